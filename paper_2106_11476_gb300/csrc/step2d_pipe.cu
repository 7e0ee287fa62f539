// Pipelined persistent 2D half steps (sm_103a); same arithmetic as the tile
// functions of tile2d.cuh, one launch per half step.
//
// A grid of one block per SM first runs the edge tiles of the grid (tiles
// that touch a C-PML strip or the outer boundary) through the general tile
// path, then walks the interior in half tiles of 128 x 8 cells with a
// two-stage pipeline: for the next half tile it issues cp.async copies of the
// stencil operand with its halo, of the density (or tissue-index) tile and of
// every streamed array of its cells into one shared-memory stage, while it
// computes the current half tile from the other.  The copies hold no
// registers, so a block keeps a whole stage (up to ~95 KB) of loads in
// flight; results go straight from registers to HBM.  Dense float maps and
// the tissue-index form take this path.
#include "tile2d.cuh"

namespace fw2 {

namespace {

constexpr int kHT = 8;              // rows of a half tile
constexpr int kCW = kTX + 8;        // staged operand columns x0-4 .. x0+TX+3 (= kPW)
constexpr int kRWp = kTX + 4;       // density / index tile columns x0 .. x0+TX+3 (= kRW)
constexpr int kArr = kHT * kTX;     // floats of one streamed array per half tile

__device__ __forceinline__ void cp16(void *smem, const void *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp4(void *smem, const void *gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory"); }

__device__ __forceinline__ float4 sld4(const float *s) { return *reinterpret_cast<const float4 *>(s); }

template <typename Maps>
struct IsIdx {
  static constexpr bool value = false;
};
template <>
struct IsIdx<IdxMaps> {
  static constexpr bool value = true;
};

constexpr int round4(int n) { return (n + 3) & ~3; }

// Tile bookkeeping: the interior region [tx_lo, tx_lo+ntx) x [ty_lo, ty_lo+nty)
// in 128 x 16 tile units (exactly the tiles interior_tile accepts) and the
// frame of edge tiles around it in a grid of tnx x tny tiles.
struct Region {
  int tnx, tny, tx_lo, ntx, ty_lo, nty;
  __device__ __forceinline__ int halves() const { return 2 * ntx * nty; }
  __device__ __forceinline__ void half_origin(int h, int &x0, int &y0) const {
    const int t = h >> 1;
    x0 = (tx_lo + t % ntx) * kTX;
    y0 = (ty_lo + t / ntx) * kTY + (h & 1) * kHT;
  }
  __device__ __forceinline__ int edges() const { return tnx * tny - ntx * nty; }
  // e-th edge tile: the rows below the interior, the side tiles of the
  // interior rows, then the rows above
  __device__ __forceinline__ void edge_origin(int e, int &x0, int &y0) const {
    int tx, ty;
    const int low = ty_lo * tnx, side = tnx - ntx;
    if (e < low) {
      ty = e / tnx;
      tx = e % tnx;
    } else if (e - low < nty * side) {
      const int k = e - low;
      ty = ty_lo + k / side;
      const int s = k % side;
      tx = s < tx_lo ? s : s + ntx;
    } else {
      const int k = e - low - nty * side;
      ty = ty_lo + nty + k / tnx;
      tx = k % tnx;
    }
    x0 = tx * kTX;
    y0 = ty * kTY;
  }
};

// ---------------------------------------------------------------- stages ---
// velocity: operand p rows y0-3 .. y0+kHT+3; density tile rows y0 .. y0+kHT;
// streamed arrays [ns][kHT][kTX]; tissue bytes rows y0 .. y0+kHT (index form)
template <int N, typename Maps>
struct VelStage {
  static constexpr bool kIdx = IsIdx<Maps>::value;
  // dense: v_x, v_y, psi_x[N], psi_y[N], 1/kappa1, a1[N], b1[N];
  // index: v_x, v_y, psi_x[N], psi_y[N]
  static constexpr int kNs = kIdx ? 2 + 2 * N : 3 + 4 * N;
  static constexpr int kP = (kHT + 7) * kCW;
  static constexpr int kR = (kHT + 1) * kRWp;
  static constexpr int kS = kNs * kArr;
  static constexpr int kI = kIdx ? (kHT + 1) * kRWp / 4 : 0;  // bytes / 4
  static constexpr int kFloats = round4(kP + kR + kS + kI);
  static constexpr int kEdge = kPH * kPW + kRH * kRW;         // general tile
};

// pressure: v_x rows y0-1 .. y0+kHT, v_y rows y0-4 .. y0+kHT+2; streamed
// arrays; tissue bytes of the half tile (index form)
template <int N, typename Maps>
struct PrsStage {
  static constexpr bool kIdx = IsIdx<Maps>::value;
  // dense: p, psi_x[N], psi_y[N], 1/kappa2, K, chi, a2[N], b2[N];
  // index: p, psi_x[N], psi_y[N]
  static constexpr int kNs = kIdx ? 1 + 2 * N : 4 + 4 * N;
  static constexpr int kX = (kHT + 2) * kCW;
  static constexpr int kY = (kHT + 7) * kCW;
  static constexpr int kS = kNs * kArr;
  static constexpr int kI = kIdx ? kHT * kTX / 4 : 0;
  static constexpr int kFloats = round4(kX + kY + kS + kI);
  static constexpr int kEdge = kHX * kPW + kHY * kPW;
};

template <int N, typename Maps>
__device__ __forceinline__ void vel_prefetch(const StepParams &P, float *st, int x0, int y0, int tid) {
  using S = VelStage<N, Maps>;
  float *sp = st, *sr = st + S::kP, *ss = sr + S::kR;
  for (int t = tid; t < (kHT + 7) * (kCW / 4); t += 256) {
    const int r = t / (kCW / 4), c4 = t % (kCW / 4);
    cp16(sp + r * kCW + 4 * c4, P.p + (long long)(y0 - 3 + r) * P.pitch + x0 - 4 + 4 * c4);
  }
  const int row = tid >> 5, col = (tid & 31) * 4;
  const long long c = (long long)(y0 + row) * P.pitch + x0 + col;
  const long long Sn = P.npts_alloc;
  float *dst = ss + row * kTX + col;
  cp16(dst, P.v[0] + c);
  cp16(dst + kArr, P.v[1] + c);
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    cp16(dst + (2 + nu) * kArr, P.psi1[0] + nu * Sn + c);
    cp16(dst + (2 + N + nu) * kArr, P.psi1[1] + nu * Sn + c);
  }
  if constexpr (!S::kIdx) {
    const float *ik1 = static_cast<const float *>(P.ik1);
    const float *a1 = static_cast<const float *>(P.a1), *b1 = static_cast<const float *>(P.b1);
    cp16(dst + (2 + 2 * N) * kArr, ik1 + c);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      cp16(dst + (3 + 2 * N + nu) * kArr, a1 + nu * Sn + c);
      cp16(dst + (3 + 3 * N + nu) * kArr, b1 + nu * Sn + c);
    }
    const float *rho = static_cast<const float *>(P.rho);
    for (int t = tid; t < (kHT + 1) * (kRWp / 4); t += 256) {
      const int r = t / (kRWp / 4), c4 = t % (kRWp / 4);
      cp16(sr + r * kRWp + 4 * c4, rho + (long long)(y0 + r) * P.pitch + x0 + 4 * c4);
    }
  } else {
    // the uint8 rows start on 4-byte boundaries only
    unsigned char *si = reinterpret_cast<unsigned char *>(ss + S::kS);
    for (int t = tid; t < (kHT + 1) * (kRWp / 4); t += 256) {
      const int r = t / (kRWp / 4), c4 = t % (kRWp / 4);
      cp4(si + r * kRWp + 4 * c4, P.tissue + (long long)(y0 + r) * P.pitch + x0 + 4 * c4);
    }
  }
}

template <int N, typename Maps>
__device__ __forceinline__ void vel_compute(const StepParams &P, const Maps &M, float *st, int x0, int y0,
                                            int tid) {
  using S = VelStage<N, Maps>;
  const float *sp = st;
  float *sr = st + S::kP;
  const float *ss = sr + S::kR;
  if constexpr (S::kIdx) {
    // density tile from the staged index and the table
    const unsigned char *si = reinterpret_cast<const unsigned char *>(ss + S::kS);
    for (int t = tid; t < (kHT + 1) * kRWp; t += 256) sr[t] = M.tab[kTabRho * kTissues + si[t]];
    __syncthreads();
  }
  const int tx = tid & 31, ly = tid >> 5, lx = 4 * tx;
  const long long c = (long long)(y0 + ly) * P.pitch + x0 + lx;
  const long long Sn = P.npts_alloc;
  const float *own = ss + ly * kTX + lx;
  float4 Dx, Dy;
  vel_derivs(P, reinterpret_cast<const float(*)[kCW]>(sp), ly + 3, tx, Dx, Dy);
  float4 k1, A[N > 0 ? N : 1], B[N > 0 ? N : 1];
  if constexpr (S::kIdx) {
    const unsigned char *si = reinterpret_cast<const unsigned char *>(ss + S::kS);
    typename Maps::Cell cell;
    cell.t = *reinterpret_cast<const uchar4 *>(si + ly * kRWp + lx);
    k1 = M.ik1(cell);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      A[nu] = M.template a<1>(cell, nu);
      B[nu] = M.template b<1>(cell, nu);
    }
  } else {
    k1 = sld4(own + (2 + 2 * N) * kArr);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      A[nu] = sld4(own + (3 + 2 * N + nu) * kArr);
      B[nu] = sld4(own + (3 + 3 * N + nu) * kArr);
    }
  }
  float4 vx = sld4(own), vy = sld4(own + kArr);
  float4 Sx = make_float4(Dx.x * k1.x, Dx.y * k1.y, Dx.z * k1.z, Dx.w * k1.w);
  float4 Sy = make_float4(Dy.x * k1.x, Dy.y * k1.y, Dy.z * k1.z, Dy.w * k1.w);
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    const float4 px = sld4(own + (2 + nu) * kArr), py = sld4(own + (2 + N + nu) * kArr);
    float4 nx_, ny_;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el(nx_, e) = fmaf(el(B[nu], e), el(px, e), el(A[nu], e) * el(Dx, e));
      el(ny_, e) = fmaf(el(B[nu], e), el(py, e), el(A[nu], e) * el(Dy, e));
      el(Sx, e) += fmaf(P.w_new, el(nx_, e), P.w_old * el(px, e));
      el(Sy, e) += fmaf(P.w_new, el(ny_, e), P.w_old * el(py, e));
    }
    st_state4(P.psi1[0], nu * Sn + c, nx_);
    st_state4(P.psi1[1], nu * Sn + c, ny_);
  }
  const float4 r0 = sld4(sr + ly * kRWp + lx);
  const float r4 = sr[ly * kRWp + lx + 4];
  const float4 ru = sld4(sr + (ly + 1) * kRWp + lx);
  vx.x -= P.two_dt / (r0.x + r0.y) * Sx.x;
  vx.y -= P.two_dt / (r0.y + r0.z) * Sx.y;
  vx.z -= P.two_dt / (r0.z + r0.w) * Sx.z;
  vx.w -= P.two_dt / (r0.w + r4) * Sx.w;
  vy.x -= P.two_dt / (r0.x + ru.x) * Sy.x;
  vy.y -= P.two_dt / (r0.y + ru.y) * Sy.y;
  vy.z -= P.two_dt / (r0.z + ru.z) * Sy.z;
  vy.w -= P.two_dt / (r0.w + ru.w) * Sy.w;
  st_state4(P.v[0], c, vx);
  st_state4(P.v[1], c, vy);
}

template <int N, typename Maps>
__device__ __forceinline__ void prs_prefetch(const StepParams &P, float *st, int x0, int y0, int tid) {
  using S = PrsStage<N, Maps>;
  float *sx = st, *sy = st + S::kX, *ss = sy + S::kY;
  for (int t = tid; t < (kHT + 2) * (kCW / 4); t += 256) {
    const int r = t / (kCW / 4), c4 = t % (kCW / 4);
    cp16(sx + r * kCW + 4 * c4, P.v[0] + (long long)(y0 - 1 + r) * P.pitch + x0 - 4 + 4 * c4);
  }
  for (int t = tid; t < (kHT + 7) * (kCW / 4); t += 256) {
    const int r = t / (kCW / 4), c4 = t % (kCW / 4);
    cp16(sy + r * kCW + 4 * c4, P.v[1] + (long long)(y0 - 4 + r) * P.pitch + x0 - 4 + 4 * c4);
  }
  const int row = tid >> 5, col = (tid & 31) * 4;
  const long long c = (long long)(y0 + row) * P.pitch + x0 + col;
  const long long Sn = P.npts_alloc;
  float *dst = ss + row * kTX + col;
  cp16(dst, P.p + c);
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    cp16(dst + (1 + nu) * kArr, P.psi2[0] + nu * Sn + c);
    cp16(dst + (1 + N + nu) * kArr, P.psi2[1] + nu * Sn + c);
  }
  if constexpr (!S::kIdx) {
    const float *ik2 = static_cast<const float *>(P.ik2), *K = static_cast<const float *>(P.K);
    const float *a2 = static_cast<const float *>(P.a2), *b2 = static_cast<const float *>(P.b2);
    cp16(dst + (1 + 2 * N) * kArr, ik2 + c);
    cp16(dst + (2 + 2 * N) * kArr, K + c);
    if (P.nl) cp16(dst + (3 + 2 * N) * kArr, static_cast<const float *>(P.chi) + c);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      cp16(dst + (4 + 2 * N + nu) * kArr, a2 + nu * Sn + c);
      cp16(dst + (4 + 3 * N + nu) * kArr, b2 + nu * Sn + c);
    }
  } else {
    unsigned char *si = reinterpret_cast<unsigned char *>(ss + S::kS);
    cp4(si + row * kTX + col, P.tissue + c);
  }
}

template <int N, typename Maps>
__device__ __forceinline__ void prs_compute(const StepParams &P, const Maps &M, const float *st, int x0, int y0,
                                            int tid) {
  using S = PrsStage<N, Maps>;
  const float *sx = st, *sy = st + S::kX, *ss = sy + S::kY;
  const int tx = tid & 31, ly = tid >> 5, lx = 4 * tx;
  const long long c = (long long)(y0 + ly) * P.pitch + x0 + lx;
  const long long Sn = P.npts_alloc;
  const float *own = ss + ly * kTX + lx;
  float4 Dx, Dy;
  prs_derivs(P, reinterpret_cast<const float(*)[kCW]>(sx), reinterpret_cast<const float(*)[kCW]>(sy), ly, tx,
             Dx, Dy);
  float4 k2, K, ch = make_float4(0.f, 0.f, 0.f, 0.f), A[N > 0 ? N : 1], B[N > 0 ? N : 1];
  if constexpr (S::kIdx) {
    const unsigned char *si = reinterpret_cast<const unsigned char *>(ss + S::kS);
    typename Maps::Cell cell;
    cell.t = *reinterpret_cast<const uchar4 *>(si + ly * kTX + lx);
    k2 = M.ik2(cell);
    K = M.Kv(cell);
    if (P.nl) ch = M.chiv(cell);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      A[nu] = M.template a<2>(cell, nu);
      B[nu] = M.template b<2>(cell, nu);
    }
  } else {
    k2 = sld4(own + (1 + 2 * N) * kArr);
    K = sld4(own + (2 + 2 * N) * kArr);
    if (P.nl) ch = sld4(own + (3 + 2 * N) * kArr);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      A[nu] = sld4(own + (4 + 2 * N + nu) * kArr);
      B[nu] = sld4(own + (4 + 3 * N + nu) * kArr);
    }
  }
  float4 p = sld4(own);
  float4 Sx = make_float4(Dx.x * k2.x, Dx.y * k2.y, Dx.z * k2.z, Dx.w * k2.w);
  float4 Sy = make_float4(Dy.x * k2.x, Dy.y * k2.y, Dy.z * k2.z, Dy.w * k2.w);
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    const float4 px = sld4(own + (1 + nu) * kArr), py = sld4(own + (1 + N + nu) * kArr);
    float4 nx_, ny_;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el(nx_, e) = fmaf(el(B[nu], e), el(px, e), el(A[nu], e) * el(Dx, e));
      el(ny_, e) = fmaf(el(B[nu], e), el(py, e), el(A[nu], e) * el(Dy, e));
      el(Sx, e) += fmaf(P.w_new, el(nx_, e), P.w_old * el(px, e));
      el(Sy, e) += fmaf(P.w_new, el(ny_, e), P.w_old * el(py, e));
    }
    st_state4(P.psi2[0], nu * Sn + c, nx_);
    st_state4(P.psi2[1], nu * Sn + c, ny_);
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float upd = P.dt * el(K, e) * (el(Sx, e) + el(Sy, e));
    if (P.nl) upd /= fmaf(el(ch, e), el(p, e), 1.f);
    el(p, e) -= upd;
  }
  st_state4(P.p, c, p);
}

// One half step: edge tiles by the general path, then the interior half
// tiles through the two-stage pipeline.  Block (32, 8).
template <int N, typename Maps, bool VEL>
__global__ void __launch_bounds__(256, 1) pipe2d_kernel(const StepParams P, const Region R) {
  extern __shared__ __align__(16) float smem[];
  using VS = VelStage<N, Maps>;
  using PS = PrsStage<N, Maps>;
  constexpr int kStage = VEL ? VS::kFloats : PS::kFloats;
  static_assert((VEL ? VS::kEdge : PS::kEdge) <= 2 * kStage, "edge tile must fit in the stages");
  float *tab = smem + 2 * kStage;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  Maps M(P);
  M.stage(P, tab, tid);  // made visible by the first barrier below
  M.bind(tab);
  const int ne = R.edges();
  for (int e = blockIdx.x; e < ne; e += gridDim.x) {
    int x0, y0;
    R.edge_origin(e, x0, y0);
    if (VEL)
      vel2d_tile<N, Maps>(P, x0, y0, reinterpret_cast<float(*)[kPW]>(smem),
                          reinterpret_cast<float(*)[kRW]>(smem + kPH * kPW), tab, false);
    else
      prs2d_tile<N, Maps>(P, x0, y0, reinterpret_cast<float(*)[kPW]>(smem),
                          reinterpret_cast<float(*)[kPW]>(smem + kHX * kPW), tab, false);
    __syncthreads();
  }
  const int nh = R.halves();
  int h = blockIdx.x;
  if (h >= nh) return;
  int x0, y0;
  R.half_origin(h, x0, y0);
  if (VEL) vel_prefetch<N, Maps>(P, smem, x0, y0, tid);
  else prs_prefetch<N, Maps>(P, smem, x0, y0, tid);
  cp_commit();
  int s = 0;
#pragma unroll 1
  for (; h < nh; h += gridDim.x) {
    const int hn = h + gridDim.x;
    int xn = 0, yn = 0;
    if (hn < nh) {
      R.half_origin(hn, xn, yn);
      if (VEL) vel_prefetch<N, Maps>(P, smem + (s ^ 1) * kStage, xn, yn, tid);
      else prs_prefetch<N, Maps>(P, smem + (s ^ 1) * kStage, xn, yn, tid);
      cp_commit();
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    if (VEL) vel_compute<N, Maps>(P, M, smem + s * kStage, x0, y0, tid);
    else prs_compute<N, Maps>(P, M, smem + s * kStage, x0, y0, tid);
    __syncthreads();
    x0 = xn;
    y0 = yn;
    s ^= 1;
  }
}

template <int N, typename Maps, bool VEL>
cudaError_t pipe_launch(const StepParams &P, const Region &R, int grid, cudaStream_t st) {
  constexpr int stage = VEL ? VelStage<N, Maps>::kFloats : PrsStage<N, Maps>::kFloats;
  constexpr size_t bytes = sizeof(float) * (2 * (size_t)stage + Maps::kSmemFloats);
  static_assert(bytes <= 227 * 1024, "stages exceed shared memory");
  cudaError_t e = cudaFuncSetAttribute(pipe2d_kernel<N, Maps, VEL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  pipe2d_kernel<N, Maps, VEL><<<grid, dim3(32, kBY), bytes, st>>>(P, R);
  return cudaGetLastError();
}

template <typename Maps, bool VEL>
cudaError_t pipe_dispatch(const StepParams &P, const Region &R, int grid, cudaStream_t st) {
  switch (P.n_relax) {
    case 0: return pipe_launch<0, Maps, VEL>(P, R, grid, st);
    case 1: return pipe_launch<1, Maps, VEL>(P, R, grid, st);
    case 2: return pipe_launch<2, Maps, VEL>(P, R, grid, st);
    case 3: return pipe_launch<3, Maps, VEL>(P, R, grid, st);
    case 4: return pipe_launch<4, Maps, VEL>(P, R, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

// interior tiles as interior_tile defines them: x0 >= Lx, x0 + kTX + Lx <= nx
Region region_of(const StepParams &P) {
  Region R;
  const int Lx = P.L[0] > 4 ? P.L[0] : 4, Ly = P.L[1] > 4 ? P.L[1] : 4;
  R.tnx = (P.nx + kTX - 1) / kTX;
  R.tny = (P.ny + kTY - 1) / kTY;
  R.tx_lo = (Lx + kTX - 1) / kTX;
  R.ty_lo = (Ly + kTY - 1) / kTY;
  R.ntx = (P.nx - Lx) / kTX - R.tx_lo;
  R.nty = (P.ny - Ly) / kTY - R.ty_lo;
  if (R.ntx <= 0 || R.nty <= 0) {
    R.ntx = 0;
    R.nty = 0;
    R.tx_lo = 0;
    R.ty_lo = 0;
  }
  return R;
}

}  // namespace

bool pipe2d_supported(const StepParams &P, int map_kind) {
  return P.nz == 1 && (map_kind == 0 || map_kind == 2) && P.n_relax >= 0 && P.n_relax <= kMaxRelax;
}

bool pipe2d_preferred(const StepParams &P, int map_kind) {
  // measured on a 4096^2 N = 4 grid: faster than the tile kernels for the
  // tissue index (the tile kernels' table lookups stall them), slower for
  // dense float maps
  return pipe2d_supported(P, map_kind) && map_kind == 2;
}

cudaError_t launch_pipe2d(bool vel, const StepParams &P, int map_kind, int grid, cudaStream_t st) {
  const Region R = region_of(P);
  if (map_kind == 2)
    return vel ? pipe_dispatch<IdxMaps, true>(P, R, grid, st) : pipe_dispatch<IdxMaps, false>(P, R, grid, st);
  if (map_kind == 0)
    return vel ? pipe_dispatch<DenseMaps<float>, true>(P, R, grid, st)
               : pipe_dispatch<DenseMaps<float>, false>(P, R, grid, st);
  return cudaErrorInvalidValue;
}

}  // namespace fw2
