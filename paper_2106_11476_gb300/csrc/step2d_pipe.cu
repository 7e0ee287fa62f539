// Pipelined persistent 2D half steps (sm_103a); same arithmetic as the tile
// functions of tile2d.cuh (bitwise the same results), one launch per half
// step, one block per SM.
//
// The grid is walked in half tiles of 128 x 8 cells through a ring of two to
// four shared-memory stages (as many as fit).  For a coming half tile one
// thread issues tiled TMA tensor copies into a free stage, one box per array:
// the stencil operand with its halo, the density tile (or the uint8 tissue
// index), every streamed array, the N mechanisms of a memory variable or of a
// relaxation map in one 3D box.  They complete on the stage's mbarrier while
// all warps compute the current half tile from another stage, so up to
// ~190 KB stay in flight per SM without registers or load instructions of the
// computing threads; results go straight from registers to HBM.
//
// Boundaries: the copies read zero outside the grid (the zero-outside rule of
// the operand halo); half tiles at the edge of the grid or in a C-PML strip
// (edge half tiles) also clamp the density tile to the last cell, take the
// C-PML coefficients of each axis from its strip, and store nothing outside
// the grid (zeros in the row padding).  With a periodic axis the tiles next
// to the boundary run the general tile path first and only the rest is staged.
// Dense float maps and the tissue-index form take this path.
#include "async.cuh"
#include "tile2d.cuh"
#include "tmap.h"

namespace fw2 {

namespace {

constexpr int kHT = 8;              // rows of a half tile
constexpr int kCW = kTX + 8;        // staged operand columns x0-4 .. x0+TX+3 (= kPW)
constexpr int kRWp = kTX + 4;       // density tile columns x0 .. x0+TX+3 (= kRW)
constexpr int kIW = kTX + 16;       // staged index bytes per row x0 .. x0+TX+15
constexpr int kArr = kHT * kTX;     // floats of one streamed array per half tile

__device__ __forceinline__ float4 sld4(const float *s) { return *reinterpret_cast<const float4 *>(s); }

template <typename Maps>
struct IsIdx {
  static constexpr bool value = false;
};
template <>
struct IsIdx<IdxMaps> {
  static constexpr bool value = true;
};

// shared-memory regions start on 128-byte boundaries (TMA destinations)
constexpr int round32(int n) { return (n + 31) & ~31; }

// Work of one launch.  Staged: the half tiles [tx_lo, tx_lo+ntx) x
// [hy_lo, hy_lo+nhy) (x in tiles of 128, y in half tiles of 8 rows), x
// fastest: the whole grid, or with `split` (a periodic axis) the interior
// tiles [tx_lo, tx_lo+ntx) x [ty_lo, ty_lo+nty) of 128 x 16 (the tiles
// interior_tile accepts), the frame of tiles around them going through the
// general tile path.
struct Region {
  int nx, ny, Lx, Ly;             // grid, boundary width (at least the halo, 4)
  int tnx, tny;                   // tiles of 128 x 16
  int split;
  int tx_lo, ntx, ty_lo, nty;     // interior tiles (split)
  int hy_lo, nhy;                 // staged half-tile rows
  __device__ __forceinline__ int halves() const { return ntx * nhy; }
  __device__ __forceinline__ void half_origin(int h, int &x0, int &y0) const {
    x0 = (tx_lo + h % ntx) * kTX;
    y0 = (hy_lo + h / ntx) * kHT;
  }
  // a staged half tile clear of the boundary rules and of the C-PML strips
  __device__ __forceinline__ bool interior(int x0, int y0) const {
    return x0 >= Lx && x0 + kTX + Lx <= nx && y0 >= Ly && y0 + kHT + Ly <= ny;
  }
  __device__ __forceinline__ int edges() const { return split ? tnx * tny - ntx * nty : 0; }
  // e-th general-path tile (split): the rows below the staged tiles, the
  // side tiles of their rows, then the rows above
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
  static constexpr int kPb = (kHT + 7) * kCW;    // operand box
  static constexpr int kRb = (kHT + 1) * kRWp;   // density box
  static constexpr int kP = round32(kPb);
  static constexpr int kR = round32(kRb);
  static constexpr int kS = kNs * kArr;
  static constexpr int kI = kIdx ? (kHT + 1) * kIW / 4 : 0;  // index bytes / 4
  static constexpr int kFloats = round32(kP + kR + kS + kI);
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
  static constexpr int kXb = (kHT + 2) * kCW;
  static constexpr int kYb = (kHT + 7) * kCW;
  static constexpr int kX = round32(kXb);
  static constexpr int kY = round32(kYb);
  static constexpr int kS = kNs * kArr;
  static constexpr int kI = kIdx ? kHT * kTX / 4 : 0;
  static constexpr int kFloats = round32(kX + kY + kS + kI);
  static constexpr int kEdge = kHX * kPW + kHY * kPW;
};

// Bytes one stage receives through the tensor maps (the chi box only with
// the nonlinear term).
template <int N, typename Maps, bool VEL>
__host__ __device__ constexpr unsigned stage_bytes(bool nl) {
  if (VEL) {
    using S = VelStage<N, Maps>;
    return 4u * (S::kPb + (S::kIdx ? 0 : S::kRb) + S::kNs * kArr) + (S::kIdx ? (kHT + 1) * kIW : 0);
  } else {
    using S = PrsStage<N, Maps>;
    return 4u * (S::kXb + S::kYb + S::kNs * kArr) - ((!S::kIdx && !nl) ? 4u * kArr : 0u) +
           (S::kIdx ? kHT * kTX : 0);
  }
}

// Issue the tensor copies of one half tile into a stage (one thread; it
// first announces the stage's bytes on the stage's mbarrier).  Boxes may
// reach outside the grid: those cells read as zero.
template <int N, typename Maps, bool VEL>
__device__ __forceinline__ void issue_stage(const StepParams &P, const PipeMaps &T, float *st, uint64_t *bar,
                                            int x0, int y0) {
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(bar, stage_bytes<N, Maps, VEL>(P.nl != 0));
  if (VEL) {
    using S = VelStage<N, Maps>;
    tma_load_2d(st, &T.m[0], x0 - 4, y0 - 3, bar);
    if (!S::kIdx) tma_load_2d(st + S::kP, &T.m[1], x0, y0, bar);
    float *ss = st + S::kP + S::kR;
    tma_load_2d(ss, &T.m[2], x0, y0, bar);
    tma_load_2d(ss + kArr, &T.m[3], x0, y0, bar);
    if (N > 0) {
      tma_load_3d(ss + 2 * kArr, &T.m[4], x0, y0, 0, bar);
      tma_load_3d(ss + (2 + N) * kArr, &T.m[5], x0, y0, 0, bar);
    }
    if (!S::kIdx) {
      tma_load_2d(ss + (2 + 2 * N) * kArr, &T.m[6], x0, y0, bar);
      if (N > 0) {
        tma_load_3d(ss + (3 + 2 * N) * kArr, &T.m[7], x0, y0, 0, bar);
        tma_load_3d(ss + (3 + 3 * N) * kArr, &T.m[8], x0, y0, 0, bar);
      }
    } else {
      tma_load_2d(ss + S::kS, &T.m[1], x0, y0, bar);  // tissue index
    }
  } else {
    using S = PrsStage<N, Maps>;
    tma_load_2d(st, &T.m[0], x0 - 4, y0 - 1, bar);
    tma_load_2d(st + S::kX, &T.m[1], x0 - 4, y0 - 4, bar);
    float *ss = st + S::kX + S::kY;
    tma_load_2d(ss, &T.m[2], x0, y0, bar);
    if (N > 0) {
      tma_load_3d(ss + kArr, &T.m[3], x0, y0, 0, bar);
      tma_load_3d(ss + (1 + N) * kArr, &T.m[4], x0, y0, 0, bar);
    }
    if (!S::kIdx) {
      tma_load_2d(ss + (1 + 2 * N) * kArr, &T.m[5], x0, y0, bar);
      tma_load_2d(ss + (2 + 2 * N) * kArr, &T.m[6], x0, y0, bar);
      if (P.nl) tma_load_2d(ss + (3 + 2 * N) * kArr, &T.m[7], x0, y0, bar);
      if (N > 0) {
        tma_load_3d(ss + (4 + 2 * N) * kArr, &T.m[8], x0, y0, 0, bar);
        tma_load_3d(ss + (4 + 3 * N) * kArr, &T.m[9], x0, y0, 0, bar);
      }
    } else {
      tma_load_2d(ss + S::kS, &T.m[5], x0, y0, bar);  // tissue index
    }
  }
}

// Density tile rows y0 .. y0+kHT, columns x0 .. x0+kTX+3.  Cells beyond the
// last one along an axis take that cell's value (rho_coord of the tile path):
// dense maps fix the staged tile in place (the entries inside the grid are
// the sources); the index form gathers the tile through the table from the
// staged index (zero outside the grid, hence the clamp).
template <typename Maps, bool EDGE>
__device__ __forceinline__ void density_tile(const StepParams &P, const Maps &M, float *sr,
                                             const unsigned char *si, int x0, int y0, int tid) {
  for (int t = tid; t < (kHT + 1) * kRWp; t += 256) {
    const int r = t / kRWp, cc = t % kRWp;
    int sxi = cc, syi = r;
    if (EDGE) {
      if (x0 + cc >= P.nx) sxi = P.nx - 1 - x0;
      if (y0 + r >= P.ny) syi = P.ny - 1 - y0;
    }
    if constexpr (IsIdx<Maps>::value) {
      sr[t] = M.tab[kTabRho * kTissues + si[syi * kIW + sxi]];
    } else {
      if (sxi != cc || syi != r) sr[t] = sr[syi * kRWp + sxi];
    }
  }
}

// a, b of mechanism nu along x at the four cells of an edge group: from the
// x strip inside its C-PML region (zero beyond the grid), else the interior
// values A, B (coef_edge of the tile path)
template <int OP, typename Maps>
__device__ __forceinline__ void x_strip_coef(const StepParams &P, int nu, int i0, int j, float4 &a, float4 &b) {
  using ST = typename Maps::StripT;
  const int L = P.L[0];
  if (!(L > 0 && (i0 < L || i0 + 3 >= P.nx - L))) return;
  const ST *sa = static_cast<const ST *>(OP == 1 ? P.sa1[0] : P.sa2[0]);
  const ST *sb = static_cast<const ST *>(OP == 1 ? P.sb1[0] : P.sb2[0]);
  const long long row = (long long)nu * P.strip_nu[0] + (long long)j * (2 * L);
  // a group wholly inside one side of the strip reads 16 aligned bytes when
  // the strip rows (2L values) and the high side's offset keep that alignment
  if ((L & 1) == 0) {
    int sc0 = -1;
    if (i0 + 3 < L) sc0 = i0;
    else if ((P.nx & 3) == 0 && i0 >= P.nx - L && i0 + 3 < P.nx) sc0 = i0 - (P.nx - 2 * L);
    if (sc0 >= 0) {
      a = ldmap4(sa, row + sc0);
      b = ldb4(sb, row + sc0);
      return;
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int x = i0 + e;
    if (x >= P.nx) {
      el(a, e) = 0.f;
      el(b, e) = 0.f;
    } else {
      const int sc = strip_coord(x, P.nx, L);
      if (sc >= 0) {
        el(a, e) = ldmap(sa, row + sc);
        el(b, e) = ldb(sb, row + sc);
      }
    }
  }
}

// a, b along y at the four cells of an edge group inside the y strip
template <int OP, typename Maps>
__device__ __forceinline__ void y_strip_coef(const StepParams &P, int nu, int i0, int sc, float4 &a, float4 &b) {
  using ST = typename Maps::StripT;
  const ST *sa = static_cast<const ST *>(OP == 1 ? P.sa1[1] : P.sa2[1]);
  const ST *sb = static_cast<const ST *>(OP == 1 ? P.sb1[1] : P.sb2[1]);
  const long long off = (long long)nu * P.strip_nu[1] + (long long)sc * P.pitch + i0;
  a = ldmap4(sa, off);
  b = ldb4(sb, off);
}

template <int N, typename Maps, bool EDGE>
__device__ __forceinline__ void vel_compute(const StepParams &P, const Maps &M, float *st, int x0, int y0,
                                            int tid) {
  using S = VelStage<N, Maps>;
  const float *sp = st;
  float *sr = st + S::kP;
  const float *ss = sr + S::kR;
  const unsigned char *si = reinterpret_cast<const unsigned char *>(ss + S::kS);
  if (EDGE || S::kIdx) {
    density_tile<Maps, EDGE>(P, M, sr, si, x0, y0, tid);
    __syncthreads();
  }
  const int tx = tid & 31, ly = tid >> 5, lx = 4 * tx;
  const int i0 = x0 + lx, j = y0 + ly;
  if (EDGE && (i0 >= P.nx || j >= P.ny)) return;
  const long long c = (long long)j * P.pitch + i0;
  const long long Sn = P.npts_alloc;
  const float *own = ss + ly * kTX + lx;
  float4 Dx, Dy;
  vel_derivs(P, reinterpret_cast<const float(*)[kCW]>(sp), ly + 3, tx, Dx, Dy);
  float4 k1, A[N > 0 ? N : 1], B[N > 0 ? N : 1];
  if constexpr (S::kIdx) {
    typename Maps::Cell cell;
    cell.t = *reinterpret_cast<const uchar4 *>(si + ly * kIW + lx);
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
  // per-axis coefficients; in an edge group the C-PML strips replace them,
  // every strip value loaded before the first store (one memory latency)
  float4 AX[N > 0 ? N : 1], BX[N > 0 ? N : 1], AY[N > 0 ? N : 1], BY[N > 0 ? N : 1];
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    AX[nu] = A[nu]; BX[nu] = B[nu]; AY[nu] = A[nu]; BY[nu] = B[nu];
  }
  if (EDGE) {
    const int scy = strip_coord(j, P.ny, P.L[1]);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      x_strip_coef<1, Maps>(P, nu, i0, j, AX[nu], BX[nu]);
      if (scy >= 0) y_strip_coef<1, Maps>(P, nu, i0, scy, AY[nu], BY[nu]);
    }
  }
  float4 vx = sld4(own), vy = sld4(own + kArr);
  float4 Sx = make_float4(Dx.x * k1.x, Dx.y * k1.y, Dx.z * k1.z, Dx.w * k1.w);
  float4 Sy = make_float4(Dy.x * k1.x, Dy.y * k1.y, Dy.z * k1.z, Dy.w * k1.w);
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    const float4 px = sld4(own + (2 + nu) * kArr), py = sld4(own + (2 + N + nu) * kArr);
    const float4 ax = AX[nu], bx = BX[nu], ay = AY[nu], by = BY[nu];
    float4 nx_, ny_;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el(nx_, e) = fmaf(el(bx, e), el(px, e), el(ax, e) * el(Dx, e));
      el(ny_, e) = fmaf(el(by, e), el(py, e), el(ay, e) * el(Dy, e));
      el(Sx, e) += fmaf(P.w_new, el(nx_, e), P.w_old * el(px, e));
      el(Sy, e) += fmaf(P.w_new, el(ny_, e), P.w_old * el(py, e));
    }
    if (EDGE) {
      nx_ = mask_pad(nx_, i0, P.nx);
      ny_ = mask_pad(ny_, i0, P.nx);
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
  if (EDGE) {
    vx = mask_pad(vx, i0, P.nx);
    vy = mask_pad(vy, i0, P.nx);
  }
  st_state4(P.v[0], c, vx);
  st_state4(P.v[1], c, vy);
}

template <int N, typename Maps, bool EDGE>
__device__ __forceinline__ void prs_compute(const StepParams &P, const Maps &M, const float *st, int x0, int y0,
                                            int tid) {
  using S = PrsStage<N, Maps>;
  const float *sx = st, *sy = st + S::kX, *ss = sy + S::kY;
  const int tx = tid & 31, ly = tid >> 5, lx = 4 * tx;
  const int i0 = x0 + lx, j = y0 + ly;
  if (EDGE && (i0 >= P.nx || j >= P.ny)) return;
  const long long c = (long long)j * P.pitch + i0;
  const long long Sn = P.npts_alloc;
  const float *own = ss + ly * kTX + lx;
  float4 Dx, Dy;
  prs_derivs(P, reinterpret_cast<const float(*)[kCW]>(sx), reinterpret_cast<const float(*)[kCW]>(sy), ly, tx,
             Dx, Dy);
  float4 k2, K, ch = make_float4(0.f, 0.f, 0.f, 0.f), A[N > 0 ? N : 1], B[N > 0 ? N : 1];
  if constexpr (S::kIdx) {
    typename Maps::Cell cell;
    cell.t = *reinterpret_cast<const uchar4 *>(reinterpret_cast<const unsigned char *>(ss + S::kS) + ly * kTX + lx);
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
  float4 AX[N > 0 ? N : 1], BX[N > 0 ? N : 1], AY[N > 0 ? N : 1], BY[N > 0 ? N : 1];
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    AX[nu] = A[nu]; BX[nu] = B[nu]; AY[nu] = A[nu]; BY[nu] = B[nu];
  }
  if (EDGE) {
    const int scy = strip_coord(j, P.ny, P.L[1]);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      x_strip_coef<2, Maps>(P, nu, i0, j, AX[nu], BX[nu]);
      if (scy >= 0) y_strip_coef<2, Maps>(P, nu, i0, scy, AY[nu], BY[nu]);
    }
  }
  float4 p = sld4(own);
  float4 Sx = make_float4(Dx.x * k2.x, Dx.y * k2.y, Dx.z * k2.z, Dx.w * k2.w);
  float4 Sy = make_float4(Dy.x * k2.x, Dy.y * k2.y, Dy.z * k2.z, Dy.w * k2.w);
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    const float4 px = sld4(own + (1 + nu) * kArr), py = sld4(own + (1 + N + nu) * kArr);
    const float4 ax = AX[nu], bx = BX[nu], ay = AY[nu], by = BY[nu];
    float4 nx_, ny_;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el(nx_, e) = fmaf(el(bx, e), el(px, e), el(ax, e) * el(Dx, e));
      el(ny_, e) = fmaf(el(by, e), el(py, e), el(ay, e) * el(Dy, e));
      el(Sx, e) += fmaf(P.w_new, el(nx_, e), P.w_old * el(px, e));
      el(Sy, e) += fmaf(P.w_new, el(ny_, e), P.w_old * el(py, e));
    }
    if (EDGE) {
      nx_ = mask_pad(nx_, i0, P.nx);
      ny_ = mask_pad(ny_, i0, P.nx);
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
  if (EDGE) p = mask_pad(p, i0, P.nx);
  st_state4(P.p, c, p);
}

// Ring of stages: as many as fit next to the maps' table (2 .. 4).
template <int N, typename Maps, bool VEL>
struct Ring {
  static constexpr int kStage = VEL ? VelStage<N, Maps>::kFloats : PrsStage<N, Maps>::kFloats;
  static constexpr int kEdge = VEL ? VelStage<N, Maps>::kEdge : PrsStage<N, Maps>::kEdge;
  static constexpr int kBudget = (220 * 1024 - 128) / 4 - Maps::kSmemFloats;  // floats
  static constexpr int kFit = kBudget / kStage;
  static constexpr int kStages = kFit > 4 ? 4 : kFit;
  static constexpr size_t kBytes = sizeof(float) * ((size_t)kStages * kStage + Maps::kSmemFloats) + 128;
  static_assert(kStages >= 2, "two stages must fit in shared memory");
  static_assert(kEdge <= kStages * kStage, "a general tile must fit in the stages");
};

// One half step.  Block (32, 8), one per SM.
template <int N, typename Maps, bool VEL>
__global__ void __launch_bounds__(256, 1)
    pipe2d_kernel(const StepParams P, const Region R, const __grid_constant__ PipeMaps T) {
  using G = Ring<N, Maps, VEL>;
  constexpr int kS = G::kStages, kStage = G::kStage;
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ __align__(8) uint64_t bar[kS];
  __shared__ int ok;
  // TMA destinations need 128-byte alignment: round the base up (the launch
  // adds 128 bytes of slack)
  float *smem = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float *tab = smem + kS * kStage;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  Maps M(P);
  M.stage(P, tab, tid);  // made visible by the first barrier below
  M.bind(tab);
  if (tid == 0) {
    for (int q = 0; q < kS; ++q) mbar_init(&bar[q], 1);
    fence_mbarrier_init();
  }
  // general-path tiles (periodic axes only)
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
  __syncthreads();  // barriers initialised, table staged, general tiles done with the stages
  const int nh = R.halves();
  int h = blockIdx.x;
  if (h >= nh) return;
  // this block's half tiles are h, h + grid, ...; the first kS - 1 go out now,
  // then each iteration issues one more into the stage freed last
  unsigned phase = 0;    // bit q: parity of the next completion of stage q
  unsigned pending = 0;  // bit q: copies issued into stage q, not consumed
  int hs = h;            // next half tile to issue
  for (int q = 0; q < kS - 1; ++q, hs += gridDim.x) {
    if (hs >= nh) break;
    if (tid == 0) {
      int xq, yq;
      R.half_origin(hs, xq, yq);
      issue_stage<N, Maps, VEL>(P, T, smem + q * kStage, &bar[q], xq, yq);
    }
    pending |= 1u << q;
  }
  int s = 0;
#pragma unroll 1
  for (; h < nh; h += gridDim.x) {
    if (hs < nh) {
      const int q = (s + kS - 1) % kS;  // computed in the previous iteration
      if (tid == 0) {
        int xq, yq;
        R.half_origin(hs, xq, yq);
        issue_stage<N, Maps, VEL>(P, T, smem + q * kStage, &bar[q], xq, yq);
      }
      pending |= 1u << q;
      hs += gridDim.x;
    }
    if (tid == 0) ok = mbar_wait_bounded(&bar[s], (phase >> s) & 1u);
    __syncthreads();
    if (!ok) {
      // a copy never landed: report, let the other stages' copies finish
      // (bounded), and leave
      if (tid == 0) {
        report_status(P.status, kStatusWaitTimeout);
        for (int q = 0; q < kS; ++q)
          if (q != s && ((pending >> q) & 1u)) mbar_wait_bounded(&bar[q], (phase >> q) & 1u);
      }
      return;
    }
    phase ^= 1u << s;
    pending &= ~(1u << s);
    int x0, y0;
    R.half_origin(h, x0, y0);
    float *cur = smem + s * kStage;
    if (R.interior(x0, y0)) {
      if (VEL) vel_compute<N, Maps, false>(P, M, cur, x0, y0, tid);
      else prs_compute<N, Maps, false>(P, M, cur, x0, y0, tid);
    } else {
      if (VEL) vel_compute<N, Maps, true>(P, M, cur, x0, y0, tid);
      else prs_compute<N, Maps, true>(P, M, cur, x0, y0, tid);
    }
    __syncthreads();
    s = (s + 1) % kS;
  }
}

// Batched half step over a unit table of several contexts (one group: same
// N and map kind, no periodic axis): entry (ctx, x0, y0, interior).  The
// contexts' step parameters and tensor maps sit in device memory (TMA reads
// the maps from there); a block copies a context's parameters to shared
// memory, and stages its tissue-index table, when the context changes.
template <int N, typename Maps, bool VEL>
__global__ void __launch_bounds__(256, 1)
    pipe2d_batched_kernel(const StepParams *Ps, const PipeMaps *Ts, const int4 *units, int n_units) {
  using G = Ring<N, Maps, VEL>;
  constexpr int kS = G::kStages, kStage = G::kStage;
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ __align__(8) uint64_t bar[kS];
  __shared__ __align__(16) StepParams sP;
  __shared__ int ok;
  float *smem = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float *tab = smem + kS * kStage;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid == 0) {
    for (int q = 0; q < kS; ++q) mbar_init(&bar[q], 1);
    fence_mbarrier_init();
  }
  __syncthreads();
  // a contiguous run of units per block: consecutive units share a context
  // (one parameter and table load per context) and halo rows (L2)
  const int h_end = (int)(((long long)n_units * (blockIdx.x + 1)) / gridDim.x);
  int h = (int)(((long long)n_units * blockIdx.x) / gridDim.x);
  if (h >= h_end) return;
  unsigned phase = 0, pending = 0;
  int hs = h;
  for (int q = 0; q < kS - 1; ++q, ++hs) {
    if (hs >= h_end) break;
    if (tid == 0) {
      const int4 e = units[hs];
      issue_stage<N, Maps, VEL>(Ps[e.x], Ts[e.x], smem + q * kStage, &bar[q], e.y, e.z);
    }
    pending |= 1u << q;
  }
  int s = 0, cur = -1;
#pragma unroll 1
  for (; h < h_end; ++h) {
    if (hs < h_end) {
      const int q = (s + kS - 1) % kS;
      if (tid == 0) {
        const int4 e = units[hs];
        issue_stage<N, Maps, VEL>(Ps[e.x], Ts[e.x], smem + q * kStage, &bar[q], e.y, e.z);
      }
      pending |= 1u << q;
      ++hs;
    }
    const int4 e = units[h];
    if (e.x != cur) {
      // new context: parameters (and index table) into shared memory; the
      // previous unit's compute finished at the last barrier
      const int *src = reinterpret_cast<const int *>(Ps + e.x);
      int *dst = reinterpret_cast<int *>(&sP);
      for (int w = tid; w < (int)(sizeof(StepParams) / 4); w += 256) dst[w] = __ldg(src + w);
      __syncthreads();
      Maps(sP).stage(sP, tab, tid);
      cur = e.x;
    }
    if (tid == 0) ok = mbar_wait_bounded(&bar[s], (phase >> s) & 1u);
    __syncthreads();
    if (!ok) {
      if (tid == 0) {
        report_status(sP.status, kStatusWaitTimeout);
        for (int q = 0; q < kS; ++q)
          if (q != s && ((pending >> q) & 1u)) mbar_wait_bounded(&bar[q], (phase >> q) & 1u);
      }
      return;
    }
    phase ^= 1u << s;
    pending &= ~(1u << s);
    Maps M(sP);
    M.bind(tab);
    float *stp = smem + s * kStage;
    if (e.w) {
      if (VEL) vel_compute<N, Maps, false>(sP, M, stp, e.y, e.z, tid);
      else prs_compute<N, Maps, false>(sP, M, stp, e.y, e.z, tid);
    } else {
      if (VEL) vel_compute<N, Maps, true>(sP, M, stp, e.y, e.z, tid);
      else prs_compute<N, Maps, true>(sP, M, stp, e.y, e.z, tid);
    }
    __syncthreads();
    s = (s + 1) % kS;
  }
}

template <int N, typename Maps, bool VEL>
cudaError_t pipe_batched_launch(const StepParams *Ps, const PipeMaps *Ts, const int4 *units, int n_units, int grid,
                                cudaStream_t st) {
  constexpr size_t bytes = Ring<N, Maps, VEL>::kBytes;
  cudaError_t e = cudaFuncSetAttribute(pipe2d_batched_kernel<N, Maps, VEL>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  pipe2d_batched_kernel<N, Maps, VEL><<<grid, dim3(32, kBY), bytes, st>>>(Ps, Ts, units, n_units);
  return cudaGetLastError();
}

template <typename Maps, bool VEL>
cudaError_t pipe_batched_dispatch(const StepParams *Ps, const PipeMaps *Ts, const int4 *units, int n_units,
                                  int n_relax, int grid, cudaStream_t st) {
  switch (n_relax) {
    case 0: return pipe_batched_launch<0, Maps, VEL>(Ps, Ts, units, n_units, grid, st);
    case 1: return pipe_batched_launch<1, Maps, VEL>(Ps, Ts, units, n_units, grid, st);
    case 2: return pipe_batched_launch<2, Maps, VEL>(Ps, Ts, units, n_units, grid, st);
    case 3: return pipe_batched_launch<3, Maps, VEL>(Ps, Ts, units, n_units, grid, st);
    case 4: return pipe_batched_launch<4, Maps, VEL>(Ps, Ts, units, n_units, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int N, typename Maps, bool VEL>
cudaError_t pipe_launch(const StepParams &P, const Region &R, int grid, const PipeMaps &T, cudaStream_t st) {
  constexpr size_t bytes = Ring<N, Maps, VEL>::kBytes;
  cudaError_t e = cudaFuncSetAttribute(pipe2d_kernel<N, Maps, VEL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  pipe2d_kernel<N, Maps, VEL><<<grid, dim3(32, kBY), bytes, st>>>(P, R, T);
  return cudaGetLastError();
}

template <typename Maps, bool VEL>
cudaError_t pipe_dispatch(const StepParams &P, const Region &R, int grid, const PipeMaps &T, cudaStream_t st) {
  switch (P.n_relax) {
    case 0: return pipe_launch<0, Maps, VEL>(P, R, grid, T, st);
    case 1: return pipe_launch<1, Maps, VEL>(P, R, grid, T, st);
    case 2: return pipe_launch<2, Maps, VEL>(P, R, grid, T, st);
    case 3: return pipe_launch<3, Maps, VEL>(P, R, grid, T, st);
    case 4: return pipe_launch<4, Maps, VEL>(P, R, grid, T, st);
    default: return cudaErrorInvalidValue;
  }
}

Region region_of(const StepParams &P) {
  Region R;
  R.nx = P.nx;
  R.ny = P.ny;
  R.Lx = P.L[0] > 4 ? P.L[0] : 4;
  R.Ly = P.L[1] > 4 ? P.L[1] : 4;
  R.tnx = (P.nx + kTX - 1) / kTX;
  R.tny = (P.ny + kTY - 1) / kTY;
  R.split = P.periodic[0] || P.periodic[1];
  if (!R.split) {
    // every half tile of the grid is staged
    R.tx_lo = 0;
    R.ntx = R.tnx;
    R.ty_lo = 0;
    R.nty = 0;
    R.hy_lo = 0;
    R.nhy = (P.ny + kHT - 1) / kHT;
    return R;
  }
  // interior tiles as interior_tile defines them: x0 >= Lx, x0 + kTX + Lx <= nx
  R.tx_lo = (R.Lx + kTX - 1) / kTX;
  R.ty_lo = (R.Ly + kTY - 1) / kTY;
  R.ntx = (P.nx - R.Lx) / kTX - R.tx_lo;
  R.nty = (P.ny - R.Ly) / kTY - R.ty_lo;
  if (R.ntx <= 0 || R.nty <= 0) {
    R.ntx = 0;
    R.nty = 0;
    R.tx_lo = 0;
    R.ty_lo = 0;
  }
  R.hy_lo = 2 * R.ty_lo;
  R.nhy = 2 * R.nty;
  return R;
}

}  // namespace

bool pipe2d_supported(const StepParams &P, int map_kind) {
  return P.nz == 1 && (map_kind == 0 || map_kind == 2) && P.n_relax >= 0 && P.n_relax <= kMaxRelax;
}

bool pipe2d_preferred(const StepParams &P, int map_kind) { return pipe2d_supported(P, map_kind); }

bool pipe2d_interior_half(const StepParams &P, int x0, int y0) {
  const int Lx = P.L[0] > 4 ? P.L[0] : 4, Ly = P.L[1] > 4 ? P.L[1] : 4;
  return x0 >= Lx && x0 + kTX + Lx <= P.nx && y0 >= Ly && y0 + kHT + Ly <= P.ny;
}

cudaError_t launch_pipe2d_batched(bool vel, const StepParams *Ps, const PipeMaps *Ts, const int4 *units,
                                  int n_units, int n_relax, int map_kind, int grid, cudaStream_t st) {
  if (n_units <= 0) return cudaSuccess;
  if (map_kind == 2)
    return vel ? pipe_batched_dispatch<IdxMaps, true>(Ps, Ts, units, n_units, n_relax, grid, st)
               : pipe_batched_dispatch<IdxMaps, false>(Ps, Ts, units, n_units, n_relax, grid, st);
  if (map_kind == 0)
    return vel ? pipe_batched_dispatch<DenseMaps<float>, true>(Ps, Ts, units, n_units, n_relax, grid, st)
               : pipe_batched_dispatch<DenseMaps<float>, false>(Ps, Ts, units, n_units, n_relax, grid, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_pipe2d(bool vel, const StepParams &P, int map_kind, int grid, const PipeMaps &T,
                          cudaStream_t st) {
  const Region R = region_of(P);
  if (map_kind == 2)
    return vel ? pipe_dispatch<IdxMaps, true>(P, R, grid, T, st) : pipe_dispatch<IdxMaps, false>(P, R, grid, T, st);
  if (map_kind == 0)
    return vel ? pipe_dispatch<DenseMaps<float>, true>(P, R, grid, T, st)
               : pipe_dispatch<DenseMaps<float>, false>(P, R, grid, T, st);
  return cudaErrorInvalidValue;
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeTiled>(f);
  }();
  return fn;
}

// float (or uint8) tensor map over [ny][nx] (rank 2, row stride pitch) or
// [n3][ny][nx] (rank 3, plane stride s3 elements) with a box of bx x by
// (x bz)
bool encode(CUtensorMap *m, const void *base, const StepParams &P, int rank, int n3, long long s3, int bx, int by,
            int bz, bool u8 = false) {
  const unsigned long long es = u8 ? 1 : 4;
  const unsigned long long dims[3] = {(unsigned long long)P.nx, (unsigned long long)P.ny, (unsigned long long)n3};
  const unsigned long long strides[2] = {(unsigned long long)P.pitch * es, (unsigned long long)s3 * es};
  const unsigned box[3] = {(unsigned)bx, (unsigned)by, (unsigned)bz};
  return encode_tensor_map(m, base, (int)es, rank, dims, strides, box);
}

}  // namespace

bool encode_tensor_map(CUtensorMap *m, const void *base, int elem_bytes, int rank, const unsigned long long *dims,
                       const unsigned long long *strides_bytes, const unsigned *box) {
  EncodeTiled fn = encoder();
  if (!fn || !base || rank < 2 || rank > 5) return false;
  cuuint64_t d[5], st[4];
  cuuint32_t b[5], e[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = dims[i];
    b[i] = box[i];
    e[i] = 1;
  }
  for (int i = 0; i + 1 < rank; ++i) st[i] = strides_bytes[i];
  const CUtensorMapDataType t = elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                : elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  return fn(m, t, (cuuint32_t)rank, const_cast<void *>(base), d, st, b, e, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

cudaError_t build_pipe2d_maps(const StepParams &P, int map_kind, PipeMaps *vel, PipeMaps *prs, const char **why) {
  *vel = PipeMaps{};
  *prs = PipeMaps{};
  if (!encoder()) {
    *why = "cuTensorMapEncodeTiled is not available from the driver";
    return cudaErrorInvalidValue;
  }
  const int N = P.n_relax;
  const long long S = P.npts_alloc;
  const bool dense = map_kind == 0;
  bool ok = true;
  // velocity half step
  ok = ok && encode(&vel->m[0], P.p, P, 2, 1, S, kCW, kHT + 7, 1);
  if (dense) ok = ok && encode(&vel->m[1], P.rho, P, 2, 1, S, kRWp, kHT + 1, 1);
  else ok = ok && encode(&vel->m[1], P.tissue, P, 2, 1, S, kIW, kHT + 1, 1, true);
  ok = ok && encode(&vel->m[2], P.v[0], P, 2, 1, S, kTX, kHT, 1);
  ok = ok && encode(&vel->m[3], P.v[1], P, 2, 1, S, kTX, kHT, 1);
  if (N > 0) {
    ok = ok && encode(&vel->m[4], P.psi1[0], P, 3, N, S, kTX, kHT, N);
    ok = ok && encode(&vel->m[5], P.psi1[1], P, 3, N, S, kTX, kHT, N);
  }
  if (dense) {
    ok = ok && encode(&vel->m[6], P.ik1, P, 2, 1, S, kTX, kHT, 1);
    if (N > 0) {
      ok = ok && encode(&vel->m[7], P.a1, P, 3, N, S, kTX, kHT, N);
      ok = ok && encode(&vel->m[8], P.b1, P, 3, N, S, kTX, kHT, N);
    }
  }
  // pressure half step
  ok = ok && encode(&prs->m[0], P.v[0], P, 2, 1, S, kCW, kHT + 2, 1);
  ok = ok && encode(&prs->m[1], P.v[1], P, 2, 1, S, kCW, kHT + 7, 1);
  ok = ok && encode(&prs->m[2], P.p, P, 2, 1, S, kTX, kHT, 1);
  if (N > 0) {
    ok = ok && encode(&prs->m[3], P.psi2[0], P, 3, N, S, kTX, kHT, N);
    ok = ok && encode(&prs->m[4], P.psi2[1], P, 3, N, S, kTX, kHT, N);
  }
  if (!dense) ok = ok && encode(&prs->m[5], P.tissue, P, 2, 1, S, kTX, kHT, 1, true);
  if (dense) {
    ok = ok && encode(&prs->m[5], P.ik2, P, 2, 1, S, kTX, kHT, 1);
    ok = ok && encode(&prs->m[6], P.K, P, 2, 1, S, kTX, kHT, 1);
    if (P.nl) ok = ok && encode(&prs->m[7], P.chi, P, 2, 1, S, kTX, kHT, 1);
    if (N > 0) {
      ok = ok && encode(&prs->m[8], P.a2, P, 3, N, S, kTX, kHT, N);
      ok = ok && encode(&prs->m[9], P.b2, P, 3, N, S, kTX, kHT, N);
    }
  }
  if (!ok) {
    *why = "cuTensorMapEncodeTiled rejected a map";
    return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

}  // namespace fw2
