// Pipelined persistent 2D half steps (sm_103a); the arithmetic of the tile
// kernels (tile2d.cuh) cell for cell, so the results are bitwise the same;
// one launch per half step, one block of 512 threads per SM.
//
// The grid is walked in half tiles of 128 x 8 cells through a ring of two to
// four shared-memory stages (as many as fit).  For a coming half tile one
// thread issues tiled TMA tensor copies into a free stage, one box per array:
// the stencil operand with its halo, the density tile (or the uint8 tissue
// index), every streamed array, the N mechanisms of a memory variable or of a
// relaxation map in one 3D box.  They complete on the stage's mbarrier while
// all threads compute the current half tile from another stage, two cells
// each, so up to ~190 KB stay in flight per SM without registers or load
// instructions of the computing threads.  With float maps the updated arrays
// are written back into the stage and leave for HBM as TMA tensor stores;
// with the index form every thread stores its own results.
//
// Boundaries: the copies read zero outside the grid (the zero-outside rule of
// the operand halo); half tiles at the edge of the grid or in a C-PML strip
// (edge half tiles) also clamp the density tile to the last cell, take the
// C-PML coefficients of each axis from its strip, and store nothing outside
// the grid (zeros in the row padding).  Periodic grids take the tile kernels.
// Dense float maps and the tissue-index form take this path.
#include "async.cuh"
#include "coef.cuh"
#include "maps.cuh"
#include "tmap.h"

namespace fw2 {

namespace {

constexpr int kHT = 8;              // rows of a half tile
constexpr int kCW = kTX + 8;        // staged operand columns x0-4 .. x0+TX+3 (= kPW)
constexpr int kRWp = kTX + 4;       // density tile columns x0 .. x0+TX+3 (= kRW)
constexpr int kIW = kTX + 16;       // staged index bytes per row x0 .. x0+TX+15
constexpr int kArr = kHT * kTX;     // floats of one streamed array per half tile


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

// Work of one launch: the half tiles of the grid (tiles of 128 x 8 cells,
// x fastest).
struct Region {
  int nx, ny, Lx, Ly;  // grid, boundary width (at least the halo, 4)
  int ntx, nhy;        // tiles along x, half-tile rows
  __device__ __forceinline__ int halves() const { return ntx * nhy; }
  __device__ __forceinline__ void half_origin(int h, int &x0, int &y0) const {
    x0 = (h % ntx) * kTX;
    y0 = (h / ntx) * kHT;
  }
  // a half tile clear of the boundary rules and of the C-PML strips
  __device__ __forceinline__ bool interior(int x0, int y0) const {
    return x0 >= Lx && x0 + kTX + Lx <= nx && y0 >= Ly && y0 + kHT + Ly <= ny;
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
  static constexpr int kR = kIdx ? 0 : round32(kRb);  // the index form looks the density up
  static constexpr int kS = kNs * kArr;
  static constexpr int kI = kIdx ? (kHT + 1) * kIW / 4 : 0;  // index bytes / 4
  // dense, literal nonlinear system: K box of the density box's shape
  static constexpr int kK = kIdx ? 0 : kR;
  static constexpr int kFloats = round32(kP + kR + kS + kI + kK);
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
};

// Bytes one stage receives through the tensor maps (the chi box only with
// the nonlinear term, the velocity's K box only with the literal system).
template <int N, typename Maps, bool VEL>
__host__ __device__ constexpr unsigned stage_bytes(bool nl, bool nl_vel) {
  if (VEL) {
    using S = VelStage<N, Maps>;
    return 4u * (S::kPb + (S::kIdx ? 0 : S::kRb) + S::kNs * kArr) + (S::kIdx ? (kHT + 1) * kIW : 0) +
           ((!S::kIdx && nl_vel) ? 4u * S::kRb : 0u);
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
  mbar_arrive_expect_tx(bar, stage_bytes<N, Maps, VEL>(P.nl != 0, P.nl_vel != 0));
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
      if (P.nl_vel) tma_load_2d(ss + S::kS, &T.m[9], x0, y0, bar);  // K, density-box shape
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

// Store the updated arrays of a half tile from its stage (one thread, after
// every thread's fence and a barrier): velocity v_x, v_y, psi1_x, psi1_y;
// pressure p, psi2_x, psi2_y.  The copies write nothing outside the grid.
template <int N, typename Maps, bool VEL>
__device__ __forceinline__ void store_stage(const PipeMaps &T, const float *st, int x0, int y0) {
  if (VEL) {
    using S = VelStage<N, Maps>;
    const float *ss = st + S::kP + S::kR;
    tma_store_2d(&T.m[2], x0, y0, ss);
    tma_store_2d(&T.m[3], x0, y0, ss + kArr);
    if (N > 0) {
      tma_store_3d(&T.m[4], x0, y0, 0, ss + 2 * kArr);
      tma_store_3d(&T.m[5], x0, y0, 0, ss + (2 + N) * kArr);
    }
  } else {
    using S = PrsStage<N, Maps>;
    const float *ss = st + S::kX + S::kY;
    tma_store_2d(&T.m[2], x0, y0, ss);
    if (N > 0) {
      tma_store_3d(&T.m[3], x0, y0, 0, ss + kArr);
      tma_store_3d(&T.m[4], x0, y0, 0, ss + (1 + N) * kArr);
    }
  }
  bulk_commit();
}

// ------------------------------------------------------------ compute ---
// 512 threads per block, two consecutive x cells each: thread t of row ly
// (64 threads per row) owns cells x0 + 2t, x0 + 2t + 1.  Every cell sees the
// operations of the tile path in the same order, so results are bitwise the
// same.
constexpr int kThreads = 512;

__device__ __forceinline__ float2 sld2(const float *s) { return *reinterpret_cast<const float2 *>(s); }
__device__ __forceinline__ void st_state2(float *p, long long i, float2 v) {
  __stcs(reinterpret_cast<float2 *>(p + i), v);
}
// zero the cells of a pair that fall in the row padding (x >= nx)
__device__ __forceinline__ float2 mask_pad2(float2 v, int i0, int nx) {
  if (i0 + 1 >= nx) v.y = 0.f;
  if (i0 >= nx) v.x = 0.f;
  return v;
}
// Results leave through the stage and TMA tensor stores (fewer store
// instructions than per-thread stores; the store of a unit overlaps the
// compute of the next).
template <typename Maps>
struct TmaStore {
  static constexpr bool value = true;
};
// one result pair of array `a` (stage offset in arrays) of cell c
template <typename Maps, bool EDGE>
__device__ __forceinline__ void put2(float *own, int a, float *g, long long gi, float2 v, int i0, int nx) {
  if constexpr (TmaStore<Maps>::value) {
    *reinterpret_cast<float2 *>(own + a * kArr) = v;
  } else {
    st_state2(g, gi, EDGE ? mask_pad2(v, i0, nx) : v);
  }
}
__device__ __forceinline__ float &el2(float2 &v, int e) { return e == 0 ? v.x : v.y; }
__device__ __forceinline__ float el2(const float2 &v, int e) { return e == 0 ? v.x : v.y; }
// ten consecutive shared-memory values from column c of a row (c even)
struct Win10 {
  float v[10];
};
__device__ __forceinline__ Win10 win10(const float *row, int c) {
  Win10 w;
  const float2 *r2 = reinterpret_cast<const float2 *>(row + c);
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float2 t = r2[i];
    w.v[2 * i] = t.x;
    w.v[2 * i + 1] = t.y;
  }
  return w;
}

// x and y derivatives of the staged p at the faces of cells x0+lx, x0+lx+1
// (operand rows y0-3.., columns x0-4..; cell e sits at column lx + 4 + e)
__device__ __forceinline__ void vel_derivs2(const StepParams &P, const float *sp, int sy, int lx, float2 &Dx,
                                            float2 &Dy) {
  const Win10 w = win10(sp + sy * kCW, lx);  // columns lx .. lx+9
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    float d = 0.f;
#pragma unroll
    for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m] - w.v[4 + e - m + 1], d);
    el2(Dx, e) = d;
  }
  float2 col[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) col[m] = sld2(sp + (sy - 3 + m) * kCW + lx + 4);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    float d = 0.f;
#pragma unroll
    for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el2(col[3 + m], e) - el2(col[4 - m], e), d);
    el2(Dy, e) = d;
  }
  if (P.g11h != 0.f) {
    const Win10 up = win10(sp + (sy + 1) * kCW, lx), dn = win10(sp + (sy - 1) * kCW, lx);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      el2(Dx, e) += P.g11h * ((up.v[5 + e] - up.v[4 + e]) + (dn.v[5 + e] - dn.v[4 + e]));
      el2(Dy, e) += P.g11h * ((up.v[5 + e] - w.v[5 + e]) + (up.v[3 + e] - w.v[3 + e]));
    }
  }
}

// x and y derivatives of v_x (rows y0-1..), v_y (rows y0-4..) at the centres
__device__ __forceinline__ void prs_derivs2(const StepParams &P, const float *svx, const float *svy, int ly,
                                            int lx, float2 &Dx, float2 &Dy) {
  const Win10 w = win10(svx + (ly + 1) * kCW, lx);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    float d = 0.f;
#pragma unroll
    for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m - 1] - w.v[4 + e - m], d);
    el2(Dx, e) = d;
  }
  float2 col[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) col[m] = sld2(svy + (ly + m) * kCW + lx + 4);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    float d = 0.f;
#pragma unroll
    for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el2(col[4 + m - 1], e) - el2(col[4 - m], e), d);
    el2(Dy, e) = d;
  }
  if (P.g11h != 0.f) {
    const Win10 up = win10(svx + (ly + 2) * kCW, lx), dn = win10(svx + ly * kCW, lx);
    const Win10 y0w = win10(svy + (ly + 4) * kCW, lx), y1w = win10(svy + (ly + 3) * kCW, lx);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      el2(Dx, e) += P.g11h * ((up.v[4 + e] - up.v[3 + e]) + (dn.v[4 + e] - dn.v[3 + e]));
      el2(Dy, e) += P.g11h * ((y0w.v[5 + e] - y1w.v[5 + e]) + (y0w.v[3 + e] - y1w.v[3 + e]));
    }
  }
}

// per-tissue table of the index form into shared memory (all threads)
template <typename Maps>
__device__ __forceinline__ void stage_table(const StepParams &P, float *tab, int tid) {
  if constexpr (IsIdx<Maps>::value) {
    const float4 *src = reinterpret_cast<const float4 *>(P.table);
    float4 *dst = reinterpret_cast<float4 *>(tab);
    for (int t = tid; t < kTableFields * kTissues / 4; t += kThreads) dst[t] = __ldg(src + t);
  }
}

// coefficient of field f at the two cells of a pair (index form)
__device__ __forceinline__ float2 look2(const float *tab, int f, uchar2 t) {
  const float *r = tab + f * kTissues;
  return make_float2(r[t.x], r[t.y]);
}

// Densities at the faces of a pair, read where the thread needs them: cells
// (lx, ly), (lx + 1, ly), (lx + 2, ly), (lx, ly + 1), (lx + 1, ly + 1) of the
// half tile.  Cells beyond the last one along an axis take that cell's value
// (rho_coord of the tile path).  Dense maps read the staged density box; the
// index form looks the staged index up in the table.
struct FaceRho {
  float r0, r1, r2, u0, u1;  // row ly: lx .. lx+2; row ly+1: lx, lx+1
};
template <typename Maps, bool EDGE>
__device__ __forceinline__ FaceRho face_rho(const StepParams &P, const float *tab, const float *sr,
                                            const unsigned char *si, int x0, int y0, int lx, int ly) {
  int c0 = lx, c1 = lx + 1, c2 = lx + 2, r0 = ly, r1 = ly + 1;
  if (EDGE) {
    const int mx = P.nx - 1 - x0, my = P.ny - 1 - y0;  // last cell inside, tile coordinates
    c0 = min(c0, mx);
    c1 = min(c1, mx);
    c2 = min(c2, mx);
    r0 = min(r0, my);
    r1 = min(r1, my);
  }
  auto at = [&](int r, int cc) -> float {
    if constexpr (IsIdx<Maps>::value) return tab[kTabRho * kTissues + si[r * kIW + cc]];
    else return sr[r * kRWp + cc];
  };
  return FaceRho{at(r0, c0), at(r0, c1), at(r0, c2), at(r1, c0), at(r1, c1)};
}

// Momentum factors of the literal nonlinear system (Eq. general5) at the x
// and y faces of the pair: p from the staged operand (cell e at column
// lx + 4 + e of row sy; zero beyond the grid), K from the staged K box (float
// maps; the density box's shape) or the staged index (index form),
// neighbours clamped to the last cell.
template <typename Maps, bool EDGE>
__device__ __forceinline__ void mom_factors2(const StepParams &P, const float *tab, const unsigned char *si,
                                             const float *sk, const float *sp, int sy, int lx, int ly, int x0,
                                             int y0, float2 &fx, float2 &fy) {
  const float *row = sp + sy * kCW + lx + 4, *up = sp + (sy + 1) * kCW + lx + 4;
  const int mx = P.nx - 1 - x0, my = P.ny - 1 - y0;
  const int r1 = EDGE ? min(ly + 1, my) : ly + 1;
  auto K = [&](int r, int cc) -> float {
    if constexpr (IsIdx<Maps>::value) return tab[kTabK * kTissues + si[r * kIW + cc]];
    else return sk[r * kRWp + cc];
  };
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int c0 = EDGE ? min(lx + e, mx) : lx + e, c1 = EDGE ? min(lx + e + 1, mx) : lx + e + 1;
    const float Kc = K(ly, c0), Kx = K(ly, c1), Ky = K(r1, c0);
    el2(fx, e) = mom_factor(Kc, Kx, row[e], row[e + 1]);
    el2(fy, e) = mom_factor(Kc, Ky, row[e], up[e]);
  }
}

// a, b of mechanism nu along x at the two cells of an edge pair: from the x
// strip inside its C-PML region, else unchanged (coef_edge of the tile path;
// its zero beyond the grid only reaches cells that are masked)
template <int OP, typename Maps>
__device__ __forceinline__ void x_strip_coef2(const StepParams &P, int nu, int i0, int j, float2 &a, float2 &b) {
  using ST = typename Maps::StripT;
  static_assert(sizeof(ST) == 4, "the pipelined 2D kernels read float strips");
  const int L = P.L[0];
  if (!(L > 0 && (i0 < L || i0 + 1 >= P.nx - L))) return;
  const float *sa = static_cast<const float *>(OP == 1 ? P.sa1[0] : P.sa2[0]);
  const float *sb = static_cast<const float *>(OP == 1 ? P.sb1[0] : P.sb2[0]);
  const long long row = (long long)nu * P.strip_nu[0] + (long long)j * (2 * L);
  // both cells on one side of the strip: one aligned pair (i0 and the high
  // side's offset nx - 2L are even)
  int sc0 = -1;
  if (i0 + 1 < L) sc0 = i0;
  else if (i0 >= P.nx - L && i0 + 1 < P.nx && ((P.nx - 2 * L) & 1) == 0) sc0 = i0 - (P.nx - 2 * L);
  if (sc0 >= 0) {
    a = __ldg(reinterpret_cast<const float2 *>(sa + row + sc0));
    b = __ldg(reinterpret_cast<const float2 *>(sb + row + sc0));
    return;
  }
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int x = i0 + e;
    if (x >= P.nx) {
      el2(a, e) = 0.f;
      el2(b, e) = 0.f;
    } else {
      const int sc = strip_coord(x, P.nx, L);
      if (sc >= 0) {
        el2(a, e) = ldmap(sa, row + sc);
        el2(b, e) = ldb(sb, row + sc);
      }
    }
  }
}

// a, b along y at the two cells of an edge pair inside the y strip (an
// aligned pair: i0 even, pitch a multiple of 16)
template <int OP, typename Maps>
__device__ __forceinline__ void y_strip_coef2(const StepParams &P, int nu, int i0, int sc, float2 &a, float2 &b) {
  const float *sa = static_cast<const float *>(OP == 1 ? P.sa1[1] : P.sa2[1]);
  const float *sb = static_cast<const float *>(OP == 1 ? P.sb1[1] : P.sb2[1]);
  const long long off = (long long)nu * P.strip_nu[1] + (long long)sc * P.pitch + i0;
  a = __ldg(reinterpret_cast<const float2 *>(sa + off));
  b = __ldg(reinterpret_cast<const float2 *>(sb + off));
}

// Prefetch into L2 the C-PML strip rows an edge half tile will read (warp 0,
// when its copies are issued): otherwise they come straight from DRAM while
// the half tile computes.  OP: 1 velocity (a1, b1), 2 pressure (a2, b2).
__device__ __forceinline__ void l2_line(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
template <int N, int OP>
__device__ __forceinline__ void prefetch_strips2(const StepParams &P, int x0, int y0, int lane) {
  if constexpr (N > 0) {
    const float *sa[2], *sb[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      sa[q] = static_cast<const float *>(OP == 1 ? P.sa1[q] : P.sa2[q]);
      sb[q] = static_cast<const float *>(OP == 1 ? P.sb1[q] : P.sb2[q]);
    }
    const int Lx = P.L[0];
    if (Lx > 0 && (x0 < Lx || x0 + kTX > P.nx - Lx)) {
      for (int t = lane; t < kHT * N * 2; t += 32) {
        const int r = t % kHT, nu = (t / kHT) % N, ab = t / (kHT * N);
        const int y = y0 + r;
        if (y >= P.ny) continue;
        const float *b = (ab ? sb[0] : sa[0]) + nu * P.strip_nu[0] + (long long)y * (2 * Lx);
        for (int o = 0; o < 2 * Lx; o += 32) l2_line(b + o);  // 128-byte lines
      }
    }
    const int Ly = P.L[1];
    if (Ly > 0) {
      for (int t = lane; t < kHT * N * 2; t += 32) {
        const int r = t % kHT, nu = (t / kHT) % N, ab = t / (kHT * N);
        const int y = y0 + r;
        const int sc = y < P.ny ? strip_coord(y, P.ny, Ly) : -1;
        if (sc < 0) continue;
        const float *b = (ab ? sb[1] : sa[1]) + nu * P.strip_nu[1] + (long long)sc * P.pitch + x0;
        for (int o = 0; o < kTX && x0 + o < P.nx; o += 32) l2_line(b + o);
      }
    }
  }
}

template <int N, typename Maps, bool EDGE>
__device__ __forceinline__ void vel_compute(const StepParams &P, const float *tab, float *st, int x0, int y0,
                                            int tid) {
  using S = VelStage<N, Maps>;
  const float *sp = st;
  const float *sr = st + S::kP;
  const float *ss = sr + S::kR;
  const unsigned char *si = reinterpret_cast<const unsigned char *>(ss + S::kS);
  const int t2 = tid & 63, ly = tid >> 6, lx = 2 * t2;
  const int i0 = x0 + lx, j = y0 + ly;
  if (EDGE && (i0 >= P.nx || j >= P.ny)) return;
  float *own = const_cast<float *>(ss) + ly * kTX + lx;
  const long long c = (long long)j * P.pitch + i0;
  const long long Sn = P.npts_alloc;
  float2 Dx, Dy;
  vel_derivs2(P, sp, ly + 3, lx, Dx, Dy);
  float2 k1, A[N > 0 ? N : 1], B[N > 0 ? N : 1];
  if constexpr (S::kIdx) {
    const uchar2 cell = *reinterpret_cast<const uchar2 *>(si + ly * kIW + lx);
    k1 = look2(tab, kTabIk1, cell);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      A[nu] = look2(tab, kTabRelax + nu, cell);
      B[nu] = look2(tab, kTabRelax + kTabSlots + nu, cell);
    }
  } else {
    k1 = sld2(own + (2 + 2 * N) * kArr);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      A[nu] = sld2(own + (3 + 2 * N + nu) * kArr);
      B[nu] = sld2(own + (3 + 3 * N + nu) * kArr);
    }
  }
  // per-axis coefficients; in an edge pair the C-PML strips replace them,
  // every strip value loaded before the first store (one memory latency)
  float2 AX[N > 0 ? N : 1], BX[N > 0 ? N : 1], AY[N > 0 ? N : 1], BY[N > 0 ? N : 1];
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    AX[nu] = A[nu]; BX[nu] = B[nu]; AY[nu] = A[nu]; BY[nu] = B[nu];
  }
  if (EDGE) {
    const int scy = strip_coord(j, P.ny, P.L[1]);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      x_strip_coef2<1, Maps>(P, nu, i0, j, AX[nu], BX[nu]);
      if (scy >= 0) y_strip_coef2<1, Maps>(P, nu, i0, scy, AY[nu], BY[nu]);
    }
  }
  float2 vx = sld2(own), vy = sld2(own + kArr);
  float2 Sx = make_float2(Dx.x * k1.x, Dx.y * k1.y);
  float2 Sy = make_float2(Dy.x * k1.x, Dy.y * k1.y);
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    const float2 px = sld2(own + (2 + nu) * kArr), py = sld2(own + (2 + N + nu) * kArr);
    float2 nx_, ny_;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      el2(nx_, e) = fmaf(el2(BX[nu], e), el2(px, e), el2(AX[nu], e) * el2(Dx, e));
      el2(ny_, e) = fmaf(el2(BY[nu], e), el2(py, e), el2(AY[nu], e) * el2(Dy, e));
      el2(Sx, e) += fmaf(P.w_new, el2(nx_, e), P.w_old * el2(px, e));
      el2(Sy, e) += fmaf(P.w_new, el2(ny_, e), P.w_old * el2(py, e));
    }
    put2<Maps, EDGE>(own, 2 + nu, P.psi1[0], nu * Sn + c, nx_, i0, P.nx);
    put2<Maps, EDGE>(own, 2 + N + nu, P.psi1[1], nu * Sn + c, ny_, i0, P.nx);
  }
  const FaceRho fr = face_rho<Maps, EDGE>(P, tab, sr, si, x0, y0, lx, ly);
  if (P.nl_vel) {
    float2 fx, fy;
    mom_factors2<Maps, EDGE>(P, tab, si, ss + S::kS, sp, ly + 3, lx, ly, x0, y0, fx, fy);
    vx.x = vel_upd(vx.x, qdiv(P.two_dt, fr.r0 + fr.r1), Sx.x, fx.x);
    vx.y = vel_upd(vx.y, qdiv(P.two_dt, fr.r1 + fr.r2), Sx.y, fx.y);
    vy.x = vel_upd(vy.x, qdiv(P.two_dt, fr.r0 + fr.u0), Sy.x, fy.x);
    vy.y = vel_upd(vy.y, qdiv(P.two_dt, fr.r1 + fr.u1), Sy.y, fy.y);
  } else {
    vx.x = vel_upd(vx.x, qdiv(P.two_dt, fr.r0 + fr.r1), Sx.x);
    vx.y = vel_upd(vx.y, qdiv(P.two_dt, fr.r1 + fr.r2), Sx.y);
    vy.x = vel_upd(vy.x, qdiv(P.two_dt, fr.r0 + fr.u0), Sy.x);
    vy.y = vel_upd(vy.y, qdiv(P.two_dt, fr.r1 + fr.u1), Sy.y);
  }
  put2<Maps, EDGE>(own, 0, P.v[0], c, vx, i0, P.nx);
  put2<Maps, EDGE>(own, 1, P.v[1], c, vy, i0, P.nx);
}

template <int N, typename Maps, bool EDGE>
__device__ __forceinline__ void prs_compute(const StepParams &P, const float *tab, float *st, int x0, int y0,
                                            int tid) {
  using S = PrsStage<N, Maps>;
  const float *sx = st, *sy = st + S::kX;
  float *ss = st + S::kX + S::kY;
  const int t2 = tid & 63, ly = tid >> 6, lx = 2 * t2;
  const int i0 = x0 + lx, j = y0 + ly;
  if (EDGE && (i0 >= P.nx || j >= P.ny)) return;
  float *own = ss + ly * kTX + lx;
  const long long c = (long long)j * P.pitch + i0;
  const long long Sn = P.npts_alloc;
  float2 Dx, Dy;
  prs_derivs2(P, sx, sy, ly, lx, Dx, Dy);
  float2 k2, K, ch = make_float2(0.f, 0.f), A[N > 0 ? N : 1], B[N > 0 ? N : 1];
  if constexpr (S::kIdx) {
    const uchar2 cell =
        *reinterpret_cast<const uchar2 *>(reinterpret_cast<const unsigned char *>(ss + S::kS) + ly * kTX + lx);
    k2 = look2(tab, kTabIk2, cell);
    K = look2(tab, kTabK, cell);
    if (P.nl) ch = look2(tab, kTabChi, cell);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      A[nu] = look2(tab, kTabRelax + 2 * kTabSlots + nu, cell);
      B[nu] = look2(tab, kTabRelax + 3 * kTabSlots + nu, cell);
    }
  } else {
    k2 = sld2(own + (1 + 2 * N) * kArr);
    K = sld2(own + (2 + 2 * N) * kArr);
    if (P.nl) ch = sld2(own + (3 + 2 * N) * kArr);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      A[nu] = sld2(own + (4 + 2 * N + nu) * kArr);
      B[nu] = sld2(own + (4 + 3 * N + nu) * kArr);
    }
  }
  float2 AX[N > 0 ? N : 1], BX[N > 0 ? N : 1], AY[N > 0 ? N : 1], BY[N > 0 ? N : 1];
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    AX[nu] = A[nu]; BX[nu] = B[nu]; AY[nu] = A[nu]; BY[nu] = B[nu];
  }
  if (EDGE) {
    const int scy = strip_coord(j, P.ny, P.L[1]);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      x_strip_coef2<2, Maps>(P, nu, i0, j, AX[nu], BX[nu]);
      if (scy >= 0) y_strip_coef2<2, Maps>(P, nu, i0, scy, AY[nu], BY[nu]);
    }
  }
  float2 p = sld2(own);
  float2 Sx = make_float2(Dx.x * k2.x, Dx.y * k2.y);
  float2 Sy = make_float2(Dy.x * k2.x, Dy.y * k2.y);
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    const float2 px = sld2(own + (1 + nu) * kArr), py = sld2(own + (1 + N + nu) * kArr);
    float2 nx_, ny_;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      el2(nx_, e) = fmaf(el2(BX[nu], e), el2(px, e), el2(AX[nu], e) * el2(Dx, e));
      el2(ny_, e) = fmaf(el2(BY[nu], e), el2(py, e), el2(AY[nu], e) * el2(Dy, e));
      el2(Sx, e) += fmaf(P.w_new, el2(nx_, e), P.w_old * el2(px, e));
      el2(Sy, e) += fmaf(P.w_new, el2(ny_, e), P.w_old * el2(py, e));
    }
    put2<Maps, EDGE>(own, 1 + nu, P.psi2[0], nu * Sn + c, nx_, i0, P.nx);
    put2<Maps, EDGE>(own, 1 + N + nu, P.psi2[1], nu * Sn + c, ny_, i0, P.nx);
  }
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    float upd = P.dt * el2(K, e) * (el2(Sx, e) + el2(Sy, e));
    if (P.nl) upd = qdiv(upd, fmaf(el2(ch, e), el2(p, e), 1.f));
    el2(p, e) -= upd;
  }
  put2<Maps, EDGE>(own, 0, P.p, c, p, i0, P.nx);
}

// Ring of stages: as many as fit next to the maps' table (2 .. 4).
template <int N, typename Maps, bool VEL>
struct Ring {
  static constexpr int kStage = VEL ? VelStage<N, Maps>::kFloats : PrsStage<N, Maps>::kFloats;
  static constexpr int kBudget = (224 * 1024 - 128) / 4 - Maps::kSmemFloats;  // floats
  static constexpr int kFit = kBudget / kStage;
  static constexpr int kStages = kFit > 4 ? 4 : kFit;
  // With four stages a stage is refilled one unit after its results were
  // stored (the store has read it by then: no wait on it), two units ahead
  // of its compute; with two or three, right after its store, kStages - 1
  // units ahead.
  static constexpr int kLag = (TmaStore<Maps>::value && kStages >= 4) ? 1 : 0;
  static constexpr int kAhead = kStages - 1 - kLag;
  static constexpr size_t kBytes = sizeof(float) * ((size_t)kStages * kStage + Maps::kSmemFloats) + 128;
  static_assert(kStages >= 2, "two stages must fit in shared memory");
  static_assert(kBytes + 1024 <= 227 * 1024, "stages and table leave 1 KB for static shared memory");
};

// One half step.  Block (32, 16), one per SM.
template <int N, typename Maps, bool VEL>
__global__ void __launch_bounds__(kThreads, 1)
    pipe2d_kernel(const StepParams P, const Region R, const __grid_constant__ PipeMaps T) {
  using G = Ring<N, Maps, VEL>;
  constexpr int kS = G::kStages, kStage = G::kStage;
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ __align__(8) uint64_t bar[kS];
  __shared__ int ok[kS];  // per stage: thread 0 never rewrites a flag a thread has yet to read
  // TMA destinations need 128-byte alignment: round the base up (the launch
  // adds 128 bytes of slack)
  float *smem = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float *tab = smem + kS * kStage;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  stage_table<Maps>(P, tab, tid);  // made visible by the barrier below
  if (tid == 0) {
    for (int q = 0; q < kS; ++q) mbar_init(&bar[q], 1);
    fence_mbarrier_init();
  }
  __syncthreads();
  const int nh = R.halves();
  int h = blockIdx.x;
  if (h >= nh) return;
  // this block's half tiles are h, h + grid, ...; the first kS - 1 go out now,
  // then each iteration issues one more into the stage freed last
  unsigned phase = 0;    // bit q: parity of the next completion of stage q
  unsigned pending = 0;  // bit q: copies issued into stage q, not consumed
  int hs = h;            // next half tile to issue
  for (int q = 0; q < G::kAhead; ++q, hs += gridDim.x) {
    if (hs >= nh) break;
    if (tid == 0) {
      int xq, yq;
      R.half_origin(hs, xq, yq);
      issue_stage<N, Maps, VEL>(P, T, smem + q * kStage, &bar[q], xq, yq);
    }
    pending |= 1u << q;
  }
  int s = 0;
  // One barrier per half tile: after the wait for stage s it also marks
  // the previous half tile computed, so its stage is refilled (and, with
  // TMA stores, its results sent) right after it.
  int xp = -1, yp = -1;  // previous half tile of this block
#pragma unroll 1
  for (; h < nh; h += gridDim.x) {
    if (tid == 0) ok[s] = mbar_wait_bounded(&bar[s], (phase >> s) & 1u);
    __syncthreads();
    if (!ok[s]) {
      if (tid == 0) {
        report_status(P.status, kStatusWaitTimeout);
        for (int q = 0; q < kS; ++q)
          if (q != s && ((pending >> q) & 1u)) mbar_wait_bounded(&bar[q], (phase >> q) & 1u);
        bulk_wait_all();
      }
      return;
    }
    phase ^= 1u << s;
    pending &= ~(1u << s);
    const int sp = (s + kS - 1) % kS;       // the previous half tile's stage
    const int q = (s + G::kAhead) % kS;     // the stage refilled now
    if constexpr (TmaStore<Maps>::value) {
      if (tid == 0 && xp >= 0) store_stage<N, Maps, VEL>(T, smem + sp * kStage, xp, yp);
    }
    if (hs < nh) {
      if (tid < 32) {
        int xq, yq;
        R.half_origin(hs, xq, yq);
        if (tid == 0) {
          bulk_wait_read<G::kLag>();
          issue_stage<N, Maps, VEL>(P, T, smem + q * kStage, &bar[q], xq, yq);
        }
        if (!R.interior(xq, yq)) prefetch_strips2<N, VEL ? 1 : 2>(P, xq, yq, tid);
      }
      pending |= 1u << q;
      hs += gridDim.x;
    }
    int x0, y0;
    R.half_origin(h, x0, y0);
    float *cur = smem + s * kStage;
    if (R.interior(x0, y0)) {
      if (VEL) vel_compute<N, Maps, false>(P, tab, cur, x0, y0, tid);
      else prs_compute<N, Maps, false>(P, tab, cur, x0, y0, tid);
    } else {
      if (VEL) vel_compute<N, Maps, true>(P, tab, cur, x0, y0, tid);
      else prs_compute<N, Maps, true>(P, tab, cur, x0, y0, tid);
    }
    if constexpr (TmaStore<Maps>::value) fence_proxy_async_smem();
    xp = x0;
    yp = y0;
    s = (s + 1) % kS;
  }
  if constexpr (TmaStore<Maps>::value) {
    __syncthreads();
    if (tid == 0 && xp >= 0) store_stage<N, Maps, VEL>(T, smem + ((s + kS - 1) % kS) * kStage, xp, yp);
  }
  if (tid == 0) bulk_wait_all();
}

// Batched half step over a unit table of several contexts (one group: same
// N and map kind, no periodic axis): entry (ctx, x0, y0, interior).  The
// contexts' step parameters and tensor maps sit in device memory (TMA reads
// the maps from there); a block copies a context's parameters to shared
// memory, and stages its tissue-index table, when the context changes.
template <int N, typename Maps, bool VEL>
__global__ void __launch_bounds__(kThreads, 1)
    pipe2d_batched_kernel(const StepParams *Ps, const PipeMaps *Ts, const int4 *units, const int *runs) {
  using G = Ring<N, Maps, VEL>;
  constexpr int kS = G::kStages, kStage = G::kStage;
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ __align__(8) uint64_t bar[kS];
  __shared__ __align__(16) StepParams sP;
  __shared__ int ok[kS];  // per stage: thread 0 never rewrites a flag a thread has yet to read
  float *smem = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float *tab = smem + kS * kStage;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid == 0) {
    for (int q = 0; q < kS; ++q) mbar_init(&bar[q], 1);
    fence_mbarrier_init();
  }
  __syncthreads();
  // a contiguous run of units per block (runs[b] .. runs[b + 1]; the host
  // balances the runs by the units' cost): consecutive units share a context
  // (one parameter and table load per context) and halo rows (L2)
  const int h_end = runs[blockIdx.x + 1];
  int h = runs[blockIdx.x];
  if (h >= h_end) return;
  unsigned phase = 0, pending = 0;
  // thread 0: the context whose tensor maps it last acquired (the runs of
  // units are contiguous per context, so each map is acquired about once)
  int fenced = -1;
  auto acquire = [&](int c) {
    if (c == fenced) return;
    for (int m = 0; m < kPipeMaps; ++m) fence_tensormap_acquire(&Ts[c].m[m]);
    fenced = c;
  };
  int hs = h;
  for (int q = 0; q < G::kAhead; ++q, ++hs) {
    if (hs >= h_end) break;
    if (tid == 0) {
      const int4 e = units[hs];
      acquire(e.x);
      issue_stage<N, Maps, VEL>(Ps[e.x], Ts[e.x], smem + q * kStage, &bar[q], e.y, e.z);
    }
    pending |= 1u << q;
  }
  int s = 0, cur = -1;
  // one barrier per unit (see pipe2d_kernel); a context change adds one
  int4 prev = make_int4(-1, 0, 0, 0);
#pragma unroll 1
  for (; h < h_end; ++h) {
    if (tid == 0) ok[s] = mbar_wait_bounded(&bar[s], (phase >> s) & 1u);
    __syncthreads();
    if (!ok[s]) {
      if (tid == 0) {
        report_status(Ps[units[h].x].status, kStatusWaitTimeout);
        for (int q = 0; q < kS; ++q)
          if (q != s && ((pending >> q) & 1u)) mbar_wait_bounded(&bar[q], (phase >> q) & 1u);
        bulk_wait_all();
      }
      return;
    }
    phase ^= 1u << s;
    pending &= ~(1u << s);
    const int sp = (s + kS - 1) % kS;       // the previous unit's stage
    const int q = (s + G::kAhead) % kS;     // the stage refilled now
    if constexpr (TmaStore<Maps>::value) {
      if (tid == 0 && prev.x >= 0) store_stage<N, Maps, VEL>(Ts[prev.x], smem + sp * kStage, prev.y, prev.z);
    }
    const int4 e = units[h];
    if (e.x != cur) {
      // new context: parameters (and index table) into shared memory
      const int *src = reinterpret_cast<const int *>(Ps + e.x);
      int *dst = reinterpret_cast<int *>(&sP);
      for (int w = tid; w < (int)(sizeof(StepParams) / 4); w += kThreads) dst[w] = __ldg(src + w);
      __syncthreads();
      stage_table<Maps>(sP, tab, tid);
      __syncthreads();
      cur = e.x;
    }
    if (hs < h_end) {
      if (tid < 32) {
        const int4 en = units[hs];
        if (tid == 0) {
          bulk_wait_read<G::kLag>();
          acquire(en.x);
          issue_stage<N, Maps, VEL>(Ps[en.x], Ts[en.x], smem + q * kStage, &bar[q], en.y, en.z);
        }
        if (!en.w && en.x == cur) prefetch_strips2<N, VEL ? 1 : 2>(sP, en.y, en.z, tid);
      }
      pending |= 1u << q;
      ++hs;
    }
    float *stp = smem + s * kStage;
    if (e.w) {
      if (VEL) vel_compute<N, Maps, false>(sP, tab, stp, e.y, e.z, tid);
      else prs_compute<N, Maps, false>(sP, tab, stp, e.y, e.z, tid);
    } else {
      if (VEL) vel_compute<N, Maps, true>(sP, tab, stp, e.y, e.z, tid);
      else prs_compute<N, Maps, true>(sP, tab, stp, e.y, e.z, tid);
    }
    if constexpr (TmaStore<Maps>::value) fence_proxy_async_smem();
    prev = e;
    s = (s + 1) % kS;
  }
  if constexpr (TmaStore<Maps>::value) {
    __syncthreads();
    if (tid == 0 && prev.x >= 0)
      store_stage<N, Maps, VEL>(Ts[prev.x], smem + ((s + kS - 1) % kS) * kStage, prev.y, prev.z);
  }
  if (tid == 0) bulk_wait_all();
}

template <int N, typename Maps, bool VEL>
cudaError_t pipe_batched_launch(const StepParams *Ps, const PipeMaps *Ts, const int4 *units, const int *runs, int grid,
                                cudaStream_t st) {
  constexpr size_t bytes = Ring<N, Maps, VEL>::kBytes;
  cudaError_t e = cudaFuncSetAttribute(pipe2d_batched_kernel<N, Maps, VEL>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  pipe2d_batched_kernel<N, Maps, VEL><<<grid, dim3(32, kThreads / 32), bytes, st>>>(Ps, Ts, units, runs);
  return cudaGetLastError();
}

template <typename Maps, bool VEL>
cudaError_t pipe_batched_dispatch(const StepParams *Ps, const PipeMaps *Ts, const int4 *units, const int *runs,
                                  int n_relax, int grid, cudaStream_t st) {
  switch (n_relax) {
    case 0: return pipe_batched_launch<0, Maps, VEL>(Ps, Ts, units, runs, grid, st);
    case 1: return pipe_batched_launch<1, Maps, VEL>(Ps, Ts, units, runs, grid, st);
    case 2: return pipe_batched_launch<2, Maps, VEL>(Ps, Ts, units, runs, grid, st);
    case 3: return pipe_batched_launch<3, Maps, VEL>(Ps, Ts, units, runs, grid, st);
    case 4: return pipe_batched_launch<4, Maps, VEL>(Ps, Ts, units, runs, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int N, typename Maps, bool VEL>
cudaError_t pipe_launch(const StepParams &P, const Region &R, int grid, const PipeMaps &T, cudaStream_t st) {
  constexpr size_t bytes = Ring<N, Maps, VEL>::kBytes;
  cudaError_t e = cudaFuncSetAttribute(pipe2d_kernel<N, Maps, VEL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)bytes);
  if (e != cudaSuccess) return e;
  pipe2d_kernel<N, Maps, VEL><<<grid, dim3(32, kThreads / 32), bytes, st>>>(P, R, T);
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
  R.ntx = (P.nx + kTX - 1) / kTX;
  R.nhy = (P.ny + kHT - 1) / kHT;
  return R;
}

}  // namespace

bool pipe2d_supported(const StepParams &P, int map_kind) {
  // the copies read zero outside the grid: the zero-outside boundary only
  return P.nz == 1 && (map_kind == 0 || map_kind == 2) && P.n_relax >= 0 && P.n_relax <= kPipe2dMaxRelax &&
         !P.periodic[0] && !P.periodic[1];
}

bool pipe2d_preferred(const StepParams &P, int map_kind) { return pipe2d_supported(P, map_kind); }

bool pipe2d_interior_half(const StepParams &P, int x0, int y0) {
  const int Lx = P.L[0] > 4 ? P.L[0] : 4, Ly = P.L[1] > 4 ? P.L[1] : 4;
  return x0 >= Lx && x0 + kTX + Lx <= P.nx && y0 >= Ly && y0 + kHT + Ly <= P.ny;
}

cudaError_t launch_pipe2d_batched(bool vel, const StepParams *Ps, const PipeMaps *Ts, const int4 *units,
                                  int n_units, const int *runs, int n_relax, int map_kind, int grid,
                                  cudaStream_t st) {
  if (n_units <= 0) return cudaSuccess;
  if (map_kind == 2)
    return vel ? pipe_batched_dispatch<IdxMaps, true>(Ps, Ts, units, runs, n_relax, grid, st)
               : pipe_batched_dispatch<IdxMaps, false>(Ps, Ts, units, runs, n_relax, grid, st);
  if (map_kind == 0)
    return vel ? pipe_batched_dispatch<DenseMaps<float>, true>(Ps, Ts, units, runs, n_relax, grid, st)
               : pipe_batched_dispatch<DenseMaps<float>, false>(Ps, Ts, units, runs, n_relax, grid, st);
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
  if (dense && P.nl_vel) ok = ok && encode(&vel->m[9], P.K, P, 2, 1, S, kRWp, kHT + 1, 1);
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
