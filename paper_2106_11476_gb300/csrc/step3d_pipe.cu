// Pipelined persistent 3D half steps (sm_103a) for bf16 coefficient maps;
// same arithmetic as step3d.cu (bitwise the same results), one launch per
// half step, one block of 512 threads per SM (two x cells per thread).
//
// Work unit: a 128 x 8 half tile of one z plane.  A block marches a column
// of units through z (a work item: one xy position and a range of planes;
// items are numbered xy position first, so the blocks running at one time
// hold neighbouring columns at about the same depth and share the halo rows
// in L2).  The operand planes a unit's z taps need stay in a ring of nine
// plane slots in shared memory (velocity: p planes k-3 .. k+4 with their xy
// halo, which also give the x and y taps; pressure: v_z planes k-4 .. k+3), so
// each unit adds one plane.  For a coming unit one thread issues tiled TMA
// tensor copies, one box per array, into a free stage of a two-stage ring:
// the operand plane the unit adds (into the plane ring), the density of the
// plane and of the next one, the velocity (or pressure) of the unit, all 3N
// memory variables of the half step in one 4D box, and the bf16 maps (a and b
// of the N mechanisms in one 4D box each).  The first unit of an item loads
// its eight planes after the previous unit's compute.  Copies complete on
// the stage's mbarrier while all threads compute the current unit from the
// other stage; no computing thread issues a global load outside the C-PML
// strips.
//
// Boundaries as in the 2D pipeline: the copies read zero outside the grid;
// units at the grid's edge or in a C-PML strip clamp the density to the last
// cell, take each axis' C-PML coefficients from its strip (all mechanisms
// loaded before the first store) and store nothing outside the grid.
// Periodic axes are not taken by this path (the tile kernels run them).
#include "async.cuh"
#include "coef.cuh"
#include "tmap.h"

namespace fw2 {

namespace {

constexpr int kHT = 8;            // rows of a unit
constexpr int kCW = kTX + 8;      // operand halo columns x0-4 .. x0+TX+3
constexpr int kRWb = kTX + 8;     // staged bf16 density columns x0 .. x0+TX+7 (16-byte rows)
constexpr int kArr = kHT * kTX;   // elements of one array per unit

using bf16 = __nv_bfloat16;

constexpr int round32(int n) { return (n + 31) & ~31; }  // floats: 128-byte regions
constexpr int fl(int bytes) { return (bytes + 3) / 4; }

// ------------------------------------------------------------- stages ---
constexpr int kSlots = 9;  // plane ring: the eight planes of a unit and the one the next unit adds
constexpr int kXsMax = 64; // widest x C-PML strip (cells per side) staged by TMA

// x-strip region of a stage: a then b, each [N][8][L] bf16 (L <= kXsMax)
template <int N>
struct XStrip {
  static constexpr int kHalf = N * kHT * kXsMax / 2;  // floats of a (or b); 128-byte multiple
  static constexpr int kFloats = 2 * kHalf;
};

__host__ __device__ constexpr int ring_slot(int k) { return ((k % kSlots) + kSlots) % kSlots; }

// velocity stage: density bf16 [2][9][136] (planes k, k+1), v [3][8][128],
// psi1 [3N][8][128], 1/kappa1 bf16 [8][128], a1, b1 bf16 [N][8][128];
// plane ring: p planes [15][136] (rows y0-3 .. y0+11, columns x0-4 ..)
template <int N>
struct Vel3 {
  static constexpr int kRho = round32(fl(2 * (kHT + 1) * kRWb * 2));
  static constexpr int kV = 3 * kArr;
  static constexpr int kPsi = 3 * N * kArr;
  static constexpr int kK = round32(fl(kArr * 2));
  static constexpr int kAB = round32(fl(N * kArr * 2));
  static constexpr int oRho = 0, oV = oRho + kRho, oPsi = oV + kV, oK = oPsi + kPsi, oA = oK + kK, oB = oA + kAB,
                       oXs = oB + kAB;
  static constexpr int kFloats = round32(oXs + XStrip<N>::kFloats);
  static constexpr unsigned kBytes = 4u * (kV + kPsi) + 2u * (2 * (kHT + 1) * kRWb + kArr + 2 * N * kArr);
  static constexpr int kPlane = round32((kHT + 7) * kCW);
  static constexpr unsigned kPlaneBytes = 4u * (kHT + 7) * kCW;
};

// pressure stage: v_x plane [8][136] (x halo), v_y plane [15][128] (rows
// y0-4 ..), p [8][128], psi2 [3N][8][128], 1/kappa2, K, chi bf16 [8][128],
// a2, b2 bf16 [N][8][128]; plane ring: v_z planes [8][128]
template <int N>
struct Prs3 {
  static constexpr int kVx = round32(kHT * kCW);
  static constexpr int kVy = round32((kHT + 7) * kTX);
  static constexpr int kP = kArr;
  static constexpr int kPsi = 3 * N * kArr;
  static constexpr int kK = round32(fl(kArr * 2));
  static constexpr int kAB = round32(fl(N * kArr * 2));
  static constexpr int oVx = 0, oVy = oVx + kVx, oP = oVy + kVy, oPsi = oP + kP, oIk = oPsi + kPsi,
                       oKm = oIk + kK, oChi = oKm + kK, oA = oChi + kK, oB = oA + kAB, oXs = oB + kAB;
  static constexpr int kFloats = round32(oXs + XStrip<N>::kFloats);
  static constexpr unsigned kBytesNoChi =
      4u * (kHT * kCW + (kHT + 7) * kTX + kP + kPsi) + 2u * (2 * kArr + 2 * N * kArr);
  static constexpr int kPlane = kArr;
  static constexpr unsigned kPlaneBytes = 4u * kArr;
};

template <int N, bool VEL>
struct Ring3 {
  static constexpr int kStage = VEL ? Vel3<N>::kFloats : Prs3<N>::kFloats;
  static constexpr int kPlane = VEL ? Vel3<N>::kPlane : Prs3<N>::kPlane;
  static constexpr unsigned kPlaneBytes = VEL ? Vel3<N>::kPlaneBytes : Prs3<N>::kPlaneBytes;
  static constexpr size_t kBytes = sizeof(float) * (2 * (size_t)kStage + (size_t)kSlots * kPlane) + 128;
};

// Work items: a column of units (xy position, x fastest) and a range of
// planes; item it covers column it % ncols, planes seg * seglen ..
struct Region3 {
  int nx, ny, nz, Lx, Ly, Lz;
  int tnx, nhy;      // x tiles, half-tile rows per plane
  int seglen, nseg;  // planes per item, items per column
  int xsL;           // x C-PML strip cells per side when its coefficients come by TMA, else 0
  // the side of the x strip a unit at x0 reaches: 0 low, 1 high, -1 none
  // (with xsL set no unit reaches both)
  __device__ __forceinline__ int xs_side(int x0) const {
    if (xsL == 0) return -1;
    return x0 < xsL ? 0 : (x0 + kTX > nx - xsL ? 1 : -1);
  }
  __device__ __forceinline__ long long items() const { return (long long)tnx * nhy * nseg; }
  __device__ __forceinline__ void item(long long it, int &x0, int &y0, int &k0, int &k1) const {
    const int ncols = tnx * nhy;
    const int col = (int)(it % ncols), seg = (int)(it / ncols);
    x0 = (col % tnx) * kTX;
    y0 = (col / tnx) * kHT;
    k0 = seg * seglen;
    k1 = min(nz, k0 + seglen);
  }
  __device__ __forceinline__ bool interior(int x0, int y0, int k) const {
    return x0 >= Lx && x0 + kTX + Lx <= nx && y0 >= Ly && y0 + kHT + Ly <= ny && k >= Lz && k + Lz < nz;
  }
};

// first plane of the operand ring a unit at plane k reads (8 planes)
template <bool VEL>
__host__ __device__ constexpr int ring_first(int k) { return VEL ? k - 3 : k - 4; }

// Issue the copies of a unit at (x0, y0, k): its stage and the operand
// planes k_lo .. k_hi of the plane ring (one plane, or eight for the first
// unit of an item), all completing on the stage's mbarrier.
template <int N, bool VEL>
__device__ __forceinline__ void issue3(const PipeMaps &T, float *st, float *ring, uint64_t *bar, int x0, int y0,
                                       int k, int k_lo, int k_hi, bool nl, int xs_side, int xsL) {
  using G = Ring3<N, VEL>;
  fence_proxy_async_smem();
  const unsigned planes = G::kPlaneBytes * (unsigned)(k_hi - k_lo + 1);
  // the x strip's coefficients of the unit's rows: one box of a and one of b
  // (L values of the side the unit reaches, all mechanisms)
  const unsigned xs = (N > 0 && xs_side >= 0) ? 2u * 2u * (unsigned)(N * kHT * xsL) : 0u;
  auto load_xs = [&] {
    if (xs) {
      float *d = st + (VEL ? Vel3<N>::oXs : Prs3<N>::oXs);
      tma_load_4d(d, &T.m[10], xs_side * xsL, y0, k, 0, bar);
      tma_load_4d(d + XStrip<N>::kHalf, &T.m[11], xs_side * xsL, y0, k, 0, bar);
    }
  };
  if (VEL) {
    using S = Vel3<N>;
    mbar_arrive_expect_tx(bar, S::kBytes + planes + xs);
    load_xs();
    for (int kp = k_lo; kp <= k_hi; ++kp) tma_load_3d(ring + ring_slot(kp) * G::kPlane, &T.m[0], x0 - 4, y0 - 3, kp, bar);
    tma_load_3d(st + S::oRho, &T.m[2], x0, y0, k, bar);
    tma_load_4d(st + S::oV, &T.m[3], x0, y0, k, 0, bar);
    if (N > 0) tma_load_4d(st + S::oPsi, &T.m[4], x0, y0, k, 0, bar);
    tma_load_3d(st + S::oK, &T.m[5], x0, y0, k, bar);
    if (N > 0) {
      tma_load_4d(st + S::oA, &T.m[6], x0, y0, k, 0, bar);
      tma_load_4d(st + S::oB, &T.m[7], x0, y0, k, 0, bar);
    }
  } else {
    using S = Prs3<N>;
    mbar_arrive_expect_tx(bar, S::kBytesNoChi + (nl ? 2u * kArr : 0u) + planes + xs);
    load_xs();
    for (int kp = k_lo; kp <= k_hi; ++kp) tma_load_3d(ring + ring_slot(kp) * G::kPlane, &T.m[2], x0, y0, kp, bar);
    tma_load_3d(st + S::oVx, &T.m[0], x0 - 4, y0, k, bar);
    tma_load_3d(st + S::oVy, &T.m[1], x0, y0 - 4, k, bar);
    tma_load_3d(st + S::oP, &T.m[3], x0, y0, k, bar);
    if (N > 0) tma_load_4d(st + S::oPsi, &T.m[4], x0, y0, k, 0, bar);
    tma_load_3d(st + S::oIk, &T.m[5], x0, y0, k, bar);
    tma_load_3d(st + S::oKm, &T.m[6], x0, y0, k, bar);
    if (nl) tma_load_3d(st + S::oChi, &T.m[7], x0, y0, k, bar);
    if (N > 0) {
      tma_load_4d(st + S::oA, &T.m[8], x0, y0, k, 0, bar);
      tma_load_4d(st + S::oB, &T.m[9], x0, y0, k, 0, bar);
    }
  }
}

// ------------------------------------------------------------ compute ---
// 512 threads, two consecutive x cells each (64 threads per row); every cell
// sees the operations of the tile kernels in the same order.
constexpr int kThreads = 512;

__device__ __forceinline__ float2 sld2(const float *s) { return *reinterpret_cast<const float2 *>(s); }
__device__ __forceinline__ float2 sldh2(const bf16 *s) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(s));
}
__device__ __forceinline__ float2 sldb2(const bf16 *s) {  // bf16 maps hold 1 - b
  const float2 v = sldh2(s);
  return make_float2(1.f - v.x, 1.f - v.y);
}
__device__ __forceinline__ void st_state2(float *p, long long i, float2 v) {
  __stcs(reinterpret_cast<float2 *>(p + i), v);
}
__device__ __forceinline__ float &el2(float2 &v, int e) { return e == 0 ? v.x : v.y; }
__device__ __forceinline__ float el2(const float2 &v, int e) { return e == 0 ? v.x : v.y; }
__device__ __forceinline__ float2 mask_pad2(float2 v, int i0, int nx) {
  if (i0 + 1 >= nx) v.y = 0.f;
  if (i0 >= nx) v.x = 0.f;
  return v;
}
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

// a, b along axis Q (OP: 1 faces, 2 centres) of mechanism nu at the two
// cells of an edge pair, from that axis' C-PML strip where the cells lie in
// it (coef4 of the tile kernels; its zero beyond the grid only reaches
// masked cells); unchanged elsewhere
template <int Q, int OP>
__device__ __forceinline__ void strip3(const StepParams &P, int nu, int i0, int j, int k, float2 &a, float2 &b) {
  const bf16 *sa = static_cast<const bf16 *>(OP == 1 ? P.sa1[Q] : P.sa2[Q]);
  const bf16 *sb = static_cast<const bf16 *>(OP == 1 ? P.sb1[Q] : P.sb2[Q]);
  const int L = P.L[Q];
  if (L <= 0) return;
  if (Q == 0) {
    if (!(i0 < L || i0 + 1 >= P.nx - L)) return;
    const long long row = (long long)nu * P.strip_nu[0] + ((long long)k * P.ny + j) * (2 * L);
    // both cells on one side of the strip: one aligned bf16 pair (i0 and
    // the high side's offset nx - 2L are even)
    int sc0 = -1;
    if (i0 + 1 < L) sc0 = i0;
    else if (i0 >= P.nx - L && i0 + 1 < P.nx && ((P.nx - 2 * L) & 1) == 0) sc0 = i0 - (P.nx - 2 * L);
    if (sc0 >= 0) {
      const float2 va = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(sa + row + sc0));
      const float2 vb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(sb + row + sc0));
      a = va;
      b = make_float2(1.f - vb.x, 1.f - vb.y);
      return;
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int x = i0 + e;
      if (x < P.nx) {
        const int sc = strip_coord(x, P.nx, L);
        if (sc >= 0) {
          el2(a, e) = ldmap(sa, row + sc);
          el2(b, e) = ldb(sb, row + sc);
        }
      }
    }
  } else {
    const int sc = Q == 1 ? strip_coord(j, P.ny, L) : strip_coord(k, P.nz, L);
    if (sc < 0) return;
    const long long off = Q == 1 ? (long long)nu * P.strip_nu[1] + ((long long)k * (2 * L) + sc) * P.pitch + i0
                                 : (long long)nu * P.strip_nu[2] + ((long long)sc * P.ny + j) * P.pitch + i0;
    // i0 even, pitch a multiple of 16: an aligned bf16 pair
    const float2 va = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(sa + off));
    const float2 vb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(sb + off));
    a = va;
    b = make_float2(1.f - vb.x, 1.f - vb.y);
  }
}

// a, b of the x strip at the two cells of an edge pair from the staged boxes
// (a then b, each [N][8][L] bf16, the side the unit reaches): the values
// strip3<0> reads from global memory, for the cells in the strip
__device__ __forceinline__ void strip3x_staged(const StepParams &P, const bf16 *xa, const bf16 *xb, int xsL, int nu,
                                               int i0, int ly, float2 &a, float2 &b) {
  const int L = P.L[0];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int x = i0 + e;
    if (x < P.nx) {
      const int sc = strip_coord(x, P.nx, L);
      if (sc >= 0) {
        const int i = (nu * kHT + ly) * xsL + (sc >= L ? sc - L : sc);
        el2(a, e) = __bfloat162float(xa[i]);
        el2(b, e) = 1.f - __bfloat162float(xb[i]);
      }
    }
  }
}

// Prefetch into L2 the C-PML strip rows an edge unit will read (warp 0, one
// unit ahead): its C-PML coefficients are otherwise read straight from DRAM
// while the unit computes.  OP: 1 velocity (a1, b1), 2 pressure (a2, b2).
__device__ __forceinline__ void l2_line(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
template <int N, int OP>
__device__ __forceinline__ void prefetch_strips(const StepParams &P, int x0, int y0, int k, int lane, bool xs_staged) {
  if constexpr (N > 0) {
    const bf16 *sa[3], *sb[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      sa[q] = static_cast<const bf16 *>(OP == 1 ? P.sa1[q] : P.sa2[q]);
      sb[q] = static_cast<const bf16 *>(OP == 1 ? P.sb1[q] : P.sb2[q]);
    }
    // x strip: rows (k, y) of 2L values, for units reaching into it
    const int Lx = P.L[0];
    if (!xs_staged && Lx > 0 && (x0 < Lx || x0 + kTX > P.nx - Lx)) {
      for (int t = lane; t < kHT * N * 2; t += 32) {
        const int r = t % kHT, nu = (t / kHT) % N, ab = t / (kHT * N);
        const int y = y0 + r;
        if (y >= P.ny) continue;
        const bf16 *b = (ab ? sb[0] : sa[0]) + nu * P.strip_nu[0] + ((long long)k * P.ny + y) * (2 * Lx);
        for (int o = 0; o < 2 * Lx; o += 64) l2_line(b + o);  // 128-byte lines
      }
    }
    // y strip: rows (k, sc) of the unit's 128 columns
    const int Ly = P.L[1];
    if (Ly > 0) {
      for (int t = lane; t < kHT * N * 2; t += 32) {
        const int r = t % kHT, nu = (t / kHT) % N, ab = t / (kHT * N);
        const int y = y0 + r;
        const int sc = y < P.ny ? strip_coord(y, P.ny, Ly) : -1;
        if (sc < 0) continue;
        const bf16 *b = (ab ? sb[1] : sa[1]) + nu * P.strip_nu[1] + ((long long)k * (2 * Ly) + sc) * P.pitch + x0;
        l2_line(b);
        if (x0 + 64 < P.nx) l2_line(b + 64);
      }
    }
    // z strip: plane sc, rows y of the unit
    const int Lz = P.L[2];
    const int scz = Lz > 0 ? strip_coord(k, P.nz, Lz) : -1;
    if (scz >= 0) {
      for (int t = lane; t < kHT * N * 2; t += 32) {
        const int r = t % kHT, nu = (t / kHT) % N, ab = t / (kHT * N);
        const int y = y0 + r;
        if (y >= P.ny) continue;
        const bf16 *b = (ab ? sb[2] : sa[2]) + nu * P.strip_nu[2] + ((long long)scz * P.ny + y) * P.pitch + x0;
        l2_line(b);
        if (x0 + 64 < P.nx) l2_line(b + 64);
      }
    }
  }
}

// Densities at the faces of a pair, read from the staged bf16 box [2][9][136]
// (planes k, k + 1) where the thread needs them: plane k row ly at lx .. lx+2,
// row ly+1 at lx, lx+1; plane k+1 row ly at lx, lx+1.  Cells beyond the last
// one along an axis take that cell's value (rho_coord of the tile kernels).
struct FaceRho3 {
  float r0, r1, r2, u0, u1, z0, z1;
};
template <bool EDGE>
__device__ __forceinline__ FaceRho3 face_rho3(const StepParams &P, const bf16 *rb, int x0, int y0, int k, int lx,
                                              int ly) {
  int c0 = lx, c1 = lx + 1, c2 = lx + 2, r0 = ly, r1 = ly + 1, pz = 1;
  if (EDGE) {
    const int mx = P.nx - 1 - x0, my = P.ny - 1 - y0;
    c0 = min(c0, mx);
    c1 = min(c1, mx);
    c2 = min(c2, mx);
    r0 = min(r0, my);
    r1 = min(r1, my);
    if (k + 1 >= P.nz) pz = 0;
  }
  auto at = [&](int z, int r, int cc) { return __bfloat162float(rb[(z * (kHT + 1) + r) * kRWb + cc]); };
  return FaceRho3{at(0, r0, c0), at(0, r0, c1), at(0, r0, c2), at(0, r1, c0), at(0, r1, c1),
                  at(pz, r0, c0), at(pz, r0, c1)};
}

template <int N, bool EDGE>
__device__ __forceinline__ void vel3_compute(const StepParams &P, float *st, const float *ring, int x0, int y0, int k,
                                             int tid, int xs_side, int xsL) {
  using S = Vel3<N>;
  const int lx = 2 * (tid & 63), ly = tid >> 6;
  const int i0 = x0 + lx, j = y0 + ly;
  if (EDGE && (i0 >= P.nx || j >= P.ny)) return;
  const long long c = (long long)k * P.plane + (long long)j * P.pitch + i0;
  const long long Sn = P.npts_alloc;
  const int o = ly * kTX + lx;
  // derivatives: x, y from the halo plane of k (cell e at column lx + 4 + e),
  // z from the same cell of planes k-3 .. k+4 in the ring
  constexpr int kPl = Vel3<N>::kPlane;
  const float *sp = ring + ring_slot(k) * kPl;
  const int sy = ly + 3;
  float2 Dx, Dy, Dz;
  {
    const Win10 w = win10(sp + sy * kCW, lx);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m] - w.v[4 + e - m + 1], d);
      el2(Dx, e) = d;
    }
  }
  {
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
  }
  {
    float2 zc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) zc[m] = sld2(ring + ring_slot(k - 3 + m) * kPl + sy * kCW + lx + 4);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el2(zc[3 + m], e) - el2(zc[4 - m], e), d);
      el2(Dz, e) = d;
    }
  }
  const float2 k1 = sldh2(reinterpret_cast<const bf16 *>(st + S::oK) + o);
  float2 A[3][N > 0 ? N : 1], B[3][N > 0 ? N : 1];
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    const float2 a = sldh2(reinterpret_cast<const bf16 *>(st + S::oA) + nu * kArr + o);
    const float2 b = sldb2(reinterpret_cast<const bf16 *>(st + S::oB) + nu * kArr + o);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      A[q][nu] = a;
      B[q][nu] = b;
    }
  }
  if (EDGE) {
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      if (xs_side >= 0)
        strip3x_staged(P, reinterpret_cast<const bf16 *>(st + S::oXs),
                       reinterpret_cast<const bf16 *>(st + S::oXs + XStrip<N>::kHalf), xsL, nu, i0, ly, A[0][nu],
                       B[0][nu]);
      else
        strip3<0, 1>(P, nu, i0, j, k, A[0][nu], B[0][nu]);
      strip3<1, 1>(P, nu, i0, j, k, A[1][nu], B[1][nu]);
      strip3<2, 1>(P, nu, i0, j, k, A[2][nu], B[2][nu]);
    }
  }
  float2 v0 = sld2(st + S::oV + o), v1 = sld2(st + S::oV + kArr + o), v2 = sld2(st + S::oV + 2 * kArr + o);
  float2 S0, S1, S2;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    el2(S0, e) = el2(Dx, e) * el2(k1, e);
    el2(S1, e) = el2(Dy, e) * el2(k1, e);
    el2(S2, e) = el2(Dz, e) * el2(k1, e);
  }
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    const float2 q0 = sld2(st + S::oPsi + nu * kArr + o);
    const float2 q1 = sld2(st + S::oPsi + (N + nu) * kArr + o);
    const float2 q2 = sld2(st + S::oPsi + (2 * N + nu) * kArr + o);
    float2 n0, n1, n2;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      el2(n0, e) = fmaf(el2(B[0][nu], e), el2(q0, e), el2(A[0][nu], e) * el2(Dx, e));
      el2(n1, e) = fmaf(el2(B[1][nu], e), el2(q1, e), el2(A[1][nu], e) * el2(Dy, e));
      el2(n2, e) = fmaf(el2(B[2][nu], e), el2(q2, e), el2(A[2][nu], e) * el2(Dz, e));
      el2(S0, e) += fmaf(P.w_new, el2(n0, e), P.w_old * el2(q0, e));
      el2(S1, e) += fmaf(P.w_new, el2(n1, e), P.w_old * el2(q1, e));
      el2(S2, e) += fmaf(P.w_new, el2(n2, e), P.w_old * el2(q2, e));
    }
    if (EDGE) {
      n0 = mask_pad2(n0, i0, P.nx);
      n1 = mask_pad2(n1, i0, P.nx);
      n2 = mask_pad2(n2, i0, P.nx);
    }
    st_state2(P.psi1[0], nu * Sn + c, n0);
    st_state2(P.psi1[1], nu * Sn + c, n1);
    st_state2(P.psi1[2], nu * Sn + c, n2);
  }
  const FaceRho3 f = face_rho3<EDGE>(P, reinterpret_cast<const bf16 *>(st + S::oRho), x0, y0, k, lx, ly);
  const float rr[3] = {f.r0, f.r1, f.r2}, ru[2] = {f.u0, f.u1}, rz[2] = {f.z0, f.z1};
  if (P.nl_vel) {
    // momentum factors of the literal system (Eq. general5) at the x, y, z
    // faces: p from the staged planes (zero beyond the grid), K of the cell
    // and of its +1 neighbours from the map, clamped to the last cell
    const bf16 *Km = static_cast<const bf16 *>(P.K);
    const int jn = min(j + 1, P.ny - 1), kn = min(k + 1, P.nz - 1);
    const long long row = (long long)k * P.plane + (long long)j * P.pitch;
    const long long rowy = (long long)k * P.plane + (long long)jn * P.pitch;
    const long long rowz = (long long)kn * P.plane + (long long)j * P.pitch;
    const float *pr = sp + sy * kCW + lx + 4, *pu = sp + (sy + 1) * kCW + lx + 4;
    const float *pz = ring + ring_slot(k + 1) * kPl + sy * kCW + lx + 4;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int x = min(i0 + e, P.nx - 1), xn = min(i0 + e + 1, P.nx - 1);
      const float Kc = ldmap(Km, row + x);
      const float fx = mom_factor(Kc, ldmap(Km, row + xn), pr[e], pr[e + 1]);
      const float fy = mom_factor(Kc, ldmap(Km, rowy + x), pr[e], pu[e]);
      const float fz = mom_factor(Kc, ldmap(Km, rowz + x), pr[e], pz[e]);
      el2(v0, e) = vel_upd(el2(v0, e), P.two_dt / (rr[e] + rr[e + 1]), el2(S0, e), fx);
      el2(v1, e) = vel_upd(el2(v1, e), P.two_dt / (rr[e] + ru[e]), el2(S1, e), fy);
      el2(v2, e) = vel_upd(el2(v2, e), P.two_dt / (rr[e] + rz[e]), el2(S2, e), fz);
    }
  } else {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      el2(v0, e) = vel_upd(el2(v0, e), P.two_dt / (rr[e] + rr[e + 1]), el2(S0, e));
      el2(v1, e) = vel_upd(el2(v1, e), P.two_dt / (rr[e] + ru[e]), el2(S1, e));
      el2(v2, e) = vel_upd(el2(v2, e), P.two_dt / (rr[e] + rz[e]), el2(S2, e));
    }
  }
  if (EDGE) {
    v0 = mask_pad2(v0, i0, P.nx);
    v1 = mask_pad2(v1, i0, P.nx);
    v2 = mask_pad2(v2, i0, P.nx);
  }
  st_state2(P.v[0], c, v0);
  st_state2(P.v[1], c, v1);
  st_state2(P.v[2], c, v2);
}

template <int N, bool EDGE>
__device__ __forceinline__ void prs3_compute(const StepParams &P, const float *st, const float *ring, int x0, int y0,
                                             int k, int tid, int xs_side, int xsL) {
  using S = Prs3<N>;
  const int lx = 2 * (tid & 63), ly = tid >> 6;
  const int i0 = x0 + lx, j = y0 + ly;
  if (EDGE && (i0 >= P.nx || j >= P.ny)) return;
  const long long c = (long long)k * P.plane + (long long)j * P.pitch + i0;
  const long long Sn = P.npts_alloc;
  const int o = ly * kTX + lx;
  float2 Dx, Dy, Dz;
  {
    const Win10 w = win10(st + S::oVx + ly * kCW, lx);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m - 1] - w.v[4 + e - m], d);
      el2(Dx, e) = d;
    }
  }
  {
    float2 col[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) col[m] = sld2(st + S::oVy + (ly + m) * kTX + lx);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el2(col[4 + m - 1], e) - el2(col[4 - m], e), d);
      el2(Dy, e) = d;
    }
  }
  {
    float2 zc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) zc[m] = sld2(ring + ring_slot(k - 4 + m) * kArr + o);  // v_z planes k-4 ..
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el2(zc[4 + m - 1], e) - el2(zc[4 - m], e), d);
      el2(Dz, e) = d;
    }
  }
  const float2 k2 = sldh2(reinterpret_cast<const bf16 *>(st + S::oIk) + o);
  const float2 K = sldh2(reinterpret_cast<const bf16 *>(st + S::oKm) + o);
  float2 ch = make_float2(0.f, 0.f);
  if (P.nl) ch = sldh2(reinterpret_cast<const bf16 *>(st + S::oChi) + o);
  float2 A[3][N > 0 ? N : 1], B[3][N > 0 ? N : 1];
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    const float2 a = sldh2(reinterpret_cast<const bf16 *>(st + S::oA) + nu * kArr + o);
    const float2 b = sldb2(reinterpret_cast<const bf16 *>(st + S::oB) + nu * kArr + o);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      A[q][nu] = a;
      B[q][nu] = b;
    }
  }
  if (EDGE) {
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      if (xs_side >= 0)
        strip3x_staged(P, reinterpret_cast<const bf16 *>(st + S::oXs),
                       reinterpret_cast<const bf16 *>(st + S::oXs + XStrip<N>::kHalf), xsL, nu, i0, ly, A[0][nu],
                       B[0][nu]);
      else
        strip3<0, 2>(P, nu, i0, j, k, A[0][nu], B[0][nu]);
      strip3<1, 2>(P, nu, i0, j, k, A[1][nu], B[1][nu]);
      strip3<2, 2>(P, nu, i0, j, k, A[2][nu], B[2][nu]);
    }
  }
  float2 p = sld2(st + S::oP + o);
  float2 S0, S1, S2;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    el2(S0, e) = el2(Dx, e) * el2(k2, e);
    el2(S1, e) = el2(Dy, e) * el2(k2, e);
    el2(S2, e) = el2(Dz, e) * el2(k2, e);
  }
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    const float2 q0 = sld2(st + S::oPsi + nu * kArr + o);
    const float2 q1 = sld2(st + S::oPsi + (N + nu) * kArr + o);
    const float2 q2 = sld2(st + S::oPsi + (2 * N + nu) * kArr + o);
    float2 n0, n1, n2;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      el2(n0, e) = fmaf(el2(B[0][nu], e), el2(q0, e), el2(A[0][nu], e) * el2(Dx, e));
      el2(n1, e) = fmaf(el2(B[1][nu], e), el2(q1, e), el2(A[1][nu], e) * el2(Dy, e));
      el2(n2, e) = fmaf(el2(B[2][nu], e), el2(q2, e), el2(A[2][nu], e) * el2(Dz, e));
      el2(S0, e) += fmaf(P.w_new, el2(n0, e), P.w_old * el2(q0, e));
      el2(S1, e) += fmaf(P.w_new, el2(n1, e), P.w_old * el2(q1, e));
      el2(S2, e) += fmaf(P.w_new, el2(n2, e), P.w_old * el2(q2, e));
    }
    if (EDGE) {
      n0 = mask_pad2(n0, i0, P.nx);
      n1 = mask_pad2(n1, i0, P.nx);
      n2 = mask_pad2(n2, i0, P.nx);
    }
    st_state2(P.psi2[0], nu * Sn + c, n0);
    st_state2(P.psi2[1], nu * Sn + c, n1);
    st_state2(P.psi2[2], nu * Sn + c, n2);
  }
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    float upd = P.dt * el2(K, e) * (el2(S0, e) + el2(S1, e) + el2(S2, e));
    if (P.nl) upd /= fmaf(el2(ch, e), el2(p, e), 1.f);
    el2(p, e) -= upd;
  }
  if (EDGE) p = mask_pad2(p, i0, P.nx);
  st_state2(P.p, c, p);
}

// One half step.  Block (32, 16), one per SM; items blockIdx.x,
// blockIdx.x + gridDim.x, ...; within an item the units k0 .. k1-1 in order.
template <int N, bool VEL>
__global__ void __launch_bounds__(kThreads, 1)
    pipe3d_kernel(const StepParams P, const Region3 R, const __grid_constant__ PipeMaps T) {
  using G = Ring3<N, VEL>;
  constexpr int kStage = G::kStage;
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int ok[2];  // per stage: thread 0 never rewrites a flag a thread has yet to read
  float *smem = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float *ring = smem + 2 * kStage;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbarrier_init();
  }
  __syncthreads();
  const long long n_items = R.items();
  long long it = blockIdx.x;
  if (it >= n_items) return;
  int x0, y0, k0, k1;
  R.item(it, x0, y0, k0, k1);
  int k = k0;
  unsigned phase = 0, pending = 0;
  if (tid == 0)
    issue3<N, VEL>(T, smem, ring, &bar[0], x0, y0, k, ring_first<VEL>(k), ring_first<VEL>(k) + 7, P.nl != 0,
                   R.xs_side(x0), R.xsL);
  pending |= 1u;
  int s = 0;
#pragma unroll 1
  while (true) {
    if (tid == 0) ok[s] = mbar_wait_bounded(&bar[s], (phase >> s) & 1u);
    __syncthreads();
    if (!ok[s]) {
      if (tid == 0) {
        report_status(P.status, kStatusWaitTimeout);
        if ((pending >> (s ^ 1)) & 1u) mbar_wait_bounded(&bar[s ^ 1], (phase >> (s ^ 1)) & 1u);
      }
      return;
    }
    phase ^= 1u << s;
    pending &= ~(1u << s);
    // the next unit: the next plane of this item, or the first of the next
    long long nit = it;
    int nx0 = x0, ny0 = y0, nk0 = k0, nk1 = k1, nk = k + 1;
    if (nk >= k1) {
      nit = it + gridDim.x;
      if (nit < n_items) R.item(nit, nx0, ny0, nk0, nk1);
      nk = nk0;
    }
    const bool more = nit < n_items, fresh = nit != it;
    const int q = s ^ 1;
    if (more && !fresh) {  // one new ring plane, into the slot no unit of this item reads any more
      if (tid < 32) {
        const int kp = ring_first<VEL>(nk) + 7;
        if (tid == 0)
          issue3<N, VEL>(T, smem + q * kStage, ring, &bar[q], nx0, ny0, nk, kp, kp, P.nl != 0, R.xs_side(nx0),
                         R.xsL);
        if (!R.interior(nx0, ny0, nk)) prefetch_strips<N, VEL ? 1 : 2>(P, nx0, ny0, nk, tid, R.xsL > 0);
      }
      pending |= 1u << q;
    }
    float *cur = smem + s * kStage;
    if (R.interior(x0, y0, k)) {
      if (VEL) vel3_compute<N, false>(P, cur, ring, x0, y0, k, tid, -1, 0);
      else prs3_compute<N, false>(P, cur, ring, x0, y0, k, tid, -1, 0);
    } else {
      const int xside = R.xs_side(x0);
      if (VEL) vel3_compute<N, true>(P, cur, ring, x0, y0, k, tid, xside, R.xsL);
      else prs3_compute<N, true>(P, cur, ring, x0, y0, k, tid, xside, R.xsL);
    }
    if (!more) break;
    if (fresh) {  // a new column: all eight ring planes, once every thread is done with the ring
      __syncthreads();
      if (tid == 0)
        issue3<N, VEL>(T, smem + q * kStage, ring, &bar[q], nx0, ny0, nk, ring_first<VEL>(nk),
                       ring_first<VEL>(nk) + 7, P.nl != 0, R.xs_side(nx0), R.xsL);
      pending |= 1u << q;
    }
    it = nit;
    x0 = nx0; y0 = ny0; k0 = nk0; k1 = nk1; k = nk;
    s = q;
  }
}

template <int N, bool VEL>
cudaError_t pipe3_launch(const StepParams &P, const Region3 &R, int grid, const PipeMaps &T, cudaStream_t st) {
  constexpr size_t bytes = Ring3<N, VEL>::kBytes;
  static_assert(bytes <= 227 * 1024, "stages exceed shared memory");
  cudaError_t e =
      cudaFuncSetAttribute(pipe3d_kernel<N, VEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  pipe3d_kernel<N, VEL><<<grid, dim3(32, kThreads / 32), bytes, st>>>(P, R, T);
  return cudaGetLastError();
}

template <bool VEL>
cudaError_t pipe3_dispatch(const StepParams &P, const Region3 &R, int grid, const PipeMaps &T, cudaStream_t st) {
  switch (P.n_relax) {
    case 0: return pipe3_launch<0, VEL>(P, R, grid, T, st);
    case 1: return pipe3_launch<1, VEL>(P, R, grid, T, st);
    case 2: return pipe3_launch<2, VEL>(P, R, grid, T, st);
    case 3: return pipe3_launch<3, VEL>(P, R, grid, T, st);
    default: return cudaErrorInvalidValue;
  }
}

// The x strip's coefficients come by TMA when a box of L values per row
// starts on a 16-byte boundary and fits the stage (L a multiple of 8, at
// most kXsMax), and no unit reaches both sides (nx >= 128 + L).
bool x_strip_staged(const StepParams &P) {
  const int L = P.L[0];
  return P.n_relax > 0 && L > 0 && L % 8 == 0 && L <= kXsMax && P.nx >= kTX + L && P.sa1[0] != nullptr;
}

// Planes per item: the split of each column into items that minimises the
// busiest block's work, counting each item's start (eight ring planes and
// one exposed copy latency) as about 1.5 units.
Region3 region3_of(const StepParams &P, int grid) {
  Region3 R;
  R.nx = P.nx;
  R.ny = P.ny;
  R.nz = P.nz;
  R.Lx = P.L[0] > 4 ? P.L[0] : 4;
  R.Ly = P.L[1] > 4 ? P.L[1] : 4;
  R.Lz = P.L[2] > 4 ? P.L[2] : 4;
  R.tnx = (P.nx + kTX - 1) / kTX;
  R.nhy = (P.ny + kHT - 1) / kHT;
  R.xsL = x_strip_staged(P) ? P.L[0] : 0;
  const long long ncols = (long long)R.tnx * R.nhy;
  double best = 1e300;
  R.seglen = P.nz;
  R.nseg = 1;
  for (int nseg = 1; nseg <= P.nz && nseg <= 64; ++nseg) {
    const int seglen = (P.nz + nseg - 1) / nseg;
    const int used = (P.nz + seglen - 1) / seglen;
    const long long items = ncols * used;
    const long long rounds = (items + grid - 1) / grid;
    const double cost = (double)rounds * (seglen + 1.5);
    if (cost < best - 1e-9) {
      best = cost;
      R.seglen = seglen;
      R.nseg = used;
    }
  }
  return R;
}

}  // namespace

bool pipe3d_supported(const StepParams &P, int map_kind) {
  // bf16 maps (two stages of ~107 KB fit); N <= 3 keeps the 4D boxes and
  // the stage within shared memory; no periodic axis; the cross taps are
  // left to the tile kernels
  return P.nz > 1 && map_kind == 1 && P.n_relax >= 0 && P.n_relax <= 3 && !P.periodic[0] && !P.periodic[1] &&
         !P.periodic[2] && P.g11h == 0.f;
}

cudaError_t build_pipe3d_maps(const StepParams &P, PipeMaps *vel, PipeMaps *prs, const char **why) {
  *vel = PipeMaps{};
  *prs = PipeMaps{};
  const int N = P.n_relax;
  using ull = unsigned long long;
  const ull nx = P.nx, ny = P.ny, nz = P.nz, S = P.npts_alloc;
  const ull f3[2] = {(ull)P.pitch * 4, (ull)P.plane * 4}, h3[2] = {(ull)P.pitch * 2, (ull)P.plane * 2};
  const ull f4[3] = {(ull)P.pitch * 4, (ull)P.plane * 4, S * 4}, h4[3] = {(ull)P.pitch * 2, (ull)P.plane * 2, S * 2};
  const ull d3[3] = {nx, ny, nz};
  const ull dv[4] = {nx, ny, nz, 3}, dpsi[4] = {nx, ny, nz, (ull)(3 * N)}, dab[4] = {nx, ny, nz, (ull)N};
  const unsigned halo[3] = {kCW, kHT + 7, 1}, rho[3] = {kRWb, kHT + 1, 2},
                 one[3] = {kTX, kHT, 1}, v4[4] = {kTX, kHT, 1, 3}, psi4[4] = {kTX, kHT, 1, (unsigned)(3 * N)},
                 ab4[4] = {kTX, kHT, 1, (unsigned)N}, vx[3] = {kCW, kHT, 1}, vy[3] = {kTX, kHT + 7, 1};
  bool ok = true;
  // velocity half step
  ok = ok && encode_tensor_map(&vel->m[0], P.p, 4, 3, d3, f3, halo);
  ok = ok && encode_tensor_map(&vel->m[2], P.rho, 2, 3, d3, h3, rho);
  ok = ok && encode_tensor_map(&vel->m[3], P.v[0], 4, 4, dv, f4, v4);
  if (N > 0) ok = ok && encode_tensor_map(&vel->m[4], P.psi1[0], 4, 4, dpsi, f4, psi4);
  ok = ok && encode_tensor_map(&vel->m[5], P.ik1, 2, 3, d3, h3, one);
  if (N > 0) {
    ok = ok && encode_tensor_map(&vel->m[6], P.a1, 2, 4, dab, h4, ab4);
    ok = ok && encode_tensor_map(&vel->m[7], P.b1, 2, 4, dab, h4, ab4);
  }
  // pressure half step
  ok = ok && encode_tensor_map(&prs->m[0], P.v[0], 4, 3, d3, f3, vx);
  ok = ok && encode_tensor_map(&prs->m[1], P.v[1], 4, 3, d3, f3, vy);
  ok = ok && encode_tensor_map(&prs->m[2], P.v[2], 4, 3, d3, f3, one);
  ok = ok && encode_tensor_map(&prs->m[3], P.p, 4, 3, d3, f3, one);
  if (N > 0) ok = ok && encode_tensor_map(&prs->m[4], P.psi2[0], 4, 4, dpsi, f4, psi4);
  ok = ok && encode_tensor_map(&prs->m[5], P.ik2, 2, 3, d3, h3, one);
  ok = ok && encode_tensor_map(&prs->m[6], P.K, 2, 3, d3, h3, one);
  if (P.nl) ok = ok && encode_tensor_map(&prs->m[7], P.chi, 2, 3, d3, h3, one);
  if (N > 0) {
    ok = ok && encode_tensor_map(&prs->m[8], P.a2, 2, 4, dab, h4, ab4);
    ok = ok && encode_tensor_map(&prs->m[9], P.b2, 2, 4, dab, h4, ab4);
  }
  if (x_strip_staged(P)) {  // x strips [N][z][y][2L] bf16, boxes L x 8 x 1 x N
    const ull L = (ull)P.L[0];
    const ull dxs[4] = {2 * L, ny, nz, (ull)N}, sxs[3] = {2 * L * 2, ny * 2 * L * 2, (ull)P.strip_nu[0] * 2};
    const unsigned bxs[4] = {(unsigned)L, kHT, 1, (unsigned)N};
    ok = ok && encode_tensor_map(&vel->m[10], P.sa1[0], 2, 4, dxs, sxs, bxs);
    ok = ok && encode_tensor_map(&vel->m[11], P.sb1[0], 2, 4, dxs, sxs, bxs);
    ok = ok && encode_tensor_map(&prs->m[10], P.sa2[0], 2, 4, dxs, sxs, bxs);
    ok = ok && encode_tensor_map(&prs->m[11], P.sb2[0], 2, 4, dxs, sxs, bxs);
  }
  if (!ok) {
    *why = "cuTensorMapEncodeTiled rejected a 3D map (or the driver entry point is missing)";
    return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t launch_pipe3d(bool vel, const StepParams &P, int grid, const PipeMaps &T, cudaStream_t st) {
  const Region3 R = region3_of(P, grid);
  return vel ? pipe3_dispatch<true>(P, R, grid, T, st) : pipe3_dispatch<false>(P, R, grid, T, st);
}

}  // namespace fw2
