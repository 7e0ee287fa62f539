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
// halo, which also give the x and y taps and the g_{1,1} cross taps of
// planes k-1 .. k+1; pressure: v_z planes k-4 .. k+3), so each unit adds one
// plane.  With cross taps the pressure half step also keeps v_x and v_y
// planes k-1 .. k+1 (with a one-cell halo) in rings of four slots, and its
// v_z slots carry the same halo.  For a coming unit one thread issues tiled
// TMA tensor copies, one box per array, into a free stage of a two-stage
// ring: the operand planes the unit adds, the density of the plane and of
// the next one, the velocity (or pressure) of the unit, the bf16 maps (a and
// b of the N mechanisms in one 4D box each), K of planes k and k + 1 for the
// literal system's momentum factor, and in edge units the C-PML strip
// coefficients of each axis the unit reaches.  The memory variables, read
// once and written once by the thread that owns the cell, bypass shared
// memory: every thread loads the next unit's into registers while it
// computes the current one.  Copies complete on the stage's mbarrier while
// all threads compute the current unit from the other stage.
//
// Boundaries as in the 2D pipeline: the copies read zero outside the grid;
// units at the grid's edge or in a C-PML strip clamp the density to the last
// cell, take each axis' C-PML coefficients from its strip (staged, or read
// per cell where a box cannot serve: a strip wider than 64 cells or not a
// multiple of 8 along x, a grid too small for a unit to reach one side only
// along y) and store nothing outside the grid.  Periodic axes are not taken
// by this path (the tile kernels run them).
#include <climits>
#include <cstring>

#include "async.cuh"
#include "coef.cuh"
#include "tmap.h"

namespace fw2 {

namespace {

constexpr int kHT = 8;            // rows of a unit
constexpr int kCW = kTX + 8;      // halo columns x0-4 .. x0+TX+3
constexpr int kRWb = kTX + 8;     // staged bf16 density / K columns x0 .. x0+TX+7 (16-byte rows)
constexpr int kArr = kHT * kTX;   // elements of one array per unit

using bf16 = __nv_bfloat16;

constexpr int round32(int n) { return (n + 31) & ~31; }  // floats: 128-byte regions
constexpr int fl(int bytes) { return (bytes + 3) / 4; }

constexpr int kSlots = 9;  // operand ring: the eight planes of a unit and the one the next unit adds
constexpr int kSub = 4;    // cross-tap rings of v_x, v_y: planes k-1 .. k+1 and the one the next unit adds
constexpr int kXsMax = 64; // widest x C-PML strip (cells per side) staged by TMA

__host__ __device__ constexpr int ring_slot(int k) { return ((k % kSlots) + kSlots) % kSlots; }
static_assert((kSub & (kSub - 1)) == 0, "the sub-rings index by a mask");
__host__ __device__ constexpr int sub_slot(int k) { return k & (kSub - 1); }
// slot of plane k0 + m (0 <= m < kSlots) from the slot s0 of plane k0: one
// modulo per unit instead of one per plane
__device__ __forceinline__ int slot_after(int s0, int m) {
  const int s = s0 + m;
  return s >= kSlots ? s - kSlots : s;
}

// C-PML strip coefficients of a stage (bf16): x strip a then b, each
// [N][8][L] (L <= kXsMax); y strip a, b and z strip a, b, each [N][8][128]
// (not in the layout that stages the memory variables, PS)
template <int N, bool PS>
struct Strips {
  static constexpr int kX = N * kHT * kXsMax / 2;    // floats of the x strip's a (or b)
  static constexpr int kYZ = PS ? 0 : N * kArr / 2;  // floats of a y or z strip's a (or b)
  static constexpr int oXa = 0, oXb = kX, oYa = 2 * kX, oYb = oYa + kYZ, oZa = oYb + kYZ, oZb = oZa + kYZ;
  static constexpr int kFloats = oZb + kYZ;
};

// velocity stage: density bf16 [2][9][136] (planes k, k+1), v [3][8][128],
// 1/kappa1 bf16 [8][128], a1, b1 bf16 [N][8][128], then either (PS) the 3N
// memory variables [3N][8][128] and the x strip, or K bf16 [2][9][136]
// (literal system) and the strips of all axes; plane ring: p planes
// [15][136] (rows y0-3 .. y0+11, columns x0-4 ..)
template <int N, bool PS>
struct Vel3 {
  static constexpr int kRho = round32(fl(2 * (kHT + 1) * kRWb * 2));
  static constexpr int kV = 3 * kArr;
  static constexpr int kK = round32(fl(kArr * 2));
  static constexpr int kAB = round32(fl(N * kArr * 2));
  static constexpr int kPsi = PS ? 3 * N * kArr : 0;
  static constexpr int kKmF = PS ? 0 : kRho;
  static constexpr int oRho = 0, oV = oRho + kRho, oK = oV + kV, oA = oK + kK, oB = oA + kAB, oPsi = oB + kAB,
                       oKm = oPsi + kPsi, oS = oKm + kKmF;
  static constexpr int kFloats = round32(oS + Strips<N, PS>::kFloats);
  static constexpr unsigned kBytes = 4u * (kV + kPsi) + 2u * (2 * (kHT + 1) * kRWb + kArr + 2 * N * kArr);
  static constexpr unsigned kKmBytes = 2u * 2 * (kHT + 1) * kRWb;
  static constexpr int kPlane = round32((kHT + 7) * kCW);
  static constexpr unsigned kPlaneBytes = 4u * (kHT + 7) * kCW;
};

// pressure stage: p [8][128], 1/kappa2, K, chi bf16 [8][128], a2, b2 bf16
// [N][8][128], then either (PS) the 3N memory variables and the x strip or
// the strips of all axes; without cross taps also v_x [8][136] (x halo) and
// v_y [15][128] (rows y0-4 ..), with the plane ring of v_z [8][128]; with
// cross taps (never PS) the rings hold v_z [10][136] (rows y0-1 .., columns
// x0-4 ..), v_x [10][136] (rows y0-1 ..) and v_y [15][136] (rows y0-4 ..)
template <int N, bool CROSS, bool PS>
struct Prs3 {
  static constexpr int kVx = CROSS ? 0 : round32(kHT * kCW);
  static constexpr int kVy = CROSS ? 0 : round32((kHT + 7) * kTX);
  static constexpr int kP = kArr;
  static constexpr int kK = round32(fl(kArr * 2));
  static constexpr int kAB = round32(fl(N * kArr * 2));
  static constexpr int kPsi = PS ? 3 * N * kArr : 0;
  static constexpr int oVx = 0, oVy = oVx + kVx, oP = oVy + kVy, oIk = oP + kP, oKm = oIk + kK, oChi = oKm + kK,
                       oA = oChi + kK, oB = oA + kAB, oPsi = oB + kAB, oS = oPsi + kPsi;
  static constexpr int kFloats = round32(oS + Strips<N, PS>::kFloats);
  static constexpr unsigned kBytesNoChi =
      4u * ((CROSS ? kP : kHT * kCW + (kHT + 7) * kTX + kP) + kPsi) + 2u * (2 * kArr + 2 * N * kArr);
  // v_z ring slot; with cross taps also the v_x and v_y ring slots
  static constexpr int kPlane = CROSS ? round32((kHT + 2) * kCW) : kArr;
  static constexpr unsigned kPlaneBytes = 4u * (CROSS ? (kHT + 2) * kCW : kArr);
  static constexpr int kXPlane = round32((kHT + 2) * kCW);
  static constexpr unsigned kXPlaneBytes = 4u * (kHT + 2) * kCW;
  static constexpr int kYPlane = round32((kHT + 7) * kCW);
  static constexpr unsigned kYPlaneBytes = 4u * (kHT + 7) * kCW;
};

template <int N, bool VEL, bool CROSS, bool PS>
struct Ring3 {
  static constexpr int kStage = VEL ? Vel3<N, PS>::kFloats : Prs3<N, CROSS, PS>::kFloats;
  static constexpr int kPlane = VEL ? Vel3<N, PS>::kPlane : Prs3<N, CROSS, PS>::kPlane;
  static constexpr unsigned kPlaneBytes = VEL ? Vel3<N, PS>::kPlaneBytes : Prs3<N, CROSS, PS>::kPlaneBytes;
  static constexpr int kSubFloats =
      (!VEL && CROSS) ? kSub * (Prs3<N, CROSS, PS>::kXPlane + Prs3<N, CROSS, PS>::kYPlane) : 0;
  static constexpr size_t kBytes =
      sizeof(float) * (2 * (size_t)kStage + (size_t)kSlots * kPlane + (size_t)kSubFloats) + 128;
};

// Work items: a column of units (xy position, x fastest) and a range of
// planes; item it covers column it % ncols, planes seg * seglen ..
struct Region3 {
  int nx, ny, nz, Lx, Ly, Lz;
  int tnx, nhy;      // x tiles, half-tile rows per plane
  int seglen, nseg;  // planes per item, items per column
  int xsL;           // x C-PML strip cells per side when its coefficients come by TMA, else 0
  int ysL, zsL;      // the same for the y and z strips
  // the side of the x strip a unit at x0 reaches: 0 low, 1 high, -1 none
  // (with xsL set no unit reaches both)
  __device__ __forceinline__ int xs_side(int x0) const {
    if (xsL == 0) return -1;
    return x0 < xsL ? 0 : (x0 + kTX > nx - xsL ? 1 : -1);
  }
  // first strip row of the y box of a unit at y0 (INT_MIN: none)
  __device__ __forceinline__ int ys_row(int y0) const {
    if (ysL == 0) return INT_MIN;
    if (y0 < ysL) return y0;
    if (y0 + kHT > ny - ysL) return y0 - (ny - 2 * ysL);
    return INT_MIN;
  }
  __device__ __forceinline__ int zs_plane(int k) const {
    if (zsL == 0) return -1;
    return strip_coord(k, nz, zsL);
  }
  __host__ __device__ __forceinline__ long long items() const { return (long long)tnx * nhy * nseg; }
  __host__ __device__ __forceinline__ void item(long long it, int &x0, int &y0, int &k0, int &k1) const {
    const int ncols = tnx * nhy;
    const int col = (int)(it % ncols), seg = (int)(it / ncols);
    x0 = (col % tnx) * kTX;
    y0 = (col / tnx) * kHT;
    k0 = seg * seglen;
    k1 = k0 + seglen < nz ? k0 + seglen : nz;
  }
  __host__ __device__ __forceinline__ bool interior(int x0, int y0, int k) const {
    return x0 >= Lx && x0 + kTX + Lx <= nx && y0 >= Ly && y0 + kHT + Ly <= ny && k >= Lz && k + Lz < nz;
  }
};

// first plane of the operand ring a unit at plane k reads (8 planes)
template <bool VEL>
__host__ __device__ constexpr int ring_first(int k) { return VEL ? k - 3 : k - 4; }

// Issue the copies of a unit at (x0, y0, k): its stage, the operand planes
// k_lo .. k_hi of the plane ring (one plane, or eight for the first unit of
// an item) and, with cross taps in the pressure half step, the v_x and v_y
// planes s_lo .. s_hi of their rings, all completing on the stage's mbarrier.
template <int N, bool VEL, bool CROSS, bool PS>
__device__ __forceinline__ void issue3(const PipeMaps &T, const Region3 &R, float *st, float *ring, float *sub,
                                       uint64_t *bar, int x0, int y0, int k, int k_lo, int k_hi, int s_lo, int s_hi,
                                       bool nl, bool nl_vel) {
  using G = Ring3<N, VEL, CROSS, PS>;
  using SS = Strips<N, PS>;
  fence_proxy_async_smem();
  const unsigned planes = G::kPlaneBytes * (unsigned)(k_hi - k_lo + 1);
  // C-PML strip boxes of the axes the unit reaches (all mechanisms)
  const int xside = N > 0 ? R.xs_side(x0) : -1;
  const int yrow = N > 0 ? R.ys_row(y0) : INT_MIN;
  const int zpl = N > 0 ? R.zs_plane(k) : -1;
  const unsigned xs = xside >= 0 ? 2u * 2u * (unsigned)(N * kHT * R.xsL) : 0u;
  const unsigned yz = (yrow != INT_MIN ? 2u * 2u * N * kArr : 0u) + (zpl >= 0 ? 2u * 2u * N * kArr : 0u);
  float *ss = st + (VEL ? Vel3<N, PS>::oS : Prs3<N, CROSS, PS>::oS);
  auto load_strips = [&] {
    if (xside >= 0) {
      tma_load_4d(ss + SS::oXa, &T.m[10], xside * R.xsL, y0, k, 0, bar);
      tma_load_4d(ss + SS::oXb, &T.m[11], xside * R.xsL, y0, k, 0, bar);
    }
    if (yrow != INT_MIN) {
      tma_load_4d(ss + SS::oYa, &T.m[13], x0, yrow, k, 0, bar);
      tma_load_4d(ss + SS::oYb, &T.m[14], x0, yrow, k, 0, bar);
    }
    if (zpl >= 0) {
      tma_load_4d(ss + SS::oZa, &T.m[15], x0, y0, zpl, 0, bar);
      tma_load_4d(ss + SS::oZb, &T.m[16], x0, y0, zpl, 0, bar);
    }
  };
  if (VEL) {
    using S = Vel3<N, PS>;
    mbar_arrive_expect_tx(bar, S::kBytes + (nl_vel ? S::kKmBytes : 0u) + planes + xs + yz);
    load_strips();
    for (int kp = k_lo; kp <= k_hi; ++kp) tma_load_3d(ring + ring_slot(kp) * G::kPlane, &T.m[0], x0 - 4, y0 - 3, kp, bar);
    tma_load_3d(st + S::oRho, &T.m[2], x0, y0, k, bar);
    tma_load_4d(st + S::oV, &T.m[3], x0, y0, k, 0, bar);
    tma_load_3d(st + S::oK, &T.m[5], x0, y0, k, bar);
    if (N > 0) {
      tma_load_4d(st + S::oA, &T.m[6], x0, y0, k, 0, bar);
      tma_load_4d(st + S::oB, &T.m[7], x0, y0, k, 0, bar);
      if (PS) tma_load_4d(st + S::oPsi, &T.m[4], x0, y0, k, 0, bar);
    }
    if (!PS && nl_vel) tma_load_3d(st + S::oKm, &T.m[12], x0, y0, k, bar);
  } else {
    using S = Prs3<N, CROSS, PS>;
    const unsigned subs = CROSS ? (S::kXPlaneBytes + S::kYPlaneBytes) * (unsigned)(s_hi - s_lo + 1) : 0u;
    mbar_arrive_expect_tx(bar, S::kBytesNoChi + (nl ? 2u * kArr : 0u) + planes + subs + xs + yz);
    load_strips();
    if (CROSS) {
      for (int kp = k_lo; kp <= k_hi; ++kp) tma_load_3d(ring + ring_slot(kp) * G::kPlane, &T.m[2], x0 - 4, y0 - 1, kp, bar);
      float *sx = sub, *sy = sub + kSub * S::kXPlane;
      for (int kp = s_lo; kp <= s_hi; ++kp) {
        tma_load_3d(sx + sub_slot(kp) * S::kXPlane, &T.m[0], x0 - 4, y0 - 1, kp, bar);
        tma_load_3d(sy + sub_slot(kp) * S::kYPlane, &T.m[1], x0 - 4, y0 - 4, kp, bar);
      }
    } else {
      for (int kp = k_lo; kp <= k_hi; ++kp) tma_load_3d(ring + ring_slot(kp) * G::kPlane, &T.m[2], x0, y0, kp, bar);
      tma_load_3d(st + S::oVx, &T.m[0], x0 - 4, y0, k, bar);
      tma_load_3d(st + S::oVy, &T.m[1], x0, y0 - 4, k, bar);
    }
    tma_load_3d(st + S::oP, &T.m[3], x0, y0, k, bar);
    tma_load_3d(st + S::oIk, &T.m[5], x0, y0, k, bar);
    tma_load_3d(st + S::oKm, &T.m[6], x0, y0, k, bar);
    if (nl) tma_load_3d(st + S::oChi, &T.m[7], x0, y0, k, bar);
    if (N > 0) {
      tma_load_4d(st + S::oA, &T.m[8], x0, y0, k, 0, bar);
      tma_load_4d(st + S::oB, &T.m[9], x0, y0, k, 0, bar);
      if (PS) tma_load_4d(st + S::oPsi, &T.m[4], x0, y0, k, 0, bar);
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
// columns c+2 .. c+7 of a halo row (v[2 + e] is the cell e of a pair at c+4)
struct Win6 {
  float v[6];
};
__device__ __forceinline__ Win6 win6(const float *row, int c) {
  Win6 w;
  const float2 *r2 = reinterpret_cast<const float2 *>(row + c + 2);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float2 t = r2[i];
    w.v[2 * i] = t.x;
    w.v[2 * i + 1] = t.y;
  }
  return w;
}

// Memory variables of a thread's two cells: q[axis][nu], loaded one unit
// ahead (zero for a pair outside the grid, like the padding it would read).
template <int N>
using Psi = float2[3][N > 0 ? N : 1];
template <int N>
__device__ __forceinline__ void load_psi(float *const *psi, long long Sn, long long c, bool ok, Psi<N> &q) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int nu = 0; nu < N; ++nu)
      q[a][nu] = ok ? __ldcs(reinterpret_cast<const float2 *>(psi[a] + nu * Sn + c)) : make_float2(0.f, 0.f);
}

// a, b along axis Q (OP: 1 faces, 2 centres) of mechanism nu at the two
// cells of an edge pair, from that axis' C-PML strip in global memory where
// the cells lie in it (coef4 of the tile kernels; its zero beyond the grid
// only reaches masked cells); unchanged elsewhere
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
// (each [N][8][L] bf16, the side the unit reaches): the values strip3<0>
// reads from global memory, for the cells in the strip
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

// All C-PML coefficient overrides of an edge pair for mechanism nu (axes x,
// y, z), from the staged boxes where the unit has them, else global memory.
template <int N, int OP, bool PS>
__device__ __forceinline__ void strips_of(const StepParams &P, const Region3 &R, const float *ss, int xside, bool ys,
                                          bool zs, int nu, int i0, int j, int k, int ly, int lx, float2 (&A)[3],
                                          float2 (&B)[3]) {
  using SS = Strips<N, PS>;
  if (xside >= 0)
    strip3x_staged(P, reinterpret_cast<const bf16 *>(ss + SS::oXa), reinterpret_cast<const bf16 *>(ss + SS::oXb),
                   R.xsL, nu, i0, ly, A[0], B[0]);
  else
    strip3<0, OP>(P, nu, i0, j, k, A[0], B[0]);
  if (ys) {
    if (strip_coord(j, P.ny, P.L[1]) >= 0) {
      const int o = nu * kArr + ly * kTX + lx;
      A[1] = sldh2(reinterpret_cast<const bf16 *>(ss + SS::oYa) + o);
      B[1] = sldb2(reinterpret_cast<const bf16 *>(ss + SS::oYb) + o);
    }
  } else {
    strip3<1, OP>(P, nu, i0, j, k, A[1], B[1]);
  }
  if (zs) {
    const int o = nu * kArr + ly * kTX + lx;
    A[2] = sldh2(reinterpret_cast<const bf16 *>(ss + SS::oZa) + o);
    B[2] = sldb2(reinterpret_cast<const bf16 *>(ss + SS::oZb) + o);
  } else {
    strip3<2, OP>(P, nu, i0, j, k, A[2], B[2]);
  }
}

// Prefetch into L2 the C-PML strip rows an edge unit will read per cell from
// global memory (warp 0, one unit ahead): only strips without a staged box.
// OP: 1 velocity (a1, b1), 2 pressure (a2, b2).
__device__ __forceinline__ void l2_line(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }
template <int N, int OP>
__device__ __forceinline__ void prefetch_strips(const StepParams &P, const Region3 &R, int x0, int y0, int k,
                                                int lane) {
  if constexpr (N > 0) {
    const bf16 *sa[3], *sb[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      sa[q] = static_cast<const bf16 *>(OP == 1 ? P.sa1[q] : P.sa2[q]);
      sb[q] = static_cast<const bf16 *>(OP == 1 ? P.sb1[q] : P.sb2[q]);
    }
    // x strip: rows (k, y) of 2L values, for units reaching into it
    const int Lx = P.L[0];
    if (R.xsL == 0 && Lx > 0 && (x0 < Lx || x0 + kTX > P.nx - Lx)) {
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
    if (R.ysL == 0 && Ly > 0) {
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
    const int scz = (R.zsL == 0 && Lz > 0) ? strip_coord(k, P.nz, Lz) : -1;
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

// mom_factor (coef.cuh) from the reciprocals 1 / K of the two cells, taken
// once per cell: the same value for the same operands
__device__ __forceinline__ float mom_factor_ik(float ika, float ikb, float pa, float pb) {
  return fmaf(0.5f * (ika + ikb), 0.5f * (pa + pb), 1.f);
}

// Values at the faces of a pair read from a staged bf16 box [2][9][136]
// (planes k, k + 1: the density, or K): plane k row ly at lx .. lx+2, row
// ly+1 at lx, lx+1; plane k+1 row ly at lx, lx+1.  Cells beyond the last one
// along an axis take that cell's value (rho_coord of the tile kernels).
struct Face3 {
  float r0, r1, r2, u0, u1, z0, z1;
};
template <bool EDGE>
__device__ __forceinline__ Face3 face3(const StepParams &P, const bf16 *rb, int x0, int y0, int k, int lx, int ly) {
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
  return Face3{at(0, r0, c0), at(0, r0, c1), at(0, r0, c2), at(0, r1, c0), at(0, r1, c1),
               at(pz, r0, c0), at(pz, r0, c1)};
}

// The memory-variable update of mechanism nu on the three axes and its
// contribution to the stretched derivatives (Eqs. relaxation4,
// relaxation_psi), writing psi back; A[a], B[a] are the coefficients of
// axis a, q[a] its memory variable before the update.
__device__ __forceinline__ void relax3(const StepParams &P, float *const *psi, long long o, int i0, bool edge,
                                       const float2 (&q)[3], const float2 (&A)[3], const float2 (&B)[3],
                                       const float2 (&D)[3], float2 (&S)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 n;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      el2(n, e) = fmaf(el2(B[a], e), el2(q[a], e), el2(A[a], e) * el2(D[a], e));
      el2(S[a], e) += fmaf(P.w_new, el2(n, e), P.w_old * el2(q[a], e));
    }
    if (edge) n = mask_pad2(n, i0, P.nx);
    st_state2(psi[a], o, n);
  }
}

template <int N, bool EDGE, bool CROSS, bool PS>
__device__ __forceinline__ void vel3_compute(const StepParams &P, const Region3 &R, float *st, const float *ring,
                                             int x0, int y0, int k, int tid, const Psi<N> &q) {
  using S = Vel3<N, PS>;
  const int lx = 2 * (tid & 63), ly = tid >> 6;
  const int i0 = x0 + lx, j = y0 + ly;
  if (EDGE && (i0 >= P.nx || j >= P.ny)) return;
  const long long c = (long long)k * P.plane + (long long)j * P.pitch + i0;
  const long long Sn = P.npts_alloc;
  const int o = ly * kTX + lx;
  // derivatives: x, y from the halo plane of k (cell e at column lx + 4 + e),
  // z from the same cell of planes k-3 .. k+4 in the ring
  constexpr int kPl = S::kPlane;
  const int s0 = ring_slot(k - 3);  // planes k-3 .. k+4 of the ring: slots s0 + 0 .. 7
  const float *sp = ring + slot_after(s0, 3) * kPl;
  const int sy = ly + 3;
  float2 D[3];
  {
    const Win10 w = win10(sp + sy * kCW, lx);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m] - w.v[4 + e - m + 1], d);
      el2(D[0], e) = d;
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
      el2(D[1], e) = d;
    }
  }
  {
    float2 zc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) zc[m] = sld2(ring + slot_after(s0, m) * kPl + sy * kCW + lx + 4);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el2(zc[3 + m], e) - el2(zc[4 - m], e), d);
      el2(D[2], e) = d;
    }
  }
  if (CROSS) {
    // cross taps (Sec. 3.1) over both transverse axes, in the order of the
    // tile kernels: w row j, up / dn rows j +- 1 of plane k; zp, zm row j of
    // planes k +- 1; zp_up, zm_up row j+1, zp_dn row j-1 of those planes
    const float *pp = ring + slot_after(s0, 4) * kPl, *pm = ring + slot_after(s0, 2) * kPl;
    const Win6 w = win6(sp + sy * kCW, lx), up = win6(sp + (sy + 1) * kCW, lx), dn = win6(sp + (sy - 1) * kCW, lx);
    const Win6 zp = win6(pp + sy * kCW, lx), zm = win6(pm + sy * kCW, lx);
    const Win6 zp_up = win6(pp + (sy + 1) * kCW, lx), zm_up = win6(pm + (sy + 1) * kCW, lx);
    const Win6 zp_dn = win6(pp + (sy - 1) * kCW, lx);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      el2(D[0], e) = fmaf(P.g11h, (((up.v[3 + e] - up.v[2 + e]) + (dn.v[3 + e] - dn.v[2 + e])) +
                                ((zp.v[3 + e] - zp.v[2 + e]) + (zm.v[3 + e] - zm.v[2 + e]))), el2(D[0], e));
      el2(D[1], e) = fmaf(P.g11h, (((up.v[3 + e] - w.v[3 + e]) + (up.v[1 + e] - w.v[1 + e])) +
                                ((zp_up.v[2 + e] - zp.v[2 + e]) + (zm_up.v[2 + e] - zm.v[2 + e]))), el2(D[1], e));
      el2(D[2], e) = fmaf(P.g11h, (((zp.v[3 + e] - w.v[3 + e]) + (zp.v[1 + e] - w.v[1 + e])) +
                                ((zp_up.v[2 + e] - up.v[2 + e]) + (zp_dn.v[2 + e] - dn.v[2 + e]))), el2(D[2], e));
    }
  }
  const float2 k1 = sldh2(reinterpret_cast<const bf16 *>(st + S::oK) + o);
  float2 v0 = sld2(st + S::oV + o), v1 = sld2(st + S::oV + kArr + o), v2 = sld2(st + S::oV + 2 * kArr + o);
  float2 Sd[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int e = 0; e < 2; ++e) el2(Sd[a], e) = el2(D[a], e) * el2(k1, e);
  const int xside = EDGE ? R.xs_side(x0) : -1;
  const bool ys = EDGE && R.ys_row(y0) != INT_MIN, zs = EDGE && R.zs_plane(k) >= 0;
  // coefficients of every mechanism and axis first, C-PML strips included,
  // so that the strip loads a staged-layout edge unit reads from global
  // memory are all in flight together
  float2 A[N > 0 ? N : 1][3], B[N > 0 ? N : 1][3];
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    const float2 a = sldh2(reinterpret_cast<const bf16 *>(st + S::oA) + nu * kArr + o);
    const float2 b = sldb2(reinterpret_cast<const bf16 *>(st + S::oB) + nu * kArr + o);
#pragma unroll
    for (int a3 = 0; a3 < 3; ++a3) {
      A[nu][a3] = a;
      B[nu][a3] = b;
    }
    if (EDGE) strips_of<N, 1, PS>(P, R, st + S::oS, xside, ys, zs, nu, i0, j, k, ly, lx, A[nu], B[nu]);
  }
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    float2 qq[3];
#pragma unroll
    for (int a3 = 0; a3 < 3; ++a3) qq[a3] = PS ? sld2(st + S::oPsi + (a3 * N + nu) * kArr + o) : q[a3][nu];
    relax3(P, P.psi1, nu * Sn + c, i0, EDGE, qq, A[nu], B[nu], D, Sd);
  }
  const Face3 f = face3<EDGE>(P, reinterpret_cast<const bf16 *>(st + S::oRho), x0, y0, k, lx, ly);
  const float rr[3] = {f.r0, f.r1, f.r2}, ru[2] = {f.u0, f.u1}, rz[2] = {f.z0, f.z1};
  if (P.nl_vel) {
    // momentum factors of the literal system (Eq. general5) at the x, y, z
    // faces: p from the staged planes (zero beyond the grid), K of the cell
    // and of its +1 neighbours from the staged K box, clamped to the last cell
    const Face3 g = face3<EDGE>(P, reinterpret_cast<const bf16 *>(st + S::oKm), x0, y0, k, lx, ly);
    // 1 / K of each of the seven cells once (mom_factor takes them the same way)
    const float Kr[3] = {qdiv(1.f, g.r0), qdiv(1.f, g.r1), qdiv(1.f, g.r2)};
    const float Ku[2] = {qdiv(1.f, g.u0), qdiv(1.f, g.u1)}, Kz[2] = {qdiv(1.f, g.z0), qdiv(1.f, g.z1)};
    const float *pr = sp + sy * kCW + lx + 4, *pu = sp + (sy + 1) * kCW + lx + 4;
    const float *pz = ring + slot_after(s0, 4) * kPl + sy * kCW + lx + 4;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float fx = mom_factor_ik(Kr[e], Kr[e + 1], pr[e], pr[e + 1]);
      const float fy = mom_factor_ik(Kr[e], Ku[e], pr[e], pu[e]);
      const float fz = mom_factor_ik(Kr[e], Kz[e], pr[e], pz[e]);
      el2(v0, e) = vel_upd(el2(v0, e), qdiv(P.two_dt, rr[e] + rr[e + 1]), el2(Sd[0], e), fx);
      el2(v1, e) = vel_upd(el2(v1, e), qdiv(P.two_dt, rr[e] + ru[e]), el2(Sd[1], e), fy);
      el2(v2, e) = vel_upd(el2(v2, e), qdiv(P.two_dt, rr[e] + rz[e]), el2(Sd[2], e), fz);
    }
  } else {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      el2(v0, e) = vel_upd(el2(v0, e), qdiv(P.two_dt, rr[e] + rr[e + 1]), el2(Sd[0], e));
      el2(v1, e) = vel_upd(el2(v1, e), qdiv(P.two_dt, rr[e] + ru[e]), el2(Sd[1], e));
      el2(v2, e) = vel_upd(el2(v2, e), qdiv(P.two_dt, rr[e] + rz[e]), el2(Sd[2], e));
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

template <int N, bool EDGE, bool CROSS, bool PS>
__device__ __forceinline__ void prs3_compute(const StepParams &P, const Region3 &R, const float *st, const float *ring,
                                             const float *sub, int x0, int y0, int k, int tid, const Psi<N> &q) {
  using S = Prs3<N, CROSS, PS>;
  const int lx = 2 * (tid & 63), ly = tid >> 6;
  const int i0 = x0 + lx, j = y0 + ly;
  if (EDGE && (i0 >= P.nx || j >= P.ny)) return;
  const long long c = (long long)k * P.plane + (long long)j * P.pitch + i0;
  const long long Sn = P.npts_alloc;
  const int o = ly * kTX + lx;
  constexpr int kPl = S::kPlane;
  const int s0 = ring_slot(k - 4);  // planes k-4 .. k+3 of the ring: slots s0 + 0 .. 7
  const float *subx = sub, *suby = sub + kSub * S::kXPlane;
  float2 D[3];
  {
    // v_x row j of plane k (stage rows y0 .., or ring rows y0-1 ..), columns x0-4 ..
    const float *row = CROSS ? subx + sub_slot(k) * S::kXPlane + (ly + 1) * kCW : st + S::oVx + ly * kCW;
    const Win10 w = win10(row, lx);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m - 1] - w.v[4 + e - m], d);
      el2(D[0], e) = d;
    }
  }
  {
    // v_y rows j-4 .. j+3 of plane k
    float2 col[8];
#pragma unroll
    for (int m = 0; m < 8; ++m)
      col[m] = CROSS ? sld2(suby + sub_slot(k) * S::kYPlane + (ly + m) * kCW + lx + 4)
                     : sld2(st + S::oVy + (ly + m) * kTX + lx);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el2(col[4 + m - 1], e) - el2(col[4 - m], e), d);
      el2(D[1], e) = d;
    }
  }
  {
    // v_z planes k-4 .. k+3 of the ring
    float2 zc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m)
      zc[m] = CROSS ? sld2(ring + slot_after(s0, m) * kPl + (ly + 1) * kCW + lx + 4)
                    : sld2(ring + slot_after(s0, m) * kPl + o);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el2(zc[4 + m - 1], e) - el2(zc[4 - m], e), d);
      el2(D[2], e) = d;
    }
  }
  if (CROSS) {
    // cross taps (Sec. 3.1) at the centres, in the order of the tile
    // kernels: g11 sum_{t != q} sum_{s = +-1} (v_q(c + s e_t) - v_q(c - e_q + s e_t))
    {
      const float *xk = subx + sub_slot(k) * S::kXPlane, *xp = subx + sub_slot(k + 1) * S::kXPlane,
                  *xm = subx + sub_slot(k - 1) * S::kXPlane;
      const Win6 a = win6(xk + (ly + 2) * kCW, lx), b = win6(xk + ly * kCW, lx);
      const Win6 cc = win6(xp + (ly + 1) * kCW, lx), dd = win6(xm + (ly + 1) * kCW, lx);
#pragma unroll
      for (int e = 0; e < 2; ++e)
        el2(D[0], e) = fmaf(P.g11h, (((a.v[2 + e] - a.v[1 + e]) + (b.v[2 + e] - b.v[1 + e])) +
                                  ((cc.v[2 + e] - cc.v[1 + e]) + (dd.v[2 + e] - dd.v[1 + e]))), el2(D[0], e));
    }
    {
      const float *yk = suby + sub_slot(k) * S::kYPlane, *yp = suby + sub_slot(k + 1) * S::kYPlane,
                  *ym = suby + sub_slot(k - 1) * S::kYPlane;
      const Win6 w0 = win6(yk + (ly + 4) * kCW, lx), w1 = win6(yk + (ly + 3) * kCW, lx);
      const Win6 zp0 = win6(yp + (ly + 4) * kCW, lx), zp1 = win6(yp + (ly + 3) * kCW, lx);
      const Win6 zm0 = win6(ym + (ly + 4) * kCW, lx), zm1 = win6(ym + (ly + 3) * kCW, lx);
#pragma unroll
      for (int e = 0; e < 2; ++e)
        el2(D[1], e) = fmaf(P.g11h, (((w0.v[3 + e] - w1.v[3 + e]) + (w0.v[1 + e] - w1.v[1 + e])) +
                                  ((zp0.v[2 + e] - zp1.v[2 + e]) + (zm0.v[2 + e] - zm1.v[2 + e]))), el2(D[1], e));
    }
    {
      const float *zk = ring + slot_after(s0, 4) * kPl, *zk1 = ring + slot_after(s0, 3) * kPl;
      const Win6 z0 = win6(zk + (ly + 1) * kCW, lx), z1 = win6(zk1 + (ly + 1) * kCW, lx);
      const Win6 u0 = win6(zk + (ly + 2) * kCW, lx), u1 = win6(zk1 + (ly + 2) * kCW, lx);
      const Win6 d0 = win6(zk + ly * kCW, lx), d1 = win6(zk1 + ly * kCW, lx);
#pragma unroll
      for (int e = 0; e < 2; ++e)
        el2(D[2], e) = fmaf(P.g11h, (((z0.v[3 + e] - z1.v[3 + e]) + (z0.v[1 + e] - z1.v[1 + e])) +
                                  ((u0.v[2 + e] - u1.v[2 + e]) + (d0.v[2 + e] - d1.v[2 + e]))), el2(D[2], e));
    }
  }
  const float2 k2 = sldh2(reinterpret_cast<const bf16 *>(st + S::oIk) + o);
  const float2 K = sldh2(reinterpret_cast<const bf16 *>(st + S::oKm) + o);
  float2 ch = make_float2(0.f, 0.f);
  if (P.nl) ch = sldh2(reinterpret_cast<const bf16 *>(st + S::oChi) + o);
  float2 p = sld2(st + S::oP + o);
  float2 Sd[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int e = 0; e < 2; ++e) el2(Sd[a], e) = el2(D[a], e) * el2(k2, e);
  const int xside = EDGE ? R.xs_side(x0) : -1;
  const bool ys = EDGE && R.ys_row(y0) != INT_MIN, zs = EDGE && R.zs_plane(k) >= 0;
  // coefficients of every mechanism and axis first, C-PML strips included,
  // so that the strip loads a staged-layout edge unit reads from global
  // memory are all in flight together
  float2 A[N > 0 ? N : 1][3], B[N > 0 ? N : 1][3];
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    const float2 a = sldh2(reinterpret_cast<const bf16 *>(st + S::oA) + nu * kArr + o);
    const float2 b = sldb2(reinterpret_cast<const bf16 *>(st + S::oB) + nu * kArr + o);
#pragma unroll
    for (int a3 = 0; a3 < 3; ++a3) {
      A[nu][a3] = a;
      B[nu][a3] = b;
    }
    if (EDGE) strips_of<N, 2, PS>(P, R, st + S::oS, xside, ys, zs, nu, i0, j, k, ly, lx, A[nu], B[nu]);
  }
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    float2 qq[3];
#pragma unroll
    for (int a3 = 0; a3 < 3; ++a3) qq[a3] = PS ? sld2(st + S::oPsi + (a3 * N + nu) * kArr + o) : q[a3][nu];
    relax3(P, P.psi2, nu * Sn + c, i0, EDGE, qq, A[nu], B[nu], D, Sd);
  }
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    float upd = P.dt * el2(K, e) * (el2(Sd[0], e) + el2(Sd[1], e) + el2(Sd[2], e));
    if (P.nl) upd = qdiv(upd, fmaf(el2(ch, e), el2(p, e), 1.f));
    el2(p, e) -= upd;
  }
  if (EDGE) p = mask_pad2(p, i0, P.nx);
  st_state2(P.p, c, p);
}

// One half step.  Block (32, 16), one per SM; items blockIdx.x,
// blockIdx.x + gridDim.x, ...; within an item the units k0 .. k1-1 in order.
template <int N, bool VEL, bool CROSS, bool PS>
__global__ void __launch_bounds__(kThreads, 1)
    pipe3d_kernel(const StepParams P, const Region3 R, const __grid_constant__ PipeMaps T) {
  using G = Ring3<N, VEL, CROSS, PS>;
  constexpr int kStage = G::kStage;
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int ok[2];  // per stage: thread 0 never rewrites a flag a thread has yet to read
  float *smem = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float *ring = smem + 2 * kStage;
  float *sub = ring + kSlots * G::kPlane;  // cross-tap rings of the pressure half step
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
  const bool nl = P.nl != 0, nlv = VEL && P.nl_vel != 0;
  if (tid == 0)
    issue3<N, VEL, CROSS, PS>(T, R, smem, ring, sub, &bar[0], x0, y0, k, ring_first<VEL>(k), ring_first<VEL>(k) + 7,
                          k - 1, k + 1, nl, nlv);
  pending |= 1u;
  // this thread's memory variables, one unit ahead of the compute
  const int lx = 2 * (tid & 63), ly = tid >> 6;
  float *const *psi = VEL ? P.psi1 : P.psi2;
  auto psi_of = [&](int ux0, int uy0, int uk, Psi<N> &q) {
    const int i0 = ux0 + lx, j = uy0 + ly;
    load_psi<N>(psi, P.npts_alloc, (long long)uk * P.plane + (long long)j * P.pitch + i0, i0 < P.nx && j < P.ny,
                q);
  };
  Psi<N> qc, qn;
  if (!PS) psi_of(x0, y0, k, qc);
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
          issue3<N, VEL, CROSS, PS>(T, R, smem + q * kStage, ring, sub, &bar[q], nx0, ny0, nk, kp, kp, nk + 1, nk + 1,
                                nl, nlv);
        if (!R.interior(nx0, ny0, nk)) prefetch_strips<N, VEL ? 1 : 2>(P, R, nx0, ny0, nk, tid);
      }
      pending |= 1u << q;
    }
    if (!PS && more) psi_of(nx0, ny0, nk, qn);
    float *cur = smem + s * kStage;
    if (R.interior(x0, y0, k)) {
      if (VEL) vel3_compute<N, false, CROSS, PS>(P, R, cur, ring, x0, y0, k, tid, qc);
      else prs3_compute<N, false, CROSS, PS>(P, R, cur, ring, sub, x0, y0, k, tid, qc);
    } else {
      if (VEL) vel3_compute<N, true, CROSS, PS>(P, R, cur, ring, x0, y0, k, tid, qc);
      else prs3_compute<N, true, CROSS, PS>(P, R, cur, ring, sub, x0, y0, k, tid, qc);
    }
    if (!more) break;
    if (fresh) {  // a new column: all ring planes, once every thread is done with the rings
      __syncthreads();
      if (tid == 0)
        issue3<N, VEL, CROSS, PS>(T, R, smem + q * kStage, ring, sub, &bar[q], nx0, ny0, nk, ring_first<VEL>(nk),
                              ring_first<VEL>(nk) + 7, nk - 1, nk + 1, nl, nlv);
      pending |= 1u << q;
    }
    it = nit;
    x0 = nx0; y0 = ny0; k0 = nk0; k1 = nk1; k = nk;
    s = q;
    if (!PS) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int nu = 0; nu < N; ++nu) qc[a][nu] = qn[a][nu];
    }
  }
}

// The same half step for several contexts in one launch (a batch of 3D
// problems): a table of work items {context, item of that context}; each
// block takes a contiguous run of the table, so consecutive items mostly
// share a context, whose parameters and work layout it keeps in shared
// memory (the tensor maps stay in global memory).  A new item always reloads
// the plane rings; the next item's first copies are issued after the
// current item's last unit, as in the single-context kernel.
template <int N, bool VEL, bool CROSS, bool PS>
__global__ void __launch_bounds__(kThreads, 1)
    pipe3d_batched_kernel(const StepParams *Ps, const Region3 *Rs, const PipeMaps *Ts, const int2 *items,
                          const int *runs) {
  using G = Ring3<N, VEL, CROSS, PS>;
  constexpr int kStage = G::kStage;
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int ok[2];
  __shared__ __align__(16) StepParams sP;
  __shared__ __align__(16) Region3 sR;
  float *smem = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float *ring = smem + 2 * kStage;
  float *sub = ring + kSlots * G::kPlane;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  // a contiguous run of items per block, balanced by the host over the
  // items' edge and interior units
  const int h_end = runs[blockIdx.x + 1];
  int h = runs[blockIdx.x];
  if (h >= h_end) return;
  auto load_ctx = [&](int c) {  // every thread; callers put barriers around it
    const int *ps = reinterpret_cast<const int *>(Ps + c);
    int *pd = reinterpret_cast<int *>(&sP);
    for (int w = tid; w < (int)(sizeof(StepParams) / 4); w += kThreads) pd[w] = __ldg(ps + w);
    const int *rs = reinterpret_cast<const int *>(Rs + c);
    int *rd = reinterpret_cast<int *>(&sR);
    for (int w = tid; w < (int)(sizeof(Region3) / 4); w += kThreads) rd[w] = __ldg(rs + w);
  };
  int2 e = items[h];
  int ctx = e.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbarrier_init();
  }
  load_ctx(ctx);
  __syncthreads();
  int x0, y0, k0, k1;
  sR.item(e.y, x0, y0, k0, k1);
  int k = k0;
  unsigned phase = 0, pending = 0;
  bool nl = sP.nl != 0, nlv = VEL && sP.nl_vel != 0;
  // thread 0 acquires a context's tensor maps (written by a host copy) before
  // its first copy through them
  auto acquire = [&](int c) {
    for (int m = 0; m < kPipeMaps; ++m) fence_tensormap_acquire(&Ts[c].m[m]);
  };
  if (tid == 0) acquire(ctx);
  if (tid == 0)
    issue3<N, VEL, CROSS, PS>(Ts[ctx], sR, smem, ring, sub, &bar[0], x0, y0, k, ring_first<VEL>(k),
                              ring_first<VEL>(k) + 7, k - 1, k + 1, nl, nlv);
  pending |= 1u;
  const int lx = 2 * (tid & 63), ly = tid >> 6;
  auto psi_of = [&](const StepParams &Q, int ux0, int uy0, int uk, Psi<N> &q) {
    const int i0 = ux0 + lx, j = uy0 + ly;
    load_psi<N>(VEL ? Q.psi1 : Q.psi2, Q.npts_alloc, (long long)uk * Q.plane + (long long)j * Q.pitch + i0,
                i0 < Q.nx && j < Q.ny, q);
  };
  Psi<N> qc, qn;
  if (!PS) psi_of(sP, x0, y0, k, qc);
  int s = 0;
#pragma unroll 1
  while (true) {
    if (tid == 0) ok[s] = mbar_wait_bounded(&bar[s], (phase >> s) & 1u);
    __syncthreads();
    if (!ok[s]) {
      if (tid == 0) {
        report_status(sP.status, kStatusWaitTimeout);
        if ((pending >> (s ^ 1)) & 1u) mbar_wait_bounded(&bar[s ^ 1], (phase >> (s ^ 1)) & 1u);
      }
      return;
    }
    phase ^= 1u << s;
    pending &= ~(1u << s);
    // the next unit: the next plane of this item, or the first of the next item
    int nh = h, nctx = ctx, nx0 = x0, ny0 = y0, nk0 = k0, nk1 = k1, nk = k + 1;
    if (nk >= k1) {
      nh = h + 1;
      if (nh < h_end) {
        const int2 en = items[nh];
        nctx = en.x;
        Rs[nctx].item(en.y, nx0, ny0, nk0, nk1);
      }
      nk = nk0;
    }
    const bool more = nh < h_end, fresh = nh != h;
    const int q = s ^ 1;
    if (more && !fresh) {
      if (tid < 32) {
        const int kp = ring_first<VEL>(nk) + 7;
        if (tid == 0)
          issue3<N, VEL, CROSS, PS>(Ts[ctx], sR, smem + q * kStage, ring, sub, &bar[q], nx0, ny0, nk, kp, kp,
                                    nk + 1, nk + 1, nl, nlv);
        if (!sR.interior(nx0, ny0, nk)) prefetch_strips<N, VEL ? 1 : 2>(sP, sR, nx0, ny0, nk, tid);
      }
      pending |= 1u << q;
    }
    if (!PS && more) psi_of(nctx == ctx ? sP : Ps[nctx], nx0, ny0, nk, qn);
    float *cur = smem + s * kStage;
    if (sR.interior(x0, y0, k)) {
      if (VEL) vel3_compute<N, false, CROSS, PS>(sP, sR, cur, ring, x0, y0, k, tid, qc);
      else prs3_compute<N, false, CROSS, PS>(sP, sR, cur, ring, sub, x0, y0, k, tid, qc);
    } else {
      if (VEL) vel3_compute<N, true, CROSS, PS>(sP, sR, cur, ring, x0, y0, k, tid, qc);
      else prs3_compute<N, true, CROSS, PS>(sP, sR, cur, ring, sub, x0, y0, k, tid, qc);
    }
    if (!more) break;
    if (fresh) {  // a new item: every thread is done with the rings (and the context's parameters)
      __syncthreads();
      if (nctx != ctx) {
        load_ctx(nctx);
        __syncthreads();
        ctx = nctx;
        nl = sP.nl != 0;
        nlv = VEL && sP.nl_vel != 0;
        if (tid == 0) acquire(ctx);
      }
      if (tid == 0)
        issue3<N, VEL, CROSS, PS>(Ts[ctx], sR, smem + q * kStage, ring, sub, &bar[q], nx0, ny0, nk,
                                  ring_first<VEL>(nk), ring_first<VEL>(nk) + 7, nk - 1, nk + 1, nl, nlv);
      pending |= 1u << q;
    }
    h = nh;
    x0 = nx0; y0 = ny0; k0 = nk0; k1 = nk1; k = nk;
    s = q;
    if (!PS) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int nu = 0; nu < N; ++nu) qc[a][nu] = qn[a][nu];
    }
  }
}

template <int N, bool VEL, bool CROSS, bool PS>
cudaError_t pipe3_batched_launch(const StepParams *Ps, const Region3 *Rs, const PipeMaps *Ts, const int2 *items,
                                 const int *runs, int grid, cudaStream_t st) {
  constexpr size_t bytes = Ring3<N, VEL, CROSS, PS>::kBytes;
  cudaError_t e = cudaFuncSetAttribute(pipe3d_batched_kernel<N, VEL, CROSS, PS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  pipe3d_batched_kernel<N, VEL, CROSS, PS><<<grid, dim3(32, kThreads / 32), bytes, st>>>(Ps, Rs, Ts, items, runs);
  return cudaGetLastError();
}

template <bool VEL, bool CROSS, bool PS>
cudaError_t pipe3_batched_dispatch(int n_relax, const StepParams *Ps, const Region3 *Rs, const PipeMaps *Ts,
                                   const int2 *items, const int *runs, int grid, cudaStream_t st) {
  switch (n_relax) {
    case 0: return pipe3_batched_launch<0, VEL, CROSS, PS>(Ps, Rs, Ts, items, runs, grid, st);
    case 1: return pipe3_batched_launch<1, VEL, CROSS, PS>(Ps, Rs, Ts, items, runs, grid, st);
    case 2: return pipe3_batched_launch<2, VEL, CROSS, PS>(Ps, Rs, Ts, items, runs, grid, st);
    case 3: return pipe3_batched_launch<3, VEL, CROSS, PS>(Ps, Rs, Ts, items, runs, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int N, bool VEL, bool CROSS, bool PS>
cudaError_t pipe3_launch(const StepParams &P, const Region3 &R, int grid, const PipeMaps &T, cudaStream_t st) {
  constexpr size_t bytes = Ring3<N, VEL, CROSS, PS>::kBytes;
  static_assert(bytes + 64 <= 227 * 1024, "stages exceed shared memory");
  cudaError_t e = cudaFuncSetAttribute(pipe3d_kernel<N, VEL, CROSS, PS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  pipe3d_kernel<N, VEL, CROSS, PS><<<grid, dim3(32, kThreads / 32), bytes, st>>>(P, R, T);
  return cudaGetLastError();
}

template <bool VEL, bool CROSS, bool PS>
cudaError_t pipe3_dispatch(const StepParams &P, const Region3 &R, int grid, const PipeMaps &T, cudaStream_t st) {
  switch (P.n_relax) {
    case 0: return pipe3_launch<0, VEL, CROSS, PS>(P, R, grid, T, st);
    case 1: return pipe3_launch<1, VEL, CROSS, PS>(P, R, grid, T, st);
    case 2: return pipe3_launch<2, VEL, CROSS, PS>(P, R, grid, T, st);
    case 3: return pipe3_launch<3, VEL, CROSS, PS>(P, R, grid, T, st);
    default: return cudaErrorInvalidValue;
  }
}

// The layout of a half step: the memory variables staged with the other
// arrays (PS) unless the stage needs that room for the cross taps' planes
// or (velocity) the literal system's K box; then they are loaded into
// registers one unit ahead and the C-PML strips of every axis are staged.
bool psi_staged(bool vel, const StepParams &P) { return P.g11h == 0.f && !(vel && P.nl_vel); }

// The x strip's coefficients come by TMA when a box of L values per row
// starts on a 16-byte boundary and fits the stage (L a multiple of 8, at
// most kXsMax), and no unit reaches both sides (nx >= 128 + L).
bool x_strip_staged(const StepParams &P) {
  const int L = P.L[0];
  return P.n_relax > 0 && L > 0 && L % 8 == 0 && L <= kXsMax && P.nx >= kTX + L && P.ny >= kHT &&
         P.sa1[0] != nullptr;
}
// The y strip's by TMA when no unit reaches both sides (ny >= 2L + 8) and
// the strip holds at least a unit's rows; the z strip's always (a unit is
// one plane).
bool y_strip_staged(const StepParams &P) {
  const int L = P.L[1];
  return P.n_relax > 0 && L >= kHT / 2 && P.ny >= 2 * L + kHT && P.sa1[1] != nullptr;
}
bool z_strip_staged(const StepParams &P) {
  const int L = P.L[2];
  return P.n_relax > 0 && L > 0 && P.ny >= kHT && P.sa1[2] != nullptr;
}

// Planes per item: the split of each column into items that minimises the
// busiest block's work, counting each item's start (eight ring planes and
// one exposed copy latency) as about 1.5 units.  ps: the layout stages the
// memory variables, so the y and z strips are read per cell.
Region3 region3_of(const StepParams &P, int grid, bool ps) {
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
  R.ysL = !ps && y_strip_staged(P) ? P.L[1] : 0;
  R.zsL = !ps && z_strip_staged(P) ? P.L[2] : 0;
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
  // bf16 maps; N <= 3 keeps the 4D boxes and the stages within shared
  // memory; no periodic axis
  return P.nz > 1 && map_kind == 1 && P.n_relax >= 0 && P.n_relax <= 3 && !P.periodic[0] && !P.periodic[1] &&
         !P.periodic[2];
}

cudaError_t build_pipe3d_maps(const StepParams &P, PipeMaps *vel, PipeMaps *prs, const char **why) {
  *vel = PipeMaps{};
  *prs = PipeMaps{};
  const int N = P.n_relax;
  const bool cross = P.g11h != 0.f;
  using ull = unsigned long long;
  const ull nx = P.nx, ny = P.ny, nz = P.nz, S = P.npts_alloc;
  const ull f3[2] = {(ull)P.pitch * 4, (ull)P.plane * 4}, h3[2] = {(ull)P.pitch * 2, (ull)P.plane * 2};
  const ull f4[3] = {(ull)P.pitch * 4, (ull)P.plane * 4, S * 4}, h4[3] = {(ull)P.pitch * 2, (ull)P.plane * 2, S * 2};
  const ull d3[3] = {nx, ny, nz};
  const ull dv[4] = {nx, ny, nz, 3}, dab[4] = {nx, ny, nz, (ull)N}, dpsi[4] = {nx, ny, nz, (ull)(3 * N)};
  const unsigned halo[3] = {kCW, kHT + 7, 1}, rho[3] = {kRWb, kHT + 1, 2}, one[3] = {kTX, kHT, 1},
                 v4[4] = {kTX, kHT, 1, 3}, ab4[4] = {kTX, kHT, 1, (unsigned)N},
                 psi4[4] = {kTX, kHT, 1, (unsigned)(3 * N)}, vx[3] = {kCW, kHT, 1},
                 vy[3] = {kTX, kHT + 7, 1}, halo1[3] = {kCW, kHT + 2, 1};
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
  if (P.nl_vel) ok = ok && encode_tensor_map(&vel->m[12], P.K, 2, 3, d3, h3, rho);
  // pressure half step
  if (cross) {
    ok = ok && encode_tensor_map(&prs->m[0], P.v[0], 4, 3, d3, f3, halo1);
    ok = ok && encode_tensor_map(&prs->m[1], P.v[1], 4, 3, d3, f3, halo);
    ok = ok && encode_tensor_map(&prs->m[2], P.v[2], 4, 3, d3, f3, halo1);
  } else {
    ok = ok && encode_tensor_map(&prs->m[0], P.v[0], 4, 3, d3, f3, vx);
    ok = ok && encode_tensor_map(&prs->m[1], P.v[1], 4, 3, d3, f3, vy);
    ok = ok && encode_tensor_map(&prs->m[2], P.v[2], 4, 3, d3, f3, one);
  }
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
  if (y_strip_staged(P)) {  // y strips [N][z][2L][x] bf16, boxes 128 x 8 x 1 x N
    const ull L = (ull)P.L[1];
    const ull dys[4] = {nx, 2 * L, nz, (ull)N},
              sys[3] = {(ull)P.pitch * 2, 2 * L * (ull)P.pitch * 2, (ull)P.strip_nu[1] * 2};
    ok = ok && encode_tensor_map(&vel->m[13], P.sa1[1], 2, 4, dys, sys, ab4);
    ok = ok && encode_tensor_map(&vel->m[14], P.sb1[1], 2, 4, dys, sys, ab4);
    ok = ok && encode_tensor_map(&prs->m[13], P.sa2[1], 2, 4, dys, sys, ab4);
    ok = ok && encode_tensor_map(&prs->m[14], P.sb2[1], 2, 4, dys, sys, ab4);
  }
  if (z_strip_staged(P)) {  // z strips [N][2L][y][x] bf16, boxes 128 x 8 x 1 x N
    const ull L = (ull)P.L[2];
    const ull dzs[4] = {nx, ny, 2 * L, (ull)N},
              szs[3] = {(ull)P.pitch * 2, ny * (ull)P.pitch * 2, (ull)P.strip_nu[2] * 2};
    ok = ok && encode_tensor_map(&vel->m[15], P.sa1[2], 2, 4, dzs, szs, ab4);
    ok = ok && encode_tensor_map(&vel->m[16], P.sb1[2], 2, 4, dzs, szs, ab4);
    ok = ok && encode_tensor_map(&prs->m[15], P.sa2[2], 2, 4, dzs, szs, ab4);
    ok = ok && encode_tensor_map(&prs->m[16], P.sb2[2], 2, 4, dzs, szs, ab4);
  }
  if (!ok) {
    *why = "cuTensorMapEncodeTiled rejected a 3D map (or the driver entry point is missing)";
    return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

bool pipe3d_layout_allowed(bool vel, const StepParams &P, int layout) {
  return layout != kLayoutStaged || psi_staged(vel, P);
}

size_t pipe3d_region_bytes() { return sizeof(Region3); }

long long pipe3d_region(const StepParams &P, int grid, bool vel, void *out) {
  const Region3 R = region3_of(P, grid, psi_staged(vel, P));
  std::memcpy(out, &R, sizeof R);
  return (long long)R.tnx * R.nhy * R.nseg;
}

bool pipe3d_staged_layout(bool vel, const StepParams &P) { return psi_staged(vel, P); }

void pipe3d_item_units(const StepParams &P, int grid, bool vel, int *n_edge, int *n_all) {
  const Region3 R = region3_of(P, grid, psi_staged(vel, P));
  const long long n = R.items();
  for (long long it = 0; it < n; ++it) {
    int x0, y0, k0, k1;
    R.item(it, x0, y0, k0, k1);
    int e = 0;
    for (int k = k0; k < k1; ++k) e += R.interior(x0, y0, k) ? 0 : 1;
    n_edge[it] = e;
    n_all[it] = k1 - k0;
  }
}

cudaError_t launch_pipe3d_batched(bool vel, bool cross, bool ps, int n_relax, const StepParams *Ps,
                                  const void *Rs, const PipeMaps *Ts, const int2 *items, const int *runs, int grid,
                                  cudaStream_t st) {
  const Region3 *R = static_cast<const Region3 *>(Rs);
  if (cross)
    return vel ? pipe3_batched_dispatch<true, true, false>(n_relax, Ps, R, Ts, items, runs, grid, st)
               : pipe3_batched_dispatch<false, true, false>(n_relax, Ps, R, Ts, items, runs, grid, st);
  if (vel)
    return ps ? pipe3_batched_dispatch<true, false, true>(n_relax, Ps, R, Ts, items, runs, grid, st)
              : pipe3_batched_dispatch<true, false, false>(n_relax, Ps, R, Ts, items, runs, grid, st);
  return ps ? pipe3_batched_dispatch<false, false, true>(n_relax, Ps, R, Ts, items, runs, grid, st)
            : pipe3_batched_dispatch<false, false, false>(n_relax, Ps, R, Ts, items, runs, grid, st);
}

cudaError_t launch_pipe3d(bool vel, const StepParams &P, int grid, const PipeMaps &T, cudaStream_t st, int layout) {
  const bool ps = layout == kLayoutRegisters ? false : psi_staged(vel, P);
  const Region3 R = region3_of(P, grid, ps);
  if (P.g11h != 0.f)
    return vel ? pipe3_dispatch<true, true, false>(P, R, grid, T, st)
               : pipe3_dispatch<false, true, false>(P, R, grid, T, st);
  if (vel)
    return ps ? pipe3_dispatch<true, false, true>(P, R, grid, T, st)
              : pipe3_dispatch<true, false, false>(P, R, grid, T, st);
  return ps ? pipe3_dispatch<false, false, true>(P, R, grid, T, st)
            : pipe3_dispatch<false, false, false>(P, R, grid, T, st);
}

}  // namespace fw2
