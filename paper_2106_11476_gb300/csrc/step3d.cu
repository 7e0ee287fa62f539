// 3D fused velocity and pressure half steps (sm_103a).
//
// Same arithmetic as the 2D kernels (Sec. 3.1 updates, Eqs. relaxation4,
// relaxation_psi, general6) with the third axis.  Each block owns a 128 x 8
// tile of an xy plane (256 threads, two rows each) and marches through kTZ
// planes along z; the xy stencil
// operand of the current plane is staged in shared memory with its halo, the
// z taps of each cell's own column are read through L2.
#include <type_traits>

#include "coef.cuh"
#include "maps.cuh"

namespace fw2 {

namespace {

// Map access of the 3D tile kernels; a map is named by its slot of
// StepParams::ms (kMsK, kMsRho, kMsChi, kMsIk1, kMsIk2, kMsA1 + nu, kMsB1 +
// nu, kMsA2 + nu, kMsB2 + nu), and v1 / v4 give its value at one cell / at
// the four cells c .. c + 3 (b as b).
// Dense3<MT>: one value per cell (float, bf16 or FP16 with the map's scale;
// bf16 and FP16 keep b as 1 - b).
template <typename MT>
struct Dense3 {
  using StripT = MT;
  static __device__ __forceinline__ const MT *base(const StepParams &P, int id, long long &off) {
    const long long S = P.npts_alloc;
    if (id >= kMsB2) { off = (id - kMsB2) * S; return static_cast<const MT *>(P.b2); }
    if (id >= kMsA2) { off = (id - kMsA2) * S; return static_cast<const MT *>(P.a2); }
    if (id >= kMsB1) { off = (id - kMsB1) * S; return static_cast<const MT *>(P.b1); }
    if (id >= kMsA1) { off = (id - kMsA1) * S; return static_cast<const MT *>(P.a1); }
    off = 0;
    return static_cast<const MT *>(id == kMsK ? P.K : id == kMsRho ? P.rho : id == kMsChi ? P.chi
                                   : id == kMsIk1 ? P.ik1 : P.ik2);
  }
  static __device__ __forceinline__ bool is_b(int id) {
    return (id >= kMsB1 && id < kMsA2) || id >= kMsB2;
  }
  static __device__ __forceinline__ float v1(const StepParams &P, int id, long long c) {
    long long off;
    const MT *p = base(P, id, off);
    return is_b(id) ? ldb(p, off + c, P.ms[id]) : ldmap(p, off + c, P.ms[id]);
  }
  static __device__ __forceinline__ float4 v4(const StepParams &P, int id, long long c) {
    long long off;
    const MT *p = base(P, id, off);
    return is_b(id) ? ldb4(p, off + c, P.ms[id]) : ldmap4(p, off + c, P.ms[id]);
  }
};
// Idx3<IT>: a tissue index per cell (uint8 or uint16) into the per-tissue
// float tables ([field][tab_stride] in global memory, read through L2 and the
// read-only cache; maps.cuh field order); the C-PML strips stay per cell.
template <typename IT>
struct Idx3 {
  using StripT = float;
  static __device__ __forceinline__ int field(int id) {
    return id == kMsK ? kTabK : id == kMsRho ? kTabRho : id == kMsChi ? kTabChi : id == kMsIk1 ? kTabIk1
         : id == kMsIk2 ? kTabIk2 : id < kMsB1 ? kTabRelax + (id - kMsA1)
         : id < kMsA2 ? kTabRelax + kTabSlots + (id - kMsB1) : id < kMsB2 ? kTabRelax + 2 * kTabSlots + (id - kMsA2)
                      : kTabRelax + 3 * kTabSlots + (id - kMsB2);
  }
  static __device__ __forceinline__ float v1(const StepParams &P, int id, long long c) {
    const int t = __ldg(reinterpret_cast<const IT *>(P.tissue) + c);
    return __ldg(P.table + (long long)field(id) * P.tab_stride + t);
  }
  static __device__ __forceinline__ float4 v4(const StepParams &P, int id, long long c) {
    const float *f = P.table + (long long)field(id) * P.tab_stride;
    if constexpr (sizeof(IT) == 1) {
      const uchar4 t = __ldg(reinterpret_cast<const uchar4 *>(P.tissue + c));
      return make_float4(__ldg(f + t.x), __ldg(f + t.y), __ldg(f + t.z), __ldg(f + t.w));
    } else {
      const ushort4 t = __ldg(reinterpret_cast<const ushort4 *>(reinterpret_cast<const IT *>(P.tissue) + c));
      return make_float4(__ldg(f + t.x), __ldg(f + t.y), __ldg(f + t.z), __ldg(f + t.w));
    }
  }
};
template <typename M>
constexpr bool kIndexed3 = std::is_same<M, Idx3<unsigned char>>::value || std::is_same<M, Idx3<unsigned short>>::value;

// a, b of mechanism nu for the derivative along axis Q at the four cells
// i0..i0+3 of row (j, k): from the boundary strip of axis Q when the cell
// lies inside the C-PML region of that axis (Sec. 3.3: each axis' parameters
// depend on the distance along that axis only), else from the interior maps.
// OP = 1: nabla_1 (faces), OP = 2: nabla_2 (centres).
template <int Q, int OP, typename M>
__device__ __forceinline__ void coef4(const StepParams &P, int nu, long long c, int i0, int j, int k, float4 &a,
                                      float4 &b) {
  using ST = typename M::StripT;
  const int ia = (OP == 1 ? kMsA1 : kMsA2) + nu, ib = (OP == 1 ? kMsB1 : kMsB2) + nu;
  const ST *sa = static_cast<const ST *>(OP == 1 ? P.sa1[Q] : P.sa2[Q]);
  const ST *sb = static_cast<const ST *>(OP == 1 ? P.sb1[Q] : P.sb2[Q]);
  const float s_a = P.ms[ia], s_b = P.ms[ib];
  const int L = P.L[Q];
  if (Q == 0) {
    const bool any = L > 0 && (i0 < L || i0 + 3 >= P.nx - L);
    if (!any) {
      a = M::v4(P, ia, c);
      b = M::v4(P, ib, c);
      return;
    }
    const long long row = (long long)nu * P.strip_nu[0] + ((long long)k * P.ny + j) * (2 * L);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int x = i0 + e;
      float av = 0.f, bv = 0.f;
      if (x < P.nx) {
        const int sc = strip_coord(x, P.nx, L);
        if (sc >= 0) {
          av = ldmap(sa, row + sc, s_a);
          bv = ldb(sb, row + sc, s_b);
        } else {
          av = M::v1(P, ia, c + e);
          bv = M::v1(P, ib, c + e);
        }
      }
      el(a, e) = av;
      el(b, e) = bv;
    }
  } else {
    const int sc = Q == 1 ? strip_coord(j, P.ny, L) : strip_coord(k, P.nz, L);
    if (sc < 0) {
      a = M::v4(P, ia, c);
      b = M::v4(P, ib, c);
    } else {
      const long long off =
          Q == 1 ? (long long)nu * P.strip_nu[1] + ((long long)k * (2 * L) + sc) * P.pitch + i0
                 : (long long)nu * P.strip_nu[2] + ((long long)sc * P.ny + j) * P.pitch + i0;
      a = ldmap4(sa, off, s_a);
      b = ldb4(sb, off, s_b);
    }
  }
}

// Stretched derivative of Eq. (relaxation4) for four cells:
//   S = D / kappa + sum_nu (w_new psi_new + w_old psi_old),
//   psi_new = b psi_old + a D    (Eq. relaxation_psi), psi written back.
template <int Q, int OP, int N, typename M>
__device__ __forceinline__ float4 stretch4(const StepParams &P, float *psi, float4 D, float4 ik, long long c, int i0,
                                           int j, int k) {
  float4 S = make_float4(D.x * ik.x, D.y * ik.y, D.z * ik.z, D.w * ik.w);
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    float4 a, b;
    coef4<Q, OP, M>(P, nu, c, i0, j, k, a, b);
    const long long o = (long long)nu * P.npts_alloc + c;
    const float4 ps = ld_state4(psi, o);
    float4 pn;
    pn.x = fmaf(b.x, ps.x, a.x * D.x);
    pn.y = fmaf(b.y, ps.y, a.y * D.y);
    pn.z = fmaf(b.z, ps.z, a.z * D.z);
    pn.w = fmaf(b.w, ps.w, a.w * D.w);
    S.x += fmaf(P.w_new, pn.x, P.w_old * ps.x);
    S.y += fmaf(P.w_new, pn.y, P.w_old * ps.y);
    S.z += fmaf(P.w_new, pn.z, P.w_old * ps.z);
    S.w += fmaf(P.w_new, pn.w, P.w_old * ps.w);
    st_state4(psi, o, pn);
  }
  return S;
}

constexpr int kTY3 = 16;  // tile rows (two per thread row)
constexpr int kBY3 = 8;   // thread rows
constexpr int kTZ = 8;    // planes per block

struct Win12 {
  float v[12];
};
__device__ __forceinline__ Win12 win12(const float *row, int tx) {
  Win12 w;
  const float4 *r4 = reinterpret_cast<const float4 *>(row) + tx;
  float4 a = r4[0], b = r4[1], c = r4[2];
  w.v[0] = a.x; w.v[1] = a.y; w.v[2] = a.z; w.v[3] = a.w;
  w.v[4] = b.x; w.v[5] = b.y; w.v[6] = b.z; w.v[7] = b.w;
  w.v[8] = c.x; w.v[9] = c.y; w.v[10] = c.z; w.v[11] = c.w;
  return w;
}


// xy tile and plane k clear of every C-PML strip and of the outer boundary:
// all three axes use the interior maps and no boundary rule applies.
__device__ __forceinline__ bool interior_xy(const StepParams &P, int x0, int y0) {
  const int Lx = P.L[0] > 4 ? P.L[0] : 4, Ly = P.L[1] > 4 ? P.L[1] : 4;
  return x0 >= Lx && x0 + kTX + Lx <= P.nx && y0 >= Ly && y0 + kTY3 + Ly <= P.ny;
}
__device__ __forceinline__ bool interior_z(const StepParams &P, int k) {
  const int Lz = P.L[2] > 4 ? P.L[2] : 4;
  return k >= Lz && k + Lz < P.nz;
}

// Twelve values x = i0-4 .. i0+7 of row (j, k) of a cell-indexed field read
// from global memory under the outer boundary rule (v[4 + e] is x = i0 + e);
// the cross taps' rows in planes the tile does not stage.
__device__ __forceinline__ Win12 win12_g(const StepParams &P, const float *f, int i0, int j, int k) {
  const float4 a = load_chunk(P, f, i0 - 4, j, k), b = load_chunk(P, f, i0, j, k), c = load_chunk(P, f, i0 + 4, j, k);
  Win12 w;
  w.v[0] = a.x; w.v[1] = a.y; w.v[2] = a.z; w.v[3] = a.w;
  w.v[4] = b.x; w.v[5] = b.y; w.v[6] = b.z; w.v[7] = b.w;
  w.v[8] = c.x; w.v[9] = c.y; w.v[10] = c.z; w.v[11] = c.w;
  return w;
}

// Cross taps of Sec. 3.1 over both transverse axes at the faces of the four
// cells i0..i0+3 of row (j, k): for the face of axis q,
// g11 sum_{t != q} sum_{s = +-1} (p(c + e_q + s e_t) - p(c + s e_t)).
// sp row sy is row j of plane k (rows sy +- 1 are j +- 1).
__device__ __forceinline__ void vel3_cross(const StepParams &P, const float (*sp)[kTX + 8], int sy, int tx, int i0,
                                           int j, int k, float4 &Dx, float4 &Dy, float4 &Dz) {
  const Win12 w = win12(sp[sy], tx), up = win12(sp[sy + 1], tx), dn = win12(sp[sy - 1], tx);
  const Win12 zp = win12_g(P, P.p, i0, j, k + 1), zm = win12_g(P, P.p, i0, j, k - 1);
  const Win12 zp_up = win12_g(P, P.p, i0, j + 1, k + 1), zm_up = win12_g(P, P.p, i0, j + 1, k - 1);
  const Win12 zp_dn = win12_g(P, P.p, i0, j - 1, k + 1);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    el(Dx, e) = fmaf(P.g11h, (((up.v[5 + e] - up.v[4 + e]) + (dn.v[5 + e] - dn.v[4 + e])) +
                           ((zp.v[5 + e] - zp.v[4 + e]) + (zm.v[5 + e] - zm.v[4 + e]))), el(Dx, e));
    el(Dy, e) = fmaf(P.g11h, (((up.v[5 + e] - w.v[5 + e]) + (up.v[3 + e] - w.v[3 + e])) +
                           ((zp_up.v[4 + e] - zp.v[4 + e]) + (zm_up.v[4 + e] - zm.v[4 + e]))), el(Dy, e));
    el(Dz, e) = fmaf(P.g11h, (((zp.v[5 + e] - w.v[5 + e]) + (zp.v[3 + e] - w.v[3 + e])) +
                           ((zp_up.v[4 + e] - up.v[4 + e]) + (zp_dn.v[4 + e] - dn.v[4 + e]))), el(Dz, e));
  }
}

// The same at the cell centres of the pressure half step, for axis q:
// g11 sum_{t != q} sum_{s = +-1} (v_q(c + s e_t) - v_q(c - e_q + s e_t)).
__device__ __forceinline__ void prs3_cross(const StepParams &P, int i0, int j, int k, float4 &Dx, float4 &Dy,
                                           float4 &Dz) {
  {
    const Win12 a = win12_g(P, P.v[0], i0, j + 1, k), b = win12_g(P, P.v[0], i0, j - 1, k);
    const Win12 c = win12_g(P, P.v[0], i0, j, k + 1), d = win12_g(P, P.v[0], i0, j, k - 1);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      el(Dx, e) = fmaf(P.g11h, (((a.v[4 + e] - a.v[3 + e]) + (b.v[4 + e] - b.v[3 + e])) +
                             ((c.v[4 + e] - c.v[3 + e]) + (d.v[4 + e] - d.v[3 + e]))), el(Dx, e));
  }
  {
    const Win12 y0 = win12_g(P, P.v[1], i0, j, k), y1 = win12_g(P, P.v[1], i0, j - 1, k);
    const Win12 zp0 = win12_g(P, P.v[1], i0, j, k + 1), zp1 = win12_g(P, P.v[1], i0, j - 1, k + 1);
    const Win12 zm0 = win12_g(P, P.v[1], i0, j, k - 1), zm1 = win12_g(P, P.v[1], i0, j - 1, k - 1);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      el(Dy, e) = fmaf(P.g11h, (((y0.v[5 + e] - y1.v[5 + e]) + (y0.v[3 + e] - y1.v[3 + e])) +
                             ((zp0.v[4 + e] - zp1.v[4 + e]) + (zm0.v[4 + e] - zm1.v[4 + e]))), el(Dy, e));
  }
  {
    const Win12 z0 = win12_g(P, P.v[2], i0, j, k), z1 = win12_g(P, P.v[2], i0, j, k - 1);
    const Win12 u0 = win12_g(P, P.v[2], i0, j + 1, k), u1 = win12_g(P, P.v[2], i0, j + 1, k - 1);
    const Win12 d0 = win12_g(P, P.v[2], i0, j - 1, k), d1 = win12_g(P, P.v[2], i0, j - 1, k - 1);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      el(Dz, e) = fmaf(P.g11h, (((z0.v[5 + e] - z1.v[5 + e]) + (z0.v[3 + e] - z1.v[3 + e])) +
                             ((u0.v[4 + e] - u1.v[4 + e]) + (d0.v[4 + e] - d1.v[4 + e]))), el(Dz, e));
  }
}

// Momentum factors of the literal nonlinear system (Eq. general5) at the x, y
// and z faces of the four cells i0..i0+3 of row (j, k): p from the staged
// plane (row sy of sp) and the z column (pz1 = p at k+1), K from the map with
// the density's neighbour rule; cells past nx are clamped (masked later).
template <typename M>
__device__ __forceinline__ void mom_factors3(const StepParams &P, const float (*sp)[kTX + 8], int sy, int tx, int i0,
                                             int j, int k, const float4 &pz1, float4 &fx, float4 &fy, float4 &fz) {
  const Win12 w = win12(sp[sy], tx), up = win12(sp[sy + 1], tx);
  const int jn = rho_coord(j + 1, P.ny, P.periodic[1]), kn = rho_coord(k + 1, P.nz, P.periodic[2]);
  const long long row = (long long)k * P.plane + (long long)j * P.pitch;
  const long long rowy = (long long)k * P.plane + (long long)jn * P.pitch;
  const long long rowz = (long long)kn * P.plane + (long long)j * P.pitch;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int x = min(i0 + e, P.nx - 1);
    const int xn = rho_coord(min(i0 + e + 1, P.nx), P.nx, P.periodic[0]);
    const float Kc = M::v1(P, kMsK, row + x);
    el(fx, e) = mom_factor(Kc, M::v1(P, kMsK, row + xn), w.v[4 + e], w.v[5 + e]);
    el(fy, e) = mom_factor(Kc, M::v1(P, kMsK, rowy + x), w.v[4 + e], up.v[4 + e]);
    el(fz, e) = mom_factor(Kc, M::v1(P, kMsK, rowz + x), w.v[4 + e], el(pz1, e));
  }
}

// Interior plane of the velocity half step: z taps first (L2), then every
// streaming load of the plane row before any store.
template <int N, typename M>
__device__ __forceinline__ void vel3d_fast(const StepParams &P, const float (*sp)[kTX + 8],
                                           const float (*sr)[kTX + 4], int i0, int j, int k, int tx, int ty) {
  const long long c = (long long)k * P.plane + (long long)j * P.pitch + i0;
  const long long S = P.npts_alloc;
  float4 Dz, pz1;
  {
    float4 zc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m)
      zc[m] = __ldg(reinterpret_cast<const float4 *>(P.p + c + (long long)(m - 3) * P.plane));
    pz1 = zc[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el(zc[3 + m], e) - el(zc[4 - m], e), d);
      el(Dz, e) = d;
    }
  }
  float4 v0 = ld_state4(P.v[0], c), v1 = ld_state4(P.v[1], c), v2 = ld_state4(P.v[2], c);
  const float4 k1 = M::v4(P, kMsIk1, c);
  const float4 rz = M::v4(P, kMsRho, c + P.plane);
  float4 A[N > 0 ? N : 1], B[N > 0 ? N : 1], Q0[N > 0 ? N : 1], Q1[N > 0 ? N : 1], Q2[N > 0 ? N : 1];
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    A[nu] = M::v4(P, kMsA1 + nu, c);
    B[nu] = M::v4(P, kMsB1 + nu, c);
    Q0[nu] = ld_state4(P.psi1[0], nu * S + c);
    Q1[nu] = ld_state4(P.psi1[1], nu * S + c);
    Q2[nu] = ld_state4(P.psi1[2], nu * S + c);
  }
  const int sy = ty + 3;
  const Win12 w = win12(sp[sy], tx);
  float4 Dx, Dy;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float d = 0.f;
#pragma unroll
    for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m] - w.v[4 + e - m + 1], d);
    el(Dx, e) = d;
  }
  {
    float4 col[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) col[m] = *reinterpret_cast<const float4 *>(&sp[sy - 3 + m][4 * tx + 4]);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el(col[3 + m], e) - el(col[4 - m], e), d);
      el(Dy, e) = d;
    }
  }
  const int lx = 4 * tx;
  const float4 r0 = *reinterpret_cast<const float4 *>(&sr[ty][lx]);
  const float r4 = sr[ty][lx + 4];
  const float4 ru = *reinterpret_cast<const float4 *>(&sr[ty + 1][lx]);
  float4 S0, S1, S2;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    el(S0, e) = el(Dx, e) * el(k1, e);
    el(S1, e) = el(Dy, e) * el(k1, e);
    el(S2, e) = el(Dz, e) * el(k1, e);
  }
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    float4 n0, n1, n2;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el(n0, e) = fmaf(el(B[nu], e), el(Q0[nu], e), el(A[nu], e) * el(Dx, e));
      el(n1, e) = fmaf(el(B[nu], e), el(Q1[nu], e), el(A[nu], e) * el(Dy, e));
      el(n2, e) = fmaf(el(B[nu], e), el(Q2[nu], e), el(A[nu], e) * el(Dz, e));
      el(S0, e) += fmaf(P.w_new, el(n0, e), P.w_old * el(Q0[nu], e));
      el(S1, e) += fmaf(P.w_new, el(n1, e), P.w_old * el(Q1[nu], e));
      el(S2, e) += fmaf(P.w_new, el(n2, e), P.w_old * el(Q2[nu], e));
    }
    st_state4(P.psi1[0], nu * S + c, n0);
    st_state4(P.psi1[1], nu * S + c, n1);
    st_state4(P.psi1[2], nu * S + c, n2);
  }
  const float rr[5] = {r0.x, r0.y, r0.z, r0.w, r4};
  if (P.nl_vel) {
    float4 fx, fy, fz;
    mom_factors3<M>(P, sp, sy, tx, i0, j, k, pz1, fx, fy, fz);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el(v0, e) = vel_upd(el(v0, e), qdiv(P.two_dt, rr[e] + rr[e + 1]), el(S0, e), el(fx, e));
      el(v1, e) = vel_upd(el(v1, e), qdiv(P.two_dt, rr[e] + el(ru, e)), el(S1, e), el(fy, e));
      el(v2, e) = vel_upd(el(v2, e), qdiv(P.two_dt, rr[e] + el(rz, e)), el(S2, e), el(fz, e));
    }
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el(v0, e) = vel_upd(el(v0, e), qdiv(P.two_dt, rr[e] + rr[e + 1]), el(S0, e));
      el(v1, e) = vel_upd(el(v1, e), qdiv(P.two_dt, rr[e] + el(ru, e)), el(S1, e));
      el(v2, e) = vel_upd(el(v2, e), qdiv(P.two_dt, rr[e] + el(rz, e)), el(S2, e));
    }
  }
  st_state4(P.v[0], c, v0);
  st_state4(P.v[1], c, v1);
  st_state4(P.v[2], c, v2);
}

// Interior plane of the pressure half step (same structure).
template <int N, typename M>
__device__ __forceinline__ void prs3d_fast(const StepParams &P, const float (*svx)[kTX + 8],
                                           const float (*svy)[kTX + 8], int i0, int j, int k, int tx, int ty) {
  const long long c = (long long)k * P.plane + (long long)j * P.pitch + i0;
  const long long S = P.npts_alloc;
  float4 Dz;
  {
    float4 zc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m)
      zc[m] = __ldg(reinterpret_cast<const float4 *>(P.v[2] + c + (long long)(m - 4) * P.plane));
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el(zc[4 + m - 1], e) - el(zc[4 - m], e), d);
      el(Dz, e) = d;
    }
  }
  float4 p = ld_state4(P.p, c);
  const float4 k2 = M::v4(P, kMsIk2, c);
  const float4 K = M::v4(P, kMsK, c);
  float4 ch = make_float4(0.f, 0.f, 0.f, 0.f);
  if (P.nl) ch = M::v4(P, kMsChi, c);
  float4 A[N > 0 ? N : 1], B[N > 0 ? N : 1], Q0[N > 0 ? N : 1], Q1[N > 0 ? N : 1], Q2[N > 0 ? N : 1];
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    A[nu] = M::v4(P, kMsA2 + nu, c);
    B[nu] = M::v4(P, kMsB2 + nu, c);
    Q0[nu] = ld_state4(P.psi2[0], nu * S + c);
    Q1[nu] = ld_state4(P.psi2[1], nu * S + c);
    Q2[nu] = ld_state4(P.psi2[2], nu * S + c);
  }
  const Win12 w = win12(svx[ty], tx);
  float4 Dx, Dy;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float d = 0.f;
#pragma unroll
    for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m - 1] - w.v[4 + e - m], d);
    el(Dx, e) = d;
  }
  {
    float4 col[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) col[m] = *reinterpret_cast<const float4 *>(&svy[ty + m][4 * tx + 4]);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el(col[4 + m - 1], e) - el(col[4 - m], e), d);
      el(Dy, e) = d;
    }
  }
  float4 S0, S1, S2;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    el(S0, e) = el(Dx, e) * el(k2, e);
    el(S1, e) = el(Dy, e) * el(k2, e);
    el(S2, e) = el(Dz, e) * el(k2, e);
  }
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    float4 n0, n1, n2;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el(n0, e) = fmaf(el(B[nu], e), el(Q0[nu], e), el(A[nu], e) * el(Dx, e));
      el(n1, e) = fmaf(el(B[nu], e), el(Q1[nu], e), el(A[nu], e) * el(Dy, e));
      el(n2, e) = fmaf(el(B[nu], e), el(Q2[nu], e), el(A[nu], e) * el(Dz, e));
      el(S0, e) += fmaf(P.w_new, el(n0, e), P.w_old * el(Q0[nu], e));
      el(S1, e) += fmaf(P.w_new, el(n1, e), P.w_old * el(Q1[nu], e));
      el(S2, e) += fmaf(P.w_new, el(n2, e), P.w_old * el(Q2[nu], e));
    }
    st_state4(P.psi2[0], nu * S + c, n0);
    st_state4(P.psi2[1], nu * S + c, n1);
    st_state4(P.psi2[2], nu * S + c, n2);
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float upd = P.dt * el(K, e) * (el(S0, e) + el(S1, e) + el(S2, e));
    if (P.nl) upd = qdiv(upd, fmaf(el(ch, e), el(p, e), 1.f));
    el(p, e) -= upd;
  }
  st_state4(P.p, c, p);
}

template <int N, typename M>
__global__ void __launch_bounds__(256, 2) vel3d_kernel(const StepParams P) {
  constexpr int PW = kTX + 8, PH = kTY3 + 7;  // p plane tile: x0-4.., y0-3..
  constexpr int RW = kTX + 4, RH = kTY3 + 1;  // rho plane tile: x0.., y0..
  __shared__ __align__(16) float sp[PH][PW];
  __shared__ __align__(16) float sr[RH][RW];
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY3, z0 = blockIdx.z * kTZ;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int i0 = x0 + 4 * tx;
  const bool fast_xy = interior_xy(P, x0, y0) && P.g11h == 0.f;  // cross taps: general path
  const int zend = min(z0 + kTZ, P.nz);
#pragma unroll 1
  for (int k = z0; k < zend; ++k) {
    __syncthreads();
    for (int t = tid; t < PH * (PW / 4); t += 256) {
      const int r = t / (PW / 4), c4 = t % (PW / 4);
      *reinterpret_cast<float4 *>(&sp[r][4 * c4]) = load_chunk(P, P.p, x0 - 4 + 4 * c4, y0 - 3 + r, k);
    }
    for (int t = tid; t < RH * RW; t += 256) {
      const int r = t / RW, cc = t % RW;
      const int gx = rho_coord(x0 + cc, P.nx, P.periodic[0]);
      const int gy = rho_coord(y0 + r, P.ny, P.periodic[1]);
      sr[r][cc] = M::v1(P, kMsRho, (long long)k * P.plane + (long long)gy * P.pitch + gx);
    }
    __syncthreads();
#pragma unroll 1
    for (int rr = 0; rr < kTY3 / kBY3; ++rr) {
    const int ly = ty + rr * kBY3, j = y0 + ly;
    if (i0 >= P.nx || j >= P.ny) continue;
    if (fast_xy && interior_z(P, k)) {
      vel3d_fast<N, M>(P, sp, sr, i0, j, k, tx, ly);
      continue;
    }
    const long long c = (long long)k * P.plane + (long long)j * P.pitch + i0;
    const int sy = ly + 3;
    const Win12 w = win12(sp[sy], tx);
    float4 Dx, Dy, Dz;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m] - w.v[4 + e - m + 1], d);
      el(Dx, e) = d;
    }
    {
      float4 col[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) col[m] = *reinterpret_cast<const float4 *>(&sp[sy - 3 + m][4 * tx + 4]);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float d = 0.f;
#pragma unroll
        for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el(col[3 + m], e) - el(col[4 - m], e), d);
        el(Dy, e) = d;
      }
    }
    float4 pz1;
    {
      // d/dz at faces k+1/2: sum_m g_m (p[k+m] - p[k-m+1]) on the cell's own column
      float4 zc[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) zc[m] = load_chunk(P, P.p, i0, j, k - 3 + m);
      pz1 = zc[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float d = 0.f;
#pragma unroll
        for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el(zc[3 + m], e) - el(zc[4 - m], e), d);
        el(Dz, e) = d;
      }
    }
    if (P.g11h != 0.f) vel3_cross(P, sp, sy, tx, i0, j, k, Dx, Dy, Dz);
    float4 bx, by, bz;
    {
      const int lx = 4 * tx;
      const float4 r0 = *reinterpret_cast<const float4 *>(&sr[ly][lx]);
      const float r4 = sr[ly][lx + 4];
      const float4 ru = *reinterpret_cast<const float4 *>(&sr[ly + 1][lx]);
      const int kz = rho_coord(k + 1, P.nz, P.periodic[2]);
      float4 rz;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int x = min(i0 + e, P.nx - 1);
        el(rz, e) = M::v1(P, kMsRho, (long long)kz * P.plane + (long long)j * P.pitch + x);
      }
      bx = make_float4(qdiv(P.two_dt, r0.x + r0.y), qdiv(P.two_dt, r0.y + r0.z), qdiv(P.two_dt, r0.z + r0.w),
                       qdiv(P.two_dt, r0.w + r4));
      by = make_float4(qdiv(P.two_dt, r0.x + ru.x), qdiv(P.two_dt, r0.y + ru.y), qdiv(P.two_dt, r0.z + ru.z),
                       qdiv(P.two_dt, r0.w + ru.w));
      bz = make_float4(qdiv(P.two_dt, r0.x + rz.x), qdiv(P.two_dt, r0.y + rz.y), qdiv(P.two_dt, r0.z + rz.z),
                       qdiv(P.two_dt, r0.w + rz.w));
    }
    const float4 k1 = M::v4(P, kMsIk1, c);
    float4 fx = make_float4(1.f, 1.f, 1.f, 1.f), fy = fx, fz = fx;
    if (P.nl_vel) mom_factors3<M>(P, sp, ly + 3, tx, i0, j, k, pz1, fx, fy, fz);
    const float4 bb[3] = {bx, by, bz}, ff[3] = {fx, fy, fz};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float4 S = q == 0 ? stretch4<0, 1, N, M>(P, P.psi1[0], Dx, k1, c, i0, j, k)
                     : q == 1 ? stretch4<1, 1, N, M>(P, P.psi1[1], Dy, k1, c, i0, j, k)
                              : stretch4<2, 1, N, M>(P, P.psi1[2], Dz, k1, c, i0, j, k);
      float4 v = ld_state4(P.v[q], c);
      if (P.nl_vel) {
#pragma unroll
        for (int e = 0; e < 4; ++e) el(v, e) = vel_upd(el(v, e), el(bb[q], e), el(S, e), el(ff[q], e));
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) el(v, e) = vel_upd(el(v, e), el(bb[q], e), el(S, e));
      }
      st_state4(P.v[q], c, mask_pad(v, i0, P.nx));
    }
    }
  }
}

template <int N, typename M>
__global__ void __launch_bounds__(256, 2) prs3d_kernel(const StepParams P) {
  constexpr int W = kTX + 8;
  constexpr int HX = kTY3;      // v_x rows y0 .. y0+TY-1
  constexpr int HY = kTY3 + 7;  // v_y rows y0-4 .. y0+TY+2
  __shared__ __align__(16) float svx[HX][W];
  __shared__ __align__(16) float svy[HY][W];
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY3, z0 = blockIdx.z * kTZ;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int i0 = x0 + 4 * tx;
  const bool fast_xy = interior_xy(P, x0, y0) && P.g11h == 0.f;  // cross taps: general path
  const int zend = min(z0 + kTZ, P.nz);
#pragma unroll 1
  for (int k = z0; k < zend; ++k) {
    __syncthreads();
    for (int t = tid; t < HX * (W / 4); t += 256) {
      const int r = t / (W / 4), c4 = t % (W / 4);
      *reinterpret_cast<float4 *>(&svx[r][4 * c4]) = load_chunk(P, P.v[0], x0 - 4 + 4 * c4, y0 + r, k);
    }
    for (int t = tid; t < HY * (W / 4); t += 256) {
      const int r = t / (W / 4), c4 = t % (W / 4);
      *reinterpret_cast<float4 *>(&svy[r][4 * c4]) = load_chunk(P, P.v[1], x0 - 4 + 4 * c4, y0 - 4 + r, k);
    }
    __syncthreads();
#pragma unroll 1
    for (int rr = 0; rr < kTY3 / kBY3; ++rr) {
    const int ly = ty + rr * kBY3, j = y0 + ly;
    if (i0 >= P.nx || j >= P.ny) continue;
    if (fast_xy && interior_z(P, k)) {
      prs3d_fast<N, M>(P, svx, svy, i0, j, k, tx, ly);
      continue;
    }
    const long long c = (long long)k * P.plane + (long long)j * P.pitch + i0;
    const Win12 w = win12(svx[ly], tx);
    float4 Dx, Dy, Dz;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m - 1] - w.v[4 + e - m], d);
      el(Dx, e) = d;
    }
    {
      float4 col[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) col[m] = *reinterpret_cast<const float4 *>(&svy[ly + m][4 * tx + 4]);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float d = 0.f;
#pragma unroll
        for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el(col[4 + m - 1], e) - el(col[4 - m], e), d);
        el(Dy, e) = d;
      }
    }
    {
      // d/dz v_z at centres: sum_m g_m (vz[k+m-1] - vz[k-m]); zc[4] is plane k
      float4 zc[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) zc[m] = load_chunk(P, P.v[2], i0, j, k - 4 + m);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float d = 0.f;
#pragma unroll
        for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el(zc[4 + m - 1], e) - el(zc[4 - m], e), d);
        el(Dz, e) = d;
      }
    }
    if (P.g11h != 0.f) prs3_cross(P, i0, j, k, Dx, Dy, Dz);
    const float4 k2 = M::v4(P, kMsIk2, c);
    const float4 Sx = stretch4<0, 2, N, M>(P, P.psi2[0], Dx, k2, c, i0, j, k);
    const float4 Sy = stretch4<1, 2, N, M>(P, P.psi2[1], Dy, k2, c, i0, j, k);
    const float4 Sz = stretch4<2, 2, N, M>(P, P.psi2[2], Dz, k2, c, i0, j, k);
    const float4 K = M::v4(P, kMsK, c);
    float4 p = ld_state4(P.p, c);
    float4 upd = make_float4(P.dt * K.x * (Sx.x + Sy.x + Sz.x), P.dt * K.y * (Sx.y + Sy.y + Sz.y),
                             P.dt * K.z * (Sx.z + Sy.z + Sz.z), P.dt * K.w * (Sx.w + Sy.w + Sz.w));
    if (P.nl) {
      const float4 ch = M::v4(P, kMsChi, c);
      upd.x = qdiv(upd.x, fmaf(ch.x, p.x, 1.f)); upd.y = qdiv(upd.y, fmaf(ch.y, p.y, 1.f));
      upd.z = qdiv(upd.z, fmaf(ch.z, p.z, 1.f)); upd.w = qdiv(upd.w, fmaf(ch.w, p.w, 1.f));
    }
    p.x -= upd.x; p.y -= upd.y; p.z -= upd.z; p.w -= upd.w;
    st_state4(P.p, c, mask_pad(p, i0, P.nx));
    }
  }
}

// The mechanism counts this compilation instantiates: 0..4, or 5..8 when
// built with FW2_WIDE_RELAX (the second object of this file).
#ifdef FW2_WIDE_RELAX
constexpr int kNLo = 5, kNHi = kMaxRelax;
#else
constexpr int kNLo = 0, kNHi = 4;
#endif

template <int N, typename M>
cudaError_t vel3d_at(const StepParams &P, dim3 g, dim3 b, cudaStream_t s) {
  if constexpr (N > kNHi) {
    return cudaErrorInvalidValue;
  } else {
    if (P.n_relax != N) return vel3d_at<N + 1, M>(P, g, b, s);
    if constexpr (kIndexed3<M> && N > kTabSlots) return cudaErrorInvalidValue;  // tables hold kTabSlots
    else vel3d_kernel<N, M><<<g, b, 0, s>>>(P);
    return cudaGetLastError();
  }
}

template <int N, typename M>
cudaError_t prs3d_at(const StepParams &P, dim3 g, dim3 b, cudaStream_t s) {
  if constexpr (N > kNHi) {
    return cudaErrorInvalidValue;
  } else {
    if (P.n_relax != N) return prs3d_at<N + 1, M>(P, g, b, s);
    if constexpr (kIndexed3<M> && N > kTabSlots) return cudaErrorInvalidValue;  // tables hold kTabSlots
    else prs3d_kernel<N, M><<<g, b, 0, s>>>(P);
    return cudaGetLastError();
  }
}

}  // namespace

#ifdef FW2_WIDE_RELAX
cudaError_t launch_vel3d_wide(const StepParams &P, int map_kind, cudaStream_t s) {
#else
cudaError_t launch_vel3d(const StepParams &P, int map_kind, cudaStream_t s) {
  if (P.n_relax > kNHi) return launch_vel3d_wide(P, map_kind, s);
#endif
  dim3 g((P.nx + kTX - 1) / kTX, (P.ny + kTY3 - 1) / kTY3, (P.nz + kTZ - 1) / kTZ), b(32, kBY3);
  switch (map_kind) {
    case 0: return vel3d_at<kNLo, Dense3<float>>(P, g, b, s);
    case 1: return vel3d_at<kNLo, Dense3<__nv_bfloat16>>(P, g, b, s);
    case 2: return vel3d_at<kNLo, Idx3<unsigned char>>(P, g, b, s);
    case 3: return vel3d_at<kNLo, Idx3<unsigned short>>(P, g, b, s);
    case 4: return vel3d_at<kNLo, Dense3<__half>>(P, g, b, s);
    default: return cudaErrorInvalidValue;
  }
}

#ifdef FW2_WIDE_RELAX
cudaError_t launch_prs3d_wide(const StepParams &P, int map_kind, cudaStream_t s) {
#else
cudaError_t launch_prs3d(const StepParams &P, int map_kind, cudaStream_t s) {
  if (P.n_relax > kNHi) return launch_prs3d_wide(P, map_kind, s);
#endif
  dim3 g((P.nx + kTX - 1) / kTX, (P.ny + kTY3 - 1) / kTY3, (P.nz + kTZ - 1) / kTZ), b(32, kBY3);
  switch (map_kind) {
    case 0: return prs3d_at<kNLo, Dense3<float>>(P, g, b, s);
    case 1: return prs3d_at<kNLo, Dense3<__nv_bfloat16>>(P, g, b, s);
    case 2: return prs3d_at<kNLo, Idx3<unsigned char>>(P, g, b, s);
    case 3: return prs3d_at<kNLo, Idx3<unsigned short>>(P, g, b, s);
    case 4: return prs3d_at<kNLo, Dense3<__half>>(P, g, b, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fw2
