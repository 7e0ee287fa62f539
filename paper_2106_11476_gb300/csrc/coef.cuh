// Per-axis relaxation coefficient fetch and memory-variable update, shared by
// the 2D and 3D step kernels.
#pragma once
#include "fw2_internal.cuh"

namespace fw2 {

// a, b of mechanism nu for the derivative along axis Q at the four cells
// i0..i0+3 of row (j, k): from the boundary strip of axis Q when the cell
// lies inside the C-PML region of that axis (Sec. 3.3: each axis' parameters
// depend on the distance along that axis only), else from the interior maps.
// OP = 1: nabla_1 (faces), OP = 2: nabla_2 (centres).
template <int Q, int OP, typename MT>
__device__ __forceinline__ void coef4(const StepParams &P, int nu, long long c, int i0, int j,
                                      int k, float4 &a, float4 &b) {
  const MT *ia = static_cast<const MT *>(OP == 1 ? P.a1 : P.a2);
  const MT *ib = static_cast<const MT *>(OP == 1 ? P.b1 : P.b2);
  const long long iso = (long long)nu * P.npts_alloc + c;
  const MT *sa = static_cast<const MT *>(OP == 1 ? P.sa1[Q] : P.sa2[Q]);
  const MT *sb = static_cast<const MT *>(OP == 1 ? P.sb1[Q] : P.sb2[Q]);
  const float s_a = P.ms[(OP == 1 ? kMsA1 : kMsA2) + nu], s_b = P.ms[(OP == 1 ? kMsB1 : kMsB2) + nu];
  const int L = P.L[Q];
  if (Q == 0) {
    const bool any = L > 0 && (i0 < L || i0 + 3 >= P.nx - L);
    if (!any) {
      a = ldmap4(ia, iso, s_a);
      b = ldb4(ib, iso, s_b);
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
          av = ldmap(ia, iso + e, s_a);
          bv = ldb(ib, iso + e, s_b);
        }
      }
      el(a, e) = av;
      el(b, e) = bv;
    }
  } else {
    const int sc = Q == 1 ? strip_coord(j, P.ny, L) : strip_coord(k, P.nz, L);
    if (sc < 0) {
      a = ldmap4(ia, iso, s_a);
      b = ldb4(ib, iso, s_b);
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
template <int Q, int OP, int N, typename MT>
__device__ __forceinline__ float4 stretch4(const StepParams &P, float *psi, float4 D, float4 ik,
                                           long long c, int i0, int j, int k) {
  float4 S = make_float4(D.x * ik.x, D.y * ik.y, D.z * ik.z, D.w * ik.w);
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    float4 a, b;
    coef4<Q, OP, MT>(P, nu, c, i0, j, k, a, b);
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

// zero the lanes of a 4-cell group that fall in the row padding (x >= nx)
__device__ __forceinline__ float4 mask_pad(float4 v, int i0, int nx) {
  if (i0 + 3 >= nx) {
    if (i0 + 1 >= nx) v.y = 0.f;
    if (i0 + 2 >= nx) v.z = 0.f;
    if (i0 + 3 >= nx) v.w = 0.f;
    if (i0 >= nx) v.x = 0.f;
  }
  return v;
}

// Wrap or drop an out-of-range coordinate: returns -1 when the value is zero
// (zero-outside boundary), the wrapped coordinate when periodic.
__device__ __forceinline__ int bc_coord(int x, int n, int periodic) {
  if (x >= 0 && x < n) return x;
  if (!periodic) return -1;
  x %= n;
  return x < 0 ? x + n : x;
}

// Four consecutive values of a cell-indexed float field starting at the
// 4-aligned column gx of row (gy, gz), following the outer boundary rule.
__device__ __forceinline__ float4 load_chunk(const StepParams &P, const float *f, int gx, int gy,
                                             int gz) {
  const int y = bc_coord(gy, P.ny, P.periodic[1]);
  const int z = bc_coord(gz, P.nz, P.periodic[2]);
  if (y < 0 || z < 0) return make_float4(0.f, 0.f, 0.f, 0.f);
  const long long rowoff = (long long)z * P.plane + (long long)y * P.pitch;
  if (gx >= 0 && gx + 3 < P.nx) return __ldg(reinterpret_cast<const float4 *>(f + rowoff + gx));
  float4 v;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int x = bc_coord(gx + e, P.nx, P.periodic[0]);
    el(v, e) = x < 0 ? 0.f : __ldg(f + rowoff + x);
  }
  return v;
}

// Quotients of the half steps (the face coefficient 2 dt / (rho_a + rho_b),
// the momentum factor, the nonlinear denominator 1 + chi p): x times the
// approximate reciprocal of y, within 2 ulp of the rounded quotient, two
// instructions where the rounded division takes a dozen and a slow-path
// check.  The product is rounded on its own (__fmul_rn is never contracted
// into a neighbouring add), so every kernel of a half step computes the same
// value whatever its surrounding code: all paths agree bitwise.
__device__ __forceinline__ float qdiv(float x, float y) { return __fmul_rn(x, __fdividef(1.f, y)); }

// Momentum factor of the literal nonlinear system (Eq. general5,
// rho_0 (1 + kappa_0 p)) at the face between cells a and b: 1 + kappa0_face
// p_face, both the mean of the two cells (kappa0 = 1 / K).
__device__ __forceinline__ float mom_factor(float Ka, float Kb, float pa, float pb) {
  return fmaf(0.5f * (qdiv(1.f, Ka) + qdiv(1.f, Kb)), 0.5f * (pa + pb), 1.f);
}

// The velocity update v - b S (Eq. general5, b = 2 dt / (rho_a + rho_b)),
// and with the literal system's momentum factor f, v - b (S / f).  One fused
// multiply-add each, written out so that every kernel of the half step
// rounds alike whatever the compiler's contraction choices.
__device__ __forceinline__ float vel_upd(float v, float b, float S) { return fmaf(-b, S, v); }
__device__ __forceinline__ float vel_upd(float v, float b, float S, float f) { return fmaf(-b, qdiv(S, f), v); }

// Density used for the face average: cells beyond the last one along an
// axis take the last cell's value (zero-outside boundary) or wrap (periodic).
__device__ __forceinline__ int rho_coord(int x, int n, int periodic) {
  if (x < n) return x;
  return periodic ? x % n : n - 1;
}

}  // namespace fw2
