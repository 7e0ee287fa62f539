// Helpers shared by the 2D and 3D step kernels: the outer boundary rule of
// the operand loads, padding masks, the face-density coordinate rule, the
// half-step quotient, the literal system's momentum factor and the velocity
// update.
#pragma once
#include "fw2_internal.cuh"

namespace fw2 {

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
