// 3D fused velocity and pressure half steps (sm_103a).
//
// Same arithmetic as the 2D kernels (Sec. 3.1 updates, Eqs. relaxation4,
// relaxation_psi, general6) with the third axis.  Each block owns a 128 x 8
// tile of an xy plane (256 threads, two rows each) and marches through kTZ
// planes along z; the xy stencil
// operand of the current plane is staged in shared memory with its halo, the
// z taps of each cell's own column are read through L2.
#include "coef.cuh"

namespace fw2 {

namespace {

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
template <typename MT>
__device__ __forceinline__ void mom_factors3(const StepParams &P, const float (*sp)[kTX + 8], int sy, int tx, int i0,
                                             int j, int k, const float4 &pz1, float4 &fx, float4 &fy, float4 &fz) {
  const MT *Km = static_cast<const MT *>(P.K);
  const Win12 w = win12(sp[sy], tx), up = win12(sp[sy + 1], tx);
  const int jn = rho_coord(j + 1, P.ny, P.periodic[1]), kn = rho_coord(k + 1, P.nz, P.periodic[2]);
  const long long row = (long long)k * P.plane + (long long)j * P.pitch;
  const long long rowy = (long long)k * P.plane + (long long)jn * P.pitch;
  const long long rowz = (long long)kn * P.plane + (long long)j * P.pitch;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int x = min(i0 + e, P.nx - 1);
    const int xn = rho_coord(min(i0 + e + 1, P.nx), P.nx, P.periodic[0]);
    const float sK = P.ms[kMsK];
    const float Kc = ldmap(Km, row + x, sK);
    el(fx, e) = mom_factor(Kc, ldmap(Km, row + xn, sK), w.v[4 + e], w.v[5 + e]);
    el(fy, e) = mom_factor(Kc, ldmap(Km, rowy + x, sK), w.v[4 + e], up.v[4 + e]);
    el(fz, e) = mom_factor(Kc, ldmap(Km, rowz + x, sK), w.v[4 + e], el(pz1, e));
  }
}

// Interior plane of the velocity half step: z taps first (L2), then every
// streaming load of the plane row before any store.
template <int N, typename MT>
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
  const MT *ik1 = static_cast<const MT *>(P.ik1);
  const MT *a1 = static_cast<const MT *>(P.a1);
  const MT *b1 = static_cast<const MT *>(P.b1);
  const MT *rho = static_cast<const MT *>(P.rho);
  float4 v0 = ld_state4(P.v[0], c), v1 = ld_state4(P.v[1], c), v2 = ld_state4(P.v[2], c);
  const float4 k1 = ldmap4(ik1, c, P.ms[kMsIk1]);
  const float4 rz = ldmap4(rho, c + P.plane, P.ms[kMsRho]);
  float4 A[N > 0 ? N : 1], B[N > 0 ? N : 1], Q0[N > 0 ? N : 1], Q1[N > 0 ? N : 1], Q2[N > 0 ? N : 1];
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    A[nu] = ldmap4(a1, nu * S + c, P.ms[kMsA1 + nu]);
    B[nu] = ldb4(b1, nu * S + c, P.ms[kMsB1 + nu]);
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
    mom_factors3<MT>(P, sp, sy, tx, i0, j, k, pz1, fx, fy, fz);
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
template <int N, typename MT>
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
  const MT *ik2 = static_cast<const MT *>(P.ik2);
  const MT *a2 = static_cast<const MT *>(P.a2);
  const MT *b2 = static_cast<const MT *>(P.b2);
  const MT *Km = static_cast<const MT *>(P.K);
  const MT *chim = static_cast<const MT *>(P.chi);
  float4 p = ld_state4(P.p, c);
  const float4 k2 = ldmap4(ik2, c, P.ms[kMsIk2]);
  const float4 K = ldmap4(Km, c, P.ms[kMsK]);
  float4 ch = make_float4(0.f, 0.f, 0.f, 0.f);
  if (P.nl) ch = ldmap4(chim, c, P.ms[kMsChi]);
  float4 A[N > 0 ? N : 1], B[N > 0 ? N : 1], Q0[N > 0 ? N : 1], Q1[N > 0 ? N : 1], Q2[N > 0 ? N : 1];
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    A[nu] = ldmap4(a2, nu * S + c, P.ms[kMsA2 + nu]);
    B[nu] = ldb4(b2, nu * S + c, P.ms[kMsB2 + nu]);
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

template <int N, typename MT>
__global__ void __launch_bounds__(256, 2) vel3d_kernel(const StepParams P) {
  constexpr int PW = kTX + 8, PH = kTY3 + 7;  // p plane tile: x0-4.., y0-3..
  constexpr int RW = kTX + 4, RH = kTY3 + 1;  // rho plane tile: x0.., y0..
  __shared__ __align__(16) float sp[PH][PW];
  __shared__ __align__(16) float sr[RH][RW];
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY3, z0 = blockIdx.z * kTZ;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const MT *rho = static_cast<const MT *>(P.rho);
  const MT *ik1 = static_cast<const MT *>(P.ik1);
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
      sr[r][cc] = ldmap(rho, (long long)k * P.plane + (long long)gy * P.pitch + gx, P.ms[kMsRho]);
    }
    __syncthreads();
#pragma unroll 1
    for (int rr = 0; rr < kTY3 / kBY3; ++rr) {
    const int ly = ty + rr * kBY3, j = y0 + ly;
    if (i0 >= P.nx || j >= P.ny) continue;
    if (fast_xy && interior_z(P, k)) {
      vel3d_fast<N, MT>(P, sp, sr, i0, j, k, tx, ly);
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
        el(rz, e) = ldmap(rho, (long long)kz * P.plane + (long long)j * P.pitch + x, P.ms[kMsRho]);
      }
      bx = make_float4(qdiv(P.two_dt, r0.x + r0.y), qdiv(P.two_dt, r0.y + r0.z), qdiv(P.two_dt, r0.z + r0.w),
                       qdiv(P.two_dt, r0.w + r4));
      by = make_float4(qdiv(P.two_dt, r0.x + ru.x), qdiv(P.two_dt, r0.y + ru.y), qdiv(P.two_dt, r0.z + ru.z),
                       qdiv(P.two_dt, r0.w + ru.w));
      bz = make_float4(qdiv(P.two_dt, r0.x + rz.x), qdiv(P.two_dt, r0.y + rz.y), qdiv(P.two_dt, r0.z + rz.z),
                       qdiv(P.two_dt, r0.w + rz.w));
    }
    const float4 k1 = ldmap4(ik1, c, P.ms[kMsIk1]);
    float4 fx = make_float4(1.f, 1.f, 1.f, 1.f), fy = fx, fz = fx;
    if (P.nl_vel) mom_factors3<MT>(P, sp, ly + 3, tx, i0, j, k, pz1, fx, fy, fz);
    const float4 bb[3] = {bx, by, bz}, ff[3] = {fx, fy, fz};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float4 S = q == 0 ? stretch4<0, 1, N, MT>(P, P.psi1[0], Dx, k1, c, i0, j, k)
                     : q == 1 ? stretch4<1, 1, N, MT>(P, P.psi1[1], Dy, k1, c, i0, j, k)
                              : stretch4<2, 1, N, MT>(P, P.psi1[2], Dz, k1, c, i0, j, k);
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

template <int N, typename MT>
__global__ void __launch_bounds__(256, 2) prs3d_kernel(const StepParams P) {
  constexpr int W = kTX + 8;
  constexpr int HX = kTY3;      // v_x rows y0 .. y0+TY-1
  constexpr int HY = kTY3 + 7;  // v_y rows y0-4 .. y0+TY+2
  __shared__ __align__(16) float svx[HX][W];
  __shared__ __align__(16) float svy[HY][W];
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY3, z0 = blockIdx.z * kTZ;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const MT *ik2 = static_cast<const MT *>(P.ik2);
  const MT *Km = static_cast<const MT *>(P.K);
  const MT *chim = static_cast<const MT *>(P.chi);
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
      prs3d_fast<N, MT>(P, svx, svy, i0, j, k, tx, ly);
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
    const float4 k2 = ldmap4(ik2, c, P.ms[kMsIk2]);
    const float4 Sx = stretch4<0, 2, N, MT>(P, P.psi2[0], Dx, k2, c, i0, j, k);
    const float4 Sy = stretch4<1, 2, N, MT>(P, P.psi2[1], Dy, k2, c, i0, j, k);
    const float4 Sz = stretch4<2, 2, N, MT>(P, P.psi2[2], Dz, k2, c, i0, j, k);
    const float4 K = ldmap4(Km, c, P.ms[kMsK]);
    float4 p = ld_state4(P.p, c);
    float4 upd = make_float4(P.dt * K.x * (Sx.x + Sy.x + Sz.x), P.dt * K.y * (Sx.y + Sy.y + Sz.y),
                             P.dt * K.z * (Sx.z + Sy.z + Sz.z), P.dt * K.w * (Sx.w + Sy.w + Sz.w));
    if (P.nl) {
      const float4 ch = ldmap4(chim, c, P.ms[kMsChi]);
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

template <int N, typename MT>
cudaError_t vel3d_at(const StepParams &P, dim3 g, dim3 b, cudaStream_t s) {
  if constexpr (N > kNHi) {
    return cudaErrorInvalidValue;
  } else {
    if (P.n_relax != N) return vel3d_at<N + 1, MT>(P, g, b, s);
    vel3d_kernel<N, MT><<<g, b, 0, s>>>(P);
    return cudaGetLastError();
  }
}

template <int N, typename MT>
cudaError_t prs3d_at(const StepParams &P, dim3 g, dim3 b, cudaStream_t s) {
  if constexpr (N > kNHi) {
    return cudaErrorInvalidValue;
  } else {
    if (P.n_relax != N) return prs3d_at<N + 1, MT>(P, g, b, s);
    prs3d_kernel<N, MT><<<g, b, 0, s>>>(P);
    return cudaGetLastError();
  }
}

}  // namespace

#ifdef FW2_WIDE_RELAX
cudaError_t launch_vel3d_wide(const StepParams &P, int map_kind, cudaStream_t s) {
#else
cudaError_t launch_vel3d(const StepParams &P, int map_kind, cudaStream_t s) {  // map kind 0, 1 or 4
  if (P.n_relax > kNHi) return launch_vel3d_wide(P, map_kind, s);
#endif
  dim3 g((P.nx + kTX - 1) / kTX, (P.ny + kTY3 - 1) / kTY3, (P.nz + kTZ - 1) / kTZ), b(32, kBY3);
  if (map_kind == 4) return vel3d_at<kNLo, __half>(P, g, b, s);
  return map_kind == 1 ? vel3d_at<kNLo, __nv_bfloat16>(P, g, b, s) : vel3d_at<kNLo, float>(P, g, b, s);
}

#ifdef FW2_WIDE_RELAX
cudaError_t launch_prs3d_wide(const StepParams &P, int map_kind, cudaStream_t s) {
#else
cudaError_t launch_prs3d(const StepParams &P, int map_kind, cudaStream_t s) {
  if (P.n_relax > kNHi) return launch_prs3d_wide(P, map_kind, s);
#endif
  dim3 g((P.nx + kTX - 1) / kTX, (P.ny + kTY3 - 1) / kTY3, (P.nz + kTZ - 1) / kTZ), b(32, kBY3);
  if (map_kind == 4) return prs3d_at<kNLo, __half>(P, g, b, s);
  return map_kind == 1 ? prs3d_at<kNLo, __nv_bfloat16>(P, g, b, s) : prs3d_at<kNLo, float>(P, g, b, s);
}

}  // namespace fw2
