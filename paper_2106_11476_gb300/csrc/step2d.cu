// 2D fused velocity and pressure half steps (sm_103a).
//
// Velocity half step (Sec. 3.1 u, v updates; Eqs. relaxation4 and
// relaxation_psi for nabla_1):
//   D_q      = staggered 8th-order derivative of p^n at the face of axis q
//   psi1_q  <- b psi1_q + a D_q                      (per mechanism)
//   v_q     <- v_q - dt / rho_face * (D_q / kappa1 + sum memory terms)
// Pressure half step (Sec. 3.1 p update; Eq. general6 for the nonlinear
// factor):
//   D_q      = staggered derivative of v_q at the cell centre
//   psi2_q  <- b psi2_q + a D_q
//   p       <- p - dt K sum_q (D_q / kappa2 + memory) / (1 + chi p)
//
// Each block owns a 128 x 16 tile; 256 threads, 4 consecutive x cells per
// thread (128-bit loads and stores of every streamed array), two rows each.
// The stencil operand (p, or v_x / v_y) is staged in shared memory with its
// halo; every other array is read once and written once.
#include "coef.cuh"

namespace fw2 {

namespace {

constexpr int kRows = kTY / kBY;  // rows per thread

// 12 consecutive shared-memory values starting at column 4*tx of a row
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


// x and y derivatives of v_x, v_y at the four centres of a thread (pressure)
__device__ __forceinline__ void prs_derivs(const StepParams &P, const float (*svx)[kTX + 8],
                                           const float (*svy)[kTX + 8], int ly, int tx, float4 &Dx, float4 &Dy) {
  const Win12 w = win12(svx[ly + 1], tx);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float d = 0.f;
#pragma unroll
    for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m - 1] - w.v[4 + e - m], d);
    el(Dx, e) = d;
  }
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
  if (P.g11h != 0.f) {
    const Win12 up = win12(svx[ly + 2], tx), dn = win12(svx[ly], tx);
    const Win12 y0w = win12(svy[ly + 4], tx), y1w = win12(svy[ly + 3], tx);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el(Dx, e) += P.g11h * ((up.v[4 + e] - up.v[3 + e]) + (dn.v[4 + e] - dn.v[3 + e]));
      el(Dy, e) += P.g11h * ((y0w.v[5 + e] - y1w.v[5 + e]) + (y0w.v[3 + e] - y1w.v[3 + e]));
    }
  }
}

// A tile whose cells, stencil halo and face neighbours all lie inside the
// grid and outside every C-PML strip: every cell uses the interior maps for
// both axes, and no boundary rule applies.
__device__ __forceinline__ bool interior_tile(const StepParams &P, int x0, int y0) {
  const int Lx = P.L[0] > 4 ? P.L[0] : 4, Ly = P.L[1] > 4 ? P.L[1] : 4;
  return x0 >= Lx && x0 + kTX + Lx <= P.nx && y0 >= Ly && y0 + kTY + Ly <= P.ny;
}

// x and y derivatives of the staged operand at the four faces of a thread
// (velocity) -- shared by both paths
__device__ __forceinline__ void vel_derivs(const StepParams &P, const float (*sp)[kTX + 8], int sy, int tx,
                                           float4 &Dx, float4 &Dy) {
  const Win12 w = win12(sp[sy], tx);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float d = 0.f;
#pragma unroll
    for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m] - w.v[4 + e - m + 1], d);
    el(Dx, e) = d;
  }
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
  if (P.g11h != 0.f) {
    const Win12 up = win12(sp[sy + 1], tx), dn = win12(sp[sy - 1], tx);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el(Dx, e) += P.g11h * ((up.v[5 + e] - up.v[4 + e]) + (dn.v[5 + e] - dn.v[4 + e]));
      el(Dy, e) += P.g11h * ((up.v[5 + e] - w.v[5 + e]) + (up.v[3 + e] - w.v[3 + e]));
    }
  }
}

// Interior rows of the velocity half step.  Every global load of a row (both
// velocity components, 1/kappa1, the shared interior a, b and the memory
// variables of both axes) is issued before any store, so a row pays one
// memory latency instead of one per mechanism.
template <int N, typename MT>
__device__ __forceinline__ void vel2d_fast_rows(const StepParams &P, const float (*sp)[kTX + 8],
                                                const float (*sr)[kTX + 4], int x0, int y0, int tx, int ty) {
  const MT *ik1 = static_cast<const MT *>(P.ik1);
  const MT *a1 = static_cast<const MT *>(P.a1);
  const MT *b1 = static_cast<const MT *>(P.b1);
  float *psx = P.psi1[0], *psy = P.psi1[1];
  const long long S = P.npts_alloc;
  const int i0 = x0 + 4 * tx;
#pragma unroll 1
  for (int rr = 0; rr < kRows; ++rr) {
    const int ly = ty + rr * kBY;
    const int j = y0 + ly;
    const long long c = (long long)j * P.pitch + i0;
    float4 vx = ld_state4(P.v[0], c), vy = ld_state4(P.v[1], c);
    const float4 k1 = ldmap4(ik1, c);
    float4 A[N > 0 ? N : 1], B[N > 0 ? N : 1], Px[N > 0 ? N : 1], Py[N > 0 ? N : 1];
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      A[nu] = ldmap4(a1, nu * S + c);
      B[nu] = ldmap4(b1, nu * S + c);
      Px[nu] = ld_state4(psx, nu * S + c);
      Py[nu] = ld_state4(psy, nu * S + c);
    }
    float4 Dx, Dy;
    vel_derivs(P, sp, ly + 3, tx, Dx, Dy);
    const int lx = 4 * tx;
    const float4 r0 = *reinterpret_cast<const float4 *>(&sr[ly][lx]);
    const float r4 = sr[ly][lx + 4];
    const float4 ru = *reinterpret_cast<const float4 *>(&sr[ly + 1][lx]);
    float4 Sx = make_float4(Dx.x * k1.x, Dx.y * k1.y, Dx.z * k1.z, Dx.w * k1.w);
    float4 Sy = make_float4(Dy.x * k1.x, Dy.y * k1.y, Dy.z * k1.z, Dy.w * k1.w);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      float4 nx_, ny_;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        el(nx_, e) = fmaf(el(B[nu], e), el(Px[nu], e), el(A[nu], e) * el(Dx, e));
        el(ny_, e) = fmaf(el(B[nu], e), el(Py[nu], e), el(A[nu], e) * el(Dy, e));
        el(Sx, e) += fmaf(P.w_new, el(nx_, e), P.w_old * el(Px[nu], e));
        el(Sy, e) += fmaf(P.w_new, el(ny_, e), P.w_old * el(Py[nu], e));
      }
      st_state4(psx, nu * S + c, nx_);
      st_state4(psy, nu * S + c, ny_);
    }
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
}

// Interior rows of the pressure half step (same load-first structure).
template <int N, typename MT>
__device__ __forceinline__ void prs2d_fast_rows(const StepParams &P, const float (*svx)[kTX + 8],
                                                const float (*svy)[kTX + 8], int x0, int y0, int tx, int ty) {
  const MT *ik2 = static_cast<const MT *>(P.ik2);
  const MT *a2 = static_cast<const MT *>(P.a2);
  const MT *b2 = static_cast<const MT *>(P.b2);
  const MT *Km = static_cast<const MT *>(P.K);
  const MT *chim = static_cast<const MT *>(P.chi);
  float *psx = P.psi2[0], *psy = P.psi2[1];
  const long long S = P.npts_alloc;
  const int i0 = x0 + 4 * tx;
#pragma unroll 1
  for (int rr = 0; rr < kRows; ++rr) {
    const int ly = ty + rr * kBY;
    const int j = y0 + ly;
    const long long c = (long long)j * P.pitch + i0;
    float4 p = ld_state4(P.p, c);
    const float4 k2 = ldmap4(ik2, c);
    const float4 K = ldmap4(Km, c);
    float4 ch = make_float4(0.f, 0.f, 0.f, 0.f);
    if (P.nl) ch = ldmap4(chim, c);
    float4 A[N > 0 ? N : 1], B[N > 0 ? N : 1], Px[N > 0 ? N : 1], Py[N > 0 ? N : 1];
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      A[nu] = ldmap4(a2, nu * S + c);
      B[nu] = ldmap4(b2, nu * S + c);
      Px[nu] = ld_state4(psx, nu * S + c);
      Py[nu] = ld_state4(psy, nu * S + c);
    }
    float4 Dx, Dy;
    prs_derivs(P, svx, svy, ly, tx, Dx, Dy);
    float4 Sx = make_float4(Dx.x * k2.x, Dx.y * k2.y, Dx.z * k2.z, Dx.w * k2.w);
    float4 Sy = make_float4(Dy.x * k2.x, Dy.y * k2.y, Dy.z * k2.z, Dy.w * k2.w);
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      float4 nx_, ny_;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        el(nx_, e) = fmaf(el(B[nu], e), el(Px[nu], e), el(A[nu], e) * el(Dx, e));
        el(ny_, e) = fmaf(el(B[nu], e), el(Py[nu], e), el(A[nu], e) * el(Dy, e));
        el(Sx, e) += fmaf(P.w_new, el(nx_, e), P.w_old * el(Px[nu], e));
        el(Sy, e) += fmaf(P.w_new, el(ny_, e), P.w_old * el(Py[nu], e));
      }
      st_state4(psx, nu * S + c, nx_);
      st_state4(psy, nu * S + c, ny_);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float upd = P.dt * el(K, e) * (el(Sx, e) + el(Sy, e));
      if (P.nl) upd /= fmaf(el(ch, e), el(p, e), 1.f);
      el(p, e) -= upd;
    }
    st_state4(P.p, c, p);
  }
}

template <int N, typename MT>
__global__ void __launch_bounds__(256, 2) vel2d_kernel(const StepParams P) {
  constexpr int PW = kTX + 8;  // p tile columns: x0-4 .. x0+TX+3
  constexpr int PH = kTY + 7;  // p tile rows:    y0-3 .. y0+TY+3
  constexpr int RW = kTX + 4;  // rho tile columns: x0 .. x0+TX+3
  constexpr int RH = kTY + 1;  // rho tile rows:    y0 .. y0+TY
  __shared__ __align__(16) float sp[PH][PW];
  __shared__ __align__(16) float sr[RH][RW];

  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  const MT *rho = static_cast<const MT *>(P.rho);

  for (int t = tid; t < PH * (PW / 4); t += 256) {
    const int r = t / (PW / 4), c4 = t % (PW / 4);
    const float4 v = load_chunk(P, P.p, x0 - 4 + 4 * c4, y0 - 3 + r, 0);
    *reinterpret_cast<float4 *>(&sp[r][4 * c4]) = v;
  }
  for (int t = tid; t < RH * RW; t += 256) {
    const int r = t / RW, cc = t % RW;
    const int gx = rho_coord(x0 + cc, P.nx, P.periodic[0]);
    const int gy = rho_coord(y0 + r, P.ny, P.periodic[1]);
    sr[r][cc] = ldmap(rho, (long long)gy * P.pitch + gx);
  }
  __syncthreads();

  const int i0 = x0 + 4 * tx;
  if (i0 >= P.nx) return;
  const MT *ik1 = static_cast<const MT *>(P.ik1);
  if (interior_tile(P, x0, y0)) {
    vel2d_fast_rows<N, MT>(P, sp, sr, x0, y0, tx, ty);
    return;
  }
#pragma unroll 1
  for (int rr = 0; rr < kRows; ++rr) {
    const int ly = ty + rr * kBY;
    const int j = y0 + ly;
    if (j >= P.ny) break;
    const long long c = (long long)j * P.pitch + i0;
    const int sy = ly + 3;  // tile row of j
    // d/dx at faces i+1/2: sum_m g_m (p[i+m] - p[i-m+1]); window col 4 is i0
    const Win12 w = win12(sp[sy], tx);
    float4 Dx, Dy;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m] - w.v[4 + e - m + 1], d);
      el(Dx, e) = d;
    }
    // d/dy at faces j+1/2: sum_m g_m (p[j+m] - p[j-m+1])
    {
      float4 col[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) col[m] = *reinterpret_cast<const float4 *>(&sp[sy - 3 + m][4 * tx + 4]);
      // col[3] is row j, col[3 + m] row j+m, col[3 - m + 1] row j-m+1
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float d = 0.f;
#pragma unroll
        for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], el(col[3 + m], e) - el(col[4 - m], e), d);
        el(Dy, e) = d;
      }
    }
    if (P.g11h != 0.f) {
      // cross taps of Sec. 3.1: g11 sum_s (p(i+1, j+s) - p(i, j+s)) for x,
      // g11 sum_s (p(i+s, j+1) - p(i+s, j)) for y
      const Win12 up = win12(sp[sy + 1], tx), dn = win12(sp[sy - 1], tx);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        el(Dx, e) += P.g11h * ((up.v[5 + e] - up.v[4 + e]) + (dn.v[5 + e] - dn.v[4 + e]));
        el(Dy, e) += P.g11h * ((up.v[5 + e] - w.v[5 + e]) + (up.v[3 + e] - w.v[3 + e]));
      }
    }
    // dt / rho at the faces: 2 dt / (rho_i + rho_{i+1})
    float4 bx, by;
    {
      const int lx = 4 * tx;
      const float4 r0 = *reinterpret_cast<const float4 *>(&sr[ly][lx]);
      const float r4 = sr[ly][lx + 4];
      const float4 ru = *reinterpret_cast<const float4 *>(&sr[ly + 1][lx]);
      bx = make_float4(P.two_dt / (r0.x + r0.y), P.two_dt / (r0.y + r0.z), P.two_dt / (r0.z + r0.w),
                       P.two_dt / (r0.w + r4));
      by = make_float4(P.two_dt / (r0.x + ru.x), P.two_dt / (r0.y + ru.y), P.two_dt / (r0.z + ru.z),
                       P.two_dt / (r0.w + ru.w));
    }
    const float4 k1 = ldmap4(ik1, c);
    {
      const float4 S = stretch4<0, 1, N, MT>(P, P.psi1[0], Dx, k1, c, i0, j, 0);
      float4 v = ld_state4(P.v[0], c);
      v.x -= bx.x * S.x; v.y -= bx.y * S.y; v.z -= bx.z * S.z; v.w -= bx.w * S.w;
      st_state4(P.v[0], c, mask_pad(v, i0, P.nx));
    }
    {
      const float4 S = stretch4<1, 1, N, MT>(P, P.psi1[1], Dy, k1, c, i0, j, 0);
      float4 v = ld_state4(P.v[1], c);
      v.x -= by.x * S.x; v.y -= by.y * S.y; v.z -= by.z * S.z; v.w -= by.w * S.w;
      st_state4(P.v[1], c, mask_pad(v, i0, P.nx));
    }
  }
}

template <int N, typename MT>
__global__ void __launch_bounds__(256, 2) prs2d_kernel(const StepParams P) {
  constexpr int W = kTX + 8;   // columns x0-4 .. x0+TX+3
  constexpr int HX = kTY + 2;  // v_x rows y0-1 .. y0+TY
  constexpr int HY = kTY + 7;  // v_y rows y0-4 .. y0+TY+2
  __shared__ __align__(16) float svx[HX][W];
  __shared__ __align__(16) float svy[HY][W];

  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  for (int t = tid; t < HX * (W / 4); t += 256) {
    const int r = t / (W / 4), c4 = t % (W / 4);
    *reinterpret_cast<float4 *>(&svx[r][4 * c4]) = load_chunk(P, P.v[0], x0 - 4 + 4 * c4, y0 - 1 + r, 0);
  }
  for (int t = tid; t < HY * (W / 4); t += 256) {
    const int r = t / (W / 4), c4 = t % (W / 4);
    *reinterpret_cast<float4 *>(&svy[r][4 * c4]) = load_chunk(P, P.v[1], x0 - 4 + 4 * c4, y0 - 4 + r, 0);
  }
  __syncthreads();

  const int i0 = x0 + 4 * tx;
  if (i0 >= P.nx) return;
  if (interior_tile(P, x0, y0)) {
    prs2d_fast_rows<N, MT>(P, svx, svy, x0, y0, tx, ty);
    return;
  }
  const MT *ik2 = static_cast<const MT *>(P.ik2);
  const MT *Km = static_cast<const MT *>(P.K);
  const MT *chim = static_cast<const MT *>(P.chi);
#pragma unroll 1
  for (int rr = 0; rr < kRows; ++rr) {
    const int ly = ty + rr * kBY;
    const int j = y0 + ly;
    if (j >= P.ny) break;
    const long long c = (long long)j * P.pitch + i0;
    // d/dx v_x at centres: sum_m g_m (vx[i+m-1] - vx[i-m]); window col 4 is i0
    const Win12 w = win12(svx[ly + 1], tx);
    float4 Dx, Dy;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float d = 0.f;
#pragma unroll
      for (int m = 1; m <= 4; ++m) d = fmaf(P.gh[m - 1], w.v[4 + e + m - 1] - w.v[4 + e - m], d);
      el(Dx, e) = d;
    }
    {
      // d/dy v_y at centres: sum_m g_m (vy[j+m-1] - vy[j-m]); col[4] is row j
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
    if (P.g11h != 0.f) {
      // g11 sum_s (vx(i, j+s) - vx(i-1, j+s)) and g11 sum_s (vy(i+s, j) - vy(i+s, j-1))
      const Win12 up = win12(svx[ly + 2], tx), dn = win12(svx[ly], tx);
      const Win12 y0w = win12(svy[ly + 4], tx), y1w = win12(svy[ly + 3], tx);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        el(Dx, e) += P.g11h * ((up.v[4 + e] - up.v[3 + e]) + (dn.v[4 + e] - dn.v[3 + e]));
        el(Dy, e) += P.g11h * ((y0w.v[5 + e] - y1w.v[5 + e]) + (y0w.v[3 + e] - y1w.v[3 + e]));
      }
    }
    const float4 k2 = ldmap4(ik2, c);
    const float4 Sx = stretch4<0, 2, N, MT>(P, P.psi2[0], Dx, k2, c, i0, j, 0);
    const float4 Sy = stretch4<1, 2, N, MT>(P, P.psi2[1], Dy, k2, c, i0, j, 0);
    const float4 K = ldmap4(Km, c);
    float4 p = ld_state4(P.p, c);
    float4 upd = make_float4(P.dt * K.x * (Sx.x + Sy.x), P.dt * K.y * (Sx.y + Sy.y),
                             P.dt * K.z * (Sx.z + Sy.z), P.dt * K.w * (Sx.w + Sy.w));
    if (P.nl) {
      const float4 ch = ldmap4(chim, c);
      upd.x /= fmaf(ch.x, p.x, 1.f); upd.y /= fmaf(ch.y, p.y, 1.f);
      upd.z /= fmaf(ch.z, p.z, 1.f); upd.w /= fmaf(ch.w, p.w, 1.f);
    }
    p.x -= upd.x; p.y -= upd.y; p.z -= upd.z; p.w -= upd.w;
    st_state4(P.p, c, mask_pad(p, i0, P.nx));
  }
}

template <typename MT>
cudaError_t vel2d_dispatch(const StepParams &P, dim3 g, dim3 b, cudaStream_t s) {
  switch (P.n_relax) {
    case 0: vel2d_kernel<0, MT><<<g, b, 0, s>>>(P); break;
    case 1: vel2d_kernel<1, MT><<<g, b, 0, s>>>(P); break;
    case 2: vel2d_kernel<2, MT><<<g, b, 0, s>>>(P); break;
    case 3: vel2d_kernel<3, MT><<<g, b, 0, s>>>(P); break;
    case 4: vel2d_kernel<4, MT><<<g, b, 0, s>>>(P); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename MT>
cudaError_t prs2d_dispatch(const StepParams &P, dim3 g, dim3 b, cudaStream_t s) {
  switch (P.n_relax) {
    case 0: prs2d_kernel<0, MT><<<g, b, 0, s>>>(P); break;
    case 1: prs2d_kernel<1, MT><<<g, b, 0, s>>>(P); break;
    case 2: prs2d_kernel<2, MT><<<g, b, 0, s>>>(P); break;
    case 3: prs2d_kernel<3, MT><<<g, b, 0, s>>>(P); break;
    case 4: prs2d_kernel<4, MT><<<g, b, 0, s>>>(P); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_vel2d(const StepParams &P, int map_bf16, cudaStream_t s) {
  dim3 g((P.nx + kTX - 1) / kTX, (P.ny + kTY - 1) / kTY), b(32, kBY);
  return map_bf16 ? vel2d_dispatch<__nv_bfloat16>(P, g, b, s) : vel2d_dispatch<float>(P, g, b, s);
}

cudaError_t launch_prs2d(const StepParams &P, int map_bf16, cudaStream_t s) {
  dim3 g((P.nx + kTX - 1) / kTX, (P.ny + kTY - 1) / kTY), b(32, kBY);
  return map_bf16 ? prs2d_dispatch<__nv_bfloat16>(P, g, b, s) : prs2d_dispatch<float>(P, g, b, s);
}

}  // namespace fw2
