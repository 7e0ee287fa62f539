// General 2D tile functions of the velocity and pressure half steps.
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
// A tile is 128 x 16 cells for a block of (32, 8) threads, 4 consecutive x
// cells per thread (128-bit loads and stores of every streamed array), two
// rows each.  The stencil operand (p, or v_x / v_y) is staged in shared
// memory with its halo; every other array is read once and written once.
// Interior tiles issue every global load of a row before the first store.
// Coefficient maps are read through a policy (maps.cuh): dense float / bf16
// maps, or a uint8 tissue index into per-tissue tables in shared memory.
// Included by the translation units that launch 2D half steps.
#pragma once
#include "coef.cuh"
#include "maps.cuh"

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

// A tile whose cells, stencil halo and face neighbours all lie inside the
// grid and outside every C-PML strip: every cell uses the interior maps for
// both axes, and no boundary rule applies.
__device__ __forceinline__ bool interior_tile(const StepParams &P, int x0, int y0) {
  const int Lx = P.L[0] > 4 ? P.L[0] : 4, Ly = P.L[1] > 4 ? P.L[1] : 4;
  return x0 >= Lx && x0 + kTX + Lx <= P.nx && y0 >= Ly && y0 + kTY + Ly <= P.ny;
}

// x and y derivatives of the staged p at the four faces of a thread
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
    // cross taps of Sec. 3.1: g11 sum_s (p(i+1, j+s) - p(i, j+s)) for x,
    // g11 sum_s (p(i+s, j+1) - p(i+s, j)) for y
    const Win12 up = win12(sp[sy + 1], tx), dn = win12(sp[sy - 1], tx);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el(Dx, e) += P.g11h * ((up.v[5 + e] - up.v[4 + e]) + (dn.v[5 + e] - dn.v[4 + e]));
      el(Dy, e) += P.g11h * ((up.v[5 + e] - w.v[5 + e]) + (up.v[3 + e] - w.v[3 + e]));
    }
  }
}

// x and y derivatives of v_x, v_y at the four centres of a thread
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
    // g11 sum_s (vx(i, j+s) - vx(i-1, j+s)) and g11 sum_s (vy(i+s, j) - vy(i+s, j-1))
    const Win12 up = win12(svx[ly + 2], tx), dn = win12(svx[ly], tx);
    const Win12 y0w = win12(svy[ly + 4], tx), y1w = win12(svy[ly + 3], tx);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el(Dx, e) += P.g11h * ((up.v[4 + e] - up.v[3 + e]) + (dn.v[4 + e] - dn.v[3 + e]));
      el(Dy, e) += P.g11h * ((y0w.v[5 + e] - y1w.v[5 + e]) + (y0w.v[3 + e] - y1w.v[3 + e]));
    }
  }
}

// a, b of mechanism nu for axis Q at the cells of a group (edge path):
// from the boundary strip of axis Q inside its C-PML region (Sec. 3.3: each
// axis' parameters depend on the distance along that axis only), else from
// the interior maps.
template <int Q, int OP, typename Maps>
__device__ __forceinline__ void coef_edge(const StepParams &P, const Maps &M, typename Maps::Cell cell, int nu,
                                          int i0, int j, float4 &a, float4 &b) {
  using ST = typename Maps::StripT;
  const ST *sa = static_cast<const ST *>(OP == 1 ? P.sa1[Q] : P.sa2[Q]);
  const ST *sb = static_cast<const ST *>(OP == 1 ? P.sb1[Q] : P.sb2[Q]);
  const int L = P.L[Q];
  if (Q == 0) {
    const bool any = L > 0 && (i0 < L || i0 + 3 >= P.nx - L);
    if (!any) {
      a = M.template a<OP>(cell, nu);
      b = M.template b<OP>(cell, nu);
      return;
    }
    const long long row = (long long)nu * P.strip_nu[0] + (long long)j * (2 * L);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int x = i0 + e;
      float av = 0.f, bv = 0.f;
      if (x < P.nx) {
        const int sc = strip_coord(x, P.nx, L);
        if (sc >= 0) {
          av = ldmap(sa, row + sc, P.ms[(OP == 1 ? kMsA1 : kMsA2) + nu]);
          bv = ldb(sb, row + sc, P.ms[(OP == 1 ? kMsB1 : kMsB2) + nu]);
        } else {
          av = M.template a1c<OP>(cell, nu, e);
          bv = M.template b1c<OP>(cell, nu, e);
        }
      }
      el(a, e) = av;
      el(b, e) = bv;
    }
  } else {
    const int sc = strip_coord(j, P.ny, L);
    if (sc < 0) {
      a = M.template a<OP>(cell, nu);
      b = M.template b<OP>(cell, nu);
    } else {
      const long long off = (long long)nu * P.strip_nu[1] + (long long)sc * P.pitch + i0;
      a = ldmap4(sa, off, P.ms[(OP == 1 ? kMsA1 : kMsA2) + nu]);
      b = ldb4(sb, off, P.ms[(OP == 1 ? kMsB1 : kMsB2) + nu]);
    }
  }
}

// Stretched derivative of Eq. (relaxation4) for the four cells of a group
// (edge path): S = D / kappa + sum_nu (w_new psi_new + w_old psi_old),
// psi_new = b psi_old + a D (Eq. relaxation_psi), psi written back.
template <int Q, int OP, int N, typename Maps>
__device__ __forceinline__ float4 stretch_edge(const StepParams &P, const Maps &M, typename Maps::Cell cell,
                                               float *psi, float4 D, float4 ik, long long c, int i0, int j) {
  float4 S = make_float4(D.x * ik.x, D.y * ik.y, D.z * ik.z, D.w * ik.w);
#pragma unroll
  for (int nu = 0; nu < N; ++nu) {
    float4 a, b;
    coef_edge<Q, OP>(P, M, cell, nu, i0, j, a, b);
    const long long o = (long long)nu * P.npts_alloc + c;
    const float4 ps = ld_state4(psi, o);
    float4 pn;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      el(pn, e) = fmaf(el(b, e), el(ps, e), el(a, e) * el(D, e));
      el(S, e) += fmaf(P.w_new, el(pn, e), P.w_old * el(ps, e));
    }
    st_state4(psi, o, mask_pad(pn, i0, P.nx));
  }
  return S;
}

// Momentum factors of the literal nonlinear system (Eq. general5) at the x
// and y faces of the four cells i0..i0+3 of row j: p from the staged operand
// (row sy of sp; zero or wrapped beyond the grid), K through the maps with
// the density's neighbour rule.  Cells past nx are clamped (their results are
// masked).
template <typename Maps>
__device__ __forceinline__ void mom_factors(const StepParams &P, const Maps &M, const float (*sp)[kTX + 8], int sy,
                                            int tx, int i0, int j, float4 &fx, float4 &fy) {
  const Win12 w = win12(sp[sy], tx), up = win12(sp[sy + 1], tx);
  const int jn = rho_coord(j + 1, P.ny, P.periodic[1]);
  const long long row = (long long)j * P.pitch, rown = (long long)jn * P.pitch;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int x = min(i0 + e, P.nx - 1);
    const int xn = rho_coord(min(i0 + e + 1, P.nx), P.nx, P.periodic[0]);
    const float Kc = M.K_at(row + x), Kx = M.K_at(row + xn), Ky = M.K_at(rown + x);
    el(fx, e) = mom_factor(Kc, Kx, w.v[4 + e], w.v[5 + e]);
    el(fy, e) = mom_factor(Kc, Ky, w.v[4 + e], up.v[4 + e]);
  }
}

// Interior rows of the velocity half step.  Every global load of a row (both
// velocity components, the maps and the memory variables of both axes) is
// issued before any store, so a row pays one memory latency instead of one
// per mechanism.
template <int N, typename Maps>
__device__ __forceinline__ void vel2d_fast_rows(const StepParams &P, const Maps &M, const float (*sp)[kTX + 8],
                                                const float (*sr)[kTX + 4], int x0, int y0, int tx, int ty) {
  float *psx = P.psi1[0], *psy = P.psi1[1];
  const long long S = P.npts_alloc;
  const int i0 = x0 + 4 * tx;
#pragma unroll 1
  for (int rr = 0; rr < kRows; ++rr) {
    const int ly = ty + rr * kBY;
    const int j = y0 + ly;
    const long long c = (long long)j * P.pitch + i0;
    const typename Maps::Cell cell = M.cell(c);
    float4 vx = ld_state4(P.v[0], c), vy = ld_state4(P.v[1], c);
    float4 Px[N > 0 ? N : 1], Py[N > 0 ? N : 1];
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      Px[nu] = ld_state4(psx, nu * S + c);
      Py[nu] = ld_state4(psy, nu * S + c);
    }
    const float4 k1 = M.ik1(cell);
    float4 A[N > 0 ? N : 1], B[N > 0 ? N : 1];
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      A[nu] = M.template a<1>(cell, nu);
      B[nu] = M.template b<1>(cell, nu);
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
    if (P.nl_vel) {
      float4 fx, fy;
      mom_factors(P, M, sp, ly + 3, tx, i0, j, fx, fy);
      vx.x = vel_upd(vx.x, qdiv(P.two_dt, r0.x + r0.y), Sx.x, fx.x);
      vx.y = vel_upd(vx.y, qdiv(P.two_dt, r0.y + r0.z), Sx.y, fx.y);
      vx.z = vel_upd(vx.z, qdiv(P.two_dt, r0.z + r0.w), Sx.z, fx.z);
      vx.w = vel_upd(vx.w, qdiv(P.two_dt, r0.w + r4), Sx.w, fx.w);
      vy.x = vel_upd(vy.x, qdiv(P.two_dt, r0.x + ru.x), Sy.x, fy.x);
      vy.y = vel_upd(vy.y, qdiv(P.two_dt, r0.y + ru.y), Sy.y, fy.y);
      vy.z = vel_upd(vy.z, qdiv(P.two_dt, r0.z + ru.z), Sy.z, fy.z);
      vy.w = vel_upd(vy.w, qdiv(P.two_dt, r0.w + ru.w), Sy.w, fy.w);
    } else {
      vx.x = vel_upd(vx.x, qdiv(P.two_dt, r0.x + r0.y), Sx.x);
      vx.y = vel_upd(vx.y, qdiv(P.two_dt, r0.y + r0.z), Sx.y);
      vx.z = vel_upd(vx.z, qdiv(P.two_dt, r0.z + r0.w), Sx.z);
      vx.w = vel_upd(vx.w, qdiv(P.two_dt, r0.w + r4), Sx.w);
      vy.x = vel_upd(vy.x, qdiv(P.two_dt, r0.x + ru.x), Sy.x);
      vy.y = vel_upd(vy.y, qdiv(P.two_dt, r0.y + ru.y), Sy.y);
      vy.z = vel_upd(vy.z, qdiv(P.two_dt, r0.z + ru.z), Sy.z);
      vy.w = vel_upd(vy.w, qdiv(P.two_dt, r0.w + ru.w), Sy.w);
    }
    st_state4(P.v[0], c, vx);
    st_state4(P.v[1], c, vy);
  }
}

// Interior rows of the pressure half step (same load-first structure).
template <int N, typename Maps>
__device__ __forceinline__ void prs2d_fast_rows(const StepParams &P, const Maps &M, const float (*svx)[kTX + 8],
                                                const float (*svy)[kTX + 8], int x0, int y0, int tx, int ty) {
  float *psx = P.psi2[0], *psy = P.psi2[1];
  const long long S = P.npts_alloc;
  const int i0 = x0 + 4 * tx;
#pragma unroll 1
  for (int rr = 0; rr < kRows; ++rr) {
    const int ly = ty + rr * kBY;
    const int j = y0 + ly;
    const long long c = (long long)j * P.pitch + i0;
    const typename Maps::Cell cell = M.cell(c);
    float4 p = ld_state4(P.p, c);
    float4 Px[N > 0 ? N : 1], Py[N > 0 ? N : 1];
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      Px[nu] = ld_state4(psx, nu * S + c);
      Py[nu] = ld_state4(psy, nu * S + c);
    }
    const float4 k2 = M.ik2(cell);
    const float4 K = M.Kv(cell);
    float4 ch = make_float4(0.f, 0.f, 0.f, 0.f);
    if (P.nl) ch = M.chiv(cell);
    float4 A[N > 0 ? N : 1], B[N > 0 ? N : 1];
#pragma unroll
    for (int nu = 0; nu < N; ++nu) {
      A[nu] = M.template a<2>(cell, nu);
      B[nu] = M.template b<2>(cell, nu);
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
      if (P.nl) upd = qdiv(upd, fmaf(el(ch, e), el(p, e), 1.f));
      el(p, e) -= upd;
    }
    st_state4(P.p, c, p);
  }
}

constexpr int kPW = kTX + 8;  // p tile columns: x0-4 .. x0+TX+3
constexpr int kPH = kTY + 7;  // p tile rows:    y0-3 .. y0+TY+3
constexpr int kRW = kTX + 4;  // rho tile columns: x0 .. x0+TX+3
constexpr int kRH = kTY + 1;  // rho tile rows:    y0 .. y0+TY

// One 128 x 16 tile of the velocity half step.  `stage` false skips copying
// the maps' shared-memory table (already staged for this context).
template <int N, typename Maps>
__device__ __forceinline__ void vel2d_tile(const StepParams &P, int x0, int y0, float (*sp)[kPW],
                                           float (*sr)[kRW], float *stab, bool stage) {
  constexpr int PW = kPW, PH = kPH, RW = kRW, RH = kRH;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  Maps M(P);
  if (stage) M.stage(P, stab, tid);
  for (int t = tid; t < PH * (PW / 4); t += 256) {
    const int r = t / (PW / 4), c4 = t % (PW / 4);
    const float4 v = load_chunk(P, P.p, x0 - 4 + 4 * c4, y0 - 3 + r, 0);
    *reinterpret_cast<float4 *>(&sp[r][4 * c4]) = v;
  }
  __syncthreads();  // the table must be staged before the rho tile reads it
  M.bind(stab);
  for (int t = tid; t < RH * RW; t += 256) {
    const int r = t / RW, cc = t % RW;
    const int gx = rho_coord(x0 + cc, P.nx, P.periodic[0]);
    const int gy = rho_coord(y0 + r, P.ny, P.periodic[1]);
    sr[r][cc] = M.rho_at((long long)gy * P.pitch + gx);
  }
  __syncthreads();

  const int i0 = x0 + 4 * tx;
  if (i0 >= P.nx) return;
  if (interior_tile(P, x0, y0)) {
    vel2d_fast_rows<N>(P, M, sp, sr, x0, y0, tx, ty);
    return;
  }
#pragma unroll 1
  for (int rr = 0; rr < kRows; ++rr) {
    const int ly = ty + rr * kBY;
    const int j = y0 + ly;
    if (j >= P.ny) break;
    const long long c = (long long)j * P.pitch + i0;
    const typename Maps::Cell cell = M.cell(c);
    float4 Dx, Dy;
    vel_derivs(P, sp, ly + 3, tx, Dx, Dy);
    // dt / rho at the faces: 2 dt / (rho_i + rho_{i+1})
    float4 bx, by;
    {
      const int lx = 4 * tx;
      const float4 r0 = *reinterpret_cast<const float4 *>(&sr[ly][lx]);
      const float r4 = sr[ly][lx + 4];
      const float4 ru = *reinterpret_cast<const float4 *>(&sr[ly + 1][lx]);
      bx = make_float4(qdiv(P.two_dt, r0.x + r0.y), qdiv(P.two_dt, r0.y + r0.z), qdiv(P.two_dt, r0.z + r0.w),
                       qdiv(P.two_dt, r0.w + r4));
      by = make_float4(qdiv(P.two_dt, r0.x + ru.x), qdiv(P.two_dt, r0.y + ru.y), qdiv(P.two_dt, r0.z + ru.z),
                       qdiv(P.two_dt, r0.w + ru.w));
    }
    const float4 k1 = M.ik1(cell);
    float4 fx = make_float4(1.f, 1.f, 1.f, 1.f), fy = fx;
    if (P.nl_vel) mom_factors(P, M, sp, ly + 3, tx, i0, j, fx, fy);
    {
      const float4 S = stretch_edge<0, 1, N>(P, M, cell, P.psi1[0], Dx, k1, c, i0, j);
      float4 v = ld_state4(P.v[0], c);
      if (P.nl_vel) {
        v.x = vel_upd(v.x, bx.x, S.x, fx.x); v.y = vel_upd(v.y, bx.y, S.y, fx.y);
        v.z = vel_upd(v.z, bx.z, S.z, fx.z); v.w = vel_upd(v.w, bx.w, S.w, fx.w);
      } else {
        v.x = vel_upd(v.x, bx.x, S.x); v.y = vel_upd(v.y, bx.y, S.y);
        v.z = vel_upd(v.z, bx.z, S.z); v.w = vel_upd(v.w, bx.w, S.w);
      }
      st_state4(P.v[0], c, mask_pad(v, i0, P.nx));
    }
    {
      const float4 S = stretch_edge<1, 1, N>(P, M, cell, P.psi1[1], Dy, k1, c, i0, j);
      float4 v = ld_state4(P.v[1], c);
      if (P.nl_vel) {
        v.x = vel_upd(v.x, by.x, S.x, fy.x); v.y = vel_upd(v.y, by.y, S.y, fy.y);
        v.z = vel_upd(v.z, by.z, S.z, fy.z); v.w = vel_upd(v.w, by.w, S.w, fy.w);
      } else {
        v.x = vel_upd(v.x, by.x, S.x); v.y = vel_upd(v.y, by.y, S.y);
        v.z = vel_upd(v.z, by.z, S.z); v.w = vel_upd(v.w, by.w, S.w);
      }
      st_state4(P.v[1], c, mask_pad(v, i0, P.nx));
    }
  }
}

constexpr int kHX = kTY + 2;  // v_x rows y0-1 .. y0+TY
constexpr int kHY = kTY + 7;  // v_y rows y0-4 .. y0+TY+2

// One 128 x 16 tile of the pressure half step.
template <int N, typename Maps>
__device__ __forceinline__ void prs2d_tile(const StepParams &P, int x0, int y0, float (*svx)[kPW],
                                           float (*svy)[kPW], float *stab, bool stage) {
  constexpr int W = kPW, HX = kHX, HY = kHY;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * 32 + tx;
  Maps M(P);
  if (stage) M.stage(P, stab, tid);
  for (int t = tid; t < HX * (W / 4); t += 256) {
    const int r = t / (W / 4), c4 = t % (W / 4);
    *reinterpret_cast<float4 *>(&svx[r][4 * c4]) = load_chunk(P, P.v[0], x0 - 4 + 4 * c4, y0 - 1 + r, 0);
  }
  for (int t = tid; t < HY * (W / 4); t += 256) {
    const int r = t / (W / 4), c4 = t % (W / 4);
    *reinterpret_cast<float4 *>(&svy[r][4 * c4]) = load_chunk(P, P.v[1], x0 - 4 + 4 * c4, y0 - 4 + r, 0);
  }
  __syncthreads();
  M.bind(stab);

  const int i0 = x0 + 4 * tx;
  if (i0 >= P.nx) return;
  if (interior_tile(P, x0, y0)) {
    prs2d_fast_rows<N>(P, M, svx, svy, x0, y0, tx, ty);
    return;
  }
#pragma unroll 1
  for (int rr = 0; rr < kRows; ++rr) {
    const int ly = ty + rr * kBY;
    const int j = y0 + ly;
    if (j >= P.ny) break;
    const long long c = (long long)j * P.pitch + i0;
    const typename Maps::Cell cell = M.cell(c);
    float4 Dx, Dy;
    prs_derivs(P, svx, svy, ly, tx, Dx, Dy);
    const float4 k2 = M.ik2(cell);
    const float4 Sx = stretch_edge<0, 2, N>(P, M, cell, P.psi2[0], Dx, k2, c, i0, j);
    const float4 Sy = stretch_edge<1, 2, N>(P, M, cell, P.psi2[1], Dy, k2, c, i0, j);
    const float4 K = M.Kv(cell);
    float4 p = ld_state4(P.p, c);
    float4 upd = make_float4(P.dt * K.x * (Sx.x + Sy.x), P.dt * K.y * (Sx.y + Sy.y),
                             P.dt * K.z * (Sx.z + Sy.z), P.dt * K.w * (Sx.w + Sy.w));
    if (P.nl) {
      const float4 ch = M.chiv(cell);
      upd.x = qdiv(upd.x, fmaf(ch.x, p.x, 1.f)); upd.y = qdiv(upd.y, fmaf(ch.y, p.y, 1.f));
      upd.z = qdiv(upd.z, fmaf(ch.z, p.z, 1.f)); upd.w = qdiv(upd.w, fmaf(ch.w, p.w, 1.f));
    }
    p.x -= upd.x; p.y -= upd.y; p.z -= upd.z; p.w -= upd.w;
    st_state4(P.p, c, mask_pad(p, i0, P.nx));
  }
}

}  // namespace

}  // namespace fw2
