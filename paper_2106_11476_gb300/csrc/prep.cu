// One-time coefficient preparation on the device (Sec. 3.2, 3.3): FP64 for
// everything but the relaxation pair a, b, which is float (relax_ab32).
//
// From the raw per-cell medium (c, rho, beta) and relaxation parameters
// (kappa1, kappa2, d^nu, alpha^nu for nabla_1 and nabla_2) it writes the maps
// the step kernels stream:
//   K = rho c^2, rho, chi (nonlinear factor of Eq. general6),
//   1/kappa1, 1/kappa2,
//   interior a, b (Eqs. relaxation_a, relaxation_b) of every cell, and
//   per-axis a, b inside the boundary strips, where d and alpha follow the
//   two-stage C-PML ramps of Table 1:  X = (X_target - X_0) g + X_0 with
//   g = (x/L)^npow (nu = 1, d), x/L (nu = 1, alpha) and
//   (1 - cos(pi x / L_T)) / 2 over the transition layer (nu >= 2).  In
//   reading C alpha^{nu=1} is blended by that cosine into the C-PML profile
//   d_target (1 - x/L).
// The profile of a face is evaluated at its exact staggered coordinate; the
// relaxation parameters of a face are those of its lower-index cell.
#include "fw2_prep.cuh"
#include <type_traits>

#include "maps.cuh"

namespace fw2 {

namespace {

// tissue index of input cell t (index form)
__device__ __forceinline__ int tissue_at(const PrepParams &Q, long long t) {
  return Q.tissue_wide ? (int)static_cast<const unsigned short *>(Q.tissue_in)[t]
                       : (int)static_cast<const unsigned char *>(Q.tissue_in)[t];
}
// raw parameter of cell t (dense inputs) or of its tissue (index form)
__device__ __forceinline__ long long src_of(const PrepParams &Q, long long t) {
  return Q.tissue_in ? (long long)tissue_at(Q, t) : t;
}
__device__ __forceinline__ long long n_src(const PrepParams &Q) {
  return Q.tissue_in ? (long long)Q.n_tissue : (long long)Q.nx * Q.ny * Q.nz;
}

__device__ __forceinline__ void store(float *p, long long i, double v) { p[i] = (float)v; }
__device__ __forceinline__ void store(__nv_bfloat16 *p, long long i, double v) {
  p[i] = __float2bfloat16_rn((float)v);
}
// FP16 maps: the value times the map's inverse scale (a power of two, exact),
// rounded to float then to half
__device__ __forceinline__ void store(__half *p, long long i, double v, double inv) {
  p[i] = __float2half_rn((float)(v * inv));
}
__device__ __forceinline__ void store(float *p, long long i, double v, double) { store(p, i, v); }
__device__ __forceinline__ void store(__nv_bfloat16 *p, long long i, double v, double) { store(p, i, v); }

// Where the map kernels put a value: stored (scaled for FP16), or, in the
// scan pass of the FP16 maps, folded into this thread's largest magnitude of
// the map; flush() combines the threads' maxima (warp reduction, one atomic
// per warp and map).
template <typename MT, bool SCAN>
struct MapSink {
  const PrepParams &Q;
  float mx[SCAN ? kMapScales : 1];
  __device__ __forceinline__ explicit MapSink(const PrepParams &q) : Q(q) {
    if (SCAN)
      for (int m = 0; m < kMapScales; ++m) mx[m] = 0.f;
  }
  __device__ __forceinline__ void put(int id, void *p, long long i, double v) {
    if constexpr (SCAN) mx[id] = fmaxf(mx[id], (float)fabs(v));
    else store(static_cast<MT *>(p), i, v, Q.inv_scale[id]);
  }
  // decay factor b with 1 - b given: float maps keep b, bf16 and FP16 maps
  // 1 - b (FP16 times the map's inverse scale)
  __device__ __forceinline__ void put_b2(int id, void *p, long long i, float b, float omb) {
    if constexpr (SCAN) {
      mx[id] = fmaxf(mx[id], fabsf(omb));
    } else if constexpr (std::is_same<MT, float>::value) {
      static_cast<float *>(p)[i] = b;
    } else if constexpr (std::is_same<MT, __nv_bfloat16>::value) {
      static_cast<__nv_bfloat16 *>(p)[i] = __float2bfloat16_rn(omb);
    } else {
      static_cast<__half *>(p)[i] = __float2half_rn((float)((double)omb * Q.inv_scale[id]));
    }
  }
  __device__ __forceinline__ void flush() {
    if constexpr (SCAN) {
      const unsigned lane = threadIdx.x & 31;
      for (int m = 0; m < kMapScales; ++m) {
        const unsigned v = __reduce_max_sync(0xffffffffu, __float_as_uint(mx[m]));
        if (lane == 0 && v) atomicMax(Q.f16_max + m, v);
      }
    }
  }
};

// Relaxation coefficients of Eqs. (relaxation_a), (relaxation_b) (Sec. 3.2)
// in float arithmetic, for the cell maps, the C-PML strips and the tissue
// tables alike (GB300's FP64 rate would make the build an order of magnitude
// slower):
//   b = exp(-(d/kappa + alpha) dt),  a = d (b - 1) / (kappa (d + kappa alpha)).
// em = expm1(-(d/kappa + alpha) dt) keeps b - 1 accurate when b is near 1;
// b = 1 + em, 1 - b = -em (what bf16 and FP16 maps store), and
// a = (d/kappa) em / (d + kappa alpha).  A few float ulps from the FP64
// values, far inside the parity bound.  One function everywhere keeps the
// index form bitwise equal to the gathered dense maps, and a strip cell at
// depth 0 (a subdomain's cut side) equal to the interior cell it continues.
__device__ __forceinline__ void relax_ab32(float d, float alpha, float kappa, float ik, float dt, float &a,
                                           float &b, float &omb) {
  const float dk = d * ik;
  const float em = expm1f(-(dk + alpha) * dt);
  b = 1.f + em;
  omb = -em;
  const float den = d + kappa * alpha;
  a = (d == 0.f || den == 0.f) ? 0.f : dk * em / den;
}

// depth (cells, 0..L) into the boundary region of coordinate x on an axis of
// n cells whose outer L cells on each side form the region
__device__ __forceinline__ double depth_of(double x, int n, int L) {
  if (L <= 0) return 0.0;
  const double lo = L - 0.5, hi = n - L - 0.5;
  double d = 0.0;
  if (x < lo) d = lo - x;
  else if (x > hi) d = x - hi;
  return d < (double)L ? d : (double)L;
}

// C-PML / transition value of parameter X0 at `depth` (Table 1).
// nu is 0-based here (nu = 0 is the paper's nu = 1); is_d selects d or alpha.
__device__ double ramp(const PrepParams &Q, double X0, double depth, int nu, bool is_d) {
  if (depth <= 0.0) return X0;
  const int LT = Q.LT, LB = Q.LB, L = LT + LB;
  if (nu == 0 && !is_d && (Q.reading == 2 || Q.reading == 3)) {
    // reading C: the tissue's alpha is blended (cosine over the transition
    // layer) into the C-PML profile d_target (1 - x/L), linear to 0 at the
    // outer edge
    double gT = 1.0;
    if (LT > 0 && depth < LT) gT = 0.5 * (1.0 - cos(M_PI * depth / LT));
    const double a_cfs = Q.d_target * (1.0 - depth / L);
    return (1.0 - gT) * X0 + gT * a_cfs;
  }
  if (nu == 0) {
    const double s = depth / L;
    if (is_d) return (Q.d_target - X0) * pow(s, Q.npow) + X0;
    return (0.0 - X0) * s + X0;
  }
  if (Q.reading == 3) return X0;  // no transition layer: nu >= 2 kept (unstable, Sec. 3.3)
  double g = 1.0;
  if (LT > 0 && depth < LT) g = 0.5 * (1.0 - cos(M_PI * depth / LT));
  return (0.0 - X0) * g + X0;
}

template <typename MT, bool SCAN>
__global__ void cell_maps_kernel(const PrepParams Q) {
  const long long n = (long long)Q.nx * Q.ny * Q.nz;
  MapSink<MT, SCAN> out(Q);
  // every thread runs the same number of iterations: the scan pass's warp
  // reduction at the end needs the whole warp
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t0 = blockIdx.x * (long long)blockDim.x; t0 < n; t0 += stride) {
    const long long t = t0 + threadIdx.x;
    if (t >= n) continue;
    const int i = (int)(t % Q.nx);
    const long long r = t / Q.nx;
    const int j = (int)(r % Q.ny);
    const int k = (int)(r / Q.ny);
    const long long o = (long long)k * Q.plane + (long long)j * Q.pitch + i;
    const double c = Q.c[t], rho = Q.rho[t];
    const double K = rho * c * c;
    out.put(kMsK, Q.K, o, K);
    out.put(kMsRho, Q.rho_o, o, rho);
    if (Q.nl_mode != 0) {
      const double beta = Q.beta[t];
      const double chi = Q.nl_mode != 2 ? (1.0 - 2.0 * beta) / K : -2.0 * beta / K;  // 1, 3: Eq. general6
      out.put(kMsChi, Q.chi, o, chi);
    }
    const double k1 = Q.N ? (double)Q.k1[t] : 1.0, k2 = Q.N ? (double)Q.k2[t] : 1.0;
    const double ik1 = 1.0 / k1, ik2 = 1.0 / k2;
    out.put(kMsIk1, Q.ik1, o, ik1);
    out.put(kMsIk2, Q.ik2, o, ik2);
    const float dt = (float)Q.dt;
    for (int nu = 0; nu < Q.N; ++nu) {
      float a, b, omb;
      relax_ab32(Q.d1[nu * n + t], Q.al1[nu * n + t], (float)k1, (float)ik1, dt, a, b, omb);
      out.put(kMsA1 + nu, Q.a1, nu * Q.npts_alloc + o, a);
      out.put_b2(kMsB1 + nu, Q.b1, nu * Q.npts_alloc + o, b, omb);
      relax_ab32(Q.d2[nu * n + t], Q.al2[nu * n + t], (float)k2, (float)ik2, dt, a, b, omb);
      out.put(kMsA2 + nu, Q.a2, nu * Q.npts_alloc + o, a);
      out.put_b2(kMsB2 + nu, Q.b2, nu * Q.npts_alloc + o, b, omb);
    }
  }
  out.flush();
}

// Tissue-index form: per-tissue coefficient table ([field][tab_stride],
// field order of maps.cuh) with the same arithmetic as the per-cell maps, and
// the index copied into the pitched cell layout.
__global__ void table_kernel(const PrepParams Q) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Q.n_tissue) return;
  float *T = Q.table_out;
  const int S = Q.tab_stride;  // field stride of this table
  const double c = Q.c[t], rho = Q.rho[t];
  const double K = rho * c * c;
  T[kTabK * S + t] = (float)K;
  T[kTabRho * S + t] = (float)rho;
  if (Q.nl_mode != 0) {
    const double beta = Q.beta[t];
    T[kTabChi * S + t] = (float)(Q.nl_mode != 2 ? (1.0 - 2.0 * beta) / K : -2.0 * beta / K);
  }
  const double k1 = Q.N ? (double)Q.k1[t] : 1.0, k2 = Q.N ? (double)Q.k2[t] : 1.0;
  T[kTabIk1 * S + t] = (float)(1.0 / k1);
  T[kTabIk2 * S + t] = (float)(1.0 / k2);
  const float dt = (float)Q.dt;
  for (int nu = 0; nu < Q.N; ++nu) {
    float a, b, omb;
    relax_ab32(Q.d1[nu * Q.n_tissue + t], Q.al1[nu * Q.n_tissue + t], (float)k1, (float)(1.0 / k1), dt, a, b, omb);
    T[(kTabRelax + nu) * S + t] = a;
    T[(kTabRelax + kTabSlots + nu) * S + t] = b;
    relax_ab32(Q.d2[nu * Q.n_tissue + t], Q.al2[nu * Q.n_tissue + t], (float)k2, (float)(1.0 / k2), dt, a, b, omb);
    T[(kTabRelax + 2 * kTabSlots + nu) * S + t] = a;
    T[(kTabRelax + 3 * kTabSlots + nu) * S + t] = b;
  }
}

__global__ void index_copy_kernel(const PrepParams Q) {
  const long long n = (long long)Q.nx * Q.ny * Q.nz;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t % Q.nx);
    const long long r = t / Q.nx;
    const int j = (int)(r % Q.ny);
    const int k = (int)(r / Q.ny);
    const long long o = (long long)k * Q.plane + (long long)j * Q.pitch + i;
    if (Q.tissue_wide) static_cast<unsigned short *>(Q.tissue_out)[o] = (unsigned short)tissue_at(Q, t);
    else static_cast<unsigned char *>(Q.tissue_out)[o] = (unsigned char)tissue_at(Q, t);
  }
}

// One thread per (strip coordinate, other two coordinates) of axis `axis`.
template <typename MT, bool SCAN>
__global__ void strip_maps_kernel(const PrepParams Q, int axis) {
  const int L = Q.LT + Q.LB;
  const int ext[3] = {Q.nx, Q.ny, Q.nz};
  // strip extents: the axis has 2L entries, the others their full extent
  int se[3] = {Q.nx, Q.ny, Q.nz};
  se[axis] = 2 * L;
  const long long total = (long long)se[0] * se[1] * se[2];
  const long long pitch_out = axis == 0 ? 2 * L : Q.pitch;
  MapSink<MT, SCAN> sink(Q);
  // the same number of iterations in every thread (see cell_maps_kernel)
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t0 = blockIdx.x * (long long)blockDim.x; t0 < total; t0 += stride) {
    const long long t = t0 + threadIdx.x;
    if (t >= total) continue;
    int s[3];
    s[0] = (int)(t % se[0]);
    const long long r = t / se[0];
    s[1] = (int)(r % se[1]);
    s[2] = (int)(r / se[1]);
    int cell[3] = {s[0], s[1], s[2]};
    const int sc = s[axis];
    cell[axis] = sc < L ? sc : ext[axis] - 2 * L + sc;
    const long long src = cell[0] + (long long)Q.nx * (cell[1] + (long long)Q.ny * cell[2]);
    // output index in the strip layout
    long long out;
    if (axis == 0) out = ((long long)s[2] * Q.ny + s[1]) * pitch_out + s[0];
    else if (axis == 1) out = ((long long)s[2] * (2 * L) + s[1]) * pitch_out + s[0];
    else out = ((long long)s[2] * Q.ny + s[1]) * pitch_out + s[0];
    const double dface = depth_of(Q.goff[axis] + cell[axis] + 0.5, Q.gext[axis], L);
    const double dcent = depth_of((double)(Q.goff[axis] + cell[axis]), Q.gext[axis], L);
    const long long ri = src_of(Q, src), nr = n_src(Q);
    const double k1 = Q.k1[ri], k2 = Q.k2[ri];
    const float ik1 = (float)(1.0 / k1), ik2 = (float)(1.0 / k2), dt = (float)Q.dt;
    // the ramped parameters (FP64) through the float coefficients of the cells
    for (int nu = 0; nu < Q.N; ++nu) {
      float a, b, omb;
      const double d1 = ramp(Q, Q.d1[nu * nr + ri], dface, nu, true);
      const double al1 = ramp(Q, Q.al1[nu * nr + ri], dface, nu, false);
      relax_ab32((float)d1, (float)al1, (float)k1, ik1, dt, a, b, omb);
      sink.put(kMsA1 + nu, Q.sa1[axis], nu * Q.strip_nu[axis] + out, a);
      sink.put_b2(kMsB1 + nu, Q.sb1[axis], nu * Q.strip_nu[axis] + out, b, omb);
      const double d2 = ramp(Q, Q.d2[nu * nr + ri], dcent, nu, true);
      const double al2 = ramp(Q, Q.al2[nu * nr + ri], dcent, nu, false);
      relax_ab32((float)d2, (float)al2, (float)k2, ik2, dt, a, b, omb);
      sink.put(kMsA2 + nu, Q.sa2[axis], nu * Q.strip_nu[axis] + out, a);
      sink.put_b2(kMsB2 + nu, Q.sb2[axis], nu * Q.strip_nu[axis] + out, b, omb);
    }
  }
  sink.flush();
}

// Largest c / sqrt(kappa1 kappa2) and largest c (FP64, as ordered bit
// patterns of positive doubles) and a count of invalid cells.
__global__ void medium_scan_kernel(const PrepParams Q, unsigned long long *maxbits, int *bad) {
  const long long n = (long long)Q.nx * Q.ny * Q.nz;
  double m_eff = 0.0, m_c = 0.0;
  int nbad = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    if (Q.tissue_in && tissue_at(Q, t) >= Q.n_tissue) {
      ++nbad;
      continue;
    }
    const long long r = src_of(Q, t);
    const double c = Q.c[r], rho = Q.rho[r];
    double k1 = 1.0, k2 = 1.0;
    if (Q.N) {
      k1 = Q.k1[r];
      k2 = Q.k2[r];
    }
    const bool ok = isfinite(c) && c > 0.0 && isfinite(rho) && rho > 0.0 && isfinite(k1) && k1 > 0.0 &&
                    isfinite(k2) && k2 > 0.0 && (Q.nl_mode == 0 || isfinite((double)Q.beta[r]));
    if (!ok) {
      ++nbad;
      continue;
    }
    const double ce = c / sqrt(k1 * k2);
    m_eff = ce > m_eff ? ce : m_eff;
    m_c = c > m_c ? c : m_c;
  }
  if (m_eff > 0.0) atomicMax(&maxbits[0], (unsigned long long)__double_as_longlong(m_eff));
  if (m_c > 0.0) atomicMax(&maxbits[1], (unsigned long long)__double_as_longlong(m_c));
  if (nbad) atomicAdd(bad, nbad);
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_medium_scan(const PrepParams &Q, unsigned long long *maxbits, int *bad,
                               cudaStream_t s) {
  const long long n = (long long)Q.nx * Q.ny * Q.nz;
  medium_scan_kernel<<<grid_for(n), 256, 0, s>>>(Q, maxbits, bad);
  return cudaGetLastError();
}

namespace {
template <typename MT, bool SCAN>
cudaError_t launch_strips(const PrepParams &Q, cudaStream_t s) {
  const long long n = (long long)Q.nx * Q.ny * Q.nz;
  const int L = Q.LT + Q.LB;
  if (L > 0 && Q.N > 0) {
    for (int axis = 0; axis < Q.nd; ++axis) {
      long long total = 2LL * L * n / (axis == 0 ? Q.nx : axis == 1 ? Q.ny : Q.nz);
      strip_maps_kernel<MT, SCAN><<<grid_for(total), 256, 0, s>>>(Q, axis);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}
}  // namespace

cudaError_t launch_prep(const PrepParams &Q, int map_kind, cudaStream_t s) {
  const long long n = (long long)Q.nx * Q.ny * Q.nz;
  if (map_kind == 2 || map_kind == 3) {
    table_kernel<<<(Q.n_tissue + 255) / 256, 256, 0, s>>>(Q);
    index_copy_kernel<<<grid_for(n), 256, 0, s>>>(Q);
  } else if (map_kind == 1) {
    cell_maps_kernel<__nv_bfloat16, false><<<grid_for(n), 256, 0, s>>>(Q);
  } else if (map_kind == 4) {
    cell_maps_kernel<__half, false><<<grid_for(n), 256, 0, s>>>(Q);
  } else {
    cell_maps_kernel<float, false><<<grid_for(n), 256, 0, s>>>(Q);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (map_kind == 1) return launch_strips<__nv_bfloat16, false>(Q, s);
  if (map_kind == 4) return launch_strips<__half, false>(Q, s);
  return launch_strips<float, false>(Q, s);
}

cudaError_t launch_prep_scan(const PrepParams &Q, cudaStream_t s) {
  const long long n = (long long)Q.nx * Q.ny * Q.nz;
  cell_maps_kernel<__half, true><<<grid_for(n), 256, 0, s>>>(Q);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_strips<__half, true>(Q, s);
}

}  // namespace fw2
