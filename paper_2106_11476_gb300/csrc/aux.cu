// Source injection, sensor recording, the field scan and the self-test of
// the bounded wait (sm_103a).
#include "async.cuh"
#include "fw2_prep.cuh"

namespace fw2 {

namespace {

// One thread per distinct target cell: the entries feeding it are summed in
// a fixed order, so repeated runs give identical results (no atomics).
__global__ void inject_kernel(float *field, const long long *tgt, const int *off, const int *col,
                              const float *row, int n_tgt) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n_tgt) return;
  float s = 0.f;
  for (int e = off[u]; e < off[u + 1]; ++e) s += __ldg(row + col[e]);
  field[tgt[u]] += s;
}

// One thread per sensor group: mean of p over the group's cells.
__global__ void record_kernel(const float *p, const long long *cell, const int *off, int n_groups,
                              float *out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_groups) return;
  const int b = off[g], e = off[g + 1];
  float s = 0.f;
  for (int i = b; i < e; ++i) s += p[cell[i]];
  out[g] = e > b ? s / (float)(e - b) : 0.f;
}

// max |x| over the valid cells, non-finite values count as +inf.  Each block
// reduces in shared memory and folds its result into *out_bits with an
// integer atomicMax (non-negative floats order like their bit patterns).
__global__ void absmax_kernel(const float *f, int nx, int pitch, long long rows, unsigned int *out_bits) {
  __shared__ float red[256];
  float m = 0.f;
  const long long n = rows * (long long)nx;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / nx;
    const int i = (int)(t - r * nx);
    const float v = fabsf(f[r * pitch + i]);
    m = isfinite(v) ? fmaxf(m, v) : __int_as_float(0x7f800000);
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out_bits, __float_as_uint(red[0]));
}

}  // namespace

cudaError_t launch_inject(float *field, const long long *tgt, const int *off, const int *col,
                          const float *row, int n_tgt, cudaStream_t s) {
  if (n_tgt <= 0) return cudaSuccess;
  inject_kernel<<<(n_tgt + 127) / 128, 128, 0, s>>>(field, tgt, off, col, row, n_tgt);
  return cudaGetLastError();
}

cudaError_t launch_record(const float *p, const long long *cell, const int *off, int n_groups,
                          float *out, cudaStream_t s) {
  if (n_groups <= 0) return cudaSuccess;
  record_kernel<<<(n_groups + 127) / 128, 128, 0, s>>>(p, cell, off, n_groups, out);
  return cudaGetLastError();
}

cudaError_t launch_absmax(const float *f, int nx, int pitch, long long rows, unsigned int *out_bits,
                          cudaStream_t s) {
  long long n = rows * (long long)nx;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  absmax_kernel<<<(int)blocks, 256, 0, s>>>(f, nx, pitch, rows, out_bits);
  return cudaGetLastError();
}

namespace {
// one thread waits on an mbarrier that never completes (count 1, no arrival)
__global__ void bounded_wait_kernel(unsigned long long limit_ns, int *timed_out) {
  __shared__ __align__(8) uint64_t bar;
  mbar_init(&bar, 1);
  fence_mbarrier_init();
  *timed_out = mbar_wait_bounded(&bar, 0, limit_ns) ? 0 : 1;
}
}  // namespace

cudaError_t launch_bounded_wait_selftest(unsigned long long limit_ns, int *timed_out) {
  bounded_wait_kernel<<<1, 1>>>(limit_ns, timed_out);
  return cudaGetLastError();
}

}  // namespace fw2
