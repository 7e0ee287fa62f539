// Field scan that allocates nothing: fw2_field_absmax_noalloc.
//
// Same result as the scan behind fw2_check_field (max |x|, +inf when any
// value is non-finite) for callers that cannot allocate device memory: an
// application that owns every device allocation itself (a host framework's
// allocator or a fixed memory budget that must account for each byte), or
// a latency-critical loop that cannot afford the device-wide synchronisation
// cudaMalloc / cudaFree may cause.  Its scratch is the file-scope device
// array below, held by every GPU that loads the library until exit.
#include "fw2.h"
#include "fw2_internal.cuh"

namespace fw2 {
void set_global_error(const char *msg);
}

namespace {

// Capacity of the scratch: one partial maximum per field row (4 MiB).
constexpr long long kScratchRows = 1LL << 20;
__device__ __align__(256) float g_row_absmax[kScratchRows];

// One warp per row: max |x| over the row's row_len values, +inf if any is
// non-finite; every row r < n_rows of the scratch is overwritten.
__global__ void row_absmax_kernel(const float *f, long long row_len, long long n_rows, long long pitch,
                                  float *rowmax) {
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = warp; r < n_rows; r += nwarps) {
    const float *row = f + r * pitch;
    float m = 0.f;
    for (long long i = lane; i < row_len; i += 32) {
      const float v = fabsf(row[i]);
      m = isfinite(v) ? fmaxf(m, v) : __int_as_float(0x7f800000);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) rowmax[r] = m;
  }
}

// One block folds the row maxima into *out.
__global__ void rows_fold_kernel(const float *rowmax, long long n_rows, float *out) {
  __shared__ float red[1024];
  float m = 0.f;
  for (long long r = threadIdx.x; r < n_rows; r += blockDim.x) m = fmaxf(m, rowmax[r]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Device address of the scratch in the current device's context.  Host code
// may not use the array's name as a device address, so it is looked up on
// every call: a lookup is cheap once the module is loaded, and nothing is
// cached that a device reset (a new primary context) would leave stale.
cudaError_t scratch_for_current_device(float **ptr) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_row_absmax);
  if (e != cudaSuccess) return e;
  *ptr = static_cast<float *>(p);
  return cudaSuccess;
}

// True when p is device (or managed) memory that the current device owns;
// host memory, pinned or not, and memory of another device are refused
// before any kernel could dereference them.  Queries only, no allocation.
bool on_current_device(const void *p) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error so the next runtime call does not report it
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" fw2_status fw2_field_absmax_noalloc(const float *field, int64_t row_len, int64_t n_rows,
                                               int64_t row_pitch, float *out, void *stream) {
  if (!field || !out) {
    fw2::set_global_error("fw2_field_absmax_noalloc: field and out must be device pointers");
    return FW2_EINVAL;
  }
  if (!on_current_device(field) || !on_current_device(out)) {
    fw2::set_global_error(
        "fw2_field_absmax_noalloc: field and out must be device memory of the current device");
    return FW2_EINVAL;
  }
  if (row_len < 1 || n_rows < 1 || row_pitch < row_len) {
    fw2::set_global_error("fw2_field_absmax_noalloc: need row_len >= 1, n_rows >= 1, row_pitch >= row_len");
    return FW2_EINVAL;
  }
  if (n_rows > kScratchRows) {
    fw2::set_global_error("fw2_field_absmax_noalloc: n_rows exceeds the 1048576 rows of its static scratch");
    return FW2_EINVAL;
  }
  float *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    fw2::set_global_error(cudaGetErrorString(e));
    return FW2_ECUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  long long warps = n_rows < 152LL * 64 ? n_rows : 152LL * 64;
  const int blocks = (int)((warps * 32 + 255) / 256);
  row_absmax_kernel<<<blocks, 256, 0, s>>>(field, row_len, n_rows, row_pitch, scratch);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    rows_fold_kernel<<<1, 1024, 0, s>>>(scratch, n_rows, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    fw2::set_global_error(cudaGetErrorString(e));
    return FW2_ECUDA;
  }
  return FW2_OK;
}
