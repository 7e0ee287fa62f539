// Internal declarations shared by the CUDA translation units of libfw2.
//
// Device layout (all arrays in HBM, one allocation per context):
//   every per-cell array is [nz][ny][pitch] (pitch = nx rounded up to 16
//   elements, so each row starts on a 16-byte boundary for 128-bit accesses
//   and tensor copies of every element type; the padding columns of state
//   arrays stay zero);
//   memory variables psi1_q / psi2_q are [N][nz][ny][pitch];
//   coefficient maps use the same cell layout in float or bf16;
//   boundary strips hold the per-axis a, b of the C-PML region only:
//     x: [N][nz][ny][2L], y: [N][nz][2L][pitch], z: [N][2L][ny][pitch],
//   indexed by the strip coordinate (low side 0..L-1, high side L..2L-1).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fw2 {

// mechanisms per context: up to 8 on the tile kernels (dense float or bf16
// maps); the pipelined 2D half steps and the tissue-index tables take up to
// 4, the pipelined 3D half steps up to 3
constexpr int kMaxRelax = 8;
// Scales of the FP16 maps (StepParams::ms): every map is stored divided by a
// power of two chosen from its largest magnitude; slots per map, per
// mechanism for the relaxation coefficients (b kept as 1 - b)
enum {
  kMsK = 0, kMsRho = 1, kMsChi = 2, kMsIk1 = 3, kMsIk2 = 4,
  kMsA1 = 5, kMsB1 = kMsA1 + kMaxRelax, kMsA2 = kMsB1 + kMaxRelax, kMsB2 = kMsA2 + kMaxRelax,
  kMapScales = kMsB2 + kMaxRelax
};
constexpr int kTabSlots = 4;       // mechanism slots of the tissue-index tables
constexpr int kPipe2dMaxRelax = 4;

struct StepParams {
  int nx, ny, nz;        // logical extent
  int pitch;             // row pitch in elements (multiple of 16)
  long long plane;       // pitch * ny
  long long npts_alloc;  // plane * nz
  int L[3];              // boundary cells per side on each axis (0: no strip)
  int periodic[3];
  float dt, two_dt;
  float gh[4];           // g_i / h
  float g11h;            // g_{1,1} / h
  float w_new, w_old;    // memory-term weights: centred (0.5, 0.5), endpoint (1, 0)
  int nl;                // nonlinear factor present
  int nl_vel;            // momentum factor 1 + kappa0 p at the faces (literal system)
  int n_relax;
  // state (float)
  float *p;
  float *v[3];
  float *psi1[3];        // [N][npts_alloc]
  float *psi2[3];
  // maps (float or bf16, see MapT)
  const void *K;         // rho c^2
  const void *rho;
  const void *chi;
  const void *ik1, *ik2; // 1/kappa1, 1/kappa2
  const void *a1, *b1, *a2, *b2;          // interior [N][npts_alloc]
  const void *sa1[3], *sb1[3], *sa2[3], *sb2[3];  // strips
  long long strip_nu[3]; // elements between mechanisms in a strip array
  // tissue-index form: index per cell (uint8, or uint16 for the wide form)
  // and per-tissue tables ([field][tab_stride] floats, field order of
  // maps.cuh; tab_stride 256 for uint8)
  const unsigned char *tissue;
  const float *table;
  int tab_stride;
  unsigned int *status;  // device status word: bit 0 set when a bounded wait gave up
  float ms[kMapScales];  // FP16 maps: value = stored x ms[map] (1 for the other storages)
};

// ---------------------------------------------------------------- loads ---
__device__ __forceinline__ float ldmap(const float *p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ float ldmap(const __nv_bfloat16 *p, long long i) {
  return __bfloat162float(p[i]);
}
__device__ __forceinline__ float4 ldmap4(const float *p, long long i) {
  return __ldg(reinterpret_cast<const float4 *>(p + i));
}
__device__ __forceinline__ float4 ldmap4(const __nv_bfloat16 *p, long long i) {
  uint2 u = __ldg(reinterpret_cast<const uint2 *>(p + i));
  __nv_bfloat162 lo = *reinterpret_cast<__nv_bfloat162 *>(&u.x);
  __nv_bfloat162 hi = *reinterpret_cast<__nv_bfloat162 *>(&u.y);
  float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
  return make_float4(a.x, a.y, b.x, b.y);
}
// Decay factors b of the recursion: float maps hold b, bf16 maps hold 1 - b
// (bf16 cannot resolve b close to 1, e.g. 0.9999 would round to 1.0).
__device__ __forceinline__ float4 ldb4(const float *p, long long i) { return ldmap4(p, i); }
__device__ __forceinline__ float4 ldb4(const __nv_bfloat16 *p, long long i) {
  const float4 v = ldmap4(p, i);
  return make_float4(1.f - v.x, 1.f - v.y, 1.f - v.z, 1.f - v.w);
}
__device__ __forceinline__ float ldb(const float *p, long long i) { return ldmap(p, i); }
__device__ __forceinline__ float ldb(const __nv_bfloat16 *p, long long i) { return 1.f - ldmap(p, i); }

// The same loads with the map's scale s: FP16 maps hold value / s (s a power
// of two, so the product is exact); float and bf16 maps ignore s.
__device__ __forceinline__ float ldmap(const float *p, long long i, float) { return ldmap(p, i); }
__device__ __forceinline__ float ldmap(const __nv_bfloat16 *p, long long i, float) { return ldmap(p, i); }
__device__ __forceinline__ float ldmap(const __half *p, long long i, float s) { return __half2float(p[i]) * s; }
__device__ __forceinline__ float4 ldmap4(const float *p, long long i, float) { return ldmap4(p, i); }
__device__ __forceinline__ float4 ldmap4(const __nv_bfloat16 *p, long long i, float) { return ldmap4(p, i); }
__device__ __forceinline__ float4 ldmap4(const __half *p, long long i, float s) {
  uint2 u = __ldg(reinterpret_cast<const uint2 *>(p + i));
  const float2 a = __half22float2(*reinterpret_cast<__half2 *>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<__half2 *>(&u.y));
  return make_float4(a.x * s, a.y * s, b.x * s, b.y * s);
}
__device__ __forceinline__ float ldb(const float *p, long long i, float) { return ldb(p, i); }
__device__ __forceinline__ float ldb(const __nv_bfloat16 *p, long long i, float) { return ldb(p, i); }
__device__ __forceinline__ float ldb(const __half *p, long long i, float s) { return 1.f - ldmap(p, i, s); }
__device__ __forceinline__ float4 ldb4(const float *p, long long i, float) { return ldb4(p, i); }
__device__ __forceinline__ float4 ldb4(const __nv_bfloat16 *p, long long i, float) { return ldb4(p, i); }
__device__ __forceinline__ float4 ldb4(const __half *p, long long i, float s) {
  const float4 v = ldmap4(p, i, s);
  return make_float4(1.f - v.x, 1.f - v.y, 1.f - v.z, 1.f - v.w);
}

// streaming state loads/stores: read once, write once per step
__device__ __forceinline__ float4 ld_state4(const float *p, long long i) {
  return __ldcs(reinterpret_cast<const float4 *>(p + i));
}
__device__ __forceinline__ void st_state4(float *p, long long i, float4 v) {
  __stcs(reinterpret_cast<float4 *>(p + i), v);
}

__device__ __forceinline__ float &el(float4 &v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
__device__ __forceinline__ float el(const float4 &v, int e) {
  return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

// Strip coordinate along an axis of extent n with L boundary cells per side,
// or -1 in the interior.
__device__ __forceinline__ int strip_coord(int i, int n, int L) {
  if (L <= 0) return -1;
  if (i < L) return i;
  if (i >= n - L) return i - (n - 2 * L);
  return -1;
}

// ------------------------------------------------------------- launches ---
// 2D kernels: tile of kTX x kTY cells, block (32, 8), 4 x-cells per thread.
constexpr int kTX = 128;
constexpr int kTY = 16;
constexpr int kBY = 8;

// map_kind: 0 float maps, 1 bf16 maps, 2 uint8 tissue index + tables in
// shared memory, 3 uint16 tissue index + tables read through L2 (tile path),
// 4 FP16 maps with a power-of-two scale per map (tile path)
cudaError_t launch_vel2d(const StepParams &P, int map_kind, cudaStream_t s);
cudaError_t launch_prs2d(const StepParams &P, int map_kind, cudaStream_t s);
// the same for 5..8 mechanisms (dense maps; a second compilation of the tile
// kernels, so the two sets build in parallel)
cudaError_t launch_vel2d_wide(const StepParams &P, int map_kind, cudaStream_t s);
cudaError_t launch_prs2d_wide(const StepParams &P, int map_kind, cudaStream_t s);
cudaError_t launch_batched2d_wide(bool vel, const StepParams *Ps, const int4 *tiles, int n_tiles, int n_relax,
                                  int map_kind, int grid, cudaStream_t s);
// persistent batched 2D half step over a tile table {ctx, x0, y0, -} of
// several contexts sharing N and the map kind (vel: velocity, else pressure)
cudaError_t launch_batched2d(bool vel, const StepParams *Ps, const int4 *tiles, int n_tiles, int n_relax,
                             int map_kind, int grid, cudaStream_t s);
// persistent pipelined 2D half step (one block per SM: grid = SM count):
// edge tiles by the tile path, interior half tiles staged by cp.async;
// float maps (map_kind 0) and the tissue index (2)
struct PipeMaps;
bool pipe2d_supported(const StepParams &P, int map_kind);
bool pipe2d_preferred(const StepParams &P, int map_kind);
// encode the tensor maps of both half steps (host); cudaErrorInvalidValue
// when the driver rejects one (message in *why)
cudaError_t build_pipe2d_maps(const StepParams &P, int map_kind, PipeMaps *vel, PipeMaps *prs, const char **why);
cudaError_t launch_pipe2d(bool vel, const StepParams &P, int map_kind, int grid, const PipeMaps &T,
                          cudaStream_t s);
// batched form over a unit table {ctx, x0, y0, interior} of 128 x 8 half
// tiles (no periodic context); Ps and Ts in device memory, one per context;
// block b takes the units runs[b] .. runs[b + 1] - 1 (grid + 1 entries)
constexpr int kPipeHalf = 8;  // rows of a pipelined half tile
bool pipe2d_interior_half(const StepParams &P, int x0, int y0);
cudaError_t launch_pipe2d_batched(bool vel, const StepParams *Ps, const PipeMaps *Ts, const int4 *units,
                                  int n_units, const int *runs, int n_relax, int map_kind, int grid,
                                  cudaStream_t s);
// persistent pipelined 3D half step (bf16 maps, N <= 3, no periodic axis),
// in one of two layouts that compute the same result: the memory variables
// staged in shared memory with the other arrays (kLayoutStaged; not with
// cross taps, nor for the literal system's velocity half step), or loaded
// into registers one unit ahead with every C-PML strip staged
// (kLayoutRegisters); kLayoutDefault takes the staged one where it applies
constexpr int kLayoutDefault = 0, kLayoutStaged = 1, kLayoutRegisters = 2;
bool pipe3d_supported(const StepParams &P, int map_kind);
bool pipe3d_layout_allowed(bool vel, const StepParams &P, int layout);
cudaError_t build_pipe3d_maps(const StepParams &P, PipeMaps *vel, PipeMaps *prs, const char **why);
cudaError_t launch_pipe3d(bool vel, const StepParams &P, int grid, const PipeMaps &T, cudaStream_t s,
                          int layout = kLayoutDefault);
// batched form: per context the parameters, the work layout (an opaque
// record of pipe3d_region_bytes(), written by pipe3d_region, which returns
// the context's item count) and the tensor maps, in device memory; items
// {context, item}; the layout of every context is the default one
// (pipe3d_staged_layout), which must agree within a launch
size_t pipe3d_region_bytes();
long long pipe3d_region(const StepParams &P, int grid, bool vel, void *out);
// edge units of each of the context's items (n_edge) and units per item
// (n_all), arrays of the item count pipe3d_region returns
void pipe3d_item_units(const StepParams &P, int grid, bool vel, int *n_edge, int *n_all);
bool pipe3d_staged_layout(bool vel, const StepParams &P);
// block b takes the items runs[b] .. runs[b + 1] - 1 (grid + 1 entries)
cudaError_t launch_pipe3d_batched(bool vel, bool cross, bool ps, int n_relax, const StepParams *Ps,
                                  const void *Rs, const PipeMaps *Ts, const int2 *items, const int *runs,
                                  int grid, cudaStream_t s);
// 3D tile kernels: map_kind 0 float, 1 bf16, 4 FP16, 2 and 3 the uint8 and
// uint16 tissue index (tables read through L2)
cudaError_t launch_vel3d(const StepParams &P, int map_kind, cudaStream_t s);
cudaError_t launch_prs3d(const StepParams &P, int map_kind, cudaStream_t s);
cudaError_t launch_vel3d_wide(const StepParams &P, int map_kind, cudaStream_t s);
cudaError_t launch_prs3d_wide(const StepParams &P, int map_kind, cudaStream_t s);

}  // namespace fw2
