// 2D fused velocity and pressure half steps (sm_103a): one block per
// 128 x 16 tile (tile2d.cuh), and the persistent batched form that walks a
// tile table of several contexts.
#include <type_traits>

#include "tile2d.cuh"

namespace fw2 {

namespace {

template <int N, typename Maps>
__global__ void __launch_bounds__(256, 2) vel2d_kernel(const StepParams P) {
  __shared__ __align__(16) float sp[kPH][kPW];
  __shared__ __align__(16) float sr[kRH][kRW];
  __shared__ __align__(16) float stab[Maps::kSmemFloats];
  vel2d_tile<N, Maps>(P, blockIdx.x * kTX, blockIdx.y * kTY, sp, sr, stab, true);
}

template <int N, typename Maps>
__global__ void __launch_bounds__(256, 2) prs2d_kernel(const StepParams P) {
  __shared__ __align__(16) float svx[kHX][kPW];
  __shared__ __align__(16) float svy[kHY][kPW];
  __shared__ __align__(16) float stab[Maps::kSmemFloats];
  prs2d_tile<N, Maps>(P, blockIdx.x * kTX, blockIdx.y * kTY, svx, svy, stab, true);
}

// Persistent batched half steps: blocks walk the tile table round-robin;
// entry (ctx, x0, y0).  The context's parameter block is copied to shared
// memory when the context changes (the table stays staged with it).
__device__ __forceinline__ bool load_ctx(const StepParams *Ps, int ctx, StepParams *sP, int *cur) {
  if (*cur == ctx) return false;
  __syncthreads();
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int *src = reinterpret_cast<const int *>(Ps + ctx);
  int *dst = reinterpret_cast<int *>(sP);
  for (int w = tid; w < (int)(sizeof(StepParams) / 4); w += 256) dst[w] = __ldg(src + w);
  __syncthreads();
  *cur = ctx;
  return true;
}

template <int N, typename Maps>
__global__ void __launch_bounds__(256, 2) vel2d_batched(const StepParams *Ps, const int4 *tiles, int n_tiles) {
  __shared__ __align__(16) float sp[kPH][kPW];
  __shared__ __align__(16) float sr[kRH][kRW];
  __shared__ __align__(16) float stab[Maps::kSmemFloats];
  __shared__ __align__(16) StepParams sP;
  int cur = -1;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int4 e = tiles[t];
    const bool fresh = load_ctx(Ps, e.x, &sP, &cur);
    vel2d_tile<N, Maps>(sP, e.y, e.z, sp, sr, stab, fresh);
    __syncthreads();
  }
}

template <int N, typename Maps>
__global__ void __launch_bounds__(256, 2) prs2d_batched(const StepParams *Ps, const int4 *tiles, int n_tiles) {
  __shared__ __align__(16) float svx[kHX][kPW];
  __shared__ __align__(16) float svy[kHY][kPW];
  __shared__ __align__(16) float stab[Maps::kSmemFloats];
  __shared__ __align__(16) StepParams sP;
  int cur = -1;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int4 e = tiles[t];
    const bool fresh = load_ctx(Ps, e.x, &sP, &cur);
    prs2d_tile<N, Maps>(sP, e.y, e.z, svx, svy, stab, fresh);
    __syncthreads();
  }
}

// The mechanism counts this compilation instantiates: 0..4, or 5..8 when
// built with FW2_WIDE_RELAX (the second object of this file).
#ifdef FW2_WIDE_RELAX
constexpr int kNLo = 5, kNHi = kMaxRelax;
#else
constexpr int kNLo = 0, kNHi = 4;
#endif

// tissue-index tables hold kTabSlots mechanisms
template <int N, typename Maps>
constexpr bool kHasN = !((std::is_same<Maps, IdxMaps>::value || std::is_same<Maps, IdxMaps16>::value) &&
                         N > kTabSlots);

template <int N, typename Maps>
cudaError_t vel2d_at(const StepParams &P, dim3 g, dim3 b, cudaStream_t s) {
  if constexpr (N > kNHi) {
    return cudaErrorInvalidValue;
  } else {
    if (P.n_relax != N) return vel2d_at<N + 1, Maps>(P, g, b, s);
    if constexpr (!kHasN<N, Maps>) return cudaErrorInvalidValue;
    else vel2d_kernel<N, Maps><<<g, b, 0, s>>>(P);
    return cudaGetLastError();
  }
}

template <int N, typename Maps>
cudaError_t prs2d_at(const StepParams &P, dim3 g, dim3 b, cudaStream_t s) {
  if constexpr (N > kNHi) {
    return cudaErrorInvalidValue;
  } else {
    if (P.n_relax != N) return prs2d_at<N + 1, Maps>(P, g, b, s);
    if constexpr (!kHasN<N, Maps>) return cudaErrorInvalidValue;
    else prs2d_kernel<N, Maps><<<g, b, 0, s>>>(P);
    return cudaGetLastError();
  }
}

template <int N, typename Maps>
cudaError_t batched_at(bool vel, const StepParams *Ps, const int4 *tiles, int n_tiles, int n_relax, int grid,
                       cudaStream_t s) {
  if constexpr (N > kNHi) {
    return cudaErrorInvalidValue;
  } else {
    if (n_relax != N) return batched_at<N + 1, Maps>(vel, Ps, tiles, n_tiles, n_relax, grid, s);
    if constexpr (!kHasN<N, Maps>) {
      return cudaErrorInvalidValue;
    } else {
      const dim3 b(32, kBY);
      if (vel) vel2d_batched<N, Maps><<<grid, b, 0, s>>>(Ps, tiles, n_tiles);
      else prs2d_batched<N, Maps><<<grid, b, 0, s>>>(Ps, tiles, n_tiles);
    }
    return cudaGetLastError();
  }
}

template <typename Maps>
cudaError_t vel2d_dispatch(const StepParams &P, dim3 g, dim3 b, cudaStream_t s) {
  return vel2d_at<kNLo, Maps>(P, g, b, s);
}
template <typename Maps>
cudaError_t prs2d_dispatch(const StepParams &P, dim3 g, dim3 b, cudaStream_t s) {
  return prs2d_at<kNLo, Maps>(P, g, b, s);
}
template <typename Maps>
cudaError_t batched_dispatch(bool vel, const StepParams *Ps, const int4 *tiles, int n_tiles, int n_relax, int grid,
                             cudaStream_t s) {
  return batched_at<kNLo, Maps>(vel, Ps, tiles, n_tiles, n_relax, grid, s);
}

}  // namespace

#ifdef FW2_WIDE_RELAX
cudaError_t launch_vel2d_wide(const StepParams &P, int map_kind, cudaStream_t s) {
#else
cudaError_t launch_vel2d(const StepParams &P, int map_kind, cudaStream_t s) {
  if (P.n_relax > kNHi) return launch_vel2d_wide(P, map_kind, s);
#endif
  dim3 g((P.nx + kTX - 1) / kTX, (P.ny + kTY - 1) / kTY), b(32, kBY);
  if (map_kind == 2) return vel2d_dispatch<IdxMaps>(P, g, b, s);
  if (map_kind == 3) return vel2d_dispatch<IdxMaps16>(P, g, b, s);
  if (map_kind == 4) return vel2d_dispatch<DenseMaps<__half>>(P, g, b, s);
  return map_kind ? vel2d_dispatch<DenseMaps<__nv_bfloat16>>(P, g, b, s) : vel2d_dispatch<DenseMaps<float>>(P, g, b, s);
}

#ifdef FW2_WIDE_RELAX
cudaError_t launch_prs2d_wide(const StepParams &P, int map_kind, cudaStream_t s) {
#else
cudaError_t launch_prs2d(const StepParams &P, int map_kind, cudaStream_t s) {
  if (P.n_relax > kNHi) return launch_prs2d_wide(P, map_kind, s);
#endif
  dim3 g((P.nx + kTX - 1) / kTX, (P.ny + kTY - 1) / kTY), b(32, kBY);
  if (map_kind == 2) return prs2d_dispatch<IdxMaps>(P, g, b, s);
  if (map_kind == 3) return prs2d_dispatch<IdxMaps16>(P, g, b, s);
  if (map_kind == 4) return prs2d_dispatch<DenseMaps<__half>>(P, g, b, s);
  return map_kind ? prs2d_dispatch<DenseMaps<__nv_bfloat16>>(P, g, b, s) : prs2d_dispatch<DenseMaps<float>>(P, g, b, s);
}

#ifdef FW2_WIDE_RELAX
cudaError_t launch_batched2d_wide(bool vel, const StepParams *Ps, const int4 *tiles, int n_tiles, int n_relax,
                                  int map_kind, int grid, cudaStream_t s) {
#else
cudaError_t launch_batched2d(bool vel, const StepParams *Ps, const int4 *tiles, int n_tiles, int n_relax,
                             int map_kind, int grid, cudaStream_t s) {
  if (n_relax > kNHi) return launch_batched2d_wide(vel, Ps, tiles, n_tiles, n_relax, map_kind, grid, s);
#endif
  if (n_tiles <= 0) return cudaSuccess;
  if (map_kind == 2) return batched_dispatch<IdxMaps>(vel, Ps, tiles, n_tiles, n_relax, grid, s);
  if (map_kind == 3) return batched_dispatch<IdxMaps16>(vel, Ps, tiles, n_tiles, n_relax, grid, s);
  if (map_kind == 1) return batched_dispatch<DenseMaps<__nv_bfloat16>>(vel, Ps, tiles, n_tiles, n_relax, grid, s);
  if (map_kind == 4) return batched_dispatch<DenseMaps<__half>>(vel, Ps, tiles, n_tiles, n_relax, grid, s);
  return batched_dispatch<DenseMaps<float>>(vel, Ps, tiles, n_tiles, n_relax, grid, s);
}

}  // namespace fw2
