// Internal definition of a context (shared by api.cu and batch.cu).
#pragma once
#include <string>
#include <vector>

#include "fw2.h"
#include "fw2_prep.cuh"
#include "maps.cuh"
#include "tmap.h"

namespace fw2 {

struct HostSource {
  int kind;
  std::vector<long long> idx;   // flat dense cell index
  std::vector<int> group;
  std::vector<float> signal;    // [n_steps][n_groups]
  long long n_groups = 0, n_steps = 0;
};

struct DevSource {
  long long *tgt = nullptr;
  int *off = nullptr;
  int *col = nullptr;
  int n_tgt = 0;
};

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace fw2

struct fw2_ctx {
  using HostSource = fw2::HostSource;
  using DevSource = fw2::DevSource;
  using StepParams = fw2::StepParams;
  fw2_config cfg;
  int nd = 2, N = 0, nx = 1, ny = 1, nz = 1, pitch = 4;
  long long plane = 0, npts_alloc = 0, n_pts = 0;
  cudaStream_t stream = nullptr;
  std::string err = "no error";
  // device memory
  std::vector<void *> allocs;
  long long dev_bytes = 0;
  char *state = nullptr;
  size_t state_bytes = 0;
  float *p = nullptr, *v[3] = {nullptr, nullptr, nullptr};
  float *psi1[3] = {nullptr, nullptr, nullptr}, *psi2[3] = {nullptr, nullptr, nullptr};
  // raw inputs (device, dense)
  float *raw_c = nullptr, *raw_rho = nullptr, *raw_beta = nullptr;
  float *raw_k1 = nullptr, *raw_k2 = nullptr, *raw_d1 = nullptr, *raw_al1 = nullptr, *raw_d2 = nullptr,
        *raw_al2 = nullptr;
  void *raw_tissue = nullptr;  // tissue-index form (uint8 or uint16 per cell)
  float map_scale[fw2::kMapScales] = {};  // FP16 maps: value = stored x scale
  int n_tissue = 0;
  bool medium_set = false, relax_set = false, finalized = false;
  // coefficient maps
  char *maps = nullptr;
  StepParams P{};
  int map_kind = 0;  // FW2_MAP_*
  int n_sm = 152;    // multiprocessors of the device
  bool pipe = false; // 2D half steps by the pipelined kernels
  fw2::PipeMaps tm_vel{}, tm_prs{};  // their tensor maps
  double dt = 0.0, cmax_eff = 0.0, cmax = 0.0;
  // sources
  std::vector<HostSource> sources;
  bool src_dirty = false;
  DevSource dsrc[4];
  float *d_signal = nullptr;
  long long sig_steps = 0, sig_cols = 0;
  // recording
  long long *rec_cell = nullptr;
  int *rec_off = nullptr;
  int rec_groups = 0;
  float *rec_out = nullptr;
  long long rec_steps = 0;
  // scratch words for scans
  unsigned long long *d_scan = nullptr;
  int *d_bad = nullptr;
  unsigned int *d_absmax = nullptr;
  unsigned int *d_status = nullptr;  // bit 0: a bounded device-side wait gave up
  long long step = 0, launches = 0;
  // optional per-kernel event timing
  bool profiling = false;
  // 3D pipelined layout per half step (velocity, pressure), chosen by timing
  // both on the first steps: 0 until then, else kLayoutStaged / kLayoutRegisters
  int layout3[2] = {0, 0};
  int layout_trial = 0;
  float layout_ms[2][2] = {{0.f, 0.f}, {0.f, 0.f}};  // [layout - 1][half]
  // subdomain of a larger grid (fw2_set_subdomain): its extent and this
  // context's offset along each axis; half = 1 between the two parts of a
  // step taken with fw2_step_part
  bool subdomain = false;
  long long gext[3] = {0, 0, 0}, goff[3] = {0, 0, 0};
  int half = 0;
  // in-loop blow-up detection: scan p every watch_every steps (0: off)
  long long watch_every = 0;
  float watch_bound = 0.f;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_vel, ev_prs;
};


namespace fw2 {
// finalize the coefficient maps and upload pending sources (status; the
// message goes to the context)
fw2_status ctx_prepare(fw2_ctx *c);
fw2_status ctx_fail(fw2_ctx *c, fw2_status s, const char *msg);
}  // namespace fw2
