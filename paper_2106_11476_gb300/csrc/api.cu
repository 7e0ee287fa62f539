// C ABI of libfw2 (declared in include/fw2.h): context management, input
// validation and staging, device coefficient build, the time-step loop.
#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

using namespace fw2;

namespace {
thread_local std::string g_create_error = "no error";
}

namespace fw2 {
// error text of calls without a context (fw2_last_error(NULL))
void set_global_error(const char *msg) { g_create_error = msg; }
}  // namespace fw2

namespace {

fw2_status fail(fw2_ctx *c, fw2_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_create_error = buf;
  return s;
}

fw2_status cuda_fail(fw2_ctx *c, cudaError_t e, const char *what) {
  return fail(c, e == cudaErrorMemoryAllocation ? FW2_ENOMEM : FW2_ECUDA, "%s: %s (%s)", what,
              cudaGetErrorString(e), cudaGetErrorName(e));
}

#define CK(ctx, call)                                       \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

// Device memory of the contexts comes from a stream-ordered pool the library
// owns, one per device: what a destroyed context (or a finished coefficient
// build) returns stays in the pool for the next allocation of the process
// instead of going back to the driver, so contexts created one after another
// (the transmit events of a sequence, served requests) do not map fresh
// memory each time.  fw2_release_memory hands the pool's free memory back.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaError_t pool_of_current_device(cudaMemPool_t *pool) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  if (!g_pool[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    unsigned long long keep = ~0ull;  // keep freed memory for reuse
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return e;
    }
    g_pool[dev] = p;
  }
  *pool = g_pool[dev];
  return cudaSuccess;
}

fw2_status dalloc(fw2_ctx *c, size_t bytes, void **out) {
  *out = nullptr;
  if (bytes == 0) bytes = 256;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = pool_of_current_device(&pool);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(out, bytes, pool, c->stream);
  if (e != cudaSuccess) {
    *out = nullptr;
    return fail(c, FW2_ENOMEM, "allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  c->allocs.push_back(*out);
  c->dev_bytes += (long long)bytes;
  return FW2_OK;
}

// returned to the pool in stream order: work already queued on the context
// stream that reads the buffer completes first
void dfree(fw2_ctx *c, void *p) {
  if (!p) return;
  auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
  if (it != c->allocs.end()) c->allocs.erase(it);
  cudaFreeAsync(p, c->stream);
}

// copy n floats (or other POD) from host or device into a device buffer
fw2_status copy_in(fw2_ctx *c, void *dst, const void *src, size_t bytes, int mem_space) {
  if (bytes == 0) return FW2_OK;
  if (!src) return fail(c, FW2_EINVAL, "null input pointer");
  const cudaMemcpyKind kind = mem_space == FW2_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(c, cudaMemcpyAsync(dst, src, bytes, kind, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return FW2_OK;
}

// copy an input array to host memory (for index lists)
template <typename T>
fw2_status copy_to_host(fw2_ctx *c, std::vector<T> &out, const T *src, size_t n, int mem_space) {
  out.resize(n);
  if (n == 0) return FW2_OK;
  if (!src) return fail(c, FW2_EINVAL, "null index pointer");
  if (mem_space == FW2_MEM_DEVICE) {
    CK(c, cudaMemcpyAsync(out.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
  } else {
    std::memcpy(out.data(), src, n * sizeof(T));
  }
  return FW2_OK;
}

long long to_pitched(const fw2_ctx *c, long long flat) {
  const long long i = flat % c->nx;
  const long long r = flat / c->nx;
  const long long j = r % c->ny;
  const long long k = r / c->ny;
  return k * c->plane + j * c->pitch + i;
}

double taps_abs_sum(const fw2_config &cfg) {
  double s = 0.0;
  for (int i = 0; i < 4; ++i) s += std::fabs(cfg.g[i]);
  return s;
}

fw2_status finalize(fw2_ctx *c) {
  if (c->finalized) return FW2_OK;
  if (!c->medium_set) return fail(c, FW2_ESTATE, "fw2_set_medium must be called before stepping");
  if (c->N > 0 && !c->relax_set) return fail(c, FW2_ESTATE, "fw2_set_relaxation is required when n_relax > 0");
  const fw2_config &cfg = c->cfg;
  PrepParams Q{};
  Q.nx = c->nx; Q.ny = c->ny; Q.nz = c->nz; Q.nd = c->nd; Q.pitch = c->pitch;
  Q.plane = c->plane; Q.npts_alloc = c->npts_alloc; Q.N = c->N;
  Q.c = c->raw_c; Q.rho = c->raw_rho; Q.beta = c->raw_beta;
  Q.k1 = c->raw_k1; Q.k2 = c->raw_k2; Q.d1 = c->raw_d1; Q.al1 = c->raw_al1; Q.d2 = c->raw_d2; Q.al2 = c->raw_al2;
  Q.nl_mode = cfg.nl_mode;
  const long long ext[3] = {c->nx, c->ny, c->nz};
  for (int q = 0; q < 3; ++q) {
    Q.gext[q] = (int)(c->subdomain ? c->gext[q] : ext[q]);
    Q.goff[q] = (int)(c->subdomain ? c->goff[q] : 0);
  }
  const bool indexed = c->map_kind == FW2_MAP_IDX_U8 || c->map_kind == FW2_MAP_IDX_U16;
  const bool wide = c->map_kind == FW2_MAP_IDX_U16;
  Q.tissue_in = indexed ? c->raw_tissue : nullptr;
  Q.tissue_wide = wide ? 1 : 0;
  Q.n_tissue = c->n_tissue;
  // table field stride: 256 for the uint8 form (its kernels stage the table
  // at that stride), the tissue count rounded up to 4 for the uint16 form
  Q.tab_stride = wide ? (c->n_tissue + 3) / 4 * 4 : kTissues;
  // medium scan: c_max (high-frequency) and validity
  CK(c, cudaMemsetAsync(c->d_scan, 0, 2 * sizeof(unsigned long long), c->stream));
  CK(c, cudaMemsetAsync(c->d_bad, 0, sizeof(int), c->stream));
  CK(c, launch_medium_scan(Q, c->d_scan, c->d_bad, c->stream));
  c->launches++;
  unsigned long long mx[2];
  int bad = 0;
  CK(c, cudaMemcpyAsync(mx, c->d_scan, sizeof mx, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(&bad, c->d_bad, sizeof bad, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (bad) return fail(c, FW2_EINVAL, "%d cells have non-positive or non-finite c, rho, kappa or beta", bad);
  double ce, cm;
  std::memcpy(&ce, &mx[0], 8);
  std::memcpy(&cm, &mx[1], 8);
  c->cmax_eff = ce;
  c->cmax = cm;
  c->dt = cfg.dt > 0.0 ? cfg.dt : cfg.cfl * cfg.h / ce;
  // stability of the leapfrog staggered scheme: (c dt / h) sqrt(nd) (sum |g| + 2 |g11| (nd - 1)) <= 1
  const double bound = taps_abs_sum(cfg) + 2.0 * std::fabs(cfg.g[4]) * (c->nd - 1);
  const double courant = ce * c->dt / cfg.h * std::sqrt((double)c->nd) * bound;
  if (!(courant <= 1.0))
    return fail(c, FW2_EINVAL, "time step %.6g s exceeds the stability limit (Courant factor %.4f > 1)", c->dt, courant);
  Q.dt = c->dt;
  const int L = cfg.pml_transition + cfg.pml_bound;
  Q.LT = cfg.pml_transition; Q.LB = cfg.pml_bound; Q.reading = cfg.pml_reading; Q.npow = cfg.pml_npow;
  const double cp = cfg.pml_cp > 0.0 ? cfg.pml_cp : cm;
  Q.d_target = L > 0 ? -(cfg.pml_npow + 1.0) * cp * std::log(cfg.pml_rc) / (2.0 * L * cfg.h) : 0.0;
  // map allocation: 5 cell maps + 4N interior + strips (dense forms), or the
  // per-tissue table + the pitched index + strips (index form)
  const size_t es = (c->map_kind == FW2_MAP_BF16 || c->map_kind == FW2_MAP_F16) ? 2 : 4;
  const size_t cell_bytes = indexed ? 0 : align256(es * (size_t)c->npts_alloc);
  long long strip_nu[3] = {0, 0, 0};
  const bool strips = L > 0 && c->N > 0;
  if (strips) {
    strip_nu[0] = (long long)c->nz * c->ny * 2 * L;
    strip_nu[1] = (long long)c->nz * 2 * L * c->pitch;
    if (c->nd == 3) strip_nu[2] = (long long)2 * L * c->ny * c->pitch;
  }
  const size_t table_bytes = indexed ? align256(sizeof(float) * kTableFields * (size_t)Q.tab_stride) : 0;
  const size_t index_bytes = indexed ? align256((wide ? 2 : 1) * (size_t)c->npts_alloc) : 0;
  size_t total = 5 * cell_bytes + 4 * (size_t)c->N * cell_bytes + table_bytes + index_bytes;
  size_t strip_bytes[3];
  for (int q = 0; q < 3; ++q) {
    strip_bytes[q] = align256(es * (size_t)(strip_nu[q] * (c->N ? c->N : 1)));
    if (strip_nu[q]) total += 4 * strip_bytes[q];
  }
  if (c->maps) {
    dfree(c, c->maps);
    c->maps = nullptr;
  }
  void *m;
  fw2_status st = dalloc(c, total, &m);
  if (st != FW2_OK) return st;
  c->maps = (char *)m;
  CK(c, cudaMemsetAsync(c->maps, 0, total, c->stream));
  char *cur = c->maps;
  auto take = [&](size_t b) { char *r = cur; cur += b; return (void *)r; };
  Q.table_out = indexed ? (float *)take(table_bytes) : nullptr;
  Q.tissue_out = indexed ? take(index_bytes) : nullptr;
  Q.K = take(cell_bytes); Q.rho_o = take(cell_bytes); Q.chi = take(cell_bytes);
  Q.ik1 = take(cell_bytes); Q.ik2 = take(cell_bytes);
  const size_t iso = (size_t)c->N * cell_bytes;
  Q.a1 = take(iso); Q.b1 = take(iso); Q.a2 = take(iso); Q.b2 = take(iso);
  for (int q = 0; q < 3; ++q) {
    Q.strip_nu[q] = strip_nu[q];
    if (strip_nu[q]) {
      Q.sa1[q] = take(strip_bytes[q]); Q.sb1[q] = take(strip_bytes[q]);
      Q.sa2[q] = take(strip_bytes[q]); Q.sb2[q] = take(strip_bytes[q]);
    }
  }
  // FP16 maps: a scan pass for the largest magnitude of every map, then a
  // power-of-two scale per map that puts it in [2^14, 2^15)
  float scale[kMapScales];
  for (int m = 0; m < kMapScales; ++m) {
    scale[m] = 1.f;
    Q.inv_scale[m] = 1.0;
  }
  if (c->map_kind == FW2_MAP_F16) {
    void *mb;
    fw2_status sm = dalloc(c, sizeof(unsigned int) * kMapScales, &mb);
    if (sm != FW2_OK) return sm;
    Q.f16_max = static_cast<unsigned int *>(mb);
    unsigned int bits[kMapScales];
    cudaError_t e = cudaMemsetAsync(mb, 0, sizeof bits, c->stream);
    if (e == cudaSuccess) e = launch_prep_scan(Q, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bits, mb, sizeof bits, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, mb);
    Q.f16_max = nullptr;
    CK(c, e);
    c->launches += 1 + (strips ? c->nd : 0);
    for (int m = 0; m < kMapScales; ++m) {
      float mx;
      std::memcpy(&mx, &bits[m], 4);
      if (mx > 0.f && std::isfinite(mx)) {
        int ex;
        std::frexp((double)mx, &ex);             // mx in [2^(ex-1), 2^ex)
        scale[m] = (float)std::ldexp(1.0, ex - 15);  // mx / scale in [2^14, 2^15)
        Q.inv_scale[m] = std::ldexp(1.0, 15 - ex);
      }
    }
  }
  for (int m = 0; m < kMapScales; ++m) c->map_scale[m] = scale[m];
  CK(c, launch_prep(Q, c->map_kind, c->stream));
  c->launches += (indexed ? 2 : 1) + (strips ? c->nd : 0);
  CK(c, cudaStreamSynchronize(c->stream));
  // raw inputs are no longer needed
  float **raws[] = {&c->raw_c, &c->raw_rho, &c->raw_beta, &c->raw_k1, &c->raw_k2,
                    &c->raw_d1, &c->raw_al1, &c->raw_d2, &c->raw_al2};
  for (float **r : raws) {
    dfree(c, *r);
    *r = nullptr;
  }
  dfree(c, c->raw_tissue);
  c->raw_tissue = nullptr;
  c->medium_set = c->relax_set = false;
  // step parameters
  StepParams &P = c->P;
  P = StepParams{};
  P.nx = c->nx; P.ny = c->ny; P.nz = c->nz; P.pitch = c->pitch; P.plane = c->plane; P.npts_alloc = c->npts_alloc;
  for (int q = 0; q < 3; ++q) {
    P.L[q] = (strips && q < c->nd) ? L : 0;
    P.periodic[q] = q < c->nd ? (cfg.bc[q] == FW2_BC_PERIODIC) : 0;
    P.strip_nu[q] = strip_nu[q];
    P.sa1[q] = Q.sa1[q]; P.sb1[q] = Q.sb1[q]; P.sa2[q] = Q.sa2[q]; P.sb2[q] = Q.sb2[q];
    P.v[q] = c->v[q]; P.psi1[q] = c->psi1[q]; P.psi2[q] = c->psi2[q];
  }
  P.dt = (float)c->dt;
  P.two_dt = (float)(2.0 * c->dt);
  for (int i = 0; i < 4; ++i) P.gh[i] = (float)(cfg.g[i] / cfg.h);
  P.g11h = (float)(cfg.g[4] / cfg.h);
  if (cfg.mem_alignment == FW2_MEM_CENTRED) { P.w_new = 0.5f; P.w_old = 0.5f; }
  else { P.w_new = 1.0f; P.w_old = 0.0f; }
  P.nl = cfg.nl_mode != FW2_NL_OFF;
  P.nl_vel = cfg.nl_mode == FW2_NL_LITERAL;
  P.n_relax = c->N;
  P.p = c->p;
  P.K = Q.K; P.rho = Q.rho_o; P.chi = Q.chi; P.ik1 = Q.ik1; P.ik2 = Q.ik2;
  P.a1 = Q.a1; P.b1 = Q.b1; P.a2 = Q.a2; P.b2 = Q.b2;
  P.tissue = static_cast<const unsigned char *>(Q.tissue_out);
  P.table = Q.table_out;
  P.tab_stride = Q.tab_stride;
  for (int m = 0; m < kMapScales; ++m) P.ms[m] = c->map_scale[m];
  P.status = c->d_status;
  const bool forced_pipe = cfg.kernel_path >= FW2_PATH_PIPE;
  if (c->nd == 2)
    c->pipe = (cfg.kernel_path == FW2_PATH_AUTO && pipe2d_preferred(P, c->map_kind)) ||
              (forced_pipe && pipe2d_supported(P, c->map_kind));
  else
    c->pipe = cfg.kernel_path != FW2_PATH_TILE && pipe3d_supported(P, c->map_kind);
  if (c->nd == 3 && c->pipe && (cfg.kernel_path == FW2_PATH_PIPE_STAGED || cfg.kernel_path == FW2_PATH_PIPE_REGISTERS)) {
    const int l = cfg.kernel_path == FW2_PATH_PIPE_STAGED ? kLayoutStaged : kLayoutRegisters;
    c->layout3[0] = pipe3d_layout_allowed(true, P, l) ? l : kLayoutRegisters;
    c->layout3[1] = pipe3d_layout_allowed(false, P, l) ? l : kLayoutRegisters;
  }
  if (c->pipe) {
    const char *why = "";
    const cudaError_t e = c->nd == 2 ? build_pipe2d_maps(P, c->map_kind, &c->tm_vel, &c->tm_prs, &why)
                                     : build_pipe3d_maps(P, &c->tm_vel, &c->tm_prs, &why);
    if (e != cudaSuccess) return fail(c, FW2_ECUDA, "tensor maps of the pipelined kernels: %s", why);
  }
  c->finalized = true;
  return FW2_OK;
}

fw2_status build_sources(fw2_ctx *c) {
  if (!c->src_dirty) return FW2_OK;
  for (DevSource &d : c->dsrc) {
    dfree(c, d.tgt); dfree(c, d.off); dfree(c, d.col);
    d = DevSource{};
  }
  dfree(c, c->d_signal);
  c->d_signal = nullptr;
  long long cols = 0, steps = 0;
  for (const HostSource &s : c->sources) {
    cols += s.n_groups;
    steps = std::max(steps, s.n_steps);
  }
  c->sig_cols = cols;
  c->sig_steps = steps;
  if (cols > 0 && steps > 0) {
    std::vector<float> table((size_t)(cols * steps), 0.f);
    long long base = 0;
    for (const HostSource &s : c->sources) {
      for (long long n = 0; n < s.n_steps; ++n)
        for (long long g = 0; g < s.n_groups; ++g)
          table[(size_t)(n * cols + base + g)] = s.signal[(size_t)(n * s.n_groups + g)];
      base += s.n_groups;
    }
    void *m;
    fw2_status st = dalloc(c, table.size() * sizeof(float), &m);
    if (st != FW2_OK) return st;
    c->d_signal = (float *)m;
    CK(c, cudaMemcpyAsync(c->d_signal, table.data(), table.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
  }
  for (int kind = 0; kind < 4; ++kind) {
    struct E { long long tgt; int col; long long order; };
    std::vector<E> es;
    long long base = 0, order = 0;
    for (const HostSource &s : c->sources) {
      if (s.kind == kind)
        for (size_t e = 0; e < s.idx.size(); ++e) es.push_back({to_pitched(c, s.idx[e]), (int)(base + s.group[e]), order++});
      base += s.n_groups;
    }
    if (es.empty()) continue;
    std::stable_sort(es.begin(), es.end(), [](const E &a, const E &b) { return a.tgt < b.tgt; });
    std::vector<long long> tgt;
    std::vector<int> off, col;
    for (size_t e = 0; e < es.size(); ++e) {
      if (e == 0 || es[e].tgt != es[e - 1].tgt) {
        tgt.push_back(es[e].tgt);
        off.push_back((int)col.size());
      }
      col.push_back(es[e].col);
    }
    off.push_back((int)col.size());
    DevSource &d = c->dsrc[kind];
    void *m;
    fw2_status st;
    if ((st = dalloc(c, tgt.size() * sizeof(long long), &m)) != FW2_OK) return st;
    d.tgt = (long long *)m;
    if ((st = dalloc(c, off.size() * sizeof(int), &m)) != FW2_OK) return st;
    d.off = (int *)m;
    if ((st = dalloc(c, col.size() * sizeof(int), &m)) != FW2_OK) return st;
    d.col = (int *)m;
    d.n_tgt = (int)tgt.size();
    CK(c, cudaMemcpyAsync(d.tgt, tgt.data(), tgt.size() * sizeof(long long), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(d.off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaMemcpyAsync(d.col, col.data(), col.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
  }
  c->src_dirty = false;
  return FW2_OK;
}

cudaEvent_t take_event(fw2_ctx *c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void release_events(fw2_ctx *c) {
  for (auto &pr : c->ev_vel) { c->ev_pool.push_back(pr.first); c->ev_pool.push_back(pr.second); }
  for (auto &pr : c->ev_prs) { c->ev_pool.push_back(pr.first); c->ev_pool.push_back(pr.second); }
  c->ev_vel.clear();
  c->ev_prs.clear();
}

float *field_ptr(fw2_ctx *c, int field, int *count) {
  *count = 1;
  if (field == FW2_FIELD_P) return c->p;
  if (field >= FW2_FIELD_VX && field <= FW2_FIELD_VZ) {
    int q = field - FW2_FIELD_VX;
    return q < c->nd ? c->v[q] : nullptr;
  }
  if (field >= FW2_FIELD_PSI1X && field <= FW2_FIELD_PSI2Z) {
    const bool one = field <= FW2_FIELD_PSI1Z;
    const int q = one ? field - FW2_FIELD_PSI1X : field - FW2_FIELD_PSI2X;
    if (q >= c->nd || c->N == 0) return nullptr;
    *count = c->N;
    return one ? c->psi1[q] : c->psi2[q];
  }
  return nullptr;
}

}  // namespace

namespace fw2 {
fw2_status ctx_prepare(fw2_ctx *c) {
  fw2_status st = finalize(c);
  if (st != FW2_OK) return st;
  return build_sources(c);
}
fw2_status ctx_fail(fw2_ctx *c, fw2_status s, const char *msg) { return fail(c, s, "%s", msg); }

// Layout of the 3D pipelined half steps for the next step: the tuned one,
// or during the first four steps of a context the trial one (two steps per
// layout, the second timed); *timed tells whether to time this step.
int layout_for_step(fw2_ctx *c, bool *timed) {
  *timed = false;
  if (c->nd != 3 || !c->pipe || c->layout3[0] != 0) return -1;
  const bool choice = pipe3d_layout_allowed(true, c->P, kLayoutStaged) ||
                      pipe3d_layout_allowed(false, c->P, kLayoutStaged);
  if (!choice) {  // only the register layout applies
    c->layout3[0] = c->layout3[1] = kLayoutRegisters;
    return -1;
  }
  const int t = c->layout_trial;
  *timed = t == 1 || t == 3;
  return t < 2 ? kLayoutStaged : kLayoutRegisters;
}

// Enqueue the launches of time step n (Sec. 3.1 order): velocity half step,
// velocity sources (part 0), pressure half step, pressure sources,
// recording (part 1); part -1 enqueues both, and only whole steps take part
// in the choice of the 3D layout.
fw2_status enqueue_step(fw2_ctx *c, long long n, int part = -1) {
  const StepParams &P = c->P;
  bool trial_timed = false;
  const int trial = part < 0 ? layout_for_step(c, &trial_timed) : -1;
  auto lay = [&](bool vel) {
    const int l = trial > 0 ? trial : c->layout3[vel ? 0 : 1];
    if (l == 0) return kLayoutDefault;
    return pipe3d_layout_allowed(vel, P, l) ? l : kLayoutRegisters;
  };
  const bool do_vel = part != 1, do_prs = part != 0;
  struct TrialEvents {  // destroyed on every return, error paths included
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
    ~TrialEvents() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
  } trial_ev;
  cudaEvent_t *te = trial_ev.e;
  if (trial_timed)
    for (int i = 0; i < 4; ++i) CK(c, cudaEventCreate(&te[i]));
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (c->profiling) {
    ev = {take_event(c), take_event(c)};
    CK(c, cudaEventRecord(ev.first, c->stream));
  }
  if (do_vel) {
  if (trial_timed) CK(c, cudaEventRecord(te[0], c->stream));
  CK(c, c->pipe ? (c->nd == 2 ? launch_pipe2d(true, P, c->map_kind, c->n_sm, c->tm_vel, c->stream)
                              : launch_pipe3d(true, P, c->n_sm, c->tm_vel, c->stream, lay(true)))
                : c->nd == 2 ? launch_vel2d(P, c->map_kind, c->stream) : launch_vel3d(P, c->map_kind, c->stream));
  c->launches++;
  if (trial_timed) CK(c, cudaEventRecord(te[1], c->stream));
  if (c->profiling) {
    CK(c, cudaEventRecord(ev.second, c->stream));
    c->ev_vel.push_back(ev);
    ev = {take_event(c), take_event(c)};
  }
  if (n < c->sig_steps) {
    for (int kind = 1; kind <= c->nd; ++kind) {
      const DevSource &d = c->dsrc[kind];
      if (d.n_tgt == 0) continue;
      CK(c, launch_inject(c->v[kind - 1], d.tgt, d.off, d.col, c->d_signal + n * c->sig_cols, d.n_tgt, c->stream));
      c->launches++;
    }
  }
  }
  if (!do_prs) {
    if (c->profiling) {  // the pair taken for the pressure half step goes back unused
      c->ev_pool.push_back(ev.first);
      c->ev_pool.push_back(ev.second);
    }
    return FW2_OK;
  }
  if (c->profiling && !do_vel) ev = {take_event(c), take_event(c)};
  if (c->profiling) CK(c, cudaEventRecord(ev.first, c->stream));
  if (trial_timed) CK(c, cudaEventRecord(te[2], c->stream));
  CK(c, c->pipe ? (c->nd == 2 ? launch_pipe2d(false, P, c->map_kind, c->n_sm, c->tm_prs, c->stream)
                              : launch_pipe3d(false, P, c->n_sm, c->tm_prs, c->stream, lay(false)))
                : c->nd == 2 ? launch_prs2d(P, c->map_kind, c->stream) : launch_prs3d(P, c->map_kind, c->stream));
  c->launches++;
  if (trial_timed) CK(c, cudaEventRecord(te[3], c->stream));
  if (c->profiling) {
    CK(c, cudaEventRecord(ev.second, c->stream));
    c->ev_prs.push_back(ev);
  }
  if (n < c->sig_steps && c->dsrc[0].n_tgt > 0) {
    const DevSource &d = c->dsrc[0];
    CK(c, launch_inject(c->p, d.tgt, d.off, d.col, c->d_signal + n * c->sig_cols, d.n_tgt, c->stream));
    c->launches++;
  }
  if (c->rec_groups > 0 && n < c->rec_steps) {
    CK(c, launch_record(c->p, c->rec_cell, c->rec_off, c->rec_groups, c->rec_out + n * c->rec_groups, c->stream));
    c->launches++;
  }
  if (trial > 0) {
    if (trial_timed) {
      CK(c, cudaEventSynchronize(te[3]));
      float mv = 0.f, mp = 0.f;
      CK(c, cudaEventElapsedTime(&mv, te[0], te[1]));
      CK(c, cudaEventElapsedTime(&mp, te[2], te[3]));
      c->layout_ms[trial - 1][0] = mv;
      c->layout_ms[trial - 1][1] = mp;
    }
    if (++c->layout_trial == 4)
      for (int h = 0; h < 2; ++h) {
        const bool vel = h == 0;
        const bool both = pipe3d_layout_allowed(vel, P, kLayoutStaged);
        c->layout3[h] = both && c->layout_ms[0][h] <= c->layout_ms[1][h] ? kLayoutStaged : kLayoutRegisters;
      }
  }
  return FW2_OK;
}

// max |p| of the context (+inf when a value is not finite); synchronises the
// context stream.
fw2_status scan_p(fw2_ctx *c, float *max_abs) {
  CK(c, cudaMemsetAsync(c->d_absmax, 0, sizeof(unsigned int), c->stream));
  CK(c, launch_absmax(c->p, c->nx, c->pitch, (long long)c->ny * c->nz, c->d_absmax, c->stream));
  c->launches++;
  unsigned int bits = 0;
  CK(c, cudaMemcpyAsync(&bits, c->d_absmax, sizeof bits, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  std::memcpy(max_abs, &bits, 4);
  return FW2_OK;
}

}  // namespace fw2

extern "C" {

int32_t fw2_abi_version(void) { return 1; }

fw2_status fw2_kernel_path(fw2_ctx *c, int32_t *path) {
  if (!c || !path) return FW2_EINVAL;
  *path = !c->finalized ? FW2_PATH_AUTO : (c->pipe ? FW2_PATH_PIPE : FW2_PATH_TILE);
  return FW2_OK;
}

fw2_status fw2_taps_time_space(double r, int32_t ndim, double *g) {
  if (!g || !(r >= 0.0 && r < 1.0)) return fail(nullptr, FW2_EINVAL, "g is required and r must lie in [0, 1)");
  if (ndim != 2 && ndim != 3) return fail(nullptr, FW2_EINVAL, "ndim must be 2 or 3");
  // g_11 from the |k h|^4 term (the time error; the direction-dependent part
  // then vanishes); g_1..g_4 from the odd powers p = 1, 3, 5, 7 of the axial
  // relation, where the cross tap has ndim - 1 transverse pairs:
  //   sum_m g_m b_m^p + 2 g_11 (ndim - 1) 2^-p = r^(p-1) 2^-p,  b_m = (2m - 1) / 2
  const double g11 = r * r / 24.0;
  double A[4][5];
  for (int row = 0; row < 4; ++row) {
    const int p = 2 * row + 1;
    for (int m = 0; m < 4; ++m) A[row][m] = std::pow((2.0 * m + 1.0) / 2.0, p);
    A[row][4] = (std::pow(r, p - 1) - 2.0 * g11 * (ndim - 1)) / std::pow(2.0, p);
  }
  for (int col = 0; col < 4; ++col) {  // Gaussian elimination, partial pivoting
    int piv = col;
    for (int row = col + 1; row < 4; ++row)
      if (std::fabs(A[row][col]) > std::fabs(A[piv][col])) piv = row;
    for (int k = 0; k < 5; ++k) std::swap(A[col][k], A[piv][k]);
    for (int row = 0; row < 4; ++row) {
      if (row == col) continue;
      const double f = A[row][col] / A[col][col];
      for (int k = col; k < 5; ++k) A[row][k] -= f * A[col][k];
    }
  }
  for (int m = 0; m < 4; ++m) g[m] = A[m][4] / A[m][m];
  g[4] = g11;
  return FW2_OK;
}

fw2_status fw2_selftest_bounded_wait(int64_t limit_ns, int32_t *timed_out) {
  if (!timed_out || limit_ns < 1 || limit_ns > 10000000000ll)
    return fail(nullptr, FW2_EINVAL, "timed_out is required and limit_ns must lie in [1, 1e10]");
  int *d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d, 0xff, sizeof(int));
  if (e == cudaSuccess) e = launch_bounded_wait_selftest((unsigned long long)limit_ns, d);
  int h = -1;
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) return fail(nullptr, FW2_ECUDA, "bounded-wait self-test: %s", cudaGetErrorString(e));
  *timed_out = h;
  return FW2_OK;
}

fw2_status fw2_config_init(fw2_config *cfg) {
  if (!cfg) return FW2_EINVAL;
  std::memset(cfg, 0, sizeof *cfg);
  cfg->ndim = 2;
  cfg->n[0] = cfg->n[1] = cfg->n[2] = 1;
  cfg->cfl = 0.4;
  cfg->pml_rc = 1e-3;
  cfg->pml_npow = 2.0;
  cfg->pml_reading = FW2_PML_C;
  cfg->map_precision = FW2_MAP_F32;
  cfg->nl_mode = FW2_NL_OFF;
  cfg->mem_alignment = FW2_MEM_CENTRED;
  return FW2_OK;
}

const char *fw2_last_error(const fw2_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

fw2_status fw2_create(const fw2_config *cfg_in, fw2_ctx **out) {
  if (!out) return fail(nullptr, FW2_EINVAL, "out pointer is null");
  *out = nullptr;
  if (!cfg_in) return fail(nullptr, FW2_EINVAL, "config is null");
  fw2_config cfg = *cfg_in;
  if (cfg.ndim != 2 && cfg.ndim != 3) return fail(nullptr, FW2_EINVAL, "ndim must be 2 or 3 (got %d)", cfg.ndim);
  if (cfg.ndim == 2 && cfg.n[2] != 1) return fail(nullptr, FW2_EINVAL, "2D grids need n[2] == 1");
  for (int q = 0; q < cfg.ndim; ++q) {
    if (cfg.n[q] < 8 || cfg.n[q] > (1LL << 30))
      return fail(nullptr, FW2_EINVAL, "n[%d] = %lld outside [8, 2^30]", q, (long long)cfg.n[q]);
  }
  if (cfg.n_relax < 0 || cfg.n_relax > kMaxRelax)
    return fail(nullptr, cfg.n_relax > kMaxRelax ? FW2_EUNSUPPORTED : FW2_EINVAL, "n_relax = %d outside [0, %d]",
                cfg.n_relax, kMaxRelax);
  if (!(cfg.h > 0.0) || !std::isfinite(cfg.h)) return fail(nullptr, FW2_EINVAL, "h must be positive");
  if (!(cfg.dt > 0.0) && !(cfg.cfl > 0.0)) return fail(nullptr, FW2_EINVAL, "need dt > 0 or cfl > 0");
  if (cfg.pml_transition < 0 || cfg.pml_bound < 0) return fail(nullptr, FW2_EINVAL, "negative PML thickness");
  const int L = cfg.pml_transition + cfg.pml_bound;
  if (L > 0) {
    if (cfg.n_relax < 1) return fail(nullptr, FW2_EINVAL, "a C-PML needs at least one relaxation mechanism");
    for (int q = 0; q < cfg.ndim; ++q)
      if (2LL * L > cfg.n[q]) return fail(nullptr, FW2_EINVAL, "boundary of %d cells per side does not fit axis %d", L, q);
    if (!(cfg.pml_rc > 0.0 && cfg.pml_rc < 1.0)) return fail(nullptr, FW2_EINVAL, "pml_rc must lie in (0, 1)");
    if (!(cfg.pml_npow >= 0.0)) return fail(nullptr, FW2_EINVAL, "pml_npow must be >= 0");
  }
  if (cfg.pml_reading != FW2_PML_A && cfg.pml_reading != FW2_PML_C && cfg.pml_reading != FW2_PML_NO_TRANSITION)
    return fail(nullptr, FW2_EINVAL, "bad pml_reading (FW2_PML_A = 0, FW2_PML_C = 2 or FW2_PML_NO_TRANSITION = 3)");
  if (cfg.map_precision < FW2_MAP_F32 || cfg.map_precision > FW2_MAP_F16)
    return fail(nullptr, FW2_EINVAL, "bad map_precision");
  const bool idx_form = cfg.map_precision == FW2_MAP_IDX_U8 || cfg.map_precision == FW2_MAP_IDX_U16;
  if (idx_form && cfg.n_relax > kTabSlots)
    return fail(nullptr, FW2_EUNSUPPORTED, "tissue-index tables hold up to %d mechanisms", kTabSlots);
  if (cfg.nl_mode < FW2_NL_OFF || cfg.nl_mode > FW2_NL_LITERAL) return fail(nullptr, FW2_EINVAL, "bad nl_mode");
  if (cfg.mem_alignment != FW2_MEM_CENTRED && cfg.mem_alignment != FW2_MEM_ENDPOINT)
    return fail(nullptr, FW2_EINVAL, "bad mem_alignment");
  if (cfg.kernel_path < FW2_PATH_AUTO || cfg.kernel_path > FW2_PATH_PIPE_REGISTERS)
    return fail(nullptr, FW2_EINVAL, "bad kernel_path");
  for (int q = 0; q < 3; ++q)
    if (cfg.bc[q] != FW2_BC_ZERO && cfg.bc[q] != FW2_BC_PERIODIC) return fail(nullptr, FW2_EINVAL, "bad bc[%d]", q);
  bool taps_zero = true;
  for (int i = 0; i < 5; ++i) taps_zero = taps_zero && cfg.g[i] == 0.0;
  if (taps_zero) {
    cfg.g[0] = 1225.0 / 1024.0;
    cfg.g[1] = -245.0 / 3072.0;
    cfg.g[2] = 49.0 / 5120.0;
    cfg.g[3] = -5.0 / 7168.0;
    cfg.g[4] = 0.0;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev < 1)
    return fail(nullptr, FW2_ECUDA, "no usable CUDA device (%s)", e != cudaSuccess ? cudaGetErrorString(e) : "count 0");
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return fail(nullptr, FW2_ECUDA, "cudaGetDeviceProperties failed");
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(nullptr, FW2_EUNSUPPORTED, "libfw2 is built for sm_103a; device %d is sm_%d%d", dev, prop.major, prop.minor);

  fw2_ctx *c = new (std::nothrow) fw2_ctx();
  if (!c) return fail(nullptr, FW2_ENOMEM, "host allocation failed");
  c->cfg = cfg;
  c->nd = cfg.ndim;
  c->N = cfg.n_relax;
  c->nx = (int)cfg.n[0];
  c->ny = (int)cfg.n[1];
  c->nz = cfg.ndim == 3 ? (int)cfg.n[2] : 1;
  // rows start on 64-byte boundaries: 16-byte aligned rows for every element
  // type (the uint8 tissue index included), as the tensor copies require
  c->pitch = (c->nx + 15) & ~15;
  c->plane = (long long)c->pitch * c->ny;
  // padded to 128 elements so every per-mechanism array (float or bf16)
  // starts 256-byte aligned at nu * npts_alloc
  c->npts_alloc = (c->plane * c->nz + 127) / 128 * 128;
  c->n_pts = (long long)c->nx * c->ny * c->nz;
  c->stream = (cudaStream_t)cfg.stream;
  c->map_kind = cfg.map_precision;
  c->n_sm = prop.multiProcessorCount;
  // state: p, v_q, psi1_q[N], psi2_q[N]
  const size_t arr = align256(sizeof(float) * (size_t)c->npts_alloc);
  const int n_arrays = 1 + c->nd + 2 * c->nd * c->N;
  void *m;
  fw2_status st = dalloc(c, arr * n_arrays, &m);
  if (st == FW2_OK) {
    c->state = (char *)m;
    c->state_bytes = arr * n_arrays;
    char *cur = c->state;
    c->p = (float *)cur; cur += arr;
    for (int q = 0; q < c->nd; ++q) { c->v[q] = (float *)cur; cur += arr; }
    for (int q = 0; q < c->nd; ++q) { c->psi1[q] = (float *)cur; cur += arr * c->N; }
    for (int q = 0; q < c->nd; ++q) { c->psi2[q] = (float *)cur; cur += arr * c->N; }
    if ((st = dalloc(c, 2 * sizeof(unsigned long long), &m)) == FW2_OK) c->d_scan = (unsigned long long *)m;
    if (st == FW2_OK && (st = dalloc(c, sizeof(int), &m)) == FW2_OK) c->d_bad = (int *)m;
    if (st == FW2_OK && (st = dalloc(c, sizeof(unsigned int), &m)) == FW2_OK) c->d_absmax = (unsigned int *)m;
    if (st == FW2_OK && (st = dalloc(c, sizeof(unsigned int), &m)) == FW2_OK) c->d_status = (unsigned int *)m;
  }
  if (st == FW2_OK) {
    cudaError_t e2 = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned int), c->stream);
    if (e2 != cudaSuccess) st = cuda_fail(c, e2, "status initialisation");
  }
  if (st == FW2_OK) {
    cudaError_t e2 = cudaMemsetAsync(c->state, 0, c->state_bytes, c->stream);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(c->stream);
    if (e2 != cudaSuccess) st = cuda_fail(c, e2, "state initialisation");
  }
  if (st != FW2_OK) {
    g_create_error = c->err;
    fw2_destroy(c);
    return st;
  }
  *out = c;
  return FW2_OK;
}

fw2_status fw2_destroy(fw2_ctx *c) {
  if (!c) return FW2_OK;
  cudaStreamSynchronize(c->stream);
  release_events(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (void *p : c->allocs) cudaFreeAsync(p, c->stream);
  c->allocs.clear();
  cudaStreamSynchronize(c->stream);
  delete c;
  return FW2_OK;
}

fw2_status fw2_release_memory(void) {
  cudaMemPool_t pool = nullptr;
  cudaError_t e = pool_of_current_device(&pool);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
  if (e != cudaSuccess) {
    fw2::set_global_error(cudaGetErrorString(e));
    return FW2_ECUDA;
  }
  return FW2_OK;
}

fw2_status fw2_set_medium(fw2_ctx *c, const float *cc, const float *rho, const float *beta, int32_t mem_space) {
  if (!c) return FW2_EINVAL;
  if (c->map_kind == FW2_MAP_IDX_U8 || c->map_kind == FW2_MAP_IDX_U16)
    return fail(c, FW2_EINVAL, "tissue-index contexts take fw2_set_medium_indexed");
  if (!cc || !rho) return fail(c, FW2_EINVAL, "c and rho are required");
  if (c->cfg.nl_mode != FW2_NL_OFF && !beta) return fail(c, FW2_EINVAL, "beta is required when nl_mode != OFF");
  if (mem_space != FW2_MEM_HOST && mem_space != FW2_MEM_DEVICE) return fail(c, FW2_EINVAL, "bad mem_space");
  const size_t b = sizeof(float) * (size_t)c->n_pts;
  void *m;
  fw2_status st;
  if (!c->raw_c) { if ((st = dalloc(c, b, &m)) != FW2_OK) return st; c->raw_c = (float *)m; }
  if (!c->raw_rho) { if ((st = dalloc(c, b, &m)) != FW2_OK) return st; c->raw_rho = (float *)m; }
  if ((st = copy_in(c, c->raw_c, cc, b, mem_space)) != FW2_OK) return st;
  if ((st = copy_in(c, c->raw_rho, rho, b, mem_space)) != FW2_OK) return st;
  if (c->cfg.nl_mode != FW2_NL_OFF) {
    if (!c->raw_beta) { if ((st = dalloc(c, b, &m)) != FW2_OK) return st; c->raw_beta = (float *)m; }
    if ((st = copy_in(c, c->raw_beta, beta, b, mem_space)) != FW2_OK) return st;
  }
  c->medium_set = true;
  c->finalized = false;
  return FW2_OK;
}

fw2_status fw2_set_relaxation(fw2_ctx *c, const fw2_relax_desc *d) {
  if (!c) return FW2_EINVAL;
  if (c->map_kind == FW2_MAP_IDX_U8 || c->map_kind == FW2_MAP_IDX_U16)
    return fail(c, FW2_EINVAL, "tissue-index contexts take fw2_set_medium_indexed");
  if (!d) return fail(c, FW2_EINVAL, "relaxation descriptor is null");
  if (c->N == 0) return fail(c, FW2_EINVAL, "n_relax is 0: no relaxation parameters to set");
  if (!d->kappa1 || !d->kappa2 || !d->d1 || !d->alpha1 || !d->d2 || !d->alpha2)
    return fail(c, FW2_EINVAL, "every relaxation array is required");
  const size_t b = sizeof(float) * (size_t)c->n_pts, bN = b * c->N;
  float **dst[] = {&c->raw_k1, &c->raw_k2, &c->raw_d1, &c->raw_al1, &c->raw_d2, &c->raw_al2};
  const float *src[] = {d->kappa1, d->kappa2, d->d1, d->alpha1, d->d2, d->alpha2};
  const size_t sz[] = {b, b, bN, bN, bN, bN};
  for (int i = 0; i < 6; ++i) {
    void *m;
    fw2_status st;
    if (!*dst[i]) { if ((st = dalloc(c, sz[i], &m)) != FW2_OK) return st; *dst[i] = (float *)m; }
    if ((st = copy_in(c, *dst[i], src[i], sz[i], d->mem_space)) != FW2_OK) return st;
  }
  c->relax_set = true;
  c->finalized = false;
  return FW2_OK;
}

fw2_status fw2_set_medium_indexed(fw2_ctx *c, const void *tissue, int32_t n_tissue, const float *cc,
                                  const float *rho, const float *beta, const fw2_relax_desc *relax,
                                  int32_t mem_space) {
  if (!c) return FW2_EINVAL;
  if (c->map_kind != FW2_MAP_IDX_U8 && c->map_kind != FW2_MAP_IDX_U16)
    return fail(c, FW2_EINVAL, "fw2_set_medium_indexed needs map_precision FW2_MAP_IDX_U8 or FW2_MAP_IDX_U16");
  if (!tissue || !cc || !rho) return fail(c, FW2_EINVAL, "tissue, c and rho are required");
  const bool wide = c->map_kind == FW2_MAP_IDX_U16;
  const int max_tissue = wide ? 65536 : kTissues;
  if (n_tissue < 1 || n_tissue > max_tissue)
    return fail(c, FW2_EINVAL, "n_tissue = %d outside [1, %d]", n_tissue, max_tissue);
  if (c->cfg.nl_mode != FW2_NL_OFF && !beta) return fail(c, FW2_EINVAL, "beta is required when nl_mode != OFF");
  if (c->N > 0 && (!relax || !relax->kappa1 || !relax->kappa2 || !relax->d1 || !relax->alpha1 || !relax->d2 ||
                   !relax->alpha2))
    return fail(c, FW2_EINVAL, "every relaxation table is required when n_relax > 0");
  if (mem_space != FW2_MEM_HOST && mem_space != FW2_MEM_DEVICE) return fail(c, FW2_EINVAL, "bad mem_space");
  // drop any earlier medium
  float **raws[] = {&c->raw_c, &c->raw_rho, &c->raw_beta, &c->raw_k1, &c->raw_k2,
                    &c->raw_d1, &c->raw_al1, &c->raw_d2, &c->raw_al2};
  for (float **r : raws) {
    dfree(c, *r);
    *r = nullptr;
  }
  dfree(c, c->raw_tissue);
  c->raw_tissue = nullptr;
  void *m;
  fw2_status st;
  const size_t index_bytes = (wide ? 2 : 1) * (size_t)c->n_pts;
  if ((st = dalloc(c, index_bytes, &m)) != FW2_OK) return st;
  c->raw_tissue = m;
  if ((st = copy_in(c, c->raw_tissue, tissue, index_bytes, mem_space)) != FW2_OK) return st;
  const size_t bt = sizeof(float) * (size_t)n_tissue, btN = bt * c->N;
  struct Item { float **dst; const float *src; size_t bytes; };
  std::vector<Item> items = {{&c->raw_c, cc, bt}, {&c->raw_rho, rho, bt}};
  if (c->cfg.nl_mode != FW2_NL_OFF) items.push_back({&c->raw_beta, beta, bt});
  if (c->N > 0) {
    items.push_back({&c->raw_k1, relax->kappa1, bt});
    items.push_back({&c->raw_k2, relax->kappa2, bt});
    items.push_back({&c->raw_d1, relax->d1, btN});
    items.push_back({&c->raw_al1, relax->alpha1, btN});
    items.push_back({&c->raw_d2, relax->d2, btN});
    items.push_back({&c->raw_al2, relax->alpha2, btN});
  }
  for (const Item &it : items) {
    if ((st = dalloc(c, it.bytes, &m)) != FW2_OK) return st;
    *it.dst = (float *)m;
    if ((st = copy_in(c, *it.dst, it.src, it.bytes, mem_space)) != FW2_OK) return st;
  }
  c->n_tissue = n_tissue;
  c->medium_set = true;
  c->relax_set = true;
  c->finalized = false;
  return FW2_OK;
}

fw2_status fw2_add_source(fw2_ctx *c, int32_t kind, int64_t n_pts, const int64_t *idx, const int32_t *group,
                          const float *signal, int64_t n_groups, int64_t n_steps, int32_t mem_space) {
  if (!c) return FW2_EINVAL;
  if (kind < FW2_SRC_P || kind > FW2_SRC_VZ || (kind != FW2_SRC_P && kind - 1 >= c->nd))
    return fail(c, FW2_EINVAL, "bad source kind %d for a %dD grid", kind, c->nd);
  if (n_pts < 0 || n_groups < 1 || n_steps < 0 || n_pts > (1LL << 31))
    return fail(c, FW2_EINVAL, "bad source sizes (n_pts %lld, n_groups %lld, n_steps %lld)", (long long)n_pts,
                (long long)n_groups, (long long)n_steps);
  HostSource s;
  s.kind = kind;
  s.n_groups = n_groups;
  s.n_steps = n_steps;
  fw2_status st;
  std::vector<long long> idx_h;
  if ((st = copy_to_host(c, idx_h, (const long long *)idx, (size_t)n_pts, mem_space)) != FW2_OK) return st;
  s.idx = idx_h;
  if (group) {
    if ((st = copy_to_host(c, s.group, (const int *)group, (size_t)n_pts, mem_space)) != FW2_OK) return st;
  } else {
    s.group.assign((size_t)n_pts, 0);
  }
  if ((st = copy_to_host(c, s.signal, signal, (size_t)(n_steps * n_groups), mem_space)) != FW2_OK) return st;
  for (long long e = 0; e < n_pts; ++e) {
    if (s.idx[e] < 0 || s.idx[e] >= c->n_pts) return fail(c, FW2_EINVAL, "source index %lld out of range", s.idx[e]);
    if (s.group[e] < 0 || s.group[e] >= n_groups) return fail(c, FW2_EINVAL, "source group %d out of range", s.group[e]);
  }
  c->sources.push_back(std::move(s));
  c->src_dirty = true;
  return FW2_OK;
}

fw2_status fw2_record(fw2_ctx *c, int64_t n_pts, const int64_t *idx, const int32_t *group, int64_t n_groups,
                      float *out, int64_t n_steps, int32_t mem_space) {
  if (!c) return FW2_EINVAL;
  dfree(c, c->rec_cell); c->rec_cell = nullptr;
  dfree(c, c->rec_off); c->rec_off = nullptr;
  c->rec_groups = 0;
  c->rec_out = nullptr;
  c->rec_steps = 0;
  if (n_pts == 0) return FW2_OK;  // recording disabled
  if (n_pts < 0 || n_steps < 0 || n_pts > (1LL << 31)) return fail(c, FW2_EINVAL, "bad recording sizes");
  if (!group) n_groups = n_pts;
  if (n_groups < 1 || n_groups > (1LL << 31)) return fail(c, FW2_EINVAL, "bad n_groups");
  if (!out && n_steps > 0) return fail(c, FW2_EINVAL, "trace buffer is null");
  std::vector<long long> idx_h;
  std::vector<int> grp;
  fw2_status st;
  if ((st = copy_to_host(c, idx_h, (const long long *)idx, (size_t)n_pts, mem_space)) != FW2_OK) return st;
  if (group) {
    if ((st = copy_to_host(c, grp, (const int *)group, (size_t)n_pts, mem_space)) != FW2_OK) return st;
  } else {
    grp.resize((size_t)n_pts);
    for (long long e = 0; e < n_pts; ++e) grp[e] = (int)e;
  }
  std::vector<int> count((size_t)n_groups + 1, 0);
  for (long long e = 0; e < n_pts; ++e) {
    if (idx_h[e] < 0 || idx_h[e] >= c->n_pts) return fail(c, FW2_EINVAL, "sensor index %lld out of range", idx_h[e]);
    if (grp[e] < 0 || grp[e] >= n_groups) return fail(c, FW2_EINVAL, "sensor group %d out of range", grp[e]);
    count[grp[e] + 1]++;
  }
  for (long long g = 0; g < n_groups; ++g) count[g + 1] += count[g];
  std::vector<long long> cells((size_t)n_pts);
  std::vector<int> fill(count.begin(), count.end() - 1);
  for (long long e = 0; e < n_pts; ++e) cells[fill[grp[e]]++] = to_pitched(c, idx_h[e]);
  void *m;
  if ((st = dalloc(c, cells.size() * sizeof(long long), &m)) != FW2_OK) return st;
  c->rec_cell = (long long *)m;
  if ((st = dalloc(c, count.size() * sizeof(int), &m)) != FW2_OK) return st;
  c->rec_off = (int *)m;
  CK(c, cudaMemcpyAsync(c->rec_cell, cells.data(), cells.size() * sizeof(long long), cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemcpyAsync(c->rec_off, count.data(), count.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->rec_groups = (int)n_groups;
  c->rec_out = out;
  c->rec_steps = n_steps;
  return FW2_OK;
}

fw2_status fw2_step(fw2_ctx *c, int64_t n_steps) {
  if (!c) return FW2_EINVAL;
  if (n_steps < 0) return fail(c, FW2_EINVAL, "negative step count");
  if (c->half) return fail(c, FW2_ESTATE, "a step begun with fw2_step_part must be completed first");
  fw2_status st;
  if ((st = finalize(c)) != FW2_OK) return st;
  if ((st = build_sources(c)) != FW2_OK) return st;
  for (int64_t s = 0; s < n_steps; ++s) {
    if ((st = enqueue_step(c, c->step)) != FW2_OK) return st;
    c->step += 1;  // every launch of the step is enqueued; it counts even if a later one fails
    if (c->watch_every > 0 && c->step % c->watch_every == 0) {
      float m = 0.f;
      if ((st = scan_p(c, &m)) != FW2_OK) return st;
      if (!(m <= c->watch_bound))
        return fail(c, FW2_EUNSTABLE, "field blew up by step %lld: max |p| = %g exceeds the watch bound %g",
                    (long long)c->step, m, c->watch_bound);
    }
  }
  return FW2_OK;
}

fw2_status fw2_pipe_layout(fw2_ctx *c, int32_t *vel, int32_t *prs) {
  if (!c || !vel || !prs) return FW2_EINVAL;
  *vel = c->layout3[0];
  *prs = c->layout3[1];
  return FW2_OK;
}

fw2_status fw2_step_part(fw2_ctx *c, int32_t part) {
  if (!c) return FW2_EINVAL;
  if (part != 0 && part != 1) return fail(c, FW2_EINVAL, "part must be 0 (velocity) or 1 (pressure)");
  if (part != c->half)
    return fail(c, FW2_ESTATE, "part %d of a step requested while part %d is due", part, c->half);
  fw2_status st;
  if ((st = finalize(c)) != FW2_OK) return st;
  if ((st = build_sources(c)) != FW2_OK) return st;
  if ((st = enqueue_step(c, c->step, part)) != FW2_OK) return st;
  c->half = part == 0 ? 1 : 0;
  if (part == 1) c->step += 1;
  return FW2_OK;
}

fw2_status fw2_set_subdomain(fw2_ctx *c, const int64_t *global_n, const int64_t *offset) {
  if (!c || !global_n || !offset) return FW2_EINVAL;
  const long long ext[3] = {c->nx, c->ny, c->nz};
  for (int q = 0; q < 3; ++q) {
    const long long g = q < c->nd ? global_n[q] : 1, o = q < c->nd ? offset[q] : 0;
    if (o < 0 || g < ext[q] || o + ext[q] > g)
      return fail(c, FW2_EINVAL, "axis %d: the grid [%lld, %lld) does not lie in [0, %lld)", q, o, o + ext[q], g);
    if (q < c->nd && c->cfg.bc[q] == FW2_BC_PERIODIC && (o != 0 || g != ext[q]))
      return fail(c, FW2_EINVAL, "a periodic axis cannot be split into subdomains");
    c->gext[q] = g;
    c->goff[q] = o;
  }
  if (!(c->cfg.dt > 0.0))
    return fail(c, FW2_EINVAL, "a subdomain needs an explicit dt (that of the whole grid)");
  if (c->cfg.pml_transition + c->cfg.pml_bound > 0 && !(c->cfg.pml_cp > 0.0))
    return fail(c, FW2_EINVAL, "a subdomain with a C-PML needs an explicit pml_cp (that of the whole grid)");
  c->subdomain = true;
  c->finalized = false;
  return FW2_OK;
}

// Rows of a state array along the slowest axis (y rows in 2D, z planes in
// 3D) to or from a dense buffer [n_rows][(ny)][nx]; synchronous.
static fw2_status copy_rows(fw2_ctx *c, int32_t field, int64_t row0, int64_t n_rows, float *buf, int32_t mem_space,
                     bool out) {
  if (!c || !buf) return FW2_EINVAL;
  if (field < FW2_FIELD_P || field > FW2_FIELD_VZ || (field > FW2_FIELD_P && field - FW2_FIELD_VX >= c->nd))
    return fail(c, FW2_EINVAL, "rows are copied for p and the velocity components only");
  const long long rows = c->nd == 3 ? c->nz : c->ny;
  if (row0 < 0 || n_rows < 0 || row0 + n_rows > rows)
    return fail(c, FW2_EINVAL, "rows [%lld, %lld) outside [0, %lld)", (long long)row0, (long long)(row0 + n_rows), rows);
  if (n_rows == 0) return FW2_OK;
  float *f = field == FW2_FIELD_P ? c->p : c->v[field - FW2_FIELD_VX];
  const long long per_row = c->nd == 3 ? c->plane : c->pitch;
  const size_t height = (size_t)n_rows * (c->nd == 3 ? c->ny : 1);
  float *dev = f + row0 * per_row;
  const size_t w = sizeof(float) * c->nx, dp = sizeof(float) * c->pitch;
  const cudaMemcpyKind kind = out ? (mem_space == FW2_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost)
                                  : (mem_space == FW2_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
  if (out) CK(c, cudaMemcpy2DAsync(buf, w, dev, dp, w, height, kind, c->stream));
  else CK(c, cudaMemcpy2DAsync(dev, dp, buf, w, w, height, kind, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return FW2_OK;
}

fw2_status fw2_get_rows(fw2_ctx *c, int32_t field, int64_t row0, int64_t n_rows, float *out, int32_t mem_space) {
  return copy_rows(c, field, row0, n_rows, out, mem_space, true);
}

fw2_status fw2_set_rows(fw2_ctx *c, int32_t field, int64_t row0, int64_t n_rows, const float *in,
                        int32_t mem_space) {
  return copy_rows(c, field, row0, n_rows, const_cast<float *>(in), mem_space, false);
}

fw2_status fw2_set_watch(fw2_ctx *c, int64_t every, float bound) {
  if (!c) return FW2_EINVAL;
  if (every < 0) return fail(c, FW2_EINVAL, "negative watch interval");
  if (every > 0 && !(bound > 0.f)) return fail(c, FW2_EINVAL, "the watch bound must be positive");
  c->watch_every = every;
  c->watch_bound = bound;
  return FW2_OK;
}

fw2_status fw2_get_dt(fw2_ctx *c, double *dt) {
  if (!c || !dt) return FW2_EINVAL;
  fw2_status st = finalize(c);
  if (st != FW2_OK) return st;
  *dt = c->dt;
  return FW2_OK;
}

fw2_status fw2_get_step(fw2_ctx *c, int64_t *step) {
  if (!c || !step) return FW2_EINVAL;
  *step = c->step;
  return FW2_OK;
}

fw2_status fw2_set_step(fw2_ctx *c, int64_t step) {
  if (!c) return FW2_EINVAL;
  if (step < 0) return fail(c, FW2_EINVAL, "negative step index");
  c->step = step;
  return FW2_OK;
}

fw2_status fw2_get_field(fw2_ctx *c, int32_t field, float *out, int32_t mem_space) {
  if (!c || !out) return FW2_EINVAL;
  int count;
  float *f = field_ptr(c, field, &count);
  if (!f) return fail(c, FW2_EINVAL, "field %d does not exist in this context", field);
  const cudaMemcpyKind kind = mem_space == FW2_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int m = 0; m < count; ++m) {
    CK(c, cudaMemcpy2DAsync(out + (size_t)m * c->n_pts, sizeof(float) * c->nx, f + (size_t)m * c->npts_alloc,
                            sizeof(float) * c->pitch, sizeof(float) * c->nx, (size_t)c->ny * c->nz, kind, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  return FW2_OK;
}

fw2_status fw2_set_field(fw2_ctx *c, int32_t field, const float *in, int32_t mem_space) {
  if (!c || !in) return FW2_EINVAL;
  int count;
  float *f = field_ptr(c, field, &count);
  if (!f) return fail(c, FW2_EINVAL, "field %d does not exist in this context", field);
  const cudaMemcpyKind kind = mem_space == FW2_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  for (int m = 0; m < count; ++m) {
    CK(c, cudaMemcpy2DAsync(f + (size_t)m * c->npts_alloc, sizeof(float) * c->pitch, in + (size_t)m * c->n_pts,
                            sizeof(float) * c->nx, sizeof(float) * c->nx, (size_t)c->ny * c->nz, kind, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  return FW2_OK;
}

fw2_status fw2_reset(fw2_ctx *c) {
  if (!c) return FW2_EINVAL;
  CK(c, cudaMemsetAsync(c->state, 0, c->state_bytes, c->stream));
  CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned int), c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->step = 0;
  c->half = 0;
  return FW2_OK;
}

fw2_status fw2_synchronize(fw2_ctx *c) {
  if (!c) return FW2_EINVAL;
  unsigned int status = 0;
  CK(c, cudaMemcpyAsync(&status, c->d_status, sizeof status, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (status & 1u)
    return fail(c, FW2_ETIMEOUT, "a bounded device-side wait gave up; the state is incomplete (fw2_reset clears it)");
  return FW2_OK;
}

fw2_status fw2_check_field(fw2_ctx *c, float bound, float *max_abs) {
  if (!c) return FW2_EINVAL;
  float m = 0.f;
  const fw2_status st = scan_p(c, &m);
  if (st != FW2_OK) return st;
  if (max_abs) *max_abs = m;
  if (!(m <= bound)) return fail(c, FW2_EUNSTABLE, "field check failed: max |p| = %g exceeds %g", m, bound);
  return FW2_OK;
}

fw2_status fw2_profile(fw2_ctx *c, int32_t enable) {
  if (!c) return FW2_EINVAL;
  c->profiling = enable != 0;
  if (!c->profiling) {
    cudaStreamSynchronize(c->stream);
    release_events(c);
  }
  return FW2_OK;
}

fw2_status fw2_profile_read(fw2_ctx *c, double *vel_ms, int64_t *vel_launches, double *prs_ms,
                            int64_t *prs_launches) {
  if (!c) return FW2_EINVAL;
  CK(c, cudaStreamSynchronize(c->stream));
  double tv = 0.0, tp = 0.0;
  for (auto &pr : c->ev_vel) {
    float ms = 0.f;
    CK(c, cudaEventElapsedTime(&ms, pr.first, pr.second));
    tv += ms;
  }
  for (auto &pr : c->ev_prs) {
    float ms = 0.f;
    CK(c, cudaEventElapsedTime(&ms, pr.first, pr.second));
    tp += ms;
  }
  if (vel_ms) *vel_ms = tv;
  if (prs_ms) *prs_ms = tp;
  if (vel_launches) *vel_launches = (int64_t)c->ev_vel.size();
  if (prs_launches) *prs_launches = (int64_t)c->ev_prs.size();
  release_events(c);
  return FW2_OK;
}

fw2_status fw2_device_bytes(fw2_ctx *c, int64_t *bytes) {
  if (!c || !bytes) return FW2_EINVAL;
  *bytes = c->dev_bytes;
  return FW2_OK;
}

fw2_status fw2_kernel_launches(fw2_ctx *c, int64_t *count) {
  if (!c || !count) return FW2_EINVAL;
  *count = c->launches;
  return FW2_OK;
}

}  // extern "C"
