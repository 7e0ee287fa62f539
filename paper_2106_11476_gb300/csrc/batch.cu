// Batched stepping of many contexts (transmit events, requests of a serving
// loop) in persistent launches, with a CUDA-graph-captured step loop.
//
// The active contexts form groups that share the dimension, the mechanism
// count and the map kind (in 3D also the cross taps and the layout of each
// half step).  Per time step: for every group one persistent velocity launch
// over the group's work table (2D pipelined: units of 128 x 8 cells; 2D tile
// path: tiles; 3D: the z-marching items of every context), one launch per
// velocity source kind present (v_x, v_y, v_z) over all contexts, one
// persistent pressure launch per group, one launch for the pressure
// sources, one for the recordings, and a tick of the per-context step
// counters kept on the device.  Since every per-step index comes from those
// counters, a chunk of steps is captured once as a CUDA graph and replayed.
// Each context computes exactly what fw2_step computes for it alone (same
// per-cell arithmetic).  Contexts leave the tables when they reach their
// step budget.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

using namespace fw2;

namespace {

struct BatchCtx {
  float *p;
  float *v[3];
  const long long *tgt[4];
  const int *off[4];
  const int *col[4];
  const float *signal;
  long long sig_cols, sig_steps;
  const long long *rec_cell;
  const int *rec_off;
  float *rec_out;
  long long rec_steps;
  int rec_groups;
};

// context of flat work item t, from the per-context prefix offsets
__device__ __forceinline__ int ctx_of(const int *prefix, int n_ctx, int t) {
  int lo = 0, hi = n_ctx;  // prefix[lo] <= t < prefix[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void batch_inject_kernel(const BatchCtx *C, int n_ctx, const int *prefix, int total, int kind,
                                    const long long *steps) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int k = ctx_of(prefix, n_ctx, t);
  const BatchCtx &c = C[k];
  const long long n = steps[k];
  if (n >= c.sig_steps) return;
  const int u = t - prefix[k];
  const float *row = c.signal + n * c.sig_cols;
  float s = 0.f;
  for (int e = c.off[kind][u]; e < c.off[kind][u + 1]; ++e) s += __ldg(row + c.col[kind][e]);
  float *field = kind == 0 ? c.p : c.v[kind - 1];
  field[c.tgt[kind][u]] += s;
}

__global__ void batch_record_kernel(const BatchCtx *C, int n_ctx, const int *prefix, int total,
                                    const long long *steps) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int k = ctx_of(prefix, n_ctx, t);
  const BatchCtx &c = C[k];
  const long long n = steps[k];
  if (n >= c.rec_steps) return;
  const int g = t - prefix[k];
  const int b = c.rec_off[g], e = c.rec_off[g + 1];
  float s = 0.f;
  for (int i = b; i < e; ++i) s += c.p[c.rec_cell[i]];
  c.rec_out[n * c.rec_groups + g] = e > b ? s / (float)(e - b) : 0.f;
}

__global__ void batch_tick_kernel(long long *steps, int n_ctx) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_ctx) steps[t] += 1;
}

struct Group {
  int n_relax, map_kind;
  std::vector<int> members;
  // 3D groups (pipelined, bf16 maps): contexts sharing N, the cross taps and
  // the layout of each half step; per half step a work-layout record per
  // context and the item table {context, item}
  int nd = 2;
  bool cross = false, ps[2] = {false, false};
  unsigned char *d_regions[2] = {nullptr, nullptr};
  int2 *d_items[2] = {nullptr, nullptr};
  int n_items[2] = {0, 0};
  int *d_runs3[2][4] = {};  // per half step and edge weight: the blocks' runs of items
  StepParams *d_params = nullptr;
  int4 *d_tiles[2] = {nullptr, nullptr};  // context-major, interleaved
  int n_tiles = 0;
  // pipelined form (float or index maps, no periodic axis): units of
  // 128 x 8 cells {ctx, x0, y0, interior}, tensor maps per context
  bool pipe = false;
  int4 *d_units = nullptr;
  int n_units = 0;
  int *d_runs[4] = {};  // per edge weight: the blocks' runs of units
  PipeMaps *d_maps[2] = {nullptr, nullptr};  // velocity, pressure
};

}  // namespace

struct fw2_batch {
  std::vector<fw2_ctx *> ctxs;
  std::vector<int> active;          // contexts (indices into ctxs) the tables cover
  std::vector<long long> budget;    // step count at which each context leaves (LLONG_MAX: none)
  std::vector<void *> table_allocs; // device tables of the active set, rebuilt when it changes
  std::vector<Group> groups;
  cudaStream_t stream = nullptr;
  BatchCtx *d_ctx = nullptr;
  long long *d_step = nullptr;
  int *d_prefix[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // source kinds 0..3, record
  int total[5] = {0, 0, 0, 0, 0};
  std::string err = "no error";
  // launch configuration: persistent grid and tile order, tuned online
  int grid = 0, order = 0, cand = 0;
  int n_sm = 152;
  bool tuned = false, warmed = false;
  int trial = 0;
  std::vector<float> trial_ms[4];
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  bool graph_stale = false;  // the tables changed since the graph was captured
  long long steps_done = 0;  // batch steps since creation
  // blow-up detection: scan every context's p every watch_every steps (0: off)
  long long watch_every = 0;
  float watch_bound = 0.f;
  long long launches = 0;
};

namespace {

// Launch configurations the tuner times: persistent grid and tile order of
// the tile path, and the cost of an edge unit relative to an interior one
// (tenths) by which the pipelined groups split their unit tables into the
// blocks' contiguous runs (edge units read C-PML strips and clamp; a run
// of them takes longer than a run of interior units of the same length).
const int kCandidates[4][3] = {{152 * 2, 0, 15}, {152 * 2, 1, 25}, {152, 0, 35}, {152 * 4, 1, 50}};

// Boundaries of `grid` contiguous runs of the weighted items with about
// equal weight each (grid + 1 entries, runs[0] = 0, runs[grid] = n).
std::vector<int> balanced_runs(const std::vector<double> &w, int grid) {
  const int n = (int)w.size();
  double total = 0.0;
  for (double x : w) total += x;
  std::vector<int> runs(grid + 1, n);
  runs[0] = 0;
  double acc = 0.0;
  int b = 1;
  for (int i = 0; i < n && b < grid; ++i) {
    acc += w[i];
    while (b < grid && acc >= total * b / grid) runs[b++] = i + 1;
  }
  return runs;
}

fw2_status bfail(fw2_batch *b, fw2_status s, const char *what, cudaError_t e = cudaSuccess) {
  char buf[512];
  if (e != cudaSuccess) snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  else snprintf(buf, sizeof buf, "%s", what);
  b->err = buf;
  return s;
}

#define BCK(b, call)                                              \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return bfail(b, FW2_ECUDA, #call, e_); \
  } while (0)

template <typename T>
fw2_status bupload(fw2_batch *b, const std::vector<T> &v, T **out) {
  void *m = nullptr;
  const size_t bytes = std::max<size_t>(sizeof(T) * v.size(), 16);
  cudaError_t e = cudaMalloc(&m, bytes);
  if (e != cudaSuccess) return bfail(b, FW2_ENOMEM, "batch allocation", e);
  b->table_allocs.push_back(m);
  if (!v.empty()) {
    e = cudaMemcpy(m, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bfail(b, FW2_ECUDA, "batch upload", e);
  }
  *out = static_cast<T *>(m);
  return FW2_OK;
}

// one time step of every active context (launch sequence of the file header)
fw2_status enqueue_step(fw2_batch *b, int cand) {
  const int grid = kCandidates[cand][0], order = kCandidates[cand][1];
  const int n_ctx = (int)b->active.size();
  for (int half = 0; half < 2; ++half) {
    const bool vel = half == 0;
    for (Group &g : b->groups) {
      if (g.nd == 3)
        BCK(b, launch_pipe3d_batched(vel, g.cross, g.ps[half], g.n_relax, g.d_params, g.d_regions[half],
                                     g.d_maps[half], g.d_items[half], g.d_runs3[half][cand], b->n_sm,
                                     b->stream));
      else if (g.pipe)
        BCK(b, launch_pipe2d_batched(vel, g.d_params, g.d_maps[vel ? 0 : 1], g.d_units, g.n_units, g.d_runs[cand],
                                     g.n_relax,
                                     g.map_kind, b->n_sm, b->stream));
      else
        BCK(b, launch_batched2d(vel, g.d_params, g.d_tiles[order], g.n_tiles, g.n_relax, g.map_kind, grid,
                                b->stream));
      b->launches++;
    }
    // after the velocity half step the v_x, v_y, v_z sources, after the
    // pressure half step the p sources
    const int kinds[2][3] = {{1, 2, 3}, {0, -1, -1}};
    for (int kk = 0; kk < 3; ++kk) {
      const int kind = kinds[half][kk];
      if (kind < 0 || b->total[kind] == 0) continue;
      batch_inject_kernel<<<(b->total[kind] + 127) / 128, 128, 0, b->stream>>>(b->d_ctx, n_ctx, b->d_prefix[kind],
                                                                              b->total[kind], kind, b->d_step);
      BCK(b, cudaGetLastError());
      b->launches++;
    }
  }
  if (b->total[4] > 0) {
    batch_record_kernel<<<(b->total[4] + 127) / 128, 128, 0, b->stream>>>(b->d_ctx, n_ctx, b->d_prefix[4],
                                                                         b->total[4], b->d_step);
    BCK(b, cudaGetLastError());
    b->launches++;
  }
  batch_tick_kernel<<<(n_ctx + 127) / 128, 128, 0, b->stream>>>(b->d_step, n_ctx);
  BCK(b, cudaGetLastError());
  b->launches++;
  return FW2_OK;
}

// Device tables of the active contexts: per group (mechanism count, map
// kind) the step parameters, tile tables (context-major and interleaved)
// and, for the pipelined form, the unit table and tensor maps; the source,
// recording and step-counter arrays of all active contexts.  Replaces the
// previous tables (the captured graph, which points into them, is marked
// stale: the next run re-captures it and updates the executable in place
// when the launch sequence kept its shape).
fw2_status build_tables(fw2_batch *b) {
  b->graph_stale = true;
  cudaStreamSynchronize(b->stream);
  for (void *m : b->table_allocs) cudaFree(m);
  b->table_allocs.clear();
  b->groups.clear();
  b->d_ctx = nullptr;
  b->d_step = nullptr;
  for (int k = 0; k < 5; ++k) {
    b->d_prefix[k] = nullptr;
    b->total[k] = 0;
  }
  // groups by (dimension, mechanism count, map kind; in 3D the cross taps
  // and the layouts); members index b->active
  for (int i = 0; i < (int)b->active.size(); ++i) {
    fw2_ctx *c = b->ctxs[b->active[i]];
    const bool cross = c->nd == 3 && c->P.g11h != 0.f;
    const bool ps0 = c->nd == 3 && pipe3d_staged_layout(true, c->P), ps1 = c->nd == 3 && pipe3d_staged_layout(false, c->P);
    auto it = std::find_if(b->groups.begin(), b->groups.end(), [&](const Group &g) {
      return g.nd == c->nd && g.n_relax == c->N && g.map_kind == c->map_kind && g.cross == cross && g.ps[0] == ps0 &&
             g.ps[1] == ps1;
    });
    if (it == b->groups.end()) {
      Group g{c->N, c->map_kind, {}};
      g.nd = c->nd;
      g.cross = cross;
      g.ps[0] = ps0;
      g.ps[1] = ps1;
      b->groups.push_back(g);
      it = b->groups.end() - 1;
    }
    it->members.push_back(i);
  }
  fw2_status st = FW2_OK;
  for (Group &g : b->groups) {
    if (g.nd == 3) {
      std::vector<StepParams> params;
      std::vector<PipeMaps> mv, mp;
      std::vector<unsigned char> reg[2];
      std::vector<int2> items[2];
      std::vector<int2> units3[2];  // per item: {edge units, units}
      const size_t rb = pipe3d_region_bytes();
      for (int m = 0; m < (int)g.members.size(); ++m) {
        fw2_ctx *c = b->ctxs[b->active[g.members[m]]];
        params.push_back(c->P);
        mv.push_back(c->tm_vel);
        mp.push_back(c->tm_prs);
        for (int h = 0; h < 2; ++h) {
          reg[h].resize((m + 1) * rb);
          const long long n = pipe3d_region(c->P, b->n_sm, h == 0, reg[h].data() + m * rb);
          for (long long t = 0; t < n; ++t) items[h].push_back(make_int2(m, (int)t));
          std::vector<int> ne(n), na(n);
          pipe3d_item_units(c->P, b->n_sm, h == 0, ne.data(), na.data());
          for (long long t = 0; t < n; ++t) units3[h].push_back(make_int2(ne[t], na[t]));
        }
      }
      if ((st = bupload(b, params, &g.d_params)) != FW2_OK) break;
      if ((st = bupload(b, mv, &g.d_maps[0])) != FW2_OK) break;
      if ((st = bupload(b, mp, &g.d_maps[1])) != FW2_OK) break;
      for (int h = 0; h < 2 && st == FW2_OK; ++h) {
        g.n_items[h] = (int)items[h].size();
        if ((st = bupload(b, reg[h], &g.d_regions[h])) != FW2_OK) break;
        if ((st = bupload(b, items[h], &g.d_items[h])) != FW2_OK) break;
        for (int w = 0; w < 4 && st == FW2_OK; ++w) {
          std::vector<double> wt(units3[h].size());
          for (size_t i = 0; i < wt.size(); ++i)
            wt[i] = (units3[h][i].y - units3[h][i].x) + units3[h][i].x * (kCandidates[w][2] / 10.0);
          st = bupload(b, balanced_runs(wt, b->n_sm), &g.d_runs3[h][w]);
        }
      }
      if (st != FW2_OK) break;
      continue;
    }
    std::vector<StepParams> params;
    std::vector<std::vector<int4>> per;
    for (int m = 0; m < (int)g.members.size(); ++m) {
      fw2_ctx *c = b->ctxs[b->active[g.members[m]]];
      params.push_back(c->P);
      std::vector<int4> t;
      for (int y0 = 0; y0 < c->ny; y0 += kTY)
        for (int x0 = 0; x0 < c->nx; x0 += kTX) t.push_back(make_int4(m, x0, y0, 0));
      per.push_back(t);
    }
    std::vector<int4> major, inter;
    for (auto &t : per) major.insert(major.end(), t.begin(), t.end());
    // interleaved: tiles of the contexts in turn
    size_t longest = 0;
    for (auto &t : per) longest = std::max(longest, t.size());
    for (size_t k = 0; k < longest; ++k)
      for (auto &t : per)
        if (k < t.size()) inter.push_back(t[k]);
    g.n_tiles = (int)major.size();
    if ((st = bupload(b, params, &g.d_params)) != FW2_OK) break;
    if ((st = bupload(b, major, &g.d_tiles[0])) != FW2_OK) break;
    if ((st = bupload(b, inter, &g.d_tiles[1])) != FW2_OK) break;
    // the pipelined form when every member allows it
    g.pipe = true;
    for (const StepParams &P : params)
      if (!pipe2d_supported(P, g.map_kind) || P.periodic[0] || P.periodic[1]) g.pipe = false;
    if (g.pipe) {
      std::vector<PipeMaps> mv(params.size()), mp(params.size());
      std::vector<int4> units;
      for (int m = 0; m < (int)params.size() && g.pipe; ++m) {
        const StepParams &P = params[m];
        const char *why = "";
        if (build_pipe2d_maps(P, g.map_kind, &mv[m], &mp[m], &why) != cudaSuccess) g.pipe = false;
        for (int y0 = 0; y0 < P.ny; y0 += kPipeHalf)
          for (int x0 = 0; x0 < P.nx; x0 += kTX)
            units.push_back(make_int4(m, x0, y0, pipe2d_interior_half(P, x0, y0) ? 1 : 0));
      }
      if (g.pipe) {
        g.n_units = (int)units.size();
        if ((st = bupload(b, units, &g.d_units)) != FW2_OK) break;
        for (int w = 0; w < 4 && st == FW2_OK; ++w) {
          std::vector<double> wt(units.size());
          for (size_t i = 0; i < units.size(); ++i) wt[i] = units[i].w ? 1.0 : kCandidates[w][2] / 10.0;
          st = bupload(b, balanced_runs(wt, b->n_sm), &g.d_runs[w]);
        }
        if (st != FW2_OK) break;
        if ((st = bupload(b, mv, &g.d_maps[0])) != FW2_OK) break;
        if ((st = bupload(b, mp, &g.d_maps[1])) != FW2_OK) break;
      }
    }
  }
  if (st == FW2_OK) {
    std::vector<BatchCtx> bc;
    std::vector<int> prefix[5];
    for (int k = 0; k < 5; ++k) prefix[k].push_back(0);
    for (int i : b->active) {
      fw2_ctx *c = b->ctxs[i];
      BatchCtx x{};
      x.p = c->p;
      for (int q = 0; q < 3; ++q) x.v[q] = c->v[q];
      for (int k = 0; k < 4; ++k) {
        x.tgt[k] = c->dsrc[k].tgt;
        x.off[k] = c->dsrc[k].off;
        x.col[k] = c->dsrc[k].col;
        prefix[k].push_back(prefix[k].back() + c->dsrc[k].n_tgt);
      }
      x.signal = c->d_signal;
      x.sig_cols = c->sig_cols;
      x.sig_steps = c->sig_steps;
      x.rec_cell = c->rec_cell;
      x.rec_off = c->rec_off;
      x.rec_out = c->rec_out;
      x.rec_steps = c->rec_steps;
      x.rec_groups = c->rec_groups;
      prefix[4].push_back(prefix[4].back() + c->rec_groups);
      bc.push_back(x);
    }
    st = bupload(b, bc, &b->d_ctx);
    for (int k = 0; k < 5 && st == FW2_OK; ++k) {
      b->total[k] = prefix[k].back();
      st = bupload(b, prefix[k], &b->d_prefix[k]);
    }
    std::vector<long long> steps(b->active.size(), 0);
    if (st == FW2_OK) st = bupload(b, steps, &b->d_step);
  }
  return st;
}

}  // namespace

extern "C" {

fw2_status fw2_batch_create(fw2_ctx *const *ctxs, int32_t n_ctx, fw2_batch **out) {
  if (!out) return FW2_EINVAL;
  *out = nullptr;
  if (!ctxs || n_ctx < 1) return FW2_EINVAL;
  fw2_batch *b = new (std::nothrow) fw2_batch();
  if (!b) return FW2_ENOMEM;
  for (int i = 0; i < n_ctx; ++i) {
    fw2_ctx *c = ctxs[i];
    if (!c) {
      delete b;
      return FW2_EINVAL;
    }
    fw2_status st = ctx_prepare(c);
    if (st == FW2_OK && c->nd == 3 && !c->pipe)
      st = ctx_fail(c, FW2_EUNSUPPORTED,
                    "3D contexts join a batch on the pipelined path only (bf16 maps, N <= 3, no periodic axis)");
    if (st != FW2_OK) {
      delete b;
      return st;
    }
    b->ctxs.push_back(c);
  }
  b->n_sm = b->ctxs[0]->n_sm;
  cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    return FW2_ECUDA;
  }
  b->budget.assign(b->ctxs.size(), LLONG_MAX);
  for (int i = 0; i < n_ctx; ++i) b->active.push_back(i);
  fw2_status st = build_tables(b);
  if (st != FW2_OK) {
    for (void *m : b->table_allocs) cudaFree(m);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return st;
  }
  *out = b;
  return FW2_OK;
}

}  // extern "C"

namespace {

// Steps each launch configuration is timed over during tuning; the median
// of its trials counts.
constexpr int kTrialReps = 3;
// Steps per captured graph (replayed; a shorter tail is launched directly).
constexpr int kGraphSteps = 16;

struct EventPair {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~EventPair() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

float median_of(std::vector<float> v) {
  std::sort(v.begin(), v.end());
  return v.empty() ? 0.f : v[v.size() / 2];
}

// Enqueue n_steps batch steps; *done counts the steps enqueued (they run
// even when a later enqueue fails), b->steps_done follows it.
fw2_status batch_run(fw2_batch *b, int64_t n_steps, int64_t *done) {
  const int64_t start = *done;
  struct Count {  // keeps b->steps_done in step with *done on every return
    fw2_batch *b;
    const int64_t *done;
    int64_t start;
    ~Count() { b->steps_done += *done - start; }
  } count{b, done, start};
  n_steps += start;
  // online tuning: one warm-up step (it pays the first launch's cold start),
  // then each launch configuration for kTrialReps steps (every
  // configuration computes the same result); the fastest median wins
  if (!b->warmed && *done < n_steps) {
    fw2_status st = enqueue_step(b, 0);
    if (st != FW2_OK) return st;
    ++*done;
    b->warmed = true;
  }
  while (!b->tuned && *done < n_steps) {
    const int k = b->trial / kTrialReps;
    EventPair ev;
    BCK(b, cudaEventCreate(&ev.e0));
    BCK(b, cudaEventCreate(&ev.e1));
    BCK(b, cudaEventRecord(ev.e0, b->stream));
    fw2_status st = enqueue_step(b, k);
    if (st != FW2_OK) return st;
    ++*done;
    BCK(b, cudaEventRecord(ev.e1, b->stream));
    BCK(b, cudaEventSynchronize(ev.e1));
    float ms = 0.f;
    BCK(b, cudaEventElapsedTime(&ms, ev.e0, ev.e1));
    b->trial_ms[k].push_back(ms);
    if (++b->trial == 4 * kTrialReps) {
      int best = 0;
      for (int c = 1; c < 4; ++c)
        if (median_of(b->trial_ms[c]) < median_of(b->trial_ms[best])) best = c;
      b->grid = kCandidates[best][0];
      b->order = kCandidates[best][1];
      b->cand = best;
      b->tuned = true;
    }
  }
  const int64_t rest = n_steps - *done;
  if (rest > 0) {
    const int chunk = (int)std::min<int64_t>(rest, kGraphSteps);
    if (!b->graph || b->graph_steps != chunk || b->graph_stale) {
      cudaGraph_t g;
      BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
      fw2_status st = FW2_OK;
      for (int s = 0; s < chunk && st == FW2_OK; ++s) st = enqueue_step(b, b->cand);
      cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
      if (st != FW2_OK) return st;
      BCK(b, ec);
      // same number of steps and launches: new parameters into the
      // executable graph; otherwise a new executable
      bool updated = false;
      if (b->graph && b->graph_steps == chunk) {
        cudaGraphExecUpdateResultInfo info;
        updated = cudaGraphExecUpdate(b->graph, g, &info) == cudaSuccess;
        if (!updated) (void)cudaGetLastError();
      }
      if (!updated) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        ec = cudaGraphInstantiate(&b->graph, g, 0);
      }
      cudaGraphDestroy(g);
      BCK(b, ec);
      b->graph_steps = chunk;
      b->graph_stale = false;
    }
    int64_t left = rest;
    while (left >= chunk) {
      BCK(b, cudaGraphLaunch(b->graph, b->stream));
      *done += chunk;
      left -= chunk;
    }
    for (int64_t s = 0; s < left; ++s) {
      fw2_status st = enqueue_step(b, b->cand);
      if (st != FW2_OK) return st;
      ++*done;
    }
  }
  return FW2_OK;
}

// max |p| of every context, scanned on the batch stream; FW2_EUNSTABLE names
// the first context that holds a non-finite value or exceeds the bound.
fw2_status batch_scan(fw2_batch *b) {
  std::vector<unsigned int> bits(b->ctxs.size(), 0u);
  for (int i : b->active) {
    fw2_ctx *c = b->ctxs[i];
    BCK(b, cudaMemsetAsync(c->d_absmax, 0, sizeof(unsigned int), b->stream));
    BCK(b, launch_absmax(c->p, c->nx, c->pitch, (long long)c->ny * c->nz, c->d_absmax, b->stream));
    ++b->launches;
    BCK(b, cudaMemcpyAsync(&bits[i], c->d_absmax, sizeof(unsigned int), cudaMemcpyDeviceToHost, b->stream));
  }
  BCK(b, cudaStreamSynchronize(b->stream));
  for (int i : b->active) {
    float m;
    std::memcpy(&m, &bits[i], 4);
    if (!(m <= b->watch_bound)) {
      char msg[200];
      std::snprintf(msg, sizeof msg, "context %d blew up by batch step %lld: max |p| = %g exceeds the watch bound %g",
                    i, b->steps_done, (double)m, (double)b->watch_bound);
      return bfail(b, FW2_EUNSTABLE, msg);
    }
  }
  return FW2_OK;
}

// batch_run in segments that end where a blow-up scan is due.
fw2_status batch_advance(fw2_batch *b, int64_t n_steps, int64_t *done) {
  while (*done < n_steps) {
    int64_t seg = n_steps - *done;
    if (b->watch_every > 0) seg = std::min<int64_t>(seg, b->watch_every - b->steps_done % b->watch_every);
    const fw2_status st = batch_run(b, seg, done);
    if (st != FW2_OK) return st;
    if (b->watch_every > 0 && b->steps_done % b->watch_every == 0) {
      const fw2_status sc = batch_scan(b);
      if (sc != FW2_OK) return sc;
    }
  }
  return FW2_OK;
}

}  // namespace

extern "C" {

fw2_status fw2_batch_step(fw2_batch *b, int64_t n_steps) {
  if (!b) return FW2_EINVAL;
  if (n_steps < 0) return bfail(b, FW2_EINVAL, "negative step count");
  // work already queued on the contexts' own streams comes first
  for (fw2_ctx *c : b->ctxs) BCK(b, cudaStreamSynchronize(c->stream));
  int64_t total = 0;
  while (total < n_steps) {
    // the contexts still short of their budget; the tables follow that set
    std::vector<int> act;
    int64_t seg = n_steps - total;
    for (int i = 0; i < (int)b->ctxs.size(); ++i)
      if (b->ctxs[i]->step < b->budget[i]) {
        act.push_back(i);
        seg = std::min<int64_t>(seg, b->budget[i] - b->ctxs[i]->step);
      }
    if (act.empty()) break;
    if (act != b->active) {
      b->active = act;
      const fw2_status st = build_tables(b);
      if (st != FW2_OK) return st;
    }
    std::vector<long long> steps;
    for (int i : b->active) steps.push_back(b->ctxs[i]->step);
    BCK(b, cudaMemcpyAsync(b->d_step, steps.data(), sizeof(long long) * steps.size(), cudaMemcpyHostToDevice,
                           b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    int64_t done = 0;
    const fw2_status st = batch_advance(b, seg, &done);
    // the steps enqueued before a failure still advance the contexts
    for (int i : b->active) b->ctxs[i]->step += done;
    total += done;
    if (st != FW2_OK) return st;
  }
  return FW2_OK;
}

fw2_status fw2_batch_set_budget(fw2_batch *b, const int64_t *last_step) {
  if (!b) return FW2_EINVAL;
  for (size_t i = 0; i < b->ctxs.size(); ++i)
    b->budget[i] = (last_step && last_step[i] >= 0) ? (long long)last_step[i] : LLONG_MAX;
  return FW2_OK;
}

fw2_status fw2_batch_active(fw2_batch *b, int32_t *n_active) {
  if (!b || !n_active) return FW2_EINVAL;
  int32_t n = 0;
  for (size_t i = 0; i < b->ctxs.size(); ++i) n += b->ctxs[i]->step < b->budget[i] ? 1 : 0;
  *n_active = n;
  return FW2_OK;
}

fw2_status fw2_batch_set_watch(fw2_batch *b, int64_t every, float bound) {
  if (!b) return FW2_EINVAL;
  if (every < 0) return bfail(b, FW2_EINVAL, "negative watch interval");
  if (every > 0 && !(bound > 0.f)) return bfail(b, FW2_EINVAL, "the watch bound must be positive");
  b->watch_every = every;
  b->watch_bound = bound;
  return FW2_OK;
}

fw2_status fw2_batch_synchronize(fw2_batch *b) {
  if (!b) return FW2_EINVAL;
  BCK(b, cudaStreamSynchronize(b->stream));
  return FW2_OK;
}

fw2_status fw2_batch_info(fw2_batch *b, int32_t *grid, int32_t *order, int64_t *launches) {
  if (!b) return FW2_EINVAL;
  if (grid) *grid = b->tuned ? b->grid : 0;
  if (order) *order = b->tuned ? b->order : -1;
  if (launches) *launches = b->launches;
  return FW2_OK;
}

fw2_status fw2_batch_edge_weight(fw2_batch *b, double *weight) {
  if (!b || !weight) return FW2_EINVAL;
  *weight = b->tuned ? kCandidates[b->cand][2] / 10.0 : 0.0;
  return FW2_OK;
}

const char *fw2_batch_last_error(const fw2_batch *b) { return b ? b->err.c_str() : "null batch"; }

fw2_status fw2_batch_destroy(fw2_batch *b) {
  if (!b) return FW2_OK;
  cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void *m : b->table_allocs) cudaFree(m);
  cudaStreamDestroy(b->stream);
  delete b;
  return FW2_OK;
}

}  // extern "C"
