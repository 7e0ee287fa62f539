// Parameters of the one-time coefficient preparation and of the auxiliary
// (source, recording, check) kernels.
#pragma once
#include "fw2_internal.cuh"

namespace fw2 {

struct PrepParams {
  int nx, ny, nz, nd, pitch;
  long long plane, npts_alloc;
  int N;
  double dt;
  int LT, LB, reading;
  double npow, d_target;
  // the grid this context covers within a larger one (a subdomain): extent
  // of the whole grid and offset of this context along each axis; the
  // C-PML depth of a cell comes from its coordinate in the whole grid
  int gext[3], goff[3];
  int nl_mode;
  // raw inputs, dense [n_pts] (relaxation [N][n_pts]), device; in the
  // tissue-index form they are tables [n_tissue] ([N][n_tissue]) read
  // through tissue_in[n_pts]
  const float *c, *rho, *beta, *k1, *k2, *d1, *al1, *d2, *al2;
  const void *tissue_in;           // null: dense inputs (uint8, or uint16 when wide)
  int n_tissue;
  int tissue_wide;                 // 1: uint16 index
  void *tissue_out;                // pitched index (index form)
  float *table_out;                // [kTableFields][tab_stride] (index form)
  int tab_stride;
  // outputs (float or bf16)
  void *K, *rho_o, *chi, *ik1, *ik2, *a1, *b1, *a2, *b2;
  void *sa1[3], *sb1[3], *sa2[3], *sb2[3];
  long long strip_nu[3];
  // FP16 maps: each map is stored times inv_scale[map] (a power of two,
  // slots of StepParams::ms), chosen from the maps' largest magnitudes that
  // a scan pass first gathers into f16_max (float bits, device)
  double inv_scale[kMapScales];
  unsigned int *f16_max;
};

cudaError_t launch_medium_scan(const PrepParams &Q, unsigned long long *maxbits, int *bad,
                               cudaStream_t s);
// map_kind: 0 float, 1 bf16, 2 uint8 tissue index, 3 uint16 tissue index,
// 4 FP16 (after launch_prep_scan and with Q.inv_scale set)
cudaError_t launch_prep(const PrepParams &Q, int map_kind, cudaStream_t s);
// FP16 maps: the largest magnitude of every map (cell maps and C-PML strips,
// b as 1 - b) into Q.f16_max[kMapScales] (zeroed by the caller), as float bits
cudaError_t launch_prep_scan(const PrepParams &Q, cudaStream_t s);

// sources: field[tgt[u]] += sum_{e in [off[u], off[u+1])} row[col[e]]
cudaError_t launch_inject(float *field, const long long *tgt, const int *off, const int *col,
                          const float *row, int n_tgt, cudaStream_t s);
// recording: out[g] = mean over e in [off[g], off[g+1]) of p[cell[e]]
cudaError_t launch_record(const float *p, const long long *cell, const int *off, int n_groups,
                          float *out, cudaStream_t s);
// field scan: max |x| over the cell layout (rows of nx valid values, pitch
// apart), non-finite values reported as +inf; result in *out_bits (float bits)
cudaError_t launch_absmax(const float *f, int nx, int pitch, long long rows,
                          unsigned int *out_bits, cudaStream_t s);

// one block waits on an mbarrier that never completes, with the bounded wait
// of the pipelined kernels; *timed_out (device) = 1 when it gave up
cudaError_t launch_bounded_wait_selftest(unsigned long long limit_ns, int *timed_out);

}  // namespace fw2
