/*
 * fw2.h -- C ABI of the GB300 Fullwave 2 time stepper (libfw2.so).
 *
 * The library advances the stretched first-order pressure / particle-velocity
 * system of Sode & Pinton, "Fullwave 2" (arXiv 2106.11476), Eqs. (wave1),
 * (wave2) and their nonlinear form Eqs. (general5), (general6), on the
 * staggered grid of Sec. 3.1.  Every spatial derivative is stretched through
 * N relaxation memory variables (Eqs. relaxation1-3, relaxation4, advanced by
 * the recursion Eq. relaxation_psi with the coefficients of Eqs. relaxation_a,
 * relaxation_b).  The same recursion provides interior power-law attenuation
 * and the two-stage C-PML with its transition layer (Sec. 3.3, Table 1).
 *
 * Conventions shared by every call
 *  - Grids are nx x ny (x nz) cells, x fastest; a flat cell index is
 *    i + nx * (j + ny * k).  The boundary region lies inside the grid.
 *    p lives at cell centres, v_q at the +1/2 face of axis q of each cell.
 *  - Array arguments are plain pointers; `mem_space` says whether they are
 *    host (FW2_MEM_HOST) or device (FW2_MEM_DEVICE) memory of the current
 *    CUDA device.  Inputs are copied before the call returns (for device
 *    inputs: enqueued on the context stream, then synchronised), so the
 *    caller may free or reuse them afterwards.
 *  - Output buffers passed to fw2_record are caller-owned device memory and
 *    must stay valid while fw2_step calls that write them are in flight.
 *  - Every call returns an fw2_status; no exception or exit crosses the ABI.
 *    On failure fw2_last_error(ctx) describes the cause.  A context is not
 *    thread-safe; distinct contexts are independent.
 *  - All device work of a context runs on the stream given in fw2_config
 *    (NULL: the legacy default stream).  fw2_step is asynchronous.
 *  - Device memory of the contexts comes from a stream-ordered memory pool
 *    the library keeps per device: memory a destroyed context returns stays
 *    in the pool for the next context of the process (contexts created one
 *    after another do not map fresh memory each time) until
 *    fw2_release_memory returns it to the driver.
 */
#ifndef FW2_H
#define FW2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fw2_ctx fw2_ctx; /* opaque, owned by the library */

typedef enum {
  FW2_OK = 0,
  FW2_EINVAL = 1,       /* bad argument, size, layout or unstable time step */
  FW2_ENOMEM = 2,       /* device or host allocation failed */
  FW2_ECUDA = 3,        /* a CUDA runtime call failed (no device, launch error) */
  FW2_ESTATE = 4,       /* call out of order (e.g. step before set_medium) */
  FW2_EUNSTABLE = 5,    /* non-finite or exploding field detected */
  FW2_ETIMEOUT = 6,     /* a bounded device-side wait gave up */
  FW2_EUNSUPPORTED = 7  /* valid request the library does not implement */
} fw2_status;

enum { FW2_MEM_HOST = 0, FW2_MEM_DEVICE = 1 };
enum { FW2_BC_ZERO = 0, FW2_BC_PERIODIC = 1 };
/* nonlinear factor chi of the pressure update p -= dt K div / (1 + chi p):
 * OFF: chi = 0; PRESSURE: chi = kappa0 (1 - 2 beta), the factor printed in
 * Eq. (general6); WESTERVELT: chi = -2 beta kappa0 (kappa0 = 1 / (rho c^2)).
 * LITERAL: the system as printed, Eqs. (general5) and (general6): the
 * PRESSURE factor, and the velocity update divided by 1 + kappa0 p at the face
 * (kappa0 the mean of the two cells' 1/K, p the mean of their p^n), which
 * propagates with speed c0 + (beta - 1) v. */
enum { FW2_NL_OFF = 0, FW2_NL_PRESSURE = 1, FW2_NL_WESTERVELT = 2, FW2_NL_LITERAL = 3 };
/* storage of the coefficient maps: float, bf16 (b kept as 1 - b), FP16
 * (every map, and the C-PML strips of a mechanism with its interior map,
 * divided by a power of two chosen from the map's largest magnitude so that
 * it lies in [2^14, 2^15); b kept as 1 - b; tile kernels), or a tissue index
 * per cell into per-tissue float tables (N <= 4; set the medium with
 * fw2_set_medium_indexed): uint8 for up to 256 tissues or uint16 for up to
 * 65536.  In 2D the uint8 tables sit in shared memory (pipelined or tile
 * kernels); the uint16 tables, and every table in 3D, are read through L2 by
 * the tile kernels. */
enum { FW2_MAP_F32 = 0, FW2_MAP_BF16 = 1, FW2_MAP_IDX_U8 = 2, FW2_MAP_IDX_U16 = 3, FW2_MAP_F16 = 4 };
/* C-PML geometry (Sec. 3.3, Table 1).  In both readings the nu >= 2
 * parameters fall to zero over the inner L_T cells with the cosine transition
 * and kappa is kept, and d^{nu=1} ramps as a polynomial over all L_T + L_B
 * cells toward Table 1's d_target.
 * A: Table 1 as printed: alpha^{nu=1} falls linearly from the tissue's value
 * to zero over all L_T + L_B cells.
 * C (default): NOT Table 1's alpha^{nu=1} profile.  alpha^{nu=1} is blended
 * by the cosine transition over the inner L_T cells from the tissue's value
 * into the C-PML profile d_target (1 - x/L), which falls linearly to zero at
 * the outer edge (d_target acting as the maximum frequency shift of a
 * C-PML), so the transition layer turns the tissue's first mechanism into
 * the single C-PML mechanism.  Why: with Table 2's alpha^{nu=1} = 2.8e8 1/s,
 * far above the C-PML damping, reading A's first mechanism absorbs only in
 * the outermost cells and the boundary reflects at about -28 dB in that
 * tissue (3 + 1 wavelengths); C reflects at -53 dB there and stays stable.
 * In a non-attenuating medium both reach about -60 dB.
 * NO_TRANSITION: reading C for the first mechanism, but the nu >= 2
 * parameters keep their interior values inside the boundary: the
 * multi-mechanism C-PML without a transition layer that Sec. 3.3 reports
 * unstable (the field grows by about x1.5 every 5000 steps in Table 2
 * tissue).  It is offered to reproduce that result and to exercise the
 * blow-up detection of fw2_set_watch; do not use it for simulations.
 * The value 1 (an earlier reading that ramped the first mechanism over the
 * outer L_B cells only, reflecting at about -9 dB) is rejected with
 * FW2_EINVAL. */
enum { FW2_PML_A = 0, FW2_PML_C = 2, FW2_PML_NO_TRANSITION = 3 };
/* time alignment of the memory term in Eq. (relaxation_psi): CENTRED uses
 * the mean of the memory variable before and after its update (D^{n-1/2}
 * estimated by (D^n + D^{n-1}) / 2); ENDPOINT uses the updated value. */
enum { FW2_MEM_CENTRED = 0, FW2_MEM_ENDPOINT = 1 };
/* kernel path of the half steps (bitwise the same results on every path):
 * TILE runs one block per tile; PIPE runs the persistent kernels that stage
 * every tile through shared memory with TMA copies, where they apply (2D
 * float or tissue-index maps; 3D bf16 maps with N <= 3, g_{1,1} cross taps
 * and the literal system included; no periodic axis), and TILE elsewhere;
 * AUTO (default) is PIPE where it applies.  The 3D pipelined half steps have two layouts:
 * the memory variables staged in shared memory with the other arrays, or
 * loaded into registers one unit ahead, which leaves room to stage every
 * C-PML strip (faster where edge units dominate); the cross taps and the
 * literal system's velocity half step take the register layout only.  PIPE
 * and AUTO time both on a context's first four steps and keep the faster
 * per half step (fw2_pipe_layout reports the choice); PIPE_STAGED and
 * PIPE_REGISTERS fix one (where it applies). */
enum { FW2_PATH_AUTO = 0, FW2_PATH_TILE = 1, FW2_PATH_PIPE = 2, FW2_PATH_PIPE_STAGED = 3, FW2_PATH_PIPE_REGISTERS = 4 };
enum { FW2_SRC_P = 0, FW2_SRC_VX = 1, FW2_SRC_VY = 2, FW2_SRC_VZ = 3 };
enum {
  FW2_FIELD_P = 0, FW2_FIELD_VX = 1, FW2_FIELD_VY = 2, FW2_FIELD_VZ = 3,
  FW2_FIELD_PSI1X = 4, FW2_FIELD_PSI1Y = 5, FW2_FIELD_PSI1Z = 6,
  FW2_FIELD_PSI2X = 7, FW2_FIELD_PSI2Y = 8, FW2_FIELD_PSI2Z = 9
};

typedef struct {
  int32_t ndim;          /* 2 or 3 */
  int32_t n_relax;       /* N relaxation mechanisms, 0..8 (Sec. 2.1: N
                            memory variables per derivative); the tile
                            kernels take every N, the pipelined 2D half steps
                            N <= 4, the 3D ones N <= 3, the tissue-index
                            tables N <= 4 (FW2_EUNSUPPORTED above) */
  int64_t n[3];          /* nx, ny, nz (nz = 1 in 2D); boundary region included */
  double h;              /* grid spacing [m] */
  double dt;             /* time step [s]; <= 0: cfl * h / c_max, with c_max the
                            largest c / sqrt(kappa1 kappa2) of the medium */
  double cfl;            /* used when dt <= 0 (Sec. 3.4 uses 0.4) */
  double g[5];           /* g_{1,0}..g_{4,0}, g_{1,1} of the staggered operator
                            (Sec. 3.1); all zero: 8th-order Taylor set
                            1225/1024, -245/3072, 49/5120, -5/7168, g11 = 0 */
  int32_t pml_transition;/* L_T, cells per side (Sec. 3.3) */
  int32_t pml_bound;     /* L_B, cells per side */
  int32_t pml_reading;   /* FW2_PML_C (default), FW2_PML_A or FW2_PML_NO_TRANSITION */
  int32_t map_precision; /* FW2_MAP_F32, FW2_MAP_BF16, FW2_MAP_F16, FW2_MAP_IDX_U8 or FW2_MAP_IDX_U16 */
  double pml_rc;         /* reflection target R_c of Table 1 (default 1e-3) */
  double pml_npow;       /* polynomial order of the d ramp (default 2) */
  double pml_cp;         /* c_p of Table 1 [m/s]; <= 0: largest c of the medium */
  int32_t nl_mode;       /* FW2_NL_* */
  int32_t mem_alignment; /* FW2_MEM_CENTRED (default) or FW2_MEM_ENDPOINT */
  int32_t bc[3];         /* FW2_BC_* per axis */
  int32_t kernel_path;   /* FW2_PATH_* (default AUTO) */
  void *stream;          /* cudaStream_t, borrowed; NULL = default stream */
} fw2_config;

typedef struct {
  /* Interior relaxation parameters of every cell (Sec. 3.2, 2 + 4N values):
   * kappa1, kappa2: [n_pts]; d1, alpha1, d2, alpha2: [N][n_pts] in 1/s.
   * Inside the boundary region the library ramps d and alpha per axis
   * following Table 1; kappa is kept. */
  const float *kappa1;
  const float *kappa2;
  const float *d1;
  const float *alpha1;
  const float *d2;
  const float *alpha2;
  int32_t mem_space;
} fw2_relax_desc;

/* Fill *cfg with defaults (2D, N = 0, Taylor taps, CFL 0.4, R_c = 1e-3,
 * npow = 2, reading C, FP32 maps, linear, centred memory term, zero BC). */
fw2_status fw2_config_init(fw2_config *cfg);

/* Create a context for one grid (Sec. 3.1 staggered layout) and allocate its
 * device state: p, v_q and the 2 * ndim * N memory variables (Sec. 3.2),
 * zero-initialised.  EINVAL for bad sizes, ECUDA without a usable device. */
fw2_status fw2_create(const fw2_config *cfg, fw2_ctx **out);

/* Material of every cell (Eqs. wave1-wave2, general5-general6): sound speed
 * c [m/s], density rho [kg/m^3] and, when nl_mode != OFF, the coefficient of
 * nonlinearity beta = 1 + B/2A (nullable otherwise).  Each [n_pts]. */
fw2_status fw2_set_medium(fw2_ctx *ctx, const float *c, const float *rho,
                          const float *beta, int32_t mem_space);

/* Reduced-storage medium (map_precision FW2_MAP_IDX_U8 or FW2_MAP_IDX_U16):
 * every cell holds a tissue index tissue[n_pts] < n_tissue, uint8 with
 * n_tissue <= 256 or uint16 with n_tissue <= 65536, and the material and
 * relaxation parameters of Eqs. (wave1)-(general6) and Sec. 3.2 are
 * per-tissue tables: c, rho, beta (nullable when linear) [n_tissue];
 * relax->kappa1, kappa2 [n_tissue]; relax->d1, alpha1, d2, alpha2
 * [N][n_tissue].  The result equals fw2_set_medium + fw2_set_relaxation with
 * the tables gathered per cell; the C-PML still ramps per cell.  Replaces
 * both calls.  EINVAL on an index >= n_tissue or bad sizes. */
fw2_status fw2_set_medium_indexed(fw2_ctx *ctx, const void *tissue, int32_t n_tissue,
                                  const float *c, const float *rho, const float *beta,
                                  const fw2_relax_desc *relax, int32_t mem_space);

/* Relaxation parameters (Sec. 3.2, Table 2 shape); required when N > 0.
 * The coefficient maps (b = exp(-(d/kappa + alpha) dt),
 * a = d (b - 1) / (kappa (d + kappa alpha)), Eqs. relaxation_a/b; the C-PML
 * ramps of Table 1) are built on the device at the first fw2_step (or
 * fw2_get_dt) after medium and relaxation are set: K, rho, chi, 1/kappa and
 * the ramped d, alpha in FP64, rounded once; a and b in float (b - 1 through
 * expm1), a few float ulps from their FP64 values. */
fw2_status fw2_set_relaxation(fw2_ctx *ctx, const fw2_relax_desc *desc);

/* Add an additive source (the paper's transmit events, Sec. 4 and the
 * appendices): `kind` FW2_SRC_*; n_pts cell indices idx[] each fed by signal
 * column group[] (NULL: all column 0); signal is [n_steps][n_groups] and row n
 * is added to the field right after the half step of time step n.  Steps past
 * n_steps inject nothing.  May be called several times; entries accumulate. */
fw2_status fw2_add_source(fw2_ctx *ctx, int32_t kind, int64_t n_pts,
                          const int64_t *idx, const int32_t *group,
                          const float *signal, int64_t n_groups,
                          int64_t n_steps, int32_t mem_space);

/* Record p after every time step (sensor traces): trace row n, column g, is
 * the mean of p^{n+1} over the cells of group g (group NULL: one cell per
 * group, n_groups = n_pts).  out is caller-owned device memory of
 * [n_steps][n_groups] floats; row n is written by step n for n < n_steps.
 * idx/group follow mem_space.  Replaces any previous recording. */
fw2_status fw2_record(fw2_ctx *ctx, int64_t n_pts, const int64_t *idx,
                      const int32_t *group, int64_t n_groups, float *out,
                      int64_t n_steps, int32_t mem_space);

/* Advance n_steps time steps (Sec. 3.1 update order): velocity half step
 * with the nabla_1 memory variables, velocity sources, pressure half step
 * with the nabla_2 memory variables and the nonlinear factor, pressure
 * sources, recording.  Asynchronous on the context stream.  EINVAL when the
 * time step violates the stability limit of the staggered scheme. */
fw2_status fw2_step(fw2_ctx *ctx, int64_t n_steps);

/* Release every resource of the context (safe on NULL). */
fw2_status fw2_destroy(fw2_ctx *ctx);

/* ---- one grid split into subdomains --------------------------------------
 * The finite-difference step is local (Sec. 5 remarks that this suits
 * several GPUs): a grid split along its slowest axis (y in 2D, z in 3D) into
 * slabs advances each slab as its own context, given 4 extra rows on every
 * side where it borders another slab (the half-width of the 8th-order
 * operator).  Before each velocity half step those rows of p are copied in
 * from the neighbours, before each pressure half step those of v_q; the
 * slabs' own rows then hold exactly (bitwise) what one context of the whole
 * grid holds.  The extra rows are computed too and overwritten by the next
 * copy.  paper_2106_11476_gb300/slab.py drives this with contexts on one
 * device or with one process per device and torch.distributed for the
 * exchange. */

/* Declare the context's grid (extra rows included) as the box [offset,
 * offset + n) of a grid of extent global_n (cells per axis): the C-PML
 * depth of every cell is taken from its coordinate in the whole grid, so
 * the boundary lies at the whole grid's faces only.  Needs fw2_config.dt > 0
 * and, with a C-PML, pml_cp > 0 (the whole grid's values: a subdomain cannot
 * derive them from its own medium).  Call before the first step.  EINVAL
 * when the box leaves the grid, splits a periodic axis, or dt / pml_cp are
 * missing.  FP16 maps take their scales from the context's own cells, so
 * FP16 subdomains agree with the whole grid to the maps' rounding, not
 * bitwise (the other storages agree bitwise). */
fw2_status fw2_set_subdomain(fw2_ctx *ctx, const int64_t *global_n, const int64_t *offset);
/* One part of a time step, for an exchange between the half steps: part 0
 * is the velocity half step with the velocity sources, part 1 the pressure
 * half step with the pressure sources and the recording, after which the
 * step counter advances.  Parts alternate starting with 0; fw2_step is
 * refused (ESTATE) between the two.  Asynchronous like fw2_step. */
fw2_status fw2_step_part(fw2_ctx *ctx, int32_t part);
/* Copy rows [row0, row0 + n_rows) along the slowest axis (y rows in 2D, z
 * planes in 3D) of p or a velocity component (FW2_FIELD_P .. VZ) out to, or
 * in from, a dense buffer [n_rows][ny (3D)][nx] in host or device memory.
 * Synchronises the context stream.  EINVAL for other fields or rows outside
 * the grid. */
fw2_status fw2_get_rows(fw2_ctx *ctx, int32_t field, int64_t row0, int64_t n_rows, float *out,
                        int32_t mem_space);
fw2_status fw2_set_rows(fw2_ctx *ctx, int32_t field, int64_t row0, int64_t n_rows, const float *in,
                        int32_t mem_space);

/* In-loop blow-up detection (a numerical failure such as the C-PML
 * instability with N >= 2 and no transition layer, Sec. 3.3).  With
 * every > 0, fw2_step scans p after each step whose count is a multiple of
 * `every` and stops with FW2_EUNSTABLE when a value is not finite or
 * |p| > bound (fw2_last_error names the step and the value); the steps up to
 * the failing scan are taken and counted (fw2_get_step).  Each scan
 * synchronises the context stream once.  every = 0 (the default) switches
 * it off.  EINVAL for every < 0, or bound <= 0 with every > 0. */
fw2_status fw2_set_watch(fw2_ctx *ctx, int64_t every, float bound);

/* ---- batches ---------------------------------------------------------- */

/* Many contexts advanced together: the transmit events of a full
 * synthetic aperture sequence (appendix, abdominal wall imaging: one
 * simulation per transmitting element) or the requests of a serving loop.
 * Each context computes exactly what fw2_step computes for it alone; the
 * batch runs one persistent launch per half step over a work table of all
 * contexts (grouped by dimension, mechanism count and map kind, in 3D also
 * by the cross taps and the layout of each half step), one launch each for
 * the sources and recordings of all contexts, and replays chunks of steps
 * as a captured CUDA graph.  The first batch step warms up; the next twelve
 * time four launch configurations, three steps each, and the one with the
 * fastest median is kept; every configuration computes the same result.  A
 * configuration is a persistent grid size and tile order for the tile path
 * and, for the pipelined groups, the cost of an edge unit (C-PML strips,
 * clamps) relative to an interior one, 1.5, 2.5, 3.5 or 5, by which the work
 * table is split into the blocks' contiguous runs of about equal cost. */
typedef struct fw2_batch fw2_batch;
/* Contexts are borrowed (they must outlive the batch), with medium set;
 * their coefficient maps and sources are built here.  Re-create the batch
 * after changing a context's sources or recording.  3D contexts join on the
 * pipelined path only (bf16 maps, N <= 3, no periodic axis; EUNSUPPORTED
 * otherwise), each half step in its default layout. */
fw2_status fw2_batch_create(fw2_ctx *const *ctxs, int32_t n_ctx, fw2_batch **out);
/* Advance every context by n_steps (each from its own step counter), on the
 * batch's own stream after the contexts' streams have drained; asynchronous
 * except where the set of active contexts changes (see budgets). */
fw2_status fw2_batch_step(fw2_batch *b, int64_t n_steps);
/* Step budgets: context i leaves the batch once its step counter reaches
 * last_step[i] (< 0: no budget; NULL clears every budget).  fw2_batch_step
 * then advances each context by at most what its budget leaves; when a
 * context leaves, the launch tables are rebuilt for those that remain, so
 * finished contexts cost nothing (the transmit events of a sequence, or
 * served requests, of uneven lengths). */
fw2_status fw2_batch_set_budget(fw2_batch *b, const int64_t *last_step);
/* Number of contexts still short of their budget. */
fw2_status fw2_batch_active(fw2_batch *b, int32_t *n_active);
fw2_status fw2_batch_synchronize(fw2_batch *b);
/* Tuned persistent grid (0 before tuning), tile order (0 context-major,
 * 1 interleaved) and kernel launches (graph replays count their kernels once
 * at capture). */
fw2_status fw2_batch_info(fw2_batch *b, int32_t *grid, int32_t *order, int64_t *launches);
/* Tuned edge-unit cost of the pipelined groups' runs (0 before tuning). */
fw2_status fw2_batch_edge_weight(fw2_batch *b, double *weight);
const char *fw2_batch_last_error(const fw2_batch *b);
/* Blow-up detection for the batch (as fw2_set_watch): with every > 0, after
 * each batch step whose count (steps since the batch's first) is a multiple
 * of `every`, p of every context is scanned and fw2_batch_step stops with
 * FW2_EUNSTABLE when one holds a non-finite value or |p| > bound
 * (fw2_batch_last_error names the context); the steps up to that scan are
 * taken and counted on every context.  Synchronises the batch stream once
 * per scan.  EINVAL for every < 0, or bound <= 0 with every > 0. */
fw2_status fw2_batch_set_watch(fw2_batch *b, int64_t every, float bound);
fw2_status fw2_batch_destroy(fw2_batch *b);

/* ---- relaxation fitting (Sec. 4.1) -------------------------------------- */

/* Relaxation parameters that make the multiple-relaxation model follow a
 * power law: host computation in FP64, no device needed.  The model's
 * attenuation and phase velocity come from Eq. (dispersion_relations); the
 * cost is Eq. (relaxation_parameter_optimization),
 *   J = w_alpha NMSE(alpha_model, alpha_target) + (1 - w_alpha) NMSE(c_model, c_target),
 * NMSE = mean squared error over the variance of the target, on n_freq
 * uniform samples of [f_lo, f_hi]; the target is alpha0 f^y (dB/cm, f in MHz)
 * and its Kramers-Kronig phase velocity in the nearly-local form,
 * 1/c = 1/c0 + a0 tan(pi y / 2) (w^(y-1) - w_ref^(y-1)) (y = 1: 1/c0 -
 * (2 / pi) a0 ln(w / w_ref)), which equals c0 at f_ref.  The paper leaves
 * f_ref unstated; the default is the centre of the band, where Table 2's
 * own parameters score J = 0.024 (at 3 MHz they would score 2.2).
 * The search is the paper's: a grid of grid_points values per dimension
 * over the bounds (kappa linear, d and alpha in log10), then `refinements`
 * finer grids centred on the best point so far, each range narrower by
 * `shrink` (grid values beyond a bound move onto it), followed by an optional
 * Nelder-Mead polish in the same coordinates.  grid_points^(2 + 4N)
 * evaluations per grid (9.8e6 for N = 2 and 5 points) are spread over
 * `threads` host threads. */
#define FW2_FIT_MAX_RELAX 4
typedef struct {
  double alpha0;              /* attenuation coefficient [dB/cm/MHz^y] */
  double y;                   /* power-law exponent, 0 < y < 3 */
  int32_t n_relax;            /* N mechanisms, 1 .. FW2_FIT_MAX_RELAX */
  double c0;                  /* phase velocity at f_ref [m/s] */
  double f_ref;               /* Kramers-Kronig reference [Hz]; <= 0: band centre */
  double f_lo, f_hi;          /* fitted band [Hz] (default 1 - 20 MHz, Sec. 4.1) */
  int32_t n_freq;             /* uniform samples of the band (default 77) */
  double w_alpha;             /* weight of the attenuation term (default 0.1) */
  double kappa_bounds[2];     /* Table 2 bounds (default 0.8 - 1.2) */
  double log_d_bounds[2];     /* log10 of the d bounds [1/s] (default 2 - 10) */
  double log_alpha_bounds[2]; /* log10 of the alpha bounds [1/s] (default 5 - 12) */
  int32_t grid_points;        /* values per dimension of each grid (default 5) */
  int32_t refinements;        /* finer grids after the first (default 4) */
  double shrink;              /* range reduction per finer grid (default 0.3) */
  int32_t polish_iterations;  /* Nelder-Mead iterations after the grid (default 20000; 0: none) */
  int32_t threads;            /* host threads (0: all) */
} fw2_fit_request;
typedef struct {
  double kappa1, kappa2;      /* fitted parameters, the layout of fw2_relax_desc */
  double d1[FW2_FIT_MAX_RELAX], alpha1[FW2_FIT_MAX_RELAX];  /* [1/s] */
  double d2[FW2_FIT_MAX_RELAX], alpha2[FW2_FIT_MAX_RELAX];
  double J;                   /* cost of the result */
  double J_grid;              /* cost after the grid search, before the polish */
  double f_ref;               /* reference frequency used [Hz] */
  double max_att_rel_err;     /* max |alpha_model / alpha_target - 1| from 2 MHz up */
  double max_phase_rel_err;   /* max |c_model / c_target - 1| over the band */
  int64_t evaluations;        /* cost evaluations */
} fw2_fit_result;
/* Defaults above (alpha0 0.5, y 1, N 2, c0 1540: Table 2's target). */
fw2_status fw2_fit_request_init(fw2_fit_request *req);
/* Run the search.  EINVAL for arguments out of range or a grid of more than
 * 2e9 points; EUNSTABLE when no grid point has a finite cost. */
fw2_status fw2_fit_relaxation(const fw2_fit_request *req, fw2_fit_result *out);
/* Attenuation [dB/cm] and phase velocity [m/s] of a parameter set (the
 * first n_relax mechanisms of p) at n frequencies [Hz], from Eq.
 * (dispersion_relations) with c0 the sound speed of the medium. */
fw2_status fw2_relaxation_curves(const fw2_fit_result *p, int32_t n_relax, double c0, const double *freqs,
                                 int64_t n, double *att_db_cm, double *c);

/* ---- helpers ---------------------------------------------------------- */

/* Time step in use (builds the coefficient maps if needed). */
fw2_status fw2_get_dt(fw2_ctx *ctx, double *dt);
/* Number of time steps taken so far. */
fw2_status fw2_get_step(fw2_ctx *ctx, int64_t *step);
/* Set the step counter (source row and trace row of the next step); with
 * fw2_set_field this restores a checkpoint taken with fw2_get_step and
 * fw2_get_field. EINVAL when negative. */
fw2_status fw2_set_step(fw2_ctx *ctx, int64_t step);
/* Copy a state array (FW2_FIELD_*: p and v_q at the step's end, the memory
 * variables psi1_q, psi2_q of Eq. relaxation_psi) out into a caller-owned
 * buffer in host or device memory (mem_space) of n_pts floats, dense with x
 * fastest; the memory variables take N x n_pts ([N][n_pts]).  The buffer
 * must hold that many floats: the library cannot check its extent.
 * Synchronises the context stream.  Errors: FW2_EINVAL (a field the context
 * does not have, e.g. v_z of a 2D grid or psi with N = 0; null pointer),
 * FW2_ECUDA. */
fw2_status fw2_get_field(fw2_ctx *ctx, int32_t field, float *out, int32_t mem_space);
/* Overwrite a state array from a buffer of the same layout and extent (read
 * at call time; the caller keeps it); with fw2_set_step it restores a
 * checkpoint.  Errors as fw2_get_field. */
fw2_status fw2_set_field(fw2_ctx *ctx, int32_t field, const float *in, int32_t mem_space);
/* Zero every state array and the step counter. */
fw2_status fw2_reset(fw2_ctx *ctx);
/* Wait for the context stream.  FW2_ETIMEOUT when a bounded device-side
 * wait of a pipelined kernel gave up since the last fw2_reset (the state is
 * then incomplete; fw2_reset zeroes it and clears the flag), FW2_ECUDA on a
 * failed launch. */
fw2_status fw2_synchronize(fw2_ctx *ctx);
/* Scan p for non-finite values or |p| > bound (a numerical blow-up such as
 * the C-PML instability with N >= 2 and no transition layer, Sec. 3.3).
 * Synchronising.  *max_abs receives max |p| (inf if non-finite); returns
 * FW2_EUNSTABLE when the field fails, FW2_OK otherwise. */
fw2_status fw2_check_field(fw2_ctx *ctx, float bound, float *max_abs);
/* Field scan that allocates nothing.  The paper has no counterpart: this is
 * a service for callers that cannot allocate device memory -- applications
 * that own every device allocation themselves (a host framework's allocator,
 * a fixed memory budget that must account for each byte) or latency-critical
 * loops that cannot afford the device-wide synchronisation cudaMalloc and
 * cudaFree may cause.  It needs no context.
 * Computes max |x| over n_rows rows of row_len floats, row_pitch floats
 * apart, starting at `field` (device memory), and writes it to *out (device
 * memory); a non-finite value gives +inf.  Asynchronous on `stream` (NULL:
 * default stream).  Scratch: a file-scope device array of 2^20 floats
 * (4 MiB), one partial per row, held by every GPU that loads the library
 * until the process exits; n_rows above 2^20 is rejected with FW2_EINVAL.
 * Every call looks up that array's device address in the current context
 * (cudaGetSymbolAddress); the first call on a device may load the library's
 * device code, so it should come before any stream capture.  Calls share
 * the array: calls that overlap on the GPU race; each call overwrites every
 * row it uses, so nothing carries over.  Calls no cudaMalloc, cudaFree or
 * other allocating routine.  Errors: FW2_EINVAL (null pointer, a pointer
 * that is not device or managed memory of the current device, bad sizes),
 * FW2_ECUDA (launch failure); fw2_last_error(NULL) explains. */
fw2_status fw2_field_absmax_noalloc(const float *field, int64_t row_len, int64_t n_rows,
                                    int64_t row_pitch, float *out, void *stream);
/* Time-space optimised taps of the staggered operator of an ndim-dimensional
 * grid (2 or 3) for Courant number r = c dt / h (Sec. 3.1 cites such a set,
 * after Tan and Huang, without printing it; this is the library's derivation
 * from that principle).  Writes g[0..3] = g_{1,0}..g_{4,0} and g[4] = g_{1,1}
 * for fw2_config.g: with them the leapfrog dispersion relation
 * sin^2(w dt/2) = r^2 sum_q G_q^2 holds to order (k h)^4 in every direction
 * (4th order in time) and to (k h)^8 along the axes; at r = 0 they are the
 * Taylor set.  g_{1,1} = r^2 / 24 in both dimensions; g_{1,0} differs, since
 * along an axis of a 3D grid the cross tap has two transverse pairs.  Pure
 * host computation, no device needed.  Errors: FW2_EINVAL (g NULL, r outside
 * [0, 1), ndim not 2 or 3). */
fw2_status fw2_taps_time_space(double r, int32_t ndim, double *g);
/* Self-test of the bounded device-side wait that every pipelined kernel uses
 * on its copy barriers (the paper has no counterpart; it guards against a
 * hung GPU).  Launches one block that initialises an mbarrier nobody ever
 * arrives on and waits for it with a limit of limit_ns nanoseconds (1 ..
 * 10^10); *timed_out (host) becomes 1 when the wait gave up, as it must, and
 * 0 otherwise.  Synchronous on the default stream; needs no context.  Errors:
 * FW2_EINVAL (null pointer, limit out of range), FW2_ECUDA. */
fw2_status fw2_selftest_bounded_wait(int64_t limit_ns, int32_t *timed_out);
/* Kernel path the context's half steps take, resolved once the coefficients
 * are built (first fw2_step): FW2_PATH_TILE or FW2_PATH_PIPE; FW2_PATH_AUTO
 * before the first step. */
fw2_status fw2_kernel_path(fw2_ctx *ctx, int32_t *path);
/* Layout of the 3D pipelined velocity and pressure half steps: 1 memory
 * variables staged, 2 in registers, 0 before the choice (or not a 3D
 * pipelined context). */
fw2_status fw2_pipe_layout(fw2_ctx *ctx, int32_t *vel, int32_t *prs);
/* Return the free memory of the library's pool on the current device to
 * the driver (synchronises the device). */
fw2_status fw2_release_memory(void);
/* Bytes of device memory held by the context. */
fw2_status fw2_device_bytes(fw2_ctx *ctx, int64_t *bytes);
/* Launches of library kernels since creation (all kinds). */
fw2_status fw2_kernel_launches(fw2_ctx *ctx, int64_t *count);
/* Per-kernel timing: with enable = 1, fw2_step brackets every velocity and
 * pressure kernel launch with CUDA events on the context stream. */
fw2_status fw2_profile(fw2_ctx *ctx, int32_t enable);
/* Synchronise and return the summed event time [ms] and launch counts of the
 * velocity and pressure kernels since profiling was enabled; clears them. */
fw2_status fw2_profile_read(fw2_ctx *ctx, double *vel_ms, int64_t *vel_launches,
                            double *prs_ms, int64_t *prs_launches);
/* Last error message of the context (or of the last failed fw2_create when
 * ctx is NULL); never NULL. */
const char *fw2_last_error(const fw2_ctx *ctx);
/* ABI version of this header (incremented on incompatible change). */
int32_t fw2_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FW2_H */
