/*
 * Plain FP64 CPU oracle of the Fullwave 2 time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (Sode & Pinton, "Fullwave 2", arXiv 2106.11476):
 *   - the stretched first-order pressure / particle-velocity system,
 *     Eqs. (wave1)-(wave2), in its nonlinear form Eqs. (general5)-(general6);
 *   - on the staggered grid of Sec. 3.1 (p at cell centres, v_q at the
 *     +1/2 face along axis q), with the 2M-th order operator D of Sec. 3.1
 *     (M = 4 taps g_1..g_4 plus the g_{1,1} cross term);
 *   - each derivative stretched by Eq. (relaxation4): D/kappa + sum_nu psi^nu,
 *     with the memory variables advanced by the recursion Eq. (relaxation_psi)
 *     psi^n = b psi^{n-1} + a D^{n-1/2}.
 *
 * Time alignment of the memory term.  The staggered update only has the
 * derivative D^n at the centre of the update, not D^{n-1/2}.  The stored
 * variable chi follows chi^n = b chi^{n-1} + a D^n.  With centred = 1 the
 * stretched derivative uses (chi^n + chi^{n-1}) / 2, which is exactly the
 * recursion driven by (D^n + D^{n-1}) / 2, the second-order estimate of
 * D^{n-1/2}.  With centred = 0 it uses chi^n (endpoint: D^{n-1/2} taken as
 * D^n, the usual C-PML practice).
 *
 * The coefficients (a, b, 1/kappa, 1/rho at faces, K = rho c^2, chi) are
 * inputs here: the Python side of the oracle builds them from the paper's
 * closed forms.  Every loop below is a direct transcription of one step of
 * the method, point by point, with no tiling, fusion or reordering.
 * OpenMP only splits the outermost loop of independent points.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t ndim;      /* 1, 2 or 3 */
  int32_t nrelax;    /* N, number of relaxation mechanisms */
  int64_t n[3];      /* nx, ny, nz; unused axes have extent 1; x fastest */
  int32_t bc[3];     /* 0: fields are zero outside the grid, 1: periodic */
  int32_t centred;   /* 1: memory term time-centred, 0: endpoint (see below) */
  double dt;         /* time step [s] */
  double h;          /* grid spacing [m] */
  double g[4];       /* g_{i,0}, i = 1..4, of the staggered operator */
  double g11;        /* g_{1,1} cross-term weight */
} orc_grid;

typedef struct {
  const double *K;          /* [n] rho c^2 at cell centres */
  const double *chi;        /* [n] nonlinear coefficient, NULL when linear */
  const double *buoy[3];    /* [n] 1/rho at the +1/2 face of axis q */
  const double *ik1[3];     /* [n] 1/kappa_1 at the +1/2 face of axis q */
  const double *a1[3];      /* [N][n] recursion weight a for nabla_1, axis q */
  const double *b1[3];      /* [N][n] recursion decay b for nabla_1, axis q */
  const double *ik2[3];     /* [n] 1/kappa_2 at cell centres, axis q */
  const double *a2[3];      /* [N][n] */
  const double *b2[3];      /* [N][n] */
  const double *k0f[3];     /* [n] kappa_0 = 1/K at the +1/2 face of axis q (mean of
                               the two cells); NULL: no nonlinear factor in the
                               momentum equation */
} orc_coef;

typedef struct {
  double *p;         /* [n]    pressure at t_n */
  double *v[3];      /* [n]    velocity component q at t_{n-1/2} */
  double *psi1[3];   /* [N][n] memory variables of nabla_1 (faces) */
  double *psi2[3];   /* [N][n] memory variables of nabla_2 (centres) */
} orc_state;

typedef struct {
  int64_t n_pts;          /* number of (point, column) source entries */
  const int32_t *kind;    /* 0: pressure, 1..3: velocity component x,y,z */
  const int64_t *idx;     /* flat cell index of each entry */
  const int32_t *col;     /* column of the signal table feeding each entry */
  const double *signal;   /* [n_rows][n_cols] additive source values */
  int64_t n_cols;
  int64_t n_rows;         /* steps at or past n_rows inject nothing */
} orc_sources;

typedef struct {
  int64_t n_pts;          /* number of recorded cells */
  const int64_t *idx;     /* flat cell index */
  const int32_t *group;   /* sensor (group) of each cell */
  int64_t n_groups;
  double *trace;          /* [n_rows][n_groups], mean of p over each group */
  int64_t n_rows;         /* steps at or past n_rows record nothing */
} orc_record;

static int64_t npts(const orc_grid *G) { return G->n[0] * G->n[1] * G->n[2]; }

/* Value of a cell-indexed field at integer coordinates c, following the
 * outer boundary rule: zero outside the grid, or periodic wrap. */
static double fetch(const orc_grid *G, const double *f, int64_t i, int64_t j,
                    int64_t k) {
  int64_t c[3] = {i, j, k};
  for (int q = 0; q < 3; q++) {
    int64_t n = G->n[q];
    if (c[q] < 0 || c[q] >= n) {
      if (G->bc[q] == 1) {
        c[q] = ((c[q] % n) + n) % n;
      } else {
        return 0.0;
      }
    }
  }
  return f[c[0] + G->n[0] * (c[1] + G->n[1] * c[2])];
}

/* Staggered derivative of p along axis q at the face c + 1/2 e_q,
 * Sec. 3.1 operator D^{2M,4}:
 *   (1/h)[ sum_i g_i (p(c + i e_q) - p(c - (i-1) e_q))
 *          + g11 sum_{t != q} sum_{s=+-1} (p(c + e_q + s e_t) - p(c + s e_t)) ]
 * p(c+i e_q) is the value half a cell beyond the face plus (i-1) cells, so
 * the pair is the printed p_{i-1/2} - p_{-i+1/2}. */
static double d_face(const orc_grid *G, const double *p, int q, int64_t i,
                     int64_t j, int64_t k) {
  int64_t e[3] = {0, 0, 0};
  e[q] = 1;
  double acc = 0.0;
  for (int m = 1; m <= 4; m++) {
    double hi = fetch(G, p, i + m * e[0], j + m * e[1], k + m * e[2]);
    double lo = fetch(G, p, i - (m - 1) * e[0], j - (m - 1) * e[1],
                      k - (m - 1) * e[2]);
    acc += G->g[m - 1] * (hi - lo);
  }
  if (G->g11 != 0.0) {
    for (int t = 0; t < G->ndim; t++) {
      if (t == q) continue;
      for (int s = -1; s <= 1; s += 2) {
        int64_t o[3] = {0, 0, 0};
        o[t] = s;
        double hi = fetch(G, p, i + e[0] + o[0], j + e[1] + o[1], k + e[2] + o[2]);
        double lo = fetch(G, p, i + o[0], j + o[1], k + o[2]);
        acc += G->g11 * (hi - lo);
      }
    }
  }
  return acc / G->h;
}

/* Staggered derivative of v_q along axis q at the cell centre c.
 * v_q stored at index c lives at c + 1/2 e_q, so the pair
 * v(c + (i-1/2) e_q) - v(c - (i-1/2) e_q) is v[c + (i-1)e_q] - v[c - i e_q]. */
static double d_centre(const orc_grid *G, const double *v, int q, int64_t i,
                       int64_t j, int64_t k) {
  int64_t e[3] = {0, 0, 0};
  e[q] = 1;
  double acc = 0.0;
  for (int m = 1; m <= 4; m++) {
    double hi = fetch(G, v, i + (m - 1) * e[0], j + (m - 1) * e[1],
                      k + (m - 1) * e[2]);
    double lo = fetch(G, v, i - m * e[0], j - m * e[1], k - m * e[2]);
    acc += G->g[m - 1] * (hi - lo);
  }
  if (G->g11 != 0.0) {
    for (int t = 0; t < G->ndim; t++) {
      if (t == q) continue;
      for (int s = -1; s <= 1; s += 2) {
        int64_t o[3] = {0, 0, 0};
        o[t] = s;
        double hi = fetch(G, v, i + o[0], j + o[1], k + o[2]);
        double lo = fetch(G, v, i - e[0] + o[0], j - e[1] + o[1], k - e[2] + o[2]);
        acc += G->g11 * (hi - lo);
      }
    }
  }
  return acc / G->h;
}

/* Velocity half step, Sec. 3.1 (u, v updates) with the stretched derivative
 * of Eq. (relaxation4) and the recursion Eq. (relaxation_psi):
 *   D      = D_q p^n at the face
 *   psi_nu = b psi_nu + a D                     (nu = 1..N)
 *   S      = D / kappa_1 + sum_nu psi_nu        (or the mean of old and new
 *                                                psi_nu when centred)
 *   v_q   -= dt * (1/rho_face) * S               (Eq. general5, linear in rho)
 * With the momentum equation's nonlinear factor (k0f given, Eq. general5 as
 * printed: rho_0 (1 + kappa_0 p)) the update is divided by
 * 1 + kappa_0,face p_face, p_face the mean of p^n at the face's two cells. */
static void velocity_half_step(const orc_grid *G, const orc_coef *C,
                               orc_state *S) {
  const int64_t n = npts(G);
  const int N = G->nrelax;
  for (int q = 0; q < G->ndim; q++) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < G->n[2]; k++) {
      for (int64_t j = 0; j < G->n[1]; j++) {
        for (int64_t i = 0; i < G->n[0]; i++) {
          int64_t c = i + G->n[0] * (j + G->n[1] * k);
          double D = d_face(G, S->p, q, i, j, k);
          double stretched = D * C->ik1[q][c];
          for (int nu = 0; nu < N; nu++) {
            double *psi = &S->psi1[q][(int64_t)nu * n + c];
            double old = *psi;
            *psi = C->b1[q][(int64_t)nu * n + c] * old +
                   C->a1[q][(int64_t)nu * n + c] * D;
            stretched += G->centred ? 0.5 * (old + *psi) : *psi;
          }
          double upd = G->dt * C->buoy[q][c] * stretched;
          if (C->k0f[q]) {
            int64_t e[3] = {0, 0, 0};
            e[q] = 1;
            const double pf = 0.5 * (S->p[c] + fetch(G, S->p, i + e[0], j + e[1], k + e[2]));
            upd /= 1.0 + C->k0f[q][c] * pf;
          }
          S->v[q][c] -= upd;
        }
      }
    }
  }
}

/* Pressure half step, Sec. 3.1 (p update) with Eq. (general6):
 *   S_q = D_q v_q / kappa_2 + sum_nu psi2_nu  (psi2 advanced first)
 *   p  -= dt * K * sum_q S_q / (1 + chi p^n)
 * chi = kappa_0 (1 - 2 beta) is the factor printed in Eq. (general6); the
 * caller may pass another per-point chi (or none for the linear system). */
static void pressure_half_step(const orc_grid *G, const orc_coef *C,
                               orc_state *S) {
  const int64_t n = npts(G);
  const int N = G->nrelax;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < G->n[2]; k++) {
    for (int64_t j = 0; j < G->n[1]; j++) {
      for (int64_t i = 0; i < G->n[0]; i++) {
        int64_t c = i + G->n[0] * (j + G->n[1] * k);
        double div = 0.0;
        for (int q = 0; q < G->ndim; q++) {
          double D = d_centre(G, S->v[q], q, i, j, k);
          double stretched = D * C->ik2[q][c];
          for (int nu = 0; nu < N; nu++) {
            double *psi = &S->psi2[q][(int64_t)nu * n + c];
            double old = *psi;
            *psi = C->b2[q][(int64_t)nu * n + c] * old +
                   C->a2[q][(int64_t)nu * n + c] * D;
            stretched += G->centred ? 0.5 * (old + *psi) : *psi;
          }
          div += stretched;
        }
        double factor = 1.0;
        if (C->chi) factor = 1.0 + C->chi[c] * S->p[c];
        S->p[c] -= G->dt * C->K[c] * div / factor;
      }
    }
  }
}

/* Additive sources (the paper drives its transducers with the pulse of
 * Sec. 4.5 without stating how they couple to the field; adding the signal
 * is the plain reading): signal row `step` added to p or to one velocity
 * component at the source cells. */
static void add_sources(const orc_sources *src, orc_state *S, int64_t step,
                        int want_pressure) {
  if (!src || src->n_pts == 0 || step >= src->n_rows) return;
  for (int64_t e = 0; e < src->n_pts; e++) {
    int kind = src->kind[e];
    if ((kind == 0) != (want_pressure != 0)) continue;
    double s = src->signal[step * src->n_cols + src->col[e]];
    if (kind == 0) {
      S->p[src->idx[e]] += s;
    } else {
      S->v[kind - 1][src->idx[e]] += s;
    }
  }
}

/* Sensor traces (the recorded pressure of Secs. 4.2-4.5): trace row `step`
 * holds p^{n+1} averaged over the cells of each sensor group (array
 * elements record the mean over their cells). */
static void record(const orc_record *rec, const orc_state *S, int64_t step) {
  if (!rec || rec->n_pts == 0 || step >= rec->n_rows) return;
  double *row = rec->trace + step * rec->n_groups;
  int64_t *count = (int64_t *)calloc((size_t)rec->n_groups, sizeof(int64_t));
  for (int64_t g = 0; g < rec->n_groups; g++) row[g] = 0.0;
  for (int64_t e = 0; e < rec->n_pts; e++) {
    row[rec->group[e]] += S->p[rec->idx[e]];
    count[rec->group[e]] += 1;
  }
  for (int64_t g = 0; g < rec->n_groups; g++)
    if (count[g] > 0) row[g] /= (double)count[g];
  free(count);
}

/* One full time step n -> n+1 in the order: velocity half step, velocity
 * sources (row `step`), pressure half step, pressure sources (row `step`),
 * recording of p^{n+1} into trace row `step`. */
void orc_step(const orc_grid *G, const orc_coef *C, orc_state *S,
              const orc_sources *src, orc_record *rec, int64_t step) {
  velocity_half_step(G, C, S);
  add_sources(src, S, step, 0);
  pressure_half_step(G, C, S);
  add_sources(src, S, step, 1);
  record(rec, S, step);
}

/* n_steps time steps starting at step index `first` (source and trace rows
 * are indexed by the absolute step). */
void orc_run(const orc_grid *G, const orc_coef *C, orc_state *S,
             const orc_sources *src, orc_record *rec, int64_t first,
             int64_t n_steps) {
  for (int64_t s = 0; s < n_steps; s++) orc_step(G, C, S, src, rec, first + s);
}

/* Helpers used by the pins: the raw staggered derivatives of one field. */
void orc_derivative_face(const orc_grid *G, const double *p, int q, double *out) {
  for (int64_t k = 0; k < G->n[2]; k++)
    for (int64_t j = 0; j < G->n[1]; j++)
      for (int64_t i = 0; i < G->n[0]; i++)
        out[i + G->n[0] * (j + G->n[1] * k)] = d_face(G, p, q, i, j, k);
}

void orc_derivative_centre(const orc_grid *G, const double *v, int q, double *out) {
  for (int64_t k = 0; k < G->n[2]; k++)
    for (int64_t j = 0; j < G->n[1]; j++)
      for (int64_t i = 0; i < G->n[0]; i++)
        out[i + G->n[0] * (j + G->n[1] * k)] = d_centre(G, v, q, i, j, k);
}

int orc_abi_version(void) { return 1; }
