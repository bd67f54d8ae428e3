/*
 * bp_oracle.c -- plain, slow FP64 CPU oracle for the two-body macro-ion PIC step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load this file:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg use it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (arXiv 2208.08038, An, Chen, Sheng, Zhang):
 *   - species split of a partially ionised ion into a nucleus (q1, m1) and a
 *     combined bound electron (q2, m2)                              Sec. 2, P2
 *   - initial conditions r1 = r2 = rc, p1 + p2 = pc, q1 v1 + q2 v2 = 0  Sec. 2
 *   - modified Coulomb internal force q1 q2 r / (4 pi eps0 (r^2+ac^2)^3/2)
 *     added to the electric field seen by each body                 Sec. 2
 *   - natural frequency wc^2 = |q1 q2| / (4 pi eps0 m_r ac^3), used to map a
 *     requested bound-electron frequency onto ac                    Sec. 3.1
 *   - relativistic Boris push of each body with the fields at its own
 *     position                                                       Sec. 2, Boris equations
 *   - current of each body q v / dV added to the total current     Sec. 2
 *   - vacuum Maxwell equations, unchanged                           Sec. 3.1
 * Discrete choices the paper leaves open (documented in the design doc):
 *   Yee FDTD fields, quadratic B-spline shape for gather and deposit, the
 *   Esirkepov charge-conserving current, Mur first-order open faces, a
 *   current-sheet laser antenna, normalised units (c = 1, lengths in 1/k0,
 *   times in 1/w0, E in m_e c w0 / e, densities in n_c).
 *
 * Every loop is the definition written out: no blocking, no fusion, no
 * reordering of sums.  OpenMP is used only on per-cell field loops whose
 * iterations are independent, so the result is identical to a serial run.
 * Positions are kept unwrapped (continuous); only grid indices wrap on
 * periodic axes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXSP 8
#define OR_MAXLASER 4
#define OR_MAXPROBE 32

enum { OR_PERIODIC = 0, OR_OPEN = 1 };
enum { OR_TWO_BODY = 0, OR_FREE = 1 };

/* classical electron radius [m] (CODATA 2018) */
static const double OR_RE = 2.8179403262e-15;

typedef struct {
  int kind;
  double q1, m1, q2, m2; /* body charges [e] and masses [m_e]; free: q1, m1 only */
  double w;              /* density weight: one particle adds q*w*S to rho [n_c] */
  double kappa;          /* r_e k0: the Coulomb constant in normalised units */
  double *ac;            /* modified-Coulomb softening a_c per parameter index */
  int nac;
  int64_t n, cap;
  double *x1, *x2, *u1, *u2; /* [n][3], normalised units, positions unwrapped */
  int32_t *pidx;             /* parameter index per ion (NULL: all use ac[0]) */
  unsigned char *alive;
} or_species;

typedef struct {
  int comp; /* 1: current along y (p-polarised in x-y, or 1D y), 2: along z */
  double a0, omega, theta, waist, fwhm, t0, ramp, phase;
  long ia;  /* x node index of the antenna plane */
  double yc, zc;
} or_laser;

typedef struct {
  int comp; /* 0..8: Ex Ey Ez Bx By Bz Jx Jy Jz */
  int64_t npts;
  int64_t *idx;
  int64_t cap, count; /* samples (each npts values) */
  double *data;
} or_probe;

typedef struct or_sim {
  int D;
  long n[3];
  double dx[3];
  double dt;
  int bc[3];
  long ncell;
  double *F[9]; /* Ex Ey Ez Bx By Bz Jx Jy Jz, x fastest */
  double *Eold[3];
  int nsp;
  or_species sp[OR_MAXSP];
  int nl;
  or_laser las[OR_MAXLASER];
  int np;
  or_probe pr[OR_MAXPROBE];
  int64_t step;
  int fields_on, deposit_on;
  double free_lo[3], free_hi[3]; /* free particles leaving [lo, hi) cells on an open axis are removed */
} or_sim;

/* Yee stagger (in cells) of E, B and J components along x, y, z. */
static const double STAG_E[3][3] = {{0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}};
static const double STAG_B[3][3] = {{0, 0.5, 0.5}, {0.5, 0, 0.5}, {0.5, 0.5, 0}};

/* ------------------------------------------------------------------------ */
/* grid helpers                                                              */

static long wrap_axis(const or_sim *s, int a, long i) {
  if (a >= s->D) return (i == 0) ? 0 : -1;
  if (s->bc[a] == OR_PERIODIC) {
    long m = i % s->n[a];
    return m < 0 ? m + s->n[a] : m;
  }
  return (i < 0 || i >= s->n[a]) ? -1 : i;
}

/* linear index of (i,j,k) after periodic wrap; -1 when outside an open axis */
static long lin(const or_sim *s, long i, long j, long k) {
  long a = wrap_axis(s, 0, i), b = wrap_axis(s, 1, j), c = wrap_axis(s, 2, k);
  if (a < 0 || b < 0 || c < 0) return -1;
  return a + s->n[0] * (b + s->n[1] * c);
}

static double val(const double *F, long idx) { return idx < 0 ? 0.0 : F[idx]; }

/* ------------------------------------------------------------------------ */
/* shape: the quadratic B-spline (second order, three-point support)         */

double or_shape(double xi) {
  double a = fabs(xi);
  if (a <= 0.5) return 0.75 - xi * xi;
  if (a < 1.5) {
    double t = 1.5 - a;
    return 0.5 * t * t;
  }
  return 0.0;
}

/* ------------------------------------------------------------------------ */
/* creation                                                                  */

or_sim *or_create(int D, const long n[3], const double dx[3], double dt, const int bc[3]) {
  if (D < 1 || D > 3) return NULL;
  or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
  s->D = D;
  for (int a = 0; a < 3; ++a) {
    s->n[a] = (a < D) ? n[a] : 1;
    s->dx[a] = (a < D) ? dx[a] : 1.0;
    s->bc[a] = (a < D) ? bc[a] : OR_PERIODIC;
    s->free_lo[a] = -1e300;
    s->free_hi[a] = 1e300;
  }
  s->dt = dt;
  s->ncell = s->n[0] * s->n[1] * s->n[2];
  for (int c = 0; c < 9; ++c) s->F[c] = (double *)calloc((size_t)s->ncell, sizeof(double));
  for (int c = 0; c < 3; ++c) s->Eold[c] = (double *)calloc((size_t)s->ncell, sizeof(double));
  s->fields_on = 1;
  s->deposit_on = 1;
  return s;
}

void or_destroy(or_sim *s) {
  if (!s) return;
  for (int c = 0; c < 9; ++c) free(s->F[c]);
  for (int c = 0; c < 3; ++c) free(s->Eold[c]);
  for (int i = 0; i < s->nsp; ++i) {
    or_species *p = &s->sp[i];
    free(p->ac); free(p->x1); free(p->x2); free(p->u1); free(p->u2); free(p->pidx); free(p->alive);
  }
  for (int i = 0; i < s->np; ++i) { free(s->pr[i].idx); free(s->pr[i].data); }
  free(s);
}

double *or_field_ptr(or_sim *s, int comp) { return (comp >= 0 && comp < 9) ? s->F[comp] : NULL; }
long or_ncell(const or_sim *s) { return s->ncell; }
int64_t or_step_index(const or_sim *s) { return s->step; }
void or_set_switches(or_sim *s, int fields_on, int deposit_on) { s->fields_on = fields_on; s->deposit_on = deposit_on; }
void or_set_free_bounds(or_sim *s, const double lo[3], const double hi[3]) {
  for (int a = 0; a < 3; ++a) { s->free_lo[a] = lo[a]; s->free_hi[a] = hi[a]; }
}

/* ------------------------------------------------------------------------ */
/* species                                                                   */

/* Natural frequency of the two-body system from the Taylor expansion of the
 * modified Coulomb potential (Sec. 3.1): wc^2 = |q1 q2| kappa / (m_r ac^3),
 * solved for ac.  kappa = r_e k0 is 1/(4 pi eps0) in normalised units. */
double or_omega_to_ac(double q1, double m1, double q2, double m2, double kappa, double omega) {
  double mr = m1 * m2 / (m1 + m2);
  return cbrt(fabs(q1 * q2) * kappa / (mr * omega * omega));
}

/* Species split (Sec. 2): q2 = -Z_b e, m2 = Z_b m_e, q1 = q_c - q2, m1 = m_c - m2.
 * kappa = r_e * 2 pi / lambda0_phys.  omega_b[i] (units of w0) gives ac[i]. */
int or_add_two_body(or_sim *s, double Zb, double qc, double mc, double w, double lambda0_m,
                    const double *omega_b, int n_omega) {
  if (s->nsp >= OR_MAXSP || n_omega < 1) return -1;
  or_species *p = &s->sp[s->nsp];
  memset(p, 0, sizeof(*p));
  p->kind = OR_TWO_BODY;
  p->q2 = -Zb;
  p->m2 = Zb;
  p->q1 = qc - p->q2;
  p->m1 = mc - p->m2;
  p->w = w;
  p->kappa = OR_RE * 2.0 * M_PI / lambda0_m;
  p->nac = n_omega;
  p->ac = (double *)malloc(sizeof(double) * (size_t)n_omega);
  for (int i = 0; i < n_omega; ++i)
    p->ac[i] = or_omega_to_ac(p->q1, p->m1, p->q2, p->m2, p->kappa, omega_b[i]);
  return s->nsp++;
}

int or_add_free(or_sim *s, double q, double m, double w) {
  if (s->nsp >= OR_MAXSP) return -1;
  or_species *p = &s->sp[s->nsp];
  memset(p, 0, sizeof(*p));
  p->kind = OR_FREE;
  p->q1 = q;
  p->m1 = m;
  p->w = w;
  return s->nsp++;
}

/* out: q1 m1 q2 m2 w kappa nac n */
void or_species_info(const or_sim *s, int id, double out[8]) {
  const or_species *p = &s->sp[id];
  out[0] = p->q1; out[1] = p->m1; out[2] = p->q2; out[3] = p->m2;
  out[4] = p->w; out[5] = p->kappa; out[6] = p->nac; out[7] = (double)p->n;
}

double or_species_ac(const or_sim *s, int id, int i) { return s->sp[id].ac[i]; }

/* replace the a_c table from bound-electron frequencies (used by the adjoint's
 * finite-difference checks) */
void or_set_omega(or_sim *s, int id, const double *omega_b, int n) {
  or_species *p = &s->sp[id];
  for (int i = 0; i < n && i < p->nac; ++i)
    p->ac[i] = or_omega_to_ac(p->q1, p->m1, p->q2, p->m2, p->kappa, omega_b[i]);
}

static void reserve(or_species *p, int64_t n) {
  p->cap = n;
  p->x1 = (double *)calloc((size_t)(3 * n), sizeof(double));
  p->u1 = (double *)calloc((size_t)(3 * n), sizeof(double));
  p->x2 = (double *)calloc((size_t)(3 * n), sizeof(double));
  p->u2 = (double *)calloc((size_t)(3 * n), sizeof(double));
  p->pidx = (int32_t *)calloc((size_t)n, sizeof(int32_t));
  p->alive = (unsigned char *)malloc((size_t)n);
  memset(p->alive, 1, (size_t)n);
}

/* Load ions (or free particles) from ion-level positions xc [n][D] and
 * momenta uc = p_c/(m_c c) [n][3].  Initial conditions of Sec. 2:
 *   r1 = r2 = r_c;   p1 + p2 = p_c;   q1 v1 + q2 v2 = 0.
 * For q_c = 0 the two conditions give v1 = v2, i.e. u1 = u2 = u_c exactly.
 * For q_c != 0 the split is taken in the non-relativistic limit
 * (u ~ v): u1 = m_c u_c / (m1 - m2 q1/q2), u2 = -q1 u1 / q2. */
int or_load_ions(or_sim *s, int id, int64_t n, const double *xc, const double *uc, const int32_t *pidx) {
  or_species *p = &s->sp[id];
  if (p->n) return -1;
  reserve(p, n);
  p->n = n;
  for (int64_t i = 0; i < n; ++i) {
    for (int a = 0; a < 3; ++a) {
      double x = (a < s->D) ? xc[i * s->D + a] : 0.0;
      p->x1[3 * i + a] = x;
      p->x2[3 * i + a] = x;
    }
    if (pidx) p->pidx[i] = pidx[i];
    for (int a = 0; a < 3; ++a) {
      double u = uc ? uc[3 * i + a] : 0.0;
      if (p->kind == OR_FREE) {
        p->u1[3 * i + a] = u;
      } else if (p->q1 + p->q2 == 0.0) {
        p->u1[3 * i + a] = u;
        p->u2[3 * i + a] = u;
      } else {
        double mc = p->m1 + p->m2;
        double u1 = mc * u / (p->m1 - p->m2 * p->q1 / p->q2);
        p->u1[3 * i + a] = u1;
        p->u2[3 * i + a] = -p->q1 * u1 / p->q2;
      }
    }
  }
  return 0;
}

/* raw access to body states (tests set e.g. an initial internal displacement) */
void or_get_bodies(const or_sim *s, int id, double *x1, double *x2, double *u1, double *u2) {
  const or_species *p = &s->sp[id];
  size_t b = sizeof(double) * (size_t)(3 * p->n);
  if (x1) memcpy(x1, p->x1, b);
  if (u1) memcpy(u1, p->u1, b);
  if (p->kind == OR_TWO_BODY) {
    if (x2) memcpy(x2, p->x2, b);
    if (u2) memcpy(u2, p->u2, b);
  }
}

void or_set_bodies(or_sim *s, int id, const double *x1, const double *x2, const double *u1, const double *u2) {
  or_species *p = &s->sp[id];
  size_t b = sizeof(double) * (size_t)(3 * p->n);
  if (x1) memcpy(p->x1, x1, b);
  if (u1) memcpy(p->u1, u1, b);
  if (x2) memcpy(p->x2, x2, b);
  if (u2) memcpy(p->u2, u2, b);
}

void or_get_alive(const or_sim *s, int id, unsigned char *out) {
  memcpy(out, s->sp[id].alive, (size_t)s->sp[id].n);
}

/* ------------------------------------------------------------------------ */
/* lasers and probes                                                         */

/* p: comp a0 omega theta waist fwhm t0 ramp phase ia yc zc */
int or_add_laser(or_sim *s, const double p[12]) {
  if (s->nl >= OR_MAXLASER) return -1;
  or_laser *L = &s->las[s->nl];
  L->comp = (int)p[0];
  L->a0 = p[1]; L->omega = p[2]; L->theta = p[3]; L->waist = p[4];
  L->fwhm = p[5]; L->t0 = p[6]; L->ramp = p[7]; L->phase = p[8];
  L->ia = (long)p[9]; L->yc = p[10]; L->zc = p[11];
  return s->nl++;
}

int or_add_probe(or_sim *s, int comp, int64_t npts, const int64_t *idx, int64_t cap) {
  if (s->np >= OR_MAXPROBE) return -1;
  or_probe *P = &s->pr[s->np];
  P->comp = comp;
  P->npts = npts;
  P->idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)npts);
  memcpy(P->idx, idx, sizeof(int64_t) * (size_t)npts);
  P->cap = cap;
  P->count = 0;
  P->data = (double *)calloc((size_t)(cap * npts), sizeof(double));
  return s->np++;
}

int64_t or_probe_data(const or_sim *s, int id, double *out) {
  const or_probe *P = &s->pr[id];
  if (out) memcpy(out, P->data, sizeof(double) * (size_t)(P->count * P->npts));
  return P->count;
}

static void record_probes(or_sim *s) {
  for (int i = 0; i < s->np; ++i) {
    or_probe *P = &s->pr[i];
    if (P->count >= P->cap) continue;
    for (int64_t q = 0; q < P->npts; ++q) P->data[P->count * P->npts + q] = s->F[P->comp][P->idx[q]];
    P->count++;
  }
}

/* Antenna: a current sheet on the x node plane ia.  A sheet K radiates
 * E = -K/2 to either side (c = 1), so K = -2 f(t) launches f(t) forward.
 * The grid carries the sheet as J = K/dx on one node plane.  s-polarisation
 * (current along z) scales K by cos(theta) so the oblique wave keeps
 * amplitude a0. */
double or_laser_value(const or_laser *L, double t, double y, double z) {
  double ty = y - L->yc, tz = z - L->zc;
  double tau = t - ty * sin(L->theta);
  double env;
  if (L->fwhm > 0) {
    double d = tau - L->t0;
    env = exp(-2.0 * log(2.0) * d * d / (L->fwhm * L->fwhm));
  } else {
    if (tau <= 0) env = 0.0;
    else if (tau < L->ramp) { double sn = sin(0.5 * M_PI * tau / L->ramp); env = sn * sn; }
    else env = 1.0;
  }
  double prof = 1.0;
  if (L->waist > 0) {
    double ey = ty * cos(L->theta);
    prof = exp(-(ey * ey + tz * tz) / (L->waist * L->waist));
  }
  return L->a0 * env * prof * sin(L->omega * tau + L->phase);
}

static void add_antennas(or_sim *s, double t) {
  for (int l = 0; l < s->nl; ++l) {
    const or_laser *L = &s->las[l];
    int c = L->comp; /* 1: y, 2: z */
    double amp = -2.0 / s->dx[0] * ((c == 2) ? cos(L->theta) : 1.0);
    for (long k = 0; k < s->n[2]; ++k)
      for (long j = 0; j < s->n[1]; ++j) {
        double y = (s->D >= 2) ? (j + STAG_E[c][1]) * s->dx[1] : 0.0;
        double z = (s->D >= 3) ? (k + STAG_E[c][2]) * s->dx[2] : 0.0;
        long id = lin(s, L->ia, j, k);
        if (id < 0) continue;
        s->F[6 + c][id] += amp * or_laser_value(L, t, y, z);
      }
  }
}

/* ------------------------------------------------------------------------ */
/* gather: quadratic B-spline weights at each component's Yee location       */

/* value of field F (stagger st) at the point X (cell units) */
static double interp(const or_sim *s, const double *F, const double st[3], const double X[3]) {
  long base[3];
  int cnt[3];
  double w[3][3];
  for (int a = 0; a < 3; ++a) {
    if (a < s->D) {
      double Y = X[a] - st[a];
      long nn = (long)floor(Y + 0.5);
      double xi = Y - (double)nn;
      base[a] = nn - 1;
      cnt[a] = 3;
      for (int m = 0; m < 3; ++m) w[a][m] = or_shape(xi - (double)(m - 1));
    } else {
      base[a] = 0;
      cnt[a] = 1;
      w[a][0] = 1.0;
    }
  }
  double sum = 0.0;
  for (int k = 0; k < cnt[2]; ++k)
    for (int j = 0; j < cnt[1]; ++j)
      for (int i = 0; i < cnt[0]; ++i)
        sum += w[0][i] * w[1][j] * w[2][k] * val(F, lin(s, base[0] + i, base[1] + j, base[2] + k));
  return sum;
}

double or_interp(const or_sim *s, int comp, const double X[3]) {
  const double *st = (comp < 3) ? STAG_E[comp] : (comp < 6 ? STAG_B[comp - 3] : STAG_E[comp - 6]);
  return interp(s, s->F[comp], st, X);
}

static void to_cell(const or_sim *s, const double x[3], double X[3]) {
  for (int a = 0; a < 3; ++a) X[a] = (a < s->D) ? x[a] / s->dx[a] : 0.0;
}

static void gather(const or_sim *s, const double x[3], double E[3], double B[3]) {
  double X[3];
  to_cell(s, x, X);
  for (int c = 0; c < 3; ++c) {
    E[c] = interp(s, s->F[c], STAG_E[c], X);
    B[c] = interp(s, s->F[3 + c], STAG_B[c], X);
  }
}

/* ------------------------------------------------------------------------ */
/* internal force and Boris push                                             */

/* Field seen by a body from its partner through the modified Coulomb force
 * (Sec. 2): E = q_other * kappa * d / (|d|^2 + ac^2)^{3/2} with d = x_self -
 * x_other.  For the nucleus this is q2 r/(...) with r = r1 - r2, so the force
 * on it is the paper's q1 q2 r / (4 pi eps0 (r^2 + ac^2)^{3/2}); the
 * electron gets the opposite force. */
void or_internal_field(double q_other, double kappa, double ac, const double d[3], double out[3]) {
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double den = pow(r2 + ac * ac, 1.5);
  for (int a = 0; a < 3; ++a) out[a] = q_other * kappa * d[a] / den;
}

/* Relativistic Boris push of one body (Sec. 2 Boris equations), u = p/(mc):
 *   u-  = u + (q dt / 2m) E
 *   t   = (q dt / 2m) B / gamma-,   s = 2 t / (1 + t^2)
 *   u+  = u- + (u- + u- x t) x s
 *   u'  = u+ + (q dt / 2m) E                                           */
void or_boris(double q, double m, double dt, const double E[3], const double B[3], double u[3]) {
  double h = q * dt / (2.0 * m);
  double um[3], t[3], sv[3], up[3], c1[3];
  for (int a = 0; a < 3; ++a) um[a] = u[a] + h * E[a];
  double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  for (int a = 0; a < 3; ++a) t[a] = h * B[a] / gm;
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  for (int a = 0; a < 3; ++a) sv[a] = 2.0 * t[a] / (1.0 + t2);
  /* c1 = u- + u- x t */
  c1[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
  c1[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
  c1[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
  /* u+ = u- + c1 x s */
  up[0] = um[0] + (c1[1] * sv[2] - c1[2] * sv[1]);
  up[1] = um[1] + (c1[2] * sv[0] - c1[0] * sv[2]);
  up[2] = um[2] + (c1[0] * sv[1] - c1[1] * sv[0]);
  for (int a = 0; a < 3; ++a) u[a] = up[a] + h * E[a];
}

/* ------------------------------------------------------------------------ */
/* Esirkepov charge-conserving deposit with the quadratic shape              */

/* Adds the current of one particle of charge*weight qw moving from X0 to X1
 * (cell units) with velocity v to J.  S0, S1 are the shape factors at the
 * old and new position on a five-node window around the old nearest node;
 * W are Esirkepov's density-decomposition weights:
 *   3D: W_x = DSx (S0y S0z + DSy S0z/2 + S0y DSz/2 + DSy DSz/3), cyclic
 *   2D: W_x = DSx (S0y + DSy/2),  W_y = DSy (S0x + DSx/2),
 *       J_z uses S0x S0y + DSx S0y/2 + S0x DSy/2 + DSx DSy/3 times v_z
 *   1D: W_x = DSx;  J_y, J_z use (S0 + S1)/2 times v
 * and J_a on the faces after each node is -qw (dx_a/dt) times the running
 * sum of W_a along axis a. */
void or_deposit_one(or_sim *s, double qw, const double X0[3], const double X1[3], const double v[3]) {
  const int D = s->D;
  long n0[3] = {0, 0, 0};
  double S0[3][5], DS[3][5];
  for (int a = 0; a < 3; ++a)
    for (int m = 0; m < 5; ++m) { S0[a][m] = (a < D) ? 0.0 : (m == 2 ? 1.0 : 0.0); DS[a][m] = 0.0; }
  for (int a = 0; a < D; ++a) {
    n0[a] = (long)floor(X0[a] + 0.5);
    for (int m = 0; m < 5; ++m) {
      double node = (double)(n0[a] + m - 2);
      double s0 = or_shape(X0[a] - node), s1 = or_shape(X1[a] - node);
      S0[a][m] = s0;
      DS[a][m] = s1 - s0;
    }
  }
  double *Jx = s->F[6], *Jy = s->F[7], *Jz = s->F[8];
  if (D == 1) {
    double run = 0.0;
    for (int i = 0; i < 5; ++i) {
      run += DS[0][i];
      long id = lin(s, n0[0] + i - 2, 0, 0);
      if (id < 0) continue;
      if (i < 4) Jx[id] += -qw * (s->dx[0] / s->dt) * run;
      double sbar = S0[0][i] + 0.5 * DS[0][i];
      Jy[id] += qw * v[1] * sbar;
      Jz[id] += qw * v[2] * sbar;
    }
  } else if (D == 2) {
    /* J_x: running sum along i at each j */
    for (int j = 0; j < 5; ++j) {
      double run = 0.0;
      for (int i = 0; i < 4; ++i) {
        run += DS[0][i] * (S0[1][j] + 0.5 * DS[1][j]);
        long id = lin(s, n0[0] + i - 2, n0[1] + j - 2, 0);
        if (id >= 0) Jx[id] += -qw * (s->dx[0] / s->dt) * run;
      }
    }
    for (int i = 0; i < 5; ++i) {
      double run = 0.0;
      for (int j = 0; j < 4; ++j) {
        run += DS[1][j] * (S0[0][i] + 0.5 * DS[0][i]);
        long id = lin(s, n0[0] + i - 2, n0[1] + j - 2, 0);
        if (id >= 0) Jy[id] += -qw * (s->dx[1] / s->dt) * run;
      }
    }
    for (int j = 0; j < 5; ++j)
      for (int i = 0; i < 5; ++i) {
        double wz = S0[0][i] * S0[1][j] + 0.5 * DS[0][i] * S0[1][j] + 0.5 * S0[0][i] * DS[1][j] +
                    DS[0][i] * DS[1][j] / 3.0;
        long id = lin(s, n0[0] + i - 2, n0[1] + j - 2, 0);
        if (id >= 0) Jz[id] += qw * v[2] * wz;
      }
  } else {
    for (int k = 0; k < 5; ++k)
      for (int j = 0; j < 5; ++j) {
        double run = 0.0;
        for (int i = 0; i < 4; ++i) {
          run += DS[0][i] * (S0[1][j] * S0[2][k] + 0.5 * DS[1][j] * S0[2][k] + 0.5 * S0[1][j] * DS[2][k] +
                             DS[1][j] * DS[2][k] / 3.0);
          long id = lin(s, n0[0] + i - 2, n0[1] + j - 2, n0[2] + k - 2);
          if (id >= 0) Jx[id] += -qw * (s->dx[0] / s->dt) * run;
        }
      }
    for (int k = 0; k < 5; ++k)
      for (int i = 0; i < 5; ++i) {
        double run = 0.0;
        for (int j = 0; j < 4; ++j) {
          run += DS[1][j] * (S0[0][i] * S0[2][k] + 0.5 * DS[0][i] * S0[2][k] + 0.5 * S0[0][i] * DS[2][k] +
                             DS[0][i] * DS[2][k] / 3.0);
          long id = lin(s, n0[0] + i - 2, n0[1] + j - 2, n0[2] + k - 2);
          if (id >= 0) Jy[id] += -qw * (s->dx[1] / s->dt) * run;
        }
      }
    for (int j = 0; j < 5; ++j)
      for (int i = 0; i < 5; ++i) {
        double run = 0.0;
        for (int k = 0; k < 4; ++k) {
          run += DS[2][k] * (S0[0][i] * S0[1][j] + 0.5 * DS[0][i] * S0[1][j] + 0.5 * S0[0][i] * DS[1][j] +
                             DS[0][i] * DS[1][j] / 3.0);
          long id = lin(s, n0[0] + i - 2, n0[1] + j - 2, n0[2] + k - 2);
          if (id >= 0) Jz[id] += -qw * (s->dx[2] / s->dt) * run;
        }
      }
  }
}

/* ------------------------------------------------------------------------ */
/* Yee FDTD (vacuum Maxwell, Sec. 3.1)                                      */

/* along an open axis a, a component with node stagger has boundary nodes 0
 * and n-1 (Mur); one with half stagger has no value at n-1 (exterior). */
enum { CL_INTERIOR = 0, CL_EXTERIOR = -1 };

/* returns -1 (exterior) or the number of open axes on which (i,j,k) is a
 * boundary node of a component with stagger st; *first gets the first one */
static int classify(const or_sim *s, const double st[3], const long ijk[3], int *first) {
  int nb = 0;
  *first = -1;
  for (int a = 0; a < s->D; ++a) {
    if (s->bc[a] != OR_OPEN) continue;
    if (st[a] > 0.0) {
      if (ijk[a] == s->n[a] - 1) return CL_EXTERIOR;
    } else if (ijk[a] == 0 || ijk[a] == s->n[a] - 1) {
      if (*first < 0) *first = a;
      nb++;
    }
  }
  return nb;
}

static double dfd(const or_sim *s, const double *F, int a, long i, long j, long k, int off_lo, int off_hi) {
  /* (F[idx + off_hi e_a] - F[idx + off_lo e_a]) / dx_a, zero on non-simulated axes */
  if (a >= s->D) return 0.0;
  long p[3] = {i, j, k}, q[3] = {i, j, k};
  p[a] += off_hi;
  q[a] += off_lo;
  return (val(F, lin(s, p[0], p[1], p[2])) - val(F, lin(s, q[0], q[1], q[2]))) / s->dx[a];
}

/* B <- B - h curl E, curl E at B locations uses forward differences */
void or_yee_b(or_sim *s, double h) {
  double *Ex = s->F[0], *Ey = s->F[1], *Ez = s->F[2];
#pragma omp parallel for collapse(2) schedule(static) if (s->ncell > 65536)
  for (long k = 0; k < s->n[2]; ++k)
    for (long j = 0; j < s->n[1]; ++j)
      for (long i = 0; i < s->n[0]; ++i) {
        long ijk[3] = {i, j, k};
        long id = lin(s, i, j, k);
        int f;
        if (classify(s, STAG_B[0], ijk, &f) != CL_EXTERIOR)
          s->F[3][id] -= h * (dfd(s, Ez, 1, i, j, k, 0, 1) - dfd(s, Ey, 2, i, j, k, 0, 1));
        if (classify(s, STAG_B[1], ijk, &f) != CL_EXTERIOR)
          s->F[4][id] -= h * (dfd(s, Ex, 2, i, j, k, 0, 1) - dfd(s, Ez, 0, i, j, k, 0, 1));
        if (classify(s, STAG_B[2], ijk, &f) != CL_EXTERIOR)
          s->F[5][id] -= h * (dfd(s, Ey, 0, i, j, k, 0, 1) - dfd(s, Ex, 1, i, j, k, 0, 1));
      }
}

/* E <- E + dt (curl B - J) on interior nodes; Mur first order on the
 * tangential components of open faces:
 *   E_b(n+1) = E_adj(n) + (dt - dx)/(dt + dx) (E_adj(n+1) - E_b(n))
 * Nodes on several open faces are done after their inward neighbour. */
void or_yee_e(or_sim *s) {
  const double dt = s->dt;
  double *Bx = s->F[3], *By = s->F[4], *Bz = s->F[5];
  for (int c = 0; c < 3; ++c) memcpy(s->Eold[c], s->F[c], sizeof(double) * (size_t)s->ncell);
#pragma omp parallel for collapse(2) schedule(static) if (s->ncell > 65536)
  for (long k = 0; k < s->n[2]; ++k)
    for (long j = 0; j < s->n[1]; ++j)
      for (long i = 0; i < s->n[0]; ++i) {
        long ijk[3] = {i, j, k};
        long id = lin(s, i, j, k);
        int f;
        if (classify(s, STAG_E[0], ijk, &f) == CL_INTERIOR)
          s->F[0][id] += dt * (dfd(s, Bz, 1, i, j, k, -1, 0) - dfd(s, By, 2, i, j, k, -1, 0) - s->F[6][id]);
        if (classify(s, STAG_E[1], ijk, &f) == CL_INTERIOR)
          s->F[1][id] += dt * (dfd(s, Bx, 2, i, j, k, -1, 0) - dfd(s, Bz, 0, i, j, k, -1, 0) - s->F[7][id]);
        if (classify(s, STAG_E[2], ijk, &f) == CL_INTERIOR)
          s->F[2][id] += dt * (dfd(s, By, 0, i, j, k, -1, 0) - dfd(s, Bx, 1, i, j, k, -1, 0) - s->F[8][id]);
      }
  for (int pass = 1; pass <= 3; ++pass)
    for (int c = 0; c < 3; ++c)
      for (long k = 0; k < s->n[2]; ++k)
        for (long j = 0; j < s->n[1]; ++j)
          for (long i = 0; i < s->n[0]; ++i) {
            long ijk[3] = {i, j, k};
            int a;
            if (classify(s, STAG_E[c], ijk, &a) != pass) continue;
            long adj[3] = {i, j, k};
            adj[a] += (ijk[a] == 0) ? 1 : -1;
            long id = lin(s, i, j, k), ida = lin(s, adj[0], adj[1], adj[2]);
            double km = (dt - s->dx[a]) / (dt + s->dx[a]);
            s->F[c][id] = s->Eold[c][ida] + km * (s->F[c][ida] - s->Eold[c][id]);
          }
}

/* ------------------------------------------------------------------------ */
/* the step                                                                  */

static void push_species(or_sim *s, or_species *p) {
  const double dt = s->dt;
  for (int64_t q = 0; q < p->n; ++q) {
    if (!p->alive[q]) continue;
    double *x1 = p->x1 + 3 * q, *u1 = p->u1 + 3 * q;
    double E1[3], B1[3];
    gather(s, x1, E1, B1);
    if (p->kind == OR_FREE) {
      double X0[3], X1[3], v[3];
      to_cell(s, x1, X0);
      or_boris(p->q1, p->m1, dt, E1, B1, u1);
      double g = sqrt(1.0 + u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
      for (int a = 0; a < 3; ++a) { v[a] = u1[a] / g; x1[a] += dt * v[a]; }
      to_cell(s, x1, X1);
      if (s->deposit_on) or_deposit_one(s, p->q1 * p->w, X0, X1, v);
      for (int a = 0; a < s->D; ++a)
        if (s->bc[a] == OR_OPEN && (X1[a] < s->free_lo[a] || X1[a] >= s->free_hi[a])) p->alive[q] = 0;
      continue;
    }
    double *x2 = p->x2 + 3 * q, *u2 = p->u2 + 3 * q;
    double E2[3], B2[3];
    gather(s, x2, E2, B2);
    double ac = p->ac[p->pidx[q]];
    double d12[3], d21[3], Ei1[3], Ei2[3];
    for (int a = 0; a < 3; ++a) { d12[a] = x1[a] - x2[a]; d21[a] = -d12[a]; }
    or_internal_field(p->q2, p->kappa, ac, d12, Ei1);
    or_internal_field(p->q1, p->kappa, ac, d21, Ei2);
    for (int a = 0; a < 3; ++a) { E1[a] += Ei1[a]; E2[a] += Ei2[a]; }
    double X10[3], X20[3], X11[3], X21[3], v1[3], v2[3];
    to_cell(s, x1, X10);
    to_cell(s, x2, X20);
    or_boris(p->q1, p->m1, dt, E1, B1, u1);
    or_boris(p->q2, p->m2, dt, E2, B2, u2);
    double g1 = sqrt(1.0 + u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
    double g2 = sqrt(1.0 + u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2]);
    for (int a = 0; a < 3; ++a) {
      v1[a] = u1[a] / g1; x1[a] += dt * v1[a];
      v2[a] = u2[a] / g2; x2[a] += dt * v2[a];
    }
    to_cell(s, x1, X11);
    to_cell(s, x2, X21);
    if (s->deposit_on) {
      or_deposit_one(s, p->q1 * p->w, X10, X11, v1);
      or_deposit_one(s, p->q2 * p->w, X20, X21, v2);
    }
  }
}

/* One leapfrog step from (E^n, B^{n-1/2}, x^n, u^{n-1/2}):
 *   B^n = B^{n-1/2} - dt/2 curl E^n
 *   gather E^n, B^n at each body; add the internal field; Boris; drift
 *   J^{n+1/2} by Esirkepov for each body, plus the antenna sheet
 *   B^{n+1/2} = B^n - dt/2 curl E^n
 *   E^{n+1} = E^n + dt (curl B^{n+1/2} - J^{n+1/2})                        */
void or_step(or_sim *s, int nsteps) {
  for (int it = 0; it < nsteps; ++it) {
    if (s->fields_on) or_yee_b(s, 0.5 * s->dt);
    for (int c = 6; c < 9; ++c) memset(s->F[c], 0, sizeof(double) * (size_t)s->ncell);
    for (int i = 0; i < s->nsp; ++i) push_species(s, &s->sp[i]);
    if (s->fields_on) {
      add_antennas(s, ((double)s->step + 0.5) * s->dt);
      or_yee_b(s, 0.5 * s->dt);
      or_yee_e(s);
    }
    s->step++;
    record_probes(s);
  }
}

/* ------------------------------------------------------------------------ */
/* Gauss-law residual R = div E - rho at nodes                               */

void or_rho(const or_sim *s, double *rho) {
  memset(rho, 0, sizeof(double) * (size_t)s->ncell);
  for (int i = 0; i < s->nsp; ++i) {
    const or_species *p = &s->sp[i];
    for (int64_t q = 0; q < p->n; ++q) {
      if (!p->alive[q]) continue;
      for (int b = 0; b < (p->kind == OR_FREE ? 1 : 2); ++b) {
        const double *x = (b == 0 ? p->x1 : p->x2) + 3 * q;
        double qw = (b == 0 ? p->q1 : p->q2) * p->w;
        double X[3];
        to_cell(s, x, X);
        long base[3];
        int cnt[3];
        double w[3][3];
        for (int a = 0; a < 3; ++a) {
          if (a < s->D) {
            long nn = (long)floor(X[a] + 0.5);
            base[a] = nn - 1;
            cnt[a] = 3;
            for (int m = 0; m < 3; ++m) w[a][m] = or_shape(X[a] - (double)(nn + m - 1));
          } else { base[a] = 0; cnt[a] = 1; w[a][0] = 1.0; }
        }
        for (int kk = 0; kk < cnt[2]; ++kk)
          for (int jj = 0; jj < cnt[1]; ++jj)
            for (int ii = 0; ii < cnt[0]; ++ii) {
              long id = lin(s, base[0] + ii, base[1] + jj, base[2] + kk);
              if (id >= 0) rho[id] += qw * w[0][ii] * w[1][jj] * w[2][kk];
            }
      }
    }
  }
}

void or_residual(const or_sim *s, double *R) {
  or_rho(s, R);
  for (long k = 0; k < s->n[2]; ++k)
    for (long j = 0; j < s->n[1]; ++j)
      for (long i = 0; i < s->n[0]; ++i) {
        long id = lin(s, i, j, k);
        double div = dfd(s, s->F[0], 0, i, j, k, -1, 0) + dfd(s, s->F[1], 1, i, j, k, -1, 0) +
                     dfd(s, s->F[2], 2, i, j, k, -1, 0);
        R[id] = div - R[id];
      }
}
