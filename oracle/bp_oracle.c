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
 * Discrete choices the paper leaves open:
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

/* ======================================================================== */
/* Discrete adjoint (reverse mode) of the step above, FP64.                 */
/*                                                                          */
/* Loss: L = sum over recorded probe samples of (p - target)^2.  The        */
/* reverse pass runs the forward steps backwards, each operator replaced by */
/* its transpose (linear operators) or its vector-Jacobian product          */
/* (gather, internal force, Boris, drift, Esirkepov), from states stored    */
/* during the forward run.  Parameters: the bound-electron frequency of     */
/* every parameter index (through a_c of Sec. 3.1) and the initial ion      */
/* positions (both bodies start at the ion position, Sec. 2).               */
/* Restriction: one two-body species, no free particles.                   */
/* ======================================================================== */

/* derivative of the quadratic B-spline */
double or_dshape(double x) {
  double a = fabs(x);
  if (a <= 0.5) return -2.0 * x;
  if (a < 1.5) return (x > 0 ? -1.0 : 1.0) * (1.5 - a);
  return 0.0;
}

/* reverse of or_boris: given ubar_new (adjoint of the pushed momentum),
 * return ubar_old, Ebar, Bbar (adjoints of the inputs) */
void or_boris_adj(double q, double m, double dt, const double E[3], const double B[3], const double u0[3],
                  const double ubn[3], double ub0[3], double Eb[3], double Bb[3]) {
  double h = q * dt / (2.0 * m);
  double um[3], t[3], sv[3], c1[3];
  for (int a = 0; a < 3; ++a) um[a] = u0[a] + h * E[a];
  double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  for (int a = 0; a < 3; ++a) t[a] = h * B[a] / gm;
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  for (int a = 0; a < 3; ++a) sv[a] = 2.0 * t[a] / (1.0 + t2);
  c1[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
  c1[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
  c1[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
  double upb[3], umb[3], cb[3], sb[3], tb[3];
  for (int a = 0; a < 3; ++a) { upb[a] = ubn[a]; Eb[a] = h * ubn[a]; }
  /* up = um + c1 x s:  um += upb;  c1b = s x upb;  sb = upb x c1 */
  for (int a = 0; a < 3; ++a) umb[a] = upb[a];
  cb[0] = sv[1] * upb[2] - sv[2] * upb[1];
  cb[1] = sv[2] * upb[0] - sv[0] * upb[2];
  cb[2] = sv[0] * upb[1] - sv[1] * upb[0];
  sb[0] = upb[1] * c1[2] - upb[2] * c1[1];
  sb[1] = upb[2] * c1[0] - upb[0] * c1[2];
  sb[2] = upb[0] * c1[1] - upb[1] * c1[0];
  /* c1 = um + um x t:  umb += cb + t x cb;  tb = cb x um */
  umb[0] += cb[0] + (t[1] * cb[2] - t[2] * cb[1]);
  umb[1] += cb[1] + (t[2] * cb[0] - t[0] * cb[2]);
  umb[2] += cb[2] + (t[0] * cb[1] - t[1] * cb[0]);
  tb[0] = cb[1] * um[2] - cb[2] * um[1];
  tb[1] = cb[2] * um[0] - cb[0] * um[2];
  tb[2] = cb[0] * um[1] - cb[1] * um[0];
  /* s = 2 t / (1 + t^2) */
  double ts = t[0] * sb[0] + t[1] * sb[1] + t[2] * sb[2];
  for (int a = 0; a < 3; ++a) tb[a] += 2.0 * sb[a] / (1.0 + t2) - 4.0 * t[a] * ts / ((1.0 + t2) * (1.0 + t2));
  /* t = h B / gm */
  double gmb = 0.0;
  for (int a = 0; a < 3; ++a) {
    Bb[a] = h * tb[a] / gm;
    gmb -= h * B[a] * tb[a] / (gm * gm);
  }
  /* gm = sqrt(1 + um^2) */
  for (int a = 0; a < 3; ++a) umb[a] += um[a] * gmb / gm;
  /* um = u0 + h E */
  for (int a = 0; a < 3; ++a) {
    ub0[a] = umb[a];
    Eb[a] += h * umb[a];
  }
}

/* reverse of the internal field: out = q_other kappa d / (|d|^2 + ac^2)^{3/2};
 * given its adjoint Eb, add the adjoint of d to db and return the one of ac */
double or_internal_field_adj(double q_other, double kappa, double ac, const double d[3], const double Eb[3],
                             double db[3]) {
  double rho = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + ac * ac;
  double p32 = pow(rho, -1.5), p52 = pow(rho, -2.5);
  double ed = Eb[0] * d[0] + Eb[1] * d[1] + Eb[2] * d[2];
  for (int a = 0; a < 3; ++a) db[a] += q_other * kappa * (Eb[a] * p32 - 3.0 * ed * d[a] * p52);
  return -3.0 * q_other * kappa * ed * ac * p52;
}

/* reverse of interp(): field adjoint Fb += weights * gb; returns dE/dX . gb
 * per axis in Xb (cell units) */
static void interp_adj(const or_sim *s, const double *F, double *Fb, const double st[3], const double X[3], double gb,
                       double Xb[3]) {
  long base[3];
  int cnt[3];
  double w[3][3], dw[3][3];
  for (int a = 0; a < 3; ++a) {
    if (a < s->D) {
      double Y = X[a] - st[a];
      long nn = (long)floor(Y + 0.5);
      double xi = Y - (double)nn;
      base[a] = nn - 1;
      cnt[a] = 3;
      for (int m = 0; m < 3; ++m) {
        w[a][m] = or_shape(xi - (double)(m - 1));
        dw[a][m] = or_dshape(xi - (double)(m - 1));
      }
    } else {
      base[a] = 0; cnt[a] = 1; w[a][0] = 1.0; dw[a][0] = 0.0;
    }
  }
  for (int k = 0; k < cnt[2]; ++k)
    for (int j = 0; j < cnt[1]; ++j)
      for (int i = 0; i < cnt[0]; ++i) {
        long id = lin(s, base[0] + i, base[1] + j, base[2] + k);
        if (id < 0) continue;
        if (Fb) Fb[id] += w[0][i] * w[1][j] * w[2][k] * gb;
        double f = F[id] * gb;
        Xb[0] += dw[0][i] * w[1][j] * w[2][k] * f;
        if (s->D >= 2) Xb[1] += w[0][i] * dw[1][j] * w[2][k] * f;
        if (s->D >= 3) Xb[2] += w[0][i] * w[1][j] * dw[2][k] * f;
      }
}

/* reverse of gather(): Eb, Bb adjoints of the gathered fields at x;
 * accumulates the field adjoints FEb, FBb (may be NULL) and xb */
void or_gather_adj(const or_sim *s, const double x[3], const double Eb[3], const double Bb[3], double *const FEb[3],
                   double *const FBb[3], double xb[3]) {
  double X[3], Xb[3] = {0, 0, 0};
  to_cell(s, x, X);
  for (int c = 0; c < 3; ++c) {
    interp_adj(s, s->F[c], FEb ? FEb[c] : NULL, STAG_E[c], X, Eb[c], Xb);
    interp_adj(s, s->F[3 + c], FBb ? FBb[c] : NULL, STAG_B[c], X, Bb[c], Xb);
  }
  for (int a = 0; a < s->D; ++a) xb[a] += Xb[a] / s->dx[a];
}

/* reverse of or_deposit_one: with lam the adjoint of J (lam[0..2] arrays on
 * the grid), adds d(sum lam . J)/dX0, /dX1 (cell units) and /dv */
void or_deposit_adj(const or_sim *s, double qw, const double X0[3], const double X1[3], const double v[3],
                    const double *const lam[3], double X0b[3], double X1b[3], double vb[3]) {
  const int D = s->D;
  long n0[3] = {2, 2, 2}; /* non-simulated axes: window entry 0 maps to index 0 */
  double S0[3][5], DS[3][5], gS0[3][5], gDS[3][5];
  for (int a = 0; a < 3; ++a)
    for (int m = 0; m < 5; ++m) {
      S0[a][m] = (a < D) ? 0.0 : (m == 2 ? 1.0 : 0.0);
      DS[a][m] = 0.0; gS0[a][m] = 0.0; gDS[a][m] = 0.0;
    }
  for (int a = 0; a < D; ++a) {
    n0[a] = (long)floor(X0[a] + 0.5);
    for (int m = 0; m < 5; ++m) {
      double node = (double)(n0[a] + m - 2);
      double s0 = or_shape(X0[a] - node), s1 = or_shape(X1[a] - node);
      S0[a][m] = s0;
      DS[a][m] = s1 - s0;
    }
  }
#define LAM(c, i, j, k) val(lam[c], lin(s, n0[0] + (i) - 2, n0[1] + (j) - 2, n0[2] + (k) - 2))
  if (D == 1) {
    double cx = -qw * s->dx[0] / s->dt;
    for (int ip = 0; ip < 4; ++ip)
      for (int i = ip; i < 4; ++i) gDS[0][ip] += cx * LAM(0, i, 0, 0);
    for (int i = 0; i < 5; ++i) {
      double ly = LAM(1, i, 0, 0), lz = LAM(2, i, 0, 0);
      double sbar = S0[0][i] + 0.5 * DS[0][i];
      gS0[0][i] += qw * (v[1] * ly + v[2] * lz);
      gDS[0][i] += 0.5 * qw * (v[1] * ly + v[2] * lz);
      vb[1] += qw * ly * sbar;
      vb[2] += qw * lz * sbar;
    }
  } else if (D == 2) {
    double cx = -qw * s->dx[0] / s->dt, cy = -qw * s->dx[1] / s->dt;
    for (int j = 0; j < 5; ++j) {
      double fac = S0[1][j] + 0.5 * DS[1][j], P = 0.0;
      for (int i = 0; i < 4; ++i) {
        P += DS[0][i];
        double l = LAM(0, i, j, 0);
        for (int ip = 0; ip <= i; ++ip) gDS[0][ip] += cx * l * fac;
        gS0[1][j] += cx * l * P;
        gDS[1][j] += 0.5 * cx * l * P;
      }
    }
    for (int i = 0; i < 5; ++i) {
      double fac = S0[0][i] + 0.5 * DS[0][i], P = 0.0;
      for (int j = 0; j < 4; ++j) {
        P += DS[1][j];
        double l = LAM(1, i, j, 0);
        for (int jp = 0; jp <= j; ++jp) gDS[1][jp] += cy * l * fac;
        gS0[0][i] += cy * l * P;
        gDS[0][i] += 0.5 * cy * l * P;
      }
    }
    for (int j = 0; j < 5; ++j)
      for (int i = 0; i < 5; ++i) {
        double l = LAM(2, i, j, 0);
        double wz = S0[0][i] * S0[1][j] + 0.5 * DS[0][i] * S0[1][j] + 0.5 * S0[0][i] * DS[1][j] +
                    DS[0][i] * DS[1][j] / 3.0;
        double c = qw * v[2] * l;
        vb[2] += qw * l * wz;
        gS0[0][i] += c * (S0[1][j] + 0.5 * DS[1][j]);
        gDS[0][i] += c * (0.5 * S0[1][j] + DS[1][j] / 3.0);
        gS0[1][j] += c * (S0[0][i] + 0.5 * DS[0][i]);
        gDS[1][j] += c * (0.5 * S0[0][i] + DS[0][i] / 3.0);
      }
  } else {
    /* the three components are the same formula with the axes permuted:
     * component a runs along a with the factor of the other two (b, c) */
    for (int a = 0; a < 3; ++a) {
      int b = (a + 1) % 3, c = (a + 2) % 3;
      double ca = -qw * s->dx[a] / s->dt;
      for (int kb = 0; kb < 5; ++kb)
        for (int kc = 0; kc < 5; ++kc) {
          double fac = S0[b][kb] * S0[c][kc] + 0.5 * DS[b][kb] * S0[c][kc] + 0.5 * S0[b][kb] * DS[c][kc] +
                       DS[b][kb] * DS[c][kc] / 3.0;
          double P = 0.0;
          for (int ka = 0; ka < 4; ++ka) {
            P += DS[a][ka];
            int idx[3];
            idx[a] = ka; idx[b] = kb; idx[c] = kc;
            double l = LAM(a, idx[0], idx[1], idx[2]);
            if (l == 0.0) continue;
            for (int kp = 0; kp <= ka; ++kp) gDS[a][kp] += ca * l * fac;
            gS0[b][kb] += ca * l * P * (S0[c][kc] + 0.5 * DS[c][kc]);
            gDS[b][kb] += ca * l * P * (0.5 * S0[c][kc] + DS[c][kc] / 3.0);
            gS0[c][kc] += ca * l * P * (S0[b][kb] + 0.5 * DS[b][kb]);
            gDS[c][kc] += ca * l * P * (0.5 * S0[b][kb] + DS[b][kb] / 3.0);
          }
        }
    }
  }
#undef LAM
  /* S0 = S(X0 - node), DS = S(X1 - node) - S(X0 - node) */
  for (int a = 0; a < D; ++a)
    for (int m = 0; m < 5; ++m) {
      double node = (double)(n0[a] + m - 2);
      X0b[a] += (gS0[a][m] - gDS[a][m]) * or_dshape(X0[a] - node);
      X1b[a] += gDS[a][m] * or_dshape(X1[a] - node);
    }
}

/* transpose of or_yee_b: E adjoint -= h curl^T (B adjoint); B adjoint unchanged */
void or_yee_b_adj(const or_sim *s, double h, double *const Eb[3], const double *const Bb[3]) {
  for (long k = 0; k < s->n[2]; ++k)
    for (long j = 0; j < s->n[1]; ++j)
      for (long i = 0; i < s->n[0]; ++i) {
        long ijk[3] = {i, j, k};
        long id = lin(s, i, j, k);
        int f;
        /* forward differences (F[idx + e_a] - F[idx]) / dx_a along simulated axes */
        if (classify(s, STAG_B[0], ijk, &f) != CL_EXTERIOR) {
          double g = h * Bb[0][id];
          if (s->D >= 2) { double c = g / s->dx[1]; Eb[2][lin(s, i, j + 1, k)] -= c; Eb[2][id] += c; }
          if (s->D >= 3) { double c = g / s->dx[2]; Eb[1][lin(s, i, j, k + 1)] += c; Eb[1][id] -= c; }
        }
        if (classify(s, STAG_B[1], ijk, &f) != CL_EXTERIOR) {
          double g = h * Bb[1][id];
          if (s->D >= 3) { double c = g / s->dx[2]; Eb[0][lin(s, i, j, k + 1)] -= c; Eb[0][id] += c; }
          { double c = g / s->dx[0]; Eb[2][lin(s, i + 1, j, k)] += c; Eb[2][id] -= c; }
        }
        if (classify(s, STAG_B[2], ijk, &f) != CL_EXTERIOR) {
          double g = h * Bb[2][id];
          { double c = g / s->dx[0]; Eb[1][lin(s, i + 1, j, k)] -= c; Eb[1][id] += c; }
          if (s->D >= 2) { double c = g / s->dx[1]; Eb[0][lin(s, i, j + 1, k)] += c; Eb[0][id] -= c; }
        }
      }
}

/* transpose of or_yee_e.  G: adjoint of E^{n+1} (destroyed); outputs the
 * adjoint of E^n into Hn (overwritten), adds to the adjoint of B, and writes
 * the adjoint of J (zero off the interior nodes) */
void or_yee_e_adj(const or_sim *s, double *const G[3], double *const Hn[3], double *const Bb[3], double *const Jb[3]) {
  const double dt = s->dt;
  for (int c = 0; c < 3; ++c) {
    memset(Hn[c], 0, sizeof(double) * (size_t)s->ncell);
    memset(Jb[c], 0, sizeof(double) * (size_t)s->ncell);
  }
  /* Mur faces, last pass first */
  for (int pass = 3; pass >= 1; --pass)
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
            double g = G[c][id];
            Hn[c][ida] += g;
            G[c][ida] += km * g;
            Hn[c][id] -= km * g;
            G[c][id] = 0.0;
          }
  for (long k = 0; k < s->n[2]; ++k)
    for (long j = 0; j < s->n[1]; ++j)
      for (long i = 0; i < s->n[0]; ++i) {
        long ijk[3] = {i, j, k};
        long id = lin(s, i, j, k);
        int f;
        for (int c = 0; c < 3; ++c) {
          int cl = classify(s, STAG_E[c], ijk, &f);
          if (cl == CL_EXTERIOR) { Hn[c][id] += G[c][id]; continue; }
          if (cl != CL_INTERIOR) continue;
          double g = G[c][id];
          Hn[c][id] += g;
          Jb[c][id] = -dt * g;
          double e = dt * g;
          /* backward differences (F[idx] - F[idx - e_a]) / dx_a */
          if (c == 0) {
            if (s->D >= 2) { double q = e / s->dx[1]; Bb[2][id] += q; Bb[2][lin(s, i, j - 1, k)] -= q; }
            if (s->D >= 3) { double q = e / s->dx[2]; Bb[1][id] -= q; Bb[1][lin(s, i, j, k - 1)] += q; }
          } else if (c == 1) {
            if (s->D >= 3) { double q = e / s->dx[2]; Bb[0][id] += q; Bb[0][lin(s, i, j, k - 1)] -= q; }
            { double q = e / s->dx[0]; Bb[2][id] -= q; Bb[2][lin(s, i - 1, j, k)] += q; }
          } else {
            { double q = e / s->dx[0]; Bb[1][id] += q; Bb[1][lin(s, i - 1, j, k)] -= q; }
            if (s->D >= 2) { double q = e / s->dx[1]; Bb[0][id] -= q; Bb[0][lin(s, i, j - 1, k)] += q; }
          }
        }
      }
}

/* ---------------------------------------------------------------------- */
/* the whole run                                                           */

typedef struct ora {
  or_sim *s;
  int sid, pid, nsteps;
  int64_t n;
  double *E, *B;           /* [nsteps][3][ncell] E^n and B^n (after the first half step) */
  double *X1, *X2, *U1, *U2; /* [nsteps][n][3] particle state at step n (u at n - 1/2) */
  double *target;          /* [nsteps][npts] */
  double *probe;           /* [nsteps][npts] */
} ora;

ora *ora_create(or_sim *s, int sid) {
  ora *o = (ora *)calloc(1, sizeof(ora));
  o->s = s;
  o->sid = sid;
  return o;
}

void ora_destroy(ora *o) {
  if (!o) return;
  free(o->E); free(o->B); free(o->X1); free(o->X2); free(o->U1); free(o->U2);
  free(o->target); free(o->probe);
  free(o);
}

/* Runs nsteps forward steps storing every step's state, records probe pid
 * into probe_out [nsteps][npts] and returns L = sum (probe - target)^2. */
double ora_forward(ora *o, int nsteps, int pid, const double *target, double *probe_out, int64_t npts) {
  or_sim *s = o->s;
  or_species *p = &s->sp[o->sid];
  const size_t nc = (size_t)s->ncell, np = (size_t)p->n;
  o->nsteps = nsteps;
  o->pid = pid;
  o->n = p->n;
  o->E = (double *)malloc(sizeof(double) * 3 * nc * (size_t)nsteps);
  o->B = (double *)malloc(sizeof(double) * 3 * nc * (size_t)nsteps);
  o->X1 = (double *)malloc(sizeof(double) * 3 * np * (size_t)nsteps + 8);
  o->X2 = (double *)malloc(sizeof(double) * 3 * np * (size_t)nsteps + 8);
  o->U1 = (double *)malloc(sizeof(double) * 3 * np * (size_t)nsteps + 8);
  o->U2 = (double *)malloc(sizeof(double) * 3 * np * (size_t)nsteps + 8);
  o->target = (double *)malloc(sizeof(double) * (size_t)(nsteps * npts));
  memcpy(o->target, target, sizeof(double) * (size_t)(nsteps * npts));
  or_probe *P = &s->pr[pid];
  int64_t c0 = P->count;
  for (int it = 0; it < nsteps; ++it) {
    or_yee_b(s, 0.5 * s->dt);
    for (int c = 0; c < 3; ++c) {
      memcpy(o->E + ((size_t)it * 3 + c) * nc, s->F[c], sizeof(double) * nc);
      memcpy(o->B + ((size_t)it * 3 + c) * nc, s->F[3 + c], sizeof(double) * nc);
    }
    memcpy(o->X1 + (size_t)it * 3 * np, p->x1, sizeof(double) * 3 * np);
    memcpy(o->X2 + (size_t)it * 3 * np, p->x2, sizeof(double) * 3 * np);
    memcpy(o->U1 + (size_t)it * 3 * np, p->u1, sizeof(double) * 3 * np);
    memcpy(o->U2 + (size_t)it * 3 * np, p->u2, sizeof(double) * 3 * np);
    for (int c = 6; c < 9; ++c) memset(s->F[c], 0, sizeof(double) * nc);
    for (int i = 0; i < s->nsp; ++i) push_species(s, &s->sp[i]);
    add_antennas(s, ((double)s->step + 0.5) * s->dt);
    or_yee_b(s, 0.5 * s->dt);
    or_yee_e(s);
    s->step++;
    record_probes(s);
  }
  double L = 0.0;
  for (int it = 0; it < nsteps; ++it)
    for (int64_t q = 0; q < npts; ++q) {
      double v = P->data[(c0 + it) * P->npts + q];
      if (probe_out) probe_out[it * npts + q] = v;
      double d = v - target[it * npts + q];
      L += d * d;
    }
  o->probe = (double *)malloc(sizeof(double) * (size_t)(nsteps * npts));
  for (int it = 0; it < nsteps; ++it)
    for (int64_t q = 0; q < npts; ++q) o->probe[it * npts + q] = P->data[(c0 + it) * P->npts + q];
  return L;
}

/* Reverse pass.  grad_omega[nac]: dL/d omega_b per parameter index;
 * grad_x0[n][3]: dL/d(initial ion position) (both bodies start there). */
void ora_backward(ora *o, double *grad_omega, double *grad_x0) {
  or_sim *s = o->s;
  or_species *p = &s->sp[o->sid];
  or_probe *P = &s->pr[o->pid];
  const size_t nc = (size_t)s->ncell, np = (size_t)p->n;
  const double dt = s->dt;
  double *lamE[3], *lamB[3], *lamJ[3], *Hn[3], *Esave[3], *Bsave[3];
  for (int c = 0; c < 3; ++c) {
    lamE[c] = (double *)calloc(nc, sizeof(double));
    lamB[c] = (double *)calloc(nc, sizeof(double));
    lamJ[c] = (double *)calloc(nc, sizeof(double));
    Hn[c] = (double *)calloc(nc, sizeof(double));
    Esave[c] = s->F[c];
    Bsave[c] = s->F[3 + c];
  }
  double *x1b = (double *)calloc(3 * np + 1, sizeof(double)), *x2b = (double *)calloc(3 * np + 1, sizeof(double));
  double *u1b = (double *)calloc(3 * np + 1, sizeof(double)), *u2b = (double *)calloc(3 * np + 1, sizeof(double));
  double *acb = (double *)calloc((size_t)p->nac, sizeof(double));
  for (int it = o->nsteps - 1; it >= 0; --it) {
    /* loss on the probe sample recorded after this step */
    for (int64_t q = 0; q < P->npts; ++q)
      lamE[P->comp][P->idx[q]] += 2.0 * (o->probe[it * P->npts + q] - o->target[it * P->npts + q]);
    /* E^{n+1} = E^n + dt (curl B^{n+1/2} - J^{n+1/2}), Mur faces */
    or_yee_e_adj(s, lamE, Hn, lamB, lamJ);
    for (int c = 0; c < 3; ++c) { double *t = lamE[c]; lamE[c] = Hn[c]; Hn[c] = t; }
    /* B^{n+1/2} = B^n - dt/2 curl E^n */
    or_yee_b_adj(s, 0.5 * dt, lamE, (const double *const *)lamB);
    /* particles: the fields of step n are the stored E^n, B^n */
    for (int c = 0; c < 3; ++c) {
      s->F[c] = o->E + ((size_t)it * 3 + c) * nc;
      s->F[3 + c] = o->B + ((size_t)it * 3 + c) * nc;
    }
    const double *X1 = o->X1 + (size_t)it * 3 * np, *X2 = o->X2 + (size_t)it * 3 * np;
    const double *U1 = o->U1 + (size_t)it * 3 * np, *U2 = o->U2 + (size_t)it * 3 * np;
    for (int64_t q = 0; q < p->n; ++q) {
      const double *x1 = X1 + 3 * q, *x2 = X2 + 3 * q, *u10 = U1 + 3 * q, *u20 = U2 + 3 * q;
      double ac = p->ac[p->pidx[q]];
      /* forward recompute */
      double E1[3], B1[3], E2[3], B2[3], d12[3], d21[3], Ei1[3], Ei2[3];
      gather(s, x1, E1, B1);
      gather(s, x2, E2, B2);
      for (int a = 0; a < 3; ++a) { d12[a] = x1[a] - x2[a]; d21[a] = -d12[a]; }
      or_internal_field(p->q2, p->kappa, ac, d12, Ei1);
      or_internal_field(p->q1, p->kappa, ac, d21, Ei2);
      double Et1[3], Et2[3], u1[3], u2[3];
      for (int a = 0; a < 3; ++a) {
        Et1[a] = E1[a] + Ei1[a]; Et2[a] = E2[a] + Ei2[a];
        u1[a] = u10[a]; u2[a] = u20[a];
      }
      or_boris(p->q1, p->m1, dt, Et1, B1, u1);
      or_boris(p->q2, p->m2, dt, Et2, B2, u2);
      double g1 = sqrt(1.0 + u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
      double g2 = sqrt(1.0 + u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2]);
      double v1[3], v2[3], x1n[3], x2n[3], X10[3], X20[3], X11[3], X21[3];
      for (int a = 0; a < 3; ++a) {
        v1[a] = u1[a] / g1; v2[a] = u2[a] / g2;
        x1n[a] = x1[a] + dt * v1[a]; x2n[a] = x2[a] + dt * v2[a];
      }
      to_cell(s, x1, X10); to_cell(s, x2, X20); to_cell(s, x1n, X11); to_cell(s, x2n, X21);
      /* deposit */
      double X10b[3] = {0, 0, 0}, X11b[3] = {0, 0, 0}, X20b[3] = {0, 0, 0}, X21b[3] = {0, 0, 0};
      double v1b[3] = {0, 0, 0}, v2b[3] = {0, 0, 0};
      or_deposit_adj(s, p->q1 * p->w, X10, X11, v1, (const double *const *)lamJ, X10b, X11b, v1b);
      or_deposit_adj(s, p->q2 * p->w, X20, X21, v2, (const double *const *)lamJ, X20b, X21b, v2b);
      double *xb1 = x1b + 3 * q, *xb2 = x2b + 3 * q, *ub1 = u1b + 3 * q, *ub2 = u2b + 3 * q;
      /* adjoint of x^{n+1}: carried plus the deposit's */
      for (int a = 0; a < s->D; ++a) { xb1[a] += X11b[a] / s->dx[a]; xb2[a] += X21b[a] / s->dx[a]; }
      /* drift x^{n+1} = x^n + dt v(u^{n+1/2}): x^n gets the same adjoint */
      for (int a = 0; a < 3; ++a) { v1b[a] += dt * xb1[a]; v2b[a] += dt * xb2[a]; }
      /* v = u / gamma */
      double uv1 = u1[0] * v1b[0] + u1[1] * v1b[1] + u1[2] * v1b[2];
      double uv2 = u2[0] * v2b[0] + u2[1] * v2b[1] + u2[2] * v2b[2];
      double un1b[3], un2b[3];
      for (int a = 0; a < 3; ++a) {
        un1b[a] = ub1[a] + v1b[a] / g1 - u1[a] * uv1 / (g1 * g1 * g1);
        un2b[a] = ub2[a] + v2b[a] / g2 - u2[a] * uv2 / (g2 * g2 * g2);
      }
      /* Boris */
      double Et1b[3], Et2b[3], B1b[3], B2b[3];
      or_boris_adj(p->q1, p->m1, dt, Et1, B1, u10, un1b, ub1, Et1b, B1b);
      or_boris_adj(p->q2, p->m2, dt, Et2, B2, u20, un2b, ub2, Et2b, B2b);
      /* internal field */
      double d12b[3] = {0, 0, 0}, d21b[3] = {0, 0, 0};
      acb[p->pidx[q]] += or_internal_field_adj(p->q2, p->kappa, ac, d12, Et1b, d12b);
      acb[p->pidx[q]] += or_internal_field_adj(p->q1, p->kappa, ac, d21, Et2b, d21b);
      for (int a = 0; a < 3; ++a) {
        xb1[a] += d12b[a] - d21b[a];
        xb2[a] += d21b[a] - d12b[a];
      }
      /* gather: field adjoints of E^n and B^n, and the position gradients */
      or_gather_adj(s, x1, Et1b, B1b, lamE, lamB, xb1);
      or_gather_adj(s, x2, Et2b, B2b, lamE, lamB, xb2);
      /* old positions through the deposit */
      for (int a = 0; a < s->D; ++a) { xb1[a] += X10b[a] / s->dx[a]; xb2[a] += X20b[a] / s->dx[a]; }
    }
    /* B^n = B^{n-1/2} - dt/2 curl E^n */
    or_yee_b_adj(s, 0.5 * dt, lamE, (const double *const *)lamB);
  }
  for (int c = 0; c < 3; ++c) { s->F[c] = Esave[c]; s->F[3 + c] = Bsave[c]; }
  /* a_c(omega) = (|q1 q2| kappa / (m_r omega^2))^{1/3}: d a_c / d omega = -2 a_c / (3 omega) */
  for (int i = 0; i < p->nac; ++i) {
    double mr = p->m1 * p->m2 / (p->m1 + p->m2);
    double om = sqrt(fabs(p->q1 * p->q2) * p->kappa / (mr * p->ac[i] * p->ac[i] * p->ac[i]));
    grad_omega[i] = acb[i] * (-2.0 * p->ac[i] / (3.0 * om));
  }
  for (size_t q = 0; q < np; ++q)
    for (int a = 0; a < 3; ++a) grad_x0[3 * q + a] = x1b[3 * q + a] + x2b[3 * q + a];
  for (int c = 0; c < 3; ++c) { free(lamE[c]); free(lamB[c]); free(lamJ[c]); free(Hn[c]); }
  free(x1b); free(x2b); free(u1b); free(u2b); free(acb);
}
