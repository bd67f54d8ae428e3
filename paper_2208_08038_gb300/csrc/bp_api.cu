// bp_api.cu -- the C ABI (include/bp.h): context, species set-up (species
// split and a_c mapping of arXiv 2208.08038 Sec. 2 / Sec. 3.1, initial
// conditions of Sec. 2), and the step schedule on the caller's stream.
#include <algorithm>
#include <climits>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bp_ctx.h"
#include "bp_internal.cuh"

int sort_scan_blocks(const GridP &g);
int sort_launches();

namespace {

const double R_E = 2.8179403262e-15;  // classical electron radius [m]
using Species = bp_species_state;
using Probe = bp_probe_state;

}  // namespace

namespace {

int fail(bp_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

int cuda_fail(bp_ctx *c, cudaError_t e, const char *what) {
  return fail(c, BP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void *dalloc(bp_ctx *c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  if (c->have_alloc) {
    p = c->alloc.alloc(bytes, (void *)c->stream, c->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) {
    c->owned.push_back(p);
    cudaMemsetAsync(p, 0, bytes, c->stream);
  }
  return p;
}

void dfree(bp_ctx *c, void *p) {
  if (!p) return;
  auto it = std::find(c->owned.begin(), c->owned.end(), p);
  if (it != c->owned.end()) c->owned.erase(it);
  if (c->have_alloc) c->alloc.free(p, (void *)c->stream, c->alloc.user);
  else cudaFree(p);
}

// the device address of a host pointer into page-locked memory mapped for
// the device (pinned or registered), else nullptr
const void *mapped_host(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int check_launch(bp_ctx *c, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  return BP_OK;
}

// fixed-point scale of the sorted deposit: a power of two such that one
// particle's largest contribution (|q w| max(1, dx/dt)) maps to about 2^36.
// A node of a tile box then holds the exact sum of up to 2^26 such maximal
// contributions, and a quantum is about 1e-11 of the largest one (below the
// FP32 rounding of the contributions themselves).
// the tile marks of the push's field-box test, recomputed from E and B
// after they were written from outside the step (state file, caller,
// checkpoint)
void refresh_marks(bp_ctx *c) {
  const float *F[6] = {c->F[0], c->F[1], c->F[2], c->F[3], c->F[4], c->F[5]};
  launch_field_marks(c->g, F, c->stream);
  c->launches += 1;
  // every tile active until the next push recomputes the flags
  if (c->act) cudaMemsetAsync(c->act, 1, (size_t)c->g.ntiles, c->stream);
}

void update_jscale(bp_ctx *c) {
  if (!c->det) {
    c->jscale = c->jinv = 0.0f;
    return;
  }
  double B = 0.0, f = 1.0;
  for (int a = 0; a < c->g.D; ++a) f = std::max(f, c->g.dxd[a] / c->g.dtd);
  for (auto &s : c->sp) B = std::max({B, std::fabs(s.sp.q1d * s.sp.wd), std::fabs(s.sp.q2d * s.sp.wd)});
  if (B <= 0) B = 1.0;
  int k = 36 - (int)std::ceil(std::log2(B * f));
  k = std::max(-100, std::min(100, k));
  c->jscale = std::ldexp(1.0f, k);
  c->jinv = std::ldexp(1.0f, -k);
}

int alloc_particles(bp_ctx *c, Species &s, long long n, bool pidx) {
  c->sort_dirty = true;
  const int D = c->g.D;
  const bool two = s.sp.kind == BP_TWO_BODY;
  long long cap = std::max(1LL, n);
  PartP &p = s.p;
  if (p.cell && p.cap >= cap) {
    // reload after bp_reset: keep the arrays
    if (pidx && !p.pidx) p.pidx = (int *)dalloc(c, sizeof(int) * p.cap);
    if (!pidx) p.pidx = nullptr;
    return (pidx && !p.pidx) ? fail(c, BP_ERR_OOM, "param index array") : BP_OK;
  }
  if (p.cell) {
    void *old[] = {p.cell, p.off, p.u1, p.id, p.tstart, p.r, p.u2, p.pidx};
    for (void *q : old) dfree(c, q);
  }
  p.cap = cap;
  p.cell = (int *)dalloc(c, sizeof(int) * cap);
  p.off = (float *)dalloc(c, sizeof(float) * D * cap);
  p.u1 = (float *)dalloc(c, sizeof(float) * 3 * cap);
  p.id = (int *)dalloc(c, sizeof(int) * cap);
  p.tstart = (int *)dalloc(c, sizeof(int) * (c->g.ntiles + 1));
  if (two) {
    p.r = (float *)dalloc(c, sizeof(float) * 3 * cap);
    p.u2 = (float *)dalloc(c, sizeof(float) * 3 * cap);
  } else {
    p.r = p.u2 = nullptr;
  }
  p.pidx = pidx ? (int *)dalloc(c, sizeof(int) * cap) : nullptr;
  // on a failure nothing half-allocated stays behind: the next load starts afresh
  auto drop_particles = [&]() {
    void *got[] = {p.cell, p.off, p.u1, p.id, p.tstart, p.r, p.u2, p.pidx};
    for (void *q : got) dfree(c, q);
    p = PartP{};
  };
  if (!p.cell || !p.off || !p.u1 || !p.id || !p.tstart || (two && (!p.r || !p.u2)) || (pidx && !p.pidx)) {
    drop_particles();
    return fail(c, BP_ERR_OOM, "particle arrays (%lld particles)", n);
  }
  // sort scratch, shared by all species
  c->sort_dirty = true;
  if (!c->sb.hist || !c->sb.bsum) {
    dfree(c, c->sb.hist);
    dfree(c, c->sb.bsum);
    c->sb.hist = (int *)dalloc(c, sizeof(int) * (c->g.ncell + 1));
    c->sb.bsum = (int *)dalloc(c, sizeof(int) * (sort_scan_blocks(c->g) + 4));
    if (!c->sb.hist || !c->sb.bsum) {
      dfree(c, c->sb.hist);
      dfree(c, c->sb.bsum);
      c->sb.hist = c->sb.bsum = nullptr;
      drop_particles();
      return fail(c, BP_ERR_OOM, "sort scratch");
    }
  }
  long long need_f = (long long)(D + 9) * cap;
  if (cap > c->sort_cap) {
    dfree(c, c->sb.tmp_cell);
    dfree(c, c->sb.tmp_f);
    dfree(c, c->sb.tmp_i);
    c->sb.tmp_cell = (int *)dalloc(c, sizeof(int) * cap);
    c->sb.tmp_f = (float *)dalloc(c, sizeof(float) * need_f);
    c->sb.tmp_i = (int *)dalloc(c, sizeof(int) * 2 * cap);
    if (!c->sb.tmp_cell || !c->sb.tmp_f || !c->sb.tmp_i) {
      dfree(c, c->sb.tmp_cell);
      dfree(c, c->sb.tmp_f);
      dfree(c, c->sb.tmp_i);
      c->sb.tmp_cell = nullptr;
      c->sb.tmp_f = nullptr;
      c->sb.tmp_i = nullptr;
      c->sort_cap = 0;
      drop_particles();
      return fail(c, BP_ERR_OOM, "sort buffers");
    }
    c->sort_cap = cap;
  }
  return BP_OK;
}

// one-time full sort after a load: mark every particle as living in tile 0
// (tstart[ntiles] = n) and run the sort pipeline
int initial_sort(bp_ctx *c, Species &s, long long n) {
  std::vector<int> ts(c->g.ntiles + 1, 0);
  ts[c->g.ntiles] = (int)n;
  cudaMemcpyAsync(s.p.tstart, ts.data(), sizeof(int) * ts.size(), cudaMemcpyHostToDevice, c->stream);
  launch_set_sort_flag(c->status, c->stream);
  launch_sort(c->g, s.sp, s.p, c->sb, c->status, c->stream);
  launch_clear_sort_flag(c->status, c->stream);
  c->launches += 2 + sort_launches();
  return check_launch(c, "initial sort");
}

}  // namespace

extern "C" {

int bp_create(const bp_grid_desc *gd, const bp_allocator *al, void *stream, bp_ctx **out) {
  if (!gd || !out) return BP_ERR_ARG;
  *out = nullptr;
  bp_ctx *c = new bp_ctx();
  GridP &g = c->g;
  memset(&g, 0, sizeof g);
  const int D = gd->dims;
  if (D < 1 || D > 3) {
    delete c;
    return BP_ERR_ARG;
  }
  g.D = D;
  static const int def_tile[4][3] = {{1, 1, 1}, {Geo<1>::L0, 1, 1}, {Geo<2>::L0, Geo<2>::L1, 1},
                                     {Geo<3>::L0, Geo<3>::L1, Geo<3>::L2}};
  static const int def_margin[4] = {0, Geo<1>::M, Geo<2>::M, Geo<3>::M};
  g.M = def_margin[D];
  double inv2 = 0.0;
  long long ncell = 1;
  for (int a = 0; a < 3; ++a) {
    if (a < D) {
      if (gd->n[a] < 4 || gd->dx[a] <= 0) {
        delete c;
        return BP_ERR_ARG;
      }
      g.n[a] = (int)gd->n[a];
      g.bc[a] = gd->boundary[a] == BP_OPEN ? BP_OPEN : BP_PERIODIC;
      g.dxd[a] = gd->dx[a];
      g.L[a] = def_tile[D][a];
      if (g.n[a] % g.L[a] != 0 || (gd->tile[a] > 0 && gd->tile[a] != g.L[a])) {
        delete c;
        return BP_ERR_ARG;
      }
      inv2 += 1.0 / (gd->dx[a] * gd->dx[a]);
      g.og[a] = g.M + 2;
      g.gb[a] = g.L[a] + 2 * g.M + 5;
      g.oj[a] = g.M + 3;
      g.jb[a] = g.L[a] + 2 * g.M + 7;
    } else {
      g.n[a] = 1;
      g.bc[a] = BP_PERIODIC;
      g.dxd[a] = 1.0;
      g.L[a] = 1;
      g.og[a] = 0;
      g.gb[a] = 1;
      g.oj[a] = 0;
      g.jb[a] = 1;
    }
    g.dx[a] = (float)g.dxd[a];
    g.idx[a] = (float)(1.0 / g.dxd[a]);
    g.nt[a] = g.n[a] / g.L[a];
    ncell *= g.n[a];
  }
  if (!(gd->dt > 0) || gd->dt * std::sqrt(inv2) >= 1.0) {
    delete c;
    return BP_ERR_CFL;
  }
  if (ncell >= (1LL << 31) - 1) {
    delete c;
    return BP_ERR_ARG;
  }
  int bits = 0;
  for (int a = 0; a < 3; ++a) {
    int b = 0;
    while ((1 << b) < g.n[a]) ++b;
    g.cb[a] = b;
    g.cm[a] = (1 << b) - 1;
    bits += b;
  }
  if (bits > 31) {
    delete c;
    return BP_ERR_ARG;
  }
  g.dtd = gd->dt;
  g.dt = (float)gd->dt;
  g.ncell = ncell;
  g.ntiles = g.nt[0] * g.nt[1] * g.nt[2];
  g.cpt = g.L[0] * g.L[1] * g.L[2];
  g.gcells = g.gb[0] * g.gb[1] * g.gb[2];
  g.jcells = g.jb[0] * g.jb[1] * g.jb[2];
  c->det = gd->deposit_mode == BP_DEPOSIT_ATOMIC ? 0 : 1;
  c->stream = (cudaStream_t)stream;
  cudaGetDevice(&c->device);
  if (al && al->alloc && al->free) {
    c->alloc = *al;
    c->have_alloc = true;
  }
  for (int k = 0; k < 9; ++k) {
    c->F[k] = (float *)dalloc(c, sizeof(float) * ncell);
    if (!c->F[k]) {
      bp_destroy(c);
      return BP_ERR_OOM;
    }
  }
  // sorted deposit: the tiles add their current to a global 64-bit fixed-point
  // array; atomic deposit: per-tile FP32 boxes summed by the current-sum kernel
  if (c->det) {
    c->jfx = (unsigned long long *)dalloc(c, sizeof(unsigned long long) * 3 * (size_t)ncell);
    c->ant = (double *)dalloc(c, sizeof(double) * BP_MAX_LASER * (size_t)(ncell / g.n[0]));
    c->grec_n = (int *)dalloc(c, sizeof(int));
    c->far_n = (int *)dalloc(c, sizeof(int));
    c->far_any = (int *)dalloc(c, sizeof(int));
  }
  else c->jbox = (float *)dalloc(c, sizeof(float) * 3 * (size_t)g.jcells * g.ntiles);
  c->occ = (unsigned char *)dalloc(c, g.ntiles);
  c->jbb = (uint2 *)dalloc(c, sizeof(uint2) * g.ntiles);
  g.fnz = (unsigned char *)dalloc(c, g.ntiles);  // zero fields: no tile marked
  c->qstate = (unsigned char *)dalloc(c, g.ntiles);
  // the field kernels' active tiles (all, until the first push has run):
  // on small grids the flag's kernel would cost more than the tiles it skips
  if (g.ntiles >= 1024) {
    c->act = (unsigned char *)dalloc(c, g.ntiles);
    c->act_n = (unsigned long long *)dalloc(c, 2 * sizeof(unsigned long long));
    if (c->act) cudaMemsetAsync(c->act, 1, (size_t)g.ntiles, c->stream);
  }
  c->tile_ctr = (int *)dalloc(c, sizeof(int));
  c->tile_list = (int *)dalloc(c, sizeof(int) * g.ntiles);
  c->tile_n = (int *)dalloc(c, sizeof(int));
  c->status = (int *)dalloc(c, sizeof(int) * 4);
  c->work = (unsigned long long *)dalloc(c, sizeof(unsigned long long) * 2);
  c->clk = (long long *)dalloc(c, sizeof(long long) * kClockWords);
  long long nf = frame_floats(g);
  c->frame = nf ? (float *)dalloc(c, sizeof(float) * nf) : nullptr;
  if (!(c->det ? (void *)c->jfx : (void *)c->jbox) || (c->det && (!c->ant || !c->grec_n || !c->far_n || !c->far_any)) || !c->tile_ctr || !c->tile_list || !c->tile_n || !c->occ || !c->jbb || !g.fnz || !c->qstate || !c->status ||
      !c->work || !c->clk || (g.ntiles >= 1024 && (!c->act || !c->act_n)) || (nf && !c->frame)) {
    bp_destroy(c);
    return BP_ERR_OOM;
  }
  // 3D: tensor maps for the TMA staging of the push's field boxes (without
  // them every tile is staged by per-thread copies)
  if (encode_field_maps(g, c->F, &c->tmaps)) c->tmaps.on = 0;
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (c->sms < 1) c->sms = 1;
  if (push_prepare(g, 0, &c->push_blocks[0]) || push_prepare(g, 1, &c->push_blocks[1])) {
    bp_destroy(c);
    return BP_ERR_CUDA;
  }
  if (cudaGetLastError() != cudaSuccess) {
    bp_destroy(c);
    return BP_ERR_CUDA;
  }
  *out = c;
  return BP_OK;
}

void bp_destroy(bp_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (auto e : c->ev) cudaEventDestroy(e);
  if (c->sort_exec) cudaGraphExecDestroy(c->sort_exec);
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->read_stream) {
    cudaStreamSynchronize(c->read_stream);
    cudaStreamDestroy(c->read_stream);
  }
  for (int k = 0; k < 2; ++k) {
    if (c->snap_ready[k]) cudaEventDestroy(c->snap_ready[k]);
    if (c->snap_done[k]) cudaEventDestroy(c->snap_done[k]);
  }
  if (c->sort_runs) cudaFreeHost(c->sort_runs);
  if (c->adj.stream) {
    cudaStreamSynchronize(c->adj.stream);
    cudaStreamDestroy(c->adj.stream);
  }
  for (int k = 0; k < 2; ++k) {
    if (c->adj.rec_done[k]) cudaEventDestroy(c->adj.rec_done[k]);
    if (c->adj.rev_done[k]) cudaEventDestroy(c->adj.rev_done[k]);
  }
  std::vector<void *> all = c->owned;
  for (void *p : all) dfree(c, p);
  delete c;
}

const char *bp_last_error(const bp_ctx *c) { return c ? c->err.c_str() : "null context"; }

int bp_add_species(bp_ctx *c, const bp_species_desc *d, int *id) {
  if (!c || !d) return BP_ERR_ARG;
  if ((int)c->sp.size() >= BP_MAX_SPECIES) return fail(c, BP_ERR_ARG, "too many species");
  Species s;
  SpecP &p = s.sp;
  memset(&p, 0, sizeof p);
  p.kind = d->kind == BP_FREE ? BP_FREE : BP_TWO_BODY;
  const double dt = c->g.dtd;
  p.wd = d->weight;
  if (p.kind == BP_TWO_BODY) {
    if (!(d->Zb > 0) || !(d->mc > d->Zb) || !d->omega_b || d->n_omega < 1 || !(d->lambda0_m > 0))
      return fail(c, BP_ERR_ARG, "two-body species needs Zb > 0, mc > Zb, lambda0_m > 0, omega_b");
    // species split (Sec. 2): q2 = -Zb e, m2 = Zb m_e, q1 = qc - q2, m1 = mc - m2
    p.q2d = -d->Zb;
    p.m2d = d->Zb;
    p.q1d = d->qc - p.q2d;
    p.m1d = d->mc - p.m2d;
    const double kappa = R_E * 2.0 * M_PI / d->lambda0_m;
    const double mr = p.m1d * p.m2d / (p.m1d + p.m2d);
    std::vector<float> ac(d->n_omega);
    for (int i = 0; i < d->n_omega; ++i) {
      double w = d->omega_b[i];
      if (!(w > 0)) return fail(c, BP_ERR_ARG, "omega_b must be positive");
      // leapfrog stability of the internal oscillator
      if (w * dt >= 2.0) return fail(c, BP_ERR_CFL, "omega_b dt = %g >= 2", w * dt);
      // natural frequency (Sec. 3.1): w^2 = |q1 q2| kappa / (m_r ac^3)
      ac[i] = (float)std::cbrt(std::fabs(p.q1d * p.q2d) * kappa / (mr * w * w));
      s.omega.push_back(w);
    }
    p.kappa = (float)kappa;
    p.nac = d->n_omega;
    float *acd = (float *)dalloc(c, sizeof(float) * ac.size());
    if (!acd) return fail(c, BP_ERR_OOM, "a_c table");
    cudaMemcpyAsync(acd, ac.data(), sizeof(float) * ac.size(), cudaMemcpyHostToDevice, c->stream);
    cudaStreamSynchronize(c->stream);
    p.ac = acd;
    s.ac_dev = acd;
  } else {
    if (!(d->m > 0)) return fail(c, BP_ERR_ARG, "free species needs m > 0");
    p.q1d = d->q;
    p.m1d = d->m;
    p.q2d = p.m2d = 0.0;
  }
  p.q1 = (float)p.q1d;
  p.m1 = (float)p.m1d;
  p.q2 = (float)p.q2d;
  p.m2 = (float)p.m2d;
  p.h1 = (float)(p.q1d * dt / (2.0 * p.m1d));
  p.h2 = p.m2d > 0 ? (float)(p.q2d * dt / (2.0 * p.m2d)) : 0.0f;
  p.qw1 = (float)(p.q1d * p.wd);
  p.qw2 = (float)(p.q2d * p.wd);
  c->sp.push_back(s);
  update_jscale(c);
  if (id) *id = (int)c->sp.size() - 1;
  return BP_OK;
}

}  // extern "C"

namespace {
// the end of a load: wait for the conversion, check the status word, sort
int finish_load(bp_ctx *c, Species &s, long long n, void *stage) {
  cudaStream_t st = c->stream;
  cudaError_t e = cudaStreamSynchronize(st);
  dfree(c, stage);
  if (e != cudaSuccess) return cuda_fail(c, e, "load");
  int stw = 0;
  cudaMemcpy(&stw, c->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (stw & ST_NONFINITE) return fail(c, BP_ERR_NONFINITE, "non-finite position or momentum in the load");
  if (stw & ST_DOMAIN) return fail(c, BP_ERR_DOMAIN, "a particle lies outside the grid or has a bad param_idx");
  int rc = initial_sort(c, s, n);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(c, e, "load sort");
  if (rc) return rc;
  s.n = n;
  s.loaded = true;
  return BP_OK;
}
}  // namespace

extern "C" {

int bp_set_lattice(bp_ctx *c, int sid, const double *sites, int64_t n_sites, int per_site, double jitter,
                   uint64_t seed, double sigma_u, const int32_t *site_param) {
  if (!c || sid < 0 || sid >= (int)c->sp.size() || n_sites < 0 || per_site < 1 || (n_sites > 0 && !sites) ||
      !(jitter >= 0.0) || !(sigma_u >= 0.0))
    return BP_ERR_ARG;
  Species &s = c->sp[sid];
  if (s.loaded) return fail(c, BP_ERR_STATE, "species %d already loaded", sid);
  const long long n = n_sites * (long long)per_site;
  if (n >= (1LL << 31) - 1) return fail(c, BP_ERR_ARG, "too many particles");
  const GridP &g = c->g;
  const int D = g.D;
  int rc = alloc_particles(c, s, n, site_param != nullptr);
  if (rc) return rc;
  s.has_pidx = site_param != nullptr;
  s.pidx_host.clear();
  if (site_param) {
    s.pidx_host.resize((size_t)n);
    for (long long q = 0; q < n; ++q) s.pidx_host[q] = site_param[q / per_site];
  }
  cudaStream_t st = c->stream;
  const long long chunk = std::min<long long>(std::max<long long>(n, 1), 1LL << 25);
  const size_t rows = (size_t)chunk * (sizeof(double) * (D + 3) + sizeof(int));
  const size_t ns = (size_t)std::max<int64_t>(n_sites, 1);
  char *stage = (char *)dalloc(c, rows + (sizeof(double) * D + sizeof(int)) * ns);
  if (!stage) return fail(c, BP_ERR_OOM, "lattice staging");
  double *sx = (double *)stage;
  double *su = sx + (size_t)chunk * D;
  int *sp_ = (int *)(su + (size_t)chunk * 3);
  double *dsites = (double *)(stage + rows);
  int *dparam = (int *)(dsites + (size_t)D * ns);
  int zero = 0;
  cudaMemcpyAsync(c->status, &zero, sizeof(int), cudaMemcpyHostToDevice, st);
  if (n_sites > 0) cudaMemcpyAsync(dsites, sites, sizeof(double) * D * n_sites, cudaMemcpyHostToDevice, st);
  if (site_param && n_sites > 0) cudaMemcpyAsync(dparam, site_param, sizeof(int) * n_sites, cudaMemcpyHostToDevice, st);
  for (long long b = 0; b < n; b += chunk) {
    long long k = std::min(chunk, n - b);
    launch_gen_lattice(D, dsites, per_site, jitter, seed, sigma_u, site_param ? dparam : nullptr, b, k, sx, su,
                       site_param ? sp_ : nullptr, st);
    launch_load_convert(g, s.sp, s.p, sx, su, site_param ? sp_ : nullptr, b, k, c->status, st);
    c->launches += 2;
  }
  if ((rc = check_launch(c, "lattice generation"))) {
    dfree(c, stage);
    return rc;
  }
  return finish_load(c, s, n, stage);
}

int bp_load_particles(bp_ctx *c, int sid, const double *x, const double *u, const int32_t *pidx, int64_t n) {
  if (!c || sid < 0 || sid >= (int)c->sp.size() || n < 0 || (n > 0 && !x)) return BP_ERR_ARG;
  Species &s = c->sp[sid];
  if (s.loaded) return fail(c, BP_ERR_STATE, "species %d already loaded", sid);
  if (n >= (1LL << 31) - 1) return fail(c, BP_ERR_ARG, "too many particles");
  const GridP &g = c->g;
  const int D = g.D;
  int rc = alloc_particles(c, s, n, pidx != nullptr);
  if (rc) return rc;
  s.has_pidx = pidx != nullptr;
  if (pidx) s.pidx_host.assign(pidx, pidx + n);
  else s.pidx_host.clear();  // all 0
  cudaStream_t st = c->stream;
  const long long chunk = std::min<long long>(std::max<long long>(n, 1), 1LL << 25);
  int zero = 0;
  // Arrays in page-locked host memory that the device can address (pinned
  // or registered, e.g. torch's pin_memory()): the conversion kernel reads
  // them where they are, over the host link, with no staging copy.
  // Otherwise they are copied to a device staging buffer chunk by chunk.
  const void *dx = mapped_host(x), *du = u ? mapped_host(u) : nullptr, *dp = pidx ? mapped_host(pidx) : nullptr;
  if (dx && (!u || du) && (!pidx || dp)) {
    cudaMemcpyAsync(c->status, &zero, sizeof(int), cudaMemcpyHostToDevice, st);
    for (long long b = 0; b < n; b += chunk) {
      const long long k = std::min(chunk, n - b);
      launch_load_convert(g, s.sp, s.p, static_cast<const double *>(dx) + b * D,
                          u ? static_cast<const double *>(du) + b * 3 : nullptr,
                          pidx ? static_cast<const int *>(dp) + b : nullptr, b, k, c->status, st);
      c->launches++;
    }
    if ((rc = check_launch(c, "load conversion"))) return rc;
    return finish_load(c, s, n, nullptr);
  }
  char *stage = (char *)dalloc(c, (size_t)chunk * (sizeof(double) * (D + 3) + sizeof(int)));
  if (!stage) return fail(c, BP_ERR_OOM, "load staging");
  double *sx = (double *)stage;
  double *su = sx + (size_t)chunk * D;
  int *sp_ = (int *)(su + (size_t)chunk * 3);
  cudaMemcpyAsync(c->status, &zero, sizeof(int), cudaMemcpyHostToDevice, st);
  for (long long b = 0; b < n; b += chunk) {
    long long k = std::min(chunk, n - b);
    cudaMemcpyAsync(sx, x + b * D, sizeof(double) * k * D, cudaMemcpyHostToDevice, st);
    if (u) cudaMemcpyAsync(su, u + b * 3, sizeof(double) * k * 3, cudaMemcpyHostToDevice, st);
    if (pidx) cudaMemcpyAsync(sp_, pidx + b, sizeof(int) * k, cudaMemcpyHostToDevice, st);
    launch_load_convert(g, s.sp, s.p, sx, u ? su : nullptr, pidx ? sp_ : nullptr, b, k, c->status, st);
    c->launches++;
  }
  if ((rc = check_launch(c, "load conversion"))) {
    dfree(c, stage);
    return rc;
  }
  return finish_load(c, s, n, stage);
}

int bp_set_medium(bp_ctx *c, int sid, const int64_t lo[3], const int64_t hi[3], int ppc, uint64_t seed,
                  double sigma_u) {
  if (!c || sid < 0 || sid >= (int)c->sp.size() || !lo || !hi || ppc < 1) return BP_ERR_ARG;
  Species &s = c->sp[sid];
  if (s.loaded) return fail(c, BP_ERR_STATE, "species %d already loaded", sid);
  const GridP &g = c->g;
  int l[3] = {0, 0, 0}, h[3] = {1, 1, 1};
  long long n = ppc;
  for (int a = 0; a < g.D; ++a) {
    if (lo[a] < 0 || hi[a] > g.n[a] || hi[a] <= lo[a]) return fail(c, BP_ERR_ARG, "bad medium box");
    l[a] = (int)lo[a];
    h[a] = (int)hi[a];
    n *= (hi[a] - lo[a]);
  }
  if (n >= (1LL << 31) - 1) return fail(c, BP_ERR_ARG, "too many particles");
  int rc = alloc_particles(c, s, n, false);
  if (rc) return rc;
  s.pidx_host.clear();  // all 0
  launch_gen_medium(g, s.sp, s.p, l, h, ppc, seed, sigma_u, 0, n, c->stream);
  c->launches++;
  if ((rc = check_launch(c, "medium generation"))) return rc;
  rc = initial_sort(c, s, n);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "medium");
  if (rc) return rc;
  s.n = n;
  s.loaded = true;
  return BP_OK;
}

int bp_add_laser(bp_ctx *c, const bp_laser_desc *L) {
  if (!c || !L) return BP_ERR_ARG;
  if ((int)c->las.size() >= BP_MAX_LASER) return fail(c, BP_ERR_ARG, "too many lasers");
  if ((L->comp != 1 && L->comp != 2) || L->ia < 0 || L->ia >= c->g.n[0])
    return fail(c, BP_ERR_ARG, "laser comp must be 1 or 2 and ia inside the grid");
  LaserP p;
  p.comp = L->comp;
  p.a0 = L->a0;
  p.omega = L->omega;
  p.theta = L->theta;
  p.waist = L->waist;
  p.fwhm = L->fwhm;
  p.t0 = L->t0;
  p.ramp = L->ramp;
  p.phase = L->phase;
  p.ia = (int)L->ia;
  p.yc = L->yc;
  p.zc = L->zc;
  c->las.push_back(p);
  return BP_OK;
}

int bp_add_probe(bp_ctx *c, int comp, const int64_t *nodes, int64_t npts, int64_t capacity, int *pid) {
  if (!c || comp < 0 || comp > 8 || !nodes || npts < 1 || capacity < 1) return BP_ERR_ARG;
  if ((int)c->pr.size() >= BP_MAX_PROBE) return fail(c, BP_ERR_ARG, "too many probes");
  for (int64_t i = 0; i < npts; ++i)
    if (nodes[i] < 0 || nodes[i] >= c->g.ncell) return fail(c, BP_ERR_ARG, "probe node out of range");
  Probe p;
  p.comp = comp;
  p.npts = npts;
  p.cap = capacity;
  p.count = 0;
  p.nodes = (long long *)dalloc(c, sizeof(long long) * npts);
  p.buf = (float *)dalloc(c, sizeof(float) * npts * capacity);
  if (!p.nodes || !p.buf) return fail(c, BP_ERR_OOM, "probe buffers");
  cudaMemcpyAsync(p.nodes, nodes, sizeof(long long) * npts, cudaMemcpyHostToDevice, c->stream);
  cudaStreamSynchronize(c->stream);
  c->pr.push_back(p);
  if (pid) *pid = (int)c->pr.size() - 1;
  return BP_OK;
}

}  // extern "C"

namespace {

// sorted mode: room for the general-case records of a step, 1 in 256
// particles (at least 65,536); a step with more deposits the rest in place
void ensure_records(bp_ctx *c) {
  if (!c->det) return;
  long long n = 0;
  for (auto &s : c->sp)
    if (s.loaded) n += s.p.cap;
  const long long want =
      c->grec_fixed > 0 ? c->grec_fixed : std::min<long long>(1LL << 30, std::max<long long>(65536, n / 256));
  // the far-ion list: as many entries as the default record capacity
  const long long want_far = std::min<long long>(1LL << 30, std::max<long long>(65536, n / 256));
  if (!c->far || c->far_cap < want_far) {
    if (c->far) dfree(c, c->far);
    c->far = (int4 *)dalloc(c, sizeof(int4) * (size_t)want_far);
    c->far_cap = c->far ? want_far : 0;
  }
  if (c->grec && (c->grec_fixed > 0 ? c->grec_cap == want : c->grec_cap >= want)) return;
  if (c->grec) dfree(c, c->grec);
  c->grec = dalloc(c, push_record_bytes() * (size_t)want);
  c->grec_cap = c->grec ? want : 0;
}

PushArgs push_args(bp_ctx *c, int *nsp_out) {
  ensure_records(c);
  PushArgs A;
  memset(&A, 0, sizeof A);
  int nsp = 0;
  for (auto &s : c->sp) {
    if (!s.loaded) continue;
    A.sp[nsp] = s.sp;
    A.p[nsp] = s.p;
    ++nsp;
  }
  A.nsp = nsp;
  for (int k = 0; k < 3; ++k) {
    A.E[k] = c->F[k];
    A.B[k] = c->F[3 + k];
  }
  A.jbox = c->jbox;
  A.jfx = c->jfx;
  A.grec = c->grec;
  A.grec_n = c->grec_n;
  A.far = c->far;
  A.far_n = c->far_n;
  A.far_cap = (int)c->far_cap;
  A.far_any = c->far_any;
  A.grec_cap = (int)c->grec_cap;
  A.occ = c->occ;
  A.jbb = c->jbb;
  A.qstate = c->qstate;
  A.tile_ctr = c->tile_ctr;
  A.tile_list = c->tile_list;
  A.tile_n = c->tile_n;
  A.status = c->status;
  A.jscale = c->jscale;
  A.jinv = c->jinv;
  A.work = c->timing ? c->work : nullptr;
  A.push_blocks = c->push_blocks[c->det ? 1 : 0];
  A.sms = c->sms;
  *nsp_out = nsp;
  return A;
}

// copy of the particle arrays of one species (same capacity)
int copy_alloc(bp_ctx *c, const PartP &src, int D, bool two, PartP &dst) {
  dst = src;
  long long cap = src.cap;
  dst.cell = (int *)dalloc(c, sizeof(int) * cap);
  dst.off = (float *)dalloc(c, sizeof(float) * D * cap);
  dst.u1 = (float *)dalloc(c, sizeof(float) * 3 * cap);
  dst.id = (int *)dalloc(c, sizeof(int) * cap);
  dst.tstart = (int *)dalloc(c, sizeof(int) * (c->g.ntiles + 1));
  dst.r = two ? (float *)dalloc(c, sizeof(float) * 3 * cap) : nullptr;
  dst.u2 = two ? (float *)dalloc(c, sizeof(float) * 3 * cap) : nullptr;
  dst.pidx = src.pidx ? (int *)dalloc(c, sizeof(int) * cap) : nullptr;
  if (!dst.cell || !dst.off || !dst.u1 || !dst.id || !dst.tstart || (two && (!dst.r || !dst.u2)) ||
      (src.pidx && !dst.pidx))
    return BP_ERR_OOM;
  return BP_OK;
}

// batched device-to-device copies (one kernel per up to 32 arrays)
void cl_flush(bp_ctx *c, CopyList &L) {
  if (L.n) {
    launch_copy_many(L, c->sms, c->stream);
    c->launches++;
    L.n = 0;
  }
}
void cl_add(bp_ctx *c, CopyList &L, const void *src, void *dst, long long bytes) {
  if (L.n == CopyList::MAX) cl_flush(c, L);
  L.src[L.n] = src;
  L.dst[L.n] = dst;
  L.words[L.n] = bytes / 4;
  ++L.n;
}
void cl_parts(bp_ctx *c, CopyList &L, const PartP &src, PartP &dst, int D, bool two) {
  const long long cap = src.cap;
  cl_add(c, L, src.cell, dst.cell, sizeof(int) * cap);
  cl_add(c, L, src.off, dst.off, sizeof(float) * D * cap);
  cl_add(c, L, src.u1, dst.u1, sizeof(float) * 3 * cap);
  cl_add(c, L, src.id, dst.id, sizeof(int) * cap);
  cl_add(c, L, src.tstart, dst.tstart, sizeof(int) * (c->g.ntiles + 1));
  if (two) {
    cl_add(c, L, src.r, dst.r, sizeof(float) * 3 * cap);
    cl_add(c, L, src.u2, dst.u2, sizeof(float) * 3 * cap);
  }
  if (src.pidx) cl_add(c, L, src.pidx, dst.pidx, sizeof(int) * cap);
}

// the re-sort graph of the current particle arrays (built on first use and
// after any reallocation); false if the CUDA runtime cannot build it, in
// which case the step launches the sort pipeline directly
bool sort_graph(bp_ctx *c) {
  if (c->sort_exec && !c->sort_dirty) return true;
  if (c->sort_exec) {
    cudaGraphExecDestroy(c->sort_exec);
    c->sort_exec = nullptr;
  }
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    c->cap_stream = nullptr;
    cudaGetLastError();
    return false;
  }
  if (!c->sort_runs) {
    if (cudaHostAlloc((void **)&c->sort_runs, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&c->sort_runs_dev, c->sort_runs, 0) != cudaSuccess) {
      if (c->sort_runs) cudaFreeHost(c->sort_runs);
      c->sort_runs = nullptr;
      cudaGetLastError();
      return false;
    }
    *c->sort_runs = 0;
  }
  SpecP sp[BP_MAX_SPECIES];
  PartP pp[BP_MAX_SPECIES];
  int n = 0;
  for (auto &s : c->sp)
    if (s.loaded && n < BP_MAX_SPECIES) {
      sp[n] = s.sp;
      pp[n] = s.p;
      ++n;
    }
  cudaGraphExec_t ex = nullptr;
  if (make_sort_graph(c->g, n, sp, pp, c->sb, c->status, c->sort_runs_dev, c->cap_stream, &ex) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->sort_exec = ex;
  c->sort_nsp = n;
  c->sort_dirty = false;
  return true;
}

// the step clock from the host's state (the step number, the probes' sample
// counts and capacities); run before the first step of every call that steps
void sync_clock(bp_ctx *c, cudaStream_t st) {
  ClockState v;
  memset(&v, 0, sizeof v);
  v.step = c->step;
  v.nprobe = (int)c->pr.size();
  for (int p = 0; p < v.nprobe; ++p) {
    v.count[p] = c->pr[p].count;
    v.cap[p] = c->pr[p].cap;
  }
  launch_clock_set(c->clk, v, st);
  c->launches++;
}

// re-sort when a particle left its tile margin in the previous step
void launch_resort(bp_ctx *c, int nsp, cudaStream_t st) {
  if (!nsp) return;
  if (sort_graph(c)) {
    cudaGraphLaunch(c->sort_exec, st);
    c->launches += 1;  // the condition kernel; a re-sort that ran is counted by bp_kernel_launches
  } else {
    for (auto &s : c->sp)
      if (s.loaded) launch_sort(c->g, s.sp, s.p, c->sb, c->status, st);
    launch_clear_sort_flag(c->status, st);
    c->launches += nsp * sort_launches() + 1;
  }
}

// The launches of one leapfrog step after the re-sort, on stream st.  They
// are the same every step (the time and the probe slots come from the device
// clock), so a plain step and a replay of their captured graph do the same
// work.  When snap_fields is given, E^n and B^n (after the first half step)
// and the particle state before the push are copied there; with push timing
// on, events bracket the push.
void step_launches(bp_ctx *c, const PushArgs &A, bool probes, cudaStream_t st, float *snap_fields,
                   std::vector<bp_part_copy> *snap_parts) {
  const GridP &g = c->g;
  float *E[3] = {c->F[0], c->F[1], c->F[2]}, *B[3] = {c->F[3], c->F[4], c->F[5]}, *J[3] = {c->F[6], c->F[7], c->F[8]};
  const float *cE[3] = {E[0], E[1], E[2]}, *cB[3] = {B[0], B[1], B[2]};
  launch_yee_b(g, B, cE, 0.5f * g.dt, c->act, st);
  if (snap_fields) {
    CopyList L;
    for (int k = 0; k < 6; ++k) cl_add(c, L, c->F[k], snap_fields + (size_t)k * g.ncell, sizeof(float) * g.ncell);
    int q = 0;
    for (auto &s : c->sp)
      if (s.loaded) cl_parts(c, L, s.p, (*snap_parts)[q++].p, g.D, s.sp.kind == BP_TWO_BODY);
    cl_flush(c, L);
  }
  if (c->timing) {
    if (c->ev_used + 2 > c->ev.size()) {
      for (int k = 0; k < 64; ++k) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev.push_back(e);
      }
    }
    cudaEventRecord(c->ev[c->ev_used], st);
  }
  launch_push(g, A, c->tmaps, st);
  if (c->timing) {
    cudaEventRecord(c->ev[c->ev_used + 1], st);
    c->ev_used += 2;
  }
  if (!c->det) launch_jsum(g, c->jbox, c->occ, c->jbb, J, c->las.data(), (int)c->las.size(), c->clk, st);
  if (c->act) {
    int ia_lo = INT_MAX, ia_hi = INT_MIN;
    for (auto &L : c->las) {
      ia_lo = std::min(ia_lo, L.ia);
      ia_hi = std::max(ia_hi, L.ia);
    }
    launch_tile_active(g, c->qstate, c->far_any, ia_lo, ia_hi, c->act, c->act_n, st);
  }
  launch_yee_b(g, B, cE, 0.5f * g.dt, c->act, st);
  launch_yee_e(g, E, cB, J, c->frame, c->det ? c->jfx : nullptr, c->jinv, c->las.data(), (int)c->las.size(), c->clk,
               c->ant, c->act, st);
  if (probes)
    for (size_t p = 0; p < c->pr.size(); ++p)
      launch_probe(c->F[c->pr[p].comp], c->pr[p].nodes, c->pr[p].npts, c->pr[p].buf, c->clk, (int)p, st);
  launch_clock_tick(c->clk, probes ? (int)c->pr.size() : 0, st);
}

// the host's record of one step (the device's is the clock)
void step_account(bp_ctx *c, bool probes) {
  int nopen = 0;
  for (int a = 0; a < c->g.D; ++a) nopen += c->g.bc[a] == BP_OPEN;
  // quiet-tile pass, push, records (sorted) or current sum (atomic), antenna (sorted, with lasers),
  // Yee (3), Mur, the clock
  c->launches += (c->det ? 6 + (c->las.empty() ? 0 : 1) : 6) + (nopen ? 1 + nopen : 0) + 1 + (c->act ? 1 : 0);
  c->step++;
  if (probes)
    for (auto &p : c->pr) {
      c->launches++;
      if (p.count < p.cap) p.count++;
    }
}

// one leapfrog step, launched directly
int one_step(bp_ctx *c, const PushArgs &A, int nsp, bool probes, float *snap_fields,
             std::vector<bp_part_copy> *snap_parts) {
  launch_resort(c, nsp, c->stream);
  step_launches(c, A, probes, c->stream, snap_fields, snap_parts);
  step_account(c, probes);
  return check_launch(c, "step");
}

// one step through the step graph (step_graph succeeded for the current
// arguments): one launch when the graph holds the re-sort, else two
int graph_step(bp_ctx *c, int nsp) {
  if (c->step_sorts) c->launches += 1;  // the re-sort's condition kernel
  else launch_resort(c, nsp, c->stream);
  cudaGraphLaunch(c->step_exec, c->stream);
  step_account(c, true);
  return check_launch(c, "step graph");
}

// The graph of a plain step's launches (probes recorded, no push timing, no
// snapshots), captured on the capture stream; reused while every launch
// argument is unchanged.  False when the runtime cannot capture or
// instantiate it: the caller then launches the steps directly.
bool step_graph(bp_ctx *c, const PushArgs &A) {
  std::string key;
  auto put = [&key](const void *p, size_t n) { key.append(static_cast<const char *>(p), n); };
  put(&A, sizeof A);
  put(&c->tmaps, sizeof c->tmaps);
  put(&c->g, sizeof c->g);
  put(c->F, sizeof c->F);
  const void *ptrs[] = {c->jfx, c->jbox, c->occ, c->jbb, c->frame, c->ant, c->clk, c->sort_runs_dev};
  put(ptrs, sizeof ptrs);
  put(&c->sb, sizeof c->sb);
  put(&c->det, sizeof c->det);
  put(&c->jinv, sizeof c->jinv);
  if (!c->las.empty()) put(c->las.data(), sizeof(LaserP) * c->las.size());
  for (auto &p : c->pr) {
    const void *pp[] = {p.nodes, p.buf};
    put(pp, sizeof pp);
    put(&p.comp, sizeof p.comp);
    put(&p.npts, sizeof p.npts);
  }
  if (c->step_exec && key == c->step_key) return true;
  if (c->step_exec) {
    cudaGraphExecDestroy(c->step_exec);
    c->step_exec = nullptr;
  }
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    c->cap_stream = nullptr;
    cudaGetLastError();
    return false;
  }
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  step_launches(c, A, true, c->cap_stream, nullptr, nullptr);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
  cudaGraphExec_t ex = nullptr;
  // the re-sort's conditional node first, the captured launches after it
  // (one graph launch per step); else the captured launches alone
  bool sorts = false;
  if (e == cudaSuccess && A.nsp > 0 && sort_graph(c)) {
    SpecP sp[BP_MAX_SPECIES];
    PartP pp[BP_MAX_SPECIES];
    int n = 0;
    for (auto &s : c->sp)
      if (s.loaded && n < BP_MAX_SPECIES) {
        sp[n] = s.sp;
        pp[n] = s.p;
        ++n;
      }
    sorts = make_sort_graph(c->g, n, sp, pp, c->sb, c->status, c->sort_runs_dev, c->cap_stream, &ex, graph) ==
            cudaSuccess;
    if (!sorts) {
      ex = nullptr;
      cudaGetLastError();
    }
  }
  if (e == cudaSuccess && !sorts) e = cudaGraphInstantiate(&ex, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    if (ex) cudaGraphExecDestroy(ex);
    cudaGetLastError();
    return false;
  }
  c->step_exec = ex;
  c->step_sorts = sorts;
  c->step_key = key;
  return true;
}

}  // namespace

extern "C" {

int bp_step(bp_ctx *c, int64_t nsteps) {
  if (!c || nsteps < 0) return BP_ERR_ARG;
  if (nsteps == 0) return BP_OK;
  int nsp = 0;
  PushArgs A = push_args(c, &nsp);
  sync_clock(c, c->stream);
  // two or more steps without push timing: one graph launch per step (the
  // conditional re-sort, then the step's kernels)
  const bool graph = nsteps >= 2 && !c->timing && step_graph(c, A);
  for (int64_t it = 0; it < nsteps; ++it) {
    int rc;
    rc = graph ? graph_step(c, nsp) : one_step(c, A, nsp, true, nullptr, nullptr);
    if (rc) return rc;
  }
  return BP_OK;
}

int bp_sync(bp_ctx *c) {
  if (!c) return BP_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess && c->read_stream) e = cudaStreamSynchronize(c->read_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "sync");
  if (c->timing && c->ev_used) {
    for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]);
      c->push_ms += ms;
      c->push_launches++;
    }
    c->ev_used = 0;
  }
  int st = 0;
  e = cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "status");
  if (st & ST_NONFINITE) return fail(c, BP_ERR_NONFINITE, "non-finite momentum");
  if (st & ST_DOMAIN) return fail(c, BP_ERR_DOMAIN, "a two-body ion left the region its tile handles or the grid");
  if (st & ST_TIMEOUT) return fail(c, BP_ERR_TIMEOUT, "device wait timed out");
  return BP_OK;
}

int bp_read_field(bp_ctx *c, int comp, float *dst, int on_device) {
  if (!c || comp < 0 || comp > 8 || !dst) return BP_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(dst, c->F[comp], sizeof(float) * c->g.ncell,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? BP_OK : cuda_fail(c, e, "read field");
}

int bp_read_field_async(bp_ctx *c, int comp, float *dst) {
  if (!c || comp < 0 || comp > 8 || !dst) return BP_ERR_ARG;
  const size_t bytes = sizeof(float) * c->g.ncell;
  if (!c->snap[0]) {
    c->snap[0] = (float *)dalloc(c, bytes);
    c->snap[1] = (float *)dalloc(c, bytes);
    if (!c->snap[0] || !c->snap[1]) return fail(c, BP_ERR_OOM, "read snapshots");
    if (cudaStreamCreateWithFlags(&c->read_stream, cudaStreamNonBlocking) != cudaSuccess) {
      c->read_stream = nullptr;
      return cuda_fail(c, cudaGetLastError(), "read stream");
    }
    for (int k = 0; k < 2; ++k) {
      cudaEventCreateWithFlags(&c->snap_ready[k], cudaEventDisableTiming);
      cudaEventCreateWithFlags(&c->snap_done[k], cudaEventDisableTiming);
      cudaEventRecord(c->snap_done[k], c->read_stream);
    }
  }
  const int k = c->snap_next;
  c->snap_next ^= 1;
  // snapshot k may be overwritten once its previous copy to the host is done
  cudaStreamWaitEvent(c->stream, c->snap_done[k], 0);
  cudaError_t e = cudaMemcpyAsync(c->snap[k], c->F[comp], bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaEventRecord(c->snap_ready[k], c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->read_stream, c->snap_ready[k], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst, c->snap[k], bytes, cudaMemcpyDeviceToHost, c->read_stream);
  if (e == cudaSuccess) e = cudaEventRecord(c->snap_done[k], c->read_stream);
  return e == cudaSuccess ? BP_OK : cuda_fail(c, e, "read field async");
}

int bp_write_field(bp_ctx *c, int comp, const float *src, int on_device) {
  if (!c || comp < 0 || comp > 8 || !src) return BP_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(c->F[comp], src, sizeof(float) * c->g.ncell,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && comp < 6) refresh_marks(c);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? BP_OK : cuda_fail(c, e, "write field");
}

int bp_read_probe(bp_ctx *c, int pid, float *dst, int64_t cap, int64_t *n) {
  if (!c || pid < 0 || pid >= (int)c->pr.size() || !dst) return BP_ERR_ARG;
  Probe &p = c->pr[pid];
  long long k = std::min<long long>(p.count, cap);
  cudaError_t e = cudaMemcpyAsync(dst, p.buf, sizeof(float) * k * p.npts, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (n) *n = p.count;
  return e == cudaSuccess ? BP_OK : cuda_fail(c, e, "read probe");
}

int bp_read_particles(bp_ctx *c, int sid, double *x1, double *x2, double *u1, double *u2, int64_t cap,
                      int64_t *nout) {
  if (!c || sid < 0 || sid >= (int)c->sp.size()) return BP_ERR_ARG;
  Species &s = c->sp[sid];
  if (!s.loaded) return fail(c, BP_ERR_STATE, "species not loaded");
  const GridP &g = c->g;
  const int D = g.D;
  const bool two = s.sp.kind == BP_TWO_BODY;
  const long long pc = s.p.cap;
  cudaStream_t st = c->stream;
  cudaStreamSynchronize(st);
  int cnt = 0;
  cudaMemcpy(&cnt, s.p.tstart + g.ntiles, sizeof(int), cudaMemcpyDeviceToHost);
  std::vector<int> cell(cnt), id(cnt);
  std::vector<float> off((size_t)D * cnt), uu1(3 * (size_t)cnt), r(two ? 3 * (size_t)cnt : 0),
      uu2(two ? 3 * (size_t)cnt : 0);
  cudaMemcpy(cell.data(), s.p.cell, sizeof(int) * cnt, cudaMemcpyDeviceToHost);
  cudaMemcpy(id.data(), s.p.id, sizeof(int) * cnt, cudaMemcpyDeviceToHost);
  for (int a = 0; a < D; ++a)
    cudaMemcpy(off.data() + (size_t)a * cnt, s.p.off + a * pc, sizeof(float) * cnt, cudaMemcpyDeviceToHost);
  for (int a = 0; a < 3; ++a) {
    cudaMemcpy(uu1.data() + (size_t)a * cnt, s.p.u1 + a * pc, sizeof(float) * cnt, cudaMemcpyDeviceToHost);
    if (two) {
      cudaMemcpy(r.data() + (size_t)a * cnt, s.p.r + a * pc, sizeof(float) * cnt, cudaMemcpyDeviceToHost);
      cudaMemcpy(uu2.data() + (size_t)a * cnt, s.p.u2 + a * pc, sizeof(float) * cnt, cudaMemcpyDeviceToHost);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "read particles");
  // alive particles, in load order
  std::vector<std::pair<int, int>> order;
  order.reserve(cnt);
  for (int q = 0; q < cnt; ++q)
    if (cell[q] >= 0) order.push_back({id[q], q});
  std::sort(order.begin(), order.end());
  long long k = 0;
  for (auto &pr : order) {
    if (k >= cap) break;
    int q = pr.second;
    int cc[3];
    unpack_cell(g, cell[q], cc);
    for (int a = 0; a < 3; ++a) {
      double xa = a < D ? ((double)cc[a] + (double)off[(size_t)a * cnt + q]) * g.dxd[a] : 0.0;
      if (x1) x1[3 * k + a] = xa;
      if (two && x2) x2[3 * k + a] = xa - (double)r[(size_t)a * cnt + q];
      if (u1) u1[3 * k + a] = uu1[(size_t)a * cnt + q];
      if (two && u2) u2[3 * k + a] = uu2[(size_t)a * cnt + q];
    }
    ++k;
  }
  if (nout) *nout = (int64_t)order.size();
  return BP_OK;
}

int bp_read_particles_by_id(bp_ctx *c, int sid, const int64_t *ids, int64_t n, double *x1, double *x2,
                            double *u1, double *u2, unsigned char *found) {
  if (!c || sid < 0 || sid >= (int)c->sp.size() || n < 0 || (n > 0 && !ids) || n > INT32_MAX) return BP_ERR_ARG;
  Species &s = c->sp[sid];
  if (!s.loaded) return fail(c, BP_ERR_STATE, "species not loaded");
  if (n == 0) return BP_OK;
  const GridP &g = c->g;
  const int D = g.D;
  const bool two = s.sp.kind == BP_TWO_BODY;
  cudaStream_t st = c->stream;
  // the ids sorted, with the output row of each
  std::vector<std::pair<long long, int>> key(n);
  for (long long k = 0; k < n; ++k) {
    if (ids[k] < 0 || ids[k] > INT32_MAX) return fail(c, BP_ERR_ARG, "bp_read_particles_by_id: id out of range");
    key[k] = {ids[k], (int)k};
  }
  std::sort(key.begin(), key.end());
  std::vector<int> sid_h(n), srow_h(n);
  for (long long k = 0; k < n; ++k) {
    sid_h[k] = (int)key[k].first;
    srow_h[k] = key[k].second;
  }
  int *d_sid = (int *)dalloc(c, sizeof(int) * n), *d_srow = (int *)dalloc(c, sizeof(int) * n);
  int *d_cell = (int *)dalloc(c, sizeof(int) * n);
  float *d_out = (float *)dalloc(c, sizeof(float) * 12 * n);
  unsigned char *d_found = (unsigned char *)dalloc(c, n);
  auto release = [&]() {
    dfree(c, d_sid);
    dfree(c, d_srow);
    dfree(c, d_cell);
    dfree(c, d_out);
    dfree(c, d_found);
  };
  if (!d_sid || !d_srow || !d_cell || !d_out || !d_found) {
    release();
    return fail(c, BP_ERR_OOM, "bp_read_particles_by_id scratch");
  }
  cudaMemcpyAsync(d_sid, sid_h.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_srow, srow_h.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(d_found, 0, n, st);
  cudaStreamSynchronize(st);
  int cnt = 0;
  cudaMemcpy(&cnt, s.p.tstart + g.ntiles, sizeof(int), cudaMemcpyDeviceToHost);
  launch_pick(s.p, D, two ? 1 : 0, cnt, d_sid, d_srow, (int)n, d_cell, d_out, d_found, st);
  c->launches++;
  std::vector<int> cell(n);
  std::vector<float> raw(12 * (size_t)n);
  std::vector<unsigned char> fnd(n);
  cudaMemcpyAsync(cell.data(), d_cell, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(raw.data(), d_out, sizeof(float) * 12 * n, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(fnd.data(), d_found, n, cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  release();
  if (e != cudaSuccess) return cuda_fail(c, e, "read particles by id");
  for (long long k = 0; k < n; ++k) {
    if (found) found[k] = fnd[k];
    int cc[3] = {0, 0, 0};
    if (fnd[k]) unpack_cell(g, cell[k], cc);
    const float *o = raw.data() + 12 * (size_t)k;
    for (int a = 0; a < 3; ++a) {
      const double xa = fnd[k] && a < D ? ((double)cc[a] + (double)o[a]) * g.dxd[a] : 0.0;
      if (x1) x1[3 * k + a] = xa;
      if (x2) x2[3 * k + a] = fnd[k] && two ? xa - (double)o[3 + a] : 0.0;
      if (u1) u1[3 * k + a] = fnd[k] ? (double)o[6 + a] : 0.0;
      if (u2) u2[3 * k + a] = fnd[k] && two ? (double)o[9 + a] : 0.0;
    }
  }
  return BP_OK;
}

// ---------------------------------------------------------------------------
// state files: header, per species (parameters, a_c, live particle arrays,
// tile offsets, parameter index per load id), E and B, the status word

}  // extern "C"

namespace {
struct StateHeader {
  char magic[8];
  int32_t version, D, n[3], bc[3], L[3], det, nsp;
  double dx[3], dt;
  int64_t step;
};
struct StateSpecies {
  int32_t kind, loaded, has_pidx, nac, dim, pad;
  double q1, m1, q2, m2, w;
  int64_t n, cnt, pcap;
};
const char kStateMagic[8] = {'B', 'P', 'S', 'T', 'A', 'T', 'E', '1'};
constexpr int32_t kStateVersion = 2;  // 2: a CRC-32 of every preceding byte ends the file

// CRC-32 of the IEEE 802.3 / zlib convention (reflected polynomial
// 0xEDB88320, initial value and final xor 0xFFFFFFFF), table-driven eight
// bytes at a time ("slicing by 8": table k gives the CRC contribution of a
// byte followed by k zero bytes).  Portable C++: the same result on any host.
struct Crc32 {
  uint32_t t[8][256];
  Crc32() {
    for (uint32_t b = 0; b < 256; ++b) {
      uint32_t c = b;
      for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
      t[0][b] = c;
    }
    for (uint32_t b = 0; b < 256; ++b)
      for (int k = 1; k < 8; ++k) t[k][b] = (t[k - 1][b] >> 8) ^ t[0][t[k - 1][b] & 0xFFu];
  }
  // continue a running CRC (pass the previous return value; start from 0)
  uint32_t update(uint32_t crc, const void *data, size_t n) const {
    const unsigned char *p = static_cast<const unsigned char *>(data);
    uint32_t c = ~crc;
    while (n >= 8) {
      const uint32_t lo = c ^ ((uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24));
      c = t[7][lo & 0xFFu] ^ t[6][(lo >> 8) & 0xFFu] ^ t[5][(lo >> 16) & 0xFFu] ^ t[4][lo >> 24] ^ t[3][p[4]] ^
          t[2][p[5]] ^ t[1][p[6]] ^ t[0][p[7]];
      p += 8;
      n -= 8;
    }
    while (n--) c = t[0][(c ^ *p++) & 0xFFu] ^ (c >> 8);
    return ~c;
  }
};
const Crc32 &crc32_tables() {
  static const Crc32 T;
  return T;
}

// the running CRC of what bp_save has written so far
thread_local uint32_t g_wr_crc = 0;
bool wr(FILE *f, const void *p, size_t bytes) {
  if (bytes == 0) return true;
  g_wr_crc = crc32_tables().update(g_wr_crc, p, bytes);
  return fwrite(p, 1, bytes, f) == bytes;
}
bool rd(FILE *f, void *p, size_t bytes) { return bytes == 0 || fread(p, 1, bytes, f) == bytes; }
bool wr_dev(FILE *f, const void *dev, size_t bytes) {
  std::vector<char> h(bytes);
  if (bytes && cudaMemcpy(h.data(), dev, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
  return wr(f, h.data(), bytes);
}

// Whether the file ends with the CRC-32 of everything before it: read once,
// in chunks, before anything is loaded, so that a truncated or corrupted file
// leaves the context untouched.
bool state_crc_ok(FILE *f) {
  if (fseek(f, 0, SEEK_END) != 0) return false;
  const long long size = ftell(f);
  if (size < (long long)sizeof(StateHeader) + 4 || fseek(f, 0, SEEK_SET) != 0) return false;
  long long left = size - 4;
  std::vector<unsigned char> buf(1 << 22);
  uint32_t crc = 0;
  while (left > 0) {
    const size_t k = (size_t)std::min<long long>(left, (long long)buf.size());
    if (fread(buf.data(), 1, k, f) != k) return false;
    crc = crc32_tables().update(crc, buf.data(), k);
    left -= (long long)k;
  }
  unsigned char tail[4];
  if (fread(tail, 1, 4, f) != 4) return false;
  const uint32_t want = (uint32_t)tail[0] | ((uint32_t)tail[1] << 8) | ((uint32_t)tail[2] << 16) | ((uint32_t)tail[3] << 24);
  return want == crc && fseek(f, 0, SEEK_SET) == 0;
}
bool rd_dev(FILE *f, void *dev, size_t bytes) {
  std::vector<char> h(bytes);
  if (!rd(f, h.data(), bytes)) return false;
  return bytes == 0 || cudaMemcpy(dev, h.data(), bytes, cudaMemcpyHostToDevice) == cudaSuccess;
}
}  // namespace

extern "C" {

int bp_save(bp_ctx *c, const char *path) {
  if (!c || !path) return BP_ERR_ARG;
  const GridP &g = c->g;
  cudaError_t e0 = cudaStreamSynchronize(c->stream);
  if (e0 != cudaSuccess) return cuda_fail(c, e0, "save");
  FILE *f = fopen(path, "wb");
  if (!f) return fail(c, BP_ERR_IO, "bp_save: cannot open %s", path);
  StateHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, kStateMagic, 8);
  h.version = kStateVersion;
  g_wr_crc = 0;
  h.D = g.D;
  h.det = c->det;
  h.nsp = (int)c->sp.size();
  for (int a = 0; a < 3; ++a) {
    h.n[a] = g.n[a];
    h.bc[a] = g.bc[a];
    h.L[a] = g.L[a];
    h.dx[a] = g.dxd[a];
  }
  h.dt = g.dtd;
  h.step = c->step;
  bool ok = wr(f, &h, sizeof h);
  const int D = g.D;
  for (auto &s : c->sp) {
    StateSpecies q;
    memset(&q, 0, sizeof q);
    q.kind = s.sp.kind;
    q.loaded = s.loaded;
    q.has_pidx = s.has_pidx;
    q.nac = s.sp.nac;
    q.dim = D;
    q.q1 = s.sp.q1d;
    q.m1 = s.sp.m1d;
    q.q2 = s.sp.q2d;
    q.m2 = s.sp.m2d;
    q.w = s.sp.wd;
    q.n = s.n;
    q.pcap = s.p.cap;
    int cnt = 0;
    if (s.loaded) cudaMemcpy(&cnt, s.p.tstart + g.ntiles, sizeof(int), cudaMemcpyDeviceToHost);
    q.cnt = cnt;
    ok = ok && wr(f, &q, sizeof q);
    if (s.sp.nac > 0 && s.ac_dev) ok = ok && wr_dev(f, s.ac_dev, sizeof(float) * s.sp.nac);
    if (!s.loaded) continue;
    const bool two = s.sp.kind == BP_TWO_BODY;
    const long long pc = s.p.cap;
    ok = ok && wr_dev(f, s.p.cell, sizeof(int) * cnt) && wr_dev(f, s.p.id, sizeof(int) * cnt);
    for (int a = 0; a < D; ++a) ok = ok && wr_dev(f, s.p.off + a * pc, sizeof(float) * cnt);
    for (int a = 0; a < 3; ++a) ok = ok && wr_dev(f, s.p.u1 + a * pc, sizeof(float) * cnt);
    if (two)
      for (int a = 0; a < 3; ++a)
        ok = ok && wr_dev(f, s.p.r + a * pc, sizeof(float) * cnt) && wr_dev(f, s.p.u2 + a * pc, sizeof(float) * cnt);
    if (s.p.pidx) ok = ok && wr_dev(f, s.p.pidx, sizeof(int) * cnt);
    ok = ok && wr_dev(f, s.p.tstart, sizeof(int) * (g.ntiles + 1));
    if (!s.pidx_host.empty()) {
      ok = ok && wr(f, s.pidx_host.data(), sizeof(int) * s.pidx_host.size());
    } else {
      // no parameter indices: n zeros (the file holds one index per particle)
      const std::vector<int> zeros(1 << 16, 0);
      for (long long q = 0; ok && q < s.n; q += (long long)zeros.size())
        ok = wr(f, zeros.data(), sizeof(int) * (size_t)std::min<long long>((long long)zeros.size(), s.n - q));
    }
  }
  for (int k = 0; k < 6; ++k) ok = ok && wr_dev(f, c->F[k], sizeof(float) * g.ncell);
  ok = ok && wr_dev(f, c->status, sizeof(int));
  // the checksum of every byte above, little-endian
  const uint32_t crc = g_wr_crc;
  const unsigned char tail[4] = {(unsigned char)(crc & 0xFFu), (unsigned char)((crc >> 8) & 0xFFu),
                                 (unsigned char)((crc >> 16) & 0xFFu), (unsigned char)(crc >> 24)};
  ok = ok && fwrite(tail, 1, 4, f) == 4;
  ok = (fclose(f) == 0) && ok;
  return ok ? BP_OK : fail(c, BP_ERR_IO, "bp_save: write to %s failed", path);
}

int bp_load(bp_ctx *c, const char *path) {
  if (!c || !path) return BP_ERR_ARG;
  const GridP &g = c->g;
  cudaError_t e0 = cudaStreamSynchronize(c->stream);
  if (e0 != cudaSuccess) return cuda_fail(c, e0, "load");
  FILE *f = fopen(path, "rb");
  if (!f) return fail(c, BP_ERR_IO, "bp_load: cannot open %s", path);
  auto bad = [&](int code, const char *why) {
    fclose(f);
    return fail(c, code, "bp_load: %s (%s)", why, path);
  };
  StateHeader h;
  if (!rd(f, &h, sizeof h) || memcmp(h.magic, kStateMagic, 8) != 0 || h.version != kStateVersion)
    return bad(BP_ERR_IO, "not a state file of this library");
  if (!state_crc_ok(f)) return bad(BP_ERR_IO, "checksum mismatch: the file is truncated or corrupted");
  if (!rd(f, &h, sizeof h)) return bad(BP_ERR_IO, "unreadable header");
  bool same = h.D == g.D && h.det == c->det && h.nsp == (int)c->sp.size() && h.dt == g.dtd;
  for (int a = 0; a < 3; ++a)
    same = same && h.n[a] == g.n[a] && h.bc[a] == g.bc[a] && h.L[a] == g.L[a] && h.dx[a] == g.dxd[a];
  if (!same) return bad(BP_ERR_ARG, "grid, deposit mode or species count differ from the context's");
  const int D = g.D;
  for (auto &s : c->sp) {
    StateSpecies q;
    if (!rd(f, &q, sizeof q)) return bad(BP_ERR_IO, "truncated species record");
    if (q.kind != s.sp.kind || q.nac != s.sp.nac || q.dim != D || q.q1 != s.sp.q1d || q.m1 != s.sp.m1d ||
        q.q2 != s.sp.q2d || q.m2 != s.sp.m2d || q.w != s.sp.wd)
      return bad(BP_ERR_ARG, "species differ from the context's");
    if (q.nac > 0 && s.ac_dev && !rd_dev(f, s.ac_dev, sizeof(float) * q.nac)) return bad(BP_ERR_IO, "a_c");
    if (!q.loaded) continue;
    if (s.loaded) return bad(BP_ERR_STATE, "a species of the context is already loaded (bp_reset first)");
    if (q.cnt < 0 || q.n < 0 || q.cnt > q.pcap) return bad(BP_ERR_IO, "bad particle counts");
    const bool two = s.sp.kind == BP_TWO_BODY;
    if (alloc_particles(c, s, std::max<long long>(q.pcap, 1), q.has_pidx != 0)) {
      fclose(f);
      return BP_ERR_OOM;
    }
    const long long pc = s.p.cap, cnt = q.cnt;
    bool ok = rd_dev(f, s.p.cell, sizeof(int) * cnt) && rd_dev(f, s.p.id, sizeof(int) * cnt);
    for (int a = 0; a < D; ++a) ok = ok && rd_dev(f, s.p.off + a * pc, sizeof(float) * cnt);
    for (int a = 0; a < 3; ++a) ok = ok && rd_dev(f, s.p.u1 + a * pc, sizeof(float) * cnt);
    if (two)
      for (int a = 0; a < 3; ++a)
        ok = ok && rd_dev(f, s.p.r + a * pc, sizeof(float) * cnt) && rd_dev(f, s.p.u2 + a * pc, sizeof(float) * cnt);
    if (q.has_pidx) ok = ok && rd_dev(f, s.p.pidx, sizeof(int) * cnt);
    ok = ok && rd_dev(f, s.p.tstart, sizeof(int) * (g.ntiles + 1));
    s.pidx_host.assign((size_t)q.n, 0);
    ok = ok && rd(f, s.pidx_host.data(), sizeof(int) * (size_t)q.n);
    if (!q.has_pidx) s.pidx_host.clear();  // all 0
    if (!ok) return bad(BP_ERR_IO, "truncated particle arrays");
    s.n = q.n;
    s.has_pidx = q.has_pidx != 0;
    s.loaded = true;
  }
  bool ok = true;
  for (int k = 0; k < 6; ++k) ok = ok && rd_dev(f, c->F[k], sizeof(float) * g.ncell);
  ok = ok && rd_dev(f, c->status, sizeof(int));
  fclose(f);
  if (!ok) return fail(c, BP_ERR_IO, "bp_load: truncated fields (%s)", path);
  for (int k = 6; k < 9; ++k) cudaMemset(c->F[k], 0, sizeof(float) * g.ncell);
  if (c->jfx) cudaMemset(c->jfx, 0, sizeof(unsigned long long) * 3 * (size_t)g.ncell);
  refresh_marks(c);
  c->step = h.step;
  c->sort_dirty = true;
  update_jscale(c);
  cudaError_t e = cudaDeviceSynchronize();
  return e == cudaSuccess ? BP_OK : cuda_fail(c, e, "load");
}

int bp_residual(bp_ctx *c, double *dst, int on_device) {
  if (!c || !dst) return BP_ERR_ARG;
  const GridP &g = c->g;
  double *R = on_device ? dst : c->rho;
  if (!R) {
    c->rho = (double *)dalloc(c, sizeof(double) * g.ncell);
    if (!c->rho) return fail(c, BP_ERR_OOM, "residual scratch");
    R = c->rho;
  }
  cudaMemsetAsync(R, 0, sizeof(double) * g.ncell, c->stream);
  for (auto &s : c->sp)
    if (s.loaded) {
      launch_rho(g, s.sp, s.p, R, c->stream);
      c->launches++;
    }
  const float *E[3] = {c->F[0], c->F[1], c->F[2]};
  launch_divE_minus(g, E, R, c->stream);
  c->launches++;
  int rc = check_launch(c, "residual");
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  if (!on_device) e = cudaMemcpyAsync(dst, R, sizeof(double) * g.ncell, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? BP_OK : cuda_fail(c, e, "residual");
}

int64_t bp_kernel_launches(const bp_ctx *c) {
  if (!c) return 0;
  // re-sorts run inside the step graph are counted on the device
  const long long runs = c->sort_runs ? *(volatile int *)c->sort_runs : 0;
  return c->launches + runs * ((long long)c->sort_nsp * sort_launches() + 1);
}

int bp_set_record_capacity(bp_ctx *c, int64_t n) {
  if (!c || n < 0 || !c->det) return BP_ERR_ARG;
  cudaStreamSynchronize(c->stream);
  c->grec_fixed = std::min<long long>(n, 1LL << 30);
  ensure_records(c);
  return (c->grec || c->sp.empty()) ? BP_OK : fail(c, BP_ERR_OOM, "record buffer");
}

int bp_time_push(bp_ctx *c, int enable) {
  if (!c) return BP_ERR_ARG;
  cudaStreamSynchronize(c->stream);
  c->timing = enable != 0;
  c->ev_used = 0;
  c->push_ms = 0.0;
  c->push_launches = 0;
  cudaError_t e = cudaMemsetAsync(c->work, 0, sizeof(unsigned long long) * 2, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? BP_OK : cuda_fail(c, e, "time push");
}

int bp_push_work(bp_ctx *c, int64_t *full, int64_t *quiet) {
  if (!c) return BP_ERR_ARG;
  unsigned long long w[2] = {0, 0};
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaMemcpy(w, c->work, sizeof w, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "push work");
  if (full) *full = (int64_t)w[0];
  if (quiet) *quiet = (int64_t)w[1];
  return BP_OK;
}

int bp_field_work(bp_ctx *c, int64_t *active_tiles, int64_t *steps) {
  if (!c) return BP_ERR_ARG;
  unsigned long long w[2] = {0, 0};
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess && c->act_n) e = cudaMemcpy(w, c->act_n, sizeof w, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && c->act_n) e = cudaMemset(c->act_n, 0, sizeof w);
  if (e != cudaSuccess) return cuda_fail(c, e, "field work");
  if (active_tiles) *active_tiles = (int64_t)w[0];
  if (steps) *steps = (int64_t)w[1];
  return BP_OK;
}

int bp_push_time(bp_ctx *c, double *ms, int64_t *launches) {
  if (!c) return BP_ERR_ARG;
  if (ms) *ms = c->push_ms;
  if (launches) *launches = c->push_launches;
  return BP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// reset, parameters, checkpointed forward and the discrete adjoint

extern "C" {

int bp_reset(bp_ctx *c) {
  if (!c) return BP_ERR_ARG;
  cudaStream_t st = c->stream;
  for (int k = 0; k < 9; ++k) cudaMemsetAsync(c->F[k], 0, sizeof(float) * c->g.ncell, st);
  cudaMemsetAsync(c->g.fnz, 0, (size_t)c->g.ntiles, st);
  if (c->act) cudaMemsetAsync(c->act, 1, (size_t)c->g.ntiles, st);
  if (c->jfx) cudaMemsetAsync(c->jfx, 0, sizeof(unsigned long long) * 3 * (size_t)c->g.ncell, st);
  cudaMemsetAsync(c->status, 0, sizeof(int) * 4, st);
  c->step = 0;
  for (auto &p : c->pr) p.count = 0;
  for (auto &s : c->sp) s.loaded = false;
  c->adj.ready = false;
  cudaError_t e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? BP_OK : cuda_fail(c, e, "reset");
}

int bp_set_omega(bp_ctx *c, int sid, const double *omega_b, int n) {
  if (!c || sid < 0 || sid >= (int)c->sp.size() || !omega_b) return BP_ERR_ARG;
  Species &s = c->sp[sid];
  if (s.sp.kind != BP_TWO_BODY || n != s.sp.nac) return fail(c, BP_ERR_ARG, "bp_set_omega: %d values for %d", n, s.sp.nac);
  const double mr = s.sp.m1d * s.sp.m2d / (s.sp.m1d + s.sp.m2d);
  std::vector<float> ac(n);
  for (int i = 0; i < n; ++i) {
    double w = omega_b[i];
    if (!(w > 0)) return fail(c, BP_ERR_ARG, "omega_b must be positive");
    if (w * c->g.dtd >= 2.0) return fail(c, BP_ERR_CFL, "omega_b dt = %g >= 2", w * c->g.dtd);
    ac[i] = (float)std::cbrt(std::fabs(s.sp.q1d * s.sp.q2d) * (double)s.sp.kappa / (mr * w * w));
    s.omega[i] = w;
  }
  cudaMemcpyAsync(s.ac_dev, ac.data(), sizeof(float) * n, cudaMemcpyHostToDevice, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? BP_OK : cuda_fail(c, e, "set omega");
}

int bp_forward_ckpt(bp_ctx *c, int64_t nsteps, int K) {
  if (!c || nsteps < 1 || K < 1) return BP_ERR_ARG;
  if (!c->det) return fail(c, BP_ERR_STATE, "the adjoint needs the sorted (bit-reproducible) deposit");
  const GridP &g = c->g;
  bp_adjoint &ad = c->adj;
  const int nseg = (int)((nsteps + K - 1) / K);
  // checkpoint storage (reused when it is large enough)
  bool caps_ok = !ad.ck_parts.empty() && ad.ck_parts[0].size() == c->sp.size();
  for (size_t q = 0; caps_ok && q < c->sp.size(); ++q)
    caps_ok = ad.ck_parts[0][q].p.cap == c->sp[q].p.cap && (ad.ck_parts[0][q].p.pidx != nullptr) == (c->sp[q].p.pidx != nullptr);
  if (ad.K != K || ad.nseg < nseg || !caps_ok) {
    for (float *p : ad.ck_fields) dfree(c, p);
    for (float *p : ad.st_fields) dfree(c, p);
    for (auto &v : ad.ck_parts)
      for (auto &q : v) {
        void *a[] = {q.p.cell, q.p.off, q.p.u1, q.p.id, q.p.tstart, q.p.r, q.p.u2, q.p.pidx};
        for (void *x : a) dfree(c, x);
      }
    for (auto &v : ad.st_parts)
      for (auto &q : v) {
        void *a[] = {q.p.cell, q.p.off, q.p.u1, q.p.id, q.p.tstart, q.p.r, q.p.u2, q.p.pidx};
        for (void *x : a) dfree(c, x);
      }
    ad.ck_fields.assign(nseg, nullptr);
    ad.ck_parts.assign(nseg, std::vector<bp_part_copy>(c->sp.size()));
    ad.st_fields.assign(2 * K, nullptr);
    ad.st_parts.assign(2 * K, std::vector<bp_part_copy>(c->sp.size()));
    for (int k = 0; k < nseg; ++k) {
      ad.ck_fields[k] = (float *)dalloc(c, sizeof(float) * 6 * g.ncell);
      if (!ad.ck_fields[k]) return fail(c, BP_ERR_OOM, "checkpoint fields");
      for (size_t q = 0; q < c->sp.size(); ++q)
        if (copy_alloc(c, c->sp[q].p, g.D, c->sp[q].sp.kind == BP_TWO_BODY, ad.ck_parts[k][q].p))
          return fail(c, BP_ERR_OOM, "checkpoint particles");
    }
    for (int k = 0; k < 2 * K; ++k) {
      ad.st_fields[k] = (float *)dalloc(c, sizeof(float) * 6 * g.ncell);
      if (!ad.st_fields[k]) return fail(c, BP_ERR_OOM, "step store fields");
      for (size_t q = 0; q < c->sp.size(); ++q)
        if (copy_alloc(c, c->sp[q].p, g.D, c->sp[q].sp.kind == BP_TWO_BODY, ad.st_parts[k][q].p))
          return fail(c, BP_ERR_OOM, "step store particles");
    }
    dfree(c, ad.ck_status);
    ad.ck_status = (int *)dalloc(c, sizeof(int) * 4 * nseg);
    if (!ad.ck_status) return fail(c, BP_ERR_OOM, "checkpoint status");
    ad.K = K;
    ad.nseg = nseg;
  }
  for (auto &s : c->sp)
    if (!s.loaded) return fail(c, BP_ERR_STATE, "every species must be loaded before bp_forward_ckpt");
  ad.start = c->step;
  ad.nsteps = nsteps;
  ad.probe_c0.clear();
  for (auto &p : c->pr) ad.probe_c0.push_back(p.count);
  int nsp = 0;
  PushArgs A = push_args(c, &nsp);
  cudaStream_t st = c->stream;
  sync_clock(c, st);
  const bool graph = !c->timing && step_graph(c, A);
  for (int k = 0; k < nseg; ++k) {
    // the state before step start + k K: E, B^{n-1/2}, particles
    CopyList L;
    for (int f = 0; f < 6; ++f) cl_add(c, L, c->F[f], ad.ck_fields[k] + (size_t)f * g.ncell, sizeof(float) * g.ncell);
    for (size_t q = 0; q < c->sp.size(); ++q)
      cl_parts(c, L, c->sp[q].p, ad.ck_parts[k][q].p, g.D, c->sp[q].sp.kind == BP_TWO_BODY);
    cl_add(c, L, c->status, ad.ck_status + 4 * k, sizeof(int) * 4);
    cl_flush(c, L);
    long long len = std::min<long long>(K, nsteps - (long long)k * K);
    for (long long j = 0; j < len; ++j) {
      int rc = graph ? graph_step(c, nsp) : one_step(c, A, nsp, true, nullptr, nullptr);
      if (rc) return rc;
    }
  }
  ad.ready = true;
  return BP_OK;
}

int bp_backward(bp_ctx *c, int probe_id, const float *dl_dprobe, int sid, double *grad_omega, const int32_t *group,
                int64_t n_groups, double *grad_group) {
  if (!c || probe_id < 0 || probe_id >= (int)c->pr.size() || !dl_dprobe || sid < 0 || sid >= (int)c->sp.size())
    return BP_ERR_ARG;
  bp_adjoint &ad = c->adj;
  if (!ad.ready) return fail(c, BP_ERR_STATE, "bp_backward needs a preceding bp_forward_ckpt");
  const GridP &g = c->g;
  cudaStream_t st = c->stream;
  Probe &P = c->pr[probe_id];
  if (P.comp > 2) return fail(c, BP_ERR_ARG, "bp_backward: the loss probe must record an E component");
  const long long c0 = ad.probe_c0[probe_id];
  const long long nrec = std::min<long long>(ad.nsteps, P.cap - c0);
  if (adj_prepare(g.D, &ad.push_blocks, &ad.scat_blocks)) return fail(c, BP_ERR_CUDA, "adjoint kernel set-up");
  // buffers
  if (!ad.lamE[0]) {
    for (int k = 0; k < 3; ++k) {
      ad.lamE[k] = (float *)dalloc(c, sizeof(float) * g.ncell);
      ad.lamB[k] = (float *)dalloc(c, sizeof(float) * g.ncell);
      ad.lamJ[k] = (float *)dalloc(c, sizeof(float) * g.ncell);
      ad.H[k] = (float *)dalloc(c, sizeof(float) * g.ncell);
      if (!ad.lamE[k] || !ad.lamB[k] || !ad.lamJ[k] || !ad.H[k]) return fail(c, BP_ERR_OOM, "adjoint fields");
    }
    ad.lfx = (unsigned long long *)dalloc(c, sizeof(unsigned long long) * 6 * (size_t)g.ncell);
    ad.dirty = (unsigned char *)dalloc(c, g.ntiles);
    ad.emax = (unsigned *)dalloc(c, sizeof(unsigned));
    ad.status = (int *)dalloc(c, sizeof(int));
    ad.kst = (int *)dalloc(c, sizeof(int));
    ad.nwork = (int *)dalloc(c, sizeof(int));
    if (!ad.lfx || !ad.dirty || !ad.emax || !ad.status || !ad.kst || !ad.nwork)
      return fail(c, BP_ERR_OOM, "adjoint accumulators");
  }
  // work items: every tile and species contributes at most one partial chunk
  long long want_work = 0;
  for (auto &s : c->sp) want_work += (s.p.cap + kAdjChunk - 1) / kAdjChunk + g.ntiles;
  if (want_work > INT32_MAX) return fail(c, BP_ERR_ARG, "bp_backward: too many particles for the work list");
  if (ad.work_cap < want_work) {
    dfree(c, ad.work);
    ad.work = (int4 *)dalloc(c, sizeof(int4) * (size_t)want_work);
    if (!ad.work) return fail(c, BP_ERR_OOM, "adjoint work list");
    ad.work_cap = want_work;
  }
  bool xb_ok = ad.xb.size() == c->sp.size() && ad.xb_cap.size() == c->sp.size();
  for (size_t q = 0; xb_ok && q < c->sp.size(); ++q) xb_ok = ad.xb_cap[q] == c->sp[q].p.cap;
  if (!xb_ok) {
    for (auto p : ad.xb) dfree(c, p);
    for (auto p : ad.acb) dfree(c, p);
    for (auto p : ad.eb) dfree(c, p);
    ad.xb.assign(c->sp.size(), nullptr);
    ad.acb.assign(c->sp.size(), nullptr);
    ad.eb.assign(c->sp.size(), nullptr);
    ad.xb_cap.assign(c->sp.size(), 0);
    for (size_t q = 0; q < c->sp.size(); ++q) {
      ad.xb[q] = (float *)dalloc(c, sizeof(float) * 12 * c->sp[q].p.cap);
      ad.acb[q] = (double *)dalloc(c, sizeof(double) * c->sp[q].p.cap);
      ad.eb[q] = (float *)dalloc(c, sizeof(float) * 12 * c->sp[q].p.cap);
      if (!ad.xb[q] || !ad.acb[q] || !ad.eb[q]) return fail(c, BP_ERR_OOM, "particle adjoints");
      ad.xb_cap[q] = c->sp[q].p.cap;
    }
  }
  long long need = std::max<long long>(1, nrec * P.npts);
  if (ad.dl_len < need) {
    dfree(c, ad.dl);
    ad.dl = (float *)dalloc(c, sizeof(float) * need);
    if (!ad.dl) return fail(c, BP_ERR_OOM, "probe gradient");
    ad.dl_len = need;
  }
  if (nrec > 0) cudaMemcpyAsync(ad.dl, dl_dprobe, sizeof(float) * nrec * P.npts, cudaMemcpyHostToDevice, st);
  for (int k = 0; k < 3; ++k) {
    cudaMemsetAsync(ad.lamE[k], 0, sizeof(float) * g.ncell, st);
    cudaMemsetAsync(ad.lamB[k], 0, sizeof(float) * g.ncell, st);
    cudaMemsetAsync(ad.H[k], 0, sizeof(float) * g.ncell, st);
  }
  cudaMemsetAsync(ad.emax, 0, sizeof(unsigned), st);
  cudaMemsetAsync(ad.status, 0, sizeof(int), st);
  cudaMemsetAsync(ad.nwork, 0, sizeof(int), st);
  // kept clear from step to step by k_adj_fxsum; cleared here too, in case
  // an earlier backward pass stopped on an error
  cudaMemsetAsync(ad.lfx, 0, sizeof(unsigned long long) * 6 * (size_t)g.ncell, st);
  cudaMemsetAsync(ad.dirty, 0, g.ntiles, st);
  for (size_t q = 0; q < c->sp.size(); ++q) {
    cudaMemsetAsync(ad.xb[q], 0, sizeof(float) * 12 * c->sp[q].p.cap, st);
    cudaMemsetAsync(ad.acb[q], 0, sizeof(double) * c->sp[q].p.cap, st);
  }
  int nsp = 0;
  PushArgs A = push_args(c, &nsp);
  std::vector<SpecP> sps;
  std::vector<float *> xbs, ebs;
  std::vector<double *> acbs;
  std::vector<long long> caps;
  for (size_t q = 0; q < c->sp.size(); ++q) {
    sps.push_back(c->sp[q].sp);
    xbs.push_back(ad.xb[q]);
    ebs.push_back(ad.eb[q]);
    acbs.push_back(ad.acb[q]);
    caps.push_back(c->sp[q].p.cap);
  }
  // Two streams: each segment (newest first) is recomputed on the context's
  // stream into one bank of the per-step stores, and its reverse steps run on
  // the adjoint stream from that bank; the recomputation of the next
  // (earlier) segment, into the other bank, overlaps them.  A bank is
  // recomputed again only after the reverse steps that read it are done.
  if (!ad.stream) {
    if (cudaStreamCreateWithFlags(&ad.stream, cudaStreamNonBlocking) != cudaSuccess) {
      ad.stream = nullptr;
      return cuda_fail(c, cudaGetLastError(), "adjoint stream");
    }
    for (int k = 0; k < 2; ++k) {
      cudaEventCreateWithFlags(&ad.rec_done[k], cudaEventDisableTiming);
      cudaEventCreateWithFlags(&ad.rev_done[k], cudaEventDisableTiming);
    }
  }
  cudaStream_t as = ad.stream;
  const int K = ad.K;
  const AdjBufs bufs{ad.lfx, ad.dirty, ad.kst, ad.emax, ad.nwork, ad.work, (int)ad.work_cap, kAdjChunk,
                     ad.push_blocks, ad.scat_blocks};
  auto recompute = [&](int seg) -> int {
    const int bank = seg & 1;
    // the reverse steps of segment seg + 2 read this bank
    if (seg + 2 <= ad.nseg - 1) cudaStreamWaitEvent(st, ad.rev_done[bank], 0);
    // restore the checkpoint and recompute the segment, storing each step
    CopyList L;
    for (int f = 0; f < 6; ++f) cl_add(c, L, ad.ck_fields[seg] + (size_t)f * g.ncell, c->F[f], sizeof(float) * g.ncell);
    for (size_t q = 0; q < c->sp.size(); ++q)
      cl_parts(c, L, ad.ck_parts[seg][q].p, c->sp[q].p, g.D, c->sp[q].sp.kind == BP_TWO_BODY);
    cl_add(c, L, ad.ck_status + 4 * seg, c->status, sizeof(int) * 4);
    cl_flush(c, L);
    refresh_marks(c);
    const long long base = (long long)seg * K;
    const long long len = std::min<long long>(K, ad.nsteps - base);
    c->step = ad.start + base;
    sync_clock(c, st);
    for (long long j = 0; j < len; ++j) {
      int rc = one_step(c, A, nsp, false, ad.st_fields[bank * K + j], &ad.st_parts[bank * K + j]);
      if (rc) return rc;
    }
    cudaEventRecord(ad.rec_done[bank], st);
    return BP_OK;
  };
  auto reverse = [&](int seg) -> int {
    const int bank = seg & 1;
    cudaStreamWaitEvent(as, ad.rec_done[bank], 0);
    const long long base = (long long)seg * K;
    const long long len = std::min<long long>(K, ad.nsteps - base);
    for (long long j = len - 1; j >= 0; --j) {
      const long long n = base + j;  // step n maps state n to n + 1
      // loss on the probe sample recorded after step n
      if (n < nrec) {
        launch_adj_inject(ad.lamE[P.comp], P.nodes, P.npts, ad.dl + n * P.npts, as);
        c->launches++;
      }
      // E update with Mur faces, transposed (H is clear: zeroed before the
      // first reverse step, then by the previous step's B transpose)
      launch_adj_e(g, ad.lamE, ad.H, ad.lamB, ad.lamJ, as);
      for (int k = 0; k < 3; ++k) std::swap(ad.lamE[k], ad.H[k]);
      // B^{n+1/2} = B^n - dt/2 curl E^n; clears H (the old E adjoint) for the next step
      launch_adj_b(g, ad.lamE, ad.lamB, 0.5f * g.dt, ad.H, as);
      // particles, with E^n, B^n and the particle state stored for step n
      const float *En[3], *Bn[3], *lJ[3] = {ad.lamJ[0], ad.lamJ[1], ad.lamJ[2]};
      const float *sf = ad.st_fields[bank * K + j];
      for (int k = 0; k < 3; ++k) {
        En[k] = sf + (size_t)k * g.ncell;
        Bn[k] = sf + (size_t)(3 + k) * g.ncell;
      }
      std::vector<PartP> pp;
      for (size_t q = 0; q < c->sp.size(); ++q) pp.push_back(ad.st_parts[bank * K + j][q].p);
      launch_adj_push(g, (int)c->sp.size(), sps.data(), pp.data(), xbs.data(), acbs.data(), ebs.data(), caps.data(), En,
                      Bn, lJ, bufs, ad.lamE, ad.lamB, ad.status, as);
      // B^n = B^{n-1/2} - dt/2 curl E^n
      launch_adj_b(g, ad.lamE, ad.lamB, 0.5f * g.dt, nullptr, as);
      // E transpose and its Mur passes (one per pass and open axis), two B
      // transposes, work list, particle adjoint, scatter, fixed-point sum
      int nopen = 0;
      for (int a = 0; a < g.D; ++a) nopen += g.bc[a] == BP_OPEN;
      c->launches += 1 + nopen * nopen + 2 + 4;
      int rc = check_launch(c, "backward step");
      if (rc) return rc;
    }
    cudaEventRecord(ad.rev_done[bank], as);
    return BP_OK;
  };
  {
    int rc = recompute(ad.nseg - 1);
    for (int seg = ad.nseg - 1; !rc && seg >= 0; --seg) {
      if (seg >= 1) rc = recompute(seg - 1);
      if (!rc) rc = reverse(seg);
    }
    if (rc) {
      cudaStreamSynchronize(as);
      return rc;
    }
    // the reductions below read the adjoint stream's results
    cudaStreamWaitEvent(st, ad.rev_done[0], 0);
    int ast = 0;
    cudaError_t e = cudaMemcpyAsync(&ast, ad.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "backward");
    if (ast & ST_DOMAIN)
      return fail(c, BP_ERR_DOMAIN, "bp_backward: a bound electron a cell or more from its nucleus (not followed by the reverse pass)");
  }
  // FP64 reductions in a fixed order: parameters and groups (CSR over load order)
  Species &S = c->sp[sid];
  const long long n = S.n;
  std::vector<int> ptr, ids;
  auto build_csr = [&](const int32_t *key, long long nrows) {
    ptr.assign(nrows + 1, 0);
    for (long long i = 0; i < n; ++i) ptr[key[i] + 1]++;
    for (long long r = 0; r < nrows; ++r) ptr[r + 1] += ptr[r];
    ids.assign(n, 0);
    std::vector<int> cur(ptr.begin(), ptr.end() - 1);
    for (long long i = 0; i < n; ++i) ids[cur[key[i]]++] = (int)i;
  };
  int *dptr = nullptr, *dids = nullptr;
  double *dout = nullptr, *dscale = nullptr;
  const long long nrow_max = std::max<long long>(S.sp.nac, n_groups) + 1;
  dptr = (int *)dalloc(c, sizeof(int) * (nrow_max + 1));
  dids = (int *)dalloc(c, sizeof(int) * std::max<long long>(1, n));
  dout = (double *)dalloc(c, sizeof(double) * nrow_max * 3);
  dscale = (double *)dalloc(c, sizeof(double) * nrow_max);
  if (!dptr || !dids || !dout || !dscale) return fail(c, BP_ERR_OOM, "reduction buffers");
  int rc = BP_OK;
  if (grad_omega && S.sp.kind == BP_TWO_BODY) {
    std::vector<int> zeros;
    if (S.pidx_host.empty()) zeros.assign((size_t)n, 0);  // no parameter indices: all 0
    const int *key = S.pidx_host.empty() ? zeros.data() : S.pidx_host.data();
    for (long long i = 0; i < n; ++i)
      if (key[i] < 0 || key[i] >= S.sp.nac) rc = BP_ERR_STATE;
    if (!rc) {
      build_csr(key, S.sp.nac);
      // a_c = (|q1 q2| kappa / (m_r w^2))^{1/3}: d a_c / d w = -2 a_c / (3 w)
      std::vector<double> scale(S.sp.nac);
      const double mr = S.sp.m1d * S.sp.m2d / (S.sp.m1d + S.sp.m2d);
      for (int p = 0; p < S.sp.nac; ++p) {
        double w = S.omega[p];
        double ac = std::cbrt(std::fabs(S.sp.q1d * S.sp.q2d) * (double)S.sp.kappa / (mr * w * w));
        scale[p] = -2.0 * ac / (3.0 * w);
      }
      cudaMemcpyAsync(dptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(dids, ids.data(), sizeof(int) * std::max<long long>(1, n), cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(dscale, scale.data(), sizeof(double) * scale.size(), cudaMemcpyHostToDevice, st);
      launch_csr_sum(dptr, dids, S.sp.nac, ad.xb[sid], S.p.cap, 1, ad.acb[sid], dscale, dout, st);
      cudaMemcpyAsync(grad_omega, dout, sizeof(double) * S.sp.nac, cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
    }
  }
  if (!rc && grad_group && group && n_groups > 0) {
    for (long long i = 0; i < n; ++i)
      if (group[i] < 0 || group[i] >= n_groups) rc = BP_ERR_ARG;
    if (!rc) {
      build_csr(group, n_groups);
      cudaMemcpyAsync(dptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(dids, ids.data(), sizeof(int) * std::max<long long>(1, n), cudaMemcpyHostToDevice, st);
      launch_csr_sum(dptr, dids, (int)n_groups, ad.xb[sid], S.p.cap, g.D, nullptr, nullptr, dout, st);
      cudaMemcpyAsync(grad_group, dout, sizeof(double) * n_groups * g.D, cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
    }
  }
  cudaError_t e = cudaStreamSynchronize(st);
  dfree(c, dptr);
  dfree(c, dids);
  dfree(c, dout);
  dfree(c, dscale);
  if (e != cudaSuccess) return cuda_fail(c, e, "backward");
  if (rc) return fail(c, rc, "bp_backward: bad parameter or group index");
  c->launches += 2;
  return BP_OK;
}

}  // extern "C"
