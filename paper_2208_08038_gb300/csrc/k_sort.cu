// k_sort.cu -- integer work: the counting sort of particles by tile-major cell
// (key = tile * cells_per_tile + cell within tile), run only when the device
// status word says a particle left its tile's margin; the seeded device-side
// medium generator; and the FP64 Gauss-law residual.
#include "bp_internal.cuh"

namespace {

constexpr int SCAN_BS = 1024;
constexpr int SCAN_PER = 4;                 // elements per thread
constexpr int SCAN_TILE = SCAN_BS * SCAN_PER;

// blocks for n items; the kernels launched with it are grid-stride loops, so
// the cap (two waves of 256-thread blocks on 152 SMs) only bounds the grid
int blocks_for(long long n, int bs, long long cap = 152LL * 16) {
  long long b = (n + bs - 1) / bs;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

__device__ __forceinline__ bool sorting(const int *status) { return (*(volatile const int *)status) & ST_NEED_SORT; }

__device__ __forceinline__ int sort_key(const GridP &g, int cell) {
  int cc[3];
  unpack_cell(g, cell, cc);
  const int c0 = cc[0], c1 = cc[1], c2 = cc[2];
  int t = c0 / g.L[0] + g.nt[0] * (c1 / g.L[1] + g.nt[1] * (c2 / g.L[2]));
  int l = c0 % g.L[0] + g.L[0] * (c1 % g.L[1] + g.L[1] * (c2 % g.L[2]));
  return t * g.cpt + l;
}

__global__ void k_zero_if(int *a, long long n, const int *status) {
  if (!sorting(status)) return;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    a[q] = 0;
}

__global__ void k_save_count(const int *src, int *dst, const int *status) {
  if (!sorting(status)) return;
  *dst = *src;
}

__global__ void k_count(GridP g, PartP p, int *hist, const int *nold, const int *status) {
  if (!sorting(status)) return;
  const int n = *nold;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    int c = p.cell[q];
    if (c >= 0) atomicAdd(hist + sort_key(g, c), 1);
  }
}

// exclusive scan, three passes: per-block scan + block totals, scan of the
// totals in one block, add-back
__device__ __forceinline__ int block_exclusive_scan(int v, int *sh, int &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = lane < (blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;
  }
  __syncthreads();
  int base = warp ? sh[warp - 1] : 0;
  total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + x - v;
}

__global__ void __launch_bounds__(SCAN_BS) k_scan_blocks(int *a, long long n, int *bsum, const int *status) {
  if (!sorting(status)) return;
  __shared__ int sh[32];
  long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_PER;
  int v[SCAN_PER], s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    v[k] = base + k < n ? a[base + k] : 0;
    s += v[k];
  }
  int total;
  int ex = block_exclusive_scan(s, sh, total);
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    if (base + k < n) a[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_BS) k_scan_single(int *a, int n, const int *status) {
  if (!sorting(status)) return;
  __shared__ int sh[32];
  const int per = (n + SCAN_BS - 1) / SCAN_BS;
  int s = 0;
  for (int k = 0; k < per; ++k) {
    int i = threadIdx.x * per + k;
    s += i < n ? a[i] : 0;
  }
  int total;
  int ex = block_exclusive_scan(s, sh, total);
  for (int k = 0; k < per; ++k) {
    int i = threadIdx.x * per + k;
    if (i < n) {
      int v = a[i];
      a[i] = ex;
      ex += v;
    }
  }
}

__global__ void k_scan_add(int *a, long long n, const int *bsum, const int *status) {
  if (!sorting(status)) return;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    a[q] += bsum[q / SCAN_TILE];
}

// tile ranges of the sorted order; the exclusive prefix at ncell is the count
__global__ void k_tstart(GridP g, const int *hist, int *tstart, const int *status) {
  if (!sorting(status)) return;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t <= g.ntiles;
       t += (long long)gridDim.x * blockDim.x) {
    tstart[t] = hist[t * (long long)g.cpt];
  }
}

__global__ void k_scatter(GridP g, PartP p, int *off, int *tcell, float *tf, int *ti, int nf, const int *nold,
                          const int *status) {
  if (!sorting(status)) return;
  const long long cap = p.cap;
  const int n_old = *nold;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n_old;
       q += (long long)gridDim.x * blockDim.x) {
    int c = p.cell[q];
    if (c < 0) continue;
    int dst = atomicAdd(off + sort_key(g, c), 1);
    tcell[dst] = c;
    int k = 0;
    for (int a = 0; a < g.D; ++a) tf[(k++) * cap + dst] = p.off[a * cap + q];
    for (int a = 0; a < 3; ++a) tf[(k++) * cap + dst] = p.u1[a * cap + q];
    if (nf > g.D + 3) {
      for (int a = 0; a < 3; ++a) tf[(k++) * cap + dst] = p.r[a * cap + q];
      for (int a = 0; a < 3; ++a) tf[(k++) * cap + dst] = p.u2[a * cap + q];
    }
    ti[dst] = p.id[q];
    if (p.pidx) ti[cap + dst] = p.pidx[q];
  }
}

__global__ void k_copyback(GridP g, PartP p, const int *tcell, const float *tf, const int *ti, int nf,
                           const int *status) {
  if (!sorting(status)) return;
  const long long cap = p.cap;
  const int n = p.tstart[g.ntiles];
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    p.cell[q] = tcell[q];
    int k = 0;
    for (int a = 0; a < g.D; ++a, ++k) p.off[a * cap + q] = tf[k * cap + q];
    for (int a = 0; a < 3; ++a, ++k) p.u1[a * cap + q] = tf[k * cap + q];
    if (nf > g.D + 3) {
      for (int a = 0; a < 3; ++a, ++k) p.r[a * cap + q] = tf[k * cap + q];
      for (int a = 0; a < 3; ++a, ++k) p.u2[a * cap + q] = tf[k * cap + q];
    }
    p.id[q] = ti[q];
    if (p.pidx) p.pidx[q] = ti[cap + q];
  }
}

__global__ void k_clear_flag(int *status) { atomicAnd(status, ~ST_NEED_SORT); }
__global__ void k_set_flag(int *status) { atomicOr(status, ST_NEED_SORT); }

// condition of the re-sort graph: non-zero when a particle left its tile's
// margin in the previous step; counts the sorts that run
__global__ void k_sort_cond(cudaGraphConditionalHandle h, const int *status, int *runs) {
  const bool need = (*(volatile const int *)status) & ST_NEED_SORT;
  if (need) ++*runs;
  cudaGraphSetConditional(h, need ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// device medium: ion g = cell rank * ppc + p over the cell box [lo, hi);
// position x_a = (c_a + U(3g + a)) dx_a, momentum sigma N(3g + a); the
// two bodies start together (r = 0) with u1 = u2 = u_c for neutral ions and
// the non-relativistic split of p1 + p2 = p_c, q1 v1 + q2 v2 = 0 otherwise

__global__ void k_gen_medium(GridP g, SpecP sp, PartP p, int lo0, int lo1, int lo2, int e0, int e1, int ppc,
                             uint64_t kpos, uint64_t kmom, double sigma, long long first, long long count,
                             long long out0) {
  const long long cap = p.cap;
  const int lo[3] = {lo0, lo1, lo2}, ext[3] = {e0, e1, 1};
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
       q += (long long)gridDim.x * blockDim.x) {
    long long gi = first + q;
    long long rem = gi / ppc;
    int cell[3] = {0, 0, 0};
    float off[3] = {0.0f, 0.0f, 0.0f};
    for (int a = 0; a < g.D; ++a) {
      long long e = a < 2 ? ext[a] : rem + 1;
      int ca = (int)(a < g.D - 1 ? rem % e : rem) + lo[a];
      if (a < g.D - 1) rem /= e;
      double u = sm64_uniform(kpos, (uint64_t)(3 * gi + a));
      double x = ((double)ca + u) * g.dxd[a];
      double X = x / g.dxd[a];
      double fl = floor(X);
      float f = (float)(X - fl);
      int ci = (int)fl;
      if (f >= 1.0f) { f = 0.0f; ci += 1; }
      cell[a] = ci;
      off[a] = f;
    }
    double uc[3] = {0.0, 0.0, 0.0};
    if (sigma > 0) {
      for (int a = 0; a < 3; ++a) {
        uint64_t c = (uint64_t)(3 * gi + a);
        double u1 = sm64_uniform(kmom, 2 * c), u2 = sm64_uniform(kmom, 2 * c + 1);
        uc[a] = sigma * sqrt(-2.0 * log(1.0 - u1)) * cos(6.283185307179586476925 * u2);
      }
    }
    long long o = out0 + q;
    p.cell[o] = pack_cell(g, cell[0], cell[1], cell[2]);
    for (int a = 0; a < g.D; ++a) p.off[a * cap + o] = off[a];
    if (sp.kind == BP_TWO_BODY) {
      double qc = sp.q1d + sp.q2d;
      for (int a = 0; a < 3; ++a) {
        double u1, u2;
        if (qc == 0.0) {
          u1 = u2 = uc[a];
        } else {
          u1 = (sp.m1d + sp.m2d) * uc[a] / (sp.m1d - sp.m2d * sp.q1d / sp.q2d);
          u2 = -sp.q1d * u1 / sp.q2d;
        }
        p.u1[a * cap + o] = (float)u1;
        p.u2[a * cap + o] = (float)u2;
        p.r[a * cap + o] = 0.0f;
      }
    } else {
      for (int a = 0; a < 3; ++a) p.u1[a * cap + o] = (float)uc[a];
    }
    p.id[o] = (int)gi;
    if (p.pidx) p.pidx[o] = 0;
  }
}

// ---------------------------------------------------------------------------
// FP64 Gauss-law residual: rho from the stored positions (quadratic shape at
// nodes), then R = div E - rho

__global__ void k_rho(GridP g, SpecP sp, PartP p, double *rho) {
  const long long cap = p.cap;
  const int n = p.tstart[g.ntiles];
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    int cell = p.cell[q];
    if (cell < 0) continue;
    int c[3];
    unpack_cell(g, cell, c);
    const int nb = sp.kind == BP_TWO_BODY ? 2 : 1;
    for (int b = 0; b < nb; ++b) {
      double qw = (b == 0 ? sp.q1d : sp.q2d) * sp.wd;
      int base[3], cnt[3];
      double w[3][3];
      for (int a = 0; a < 3; ++a) {
        if (a >= g.D) {
          base[a] = 0;
          cnt[a] = 1;
          w[a][0] = 1.0;
          continue;
        }
        double X = (double)c[a] + (double)p.off[a * cap + q];
        if (b == 1) X -= (double)p.r[a * cap + q] / g.dxd[a];
        double nn = floor(X + 0.5);
        double xi = X - nn;
        base[a] = (int)nn - 1;
        cnt[a] = 3;
        w[a][0] = 0.5 * (0.5 - xi) * (0.5 - xi);
        w[a][1] = 0.75 - xi * xi;
        w[a][2] = 0.5 * (0.5 + xi) * (0.5 + xi);
      }
      for (int kk = 0; kk < cnt[2]; ++kk)
        for (int jj = 0; jj < cnt[1]; ++jj)
          for (int ii = 0; ii < cnt[0]; ++ii) {
            int x[3] = {base[0] + ii, base[1] + jj, base[2] + kk};
            bool ok = true;
            for (int a = 0; a < g.D; ++a) {
              if (g.bc[a] == BP_PERIODIC) x[a] = wrap_mod(x[a], g.n[a]);
              else ok &= x[a] >= 0 && x[a] < g.n[a];
            }
            if (!ok) continue;
            long long id = x[0] + (long long)g.n[0] * (x[1] + (long long)g.n[1] * x[2]);
            atomicAdd(rho + id, qw * w[0][ii] * w[1][jj] * w[2][kk]);
          }
    }
  }
}

__global__ void k_divE(GridP g, const float *Ex, const float *Ey, const float *Ez, double *R) {
  const float *E[3] = {Ex, Ey, Ez};
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.ncell;
       q += (long long)gridDim.x * blockDim.x) {
    int c[3] = {(int)(q % g.n[0]), (int)((q / g.n[0]) % g.n[1]), (int)(q / ((long long)g.n[0] * g.n[1]))};
    double div = 0.0;
    for (int a = 0; a < g.D; ++a) {
      int x[3] = {c[0], c[1], c[2]};
      x[a] -= 1;
      double lo = 0.0;
      if (g.bc[a] == BP_PERIODIC) x[a] = wrap_mod(x[a], g.n[a]);
      if (x[a] >= 0) lo = (double)E[a][x[0] + (long long)g.n[0] * (x[1] + (long long)g.n[1] * x[2])];
      div += ((double)E[a][q] - lo) / g.dxd[a];
    }
    R[q] = div - R[q];
  }
}


// ---------------------------------------------------------------------------
// load: FP64 ion positions / momenta (caller's layout, staged on the device)
// to the particle arrays.  Initial conditions of Sec. 2: both bodies at the
// ion position (r = 0); u1 = u2 = u_c for neutral ions, else the
// non-relativistic solution of p1 + p2 = p_c, q1 v1 + q2 v2 = 0.

__global__ void k_load_convert(GridP g, SpecP sp, PartP p, const double *x, const double *u, const int *pidx,
                               long long first, long long count, int *status) {
  const long long cap = p.cap;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
       q += (long long)gridDim.x * blockDim.x) {
    const long long o = first + q;
    int cell[3] = {0, 0, 0};
    bool bad = false, nonfinite = false;
    for (int a = 0; a < g.D; ++a) {
      double xa = x[q * g.D + a];
      nonfinite |= !isfinite(xa);
      double X = xa / g.dxd[a];
      double fl = floor(X);
      float f = (float)(X - fl);
      long long ci = (long long)fl;
      if (f >= 1.0f) { f = 0.0f; ci += 1; }
      if (g.bc[a] == BP_PERIODIC) {
        long long m = ci % g.n[a];
        ci = m < 0 ? m + g.n[a] : m;
      } else if (ci < 0 || ci >= g.n[a]) {
        bad = true;
        ci = 0;
      }
      cell[a] = (int)ci;
      p.off[a * cap + o] = f;
    }
    int pi = 0;
    if (pidx) {
      pi = pidx[q];
      if (pi < 0 || (sp.kind == BP_TWO_BODY && pi >= sp.nac)) { bad = true; pi = 0; }
      p.pidx[o] = pi;
    }
    for (int a = 0; a < 3; ++a) {
      double uc = u ? u[q * 3 + a] : 0.0;
      nonfinite |= !isfinite(uc);
      if (sp.kind != BP_TWO_BODY) {
        p.u1[a * cap + o] = (float)uc;
      } else {
        double u1, u2;
        if (sp.q1d + sp.q2d == 0.0) {
          u1 = u2 = uc;
        } else {
          u1 = (sp.m1d + sp.m2d) * uc / (sp.m1d - sp.m2d * sp.q1d / sp.q2d);
          u2 = -sp.q1d * u1 / sp.q2d;
        }
        p.u1[a * cap + o] = (float)u1;
        p.u2[a * cap + o] = (float)u2;
        p.r[a * cap + o] = 0.0f;
      }
    }
    p.cell[o] = (bad || nonfinite) ? -1 : pack_cell(g, cell[0], cell[1], cell[2]);
    p.id[o] = (int)o;
    if (bad) atomicOr(status, ST_DOMAIN);
    if (nonfinite) atomicOr(status, ST_NONFINITE);
  }
}

}  // namespace

void launch_sort(const GridP &g, const SpecP &sp, PartP &p, SortBufs &b, int *status, cudaStream_t s) {
  const long long nh = g.ncell + 1;
  const int nf = g.D + (sp.kind == BP_TWO_BODY ? 9 : 3);
  const int nblk = (int)((nh + SCAN_TILE - 1) / SCAN_TILE);
  int *nold = b.bsum + nblk;
  k_save_count<<<1, 1, 0, s>>>(p.tstart + g.ntiles, nold, status);
  k_zero_if<<<blocks_for(nh, 256), 256, 0, s>>>(b.hist, nh, status);
  k_count<<<blocks_for(p.cap, 256), 256, 0, s>>>(g, p, b.hist, nold, status);
  k_scan_blocks<<<nblk, SCAN_BS, 0, s>>>(b.hist, nh, b.bsum, status);
  k_scan_single<<<1, SCAN_BS, 0, s>>>(b.bsum, nblk, status);
  k_scan_add<<<blocks_for(nh, 256), 256, 0, s>>>(b.hist, nh, b.bsum, status);
  k_tstart<<<blocks_for(g.ntiles + 1, 256), 256, 0, s>>>(g, b.hist, p.tstart, status);
  k_scatter<<<blocks_for(p.cap, 256), 256, 0, s>>>(g, p, b.hist, b.tmp_cell, b.tmp_f, b.tmp_i, nf, nold, status);
  k_copyback<<<blocks_for(p.cap, 256), 256, 0, s>>>(g, p, b.tmp_cell, b.tmp_f, b.tmp_i, nf, status);
}

int sort_scan_blocks(const GridP &g) { return (int)((g.ncell + 1 + SCAN_TILE - 1) / SCAN_TILE); }
int sort_launches() { return 9; }

void launch_clear_sort_flag(int *status, cudaStream_t s) { k_clear_flag<<<1, 1, 0, s>>>(status); }

// The per-step re-sort as one graph: a one-thread kernel reads the status
// word and sets the condition of an IF node whose body is the sort pipeline
// of every species followed by the flag reset.  A step in which no particle
// left its tile's margin then costs that one kernel instead of the pipeline's
// nine launches per species.  Captured on the private stream cap (the
// caller's stream may be one that cannot capture); the executable graph is
// launched on any stream of the context.  Valid while the particle arrays,
// the sort scratch and the status word keep their addresses.
cudaError_t make_sort_graph(const GridP &g, int nsp, const SpecP *sp, PartP *p, SortBufs &b, int *status, int *runs,
                            cudaStream_t cap, cudaGraphExec_t *out, cudaGraph_t tail) {
  *out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaGraphCreate(&graph, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  cudaGraphNode_t ncond = nullptr, nif = nullptr;
  e = cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    const int *cs = status;
    void *args[3] = {&h, (void *)&cs, &runs};
    cudaKernelNodeParams kp{};
    kp.func = (void *)k_sort_cond;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&ncond, graph, nullptr, 0, &kp);
  }
  cudaGraph_t body = nullptr;
  if (e == cudaSuccess) {
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&nif, graph, &ncond, nullptr, 1, &np);
    if (e == cudaSuccess) body = np.conditional.phGraph_out[0];
  }
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    for (int q = 0; q < nsp; ++q) launch_sort(g, sp[q], p[q], b, status, cap);
    launch_clear_sort_flag(status, cap);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cap, &captured);
  }
  // the rest of a step, when given, after the conditional re-sort (a copy of
  // the tail graph becomes a child node)
  cudaGraphNode_t ntail = nullptr;
  if (e == cudaSuccess && tail) e = cudaGraphAddChildGraphNode(&ntail, graph, &nif, 1, tail);
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) *out = nullptr;
  return e;
}
void launch_set_sort_flag(int *status, cudaStream_t s) { k_set_flag<<<1, 1, 0, s>>>(status); }

// particles whose load id is in the sorted list sid[0..n): copy the raw
// state of particle slot i to row k of out (k = position of its id in the
// list): cell, then D offsets, r[3], u1[3], u2[3] as floats
__global__ void k_pick(PartP p, int D, int two, long long count, const int *sid, const int *srow, int n, int *cell_out,
                       float *out, unsigned char *found) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = p.cell[i];
    if (c < 0) continue;
    const int id = p.id[i];
    int lo = 0, hi = n;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sid[mid] < id) lo = mid + 1;
      else hi = mid;
    }
    if (lo >= n || sid[lo] != id) continue;
    const int k = srow[lo];
    cell_out[k] = c;
    float *o = out + (size_t)k * 12;
    for (int a = 0; a < D; ++a) o[a] = p.off[a * p.cap + i];
    for (int a = 0; a < 3; ++a) {
      o[3 + a] = two ? p.r[a * p.cap + i] : 0.0f;
      o[6 + a] = p.u1[a * p.cap + i];
      o[9 + a] = two ? p.u2[a * p.cap + i] : 0.0f;
    }
    found[k] = 1;
  }
}

void launch_pick(const PartP &p, int D, int two, long long count, const int *sid, const int *srow, int n,
                 int *cell_out, float *out, unsigned char *found, cudaStream_t s) {
  k_pick<<<blocks_for(count, 256), 256, 0, s>>>(p, D, two, count, sid, srow, n, cell_out, out, found);
}

// seeded lattice: ion g = site * per_site + p sits at its site plus a
// Gaussian jitter (normals D g + a of the jitter stream) and takes momenta
// sigma N (normals 3 g + a of the momentum stream); written as FP64 position
// and momentum rows for the load conversion
__device__ __forceinline__ double sm64_normal(uint64_t key, uint64_t c) {
  const double u1 = sm64_uniform(key, 2 * c), u2 = sm64_uniform(key, 2 * c + 1);
  return sqrt(-2.0 * log(1.0 - u1)) * cos(6.283185307179586476925 * u2);
}

__global__ void k_gen_lattice(int D, const double *sites, int per_site, double jitter, uint64_t kj, uint64_t km,
                              double sigma, const int *site_param, long long first, long long count, double *x,
                              double *u, int *pidx) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < count;
       q += (long long)gridDim.x * blockDim.x) {
    const long long gi = first + q, site = gi / per_site;
    for (int a = 0; a < D; ++a)
      x[q * D + a] = sites[site * D + a] + (jitter > 0.0 ? jitter * sm64_normal(kj, (uint64_t)(D * gi + a)) : 0.0);
    for (int a = 0; a < 3; ++a) u[q * 3 + a] = sigma > 0.0 ? sigma * sm64_normal(km, (uint64_t)(3 * gi + a)) : 0.0;
    if (pidx) pidx[q] = site_param[site];
  }
}

void launch_gen_lattice(int D, const double *sites, int per_site, double jitter, uint64_t seed, double sigma,
                        const int *site_param, long long first, long long count, double *x, double *u, int *pidx,
                        cudaStream_t s) {
  k_gen_lattice<<<blocks_for(count, 256), 256, 0, s>>>(D, sites, per_site, jitter, sm64_key(seed, 2),
                                                        sm64_key(seed, 3), sigma, site_param, first, count, x, u,
                                                        pidx);
}

void launch_gen_medium(const GridP &g, const SpecP &sp, PartP &p, const int lo[3], const int hi[3], int ppc,
                       uint64_t seed, double sigma, long long first, long long count, cudaStream_t s) {
  uint64_t kpos = sm64_key(seed, 1), kmom = sm64_key(seed, 3);
  k_gen_medium<<<blocks_for(count, 256), 256, 0, s>>>(g, sp, p, lo[0], lo[1], lo[2], hi[0] - lo[0], hi[1] - lo[1], ppc,
                                                       kpos, kmom, sigma, first, count, first);
}

void launch_rho(const GridP &g, const SpecP &sp, const PartP &p, double *rho, cudaStream_t s) {
  k_rho<<<blocks_for(p.cap, 256), 256, 0, s>>>(g, sp, p, rho);
}

void launch_divE_minus(const GridP &g, const float *const E[3], double *R, cudaStream_t s) {
  k_divE<<<blocks_for(g.ncell, 256), 256, 0, s>>>(g, E[0], E[1], E[2], R);
}

void launch_load_convert(const GridP &g, const SpecP &sp, PartP &p, const double *x, const double *u, const int *pidx,
                         long long first, long long count, int *status, cudaStream_t s) {
  k_load_convert<<<blocks_for(count, 256), 256, 0, s>>>(g, sp, p, x, u, pidx, first, count, status);
}
