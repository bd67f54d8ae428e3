// k_fields.cu -- Yee FDTD for the vacuum Maxwell equations (the medium's
// response comes only from the particles' current, arXiv 2208.08038 Sec. 3.1),
// first-order Mur open faces, the fixed-order sum of the per-tile current
// boxes plus the laser antenna, and probes.  All FP32, memory bound: one
// thread per cell, coalesced along x.
#include "bp_internal.cuh"

namespace {

// along an open axis a component with half stagger has no value at n-1
// (exterior), one with node stagger has Mur boundary nodes at 0 and n-1
__device__ __forceinline__ bool exterior(const GridP &g, int pat, const int c[3]) {
  bool e = false;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a < g.D && g.bc[a] == BP_OPEN && ((pat >> a) & 1)) e |= c[a] == g.n[a] - 1;
  return e;
}
__device__ __forceinline__ int nbound(const GridP &g, int pat, const int c[3], int *first) {
  int k = 0;
  *first = -1;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a < g.D && g.bc[a] == BP_OPEN && !((pat >> a) & 1) && (c[a] == 0 || c[a] == g.n[a] - 1)) {
      if (*first < 0) *first = a;
      ++k;
    }
  return k;
}

// stagger pattern of E_x, E_y, E_z (bit a: half cell along axis a)
__device__ __forceinline__ int pat_e(int comp) { return 1 << comp; }

// B <- B - h curl E (forward differences to the B locations)
template <int D>
__global__ void __launch_bounds__(256) k_yee_b(GridP g, float *Bx, float *By, float *Bz, const float *__restrict__ Ex,
                                               const float *__restrict__ Ey, const float *__restrict__ Ez, float h) {
  Cell C;
  if (!row_cell<D>(g, C)) return;
  const long long q = C.q;
  bool nz = false;
  if (!exterior_c<D>(g, 6, C.c)) {
    float d = 0.0f;
    if (D >= 2) d += (Ez[q + C.up[1]] - Ez[q]) * g.idx[1];
    if (D >= 3) d -= (Ey[q + C.up[2]] - Ey[q]) * g.idx[2];
    const float v = Bx[q] - h * d;
    Bx[q] = v;
    nz |= v != 0.0f;
  }
  if (!exterior_c<D>(g, 5, C.c)) {
    float d = -(Ez[q + C.up[0]] - Ez[q]) * g.idx[0];
    if (D >= 3) d += (Ex[q + C.up[2]] - Ex[q]) * g.idx[2];
    const float v = By[q] - h * d;
    By[q] = v;
    nz |= v != 0.0f;
  }
  if (!exterior_c<D>(g, 3, C.c)) {
    float d = (Ey[q + C.up[0]] - Ey[q]) * g.idx[0];
    if (D >= 2) d -= (Ex[q + C.up[1]] - Ex[q]) * g.idx[1];
    const float v = Bz[q] - h * d;
    Bz[q] = v;
    nz |= v != 0.0f;
  }
  mark_nonzero<D>(g, C.c, nz);
}

// E <- E + dt (curl B - J) on interior nodes (backward differences)
template <int D>
__global__ void __launch_bounds__(256) k_yee_e(GridP g, float *Ex, float *Ey, float *Ez, const float *__restrict__ Bx,
                                               const float *__restrict__ By, const float *__restrict__ Bz,
                                               const float *__restrict__ Jx, const float *__restrict__ Jy,
                                               const float *__restrict__ Jz) {
  Cell C;
  if (!row_cell<D>(g, C)) return;
  const long long q = C.q;
  bool nz = false;
  if (!exterior_c<D>(g, 1, C.c) && !mur_node<D>(g, 1, C.c)) {
    float d = 0.0f;
    if (D >= 2) d += (Bz[q] - Bz[q + C.dn[1]]) * g.idx[1];
    if (D >= 3) d -= (By[q] - By[q + C.dn[2]]) * g.idx[2];
    const float v = Ex[q] + g.dt * (d - Jx[q]);
    Ex[q] = v;
    nz |= v != 0.0f;
  }
  if (!exterior_c<D>(g, 2, C.c) && !mur_node<D>(g, 2, C.c)) {
    float d = -(Bz[q] - Bz[q + C.dn[0]]) * g.idx[0];
    if (D >= 3) d += (Bx[q] - Bx[q + C.dn[2]]) * g.idx[2];
    const float v = Ey[q] + g.dt * (d - Jy[q]);
    Ey[q] = v;
    nz |= v != 0.0f;
  }
  if (!exterior_c<D>(g, 4, C.c) && !mur_node<D>(g, 4, C.c)) {
    float d = (By[q] - By[q + C.dn[0]]) * g.idx[0];
    if (D >= 2) d -= (Bx[q] - Bx[q + C.dn[1]]) * g.idx[1];
    const float v = Ez[q] + g.dt * (d - Jz[q]);
    Ez[q] = v;
    nz |= v != 0.0f;
  }
  mark_nonzero<D>(g, C.c, nz);
}

// the marks of the fields as they are (after a write from outside the step):
// every tile holding a non-zero E or B component (marks cleared before)
template <int D>
__global__ void __launch_bounds__(256) k_field_marks(GridP g, const float *__restrict__ Ex,
                                                     const float *__restrict__ Ey, const float *__restrict__ Ez,
                                                     const float *__restrict__ Bx, const float *__restrict__ By,
                                                     const float *__restrict__ Bz) {
  Cell C;
  if (!row_cell<D>(g, C)) return;
  const long long q = C.q;
  const bool nz = Ex[q] != 0.0f || Ey[q] != 0.0f || Ez[q] != 0.0f || Bx[q] != 0.0f || By[q] != 0.0f ||
                  Bz[q] != 0.0f;
  mark_nonzero<D>(g, C.c, nz);
}

// ---------------------------------------------------------------------------
// Mur faces.  frame[] holds, for every open face, the old values of the two
// tangential components on the boundary layer (l = 0) and the adjacent layer
// (l = 1): frame[base(a) + (((side * 2 + l) * 2 + ci) * face + pos)].

__device__ __forceinline__ long long face_size(const GridP &g, int a) { return g.ncell / g.n[a]; }

__device__ __forceinline__ void face_node(const GridP &g, int a, int side, int layer, long long pos, int c[3]) {
  int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
  int lo = o1 < o2 ? o1 : o2, hi = o1 < o2 ? o2 : o1;
  c[lo] = (int)(pos % g.n[lo]);
  c[hi] = (int)(pos / g.n[lo]);
  c[a] = side == 0 ? layer : g.n[a] - 1 - layer;
}

__device__ __forceinline__ int tang_comp(int a, int ci) {
  // the two components other than a, in increasing order
  int c0 = a == 0 ? 1 : 0;
  int c1 = a == 2 ? 1 : 2;
  return ci == 0 ? c0 : c1;
}

__global__ void k_frame_save(GridP g, const float *Ex, const float *Ey, const float *Ez, float *frame,
                             long long total) {
  const float *E[3] = {Ex, Ey, Ez};
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    long long base = 0, rem = q;
    int a = 0;
    for (; a < g.D; ++a) {
      if (g.bc[a] != BP_OPEN) continue;
      long long n = 8 * face_size(g, a);
      if (rem < n) break;
      rem -= n;
      base += n;
    }
    long long F = face_size(g, a);
    long long pos = rem % F;
    int t = (int)(rem / F);  // ((side * 2 + l) * 2 + ci)
    int ci = t & 1, l = (t >> 1) & 1, side = t >> 2;
    int c[3];
    face_node(g, a, side, l, pos, c);
    long long id = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
    frame[q] = E[tang_comp(a, ci)][id];
  }
}

// E_b(n+1) = E_adj(n) + (dt - dx)/(dt + dx) (E_adj(n+1) - E_b(n)); a node
// on p open faces is done in pass p, through its first open axis
__global__ void k_mur(GridP g, float *Ex, float *Ey, float *Ez, const float *frame, long long nbnd, int pass) {
  float *E[3] = {Ex, Ey, Ez};
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nbnd;
       q += (long long)gridDim.x * blockDim.x) {
    long long base = 0, rem = q;
    int a = 0;
    for (; a < g.D; ++a) {
      if (g.bc[a] != BP_OPEN) continue;
      long long n = 4 * face_size(g, a);
      if (rem < n) break;
      rem -= n;
      base += 8 * face_size(g, a);
    }
    long long F = face_size(g, a);
    long long pos = rem % F;
    int t = (int)(rem / F);  // side * 2 + ci
    int ci = t & 1, side = t >> 1;
    int comp = tang_comp(a, ci);
    int c[3];
    face_node(g, a, side, 0, pos, c);
    int first;
    if (exterior(g, pat_e(comp), c)) continue;
    if (nbound(g, pat_e(comp), c, &first) != pass || first != a) continue;
    int ca[3] = {c[0], c[1], c[2]};
    ca[a] += side == 0 ? 1 : -1;
    long long id = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
    long long ida = ca[0] + (long long)g.n[0] * (ca[1] + (long long)g.n[1] * ca[2]);
    float old_b = frame[base + ((side * 2 + 0) * 2 + ci) * F + pos];
    float old_a = frame[base + ((side * 2 + 1) * 2 + ci) * F + pos];
    float km = (g.dt - g.dx[a]) / (g.dt + g.dx[a]);
    const float v = old_a + km * (E[comp][ida] - old_b);
    E[comp][id] = v;
    if (v != 0.0f) {
      unsigned char *f = g.fnz + tile_of(g, c);
      if (*f == 0) *f = 1;
    }
  }
}

// ---------------------------------------------------------------------------
// current: J(cell) = sum of the boxes of the tiles covering the cell, in a
// fixed order (z, y, x candidates ascending), plus the antenna sheets

__device__ double laser_value(const LaserP &L, double t, double y, double z) {
  double ty = y - L.yc, tz = z - L.zc;
  double tau = t - ty * sin(L.theta);
  double env;
  if (L.fwhm > 0) {
    double d = tau - L.t0;
    env = exp(-2.0 * 0.69314718055994530942 * d * d / (L.fwhm * L.fwhm));
  } else if (tau <= 0) {
    env = 0.0;
  } else if (tau < L.ramp) {
    double s = sin(0.5 * 3.14159265358979323846 * tau / L.ramp);
    env = s * s;
  } else {
    env = 1.0;
  }
  double prof = 1.0;
  if (L.waist > 0) {
    double ey = ty * cos(L.theta);
    prof = exp(-(ey * ey + tz * tz) / (L.waist * L.waist));
  }
  return L.a0 * env * prof * sin(L.omega * tau + L.phase);
}

struct LaserSet {
  int n;
  LaserP l[BP_MAX_LASER];
};

template <int D>
__global__ void __launch_bounds__(256) k_jsum(GridP g, const float *__restrict__ jbox,
                                              const unsigned char *__restrict__ occ, const uint2 *__restrict__ jbb,
                                              float *Jx, float *Jy, float *Jz, LaserSet las, double t) {
  Cell C;
  if (!row_cell<D>(g, C)) return;
  const int *c = C.c;
  // the (up to three per axis) tiles whose boxes cover the cell, ascending
  int tw[3][3], loc[3][3], nc[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    nc[a] = 0;
    if (a >= D) {
      tw[a][0] = 0;
      loc[a][0] = 0;
      nc[a] = 1;
      continue;
    }
    const int tb = c[a] / g.L[a];
#pragma unroll
    for (int dt = -1; dt <= 1; ++dt) {
      const int tu = tb + dt;
      const int l = c[a] - (tu * g.L[a] - g.oj[a]);
      if (l < 0 || l >= g.jb[a]) continue;
      int tt = tu;
      if (g.bc[a] == BP_PERIODIC) tt = wrap_once(tu, g.nt[a]);
      else if (tu < 0 || tu >= g.nt[a]) continue;
      tw[a][nc[a]] = tt;
      loc[a][nc[a]] = l;
      ++nc[a];
    }
  }
  float sx = 0.0f, sy = 0.0f, sz = 0.0f;
  for (int k = 0; k < nc[2]; ++k)
    for (int j = 0; j < nc[1]; ++j)
      for (int i = 0; i < nc[0]; ++i) {
        const int tile = tw[0][i] + g.nt[0] * (tw[1][j] + g.nt[1] * tw[2][k]);
        if (!occ[tile]) continue;
        // outside the tile's deposit box every entry is zero (and unwritten)
        const uint2 bb = jbb[tile];
        const int l0 = loc[0][i], l1 = loc[1][j], l2 = loc[2][k];
        if (l0 < (int)(bb.x & 255u) || l0 > (int)(bb.y & 255u) || l1 < (int)((bb.x >> 8) & 255u) ||
            l1 > (int)((bb.y >> 8) & 255u) || l2 < (int)((bb.x >> 16) & 255u) || l2 > (int)((bb.y >> 16) & 255u))
          continue;
        const long long l = l0 + (long long)g.jb[0] * (l1 + (long long)g.jb[1] * l2);
        const float *b = jbox + (size_t)tile * 3 * g.jcells;
        sx += b[l];
        sy += b[g.jcells + l];
        sz += b[2 * g.jcells + l];
      }
  for (int s = 0; s < las.n; ++s) {
    const LaserP &L = las.l[s];
    if (c[0] != L.ia) continue;
    // the antenna current sits on the E_y (comp 1) or E_z (comp 2) location
    double y = D >= 2 ? (c[1] + (L.comp == 1 ? 0.5 : 0.0)) * g.dxd[1] : 0.0;
    double z = D >= 3 ? (c[2] + (L.comp == 2 ? 0.5 : 0.0)) * g.dxd[2] : 0.0;
    double amp = -2.0 / g.dxd[0] * (L.comp == 2 ? cos(L.theta) : 1.0);
    double v = amp * laser_value(L, t, y, z);
    if (L.comp == 1) sy = (float)((double)sy + v);
    else sz = (float)((double)sz + v);
  }
  Jx[C.q] = sx;
  Jy[C.q] = sy;
  Jz[C.q] = sz;
}

__global__ void k_probe(const float *F, const long long *nodes, long long npts, float *buf) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < npts; q += (long long)gridDim.x * blockDim.x)
    buf[q] = F[nodes[q]];
}

int grid_blocks(long long n, int bs) {
  long long b = (n + bs - 1) / bs;
  long long cap = 152LL * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

long long frame_floats(const GridP &g) {
  long long t = 0;
  for (int a = 0; a < g.D; ++a)
    if (g.bc[a] == BP_OPEN) t += 8 * (g.ncell / g.n[a]);
  return t;
}

void launch_yee_b(const GridP &g, float *const B[3], const float *const E[3], float h, cudaStream_t s) {
  const int nb = row_blocks(g, 256);
  if (g.D == 1) k_yee_b<1><<<nb, 256, 0, s>>>(g, B[0], B[1], B[2], E[0], E[1], E[2], h);
  else if (g.D == 2) k_yee_b<2><<<nb, 256, 0, s>>>(g, B[0], B[1], B[2], E[0], E[1], E[2], h);
  else k_yee_b<3><<<nb, 256, 0, s>>>(g, B[0], B[1], B[2], E[0], E[1], E[2], h);
}

void launch_yee_e(const GridP &g, float *const E[3], const float *const B[3], const float *const J[3], float *frame,
                  cudaStream_t s) {
  long long nf = frame_floats(g);
  if (nf) k_frame_save<<<grid_blocks(nf, 256), 256, 0, s>>>(g, E[0], E[1], E[2], frame, nf);
  const int nb = row_blocks(g, 256);
  if (g.D == 1) k_yee_e<1><<<nb, 256, 0, s>>>(g, E[0], E[1], E[2], B[0], B[1], B[2], J[0], J[1], J[2]);
  else if (g.D == 2) k_yee_e<2><<<nb, 256, 0, s>>>(g, E[0], E[1], E[2], B[0], B[1], B[2], J[0], J[1], J[2]);
  else k_yee_e<3><<<nb, 256, 0, s>>>(g, E[0], E[1], E[2], B[0], B[1], B[2], J[0], J[1], J[2]);
  if (nf) {
    int nopen = 0;
    for (int a = 0; a < g.D; ++a) nopen += g.bc[a] == BP_OPEN;
    for (int p = 1; p <= nopen; ++p)
      k_mur<<<grid_blocks(nf / 2, 256), 256, 0, s>>>(g, E[0], E[1], E[2], frame, nf / 2, p);
  }
}

void launch_field_marks(const GridP &g, const float *const F[6], cudaStream_t s) {
  cudaMemsetAsync(g.fnz, 0, (size_t)g.ntiles, s);
  const int nb = row_blocks(g, 256);
  if (g.D == 1) k_field_marks<1><<<nb, 256, 0, s>>>(g, F[0], F[1], F[2], F[3], F[4], F[5]);
  else if (g.D == 2) k_field_marks<2><<<nb, 256, 0, s>>>(g, F[0], F[1], F[2], F[3], F[4], F[5]);
  else k_field_marks<3><<<nb, 256, 0, s>>>(g, F[0], F[1], F[2], F[3], F[4], F[5]);
}

void launch_jsum(const GridP &g, const float *jbox, const unsigned char *occ, const uint2 *jbb, float *const J[3],
                 const LaserP *las, int nlas, double t, cudaStream_t s) {
  LaserSet ls;
  ls.n = nlas;
  for (int i = 0; i < nlas; ++i) ls.l[i] = las[i];
  const int nb = row_blocks(g, 256);
  if (g.D == 1) k_jsum<1><<<nb, 256, 0, s>>>(g, jbox, occ, jbb, J[0], J[1], J[2], ls, t);
  else if (g.D == 2) k_jsum<2><<<nb, 256, 0, s>>>(g, jbox, occ, jbb, J[0], J[1], J[2], ls, t);
  else k_jsum<3><<<nb, 256, 0, s>>>(g, jbox, occ, jbb, J[0], J[1], J[2], ls, t);
}

// one block row per copy; 16-byte moves when both ends allow, then the tail
__global__ void k_copy_many(CopyList L) {
  const int k = blockIdx.y;
  const long long n = L.words[k];
  const unsigned *src = static_cast<const unsigned *>(L.src[k]);
  unsigned *dst = static_cast<unsigned *>(L.dst[k]);
  const bool v4 = (((size_t)src | (size_t)dst) & 15) == 0;
  const long long nv = v4 ? n / 4 : 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv; i += stride)
    reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(src)[i];
  for (long long i = 4 * nv + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

void launch_copy_many(const CopyList &L, cudaStream_t s) {
  if (L.n <= 0) return;
  long long most = 0;
  for (int k = 0; k < L.n; ++k) most = most > L.words[k] ? most : L.words[k];
  long long bx = (most / 4 + 255) / 256;
  bx = bx < 1 ? 1 : (bx > 152 * 8 ? 152 * 8 : bx);
  k_copy_many<<<dim3((unsigned)bx, (unsigned)L.n), 256, 0, s>>>(L);
}

void launch_probe(const float *F, const long long *nodes, long long npts, float *buf, long long slot,
                  cudaStream_t s) {
  k_probe<<<grid_blocks(npts, 256), 256, 0, s>>>(F, nodes, npts, buf + slot * npts);
}
