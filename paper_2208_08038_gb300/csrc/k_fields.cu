// k_fields.cu -- Yee FDTD for the vacuum Maxwell equations (the medium's
// response comes only from the particles' current, arXiv 2208.08038 Sec. 3.1),
// first-order Mur open faces, the laser antenna, the current (sorted deposit:
// formed in the E update from the 64-bit fixed-point accumulator; atomic
// deposit: the fixed-order sum of the per-tile boxes), the tile marks of
// non-zero fields, the device step clock (step number and probe sample
// counts, so a step's launches are the same every step), and probes.  All
// FP32, memory bound: the Yee updates take four consecutive x cells per
// thread (16-byte vector loads and stores, coalesced along x) and return at
// once in tiles the per-step activity flags mark inactive (E, B and J are
// zero there and would stay zero); the other kernels one cell per thread.
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

// whether cell x of the group is an exterior position (open axis, half
// stagger, last cell) or a Mur node (open axis, node stagger, first or last
// cell) of a component with stagger pattern pat
template <int D>
__device__ __forceinline__ bool skip_cell(const GridP &g, int pat, const int c[3], int i, bool mur) {
  int ci[3] = {c[0] + i, c[1], c[2]};
  return exterior_c<D>(g, pat, ci) || (mur && mur_node<D>(g, pat, ci));
}

// the tile mark of a group of four cells (see mark_nonzero): the lowest lane
// of each tile segment (L0 / 4 lanes) that holds a non-zero value writes it
template <int D>
__device__ __forceinline__ void mark_nonzero4(const GridP &g, const int c[3], bool nz) {
  const unsigned m = __ballot_sync(__activemask(), nz);
  if (!nz) return;
  constexpr int LANES = Geo<D>::L0 / 4;
  static_assert(LANES >= 1 && LANES <= 32 && (LANES & (LANES - 1)) == 0, "a tile segment lies inside one warp");
  const int lane = (int)(threadIdx.x & 31u);
  const int base = lane & ~(LANES - 1);
  if (m & ((1u << lane) - 1u) & ~((1u << base) - 1u)) return;
  unsigned char *f = g.fnz + tile_of(g, c);
  if (*f == 0) *f = 1;
}

// B <- B - h curl E (forward differences to the B locations)
template <int D>
__global__ void __launch_bounds__(128) k_yee_b(GridP g, float *Bx, float *By, float *Bz, const float *__restrict__ Ex,
                                               const float *__restrict__ Ey, const float *__restrict__ Ez, float h,
                                               const unsigned char *__restrict__ act) {
  Cell4 C;
  if (!row_cell4<D>(g, C)) return;
  if (act && !act[tile_of(g, C.c)]) return;  // E and B zero around the tile: B stays zero
  const long long q = C.q;
  const float4 ex = ld4(Ex + q), ey = ld4(Ey + q), ez = ld4(Ez + q);
  const float eyn = Ey[q + C.up[0]], ezn = Ez[q + C.up[0]];  // x neighbours of the last cell
  float4 ezy = ez, exy = ex, eyz = ey, exz = ex;
  if (D >= 2) {
    ezy = ld4(Ez + q + C.up[1]);
    exy = ld4(Ex + q + C.up[1]);
  }
  if (D >= 3) {
    eyz = ld4(Ey + q + C.up[2]);
    exz = ld4(Ex + q + C.up[2]);
  }
  float4 bx = ld4(Bx + q), by = ld4(By + q), bz = ld4(Bz + q);
  bool nz = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float ezi = el(ez, i), eyi = el(ey, i), exi = el(ex, i);
    const float ezx = i < 3 ? el(ez, i + 1) : ezn, eyx = i < 3 ? el(ey, i + 1) : eyn;
    if (!skip_cell<D>(g, 6, C.c, i, false)) {
      float d = 0.0f;
      if (D >= 2) d += (el(ezy, i) - ezi) * g.idx[1];
      if (D >= 3) d -= (el(eyz, i) - eyi) * g.idx[2];
      const float v = el(bx, i) - h * d;
      set_el(bx, i, v);
      nz |= v != 0.0f;
    }
    if (!skip_cell<D>(g, 5, C.c, i, false)) {
      float d = -(ezx - ezi) * g.idx[0];
      if (D >= 3) d += (el(exz, i) - exi) * g.idx[2];
      const float v = el(by, i) - h * d;
      set_el(by, i, v);
      nz |= v != 0.0f;
    }
    if (!skip_cell<D>(g, 3, C.c, i, false)) {
      float d = (eyx - eyi) * g.idx[0];
      if (D >= 2) d -= (el(exy, i) - exi) * g.idx[1];
      const float v = el(bz, i) - h * d;
      set_el(bz, i, v);
      nz |= v != 0.0f;
    }
  }
  st4(Bx + q, bx);
  st4(By + q, by);
  st4(Bz + q, bz);
  mark_nonzero4<D>(g, C.c, nz);
}

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
  int lo, hi;  // lowest and highest antenna plane
  LaserP l[BP_MAX_LASER];
};

LaserSet make_laser_set(const LaserP *las, int nlas) {
  LaserSet ls;
  ls.n = nlas;
  ls.lo = 1 << 30;
  ls.hi = -1;
  for (int i = 0; i < nlas; ++i) {
    ls.l[i] = las[i];
    ls.lo = las[i].ia < ls.lo ? las[i].ia : ls.lo;
    ls.hi = las[i].ia > ls.hi ? las[i].ia : ls.hi;
  }
  return ls;
}

// v * s for a 64-bit fixed-point value v and a power-of-two scale s, rounded
// once: v = a 2^24 + b with 0 <= b < 2^24, both exact in FP32 while
// |v| < 2^48, so the fma rounds the exact product (the 64-bit integer
// conversion would run on the slow FP64 path)
__device__ __forceinline__ float fx_to_float(long long v, float s) {
  const float a = (float)(int)(v >> 24);
  const float b = (float)(int)(v & 0xFFFFFFLL);
  return fmaf(a, 16777216.0f * s, b * s);
}

// The step clock in device memory, so that a step's launches are the same
// every step (one CUDA graph replayed): clk[0] the step number n,
// clk[1 + p] probe p's samples so far, clk[1 + BP_MAX_PROBE + p] its
// capacity.  The current J^{n+1/2} and the antenna's sheet take time
// (n + 1/2) dt.
__device__ __forceinline__ double current_time(const GridP &g, const long long *clk) {
  return ((double)clk[0] + 0.5) * g.dtd;
}

// the antenna sheets' current on their planes at the current's time, FP64:
// ant[s][y + ny z] for laser s (the value the current sum adds at cell
// (L.ia, y, z))
template <int D>
__global__ void k_antenna(GridP g, LaserSet las, const long long *clk, double *ant) {
  const double t = current_time(g, clk);
  const long long nyz = g.ncell / g.n[0];
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < las.n * nyz;
       q += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(q / nyz);
    const long long yz = q - s * nyz;
    const int cy = (int)(yz % g.n[1]), cz = (int)(yz / g.n[1]);
    const LaserP &L = las.l[s];
    double y = D >= 2 ? (cy + (L.comp == 1 ? 0.5 : 0.0)) * g.dxd[1] : 0.0;
    double z = D >= 3 ? (cz + (L.comp == 2 ? 0.5 : 0.0)) * g.dxd[2] : 0.0;
    double amp = -2.0 / g.dxd[0] * (L.comp == 2 ? cos(L.theta) : 1.0);
    ant[q] = amp * laser_value(L, t, y, z);
  }
}

// the antenna part of the sheets covering cell c: only which laser sits on
// which plane and component is needed here
struct AntSet {
  int n, lo, hi;
  int ia[BP_MAX_LASER], comp[BP_MAX_LASER];
};

// E <- E + dt (curl B - J) on interior nodes (backward differences).  FX:
// J^{n+1/2} is formed here from the 64-bit fixed-point accumulator (one
// rounding: the scale jinv is a power of two) plus the antenna (added in
// FP64 before the rounding) and stored in J; the launcher then clears the
// accumulator for the next deposit with one memset (clearing it here, after
// the loads, ran the kernel at a third of the bandwidth).
template <int D, bool FX>
__global__ void __launch_bounds__(128) k_yee_e(GridP g, float *Ex, float *Ey, float *Ez, const float *__restrict__ Bx,
                                               const float *__restrict__ By, const float *__restrict__ Bz, float *Jx,
                                               float *Jy, float *Jz, unsigned long long *jfx, float jinv,
                                               AntSet as, const double *__restrict__ ant,
                                               const unsigned char *__restrict__ act) {
  Cell4 C;
  if (!row_cell4<D>(g, C)) return;
  if (act && !act[tile_of(g, C.c)]) return;  // no field and no current around the tile: E stays zero
  const long long q = C.q;
  float4 jx, jy, jz;
  if constexpr (FX) {
    const long long nc = g.ncell;
    const ulonglong2 *px = reinterpret_cast<const ulonglong2 *>(jfx + q);
    const ulonglong2 *py = reinterpret_cast<const ulonglong2 *>(jfx + nc + q);
    const ulonglong2 *pz = reinterpret_cast<const ulonglong2 *>(jfx + 2 * nc + q);
    const ulonglong2 x0 = px[0], x1 = px[1], y0 = py[0], y1 = py[1], z0 = pz[0], z1 = pz[1];
    const long long fx[4] = {(long long)x0.x, (long long)x0.y, (long long)x1.x, (long long)x1.y};
    const long long fy[4] = {(long long)y0.x, (long long)y0.y, (long long)y1.x, (long long)y1.y};
    const long long fz[4] = {(long long)z0.x, (long long)z0.y, (long long)z1.x, (long long)z1.y};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      set_el(jx, i, fx_to_float(fx[i], jinv));
      set_el(jy, i, fx_to_float(fy[i], jinv));
      set_el(jz, i, fx_to_float(fz[i], jinv));
    }
    if (as.n > 0 && C.c[0] + 3 >= as.lo && C.c[0] <= as.hi) {
      // an antenna plane in the group: its sheet current added in FP64
      // before the one rounding
      const long long yz = q / g.n[0], nyz = g.ncell / g.n[0];
      for (int i = 0; i < 4; ++i) {
        double ay = 0.0, az = 0.0;
        bool on = false;
#pragma unroll
        for (int k = 0; k < BP_MAX_LASER; ++k) {
          if (k >= as.n || C.c[0] + i != as.ia[k]) continue;
          on = true;
          if (as.comp[k] == 1) ay += ant[k * nyz + yz];
          else az += ant[k * nyz + yz];
        }
        if (on) {
          set_el(jy, i, (float)((double)fy[i] * (double)jinv + ay));
          set_el(jz, i, (float)((double)fz[i] * (double)jinv + az));
        }
      }
    }
    st4(Jx + q, jx);
    st4(Jy + q, jy);
    st4(Jz + q, jz);
  } else {
    jx = ld4(Jx + q);
    jy = ld4(Jy + q);
    jz = ld4(Jz + q);
  }
  const float4 bx = ld4(Bx + q), by = ld4(By + q), bz = ld4(Bz + q);
  const float byp = By[q + C.dn[0]], bzp = Bz[q + C.dn[0]];  // x neighbours of the first cell
  float4 bzy = bz, bxy = bx, byz = by, bxz = bx;
  if (D >= 2) {
    bzy = ld4(Bz + q + C.dn[1]);
    bxy = ld4(Bx + q + C.dn[1]);
  }
  if (D >= 3) {
    byz = ld4(By + q + C.dn[2]);
    bxz = ld4(Bx + q + C.dn[2]);
  }
  float4 ex = ld4(Ex + q), ey = ld4(Ey + q), ez = ld4(Ez + q);
  bool nz = false;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float bxi = el(bx, i), byi = el(by, i), bzi = el(bz, i);
    const float byx = i > 0 ? el(by, i - 1) : byp, bzx = i > 0 ? el(bz, i - 1) : bzp;
    if (!skip_cell<D>(g, 1, C.c, i, true)) {
      float d = 0.0f;
      if (D >= 2) d += (bzi - el(bzy, i)) * g.idx[1];
      if (D >= 3) d -= (byi - el(byz, i)) * g.idx[2];
      const float v = el(ex, i) + g.dt * (d - el(jx, i));
      set_el(ex, i, v);
      nz |= v != 0.0f;
    }
    if (!skip_cell<D>(g, 2, C.c, i, true)) {
      float d = -(bzi - bzx) * g.idx[0];
      if (D >= 3) d += (bxi - el(bxz, i)) * g.idx[2];
      const float v = el(ey, i) + g.dt * (d - el(jy, i));
      set_el(ey, i, v);
      nz |= v != 0.0f;
    }
    if (!skip_cell<D>(g, 4, C.c, i, true)) {
      float d = (byi - byx) * g.idx[0];
      if (D >= 2) d -= (bxi - el(bxy, i)) * g.idx[1];
      const float v = el(ez, i) + g.dt * (d - el(jz, i));
      set_el(ez, i, v);
      nz |= v != 0.0f;
    }
  }
  st4(Ex + q, ex);
  st4(Ey + q, ey);
  st4(Ez + q, ez);
  mark_nonzero4<D>(g, C.c, nz);
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

template <int D>
__global__ void __launch_bounds__(256) k_jsum(GridP g, const float *__restrict__ jbox,
                                              const unsigned char *__restrict__ occ, const uint2 *__restrict__ jbb,
                                              float *Jx, float *Jy, float *Jz, LaserSet las, const long long *clk) {
  Cell C;
  if (!row_cell<D>(g, C)) return;
  const double t = current_time(g, clk);
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

// The same sum with one block per destination tile (2D, 3D): the block's
// cells are covered only by the boxes of the tile's 3^D neighbours, whose
// occupancy and bounding boxes are read once into shared memory; each cell
// adds the covering boxes in the same order as k_jsum (source tiles by
// ascending z, y, x offset), so the result is the same.
template <int D>
__global__ void __launch_bounds__(Geo<D>::L0 * Geo<D>::L1 * Geo<D>::L2)
    k_jsum_tile(GridP g, const float *__restrict__ jbox, const unsigned char *__restrict__ occ,
                const uint2 *__restrict__ jbb, float *Jx, float *Jy, float *Jz, LaserSet las, const long long *clk) {
  static_assert(D >= 2, "tile form for 2D and 3D");
  const double t = current_time(g, clk);
  constexpr int L0 = Geo<D>::L0, L1 = Geo<D>::L1, L2 = Geo<D>::L2;
  constexpr int NC = D == 3 ? 27 : 9;
  __shared__ int ctile[NC], corg[NC][3];
  __shared__ uint2 cbb[NC];
  const int tile = blockIdx.x, tid = threadIdx.x;
  const int tc[3] = {tile % g.nt[0], (tile / g.nt[0]) % g.nt[1], tile / (g.nt[0] * g.nt[1])};
  if (tid < NC) {
    const int o[3] = {tid % 3 - 1, (tid / 3) % 3 - 1, D == 3 ? tid / 9 - 1 : 0};
    bool use = true;
    int nb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int tu = tc[a] + o[a];
      // first box cell of the source tile, in the (unwrapped) coordinates of this tile's cells
      corg[tid][a] = a < D ? tu * g.L[a] - g.oj[a] : 0;
      nb[a] = tu;
      if (a < D) {
        if (g.bc[a] == BP_PERIODIC) nb[a] = wrap_once(tu, g.nt[a]);
        else use &= tu >= 0 && tu < g.nt[a];
      }
    }
    const int src = nb[0] + g.nt[0] * (nb[1] + g.nt[1] * nb[2]);
    ctile[tid] = use && occ[src] ? src : -1;
    cbb[tid] = use ? jbb[src] : make_uint2(0u, 0u);
  }
  __syncthreads();
  const int c[3] = {tc[0] * L0 + tid % L0, tc[1] * L1 + (tid / L0) % L1, tc[2] * L2 + tid / (L0 * L1)};
  float sx = 0.0f, sy = 0.0f, sz = 0.0f;
  // unrolled: every covering box's loads are issued before the in-order adds
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const int src = ctile[k];
    if (src < 0) continue;
    const uint2 bb = cbb[k];
    const int l0 = c[0] - corg[k][0], l1 = c[1] - corg[k][1], l2 = c[2] - corg[k][2];
    // outside the tile's deposit box every entry is zero (and unwritten)
    if (l0 < (int)(bb.x & 255u) || l0 > (int)(bb.y & 255u) || l1 < (int)((bb.x >> 8) & 255u) ||
        l1 > (int)((bb.y >> 8) & 255u) || l2 < (int)((bb.x >> 16) & 255u) || l2 > (int)((bb.y >> 16) & 255u))
      continue;
    const long long l = l0 + (long long)g.jb[0] * (l1 + (long long)g.jb[1] * l2);
    const float *b = jbox + (size_t)src * 3 * g.jcells;
    sx += b[l];
    sy += b[g.jcells + l];
    sz += b[2 * g.jcells + l];
  }
  for (int s = 0; s < las.n; ++s) {
    const LaserP &L = las.l[s];
    if (c[0] != L.ia) continue;
    double y = (c[1] + (L.comp == 1 ? 0.5 : 0.0)) * g.dxd[1];
    double z = D >= 3 ? (c[2] + (L.comp == 2 ? 0.5 : 0.0)) * g.dxd[2] : 0.0;
    double amp = -2.0 / g.dxd[0] * (L.comp == 2 ? cos(L.theta) : 1.0);
    double v = amp * laser_value(L, t, y, z);
    if (L.comp == 1) sy = (float)((double)sy + v);
    else sz = (float)((double)sz + v);
  }
  const long long q = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
  Jx[q] = sx;
  Jy[q] = sy;
  Jz[q] = sz;
}

// probe p's sample of this step into its next slot, while it has room
__global__ void k_probe(const float *F, const long long *nodes, long long npts, float *buf, const long long *clk,
                        int p) {
  const long long slot = clk[1 + p];
  if (slot >= clk[1 + BP_MAX_PROBE + p]) return;
  float *out = buf + slot * npts;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < npts; q += (long long)gridDim.x * blockDim.x)
    out[q] = F[nodes[q]];
}

// the end of a step: the clock advances, and the sample count of each of
// the first nprobe probes (those recorded this step) while it has room
__global__ void k_clock_tick(long long *clk, int nprobe) {
  if (threadIdx.x == 0) clk[0] += 1;
  if ((int)threadIdx.x < nprobe && clk[1 + threadIdx.x] < clk[1 + BP_MAX_PROBE + threadIdx.x]) clk[1 + threadIdx.x] += 1;
}

// the clock set from the host's state
__global__ void k_clock_set(long long *clk, ClockState v) {
  const int i = threadIdx.x;
  if (i == 0) clk[0] = v.step;
  if (i < BP_MAX_PROBE) {
    clk[1 + i] = i < v.nprobe ? v.count[i] : 0;
    clk[1 + BP_MAX_PROBE + i] = i < v.nprobe ? v.cap[i] : 0;
  }
}

// blocks for n items; the kernels launched with it are grid-stride loops, so
// the cap (two waves of 256-thread blocks on 152 SMs) only bounds the grid
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

void launch_yee_b(const GridP &g, float *const B[3], const float *const E[3], float h, const unsigned char *act,
                  cudaStream_t s) {
  const int nb = row_blocks4(g, 128);
  if (g.D == 1) k_yee_b<1><<<nb, 128, 0, s>>>(g, B[0], B[1], B[2], E[0], E[1], E[2], h, act);
  else if (g.D == 2) k_yee_b<2><<<nb, 128, 0, s>>>(g, B[0], B[1], B[2], E[0], E[1], E[2], h, act);
  else k_yee_b<3><<<nb, 128, 0, s>>>(g, B[0], B[1], B[2], E[0], E[1], E[2], h, act);
}

void launch_yee_e(const GridP &g, float *const E[3], const float *const B[3], float *const J[3], float *frame,
                  unsigned long long *jfx, float jinv, const LaserP *las, int nlas, const long long *clk,
                  double *ant, const unsigned char *act, cudaStream_t s) {
  long long nf = frame_floats(g);
  if (nf) k_frame_save<<<grid_blocks(nf, 256), 256, 0, s>>>(g, E[0], E[1], E[2], frame, nf);
  const int nb = row_blocks4(g, 128);
  AntSet as;
  as.n = jfx ? nlas : 0;
  as.lo = 1 << 30;
  as.hi = -1;
  for (int i = 0; i < as.n; ++i) {
    as.ia[i] = las[i].ia;
    as.comp[i] = las[i].comp;
    as.lo = las[i].ia < as.lo ? las[i].ia : as.lo;
    as.hi = las[i].ia > as.hi ? las[i].ia : as.hi;
  }
  if (as.n > 0) {
    const LaserSet ls = make_laser_set(las, nlas);
    const long long nant = (long long)nlas * (g.ncell / g.n[0]);
    // small blocks: the FP64 exp / sin of the antenna planes spread over many SMs
    if (g.D == 1) k_antenna<1><<<grid_blocks(nant, 64), 64, 0, s>>>(g, ls, clk, ant);
    else if (g.D == 2) k_antenna<2><<<grid_blocks(nant, 64), 64, 0, s>>>(g, ls, clk, ant);
    else k_antenna<3><<<grid_blocks(nant, 64), 64, 0, s>>>(g, ls, clk, ant);
  }
#define YEE_E(DD, FF) \
  k_yee_e<DD, FF><<<nb, 128, 0, s>>>(g, E[0], E[1], E[2], B[0], B[1], B[2], J[0], J[1], J[2], jfx, jinv, as, ant, act)
  if (jfx) {
    if (g.D == 1) YEE_E(1, true);
    else if (g.D == 2) YEE_E(2, true);
    else YEE_E(3, true);
  } else {
    if (g.D == 1) YEE_E(1, false);
    else if (g.D == 2) YEE_E(2, false);
    else YEE_E(3, false);
  }
#undef YEE_E
  if (jfx) cudaMemsetAsync(jfx, 0, sizeof(unsigned long long) * 3 * (size_t)g.ncell, s);
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
                 const LaserP *las, int nlas, const long long *clk, cudaStream_t s) {
  const LaserSet ls = make_laser_set(las, nlas);
  if (g.D == 1) {
    k_jsum<1><<<row_blocks(g, 256), 256, 0, s>>>(g, jbox, occ, jbb, J[0], J[1], J[2], ls, clk);
  } else if (g.D == 2) {
    constexpr int nt = Geo<2>::L0 * Geo<2>::L1 * Geo<2>::L2;
    k_jsum_tile<2><<<g.ntiles, nt, 0, s>>>(g, jbox, occ, jbb, J[0], J[1], J[2], ls, clk);
  } else {
    constexpr int nt = Geo<3>::L0 * Geo<3>::L1 * Geo<3>::L2;
    k_jsum_tile<3><<<g.ntiles, nt, 0, s>>>(g, jbox, occ, jbb, J[0], J[1], J[2], ls, clk);
  }
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

void launch_copy_many(const CopyList &L, int sms, cudaStream_t s) {
  if (L.n <= 0) return;
  long long most = 0;
  for (int k = 0; k < L.n; ++k) most = most > L.words[k] ? most : L.words[k];
  long long bx = (most / 4 + 255) / 256;
  const long long cap = 8LL * (sms > 0 ? sms : 1);  // grid-stride: any count >= 1 covers the copy
  bx = bx < 1 ? 1 : (bx > cap ? cap : bx);
  k_copy_many<<<dim3((unsigned)bx, (unsigned)L.n), 256, 0, s>>>(L);
}

void launch_probe(const float *F, const long long *nodes, long long npts, float *buf, const long long *clk, int p,
                  cudaStream_t s) {
  k_probe<<<grid_blocks(npts, 256), 256, 0, s>>>(F, nodes, npts, buf, clk, p);
}

void launch_clock_tick(long long *clk, int nprobe, cudaStream_t s) { k_clock_tick<<<1, 32, 0, s>>>(clk, nprobe); }

void launch_clock_set(long long *clk, const ClockState &v, cudaStream_t s) {
  k_clock_set<<<1, BP_MAX_PROBE, 0, s>>>(clk, v);
}
