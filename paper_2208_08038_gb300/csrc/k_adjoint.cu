// k_adjoint.cu -- discrete adjoint of the PIC step (reverse mode), FP32 with
// FP64 parameter-gradient reductions.
//
// Each forward operator is replaced by its transpose or vector-Jacobian
// product, applied in reverse order:
//   E^{n+1} = E^n + dt (curl B^{n+1/2} - J) with Mur faces  ->  k_adj_mur (last
//       pass first) + k_adj_e (gathers curl^T of the interior adjoint, J adjoint)
//   B^{n+1/2} = B^n - dt/2 curl E^n                          ->  k_adj_b
//   per particle: Esirkepov deposit, drift, Boris, internal modified-Coulomb
//       field (arXiv 2208.08038 Sec. 2), gather              ->  k_adj_work
//       (the step's list of 256-ion chunks of the occupied tiles), k_adj_push
//       (recompute of the push; the deposit's transpose reads the current
//       adjoint like a gather; Boris, force and drift transposes; the
//       gather's position derivatives; stores each ion's gathered-field
//       adjoints), k_adj_scatter (the gather's transpose: those adjoints
//       scattered like a deposit into a 64-bit fixed-point box per chunk,
//       added into a per-cell accumulator), k_adj_fxsum (the accumulator
//       converted once and added to the field adjoints, then cleared)
//   B^n = B^{n-1/2} - dt/2 curl E^n                          ->  k_adj_b
// The particle adjoints are indexed by load order, so re-sorting between
// steps does not disturb them.
#include "bp_internal.cuh"
#include "bp_particle.cuh"

namespace {

// 2^k as two factors 2^(k/2) and 2^(k - k/2), each a normal float for
// |k| <= 252: x * f.x * f.y scales by 2^k exactly while x 2^k is a normal
// float (and the intermediate lies between x and the result)
__device__ __forceinline__ float2 pow2_split(int k) {
  const int a = k / 2, b = k - a;
  return make_float2(__int_as_float((127 + a) << 23), __int_as_float((127 + b) << 23));
}

// blocks for n items; the kernels launched with it are grid-stride loops, so
// the cap (two waves of 256-thread blocks on 152 SMs) only bounds the grid
int blocks_for(long long n, int bs) {
  long long b = (n + bs - 1) / bs;
  long long cap = 152LL * 16;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

__device__ __forceinline__ bool ext(const GridP &g, int pat, const int c[3]) {
  bool e = false;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (a < g.D && g.bc[a] == BP_OPEN && ((pat >> a) & 1)) e |= c[a] == g.n[a] - 1;
  return e;
}
__device__ __forceinline__ int nbnd(const GridP &g, int pat, const int c[3], int *first) {
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
__global__ void k_adj_inject(float *lam, const long long *nodes, long long npts, const float *dl) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < npts; q += (long long)gridDim.x * blockDim.x)
    atomicAdd(lam + nodes[q], dl[q]);
}

// Mur faces, one (pass, axis) per launch: E_b(n+1) = E_a(n) + k (E_a(n+1) - E_b(n))
__global__ void k_adj_mur(GridP g, float *G0, float *G1, float *G2, float *H0, float *H1, float *H2, int axis,
                          int pass) {
  float *G[3] = {G0, G1, G2}, *H[3] = {H0, H1, H2};
  const int a = axis;
  const long long F = g.ncell / g.n[a];
  const long long total = 4 * F;  // 2 sides x 2 tangential components
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    long long pos = q % F;
    int t = (int)(q / F);
    int ci = t & 1, side = t >> 1;
    int comp = ci == 0 ? (a == 0 ? 1 : 0) : (a == 2 ? 1 : 2);
    int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
    int lo = o1 < o2 ? o1 : o2, hi = o1 < o2 ? o2 : o1;
    int c[3];
    c[lo] = (int)(pos % g.n[lo]);
    c[hi] = (int)(pos / g.n[lo]);
    c[a] = side == 0 ? 0 : g.n[a] - 1;
    int first;
    if (ext(g, 1 << comp, c)) continue;
    if (nbnd(g, 1 << comp, c, &first) != pass || first != a) continue;
    int ca[3] = {c[0], c[1], c[2]};
    ca[a] += side == 0 ? 1 : -1;
    long long id = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
    long long ida = ca[0] + (long long)g.n[0] * (ca[1] + (long long)g.n[1] * ca[2]);
    float km = (g.dt - g.dx[a]) / (g.dt + g.dx[a]);
    float v = G[comp][id];
    H[comp][ida] += v;
    G[comp][ida] += km * v;
    H[comp][id] -= km * v;
    G[comp][id] = 0.0f;
  }
}

// E node of component comp at coordinates x updated by the interior formula
template <int D>
__device__ __forceinline__ bool e_int(const GridP &g, int comp, const int x[3]) {
  return !exterior_c<D>(g, 1 << comp, x) && !mur_node<D>(g, 1 << comp, x);
}
// Both transposes take four consecutive x cells per thread (float4 loads
// and stores, as the forward Yee kernels); the masks are those of the
// forward update, cell by cell.
//
// G of component comp at cell i of a group (G: the group), at its +1
// neighbour along x (gn: the value after the group's last cell) and along y
// or z (Gu: the group one row or plane up), masked to interior E nodes (0
// off an open face)
template <int D>
__device__ __forceinline__ float g_here4(const GridP &g, const float4 &G, int comp, const int c[3], int i) {
  const int x[3] = {c[0] + i, c[1], c[2]};
  return e_int<D>(g, comp, x) ? el(G, i) : 0.0f;
}
template <int D>
__device__ __forceinline__ float g_up_x4(const GridP &g, const float4 &G, float gn, int comp, const int c[3], int i) {
  int x[3] = {c[0] + i + 1, c[1], c[2]};
  if (x[0] >= g.n[0]) {
    if (g.bc[0] != BP_PERIODIC) return 0.0f;
    x[0] = 0;
  }
  return e_int<D>(g, comp, x) ? (i < 3 ? el(G, i + 1) : gn) : 0.0f;
}
template <int D>
__device__ __forceinline__ float g_up_a4(const GridP &g, const float4 &Gu, int comp, const int c[3], int i, int a) {
  int x[3] = {c[0] + i, c[1], c[2]};
  if (++x[a] >= g.n[a]) {
    if (g.bc[a] != BP_PERIODIC) return 0.0f;
    x[a] = 0;
  }
  return e_int<D>(g, comp, x) ? el(Gu, i) : 0.0f;
}

// interior E update transposed: H += G (interior and exterior nodes),
// lamJ = -dt G (interior), lamB += dt curl_B^T (G on interior nodes)
template <int D>
__global__ void __launch_bounds__(128) k_adj_e(GridP g, const float *G0, const float *G1, const float *G2, float *H0,
                                               float *H1, float *H2, float *B0, float *B1, float *B2, float *J0,
                                               float *J1, float *J2) {
  Cell4 C;
  if (!row_cell4<D>(g, C)) return;
  const long long q = C.q;
  const float dt = g.dt;
  const float4 g0 = ld4(G0 + q), g1 = ld4(G1 + q), g2 = ld4(G2 + q);
  {
    const float4 gg[3] = {g0, g1, g2};
    float *H[3] = {H0, H1, H2}, *J[3] = {J0, J1, J2};
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
      float4 h = ld4(H[comp] + q), j;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int x[3] = {C.c[0] + i, C.c[1], C.c[2]};
        const bool ex = exterior_c<D>(g, 1 << comp, x);
        const bool in = !ex && !mur_node<D>(g, 1 << comp, x);
        const float v = el(gg[comp], i);
        if (in || ex) set_el(h, i, el(h, i) + v);
        set_el(j, i, in ? -dt * v : 0.0f);
      }
      st4(H[comp] + q, h);
      st4(J[comp] + q, j);
    }
  }
  const float g1n = G1[q + C.up[0]], g2n = G2[q + C.up[0]];  // x neighbours of the last cell
  float4 g2y = g2, g0y = g0, g1z = g1, g0z = g0;
  if (D >= 2) {
    g2y = ld4(G2 + q + C.up[1]);
    g0y = ld4(G0 + q + C.up[1]);
  }
  if (D >= 3) {
    g1z = ld4(G1 + q + C.up[2]);
    g0z = ld4(G0 + q + C.up[2]);
  }
  float4 b0 = ld4(B0 + q), b1 = ld4(B1 + q), b2 = ld4(B2 + q);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float bx = 0.0f, by = 0.0f, bz = 0.0f;
    if (D >= 3) bx += (g_here4<D>(g, g1, 1, C.c, i) - g_up_a4<D>(g, g1z, 1, C.c, i, 2)) * g.idx[2];
    if (D >= 2) bx -= (g_here4<D>(g, g2, 2, C.c, i) - g_up_a4<D>(g, g2y, 2, C.c, i, 1)) * g.idx[1];
    if (D >= 3) by -= (g_here4<D>(g, g0, 0, C.c, i) - g_up_a4<D>(g, g0z, 0, C.c, i, 2)) * g.idx[2];
    by += (g_here4<D>(g, g2, 2, C.c, i) - g_up_x4<D>(g, g2, g2n, 2, C.c, i)) * g.idx[0];
    if (D >= 2) bz += (g_here4<D>(g, g0, 0, C.c, i) - g_up_a4<D>(g, g0y, 0, C.c, i, 1)) * g.idx[1];
    bz -= (g_here4<D>(g, g1, 1, C.c, i) - g_up_x4<D>(g, g1, g1n, 1, C.c, i)) * g.idx[0];
    set_el(b0, i, el(b0, i) + dt * bx);
    set_el(b1, i, el(b1, i) + dt * by);
    set_el(b2, i, el(b2, i) + dt * bz);
  }
  st4(B0 + q, b0);
  st4(B1 + q, b1);
  st4(B2 + q, b2);
}

// B adjoint of component stagger pat (6, 5, 3 for x, y, z) at cell i of a
// group (B: the group), at its -1 neighbour along x (bp: the value before the
// group's first cell) and along y or z (Bd: the group one row or plane
// down), masked to non-exterior B nodes (0 off an open face)
template <int D>
__device__ __forceinline__ float b_here4(const GridP &g, const float4 &B, int pat, const int c[3], int i) {
  const int x[3] = {c[0] + i, c[1], c[2]};
  return exterior_c<D>(g, pat, x) ? 0.0f : el(B, i);
}
template <int D>
__device__ __forceinline__ float b_dn_x4(const GridP &g, const float4 &B, float bp, int pat, const int c[3], int i) {
  int x[3] = {c[0] + i - 1, c[1], c[2]};
  if (x[0] < 0) {
    if (g.bc[0] != BP_PERIODIC) return 0.0f;
    x[0] = g.n[0] - 1;
  }
  return exterior_c<D>(g, pat, x) ? 0.0f : (i > 0 ? el(B, i - 1) : bp);
}
template <int D>
__device__ __forceinline__ float b_dn_a4(const GridP &g, const float4 &Bd, int pat, const int c[3], int i, int a) {
  int x[3] = {c[0] + i, c[1], c[2]};
  if (--x[a] < 0) {
    if (g.bc[a] != BP_PERIODIC) return 0.0f;
    x[a] = g.n[a] - 1;
  }
  return exterior_c<D>(g, pat, x) ? 0.0f : el(Bd, i);
}

// B <- B - h curl E transposed: E adjoint -= h curl_E^T (B adjoint on
// non-exterior B nodes); the B adjoint itself passes through.  Z0..Z2, when
// given, are cleared on the way (the buffer the next E transpose fills).
template <int D>
__global__ void __launch_bounds__(128) k_adj_b(GridP g, float *E0, float *E1, float *E2, const float *B0,
                                               const float *B1, const float *B2, float h, float *Z0, float *Z1,
                                               float *Z2) {
  Cell4 C;
  if (!row_cell4<D>(g, C)) return;
  const long long q = C.q;
  const float4 b0 = ld4(B0 + q), b1 = ld4(B1 + q), b2 = ld4(B2 + q);
  const float b1p = B1[q + C.dn[0]], b2p = B2[q + C.dn[0]];  // x neighbours of the first cell
  float4 b1z = b1, b2y = b2, b0z = b0, b0y = b0;
  if (D >= 2) {
    b2y = ld4(B2 + q + C.dn[1]);
    b0y = ld4(B0 + q + C.dn[1]);
  }
  if (D >= 3) {
    b1z = ld4(B1 + q + C.dn[2]);
    b0z = ld4(B0 + q + C.dn[2]);
  }
  float4 e0 = ld4(E0 + q), e1 = ld4(E1 + q), e2 = ld4(E2 + q);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float ex = 0.0f, ey = 0.0f, ez = 0.0f;
    if (D >= 3) ex += (b_dn_a4<D>(g, b1z, 5, C.c, i, 2) - b_here4<D>(g, b1, 5, C.c, i)) * g.idx[2];
    if (D >= 2) ex -= (b_dn_a4<D>(g, b2y, 3, C.c, i, 1) - b_here4<D>(g, b2, 3, C.c, i)) * g.idx[1];
    if (D >= 3) ey -= (b_dn_a4<D>(g, b0z, 6, C.c, i, 2) - b_here4<D>(g, b0, 6, C.c, i)) * g.idx[2];
    ey += (b_dn_x4<D>(g, b2, b2p, 3, C.c, i) - b_here4<D>(g, b2, 3, C.c, i)) * g.idx[0];
    if (D >= 2) ez += (b_dn_a4<D>(g, b0y, 6, C.c, i, 1) - b_here4<D>(g, b0, 6, C.c, i)) * g.idx[1];
    ez -= (b_dn_x4<D>(g, b1, b1p, 5, C.c, i) - b_here4<D>(g, b1, 5, C.c, i)) * g.idx[0];
    set_el(e0, i, el(e0, i) - h * ex);
    set_el(e1, i, el(e1, i) - h * ey);
    set_el(e2, i, el(e2, i) - h * ez);
  }
  st4(E0 + q, e0);
  st4(E1 + q, e1);
  st4(E2 + q, e2);
  if (Z0) {
    const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    st4(Z0 + q, z);
    st4(Z1 + q, z);
    st4(Z2 + q, z);
  }
}

// ---------------------------------------------------------------------------
// particles

__device__ __forceinline__ float dqshape(float x) {
  float a = fabsf(x);
  if (a <= 0.5f) return -2.0f * x;
  if (a < 1.5f) return (x > 0.0f ? -1.0f : 1.0f) * (1.5f - a);
  return 0.0f;
}

// reverse of boris(): given the adjoint of the pushed momentum, the adjoints
// of the old momentum, E and B
__device__ __forceinline__ void boris_adj(float h, const float E[3], const float B[3], const float u0[3], const float ubn[3],
                          float ub0[3], float Eb[3], float Bb[3]) {
  float um[3], t[3], sv[3], c1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) um[a] = u0[a] + h * E[a];
  float gm = sqrtf(1.0f + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) t[a] = h * B[a] / gm;
  float t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) sv[a] = 2.0f * t[a] / (1.0f + t2);
  c1[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
  c1[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
  c1[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
  float umb[3], cb[3], sb[3], tb[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Eb[a] = h * ubn[a];
    umb[a] = ubn[a];
  }
  cb[0] = sv[1] * ubn[2] - sv[2] * ubn[1];
  cb[1] = sv[2] * ubn[0] - sv[0] * ubn[2];
  cb[2] = sv[0] * ubn[1] - sv[1] * ubn[0];
  sb[0] = ubn[1] * c1[2] - ubn[2] * c1[1];
  sb[1] = ubn[2] * c1[0] - ubn[0] * c1[2];
  sb[2] = ubn[0] * c1[1] - ubn[1] * c1[0];
  umb[0] += cb[0] + (t[1] * cb[2] - t[2] * cb[1]);
  umb[1] += cb[1] + (t[2] * cb[0] - t[0] * cb[2]);
  umb[2] += cb[2] + (t[0] * cb[1] - t[1] * cb[0]);
  tb[0] = cb[1] * um[2] - cb[2] * um[1];
  tb[1] = cb[2] * um[0] - cb[0] * um[2];
  tb[2] = cb[0] * um[1] - cb[1] * um[0];
  float ts = t[0] * sb[0] + t[1] * sb[1] + t[2] * sb[2];
  float i1 = 1.0f / (1.0f + t2);
#pragma unroll
  for (int a = 0; a < 3; ++a) tb[a] += 2.0f * sb[a] * i1 - 4.0f * t[a] * ts * i1 * i1;
  float gmb = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Bb[a] = h * tb[a] / gm;
    gmb -= h * B[a] * tb[a] / (gm * gm);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    umb[a] += um[a] * gmb / gm;
    ub0[a] = umb[a];
    Eb[a] += h * umb[a];
  }
}

// Gather transposed, part 1: the derivatives of the gathered fields with
// respect to the bodies' positions, taken with the forward recompute (the
// field adjoints that weight them come later, from the Boris transpose).
// Part 2, the scatter of e w into the field adjoints, is the separate kernel
// k_adj_scatter (fixed point, exact and order-free).
//
// One gathered component (stagger PAT) at one body, with its derivatives
// with respect to the body's position (in cells) along each simulated axis:
// the value by the forward gather's arithmetic (the same contractions in the
// same order: x, then y, then z), the derivatives from the same node loads
// with the weights' derivatives in place of the weights along one axis.
template <int D, int PAT>
__device__ __forceinline__ float gather_vd(const float *__restrict__ G, const int d[3], const float f[3],
                                           float dv[3]) {
  int b[3];
  float w[3][3], dw[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < D) {
      const bool half = (PAT >> a) & 1;
      float xi;
      if (half) {
        b[a] = d[a] + Box<D>::OG - 1;
        xi = f[a] - 0.5f;
      } else {
        const int up = f[a] >= 0.5f ? 1 : 0;
        b[a] = d[a] + Box<D>::OG + up - 1;
        xi = f[a] - (float)up;
      }
      qweights(xi, w[a]);
      dw[a][0] = -(0.5f - xi);
      dw[a][1] = -2.0f * xi;
      dw[a][2] = 0.5f + xi;
    } else {
      b[a] = 0;
      w[a][0] = 1.0f;
      w[a][1] = w[a][2] = 0.0f;
      dw[a][0] = dw[a][1] = dw[a][2] = 0.0f;
    }
  }
  constexpr int NJ = D >= 2 ? 3 : 1, NK = D >= 3 ? 3 : 1;
  float sa = 0.0f, sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
  for (int k = 0; k < NK; ++k) {
    float pa = 0.0f, px = 0.0f, py = 0.0f;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const float *row = G + Box<D>::gi(b[0], b[1] + j, b[2] + k);
      float ra = 0.0f, rd = 0.0f;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const float v = row[i];
        ra = fmaf(w[0][i], v, ra);
        rd = fmaf(dw[0][i], v, rd);
      }
      pa = fmaf(w[1][j], ra, pa);
      px = fmaf(w[1][j], rd, px);
      py = fmaf(dw[1][j], ra, py);
    }
    sa = fmaf(w[2][k], pa, sa);
    sx = fmaf(w[2][k], px, sx);
    sy = fmaf(w[2][k], py, sy);
    sz = fmaf(dw[2][k], pa, sz);
  }
  dv[0] = sx;
  dv[1] = sy;
  dv[2] = sz;
  return sa;
}

// the six components at one body (E_x, E_y, E_z, B_x, B_y, B_z), their
// derivatives to the thread's slice of shared memory: component q, axis a
// at dst[(q D + a) * stride]
template <int D>
__device__ __forceinline__ void gather_vd_body(const float *G, const int d[3], const float f[3], float E[3], float B[3],
                                               float *dst, int stride) {
  constexpr int gc = Box<D>::GCELLS;
  float dv[3];
  auto put = [&](int q) {
#pragma unroll
    for (int a = 0; a < D; ++a) dst[(q * D + a) * stride] = dv[a];
  };
  E[0] = gather_vd<D, 1>(G + 0 * gc, d, f, dv); put(0);
  E[1] = gather_vd<D, 2>(G + 1 * gc, d, f, dv); put(1);
  E[2] = gather_vd<D, 4>(G + 2 * gc, d, f, dv); put(2);
  B[0] = gather_vd<D, 6>(G + 3 * gc, d, f, dv); put(3);
  B[1] = gather_vd<D, 5>(G + 4 * gc, d, f, dv); put(4);
  B[2] = gather_vd<D, 3>(G + 5 * gc, d, f, dv); put(5);
}

// Esirkepov transposed on a window of W nodes per axis (W = 3: every
// position keeps one nearest node; W = 5: general), for NB bodies sharing the
// window: reads the current adjoint lam once (like a gather) and returns, per
// body, d(lam . J)/dX0, /dX1 (cells) and /dv.  S0 = S(xi - m), DS = S(xi + de -
// m) - S(xi - m) on the window; then X0b = sum (gS0 - gDS) S'(xi - m),
// X1b = sum gDS S'(xi + de - m).
template <int D, int W, int NB>
__device__ __forceinline__ void deposit_adj(const float *__restrict__ Jl, const int n0[3], const float (*xi)[3],
                            const float (*de)[3], const float *qw, const float (*v)[3], const float dxdt[3],
                            float (*X0b)[3], float (*X1b)[3], float (*vb)[3]) {
  constexpr int jc = Box<D>::JCELLS;
  constexpr int H = W / 2;  // window nodes n0 - H .. n0 + H
  float S0[NB][3][W], DS[NB][3][W], gS0[NB][3][W], gDS[NB][3][W];
#pragma unroll
  for (int q = 0; q < NB; ++q)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int m = 0; m < W; ++m) {
        if (a < D && W == 3) {
          // every position keeps its nearest node: closed forms in xi and
          // the move d (as in the forward fast path)
          const float x = xi[q][a], dd = de[q][a];
          float w3[3];
          qweights(x, w3);
          S0[q][a][m] = w3[m];
          DS[q][a][m] = m == 0 ? -0.5f * dd * (1.0f - 2.0f * x - dd)
                               : (m == 1 ? -dd * (2.0f * x + dd) : 0.5f * dd * (1.0f + 2.0f * x + dd));
        } else if (a < D) {
          const float u = xi[q][a] - (float)(m - H);
          S0[q][a][m] = qshape(u);
          DS[q][a][m] = qshape(u + de[q][a]) - S0[q][a][m];
        } else {
          S0[q][a][m] = m == H ? 1.0f : 0.0f;
          DS[q][a][m] = 0.0f;
        }
        gS0[q][a][m] = gDS[q][a][m] = 0.0f;
      }
  const int bx = n0[0] - H, by = D >= 2 ? n0[1] - H : 0, bz = D >= 3 ? n0[2] - H : 0;
  auto L = [&](int comp, int i, int j, int k) -> float {
    return Jl[comp * jc + Box<D>::ji(bx + i, by + j, bz + k)];
  };
  if constexpr (D == 1) {
    float suf = 0.0f;
#pragma unroll
    for (int i = W - 2; i >= 0; --i) {
      suf += L(0, i, 0, 0);
#pragma unroll
      for (int q = 0; q < NB; ++q) gDS[q][0][i] += -qw[q] * dxdt[0] * suf;
    }
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const float ly = L(1, i, 0, 0), lz = L(2, i, 0, 0);
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        const float sbar = S0[q][0][i] + 0.5f * DS[q][0][i];
        const float t = qw[q] * (v[q][1] * ly + v[q][2] * lz);
        gS0[q][0][i] += t;
        gDS[q][0][i] += 0.5f * t;
        vb[q][1] += qw[q] * ly * sbar;
        vb[q][2] += qw[q] * lz * sbar;
      }
    }
  } else if constexpr (D == 2) {
    // J_x on faces i (W - 1 of them) at rows j, J_y likewise with axes swapped
#pragma unroll
    for (int ax = 0; ax < 2; ++ax) {
      const int ox = 1 - ax;  // the other axis
#pragma unroll
      for (int t = 0; t < W; ++t) {
        float lv[W - 1];
#pragma unroll
        for (int s = 0; s < W - 1; ++s) lv[s] = ax == 0 ? L(0, s, t, 0) : L(1, t, s, 0);
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          const float c = -qw[q] * dxdt[ax];
          const float fac = S0[q][ox][t] + 0.5f * DS[q][ox][t];
          float suf = 0.0f, P = 0.0f, sumLP = 0.0f;
#pragma unroll
          for (int s = W - 2; s >= 0; --s) {
            suf += lv[s];
            gDS[q][ax][s] += c * suf * fac;
          }
#pragma unroll
          for (int s = 0; s < W - 1; ++s) {
            P += DS[q][ax][s];
            sumLP += lv[s] * P;
          }
          gS0[q][ox][t] += c * sumLP;
          gDS[q][ox][t] += 0.5f * c * sumLP;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < W; ++j)
#pragma unroll
      for (int i = 0; i < W; ++i) {
        const float l = L(2, i, j, 0);
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          const float wz = S0[q][0][i] * S0[q][1][j] + 0.5f * (DS[q][0][i] * S0[q][1][j] + S0[q][0][i] * DS[q][1][j]) +
                           (1.0f / 3.0f) * DS[q][0][i] * DS[q][1][j];
          const float c = qw[q] * v[q][2] * l;
          vb[q][2] += qw[q] * l * wz;
          gS0[q][0][i] += c * (S0[q][1][j] + 0.5f * DS[q][1][j]);
          gDS[q][0][i] += c * (0.5f * S0[q][1][j] + (1.0f / 3.0f) * DS[q][1][j]);
          gS0[q][1][j] += c * (S0[q][0][i] + 0.5f * DS[q][0][i]);
          gDS[q][1][j] += c * (0.5f * S0[q][0][i] + (1.0f / 3.0f) * DS[q][0][i]);
        }
      }
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int b = (a + 1) % 3, c = (a + 2) % 3;
#pragma unroll 1
      for (int kb = 0; kb < W; ++kb)
#pragma unroll 1
        for (int kc = 0; kc < W; ++kc) {
          float lv[W - 1];
#pragma unroll
          for (int ka = 0; ka < W - 1; ++ka) {
            int idx[3];
            idx[a] = ka;
            idx[b] = kb;
            idx[c] = kc;
            lv[ka] = L(a, idx[0], idx[1], idx[2]);
          }
#pragma unroll
          for (int q = 0; q < NB; ++q) {
            const float ca = -qw[q] * dxdt[a];
            const float fac = S0[q][b][kb] * S0[q][c][kc] +
                              0.5f * (DS[q][b][kb] * S0[q][c][kc] + S0[q][b][kb] * DS[q][c][kc]) +
                              (1.0f / 3.0f) * DS[q][b][kb] * DS[q][c][kc];
            float suf = 0.0f, P = 0.0f, sumLP = 0.0f;
#pragma unroll
            for (int ka = W - 2; ka >= 0; --ka) {
              suf += lv[ka];
              gDS[q][a][ka] += ca * suf * fac;
            }
#pragma unroll
            for (int ka = 0; ka < W - 1; ++ka) {
              P += DS[q][a][ka];
              sumLP += lv[ka] * P;
            }
            gS0[q][b][kb] += ca * sumLP * (S0[q][c][kc] + 0.5f * DS[q][c][kc]);
            gDS[q][b][kb] += ca * sumLP * (0.5f * S0[q][c][kc] + (1.0f / 3.0f) * DS[q][c][kc]);
            gS0[q][c][kc] += ca * sumLP * (S0[q][b][kb] + 0.5f * DS[q][b][kb]);
            gDS[q][c][kc] += ca * sumLP * (0.5f * S0[q][b][kb] + (1.0f / 3.0f) * DS[q][b][kb]);
          }
        }
    }
  }
#pragma unroll
  for (int q = 0; q < NB; ++q)
#pragma unroll
    for (int a = 0; a < D; ++a) {
      float x0 = 0.0f, x1 = 0.0f;
#pragma unroll
      for (int m = 0; m < W; ++m) {
        float d0, d1;
        if (W == 3) {
          // S'(x - node) on the three nodes around the nearest one
          const float x = xi[q][a], y = x + de[q][a];
          d0 = m == 0 ? -(0.5f - x) : (m == 1 ? -2.0f * x : 0.5f + x);
          d1 = m == 0 ? -(0.5f - y) : (m == 1 ? -2.0f * y : 0.5f + y);
        } else {
          const float u = xi[q][a] - (float)(m - H);
          d0 = dqshape(u);
          d1 = dqshape(u + de[q][a]);
        }
        x0 += (gS0[q][a][m] - gDS[q][a][m]) * d0;
        x1 += gDS[q][a][m] * d1;
      }
      X0b[q][a] += x0;
      X1b[q][a] += x1;
    }
}

// the rare case out of line, its inputs and results in one object built
// inside the rare branch (the fast path's arrays stay in registers)
struct AdjGen {
  int nn[3], n2[3];
  float xi[2][3], dd[2][3], qw[2], vv[2][3], dxdt[3];
  float X0[2][3], X1[2][3], vb[2][3];
  int two;
};

template <int D>
__device__ __noinline__ void deposit_adj_general(const float *Jl, AdjGen &A) {
  deposit_adj<D, 5, 1>(Jl, A.nn, A.xi, A.dd, A.qw, A.vv, A.dxdt, A.X0, A.X1, A.vb);
  if (A.two) deposit_adj<D, 5, 1>(Jl, A.n2, A.xi + 1, A.dd + 1, A.qw + 1, A.vv + 1, A.dxdt, A.X0 + 1, A.X1 + 1, A.vb + 1);
}

// The step's work: every occupied tile's particles of each species, cut
// into chunks of at most `chunk` particles; an item is (tile, species,
// first, end) in the stored particle arrays.  k_adj_push and k_adj_scatter
// hand the items to their resident blocks round-robin, so the blocks stay
// busy whatever the number of occupied tiles and their populations.  Each
// particle's results depend on the particle alone (its adjoint state is
// written by load id, its field-adjoint adds are exact integers), so the
// order of the list, which the appends leave open, changes nothing.
struct AdjWork {
  int *n;       // items in the list (cleared by k_adj_fxsum)
  int4 *item;
  int cap;
};

struct AdjState {
  float *xb;      // [12][cap] by load id: x1b(3) x2b(3) u1b(3) u2b(3)
  double *acb;    // [cap] adjoint of a_c, accumulated over steps
  float *eb;      // [12][cap] by slot: adjoints of the gathered E1 B1 E2 B2 (this step)
  long long cap;
  int *status;    // the reverse pass's status word (ST_DOMAIN)
};

struct AdjArgs {
  int nsp;
  SpecP sp[BP_MAX_SPECIES];
  PartP p[BP_MAX_SPECIES];       // particle state of step n
  AdjState st[BP_MAX_SPECIES];
  const float *E[3], *B[3];      // E^n, B^n
  const float *lamJ[3];
  unsigned *emax;                // largest |gathered-field adjoint| of the step (float bits)
};

template <int D>
__device__ void adj_particle(const GridP &g, const SpecP &sp, const PartP &P, AdjState &S, long long i,
                             const int T0[3], const float *Gsm, const float *Jl, float *stash, float &emax) {
  const long long cap = P.cap;
  const bool two = sp.kind == BP_TWO_BODY;
  const int cell = P.cell[i];
  if (cell < 0) return;
  const int id = P.id[i];
  int c[3];
  unpack_cell(g, cell, c);
  float f[3] = {0.0f, 0.0f, 0.0f}, r[3] = {0.0f, 0.0f, 0.0f}, u1[3], u2[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int a = 0; a < D; ++a) f[a] = P.off[a * cap + i];
#pragma unroll
  for (int a = 0; a < 3; ++a) u1[a] = P.u1[a * cap + i];
  if (two) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      r[a] = P.r[a * cap + i];
      u2[a] = P.u2[a * cap + i];
    }
  }
  int d[3] = {0, 0, 0}, d2[3] = {0, 0, 0};
  float f2[3] = {0.0f, 0.0f, 0.0f};
  bool bad = false;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    d[a] = rel_cell<D>(g, a, c[a], T0[a]);
    bad |= outside_margin<D>(a, d[a]) || !(fabsf(r[a] * g.idx[a]) < 1.0f);
    float X = f[a] - r[a] * g.idx[a];
    float fl = floorf(X);
    float fr = X - fl;
    int di = (int)fl;
    if (fr >= 1.0f) { fr = 0.0f; di += 1; }
    d2[a] = d[a] + di;
    f2[a] = fr;
  }
  if (bad) {
    // a body outside the tile's reach: the forward push either skipped it
    // (a domain error) or, for a bound electron a cell or more from its
    // nucleus, moved it on the global grid, which this reverse step does not
    // follow: reported, never skipped silently
    atomicOr(S.status, ST_DOMAIN);
    return;
  }
  // forward recompute: the gathered fields, and their derivatives with
  // respect to the bodies' positions kept in the thread's slice of shared
  // memory for the gather's transpose below
  float E1[3], B1[3], E2[3] = {0.0f, 0.0f, 0.0f}, B2[3] = {0.0f, 0.0f, 0.0f};
  float *dvs = stash + threadIdx.x;
  gather_vd_body<D>(Gsm, d, f, E1, B1, dvs, blockDim.x);
  if (two) gather_vd_body<D>(Gsm, d2, f2, E2, B2, dvs + 6 * D * blockDim.x, blockDim.x);
  float ac = 0.0f, rr = 1.0f, s3 = 0.0f;
  if (two) {
    const int pi = P.pidx ? P.pidx[i] : 0;
    ac = sp.ac[pi];
    rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + ac * ac;
    float rs = rsqrtf(rr);
    s3 = sp.kappa * rs * rs * rs;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      E1[a] = fmaf(sp.q2 * s3, r[a], E1[a]);
      E2[a] = fmaf(-sp.q1 * s3, r[a], E2[a]);
    }
  }
  float un1[3] = {u1[0], u1[1], u1[2]}, un2[3] = {u2[0], u2[1], u2[2]};
  boris(sp.h1, E1, B1, un1);
  if (two) boris(sp.h2, E2, B2, un2);
  float gi1 = rsqrtf(1.0f + un1[0] * un1[0] + un1[1] * un1[1] + un1[2] * un1[2]);
  float gi2 = rsqrtf(1.0f + un2[0] * un2[0] + un2[1] * un2[1] + un2[2] * un2[2]);
  float v1[3], v2[3], de1[3] = {0.0f, 0.0f, 0.0f}, de2[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v1[a] = un1[a] * gi1;
    v2[a] = un2[a] * gi2;
    if (a < D) {
      de1[a] = g.dt * v1[a] * g.idx[a];
      de2[a] = g.dt * v2[a] * g.idx[a];
    }
  }
  const float dxdt[3] = {g.dx[0] / g.dt, g.dx[1] / g.dt, g.dx[2] / g.dt};
  // deposit transposed: three-node window shared by both bodies when every
  // position keeps one nearest node, else five-node windows per body
  float X10b[3] = {0, 0, 0}, X11b[3] = {0, 0, 0}, X20b[3] = {0, 0, 0}, X21b[3] = {0, 0, 0};
  float v1b[3] = {0, 0, 0}, v2b[3] = {0, 0, 0};
  {
    bool fast = true;
    float xi[2][3] = {{0, 0, 0}, {0, 0, 0}}, dd[2][3], vv[2][3];
    int nn[3] = {2, 2, 2}, n2[3] = {2, 2, 2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dd[0][a] = de1[a];
      dd[1][a] = de2[a];
      vv[0][a] = v1[a];
      vv[1][a] = v2[a];
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int up1 = f[a] >= 0.5f ? 1 : 0, up2 = f2[a] >= 0.5f ? 1 : 0;
      xi[0][a] = f[a] - (float)up1;
      xi[1][a] = f2[a] - (float)up2;
      nn[a] = d[a] + Box<D>::OJ + up1;
      n2[a] = d2[a] + Box<D>::OJ + up2;
      const float x1n = xi[0][a] + de1[a], x2n = xi[1][a] + de2[a];
      fast &= x1n >= -0.5f && x1n < 0.5f;
      if (two) fast &= nn[a] == n2[a] && x2n >= -0.5f && x2n < 0.5f;
    }
    const float qw[2] = {sp.qw1, sp.qw2};
    float X0[2][3] = {{0, 0, 0}, {0, 0, 0}}, X1[2][3] = {{0, 0, 0}, {0, 0, 0}}, vb[2][3] = {{0, 0, 0}, {0, 0, 0}};
    if (fast && two) {
      deposit_adj<D, 3, 2>(Jl, nn, xi, dd, qw, vv, dxdt, X0, X1, vb);
    } else if (fast) {
      deposit_adj<D, 3, 1>(Jl, nn, xi, dd, qw, vv, dxdt, X0, X1, vb);
    } else {
      AdjGen G;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        G.nn[a] = nn[a]; G.n2[a] = n2[a]; G.dxdt[a] = dxdt[a];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          G.xi[q][a] = xi[q][a]; G.dd[q][a] = dd[q][a]; G.vv[q][a] = vv[q][a];
          G.X0[q][a] = G.X1[q][a] = G.vb[q][a] = 0.0f;
        }
      }
      G.qw[0] = qw[0];
      G.qw[1] = qw[1];
      G.two = two;
      deposit_adj_general<D>(Jl, G);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          X0[q][a] = G.X0[q][a]; X1[q][a] = G.X1[q][a]; vb[q][a] = G.vb[q][a];
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      X10b[a] = X0[0][a]; X11b[a] = X1[0][a]; v1b[a] = vb[0][a];
      X20b[a] = X0[1][a]; X21b[a] = X1[1][a]; v2b[a] = vb[1][a];
    }
  }
  // carried adjoints of x^{n+1}, u^{n+1/2}
  const long long sc = S.cap;
  float xb1[3], xb2[3], ub1[3], ub2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    xb1[a] = S.xb[(0 + a) * sc + id];
    xb2[a] = S.xb[(3 + a) * sc + id];
    ub1[a] = S.xb[(6 + a) * sc + id];
    ub2[a] = S.xb[(9 + a) * sc + id];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    xb1[a] += X11b[a] * g.idx[a];
    xb2[a] += X21b[a] * g.idx[a];
  }
  // drift x^{n+1} = x^n + dt v: v adjoint; v = u / gamma
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v1b[a] += g.dt * xb1[a];
    v2b[a] += g.dt * xb2[a];
  }
  float uv1 = un1[0] * v1b[0] + un1[1] * v1b[1] + un1[2] * v1b[2];
  float uv2 = un2[0] * v2b[0] + un2[1] * v2b[1] + un2[2] * v2b[2];
  float g31 = gi1 * gi1 * gi1, g32 = gi2 * gi2 * gi2;
  float unb1[3], unb2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    unb1[a] = ub1[a] + v1b[a] * gi1 - un1[a] * uv1 * g31;
    unb2[a] = ub2[a] + v2b[a] * gi2 - un2[a] * uv2 * g32;
  }
  // Boris transposed
  float Eb1[3], Bb1[3], Eb2[3] = {0, 0, 0}, Bb2[3] = {0, 0, 0};
  boris_adj(sp.h1, E1, B1, u1, unb1, ub1, Eb1, Bb1);
  if (two) boris_adj(sp.h2, E2, B2, u2, unb2, ub2, Eb2, Bb2);
  // internal field transposed: w = q2 Eb1 - q1 Eb2 against kappa r rho^{-3/2}
  if (two) {
    float w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) w[a] = sp.q2 * Eb1[a] - sp.q1 * Eb2[a];
    float wr = w[0] * r[0] + w[1] * r[1] + w[2] * r[2];
    float p52 = s3 / (sp.kappa * rr);  // rho^{-5/2}
    float p32 = s3 / sp.kappa;         // rho^{-3/2}
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float rb = sp.kappa * (w[a] * p32 - 3.0f * wr * r[a] * p52);
      xb1[a] += rb;
      xb2[a] -= rb;
    }
    S.acb[id] += (double)(-3.0f * sp.kappa * wr * ac * p52);
  }
  // gather transposed: position derivatives here, the field-adjoint scatter
  // by k_adj_scatter from the stored Eb, Bb; old positions through the deposit
  float Xg1[3] = {0, 0, 0}, Xg2[3] = {0, 0, 0};
  {
    const float e1[6] = {Eb1[0], Eb1[1], Eb1[2], Bb1[0], Bb1[1], Bb1[2]};
    const float e2[6] = {Eb2[0], Eb2[1], Eb2[2], Bb2[0], Bb2[1], Bb2[2]};
#pragma unroll
    for (int q = 0; q < 6; ++q)
#pragma unroll
      for (int a = 0; a < D; ++a) Xg1[a] += e1[q] * dvs[(q * D + a) * blockDim.x];
    if (two)
#pragma unroll
      for (int q = 0; q < 6; ++q)
#pragma unroll
        for (int a = 0; a < D; ++a) Xg2[a] += e2[q] * dvs[((6 + q) * D + a) * blockDim.x];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    S.eb[(0 + a) * sc + i] = Eb1[a];
    S.eb[(3 + a) * sc + i] = Bb1[a];
    S.eb[(6 + a) * sc + i] = Eb2[a];
    S.eb[(9 + a) * sc + i] = Bb2[a];
    emax = fmaxf(emax, fmaxf(fmaxf(fabsf(Eb1[a]), fabsf(Bb1[a])), fmaxf(fabsf(Eb2[a]), fabsf(Bb2[a]))));
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    xb1[a] += (Xg1[a] + X10b[a]) * g.idx[a];
    xb2[a] += (Xg2[a] + X20b[a]) * g.idx[a];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    S.xb[(0 + a) * sc + id] = xb1[a];
    S.xb[(3 + a) * sc + id] = two ? xb2[a] : 0.0f;
    S.xb[(6 + a) * sc + id] = ub1[a];
    S.xb[(9 + a) * sc + id] = two ? ub2[a] : 0.0f;
  }
}

// one thread per tile and species: the chunks of its particles appended
__global__ void k_adj_work(GridP g, AdjArgs A, AdjWork W, int chunk) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= g.ntiles * A.nsp) return;
  const int t = q % g.ntiles, s = q / g.ntiles;
  const int beg = A.p[s].tstart[t], end = A.p[s].tstart[t + 1];
  if (end <= beg) return;
  const int m = (end - beg + chunk - 1) / chunk;
  const int at = atomicAdd(W.n, m);
  for (int k = 0; k < m && at + k < W.cap; ++k)
    W.item[at + k] = make_int4(t, s, beg + k * chunk, min(beg + (k + 1) * chunk, end));
}

// The staged boxes of tile t: E^n, B^n (gather box) and the J adjoint, as
// per-thread asynchronous 4-byte copies (zero fill outside open faces),
// completed by cp.async.wait_all; T0 receives the tile's first cell.
template <int D>
__device__ __forceinline__ void adj_stage(const GridP &g, const AdjArgs &A, int t, int T0[3], float *Gsm, float *Jl) {
  using BX = Box<D>;
  constexpr int GC = BX::GCELLS, JC = BX::JCELLS;
  const int tid = threadIdx.x, bs = blockDim.x;
  const int tc[3] = {t % g.nt[0], (t / g.nt[0]) % g.nt[1], t / (g.nt[0] * g.nt[1])};
  T0[0] = tc[0] * Geo<D>::L0;
  T0[1] = tc[1] * Geo<D>::L1;
  T0[2] = tc[2] * Geo<D>::L2;
  const unsigned gbase = (unsigned)__cvta_generic_to_shared(Gsm), jbase = (unsigned)__cvta_generic_to_shared(Jl);
  for (int q = tid; q < BX::GCOMP; q += bs) {
    int bidx[3] = {q % BX::G0, (q / BX::G0) % BX::G1, q / (BX::G0 * BX::G1)};
    const int si = BX::gi(bidx[0], bidx[1], bidx[2]);
    long long gi = 0, stride = 1;
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int x = T0[a] - (a < D ? BX::OG : 0) + bidx[a];
      if (a < D) {
        if (g.bc[a] == BP_PERIODIC) x = wrap_once(x, g.n[a]);
        else ok &= (x >= 0 && x < g.n[a]);
      }
      gi += (long long)x * stride;
      stride *= g.n[a];
    }
    if (!ok) gi = 0;  // a zero fill: nothing is read
    const unsigned src = ok ? 4u : 0u;
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) {
      const float *gp = (cc < 3 ? A.E[cc] : A.B[cc - 3]) + gi;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(gbase + 4u * (unsigned)(cc * GC + si)),
                   "l"(gp), "r"(src)
                   : "memory");
    }
  }
  for (int q = tid; q < BX::JCOMP; q += bs) {
    int bidx[3] = {q % BX::J0, (q / BX::J0) % BX::J1, q / (BX::J0 * BX::J1)};
    const int si = BX::ji(bidx[0], bidx[1], bidx[2]);
    long long gi = 0, stride = 1;
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int x = T0[a] - (a < D ? BX::OJ : 0) + bidx[a];
      if (a < D) {
        if (g.bc[a] == BP_PERIODIC) x = wrap_once(x, g.n[a]);
        else ok &= (x >= 0 && x < g.n[a]);
      }
      gi += (long long)x * stride;
      stride *= g.n[a];
    }
    if (!ok) gi = 0;
    const unsigned src = ok ? 4u : 0u;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(jbase + 4u * (unsigned)(cc * JC + si)),
                   "l"(A.lamJ[cc] + gi), "r"(src)
                   : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// box sets of the reversed push in shared memory: two in 1D and 2D (the next
// work item's boxes are staged while the current item is processed), one in
// 3D (a set fills most of the shared memory)
__host__ __device__ constexpr int adj_push_bufs(int D) { return D == 3 ? 1 : 2; }
template <int D>
__host__ __device__ constexpr int adj_box_floats() {
  return 6 * Box<D>::GCELLS + 3 * Box<D>::JCELLS;
}

// the reversed push of the step's work items, round-robin over the
// resident blocks
template <int D>
__global__ void __launch_bounds__(256, D == 3 ? 1 : 2) k_adj_push(GridP g, AdjArgs A, AdjWork W) {
  using BX = Box<D>;
  constexpr int GC = BX::GCELLS, NB = adj_push_bufs(D), BOX = adj_box_floats<D>();
  extern __shared__ __align__(16) unsigned char smem[];
  float *buf = reinterpret_cast<float *>(smem);  // NB x [E^n, B^n (6 GC) | J adjoint (3 JC)]
  float *stash = buf + NB * BOX;                 // [12 D][blockDim]: the gather's position derivatives
  const int tid = threadIdx.x, bs = blockDim.x;
  const int nw = min(*W.n, W.cap);
  float emax = 0.0f;
  int w = blockIdx.x, cur = 0, T0[3], Tn[3];
  if (w < nw) {
    int4 it = W.item[w];
    adj_stage<D>(g, A, it.x, T0, buf, buf + 6 * GC);
    for (;;) {
      const int wn = w + (int)gridDim.x;
      const bool more = wn < nw;
      const int4 nx = more ? W.item[wn] : make_int4(0, 0, 0, 0);
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();  // the current boxes have landed; the other set is no longer read
      float *Gsm = buf + cur * BOX;
      if (NB == 2 && more) adj_stage<D>(g, A, nx.x, Tn, buf + (cur ^ 1) * BOX, buf + (cur ^ 1) * BOX + 6 * GC);
      const int s = it.y;
      for (long long i = it.z + tid; i < it.w; i += bs)
        adj_particle<D>(g, A.sp[s], A.p[s], A.st[s], i, T0, Gsm, Gsm + 6 * GC, stash, emax);
      if (!more) break;
      if (NB == 1) {
        __syncthreads();  // every thread is done with the set before it is restaged
        adj_stage<D>(g, A, nx.x, Tn, buf, buf + 6 * GC);
      }
      it = nx;
      w = wn;
      T0[0] = Tn[0];
      T0[1] = Tn[1];
      T0[2] = Tn[2];
      if (NB == 2) cur ^= 1;
    }
  }
  // non-negative floats order like their bit patterns
  const unsigned m = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(emax));
  if ((tid & 31) == 0 && m) atomicMax(A.emax, m);
}

// Gather transposed, part 2: scatter the stored field adjoints e of both
// bodies with the gather weights, in 64-bit fixed point (exact, independent
// of the order of the adds; the scale puts the step's largest |e| at 2^30,
// so a quantum is below 1e-9 of it).  A block takes a work item (a chunk of
// one tile's particles), adds into the tile's box in shared memory with the
// forward deposit's split (fx_add: non-returning 32-bit shared atomics, the
// high word only when needed), then adds the box's non-zero nodes into the
// per-cell 64-bit accumulator lfx (integer adds: exact in any order) and
// marks the tiles the box reaches; k_adj_fxsum converts the marked tiles'
// cells once to FP32 and adds them to the field adjoints.
struct ScatArgs {
  int nsp;
  SpecP sp[BP_MAX_SPECIES];
  PartP p[BP_MAX_SPECIES];
  const float *eb[BP_MAX_SPECIES];
  long long ecap[BP_MAX_SPECIES];
  const unsigned *emax;
  unsigned long long *lfx;  // [6][ncell] field-adjoint sums, fixed point, scale 2^k
  unsigned char *dirty;     // [ntiles] a box added into the tile's cells
  int *kst;                 // k of this step, for k_adj_fxsum
};

// stencil base and weights of component PAT at one body
template <int D, int PAT>
__device__ __forceinline__ void scat_loc(const int d[3], const float f[3], int b[3], float w[3][3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < D) {
      const bool half = (PAT >> a) & 1;
      const int up = half ? 0 : (f[a] >= 0.5f ? 1 : 0);
      b[a] = d[a] + Box<D>::OG + up - 1;
      qweights(half ? f[a] - 0.5f : f[a] - (float)up, w[a]);
    } else {
      b[a] = 0;
      w[a][0] = 1.0f;
      w[a][1] = w[a][2] = 0.0f;
    }
  }
}

// one component PAT: add e1 w(body 1) + e2 w(body 2) (one add per node when
// both stencils start at the same node -- a decision of the ion alone, so
// the rounding does not depend on which ions share a warp)
template <int D, int PAT>
__device__ __forceinline__ void scatter_comp(unsigned *A, const int d1[3], const float f1[3], float e1,
                                             const int d2[3], const float f2[3], float e2, bool two) {
  constexpr int hoff = 6 * Box<D>::GCELLS;
  constexpr int NJ = D >= 2 ? 3 : 1, NK = D >= 3 ? 3 : 1;
  int b1[3], b2[3];
  float w1[3][3], w2[3][3];
  scat_loc<D, PAT>(d1, f1, b1, w1);
  scat_loc<D, PAT>(d2, f2, b2, w2);
  const bool same = two && b1[0] == b2[0] && b1[1] == b2[1] && b1[2] == b2[2];
#pragma unroll
  for (int k = 0; k < NK; ++k)
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const float a1 = e1 * w1[1][j] * w1[2][k];
      if (same) {
        const float a2 = e2 * w2[1][j] * w2[2][k];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          fx_add(A + Box<D>::gi(b1[0] + i, b1[1] + j, b1[2] + k), hoff, __fadd_rn(a1 * w1[0][i], a2 * w2[0][i]));
      } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) fx_add(A + Box<D>::gi(b1[0] + i, b1[1] + j, b1[2] + k), hoff, a1 * w1[0][i]);
      }
    }
  if (two && !same) {
#pragma unroll
    for (int k = 0; k < NK; ++k)
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const float a2 = e2 * w2[1][j] * w2[2][k];
#pragma unroll
        for (int i = 0; i < 3; ++i) fx_add(A + Box<D>::gi(b2[0] + i, b2[1] + j, b2[2] + k), hoff, a2 * w2[0][i]);
      }
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_adj_scatter(GridP g, ScatArgs S, AdjWork W) {
  using BX = Box<D>;
  constexpr int GC = BX::GCELLS;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned *A = reinterpret_cast<unsigned *>(smem);  // [6][GC] low words, then [6][GC] high words
  const int tid = threadIdx.x, bs = blockDim.x;
  const unsigned mbits = *S.emax;
  if (mbits == 0) return;  // every gathered-field adjoint is zero
  const int nw = min(*W.n, W.cap);
  int ex;
  frexpf(__uint_as_float(mbits), &ex);  // emax < 2^ex
  const int k = 30 - ex;
  const float2 sk = pow2_split(k);  // the fixed-point scale 2^k
  if (blockIdx.x == 0 && tid == 0) *S.kst = k;
  __shared__ int sbb[6];  // the chunk's body cells (box coordinates): lowest, highest per axis
  for (int q = tid; q < 12 * GC; q += bs) A[q] = 0u;
  for (int w = blockIdx.x; w < nw; w += gridDim.x) {
    const int4 it = W.item[w];
    const int t = it.x, s = it.y;
    const int tc[3] = {t % g.nt[0], (t / g.nt[0]) % g.nt[1], t / (g.nt[0] * g.nt[1])};
    const int T0[3] = {tc[0] * Geo<D>::L0, tc[1] * Geo<D>::L1, tc[2] * Geo<D>::L2};
    if (tid < 3) {
      sbb[tid] = 1 << 30;
      sbb[3 + tid] = -(1 << 30);
    }
    __syncthreads();  // the box is clear (the previous item's flush cleared what it read)
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    const PartP &P = S.p[s];
    const bool two = S.sp[s].kind == BP_TWO_BODY;
    const long long cap = P.cap, ec = S.ecap[s];
    for (long long i = it.z + tid; i < it.w; i += bs) {
      const int cell = P.cell[i];
      if (cell < 0) continue;
      int c[3];
      unpack_cell(g, cell, c);
      int d[3] = {0, 0, 0}, d2[3] = {0, 0, 0};
      float f[3] = {0.0f, 0.0f, 0.0f}, f2[3] = {0.0f, 0.0f, 0.0f};
      bool bad = false;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        f[a] = P.off[a * cap + i];
        const float ra = two ? P.r[a * cap + i] : 0.0f;
        // body positions exactly as the adjoint push places them
        d[a] = rel_cell<D>(g, a, c[a], T0[a]);
        bad |= outside_margin<D>(a, d[a]) || !(fabsf(ra * g.idx[a]) < 1.0f);
        float X = f[a] - ra * g.idx[a];
        float fl = floorf(X);
        float fr = X - fl;
        int di = (int)fl;
        if (fr >= 1.0f) { fr = 0.0f; di += 1; }
        d2[a] = d[a] + di;
        f2[a] = fr;
      }
      if (bad) continue;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        lo[a] = min(lo[a], min(d[a], d2[a]));
        hi[a] = max(hi[a], max(d[a], d2[a]));
      }
      float e[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) e[q] = S.eb[s][q * ec + i] * sk.x * sk.y;
      scatter_comp<D, 1>(A + 0 * GC, d, f, e[0], d2, f2, e[6], two);
      scatter_comp<D, 2>(A + 1 * GC, d, f, e[1], d2, f2, e[7], two);
      scatter_comp<D, 4>(A + 2 * GC, d, f, e[2], d2, f2, e[8], two);
      scatter_comp<D, 6>(A + 3 * GC, d, f, e[3], d2, f2, e[9], two);
      scatter_comp<D, 5>(A + 4 * GC, d, f, e[4], d2, f2, e[10], two);
      scatter_comp<D, 3>(A + 5 * GC, d, f, e[5], d2, f2, e[11], two);
    }
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const int l = __reduce_min_sync(0xFFFFFFFFu, lo[a]), h = __reduce_max_sync(0xFFFFFFFFu, hi[a]);
      if ((tid & 31) == 0 && l <= h) {
        atomicMin(&sbb[a], l);
        atomicMax(&sbb[3 + a], h);
      }
    }
    __syncthreads();
    // the box's non-zero nodes into lfx (nodes beyond an open face carry no
    // field the gather read), each node cleared once read.  A body in cell d
    // (box coordinates) reaches the nodes d + OG - 1 .. d + OG + 2 along each
    // axis, so only the chunk's bounding box of those is visited.
    int b0[3] = {0, 0, 0}, ext[3] = {1, 1, 1};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      b0[a] = max(sbb[a] + BX::OG - 1, 0);
      ext[a] = min(sbb[3 + a] + BX::OG + 2, (a == 0 ? BX::G0 : (a == 1 ? BX::G1 : BX::G2)) - 1) - b0[a] + 1;
    }
    const bool none = sbb[0] > sbb[3];
    __syncthreads();  // every thread has read the bounds: the next item may reset them
    if (none) continue;  // no body scattered
    const int nb = ext[0] * ext[1] * ext[2];
    for (int q = tid; q < 6 * nb; q += bs) {
      const int cc = q / nb, r = q - cc * nb;
      const int bidx[3] = {b0[0] + r % ext[0], b0[1] + (r / ext[0]) % ext[1], b0[2] + r / (ext[0] * ext[1])};
      const int si = cc * GC + BX::gi(bidx[0], bidx[1], bidx[2]);
      const unsigned lo = A[si], hi = A[si + 6 * GC];
      if ((lo | hi) == 0u) continue;
      A[si] = 0u;
      A[si + 6 * GC] = 0u;
      const long long v = (long long)(int)hi * 65536LL + (long long)(int)lo;  // fx_value
      if (v == 0) continue;
      long long gidx = 0, stride = 1;
      bool ok = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        int x = T0[a] - (a < D ? BX::OG : 0) + bidx[a];
        if (a < D) {
          if (g.bc[a] == BP_PERIODIC) x = wrap_once(x, g.n[a]);
          else ok &= (x >= 0 && x < g.n[a]);
        }
        gidx += (long long)x * stride;
        stride *= g.n[a];
      }
      if (ok) atomicAdd(S.lfx + (size_t)cc * g.ncell + gidx, (unsigned long long)v);
    }
    // the box spans the tile and less than one tile on each side
    constexpr int NM = D == 1 ? 3 : (D == 2 ? 9 : 27);
    if (tid < NM) {
      int o[3] = {tid % 3 - 1, D >= 2 ? (tid / 3) % 3 - 1 : 0, D >= 3 ? tid / 9 - 1 : 0};
      int u[3];
      bool ok = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        u[a] = tc[a] + o[a];
        if (a < D && g.bc[a] == BP_PERIODIC) u[a] = wrap_once(u[a], g.nt[a]);
        else ok &= u[a] >= 0 && u[a] < g.nt[a];
      }
      if (ok) S.dirty[u[0] + g.nt[0] * (u[1] + g.nt[1] * u[2])] = 1;
    }
  }
}

// the marked tiles' cells: lfx to FP32 (one rounding of the exact sum) added
// to the field adjoints, lfx cleared; the step's emax and work list cleared
template <int D>
__global__ void __launch_bounds__(256) k_adj_fxsum(GridP g, unsigned long long *lfx, unsigned char *dirty,
                                                   const int *kst, float *E0, float *E1, float *E2, float *B0,
                                                   float *B1, float *B2, unsigned *emax, int *nwork) {
  const int t = blockIdx.x, tid = threadIdx.x;
  if (t == 0 && tid == 0) {
    *emax = 0u;  // read by this step's scatter
    *nwork = 0;  // read by this step's push and scatter
  }
  const bool mine = dirty[t] != 0;
  __syncthreads();  // every thread has read the mark before it is cleared
  if (!mine) return;
  float *out[6] = {E0, E1, E2, B0, B1, B2};
  const float2 sk = pow2_split(-*kst);  // back from the fixed-point scale
  constexpr int L0 = Geo<D>::L0, L1 = Geo<D>::L1, L2 = Geo<D>::L2;
  const int tc[3] = {t % g.nt[0], (t / g.nt[0]) % g.nt[1], t / (g.nt[0] * g.nt[1])};
  for (int q = tid; q < L0 * L1 * L2; q += blockDim.x) {
    const int x = tc[0] * L0 + q % L0, y = tc[1] * L1 + (q / L0) % L1, z = tc[2] * L2 + q / (L0 * L1);
    const long long cell = x + (long long)g.n[0] * (y + (long long)g.n[1] * z);
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) {
      unsigned long long *p = lfx + (size_t)cc * g.ncell + cell;
      const long long v = (long long)*p;
      if (v == 0) continue;
      *p = 0ull;
      out[cc][cell] += __ll2float_rn(v) * sk.x * sk.y;
    }
  }
  if (tid == 0) dirty[t] = 0;
}

// deterministic FP64 row sums: out[r * ncomp + k] = scale[r] * sum over the
// ids of row r (CSR, fixed order) of val(id, k)
__global__ void k_csr_sum(const int *ptr, const int *ids, int nrows, const float *xb, long long cap, int ncomp,
                          const double *acb, const double *scale, double *out) {
  __shared__ double sh[256];
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    for (int k = 0; k < ncomp; ++k) {
      double s = 0.0;
      for (int j = ptr[r] + threadIdx.x; j < ptr[r + 1]; j += blockDim.x) {
        const int id = ids[j];
        // positions: adjoint of the ion position = x1b + x2b (both bodies start there)
        s += acb ? acb[id] : (double)xb[(size_t)k * cap + id] + (double)xb[(size_t)(3 + k) * cap + id];
      }
      sh[threadIdx.x] = s;
      __syncthreads();
      for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
      }
      if (threadIdx.x == 0) out[(size_t)r * ncomp + k] = sh[0] * (scale ? scale[r] : 1.0);
      __syncthreads();
    }
  }
}

}  // namespace

void launch_adj_inject(float *lam, const long long *nodes, long long npts, const float *dl, cudaStream_t s) {
  k_adj_inject<<<blocks_for(npts, 256), 256, 0, s>>>(lam, nodes, npts, dl);
}

void launch_adj_e(const GridP &g, float *G[3], float *H[3], float *lamB[3], float *lamJ[3], cudaStream_t s) {
  int nopen = 0;
  for (int a = 0; a < g.D; ++a) nopen += g.bc[a] == BP_OPEN;
  for (int p = nopen; p >= 1; --p)
    for (int a = 0; a < g.D; ++a)
      if (g.bc[a] == BP_OPEN)
        k_adj_mur<<<blocks_for(4 * (g.ncell / g.n[a]), 256), 256, 0, s>>>(g, G[0], G[1], G[2], H[0], H[1], H[2], a, p);
  const int nb = row_blocks4(g, 128);
  if (g.D == 1) k_adj_e<1><<<nb, 128, 0, s>>>(g, G[0], G[1], G[2], H[0], H[1], H[2], lamB[0], lamB[1], lamB[2], lamJ[0], lamJ[1], lamJ[2]);
  else if (g.D == 2) k_adj_e<2><<<nb, 128, 0, s>>>(g, G[0], G[1], G[2], H[0], H[1], H[2], lamB[0], lamB[1], lamB[2], lamJ[0], lamJ[1], lamJ[2]);
  else k_adj_e<3><<<nb, 128, 0, s>>>(g, G[0], G[1], G[2], H[0], H[1], H[2], lamB[0], lamB[1], lamB[2], lamJ[0], lamJ[1], lamJ[2]);
}

void launch_adj_b(const GridP &g, float *lamE[3], float *lamB[3], float h, float *zero[3], cudaStream_t s) {
  const int nb = row_blocks4(g, 128);
  float *z0 = zero ? zero[0] : nullptr, *z1 = zero ? zero[1] : nullptr, *z2 = zero ? zero[2] : nullptr;
  if (g.D == 1) k_adj_b<1><<<nb, 128, 0, s>>>(g, lamE[0], lamE[1], lamE[2], lamB[0], lamB[1], lamB[2], h, z0, z1, z2);
  else if (g.D == 2) k_adj_b<2><<<nb, 128, 0, s>>>(g, lamE[0], lamE[1], lamE[2], lamB[0], lamB[1], lamB[2], h, z0, z1, z2);
  else k_adj_b<3><<<nb, 128, 0, s>>>(g, lamE[0], lamE[1], lamE[2], lamB[0], lamB[1], lamB[2], h, z0, z1, z2);
}

// box sets, then the 256 threads' slices of gather derivatives (12 D floats each)
size_t adj_push_smem(int D) {
  const size_t stash = sizeof(float) * 12 * (size_t)D * 256;
  if (D == 1) return sizeof(float) * adj_push_bufs(1) * adj_box_floats<1>() + stash;
  if (D == 2) return sizeof(float) * adj_push_bufs(2) * adj_box_floats<2>() + stash;
  return sizeof(float) * adj_push_bufs(3) * adj_box_floats<3>() + stash;
}
size_t adj_scatter_smem(int D) {
  if (D == 1) return sizeof(unsigned) * 12 * Box<1>::GCELLS;
  if (D == 2) return sizeof(unsigned) * 12 * Box<2>::GCELLS;
  return sizeof(unsigned) * 12 * Box<3>::GCELLS;
}

template <int D>
cudaError_t adj_prepare_one(int *push_blocks, int *scat_blocks) {
  cudaError_t e = cudaFuncSetAttribute(k_adj_push<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj_push_smem(D));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_scatter<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj_scatter_smem(D));
  int dev = 0, sms = 0, bp = 0, bsc = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bp, k_adj_push<D>, 256, adj_push_smem(D));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bsc, k_adj_scatter<D>, 256, adj_scatter_smem(D));
  *push_blocks = sms * (bp < 1 ? 1 : bp);
  *scat_blocks = sms * (bsc < 1 ? 1 : bsc);
  return e;
}

// kernel attributes and the resident grids of the two work-list kernels
int adj_prepare(int D, int *push_blocks, int *scat_blocks) {
  cudaError_t e = D == 1   ? adj_prepare_one<1>(push_blocks, scat_blocks)
                  : D == 2 ? adj_prepare_one<2>(push_blocks, scat_blocks)
                           : adj_prepare_one<3>(push_blocks, scat_blocks);
  return e == cudaSuccess ? 0 : -1;
}

template <int D>
void adj_launch_all(const GridP &g, const AdjArgs &A, const ScatArgs &S, const AdjWork &W, const AdjBufs &b,
                    float *lamE[3], float *lamB[3], cudaStream_t s) {
  const int nq = g.ntiles * A.nsp;
  k_adj_work<<<(nq + 255) / 256, 256, 0, s>>>(g, A, W, b.chunk);
  k_adj_push<D><<<b.push_blocks, 256, adj_push_smem(D), s>>>(g, A, W);
  k_adj_scatter<D><<<b.scat_blocks, 256, adj_scatter_smem(D), s>>>(g, S, W);
  k_adj_fxsum<D><<<g.ntiles, 256, 0, s>>>(g, b.lfx, b.dirty, b.kst, lamE[0], lamE[1], lamE[2], lamB[0], lamB[1],
                                           lamB[2], b.emax, b.nwork);
}

// the particle adjoint of one step: the work list, the reversed push with
// the position derivatives of the gather (k_adj_push), the field-adjoint
// scatter (k_adj_scatter), then its sum into lamE, lamB (k_adj_fxsum)
void launch_adj_push(const GridP &g, int nsp, const SpecP *sp, const PartP *p, float *const xb[], double *const acb[],
                     float *const eb[], const long long *cap, const float *const E[3], const float *const B[3],
                     const float *const lamJ[3], const AdjBufs &b, float *lamE[3], float *lamB[3], int *status,
                     cudaStream_t s) {
  AdjArgs A;
  memset(&A, 0, sizeof A);
  ScatArgs S;
  memset(&S, 0, sizeof S);
  A.nsp = S.nsp = nsp;
  for (int k = 0; k < nsp; ++k) {
    A.sp[k] = S.sp[k] = sp[k];
    A.p[k] = S.p[k] = p[k];
    A.st[k].xb = xb[k];
    A.st[k].acb = acb[k];
    A.st[k].eb = eb[k];
    A.st[k].cap = cap[k];
    A.st[k].status = status;
    S.eb[k] = eb[k];
    S.ecap[k] = cap[k];
  }
  for (int c = 0; c < 3; ++c) {
    A.E[c] = E[c];
    A.B[c] = B[c];
    A.lamJ[c] = lamJ[c];
  }
  A.emax = b.emax;
  S.emax = b.emax;
  S.lfx = b.lfx;
  S.dirty = b.dirty;
  S.kst = b.kst;
  AdjWork W{b.nwork, b.work, b.work_cap};
  if (g.D == 1) adj_launch_all<1>(g, A, S, W, b, lamE, lamB, s);
  else if (g.D == 2) adj_launch_all<2>(g, A, S, W, b, lamE, lamB, s);
  else adj_launch_all<3>(g, A, S, W, b, lamE, lamB, s);
}

void launch_csr_sum(const int *ptr, const int *ids, int nrows, const float *xb, long long cap, int ncomp,
                    const double *acb, const double *scale, double *out, cudaStream_t s) {
  int nb = nrows < 4096 ? (nrows < 1 ? 1 : nrows) : 4096;
  k_csr_sum<<<nb, 256, 0, s>>>(ptr, ids, nrows, xb, cap, ncomp, acb, scale, out);
}
