// bp_particle.cuh -- device helpers shared by the particle kernels (the
// forward push/deposit and its adjoint): staggered quadratic-shape gather
// from a staged field box, the relativistic Boris rotation, the five-node
// shape windows of the Esirkepov deposit, tile-relative cell coordinates.
#pragma once
#include "bp_internal.cuh"

namespace {

struct Loc {
  int bn[3], bh[3];        // first box index of the node- / half-staggered stencil
  float wn[3][3], wh[3][3];
};

template <int D>
__device__ __forceinline__ void make_loc(const int d[3], const float f[3], Loc &L) {
  constexpr int og = Box<D>::OG;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < D) {
      int up = f[a] >= 0.5f ? 1 : 0;
      L.bn[a] = d[a] + og + up - 1;
      qweights(f[a] - (float)up, L.wn[a]);
      L.bh[a] = d[a] + og - 1;
      qweights(f[a] - 0.5f, L.wh[a]);
    } else {
      L.bn[a] = L.bh[a] = 0;
      L.wn[a][0] = L.wh[a][0] = 1.0f;
      L.wn[a][1] = L.wn[a][2] = L.wh[a][1] = L.wh[a][2] = 0.0f;
    }
  }
}

// one field component with stagger pattern PAT (bit a: half cell along a)
// at two bodies; loads are shared when both stencils start at the same node
// for every active lane of the warp (a warp-uniform choice: both forms give
// the same sums, and a uniform branch keeps the warp from running both)
template <int D, int PAT>
__device__ __forceinline__ void gather_comp(const float *__restrict__ G, const Loc &A, const Loc &Bo, float &oa,
                                            float &ob) {
  int ba[3], bb[3];
  const float *wa[3];
  const float *wb[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const bool half = (PAT >> a) & 1;
    ba[a] = half ? A.bh[a] : A.bn[a];
    bb[a] = half ? Bo.bh[a] : Bo.bn[a];
    wa[a] = half ? A.wh[a] : A.wn[a];
    wb[a] = half ? Bo.wh[a] : Bo.wn[a];
  }
  constexpr int NJ = D >= 2 ? 3 : 1, NK = D >= 3 ? 3 : 1;
  const bool same = __all_sync(__activemask(),
                               (ba[0] == bb[0]) && (D < 2 || ba[1] == bb[1]) && (D < 3 || ba[2] == bb[2]));
  // contraction x, then y, then z: 3 + 3 + 3 weights per row, plane, box
  float sa = 0.0f, sb = 0.0f;
  if (same) {
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      float pa = 0.0f, pb = 0.0f;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const float *row = G + Box<D>::gi(ba[0], ba[1] + j, ba[2] + k);
        float ra = 0.0f, rb = 0.0f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          float v = row[i];
          ra = fmaf(wa[0][i], v, ra);
          rb = fmaf(wb[0][i], v, rb);
        }
        pa = fmaf(wa[1][j], ra, pa);
        pb = fmaf(wb[1][j], rb, pb);
      }
      sa = fmaf(wa[2][k], pa, sa);
      sb = fmaf(wb[2][k], pb, sb);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      float pa = 0.0f, pb = 0.0f;
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const float *ra_ = G + Box<D>::gi(ba[0], ba[1] + j, ba[2] + k);
        const float *rb_ = G + Box<D>::gi(bb[0], bb[1] + j, bb[2] + k);
        float ra = 0.0f, rb = 0.0f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          ra = fmaf(wa[0][i], ra_[i], ra);
          rb = fmaf(wb[0][i], rb_[i], rb);
        }
        pa = fmaf(wa[1][j], ra, pa);
        pb = fmaf(wb[1][j], rb, pb);
      }
      sa = fmaf(wa[2][k], pa, sa);
      sb = fmaf(wb[2][k], pb, sb);
    }
  }
  oa = sa;
  ob = sb;
}

template <int D>
__device__ __forceinline__ void gather_all(const float *G, const Loc &A, const Loc &Bo, float Ea[3], float Ba[3],
                                           float Eb[3], float Bb[3]) {
  constexpr int gc = Box<D>::GCELLS;
  gather_comp<D, 1>(G + 0 * gc, A, Bo, Ea[0], Eb[0]);
  gather_comp<D, 2>(G + 1 * gc, A, Bo, Ea[1], Eb[1]);
  gather_comp<D, 4>(G + 2 * gc, A, Bo, Ea[2], Eb[2]);
  gather_comp<D, 6>(G + 3 * gc, A, Bo, Ba[0], Bb[0]);
  gather_comp<D, 5>(G + 4 * gc, A, Bo, Ba[1], Bb[1]);
  gather_comp<D, 3>(G + 5 * gc, A, Bo, Ba[2], Bb[2]);
}

// ---------------------------------------------------------------------------
// The 3D gather on packed pairs (FFMA2): the six components go in pairs
// (E_x, B_y), (E_y, B_x), (E_z, B_z); a pair's lanes carry one component
// each, with that component's stagger weights, so each row value pair comes
// from two shared-memory loads and every multiply-add serves two components.
// Per lane the arithmetic is the scalar gather's.

// a body's position for the gather: offsets from the nearest node (xn) and
// from the cell centre (xh), and the first box index of each stencil
struct Pos {
  float xn[3], xh[3];
  int bn[3], bh[3];
};

template <int D>
__device__ __forceinline__ void make_pos(const int d[3], const float f[3], Pos &P) {
  constexpr int og = Box<D>::OG;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < D) {
      const int up = f[a] >= 0.5f ? 1 : 0;
      P.bn[a] = d[a] + og + up - 1;
      P.xn[a] = f[a] - (float)up;
      P.bh[a] = d[a] + og - 1;
      P.xh[a] = f[a] - 0.5f;
    } else {
      P.bn[a] = P.bh[a] = 0;
      P.xn[a] = P.xh[a] = 0.0f;
    }
  }
}

// qweights on a pair of offsets
__device__ __forceinline__ void qweights2(float2 xi, float2 w[3]) {
  const float2 H = make_float2(0.5f, 0.5f), M1 = make_float2(-1.0f, -1.0f);
  const float2 a = __ffma2_rn(xi, M1, H), b = __fadd2_rn(xi, H);
  w[0] = __fmul2_rn(__fmul2_rn(a, H), a);
  w[1] = __ffma2_rn(__fmul2_rn(xi, M1), xi, make_float2(0.75f, 0.75f));
  w[2] = __fmul2_rn(__fmul2_rn(b, H), b);
}

// components c1, c2 (stagger patterns P1, P2; boxes G1, G2) at bodies A, B;
// same: every active lane's bodies share all their stencil origins (both
// forms give the same sums; the shared form loads each row once)
template <int P1, int P2>
__device__ __forceinline__ void gather_pair3(const float *__restrict__ G1, const float *__restrict__ G2, const Pos &A,
                                             const Pos &B, bool same, float2 &oa, float2 &ob) {
  float2 wa[3][3], wb[3][3];
  int a1[3], a2[3], b1[3], b2[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const bool h1 = (P1 >> ax) & 1, h2 = (P2 >> ax) & 1;
    qweights2(make_float2(h1 ? A.xh[ax] : A.xn[ax], h2 ? A.xh[ax] : A.xn[ax]), wa[ax]);
    qweights2(make_float2(h1 ? B.xh[ax] : B.xn[ax], h2 ? B.xh[ax] : B.xn[ax]), wb[ax]);
    a1[ax] = h1 ? A.bh[ax] : A.bn[ax];
    a2[ax] = h2 ? A.bh[ax] : A.bn[ax];
    b1[ax] = h1 ? B.bh[ax] : B.bn[ax];
    b2[ax] = h2 ? B.bh[ax] : B.bn[ax];
  }
  float2 sa = make_float2(0.0f, 0.0f), sb = sa;
  if (same) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float2 pa = make_float2(0.0f, 0.0f), pb = pa;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float *r1 = G1 + Box<3>::gi(a1[0], a1[1] + j, a1[2] + k);
        const float *r2 = G2 + Box<3>::gi(a2[0], a2[1] + j, a2[2] + k);
        float2 ra = make_float2(0.0f, 0.0f), rb = ra;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const float2 v = make_float2(r1[i], r2[i]);
          ra = __ffma2_rn(wa[0][i], v, ra);
          rb = __ffma2_rn(wb[0][i], v, rb);
        }
        pa = __ffma2_rn(wa[1][j], ra, pa);
        pb = __ffma2_rn(wb[1][j], rb, pb);
      }
      sa = __ffma2_rn(wa[2][k], pa, sa);
      sb = __ffma2_rn(wb[2][k], pb, sb);
    }
  } else {
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
      float2 pa = make_float2(0.0f, 0.0f), pb = pa;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float *ra1 = G1 + Box<3>::gi(a1[0], a1[1] + j, a1[2] + k);
        const float *ra2 = G2 + Box<3>::gi(a2[0], a2[1] + j, a2[2] + k);
        const float *rb1 = G1 + Box<3>::gi(b1[0], b1[1] + j, b1[2] + k);
        const float *rb2 = G2 + Box<3>::gi(b2[0], b2[1] + j, b2[2] + k);
        float2 ra = make_float2(0.0f, 0.0f), rb = ra;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          ra = __ffma2_rn(wa[0][i], make_float2(ra1[i], ra2[i]), ra);
          rb = __ffma2_rn(wb[0][i], make_float2(rb1[i], rb2[i]), rb);
        }
        pa = __ffma2_rn(wa[1][j], ra, pa);
        pb = __ffma2_rn(wb[1][j], rb, pb);
      }
      // wz[k]: the weights are selected by a loop index here (rolled loop)
      const float2 wza = k == 0 ? wa[2][0] : (k == 1 ? wa[2][1] : wa[2][2]);
      const float2 wzb = k == 0 ? wb[2][0] : (k == 1 ? wb[2][1] : wb[2][2]);
      sa = __ffma2_rn(wza, pa, sa);
      sb = __ffma2_rn(wzb, pb, sb);
    }
  }
  oa = sa;
  ob = sb;
}

__device__ __forceinline__ void gather_all_p3(const float *G, const Pos &A, const Pos &Bo, float Ea[3], float Ba[3],
                                              float Eb[3], float Bb[3]) {
  constexpr int gc = Box<3>::GCELLS;
  // one warp vote for the three pairs: both bodies on the same node and
  // half-node stencils along every axis
  const bool same = __all_sync(__activemask(), A.bn[0] == Bo.bn[0] && A.bn[1] == Bo.bn[1] && A.bn[2] == Bo.bn[2] &&
                                                   A.bh[0] == Bo.bh[0] && A.bh[1] == Bo.bh[1] && A.bh[2] == Bo.bh[2]);
  float2 a, b;
  gather_pair3<1, 5>(G + 0 * gc, G + 4 * gc, A, Bo, same, a, b);  // E_x, B_y
  Ea[0] = a.x; Ba[1] = a.y; Eb[0] = b.x; Bb[1] = b.y;
  gather_pair3<2, 6>(G + 1 * gc, G + 3 * gc, A, Bo, same, a, b);  // E_y, B_x
  Ea[1] = a.x; Ba[0] = a.y; Eb[1] = b.x; Bb[0] = b.y;
  gather_pair3<4, 3>(G + 2 * gc, G + 5 * gc, A, Bo, same, a, b);  // E_z, B_z
  Ea[2] = a.x; Ba[2] = a.y; Eb[2] = b.x; Bb[2] = b.y;
}

// relativistic Boris (Sec. 2): u- = u + hE; t = hB/gamma-; s = 2t/(1+t^2);
// u+ = u- + (u- + u- x t) x s; u = u+ + hE
__device__ __forceinline__ void boris(float h, const float E[3], const float B[3], float u[3]) {
  float um0 = fmaf(h, E[0], u[0]), um1 = fmaf(h, E[1], u[1]), um2 = fmaf(h, E[2], u[2]);
  float gi = rsqrtf(1.0f + um0 * um0 + um1 * um1 + um2 * um2);
  float t0 = h * B[0] * gi, t1 = h * B[1] * gi, t2 = h * B[2] * gi;
  float sf = __fdividef(2.0f, 1.0f + t0 * t0 + t1 * t1 + t2 * t2);
  float s0 = t0 * sf, s1 = t1 * sf, s2 = t2 * sf;
  float c0 = um0 + (um1 * t2 - um2 * t1);
  float c1 = um1 + (um2 * t0 - um0 * t2);
  float c2 = um2 + (um0 * t1 - um1 * t0);
  float up0 = um0 + (c1 * s2 - c2 * s1);
  float up1 = um1 + (c2 * s0 - c0 * s2);
  float up2 = um2 + (c0 * s1 - c1 * s0);
  u[0] = fmaf(h, E[0], up0);
  u[1] = fmaf(h, E[1], up1);
  u[2] = fmaf(h, E[2], up2);
}

// shape factors on the five-node window around the old nearest node:
// S0[m] at the old position, DS[m] = S1[m] - S0[m], node n0 - 2 + m
template <int D>
__device__ __forceinline__ void window(const float f[3], const float de[3], float S0[3][5], float DS[3][5],
                                       int n0[3], const int d[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < D) {
      int up = f[a] >= 0.5f ? 1 : 0;
      float xi = f[a] - (float)up;
      n0[a] = d[a] + Box<D>::OJ + up;
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        float u = xi - (float)(m - 2);
        S0[a][m] = qshape(u);
        DS[a][m] = qshape_delta(u, de[a]);
      }
    } else {
      n0[a] = 2;
#pragma unroll
      for (int m = 0; m < 5; ++m) { S0[a][m] = (m == 2) ? 1.0f : 0.0f; DS[a][m] = 0.0f; }
    }
  }
}

// particle of a tile handled by thread tid in the chunk starting at k0: the
// lanes of a warp take particles bs/32 apart (bs = block size, a multiple of
// 32), so that in cell-sorted order they sit in different cells and rarely
// add to the same shared-memory node at once; the chunk [k0, k0 + bs) is
// still covered exactly once
__device__ __forceinline__ int spread_index(int k0, int tid, int bs) { return k0 + (tid & 31) * (bs >> 5) + (tid >> 5); }

// tile-relative cell of a global cell coordinate (periodic: nearest image)
template <int D>
__device__ __forceinline__ int rel_cell(const GridP &g, int a, int c, int T0) {
  constexpr int M = Geo<D>::M;
  const int L = a == 0 ? Geo<D>::L0 : (a == 1 ? Geo<D>::L1 : Geo<D>::L2);
  int d = c - T0;
  if (g.bc[a] == BP_PERIODIC) {
    if (d < -M) d += g.n[a];
    else if (d >= L + M) d -= g.n[a];
  }
  return d;
}

template <int D>
__device__ __forceinline__ bool outside_margin(int a, int d) {
  constexpr int M = Geo<D>::M;
  const int L = a == 0 ? Geo<D>::L0 : (a == 1 ? Geo<D>::L1 : Geo<D>::L2);
  return d < -M || d >= L + M;
}



}  // namespace
