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
