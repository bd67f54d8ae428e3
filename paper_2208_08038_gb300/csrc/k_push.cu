// k_push.cu -- the per-tile particle kernel: gather at both bodies, internal
// modified-Coulomb field, relativistic Boris push of both bodies, drift and
// Esirkepov (quadratic shape) current deposit into a shared-memory tile.
//
// Method: arXiv 2208.08038 Sec. 2 (two-body macro-ion, Boris equations,
// modified Coulomb force, body currents q v / dV).  One CTA per tile:
//   1. stage E and B of the tile plus halo in shared memory (FP32),
//   2. push every particle of the tile (all species), accumulating the
//      current of both bodies in a shared-memory box (tile + halo):
//        BP_DEPOSIT_SORTED: 64-bit fixed point (integer adds are associative,
//                           so the box is bit-identical whatever the order),
//        BP_DEPOSIT_ATOMIC: FP32 shared atomics,
//   3. write the box to the tile's slot of the global box array; the
//      current-sum kernel adds the overlapping boxes of neighbouring tiles
//      in a fixed order.
#include <type_traits>

#include "bp_internal.cuh"
#include "bp_particle.cuh"

namespace {

template <bool DET, typename JT>
__device__ __forceinline__ void jadd(JT *p, float v, float scale) {
  if (v == 0.0f) return;
  if constexpr (DET) {
    long long q = __float2ll_rn(v * scale);
    if (q) atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)q);
  } else {
    atomicAdd(p, v);
  }
}

// Esirkepov density decomposition for NB bodies sharing one window:
//   3D W_x = DSx (S0y S0z + (DSy S0z + S0y DSz)/2 + DSy DSz/3) (cyclic),
//   2D W_x = DSx (S0y + DSy/2), J_z with S0x S0y + (DSx S0y + S0x DSy)/2 + DSx DSy/3,
//   1D W_x = DSx, J_y/z with S0 + DS/2,
// J_a on the face after node i = -qw dx_a/dt * sum_{i' <= i} W_a(i').
template <int D, bool DET, int NB, typename JT>
__device__ __forceinline__ void esirkepov(JT *__restrict__ J, const int n0[3], const float (*S0)[3][5],
                                          const float (*DS)[3][5], const float *qw, const float (*v)[3],
                                          const float dxdt[3], float scale) {
  constexpr int jcells = Box<D>::JCELLS, jb0 = Box<D>::J0, jb1 = Box<D>::J1;
  JT *Jx = J, *Jy = J + jcells, *Jz = J + 2 * jcells;
  const int bx = n0[0] - 2, by = n0[1] - 2, bz = n0[2] - 2;
  if constexpr (D == 1) {
    float run[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) run[b] = 0.0f;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      float jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        run[b] += DS[b][0][i];
        jx += -qw[b] * dxdt[0] * run[b];
        float sb = S0[b][0][i] + 0.5f * DS[b][0][i];
        jy += qw[b] * v[b][1] * sb;
        jz += qw[b] * v[b][2] * sb;
      }
      if (i < 4) jadd<DET>(Jx + bx + i, jx, scale);
      jadd<DET>(Jy + bx + i, jy, scale);
      jadd<DET>(Jz + bx + i, jz, scale);
    }
  } else if constexpr (D == 2) {
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      float fac[NB];
      bool any = false;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        fac[b] = S0[b][1][j] + 0.5f * DS[b][1][j];
        any |= fac[b] != 0.0f;
      }
      if (!any) continue;
      float run[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) run[b] = 0.0f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float jx = 0.0f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          run[b] += DS[b][0][i];
          jx += -qw[b] * dxdt[0] * run[b] * fac[b];
        }
        jadd<DET>(Jx + (bx + i) + jb0 * (by + j), jx, scale);
      }
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      float fac[NB];
      bool any = false;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        fac[b] = S0[b][0][i] + 0.5f * DS[b][0][i];
        any |= fac[b] != 0.0f;
      }
      if (!any) continue;
      float run[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) run[b] = 0.0f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float jy = 0.0f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          run[b] += DS[b][1][j];
          jy += -qw[b] * dxdt[1] * run[b] * fac[b];
        }
        jadd<DET>(Jy + (bx + i) + jb0 * (by + j), jy, scale);
      }
    }
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        float jz = 0.0f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          float w = S0[b][0][i] * S0[b][1][j] + 0.5f * (DS[b][0][i] * S0[b][1][j] + S0[b][0][i] * DS[b][1][j]) +
                    (1.0f / 3.0f) * DS[b][0][i] * DS[b][1][j];
          jz += qw[b] * v[b][2] * w;
        }
        jadd<DET>(Jz + (bx + i) + jb0 * (by + j), jz, scale);
      }
  } else {
    // J_x
#pragma unroll 1
    for (int k = 0; k < 5; ++k)
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        float fac[NB];
        bool any = false;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          fac[b] = S0[b][1][j] * S0[b][2][k] + 0.5f * (DS[b][1][j] * S0[b][2][k] + S0[b][1][j] * DS[b][2][k]) +
                   (1.0f / 3.0f) * DS[b][1][j] * DS[b][2][k];
          any |= fac[b] != 0.0f;
        }
        if (!any) continue;
        float run[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) run[b] = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float jx = 0.0f;
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            run[b] += DS[b][0][i];
            jx += -qw[b] * dxdt[0] * run[b] * fac[b];
          }
          jadd<DET>(Jx + (bx + i) + jb0 * ((by + j) + jb1 * (bz + k)), jx, scale);
        }
      }
    // J_y
#pragma unroll 1
    for (int k = 0; k < 5; ++k)
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        float fac[NB];
        bool any = false;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          fac[b] = S0[b][0][i] * S0[b][2][k] + 0.5f * (DS[b][0][i] * S0[b][2][k] + S0[b][0][i] * DS[b][2][k]) +
                   (1.0f / 3.0f) * DS[b][0][i] * DS[b][2][k];
          any |= fac[b] != 0.0f;
        }
        if (!any) continue;
        float run[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) run[b] = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float jy = 0.0f;
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            run[b] += DS[b][1][j];
            jy += -qw[b] * dxdt[1] * run[b] * fac[b];
          }
          jadd<DET>(Jy + (bx + i) + jb0 * ((by + j) + jb1 * (bz + k)), jy, scale);
        }
      }
    // J_z
#pragma unroll 1
    for (int j = 0; j < 5; ++j)
#pragma unroll
      for (int i = 0; i < 5; ++i) {
        float fac[NB];
        bool any = false;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          fac[b] = S0[b][0][i] * S0[b][1][j] + 0.5f * (DS[b][0][i] * S0[b][1][j] + S0[b][0][i] * DS[b][1][j]) +
                   (1.0f / 3.0f) * DS[b][0][i] * DS[b][1][j];
          any |= fac[b] != 0.0f;
        }
        if (!any) continue;
        float run[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) run[b] = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          float jz = 0.0f;
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            run[b] += DS[b][2][k];
            jz += -qw[b] * dxdt[2] * run[b] * fac[b];
          }
          jadd<DET>(Jz + (bx + i) + jb0 * ((by + j) + jb1 * (bz + k)), jz, scale);
        }
      }
  }
}


// Fast path: all four positions (both bodies, before and after the move)
// share one nearest node per axis, so the window is the three nodes around
// it and S1 - S0 has a closed form in the move d (no cancellation):
//   node n-1: -d (1 - 2 xi - d) / 2,  node n: -d (2 xi + d),  node n+1: d (1 + 2 xi + d) / 2
// with xi = old position - n.  J along a simulated axis then lives on the two
// faces inside the window.
template <int D, bool DET, int NB, typename JT>
__device__ __forceinline__ void esirkepov3(JT *__restrict__ J, const int n[3], const float (*xi)[3],
                                           const float (*de)[3], const float *qw, const float (*v)[3],
                                           const float dxdt[3], float scale) {
  constexpr int jcells = Box<D>::JCELLS, jb0 = Box<D>::J0, jb1 = Box<D>::J1;
  float S0[NB][3][3], DS[NB][3][3], P[NB][3][2];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a < D) {
        const float x = xi[b][a], d = de[b][a];
        qweights(x, S0[b][a]);
        DS[b][a][0] = -0.5f * d * (1.0f - 2.0f * x - d);
        DS[b][a][1] = -d * (2.0f * x + d);
        DS[b][a][2] = 0.5f * d * (1.0f + 2.0f * x + d);
        P[b][a][0] = DS[b][a][0];
        P[b][a][1] = DS[b][a][0] + DS[b][a][1];
      } else {
        S0[b][a][0] = S0[b][a][2] = 0.0f;
        S0[b][a][1] = 1.0f;
        DS[b][a][0] = DS[b][a][1] = DS[b][a][2] = 0.0f;
        P[b][a][0] = P[b][a][1] = 0.0f;
      }
    }
  JT *Jx = J, *Jy = J + jcells, *Jz = J + 2 * jcells;
  const int bx = n[0] - 1, by = n[1] - 1, bz = n[2] - 1;
  float cq[NB][3];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) cq[b][a] = -qw[b] * dxdt[a];
  if constexpr (D == 1) {
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      float jx = 0.0f;
#pragma unroll
      for (int b = 0; b < NB; ++b) jx = __fadd_rn(jx, __fmul_rn(cq[b][0], P[b][0][f]));
      jadd<DET>(Jx + bx + f, jx, scale);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float jy = 0.0f, jz = 0.0f;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        float sb = S0[b][0][i] + 0.5f * DS[b][0][i];
        jy = __fadd_rn(jy, __fmul_rn(qw[b] * v[b][1], sb));
        jz = __fadd_rn(jz, __fmul_rn(qw[b] * v[b][2], sb));
      }
      jadd<DET>(Jy + bx + i, jy, scale);
      jadd<DET>(Jz + bx + i, jz, scale);
    }
  } else if constexpr (D == 2) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        float jx = 0.0f;
#pragma unroll
        for (int b = 0; b < NB; ++b)
          jx = __fadd_rn(jx, __fmul_rn(cq[b][0] * P[b][0][f], S0[b][1][j] + 0.5f * DS[b][1][j]));
        jadd<DET>(Jx + (bx + f) + jb0 * (by + j), jx, scale);
      }
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float jy = 0.0f;
#pragma unroll
        for (int b = 0; b < NB; ++b)
          jy = __fadd_rn(jy, __fmul_rn(cq[b][1] * P[b][1][g], S0[b][0][i] + 0.5f * DS[b][0][i]));
        jadd<DET>(Jy + (bx + i) + jb0 * (by + g), jy, scale);
      }
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float jz = 0.0f;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          float w = S0[b][0][i] * S0[b][1][j] + 0.5f * (DS[b][0][i] * S0[b][1][j] + S0[b][0][i] * DS[b][1][j]) +
                    (1.0f / 3.0f) * DS[b][0][i] * DS[b][1][j];
          jz = __fadd_rn(jz, __fmul_rn(qw[b] * v[b][2], w));
        }
        jadd<DET>(Jz + (bx + i) + jb0 * (by + j), jz, scale);
      }
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        float F[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b)
          F[b] = S0[b][1][j] * S0[b][2][k] + 0.5f * (DS[b][1][j] * S0[b][2][k] + S0[b][1][j] * DS[b][2][k]) +
                 (1.0f / 3.0f) * DS[b][1][j] * DS[b][2][k];
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          float jx = 0.0f;
#pragma unroll
          for (int b = 0; b < NB; ++b) jx = __fadd_rn(jx, __fmul_rn(cq[b][0] * P[b][0][f], F[b]));
          jadd<DET>(Jx + (bx + f) + jb0 * ((by + j) + jb1 * (bz + k)), jx, scale);
        }
      }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float F[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b)
          F[b] = S0[b][0][i] * S0[b][2][k] + 0.5f * (DS[b][0][i] * S0[b][2][k] + S0[b][0][i] * DS[b][2][k]) +
                 (1.0f / 3.0f) * DS[b][0][i] * DS[b][2][k];
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          float jy = 0.0f;
#pragma unroll
          for (int b = 0; b < NB; ++b) jy = __fadd_rn(jy, __fmul_rn(cq[b][1] * P[b][1][g], F[b]));
          jadd<DET>(Jy + (bx + i) + jb0 * ((by + g) + jb1 * (bz + k)), jy, scale);
        }
      }
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float F[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b)
          F[b] = S0[b][0][i] * S0[b][1][j] + 0.5f * (DS[b][0][i] * S0[b][1][j] + S0[b][0][i] * DS[b][1][j]) +
                 (1.0f / 3.0f) * DS[b][0][i] * DS[b][1][j];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float jz = 0.0f;
#pragma unroll
          for (int b = 0; b < NB; ++b) jz = __fadd_rn(jz, __fmul_rn(cq[b][2] * P[b][2][h], F[b]));
          jadd<DET>(Jz + (bx + i) + jb0 * ((by + j) + jb1 * (bz + h)), jz, scale);
        }
      }
  }
}

// general case (a position changes nearest node, or the bodies straddle a
// node boundary): five-node windows per body; kept out of line so the fast
// path keeps its registers
template <int D, bool DET, typename JT>
__device__ __noinline__ void general_deposit(JT *Jsm, const GridP &g, const float *f, const float *de1, const int *d,
                                             const float *f2, const float *de2, const int *d2, bool two, float qw1,
                                             float qw2, const float *v1, const float *v2, float scale) {
  const float dxdt[3] = {g.dx[0] / g.dt, g.dx[1] / g.dt, g.dx[2] / g.dt};
  float S0[2][3][5], DS[2][3][5];
  float vv[2][3];
  float qw[2] = {qw1, qw2};
  int n1[3], n2[3];
  float fa[3], fb[3], da[3], db[3];
  int ia[3], ib[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    vv[0][a] = v1[a];
    vv[1][a] = v2[a];
    fa[a] = f[a]; fb[a] = f2[a]; da[a] = de1[a]; db[a] = de2[a]; ia[a] = d[a]; ib[a] = d2[a];
  }
  window<D>(fa, da, S0[0], DS[0], n1, ia);
  if (two) {
    window<D>(fb, db, S0[1], DS[1], n2, ib);
    const bool same = (n1[0] == n2[0]) && (D < 2 || n1[1] == n2[1]) && (D < 3 || n1[2] == n2[2]);
    if (same) {
      esirkepov<D, DET, 2>(Jsm, n1, S0, DS, qw, vv, dxdt, scale);
    } else {
      esirkepov<D, DET, 1>(Jsm, n1, S0, DS, qw, vv, dxdt, scale);
      esirkepov<D, DET, 1>(Jsm, n2, S0 + 1, DS + 1, qw + 1, vv + 1, dxdt, scale);
    }
  } else {
    esirkepov<D, DET, 1>(Jsm, n1, S0, DS, qw, vv, dxdt, scale);
  }
}

template <int D, bool DET, typename JT>
__device__ void push_particle(const GridP &g, const SpecP &sp, const PartP &P, long long i, const int T0[3],
                              const float *Gsm, JT *Jsm, int *status, float scale, int *qbuf, int *qn, int qmax) {
  const long long cap = P.cap;
  const bool two = sp.kind == BP_TWO_BODY;
  int cell = P.cell[i];
  if (cell < 0) return;
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
    bad |= outside_margin<D>(a, d[a]);
    // body 2 sits at x1 - r
    float rc = r[a] * g.idx[a];
    bad |= !(fabsf(rc) < 1.0f);
    float X = f[a] - rc;
    float fl = floorf(X);
    float fr = X - fl;
    int di = (int)fl;
    if (fr >= 1.0f) { fr = 0.0f; di += 1; }
    d2[a] = d[a] + di;
    f2[a] = fr;
  }
  if (bad) {
    atomicOr(status, ST_DOMAIN);
    return;
  }
  float E1[3], B1[3], E2[3], B2[3];
  {
    Loc L1, L2;
    make_loc<D>(d, f, L1);
    make_loc<D>(two ? d2 : d, two ? f2 : f, L2);
    gather_all<D>(Gsm, L1, L2, E1, B1, E2, B2);
  }
  float v1[3], v2[3] = {0.0f, 0.0f, 0.0f};
  if (two) {
    // modified Coulomb field (Sec. 2): on the nucleus q2 kappa r / (r^2 + ac^2)^{3/2},
    // on the bound electron -q1 kappa r / (...), r = x1 - x2
    const int pi = P.pidx ? P.pidx[i] : 0;
    const float ac = sp.ac[pi];
    float rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + ac * ac;
    float rs = rsqrtf(rr);
    float s = sp.kappa * rs * rs * rs;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      E1[a] = fmaf(sp.q2 * s, r[a], E1[a]);
      E2[a] = fmaf(-sp.q1 * s, r[a], E2[a]);
    }
    boris(sp.h2, E2, B2, u2);
    float g2 = rsqrtf(1.0f + u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) v2[a] = u2[a] * g2;
  }
  boris(sp.h1, E1, B1, u1);
  {
    float g1 = rsqrtf(1.0f + u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) v1[a] = u1[a] * g1;
  }
  // drift: body 1 moves in cells by dt v / dx; the internal displacement by
  // dt (v1 - v2) on all three axes; the deposited moves are the ones the
  // stored FP32 state actually makes
  float fn[3] = {0.0f, 0.0f, 0.0f}, de1[3] = {0.0f, 0.0f, 0.0f}, de2[3] = {0.0f, 0.0f, 0.0f}, rn[3];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    fn[a] = f[a] + g.dt * v1[a] * g.idx[a];
    de1[a] = fn[a] - f[a];
  }
  if (two) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      rn[a] = r[a] + g.dt * (v1[a] - v2[a]);
      float dr = rn[a] - r[a];
      if (a < D) de2[a] = de1[a] - dr * g.idx[a];
    }
  }
  const float dxdt[3] = {g.dx[0] / g.dt, g.dx[1] / g.dt, g.dx[2] / g.dt};
  // fast path when every position keeps one nearest node per axis
  bool fast = true;
  float xi[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
  int nn[3] = {2, 2, 2};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const float u1p = f[a] >= 0.5f ? 1.0f : 0.0f;
    xi[0][a] = f[a] - u1p;
    const float x1n = xi[0][a] + de1[a];
    fast &= (x1n >= -0.5f) && (x1n < 0.5f);
    nn[a] = d[a] + Box<D>::OJ + (int)u1p;
    if (two) {
      const float u2p = f2[a] >= 0.5f ? 1.0f : 0.0f;
      xi[1][a] = f2[a] - u2p;
      const float x2n = xi[1][a] + de2[a];
      fast &= (d2[a] == d[a]) && (u2p == u1p) && (x2n >= -0.5f) && (x2n < 0.5f);
    }
  }
  if (!fast && qbuf) {
    int slot = atomicAdd(qn, 1);
    if (slot < qmax) {
      qbuf[slot] = (int)i;  // redone by the whole block after the main pass
      return;
    }
  }
  if (fast) {
    float qw[2] = {sp.qw1, sp.qw2};
    float vv[2][3];
    float dd[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      vv[0][a] = v1[a];
      vv[1][a] = v2[a];
      dd[0][a] = de1[a];
      dd[1][a] = de2[a];
    }
    if (two) esirkepov3<D, DET, 2>(Jsm, nn, xi, dd, qw, vv, dxdt, scale);
    else esirkepov3<D, DET, 1>(Jsm, nn, xi, dd, qw, vv, dxdt, scale);
  } else {
    general_deposit<D, DET, JT>(Jsm, g, f, de1, d, f2, de2, d2, two, sp.qw1, sp.qw2, v1, v2, scale);
  }
  // new cell of body 1.  On open axes a free particle whose cell leaves
  // [2, n-2) is removed (after its last deposit); a two-body ion leaving the
  // grid is a domain error.
  bool need_sort = false, nonfinite = false, removed = false;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (fn[a] >= 1.0f) {
      fn[a] -= 1.0f;
      c[a] += 1;
    } else if (fn[a] < 0.0f) {
      fn[a] += 1.0f;
      c[a] -= 1;
      if (fn[a] >= 1.0f) { fn[a] = 0.0f; c[a] += 1; }
    }
    if (g.bc[a] == BP_PERIODIC) {
      c[a] = wrap_mod(c[a], g.n[a]);
    } else if (two) {
      bad |= (c[a] < 0 || c[a] >= g.n[a]);
    } else {
      removed |= (c[a] < 2 || c[a] >= g.n[a] - 2);
    }
    int dn = rel_cell<D>(g, a, c[a], T0[a]);
    need_sort |= outside_margin<D>(a, dn);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) nonfinite |= !isfinite(u1[a]) || !isfinite(u2[a]);
  if (bad) atomicOr(status, ST_DOMAIN);
  if (nonfinite) atomicOr(status, ST_NONFINITE);
  if (bad || removed) {
    P.cell[i] = -1;
    return;
  }
  if (need_sort) atomicOr(status, ST_NEED_SORT);
  P.cell[i] = pack_cell(g, c[0], c[1], c[2]);
#pragma unroll
  for (int a = 0; a < D; ++a) P.off[a * cap + i] = fn[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) P.u1[a * cap + i] = u1[a];
  if (two) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      P.r[a * cap + i] = rn[a];
      P.u2[a * cap + i] = u2[a];
    }
  }
}

template <int D, bool DET>
__global__ void __launch_bounds__(D == 3 ? 512 : 256) k_push(GridP g, PushArgs A) {
  using JT = typename std::conditional<DET, long long, float>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  using BX = Box<D>;
  constexpr int JC = BX::JCELLS, GC = BX::GCELLS;
  JT *Jsm = reinterpret_cast<JT *>(smem);
  float *Gsm = reinterpret_cast<float *>(smem + sizeof(JT) * 3 * (size_t)JC);
  const int t = blockIdx.x;
  const int tid = threadIdx.x, bs = blockDim.x;
  int total = 0;
  for (int s = 0; s < A.nsp; ++s) total += A.p[s].tstart[t + 1] - A.p[s].tstart[t];
  if (total == 0) {
    if (tid == 0) A.occ[t] = 0;
    return;
  }
  int tc[3];
  tc[0] = t % g.nt[0];
  tc[1] = (t / g.nt[0]) % g.nt[1];
  tc[2] = t / (g.nt[0] * g.nt[1]);
  const int T0[3] = {tc[0] * Geo<D>::L0, tc[1] * Geo<D>::L1, tc[2] * Geo<D>::L2};
  for (int q = tid; q < 3 * JC; q += bs) Jsm[q] = (JT)0;
  // stage E, B of the tile plus halo (zero outside open faces)
  for (int q = tid; q < GC; q += bs) {
    int b0 = q % BX::G0, b1 = (q / BX::G0) % BX::G1, b2 = q / (BX::G0 * BX::G1);
    int bidx[3] = {b0, b1, b2};
    long long gi = 0, stride = 1;
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int x = T0[a] - (a < D ? BX::OG : 0) + bidx[a];
      if (a < D) {
        if (g.bc[a] == BP_PERIODIC) x = wrap_mod(x, g.n[a]);
        else ok &= (x >= 0 && x < g.n[a]);
      }
      gi += (long long)x * stride;
      stride *= g.n[a];
    }
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      Gsm[cc * GC + q] = ok ? __ldg(A.E[cc] + gi) : 0.0f;
      Gsm[(3 + cc) * GC + q] = ok ? __ldg(A.B[cc] + gi) : 0.0f;
    }
  }
  __syncthreads();
  constexpr int QMAX = 512;
  __shared__ int qbuf[QMAX];
  __shared__ int qn;
  for (int s = 0; s < A.nsp; ++s) {
    if (tid == 0) qn = 0;
    __syncthreads();
    const int beg = A.p[s].tstart[t], end = A.p[s].tstart[t + 1];
    for (long long i = beg + tid; i < end; i += bs)
      push_particle<D, DET, JT>(g, A.sp[s], A.p[s], i, T0, Gsm, Jsm, A.status, A.jscale, qbuf, &qn, QMAX);
    __syncthreads();
    // particles leaving their node: general five-node window, compacted
    const int nq = min(qn, QMAX);
    for (int k = tid; k < nq; k += bs)
      push_particle<D, DET, JT>(g, A.sp[s], A.p[s], qbuf[k], T0, Gsm, Jsm, A.status, A.jscale, nullptr, nullptr, 0);
    __syncthreads();
  }
  float *out = A.jbox + (size_t)t * 3 * JC;
  for (int q = tid; q < 3 * JC; q += bs) {
    if constexpr (DET) out[q] = (float)((double)Jsm[q] * (double)A.jinv);
    else out[q] = Jsm[q];
  }
  if (tid == 0) A.occ[t] = 1;
}

template <int D, bool DET>
void launch_one(const GridP &g, const PushArgs &a, cudaStream_t s) {
  size_t smem = push_smem_bytes(g, DET);
  k_push<D, DET><<<g.ntiles, D == 3 ? 512 : 256, smem, s>>>(g, a);
}

template <int D, bool DET>
int prepare_one(const GridP &g) {
  size_t smem = push_smem_bytes(g, DET);
  cudaError_t e = cudaFuncSetAttribute(k_push<D, DET>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e == cudaSuccess ? 0 : -1;
}

}  // namespace

size_t push_smem_bytes(const GridP &g, int det) {
  int jc = 0, gc = 0;
  if (g.D == 1) { jc = Box<1>::JCELLS; gc = Box<1>::GCELLS; }
  if (g.D == 2) { jc = Box<2>::JCELLS; gc = Box<2>::GCELLS; }
  if (g.D == 3) { jc = Box<3>::JCELLS; gc = Box<3>::GCELLS; }
  return (det ? 8 : 4) * (size_t)3 * jc + 4 * (size_t)6 * gc;
}

int push_prepare(const GridP &g, int det) {
  switch (g.D * 2 + (det ? 1 : 0)) {
    case 2: return prepare_one<1, false>(g);
    case 3: return prepare_one<1, true>(g);
    case 4: return prepare_one<2, false>(g);
    case 5: return prepare_one<2, true>(g);
    case 6: return prepare_one<3, false>(g);
    default: return prepare_one<3, true>(g);
  }
}

void launch_push(const GridP &g, const PushArgs &a, cudaStream_t s) {
  const bool det = a.jscale != 0.0f;
  switch (g.D * 2 + (det ? 1 : 0)) {
    case 2: launch_one<1, false>(g, a, s); break;
    case 3: launch_one<1, true>(g, a, s); break;
    case 4: launch_one<2, false>(g, a, s); break;
    case 5: launch_one<2, true>(g, a, s); break;
    case 6: launch_one<3, false>(g, a, s); break;
    default: launch_one<3, true>(g, a, s); break;
  }
}
