// k_push.cu -- the particle step: gather at both bodies, internal
// modified-Coulomb field, relativistic Boris push of both bodies, drift and
// Esirkepov (quadratic shape) current deposit.
//
// Method: arXiv 2208.08038 Sec. 2 (two-body macro-ion, Boris equations,
// modified Coulomb force, body currents q v / dV).  Per step:
//   k_push_quiet  tiles whose neighbourhood never held a field (the field
//                 kernels' tile marks): their co-moving neutral ions only
//                 drift; the other tiles go on a list for the push,
//   k_push        persistent blocks walk that list; per tile:
//     1. stage E and B of the tile plus halo in shared memory (FP32, by
//        asynchronous copies issued while the block finishes the previous
//        tile),
//     2. push every particle of the tile (all species), accumulating the
//        current of both bodies in a shared-memory box (tile + halo).  A
//        particle whose bodies keep their nearest nodes deposits on the spot
//        (three-node windows); the others leave a five-node record.  The box
//        holds
//          BP_DEPOSIT_SORTED: 64-bit fixed point (integer adds are
//                             associative: the same sums in any order),
//          BP_DEPOSIT_ATOMIC: FP32 shared atomics,
//     3. sorted mode: add every non-zero node of the box to the global 64-bit
//        fixed-point current; atomic mode: write the box to the tile's slot
//        for the current-sum kernel (and deposit the records from a
//        shared-memory queue before that),
//   k_records     sorted mode: the records' rows added to the fixed-point
//                 current,
//   k_push_far    sorted mode: the ions k_push left on the far list (a bound
//                 electron a cell or more from its nucleus), pushed with the
//                 global fields and deposited as one-body records,
//   k_tile_active the tiles the field kernels update this step: those whose
//                 neighbourhood has held a field or holds moved particles,
//                 those next to an antenna plane, every tile after a far push.
#include <type_traits>

#include "bp_internal.cuh"
#include "bp_particle.cuh"

namespace {

// capacity of the deferred-deposit records per tile (shared memory); a tile
// with more general-case particles deposits the rest in place
__host__ __device__ constexpr int push_qmax(int D) { return D == 2 ? 128 : 64; }
// threads of a push block
__host__ __device__ constexpr int push_threads(int D) { return D == 3 ? 512 : 256; }

// add v (already in fixed-point units in the sorted mode) to a current node:
// sorted mode, the exact fixed-point add fx_add (low words of the box, high
// words 3 * JCELLS entries later); atomic mode, an FP32 shared atomic.  Zero
// contributions are skipped where SKIP0.
template <int D, bool DET, bool SKIP0 = true, typename JT>
__device__ __forceinline__ void jput(JT *p, float v) {
  if constexpr (DET) {
    if (SKIP0 && fabsf(v) <= 0.5f) return;
    fx_add(p, 3 * Box<D>::JCELLS, v);
  } else {
    if (SKIP0 && v == 0.0f) return;
    atomicAdd(p, v);
  }
}

template <int D, bool DET, typename JT>
__device__ __forceinline__ void jadd(JT *p, float v, float scale) {
  jput<D, DET>(p, DET ? v * scale : v);
}

// Fast path: all four positions (both bodies, before and after the move)
// share one nearest node per axis, so the window is the three nodes around
// it and S1 - S0 has a closed form in the move d (no cancellation):
//   node n-1: -d (1 - 2 xi - d) / 2,  node n: -d (2 xi + d),  node n+1: d (1 + 2 xi + d) / 2
// with xi = old position - n.  J along a simulated axis then lives on the two
// faces inside the window, with partial sums DS(n-1) and DS(n-1) + DS(n) =
// -DS(n+1).  The Esirkepov factor of the two transverse axes is written
//   S0y S0z + (DSy S0z + S0y DSz)/2 + DSy DSz/3 = Ay Az + DSy DSz/12,
// A = S0 + DS/2 the mid-step shape.  In the sorted mode the charge factors
// carry the fixed-point scale (a power of two, so the products round
// exactly as unscaled ones).  The two bodies' terms are added without FMA
// contraction so that a neutral pair moving together cancels exactly.
template <int D, bool DET, int NB, typename JT>
__device__ __forceinline__ void esirkepov3(JT *__restrict__ J, const int n[3], const float (*xi)[3],
                                           const float (*de)[3], const float *qw, const float (*v)[3],
                                           const float dxdt[3], float scale) {
  constexpr int jcells = Box<D>::JCELLS;
  constexpr float K12 = 1.0f / 12.0f;
  const float sc = DET ? scale : 1.0f;
  float A[NB][3][3], DS[NB][3][3], DK[NB][3][3], cP[NB][3][2];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a < D) {
        const float x = xi[b][a], d = de[b][a];
        float S0[3];
        qweights(x, S0);
        const float d0 = -0.5f * d * (1.0f - 2.0f * x - d);
        const float d1 = -d * (2.0f * x + d);
        const float d2 = 0.5f * d * (1.0f + 2.0f * x + d);
        A[b][a][0] = fmaf(0.5f, d0, S0[0]);
        A[b][a][1] = fmaf(0.5f, d1, S0[1]);
        A[b][a][2] = fmaf(0.5f, d2, S0[2]);
        DS[b][a][0] = d0;
        DS[b][a][1] = d1;
        DS[b][a][2] = d2;
        DK[b][a][0] = K12 * d0;
        DK[b][a][1] = K12 * d1;
        DK[b][a][2] = K12 * d2;
        const float c = -qw[b] * dxdt[a] * sc;
        cP[b][a][0] = c * d0;
        cP[b][a][1] = -c * d2;
      } else {
        A[b][a][0] = A[b][a][2] = 0.0f;
        A[b][a][1] = 1.0f;
        DS[b][a][0] = DS[b][a][1] = DS[b][a][2] = 0.0f;
        DK[b][a][0] = DK[b][a][1] = DK[b][a][2] = 0.0f;
        cP[b][a][0] = cP[b][a][1] = 0.0f;
      }
    }
  JT *Jx = J, *Jy = J + jcells, *Jz = J + 2 * jcells;
  const int bx = n[0] - 1, by = n[1] - 1, bz = n[2] - 1;
  if constexpr (D == 1) {
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      float jx = cP[0][0][f];
      if constexpr (NB == 2) jx = __fadd_rn(jx, cP[1][0][f]);
      jput<D, DET, false>(Jx + bx + f, jx);
    }
    float qy[NB], qz[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      qy[b] = qw[b] * v[b][1] * sc;
      qz[b] = qw[b] * v[b][2] * sc;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float jy = __fmul_rn(qy[0], A[0][0][i]), jz = __fmul_rn(qz[0], A[0][0][i]);
      if constexpr (NB == 2) {
        jy = __fadd_rn(jy, __fmul_rn(qy[1], A[1][0][i]));
        jz = __fadd_rn(jz, __fmul_rn(qz[1], A[1][0][i]));
      }
      jput<D, DET, false>(Jy + bx + i, jy);
      jput<D, DET, false>(Jz + bx + i, jz);
    }
  } else if constexpr (D == 2) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int f = 0; f < 2; ++f) {
        float jx = __fmul_rn(cP[0][0][f], A[0][1][j]);
        if constexpr (NB == 2) jx = __fadd_rn(jx, __fmul_rn(cP[1][0][f], A[1][1][j]));
        jput<D, DET, false>(Jx + Box<D>::ji(bx + f, by + j, 0), jx);
      }
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float jy = __fmul_rn(cP[0][1][g], A[0][0][i]);
        if constexpr (NB == 2) jy = __fadd_rn(jy, __fmul_rn(cP[1][1][g], A[1][0][i]));
        jput<D, DET, false>(Jy + Box<D>::ji(bx + i, by + g, 0), jy);
      }
    float qz[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) qz[b] = qw[b] * v[b][2] * sc;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float jz = __fmul_rn(qz[0], fmaf(A[0][0][i], A[0][1][j], DK[0][0][i] * DS[0][1][j]));
        if constexpr (NB == 2)
          jz = __fadd_rn(jz, __fmul_rn(qz[1], fmaf(A[1][0][i], A[1][1][j], DK[1][0][i] * DS[1][1][j])));
        jput<D, DET, false>(Jz + Box<D>::ji(bx + i, by + j, 0), jz);
      }
  } else {
    // The outer loop of each pass stays rolled (its weights picked by
    // selects): the fully unrolled 54-node form is about three times the
    // code, and the kernel's hot path then outgrows the instruction caches.
#pragma unroll 1
    for (int k = 0; k < 3; ++k) {
      float azk[NB], dzk[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        azk[b] = k == 0 ? A[b][2][0] : (k == 1 ? A[b][2][1] : A[b][2][2]);
        dzk[b] = k == 0 ? DS[b][2][0] : (k == 1 ? DS[b][2][1] : DS[b][2][2]);
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        float F[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) F[b] = fmaf(A[b][1][j], azk[b], DK[b][1][j] * dzk[b]);
#pragma unroll
        for (int f = 0; f < 2; ++f) {
          float jx = __fmul_rn(cP[0][0][f], F[0]);
          if constexpr (NB == 2) jx = __fadd_rn(jx, __fmul_rn(cP[1][0][f], F[1]));
          jput<D, DET, false>(Jx + Box<D>::ji(bx + f, by + j, bz + k), jx);
        }
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float F[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) F[b] = fmaf(A[b][0][i], azk[b], DK[b][0][i] * dzk[b]);
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          float jy = __fmul_rn(cP[0][1][g], F[0]);
          if constexpr (NB == 2) jy = __fadd_rn(jy, __fmul_rn(cP[1][1][g], F[1]));
          jput<D, DET, false>(Jy + Box<D>::ji(bx + i, by + g, bz + k), jy);
        }
      }
    }
#pragma unroll 1
    for (int j = 0; j < 3; ++j) {
      float ayj[NB], dyj[NB];
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        ayj[b] = j == 0 ? A[b][1][0] : (j == 1 ? A[b][1][1] : A[b][1][2]);
        dyj[b] = j == 0 ? DS[b][1][0] : (j == 1 ? DS[b][1][1] : DS[b][1][2]);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float F[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) F[b] = fmaf(A[b][0][i], ayj[b], DK[b][0][i] * dyj[b]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float jz = __fmul_rn(cP[0][2][h], F[0]);
          if constexpr (NB == 2) jz = __fadd_rn(jz, __fmul_rn(cP[1][2][h], F[1]));
          jput<D, DET, false>(Jz + Box<D>::ji(bx + i, by + j, bz + h), jz);
        }
      }
    }
  }
}

__device__ __forceinline__ float2 sel3(int k, const float2 *a) { return k == 0 ? a[0] : (k == 1 ? a[1] : a[2]); }

// esirkepov3 for a two-body ion in 3D, sorted mode, on Blackwell's packed
// FP32 pairs (FFMA2): the two bodies in the lanes of every setup term and of
// each row's transverse factor F; a node's value is the bodies' two products
// (one packed multiply) added, and a row's two nodes go through one packed
// fixed-point split (fx_add2).  The outer loops stay rolled as in the scalar
// form (code size).
__device__ __forceinline__ void esirkepov3_p3(unsigned int *__restrict__ J, const int n[3], const float (*xi)[3],
                                              const float (*de)[3], const float *qw, const float dxdt[3],
                                              float scale) {
  constexpr int jcells = Box<3>::JCELLS;
  constexpr int hoff = 3 * jcells;
  const float2 K12 = make_float2(1.0f / 12.0f, 1.0f / 12.0f), H = make_float2(0.5f, 0.5f);
  const float2 M1 = make_float2(-1.0f, -1.0f), ONE = make_float2(1.0f, 1.0f);
  float2 A[3][3], DS[3][3], DK[3][3], cP[3][2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float2 x = make_float2(xi[0][a], xi[1][a]), d = make_float2(de[0][a], de[1][a]);
    float2 S0[3];
    qweights2(x, S0);
    const float2 u = __fadd2_rn(__fadd2_rn(x, x), d);
    float2 dd[3];
    dd[0] = __fmul2_rn(__fmul2_rn(d, make_float2(-0.5f, -0.5f)), __ffma2_rn(u, M1, ONE));
    dd[1] = __fmul2_rn(__fmul2_rn(d, M1), u);
    dd[2] = __fmul2_rn(__fmul2_rn(d, H), __fadd2_rn(u, ONE));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      A[a][i] = __ffma2_rn(H, dd[i], S0[i]);
      DS[a][i] = dd[i];
      DK[a][i] = __fmul2_rn(K12, dd[i]);
    }
    const float2 c = make_float2(-qw[0] * dxdt[a] * scale, -qw[1] * dxdt[a] * scale);
    cP[a][0] = __fmul2_rn(c, dd[0]);
    cP[a][1] = __fmul2_rn(__fmul2_rn(c, M1), dd[2]);
  }
  unsigned int *Jx = J, *Jy = J + jcells, *Jz = J + 2 * jcells;
  const int bx = n[0] - 1, by = n[1] - 1, bz = n[2] - 1;
#pragma unroll 1
  for (int k = 0; k < 3; ++k) {
    const float2 az = sel3(k, A[2]), dz = sel3(k, DS[2]);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float2 F = __ffma2_rn(A[1][j], az, __fmul2_rn(DK[1][j], dz));
      const float2 t0 = __fmul2_rn(cP[0][0], F), t1 = __fmul2_rn(cP[0][1], F);
      unsigned int *p = Jx + Box<3>::ji(bx, by + j, bz + k);
      fx_add2(p, p + 1, hoff, make_float2(__fadd_rn(t0.x, t0.y), __fadd_rn(t1.x, t1.y)));
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float2 F = __ffma2_rn(A[0][i], az, __fmul2_rn(DK[0][i], dz));
      const float2 t0 = __fmul2_rn(cP[1][0], F), t1 = __fmul2_rn(cP[1][1], F);
      unsigned int *p = Jy + Box<3>::ji(bx + i, by, bz + k);
      fx_add2(p, p + Box<3>::J0, hoff, make_float2(__fadd_rn(t0.x, t0.y), __fadd_rn(t1.x, t1.y)));
    }
  }
#pragma unroll 1
  for (int j = 0; j < 3; ++j) {
    const float2 ay = sel3(j, A[1]), dy = sel3(j, DS[1]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float2 F = __ffma2_rn(A[0][i], ay, __fmul2_rn(DK[0][i], dy));
      const float2 t0 = __fmul2_rn(cP[2][0], F), t1 = __fmul2_rn(cP[2][1], F);
      unsigned int *p = Jz + Box<3>::ji(bx + i, by + j, bz);
      fx_add2(p, p + Box<3>::JP, hoff, make_float2(__fadd_rn(t0.x, t0.y), __fadd_rn(t1.x, t1.y)));
    }
  }
}

// Deferred general deposits.  A thread whose particle leaves the fast path
// finishes the push and stores the particle's five-node windows in a record,
// deposited row by row (one row: one current component along one line of the
// window) by many threads, so the rare general case does not leave most of a
// block idle.  Sorted mode: the records go to a global buffer and a separate
// kernel adds their rows to the fixed-point current; atomic mode: a
// shared-memory queue the block deposits after its pass.
struct QRec {
  float S0[2][3][5];
  float DS[2][3][5];
  float cq[2][3];  // component along a simulated axis: -qw dx/dt; otherwise qw v
  int n0[2][3];    // window centre, box coordinates
  int nb;
  int org[3];      // grid coordinates of box node 0 (unwrapped)
};

// a general-case particle's deposit inputs, gathered into one object inside
// the rare branch (so the main path's arrays stay in registers)
struct QIn {
  float f[3], de1[3], f2[3], de2[3], v1[3], v2[3], dxdt[3];
  int d[3], d2[3];
  float qw1, qw2;
  int two;
};

template <int D>
__device__ __noinline__ void queue_record(QRec &R, const QIn &in) {
  float S0[3][5], DS[3][5];
  int n0[3];
  const int nb = in.two ? 2 : 1;
  for (int b = 0; b < nb; ++b) {
    window<D>(b ? in.f2 : in.f, b ? in.de2 : in.de1, S0, DS, n0, b ? in.d2 : in.d);
    const float qw = b ? in.qw2 : in.qw1;
    const float *v = b ? in.v2 : in.v1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        R.S0[b][a][m] = S0[a][m];
        R.DS[b][a][m] = DS[a][m];
      }
      R.n0[b][a] = n0[a];
      R.cq[b][a] = a < D ? -qw * in.dxdt[a] : qw * v[a];
    }
  }
  R.nb = nb;
}

// rows of component c: one per node of the window along each simulated axis
// other than c
template <int D>
__host__ __device__ constexpr int qrows(int c) {
  return (((c == 0 ? 1 : 0) < D) ? 5 : 1) * (((c == 2 ? 1 : 2) < D) ? 5 : 1);
}

// the contributions of one row: sink(c, x, y, z, v) per node, box
// coordinates, v in the deposit's units before the fixed-point scale
template <int D, typename Sink>
__device__ __forceinline__ void record_row(const QRec &R, int b, int c, int row, Sink &&sink) {
  const int p = c == 0 ? 1 : 0, q = c == 2 ? 1 : 2;  // the other two axes, p < q
  const int ip = p < D ? row % 5 : 2, iq = q < D ? row / 5 : 2;
  const float sp = R.S0[b][p][ip], dp = R.DS[b][p][ip], sq = R.S0[b][q][iq], dq = R.DS[b][q][iq];
  const float fac = sp * sq + 0.5f * (dp * sq + sp * dq) + (1.0f / 3.0f) * dp * dq;
  if (fac == 0.0f) return;
  int node[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) node[a] = 0;
  if (p < D) node[p] = R.n0[b][p] - 2 + ip;
  if (q < D) node[q] = R.n0[b][q] - 2 + iq;
  const float cq = R.cq[b][c];
  if (c < D) {
    float run = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      run += R.DS[b][c][i];
      node[c] = R.n0[b][c] - 2 + i;
      sink(c, node[0], node[1], node[2], cq * run * fac);
    }
  } else {
    sink(c, node[0], node[1], node[2], cq * fac);
  }
}

template <int D, bool DET, typename JT>
__device__ __forceinline__ void queued_row(JT *J, const QRec &R, int b, int c, int row, float scale) {
  record_row<D>(R, b, c, row, [&](int cc, int x, int y, int z, float v) {
    jadd<D, DET>(J + cc * Box<D>::JCELLS + Box<D>::ji(x, y, z), v, scale);
  });
}

// a general-case particle when the record queue is full: the same rows, in
// place (so the sorted mode's sums do not depend on which particles overflow)
template <int D, bool DET, typename JT>
__device__ __noinline__ void deposit_in_place(JT *Jsm, const QIn &in, float scale) {
  QRec R;
  queue_record<D>(R, in);
  constexpr int NR0 = qrows<D>(0), NR1 = qrows<D>(1), IPB = NR0 + NR1 + qrows<D>(2);
  for (int b = 0; b < R.nb; ++b)
    for (int it = 0; it < IPB; ++it) {
      const int c = it < NR0 ? 0 : (it < NR0 + NR1 ? 1 : 2);
      const int row = it - (c == 0 ? 0 : (c == 1 ? NR0 : NR0 + NR1));
      queued_row<D, DET, JT>(Jsm, R, b, c, row, scale);
    }
}

// one row of a record added to the global fixed-point current (sorted
// mode): each contribution rounded to the fixed-point unit as the
// shared-memory path rounds it; grid coordinates = the record's origin + box
// coordinates (periodic axes wrapped, nodes beyond an open face dropped, as
// the push drops them)
template <int D>
__device__ __forceinline__ void record_row_global(const GridP &g, const QRec &R, int b, int c, int row,
                                                  unsigned long long *jfx, float scale) {
  record_row<D>(R, b, c, row, [&](int cc, int x, int y, int z, float v) {
    const float vs = v * scale;
    if (fabsf(vs) <= 0.5f) return;  // rounds to zero
    const int bx[3] = {x, y, z};
    long long gidx = 0, stride = 1;
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int cg = R.org[a] + bx[a];
      if (a < D) {
        if (g.bc[a] == BP_PERIODIC) cg = wrap_once(cg, g.n[a]);
        else ok &= (cg >= 0 && cg < g.n[a]);
      }
      gidx += (long long)cg * stride;
      stride *= g.n[a];
    }
    if (ok) atomicAdd(jfx + (size_t)cc * g.ncell + gidx, (unsigned long long)f2ll_rn(vs));
  });
}

// a one-body deposit with its own grid origin org (a bound electron pulled
// a cell or more from its nucleus, outside the tile's current box): queued as
// a record for k_records, or, when the record buffer is full, added to the
// global current here
template <int D>
__device__ __noinline__ void deposit_far(const GridP &g, const QIn &in, const int org[3], QRec *qrec, int *qn,
                                         int qmax, unsigned long long *jfx, float scale) {
  const int slot = atomicAdd(qn, 1);
  if (slot < qmax) {
    queue_record<D>(qrec[slot], in);
#pragma unroll
    for (int a = 0; a < 3; ++a) qrec[slot].org[a] = org[a];
    return;
  }
  QRec R;
  queue_record<D>(R, in);
#pragma unroll
  for (int a = 0; a < 3; ++a) R.org[a] = org[a];
  constexpr int NR0 = qrows<D>(0), NR1 = qrows<D>(1), IPB = NR0 + NR1 + qrows<D>(2);
  for (int it = 0; it < IPB; ++it) {
    const int c = it < NR0 ? 0 : (it < NR0 + NR1 ? 1 : 2);
    const int row = it - (c == 0 ? 0 : (c == 1 ? NR0 : NR0 + NR1));
    record_row_global<D>(g, R, 0, c, row, jfx, scale);
  }
}

// E and B of one body read from the global fields (a body outside the
// tile's staged box): the staggered quadratic gather over the body's cell c
// and offset f, periodic axes wrapped, zero beyond open faces
template <int D>
__device__ __noinline__ void gather_global(const GridP &g, const float *const *Eg, const float *const *Bg,
                                           const int c[3], const float f[3], float E[3], float B[3]) {
#pragma unroll 1
  for (int cc = 0; cc < 6; ++cc) {
    // stagger pattern of component cc: bit a set when it sits half a cell along a
    const int pat = cc < 3 ? (1 << cc) : (7 & ~(1 << (cc - 3)));
    const float *F = cc < 3 ? Eg[cc] : Bg[cc - 3];
    int base[3];
    float w[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a < D) {
        const bool half = (pat >> a) & 1;
        const int up = half ? 0 : (f[a] >= 0.5f ? 1 : 0);
        base[a] = c[a] + up - 1;
        qweights(half ? f[a] - 0.5f : f[a] - (float)up, w[a]);
      } else {
        base[a] = 0;
        w[a][0] = 1.0f;
        w[a][1] = w[a][2] = 0.0f;
      }
    }
    float acc = 0.0f;
    for (int k = 0; k < (D >= 3 ? 3 : 1); ++k)
      for (int j = 0; j < (D >= 2 ? 3 : 1); ++j)
        for (int i = 0; i < 3; ++i) {
          const int n[3] = {base[0] + i, base[1] + j, base[2] + k};
          long long gi = 0, stride = 1;
          bool ok = true;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            int x = n[a];
            if (a < D) {
              if (g.bc[a] == BP_PERIODIC) x = wrap_once(x, g.n[a]);
              else ok &= (x >= 0 && x < g.n[a]);
            } else {
              x = 0;
            }
            gi += (long long)x * stride;
            stride *= g.n[a];
          }
          if (ok) acc = fmaf(w[0][i] * w[1][j] * w[2][k], F[gi], acc);
        }
    if (cc < 3) E[cc] = acc;
    else B[cc - 3] = acc;
  }
}

// node bounding box of a thread's deposits, one byte per axis (box
// coordinates are below 256); axes the grid does not simulate stay at 0
template <int D>
__device__ __forceinline__ void bb_add(unsigned &lo, unsigned &hi, const int n[3], int below, int above) {
  unsigned l = 0, h = 0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    l |= (unsigned)(n[a] - below) << (8 * a);
    h |= (unsigned)(n[a] + above) << (8 * a);
  }
  lo = __vminu4(lo, l);
  hi = __vmaxu4(hi, h);
}

// the five-node window's centre node (as window() places it)
template <int D>
__device__ __forceinline__ void window_centre(const float *f, const int *d, int n0[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) n0[a] = a < D ? d[a] + Box<D>::OJ + (f[a] >= 0.5f ? 1 : 0) : 0;
}

// 1 / gamma of a momentum u = p / (m c), one fixed evaluation order (the
// quiet pass and the full push must move a particle identically)
__device__ __forceinline__ float inv_gamma(const float u[3]) {
  return rsqrtf(fmaf(u[2], u[2], fmaf(u[1], u[1], fmaf(u[0], u[0], 1.0f))));
}

// body 1's offset after the drift x += dt v, in cells
__device__ __forceinline__ float drift_offset(const GridP &g, int a, float f, float v) {
  return fmaf(g.dt * v, g.idx[a], f);
}

// new cell of body 1 from its moved offset fn (renormalised to [0, 1)).  On
// open axes a free particle whose cell leaves [2, n-2) is removed (after its
// last deposit); a two-body ion leaving the grid is a domain error.
template <int D>
__device__ __forceinline__ void advance_cell(const GridP &g, const int T0[3], bool two, int c[3], float fn[3],
                                             bool &bad, bool &removed, bool &need_sort) {
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
      c[a] = wrap_once(c[a], g.n[a]);
    } else if (two) {
      bad |= (c[a] < 0 || c[a] >= g.n[a]);
    } else {
      removed |= (c[a] < 2 || c[a] >= g.n[a] - 2);
    }
    const int dn = rel_cell<D>(g, a, c[a], T0[a]);
    need_sort |= outside_margin<D>(a, dn);
  }
}

// A quiet ion: a neutral two-body ion whose bodies coincide (r = 0) and move
// together (u1 = u2, finite) in a tile whose staged fields are all zero.  The
// full push leaves its momenta and r exactly as they are (zero internal force
// at r = 0, zero fields) and deposits nothing (its bodies' terms cancel), so
// only body 1's drift remains.
__device__ __forceinline__ bool quiet_state(const float r[3], const float u1[3], const float u2[3]) {
  bool q = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) q &= (r[a] == 0.0f) && (u1[a] == u2[a]) && isfinite(u1[a]);
  return q;
}

// The quiet pass over QB particles of a thread (i0, i0 + bs, ...): all loads
// first, so that many are in flight, then the drift of the quiet ones, which
// writes only the cell and the offset.  Returns true when one of them is not
// quiet (left for the full push).
template <int D, int QB>
__device__ __forceinline__ bool quiet_batch(const GridP &g, const PartP &P, long long i0, int bs, long long end,
                                            const int T0[3], int *status, unsigned &moved) {
  const long long cap = P.cap;
  int cell[QB];
  float f[QB][3], u1[QB][3], u2[QB][3], r[QB][3];
#pragma unroll
  for (int q = 0; q < QB; ++q) {
    const long long i = i0 + (long long)q * bs;
    cell[q] = i < end ? P.cell[i] : -1;
    if (cell[q] >= 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        f[q][a] = a < D ? P.off[a * cap + i] : 0.0f;
        u1[q][a] = P.u1[a * cap + i];
        u2[q][a] = P.u2[a * cap + i];
        r[q][a] = P.r[a * cap + i];
      }
    }
  }
  bool left = false;
#pragma unroll
  for (int q = 0; q < QB; ++q) {
    if (cell[q] < 0) continue;
    if (!quiet_state(r[q], u1[q], u2[q])) {
      left = true;
      continue;
    }
    const long long i = i0 + (long long)q * bs;
    int c[3];
    unpack_cell(g, cell[q], c);
    bool bad = false, removed = false, need_sort = false;
#pragma unroll
    for (int a = 0; a < D; ++a) bad |= outside_margin<D>(a, rel_cell<D>(g, a, c[a], T0[a]));
    if (bad) {
      atomicOr(status, ST_DOMAIN);
      continue;
    }
    const float gi = inv_gamma(u1[q]);
    float fn[3];
#pragma unroll
    for (int a = 0; a < D; ++a) fn[a] = drift_offset(g, a, f[q][a], u1[q][a] * gi);
    advance_cell<D>(g, T0, true, c, fn, bad, removed, need_sort);
    if (bad) {
      atomicOr(status, ST_DOMAIN);
      P.cell[i] = -1;
      continue;
    }
    if (need_sort) atomicOr(status, ST_NEED_SORT);
    P.cell[i] = pack_cell(g, c[0], c[1], c[2]);
#pragma unroll
    for (int a = 0; a < D; ++a) P.off[a * cap + i] = fn[a];
    ++moved;
  }
  return left;
}

// add a per-thread count to a global work counter: one atomic per warp
__device__ __forceinline__ void count_work(unsigned long long *ctr, unsigned n) {
  const unsigned s = __reduce_add_sync(0xFFFFFFFFu, n);
  if ((threadIdx.x & 31u) == 0 && s) atomicAdd(ctr, (unsigned long long)s);
}

// whether the quiet pass has already moved particle i (its state is still
// quiet after the move: r, u1, u2 unchanged)
__device__ __forceinline__ bool quiet_done(const PartP &P, long long i) {
  const long long cap = P.cap;
  if (P.cell[i] < 0) return true;
  float r[3], u1[3], u2[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r[a] = P.r[a * cap + i];
    u1[a] = P.u1[a * cap + i];
    u2[a] = P.u2[a * cap + i];
  }
  return quiet_state(r, u1, u2);
}

// The whole step of a two-body ion whose bound electron is a cell or more
// from its nucleus (a strong field pulls it into the Coulomb tail of the
// modified potential), sorted mode: outside the tile's boxes, so both bodies
// gather from the global E and B and deposit as one-body records at their own
// grid origins (k_records adds them to the fixed-point current; directly
// when the record buffer is full).  The same arithmetic as push_particle's.
// Out of line and self-contained (it reloads the particle), so the common
// path carries none of it.  Returns false when the ion cannot be moved this
// way (body 1 outside its tile's margin, body 2 beyond an open face or a
// displacement that is not finite): a domain error for the caller.
template <int D>
__device__ __noinline__ bool push_far(const GridP &g, const SpecP &sp, const PartP &P, long long i, int t0x, int t0y,
                                      int t0z, int *status, QRec *qrec, int *qn, int qmax, const float *const *Eg,
                                      const float *const *Bg, unsigned long long *jfx, float scale) {
  const long long cap = P.cap;
  const int T0[3] = {t0x, t0y, t0z};
  int c[3];
  unpack_cell(g, P.cell[i], c);
  float f[3] = {0.0f, 0.0f, 0.0f}, r[3], u1[3], u2[3];
#pragma unroll
  for (int a = 0; a < D; ++a) f[a] = P.off[a * cap + i];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r[a] = P.r[a * cap + i];
    u1[a] = P.u1[a * cap + i];
    u2[a] = P.u2[a * cap + i];
  }
  int c2[3] = {0, 0, 0};
  float f2[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (outside_margin<D>(a, rel_cell<D>(g, a, c[a], T0[a]))) return false;
    const float rc = r[a] * g.idx[a];
    if (!(fabsf(rc) < (float)g.n[a])) return false;
    const float X = f[a] - rc;
    const float fl = floorf(X);
    float fr = X - fl;
    int di = (int)fl;
    if (fr >= 1.0f) { fr = 0.0f; di += 1; }
    c2[a] = c[a] + di;
    if (g.bc[a] == BP_PERIODIC) c2[a] = wrap_mod(c2[a], g.n[a]);
    else if (c2[a] < 0 || c2[a] >= g.n[a]) return false;
    f2[a] = fr;
  }
  float E1[3], B1[3], E2[3], B2[3];
  gather_global<D>(g, Eg, Bg, c, f, E1, B1);
  gather_global<D>(g, Eg, Bg, c2, f2, E2, B2);
  const int pi = P.pidx ? P.pidx[i] : 0;
  const float ac = sp.ac[pi];
  const float rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + ac * ac;
  const float rs = rsqrtf(rr);
  const float s = sp.kappa * rs * rs * rs;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    E1[a] = fmaf(sp.q2 * s, r[a], E1[a]);
    E2[a] = fmaf(-sp.q1 * s, r[a], E2[a]);
  }
  boris(sp.h2, E2, B2, u2);
  boris(sp.h1, E1, B1, u1);
  float v1[3], v2[3];
  const float g1 = inv_gamma(u1), g2 = inv_gamma(u2);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v1[a] = u1[a] * g1;
    v2[a] = u2[a] * g2;
  }
  float fn[3] = {0.0f, 0.0f, 0.0f}, de1[3] = {0.0f, 0.0f, 0.0f}, de2[3] = {0.0f, 0.0f, 0.0f}, rn[3];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    fn[a] = drift_offset(g, a, f[a], v1[a]);
    de1[a] = fn[a] - f[a];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    rn[a] = r[a] + g.dt * (v1[a] - v2[a]);
    if (a < D) de2[a] = de1[a] - (rn[a] - r[a]) * g.idx[a];
  }
  // each body a one-body record at its own grid origin (cell - OJ)
  QIn in;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    in.f[a] = f[a]; in.de1[a] = de1[a]; in.v1[a] = v1[a]; in.dxdt[a] = g.dx[a] / g.dt; in.d[a] = 0;
    in.f2[a] = in.de2[a] = in.v2[a] = 0.0f;
    in.d2[a] = 0;
  }
  in.qw1 = sp.qw1;
  in.qw2 = 0.0f;
  in.two = 0;
  int org[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) org[a] = a < D ? c[a] - Box<D>::OJ : 0;
  deposit_far<D>(g, in, org, qrec, qn, qmax, jfx, scale);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    in.f[a] = f2[a]; in.de1[a] = de2[a]; in.v1[a] = v2[a];
    org[a] = a < D ? c2[a] - Box<D>::OJ : 0;
  }
  in.qw1 = sp.qw2;
  deposit_far<D>(g, in, org, qrec, qn, qmax, jfx, scale);
  bool bad = false, removed = false, need_sort = false, nonfinite = false;
  advance_cell<D>(g, T0, true, c, fn, bad, removed, need_sort);
#pragma unroll
  for (int a = 0; a < 3; ++a) nonfinite |= !isfinite(u1[a]) || !isfinite(u2[a]);
  if (bad) atomicOr(status, ST_DOMAIN);
  if (nonfinite) atomicOr(status, ST_NONFINITE);
  if (bad) {
    P.cell[i] = -1;
    return true;
  }
  if (need_sort) atomicOr(status, ST_NEED_SORT);
  P.cell[i] = pack_cell(g, c[0], c[1], c[2]);
#pragma unroll
  for (int a = 0; a < D; ++a) P.off[a * cap + i] = fn[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    P.u1[a * cap + i] = u1[a];
    P.r[a * cap + i] = rn[a];
    P.u2[a * cap + i] = u2[a];
  }
  return true;
}

template <int D, bool DET, typename JT>
__device__ void push_particle(const GridP &g, const SpecP &sp, const PartP &P, long long i, const int T0[3],
                              const float *Gsm, JT *Jsm, int *status, float scale, QRec *qrec, int *qn, int qmax,
                              unsigned &blo, unsigned &bhi, bool nofield, int4 *far, int *far_n, int far_cap, int s,
                              int t) {
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
    // sorted mode: perhaps a bound electron a cell or more from its nucleus,
    // which k_push_far moves on the global grid after this kernel (it
    // reports a domain error for anything else); atomic mode: a domain error
    if (DET && two) {
      const int k = atomicAdd(far_n, 1);
      if (k < far_cap) {
        far[k] = make_int4(s, (int)i, t, 0);
        return;
      }
    }
    atomicOr(status, ST_DOMAIN);
    return;
  }
  // A tile whose staged E, B are all zero (ahead of the field front) gathers
  // exact zeros, so the gather is skipped.  A neutral ion there with r = 0 and
  // u1 = u2 also keeps its momenta exactly (no internal force at r = 0, Boris
  // rotation by zero fields), so its kicks are skipped too.
  bool quiet = nofield && two && sp.qw1 == -sp.qw2;
#pragma unroll
  for (int a = 0; a < 3; ++a) quiet &= (r[a] == 0.0f) && (u1[a] == u2[a]);
  float E1[3], B1[3], E2[3], B2[3];
  if (nofield) {
#pragma unroll
    for (int a = 0; a < 3; ++a) E1[a] = B1[a] = E2[a] = B2[a] = 0.0f;
  } else {
    if constexpr (D == 3) {
      Pos P1, P2;
      make_pos<D>(d, f, P1);
      make_pos<D>(two ? d2 : d, two ? f2 : f, P2);
      gather_all_p3(Gsm, P1, P2, E1, B1, E2, B2);
    } else {
      Loc L1, L2;
      make_loc<D>(d, f, L1);
      make_loc<D>(two ? d2 : d, two ? f2 : f, L2);
      gather_all<D>(Gsm, L1, L2, E1, B1, E2, B2);
    }
  }
  float v1[3], v2[3] = {0.0f, 0.0f, 0.0f};
  if (two && !quiet) {
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
  }
  if (two) {
    const float g2 = inv_gamma(u2);
#pragma unroll
    for (int a = 0; a < 3; ++a) v2[a] = u2[a] * g2;
  }
  if (!quiet) boris(sp.h1, E1, B1, u1);
  {
    const float g1 = inv_gamma(u1);
#pragma unroll
    for (int a = 0; a < 3; ++a) v1[a] = u1[a] * g1;
  }
  // drift: body 1 moves in cells by dt v / dx; the internal displacement by
  // dt (v1 - v2) on all three axes; the deposited moves are the ones the
  // stored FP32 state actually makes
  float fn[3] = {0.0f, 0.0f, 0.0f}, de1[3] = {0.0f, 0.0f, 0.0f}, de2[3] = {0.0f, 0.0f, 0.0f}, rn[3];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    fn[a] = drift_offset(g, a, f[a], v1[a]);
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
  // a neutral ion whose bodies coincide and move together carries no
  // current (its two bodies' terms cancel exactly; Sec. 2 starts every ion
  // so, and it stays so until a field acts on it): nothing to deposit
  bool silent = two && sp.qw1 == -sp.qw2;
#pragma unroll
  for (int a = 0; a < 3; ++a) silent &= (r[a] == 0.0f) && (v1[a] == v2[a]);
  if (!silent) {
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
      if constexpr (D == 3 && DET) {
        if (two) esirkepov3_p3(Jsm, nn, xi, dd, qw, dxdt, scale);
        else esirkepov3<D, DET, 1>(Jsm, nn, xi, dd, qw, vv, dxdt, scale);
      } else if (two) esirkepov3<D, DET, 2>(Jsm, nn, xi, dd, qw, vv, dxdt, scale);
      else esirkepov3<D, DET, 1>(Jsm, nn, xi, dd, qw, vv, dxdt, scale);
      bb_add<D>(blo, bhi, nn, 1, 1);
    } else {
      QIn in;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        in.f[a] = f[a]; in.de1[a] = de1[a]; in.f2[a] = f2[a]; in.de2[a] = de2[a];
        in.v1[a] = v1[a]; in.v2[a] = v2[a]; in.dxdt[a] = dxdt[a]; in.d[a] = d[a]; in.d2[a] = d2[a];
      }
      in.qw1 = sp.qw1;
      in.qw2 = sp.qw2;
      in.two = two;
      // sorted mode: qrec, qn, qmax are the global record buffer, its counter
      // and capacity; atomic mode: the block's shared-memory queue
      const int slot = atomicAdd(qn, 1);
      const bool queued = slot < qmax;
      if (queued) {
        queue_record<D>(qrec[slot], in);
#pragma unroll
        for (int a = 0; a < 3; ++a) qrec[slot].org[a] = T0[a] - (a < D ? Box<D>::OJ : 0);
      } else {
        deposit_in_place<D, DET, JT>(Jsm, in, scale);
      }
      if (!DET || !queued) {
        int n0[3];
        window_centre<D>(f, d, n0);
        bb_add<D>(blo, bhi, n0, 2, 2);
        if (two) {
          window_centre<D>(f2, d2, n0);
          bb_add<D>(blo, bhi, n0, 2, 2);
        }
      }
    }
  }
  bool need_sort = false, nonfinite = false, removed = false;
  advance_cell<D>(g, T0, two, c, fn, bad, removed, need_sort);
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

// the state of the particle a thread takes next, brought into L1 while the
// current one is pushed (its loads would otherwise stall the warp at the
// start of the next iteration)
template <int D>
__device__ __forceinline__ void prefetch_particle(const PartP &P, long long j, bool two) {
  const long long cp = P.cap;
  asm volatile("prefetch.global.L1 [%0];" ::"l"(P.cell + j));
#pragma unroll
  for (int a = 0; a < D; ++a) asm volatile("prefetch.global.L1 [%0];" ::"l"(P.off + a * cp + j));
#pragma unroll
  for (int a = 0; a < 3; ++a) asm volatile("prefetch.global.L1 [%0];" ::"l"(P.u1 + a * cp + j));
  if (two) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      asm volatile("prefetch.global.L1 [%0];" ::"l"(P.r + a * cp + j));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(P.u2 + a * cp + j));
    }
  }
}

// clear a shared-memory current box of n nodes (and the high words in the
// sorted mode), 16 bytes per store
template <bool DET, typename JT>
__device__ __forceinline__ void zero_box(JT *J, int n, int tid, int bs) {
  constexpr int W = DET ? 2 : 1;
  uint4 *p = reinterpret_cast<uint4 *>(J);
  const int n4 = (W * n) / 4;
  for (int q = tid; q < n4; q += bs) p[q] = make_uint4(0u, 0u, 0u, 0u);
  for (int q = 4 * n4 + tid; q < W * n; q += bs) reinterpret_cast<unsigned *>(J)[q] = 0u;
}

// A tile whose 3^D neighbouring tiles have never held a non-zero E or B has
// an all-zero field box (the box lies inside them).  This light kernel takes
// such tiles before the push: it moves their quiet ions (the drift alone) at
// high occupancy (eight 128-thread blocks per SM) and leaves a state per tile:
//   QS_PUSH  the push kernel does the whole tile (fields may be non-zero),
//   QS_DONE  every particle moved, nothing deposited (occ = 0),
//   QS_REST  the quiet ions moved; the push does the others without fields.
constexpr unsigned char QS_PUSH = 0, QS_DONE = 1, QS_REST = 2;

template <int D>
__global__ void __launch_bounds__(128, 8) k_push_quiet(GridP g, PushArgs A, int qt) {
  static_assert(Box<D>::OG <= Geo<D>::L0 && Box<D>::G0 - Box<D>::OG <= 2 * Geo<D>::L0 &&
                    (D < 2 || (Box<D>::OG <= Geo<D>::L1 && Box<D>::G1 - Box<D>::OG <= 2 * Geo<D>::L1)) &&
                    (D < 3 || (Box<D>::OG <= Geo<D>::L2 && Box<D>::G2 - Box<D>::OG <= 2 * Geo<D>::L2)),
                "field box within the neighbouring tiles");
  constexpr int QB = 2;  // particles in flight per thread (measured best of 1, 2, 4, 8)
  // qt (1 to 4) tiles per block: one warp classifies each, then the whole
  // block drifts the quiet ones in turn (several tiles per block on grids
  // with many tiles, where a block per tile spent its time waiting on the
  // classification loads; one on small grids, where tiles in turn would
  // lengthen the pass)
  __shared__ int quiet[4], nquiet;
  const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int t = (int)blockIdx.x * qt + warp;
  if (tid == 0) nquiet = 0;
  bool marked = false, occupied = false;
  if (warp < qt && t < g.ntiles) {
    const int tc[3] = {t % g.nt[0], (t / g.nt[0]) % g.nt[1], t / (g.nt[0] * g.nt[1])};
    if (lane < 27) {
      const int o[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
      bool use = true;
      int nb[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        nb[a] = tc[a] + o[a];
        if (a >= D) use &= o[a] == 0;
        else if (g.bc[a] == BP_PERIODIC) nb[a] = wrap_once(nb[a], g.nt[a]);
        else use &= nb[a] >= 0 && nb[a] < g.nt[a];
      }
      if (use) marked = g.fnz[nb[0] + g.nt[0] * (nb[1] + g.nt[1] * nb[2])] != 0;
    }
    // a tile without particles has nothing to push or deposit, whatever its
    // fields: done here, so the push neither stages its fields nor visits it
    if (lane < A.nsp) occupied = A.p[lane].tstart[t + 1] > A.p[lane].tstart[t];
  }
  marked = __any_sync(0xFFFFFFFFu, marked);
  occupied = __any_sync(0xFFFFFFFFu, occupied);
  __syncthreads();  // nquiet cleared
  if (warp < qt && t < g.ntiles && lane == 0) {
    if (!occupied) {
      A.qstate[t] = QS_DONE;
      A.occ[t] = 0;
    } else if (marked) {
      A.qstate[t] = QS_PUSH;
      A.tile_list[atomicAdd(A.tile_n, 1)] = t;
    } else {
      quiet[atomicAdd(&nquiet, 1)] = t;  // each quiet tile is drifted alone: their order changes nothing
    }
  }
  __syncthreads();
  const int nq = nquiet;
  unsigned moved = 0;
  for (int k = 0; k < nq; ++k) {
    const int tq = quiet[k];
    const int T0[3] = {(tq % g.nt[0]) * Geo<D>::L0, ((tq / g.nt[0]) % g.nt[1]) * Geo<D>::L1,
                       (tq / (g.nt[0] * g.nt[1])) * Geo<D>::L2};
    bool left = false;
    for (int s = 0; s < A.nsp; ++s) {
      const int beg = A.p[s].tstart[tq], end = A.p[s].tstart[tq + 1];
      if (A.sp[s].kind == BP_TWO_BODY && A.sp[s].qw1 == -A.sp[s].qw2) {
        for (long long i0 = beg + tid; i0 < end; i0 += (long long)QB * bs)
          left |= quiet_batch<D, QB>(g, A.p[s], i0, bs, end, T0, A.status, moved);
      } else {
        left |= end > beg;
      }
    }
    left = __syncthreads_or(left);
    if (tid == 0) {
      A.qstate[tq] = left ? QS_REST : QS_DONE;
      if (!left) A.occ[tq] = 0;
      else A.tile_list[atomicAdd(A.tile_n, 1)] = tq;
    }
  }
  if (A.work) count_work(A.work + 1, moved);
}

// Tiles whose cells the field updates can change: a tile of the 3^D
// neighbourhood has held a non-zero E or B (the sticky marks), or holds
// particles the push moved this step (QS_PUSH, QS_REST: their current reaches
// the neighbouring tiles), or an antenna plane lies within one tile of it.
// Elsewhere E, B and J are zero and the Yee updates keep them exactly zero,
// so the field kernels skip those tiles.  Computed after the push; it serves
// that step's field updates and the next step's first B half step, over
// which fields spread by at most three cells, less than one tile.
template <int D>
__global__ void k_tile_active(GridP g, const unsigned char *qstate, const int *far_any, int ia_lo, int ia_hi,
                              unsigned char *act, unsigned long long *act_n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) atomicAdd(act_n + 1, 1ull);  // the steps counted
  bool a = false;
  if (t < g.ntiles) {
    const int tc[3] = {t % g.nt[0], (t / g.nt[0]) % g.nt[1], t / (g.nt[0] * g.nt[1])};
    const int x0 = tc[0] * Geo<D>::L0;
    // a far bound electron deposits at its own position: every tile then
    a = (far_any && *far_any) || (ia_hi >= x0 - Geo<D>::L0 && ia_lo < x0 + 2 * Geo<D>::L0);
    for (int o = 0; o < 27 && !a; ++o) {
      const int off[3] = {o % 3 - 1, (o / 3) % 3 - 1, o / 9 - 1};
      bool use = true;
      int nb[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        nb[k] = tc[k] + off[k];
        if (k >= D) use &= off[k] == 0;
        else if (g.bc[k] == BP_PERIODIC) nb[k] = wrap_once(nb[k], g.nt[k]);
        else use &= nb[k] >= 0 && nb[k] < g.nt[k];
      }
      if (!use) continue;
      const int u = nb[0] + g.nt[0] * (nb[1] + g.nt[1] * nb[2]);
      a = g.fnz[u] != 0 || qstate[u] != QS_DONE;
    }
    act[t] = a ? 1 : 0;
  }
  const unsigned k = __reduce_add_sync(0xFFFFFFFFu, a ? 1u : 0u);
  if ((threadIdx.x & 31u) == 0 && k) atomicAdd(act_n, (unsigned long long)k);
}

// byte offset of the field box in the push's dynamic shared memory (after the
// current box, 128-byte aligned for the TMA loads)
__host__ __device__ constexpr size_t push_gbox_offset(int D, bool det) {
  return ((det ? 8 : 4) * (size_t)3 *
              (D == 1 ? Box<1>::JCELLS : (D == 2 ? Box<2>::JCELLS : Box<3>::JCELLS)) + 127) / 128 * 128;
}

// ---------------------------------------------------------------------------
// TMA staging of 3D field boxes: one cp.async.bulk.tensor load per component,
// completing on an mbarrier (transaction bytes), issued by one thread.

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// a bounded wait for the phase of the given parity: false when it gave up
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
  for (int it = 0; it < (1 << 20); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_3d(float *dst, const CUtensorMap *map, int x, int y, int z,
                                            unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Whether tile t's field box comes by TMA: 3D with maps, and no periodic
// axis wraps inside the box (TMA fills zeros outside the grid, which is what
// an open face reads; a wrapped box is staged by per-thread copies).
template <int D>
__device__ __forceinline__ bool tma_tile(const GridP &g, const TmaMaps &T, const int T0[3]) {
  if constexpr (D != 3) {
    return false;
  } else {
    // maps present, and the block's field box 128-byte aligned in shared memory
    extern __shared__ __align__(128) unsigned char smem[];
    if (!T.on || ((smem_u32(smem) + (unsigned)push_gbox_offset(3, true)) & 127u) ||
        ((smem_u32(smem) + (unsigned)push_gbox_offset(3, false)) & 127u))
      return false;
    using BX = Box<3>;
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int lo = T0[a] - BX::OG - (a == 0 ? BX::SX : 0);
      const int ext = a == 0 ? BX::GR : (a == 1 ? BX::G1 : BX::G2);
      if (g.bc[a] == BP_PERIODIC) ok &= lo >= 0 && lo + ext <= g.n[a];
    }
    return ok;
  }
}

// Staging of a tile's field box (E, B of the tile plus halo; zero outside
// open faces), in shared memory: by TMA where tma_tile allows (one thread
// issues six box loads), else by per-thread asynchronous copies.  Neither
// holds registers, so the copies run while the block finishes the previous
// tile.  A QS_REST tile's box is all zero and is not staged.
template <int D>
__device__ __forceinline__ void stage_issue(const GridP &g, const PushArgs &A, const TmaMaps &T, int t, float *Gsm,
                                            unsigned long long *bar) {
  using BX = Box<D>;
  constexpr int GC = BX::GCELLS;
  if (A.qstate[t] != QS_PUSH) return;
  const int tc[3] = {t % g.nt[0], (t / g.nt[0]) % g.nt[1], t / (g.nt[0] * g.nt[1])};
  const int T0[3] = {tc[0] * Geo<D>::L0, tc[1] * Geo<D>::L1, tc[2] * Geo<D>::L2};
  if (tma_tile<D>(g, T, T0)) {
    if (threadIdx.x == 0) {
      // the previous tile's box was read by ordinary loads before this point
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bar, 6u * 4u * (unsigned)(BX::GP * BX::G2));
#pragma unroll
      for (int cc = 0; cc < 6; ++cc)
        tma_load_3d(Gsm + cc * GC, &T.m[cc], T0[0] - BX::OG - BX::SX, T0[1] - BX::OG, T0[2] - BX::OG, bar);
    }
    return;
  }
  const unsigned gbase = smem_u32(Gsm);
  for (int q = threadIdx.x; q < BX::GCOMP; q += blockDim.x) {
    const int b0 = q % BX::G0, b1 = (q / BX::G0) % BX::G1, b2 = q / (BX::G0 * BX::G1);
    const int bidx[3] = {b0, b1, b2};
    const int si = BX::gi(b0, b1, b2);
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
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// wait for tile t's staging (this thread's copies, or the TMA loads: the
// mbarrier phase `phase`, flipped here after each TMA tile); whether any
// staged value is non-zero.  A TMA wait that gives up sets ST_TIMEOUT and
// `failed`.
template <int D>
__device__ __forceinline__ bool stage_done(const GridP &g, const PushArgs &A, const TmaMaps &T, int t,
                                           const float *Gsm, unsigned long long *bar, unsigned &phase, bool &failed) {
  using BX = Box<D>;
  constexpr int GC = BX::GCELLS;
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  bool nz = false;
  if (A.qstate[t] != QS_PUSH) return nz;
  const int tc[3] = {t % g.nt[0], (t / g.nt[0]) % g.nt[1], t / (g.nt[0] * g.nt[1])};
  const int T0[3] = {tc[0] * Geo<D>::L0, tc[1] * Geo<D>::L1, tc[2] * Geo<D>::L2};
  if (tma_tile<D>(g, T, T0)) {
    if (!mbar_wait(bar, phase)) {
      if (threadIdx.x == 0) atomicOr(A.status, ST_TIMEOUT);
      failed = !mbar_wait(bar, phase);  // one more bounded wait for the loads in flight
    }
    phase ^= 1u;
  }
  for (int q = threadIdx.x; q < BX::GCOMP; q += blockDim.x) {
    const int b0 = q % BX::G0, b1 = (q / BX::G0) % BX::G1, b2 = q / (BX::G0 * BX::G1);
    const int si = BX::gi(b0, b1, b2);
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) nz |= Gsm[cc * GC + si] != 0.0f;
  }
  return nz;
}

// one tile of the push (the block's work for tile t)
template <int D, bool DET, typename AfterLoop>
__device__ __forceinline__ void push_tile(const GridP &g, const PushArgs &A, const TmaMaps &T, const int t,
                                          unsigned long long *bar, unsigned &phase, bool &failed,
                                          AfterLoop &&after_loop) {
  using JT = typename std::conditional<DET, unsigned int, float>::type;
  extern __shared__ __align__(128) unsigned char smem[];
  using BX = Box<D>;
  constexpr int JC = BX::JCELLS, GC = BX::GCELLS;
  constexpr size_t GOFF = push_gbox_offset(D, DET);
  JT *Jsm = reinterpret_cast<JT *>(smem);
  float *Gsm = reinterpret_cast<float *>(smem + GOFF);
  const int tid = threadIdx.x, bs = blockDim.x;
  const unsigned char qs = A.qstate[t];
  int total = 0;
  for (int s = 0; s < A.nsp; ++s) total += A.p[s].tstart[t + 1] - A.p[s].tstart[t];
  if (qs == QS_DONE || total == 0) {
    stage_done<D>(g, A, T, t, Gsm, bar, phase, failed);  // this tile's copies land before the next tile's are issued
    __syncthreads();
    if (tid == 0 && qs != QS_DONE) A.occ[t] = 0;
    after_loop();
    return;
  }
  int tc[3];
  tc[0] = t % g.nt[0];
  tc[1] = (t / g.nt[0]) % g.nt[1];
  tc[2] = t / (g.nt[0] * g.nt[1]);
  const int T0[3] = {tc[0] * Geo<D>::L0, tc[1] * Geo<D>::L1, tc[2] * Geo<D>::L2};
  zero_box<DET>(Jsm, 3 * JC, tid, bs);
  // the field box was staged asynchronously (stage_issue) by the caller
  const bool nz = stage_done<D>(g, A, T, t, Gsm, bar, phase, failed);
  const bool nofield = !__syncthreads_or(nz);
  QRec *qrec = DET ? reinterpret_cast<QRec *>(A.grec)
                   : reinterpret_cast<QRec *>(smem + GOFF + sizeof(float) * 6 * (size_t)GC);
  int *const qcount = DET ? A.grec_n : nullptr;
  const int qmax = DET ? A.grec_cap : push_qmax(D);
  constexpr int NR0 = qrows<D>(0), NR1 = qrows<D>(1), IPB = NR0 + NR1 + qrows<D>(2);
  __shared__ int qn, run;
  __shared__ unsigned sbb[6];
  if (tid < 6) sbb[tid] = tid < 3 ? 0xFFFFFFFFu : 0u;
  unsigned blo = 0xFFFFFFFFu, bhi = 0u;
  unsigned pushed = 0;
  const int lane = tid & 31;
  for (int s = 0; s < A.nsp; ++s) {
    if (tid == 0) {
      qn = 0;
      run = 0;
    }
    __syncthreads();
    const int beg = A.p[s].tstart[t], end = A.p[s].tstart[t + 1], n = end - beg;
    // in a QS_REST tile the quiet ions of this species have already moved
    const bool moved = qs == QS_REST && A.sp[s].kind == BP_TWO_BODY && A.sp[s].qw1 == -A.sp[s].qw2;
    const bool two = A.sp[s].kind == BP_TWO_BODY;
    // Each warp takes runs of 32 consecutive (cell-sorted) particles from a
    // shared counter, one lane per particle: the lanes' gather loads share
    // addresses and their state loads coalesce, and a warp whose particles
    // took the rare paths does not hold the others at the tile's end.  The
    // next run is taken before the current one is pushed, so that its
    // particle can be prefetched.
    int r = 0;
    if (lane == 0) r = atomicAdd(&run, 32);
    r = __shfl_sync(0xFFFFFFFFu, r, 0);
    while (r < n) {
      int rn = 0;
      if (lane == 0) rn = atomicAdd(&run, 32);
      rn = __shfl_sync(0xFFFFFFFFu, rn, 0);
      const long long i = beg + r + lane;
      if (i < end && !(moved && quiet_done(A.p[s], i))) {
        if (rn + lane < n) prefetch_particle<D>(A.p[s], beg + rn + lane, two);
        push_particle<D, DET, JT>(g, A.sp[s], A.p[s], i, T0, Gsm, Jsm, A.status, A.jscale, qrec,
                                  DET ? qcount : &qn, qmax, blo, bhi, nofield, A.far, A.far_n, A.far_cap, s, t);
        ++pushed;
      }
      r = rn;
    }
    __syncthreads();
    if constexpr (DET) continue;  // the records are deposited by k_records
    // the deferred general deposits, one row per thread
    const int nitem = min(qn, qmax) * 2 * IPB;
    for (int k = tid; k < nitem; k += bs) {
      const int e = k / (2 * IPB), rem = k - e * (2 * IPB), b = rem / IPB, it = rem - b * IPB;
      if (b >= qrec[e].nb) continue;
      const int c = it < NR0 ? 0 : (it < NR0 + NR1 ? 1 : 2);
      const int row = it - (c == 0 ? 0 : (c == 1 ? NR0 : NR0 + NR1));
      queued_row<D, DET, JT>(Jsm, qrec[e], b, c, row, A.jscale);
    }
    __syncthreads();
  }
  if (A.work) count_work(A.work, pushed);
  // the field box is no longer needed: the caller may start staging the next tile
  after_loop();
  // the deposits' bounding box over the block
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const unsigned l = __reduce_min_sync(0xFFFFFFFFu, blo == 0xFFFFFFFFu ? 0xFFFFFFFFu : (blo >> (8 * a)) & 255u);
    const unsigned h = __reduce_max_sync(0xFFFFFFFFu, (bhi >> (8 * a)) & 255u);
    if ((tid & 31) == 0 && l != 0xFFFFFFFFu) {
      atomicMin(&sbb[a], l);
      atomicMax(&sbb[3 + a], h);
    }
  }
  __syncthreads();
  const bool any = sbb[0] != 0xFFFFFFFFu;
  // the box's occupied part to global memory.  Sorted mode: each non-zero
  // node, an exact 64-bit fixed-point sum, is added into the global
  // fixed-point current (integer adds: the same result in any order; nodes
  // beyond an open face hold no deposit the field sees).  Atomic mode: the
  // FP32 box to the tile's slot (compact layout) for the current-sum kernel.
  constexpr int JN = BX::JCOMP;
  if (any) {
    const int lo0 = sbb[0], lo1 = sbb[1], lo2 = sbb[2];
    const int nx = sbb[3] - lo0 + 1, ny = sbb[4] - lo1 + 1, nz = sbb[5] - lo2 + 1;
    const int nbox = nx * ny * nz;
    for (int q = tid; q < 3 * nbox; q += bs) {
      const int cc = q / nbox, r = q - cc * nbox;
      const int x = lo0 + r % nx, y = lo1 + (r / nx) % ny, z = lo2 + r / (nx * ny);
      const int k = cc * JC + BX::ji(x, y, z);
      if constexpr (DET) {
        const long long v = fx_value(Jsm + k, 3 * JC);
        if (v == 0) continue;
        const int bidx[3] = {x, y, z};
        long long gidx = 0, stride = 1;
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          int c = T0[a] - (a < D ? BX::OJ : 0) + bidx[a];
          if (a < D) {
            if (g.bc[a] == BP_PERIODIC) c = wrap_once(c, g.n[a]);
            else ok &= (c >= 0 && c < g.n[a]);
          }
          gidx += (long long)c * stride;
          stride *= g.n[a];
        }
        if (ok) atomicAdd(A.jfx + (size_t)cc * g.ncell + gidx, (unsigned long long)v);
      } else {
        A.jbox[(size_t)t * 3 * JN + cc * JN + x + BX::J0 * (y + BX::J1 * z)] = Jsm[k];
      }
    }
  }
  if (tid == 0) {
    A.occ[t] = any ? 1 : 0;
    A.jbb[t] = make_uint2(sbb[0] | (sbb[1] << 8) | (sbb[2] << 16), sbb[3] | (sbb[4] << 8) | (sbb[5] << 16));
  }
}

// The push: persistent blocks (as many as fit on the GPU at once) take the
// tiles the quiet-tile pass left (its list) in order from a counter, so a
// block's shared memory and setup are reused from tile to tile, and the next
// tile's field box is staged while the block finishes the current one.
template <int D, bool DET>
__global__ void __launch_bounds__(push_threads(D)) k_push(GridP g, PushArgs A, const __grid_constant__ TmaMaps T) {
  extern __shared__ __align__(128) unsigned char smem[];
  float *Gsm = reinterpret_cast<float *>(smem + push_gbox_offset(D, DET));
  __shared__ int next;
  __shared__ __align__(8) unsigned long long bar;  // completion of the TMA staging
  __shared__ int give_up;
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    give_up = 0;
  }
  __syncthreads();
  unsigned phase = 0;
  bool failed = false;
  const int nlist = *A.tile_n;
  // The next list entry is taken only once the block has finished the
  // current tile's particles: reserving it earlier would let one block hold
  // two costly tiles in a row while others have none (grids with few
  // occupied tiles ran 20% slower that way).
  auto grab = [&]() {
    if (threadIdx.x == 0) {
      const int k = atomicAdd(A.tile_ctr, 1);
      next = k < nlist ? A.tile_list[k] : -1;
    }
    __syncthreads();
    if (next >= 0) stage_issue<D>(g, A, T, next, Gsm, &bar);
  };
  grab();
  for (int t = next; t >= 0; t = next) {
    push_tile<D, DET>(g, A, T, t, &bar, phase, failed, grab);
    if (failed) give_up = 1;
    __syncthreads();  // every thread has read `next` before it changes
    if (give_up) break;  // a staging wait gave up twice (ST_TIMEOUT is set): stop
  }
  // nothing may be in flight into this block's shared memory when it exits
  if (next >= 0 && A.qstate[next] == QS_PUSH) stage_done<D>(g, A, T, next, Gsm, &bar, phase, failed);
}

// Sorted mode: the records' rows added to the fixed-point current.  Each
// contribution is rounded to the fixed-point unit as the shared-memory path
// rounds it (the same value, so the current does not depend on which path a
// particle took); nodes beyond an open face are dropped as the push drops them.
template <int D>
__global__ void __launch_bounds__(256) k_records(GridP g, const QRec *__restrict__ rec, const int *__restrict__ count,
                                                 int cap, unsigned long long *jfx, float scale) {
  constexpr int NR0 = qrows<D>(0), NR1 = qrows<D>(1), IPB = NR0 + NR1 + qrows<D>(2);
  const long long n = (long long)min(*count, cap) * 2 * IPB;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(k / (2 * IPB)), rem = (int)(k - (long long)e * 2 * IPB), b = rem / IPB, it = rem - b * IPB;
    const QRec &R = rec[e];
    if (b >= R.nb) continue;
    const int c = it < NR0 ? 0 : (it < NR0 + NR1 ? 1 : 2);
    const int row = it - (c == 0 ? 0 : (c == 1 ? NR0 : NR0 + NR1));
    record_row_global<D>(g, R, b, c, row, jfx, scale);
  }
}

// Sorted mode: the ions the push listed as far (a bound electron a cell or
// more from its nucleus), each moved by push_far; anything push_far cannot
// move is a domain error.
template <int D>
__global__ void __launch_bounds__(128) k_push_far(GridP g, PushArgs A) {
  const int n = min(*A.far_n, A.far_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0 && A.far_any) *A.far_any = n > 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int4 e = A.far[k];
    const int t = e.z;
    const int T0[3] = {(t % g.nt[0]) * Geo<D>::L0, ((t / g.nt[0]) % g.nt[1]) * Geo<D>::L1,
                       (t / (g.nt[0] * g.nt[1])) * Geo<D>::L2};
    if (!push_far<D>(g, A.sp[e.x], A.p[e.x], e.y, T0[0], T0[1], T0[2], A.status, reinterpret_cast<QRec *>(A.grec),
                     A.grec_n, A.grec_cap, A.E, A.B, A.jfx, A.jscale))
      atomicOr(A.status, ST_DOMAIN);
  }
}

template <int D, bool DET>
void launch_one(const GridP &g, const PushArgs &a, const TmaMaps &tm, cudaStream_t s) {
  cudaMemsetAsync(a.tile_n, 0, sizeof(int), s);
  const int qt = g.ntiles >= 8192 ? 4 : 1;  // tiles per quiet-pass block
  k_push_quiet<D><<<(g.ntiles + qt - 1) / qt, 128, 0, s>>>(g, a, qt);
  const size_t smem = push_smem_bytes(g, DET);
  // as many persistent blocks as the device holds at once (worked out per
  // context for its grid and device when it was created)
  const int blocks = a.push_blocks > 0 ? a.push_blocks : 1;
  cudaMemsetAsync(a.tile_ctr, 0, sizeof(int), s);
  k_push<D, DET><<<blocks < g.ntiles ? blocks : g.ntiles, push_threads(D), smem, s>>>(g, a, tm);
  if constexpr (DET) {
    k_push_far<D><<<a.sms, 128, 0, s>>>(g, a);
    cudaMemsetAsync(a.far_n, 0, sizeof(int), s);
    k_records<D><<<a.sms * 8, 256, 0, s>>>(g, reinterpret_cast<const QRec *>(a.grec), a.grec_n, a.grec_cap, a.jfx,
                                          a.jscale);
    cudaMemsetAsync(a.grec_n, 0, sizeof(int), s);
  }
}

template <int D, bool DET>
int prepare_one(const GridP &g, int *blocks) {
  const size_t smem = push_smem_bytes(g, DET);
  cudaError_t e = cudaFuncSetAttribute(k_push<D, DET>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return -1;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_push<D, DET>, push_threads(D), smem);
  if (e != cudaSuccess) return -1;
  *blocks = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  return 0;
}

}  // namespace

size_t push_smem_bytes(const GridP &g, int det) {
  int jc = 0, gc = 0;
  if (g.D == 1) { jc = Box<1>::JCELLS; gc = Box<1>::GCELLS; }
  if (g.D == 2) { jc = Box<2>::JCELLS; gc = Box<2>::GCELLS; }
  if (g.D == 3) { jc = Box<3>::JCELLS; gc = Box<3>::GCELLS; }
  // the sorted mode keeps its records in global memory
  (void)jc;
  return push_gbox_offset(g.D, det != 0) + 4 * (size_t)6 * gc + (det ? 0 : sizeof(QRec) * (size_t)push_qmax(g.D));
}

size_t push_record_bytes() { return sizeof(QRec); }

void launch_tile_active(const GridP &g, const unsigned char *qstate, const int *far_any, int ia_lo, int ia_hi,
                        unsigned char *act, unsigned long long *act_n, cudaStream_t s) {
  const int nb = (g.ntiles + 255) / 256;
  if (g.D == 1) k_tile_active<1><<<nb, 256, 0, s>>>(g, qstate, far_any, ia_lo, ia_hi, act, act_n);
  else if (g.D == 2) k_tile_active<2><<<nb, 256, 0, s>>>(g, qstate, far_any, ia_lo, ia_hi, act, act_n);
  else k_tile_active<3><<<nb, 256, 0, s>>>(g, qstate, far_any, ia_lo, ia_hi, act, act_n);
}

int push_prepare(const GridP &g, int det, int *blocks) {
  switch (g.D * 2 + (det ? 1 : 0)) {
    case 2: return prepare_one<1, false>(g, blocks);
    case 3: return prepare_one<1, true>(g, blocks);
    case 4: return prepare_one<2, false>(g, blocks);
    case 5: return prepare_one<2, true>(g, blocks);
    case 6: return prepare_one<3, false>(g, blocks);
    default: return prepare_one<3, true>(g, blocks);
  }
}

void launch_push(const GridP &g, const PushArgs &a, const TmaMaps &tm, cudaStream_t s) {
  const bool det = a.jscale != 0.0f;
  switch (g.D * 2 + (det ? 1 : 0)) {
    case 2: launch_one<1, false>(g, a, tm, s); break;
    case 3: launch_one<1, true>(g, a, tm, s); break;
    case 4: launch_one<2, false>(g, a, tm, s); break;
    case 5: launch_one<2, true>(g, a, tm, s); break;
    case 6: launch_one<3, false>(g, a, tm, s); break;
    default: launch_one<3, true>(g, a, tm, s); break;
  }
}

// The six field maps of a 3D grid: FP32 [nz][ny][nx] (strides in bytes
// between rows and planes), box {16, 15, 15} = one staged field box, no
// swizzle, zeros outside the grid.  cuTensorMapEncodeTiled comes through the
// runtime's driver entry point, so the library does not link the driver.
int encode_field_maps(const GridP &g, float *const F[6], TmaMaps *out) {
  out->on = 0;
  if (g.D != 3) return 0;
  using encode_fn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  void *fp = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fp, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fp)
    return -1;
  const encode_fn encode = reinterpret_cast<encode_fn>(fp);
  const cuuint64_t dims[3] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2]};
  const cuuint64_t strides[2] = {(cuuint64_t)g.n[0] * 4, (cuuint64_t)g.n[0] * g.n[1] * 4};
  const cuuint32_t box[3] = {(cuuint32_t)Box<3>::GR, (cuuint32_t)Box<3>::G1, (cuuint32_t)Box<3>::G2};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (strides[0] % 16 || strides[1] % 16) return -1;
  for (int c = 0; c < 6; ++c) {
    if (reinterpret_cast<uintptr_t>(F[c]) % 16) return -1;
    CUresult r = encode(&out->m[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, F[c], dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return -1;
  }
  out->on = 1;
  return 0;
}
