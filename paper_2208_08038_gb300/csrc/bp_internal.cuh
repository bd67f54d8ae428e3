// bp_internal.cuh -- internal types and device helpers of the GB300 two-body
// PIC library.  The C ABI is include/bp.h.
#pragma once
#include <cuda.h>  // CUtensorMap (the maps are encoded through the runtime's driver entry point)
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bp.h"

#define BP_MAX_SPECIES 8
#define BP_MAX_LASER 4
#define BP_MAX_PROBE 32

// bits of the device status word
enum { ST_NEED_SORT = 1, ST_DOMAIN = 2, ST_NONFINITE = 4, ST_TIMEOUT = 8 };

// Grid geometry as the kernels see it.  Axes >= D have n = 1, L = 1, box 1.
struct GridP {
  int D;
  int n[3];
  int bc[3];
  float dx[3], idx[3];
  float dt;
  double dxd[3], dtd;
  int L[3], nt[3];
  int M;            // body 1 may sit up to M cells outside its tile
  int og[3], gb[3]; // gather box: cells before the tile start, box extent
  int oj[3], jb[3]; // current box
  int gcells, jcells;
  long long ncell;
  int ntiles;
  int cpt;          // cells per tile
  int cb[3], cm[3]; // particle cell index: bit width and mask of each axis
  unsigned char *fnz; // [ntiles] sticky mark: E or B in the tile has been non-zero
};

// Tile geometry per dimension (compile time): L cells per tile per simulated
// axis; body 1 may sit up to M cells outside its tile; the field box staged
// for the gather spans [T0 - M - 2, T0 + L + M + 2], the current box
// [T0 - M - 3, T0 + L + M + 3] (body 2 within one cell of body 1, moves
// shorter than one cell).
template <int D>
struct Geo;
template <>
struct Geo<1> {
  static constexpr int L0 = 16, L1 = 1, L2 = 1, M = 8;
};
template <>
struct Geo<2> {
  static constexpr int L0 = 16, L1 = 16, L2 = 1, M = 2;
};
template <>
struct Geo<3> {
  static constexpr int L0 = 8, L1 = 8, L2 = 8, M = 1;
};
// bank-friendly plane stride: the smallest n' >= n with n' = 8 (mod 32)
// words, so that a node's x-, y- and z-neighbours (offsets 1, row, plane)
// fall in different shared-memory banks
__host__ __device__ constexpr int pad_plane(int n) { return n + ((8 - n % 32) + 32) % 32; }

template <int D>
struct Box {
  static constexpr int M = Geo<D>::M;
  static constexpr int G0 = Geo<D>::L0 + 2 * M + 5, G1 = D >= 2 ? Geo<D>::L1 + 2 * M + 5 : 1,
                       G2 = D >= 3 ? Geo<D>::L2 + 2 * M + 5 : 1;
  static constexpr int J0 = Geo<D>::L0 + 2 * M + 7, J1 = D >= 2 ? Geo<D>::L1 + 2 * M + 7 : 1,
                       J2 = D >= 3 ? Geo<D>::L2 + 2 * M + 7 : 1;
  static constexpr int OG = M + 2, OJ = M + 3;
  // Shared-memory layout, x fastest.  The field box of a 3D tile is the
  // image of one TMA box load per component: rows of GR = 20 floats (80
  // bytes, the box's inner extent; the box's 15 x cells need 16, the other 4
  // are loaded and not read) whose first float lies SX = 1 cell before the
  // box origin T0 - OG, so that the load starts at x = T0 - 4, a multiple of
  // 4 floats (16 bytes); planes of GR * G1 = 300 floats; each component's
  // stride rounded up to 32 floats (128 bytes).  A row of 20 words puts rows
  // y and y + 1 .. y + 7 in banks 20, 8, 28, ... words apart (a 16-word row
  // put row y + 2 in the same banks and doubled the gather's shared-load
  // bank conflicts).  1D/2D: rows of G0 floats.  The current box: row stride
  // J0, padded plane stride.
  static constexpr int GR = D >= 3 ? 20 : G0, SX = D >= 3 ? 1 : 0;
  static constexpr int GP = GR * G1;
  static constexpr int JP = D >= 3 ? pad_plane(J0 * J1) : J0 * J1;
  static constexpr int GCELLS = D >= 3 ? (GP * G2 + 31) / 32 * 32 : GP * G2, JCELLS = JP * J2;
  // global per-tile box layout (compact, x fastest)
  static constexpr int GCOMP = G0 * G1 * G2, JCOMP = J0 * J1 * J2;
  __host__ __device__ static constexpr int gi(int x, int y, int z) { return x + SX + GR * y + GP * z; }
  __host__ __device__ static constexpr int ji(int x, int y, int z) { return x + J0 * y + JP * z; }
};
static_assert(Box<3>::GR >= Box<3>::G0 + Box<3>::SX, "a 3D field box row holds the box's x extent");

// particle cell index: the three cell coordinates packed in bit fields
__host__ __device__ __forceinline__ int pack_cell(const GridP &g, int c0, int c1, int c2) {
  return c0 | (c1 << g.cb[0]) | (c2 << (g.cb[0] + g.cb[1]));
}
__host__ __device__ __forceinline__ void unpack_cell(const GridP &g, int cell, int c[3]) {
  c[0] = cell & g.cm[0];
  c[1] = (cell >> g.cb[0]) & g.cm[1];
  c[2] = cell >> (g.cb[0] + g.cb[1]);
}

struct SpecP {
  int kind;                // BP_TWO_BODY / BP_FREE
  float q1, m1, q2, m2;
  float h1, h2;            // q dt / (2 m)
  float qw1, qw2;          // q * weight
  float kappa;             // r_e k0
  const float *ac;         // softening a_c per parameter index
  int nac;
  double q1d, m1d, q2d, m2d, wd;
};

struct PartP {
  int *cell;      // global linear cell of body 1 (-1: removed)
  float *off;     // [D][cap] in-cell offset of body 1, [0, 1)
  float *r;       // [3][cap] internal displacement r = x1 - x2 (two-body only)
  float *u1;      // [3][cap]
  float *u2;      // [3][cap] (two-body only)
  int *pidx;      // parameter index (NULL: 0)
  int *id;        // load order
  int *tstart;    // [ntiles + 1] particle range of each tile
  long long cap;
};

struct PushArgs {
  int nsp;
  SpecP sp[BP_MAX_SPECIES];
  PartP p[BP_MAX_SPECIES];
  const float *E[3];
  const float *B[3];
  float *jbox;             // [ntiles][3][jcells]
  unsigned char *occ;      // [ntiles] the tile's box holds a deposit
  uint2 *jbb;              // [ntiles] its bounding box: lowest / highest node, one byte per axis
  unsigned char *qstate;   // [ntiles] what the quiet-tile pass left to the push
  unsigned long long *jfx; // [3][ncell] sorted deposit: the current in 64-bit fixed point (two's complement)
  int *tile_list;          // [ntiles] tiles the quiet-tile pass left for the push
  int *tile_n;             // their number (cleared before the quiet-tile pass)
  int *tile_ctr;           // the push's next list entry (cleared before each launch)
  void *grec;              // sorted deposit: general-case deposit records (grec_cap of them)
  int *grec_n;             // their count this step (device)
  int grec_cap;
  int *status;
  float jscale, jinv;      // fixed-point scale (sorted deposit), power of two
  unsigned long long *work; // [2] ions given the full push, ions moved by the quiet-tile pass (cumulative)
  int4 *far;                // sorted deposit: two-body ions whose bound electron is a cell or more away,
  int *far_n;               //   (species, particle, tile), moved after the push by k_push_far; their count
  int far_cap;
  int *far_any;             // set by k_push_far when it moved any this step (their current may land anywhere)
  int push_blocks;          // persistent push blocks for this grid on this device
  int sms;                  // multiprocessors of the device
};

// Tensor maps of the six field components (E_x, E_y, E_z, B_x, B_y, B_z)
// for the TMA staging of 3D field boxes: FP32 [nz][ny][nx], box 16 x 15 x 15,
// zero fill outside the grid.  on = 0: no maps (1D/2D grids, or the encoding
// failed), every tile is staged by per-thread asynchronous copies.
struct TmaMaps {
  CUtensorMap m[6];
  int on;
};
// encode the maps of a 3D grid's fields F[0..5]; 0 on success
int encode_field_maps(const GridP &g, float *const F[6], TmaMaps *out);

struct LaserP {
  int comp;
  double a0, omega, theta, waist, fwhm, t0, ramp, phase;
  int ia;
  double yc, zc;
};

// ---------------------------------------------------------------------------
// small device helpers

__host__ __device__ __forceinline__ int wrap_mod(int i, int n) {
  int m = i % n;
  return m < 0 ? m + n : m;
}
// periodic wrap of an index known to lie in [-n, 2n) (a staged box or a
// one-cell move on a grid of at least one tile): no integer division
__host__ __device__ __forceinline__ int wrap_once(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// One thread per cell; a block covers a chunk of one x row (row = y + n1 z),
// so coordinates come from one division per block and the neighbours are
// fixed offsets (+-1, +-n0, +-n0 n1) with the periodic wrap applied once.
struct Cell {
  long long q;      // linear index
  int c[3];         // coordinates
  long long up[3];  // offset to the +1 neighbour along each axis (periodic wrap)
  long long dn[3];  // offset to the -1 neighbour
};

template <int D>
__device__ __forceinline__ bool row_cell(const GridP &g, Cell &C) {
  const int n0 = g.n[0];
  const int chunks = (n0 + (int)blockDim.x - 1) / (int)blockDim.x;
  const int row = (int)blockIdx.x / chunks;
  const int x = ((int)blockIdx.x - row * chunks) * (int)blockDim.x + (int)threadIdx.x;
  if (x >= n0) return false;
  C.c[0] = x;
  C.c[1] = D >= 2 ? row % g.n[1] : 0;
  C.c[2] = D >= 3 ? row / g.n[1] : 0;
  C.q = (long long)row * n0 + x;
  long long stride = 1;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int n = g.n[a];
    C.up[a] = C.c[a] + 1 < n ? stride : -stride * (n - 1);
    C.dn[a] = C.c[a] > 0 ? -stride : stride * (n - 1);
    stride *= n;
  }
  return true;
}

// along an open axis a component with half stagger has no value at n-1
// (exterior), one with node stagger has Mur boundary nodes at 0 and n-1
template <int D>
__device__ __forceinline__ bool exterior_c(const GridP &g, int pat, const int c[3]) {
  bool e = false;
#pragma unroll
  for (int a = 0; a < D; ++a)
    if (g.bc[a] == BP_OPEN && ((pat >> a) & 1)) e |= c[a] == g.n[a] - 1;
  return e;
}
template <int D>
__device__ __forceinline__ bool mur_node(const GridP &g, int pat, const int c[3]) {
  bool m = false;
#pragma unroll
  for (int a = 0; a < D; ++a)
    if (g.bc[a] == BP_OPEN && !((pat >> a) & 1)) m |= c[a] == 0 || c[a] == g.n[a] - 1;
  return m;
}

// blocks of a row-blocked launch (one block per chunk of bs cells of an x row)
inline int row_blocks(const GridP &g, int bs) {
  const long long rows = g.ncell / g.n[0];
  return (int)(rows * ((g.n[0] + bs - 1) / bs));
}

// Four consecutive x cells per thread (rows hold a multiple of 8 cells, so a
// group never straddles a row or a tile): float4 loads and stores of each
// component, index arithmetic once per thread.
struct Cell4 {
  long long q;      // linear index of the group's first cell
  int c[3];         // its coordinates
  long long up[3];  // offset to the +1 neighbour along y, z (and x for the group's last cell)
  long long dn[3];  // offset to the -1 neighbour along y, z (and x for the group's first cell)
};

template <int D>
__device__ __forceinline__ bool row_cell4(const GridP &g, Cell4 &C) {
  const int n0 = g.n[0], n4 = n0 >> 2;
  const int chunks = (n4 + (int)blockDim.x - 1) / (int)blockDim.x;
  const int row = (int)blockIdx.x / chunks;
  const int x4 = ((int)blockIdx.x - row * chunks) * (int)blockDim.x + (int)threadIdx.x;
  if (x4 >= n4) return false;
  C.c[0] = 4 * x4;
  C.c[1] = D >= 2 ? row % g.n[1] : 0;
  C.c[2] = D >= 3 ? row / g.n[1] : 0;
  C.q = (long long)row * n0 + C.c[0];
  // along x: the neighbour after the last cell and before the first one
  C.up[0] = C.c[0] + 4 < n0 ? 4 : 4 - n0;
  C.dn[0] = C.c[0] > 0 ? -1 : n0 - 1;
  long long stride = n0;
#pragma unroll
  for (int a = 1; a < 3; ++a) {
    const int n = g.n[a];
    C.up[a] = C.c[a] + 1 < n ? stride : -stride * (n - 1);
    C.dn[a] = C.c[a] > 0 ? -stride : stride * (n - 1);
    stride *= n;
  }
  return true;
}

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float el(const float4 &v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w)); }
__device__ __forceinline__ void set_el(float4 &v, int i, float x) {
  if (i == 0) v.x = x;
  else if (i == 1) v.y = x;
  else if (i == 2) v.z = x;
  else v.w = x;
}

// blocks of a four-cells-per-thread row launch (rows of n0 / 4 threads)
inline int row_blocks4(const GridP &g, int bs) {
  const long long rows = g.ncell / g.n[0];
  return (int)(rows * ((g.n[0] / 4 + bs - 1) / bs));
}

// tile of a cell (row-major over tiles, x fastest)
__host__ __device__ __forceinline__ int tile_of(const GridP &g, const int c[3]) {
  return c[0] / g.L[0] + g.nt[0] * (c[1] / g.L[1] + g.nt[1] * (c[2] / g.L[2]));
}

// Mark the tile of a cell whose new E or B value is non-zero.  The marks are
// sticky (cleared only with the fields); the push stages no field box whose
// tiles are all unmarked.  Called by every thread of a row-blocked launch that
// is still active: a warp covers 32 consecutive x cells, and only the lowest
// lane of each tile segment with a non-zero value reads (and, the first time,
// writes) the mark.
template <int D>
__device__ __forceinline__ void mark_nonzero(const GridP &g, const int c[3], bool nz) {
  const unsigned m = __ballot_sync(__activemask(), nz);
  if (!nz) return;
  constexpr int L0 = Geo<D>::L0;
  static_assert(L0 <= 32 && (L0 & (L0 - 1)) == 0, "a tile segment lies inside one warp");
  const int lane = (int)(threadIdx.x & 31u);
  const int base = lane & ~(L0 - 1);
  if (m & ((1u << lane) - 1u) & ~((1u << base) - 1u)) return;  // a lower lane of the segment marks it
  unsigned char *f = g.fnz + tile_of(g, c);
  if (*f == 0) *f = 1;
}

// float -> int64, rounded to nearest even, on the FP32 and integer pipes
// (the 64-bit conversion runs on the slow FP64 unit).  Adding 1.5 * 2^23 to
// a float of magnitude below 2^22 rounds it to an integer held in the low
// mantissa bits; x is split exactly as h 2^22 + l with h = rne(x / 2^22) and
// |l| <= 2^21, and both parts are rounded that way.  Valid for |x| < 2^44.
__device__ __forceinline__ long long f2ll_rn(float x) {
  constexpr float M = 12582912.0f;
  const float hs = __fadd_rn(x * 2.384185791015625e-07f, M);
  const float h = __fsub_rn(hs, M);
  const float l = fmaf(-h, 4194304.0f, x);
  const int hi = __float_as_int(hs) - 0x4B400000;
  const int lo = __float_as_int(__fadd_rn(l, M)) - 0x4B400000;
  return (long long)hi * 4194304LL + (long long)lo;
}

// Exact fixed-point accumulation with the GPU's native 32-bit shared atomics
// (64-bit and FP32 shared atomic adds are compare-and-swap loops on this
// GPU).  A node's 64-bit sum is kept as two signed 32-bit words, lo and hi
// (hoff words later): v is split as 2^16 h + r with h = rint(v / 2^16) and
// |r| <= 2^15, both exact in FP32, so rne(v) = 2^16 h + rne(r); lo takes
// rne(r), hi takes h (and is skipped when h = 0).  The node's value,
// 2^16 sum(h) + sum(rne(r)), is the exact sum of rne(v) whatever the order,
// while fewer than 2^16 adds reach one node.  Both roundings to an integer
// add 1.5 * 2^23 (whose ulp is 1) and read the integer off the bits, on the
// FMA pipe; that needs |v| < 2^38 (callers scale contributions to <= 2^37).
__device__ __forceinline__ void fx_add(unsigned int *lo, int hoff, float v) {
  constexpr float M = 12582912.0f;
  const float hs = fmaf(v, 1.52587890625e-05f, M);  // M + rne(v / 2^16)
  const float h = __fsub_rn(hs, M);
  const float r = fmaf(-h, 65536.0f, v);            // exact
  atomicAdd(reinterpret_cast<int *>(lo), __float_as_int(__fadd_rn(r, M)) - 0x4B400000);
  const int hh = __float_as_int(hs) - 0x4B400000;
  if (hh) atomicAdd(reinterpret_cast<int *>(lo + hoff), hh);
}
// fx_add of two values at two nodes (lo0, lo1; high words hoff later), the
// FP32 part on packed pairs: each lane rounds exactly as fx_add does
__device__ __forceinline__ void fx_add2(unsigned int *lo0, unsigned int *lo1, int hoff, float2 v) {
  constexpr float M = 12582912.0f;
  const float2 hs = __ffma2_rn(v, make_float2(1.52587890625e-05f, 1.52587890625e-05f), make_float2(M, M));
  const float2 h = __fadd2_rn(hs, make_float2(-M, -M));
  const float2 r = __ffma2_rn(h, make_float2(-65536.0f, -65536.0f), v);
  const float2 rm = __fadd2_rn(r, make_float2(M, M));
  const int l0 = __float_as_int(rm.x) - 0x4B400000, l1 = __float_as_int(rm.y) - 0x4B400000;
  const int h0 = __float_as_int(hs.x) - 0x4B400000, h1 = __float_as_int(hs.y) - 0x4B400000;
  atomicAdd(reinterpret_cast<int *>(lo0), l0);
  atomicAdd(reinterpret_cast<int *>(lo1), l1);
  if (h0) atomicAdd(reinterpret_cast<int *>(lo0 + hoff), h0);
  if (h1) atomicAdd(reinterpret_cast<int *>(lo1 + hoff), h1);
}

// the value of a pair (both words initialised to 0)
__device__ __forceinline__ long long fx_value(const unsigned int *lo, int hoff) {
  return (long long)(int)lo[hoff] * 65536LL + (long long)(int)lo[0];
}

// quadratic B-spline weights for the three nodes around the nearest node,
// xi = position - nearest node in [-1/2, 1/2)
__device__ __forceinline__ void qweights(float xi, float w[3]) {
  float a = 0.5f - xi, b = 0.5f + xi;
  w[0] = 0.5f * a * a;
  w[1] = 0.75f - xi * xi;
  w[2] = 0.5f * b * b;
}

__device__ __forceinline__ float qshape(float x) {
  float a = fabsf(x);
  if (a <= 0.5f) return 0.75f - x * x;
  if (a < 1.5f) {
    float t = 1.5f - a;
    return 0.5f * t * t;
  }
  return 0.0f;
}

// S(u + d) - S(u) for the quadratic B-spline.  When u and u + d fall on the
// same polynomial piece the difference is formed from d directly (no
// cancellation between two rounded shape values); otherwise directly.
__device__ __forceinline__ float qshape_delta(float u, float d) {
  float v = u + d;
  float au = fabsf(u), av = fabsf(v);
  if (au <= 0.5f && av <= 0.5f) return -d * (u + v);
  if (u > 0.5f && v > 0.5f && u < 1.5f && v < 1.5f) return -0.5f * d * (3.0f - u - v);
  if (u < -0.5f && v < -0.5f && u > -1.5f && v > -1.5f) return 0.5f * d * (3.0f + u + v);
  if (au >= 1.5f && av >= 1.5f && (u > 0.0f) == (v > 0.0f)) return 0.0f;
  return qshape(v) - qshape(u);
}

__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// key of stream `stream` of seed `seed`, and the counter-based draw k
__host__ __device__ __forceinline__ uint64_t sm64_key(uint64_t seed, uint64_t stream) {
  return sm64_mix(sm64_mix(seed) + stream * 0x9E3779B97F4A7C15ull);
}
__host__ __device__ __forceinline__ uint64_t sm64_draw(uint64_t key, uint64_t k) {
  return sm64_mix(key + (k + 1ull) * 0x9E3779B97F4A7C15ull);
}
__host__ __device__ __forceinline__ double sm64_uniform(uint64_t key, uint64_t k) {
  return (double)(sm64_draw(key, k) >> 11) * 0x1.0p-53;
}

// ---------------------------------------------------------------------------
// launch wrappers (host side), one translation unit each

void launch_push(const GridP &g, const PushArgs &a, const TmaMaps &tm, cudaStream_t s);
size_t push_smem_bytes(const GridP &g, int det);
size_t push_record_bytes();
// the tiles the field kernels update (see k_tile_active); ia_lo..ia_hi: the antenna planes' x range
void launch_tile_active(const GridP &g, const unsigned char *qstate, const int *far_any, int ia_lo, int ia_hi,
                        unsigned char *act, unsigned long long *act_n, cudaStream_t s);  // one general-case deposit record
// set the push kernel's shared-memory limit for this grid and return, in
// *blocks, the number of push blocks resident on the current device at once
int push_prepare(const GridP &g, int det, int *blocks);

// act (per tile, optional): tiles to update; the others keep zero E, B, J
void launch_yee_b(const GridP &g, float *const B[3], const float *const E[3], float h, const unsigned char *act,
                  cudaStream_t s);
// recompute the tile marks (g.fnz) from E, B (F[0..5]) after a write from outside the step
void launch_field_marks(const GridP &g, const float *const F[6], cudaStream_t s);
// E <- E + dt (curl B - J).  With jfx (sorted deposit) the current is first
// formed per cell from the 64-bit fixed-point accumulator (times jinv) plus
// the antenna sheets at time t (evaluated into ant, [nlas][ncell / n0] FP64),
// written to J, and the accumulator cleared;
// without it J is read as the current sum left it.
void launch_yee_e(const GridP &g, float *const E[3], const float *const B[3], float *const J[3], float *frame,
                  unsigned long long *jfx, float jinv, const LaserP *las, int nlas, const long long *clk,
                  double *ant, const unsigned char *act, cudaStream_t s);
long long frame_floats(const GridP &g);
void launch_jsum(const GridP &g, const float *jbox, const unsigned char *occ, const uint2 *jbb, float *const J[3],
                 const LaserP *las, int nlas, const long long *clk, cudaStream_t s);
// the step clock (device): [0] step number, [1 + p] probe p's samples,
// [1 + BP_MAX_PROBE + p] its capacity; read by the antenna, the current sum
// and the probes, so that one captured step serves every step
constexpr int kClockWords = 1 + 2 * BP_MAX_PROBE;
struct ClockState {
  long long step;
  int nprobe;
  long long count[BP_MAX_PROBE], cap[BP_MAX_PROBE];
};
void launch_probe(const float *F, const long long *nodes, long long npts, float *buf, const long long *clk, int p,
                  cudaStream_t s);
void launch_clock_tick(long long *clk, int nprobe, cudaStream_t s);
void launch_clock_set(long long *clk, const ClockState &v, cudaStream_t s);

struct SortBufs {
  int *hist;       // [ncell + 1]
  int *bsum;       // scan block sums
  int *tmp_cell;
  float *tmp_f;    // enough floats for the largest species' float payload
  int *tmp_i;      // pidx / id payload
};
void launch_sort(const GridP &g, const SpecP &sp, PartP &p, SortBufs &b, int *status, cudaStream_t s);
void launch_clear_sort_flag(int *status, cudaStream_t s);
void launch_gen_lattice(int D, const double *sites, int per_site, double jitter, uint64_t seed, double sigma,
                        const int *site_param, long long first, long long count, double *x, double *u, int *pidx,
                        cudaStream_t s);
void launch_pick(const PartP &p, int D, int two, long long count, const int *sid, const int *srow, int n,
                 int *cell_out, float *out, unsigned char *found, cudaStream_t s);
void launch_set_sort_flag(int *status, cudaStream_t s);
cudaError_t make_sort_graph(const GridP &g, int nsp, const SpecP *sp, PartP *p, SortBufs &b, int *status, int *runs,
                            cudaStream_t cap, cudaGraphExec_t *out, cudaGraph_t tail = nullptr);

void launch_gen_medium(const GridP &g, const SpecP &sp, PartP &p, const int lo[3], const int hi[3], int ppc,
                       uint64_t seed, double sigma, long long first, long long count, cudaStream_t s);
void launch_load_convert(const GridP &g, const SpecP &sp, PartP &p, const double *x, const double *u, const int *pidx,
                         long long first, long long count, int *status, cudaStream_t s);
void launch_rho(const GridP &g, const SpecP &sp, const PartP &p, double *rho, cudaStream_t s);
void launch_divE_minus(const GridP &g, const float *const E[3], double *R, cudaStream_t s);

// adjoint
void launch_adj_inject(float *lam, const long long *nodes, long long npts, const float *dl, cudaStream_t s);
void launch_adj_e(const GridP &g, float *G[3], float *H[3], float *lamB[3], float *lamJ[3], cudaStream_t s);
// device-to-device copies of whole 4-byte-word arrays, issued as one kernel
struct CopyList {
  static constexpr int MAX = 32;
  int n = 0;
  const void *src[MAX];
  void *dst[MAX];
  long long words[MAX];
};
void launch_copy_many(const CopyList &L, int sms, cudaStream_t s);
// zero (optional): three arrays cleared on the way
void launch_adj_b(const GridP &g, float *lamE[3], float *lamB[3], float h, float *zero[3], cudaStream_t s);
size_t adj_push_smem(int D);
constexpr int kAdjChunk = 256;  // particles per work item of the particle adjoint
int adj_prepare(int D, int *push_blocks, int *scat_blocks);
// device buffers and launch shapes of the particle adjoint
struct AdjBufs {
  unsigned long long *lfx;  // [6][ncell] field-adjoint sums in fixed point (kept zero between steps)
  unsigned char *dirty;     // [ntiles] tiles with lfx entries
  int *kst;                 // the step's fixed-point exponent
  unsigned *emax;           // the step's largest |gathered-field adjoint| (float bits)
  int *nwork;               // work items of the step
  int4 *work;
  int work_cap;
  int chunk;                // particles per work item
  int push_blocks, scat_blocks;
};
void launch_adj_push(const GridP &g, int nsp, const SpecP *sp, const PartP *p, float *const xb[], double *const acb[],
                     float *const eb[], const long long *cap, const float *const E[3], const float *const B[3],
                     const float *const lamJ[3], const AdjBufs &b, float *lamE[3], float *lamB[3], int *status,
                     cudaStream_t s);
void launch_csr_sum(const int *ptr, const int *ids, int nrows, const float *xb, long long cap, int ncomp,
                    const double *acb, const double *scale, double *out, cudaStream_t s);
