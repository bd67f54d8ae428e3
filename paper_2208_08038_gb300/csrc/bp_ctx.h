// bp_ctx.h -- the context behind the opaque bp_ctx handle (internal).
#pragma once
#include <string>
#include <vector>

#include "bp_internal.cuh"

struct bp_species_state {
  SpecP sp{};
  PartP p{};  // null until the first load (alloc_particles tests p.cell)
  long long n = 0;       // particles loaded (before any removal)
  bool loaded = false;
  bool has_pidx = false;
  std::vector<double> omega;
  std::vector<int> pidx_host;  // parameter index per particle, load order (empty: all 0)
  float *ac_dev = nullptr;
};

// particle arrays copied aside (checkpoints, per-step stores of the adjoint)
struct bp_part_copy {
  PartP p{};
};

struct bp_adjoint {
  bool ready = false;
  int K = 0, nseg = 0;
  long long start = 0, nsteps = 0;
  std::vector<long long> probe_c0;
  std::vector<float *> ck_fields;                   // [nseg] E, B (6 ncell)
  int *ck_status = nullptr;                         // [nseg][4] device status words
  std::vector<std::vector<bp_part_copy>> ck_parts;  // [nseg][species]
  // per-step stores of a recomputed segment, two banks of K steps ([bank * K
  // + j]): the reverse steps of one segment read one bank while the next
  // (earlier) segment is recomputed into the other
  std::vector<float *> st_fields;                   // [2 K] E^n, B^n
  std::vector<std::vector<bp_part_copy>> st_parts;  // [2 K][species]
  cudaStream_t stream = nullptr;                    // the reverse steps' stream
  int *status = nullptr;                            // the reverse pass's status word
  cudaEvent_t rec_done[2] = {nullptr, nullptr};     // bank b recomputed
  cudaEvent_t rev_done[2] = {nullptr, nullptr};     // bank b's reverse steps done
  float *lamE[3] = {}, *lamB[3] = {}, *lamJ[3] = {}, *H[3] = {};
  unsigned long long *lfx = nullptr;  // [6][ncell] scattered field adjoints, fixed point
  unsigned char *dirty = nullptr;     // [ntiles]
  int *kst = nullptr;                 // the step's fixed-point exponent
  int *nwork = nullptr;               // the step's work items (count, list)
  int4 *work = nullptr;
  long long work_cap = 0;
  int push_blocks = 0, scat_blocks = 0;
  std::vector<float *> xb;     // per species [12][cap]
  std::vector<double *> acb;   // per species [cap]
  std::vector<float *> eb;     // per species [12][cap], the step's gathered-field adjoints by slot
  unsigned *emax = nullptr;    // their largest magnitude (float bits)
  std::vector<long long> xb_cap;
  float *dl = nullptr;         // probe-loss gradient on the device
  long long dl_len = 0;
};

struct bp_probe_state {
  int comp;
  long long npts, cap, count;
  long long *nodes;
  float *buf;
};

struct bp_ctx {
  GridP g;
  int det = 1;
  bp_allocator alloc{};
  bool have_alloc = false;
  cudaStream_t stream = nullptr;
  int device = 0;
  float *F[9] = {};
  float *jbox = nullptr;             // atomic deposit: per-tile FP32 current boxes
  unsigned long long *jfx = nullptr; // sorted deposit: [3][ncell] current in 64-bit fixed point
  double *ant = nullptr;             // sorted deposit: antenna sheet values of a step, [laser][ncell / n0]
  void *grec = nullptr;              // sorted deposit: general-case deposit records of a step
  int *grec_n = nullptr;             // their count (device, cleared after each step)
  int4 *far = nullptr;               // sorted deposit: ions with a far bound electron, moved after the push
  int *far_n = nullptr;              // their count (device, cleared after each step)
  int *far_any = nullptr;            // whether the last push moved any (device)
  long long far_cap = 0;
  long long grec_cap = 0;
  long long grec_fixed = 0;          // capacity set by the caller (0: default)
  unsigned char *occ = nullptr;
  uint2 *jbb = nullptr;
  unsigned char *qstate = nullptr;  // per tile: left by the quiet-tile pass for the push
  unsigned char *act = nullptr;     // per tile: updated by the field kernels (grids of 1024 tiles or more)
  unsigned long long *act_n = nullptr;  // [2]: active tiles summed over steps, steps (see bp_field_work)
  int *tile_ctr = nullptr;           // the push's tile counter
  int *tile_list = nullptr;          // tiles left for the push by the quiet-tile pass, and their number
  int *tile_n = nullptr;
  // asynchronous field reads: two device snapshots, copied to the host on a
  // side stream; ready[k] marks snapshot k written, done[k] its copy finished
  float *snap[2] = {nullptr, nullptr};
  cudaStream_t read_stream = nullptr;
  cudaEvent_t snap_ready[2] = {nullptr, nullptr}, snap_done[2] = {nullptr, nullptr};
  int snap_next = 0;
  float *frame = nullptr;
  int *status = nullptr;
  unsigned long long *work = nullptr;  // [2] push work counters (see PushArgs::work)
  int push_blocks[2] = {1, 1};         // resident push blocks per deposit mode (atomic, sorted)
  int sms = 1;                         // multiprocessors of the context's device
  TmaMaps tmaps{};                     // tensor maps of E, B for the push's TMA staging (3D)
  std::vector<bp_species_state> sp;
  std::vector<LaserP> las;
  std::vector<bp_probe_state> pr;
  SortBufs sb{};
  long long sort_cap = 0;  // particles the sort scratch can hold
  long long step = 0;
  long long launches = 0;
  double *rho = nullptr;
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  double push_ms = 0.0;
  long long push_launches = 0;
  std::vector<void *> owned;
  std::string err;
  float jscale = 0.0f, jinv = 0.0f;
  bp_adjoint adj;
  // per-step re-sort as a conditional graph (rebuilt when a particle array,
  // the sort scratch or the set of loaded species changes)
  cudaGraphExec_t sort_exec = nullptr;
  cudaStream_t cap_stream = nullptr;
  bool sort_dirty = true;
  int *sort_runs = nullptr;      // host-mapped counter of re-sorts that ran
  int *sort_runs_dev = nullptr;
  int sort_nsp = 0;              // species in the graph's sort pipeline
  // the step clock (device; see kClockWords) and the graph of a step's
  // launches after the re-sort, with the launch arguments it was captured
  // with (rebuilt when any of them changes)
  long long *clk = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  bool step_sorts = false;  // the step graph begins with the conditional re-sort
  std::string step_key;
};
