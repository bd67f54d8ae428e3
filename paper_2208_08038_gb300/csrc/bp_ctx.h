// bp_ctx.h -- the context behind the opaque bp_ctx handle (internal).
#pragma once
#include <string>
#include <vector>

#include "bp_internal.cuh"

struct bp_species_state {
  SpecP sp;
  PartP p;
  long long n = 0;       // particles loaded (before any removal)
  bool loaded = false;
  bool has_pidx = false;
  std::vector<double> omega;
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
  float *jbox = nullptr;
  unsigned char *occ = nullptr;
  float *frame = nullptr;
  int *status = nullptr;
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
};
