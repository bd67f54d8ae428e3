// bp_noalloc.cu -- bp_residual_noalloc: the Gauss-law residual copied to a
// host buffer without allocating any device memory.
//
// bp_residual needs an FP64 grid of scratch on the device when its result
// goes to host memory, and it obtains that grid through the context's
// allocator the first time.  Some callers cannot let the library allocate at
// that point: a diagnostics thread of a host program that does not own the
// allocator the context was created with (PyTorch's caching allocator, say,
// which is only safe to call from the thread and stream that own it), a
// run whose device memory is fully committed to particles and fields, or a
// loop that must not touch the allocator while other work is queued.  This
// variant keeps its scratch in a fixed array in the library's static device
// memory instead, so it calls no cudaMalloc, cudaFree or allocating routine.
#include <cuda.h>

#include <cstdio>
#include <mutex>

#include "bp_ctx.h"

namespace {

// Largest grid the static scratch holds: 4,194,304 nodes (32 MiB of FP64).
// Every GPU that loads the library holds this array until the process ends.
constexpr long long kMaxNodes = 1LL << 22;
__device__ __align__(256) double g_residual_scratch[kMaxNodes];

// The device address of the array is looked up (cudaGetSymbolAddress) once
// per CUDA context and cached under the context's id, which the driver never
// reuses within a process: a context that is destroyed and created again (a
// device reset, say) gets a new id and so a fresh lookup, never a stale
// address.  In host code g_residual_scratch only names a host-side
// stand-in; the device address must come from the runtime, with the context
// current.
constexpr int kCacheSlots = 64;
struct ScratchSlot {
  unsigned long long ctx_id;
  double *addr;
};
ScratchSlot g_slots[kCacheSlots] = {};
int g_slots_used = 0, g_slots_next = 0;
std::mutex g_scratch_mu;

using ctx_get_current_fn = CUresult (*)(CUcontext *);
using ctx_get_id_fn = CUresult (*)(CUcontext, unsigned long long *);

// id of the calling thread's current CUDA context (driver entry points found
// through the runtime, so the library does not link the driver library)
int current_context_id(unsigned long long *id) {
  static ctx_get_current_fn get_current = nullptr;
  static ctx_get_id_fn get_id = nullptr;
  if (!get_current || !get_id) {
    void *a = nullptr, *b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
        qa != cudaDriverEntryPointSuccess || !a)
      return BP_ERR_CUDA;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
        qb != cudaDriverEntryPointSuccess || !b)
      return BP_ERR_CUDA;
    get_current = reinterpret_cast<ctx_get_current_fn>(a);
    get_id = reinterpret_cast<ctx_get_id_fn>(b);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return BP_ERR_STATE;
  return get_id(ctx, id) == CUDA_SUCCESS ? BP_OK : BP_ERR_CUDA;
}

// device address of the scratch array in the current context
int scratch_address(double **out) {
  unsigned long long id = 0;
  int rc = current_context_id(&id);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  for (int k = 0; k < g_slots_used; ++k)
    if (g_slots[k].ctx_id == id) {
      *out = g_slots[k].addr;
      return BP_OK;
    }
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_residual_scratch) != cudaSuccess || !p) return BP_ERR_CUDA;
  const int k = g_slots_used < kCacheSlots ? g_slots_used++ : (g_slots_next++ % kCacheSlots);
  g_slots[k] = ScratchSlot{id, static_cast<double *>(p)};
  *out = g_slots[k].addr;
  return BP_OK;
}

int set_error(bp_ctx *c, int code, const char *msg) {
  c->err = msg;
  return code;
}

}  // namespace

extern "C" int bp_residual_noalloc(bp_ctx *c, double *dst) {
  if (!c || !dst) return BP_ERR_ARG;
  const GridP &g = c->g;
  if (g.ncell > kMaxNodes) {
    char buf[160];
    snprintf(buf, sizeof buf, "bp_residual_noalloc: grid has %lld nodes, the static scratch holds at most %lld",
             g.ncell, kMaxNodes);
    return set_error(c, BP_ERR_ARG, buf);
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != c->device)
    return set_error(c, BP_ERR_STATE, "bp_residual_noalloc: call it with the context's device current");
  double *R = nullptr;
  int rc = scratch_address(&R);
  if (rc) return set_error(c, rc, "bp_residual_noalloc: no device address for the static scratch");
  // the array keeps the previous call's values: rho accumulates from zero
  cudaError_t e = cudaMemsetAsync(R, 0, sizeof(double) * g.ncell, c->stream);
  if (e != cudaSuccess) return set_error(c, BP_ERR_CUDA, cudaGetErrorString(e));
  for (auto &s : c->sp)
    if (s.loaded) {
      launch_rho(g, s.sp, s.p, R, c->stream);
      c->launches++;
    }
  const float *E[3] = {c->F[0], c->F[1], c->F[2]};
  launch_divE_minus(g, E, R, c->stream);
  c->launches++;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst, R, sizeof(double) * g.ncell, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return set_error(c, BP_ERR_CUDA, cudaGetErrorString(e));
  return BP_OK;
}
