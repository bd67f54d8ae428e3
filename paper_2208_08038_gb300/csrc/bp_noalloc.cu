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
#include <cstdio>
#include <mutex>

#include "bp_ctx.h"

namespace {

// Largest grid the static scratch holds: 4,194,304 nodes (32 MiB of FP64).
// Every GPU that loads the library holds this array until the process ends.
constexpr long long kMaxNodes = 1LL << 22;
__device__ __align__(256) double g_residual_scratch[kMaxNodes];

constexpr int kMaxDevices = 64;
double *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// In host code g_residual_scratch only names a host-side stand-in; the
// device address comes from the runtime, once per device, with that device
// current.
int scratch_address(int dev, double **out) {
  if (dev < 0 || dev >= kMaxDevices) return BP_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_residual_scratch);
    if (e != cudaSuccess) return BP_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_addr[dev];
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
  int rc = scratch_address(dev, &R);
  if (rc) return set_error(c, rc, "bp_residual_noalloc: cudaGetSymbolAddress failed");
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
