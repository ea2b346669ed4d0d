// noalloc.cu -- rbicg_op_gram_noalloc: the tall-skinny Gram G = X^H Y without any device
// allocation.  The per-row-chunk partial tiles that rbicg_op_gram keeps in cudaMalloc'd
// scratch live here in one file-scope device array of fixed size instead.
//
// Who needs this: callers that must not allocate device memory behind their back -- a
// runtime that reserves the device memory up front and forbids hidden allocations, or a
// latency-critical caller that cannot afford cudaMalloc / cudaFree and the synchronisation
// they imply.  The caller passes the inputs and the output; this entry point allocates
// nothing (no cudaMalloc, cudaFree or allocating library routine).
#include <mutex>

#include "../../include/rbicg.h"
#include "internal.cuh"

namespace rb {

// Scratch: room for RB_NOALLOC_CHUNKS x 64 x 64 complex doubles of partial sums (8 MiB): for
// mx, my <= 64 the Gram kernel writes at most that many (its row chunks times the tiles of X^H Y).
// Every GPU that loads this library holds this array until the process exits.
constexpr int RB_NOALLOC_TILE = 64;
constexpr int RB_NOALLOC_CHUNKS = 128;
constexpr size_t RB_NOALLOC_BYTES = (size_t)RB_NOALLOC_CHUNKS * RB_NOALLOC_TILE * RB_NOALLOC_TILE * sizeof(zd);
static __device__ __align__(256) unsigned char g_noalloc_scratch[RB_NOALLOC_BYTES];

// In host code the array's name is only a host-side stand-in: its device address is fetched
// once per device, with that device current, and passed to the kernels.
constexpr int RB_NOALLOC_MAXDEV = 64;
static void* g_scratch_addr[RB_NOALLOC_MAXDEV];
static std::mutex g_scratch_mu;

static cudaError_t scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= RB_NOALLOC_MAXDEV) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

void set_global_error(const char* msg);   // engine.cu: message of rbicg_last_error(NULL)

}  // namespace rb

using namespace rb;

extern "C" rbicg_status rbicg_op_gram_noalloc(rbicg_dtype dtype, int64_t n, const void* X, int mx, int ldx,
                                              const void* Y, int my, int ldy, int fp32, void* G, void* stream) {
  if (dtype != RBICG_R64 && dtype != RBICG_C128) {
    set_global_error("rbicg_op_gram_noalloc: unknown dtype");
    return RBICG_ERR_ARG;
  }
  if (n <= 0 || !X || !Y || !G || ldx < mx || ldy < my) {
    set_global_error("rbicg_op_gram_noalloc: need n > 0, non-null X, Y, G and ldx >= mx, ldy >= my");
    return RBICG_ERR_ARG;
  }
  if (mx < 1 || my < 1 || mx > RB_NOALLOC_TILE || my > RB_NOALLOC_TILE) {
    // sizes beyond the scratch array: one 64 x 64 tile of partial sums per row chunk
    set_global_error("rbicg_op_gram_noalloc: mx and my must be in 1..64 (fixed 8 MiB scratch)");
    return RBICG_ERR_ARG;
  }
  void* scratch = nullptr;
  const cudaError_t se = scratch_for_current_device(&scratch);
  if (se != cudaSuccess) {
    set_global_error(cudaGetErrorString(se));
    return RBICG_ERR_CUDA;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // Every partial tile that the reduction reads is first written by the Gram kernel of the
  // same call (whole tiles per row chunk, zero-padded), so no part of the shared scratch has to
  // start at zero; the previous call's contents are simply overwritten.
  if (dtype == RBICG_R64) {
    ColList<double> xl{}, yl{};
    for (int c = 0; c < mx; ++c) { xl.c[c].p = reinterpret_cast<const double*>(X) + c; xl.c[c].ld = ldx; }
    for (int c = 0; c < my; ++c) { yl.c[c].p = reinterpret_cast<const double*>(Y) + c; yl.c[c].ld = ldy; }
    xl.m = mx; yl.m = my;
    launch_gram<double>(xl, yl, n, fp32, scratch, RB_NOALLOC_CHUNKS, reinterpret_cast<double*>(G), s);
  } else {
    ColList<cplx<double>> xl{}, yl{};
    for (int c = 0; c < mx; ++c) { xl.c[c].p = reinterpret_cast<const cplx<double>*>(X) + c; xl.c[c].ld = ldx; }
    for (int c = 0; c < my; ++c) { yl.c[c].p = reinterpret_cast<const cplx<double>*>(Y) + c; yl.c[c].ld = ldy; }
    xl.m = mx; yl.m = my;
    launch_gram<cplx<double>>(xl, yl, n, fp32, scratch, RB_NOALLOC_CHUNKS, reinterpret_cast<zd*>(G), s);
  }
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) {
    set_global_error(cudaGetErrorString(le));
    return RBICG_ERR_CUDA;
  }
  return RBICG_OK;
}
