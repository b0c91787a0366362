// Allocation-free 2D TV prox (vrps_prox_tv2d_noalloc).  The paper has no counterpart: this
// entry point exists for callers that cannot let this library call cudaMalloc -- an
// application that owns the whole device-memory budget through its own pool allocator, or a
// latency-critical loop in which the implicit device synchronisation of an allocation is not
// acceptable.  Its scratch is a fixed array in device global memory instead of allocations.
//
// The array lives in this translation unit only, so with CUDA's default lazy module loading a
// device reserves it when this entry point first runs there (with CUDA_MODULE_LOADING=EAGER,
// every device that loads the library reserves it); it stays reserved until the process exits,
// and every call shares it.  The iterations and the output are the same launches as
// vrps_prox_tv's 2D path (fgp2d_iterate / fgp2d_output), so both give the same bits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "vrps_internal.h"

namespace vrps {
namespace {

constexpr long long NOALLOC_MAX_PIXELS = VRPS_NOALLOC_MAX_PIXELS;
// five dual-sized regions of 2 * NOALLOC_MAX_PIXELS floats: the cold-start dual and the two
// (w, z) pairs the blocked iterations alternate between
__device__ __align__(256) float g_noalloc_scratch[5 * 2 * NOALLOC_MAX_PIXELS];

constexpr int NOALLOC_MAX_DEVICES = 64;
float* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};
std::mutex g_noalloc_mu;

// Device address of the scratch array on device `dev` (the current device).  In host code the
// array's name only stands for a host-side shadow, so the address is looked up with
// cudaGetSymbolAddress once per device, with that device current, and cached for the life of
// the process (a cudaDeviceReset invalidates it; see the entry point's documentation).
int noalloc_scratch(int dev, float** out) {
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(VRPS_ERR_UNSUPPORTED, "device index %d too large", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
    g_noalloc_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return VRPS_OK;
}

}  // namespace
}  // namespace vrps

extern "C" int vrps_prox_tv2d_noalloc(int nx, int ny, const float* v, float* x, float tau, int iters, int nonneg,
                                      float* dual, vrps_stream_t stream) {
  using namespace vrps;
  if (nx <= 0 || ny <= 0) return fail(VRPS_ERR_INVALID_ARG, "sizes must be positive (nx=%d ny=%d)", nx, ny);
  if ((long long)nx * ny > NOALLOC_MAX_PIXELS)
    return fail(VRPS_ERR_INVALID_ARG, "nx*ny = %lld exceeds the fixed scratch capacity of %lld pixels",
                (long long)nx * ny, NOALLOC_MAX_PIXELS);
  if (!v || !x) return fail(VRPS_ERR_INVALID_ARG, "v or x is NULL");
  if (v == x) return fail(VRPS_ERR_INVALID_ARG, "v and x must not alias");
  if (!(tau > 0.f) || !std::isfinite(tau)) return fail(VRPS_ERR_INVALID_ARG, "tau must be > 0");
  if (iters < 0) return fail(VRPS_ERR_INVALID_ARG, "iters must be >= 0");
  int dev = -1;
  VRPS_CUDA(cudaGetDevice(&dev));
  float* base = nullptr;
  VRPS_TRY(noalloc_scratch(dev, &base));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)nx * ny, dn = 2 * n;
  const size_t cap = 2 * (size_t)NOALLOC_MAX_PIXELS;
  float* cold = base;
  float* pairs[2][2] = {{base + cap, base + 2 * cap}, {base + 3 * cap, base + 4 * cap}};
  float* d = dual;
  if (!d) {
    // the shared array keeps the previous call's contents: a cold start clears its dual
    VRPS_CUDA(cudaMemsetAsync(cold, 0, dn * sizeof(float), s));
    d = cold;
  }
  const float* w_final = d;
  VRPS_TRY(fgp2d_iterate(v, d, pairs, nx, ny, tau, iters, nonneg ? 1 : 0, 0, s, &w_final));
  ProxTail t;
  std::memset(&t, 0, sizeof(t));
  t.mode = 0;
  t.out = x;
  float* wdst = (w_final != d && dual) ? dual : nullptr;
  VRPS_TRY(fgp2d_output(v, w_final, wdst, nx, ny, tau, nonneg ? 1 : 0, t, s));
  return VRPS_OK;
}
