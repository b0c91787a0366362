// Float64 reductions (objective, power iteration), Philox4x32-10 draws and small helpers.
//
// Reductions are two-stage and deterministic: a fixed grid of NPART blocks writes one
// partial sum each (grid-stride loops, warp-shuffle + shared-memory block reduction in
// float64), then one block adds the partials in a fixed order.
#include <cmath>

#include "vrps_internal.h"

namespace vrps {
namespace {

constexpr int RED_THREADS = 256;
constexpr int NPART = 608;   // 4 blocks per SM on a 152-SM part

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[RED_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < RED_THREADS / 32; ++q) r += ws[q];
  }
  return r;
}

__global__ void __launch_bounds__(RED_THREADS) dot_partial(const float* __restrict__ a,
                                                           const float* __restrict__ b, int64_t n,
                                                           double* part) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * RED_THREADS + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * RED_THREADS)
    s += (double)a[i] * (double)b[i];
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(RED_THREADS) finalize(const double* part, int np, double* dst) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += RED_THREADS) s += part[i];
  s = block_sum(s);
  if (threadIdx.x == 0) *dst = s;
}

// isotropic TV: sum over pixels of ||forward differences||_2 (zero at the last index)
__global__ void __launch_bounds__(RED_THREADS) tv_partial(const float* __restrict__ x, int nx, int ny,
                                                          int nz, double* part) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t nxy = (int64_t)nx * ny;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * RED_THREADS + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * RED_THREADS) {
    const int ix = (int)(i % nx);
    const int iy = (int)((i / nx) % ny);
    const int iz = (int)(i / nxy);
    const double c = (double)x[i];
    const double d1 = ix < nx - 1 ? (double)x[i + 1] - c : 0.0;
    const double d2 = iy < ny - 1 ? (double)x[i + nx] - c : 0.0;
    const double d3 = iz < nz - 1 ? (double)x[i + nxy] - c : 0.0;
    s += sqrt(d1 * d1 + d2 * d2 + d3 * d3);
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Philox4x32-10 (Salmon et al., SC'11): two 32x32->64 multiplies per round, key bumped by
// the Weyl constants between the 10 rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__global__ void schedule_kernel(uint32_t k0lo, uint32_t k1hi, uint32_t job, int64_t kbase, int count,
                                uint32_t N, unsigned long long thr, int always, int32_t* out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const uint64_t k = (uint64_t)kbase + (uint64_t)q;
  const uint4 w = philox10(make_uint4((uint32_t)k, (uint32_t)(k >> 32), job, 0u), k0lo, k1hi);
  out[3 * q + 0] = (int32_t)(((uint64_t)w.x * (uint64_t)N) >> 32);
  out[3 * q + 1] = always ? 1 : ((unsigned long long)w.y < thr ? 1 : 0);
  out[3 * q + 2] = ((uint64_t)w.z < (0x100000000ull / (uint64_t)N)) ? 1 : 0;
}

__global__ void uniform_kernel(uint32_t key0, uint32_t key1, uint32_t job, uint32_t tag, float* out,
                               int64_t n) {
  const int64_t blk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blk * 4 >= n) return;
  const uint4 w = philox10(make_uint4((uint32_t)blk, (uint32_t)((uint64_t)blk >> 32), job, tag), key0, key1);
  const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
  for (int q = 0; q < 4; ++q) {
    const int64_t e = blk * 4 + q;
    if (e < n) out[e] = (float)(((double)ws[q] + 0.5) / 4294967296.0);
  }
}

__global__ void scale_kernel(float* dst, const float* src, const double* nrm2, int64_t n) {
  const double inv = 1.0 / sqrt(*nrm2);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (float)((double)src[i] * inv);
}

__global__ void gather_rows_kernel(const float* __restrict__ src, float* __restrict__ dst, const int* ids,
                                   int row_len) {
  const int r = blockIdx.y;
  const size_t so = (size_t)ids[r] * row_len, d0 = (size_t)r * row_len;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < row_len; j += gridDim.x * blockDim.x)
    dst[d0 + j] = src[so + j];
}

__global__ void scatter_rows_kernel(const float* __restrict__ src, float* __restrict__ dst, const int* ids,
                                    int row_len) {
  const int r = blockIdx.y;
  const size_t d0 = (size_t)ids[r] * row_len, so = (size_t)r * row_len;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < row_len; j += gridDim.x * blockDim.x)
    dst[d0 + j] = src[so + j];
}

__global__ void store_kernel(const float* __restrict__ src, void* __restrict__ dst, int64_t n, FwdOut f) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    st_store(f, dst, (size_t)i, src[i]);
}

__global__ void fill_kernel(float* p, float v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

}  // namespace

int dot64(const float* a, const float* b, int64_t n, double* dst, Workspace& ws, cudaStream_t s) {
  { LaunchScope _ls("dot_partial", s, (a == b ? 4.0 : 8.0) * n);
  VRPS_CUDA(launch_kernel(dot_partial, dim3(NPART), dim3(RED_THREADS), (size_t)(0), s, a, b, n, ws.partials));
  }
  VRPS_LAUNCHED("dot_partial");
  { LaunchScope _ls("finalize", s);
  VRPS_CUDA(launch_kernel(finalize, dim3(1), dim3(RED_THREADS), (size_t)(0), s, ws.partials, NPART, dst));
  }
  VRPS_LAUNCHED("finalize");
  return VRPS_OK;
}

int tv64(const vrps_geom* g, const float* x, double* dst, Workspace& ws, cudaStream_t s) {
  { LaunchScope _ls("tv_partial", s, 4.0 * g->n);
  VRPS_CUDA(launch_kernel(tv_partial, dim3(NPART), dim3(RED_THREADS), (size_t)(0), s, x, g->nx, g->ny, g->nz, ws.partials));
  }
  VRPS_LAUNCHED("tv_partial");
  { LaunchScope _ls("finalize", s);
  VRPS_CUDA(launch_kernel(finalize, dim3(1), dim3(RED_THREADS), (size_t)(0), s, ws.partials, NPART, dst));
  }
  VRPS_LAUNCHED("finalize");
  return VRPS_OK;
}

int philox_schedule(uint64_t seed, uint32_t job, int64_t k0, int count, int N, double p, int32_t* out,
                    cudaStream_t s) {
  if (count <= 0) return VRPS_OK;
  const int always = p >= 1.0 ? 1 : 0;
  const unsigned long long thr = always ? 0ull : (unsigned long long)std::floor(p * 4294967296.0);
  { LaunchScope _ls("schedule_kernel", s);
  VRPS_CUDA(launch_kernel(schedule_kernel, dim3((count + 255) / 256), dim3(256), (size_t)(0), s, (uint32_t)seed, (uint32_t)(seed >> 32), job, k0, count,
                                                      (uint32_t)N, thr, always, out));
  }
  VRPS_LAUNCHED("philox_schedule");
  return VRPS_OK;
}

int philox_uniform(uint64_t seed, uint32_t job, uint32_t tag, float* out, int64_t n, cudaStream_t s) {
  const int64_t blocks = ((n + 3) / 4 + 255) / 256;
  { LaunchScope _ls("uniform_kernel", s, 4.0 * n);
  VRPS_CUDA(launch_kernel(uniform_kernel, dim3((unsigned)blocks), dim3(256), (size_t)(0), s, (uint32_t)seed, (uint32_t)(seed >> 32), job, tag, out, n));
  }
  VRPS_LAUNCHED("philox_uniform");
  return VRPS_OK;
}

int scale_inv_sqrt(float* dst, const float* src, const double* nrm2, int64_t n, cudaStream_t s) {
  { LaunchScope _ls("scale_kernel", s, 8.0 * n);
  VRPS_CUDA(launch_kernel(scale_kernel, dim3(NPART), dim3(256), (size_t)(0), s, dst, src, nrm2, n));
  }
  VRPS_LAUNCHED("scale_inv_sqrt");
  return VRPS_OK;
}

int gather_rows(const float* src, float* dst, const int* ids, int rows, int row_len, cudaStream_t s) {
  if (rows <= 0) return VRPS_OK;
  dim3 grid((row_len + 255) / 256 < 64 ? (row_len + 255) / 256 : 64, rows);
  { LaunchScope _ls("gather_rows_kernel", s, 8.0 * rows * row_len);
  VRPS_CUDA(launch_kernel(gather_rows_kernel, dim3(grid), dim3(256), (size_t)(0), s, src, dst, ids, row_len));
  }
  VRPS_LAUNCHED("gather_rows");
  return VRPS_OK;
}

int scatter_rows(const float* src, float* dst, const int* ids, int rows, int row_len, cudaStream_t s) {
  if (rows <= 0) return VRPS_OK;
  dim3 grid((row_len + 255) / 256 < 64 ? (row_len + 255) / 256 : 64, rows);
  { LaunchScope _ls("scatter_rows_kernel", s, 8.0 * rows * row_len);
  VRPS_CUDA(launch_kernel(scatter_rows_kernel, dim3(grid), dim3(256), (size_t)(0), s, src, dst, ids, row_len));
  }
  VRPS_LAUNCHED("scatter_rows");
  return VRPS_OK;
}

int to_store(const float* src, void* dst, int64_t n, int kind, float scale, cudaStream_t s) {
  FwdOut f{};
  f.store = kind;
  f.scale = scale;
  f.inv = 1.f / scale;
  { LaunchScope _ls("store_kernel", s, (kind ? 6.0 : 8.0) * n);
  VRPS_CUDA(launch_kernel(store_kernel, dim3(NPART), dim3(256), (size_t)(0), s, src, dst, n, f));
  }
  VRPS_LAUNCHED("to_store");
  return VRPS_OK;
}

int fill(float* p, float v, int64_t n, cudaStream_t s) {
  { LaunchScope _ls("fill_kernel", s, 4.0 * n);
  VRPS_CUDA(launch_kernel(fill_kernel, dim3(NPART), dim3(256), (size_t)(0), s, p, v, n));
  }
  VRPS_LAUNCHED("fill");
  return VRPS_OK;
}

int copy_or_zero(float* dst, const float* src, int64_t n, cudaStream_t s) {
  if (src) {
    VRPS_CUDA(cudaMemcpyAsync(dst, src, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  } else {
    VRPS_CUDA(cudaMemsetAsync(dst, 0, sizeof(float) * (size_t)n, s));
  }
  return VRPS_OK;
}

}  // namespace vrps
