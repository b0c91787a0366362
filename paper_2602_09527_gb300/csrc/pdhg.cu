// Reference minimiser of Eq. (tomography_problem) by preconditioned PDHG on the GPU: the
// long-run solver the paper uses to obtain x* and F* (Section 2.1, Section 3), here as the
// reference of the relative objective gap.  Saddle form with K = [A; D]:
//   y_A <- (y_A + sigma_A (A x_bar - b)) / (1 + sigma_A)
//   y_D <- projection of y_D + sigma_D D x_bar onto {||w_p|| <= alpha}
//   x   <- max(0, x - tau (A^T y_A + D^T y_D)),  x_bar = 2 x_new - x_old
// with the diagonal steps of Pock and Chambolle (2011, exponent 1): tau_j = 1 / (column sum
// of A + column sum of |D|), sigma_A = 1 / ray sum of A, sigma_D = 1/2 on rows with a
// difference (0 on the zero rows at the last index).  Rows or columns with zero sum get
// step 0.  One iteration is a full forward, a full adjoint and three elementwise kernels.
#include <cmath>
#include <cstring>

#include "vrps_internal.h"

namespace vrps {
namespace {

struct PdDims {
  int nx, ny, nz;
  long long n;
};

__global__ void pdhg_invert(float* v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = v[i] > 0.f ? 1.f / v[i] : 0.f;
}

// tau = 1 / (A^T 1 + column sums of |D|) in place over A^T 1
__global__ void pdhg_tau(float* col, PdDims D) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < D.n; p += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(p % D.nx), iy = (int)((p / D.nx) % D.ny), iz = (int)(p / ((int64_t)D.nx * D.ny));
    int c = (ix < D.nx - 1) + (ix > 0) + (iy < D.ny - 1) + (iy > 0);
    if (D.nz > 1) c += (iz < D.nz - 1) + (iz > 0);
    const float s = col[p] + (float)c;
    col[p] = s > 0.f ? 1.f / s : 0.f;
  }
}

__global__ void pdhg_dual_a(float* ya, const float* ax, const float* b, const float* sig, int64_t m) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const float s = sig[i];
    ya[i] = fmaf(s, ax[i] - b[i], ya[i]) / (1.f + s);
  }
}

__global__ void pdhg_dual_d(float* yd, const float* xb, PdDims D, float alpha) {
  const int comps = D.nz > 1 ? 3 : 2;
  const int64_t nxy = (int64_t)D.nx * D.ny;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < D.n; p += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(p % D.nx), iy = (int)((p / D.nx) % D.ny), iz = (int)(p / nxy);
    const float c = xb[p];
    float w[3];
    w[0] = ix < D.nx - 1 ? fmaf(0.5f, xb[p + 1] - c, yd[p]) : yd[p];
    w[1] = iy < D.ny - 1 ? fmaf(0.5f, xb[p + D.nx] - c, yd[D.n + p]) : yd[D.n + p];
    w[2] = 0.f;
    if (comps == 3) w[2] = iz < D.nz - 1 ? fmaf(0.5f, xb[p + nxy] - c, yd[2 * D.n + p]) : yd[2 * D.n + p];
    const float nrm = sqrtf(fmaf(w[0], w[0], fmaf(w[1], w[1], w[2] * w[2])));
    const float sc = alpha > 0.f ? 1.f / fmaxf(1.f, nrm / alpha) : 0.f;
    for (int k = 0; k < comps; ++k) yd[k * D.n + p] = w[k] * sc;
  }
}

__global__ void pdhg_primal(float* x, float* xb, const float* aty, const float* yd, const float* tau, PdDims D,
                            int nonneg) {
  const int64_t nxy = (int64_t)D.nx * D.ny;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < D.n; p += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(p % D.nx), iy = (int)((p / D.nx) % D.ny), iz = (int)(p / nxy);
    // (D^T y)_p = sum_c y_c[p - e_c] (p - e_c has a difference) - y_c[p] (p has one)
    float dty = 0.f;
    if (ix > 0) dty += yd[p - 1];
    if (ix < D.nx - 1) dty -= yd[p];
    if (iy > 0) dty += yd[D.n + p - D.nx];
    if (iy < D.ny - 1) dty -= yd[D.n + p];
    if (D.nz > 1) {
      if (iz > 0) dty += yd[2 * D.n + p - nxy];
      if (iz < D.nz - 1) dty -= yd[2 * D.n + p];
    }
    const float xo = x[p];
    float xn = fmaf(-tau[p], aty[p] + dty, xo);
    if (nonneg) xn = fmaxf(xn, 0.f);
    x[p] = xn;
    xb[p] = 2.f * xn - xo;
  }
}

constexpr int PD_BLOCKS = 608, PD_THREADS = 256;

// inside the solver's do { } while (false): record a CUDA error and leave the block
#define PD_CUDA(call)                             \
  {                                               \
    const cudaError_t _pe = (call);               \
    if (_pe != cudaSuccess) {                     \
      rc = ::vrps::cuda_fail(_pe, #call);         \
      break;                                      \
    }                                             \
  }

}  // namespace
}  // namespace vrps

using namespace vrps;

extern "C" int vrps_pdhg(const float* b, const vrps_geom* gc, double alpha, int iters, int nonneg, int eval_every,
                         double* history, int history_cap, float* x_out, vrps_report* rep, vrps_stream_t stream) {
  if (!gc) return fail(VRPS_ERR_INVALID_ARG, "geometry handle is NULL");
  if (!b || !x_out) return fail(VRPS_ERR_INVALID_ARG, "b or x_out is NULL");
  if (!(alpha >= 0) || !std::isfinite(alpha)) return fail(VRPS_ERR_INVALID_ARG, "alpha must be >= 0");
  if (iters < 0) return fail(VRPS_ERR_INVALID_ARG, "iters must be >= 0");
  if (history && history_cap <= 0) return fail(VRPS_ERR_INVALID_ARG, "history_cap must be > 0");
  vrps_geom* g = const_cast<vrps_geom*>(gc);
  {
    int dev = -1;
    VRPS_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(VRPS_ERR_INVALID_ARG, "geometry belongs to device %d", g->device);
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = g->n, m = g->m;
  const int dims = g->dims;
  PdDims D{g->nx, g->ny, dims == 3 ? g->nz : 1, (long long)n};
  float *x = nullptr, *xb = nullptr, *tau = nullptr, *aty = nullptr, *yd = nullptr, *ya = nullptr, *sig = nullptr,
        *ax = nullptr;
  auto cleanup = [&]() {
    for (float* q : {x, xb, tau, aty, yd, ya, sig, ax})
      if (q) cudaFree(q);
  };
  auto alloc = [&](float** q, size_t count) -> int {
    if (cudaMalloc((void**)q, sizeof(float) * count) != cudaSuccess) {
      cudaGetLastError();
      return fail(VRPS_ERR_OUT_OF_MEMORY, "pdhg: %zu floats", count);
    }
    return VRPS_OK;
  };
  int rc = VRPS_OK;
  vrps_report r;
  std::memset(&r, 0, sizeof(r));
  r.objective = NAN;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  do {
    if ((rc = alloc(&x, n)) || (rc = alloc(&xb, n)) || (rc = alloc(&tau, n)) || (rc = alloc(&aty, n)) ||
        (rc = alloc(&yd, (size_t)dims * n)) || (rc = alloc(&ya, m)) || (rc = alloc(&sig, m)) || (rc = alloc(&ax, m)))
      break;
    // steps: sigma_A = 1 / (A 1), tau = 1 / (A^T 1 + |D|^T 1)
    if ((rc = fill(x, 1.f, n, s))) break;
    if ((rc = fill(ya, 1.f, m, s))) break;
    {
      FwdOut fo{sig, nullptr, nullptr};
      if ((rc = proj_forward(g, x, nullptr, g->order_natural, g->n_angles, FWD_PLAIN, fo, s))) break;
      UpdateArgs ua;
      std::memset(&ua, 0, sizeof(ua));
      ua.out = tau;
      if ((rc = proj_adjoint(g, ya, g->order_natural, g->n_angles, ua, s))) break;
    }
    {
      LaunchScope _ls("pdhg_steps", s, 8.0 * (double)(n + m));
      if (launch_kernel(pdhg_invert, dim3(PD_BLOCKS), dim3(PD_THREADS), (size_t)0, s, sig, m) != cudaSuccess ||
          launch_kernel(pdhg_tau, dim3(PD_BLOCKS), dim3(PD_THREADS), (size_t)0, s, tau, D) != cudaSuccess) {
        rc = cuda_fail(cudaGetLastError(), "pdhg steps");
        break;
      }
    }
    PD_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * n, s));
    PD_CUDA(cudaMemsetAsync(xb, 0, sizeof(float) * n, s));
    PD_CUDA(cudaMemsetAsync(ya, 0, sizeof(float) * m, s));
    PD_CUDA(cudaMemsetAsync(yd, 0, sizeof(float) * dims * n, s));
    PD_CUDA(cudaEventCreate(&e0));
    PD_CUDA(cudaEventCreate(&e1));
    PD_CUDA(cudaEventRecord(e0, s));
    int k = 0;
    for (; k < iters; ++k) {
      FwdOut fo{ax, nullptr, nullptr};
      if ((rc = proj_forward(g, xb, nullptr, g->order_natural, g->n_angles, FWD_PLAIN, fo, s))) break;
      {
        LaunchScope _ls("pdhg_dual", s, 16.0 * (double)m + 4.0 * (2 * dims + 1) * (double)n);
        if (launch_kernel(pdhg_dual_a, dim3(PD_BLOCKS), dim3(PD_THREADS), (size_t)0, s, ya, (const float*)ax, b,
                          (const float*)sig, m) != cudaSuccess ||
            launch_kernel(pdhg_dual_d, dim3(PD_BLOCKS), dim3(PD_THREADS), (size_t)0, s, yd, (const float*)xb, D,
                          (float)alpha) != cudaSuccess) {
          rc = cuda_fail(cudaGetLastError(), "pdhg dual");
          break;
        }
      }
      UpdateArgs ua;
      std::memset(&ua, 0, sizeof(ua));
      ua.out = aty;
      if ((rc = proj_adjoint(g, ya, g->order_natural, g->n_angles, ua, s))) break;
      {
        LaunchScope _ls("pdhg_primal", s, 4.0 * (6 + dims) * (double)n);
        if (launch_kernel(pdhg_primal, dim3(PD_BLOCKS), dim3(PD_THREADS), (size_t)0, s, x, xb, (const float*)aty,
                          (const float*)yd, (const float*)tau, D, nonneg) != cudaSuccess) {
          rc = cuda_fail(cudaGetLastError(), "pdhg primal");
          break;
        }
      }
      if (eval_every > 0 && (k + 1) % eval_every == 0) {
        double o3[3];
        if ((rc = vrps_objective(g, x, b, alpha, o3, stream))) break;
        r.objective = o3[0];
        if (history && r.evaluations < history_cap) {
          history[2 * (size_t)r.evaluations] = (double)(k + 1);
          history[2 * (size_t)r.evaluations + 1] = o3[0];
        }
        r.evaluations += 1;
        if (!std::isfinite(o3[0])) {
          rc = fail(VRPS_ERR_DIVERGED, "pdhg objective is not finite at iteration %d", k + 1);
          ++k;
          break;
        }
      }
    }
    if (rc != VRPS_OK) break;
    PD_CUDA(cudaEventRecord(e1, s));
    PD_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    PD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    r.iterations = k;
    r.seconds = ms * 1e-3;
    r.passes = (double)k;
    PD_CUDA(cudaMemcpyAsync(x_out, x, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    PD_CUDA(cudaStreamSynchronize(s));
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cleanup();
  if (rc == VRPS_OK && rep) *rep = r;
  return rc;
}
