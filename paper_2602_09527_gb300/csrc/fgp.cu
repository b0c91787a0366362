// FGP (Beck & Teboulle 2009) for the prox of tau (TV + I_{x>=0}), the prox step of
// Algorithm 1 (Section 2.1: fixed number of warm-started inner iterations).
//
// Dual w (one 2- or 3-vector per pixel, ||w|| <= 1).  With z the extrapolated dual,
//   x    = P_+( v + tau div z )            (D^T = -div, forward differences, Neumann)
//   w'   = P_B( z + D x / (4 d tau) )      (d = 2 or 3)
//   z'   = w' + mom_k (w' - w)             (mom from t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2)
// Kernels store only w_k and w_{k-1} and rebuild z on the fly, so one iteration reads
// v, w_k, w_{k-1} and writes w_{k+1} (7 floats per pixel in 2D, 10 per voxel in 3D).
// Three dual buffers rotate so that no launch writes a buffer another CTA still reads.
// The output kernel forms x+ = P_+(v + tau div w_K) and applies the fused tail of the
// solver (x <- x+, h += (p/gamma)(x+ - x_hat), FISTA momentum, transposed copy).
#include <cmath>
#include <vector>

#include "vrps_internal.h"

namespace vrps {
namespace {

constexpr int FX = 32, FY = 8;

__global__ void __launch_bounds__(FX* FY) fgp2d_iter(const float* __restrict__ v, const float* wc,
                                                     const float* wp, float* __restrict__ wn, int nx,
                                                     int ny, float tau, float step, float mom,
                                                     int nonneg) {
  __shared__ float z1[FY + 2][FX + 2];
  __shared__ float z2[FY + 2][FX + 2];
  __shared__ float xs[FY + 1][FX + 1];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FX + tx;
  const int ix0 = blockIdx.x * FX, iy0 = blockIdx.y * FY;
  const size_t n = (size_t)nx * ny;
  for (int e = tid; e < (FX + 2) * (FY + 2); e += FX * FY) {
    const int lx = e % (FX + 2), ly = e / (FX + 2);
    const int gx = ix0 - 1 + lx, gy = iy0 - 1 + ly;
    float a = 0.f, b = 0.f;
    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
      const size_t p = (size_t)gy * nx + gx;
      const float c1 = wc[p], c2 = wc[n + p];
      if (mom != 0.f) {
        a = c1 + mom * (c1 - wp[p]);
        b = c2 + mom * (c2 - wp[n + p]);
      } else {
        a = c1;
        b = c2;
      }
    }
    z1[ly][lx] = a;
    z2[ly][lx] = b;
  }
  __syncthreads();
  for (int e = tid; e < (FX + 1) * (FY + 1); e += FX * FY) {
    const int lx = e % (FX + 1), ly = e / (FX + 1);
    const int gx = ix0 + lx, gy = iy0 + ly;
    float xv = 0.f;
    if (gx < nx && gy < ny) {
      float d = 0.f;
      if (gx < nx - 1) d += z1[ly + 1][lx + 1];
      if (gx > 0) d -= z1[ly + 1][lx];
      if (gy < ny - 1) d += z2[ly + 1][lx + 1];
      if (gy > 0) d -= z2[ly][lx + 1];
      xv = fmaf(tau, d, v[(size_t)gy * nx + gx]);
      if (nonneg) xv = fmaxf(xv, 0.f);
    }
    xs[ly][lx] = xv;
  }
  __syncthreads();
  const int gx = ix0 + tx, gy = iy0 + ty;
  if (gx < nx && gy < ny) {
    const float xc = xs[ty][tx];
    const float d1 = gx < nx - 1 ? xs[ty][tx + 1] - xc : 0.f;
    const float d2 = gy < ny - 1 ? xs[ty + 1][tx] - xc : 0.f;
    const float q1 = fmaf(step, d1, z1[ty + 1][tx + 1]);
    const float q2 = fmaf(step, d2, z2[ty + 1][tx + 1]);
    const float den = fmaxf(1.f, sqrtf(q1 * q1 + q2 * q2));
    const size_t p = (size_t)gy * nx + gx;
    wn[p] = q1 / den;
    wn[n + p] = q2 / den;
  }
}

// x+ = P_+(v + tau div w) and the fused tail.  32x32 tile, block 32x8 (4 rows per thread).
__global__ void __launch_bounds__(256) fgp2d_out(const float* __restrict__ v, const float* __restrict__ w,
                                                 float* wdst, int nx, int ny, float tau, int nonneg,
                                                 ProxTail t) {
  __shared__ float tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const size_t n = (size_t)nx * ny;
  const bool transposed = (t.mode == 1) && (t.xT || t.yT);
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int gx = bx + threadIdx.x, gy = by + k;
    float tv_out = 0.f;
    if (gx < nx && gy < ny) {
      const size_t p = (size_t)gy * nx + gx;
      float d = 0.f;
      if (gx < nx - 1) d += w[p];
      if (gx > 0) d -= w[p - 1];
      if (gy < ny - 1) d += w[n + p];
      if (gy > 0) d -= w[n + p - nx];
      float xp = fmaf(tau, d, v[p]);
      if (nonneg) xp = fmaxf(xp, 0.f);
      if (wdst) {
        wdst[p] = w[p];
        wdst[n + p] = w[n + p];
      }
      if (t.mode == 0) {
        t.out[p] = xp;
      } else {
        const float xold = t.x[p];
        t.x[p] = xp;
        if (t.h) t.h[p] += t.p_over_gamma * (xp - t.xhat[p]);
        if (t.xprox) t.xprox[p] = xp;
        if (t.y) {
          const float yv = xp + t.mom * (xp - xold);
          t.y[p] = yv;
          tv_out = yv;
        } else {
          tv_out = xp;
        }
      }
    }
    if (transposed) tile[k][threadIdx.x] = tv_out;
  }
  if (!transposed) return;
  __syncthreads();
  float* dstT = t.y ? t.yT : t.xT;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int gy = by + threadIdx.x, gx = bx + k;
    if (gx < nx && gy < ny && dstT) dstT[(size_t)gx * ny + gy] = tile[threadIdx.x][k];
  }
}

// ---------------------------------------------------------------- 3D
struct Dims3 {
  int nx, ny, nz;
  size_t n;
};

__device__ __forceinline__ float zval(const float* wc, const float* wp, size_t idx, float mom) {
  const float c = wc[idx];
  return mom != 0.f ? c + mom * (c - wp[idx]) : c;
}

// x at (gx,gy,gz) from the extrapolated dual; caller guarantees the point is inside.
__device__ __forceinline__ float x3(const float* __restrict__ v, const float* wc, const float* wp,
                                    const Dims3 D, int gx, int gy, int gz, float tau, float mom,
                                    int nonneg) {
  const size_t p = ((size_t)gz * D.ny + gy) * D.nx + gx;
  float d = 0.f;
  if (gx < D.nx - 1) d += zval(wc, wp, p, mom);
  if (gx > 0) d -= zval(wc, wp, p - 1, mom);
  if (gy < D.ny - 1) d += zval(wc, wp, D.n + p, mom);
  if (gy > 0) d -= zval(wc, wp, D.n + p - D.nx, mom);
  if (gz < D.nz - 1) d += zval(wc, wp, 2 * D.n + p, mom);
  if (gz > 0) d -= zval(wc, wp, 2 * D.n + p - (size_t)D.nx * D.ny, mom);
  float xv = fmaf(tau, d, v[p]);
  return nonneg ? fmaxf(xv, 0.f) : xv;
}

__global__ void __launch_bounds__(256) fgp3d_iter(const float* __restrict__ v, const float* wc,
                                                  const float* wp, float* __restrict__ wn, Dims3 D,
                                                  float tau, float step, float mom, int nonneg) {
  const int gx = blockIdx.x * 32 + threadIdx.x;
  const int gy = blockIdx.y * 8 + threadIdx.y;
  const int gz = blockIdx.z;
  if (gx >= D.nx || gy >= D.ny) return;
  const size_t p = ((size_t)gz * D.ny + gy) * D.nx + gx;
  const float xc = x3(v, wc, wp, D, gx, gy, gz, tau, mom, nonneg);
  const float d1 = gx < D.nx - 1 ? x3(v, wc, wp, D, gx + 1, gy, gz, tau, mom, nonneg) - xc : 0.f;
  const float d2 = gy < D.ny - 1 ? x3(v, wc, wp, D, gx, gy + 1, gz, tau, mom, nonneg) - xc : 0.f;
  const float d3 = gz < D.nz - 1 ? x3(v, wc, wp, D, gx, gy, gz + 1, tau, mom, nonneg) - xc : 0.f;
  const float q1 = fmaf(step, d1, zval(wc, wp, p, mom));
  const float q2 = fmaf(step, d2, zval(wc, wp, D.n + p, mom));
  const float q3 = fmaf(step, d3, zval(wc, wp, 2 * D.n + p, mom));
  const float den = fmaxf(1.f, sqrtf(q1 * q1 + q2 * q2 + q3 * q3));
  wn[p] = q1 / den;
  wn[D.n + p] = q2 / den;
  wn[2 * D.n + p] = q3 / den;
}

__global__ void __launch_bounds__(256) fgp3d_out(const float* __restrict__ v, const float* __restrict__ w,
                                                 float* wdst, Dims3 D, float tau, int nonneg, ProxTail t) {
  const int gx = blockIdx.x * 32 + threadIdx.x;
  const int gy = blockIdx.y * 8 + threadIdx.y;
  const int gz = blockIdx.z;
  if (gx >= D.nx || gy >= D.ny) return;
  const size_t p = ((size_t)gz * D.ny + gy) * D.nx + gx;
  const float xp = x3(v, w, w, D, gx, gy, gz, tau, 0.f, nonneg);
  if (wdst) {
    wdst[p] = w[p];
    wdst[D.n + p] = w[D.n + p];
    wdst[2 * D.n + p] = w[2 * D.n + p];
  }
  if (t.mode == 0) {
    t.out[p] = xp;
    return;
  }
  const float xold = t.x[p];
  t.x[p] = xp;
  if (t.h) t.h[p] += t.p_over_gamma * (xp - t.xhat[p]);
  if (t.xprox) t.xprox[p] = xp;
  if (t.y) t.y[p] = xp + t.mom * (xp - xold);
}

}  // namespace

int fgp_run(const vrps_geom* g, const float* v, float tau, int iters, int nonneg, float* dual,
            const ProxTail& tail, cudaStream_t s) {
  vrps_geom* gm = const_cast<vrps_geom*>(g);
  const size_t dn = (size_t)g->dims * (size_t)g->n;
  if (iters > 0) {
    VRPS_TRY(ensure(&gm->ws.dual_s1, dn));
    VRPS_TRY(ensure(&gm->ws.dual_s2, dn));
  }
  // momentum coefficients in float64: t_0 = 1, t_{k+1} = (1+sqrt(1+4 t_k^2))/2,
  // iteration k (k >= 1) extrapolates with (t_{k-1} - 1)/t_k, iteration 0 with 0.
  std::vector<float> mom(iters > 0 ? iters : 1, 0.f);
  {
    double t = 1.0, tprev = 1.0;
    for (int k = 0; k < iters; ++k) {
      if (k >= 1) mom[k] = (float)((tprev - 1.0) / t);
      const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
      tprev = t;
      t = tn;
    }
  }
  const float step = (float)(1.0 / (4.0 * g->dims * (double)tau));
  float* buf[3] = {dual, gm->ws.dual_s1, gm->ws.dual_s2};
  int cur = 0, prev = 0;
  for (int k = 0; k < iters; ++k) {
    const int nxt = (k == 0) ? 1 : 3 - cur - prev;
    if (g->dims == 2) {
      dim3 grid((g->nx + FX - 1) / FX, (g->ny + FY - 1) / FY), block(FX, FY);
      { LaunchScope _ls("fgp2d_iter", s);
      fgp2d_iter<<<grid, block, 0, s>>>(v, buf[cur], buf[prev], buf[nxt], g->nx, g->ny, tau, step,
                                       mom[k], nonneg);
      }
    } else {
      Dims3 D{g->nx, g->ny, g->nz, (size_t)g->n};
      dim3 grid((g->nx + 31) / 32, (g->ny + 7) / 8, g->nz), block(32, 8);
      { LaunchScope _ls("fgp3d_iter", s);
      fgp3d_iter<<<grid, block, 0, s>>>(v, buf[cur], buf[prev], buf[nxt], D, tau, step, mom[k], nonneg);
      }
    }
    VRPS_LAUNCHED("fgp_iter");
    prev = cur;
    cur = nxt;
  }
  float* wdst = (cur != 0) ? dual : nullptr;
  if (g->dims == 2) {
    dim3 grid((g->nx + 31) / 32, (g->ny + 31) / 32), block(32, 8);
    { LaunchScope _ls("fgp2d_out", s);
    fgp2d_out<<<grid, block, 0, s>>>(v, buf[cur], wdst, g->nx, g->ny, tau, nonneg, tail);
    }
  } else {
    Dims3 D{g->nx, g->ny, g->nz, (size_t)g->n};
    dim3 grid((g->nx + 31) / 32, (g->ny + 7) / 8, g->nz), block(32, 8);
    { LaunchScope _ls("fgp3d_out", s);
    fgp3d_out<<<grid, block, 0, s>>>(v, buf[cur], wdst, D, tau, nonneg, tail);
    }
  }
  VRPS_LAUNCHED("fgp_out");
  return VRPS_OK;
}

}  // namespace vrps
