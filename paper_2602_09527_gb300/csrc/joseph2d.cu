// 2D parallel-beam Joseph projector: ray-driven forward (gather) with fused residual /
// estimator epilogues, and pixel-driven exact transpose with the fused ProxSkip update.
//
// Forward (Section 1.2, A_i x): one CTA row of 32 bins x 8 line phases marches the rays
// of one angle; each thread accumulates every 8th dominant-axis line, the 8 partial sums
// are reduced in shared memory in a fixed order.  Rays of angles marched along columns
// read the transposed image so that the 32 lanes always read along a row (coalesced).
//
// Adjoint (A_i^T r): one thread per pixel of a 16x16 tile.  For every angle of the launch
// the tile's footprint on the detector (at most fp bins) is staged in shared memory, then
// each pixel sums w_j r_j over the <= nc bins whose ray passes within one interpolation
// cell of its centre, with the Joseph weight of that (ray, pixel) pair.  No atomics.
#include <cstring>

#include "vrps_internal.h"

namespace vrps {
namespace {

constexpr int FWD_LANES = 32;
constexpr int FWD_PHASES = 8;
constexpr int ADJ_T = 16;
constexpr int ADJ_CHUNK = 64;

struct Fwd2DParams {
  const float* x;
  const float* xT;
  const AngleInfo2D* ang;
  const int* ids;
  int nx, ny, nb;
  float jc;
  FwdOut o;
};

template <int MODE>
__global__ void __launch_bounds__(FWD_LANES * FWD_PHASES) fwd2d_kernel(Fwd2DParams P) {
  __shared__ float red[FWD_PHASES][FWD_LANES + 1];
  const int lane = threadIdx.x, ph = threadIdx.y;
  const int j = blockIdx.x * FWD_LANES + lane;
  const int row = blockIdx.y;
  const AngleInfo2D in = P.ang[P.ids[row]];
  const bool tr = in.T != 0;
  const float* __restrict__ img = tr ? P.xT : P.x;
  const int ncols = tr ? P.ny : P.nx;
  const int nlines = tr ? P.nx : P.ny;
  const float uc = 0.5f * (float)(ncols - 1);
  const float lc = 0.5f * (float)(nlines - 1);
  float acc = 0.f;
  if (j < P.nb) {
    const float u0 = fmaf(in.A1, (float)j - P.jc, uc);   // line-range clipping only
    int lo = 0, hi = nlines - 1;
    if (in.A2 != 0.f) {
      // lines where the ray's interpolation point is in (-1, ncols); widened by one line
      float la = lc + (-1.f - u0) / in.A2;
      float lb = lc + ((float)ncols - u0) / in.A2;
      if (la > lb) {
        const float t = la;
        la = lb;
        lb = t;
      }
      la = fminf(fmaxf(la, -2.f), (float)nlines + 1.f);
      lb = fminf(fmaxf(lb, -2.f), (float)nlines + 1.f);
      lo = max(lo, (int)floorf(la) - 1);
      hi = min(hi, (int)ceilf(lb) + 1);
    } else if (!(u0 > -1.f && u0 < (float)ncols)) {
      hi = -1;
    }
    // exact fixed-point walk along the ray: U = u * 2^32
    const int l0 = lo + ph;
    long long U = (long long)(ncols - 1) * 2147483648LL + in.A1H * (long long)(2 * j - (P.nb - 1)) +
                  in.A2H * (long long)(2 * l0 - (nlines - 1));
    const long long dU = in.A2H * (2 * FWD_PHASES);
    for (int l = l0; l <= hi; l += FWD_PHASES, U += dU) {
      const int i0 = fix_floor(U);
      const float f = fix_frac(U);
      const float* rp = img + (size_t)l * ncols;
      const float v0 = (i0 >= 0 && i0 < ncols) ? __ldg(rp + i0) : 0.f;
      const float v1 = (i0 + 1 >= 0 && i0 + 1 < ncols) ? __ldg(rp + i0 + 1) : 0.f;
      acc += fmaf(f, v1 - v0, v0);
    }
  }
  red[ph][lane] = acc;
  __syncthreads();
  if (ph == 0 && j < P.nb) {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < FWD_PHASES; ++q) s += red[q][lane];
    const float r = s * in.wgt;
    const size_t idx = (size_t)row * P.nb + j;
    if (MODE == FWD_PLAIN) {
      P.o.y[idx] = r;
    } else if (MODE == FWD_RESID) {
      P.o.y[idx] = r - P.o.b[idx];
    } else if (MODE == FWD_SVRG) {
      P.o.y[idx] = r - P.o.tab[idx];
    } else if (MODE == FWD_SAGA) {
      const float res = r - P.o.b[idx];
      P.o.y[idx] = res - P.o.tab[idx];
      P.o.tab[idx] = res;
    } else {  // FWD_SNAP
      P.o.tab[idx] = r;
      P.o.y[idx] = r - P.o.b[idx];
    }
  }
}

struct Adj2DParams {
  const float* r;
  const AngleInfo2D* ang;
  const int* ids;
  int rows;
  int nx, ny, nb;
  float jc, cx, cy;
  int fp, nc, chunk;
  UpdateArgs u;
};

__global__ void __launch_bounds__(ADJ_T* ADJ_T) adj2d_kernel(Adj2DParams P) {
  extern __shared__ float sm[];  // [chunk][fp]
  __shared__ int s_jlo[ADJ_CHUNK];
  __shared__ int s_J0[ADJ_CHUNK];
  __shared__ float s_F0[ADJ_CHUNK];
  __shared__ AngleInfo2D s_ang[ADJ_CHUNK];
  __shared__ float s_tile[ADJ_T][ADJ_T + 1];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * ADJ_T + tx;
  const int ix0 = blockIdx.x * ADJ_T, iy0 = blockIdx.y * ADJ_T;
  const int ix = ix0 + tx, iy = iy0 + ty;
  const float ftx = (float)tx, fty = (float)ty;
  float acc = 0.f;
  for (int r0 = 0; r0 < P.rows; r0 += P.chunk) {
    const int nr = min(P.chunk, P.rows - r0);
    if (tid < nr) {
      // exact fractional bin of the tile origin: t = J0 + F0 (fixed point), then the
      // pixels of the tile only add small float offsets Bx tx + By ty
      const AngleInfo2D in = P.ang[P.ids[r0 + tid]];
      s_ang[tid] = in;
      const long long T0 = (long long)(P.nb - 1) * 2147483648LL + in.BxH * (long long)(2 * ix0 - (P.nx - 1)) +
                           in.ByH * (long long)(2 * iy0 - (P.ny - 1));
      const int J0 = fix_floor(T0);
      const float F0 = fix_frac(T0);
      const float e = (float)(ADJ_T - 1);
      const float tmin = F0 + fminf(0.f, in.Bx * e) + fminf(0.f, in.By * e);
      s_J0[tid] = J0;
      s_F0[tid] = F0;
      s_jlo[tid] = J0 + (int)floorf(tmin - in.hw) - 1;
    }
    __syncthreads();
    for (int e = tid; e < nr * P.fp; e += ADJ_T * ADJ_T) {
      const int q = e / P.fp;
      const int j = s_jlo[q] + (e - q * P.fp);
      sm[e] = (j >= 0 && j < P.nb) ? __ldg(P.r + (size_t)(r0 + q) * P.nb + j) : 0.f;
    }
    __syncthreads();
    for (int q = 0; q < nr; ++q) {
      const AngleInfo2D in = s_ang[q];
      const float tr = fmaf(in.By, fty, fmaf(in.Bx, ftx, s_F0[q]));   // t - J0
      const int js = (int)floorf(tr - in.hw) + 1;                      // first candidate - J0
      const int off = s_J0[q] - s_jlo[q];
      const float* row = sm + q * P.fp;
      float a = 0.f;
      for (int c = 0; c < P.nc; ++c) {
        const int jj = js + c;
        const int o = jj + off;
        const float w = fmaxf(0.f, 1.f - fabsf((float)jj - tr) * in.inv_hw);
        if (o >= 0 && o < P.fp) a = fmaf(w, row[o], a);
      }
      acc = fmaf(a, in.wgt, acc);
    }
    __syncthreads();
  }
  const bool inside = ix < P.nx && iy < P.ny;
  const size_t p = (size_t)iy * P.nx + ix;
  const UpdateArgs& u = P.u;
  if (!u.enabled) {
    if (inside) u.out[p] = acc;
    return;
  }
  // Algorithm 1, estimator + x_hat lines: G = cN g + gbar; x_hat = base - gamma (G - h)
  float xnew = 0.f;
  if (inside) {
    float G = u.cN * acc;
    if (u.gbar) {
      const float gb = u.gbar[p];
      G += gb;
      if (u.saga) u.gbar[p] = gb + acc;
    }
    const float base = u.base[p];
    if (u.h) {
      const float hp = u.h[p];
      const float xh = base - u.gamma * (G - hp);
      if (u.theta) {
        u.xhat[p] = xh;
        u.v[p] = xh - u.gamma_over_p * hp;
      } else {
        u.x[p] = xh;
        xnew = xh;
      }
    } else {
      const float xh = base - u.gamma * G;
      if (u.theta) {
        u.v[p] = xh;
      } else {
        u.x[p] = xh;
        xnew = xh;
      }
    }
  }
  if (!u.theta && u.xT) {
    s_tile[ty][tx] = xnew;
    __syncthreads();
    const int ox = ix0 + ty, oy = iy0 + tx;
    if (ox < P.nx && oy < P.ny) u.xT[(size_t)ox * P.ny + oy] = s_tile[tx][ty];
  }
}

__global__ void transpose_kernel(const float* __restrict__ in, float* __restrict__ out, int ny, int nx) {
  __shared__ float t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int x = bx + threadIdx.x, y = by + k;
    if (x < nx && y < ny) t[k][threadIdx.x] = in[(size_t)y * nx + x];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int y = by + threadIdx.x, x = bx + k;   // out[x][y]
    if (x < nx && y < ny) out[(size_t)x * ny + y] = t[threadIdx.x][k];
  }
}

}  // namespace

int transpose2d(const float* in, float* out, int ny, int nx, cudaStream_t s) {
  dim3 grid((nx + 31) / 32, (ny + 31) / 32), block(32, 8);
  { LaunchScope _ls("transpose_kernel", s);
  transpose_kernel<<<grid, block, 0, s>>>(in, out, ny, nx);
  }
  VRPS_LAUNCHED("transpose2d");
  return VRPS_OK;
}

int fwd2d(const vrps_geom* g, const float* x, const float* xT, const int* ids, int rows, int mode,
          FwdOut o, cudaStream_t s) {
  if (rows <= 0) return VRPS_OK;
  Fwd2DParams P;
  P.x = x;
  P.xT = xT;
  P.ang = g->ang2d;
  P.ids = ids;
  P.nx = g->nx;
  P.ny = g->ny;
  P.nb = g->n_bins;
  P.jc = 0.5f * (float)(g->n_bins - 1);
  P.o = o;
  dim3 grid((g->n_bins + FWD_LANES - 1) / FWD_LANES, rows), block(FWD_LANES, FWD_PHASES);
  switch (mode) {
    case FWD_PLAIN: { LaunchScope _ls("fwd2d_kernel", s); fwd2d_kernel<FWD_PLAIN><<<grid, block, 0, s>>>(P); } break;
    case FWD_RESID: { LaunchScope _ls("fwd2d_kernel", s); fwd2d_kernel<FWD_RESID><<<grid, block, 0, s>>>(P); } break;
    case FWD_SVRG: { LaunchScope _ls("fwd2d_kernel", s); fwd2d_kernel<FWD_SVRG><<<grid, block, 0, s>>>(P); } break;
    case FWD_SAGA: { LaunchScope _ls("fwd2d_kernel", s); fwd2d_kernel<FWD_SAGA><<<grid, block, 0, s>>>(P); } break;
    case FWD_SNAP: { LaunchScope _ls("fwd2d_kernel", s); fwd2d_kernel<FWD_SNAP><<<grid, block, 0, s>>>(P); } break;
    default: return fail(VRPS_ERR_INVALID_ARG, "bad forward mode %d", mode);
  }
  VRPS_LAUNCHED("fwd2d");
  return VRPS_OK;
}

int adj2d(const vrps_geom* g, const float* r, const int* ids, int rows, const UpdateArgs& u,
          cudaStream_t s) {
  Adj2DParams P;
  P.r = r;
  P.ang = g->ang2d;
  P.ids = ids;
  P.rows = rows;
  P.nx = g->nx;
  P.ny = g->ny;
  P.nb = g->n_bins;
  P.jc = 0.5f * (float)(g->n_bins - 1);
  P.cx = 0.5f * (float)(g->nx - 1);
  P.cy = 0.5f * (float)(g->ny - 1);
  P.fp = g->adj_fp;
  P.nc = g->adj_nc;
  int chunk = (int)(48 * 1024 / (sizeof(float) * (size_t)g->adj_fp));
  P.chunk = chunk < ADJ_CHUNK ? (chunk < 1 ? 1 : chunk) : ADJ_CHUNK;
  P.u = u;
  const size_t smem = sizeof(float) * (size_t)P.chunk * P.fp;
  dim3 grid((g->nx + ADJ_T - 1) / ADJ_T, (g->ny + ADJ_T - 1) / ADJ_T), block(ADJ_T, ADJ_T);
  { LaunchScope _ls("adj2d_kernel", s);
  adj2d_kernel<<<grid, block, smem, s>>>(P);
  }
  VRPS_LAUNCHED("adj2d");
  return VRPS_OK;
}

}  // namespace vrps
