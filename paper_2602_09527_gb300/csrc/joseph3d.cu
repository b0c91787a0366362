// 3D circular cone-beam Joseph projector: ray-driven forward (gather) and voxel-driven exact
// transpose (gather, no atomics), with the same fused epilogues as the 2D projector.
//
// Each ray (view, iu, iv) is marched over the planes of its dominant axis (x or y, fixed
// per detector column); on plane l its point has transverse index ft = P0 + P1 l and z index
// fz = cz + (iv - cv)(Q0 + Q1 l), both carried in 64-bit fixed point, bilinearly
// interpolated; each plane adds voxel * |d| / |d_a|.  Rays marched over x planes read the
// volume transposed in (x, y), so that for either axis the 32 lanes of a warp (adjacent
// detector columns) read along a contiguous row.  The adjoint visits, for every column of
// voxels and view, the detector columns whose rays cross the voxels' dominant plane within
// one voxel (found by projecting the two plane points at +-1 voxel onto the detector) and
// walks their detector rows in the forward's own fixed point, so that every row adds the
// identical bilinear weights to the two voxels its ray interpolates.
#include "vrps_internal.h"

namespace vrps {
namespace {


// Plane indices l in [0, nl) where intercept + slope (l - lc) lies in (-1, n); widened by 1.
__device__ __forceinline__ void clip_range(float intercept, float slope, float lc, int n, int nl, int& lo,
                                           int& hi) {
  if (slope != 0.f) {
    float a = lc + (-1.f - intercept) / slope;
    float b = lc + ((float)n - intercept) / slope;
    if (a > b) {
      const float t = a;
      a = b;
      b = t;
    }
    a = fminf(fmaxf(a, -2.f), (float)nl + 1.f);
    b = fminf(fmaxf(b, -2.f), (float)nl + 1.f);
    lo = max(lo, (int)floorf(a) - 1);
    hi = min(hi, (int)ceilf(b) + 1);
  } else if (!(intercept > -1.f && intercept < (float)n)) {
    hi = -1;
  }
}

constexpr float TWO_M32 = 2.3283064365386963e-10f;   // 2^-32

// Ray length factor voxel |d| / |d_a| = voxel sqrt(1 + P1^2 + (k R)^2) with explicit roundings
// (the same bits in every kernel that inlines it).
__device__ __forceinline__ float ray_factor(float vox, float p1, float kr) {
  return __fmul_rn(vox, sqrtf(fmaf(kr, kr, fmaf(p1, p1, 1.f))));
}

template <int MODE>
__device__ __forceinline__ void fwd3d_item(const Fwd3DParams& P, int bx, int row, int bz) {
  const int iu = bx * 32 + threadIdx.x;
  const int iv = bz * 8 + threadIdx.y;
  if (iu >= P.nu || iv >= P.nv) return;
  const int view = P.ids[row];
  const RayInfo3D ri = P.rays[(size_t)view * P.nu + iu];
  const float k = (float)iv - P.cv;
  const long long k2 = 2LL * iv - (P.nv - 1);   // 2 (iv - cv), exact
  const bool ax0 = ri.axis == 0;
  const int nl = ax0 ? P.nx : P.ny;
  const int nt = ax0 ? P.ny : P.nx;
  const float* vol = ax0 ? P.xT : P.x;          // transverse index contiguous in both cases
  const int64_t sl = nt;
  const int64_t sz = (int64_t)P.nx * P.ny;
  int lo = 0, hi = nl - 1;
  const float q0 = __ll2float_rn(ri.QF0) * TWO_M32, q1 = __ll2float_rn(ri.QF1) * TWO_M32;
  clip_range(__ll2float_rn(ri.PF0) * TWO_M32, ri.P1, 0.f, nt, nl, lo, hi);
  clip_range(fmaf(k, q0, P.cz), k * q1, 0.f, P.nz, nl, lo, hi);
  float acc = 0.f;
  // transverse position in units of 2^-32, z position in units of 2^-33
  long long ft = ri.PF0 + ri.PF1 * lo;
  const long long zstep = k2 * ri.QF1;
  long long fz = ((long long)(P.nz - 1) << 32) + k2 * ri.QF0 + zstep * lo;
  for (int l = lo; l <= hi; ++l, ft += ri.PF1, fz += zstep) {
    const int it = (int)(ft >> 32), iz = (int)(fz >> 33);
    const float f = (float)(unsigned)ft * TWO_M32;
    const float gz = (float)(unsigned)(fz >> 1) * TWO_M32;
    const bool t0 = it >= 0 && it < nt, t1 = it + 1 >= 0 && it + 1 < nt;
    const bool z0 = iz >= 0 && iz < P.nz, z1 = iz + 1 >= 0 && iz + 1 < P.nz;
    const int64_t b = (int64_t)l * sl + (int64_t)it + (int64_t)iz * sz;
    const float v00 = (t0 && z0) ? __ldg(vol + b) : 0.f;
    const float v10 = (t1 && z0) ? __ldg(vol + b + 1) : 0.f;
    const float v01 = (t0 && z1) ? __ldg(vol + b + sz) : 0.f;
    const float v11 = (t1 && z1) ? __ldg(vol + b + 1 + sz) : 0.f;
    const float lo_z = fmaf(f, v10 - v00, v00);
    const float hi_z = fmaf(f, v11 - v01, v01);
    acc += fmaf(gz, hi_z - lo_z, lo_z);
  }
  const float wgt = ray_factor(P.vox, ri.P1, k * ri.R);
  const float r = acc * wgt;
  const float ys = P.o.prescale ? wgt : 1.f;   // ray factor carried into the adjoint's input
  const size_t idx = (size_t)row * P.nu * P.nv + (size_t)iv * P.nu + iu;
  const FwdOut& o = P.o;
  if (MODE == FWD_PLAIN) {
    o.y[idx] = r * ys;
  } else if (MODE == FWD_RESID) {
    o.y[idx] = (r - ld_store(o, o.b, idx)) * ys;
  } else if (MODE == FWD_SVRG) {
    o.y[idx] = (r - ld_store(o, o.tab, idx)) * ys;
  } else if (MODE == FWD_SAGA) {
    // stored (rounded) table values on both sides, as in the 2D epilogue
    const float res = r - ld_store(o, o.b, idx);
    const float old = ld_store(o, o.tab, idx);
    o.y[idx] = (st_store(o, o.tab, idx, res) - old) * ys;
  } else {
    o.y[idx] = (st_store(o, o.tab, idx, r) - ld_store(o, o.b, idx)) * ys;
  }
}

// grid (column tiles, views, row bands): CTAs issued together cover every view of the same
// detector rows, whose rays cross the same z slab of the volume (kept in L2)
template <int MODE>
__global__ void __launch_bounds__(256) fwd3d_kernel(Fwd3DParams P) {
  fwd3d_item<MODE>(P, blockIdx.x, blockIdx.y, blockIdx.z);
}


// Fractional detector column of the ray from the source through the point (qx, qy, *).
__device__ __forceinline__ float column_of(const ViewInfo3D& vi, float qx, float qy) {
  const float ax = qx - vi.sx, ay = qy - vi.sy;
  const float num = fmaf(ax, vi.eux, ay * vi.euy);
  const float den = -fmaf(ax, vi.esx, ay * vi.esy);
  return fmaf(vi.sdd * num / den, vi.inv_du, vi.cu);
}

constexpr int ADJ3_ZC = 16;   // voxels of one z column handled by a thread (default; 32 tunable)

// r[row][iv][iu] <- r times the ray length factor voxel |d|/|d_a| (input of adj3d_kernel)
__global__ void __launch_bounds__(256) prescale3d_kernel(const float* __restrict__ r, float* __restrict__ out,
                                                         const RayInfo3D* rays, const int* ids, int nu, int nv,
                                                         float cv, float vox) {
  const int iu = blockIdx.x * 32 + threadIdx.x;
  const int iv = blockIdx.y * 8 + threadIdx.y;
  const int row = blockIdx.z;
  if (iu >= nu || iv >= nv) return;
  const RayInfo3D ri = rays[(size_t)ids[row] * nu + iu];
  const size_t idx = (size_t)row * nu * nv + (size_t)iv * nu + iu;
  out[idx] = r[idx] * ray_factor(vox, ri.P1, ((float)iv - cv) * ri.R);
}

// Voxel-driven transpose of the 3D Joseph projector.  A thread owns ZC voxels of one z
// column.  For each view and each dominant axis it projects the voxel's plane points at
// +-1 voxel onto the detector to bound the candidate columns iu; for every column whose ray
// meets the voxel's plane within one voxel (transverse weight wt, the same for the whole z
// column) it walks the detector rows whose ray crosses the column's z range.  On the
// column's plane the ray of row iv has z position fz(iv) = base + iv * 2 qf in the forward's
// 2^-33 fixed point, so every row reproduces the forward's tap exactly: z index fz >> 33
// gets weight 1 - g and the next voxel g, g the low 32 bits of fz >> 1.  The row range is
// found from a float estimate corrected by exact integer comparisons; rows add into the
// thread's own shared-memory slots (index = z index - z0 + 1, two spill slots).  r arrives
// pre-multiplied by the ray length factors.
constexpr float TWO_M33 = 1.16415321826934814453125e-10f;   // 2^-33

// First row in [0, nv] whose fixed-point z position base + iv * step reaches t (step > 0).
__device__ __forceinline__ int first_row(long long base, long long step, long long t, float iq, int nv) {
  float est = ceilf(__ll2float_rn(t - base) * TWO_M33 * iq);
  est = fminf(fmaxf(est, 0.f), (float)nv);
  int iv = (int)est;
  const long long f = base + (long long)iv * step;
  if (iv < nv && f < t) ++iv;
  else if (iv > 0 && f - step >= t) --iv;
  return iv;
}

// acc: shared [ZC + 2][256] (slot-major, one column per thread).  A voxel's contributions
// arrive in the same order (views, columns, rows ascending) whatever ZC is, so the result
// does not depend on the chunk length.
template <int ZC>
__device__ __forceinline__ void adj3d_item(const Adj3DParams& P, float* __restrict__ acc, int bx, int by, int bz) {
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int gx = bx * 32 + threadIdx.x;
  const int gy = by * 8 + threadIdx.y;
  const int z0 = bz * ZC;
  if (gx >= P.nx || gy >= P.ny) return;
  float* const a0 = acc + tid;
#pragma unroll
  for (int q = 0; q < ZC + 2; ++q) a0[q * 256] = 0.f;
  const float X = ((float)gx - P.cx) * P.vox, Y = ((float)gy - P.cy) * P.vox;
  const float lim = (float)P.nu + 2.f;
  const long long lo_t = (long long)(z0 - 1) << 33;         // rows with z index >= z0 - 1 ...
  const long long hi_t = (long long)(z0 + ZC) << 33;   // ... and < z0 + ZC
  const long long zc32 = (long long)(P.nz - 1) << 32;
  for (int q = 0; q < P.rows; ++q) {
    const int view = P.ids[q];
    const ViewInfo3D vi = P.views[view];
    const RayInfo3D* vr = P.rays + (size_t)view * P.nu;
    const float* rr = P.r + (size_t)q * P.nu * P.nv;
    for (int axis = 0; axis < 2; ++axis) {
      if (axis == 0 ? !vi.has_x : !vi.has_y) continue;
      const int tt = axis == 0 ? gy : gx;
      const long long gl = axis == 0 ? gx : gy;
      const long long tt32 = (long long)tt << 32;
      const float c0 = fminf(fmaxf(axis == 0 ? column_of(vi, X, Y - P.vox) : column_of(vi, X - P.vox, Y), -2.f), lim);
      const float c1 = fminf(fmaxf(axis == 0 ? column_of(vi, X, Y + P.vox) : column_of(vi, X + P.vox, Y), -2.f), lim);
      const int u_lo = max(0, (int)floorf(fminf(c0, c1)) - 1);
      const int u_hi = min(P.nu - 1, (int)ceilf(fmaxf(c0, c1)) + 1);
      for (int iu = u_lo; iu <= u_hi; ++iu) {
        const RayInfo3D ri = vr[iu];
        if (ri.axis != axis) continue;
        const long long dt = ri.PF0 + ri.PF1 * gl - tt32;   // (transverse - tt) 2^32, exact
        if (dt <= -(1LL << 32) || dt >= (1LL << 32)) continue;
        const float wt = 1.f - fabsf(__ll2float_rn(dt) * TWO_M32);
        const long long qf = ri.QF0 + ri.QF1 * gl;            // z voxels per row, 2^-32 (> 0)
        const long long step = 2 * qf;
        const long long base = zc32 - (long long)(P.nv - 1) * qf;
        const float iq = 1.f / (__ll2float_rn(qf) * TWO_M32);
        const int iv0 = first_row(base, step, lo_t, iq, P.nv);
        const int iv1 = first_row(base, step, hi_t, iq, P.nv);
        long long f = base + (long long)iv0 * step;
        const float* rp = rr + (size_t)iv0 * P.nu + iu;
#pragma unroll 2
        for (int iv = iv0; iv < iv1; ++iv, f += step, rp += P.nu) {
          const float wr = wt * __ldg(rp);
          const int sl = (int)(f >> 33) - z0 + 1;                  // 0 .. ZC + 1
          const float g = (float)(unsigned)(f >> 1) * TWO_M32;
          const float hi = g * wr;
          a0[sl * 256] += wr - hi;
          a0[(sl + 1) * 256] += hi;
        }
      }
    }
  }
  const UpdateArgs& u = P.u;
#pragma unroll
  for (int z = 0; z < ZC; ++z) {
    const int gz = z0 + z;
    if (gz >= P.nz) break;
    const size_t p = ((size_t)gz * P.ny + gy) * P.nx + gx;
    const float g = a0[(z + 1) * 256];
    if (!u.enabled) {
      u.out[p] = g;
      continue;
    }
    update_pixel(u, p, g);
  }
}

template <int ZC>
__global__ void __launch_bounds__(256) adj3d_kernel(Adj3DParams P) {
  __shared__ float acc[(ZC + 2) * 256];
  adj3d_item<ZC>(P, acc, blockIdx.x, blockIdx.y, blockIdx.z);
}

}  // namespace

int fwd3d_setup(const vrps_geom* g, const float* x, const float* xT, const int* ids, int rows, FwdOut o,
                Fwd3DParams* out) {
  Fwd3DParams& P = *out;
  (void)rows;
  P.x = x;
  P.xT = xT;
  P.rays = g->ray3d;
  P.ids = ids;
  P.nx = g->nx;
  P.ny = g->ny;
  P.nz = g->nz;
  P.nu = g->nu;
  P.nv = g->nv;
  P.cx = 0.5f * (float)(g->nx - 1);
  P.cy = 0.5f * (float)(g->ny - 1);
  P.cz = 0.5f * (float)(g->nz - 1);
  P.cv = 0.5f * (float)(g->nv - 1);
  P.vox = (float)g->pixel;
  P.o = o;
  return VRPS_OK;
}

int fwd3d(const vrps_geom* g, const float* x, const float* xT, const int* ids, int rows, int mode, FwdOut o,
          cudaStream_t s) {
  if (rows <= 0) return VRPS_OK;
  Fwd3DParams P;
  VRPS_TRY(fwd3d_setup(g, x, xT, ids, rows, o, &P));
  dim3 grid((g->nu + 31) / 32, rows, (g->nv + 7) / 8), block(32, 8);
  const double fb = 4.0 * g->n + fwd_mode_bytes(mode, (size_t)rows * g->nu * g->nv, o.store);
  switch (mode) {
    case FWD_PLAIN: { LaunchScope _ls("fwd3d_kernel", s, fb); VRPS_CUDA(launch_kernel(fwd3d_kernel<FWD_PLAIN>, dim3(grid), dim3(block), (size_t)(0), s, P)); } break;
    case FWD_RESID: { LaunchScope _ls("fwd3d_kernel", s, fb); VRPS_CUDA(launch_kernel(fwd3d_kernel<FWD_RESID>, dim3(grid), dim3(block), (size_t)(0), s, P)); } break;
    case FWD_SVRG: { LaunchScope _ls("fwd3d_kernel", s, fb); VRPS_CUDA(launch_kernel(fwd3d_kernel<FWD_SVRG>, dim3(grid), dim3(block), (size_t)(0), s, P)); } break;
    case FWD_SAGA: { LaunchScope _ls("fwd3d_kernel", s, fb); VRPS_CUDA(launch_kernel(fwd3d_kernel<FWD_SAGA>, dim3(grid), dim3(block), (size_t)(0), s, P)); } break;
    case FWD_SNAP: { LaunchScope _ls("fwd3d_kernel", s, fb); VRPS_CUDA(launch_kernel(fwd3d_kernel<FWD_SNAP>, dim3(grid), dim3(block), (size_t)(0), s, P)); } break;
    default: return fail(VRPS_ERR_INVALID_ARG, "bad forward mode %d", mode);
  }
  VRPS_LAUNCHED("fwd3d");
  return VRPS_OK;
}

int adj3d_setup(const vrps_geom* g, const float* r, const int* ids, int rows, const UpdateArgs& u,
                Adj3DParams* out) {
  Adj3DParams& P = *out;
  P.rays = g->ray3d;
  P.views = g->view3d;
  P.ids = ids;
  P.rows = rows;
  P.nx = g->nx;
  P.ny = g->ny;
  P.nz = g->nz;
  P.nu = g->nu;
  P.nv = g->nv;
  P.cx = 0.5f * (float)(g->nx - 1);
  P.cy = 0.5f * (float)(g->ny - 1);
  P.cz = 0.5f * (float)(g->nz - 1);
  P.cv = 0.5f * (float)(g->nv - 1);
  P.vox = (float)g->pixel;
  P.u = u;
  P.r = r;
  return VRPS_OK;
}

int adj3d(const vrps_geom* g, const float* r, const int* ids, int rows, const UpdateArgs& u, cudaStream_t s) {
  Adj3DParams P;
  VRPS_TRY(adj3d_setup(g, r, ids, rows, u, &P));
  if (!u.prescaled && rows > 0) {
    vrps_geom* gm = const_cast<vrps_geom*>(g);
    VRPS_TRY(ensure(&gm->ws.sino2, (size_t)g->m));
    dim3 pg((g->nu + 31) / 32, (g->nv + 7) / 8, rows), pb(32, 8);
    {
      LaunchScope _ls("prescale3d_kernel", s, 8.0 * rows * g->nu * g->nv);
      VRPS_CUDA(launch_kernel(prescale3d_kernel, pg, pb, (size_t)0, s, r, gm->ws.sino2, (const RayInfo3D*)g->ray3d,
                              ids, g->nu, g->nv, P.cv, P.vox));
    }
    VRPS_LAUNCHED("prescale3d");
    P.r = gm->ws.sino2;
  }
  const int zc = g->tune_adj3_zc == 32 ? 32 : ADJ3_ZC;
  dim3 grid((g->nx + 31) / 32, (g->ny + 7) / 8, (g->nz + zc - 1) / zc), block(32, 8);
  LaunchScope _ls("adj3d_kernel", s, 4.0 * rows * g->nu * g->nv + update_bytes(u, (size_t)g->n));
  if (zc == 32) VRPS_CUDA(launch_kernel(adj3d_kernel<32>, grid, block, (size_t)0, s, P));
  else VRPS_CUDA(launch_kernel(adj3d_kernel<ADJ3_ZC>, grid, block, (size_t)0, s, P));
  VRPS_LAUNCHED("adj3d");
  return VRPS_OK;
}

}  // namespace vrps

// ------------------------------------------------------------------ batched 3D launches
namespace vrps {
namespace {

__device__ __forceinline__ int b3_job(const int* pre, int n, int item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void b3_prefix(int* dst, const int* src, int n) {
  for (int i = threadIdx.y * blockDim.x + threadIdx.x; i <= n; i += blockDim.x * blockDim.y) dst[i] = src[i];
  __syncthreads();
}

__device__ __forceinline__ int b3_next(unsigned* counter, int* s_item) {
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) *s_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  return *s_item;
}

__global__ void __launch_bounds__(256) tr3_batched_kernel(char* __restrict__ slot) {
  __shared__ float t[32][33];
  __shared__ int pre[BATCH_MAX_JOBS + 1];
  __shared__ int s_item;
  const TickHeader3& H = *reinterpret_cast<const TickHeader3*>(slot);
  const int n = H.n_jobs;
  if (n <= 0) return;
  unsigned* counter = reinterpret_cast<TickHeader3*>(slot)->cnt + 0;
  const BatchTr3* jobs = reinterpret_cast<const BatchTr3*>(slot + H.off_tr);
  b3_prefix(pre, reinterpret_cast<const int*>(slot + H.off_ptr), n);
  const int total = pre[n];
  for (int item = b3_next(counter, &s_item); item < total; item = b3_next(counter, &s_item)) {
    const int j = b3_job(pre, n, item);
    const BatchTr3& J = jobs[j];
    const int local = item - pre[j];
    const int per = J.tiles_x * J.tiles_y;
    const int z = local / per, tl = local - z * per;
    const int bx = (tl % J.tiles_x) * 32, by = (tl / J.tiles_x) * 32;
    const float* in = J.in + (size_t)z * J.nx * J.ny;
    float* out = J.out + (size_t)z * J.nx * J.ny;
    for (int k = threadIdx.y; k < 32; k += 8) {
      const int x = bx + threadIdx.x, y = by + k;
      if (x < J.nx && y < J.ny) t[k][threadIdx.x] = in[(size_t)y * J.nx + x];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
      const int y = by + threadIdx.x, x = bx + k;   // out[x][y]
      if (x < J.nx && y < J.ny) out[(size_t)x * J.ny + y] = t[threadIdx.x][k];
    }
  }
}

__global__ void __launch_bounds__(256) fwd3d_batched_kernel(char* __restrict__ slot) {
  __shared__ int pre[BATCH_MAX_JOBS + 1];
  __shared__ int s_item;
  const TickHeader3& H = *reinterpret_cast<const TickHeader3*>(slot);
  const int n = H.n_jobs;
  if (n <= 0) return;
  unsigned* counter = reinterpret_cast<TickHeader3*>(slot)->cnt + 1;
  const BatchFwd3* jobs = reinterpret_cast<const BatchFwd3*>(slot + H.off_fwd);
  b3_prefix(pre, reinterpret_cast<const int*>(slot + H.off_pfwd), n);
  const int total = pre[n];
  for (int item = b3_next(counter, &s_item); item < total; item = b3_next(counter, &s_item)) {
    const int j = b3_job(pre, n, item);
    const BatchFwd3& J = jobs[j];
    const int local = item - pre[j];
    // same order as the single launch: column tiles fastest, then views, then row bands
    const int bx = local % J.tiles_u, rest = local / J.tiles_u;
    const int row = rest % J.rows, bz = rest / J.rows;
    switch (J.mode) {
      case FWD_PLAIN: fwd3d_item<FWD_PLAIN>(J.P, bx, row, bz); break;
      case FWD_RESID: fwd3d_item<FWD_RESID>(J.P, bx, row, bz); break;
      case FWD_SVRG: fwd3d_item<FWD_SVRG>(J.P, bx, row, bz); break;
      case FWD_SAGA: fwd3d_item<FWD_SAGA>(J.P, bx, row, bz); break;
      default: fwd3d_item<FWD_SNAP>(J.P, bx, row, bz); break;
    }
  }
}

__global__ void __launch_bounds__(256, 4) adj3d_batched_kernel(char* __restrict__ slot) {
  __shared__ float acc[(ADJ3_ZC + 2) * 256];   // batched jobs keep the default chunk (same results)
  __shared__ int pre[BATCH_MAX_JOBS + 1];
  __shared__ int s_item;
  const TickHeader3& H = *reinterpret_cast<const TickHeader3*>(slot);
  const int n = H.n_jobs;
  if (n <= 0) return;
  unsigned* counter = reinterpret_cast<TickHeader3*>(slot)->cnt + 2;
  const BatchAdj3* jobs = reinterpret_cast<const BatchAdj3*>(slot + H.off_adj);
  b3_prefix(pre, reinterpret_cast<const int*>(slot + H.off_padj), n);
  const int total = pre[n];
  for (int item = b3_next(counter, &s_item); item < total; item = b3_next(counter, &s_item)) {
    const int j = b3_job(pre, n, item);
    const BatchAdj3& J = jobs[j];
    const int local = item - pre[j];
    const int per = J.tiles_x * J.tiles_y;
    const int bz = local / per, tl = local - bz * per;
    const int bx = tl % J.tiles_x, by = tl / J.tiles_x;
    adj3d_item<ADJ3_ZC>(J.P, acc, bx, by, bz);
  }
}

}  // namespace

int tr3_batched(char* slot, int grid, cudaStream_t s) {
  LaunchScope _ls("tr3_batched", s);
  VRPS_CUDA(launch_kernel(tr3_batched_kernel, dim3(grid), dim3(32, 8), (size_t)0, s, slot));
  return VRPS_OK;
}

int fwd3d_batched(char* slot, int grid, cudaStream_t s) {
  LaunchScope _ls("fwd3d_batched", s);
  VRPS_CUDA(launch_kernel(fwd3d_batched_kernel, dim3(grid), dim3(32, 8), (size_t)0, s, slot));
  return VRPS_OK;
}

int adj3d_batched(char* slot, int grid, cudaStream_t s) {
  LaunchScope _ls("adj3d_batched", s);
  VRPS_CUDA(launch_kernel(adj3d_batched_kernel, dim3(grid), dim3(32, 8), (size_t)0, s, slot));
  return VRPS_OK;
}

int tr3_batch_entry(const float* in, float* out, int nx, int ny, int nz, BatchTr3* e, int* items) {
  e->in = in;
  e->out = out;
  e->nx = nx;
  e->ny = ny;
  e->nz = nz;
  e->tiles_x = (nx + 31) / 32;
  e->tiles_y = (ny + 31) / 32;
  *items = e->tiles_x * e->tiles_y * nz;
  return VRPS_OK;
}

int fwd3d_batch_entry(const vrps_geom* g, const float* x, const float* xT, const int* ids, int rows, int mode,
                      FwdOut o, BatchFwd3* e, int* items) {
  if (mode < FWD_PLAIN || mode > FWD_SNAP) return fail(VRPS_ERR_INVALID_ARG, "bad forward mode %d", mode);
  VRPS_TRY(fwd3d_setup(g, x, xT, ids, rows, o, &e->P));
  e->mode = mode;
  e->tiles_u = (g->nu + 31) / 32;
  e->rows = rows;
  e->bands_v = (g->nv + 7) / 8;
  *items = rows > 0 ? e->tiles_u * rows * e->bands_v : 0;
  return VRPS_OK;
}

int adj3d_batch_entry(const vrps_geom* g, const float* r, const int* ids, int rows, const UpdateArgs& u,
                      BatchAdj3* e, int* items) {
  if (!u.prescaled) return fail(VRPS_ERR_UNSUPPORTED, "the batched 3D adjoint reads prescaled residuals");
  VRPS_TRY(adj3d_setup(g, r, ids, rows, u, &e->P));
  e->tiles_x = (g->nx + 31) / 32;
  e->tiles_y = (g->ny + 7) / 8;
  e->chunks = (g->nz + ADJ3_ZC - 1) / ADJ3_ZC;
  *items = e->tiles_x * e->tiles_y * e->chunks;
  return VRPS_OK;
}

int batched_grid_3d_proj(int which, int* grid) {
  int dev = 0, sms = 0, per = 0;
  VRPS_CUDA(cudaGetDevice(&dev));
  VRPS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (which == 0) VRPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tr3_batched_kernel, 256, 0));
  else if (which == 1) VRPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fwd3d_batched_kernel, 256, 0));
  else VRPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, adj3d_batched_kernel, 256, 0));
  *grid = (per < 1 ? 1 : per) * sms;
  return VRPS_OK;
}

}  // namespace vrps
