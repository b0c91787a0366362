// C-ABI entry points: errors, geometry handles, operators, prox, power iteration, objective.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include "vrps_internal.h"

namespace vrps {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  return e == cudaErrorMemoryAllocation ? VRPS_ERR_OUT_OF_MEMORY : VRPS_ERR_CUDA;
}

int launch_fail(cudaError_t e, const char* name, const void* kern, dim3 grid, dim3 block, size_t smem) {
  cudaGetLastError();   // a refused launch leaves no sticky error; clear the record of it
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, kern);
  set_error("CUDA error %d (%s) launching %s: grid %u x %u, block %u x %u, %zu B dynamic shared memory "
            "(kernel: %zu B static, at most %d B dynamic, %d registers)",
            (int)e, cudaGetErrorString(e), name, grid.x, grid.y, block.x, block.y, smem, fa.sharedSizeBytes,
            fa.maxDynamicSharedSizeBytes, fa.numRegs);
  return e == cudaErrorMemoryAllocation ? VRPS_ERR_OUT_OF_MEMORY : VRPS_ERR_CUDA;
}

int smem_opt_in(const void* kern, size_t bytes) {
  // without the opt-in a kernel may use 48 KB of shared memory minus its static shared memory,
  // so sizes just under 48 KB can need it too: every nonzero size goes through the cache
  if (bytes == 0) return VRPS_OK;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  VRPS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& have = done[{kern, dev}];
  if (have >= bytes) return VRPS_OK;
  VRPS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  have = bytes;
  return VRPS_OK;
}

int ensure(float** p, size_t count) {
  if (*p) return VRPS_OK;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(float));
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMalloc(workspace)");
  }
  return VRPS_OK;
}

int ensure_d(double** p, size_t count) {
  if (*p) return VRPS_OK;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(double));
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMalloc(workspace)");
  }
  return VRPS_OK;
}

// Staggered subsets (Fig. 1 caption): subset i = {i, i+N, i+2N, ...}; subset-major order
// concatenates the subsets, so subset i occupies rows off[i] .. off[i+1]-1.
// Subset-major angle order: subset i holds angles i, i + N, i + 2N, ... (off: subset starts).
static std::vector<int> subset_order(int n_angles, int N, std::vector<int>* off) {
  std::vector<int> order;
  order.reserve(n_angles);
  if (off) off->assign(N + 1, 0);
  for (int i = 0; i < N; ++i) {
    if (off) (*off)[i] = (int)order.size();
    for (int a = i; a < n_angles; a += N) order.push_back(a);
  }
  if (off) (*off)[N] = (int)order.size();
  return order;
}

int build_order_angles(const vrps_geom* g, int N, AngleInfo2D** dev) {
  if (*dev) {
    cudaFree(*dev);
    *dev = nullptr;
  }
  if (g->dims != 2 || g->ang2d_host.empty()) return VRPS_OK;
  const std::vector<int> order = subset_order(g->n_angles, N, nullptr);
  std::vector<AngleInfo2D> rows(order.size());
  for (size_t r = 0; r < order.size(); ++r) rows[r] = g->ang2d_host[order[r]];
  VRPS_CUDA(cudaMalloc((void**)dev, sizeof(AngleInfo2D) * rows.size()));
  VRPS_CUDA(cudaMemcpy(*dev, rows.data(), sizeof(AngleInfo2D) * rows.size(), cudaMemcpyHostToDevice));
  return VRPS_OK;
}

const AngleInfo2D* angle_rows(const vrps_geom* g, const int* ids) {
  const uintptr_t p = (uintptr_t)ids;
  const size_t span = sizeof(int) * (size_t)g->n_angles;
  auto within = [&](const int* base) { return base && p >= (uintptr_t)base && p < (uintptr_t)base + span; };
  if (within(g->order_natural) && g->ang2d) return g->ang2d + (ids - g->order_natural);
  if (within(g->order_subset) && g->ang2d_sub) return g->ang2d_sub + (ids - g->order_subset);
  const Workspace& w = g->ws;
  if (within(w.order_dev) && w.ang_order_dev) return w.ang_order_dev + (ids - w.order_dev);
  return nullptr;
}

int build_order(int n_angles, int N, int** dev, std::vector<int>* off) {
  const std::vector<int> order = subset_order(n_angles, N, off);
  if (*dev) {
    cudaFree(*dev);
    *dev = nullptr;
  }
  VRPS_CUDA(cudaMalloc((void**)dev, sizeof(int) * n_angles));
  VRPS_CUDA(cudaMemcpy(*dev, order.data(), sizeof(int) * n_angles, cudaMemcpyHostToDevice));
  return VRPS_OK;
}

int subset_rows(const vrps_geom* g, int subset, const int** ids, int* rows) {
  if (subset == -1) {
    *ids = g->order_natural;
    *rows = g->n_angles;
    return VRPS_OK;
  }
  if (subset < 0 || subset >= g->n_subsets)
    return fail(VRPS_ERR_INVALID_ARG, "subset %d outside [-1, %d)", subset, g->n_subsets);
  *ids = g->order_subset + g->subset_off[subset];
  *rows = g->subset_off[subset + 1] - g->subset_off[subset];
  return VRPS_OK;
}

int proj_forward(const vrps_geom* g, const float* x, const float* xT, const int* ids, int rows,
                 int mode, FwdOut o, cudaStream_t s) {
  if (!xT) {
    vrps_geom* gm = const_cast<vrps_geom*>(g);
    VRPS_TRY(ensure(&gm->ws.xT, (size_t)g->n));
    VRPS_TRY(transpose2d(x, gm->ws.xT, g->ny, g->nx, s, g->dims == 3 ? g->nz : 1));
    xT = gm->ws.xT;
  }
  if (g->dims == 3) return fwd3d(g, x, xT, ids, rows, mode, o, s);
  return fwd2d(g, x, xT, ids, rows, mode, o, s);
}

int proj_adjoint(const vrps_geom* g, const float* r, const int* ids, int rows, const UpdateArgs& u,
                 cudaStream_t s) {
  if (g->dims == 3) return adj3d(g, r, ids, rows, u, s);
  return adj2d(g, r, ids, rows, u, s);
}

static int check_geom(const vrps_geom* g) {
  if (!g) return fail(VRPS_ERR_INVALID_ARG, "geometry handle is NULL");
  int dev = -1;
  VRPS_CUDA(cudaGetDevice(&dev));
  if (dev != g->device)
    return fail(VRPS_ERR_INVALID_ARG, "geometry was created on device %d, current device is %d",
                g->device, dev);
  return VRPS_OK;
}

static void free_ws(Workspace& w) {
  float** fl[] = {&w.xT, &w.dual_cold, &w.dual_s1, &w.dual_s2, &w.dual_s3, &w.dual_s4, &w.sino, &w.sino2, &w.img, &w.img2,
                  &w.x, &w.xf, &w.xfT, &w.h, &w.xhat, &w.v, &w.gbar, &w.xprox, &w.dual,
                  &w.b_perm, &w.tab, &w.res, &w.b16, &w.tab16};
  for (float** p : fl) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  if (w.partials) cudaFree(w.partials);
  if (w.fwd_part) cudaFree(w.fwd_part);
  if (w.fwd_count) cudaFree(w.fwd_count);
  if (w.dev_error) cudaFree(w.dev_error);
  if (w.fgp_bar) cudaFree(w.fgp_bar);
  w.fgp_bar = nullptr;
  if (w.adj_part) cudaFree(w.adj_part);
  if (w.adj_count) cudaFree(w.adj_count);
  if (w.scalars) cudaFree(w.scalars);
  if (w.sched_dev) cudaFree(w.sched_dev);
  if (w.sched_host) cudaFreeHost(w.sched_host);
  if (w.order_dev) cudaFree(w.order_dev);
  if (w.ang_order_dev) cudaFree(w.ang_order_dev);
  w.ang_order_dev = nullptr;
  w = Workspace();
}

static void free_geom(vrps_geom* g) {
  if (!g) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(g->device);
  cudaDeviceSynchronize();
  if (g->ang2d) cudaFree(g->ang2d);
  if (g->ang2d_sub) cudaFree(g->ang2d_sub);
  if (g->ray3d) cudaFree(g->ray3d);
  if (g->view3d) cudaFree(g->view3d);
  if (g->order_natural) cudaFree(g->order_natural);
  if (g->order_subset) cudaFree(g->order_subset);
  free_ws(g->ws);
  if (prev >= 0) cudaSetDevice(prev);
  delete g;
}

static int finish_common(vrps_geom* g) {
  VRPS_CUDA(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device));
  std::vector<int> nat(g->n_angles);
  for (int a = 0; a < g->n_angles; ++a) nat[a] = a;
  VRPS_CUDA(cudaMalloc((void**)&g->order_natural, sizeof(int) * g->n_angles));
  VRPS_CUDA(cudaMemcpy(g->order_natural, nat.data(), sizeof(int) * g->n_angles, cudaMemcpyHostToDevice));
  VRPS_TRY(build_order(g->n_angles, g->n_subsets, &g->order_subset, &g->subset_off));
  VRPS_TRY(ensure_d(&g->ws.partials, 1024));
  VRPS_TRY(ensure_d(&g->ws.scalars, 16));
  return VRPS_OK;
}

// 2D tables, float64 on the host (dominant-axis test included, so that it is taken in the
// same precision as by any float64 reference).
static int build_par2d(vrps_geom* g) {
  const double pix = g->pixel, ds = g->bin_spacing;
  std::vector<AngleInfo2D> tab(g->n_angles);
  double span_max = 0.0, hw_max = 0.0;
  for (int a = 0; a < g->n_angles; ++a) {
    const double th = g->angles[a];
    const double c = std::cos(th), s = std::sin(th);
    const bool rows = std::fabs(c) >= std::fabs(s);
    const double m = rows ? std::fabs(c) : std::fabs(s);
    AngleInfo2D& t = tab[a];
    if (rows) {
      t.A1 = (float)(ds / (pix * c));
      t.A2 = (float)(-s / c);
    } else {
      t.A1 = (float)(ds / (pix * s));
      t.A2 = (float)(-c / s);
    }
    t.T = rows ? 0 : 1;
    {
      const double a2 = rows ? -s / c : -c / s;
      t.inv_A2 = a2 != 0.0 ? (float)(1.0 / a2) : 0.f;
      t.pad[0] = t.pad[1] = t.pad[2] = 0;
    }
    const double two31 = 2147483648.0;
    t.A1H = std::llround((rows ? ds / (pix * c) : ds / (pix * s)) * two31);
    t.A2H = std::llround((rows ? -s / c : -c / s) * two31);
    t.BxH = std::llround(pix * c / ds * two31);
    t.ByH = std::llround(pix * s / ds * two31);
    t.wgt = (float)(pix / m);
    t.Bx = (float)(pix * c / ds);
    t.By = (float)(pix * s / ds);
    t.hw = (float)(pix * m / ds);
    t.inv_hw = (float)(ds / (pix * m));
    span_max = std::fmax(span_max, (ADJ2D_TILE_X - 1) * std::fabs(pix * c / ds) +
                                       (ADJ2D_TILE_Y - 1) * std::fabs(pix * s / ds));
    hw_max = std::fmax(hw_max, pix * m / ds);
  }
  // hw <= 1: at most two bins lie strictly within hw of a pixel's projected centre
  g->adj_nc = hw_max <= 1.0 ? 2 : (int)std::ceil(2.0 * hw_max) + 1;
  g->adj_fp = (int)std::ceil(span_max) + g->adj_nc + 4;
  VRPS_CUDA(cudaMalloc((void**)&g->ang2d, sizeof(AngleInfo2D) * g->n_angles));
  VRPS_CUDA(cudaMemcpy(g->ang2d, tab.data(), sizeof(AngleInfo2D) * g->n_angles, cudaMemcpyHostToDevice));
  g->ang2d_host = tab;
  // the rows of a subset launch read their angle constants directly, without the id hop
  VRPS_TRY(build_order_angles(g, g->n_subsets, &g->ang2d_sub));
  return VRPS_OK;
}

// 3D tables: per (view, detector column) ray constants and per view adjoint constants.
// Rays are marched over x planes when |d_x| >= |d_y| (d depends only on the column), over
// y planes otherwise; a ray whose |d_z| is not below both is rejected as unsupported.
static int build_cone3d(vrps_geom* g) {
  const double vox = g->pixel;
  const double cx = 0.5 * (g->nx - 1), cy = 0.5 * (g->ny - 1);
  const double cv = 0.5 * (g->nv - 1);
  const double vmax = std::fabs((0 - cv) * g->dv);
  std::vector<RayInfo3D> rays((size_t)g->n_angles * g->nu);
  g->view3d_host.assign(g->n_angles, ViewInfo3D());
  for (int a = 0; a < g->n_angles; ++a) {
    const double b = g->angles[a];
    const double cb = std::cos(b), sb = std::sin(b);
    const double Sx = g->sod * cb, Sy = g->sod * sb;
    const double D0x = -(g->sdd - g->sod) * cb, D0y = -(g->sdd - g->sod) * sb;
    ViewInfo3D& vi = g->view3d_host[a];
    vi.sx = (float)Sx;
    vi.sy = (float)Sy;
    vi.eux = (float)(-sb);
    vi.euy = (float)cb;
    vi.esx = (float)cb;
    vi.esy = (float)sb;
    vi.sdd = (float)g->sdd;
    vi.inv_du = (float)(1.0 / g->du);
    vi.cu = (float)(0.5 * (g->nu - 1));
    vi.has_x = 0;
    vi.has_y = 0;
    for (int iu = 0; iu < g->nu; ++iu) {
      const double u = (iu - (g->nu - 1) / 2.0) * g->du;
      const double dx = (D0x + u * (-sb)) - Sx;
      const double dy = (D0y + u * cb) - Sy;
      if (vmax >= std::fmax(std::fabs(dx), std::fabs(dy)))
        return fail(VRPS_ERR_UNSUPPORTED, "view %d column %d: ray dominant along z (cone too wide)", a, iu);
      {
        // every plane of the volume along the marching axis must lie in front of the source
        const bool ax0 = std::fabs(dx) >= std::fabs(dy);
        const double Sa = ax0 ? Sx : Sy, da = ax0 ? dx : dy;
        const int na = ax0 ? g->nx : g->ny;
        const double c = 0.5 * (na - 1);
        const double t0 = ((0 - c) * vox - Sa) / da, t1 = ((na - 1 - c) * vox - Sa) / da;
        if (!(t0 > 0.0 && t1 > 0.0))
          return fail(VRPS_ERR_INVALID_ARG, "view %d column %d: volume planes behind the source", a, iu);
      }
      RayInfo3D& r = rays[(size_t)a * g->nu + iu];
      r.pad = 0;
      // transverse index P0 + P1 (l - lc) and z step per row Q0 + Q1 (l - lc) on plane l
      double P0, P1, Q0, Q1, lc;
      if (std::fabs(dx) >= std::fabs(dy)) {
        r.axis = 0;
        P0 = cy + (Sy - Sx * dy / dx) / vox;
        P1 = dy / dx;
        Q0 = -Sx * g->dv / (dx * vox);
        Q1 = g->dv / dx;
        lc = cx;
        vi.has_x = 1;
      } else {
        r.axis = 1;
        P0 = cx + (Sx - Sy * dx / dy) / vox;
        P1 = dx / dy;
        Q0 = -Sy * g->dv / (dy * vox);
        Q1 = g->dv / dy;
        lc = cy;
        vi.has_y = 1;
      }
      r.PF0 = std::llround(std::ldexp(P0 - P1 * lc, 32));
      r.PF1 = std::llround(std::ldexp(P1, 32));
      r.QF0 = std::llround(std::ldexp(Q0 - Q1 * lc, 32));
      r.QF1 = std::llround(std::ldexp(Q1, 32));
      r.P1 = (float)P1;
      r.R = (float)Q1;
    }
  }
  VRPS_CUDA(cudaMalloc((void**)&g->ray3d, sizeof(RayInfo3D) * rays.size()));
  VRPS_CUDA(cudaMemcpy(g->ray3d, rays.data(), sizeof(RayInfo3D) * rays.size(), cudaMemcpyHostToDevice));
  VRPS_CUDA(cudaMalloc((void**)&g->view3d, sizeof(ViewInfo3D) * g->n_angles));
  VRPS_CUDA(cudaMemcpy(g->view3d, g->view3d_host.data(), sizeof(ViewInfo3D) * g->n_angles,
                       cudaMemcpyHostToDevice));
  return VRPS_OK;
}

static int fgp_dual_size(const vrps_geom* g, size_t* count) {
  *count = (size_t)g->dims * (size_t)g->n;
  return VRPS_OK;
}

int take_device_error(vrps_geom* g) {
  Workspace& w = g->ws;
  if (!w.dev_error) return VRPS_OK;
  unsigned err = 0;
  VRPS_CUDA(cudaMemcpy(&err, w.dev_error, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (!err) return VRPS_OK;
  VRPS_CUDA(cudaMemset(w.dev_error, 0, sizeof(unsigned)));
  return fail(VRPS_ERR_TIMEOUT, "a bounded device-side wait expired (error word %u)", err);
}

}  // namespace vrps

using namespace vrps;

extern "C" {

const char* vrps_last_error(void) { return g_err; }

int vrps_version(void) { return 10000; }

int vrps_geom_par2d(int nx, int ny, double pixel, int n_angles, const double* angles_rad,
                    int n_bins, double bin_spacing, int n_subsets, vrps_geom** out) {
  if (!out) return fail(VRPS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nx <= 0 || ny <= 0 || n_angles <= 0 || n_bins <= 0)
    return fail(VRPS_ERR_INVALID_ARG, "sizes must be positive (nx=%d ny=%d angles=%d bins=%d)", nx, ny,
                n_angles, n_bins);
  if (n_angles > 65535) return fail(VRPS_ERR_INVALID_ARG, "at most 65535 angles");
  if ((int64_t)nx * ny > (int64_t)1 << 30) return fail(VRPS_ERR_INVALID_ARG, "image too large");
  if (!(pixel > 0) || !(bin_spacing > 0)) return fail(VRPS_ERR_INVALID_ARG, "pixel and bin spacing must be > 0");
  if (!angles_rad) return fail(VRPS_ERR_INVALID_ARG, "angles is NULL");
  if (n_subsets < 1 || n_subsets > n_angles)
    return fail(VRPS_ERR_INVALID_ARG, "n_subsets %d outside [1, %d]", n_subsets, n_angles);
  for (int a = 0; a < n_angles; ++a)
    if (!std::isfinite(angles_rad[a])) return fail(VRPS_ERR_INVALID_ARG, "angle %d is not finite", a);
  vrps_geom* g = new (std::nothrow) vrps_geom();
  if (!g) return fail(VRPS_ERR_OUT_OF_MEMORY, "host allocation failed");
  g->dims = 2;
  g->nx = nx;
  g->ny = ny;
  g->nz = 1;
  g->pixel = pixel;
  g->n_angles = n_angles;
  g->n_bins = n_bins;
  g->bin_spacing = bin_spacing;
  g->n_subsets = n_subsets;
  g->n = (int64_t)nx * ny;
  g->m = (int64_t)n_angles * n_bins;
  g->row_len = n_bins;
  g->angles.assign(angles_rad, angles_rad + n_angles);
  cudaError_t e = cudaGetDevice(&g->device);
  int st = e == cudaSuccess ? VRPS_OK : cuda_fail(e, "cudaGetDevice");
  if (st == VRPS_OK) st = build_par2d(g);
  if (st == VRPS_OK) st = finish_common(g);
  if (st != VRPS_OK) {
    free_geom(g);
    return st;
  }
  *out = g;
  return VRPS_OK;
}

int vrps_geom_cone3d(int nx, int ny, int nz, double voxel, int n_views, const double* betas_rad,
                     int nu, int nv, double du, double dv, double sod, double sdd, int n_subsets,
                     vrps_geom** out) {
  if (!out) return fail(VRPS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nx <= 0 || ny <= 0 || nz <= 0 || n_views <= 0 || nu <= 0 || nv <= 0)
    return fail(VRPS_ERR_INVALID_ARG, "sizes must be positive");
  if (n_views > 65535) return fail(VRPS_ERR_INVALID_ARG, "at most 65535 views");
  // detector rows / columns: the adjoint's float row-range estimate stays within one row
  if (nu > 65536 || nv > 65536) return fail(VRPS_ERR_INVALID_ARG, "at most 65536 detector columns and rows");
  if ((int64_t)nx * ny * nz > ((int64_t)1 << 31) - 1) return fail(VRPS_ERR_INVALID_ARG, "volume too large");
  if ((int64_t)nu * nv * n_views > ((int64_t)1 << 31) - 1) return fail(VRPS_ERR_INVALID_ARG, "sinogram too large");
  if (!(voxel > 0) || !(du > 0) || !(dv > 0)) return fail(VRPS_ERR_INVALID_ARG, "spacings must be > 0");
  if (!betas_rad) return fail(VRPS_ERR_INVALID_ARG, "betas is NULL");
  if (n_subsets < 1 || n_subsets > n_views)
    return fail(VRPS_ERR_INVALID_ARG, "n_subsets %d outside [1, %d]", n_subsets, n_views);
  const double half = 0.5 * voxel * std::sqrt((double)nx * nx + (double)ny * ny);
  if (!(sod > half + voxel) || !(sdd > sod))
    return fail(VRPS_ERR_INVALID_ARG, "need sdd > sod > %.6g (source outside the volume)", half);
  for (int a = 0; a < n_views; ++a)
    if (!std::isfinite(betas_rad[a])) return fail(VRPS_ERR_INVALID_ARG, "view %d angle not finite", a);
  vrps_geom* g = new (std::nothrow) vrps_geom();
  if (!g) return fail(VRPS_ERR_OUT_OF_MEMORY, "host allocation failed");
  g->dims = 3;
  g->nx = nx;
  g->ny = ny;
  g->nz = nz;
  g->pixel = voxel;
  g->n_angles = n_views;
  g->nu = nu;
  g->nv = nv;
  g->du = du;
  g->dv = dv;
  g->sod = sod;
  g->sdd = sdd;
  g->n_subsets = n_subsets;
  g->n = (int64_t)nx * ny * nz;
  g->m = (int64_t)n_views * nu * nv;
  g->row_len = nu * nv;
  g->angles.assign(betas_rad, betas_rad + n_views);
  cudaError_t e = cudaGetDevice(&g->device);
  int st = e == cudaSuccess ? VRPS_OK : cuda_fail(e, "cudaGetDevice");
  if (st == VRPS_OK) st = build_cone3d(g);
  if (st == VRPS_OK) st = finish_common(g);
  if (st != VRPS_OK) {
    free_geom(g);
    return st;
  }
  *out = g;
  return VRPS_OK;
}

int vrps_geom_free(vrps_geom* g) {
  free_geom(g);
  return VRPS_OK;
}

int vrps_geom_sizes(const vrps_geom* g, int subset, int64_t* n, int64_t* m, int* rows, int* row_len,
                    int* dims) {
  if (!g) return fail(VRPS_ERR_INVALID_ARG, "geometry handle is NULL");
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (row_len) *row_len = g->row_len;
  if (dims) *dims = g->dims;
  if (rows) {
    if (subset == -1) {
      *rows = g->n_angles;
    } else {
      if (subset < 0 || subset >= g->n_subsets)
        return fail(VRPS_ERR_INVALID_ARG, "subset %d outside [-1, %d)", subset, g->n_subsets);
      *rows = g->subset_off[subset + 1] - g->subset_off[subset];
    }
  }
  return VRPS_OK;
}

// integers l in [0, nl) with lo < a + b (l - lc) < hi
static void open_interval(double a, double b, double lc, double lo, double hi, double* l0, double* l1) {
  if (b == 0.0) {
    if (!(a > lo && a < hi)) {
      *l0 = 1.0;
      *l1 = 0.0;
    }
    return;
  }
  double t0 = lc + (lo - a) / b, t1 = lc + (hi - a) / b;
  if (t0 > t1) std::swap(t0, t1);
  *l0 = std::fmax(*l0, t0);
  *l1 = std::fmin(*l1, t1);
}

static int64_t count_open(double l0, double l1, int nl) {
  // integers strictly inside (l0, l1), clipped to [0, nl-1]
  long long a = (long long)std::floor(l0) + 1, b = (long long)std::ceil(l1) - 1;
  if (a < 0) a = 0;
  if (b > nl - 1) b = nl - 1;
  return b >= a ? (int64_t)(b - a + 1) : 0;
}

int vrps_geom_samples(const vrps_geom* g, int subset, int64_t* samples) {
  if (!g || !samples) return fail(VRPS_ERR_INVALID_ARG, "NULL argument");
  std::vector<int> ids;
  if (subset == -1) {
    for (int a = 0; a < g->n_angles; ++a) ids.push_back(a);
  } else {
    if (subset < 0 || subset >= g->n_subsets) return fail(VRPS_ERR_INVALID_ARG, "bad subset %d", subset);
    for (int a = subset; a < g->n_angles; a += g->n_subsets) ids.push_back(a);
  }
  int64_t total = 0;
  if (g->dims == 2) {
    const double pix = g->pixel, ds = g->bin_spacing, jc = 0.5 * (g->n_bins - 1);
    for (int a : ids) {
      const double c = std::cos(g->angles[a]), s = std::sin(g->angles[a]);
      const bool rows = std::fabs(c) >= std::fabs(s);
      const int ncols = rows ? g->nx : g->ny, nl = rows ? g->ny : g->nx;
      const double A1 = rows ? ds / (pix * c) : ds / (pix * s), A2 = rows ? -s / c : -c / s;
      const double uc = 0.5 * (ncols - 1), lc = 0.5 * (nl - 1);
      for (int j = 0; j < g->n_bins; ++j) {
        double l0 = -1e300, l1 = 1e300;
        open_interval(uc + A1 * (j - jc), A2, lc, -1.0, (double)ncols, &l0, &l1);
        total += count_open(l0, l1, nl);
      }
    }
  } else {
    const double vox = g->pixel, cv = 0.5 * (g->nv - 1), cz = 0.5 * (g->nz - 1);
    for (int a : ids) {
      const double cb = std::cos(g->angles[a]), sb = std::sin(g->angles[a]);
      const double Sx = g->sod * cb, Sy = g->sod * sb;
      const double D0x = -(g->sdd - g->sod) * cb, D0y = -(g->sdd - g->sod) * sb;
      for (int iu = 0; iu < g->nu; ++iu) {
        const double u = (iu - (g->nu - 1) / 2.0) * g->du;
        const double dx = (D0x + u * (-sb)) - Sx, dy = (D0y + u * cb) - Sy;
        const bool ax0 = std::fabs(dx) >= std::fabs(dy);
        const double Sa = ax0 ? Sx : Sy, So = ax0 ? Sy : Sx, da = ax0 ? dx : dy, dd = ax0 ? dy : dx;
        const int nl = ax0 ? g->nx : g->ny, nt = ax0 ? g->ny : g->nx;
        const double lc = 0.5 * (nl - 1), tc = 0.5 * (nt - 1);
        const double P0 = tc + (So - Sa * dd / da) / vox, P1 = dd / da;
        const double Q0 = -Sa * g->dv / (da * vox), Q1 = g->dv / da;
        for (int iv = 0; iv < g->nv; ++iv) {
          const double k = iv - cv;
          double l0 = -1e300, l1 = 1e300;
          open_interval(P0, P1, lc, -1.0, (double)nt, &l0, &l1);
          open_interval(cz + k * Q0, k * Q1, lc, -1.0, (double)g->nz, &l0, &l1);
          if (l1 > l0) total += count_open(l0, l1, nl);
        }
      }
    }
  }
  *samples = total;
  return VRPS_OK;
}

int vrps_autotune(vrps_geom* g, int reps, double* out3, vrps_stream_t stream) {
  VRPS_TRY(check_geom(g));
  if (reps < 1) return fail(VRPS_ERR_INVALID_ARG, "reps must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  if (g->dims == 3) {
    // 3D: z planes per chunk of the streaming FGP iteration, timed on 3 iterations
    Workspace& w = g->ws;
    VRPS_TRY(ensure(&w.img, (size_t)g->n));
    VRPS_TRY(ensure(&w.img2, (size_t)g->n));
    VRPS_TRY(ensure(&w.dual, 3 * (size_t)g->n));
    VRPS_TRY(fill(w.img, 0.5f, g->n, s));
    ProxTail t;
    std::memset(&t, 0, sizeof(t));
    t.out = w.img2;
    cudaEvent_t e0, e1;
    VRPS_CUDA(cudaEventCreate(&e0));
    VRPS_CUDA(cudaEventCreate(&e1));
    const int cand[] = {4, 8, 16, 32, 64, 128};
    int best_zc = 0;
    float best = 1e30f;
    for (int zc : cand) {
      g->tune_f3_zc = zc;
      for (int r = 0; r <= reps; ++r) {
        VRPS_CUDA(cudaMemsetAsync(w.dual, 0, sizeof(float) * 3 * (size_t)g->n, s));
        VRPS_CUDA(cudaEventRecord(e0, s));
        VRPS_TRY(fgp_run(g, w.img, 0.01f, 3, 1, w.dual, t, s));
        VRPS_CUDA(cudaEventRecord(e1, s));
        VRPS_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        VRPS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0 && ms < best) {
          best = ms;
          best_zc = zc;
        }
      }
    }
    g->tune_f3_zc = best_zc;
    // adjoint voxels per thread along z (16 or 32; same results), timed on subset 0
    const int* ids = g->order_subset + g->subset_off[0];
    const int rows = g->subset_off[1] - g->subset_off[0];
    VRPS_TRY(ensure(&w.sino, (size_t)g->m));
    VRPS_TRY(fill(w.sino, 0.5f, (int64_t)rows * g->row_len, s));
    UpdateArgs ua;
    std::memset(&ua, 0, sizeof(ua));
    ua.prescaled = 1;
    ua.out = w.img2;
    int best_az = 16;
    float best_a = 1e30f;
    for (int az : {16, 32}) {
      g->tune_adj3_zc = az;
      for (int r = 0; r <= reps; ++r) {
        VRPS_CUDA(cudaEventRecord(e0, s));
        VRPS_TRY(proj_adjoint(g, w.sino, ids, rows, ua, s));
        VRPS_CUDA(cudaEventRecord(e1, s));
        VRPS_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        VRPS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0 && ms < best_a) {
          best_a = ms;
          best_az = az;
        }
      }
    }
    g->tune_adj3_zc = best_az;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (out3) {
      out3[0] = best_zc;
      out3[1] = best_az;
      out3[2] = 1e3 * (double)best;
      out3[3] = 1e3 * (double)best_a;
    }
    return VRPS_OK;
  }
  const int* ids = nullptr;
  int rows = 0;
  VRPS_TRY(subset_rows(g, 0, &ids, &rows));
  Workspace& w = g->ws;
  VRPS_TRY(ensure(&w.img, (size_t)g->n));
  VRPS_TRY(ensure(&w.img2, (size_t)g->n));
  VRPS_TRY(ensure(&w.sino, (size_t)g->m));
  VRPS_TRY(fill(w.img, 1.f, g->n, s));
  VRPS_TRY(transpose2d(w.img, w.img2, g->ny, g->nx, s));
  cudaEvent_t e0, e1;
  VRPS_CUDA(cudaEventCreate(&e0));
  VRPS_CUDA(cudaEventCreate(&e1));
  auto timed = [&](auto&& launch, float* best) -> int {
    VRPS_TRY(launch());   // warm-up
    *best = 1e30f;
    for (int r = 0; r < reps; ++r) {
      VRPS_CUDA(cudaEventRecord(e0, s));
      VRPS_TRY(launch());
      VRPS_CUDA(cudaEventRecord(e1, s));
      VRPS_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      VRPS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < *best) *best = ms;
    }
    return VRPS_OK;
  };
  FwdOut fo{w.sino, nullptr, nullptr};
  g->tune_full_fwd_bytes = g->tune_full_fwd_group = g->tune_full_adj_split = 0;   // subsets first
  const int cand[] = {16 << 10, 24 << 10, 32 << 10, 48 << 10, 64 << 10, 96 << 10};
  const int groups[] = {1, 2, 4, 8};
  int best_bytes = 0, best_group = 1;
  float best_f = 1e30f;
  for (int c : cand) {
    for (int grp : groups) {
      if (grp > 1 && (c > (64 << 10) || g->n_bins > 1536)) continue;   // two buffers; rays held in registers
      g->tune_fwd_bytes = c;
      g->tune_fwd_group = grp;
      float t = 0.f;
      const int rc = timed([&]() { return fwd2d(g, w.img, w.img2, ids, rows, FWD_PLAIN, fo, s); }, &t);
      if (rc != VRPS_OK) {
        g->tune_fwd_bytes = 0;
        g->tune_fwd_group = 0;
        return rc;
      }
      if (t < best_f) {
        best_f = t;
        best_bytes = c;
        best_group = grp;
      }
    }
  }
  g->tune_fwd_bytes = best_bytes;
  g->tune_fwd_group = best_group;
  UpdateArgs ua;
  std::memset(&ua, 0, sizeof(ua));
  ua.out = w.img;
  int best_two = 0, best_split = 1;
  float best_a = 1e30f;
  for (int split : {1, 2, 4}) {
    for (int two = 0; two < 2; ++two) {
      g->tune_adj_two = two;
      g->tune_adj_split = split;
      float t = 0.f;
      const int rc = timed([&]() { return adj2d(g, w.sino, ids, rows, ua, s); }, &t);
      if (rc != VRPS_OK) {
        g->tune_adj_two = -1;
        g->tune_adj_split = 0;
        return rc;
      }
      if (t < best_a) {
        best_a = t;
        best_two = two;
        best_split = split;
      }
    }
  }
  g->tune_adj_two = best_two;
  g->tune_adj_split = best_split;
  // all-angle passes (SVRG snapshots, full gradients): their own forward band / bands per CTA
  // and adjoint angle shares, timed on the full sinogram
  if (g->n_subsets > 1) {
    const int* all = g->order_natural;
    const int nall = g->n_angles;
    int fb = best_bytes, fg = best_group;
    float bf = 1e30f;
    for (int c : cand) {
      for (int grp : groups) {
        if (grp > 1 && (c > (64 << 10) || g->n_bins > 1536)) continue;
        g->tune_full_fwd_bytes = c;
        g->tune_full_fwd_group = grp;
        float t = 0.f;
        const int rc = timed([&]() { return fwd2d(g, w.img, w.img2, all, nall, FWD_PLAIN, fo, s); }, &t);
        if (rc != VRPS_OK) {
          g->tune_full_fwd_bytes = g->tune_full_fwd_group = 0;
          return rc;
        }
        if (t < bf) {
          bf = t;
          fb = c;
          fg = grp;
        }
      }
    }
    g->tune_full_fwd_bytes = fb;
    g->tune_full_fwd_group = fg;
    int fs = 1;
    float ba = 1e30f;
    for (int split : {1, 2, 4, 8}) {
      g->tune_full_adj_split = split;
      float t = 0.f;
      const int rc = timed([&]() { return adj2d(g, w.sino, all, nall, ua, s); }, &t);
      if (rc != VRPS_OK) {
        g->tune_full_adj_split = 0;
        return rc;
      }
      if (t < ba) {
        ba = t;
        fs = split;
      }
    }
    g->tune_full_adj_split = fs;
  }
  // 2D FGP output tile, timed on one 32-iteration prox call of a uniform random image with a
  // TV weight that saturates most of the dual (as in reconstructions: the projection onto the
  // unit ball is then active at most pixels)
  {
    VRPS_TRY(ensure(&w.dual, 2 * (size_t)g->n));
    VRPS_TRY(philox_uniform(0x5eedULL, 0u, 7u, w.img, g->n, s));
    ProxTail t;
    std::memset(&t, 0, sizeof(t));
    t.out = w.img2;
    int best_tile = 0;
    float best_p = 1e30f;
    for (int tile = 0; tile < 3; ++tile) {
      g->tune_fgp_tile = tile;
      float tp = 0.f;
      const int rc = timed([&]() -> int {
        VRPS_CUDA(cudaMemsetAsync(w.dual, 0, sizeof(float) * 2 * (size_t)g->n, s));
        return fgp_run(g, w.img, 0.25f, 32, 1, w.dual, t, s);
      }, &tp);
      if (rc != VRPS_OK) {
        g->tune_fgp_tile = 0;
        return rc;
      }
      if (tp < best_p) {
        best_p = tp;
        best_tile = tile;
      }
    }
    g->tune_fgp_tile = best_tile;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (out3) {
    out3[0] = best_bytes;
    out3[1] = best_two ? 2 : 1;
    out3[2] = 1e3 * (double)(best_f + best_a);
    out3[3] = best_group;
  }
  return VRPS_OK;
}

int vrps_launch_shape(const vrps_geom* g, int* out6) {
  VRPS_TRY(check_geom(g));
  if (!out6) return fail(VRPS_ERR_INVALID_ARG, "out6 is NULL");
  out6[0] = g->tune_fwd_bytes;
  out6[1] = g->tune_fwd_group;
  out6[2] = g->dims == 3 ? (g->tune_adj3_zc == 32 ? 32 : 16) : (g->tune_adj_two < 0 ? 0 : (g->tune_adj_two ? 2 : 1));
  out6[3] = g->dims == 3 ? fgp3_zc(g) : 0;
  out6[4] = g->tune_fgp_tile;
  out6[5] = g->tune_adj_split;
  return VRPS_OK;
}

int vrps_launch_shape_full(const vrps_geom* g, int* out3) {
  VRPS_TRY(check_geom(g));
  if (!out3) return fail(VRPS_ERR_INVALID_ARG, "out3 is NULL");
  out3[0] = g->tune_full_fwd_bytes;
  out3[1] = g->tune_full_fwd_group;
  out3[2] = g->tune_full_adj_split;
  return VRPS_OK;
}

int vrps_set_launch_shape(vrps_geom* g, int fwd_band_bytes, int fwd_group, int adj_pixels_per_thread, int fgp3_chunk,
                          int fgp_tile, int adj_split) {
  VRPS_TRY(check_geom(g));
  const bool adj_ok = g->dims == 3 ? (adj_pixels_per_thread == 0 || adj_pixels_per_thread == 16 ||
                                      adj_pixels_per_thread == 32)
                                   : (adj_pixels_per_thread >= 0 && adj_pixels_per_thread <= 2);
  if (fwd_band_bytes < 0 || fwd_band_bytes > (200 << 10) || fwd_group < 0 || fwd_group > 64 || !adj_ok ||
      fgp3_chunk < 0 || fgp_tile < 0 || fgp_tile > 4 || adj_split < 0 || adj_split > 64)
    return fail(VRPS_ERR_INVALID_ARG, "launch shape out of range");
  if (g->dims == 3) {
    g->tune_adj3_zc = adj_pixels_per_thread;
    adj_pixels_per_thread = 0;
  }
  g->tune_fgp_tile = fgp_tile;
  g->tune_adj_split = adj_split;
  g->tune_full_fwd_bytes = g->tune_full_fwd_group = g->tune_full_adj_split = 0;   // all passes alike
  g->tune_fwd_bytes = fwd_band_bytes;
  g->tune_fwd_group = fwd_group;
  g->tune_adj_two = adj_pixels_per_thread == 0 ? -1 : (adj_pixels_per_thread == 2 ? 1 : 0);
  g->tune_f3_zc = fgp3_chunk;
  return VRPS_OK;
}

int vrps_proj_fwd(const vrps_geom* g, int subset, const float* x, float* y, vrps_stream_t stream) {
  VRPS_TRY(check_geom(g));
  if (!x || !y) return fail(VRPS_ERR_INVALID_ARG, "x or y is NULL");
  const int* ids = nullptr;
  int rows = 0;
  VRPS_TRY(subset_rows(g, subset, &ids, &rows));
  FwdOut o{y, nullptr, nullptr};
  return proj_forward(g, x, nullptr, ids, rows, FWD_PLAIN, o, (cudaStream_t)stream);
}

int vrps_proj_adj(const vrps_geom* g, int subset, const float* r, float* x, vrps_stream_t stream) {
  VRPS_TRY(check_geom(g));
  if (!x || !r) return fail(VRPS_ERR_INVALID_ARG, "r or x is NULL");
  const int* ids = nullptr;
  int rows = 0;
  VRPS_TRY(subset_rows(g, subset, &ids, &rows));
  UpdateArgs u;
  std::memset(&u, 0, sizeof(u));
  u.enabled = 0;
  u.out = x;
  return proj_adjoint(g, r, ids, rows, u, (cudaStream_t)stream);
}

int vrps_prox_tv(const vrps_geom* g, const float* v, float* x, float tau, int iters, int nonneg,
                 float* dual, vrps_stream_t stream) {
  VRPS_TRY(check_geom(g));
  if (!v || !x) return fail(VRPS_ERR_INVALID_ARG, "v or x is NULL");
  if (v == x) return fail(VRPS_ERR_INVALID_ARG, "v and x must not alias");
  if (!(tau > 0.f) || !std::isfinite(tau)) return fail(VRPS_ERR_INVALID_ARG, "tau must be > 0");
  if (iters < 0) return fail(VRPS_ERR_INVALID_ARG, "iters must be >= 0");
  vrps_geom* gm = const_cast<vrps_geom*>(g);
  size_t dn = 0;
  fgp_dual_size(g, &dn);
  cudaStream_t s = (cudaStream_t)stream;
  float* d = dual;
  if (!d) {
    VRPS_TRY(ensure(&gm->ws.dual_cold, dn));
    VRPS_CUDA(cudaMemsetAsync(gm->ws.dual_cold, 0, dn * sizeof(float), s));
    d = gm->ws.dual_cold;
  }
  ProxTail t;
  std::memset(&t, 0, sizeof(t));
  t.mode = 0;
  t.out = x;
  return fgp_run(g, v, tau, iters, nonneg ? 1 : 0, d, t, s);
}

int vrps_power_iteration(const vrps_geom* g, int iters, uint64_t seed, double* L_out, vrps_stream_t stream) {
  VRPS_TRY(check_geom(g));
  if (!L_out) return fail(VRPS_ERR_INVALID_ARG, "L_out is NULL");
  if (iters < 1) return fail(VRPS_ERR_INVALID_ARG, "iters must be >= 1");
  vrps_geom* gm = const_cast<vrps_geom*>(g);
  Workspace& w = gm->ws;
  cudaStream_t s = (cudaStream_t)stream;
  VRPS_TRY(ensure(&w.img, (size_t)g->n));
  VRPS_TRY(ensure(&w.img2, (size_t)g->n));
  VRPS_TRY(ensure(&w.sino, (size_t)g->m));
  float* u = w.img;
  float* z = w.img2;
  VRPS_TRY(philox_uniform(seed, 0, 1, u, g->n, s));
  VRPS_TRY(dot64(u, u, g->n, w.scalars + 0, w, s));
  VRPS_TRY(scale_inv_sqrt(u, u, w.scalars + 0, g->n, s));
  UpdateArgs ua;
  std::memset(&ua, 0, sizeof(ua));
  ua.out = z;
  for (int it = 0; it < iters; ++it) {
    FwdOut o{w.sino, nullptr, nullptr};
    VRPS_TRY(proj_forward(g, u, nullptr, g->order_natural, g->n_angles, FWD_PLAIN, o, s));
    VRPS_TRY(proj_adjoint(g, w.sino, g->order_natural, g->n_angles, ua, s));
    VRPS_TRY(dot64(u, z, g->n, w.scalars + 1, w, s));
    VRPS_TRY(dot64(z, z, g->n, w.scalars + 2, w, s));
    VRPS_TRY(scale_inv_sqrt(u, z, w.scalars + 2, g->n, s));
  }
  double lam = 0.0;
  VRPS_CUDA(cudaMemcpyAsync(&lam, w.scalars + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
  VRPS_CUDA(cudaStreamSynchronize(s));
  VRPS_TRY(take_device_error(gm));
  *L_out = lam;
  return VRPS_OK;
}

int vrps_objective(const vrps_geom* g, const float* x, const float* b, double alpha, double* out3,
                   vrps_stream_t stream) {
  VRPS_TRY(check_geom(g));
  if (!x || !b || !out3) return fail(VRPS_ERR_INVALID_ARG, "NULL argument");
  vrps_geom* gm = const_cast<vrps_geom*>(g);
  Workspace& w = gm->ws;
  cudaStream_t s = (cudaStream_t)stream;
  VRPS_TRY(ensure(&w.sino, (size_t)g->m));
  FwdOut o{w.sino, b, nullptr};
  VRPS_TRY(proj_forward(g, x, nullptr, g->order_natural, g->n_angles, FWD_RESID, o, s));
  VRPS_TRY(dot64(w.sino, w.sino, g->m, w.scalars + 3, w, s));
  VRPS_TRY(tv64(g, x, w.scalars + 4, w, s));
  double h[2];
  VRPS_CUDA(cudaMemcpyAsync(h, w.scalars + 3, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  VRPS_CUDA(cudaStreamSynchronize(s));
  VRPS_TRY(take_device_error(gm));
  out3[1] = 0.5 * h[0];
  out3[2] = h[1];
  out3[0] = out3[1] + alpha * out3[2];
  return VRPS_OK;
}

int vrps_check_error(const vrps_geom* g, vrps_stream_t stream) {
  VRPS_TRY(check_geom(g));
  VRPS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return take_device_error(const_cast<vrps_geom*>(g));
}

int vrps_philox_schedule(uint64_t seed, uint32_t job, int64_t k0, int count, int n_subsets, double p,
                         int32_t* out, vrps_stream_t stream) {
  if (!out || count < 0 || n_subsets < 1 || !(p > 0))
    return fail(VRPS_ERR_INVALID_ARG, "bad schedule arguments");
  if (k0 < 0) return fail(VRPS_ERR_INVALID_ARG, "k0 must be >= 0");
  return philox_schedule(seed, job, k0, count, n_subsets, p, out, (cudaStream_t)stream);
}

}  // extern "C"

// ------------------------------------------------------------------ launch accounting
#include <atomic>
#include <map>
#include <mutex>

namespace vrps {
namespace {
struct PendingLaunch {
  const char* name;
  cudaEvent_t e0, e1;
  double bytes;
};
struct Totals {
  uint64_t launches = 0;
  double ms = 0.0;
  double bytes = 0.0;
};
struct ProfState {
  std::atomic<uint64_t> launches{0};
  std::atomic<bool> on{false};
  std::mutex mu;
  std::vector<PendingLaunch> pending;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, Totals> totals;
};
ProfState& prof() {
  static ProfState* st = new ProfState();   // never destroyed: safe at process exit
  return *st;
}
thread_local PendingLaunch t_open = {nullptr, nullptr, nullptr, 0.0};

cudaEvent_t take_event(ProfState& st) {
  if (!st.pool.empty()) {
    cudaEvent_t e = st.pool.back();
    st.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

void launch_begin(const char* name, cudaStream_t s, double bytes) {
  ProfState& st = prof();
  st.launches.fetch_add(1, std::memory_order_relaxed);
  t_open.name = nullptr;
  if (!st.on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(st.mu);
  cudaEvent_t e0 = take_event(st), e1 = take_event(st);
  if (!e0 || !e1) return;
  cudaEventRecord(e0, s);
  t_open = {name, e0, e1, bytes};
}

void launch_end(cudaStream_t s) {
  if (!t_open.name) return;
  ProfState& st = prof();
  cudaEventRecord(t_open.e1, s);
  std::lock_guard<std::mutex> lk(st.mu);
  st.pending.push_back(t_open);
  t_open.name = nullptr;
}

void launch_count_add(long long n) { prof().launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

bool profiling_on() { return prof().on.load(std::memory_order_relaxed); }

}  // namespace vrps

extern "C" {

uint64_t vrps_kernel_launches(void) { return vrps::prof().launches.load(); }

int vrps_profile_enable(int on) {
  vrps::ProfState& st = vrps::prof();
  std::lock_guard<std::mutex> lk(st.mu);
  if (!on) {
    cudaDeviceSynchronize();
    for (auto& p : st.pending) {
      st.pool.push_back(p.e0);
      st.pool.push_back(p.e1);
    }
    st.pending.clear();
    st.totals.clear();
  }
  st.on.store(on != 0);
  return VRPS_OK;
}

int vrps_profile_read(vrps_kernel_stat* out, int cap, int* count) {
  vrps::ProfState& st = vrps::prof();
  std::lock_guard<std::mutex> lk(st.mu);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return vrps::cuda_fail(e, "cudaDeviceSynchronize(profile)");
  for (auto& p : st.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
      auto& t = st.totals[p.name];
      t.launches += 1;
      t.ms += ms;
      t.bytes += p.bytes;
    }
    st.pool.push_back(p.e0);
    st.pool.push_back(p.e1);
  }
  st.pending.clear();
  int k = 0;
  for (auto& kv : st.totals) {
    if (out && k < cap) {
      std::snprintf(out[k].name, sizeof(out[k].name), "%s", kv.first.c_str());
      out[k].launches = kv.second.launches;
      out[k].total_ms = kv.second.ms;
      out[k].bytes = kv.second.bytes;
    }
    ++k;
  }
  if (count) *count = k;
  return VRPS_OK;
}

}  // extern "C"
