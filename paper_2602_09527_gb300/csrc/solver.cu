// vrps_solve: the iteration loop of Algorithm 1 and its family, driven from the host.
//
// Per outer iteration k the host enqueues, on one stream:
//   1. the forward projector of subset i_k (or all angles) with the estimator epilogue:
//        SGD / full:  dr = A_i x - b_i
//        SVRG:        dr = A_i x - (A x~)_i            (A x~ stored at the snapshot)
//        SAGA:        dr = (A_i x - b_i) - rho_i,  rho_i <- A_i x - b_i
//      (by linearity A_i^T dr equals grad f_i(x) - grad f_i(x~), resp. grad f_i(x) - v^i, so
//      the SAGA table of N images is held as one residual sinogram of m floats);
//   2. the pixel-driven adjoint with the update epilogue:
//        G = c A_i^T dr + gbar,   x_hat = x - gamma (G - h)            (Algorithm 1)
//        theta_k = 0: x <- x_hat;   theta_k = 1: v = x_hat - (gamma/p) h
//      (SAGA also does gbar += A_i^T dr; gbar is the table sum v-bar);
//   3. if theta_k = 1: FGP prox of v with tau = gamma alpha / p, whose output kernel writes
//      x <- x+ and h += (p/gamma)(x+ - x_hat).
// The draws (i_k, theta_k, L-SVRG coin) come from a Philox kernel and are copied to the
// host once, before the loop, so that the host knows which kernels to enqueue.
#include <cmath>
#include <cstring>
#include <vector>

#include "vrps_internal.h"

namespace vrps {
namespace {

enum Est { EST_FULL = -1 };

struct State {
  float *x, *xf, *xfT, *h, *xhat, *v, *gbar, *xprox, *dual, *b_perm, *tab, *res;
};

double step_factor(int algo, int est) {
  if (algo == VRPS_ALGO_ISTA || algo == VRPS_ALGO_PROXSKIP) return 1.99;
  if (algo == VRPS_ALGO_SAGA) return 1.0 / 3.0;
  if (algo == VRPS_ALGO_VR_PROXSKIP && est == VRPS_EST_SAGA) return 1.0 / 3.0;
  return 1.0;
}

}  // namespace

// FP16 storage scale: a power of two bringing the data's RMS into [512, 1024) (reads b_perm).
int storage_scale(vrps_geom* g, int kind, float* scale, cudaStream_t s) {
  *scale = 1.f;
  if (kind != STORE_F16) return VRPS_OK;
  Workspace& w = g->ws;
  VRPS_TRY(dot64(w.b_perm, w.b_perm, g->m, w.scalars + 7, w, s));
  double ss = 0.0;
  VRPS_CUDA(cudaMemcpyAsync(&ss, w.scalars + 7, sizeof(double), cudaMemcpyDeviceToHost, s));
  VRPS_CUDA(cudaStreamSynchronize(s));
  const double rms = std::sqrt(ss / (double)g->m);
  if (!(rms > 0.0) || !std::isfinite(rms)) return VRPS_OK;
  int e = (int)std::floor(std::log2(1024.0 / rms));
  if (e > 60) e = 60;
  if (e < -60) e = -60;
  *scale = (float)std::ldexp(1.0, e);
  return VRPS_OK;
}

int solver_alloc(vrps_geom* g, bool fista, bool bf16) {
  Workspace& w = g->ws;
  const size_t n = (size_t)g->n, m = (size_t)g->m;
  VRPS_TRY(ensure(&w.x, n));
  VRPS_TRY(ensure(&w.h, n));
  VRPS_TRY(ensure(&w.xhat, n));
  VRPS_TRY(ensure(&w.v, n));
  VRPS_TRY(ensure(&w.gbar, n));
  VRPS_TRY(ensure(&w.xprox, n));
  VRPS_TRY(ensure(&w.dual, (size_t)g->dims * n));
  VRPS_TRY(ensure(&w.b_perm, m));
  VRPS_TRY(ensure(&w.tab, m));
  VRPS_TRY(ensure(&w.res, m));
  VRPS_TRY(ensure(&w.sino, m));
  if (g->dims == 2) VRPS_TRY(ensure(&w.xfT, n));
  if (fista) VRPS_TRY(ensure(&w.xf, n));
  if (bf16) {
    VRPS_TRY(ensure(&w.b16, (m + 1) / 2));
    VRPS_TRY(ensure(&w.tab16, (m + 1) / 2));
  }
  return VRPS_OK;
}

}  // namespace vrps

using namespace vrps;

extern "C" void vrps_solve_opts_default(vrps_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->estimator = VRPS_EST_SVRG;
  o->fgp_iters = 50;
  o->max_iters = 100;
  o->nonneg = 1;
  o->power_iters = 100;
  o->eval_every = 0;
  o->f_star = 0.0;
  o->target_gap = 0.0;
}

extern "C" int vrps_solve(const float* b_in, const vrps_geom* gc, double alpha, int algo, double p,
                          double gamma, uint64_t seed, const vrps_solve_opts* opts, float* x_out,
                          vrps_report* rep, vrps_stream_t stream) {
  if (!gc) return fail(VRPS_ERR_INVALID_ARG, "geometry handle is NULL");
  if (!b_in || !x_out) return fail(VRPS_ERR_INVALID_ARG, "b or x_out is NULL");
  vrps_solve_opts o;
  if (opts) o = *opts;
  else vrps_solve_opts_default(&o);
  if (!(alpha >= 0) || !std::isfinite(alpha)) return fail(VRPS_ERR_INVALID_ARG, "alpha must be >= 0");
  if (algo < VRPS_ALGO_ISTA || algo > VRPS_ALGO_VR_PROXSKIP) return fail(VRPS_ERR_INVALID_ARG, "bad algo %d", algo);
  if (o.max_iters <= 0) return fail(VRPS_ERR_INVALID_ARG, "max_iters must be > 0");
  if (o.fgp_iters < 0) return fail(VRPS_ERR_INVALID_ARG, "fgp_iters must be >= 0");
  if (o.estimator < VRPS_EST_SVRG || o.estimator > VRPS_EST_SGD)
    return fail(VRPS_ERR_INVALID_ARG, "bad estimator %d", o.estimator);
  const bool skip = (algo == VRPS_ALGO_PROXSKIP || algo == VRPS_ALGO_VR_PROXSKIP);
  if (skip && !(p > 0.0 && p <= 1.0)) return fail(VRPS_ERR_INVALID_ARG, "p must be in (0, 1]");
  if (!skip) p = 1.0;
  if (!std::isfinite(gamma)) return fail(VRPS_ERR_INVALID_ARG, "gamma is not finite");
  if (o.history && o.history_cap <= 0) return fail(VRPS_ERR_INVALID_ARG, "history_cap must be > 0");
  if (o.storage < VRPS_STORAGE_FP32 || o.storage > VRPS_STORAGE_FP16)
    return fail(VRPS_ERR_INVALID_ARG, "bad storage %d", o.storage);
  if (o.correction_epochs < 0) return fail(VRPS_ERR_INVALID_ARG, "correction_epochs must be >= 0");
  vrps_geom* g = const_cast<vrps_geom*>(gc);
  {
    int dev = -1;
    VRPS_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return fail(VRPS_ERR_INVALID_ARG, "geometry belongs to device %d", g->device);
  }
  int est;
  switch (algo) {
    case VRPS_ALGO_SVRG: est = VRPS_EST_SVRG; break;
    case VRPS_ALGO_SAGA: est = VRPS_EST_SAGA; break;
    case VRPS_ALGO_VR_PROXSKIP: est = o.estimator; break;
    default: est = EST_FULL;
  }
  const bool fista = algo == VRPS_ALGO_FISTA;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace& w = g->ws;
  const bool bf_run = o.storage != VRPS_STORAGE_FP32;   // reduced-precision storage
  VRPS_TRY(solver_alloc(g, fista, bf_run));
  const int64_t n = g->n, m = g->m;
  const int L = g->row_len;

  // subset-major angle order for this solve's N
  int N = o.n_subsets > 0 ? o.n_subsets : g->n_subsets;
  if (N > g->n_angles) return fail(VRPS_ERR_INVALID_ARG, "n_subsets %d exceeds %d angles", N, g->n_angles);
  const int* order = g->order_subset;
  const std::vector<int>* off = &g->subset_off;
  if (N != g->n_subsets) {
    if (w.order_N != N) {
      VRPS_TRY(build_order(g->n_angles, N, &w.order_dev, &w.order_off));
      VRPS_TRY(build_order_angles(g, N, &w.ang_order_dev));
      w.order_N = N;
    }
    order = w.order_dev;
    off = &w.order_off;
  }

  // data: b (natural order, device or host) -> b_perm (subset-major)
  const float* b_dev = b_in;
  if (o.host_io) {
    VRPS_CUDA(cudaMemcpyAsync(w.sino, b_in, sizeof(float) * (size_t)m, cudaMemcpyHostToDevice, s));
    b_dev = w.sino;
  }
  VRPS_TRY(gather_rows(b_dev, w.b_perm, order, g->n_angles, L, s));
  // reduced storage: iterations k < kc read b and the estimator table as bfloat16 / float16
  const int K = o.max_iters;
  int kc = 0;
  float sc = 1.f;
  if (bf_run) {
    const long long corr = (long long)o.correction_epochs * N;
    kc = corr >= K ? 0 : (int)(K - corr);
    VRPS_TRY(storage_scale(g, o.storage, &sc, s));
    VRPS_TRY(to_store(w.b_perm, w.b16, m, o.storage, sc, s));
  }
  const float isc = 1.f / sc;

  // step size (Section 3)
  vrps_report r;
  std::memset(&r, 0, sizeof(r));
  r.objective = NAN;
  if (gamma <= 0.0) {
    double Lip = 0.0;
    VRPS_TRY(vrps_power_iteration(g, o.power_iters > 0 ? o.power_iters : 100, seed ^ 0x5bd1e995ull, &Lip, stream));
    if (!(Lip > 0.0) || !std::isfinite(Lip)) return fail(VRPS_ERR_DIVERGED, "power iteration gave L = %g", Lip);
    r.lipschitz = Lip;
    gamma = step_factor(algo, est) / Lip;
  }
  r.gamma = gamma;

  // state: x0 (or 0), h = 0, dual = 0
  float* x = w.x;
  float* xf = fista ? w.xf : w.x;   // image the gradient is taken at
  float* xfT = g->dims == 2 ? w.xfT : nullptr;
  if (o.x0 && o.host_io) {
    VRPS_CUDA(cudaMemcpyAsync(x, o.x0, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, s));
  } else {
    VRPS_TRY(copy_or_zero(x, o.x0, n, s));
  }
  if (fista) VRPS_CUDA(cudaMemcpyAsync(xf, x, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  if (xfT) VRPS_TRY(transpose2d(xf, xfT, g->ny, g->nx, s));
  VRPS_CUDA(cudaMemsetAsync(w.h, 0, sizeof(float) * (size_t)n, s));
  VRPS_CUDA(cudaMemsetAsync(w.dual, 0, sizeof(float) * (size_t)g->dims * (size_t)n, s));
  VRPS_CUDA(cudaMemcpyAsync(w.xprox, x, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, s));

  // draws
  if (w.sched_cap < K) {
    if (w.sched_dev) cudaFree(w.sched_dev);
    if (w.sched_host) cudaFreeHost(w.sched_host);
    w.sched_dev = nullptr;
    w.sched_host = nullptr;
    w.sched_cap = 0;
    VRPS_CUDA(cudaMalloc((void**)&w.sched_dev, sizeof(int32_t) * 3 * (size_t)K));
    VRPS_CUDA(cudaMallocHost((void**)&w.sched_host, sizeof(int32_t) * 3 * (size_t)K));
    w.sched_cap = K;
  }
  VRPS_TRY(philox_schedule(seed, o.job, 0, K, N, p, w.sched_dev, s));
  VRPS_CUDA(cudaMemcpyAsync(w.sched_host, w.sched_dev, sizeof(int32_t) * 3 * (size_t)K, cudaMemcpyDeviceToHost, s));

  // SAGA table at x0: rho = A x0 - b (subset-major), vbar = A^T rho
  if (est == VRPS_EST_SAGA) {
    FwdOut fo{w.tab, w.b_perm, nullptr};
    VRPS_TRY(proj_forward(g, xf, xfT, order, g->n_angles, FWD_RESID, fo, s));
    UpdateArgs ua;
    std::memset(&ua, 0, sizeof(ua));
    ua.out = w.gbar;
    VRPS_TRY(proj_adjoint(g, w.tab, order, g->n_angles, ua, s));
    if (kc > 0) VRPS_TRY(to_store(w.tab, w.tab16, m, o.storage, sc, s));
    r.passes += 1.0;
  }
  VRPS_CUDA(cudaStreamSynchronize(s));

  cudaEvent_t ev0, ev1;
  VRPS_CUDA(cudaEventCreate(&ev0));
  VRPS_CUDA(cudaEventCreate(&ev1));
  VRPS_CUDA(cudaEventRecord(ev0, s));
  // 3D: forwards that feed an adjoint leave the ray length factor on their residual
  const int pre = g->dims == 3 ? 1 : 0;
  const float tau = (float)(gamma * alpha / p);
  const float fgamma = (float)gamma, fgp = (float)(gamma / p), fpg = (float)(p / gamma);
  double t_fista = 1.0;
  int status = VRPS_OK;
  int k = 0;
  for (; k < K; ++k) {
    const int i = w.sched_host[3 * k + 0];
    const int theta = skip ? w.sched_host[3 * k + 1] : 1;
    const int coin = w.sched_host[3 * k + 2];
    const int* ids_i = order + (*off)[i];
    const int rows_i = (*off)[i + 1] - (*off)[i];
    const int bf = k < kc ? o.storage : STORE_F32;
    const size_t es = bf ? sizeof(__nv_bfloat16) : sizeof(float);
    char* const b_all = bf ? (char*)w.b16 : (char*)w.b_perm;
    char* const tab_all = bf ? (char*)w.tab16 : (char*)w.tab;
    char* b_i = b_all + es * (size_t)(*off)[i] * L;
    char* tab_i = tab_all + es * (size_t)(*off)[i] * L;
    bool force_refresh = false;
    if (bf_run && k == kc && kc > 0) {
      // switch to float32 storage from an exact float32 full gradient
      if (est == VRPS_EST_SAGA) {
        // rho = A x - b unscaled (the table), gbar = A^T rho
        FwdOut fo{w.tab, w.b_perm, nullptr};
        VRPS_TRY(proj_forward(g, xf, xfT, order, g->n_angles, FWD_RESID, fo, s));
        UpdateArgs ga;
        std::memset(&ga, 0, sizeof(ga));
        ga.out = w.gbar;
        VRPS_TRY(proj_adjoint(g, w.tab, order, g->n_angles, ga, s));
        r.passes += 1.0;
      } else {
        force_refresh = true;
      }
    }

    UpdateArgs ua;
    std::memset(&ua, 0, sizeof(ua));
    ua.enabled = 1;
    ua.prescaled = pre;
    ua.base = xf;
    ua.h = skip ? w.h : nullptr;
    ua.gamma = fgamma;
    ua.gamma_over_p = fgp;
    ua.theta = theta;
    ua.x = x;
    ua.xT = fista ? nullptr : xfT;
    ua.xhat = w.xhat;
    ua.v = w.v;

    if (est == EST_FULL) {
      FwdOut fo{w.res, b_all, nullptr, pre, bf, sc, isc};
      VRPS_TRY(proj_forward(g, xf, xfT, order, g->n_angles, FWD_RESID, fo, s));
      ua.cN = 1.f;
      VRPS_TRY(proj_adjoint(g, w.res, order, g->n_angles, ua, s));
      r.passes += 1.0;
    } else if (est == VRPS_EST_SGD) {
      FwdOut fo{w.res, b_i, nullptr, pre, bf, sc, isc};
      VRPS_TRY(proj_forward(g, xf, xfT, ids_i, rows_i, FWD_RESID, fo, s));
      ua.cN = (float)N;
      VRPS_TRY(proj_adjoint(g, w.res, ids_i, rows_i, ua, s));
      r.passes += 1.0 / N;
    } else if (est == VRPS_EST_SAGA) {
      FwdOut fo{w.res, b_i, tab_i, pre, bf, sc, isc};
      VRPS_TRY(proj_forward(g, xf, xfT, ids_i, rows_i, FWD_SAGA, fo, s));
      ua.cN = (float)N;
      ua.gbar = w.gbar;
      ua.saga = 1;
      VRPS_TRY(proj_adjoint(g, w.res, ids_i, rows_i, ua, s));
      r.passes += 1.0 / N;
    } else {  // SVRG / LSVRG
      const bool refresh = force_refresh || (est == VRPS_EST_SVRG ? (k % N == 0) : (k == 0 || coin != 0));
      if (refresh) {
        // snapshot x~ = x_k: store A x~ (subset-major), gbar = A^T (A x~ - b) and G = gbar,
        // the full adjoint's epilogue writing gbar and taking the step in one pass
        FwdOut fo{w.res, b_all, tab_all, pre, bf, sc, isc};
        VRPS_TRY(proj_forward(g, xf, xfT, order, g->n_angles, FWD_SNAP, fo, s));
        ua.cN = 0.f;
        ua.gbar = w.gbar;
        ua.snap = 1;
        VRPS_TRY(proj_adjoint(g, w.res, order, g->n_angles, ua, s));
        r.snapshots += 1;
        r.passes += 1.0;
      } else {
        FwdOut fo{w.res, nullptr, tab_i, pre, bf, sc, isc};
        VRPS_TRY(proj_forward(g, xf, xfT, ids_i, rows_i, FWD_SVRG, fo, s));
        ua.cN = (float)N;
        ua.gbar = w.gbar;
        VRPS_TRY(proj_adjoint(g, w.res, ids_i, rows_i, ua, s));
        r.passes += 1.0 / N;
      }
    }

    if (theta) {
      ProxTail t;
      std::memset(&t, 0, sizeof(t));
      t.mode = 1;
      t.x = x;
      t.xT = fista ? nullptr : xfT;
      t.h = skip ? w.h : nullptr;
      t.xhat = w.xhat;
      t.p_over_gamma = fpg;
      t.xprox = skip ? w.xprox : nullptr;
      if (fista) {
        const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t_fista * t_fista)) / 2.0;
        t.mom = (float)((t_fista - 1.0) / tn);
        t_fista = tn;
        t.y = xf;
        t.yT = xfT;
      }
      VRPS_TRY(fgp_run(g, w.v, tau, o.fgp_iters, o.nonneg ? 1 : 0, w.dual, t, s));
      r.prox_calls += 1;
    }

    if (o.eval_every > 0 && (k + 1) % o.eval_every == 0) {
      const float* xe = skip ? w.xprox : x;
      FwdOut fo{w.sino, w.b_perm, nullptr};
      VRPS_TRY(proj_forward(g, xe, nullptr, order, g->n_angles, FWD_RESID, fo, s));
      VRPS_TRY(dot64(w.sino, w.sino, m, w.scalars + 5, w, s));
      VRPS_TRY(tv64(g, xe, w.scalars + 6, w, s));
      double hv[2];
      VRPS_CUDA(cudaMemcpyAsync(hv, w.scalars + 5, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      cudaEvent_t ev2;
      VRPS_CUDA(cudaEventCreate(&ev2));
      VRPS_CUDA(cudaEventRecord(ev2, s));
      VRPS_CUDA(cudaEventSynchronize(ev2));
      float ms = 0.f;
      VRPS_CUDA(cudaEventElapsedTime(&ms, ev0, ev2));
      cudaEventDestroy(ev2);
      const double F = 0.5 * hv[0] + alpha * hv[1];
      r.objective = F;
      if (o.history && r.evaluations < o.history_cap) {
        double* row = o.history + 4 * (size_t)r.evaluations;
        row[0] = (double)(k + 1);
        row[1] = F;
        row[2] = ms * 1e-3;
        row[3] = r.passes;
      }
      r.evaluations += 1;
      if (!std::isfinite(F)) {
        status = fail(VRPS_ERR_DIVERGED, "objective is not finite at iteration %d", k + 1);
        ++k;
        break;
      }
      if (o.target_gap > 0.0 && o.f_star != 0.0 && (F - o.f_star) / std::fabs(o.f_star) <= o.target_gap) {
        r.reached = 1;
        ++k;
        break;
      }
    }
  }
  VRPS_CUDA(cudaEventRecord(ev1, s));
  VRPS_CUDA(cudaEventSynchronize(ev1));
  float ms = 0.f;
  VRPS_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  r.iterations = k;
  r.seconds = ms * 1e-3;
  if (o.host_io) {
    VRPS_CUDA(cudaMemcpyAsync(x_out, x, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost, s));
  } else {
    VRPS_CUDA(cudaMemcpyAsync(x_out, x, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  }
  VRPS_CUDA(cudaStreamSynchronize(s));
  {
    const int e = take_device_error(g);
    if (e != VRPS_OK) status = e;
  }
  if (rep) *rep = r;
  return status;
}
