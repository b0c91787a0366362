// Batched and served reconstruction: many VR-ProxSkip jobs (Algorithm 1 with a variance-
// reduced estimator), each on its own geometry and data, advance together.  A batch holds 2D
// jobs or 3D jobs (fixed by its first job).  One tick performs one iteration of every active
// job; each phase of a tick is ONE persistent launch over the tiles of all jobs, running the
// same per-tile device code as the single-job solver:
//   2D: subset forward with its estimator epilogue, adjoint with the fused update, every
//       blocked FGP launch of the prox calls due this tick, prox output;
//   3D: slice transpose of x, subset forward, adjoint with the fused update, every FGP
//       iteration of the prox calls due this tick, prox output.
// A job's arithmetic therefore does not depend on which other jobs share its ticks: its
// result is bit-identical alone, in any mix, and to vrps_solve with the same arguments.
//
// The host builds each tick's work list (per-job launch parameters and item prefix sums)
// from the jobs' precomputed Philox draws, packs it into a pinned buffer and copies it to a
// device slot; the tick's kernels read the slot.  With graphs enabled, the kernel sequence of
// each slot is captured once as a CUDA graph and replayed every tick that uses the slot
// (recaptured only when the batch's shared-memory or FGP-depth maxima grow).  Jobs are
// admitted between ticks (continuous batching) and leave at their last iteration.
#include <cmath>
#include <cstring>
#include <vector>

#include "vrps_internal.h"

namespace vrps {
namespace {

constexpr int SLOTS = 4;

struct Job {
  int id = 0;
  vrps_geom* g = nullptr;
  float* x_out = nullptr;
  double alpha = 0, p = 1, gamma = 0;
  int est = VRPS_EST_SVRG, fgp_iters = 0, K = 0, N = 1, nonneg = 1;
  bool bf_run = false;   // reduced-precision storage
  int store = 0;         // its StoreKind
  float sc = 1.f, isc = 1.f;
  int kc = 0;   // first iteration with float32 storage
  int k = 0;
  int state = 0;   // 0 running, 1 finished (kernels enqueued), 2 released
  std::vector<int32_t> sched;
  const int* order = nullptr;
  std::vector<int> off;
  float tau = 0, step = 0, fgamma = 0, fgp = 0, fpg = 0;
  vrps_report rep{};
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
};

struct Slot {
  char* pinned = nullptr;
  char* dev = nullptr;
  size_t cap = 0;
  cudaEvent_t free_ev = nullptr;
  bool used = false;
  cudaGraphExec_t graph = nullptr;
  int graph_blocks = -1;
  size_t graph_fwd_smem = 0, graph_adj_smem = 0;
  bool graph_grouped = false;
  cudaGraphExec_t graph_prox = nullptr;   // 3D: the prox launches, replayed on ticks with a prox call
  int graph_prox_iters = -1;
};

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

}  // namespace
}  // namespace vrps

using namespace vrps;

struct vrps_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;
  std::vector<Job*> jobs;   // every submitted job (index = id)
  std::vector<Job*> active;
  Slot slots[SLOTS];
  int slot_i = 0;
  int grid_fwd = 0, grid_adj = 0, grid_fgp = 0, grid_out = 0;
  size_t fwd_smem = 0, adj_smem = 0;
  bool fwd_grouped = false;   // some job's forward walks band groups
  int max_blocks = 0;
  bool graphs = true;
  long long ticks = 0;
  int dims = 0;                  // 2 or 3, set by the first job
  int grid3[5] = {0, 0, 0, 0, 0};   // 3D persistent grids: transpose, forward, adjoint, FGP, output
  int max_f3 = 0;                // 3D: most FGP iterations of any job (rows of the FGP prefix table)
  double share = 1.0;            // fraction of the resident CTA slots the persistent grids take
  std::vector<char> pack;
};

namespace {

// A persistent grid of `share` of the resident slots (at least one CTA).
int shared_grid(int grid, double share) {
  const int g = (int)(grid * share);
  return g < 1 ? 1 : g;
}

int batch_grids(vrps_batch* B) {
  VRPS_TRY(batched_grid(B->fwd_grouped ? 4 : 0, B->fwd_smem, &B->grid_fwd));
  VRPS_TRY(batched_grid(1, B->adj_smem, &B->grid_adj));
  VRPS_TRY(batched_grid(2, 0, &B->grid_fgp));
  VRPS_TRY(batched_grid(3, 0, &B->grid_out));
  B->grid_fwd = shared_grid(B->grid_fwd, B->share);
  B->grid_adj = shared_grid(B->grid_adj, B->share);
  B->grid_fgp = shared_grid(B->grid_fgp, B->share);
  B->grid_out = shared_grid(B->grid_out, B->share);
  return VRPS_OK;
}

// The tick's kernels on stream s, reading the work list at slot.
int launch_tick(vrps_batch* B, char* slot, cudaStream_t s) {
  VRPS_TRY(fwd2d_batched(slot, B->grid_fwd, B->fwd_smem, B->fwd_grouped, s));
  VRPS_TRY(adj2d_batched(slot, B->grid_adj, B->adj_smem, s));
  for (int b = 0; b < B->max_blocks; ++b) VRPS_TRY(fgp2d_block_batched(slot, b, B->grid_fgp, s));
  VRPS_TRY(fgp2d_out_batched(slot, B->grid_out, s));
  return VRPS_OK;
}

int tick_kernels(const vrps_batch* B) { return 3 + B->max_blocks; }

// Graph of the tick's kernels for one slot, captured on the batch's capture stream.
int ensure_graph(vrps_batch* B, Slot& S) {
  if (S.graph && S.graph_blocks == B->max_blocks && S.graph_fwd_smem == B->fwd_smem &&
      S.graph_adj_smem == B->adj_smem && S.graph_grouped == B->fwd_grouped)
    return VRPS_OK;
  if (S.graph) {
    cudaGraphExecDestroy(S.graph);
    S.graph = nullptr;
  }
  cudaGraph_t graph = nullptr;
  VRPS_CUDA(cudaStreamBeginCapture(B->capture, cudaStreamCaptureModeRelaxed));
  const int rc = launch_tick(B, S.dev, B->capture);
  const cudaError_t ec = cudaStreamEndCapture(B->capture, &graph);
  if (rc != VRPS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  VRPS_CUDA(ec);
  launch_count_add(-(long long)tick_kernels(B));   // counted per replay instead
  const cudaError_t ei = cudaGraphInstantiate(&S.graph, graph, 0);
  cudaGraphDestroy(graph);
  VRPS_CUDA(ei);
  S.graph_blocks = B->max_blocks;
  S.graph_fwd_smem = B->fwd_smem;
  S.graph_adj_smem = B->adj_smem;
  S.graph_grouped = B->fwd_grouped;
  return VRPS_OK;
}

// 3D ticks: the projection phase (every tick) and the prox phase (ticks with a prox call,
// `iters` FGP iteration launches then the output launch).
int launch_tick3_proj(vrps_batch* B, char* slot, cudaStream_t s) {
  VRPS_TRY(tr3_batched(slot, B->grid3[0], s));
  VRPS_TRY(fwd3d_batched(slot, B->grid3[1], s));
  VRPS_TRY(adj3d_batched(slot, B->grid3[2], s));
  return VRPS_OK;
}

int launch_tick3_prox(vrps_batch* B, char* slot, int iters, cudaStream_t s) {
  for (int it = 0; it < iters; ++it) VRPS_TRY(fgp3d_iter_batched(slot, it, B->grid3[3], s));
  VRPS_TRY(fgp3d_out_batched(slot, B->grid3[4], s));
  return VRPS_OK;
}

template <class F>
int capture(vrps_batch* B, cudaGraphExec_t* exec, int kernels, F&& body) {
  if (*exec) {
    cudaGraphExecDestroy(*exec);
    *exec = nullptr;
  }
  cudaGraph_t graph = nullptr;
  VRPS_CUDA(cudaStreamBeginCapture(B->capture, cudaStreamCaptureModeRelaxed));
  const int rc = body(B->capture);
  const cudaError_t ec = cudaStreamEndCapture(B->capture, &graph);
  if (rc != VRPS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  VRPS_CUDA(ec);
  launch_count_add(-(long long)kernels);   // counted per replay instead
  const cudaError_t ei = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  VRPS_CUDA(ei);
  return VRPS_OK;
}

int ensure_graph3(vrps_batch* B, Slot& S, bool prox) {
  if (!S.graph)
    VRPS_TRY(capture(B, &S.graph, 3, [&](cudaStream_t c) { return launch_tick3_proj(B, S.dev, c); }));
  if (prox && S.graph_prox_iters != B->max_f3) {
    VRPS_TRY(capture(B, &S.graph_prox, B->max_f3 + 1,
                     [&](cudaStream_t c) { return launch_tick3_prox(B, S.dev, B->max_f3, c); }));
    S.graph_prox_iters = B->max_f3;
  }
  return VRPS_OK;
}

// Job initialisation, identical to vrps_solve's for VR-ProxSkip (x0 = 0, h = 0, dual = 0).
int job_setup(vrps_batch* B, Job* J, const vrps_job* d) {
  vrps_geom* g = J->g;
  cudaStream_t s = B->stream;
  Workspace& w = g->ws;
  const int64_t n = g->n, m = g->m;
  const int L = g->row_len;
  const bool three = g->dims == 3;
  VRPS_TRY(solver_alloc(g, false, J->bf_run));
  VRPS_TRY(fgp_prepare(g));
  if (three) VRPS_TRY(ensure(&w.xT, (size_t)n));
  J->order = g->order_subset;
  J->off = g->subset_off;
  if (J->N != g->n_subsets) {
    if (w.order_N != J->N) {
      VRPS_TRY(build_order(g->n_angles, J->N, &w.order_dev, &w.order_off));
      VRPS_TRY(build_order_angles(g, J->N, &w.ang_order_dev));
      w.order_N = J->N;
    }
    J->order = w.order_dev;
    J->off = w.order_off;
  }
  VRPS_TRY(gather_rows(d->b, w.b_perm, J->order, g->n_angles, L, s));
  if (J->bf_run) {
    const long long corr = (long long)d->correction_epochs * J->N;
    J->kc = corr >= J->K ? 0 : (int)(J->K - corr);
    VRPS_TRY(storage_scale(g, J->store, &J->sc, s));
    J->isc = 1.f / J->sc;
    VRPS_TRY(to_store(w.b_perm, w.b16, m, J->store, J->sc, s));
  }
  VRPS_TRY(copy_or_zero(w.x, nullptr, n, s));
  if (!three) VRPS_TRY(transpose2d(w.x, w.xfT, g->ny, g->nx, s));
  VRPS_CUDA(cudaMemsetAsync(w.h, 0, sizeof(float) * (size_t)n, s));
  VRPS_CUDA(cudaMemsetAsync(w.dual, 0, sizeof(float) * g->dims * (size_t)n, s));
  VRPS_CUDA(cudaMemcpyAsync(w.xprox, w.x, sizeof(float) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  // draws, copied to the host once
  if (w.sched_cap < J->K) {
    if (w.sched_dev) cudaFree(w.sched_dev);
    if (w.sched_host) cudaFreeHost(w.sched_host);
    w.sched_dev = nullptr;
    w.sched_host = nullptr;
    w.sched_cap = 0;
    VRPS_CUDA(cudaMalloc((void**)&w.sched_dev, sizeof(int32_t) * 3 * (size_t)J->K));
    VRPS_CUDA(cudaMallocHost((void**)&w.sched_host, sizeof(int32_t) * 3 * (size_t)J->K));
    w.sched_cap = J->K;
  }
  VRPS_TRY(philox_schedule(d->seed, d->job, 0, J->K, J->N, J->p, w.sched_dev, s));
  VRPS_CUDA(cudaMemcpyAsync(w.sched_host, w.sched_dev, sizeof(int32_t) * 3 * (size_t)J->K, cudaMemcpyDeviceToHost,
                            s));
  if (J->est == VRPS_EST_SAGA) {
    FwdOut fo{w.tab, w.b_perm, nullptr};
    VRPS_TRY(proj_forward(g, w.x, three ? nullptr : w.xfT, J->order, g->n_angles, FWD_RESID, fo, s));
    UpdateArgs ua;
    std::memset(&ua, 0, sizeof(ua));
    ua.out = w.gbar;
    VRPS_TRY(proj_adjoint(g, w.tab, J->order, g->n_angles, ua, s));
    if (J->kc > 0) VRPS_TRY(to_store(w.tab, w.tab16, m, J->store, J->sc, s));
    J->rep.passes += 1.0;
  }
  VRPS_CUDA(cudaStreamSynchronize(s));
  J->sched.assign(w.sched_host, w.sched_host + 3 * (size_t)J->K);
  if (three) {
    if (J->fgp_iters > B->max_f3) B->max_f3 = J->fgp_iters;
    if (B->grid3[0] == 0)
      for (int q = 0; q < 5; ++q) {
        VRPS_TRY(batched_grid_3d(q, &B->grid3[q]));
        B->grid3[q] = shared_grid(B->grid3[q], B->share);
      }
    VRPS_CUDA(cudaEventCreate(&J->ev_start));
    VRPS_CUDA(cudaEventCreate(&J->ev_done));
    VRPS_CUDA(cudaEventRecord(J->ev_start, s));
    return VRPS_OK;
  }
  // launch constants for the batch's shared-memory maxima, over the all-angle and the subset
  // passes (their launch shapes can differ) -- this also sizes the job's partial-sum buffers
  bool regrid = false;
  for (int pass = 0; pass < 2; ++pass) {
    const int* ids = pass == 0 ? J->order : J->order + J->off[0];
    const int rows = pass == 0 ? g->n_angles : J->off[1] - J->off[0];
    Fwd2DParams fp;
    size_t fs = 0;
    bool bulk = false;
    FwdOut fo{w.res, w.b_perm, w.tab};
    VRPS_TRY(fwd2d_setup(g, w.x, w.xfT, ids, rows, fo, &fp, &fs, &bulk));
    Adj2DParams ap;
    size_t as = 0;
    int var = 0, tx = 0, ty = 0;
    UpdateArgs ua;
    std::memset(&ua, 0, sizeof(ua));
    VRPS_TRY(adj2d_setup(g, w.res, ids, rows, ua, &ap, &as, &var, &tx, &ty));
    if (fs > B->fwd_smem) {
      B->fwd_smem = fs;
      regrid = true;
    }
    if (fp.group > 1 && bulk && !B->fwd_grouped) {
      B->fwd_grouped = true;
      regrid = true;
    }
    if (as > B->adj_smem) {
      B->adj_smem = as;
      regrid = true;
    }
  }
  const int nb = (J->fgp_iters + FB_T - 1) / FB_T;
  if (nb > B->max_blocks) B->max_blocks = nb;
  if (regrid || B->grid_fwd == 0) VRPS_TRY(batch_grids(B));
  VRPS_CUDA(cudaEventCreate(&J->ev_start));
  VRPS_CUDA(cudaEventCreate(&J->ev_done));
  VRPS_CUDA(cudaEventRecord(J->ev_start, s));
  return VRPS_OK;
}

// Iteration J->k of job J (Algorithm 1, as in vrps_solve): which forward, on which rows,
// with which estimator epilogue and update; the SAGA switch to float32 storage is enqueued
// here, before the tick's kernels.
struct Plan {
  int mode;
  const int* ids;
  int rows;
  FwdOut fo;
  UpdateArgs ua;
  int theta;
};

int job_plan(vrps_batch* B, Job* J, Plan* P) {
  vrps_geom* g = J->g;
  Workspace& w = g->ws;
  const bool three = g->dims == 3;
  const int pre = three ? 1 : 0;   // 3D forwards leave the ray length factor on the residual
  float* const xT = three ? nullptr : w.xfT;
  const int k = J->k;
  const int N = J->N;
  const int L = g->row_len;
  const int i = J->sched[3 * (size_t)k + 0];
  const int theta = J->sched[3 * (size_t)k + 1];
  const int coin = J->sched[3 * (size_t)k + 2];
  const int* ids_i = J->order + J->off[i];
  const int rows_i = J->off[i + 1] - J->off[i];
  const int bf = k < J->kc ? J->store : STORE_F32;
  const size_t es = bf ? sizeof(__nv_bfloat16) : sizeof(float);
  char* const b_all = bf ? (char*)w.b16 : (char*)w.b_perm;
  char* const tab_all = bf ? (char*)w.tab16 : (char*)w.tab;
  char* b_i = b_all + es * (size_t)J->off[i] * L;
  char* tab_i = tab_all + es * (size_t)J->off[i] * L;
  bool force_refresh = false;
  if (J->bf_run && k == J->kc && J->kc > 0) {
    if (J->est == VRPS_EST_SAGA) {
      // switch to float32 storage: rho = A x - b, gbar = A^T rho (before this tick's kernels)
      FwdOut fo{w.tab, w.b_perm, nullptr};
      VRPS_TRY(proj_forward(g, w.x, xT, J->order, g->n_angles, FWD_RESID, fo, B->stream));
      UpdateArgs ga;
      std::memset(&ga, 0, sizeof(ga));
      ga.out = w.gbar;
      VRPS_TRY(proj_adjoint(g, w.tab, J->order, g->n_angles, ga, B->stream));
      J->rep.passes += 1.0;
    } else {
      force_refresh = true;
    }
  }
  UpdateArgs& ua = P->ua;
  std::memset(&ua, 0, sizeof(ua));
  ua.enabled = 1;
  ua.prescaled = pre;
  ua.base = w.x;
  ua.h = w.h;
  ua.gamma = J->fgamma;
  ua.gamma_over_p = J->fgp;
  ua.theta = theta;
  ua.x = w.x;
  ua.xT = xT;
  ua.xhat = w.xhat;
  ua.v = w.v;
  P->ids = ids_i;
  P->rows = rows_i;
  P->theta = theta;
  P->fo = FwdOut{w.res, nullptr, nullptr, pre, bf, J->sc, J->isc};
  if (J->est == VRPS_EST_SGD) {
    P->mode = FWD_RESID;
    P->fo.b = b_i;
    ua.cN = (float)N;
    J->rep.passes += 1.0 / N;
  } else if (J->est == VRPS_EST_SAGA) {
    P->mode = FWD_SAGA;
    P->fo.b = b_i;
    P->fo.tab = tab_i;
    ua.cN = (float)N;
    ua.gbar = w.gbar;
    ua.saga = 1;
    J->rep.passes += 1.0 / N;
  } else {
    const bool refresh = force_refresh || (J->est == VRPS_EST_SVRG ? (k % N == 0) : (k == 0 || coin != 0));
    if (refresh) {
      P->mode = FWD_SNAP;
      P->fo.b = b_all;
      P->fo.tab = tab_all;
      P->ids = J->order;
      P->rows = g->n_angles;
      ua.cN = 0.f;
      ua.gbar = w.gbar;
      ua.snap = 1;
      J->rep.snapshots += 1;
      J->rep.passes += 1.0;
    } else {
      P->mode = FWD_SVRG;
      P->fo.tab = tab_i;
      ua.cN = (float)N;
      ua.gbar = w.gbar;
      J->rep.passes += 1.0 / N;
    }
  }
  return VRPS_OK;
}

ProxTail prox_tail(Job* J) {
  Workspace& w = J->g->ws;
  ProxTail t;
  std::memset(&t, 0, sizeof(t));
  t.mode = 1;
  t.x = w.x;
  t.xT = J->g->dims == 2 ? w.xfT : nullptr;
  t.h = w.h;
  t.xhat = w.xhat;
  t.p_over_gamma = J->fpg;
  t.xprox = w.xprox;
  return t;
}

void job_advance(Job* J, bool prox) {
  if (prox) J->rep.prox_calls += 1;
  J->k += 1;
  J->rep.iterations = J->k;
}

// Work-list entries of a 2D job for its iteration J->k.
struct Entries {
  BatchFwd f;
  int f_items;
  BatchAdj a;
  int a_items;
  bool prox;
  BatchFgp fg;
  int fg_items;
  BatchOut o;
  int o_items;
};

int job_tick(vrps_batch* B, Job* J, Entries* E) {
  vrps_geom* g = J->g;
  Workspace& w = g->ws;
  Plan P;
  VRPS_TRY(job_plan(B, J, &P));
  size_t sm = 0;
  bool bulk = false;
  VRPS_TRY(fwd2d_setup(g, w.x, w.xfT, P.ids, P.rows, P.fo, &E->f.P, &sm, &bulk));
  // the batch's launches were sized at admission; a launch shape changed since cannot run
  if (sm > B->fwd_smem || (E->f.P.group > 1 && bulk && !B->fwd_grouped))
    return fail(VRPS_ERR_INVALID_ARG, "job %d: its geometry's launch shape changed while the job runs", J->id);
  E->f.mode = P.mode;
  E->f.bulk = bulk ? 1 : 0;
  E->f_items = E->f.P.bands * P.rows;
  int var = 0, tx = 0, ty = 0;
  VRPS_TRY(adj2d_setup(g, w.res, P.ids, P.rows, P.ua, &E->a.P, &sm, &var, &tx, &ty));
  if (sm > B->adj_smem)
    return fail(VRPS_ERR_INVALID_ARG, "job %d: its geometry's launch shape changed while the job runs", J->id);
  E->a.variant = var;
  E->a.tiles_x = tx;
  E->a_items = tx * ty * E->a.P.split;
  E->prox = P.theta != 0;
  E->fg_items = 0;
  E->o_items = 0;
  if (E->prox) {
    const int ftx = (g->nx + FGP_TILE - 1) / FGP_TILE, fty = (g->ny + FGP_TILE - 1) / FGP_TILE;
    float* pairs[2][2] = {{w.dual_s1, w.dual_s2}, {w.dual_s3, w.dual_s4}};
    const std::vector<MomBlock> moms = fgp_momentum(J->fgp_iters);
    const int nb = (int)moms.size();
    std::memset(&E->fg, 0, sizeof(E->fg));
    E->fg.nblocks = nb;
    E->fg.tiles_x = ftx;
    const float* rw = w.dual;
    const float* rz = w.dual;
    for (int b = 0; b < nb; ++b) {
      const int k0 = b * FB_T;
      const int ns = J->fgp_iters - k0 < FB_T ? J->fgp_iters - k0 : FB_T;
      float* wn = pairs[b & 1][0];
      float* zn = pairs[b & 1][1];
      E->fg.A[b] = FgpBlockArgs{w.v, rw, rz, wn, zn, g->nx, g->ny, J->tau, J->step, moms[b], ns, J->nonneg};
      rw = wn;
      rz = zn;
    }
    E->fg_items = ftx * fty;
    float* wdst = (rw != w.dual) ? w.dual : nullptr;
    E->o.A = FgpOutArgs{w.v, rw, wdst, g->nx, g->ny, J->tau, J->nonneg, prox_tail(J)};
    E->o.tiles_x = ftx;
    E->o_items = ftx * fty;
  }
  job_advance(J, E->prox);
  return VRPS_OK;
}

// Work-list entries of a 3D job for its iteration J->k.
struct Entries3 {
  BatchTr3 tr;
  int tr_items;
  BatchFwd3 f;
  int f_items;
  BatchAdj3 a;
  int a_items;
  bool prox;
  BatchFgp3 fg;
  int fg_items;
  BatchOut3 o;
  int o_items;
};

int job_tick3(vrps_batch* B, Job* J, Entries3* E) {
  vrps_geom* g = J->g;
  Workspace& w = g->ws;
  Plan P;
  VRPS_TRY(job_plan(B, J, &P));
  VRPS_TRY(tr3_batch_entry(w.x, w.xT, g->nx, g->ny, g->nz, &E->tr, &E->tr_items));
  VRPS_TRY(fwd3d_batch_entry(g, w.x, w.xT, P.ids, P.rows, P.mode, P.fo, &E->f, &E->f_items));
  VRPS_TRY(adj3d_batch_entry(g, w.res, P.ids, P.rows, P.ua, &E->a, &E->a_items));
  E->prox = P.theta != 0;
  E->fg_items = 0;
  E->o_items = 0;
  if (E->prox)
    VRPS_TRY(fgp3d_batch_entry(g, w.v, J->tau, J->fgp_iters, J->nonneg, w.dual, prox_tail(J), &E->fg, &E->fg_items,
                               &E->o, &E->o_items));
  job_advance(J, E->prox);
  return VRPS_OK;
}

// Packs the entries of the tick into B->pack; returns the packed size.
size_t pack_tick(vrps_batch* B, const std::vector<Entries>& E) {
  const int n = (int)E.size();
  int np = 0;
  for (const Entries& e : E) np += e.prox ? 1 : 0;
  TickHeader H;
  std::memset(&H, 0, sizeof(H));
  H.n_fwd = n;
  H.n_adj = n;
  H.n_prox = np;
  size_t off = align16(sizeof(TickHeader));
  H.off_fwd = (unsigned)off;
  off = align16(off + sizeof(BatchFwd) * n);
  H.off_pfwd = (unsigned)off;
  off = align16(off + sizeof(int) * (n + 1));
  H.off_adj = (unsigned)off;
  off = align16(off + sizeof(BatchAdj) * n);
  H.off_padj = (unsigned)off;
  off = align16(off + sizeof(int) * (n + 1));
  H.off_fgp = (unsigned)off;
  off = align16(off + sizeof(BatchFgp) * np);
  H.off_pfgp = (unsigned)off;
  off = align16(off + sizeof(int) * BATCH_MAX_BLOCKS * (np + 1));
  H.off_out = (unsigned)off;
  off = align16(off + sizeof(BatchOut) * np);
  H.off_pout = (unsigned)off;
  off = align16(off + sizeof(int) * (np + 1));
  B->pack.assign(off, 0);
  char* base = B->pack.data();
  std::memcpy(base, &H, sizeof(H));
  BatchFwd* F = reinterpret_cast<BatchFwd*>(base + H.off_fwd);
  int* pf = reinterpret_cast<int*>(base + H.off_pfwd);
  BatchAdj* A = reinterpret_cast<BatchAdj*>(base + H.off_adj);
  int* pa = reinterpret_cast<int*>(base + H.off_padj);
  BatchFgp* G = reinterpret_cast<BatchFgp*>(base + H.off_fgp);
  int* pg = reinterpret_cast<int*>(base + H.off_pfgp);
  BatchOut* O = reinterpret_cast<BatchOut*>(base + H.off_out);
  int* po = reinterpret_cast<int*>(base + H.off_pout);
  pf[0] = pa[0] = po[0] = 0;
  for (int b = 0; b < BATCH_MAX_BLOCKS; ++b) pg[(size_t)b * (np + 1)] = 0;
  int q = 0;
  for (int j = 0; j < n; ++j) {
    const Entries& e = E[j];
    F[j] = e.f;
    pf[j + 1] = pf[j] + e.f_items;
    A[j] = e.a;
    pa[j + 1] = pa[j] + e.a_items;
    if (e.prox) {
      G[q] = e.fg;
      O[q] = e.o;
      po[q + 1] = po[q] + e.o_items;
      for (int b = 0; b < BATCH_MAX_BLOCKS; ++b) {
        int* row = pg + (size_t)b * (np + 1);
        row[q + 1] = row[q] + (b < e.fg.nblocks ? e.fg_items : 0);
      }
      ++q;
    }
  }
  return off;
}

// Packs the entries of a 3D tick into B->pack; returns the packed size.  The FGP prefix
// table has one row per iteration up to the batch's deepest prox.
size_t pack_tick3(vrps_batch* B, const std::vector<Entries3>& E) {
  const int n = (int)E.size();
  int np = 0;
  for (const Entries3& e : E) np += e.prox ? 1 : 0;
  const int rows = B->max_f3 > 0 ? B->max_f3 : 1;
  TickHeader3 H;
  std::memset(&H, 0, sizeof(H));
  H.n_jobs = n;
  H.n_prox = np;
  size_t off = align16(sizeof(TickHeader3));
  H.off_tr = (unsigned)off;
  off = align16(off + sizeof(BatchTr3) * n);
  H.off_ptr = (unsigned)off;
  off = align16(off + sizeof(int) * (n + 1));
  H.off_fwd = (unsigned)off;
  off = align16(off + sizeof(BatchFwd3) * n);
  H.off_pfwd = (unsigned)off;
  off = align16(off + sizeof(int) * (n + 1));
  H.off_adj = (unsigned)off;
  off = align16(off + sizeof(BatchAdj3) * n);
  H.off_padj = (unsigned)off;
  off = align16(off + sizeof(int) * (n + 1));
  H.off_fgp = (unsigned)off;
  off = align16(off + sizeof(BatchFgp3) * np);
  H.off_pfgp = (unsigned)off;
  off = align16(off + sizeof(int) * (size_t)rows * (np + 1));
  H.off_out = (unsigned)off;
  off = align16(off + sizeof(BatchOut3) * np);
  H.off_pout = (unsigned)off;
  off = align16(off + sizeof(int) * (np + 1));
  B->pack.assign(off, 0);
  char* base = B->pack.data();
  std::memcpy(base, &H, sizeof(H));
  BatchTr3* T = reinterpret_cast<BatchTr3*>(base + H.off_tr);
  int* pt = reinterpret_cast<int*>(base + H.off_ptr);
  BatchFwd3* F = reinterpret_cast<BatchFwd3*>(base + H.off_fwd);
  int* pf = reinterpret_cast<int*>(base + H.off_pfwd);
  BatchAdj3* A = reinterpret_cast<BatchAdj3*>(base + H.off_adj);
  int* pa = reinterpret_cast<int*>(base + H.off_padj);
  BatchFgp3* G = reinterpret_cast<BatchFgp3*>(base + H.off_fgp);
  int* pg = reinterpret_cast<int*>(base + H.off_pfgp);
  BatchOut3* O = reinterpret_cast<BatchOut3*>(base + H.off_out);
  int* po = reinterpret_cast<int*>(base + H.off_pout);
  pt[0] = pf[0] = pa[0] = po[0] = 0;
  for (int it = 0; it < rows; ++it) pg[(size_t)it * (np + 1)] = 0;
  int q = 0;
  for (int j = 0; j < n; ++j) {
    const Entries3& e = E[j];
    T[j] = e.tr;
    pt[j + 1] = pt[j] + e.tr_items;
    F[j] = e.f;
    pf[j + 1] = pf[j] + e.f_items;
    A[j] = e.a;
    pa[j + 1] = pa[j] + e.a_items;
    if (e.prox) {
      G[q] = e.fg;
      O[q] = e.o;
      po[q + 1] = po[q] + e.o_items;
      for (int it = 0; it < rows; ++it) {
        int* row = pg + (size_t)it * (np + 1);
        row[q + 1] = row[q] + (it < e.fg.iters ? e.fg_items : 0);
      }
      ++q;
    }
  }
  return off;
}

int run_tick(vrps_batch* B) {
  Slot& S = B->slots[B->slot_i];
  B->slot_i = (B->slot_i + 1) % SLOTS;
  if (S.used) VRPS_CUDA(cudaEventSynchronize(S.free_ev));   // its pinned and device buffers are free
  const bool three = B->dims == 3;
  std::vector<Job*> finishing;
  size_t bytes = 0;
  int prox_iters = 0;   // 3D: FGP iterations of this tick's deepest prox call
  bool any_prox = false;
  if (three) {
    std::vector<Entries3> E(B->active.size());
    for (size_t j = 0; j < B->active.size(); ++j) {
      Job* J = B->active[j];
      VRPS_TRY(job_tick3(B, J, &E[j]));
      if (E[j].prox) {
        any_prox = true;
        if (E[j].fg.iters > prox_iters) prox_iters = E[j].fg.iters;
      }
      if (J->k >= J->K) finishing.push_back(J);
    }
    bytes = pack_tick3(B, E);
  } else {
    std::vector<Entries> E(B->active.size());
    for (size_t j = 0; j < B->active.size(); ++j) {
      Job* J = B->active[j];
      VRPS_TRY(job_tick(B, J, &E[j]));
      if (J->k >= J->K) finishing.push_back(J);
    }
    bytes = pack_tick(B, E);
  }
  if (bytes > S.cap) {
    if (S.pinned) cudaFreeHost(S.pinned);
    if (S.dev) cudaFree(S.dev);
    S.pinned = nullptr;
    S.dev = nullptr;
    if (S.graph) {
      cudaGraphExecDestroy(S.graph);
      S.graph = nullptr;
    }
    if (S.graph_prox) {
      cudaGraphExecDestroy(S.graph_prox);
      S.graph_prox = nullptr;
      S.graph_prox_iters = -1;
    }
    const size_t cap = bytes * 2 > (size_t)(256 << 10) ? bytes * 2 : (size_t)(256 << 10);
    VRPS_CUDA(cudaMallocHost((void**)&S.pinned, cap));
    VRPS_CUDA(cudaMalloc((void**)&S.dev, cap));
    S.cap = cap;
  }
  std::memcpy(S.pinned, B->pack.data(), bytes);
  VRPS_CUDA(cudaMemcpyAsync(S.dev, S.pinned, bytes, cudaMemcpyHostToDevice, B->stream));
  const bool graphs = B->graphs && !profiling_on();
  if (three) {
    if (graphs) {
      VRPS_TRY(ensure_graph3(B, S, any_prox));
      VRPS_CUDA(cudaGraphLaunch(S.graph, B->stream));
      launch_count_add(3);
      if (any_prox) {
        VRPS_CUDA(cudaGraphLaunch(S.graph_prox, B->stream));
        launch_count_add(B->max_f3 + 1);
      }
    } else {
      VRPS_TRY(launch_tick3_proj(B, S.dev, B->stream));
      if (any_prox) VRPS_TRY(launch_tick3_prox(B, S.dev, prox_iters, B->stream));
    }
  } else if (graphs) {
    VRPS_TRY(ensure_graph(B, S));
    VRPS_CUDA(cudaGraphLaunch(S.graph, B->stream));
    launch_count_add(tick_kernels(B));
  } else {
    VRPS_TRY(launch_tick(B, S.dev, B->stream));
  }
  if (!S.free_ev) VRPS_CUDA(cudaEventCreateWithFlags(&S.free_ev, cudaEventDisableTiming));
  VRPS_CUDA(cudaEventRecord(S.free_ev, B->stream));
  S.used = true;
  for (Job* J : finishing) {
    Workspace& w = J->g->ws;
    VRPS_CUDA(cudaMemcpyAsync(J->x_out, w.x, sizeof(float) * (size_t)J->g->n, cudaMemcpyDeviceToDevice, B->stream));
    VRPS_CUDA(cudaEventRecord(J->ev_done, B->stream));
    J->state = 1;
  }
  if (!finishing.empty()) {
    std::vector<Job*> keep;
    for (Job* J : B->active)
      if (J->state == 0) keep.push_back(J);
    B->active.swap(keep);
  }
  B->ticks += 1;
  return VRPS_OK;
}

int job_report(Job* J, vrps_report* rep) {
  vrps_report r = J->rep;
  float ms = 0.f;
  VRPS_CUDA(cudaEventElapsedTime(&ms, J->ev_start, J->ev_done));
  r.seconds = ms * 1e-3;
  r.gamma = J->gamma;
  r.objective = NAN;
  if (rep) *rep = r;
  Workspace& w = J->g->ws;
  if (w.dev_error) {
    unsigned err = 0;
    VRPS_CUDA(cudaMemcpy(&err, w.dev_error, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (err) {
      VRPS_CUDA(cudaMemset(w.dev_error, 0, sizeof(unsigned)));
      return fail(VRPS_ERR_TIMEOUT, "job %d: a bounded device-side wait expired (error word %u)", J->id, err);
    }
  }
  return VRPS_OK;
}

Job* find_job(vrps_batch* B, int id) {
  if (!B || id < 0 || id >= (int)B->jobs.size()) return nullptr;
  return B->jobs[id];
}

}  // namespace

extern "C" {

int vrps_batch_create(vrps_batch** out) {
  if (!out) return fail(VRPS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  vrps_batch* B = new (std::nothrow) vrps_batch();
  if (!B) return fail(VRPS_ERR_OUT_OF_MEMORY, "batch");
  if (cudaGetDevice(&B->device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&B->capture, cudaStreamNonBlocking) != cudaSuccess) {
    if (B->stream) cudaStreamDestroy(B->stream);
    delete B;
    return fail(VRPS_ERR_CUDA, "batch stream creation failed");
  }
  *out = B;
  return VRPS_OK;
}

int vrps_batch_free(vrps_batch* B) {
  if (!B) return VRPS_OK;
  cudaStreamSynchronize(B->stream);
  for (Slot& S : B->slots) {
    if (S.graph) cudaGraphExecDestroy(S.graph);
    if (S.graph_prox) cudaGraphExecDestroy(S.graph_prox);
    if (S.pinned) cudaFreeHost(S.pinned);
    if (S.dev) cudaFree(S.dev);
    if (S.free_ev) cudaEventDestroy(S.free_ev);
  }
  for (Job* J : B->jobs) {
    if (!J) continue;
    if (J->ev_start) cudaEventDestroy(J->ev_start);
    if (J->ev_done) cudaEventDestroy(J->ev_done);
    delete J;
  }
  cudaStreamDestroy(B->stream);
  cudaStreamDestroy(B->capture);
  delete B;
  return VRPS_OK;
}

int vrps_batch_set_graphs(vrps_batch* B, int on) {
  if (!B) return fail(VRPS_ERR_INVALID_ARG, "batch is NULL");
  B->graphs = on != 0;
  return VRPS_OK;
}

int vrps_batch_set_stream_priority(vrps_batch* B, int priority) {
  if (!B) return fail(VRPS_ERR_INVALID_ARG, "batch is NULL");
  if (!B->jobs.empty()) return fail(VRPS_ERR_INVALID_ARG, "the stream priority is set before the first job");
  int lo = 0, hi = 0;   // numerically: lo = lowest priority (largest value), hi = highest
  VRPS_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  if (priority > lo) priority = lo;
  if (priority < hi) priority = hi;
  cudaStream_t s = nullptr;
  VRPS_CUDA(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, priority));
  VRPS_CUDA(cudaStreamSynchronize(B->stream));
  cudaStreamDestroy(B->stream);
  B->stream = s;
  return VRPS_OK;
}

int vrps_batch_set_grid_share(vrps_batch* B, double share) {
  if (!B) return fail(VRPS_ERR_INVALID_ARG, "batch is NULL");
  if (!(share > 0.0 && share <= 1.0)) return fail(VRPS_ERR_INVALID_ARG, "share must be in (0, 1]");
  if (!B->jobs.empty()) return fail(VRPS_ERR_INVALID_ARG, "the grid share is set before the first job");
  B->share = share;
  return VRPS_OK;
}

int vrps_batch_submit(vrps_batch* B, const vrps_job* d, int* id) {
  if (!B || !d || !id) return fail(VRPS_ERR_INVALID_ARG, "batch, job or id is NULL");
  *id = -1;
  vrps_geom* g = const_cast<vrps_geom*>(d->geom);
  if (!g) return fail(VRPS_ERR_INVALID_ARG, "job geometry is NULL");
  if (B->dims != 0 && g->dims != B->dims)
    return fail(VRPS_ERR_INVALID_ARG, "this batch holds %dD jobs, the job is %dD", B->dims, g->dims);
  if (g->device != B->device) return fail(VRPS_ERR_INVALID_ARG, "geometry and batch are on different devices");
  if (!d->b || !d->x_out) return fail(VRPS_ERR_INVALID_ARG, "job b or x_out is NULL");
  if (!(d->alpha >= 0) || !std::isfinite(d->alpha)) return fail(VRPS_ERR_INVALID_ARG, "alpha must be >= 0");
  if (!(d->p > 0.0 && d->p <= 1.0)) return fail(VRPS_ERR_INVALID_ARG, "p must be in (0, 1]");
  if (!(d->gamma > 0.0) || !std::isfinite(d->gamma)) return fail(VRPS_ERR_INVALID_ARG, "gamma must be > 0");
  if (d->max_iters <= 0) return fail(VRPS_ERR_INVALID_ARG, "max_iters must be > 0");
  const int max_fgp = g->dims == 3 ? BATCH3_MAX_ITERS : BATCH_MAX_FGP_ITERS;
  if (d->fgp_iters < 0 || d->fgp_iters > max_fgp)
    return fail(VRPS_ERR_INVALID_ARG, "fgp_iters must be in [0, %d]", max_fgp);
  if (d->estimator < VRPS_EST_SVRG || d->estimator > VRPS_EST_SGD)
    return fail(VRPS_ERR_INVALID_ARG, "bad estimator %d", d->estimator);
  if (d->storage < VRPS_STORAGE_FP32 || d->storage > VRPS_STORAGE_FP16)
    return fail(VRPS_ERR_INVALID_ARG, "bad storage %d", d->storage);
  if (d->correction_epochs < 0) return fail(VRPS_ERR_INVALID_ARG, "correction_epochs must be >= 0");
  const int N = d->n_subsets > 0 ? d->n_subsets : g->n_subsets;
  if (N > g->n_angles) return fail(VRPS_ERR_INVALID_ARG, "n_subsets %d exceeds %d angles", N, g->n_angles);
  if ((int)B->active.size() >= BATCH_MAX_JOBS) return fail(VRPS_ERR_UNSUPPORTED, "batch is full (%d jobs)", BATCH_MAX_JOBS);
  for (Job* A : B->active)
    if (A->g == g) return fail(VRPS_ERR_INVALID_ARG, "geometry is in use by running job %d", A->id);
  Job* J = new (std::nothrow) Job();
  if (!J) return fail(VRPS_ERR_OUT_OF_MEMORY, "job");
  J->id = (int)B->jobs.size();
  J->g = g;
  J->x_out = d->x_out;
  J->alpha = d->alpha;
  J->p = d->p;
  J->gamma = d->gamma;
  J->est = d->estimator;
  J->fgp_iters = d->fgp_iters;
  J->K = d->max_iters;
  J->N = N;
  J->nonneg = d->nonneg ? 1 : 0;
  J->bf_run = d->storage != VRPS_STORAGE_FP32;
  J->store = d->storage;
  J->tau = (float)(d->gamma * d->alpha / d->p);
  J->step = (float)(1.0 / (4.0 * g->dims * (double)J->tau));
  J->fgamma = (float)d->gamma;
  J->fgp = (float)(d->gamma / d->p);
  J->fpg = (float)(d->p / d->gamma);
  J->rep.objective = NAN;
  const int rc = job_setup(B, J, d);
  if (rc != VRPS_OK) {
    if (J->ev_start) cudaEventDestroy(J->ev_start);
    if (J->ev_done) cudaEventDestroy(J->ev_done);
    delete J;
    return rc;
  }
  B->dims = g->dims;
  B->jobs.push_back(J);
  B->active.push_back(J);
  *id = J->id;
  return VRPS_OK;
}

int vrps_batch_step(vrps_batch* B, int ticks, int* active) {
  if (!B) return fail(VRPS_ERR_INVALID_ARG, "batch is NULL");
  for (int t = 0; t < ticks && !B->active.empty(); ++t) VRPS_TRY(run_tick(B));
  if (active) *active = (int)B->active.size();
  return VRPS_OK;
}

int vrps_batch_poll(vrps_batch* B, int id, int* done, vrps_report* rep) {
  Job* J = find_job(B, id);
  if (!J || !done) return fail(VRPS_ERR_INVALID_ARG, "unknown job %d", id);
  *done = 0;
  if (J->state == 0) return VRPS_OK;
  const cudaError_t e = cudaEventQuery(J->ev_done);
  if (e == cudaErrorNotReady) return VRPS_OK;
  VRPS_CUDA(e);
  *done = 1;
  return job_report(J, rep);
}

int vrps_batch_wait(vrps_batch* B, int id, vrps_report* rep) {
  if (!B) return fail(VRPS_ERR_INVALID_ARG, "batch is NULL");
  Job* J = find_job(B, id);
  if (!J) return fail(VRPS_ERR_INVALID_ARG, "unknown job %d", id);
  while (J->state == 0) VRPS_TRY(run_tick(B));
  VRPS_CUDA(cudaEventSynchronize(J->ev_done));
  return job_report(J, rep);
}

int vrps_batch_sync(vrps_batch* B) {
  if (!B) return fail(VRPS_ERR_INVALID_ARG, "batch is NULL");
  VRPS_CUDA(cudaStreamSynchronize(B->stream));
  return VRPS_OK;
}

int vrps_batch_ticks(const vrps_batch* B, long long* ticks, int* active) {
  if (!B) return fail(VRPS_ERR_INVALID_ARG, "batch is NULL");
  if (ticks) *ticks = B->ticks;
  if (active) *active = (int)B->active.size();
  return VRPS_OK;
}

int vrps_job_footprint(const vrps_geom* g, const vrps_job* d, size_t* bytes) {
  if (!g || !d || !bytes) return fail(VRPS_ERR_INVALID_ARG, "geometry, job or bytes is NULL");
  const size_t n = (size_t)g->n, m = (size_t)g->m;
  if (g->dims == 3) {
    size_t f = 0;
    f += 4 * n * 7;                 // x, h, x_hat, v, gbar, prox copy, x^T
    f += 4 * 3 * n * 3;             // dual and two rotation buffers
    f += 4 * m * 5;                 // b (subset-major), table, residual, two scratch sinograms
    if (d->storage != VRPS_STORAGE_FP32) f += 2 * m * 2;
    f += 12 * (size_t)d->max_iters + 64 * (size_t)g->n_angles;
    *bytes = f;
    return VRPS_OK;
  }
  const int maxw = g->nx > g->ny ? g->nx : g->ny;
  int band = (64 * 1024) / (int)(sizeof(float) * (maxw + 8));
  if (band < 1) band = 1;
  const size_t bands = (size_t)((maxw + band - 1) / band);
  size_t f = 0;
  f += 4 * n * 8;                   // x, h, x_hat, v, gbar, prox copy, x^T, transposed scratch
  f += 4 * 2 * n * 5;               // dual and four rotation buffers
  f += 4 * m * 4;                   // b (subset-major), table, residual, scratch sinogram
  if (d->storage != VRPS_STORAGE_FP32) f += 2 * m * 2;
  f += 4 * (size_t)g->n_angles * bands * g->n_bins;   // forward band partial sums
  f += 12 * (size_t)d->max_iters + 64 * (size_t)g->n_angles;   // draws, angle tables
  *bytes = f;
  return VRPS_OK;
}

}  // extern "C"
