// Internal declarations shared by the translation units of the CUDA library.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "vrps.h"

namespace vrps {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
// A refused kernel launch: the error with the launch's configuration and the kernel's limits.
int launch_fail(cudaError_t e, const char* name, const void* kern, dim3 grid, dim3 block, size_t smem);

#define VRPS_CUDA(call)                                        \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return ::vrps::cuda_fail(_e, #call); \
  } while (0)

#define VRPS_LAUNCHED(name)                                    \
  do {                                                         \
    cudaError_t _e = cudaGetLastError();                       \
    if (_e != cudaSuccess) return ::vrps::cuda_fail(_e, name); \
  } while (0)

#define VRPS_TRY(expr)              \
  do {                              \
    int _s = (expr);                \
    if (_s != VRPS_OK) return _s;   \
  } while (0)

// ------------------------------------------------------------------ launch accounting
// Every kernel launch is wrapped in a LaunchScope: it counts the launch and, while
// profiling is on, records CUDA events around it on the launching stream.
// `bytes` is the launch's algorithmic DRAM traffic (every array it must read or write,
// touched once, float32), summed per kernel family for the roofline; 0 where not stated.
void launch_begin(const char* name, cudaStream_t s, double bytes);
void launch_end(cudaStream_t s);
struct LaunchScope {
  cudaStream_t s;
  LaunchScope(const char* name, cudaStream_t st, double bytes = 0.0) : s(st) { launch_begin(name, st, bytes); }
  ~LaunchScope() { launch_end(s); }
};

// ------------------------------------------------------------------ launches
// Kernel launch through cudaLaunchKernelEx (one place to attach launch attributes).
// Programmatic dependent launch was measured on the 512^2 solver loop and made it 16 %
// slower (dependent CTAs parked on the SMs while the running kernel still needed them), so
// launches carry no attributes.
template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = nullptr;
  cfg.numAttrs = 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// launch_kernel, returning launch_fail's status from the enclosing function when refused.
#define VRPS_LAUNCH(name, kern, grid, block, smem, s, ...)                                      \
  do {                                                                                          \
    const cudaError_t _le = ::vrps::launch_kernel(kern, grid, block, smem, s, __VA_ARGS__);      \
    if (_le != cudaSuccess) return ::vrps::launch_fail(_le, name, (const void*)(kern), grid, block, smem); \
  } while (0)

// Opt a kernel into `bytes` of dynamic shared memory on the current device (cached: the
// runtime call is made once per kernel, device and size).
int smem_opt_in(const void* kern, size_t bytes);
// Reads and clears the handle's device error word (the caller has synchronised the work that
// could set it); VRPS_ERR_TIMEOUT when a bounded device-side wait had expired.
int take_device_error(vrps_geom* g);

// ------------------------------------------------------------------ geometry tables
// Per-angle constants of the 2D Joseph projector, derived in float64 on the host.
// Marching frame: T = 0 -> lines are image rows (iy) of x; T = 1 -> lines are columns (ix)
// read from the transposed image xT[ix][iy].  Along line l the ray of bin j meets the
// interpolation axis at u = uc + A1 (j - jc) + A2 (l - lc).  Pixel-driven adjoint: the
// pixel centre projects to fractional bin t = jc + Bx (ix - cx) + By (iy - cy); bin j gets
// weight wgt * max(0, 1 - |j - t| * inv_hw).
//
// Positions are carried in 64-bit fixed point with 32 fractional bits where float32 would
// lose precision at large coordinates: A1H, A2H, BxH, ByH hold A1, A2, Bx, By times 2^31, so
// that u * 2^32 = (ncols-1) 2^31 + A1H (2j-nb+1) + A2H (2l-nlines+1) is exact integer
// arithmetic up to the rounding of the constants (2^-32 per unit step).
struct AngleInfo2D {
  long long A1H, A2H, BxH, ByH;
  float A1, A2, wgt, Bx;
  float By, hw, inv_hw, inv_A2;   // inv_A2 = 1/A2 (0 when A2 = 0)
  int T;
  int pad[3];
};

// Fixed-point helpers: value * 2^32 held in a 64-bit integer.
__host__ __device__ __forceinline__ int fix_floor(long long v) { return (int)(v >> 32); }
// fractional part in [0, 1) from the top 23 fraction bits (exact float construction)
__device__ __forceinline__ float fix_frac(long long v) {
  return __int_as_float(0x3f800000u | ((unsigned)(unsigned long long)v >> 9)) - 1.0f;
}

// pixel tile of the 2D adjoint (the footprint size is derived from it on the host)
constexpr int ADJ2D_TILE_X = 16;
constexpr int ADJ2D_TILE_Y = 32;

// Per (view, detector column iu) constants of the 3D projector (float64-derived).
// axis 0: rays marched over x planes; axis 1: over y planes.  On dominant plane index l:
//   transverse index  ft = P0 + P1 (l - lc)
//   z index           fz = (iv - cv) (Q0 + Q1 (l - lc)) + cz
//   weight            wgt = voxel * sqrt(1 + P1^2 + ((iv - cv) R)^2),  R = dv / d_a
// Per (view, detector column) ray constants of the 3D projector.  On plane l of the ray's
// dominant axis (l = 0 .. n-1, not centred) the transverse voxel index is (PF0 + PF1 l) 2^-32
// and the z-index step per detector row is qz(l) = (QF0 + QF1 l) 2^-32: 64-bit fixed point, so
// positions stay exact to ~1e-9 voxel at any distance from the volume centre.
struct RayInfo3D {
  long long PF0, PF1;
  long long QF0, QF1;
  float P1;   // transverse slope (ray length factor)
  float R;    // z slope per detector row relative to the dominant axis (ray length factor)
  int axis;   // 0: marched over x planes, 1: over y planes
  int pad;
};

// Per view constants of the 3D voxel-driven adjoint (float64-derived).
struct ViewInfo3D {
  float sx, sy;        // source position (physical units)
  float eux, euy;      // detector u axis
  float esx, esy;      // unit vector from the origin towards the source
  float sdd, inv_du;   // source-detector distance, 1/du
  float cu;            // (nu-1)/2
  int has_x, has_y;    // whether the view has rays of each dominant axis
  int pad;
};

struct Workspace {
  // generic scratch sized by the geometry (lazily allocated)
  float* xT = nullptr;          // [n] transposed image for the 2D forward
  float* dual_cold = nullptr;   // [dims n] zero dual for cold-start prox calls
  float* dual_s1 = nullptr;     // [dims n] FGP rotation buffers
  float* dual_s2 = nullptr;
  float* dual_s3 = nullptr;
  float* dual_s4 = nullptr;
  double* partials = nullptr;   // reduction partials
  float* fwd_part = nullptr;      // 2D forward: per-band partial ray sums
  unsigned* fwd_count = nullptr;  // 2D forward: band arrival counters (one per angle row)
  size_t fwd_part_cap = 0;        // floats the partial buffer holds
  unsigned* dev_error = nullptr;  // device-side error word (bounded waits that expired)
  unsigned long long* fgp_bar = nullptr;   // arrival counter of the cooperative 2D FGP launch
  double* scalars = nullptr;    // [16] device scalars
  float* sino = nullptr;        // [m] sinogram scratch
  float* sino2 = nullptr;       // [m] second sinogram scratch (3D adjoint prescaling)
  float* img = nullptr;         // [n] image scratch
  float* img2 = nullptr;        // [n]
  // solver state (allocated on first solve)
  bool solver_ready = false;
  float *x = nullptr, *xf = nullptr, *xfT = nullptr, *h = nullptr, *xhat = nullptr, *v = nullptr,
        *gbar = nullptr, *xprox = nullptr, *dual = nullptr;
  float *b_perm = nullptr, *tab = nullptr, *res = nullptr;
  float *b16 = nullptr, *tab16 = nullptr;   // bfloat16 storage of b_perm / tab (m halves each)
  float* adj_part = nullptr;      // 2D adjoint: partial sums of the angle shares
  size_t adj_part_cap = 0;
  unsigned* adj_count = nullptr;  // 2D adjoint: per-tile arrival counters
  size_t adj_count_cap = 0;
  int32_t* sched_dev = nullptr;
  int sched_cap = 0;
  int32_t* sched_host = nullptr;   // pinned
  int* order_dev = nullptr;        // subset-major angle order for the solver's N
  int order_N = 0;
  AngleInfo2D* ang_order_dev = nullptr;   // 2D angle table in order_dev's order
  std::vector<int> order_off;      // N+1 row offsets of the subsets in subset-major order
};

}  // namespace vrps

struct vrps_geom {
  int dims = 2;
  int nx = 0, ny = 0, nz = 1;
  double pixel = 1.0;
  int n_angles = 0;      // angles (2D) or views (3D)
  int n_bins = 0;        // 2D bins
  double bin_spacing = 1.0;
  int nu = 0, nv = 0;
  double du = 1.0, dv = 1.0, sod = 0.0, sdd = 0.0;
  int n_subsets = 1;
  int64_t n = 0, m = 0;
  int row_len = 0;
  int device = 0;
  int sms = 0;           // multiprocessors of that device
  std::vector<double> angles;
  // 2D tables
  vrps::AngleInfo2D* ang2d = nullptr;
  vrps::AngleInfo2D* ang2d_sub = nullptr;         // the same rows in order_subset's order
  std::vector<vrps::AngleInfo2D> ang2d_host;      // host copy (natural order)
  int adj_fp = 0;        // footprint slots per angle of the 2D adjoint tile
  int adj_nc = 0;        // candidate bins per pixel and angle
  // launch shapes chosen by vrps_autotune (0 / -1: built-in defaults)
  int tune_fwd_bytes = 0;   // shared-memory band of the 2D forward (bytes)
  int tune_fwd_group = 0;   // bands per forward CTA item (0: one)
  int tune_adj_two = -1;    // 2D adjoint: two pixels per thread (1) or one (0)
  int tune_f3_zc = 0;       // 3D FGP: z planes per streaming chunk
  int tune_adj3_zc = 0;     // 3D adjoint: voxels per thread along z (0 = 16, or 32)
  // 2D all-angle passes (snapshots, full gradients): own forward band / bands per CTA and
  // adjoint angle shares when tuned (0 = as for subsets)
  int tune_full_fwd_bytes = 0, tune_full_fwd_group = 0, tune_full_adj_split = 0;
  int tune_fgp_tile = 0;    // 2D FGP output tile: 0 32x32, 1 32x16, 2 16x16
  int tune_adj_split = 0;   // 2D adjoint: angle shares per pixel tile (0: one)
  // 3D tables
  vrps::RayInfo3D* ray3d = nullptr;     // [n_views][nu]
  vrps::ViewInfo3D* view3d = nullptr;   // [n_views]
  std::vector<vrps::ViewInfo3D> view3d_host;
  // angle orders
  int* order_natural = nullptr;   // [n_angles] 0..n_angles-1
  int* order_subset = nullptr;    // [n_angles] subset-major for n_subsets
  std::vector<int> subset_off;    // [n_subsets+1]
  vrps::Workspace ws;
};

namespace vrps {

// subset -> (device id list, row count, row offset within the subset-major order)
int subset_rows(const vrps_geom* g, int subset, const int** ids, int* rows);
int build_order(int n_angles, int N, int** dev, std::vector<int>* off);
// 2D: the angle table permuted into the subset-major order of N subsets (device, replacing *dev).
int build_order_angles(const vrps_geom* g, int N, AngleInfo2D** dev);
// 2D: the angle table indexed by launch row for the id list ids (a subset's rows of one of the
// geometry's orders), or null when ids is none of them (the kernels then read ang[ids[row]]).
const AngleInfo2D* angle_rows(const vrps_geom* g, const int* ids);
int ensure(float** p, size_t count);
int ensure_d(double** p, size_t count);

// ---- 2D projector (joseph2d.cu)
enum FwdMode { FWD_PLAIN = 0, FWD_RESID = 1, FWD_SVRG = 2, FWD_SAGA = 3, FWD_SNAP = 4 };
// Storage of the solver's sinogram-sized rows (data b and the SVRG / SAGA table): float32,
// bfloat16, or float16 holding value * scale (scale a power of two); arithmetic is float32.
enum StoreKind { STORE_F32 = 0, STORE_BF16 = 1, STORE_F16 = 2 };
struct FwdOut {
  float* y;            // output rows (float32 always)
  const void* b;       // data rows (RESID, SAGA, SNAP), stored as `store`
  void* tab;           // table rows (SVRG read, SAGA read/write, SNAP write), likewise
  int prescale = 0;    // 3D: write y times the ray's length factor (input of a prescaled adjoint)
  int store = 0;       // StoreKind of b and tab
  float scale = 1.f;   // float16: stored = value * scale
  float inv = 1.f;     // 1 / scale (exact)
};

__device__ __forceinline__ float ld_store(const FwdOut& o, const void* p, size_t i) {
  if (o.store == STORE_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
  if (o.store == STORE_F16) return __half2float(static_cast<const __half*>(p)[i]) * o.inv;
  return static_cast<const float*>(p)[i];
}
// Stores v (rounded to nearest) and returns the value the stored entry decodes to, so that a
// table and the sums built from it use the same numbers.  float16 saturates at +-65504.
__device__ __forceinline__ float st_store(const FwdOut& o, void* p, size_t i, float v) {
  if (o.store == STORE_BF16) {
    const __nv_bfloat16 e = __float2bfloat16_rn(v);
    static_cast<__nv_bfloat16*>(p)[i] = e;
    return __bfloat162float(e);
  }
  if (o.store == STORE_F16) {
    const __half e = __float2half_rn(fminf(fmaxf(v * o.scale, -65504.f), 65504.f));
    static_cast<__half*>(p)[i] = e;
    return __half2float(e) * o.inv;
  }
  static_cast<float*>(p)[i] = v;
  return v;
}

int fwd2d(const vrps_geom* g, const float* x, const float* xT, const int* ids, int rows, int mode,
          FwdOut o, cudaStream_t s);
int transpose2d(const float* in, float* out, int ny, int nx, cudaStream_t s, int slices = 1);

// epilogue of the pixel-driven adjoint, fused ProxSkip update (Algorithm 1, x_hat line)
struct UpdateArgs {
  int enabled;            // 0: plain adjoint -> out
  float* out;             // plain output
  float cN;               // G = cN * g + gbar
  float* gbar;            // may be null; SAGA updates it in place (gbar += g)
  int saga;
  const float* base;      // point the step starts from (x, or FISTA's y)
  const float* h;         // control variate (null: not used)
  float gamma, gamma_over_p;
  int theta;
  float* x;               // theta = 0: x <- x_hat
  float* xT;              // and its transpose (may be null)
  float* xhat;            // theta = 1 and h in use: keep x_hat
  float* v;               // theta = 1: prox input
  int prescaled;          // 3D: r already carries the ray length factors (see FwdOut::prescale)
  int snap;               // SVRG snapshot: g is the full gradient; gbar <- g and G = g
};

// Algorithm 1, estimator and x_hat lines for one pixel: G = cN g + gbar,
// x_hat = base - gamma (G - h); theta = 0: x <- x_hat (returned for the transposed copy);
// theta = 1: keep x_hat and write the prox input v = x_hat - (gamma/p) h.
// (Explicit roundings and fused multiply-adds: identical bits in every kernel that inlines it.)
// The pixel's inputs of the update (gbar, base point, h), which a kernel may load before it
// computes g so that their latency hides behind the gather.
struct UpdIn {
  float gb, base, h;
};
__device__ __forceinline__ UpdIn update_load(const UpdateArgs& u, size_t p) {
  UpdIn a;
  a.gb = (!u.snap && u.gbar) ? u.gbar[p] : 0.f;
  a.base = u.base[p];
  a.h = u.h ? u.h[p] : 0.f;
  return a;
}
__device__ __forceinline__ float update_pixel_pre(const UpdateArgs& u, size_t p, float g, const UpdIn& a) {
  float G;
  if (u.snap) {            // SVRG snapshot: g is the full gradient; gbar <- g, G = g
    u.gbar[p] = g;
    G = g;
  } else if (u.gbar) {
    const float gb = a.gb;
    G = fmaf(u.cN, g, gb);
    if (u.saga) u.gbar[p] = __fadd_rn(gb, g);
  } else {
    G = __fmul_rn(u.cN, g);
  }
  const float base = a.base;
  if (u.h) {
    const float hp = a.h;
    const float xh = fmaf(-u.gamma, __fsub_rn(G, hp), base);
    if (u.theta) {
      u.xhat[p] = xh;
      u.v[p] = fmaf(-u.gamma_over_p, hp, xh);
      return 0.f;
    }
    u.x[p] = xh;
    return xh;
  }
  const float xh = fmaf(-u.gamma, G, base);
  if (u.theta) {
    u.v[p] = xh;
    return 0.f;
  }
  u.x[p] = xh;
  return xh;
}
__device__ __forceinline__ float update_pixel(const UpdateArgs& u, size_t p, float g) {
  return update_pixel_pre(u, p, g, update_load(u, p));
}
// ---- 2D projector launch parameters (joseph2d.cu)
struct Fwd2DParams {
  const float* x;
  const float* xT;
  const AngleInfo2D* ang;
  const int* ids;
  int nx, ny, nb;
  float jc;
  int band;                   // lines per band
  int nbands;                 // bands covering the longest line count
  int group;                  // bands per CTA item (walked with double-buffered copies)
  int bands;                  // band groups per row = items per row (gridDim.x)
  float* part;                // [rows][bands][nb] partial sums (one per group)
  unsigned* count;            // [rows] arrival counters, zero between launches
  unsigned* err;              // device error word
  FwdOut o;
};

struct Adj2DParams {
  const float* r;
  const AngleInfo2D* ang;
  const int* ids;
  int rows;
  int nx, ny, nb;
  int fp, nc, chunk;
  int split;                  // angle shares per tile (1: one CTA per tile)
  int tiles_x;
  float* part;                // [split][n] partial sums of the shares
  unsigned* count;            // [tiles] arrival counters, zero between launches
  UpdateArgs u;
};

int adj2d(const vrps_geom* g, const float* r, const int* ids, int rows, const UpdateArgs& u,
          cudaStream_t s);
// Launch constants of one forward / adjoint (allocating the geometry's scratch on first use).
int fwd2d_setup(const vrps_geom* g, const float* x, const float* xT, const int* ids, int rows, FwdOut o,
                Fwd2DParams* P, size_t* smem, bool* bulk);
int adj2d_setup(const vrps_geom* g, const float* r, const int* ids, int rows, const UpdateArgs& u,
                Adj2DParams* P, size_t* smem, int* variant, int* tiles_x, int* tiles_y);

// Algorithmic bytes of the image-side epilogue of an adjoint launch over n pixels.
inline double update_bytes(const UpdateArgs& u, size_t n) {
  const double f = 4.0 * (double)n;
  if (!u.enabled) return f;                        // write out
  double b = f;                                    // read base
  if (u.gbar) b += u.saga ? 2 * f : f;             // read gbar (SAGA: and write it)
  if (u.h) b += f;                                 // read h
  if (u.theta) b += u.h ? 2 * f : f;               // write v (and x_hat)
  else b += u.xT ? 2 * f : f;                      // write x (and its transpose)
  return b;
}

// Algorithmic bytes of a forward launch's sinogram epilogue over m_i rays (FwdMode).
inline double fwd_mode_bytes(int mode, size_t mi, int store = 0) {
  const double f = 4.0 * (double)mi, t = (store ? 2.0 : 4.0) * (double)mi;   // y, stored rows
  switch (mode) {
    case FWD_PLAIN: return f;              // write y
    case FWD_RESID: return f + t;          // read b, write y
    case FWD_SVRG: return f + t;           // read A x~, write y
    case FWD_SAGA: return f + 3 * t;       // read b, table; write y, table
    default: return f + 2 * t;             // snapshot: read b; write table, y
  }
}

// ---- 3D projector (joseph3d.cu)
struct Fwd3DParams {
  const float* x;    // [nz][ny][nx]
  const float* xT;   // [nz][nx][ny]
  const RayInfo3D* rays;
  const int* ids;
  int nx, ny, nz, nu, nv;
  float cx, cy, cz, cv, vox;
  FwdOut o;
};

struct Adj3DParams {
  const float* r;
  const RayInfo3D* rays;
  const ViewInfo3D* views;
  const int* ids;
  int rows;
  int nx, ny, nz, nu, nv;
  float cx, cy, cz, cv, vox;
  UpdateArgs u;
};

// Launch constants of one 3D forward / adjoint.
int fwd3d_setup(const vrps_geom* g, const float* x, const float* xT, const int* ids, int rows, FwdOut o,
                Fwd3DParams* P);
int adj3d_setup(const vrps_geom* g, const float* r, const int* ids, int rows, const UpdateArgs& u, Adj3DParams* P);

int fwd3d(const vrps_geom* g, const float* x, const float* xT, const int* ids, int rows, int mode, FwdOut o,
          cudaStream_t s);
int adj3d(const vrps_geom* g, const float* r, const int* ids, int rows, const UpdateArgs& u,
          cudaStream_t s);

// ---- FGP (fgp.cu)
struct ProxTail {
  int mode;               // 0: out = x+;  1: solver tail
  float* out;
  float* x;               // solver: x <- x+
  float* xT;              // and transposed (2D, may be null)
  float* h;               // h += (p/gamma)(x+ - xhat) when non-null
  const float* xhat;
  float p_over_gamma;
  float* xprox;           // copy of x+ (may be null)
  float* y;               // FISTA: y <- x+ + mom (x+ - x_old); yT likewise
  float* yT;
  float mom;
};
// ---- 2D FGP launch arguments (fgp.cu)
struct Dims3 {
  int nx, ny, nz;
  size_t n;
};

// The 3D FGP of one prox call: buffer rotation (0 = the warm-started dual) and extrapolation
// of every iteration, and the buffer that holds w_K.
struct Fgp3Schedule {
  std::vector<int> cur, prev, nxt;
  std::vector<float> mom;
  int final_buf = 0;
};
Fgp3Schedule fgp3_schedule(int iters);
int fgp3_zc(const vrps_geom* g);   // z planes per chunk of the streaming 3D FGP iteration
constexpr int FGP3_TX = 32, FGP3_TY = 16, FGP3_ZC = 64;   // streaming tile and default chunk

constexpr int FB_T = 6;   // iterations per block (= halo width)

struct MomBlock {
  float c[FB_T + 1];   // c[s]: extrapolation used when forming z for iteration s + 1
};

// One blocked launch: nsteps (<= FB_T) iterations from (w, z) to (wn, zn).
struct FgpBlockArgs {
  const float* v;
  const float* w;
  const float* z;
  float* wn;
  float* zn;
  int nx, ny;
  float tau, step;
  MomBlock mom;
  int nsteps, nonneg;
};

// x+ and the fused tail over a whole image.
struct FgpOutArgs {
  const float* v;
  const float* w;
  float* wdst;   // copy of w (may be null)
  int nx, ny;
  float tau;
  int nonneg;
  ProxTail t;
};

int fgp_run(const vrps_geom* g, const float* v, float tau, int iters, int nonneg, float* dual,
            const ProxTail& tail, cudaStream_t s);
// Momentum coefficients of the blocked 2D FGP launches of one prox call (t restarts at 1).
std::vector<MomBlock> fgp_momentum(int iters);
// 2D: `iters` FGP iterations from the dual w0 ([2][nx*ny]) in blocked launches whose (w, z)
// state alternates between the buffer pairs pairs[0] and pairs[1] (each [2][nx*ny]); *w_final
// receives the buffer holding w_K (w0 itself when iters = 0).  tile: 0 32 x 32 or 32 x 27 by the
// SM count, 1 32x16, 2 16x16, 3 32x32, 4 32x27.  coop_bar (device counter, nullable): run all
// blocks in one cooperative launch whose CTAs meet at a bounded grid barrier between blocks
// (err: device error word, set when a barrier wait expires), when the tiles fit the resident
// slots; otherwise, and with coop_bar null, one launch per block.
int fgp2d_iterate(const float* v, const float* w0, float* const pairs[2][2], int nx, int ny, float tau, int iters,
                  int nonneg, int tile, cudaStream_t s, const float** w_final,
                  unsigned long long* coop_bar = nullptr, unsigned* err = nullptr);
// 2D: x+ = P_+(v + tau div w) with the fused tail t; wdst (nullable) receives a copy of w.
int fgp2d_output(const float* v, const float* w, float* wdst, int nx, int ny, float tau, int nonneg,
                 const ProxTail& t, cudaStream_t s);
// Allocates the dual rotation buffers of the geometry's prox.
int fgp_prepare(vrps_geom* g);

// ---- batched persistent launches (a CTA walks items blockIdx.x, blockIdx.x + gridDim.x, ...
// over the items of many problems; the same item functions as the single-problem kernels)
constexpr int BATCH_MAX_JOBS = 256;
constexpr int BATCH_MAX_FGP_ITERS = 128;                                  // 2D inner iterations per prox call
constexpr int BATCH_MAX_BLOCKS = (BATCH_MAX_FGP_ITERS + FB_T - 1) / FB_T;   // FGP blocks per prox call
constexpr int FGP_TILE = 32;           // 2D FGP output tile (TileLarge)
struct BatchFwd {
  Fwd2DParams P;
  int mode;   // FwdMode
  int bulk;   // band staged by bulk copies
};
struct BatchAdj {
  Adj2DParams P;
  int variant;   // 2 (nc == 2) + 1 (two pixels per thread)
  int tiles_x;
};
struct BatchFgp {
  FgpBlockArgs A[BATCH_MAX_BLOCKS];   // launch b of the call
  int nblocks;
  int tiles_x;
};
struct BatchOut {
  FgpOutArgs A;
  int tiles_x;
};
// One tick's work list, packed in one buffer: the header, then the arrays at its offsets.
// Prefix arrays hold each job's first item (n + 1 entries); the FGP prefix is
// [BATCH_MAX_BLOCKS][n_prox + 1].
// cnt: item counters the launches hand out work from (0 forward, 1 adjoint, 2 prox output,
// 3 + b FGP block b); uploaded as zeros with the tick.
struct TickHeader {
  int n_fwd, n_adj, n_prox, pad;
  unsigned off_fwd, off_pfwd, off_adj, off_padj, off_fgp, off_pfgp, off_out, off_pout;
  unsigned cnt[3 + BATCH_MAX_BLOCKS];
};
int fwd2d_batched(char* slot, int grid, size_t smem, bool grouped, cudaStream_t s);
int adj2d_batched(char* slot, int grid, size_t smem, cudaStream_t s);
int fgp2d_block_batched(char* slot, int b, int grid, cudaStream_t s);
int fgp2d_out_batched(char* slot, int grid, cudaStream_t s);
// Persistent grid (CTAs resident on all SMs) of batched kernel `which` (0 fwd, 1 adj, 2 FGP
// block, 3 FGP out, 4 fwd with band groups) at `smem` bytes of dynamic shared memory.
int batched_grid(int which, size_t smem, int* grid);
int batched_grid_2d(int which, size_t smem, int* grid);

// ---- batched 3D jobs (one batch holds 2D or 3D jobs): transpose, forward, adjoint, every FGP
// iteration and the prox output are one persistent launch each over all jobs' items
constexpr int BATCH3_MAX_ITERS = 128;
struct BatchTr3 {            // x -> x^T slice by slice; items tiles_x * tiles_y * nz
  const float* in;
  float* out;
  int nx, ny, nz, tiles_x, tiles_y;
};
struct BatchFwd3 {           // items tiles_u * rows * bands_v
  Fwd3DParams P;
  int mode, tiles_u, rows, bands_v;
};
struct BatchAdj3 {           // items tiles_x * tiles_y * chunks
  Adj3DParams P;
  int tiles_x, tiles_y, chunks;
};
struct BatchFgp3 {           // iteration it: items tiles_x * tiles_y * chunks when it < iters
  const float* v;
  float* buf[3];
  Dims3 D;
  float tau, step;
  int nonneg, zc, iters, tiles_x, tiles_y, chunks;
  unsigned char cur[BATCH3_MAX_ITERS], prev[BATCH3_MAX_ITERS], nxt[BATCH3_MAX_ITERS];
  float mom[BATCH3_MAX_ITERS];
};
struct BatchOut3 {           // items tiles_x * tiles_y * nz
  const float* v;
  const float* w;
  float* wdst;
  Dims3 D;
  float tau;
  int nonneg;
  ProxTail t;
  int tiles_x, tiles_y;
};
// cnt: 0 transpose, 1 forward, 2 adjoint, 3 prox output, 4 + it FGP iteration it
struct TickHeader3 {
  int n_jobs, n_prox, pad0, pad1;
  unsigned off_tr, off_ptr, off_fwd, off_pfwd, off_adj, off_padj, off_fgp, off_pfgp, off_out, off_pout;
  unsigned cnt[4 + BATCH3_MAX_ITERS];
};
int tr3_batched(char* slot, int grid, cudaStream_t s);
int fwd3d_batched(char* slot, int grid, cudaStream_t s);
int adj3d_batched(char* slot, int grid, cudaStream_t s);
int fgp3d_iter_batched(char* slot, int it, int grid, cudaStream_t s);
int fgp3d_out_batched(char* slot, int grid, cudaStream_t s);
// persistent grids: 0 transpose, 1 forward, 2 adjoint, 3 FGP iteration, 4 prox output
int batched_grid_3d(int which, int* grid);
// work-list entries with their item counts (same launch shapes as the single-job kernels)
int tr3_batch_entry(const float* in, float* out, int nx, int ny, int nz, BatchTr3* e, int* items);
int fwd3d_batch_entry(const vrps_geom* g, const float* x, const float* xT, const int* ids, int rows, int mode,
                      FwdOut o, BatchFwd3* e, int* items);
int adj3d_batch_entry(const vrps_geom* g, const float* r, const int* ids, int rows, const UpdateArgs& u,
                      BatchAdj3* e, int* items);
int fgp3d_batch_entry(vrps_geom* g, const float* v, float tau, int iters, int nonneg, float* dual,
                      const ProxTail& t, BatchFgp3* f, int* f_items, BatchOut3* o, int* o_items);

// Algorithmic bytes of the prox output launch's tail over n pixels (beyond reading v, w).
inline double tail_bytes(const ProxTail& t, size_t n) {
  const double f = 4.0 * (double)n;
  if (t.mode == 0) return f;                       // write out
  double b = 2 * f;                                // read and write x
  if (t.h) b += 3 * f;                             // read h, x_hat; write h
  if (t.xprox) b += f;
  if (t.y) b += f;
  if (t.y ? t.yT : t.xT) b += f;                   // transposed copy
  return b;
}

// ---- reductions, Philox, misc (reduce.cu)
int dot64(const float* a, const float* b, int64_t n, double* dst, Workspace& ws, cudaStream_t s);
int tv64(const vrps_geom* g, const float* x, double* dst, Workspace& ws, cudaStream_t s);
int philox_schedule(uint64_t seed, uint32_t job, int64_t k0, int count, int N, double p,
                    int32_t* out, cudaStream_t s);
int philox_uniform(uint64_t seed, uint32_t job, uint32_t tag, float* out, int64_t n, cudaStream_t s);
int scale_inv_sqrt(float* dst, const float* src, const double* nrm2, int64_t n, cudaStream_t s);
int gather_rows(const float* src, float* dst, const int* ids, int rows, int row_len, cudaStream_t s);
int scatter_rows(const float* src, float* dst, const int* ids, int rows, int row_len, cudaStream_t s);
int fill(float* p, float v, int64_t n, cudaStream_t s);
int copy_or_zero(float* dst, const float* src, int64_t n, cudaStream_t s);
// float32 rows -> storage `kind` (StoreKind; float16 multiplied by scale).
int to_store(const float* src, void* dst, int64_t n, int kind, float scale, cudaStream_t s);
// Solver state in the geometry's workspace (solver.cu).
int solver_alloc(vrps_geom* g, bool fista, bool bf16);
int storage_scale(vrps_geom* g, int kind, float* scale, cudaStream_t s);
// Adds to the library's launch counter (kernels launched through a CUDA graph).
void launch_count_add(long long n);
// Whether per-launch event profiling is on (graphs are bypassed then).
bool profiling_on();

// projector dispatch (2D or 3D) used by the solver and the API
int proj_forward(const vrps_geom* g, const float* x, const float* xT, const int* ids, int rows,
                 int mode, FwdOut o, cudaStream_t s);
int proj_adjoint(const vrps_geom* g, const float* r, const int* ids, int rows, const UpdateArgs& u,
                 cudaStream_t s);

}  // namespace vrps
