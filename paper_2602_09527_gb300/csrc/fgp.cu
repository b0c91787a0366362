// FGP (Beck & Teboulle 2009) for the prox of tau (TV + I_{x>=0}), the prox step of
// Algorithm 1 (Section 2.1: fixed number of warm-started inner iterations).
//
// Dual w (one 2- or 3-vector per pixel, ||w|| <= 1).  With z the extrapolated dual,
//   x    = P_+( v + tau div z )            (D^T = -div, forward differences, Neumann)
//   w'   = P_B( z + D x / (4 d tau) )      (d = 2 or 3)
//   z'   = w' + mom_k (w' - w)             (mom from t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2)
// Kernels store only w_k and w_{k-1} and rebuild z on the fly.  2D runs blocks of FB_T
// iterations on shared-memory tiles (temporal blocking), all blocks of a prox call in one
// cooperative launch where the tiles fit the resident slots; 3D runs one iteration per launch
// (reads v, w_k, w_{k-1}, writes w_{k+1}: 10 floats per voxel) with three rotating buffers,
// so that no launch writes a buffer another CTA still reads.
// The output kernel forms x+ = P_+(v + tau div w_K) and applies the fused tail of the
// solver (x <- x+, h += (p/gamma)(x+ - x_hat), FISTA momentum, transposed copy).
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "vrps_internal.h"

namespace vrps {
namespace {

// 2D: T iterations per launch (temporal blocking).  A CTA owns a TX x TY output tile and
// loads v, the dual w and the extrapolated dual z on the tile grown by T pixels on every
// side; each iteration shrinks the region where values are exact by one pixel per side, so
// after T iterations the tile itself holds w_{k+T} and z_{k+T}, which are written back.
// Per iteration: x = P_+(v + tau div z) on the region, then per pixel
// w' = P_B(z + step D x) and the next extrapolation z' = w' + mom' (w' - w).
// Every thread owns fixed pixels of the grown tile (linear slots e = tid + k NT) and keeps
// their v, w, z and x in registers for the whole launch; shared memory holds only what
// neighbours read: z (for the divergence at the left / upper neighbour) and x (for the
// forward differences at the right / lower neighbour).  Reads and writes go to different
// global buffer pairs, so neighbouring CTAs never see a half-updated dual.

// Tile: TX x TY outputs per CTA of NT threads; the grown tile (EX x EY elements) is walked
// in NS linear slots per thread.  Each slot carries the depth at which it leaves the
// shrinking valid region, so one compare decides whether it works in a step.
template <int TX_, int TY_, int NT_>
struct FgpTile {
  static constexpr int TX = TX_, TY = TY_, NT = NT_;
  static constexpr int EX = TX + 2 * FB_T, EY = TY + 2 * FB_T, NE = EX * EY;
  static constexpr int NS = (NE + NT - 1) / NT;
  static constexpr size_t SMEM = sizeof(float) * 3 * NE;   // z (2 components) and x
};
// (grown tiles for FB_T = 6)
using TileLarge = FgpTile<32, 32, 512>;   // 44 x 44 grown tile, 23 KB
using TileWide = FgpTile<32, 16, 256>;    // 44 x 28, 15 KB: twice the tiles of TileLarge
using TileSmall = FgpTile<16, 16, 256>;   // 28 x 28, 9 KB: four times the tiles
using TileLow = FgpTile<32, 27, 512>;     // 44 x 39, 20 KB: 19 tile rows at 512 and 38 at 1024 rows
// the batched launches' block keeps v, w, z and x of the grown tile in shared memory
constexpr size_t BATCHED_FGP_SMEM = sizeof(float) * 6 * TileLarge::NE;   // 46 KB


// Projection onto the unit ball: g / max(1, |g|) through the hardware reciprocal square
// root (relative error a few ulp, far below the float32 tolerances of the prox).
__device__ __forceinline__ void ball2(float g1, float g2, float& n1, float& n2) {
  const float q = fmaf(g1, g1, __fmul_rn(g2, g2));
  if (q > 1.f) {
    const float r = rsqrtf(q);
    n1 = g1 * r;
    n2 = g2 * r;
  } else {
    n1 = g1;
    n2 = g2;
  }
}

// One block of A.nsteps FGP iterations on output tile (ox + FB_T, oy + FB_T) with its grown
// tile in registers (own slots) and shared memory (sz1, sz2, sx: NE floats each).
// INTERIOR: the grown tile lies strictly inside the image (no boundary or bounds tests).
template <class TL, bool INTERIOR, bool NONNEG>
__device__ __forceinline__ void fgp2d_block_regs(const FgpBlockArgs& A, int ox, int oy, float* sz1, float* sz2,
                                                 float* sx, const float* mom) {
  constexpr int EX = TL::EX, EY = TL::EY, NE = TL::NE, NT = TL::NT, NS = TL::NS;
  const int tid = threadIdx.x;
  const int nx = A.nx, ny = A.ny, nsteps = A.nsteps;
  const float tau = A.tau, step = A.step;
  const size_t n = (size_t)nx * ny;
  float rv[NS], rw1[NS], rw2[NS], rz1[NS], rz2[NS], rx[NS];
  // x at step s needs z at i-1, i-EX: valid on [s+1, EX-s); w' also needs x at i+1, i+EX:
  // valid on [s+1, EX-s-1).  dx / dw = largest step at which the slot is still inside.
  int dx[NS], dw[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int e = tid + k * NT;
    const int lx = e % EX, ly = e / EX;
    const int a = min(lx - 1, ly - 1);
    dx[k] = e < NE ? min(a, min(EX - 1 - lx, EY - 1 - ly)) : -1;
    dw[k] = e < NE ? min(a, min(EX - 2 - lx, EY - 2 - ly)) : -1;
    const int gx = ox + lx, gy = oy + ly;
    float vv = 0.f, w_a = 0.f, w_b = 0.f, z_a = 0.f, z_b = 0.f;
    if (e < NE && gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
      // the dual state through L2 only: within a cooperative launch other CTAs rewrite these
      // buffers between blocks, after this SM may have cached them
      const size_t p = (size_t)gy * nx + gx;
      vv = A.v[p];
      w_a = __ldcg(A.w + p);
      w_b = __ldcg(A.w + n + p);
      z_a = __ldcg(A.z + p);
      z_b = __ldcg(A.z + n + p);
    }
    rv[k] = vv;
    rw1[k] = w_a;
    rw2[k] = w_b;
    rz1[k] = z_a;
    rz2[k] = z_b;
    rx[k] = 0.f;
    if (e < NE) {
      sz1[e] = z_a;
      sz2[e] = z_b;
    }
  }
  __syncthreads();
  for (int s = 0; s < nsteps; ++s) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (dx[k] >= s) {
        const int i = tid + k * NT;
        float xv = 0.f;
        const int gx = ox + i % EX, gy = oy + i / EX;
        if (INTERIOR || (gx >= 0 && gx < nx && gy >= 0 && gy < ny)) {
          float d = 0.f;
          if (INTERIOR || gx < nx - 1) d += rz1[k];
          if (INTERIOR || gx > 0) d -= sz1[i - 1];
          if (INTERIOR || gy < ny - 1) d += rz2[k];
          if (INTERIOR || gy > 0) d -= sz2[i - EX];
          xv = fmaf(tau, d, rv[k]);
          if (NONNEG) xv = fmaxf(xv, 0.f);
        }
        rx[k] = xv;
        sx[i] = xv;
      }
    }
    __syncthreads();
    const float m = mom[s];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (dw[k] >= s) {
        const int i = tid + k * NT;
        float n1 = 0.f, n2 = 0.f, m1 = 0.f, m2 = 0.f;
        const int gx = ox + i % EX, gy = oy + i / EX;
        if (INTERIOR || (gx >= 0 && gx < nx && gy >= 0 && gy < ny)) {
          const float xc = rx[k];
          const float d1 = (INTERIOR || gx < nx - 1) ? sx[i + 1] - xc : 0.f;
          const float d2 = (INTERIOR || gy < ny - 1) ? sx[i + EX] - xc : 0.f;
          ball2(fmaf(step, d1, rz1[k]), fmaf(step, d2, rz2[k]), n1, n2);
          m1 = fmaf(m, n1 - rw1[k], n1);
          m2 = fmaf(m, n2 - rw2[k], n2);
        }
        rw1[k] = n1;
        rw2[k] = n2;
        rz1[k] = m1;
        rz2[k] = m2;
        sz1[i] = m1;
        sz2[i] = m2;
      }
    }
    __syncthreads();
  }
  // the output tile: every thread writes the slots it owns there
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int e = tid + k * NT;
    const int lx = e % EX, ly = e / EX;
    if (e < NE && lx >= FB_T && lx < FB_T + TL::TX && ly >= FB_T && ly < FB_T + TL::TY) {
      const int gx = ox + lx, gy = oy + ly;
      if (gx < nx && gy < ny) {
        const size_t p = (size_t)gy * nx + gx;
        A.wn[p] = rw1[k];
        A.wn[n + p] = rw2[k];
        A.zn[p] = rz1[k];
        A.zn[n + p] = rz2[k];
      }
    }
  }
}

// One output tile (bx, by) of a blocked launch; smf: dynamic shared memory (TL::SMEM bytes);
// mom: the block's momentum coefficients (FB_T + 1), staged in shared memory here.
template <class TL>
__device__ __forceinline__ void fgp2d_block_item(const FgpBlockArgs& A, int bx, int by, float* smf,
                                                 const float* mom) {
  constexpr int EX = TL::EX, EY = TL::EY, NE = TL::NE;
  __shared__ float s_mom[FB_T + 1];
  if (threadIdx.x <= FB_T) s_mom[threadIdx.x] = mom[threadIdx.x];   // visible after the load phase
  float* sz1 = smf;
  float* sz2 = sz1 + NE;
  float* sx = sz2 + NE;
  const int ox = bx * TL::TX - FB_T, oy = by * TL::TY - FB_T;
  const int nx = A.nx, ny = A.ny;
  const bool interior = ox >= 1 && oy >= 1 && ox + EX <= nx - 1 && oy + EY <= ny - 1;
  if (A.nonneg) {
    if (interior) fgp2d_block_regs<TL, true, true>(A, ox, oy, sz1, sz2, sx, s_mom);
    else fgp2d_block_regs<TL, false, true>(A, ox, oy, sz1, sz2, sx, s_mom);
  } else {
    if (interior) fgp2d_block_regs<TL, true, false>(A, ox, oy, sz1, sz2, sx, s_mom);
    else fgp2d_block_regs<TL, false, false>(A, ox, oy, sz1, sz2, sx, s_mom);
  }
}

// The batched launches' variant of the block: v, w, z and x of the grown tile all in shared
// memory (17 shared accesses per pixel-iteration, but few registers, so three or four CTAs of
// the persistent grid share an SM).  Same operations in the same order as fgp2d_block_regs:
// the same bits.  One block of nsteps FGP iterations.  INTERIOR: the grown tile
// lies strictly inside the image (no boundary or bounds tests needed).
template <class TL, bool INTERIOR, bool NONNEG>
__device__ __forceinline__ void fgp2d_steps_smem(float* sv, float* w1, float* w2, float* z1, float* z2, float* sx, int ox,
                                            int oy, int nx, int ny, float tau, float step, const MomBlock& mom,
                                            int nsteps) {
  constexpr int EX = TL::EX, EY = TL::EY, NE = TL::NE, NT = TL::NT, NS = TL::NS;
  const int tid = threadIdx.x;
  // x at step s needs z at i-1, i-EX: valid on [s+1, EX-s); w' also needs x at i+1, i+EX:
  // valid on [s+1, EX-s-1).  dx / dw = largest step at which the slot is still inside.
  int dx[NS], dw[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int e = tid + k * NT;
    const int lx = e % EX, ly = e / EX;
    const int a = min(lx - 1, ly - 1);
    dx[k] = e < NE ? min(a, min(EX - 1 - lx, EY - 1 - ly)) : -1;
    dw[k] = e < NE ? min(a, min(EX - 2 - lx, EY - 2 - ly)) : -1;
  }
  for (int s = 0; s < nsteps; ++s) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (dx[k] >= s) {
        const int i = tid + k * NT;
        float xv = 0.f;
        const int gx = ox + i % EX, gy = oy + i / EX;
        if (INTERIOR || (gx >= 0 && gx < nx && gy >= 0 && gy < ny)) {
          float d = 0.f;
          if (INTERIOR || gx < nx - 1) d += z1[i];
          if (INTERIOR || gx > 0) d -= z1[i - 1];
          if (INTERIOR || gy < ny - 1) d += z2[i];
          if (INTERIOR || gy > 0) d -= z2[i - EX];
          xv = fmaf(tau, d, sv[i]);
          if (NONNEG) xv = fmaxf(xv, 0.f);
        }
        sx[i] = xv;
      }
    }
    __syncthreads();
    const float m = mom.c[s];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      if (dw[k] >= s) {
        const int i = tid + k * NT;
        float n1 = 0.f, n2 = 0.f, m1 = 0.f, m2 = 0.f;
        const int gx = ox + i % EX, gy = oy + i / EX;
        if (INTERIOR || (gx >= 0 && gx < nx && gy >= 0 && gy < ny)) {
          const float xc = sx[i];
          const float d1 = (INTERIOR || gx < nx - 1) ? sx[i + 1] - xc : 0.f;
          const float d2 = (INTERIOR || gy < ny - 1) ? sx[i + EX] - xc : 0.f;
          ball2(fmaf(step, d1, z1[i]), fmaf(step, d2, z2[i]), n1, n2);
          m1 = fmaf(m, n1 - w1[i], n1);
          m2 = fmaf(m, n2 - w2[i], n2);
        }
        w1[i] = n1;
        w2[i] = n2;
        z1[i] = m1;
        z2[i] = m2;
      }
    }
    __syncthreads();
  }
}

// One output tile (bx, by) of a blocked launch with the whole grown tile in shared memory;
// smf: dynamic shared memory (6 TL::NE floats).
template <class TL>
__device__ __forceinline__ void fgp2d_block_item_smem(const FgpBlockArgs& A, int bx, int by, float* smf) {
  constexpr int EX = TL::EX, EY = TL::EY, NE = TL::NE, NT = TL::NT;
  const float* __restrict__ v = A.v;
  const float* __restrict__ w_g = A.w;
  const float* __restrict__ z_g = A.z;
  float* __restrict__ wn_g = A.wn;
  float* __restrict__ zn_g = A.zn;
  const int nx = A.nx, ny = A.ny, nsteps = A.nsteps;
  const float tau = A.tau, step = A.step;
  const MomBlock& mom = A.mom;
  float* sv = smf;
  float* w1 = sv + NE;
  float* w2 = w1 + NE;
  float* z1 = w2 + NE;
  float* z2 = z1 + NE;
  float* sx = z2 + NE;
  const int tid = threadIdx.x;
  const int ox = bx * TL::TX - FB_T, oy = by * TL::TY - FB_T;
  const size_t n = (size_t)nx * ny;
  for (int i = tid; i < NE; i += NT) {
    const int gx = ox + i % EX, gy = oy + i / EX;
    float vv = 0.f, a = 0.f, b = 0.f, za = 0.f, zb = 0.f;
    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
      const size_t p = (size_t)gy * nx + gx;
      vv = v[p];
      a = w_g[p];
      b = w_g[n + p];
      za = z_g[p];
      zb = z_g[n + p];
    }
    sv[i] = vv;
    w1[i] = a;
    w2[i] = b;
    z1[i] = za;
    z2[i] = zb;
  }
  __syncthreads();
  const bool interior = ox >= 1 && oy >= 1 && ox + EX <= nx - 1 && oy + EY <= ny - 1;
  if (A.nonneg) {
    if (interior)
      fgp2d_steps_smem<TL, true, true>(sv, w1, w2, z1, z2, sx, ox, oy, nx, ny, tau, step, mom, nsteps);
    else
      fgp2d_steps_smem<TL, false, true>(sv, w1, w2, z1, z2, sx, ox, oy, nx, ny, tau, step, mom, nsteps);
  } else {
    if (interior)
      fgp2d_steps_smem<TL, true, false>(sv, w1, w2, z1, z2, sx, ox, oy, nx, ny, tau, step, mom, nsteps);
    else
      fgp2d_steps_smem<TL, false, false>(sv, w1, w2, z1, z2, sx, ox, oy, nx, ny, tau, step, mom, nsteps);
  }
  for (int q = tid; q < TL::TX * TL::TY; q += NT) {
    const int lx = FB_T + q % TL::TX, ly = FB_T + q / TL::TX;
    const int gx = ox + lx, gy = oy + ly;
    if (gx < nx && gy < ny) {
      const size_t p = (size_t)gy * nx + gx;
      const int i = ly * EX + lx;
      wn_g[p] = w1[i];
      wn_g[n + p] = w2[i];
      zn_g[p] = z1[i];
      zn_g[n + p] = z2[i];
    }
  }
}

template <class TL>
__global__ void __launch_bounds__(TL::NT, 2) fgp2d_block(const __grid_constant__ FgpBlockArgs A) {
  extern __shared__ float smf[];
  fgp2d_block_item<TL>(A, blockIdx.x, blockIdx.y, smf, A.mom.c);
}

// All blocks of one 2D prox call in one cooperative launch (every CTA resident): CTA (bx, by)
// runs its tile's block, and the CTAs meet at a grid barrier before the next block reads the
// halos its neighbours wrote.  Same item function, same buffers, same order as one launch per
// block: the same bits, without the relaunch between blocks.
constexpr int FGP_COOP_MAX_BLOCKS = (256 + FB_T - 1) / FB_T;   // up to 256 iterations per prox call
constexpr unsigned FGP_BARRIER_LIMIT = 1u << 22;   // bounded polls of a grid barrier
struct FgpCoopArgs {
  const float* v;
  const float* w0;            // initial dual (also the first block's extrapolated dual)
  float* pair[2][2];          // (w, z) buffer pairs, alternating per block
  int nx, ny, iters, nblocks, nonneg;
  float tau, step;
  unsigned long long* bar;    // arrival counter, zero at launch
  unsigned* err;              // device error word (bit 4: a barrier wait expired)
  MomBlock mom[FGP_COOP_MAX_BLOCKS];
};

// Grid barrier number b (0-based) of nctas CTAs on a counter that was zero at launch: thread 0
// publishes the CTA's writes, arrives, and polls (bounded) until every CTA has arrived b + 1
// times; an expired wait sets the error word and lets the CTA go on (its results are then not
// used: the host reports the timeout).
__device__ __forceinline__ void fgp_grid_barrier(unsigned long long* bar, unsigned long long target, unsigned* err,
                                                 unsigned limit = FGP_BARRIER_LIMIT) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1ull);
    unsigned long long seen = 0;
    unsigned it = 0;
    for (;;) {
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(seen) : "l"(bar) : "memory");
      if (seen >= target || ++it >= limit) break;
      __nanosleep(32);
    }
    if (seen < target) atomicOr(err, 4u);
    __threadfence();
  }
  __syncthreads();
}

// The barrier's expiry path: a single CTA waits for a second arrival that never comes.
__global__ void bounded_wait_probe(unsigned long long* bar, unsigned* err, unsigned polls) {
  fgp_grid_barrier(bar, 2ull, err, polls);
}

template <class TL>
__global__ void __launch_bounds__(TL::NT, 2) fgp2d_coop(const __grid_constant__ FgpCoopArgs C) {
  extern __shared__ float smf[];
  const unsigned long long nctas = (unsigned long long)gridDim.x * gridDim.y;
  const float* rw = C.w0;
  const float* rz = C.w0;
  for (int b = 0; b < C.nblocks; ++b) {
    const int ns = min(FB_T, C.iters - b * FB_T);
    float* wn = C.pair[b & 1][0];
    float* zn = C.pair[b & 1][1];
    FgpBlockArgs A;
    A.v = C.v;
    A.w = rw;
    A.z = rz;
    A.wn = wn;
    A.zn = zn;
    A.nx = C.nx;
    A.ny = C.ny;
    A.tau = C.tau;
    A.step = C.step;
    A.nsteps = ns;
    A.nonneg = C.nonneg;
    fgp2d_block_item<TL>(A, blockIdx.x, blockIdx.y, smf, C.mom[b].c);
    rw = wn;
    rz = zn;
    if (b + 1 < C.nblocks) fgp_grid_barrier(C.bar, nctas * (unsigned long long)(b + 1), C.err);
  }
}

// x+ = P_+(v + tau div w) and the fused tail.  32x32 tile, block 32x8 (4 rows per thread).
__device__ __forceinline__ void fgp2d_out_item(const FgpOutArgs& A, int tbx, int tby, float (*tile)[33]) {
  const float* __restrict__ v = A.v;
  const float* __restrict__ w = A.w;
  float* wdst = A.wdst;
  const int nx = A.nx, ny = A.ny, nonneg = A.nonneg;
  const float tau = A.tau;
  const ProxTail& t = A.t;
  const int bx = tbx * 32, by = tby * 32;
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
        if (t.h) t.h[p] = fmaf(t.p_over_gamma, __fsub_rn(xp, t.xhat[p]), t.h[p]);
        if (t.xprox) t.xprox[p] = xp;
        if (t.y) {
          const float yv = fmaf(t.mom, __fsub_rn(xp, xold), xp);
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

__global__ void __launch_bounds__(256) fgp2d_out(FgpOutArgs A) {
  __shared__ float tile[32][33];
  fgp2d_out_item(A, blockIdx.x, blockIdx.y, tile);
}

// ---------------------------------------------------------------- 3D

__device__ __forceinline__ float zval(const float* wc, const float* wp, size_t idx, float mom) {
  const float c = wc[idx];
  return mom != 0.f ? fmaf(mom, __fsub_rn(c, wp[idx]), c) : c;
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

// One FGP iteration in 3D as a 2.5-D streaming stencil.  A CTA owns a F3_TX x F3_TY tile of
// z columns and walks a chunk of zc planes (tunable; by default sized to the volume).  Per
// plane it builds the extrapolated dual z = w_k + mom (w_k - w_{k-1}) on the tile grown by one
// voxel, then x = P_+(v + tau div z) on the tile grown by one voxel on the + sides; the new
// dual of plane g is finished once x of plane g+1 exists.  Each voxel's v, w_k, w_{k-1} are
// read about once (plus the tile halo) and w_{k+1} written once: 10 floats per voxel per
// iteration.  The z tiles of consecutive planes alternate between two shared buffers (the
// divergence needs the previous plane's z component), so a plane costs two barriers; every
// thread keeps fixed halo slots whose offsets are computed once per chunk, and the v loads of
// a plane are issued together with its dual loads.
constexpr int F3_TX = FGP3_TX, F3_TY = FGP3_TY, F3_ZC = FGP3_ZC;
constexpr int F3_HX = F3_TX + 2, F3_HY = F3_TY + 2;   // z tile with a one-voxel halo
constexpr int F3_XX = F3_TX + 1, F3_XY = F3_TY + 1;   // x tile with the + halo
constexpr int F3_NT = F3_TX * F3_TY;
constexpr int F3_NZ = F3_HX * F3_HY, F3_NX = F3_XX * F3_XY;   // halo slots of the z and x tiles
static_assert(F3_NZ <= 2 * F3_NT && F3_NX <= 2 * F3_NT, "two halo slots per thread");

__device__ __forceinline__ void fgp3d_stream_item(const float* __restrict__ v, const float* __restrict__ wc,
                                                  const float* __restrict__ wp, float* __restrict__ wn, Dims3 D,
                                                  float tau, float step, float mom, int nonneg, int zc, int bx, int by,
                                                  int bz) {
  __shared__ float zs[2][3][F3_NZ];      // extrapolated dual of two consecutive planes (+ halo)
  __shared__ float xs[2][F3_XY][F3_XX];  // x of two consecutive planes
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * F3_TX + tx;
  const int ix0 = bx * F3_TX, iy0 = by * F3_TY;
  const int zb = bz * zc, ze = min(zb + zc, D.nz);
  const size_t nxy = (size_t)D.nx * D.ny;
  // z-tile slots e = tid, tid + F3_NT: in-plane offset (planes hold < 2^31 voxels), or -1
  // outside the volume / tile
  int zoff[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int e = tid + k * F3_NT;
    const int ly = e / F3_HX, lx = e - ly * F3_HX;
    const int gx = ix0 + lx - 1, gy = iy0 + ly - 1;
    zoff[k] = (e < F3_NZ && gx >= 0 && gx < D.nx && gy >= 0 && gy < D.ny) ? gy * D.nx + gx : -1;
  }
  // x-tile slots: in-plane offset (or -1); z-tile index of the slot's voxel | neighbour mask << 16
  int xoff[2], xzm[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int e = tid + k * F3_NT;
    const int ly = e / F3_XX, lx = e - ly * F3_XX;
    const int gx = ix0 + lx, gy = iy0 + ly;
    const bool in = e < F3_NX && gx < D.nx && gy < D.ny;
    xoff[k] = in ? gy * D.nx + gx : -1;
    xzm[k] = ((ly + 1) * F3_HX + lx + 1) |
             (((gx < D.nx - 1 ? 1 : 0) | (gx > 0 ? 2 : 0) | (gy < D.ny - 1 ? 4 : 0) | (gy > 0 ? 8 : 0)) << 16);
  }
  auto buf_of = [&](int g) { return (g - zb + 1) & 1; };   // plane zb - 1 in buffer 0
  auto load_z = [&](int g, bool only_z3) {
    float* Z = &zs[buf_of(g)][0][0];
    const size_t base = (size_t)g * nxy;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int e = tid + k * F3_NT;
      if (k == 1 && e >= F3_NZ) break;
      float a = 0.f, b = 0.f, c = 0.f;
      if (zoff[k] >= 0) {
        const size_t p = base + (size_t)zoff[k];
        if (!only_z3) {
          a = zval(wc, wp, p, mom);
          b = zval(wc, wp, D.n + p, mom);
        }
        c = zval(wc, wp, 2 * D.n + p, mom);
      }
      Z[e] = a;
      Z[F3_NZ + e] = b;
      Z[2 * F3_NZ + e] = c;
    }
  };
  auto load_v = [&](int g, float* vr) {
    const size_t base = (size_t)g * nxy;
#pragma unroll
    for (int k = 0; k < 2; ++k) vr[k] = xoff[k] >= 0 ? __ldg(v + base + (size_t)xoff[k]) : 0.f;
  };
  auto comp_x = [&](int g, const float* vr, float (*xb)[F3_XX]) {
    const float* Z = &zs[buf_of(g)][0][0];
    const float* Zp = &zs[buf_of(g) ^ 1][2][0];   // z component of plane g - 1
    const bool up = g < D.nz - 1, down = g > 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int e = tid + k * F3_NT;
      if (k == 1 && e >= F3_NX) break;
      float xv = 0.f;
      if (xoff[k] >= 0) {
        const int q = xzm[k] & 0xffff, m = xzm[k] >> 16;
        float d = 0.f;
        if (m & 1) d += Z[q];
        if (m & 2) d -= Z[q - 1];
        if (m & 4) d += Z[F3_NZ + q];
        if (m & 8) d -= Z[F3_NZ + q - F3_HX];
        if (up) d += Z[2 * F3_NZ + q];
        if (down) d -= Zp[q];
        xv = fmaf(tau, d, vr[k]);
        if (nonneg) xv = fmaxf(xv, 0.f);
      }
      (&xb[0][0])[e] = xv;
    }
  };
  // prologue: z3 of the plane below the chunk, then plane zb and its x
  float vr[2];
  if (zb > 0) load_z(zb - 1, true);
  load_v(zb, vr);
  load_z(zb, false);
  __syncthreads();
  comp_x(zb, vr, xs[0]);
  __syncthreads();
  const int gx = ix0 + tx, gy = iy0 + ty;
  const bool own = gx < D.nx && gy < D.ny;
  const int oq = (ty + 1) * F3_HX + tx + 1;
  const float* Z0 = &zs[buf_of(zb)][0][0];
  float zo0 = Z0[oq], zo1 = Z0[F3_NZ + oq], zo2 = Z0[2 * F3_NZ + oq];
  for (int g = zb; g < ze; ++g) {
    const int cur = (g - zb) & 1, nxt = cur ^ 1;
    const bool more = g + 1 < D.nz;
    if (more) {
      load_v(g + 1, vr);
      load_z(g + 1, false);
      __syncthreads();
      comp_x(g + 1, vr, xs[nxt]);
      __syncthreads();
    }
    if (own) {
      const float xc = xs[cur][ty][tx];
      const float d1 = gx < D.nx - 1 ? xs[cur][ty][tx + 1] - xc : 0.f;
      const float d2 = gy < D.ny - 1 ? xs[cur][ty + 1][tx] - xc : 0.f;
      const float d3 = more ? xs[nxt][ty][tx] - xc : 0.f;
      const float q1 = fmaf(step, d1, zo0), q2 = fmaf(step, d2, zo1), q3 = fmaf(step, d3, zo2);
      // projection onto the unit ball: q / max(1, |q|)
      const float n2 = fmaf(q3, q3, fmaf(q2, q2, __fmul_rn(q1, q1)));
      const float inv = n2 > 1.f ? __frcp_rn(__fsqrt_rn(n2)) : 1.f;
      const size_t p = (size_t)g * nxy + (size_t)gy * D.nx + gx;
      wn[p] = __fmul_rn(q1, inv);
      wn[D.n + p] = __fmul_rn(q2, inv);
      wn[2 * D.n + p] = __fmul_rn(q3, inv);
    }
    if (more) {
      const float* Zn = &zs[buf_of(g + 1)][0][0];
      zo0 = Zn[oq];
      zo1 = Zn[F3_NZ + oq];
      zo2 = Zn[2 * F3_NZ + oq];
    }
  }
}

__global__ void __launch_bounds__(F3_TX * F3_TY, 4) fgp3d_stream(const float* __restrict__ v, const float* __restrict__ wc,
                                                             const float* __restrict__ wp, float* __restrict__ wn,
                                                             Dims3 D, float tau, float step, float mom, int nonneg,
                                                             int zc) {
  fgp3d_stream_item(v, wc, wp, wn, D, tau, step, mom, nonneg, zc, blockIdx.x, blockIdx.y, blockIdx.z);
}

__device__ __forceinline__ void fgp3d_out_item(const float* __restrict__ v, const float* __restrict__ w, float* wdst,
                                               Dims3 D, float tau, int nonneg, const ProxTail& t, int bx, int by,
                                               int gz) {
  const int gx = bx * 32 + threadIdx.x;
  const int gy = by * 8 + threadIdx.y;
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
  if (t.h) t.h[p] = fmaf(t.p_over_gamma, __fsub_rn(xp, t.xhat[p]), t.h[p]);
  if (t.xprox) t.xprox[p] = xp;
  if (t.y) t.y[p] = fmaf(t.mom, __fsub_rn(xp, xold), xp);
}

__global__ void __launch_bounds__(256) fgp3d_out(const float* __restrict__ v, const float* __restrict__ w,
                                                 float* wdst, Dims3 D, float tau, int nonneg, ProxTail t) {
  fgp3d_out_item(v, w, wdst, D, tau, nonneg, t, blockIdx.x, blockIdx.y, blockIdx.z);
}

}  // namespace

std::vector<MomBlock> fgp_momentum(int iters) {
  // t_0 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2 in float64; the z formed after iteration k
  // extrapolates with (t_k - 1) / t_{k+1}; none after the call's last iteration
  std::vector<MomBlock> out;
  double t_cur = 1.0;
  for (int k0 = 0; k0 < iters; k0 += FB_T) {
    const int ns = iters - k0 < FB_T ? iters - k0 : FB_T;
    MomBlock mb;
    for (int q = 0; q <= FB_T; ++q) {
      mb.c[q] = 0.f;
      if (q < ns) {
        const double t_next = (1.0 + std::sqrt(1.0 + 4.0 * t_cur * t_cur)) / 2.0;
        if (k0 + q + 1 < iters) mb.c[q] = (float)((t_cur - 1.0) / t_next);
        t_cur = t_next;
      }
    }
    out.push_back(mb);
  }
  return out;
}

Fgp3Schedule fgp3_schedule(int iters) {
  // iteration k extrapolates with (t_{k-1} - 1) / t_k (0 for k = 0, 1), t_0 = 1,
  // t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2 in float64; three buffers rotate, buffer 0 holding
  // the warm-started dual
  Fgp3Schedule S;
  int cur = 0, prev = 0;
  double t_prev = 1.0, t_cur = 1.0;
  for (int k = 0; k < iters; ++k) {
    const int nxt = (k == 0) ? 1 : 3 - cur - prev;
    const float mk = k >= 1 ? (float)((t_prev - 1.0) / t_cur) : 0.f;
    t_prev = t_cur;
    t_cur = (1.0 + std::sqrt(1.0 + 4.0 * t_cur * t_cur)) / 2.0;
    S.cur.push_back(cur);
    S.prev.push_back(prev);
    S.nxt.push_back(nxt);
    S.mom.push_back(mk);
    prev = cur;
    cur = nxt;
  }
  S.final_buf = cur;
  return S;
}

int fgp3_zc(const vrps_geom* g) {
  if (g->tune_f3_zc > 0) return g->tune_f3_zc;
  // untuned: the longest chunk that still gives about 8 CTAs per SM (the streaming iteration
  // is latency-bound; shorter chunks add one prologue plane each)
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 148;
  const long long tiles = (long long)((g->nx + F3_TX - 1) / F3_TX) * ((g->ny + F3_TY - 1) / F3_TY);
  for (int zc = F3_ZC; zc > 4; zc /= 2)
    if (tiles * ((g->nz + zc - 1) / zc) >= 8LL * sms) return zc;
  return 4;
}

int fgp_prepare(vrps_geom* g) {
  Workspace& ws = g->ws;
  const size_t dn = (size_t)g->dims * (size_t)g->n;
  VRPS_TRY(ensure(&ws.dual_s1, dn));
  VRPS_TRY(ensure(&ws.dual_s2, dn));
  if (g->dims == 2) {
    VRPS_TRY(ensure(&ws.dual_s3, dn));
    VRPS_TRY(ensure(&ws.dual_s4, dn));
    if (!ws.fgp_bar) {
      VRPS_CUDA(cudaMalloc((void**)&ws.fgp_bar, sizeof(unsigned long long)));
      VRPS_CUDA(cudaMemset(ws.fgp_bar, 0, sizeof(unsigned long long)));
    }
    if (!ws.dev_error) {
      VRPS_CUDA(cudaMalloc((void**)&ws.dev_error, sizeof(unsigned)));
      VRPS_CUDA(cudaMemset(ws.dev_error, 0, sizeof(unsigned)));
    }
  }
  return VRPS_OK;
}

// The 32-wide tile for an nx x ny image: the busiest SM runs ceil(tiles / SMs) tiles, each
// costing its grown tile's pixel-iterations over a block (the valid region shrinking one pixel
// per side per iteration); the height (32 or 27 rows) with the least such work wins, 32 on
// ties.  27 rows fill the resident slots evenly where 32 leave part of the last wave empty
// (512^2: 304 tiles for 2 x 152 slots instead of 256).
static bool fgp_low_tile(int nx, int ny) {
  thread_local int last_dev = -1, last_nx = -1, last_ny = -1, sms = 0;
  thread_local bool last_low = false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (dev == last_dev && nx == last_nx && ny == last_ny) return last_low;
  if (dev != last_dev && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return false;
  auto cost = [&](int tx, int ty, int ex) {
    const long long tiles = (long long)((nx + tx - 1) / tx) * ((ny + ty - 1) / ty);
    double work = 0.0;
    for (int q = 0; q < FB_T; ++q) work += (double)(ex - 2 * q) * (double)(ty + 2 * FB_T - 2 * q);
    return (double)((tiles + sms - 1) / sms) * work;
  };
  last_low = cost(TileLow::TX, TileLow::TY, TileLow::EX) < cost(TileLarge::TX, TileLarge::TY, TileLarge::EX);
  last_dev = dev;
  last_nx = nx;
  last_ny = ny;
  return last_low;
}

// One cooperative launch of fgp2d_coop<TL> for all blocks; *done = false (and nothing launched)
// when the tiles do not all fit the resident slots.
template <class TL>
static int fgp2d_coop_launch(const FgpCoopArgs& C, int ty, cudaStream_t s, bool* done) {
  *done = false;
  const int tiles_x = (C.nx + TL::TX - 1) / TL::TX, tiles_y = (C.ny + ty - 1) / ty;
  int dev = 0, sms = 0, per = 0;
  VRPS_CUDA(cudaGetDevice(&dev));
  VRPS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  VRPS_TRY(smem_opt_in((const void*)fgp2d_coop<TL>, TL::SMEM));
  VRPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fgp2d_coop<TL>, TL::NT, TL::SMEM));
  if ((long long)tiles_x * tiles_y > (long long)per * sms) return VRPS_OK;
  VRPS_CUDA(cudaMemsetAsync(C.bar, 0, sizeof(unsigned long long), s));
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(tiles_x, tiles_y);
  cfg.blockDim = dim3(TL::NT);
  cfg.dynamicSmemBytes = TL::SMEM;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  {
    LaunchScope _ls("fgp2d_coop", s, 4.0 * (double)C.nx * C.ny * (7.0 + 9.0 * (C.nblocks - 1)));
    const cudaError_t e = cudaLaunchKernelEx(&cfg, fgp2d_coop<TL>, C);
    if (e != cudaSuccess)
      return launch_fail(e, "fgp2d_coop", (const void*)fgp2d_coop<TL>, cfg.gridDim, cfg.blockDim, TL::SMEM);
  }
  VRPS_LAUNCHED("fgp2d_coop");
  *done = true;
  return VRPS_OK;
}

int fgp2d_iterate(const float* v, const float* w0, float* const pairs[2][2], int nx, int ny, float tau, int iters,
                  int nonneg, int tile, cudaStream_t s, const float** w_final, unsigned long long* coop_bar,
                  unsigned* err) {
  // blocks of FB_T iterations; the (w, z) state alternates between pairs[0] and pairs[1].  The
  // first block starts from z = w0 (iteration 0 does not extrapolate).
  const float step = (float)(1.0 / (8.0 * (double)tau));
  const float* rw = w0;
  const float* rz = w0;
  int which = 0;
  VRPS_TRY(smem_opt_in((const void*)fgp2d_block<TileLarge>, TileLarge::SMEM));
  VRPS_TRY(smem_opt_in((const void*)fgp2d_block<TileWide>, TileWide::SMEM));
  VRPS_TRY(smem_opt_in((const void*)fgp2d_block<TileSmall>, TileSmall::SMEM));
  VRPS_TRY(smem_opt_in((const void*)fgp2d_block<TileLow>, TileLow::SMEM));
  const std::vector<MomBlock> moms = fgp_momentum(iters);
  const double n = (double)nx * ny;
  const int nblocks = (iters + FB_T - 1) / FB_T;
  if (coop_bar && err && nblocks > 1 && nblocks <= FGP_COOP_MAX_BLOCKS && (tile == 0 || tile >= 3)) {
    // the 32-wide tiles in one cooperative launch
    FgpCoopArgs C;
    std::memset(&C, 0, sizeof(C));
    C.v = v;
    C.w0 = w0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) C.pair[a][b] = pairs[a][b];
    C.nx = nx;
    C.ny = ny;
    C.iters = iters;
    C.nblocks = nblocks;
    C.nonneg = nonneg;
    C.tau = tau;
    C.step = step;
    C.bar = coop_bar;
    C.err = err;
    for (int b = 0; b < nblocks; ++b) C.mom[b] = moms[b];
    const bool low = tile == 4 || (tile == 0 && fgp_low_tile(nx, ny));
    bool done = false;
    if (low) VRPS_TRY(fgp2d_coop_launch<TileLow>(C, TileLow::TY, s, &done));
    else VRPS_TRY(fgp2d_coop_launch<TileLarge>(C, TileLarge::TY, s, &done));
    if (done) {
      *w_final = pairs[(nblocks - 1) & 1][0];
      return VRPS_OK;
    }
  }
  for (int k0 = 0; k0 < iters; k0 += FB_T) {
    const int ns = iters - k0 < FB_T ? iters - k0 : FB_T;
    const MomBlock& mb = moms[k0 / FB_T];
    float* wn = pairs[which][0];
    float* zn = pairs[which][1];
    {
      // read v, w and z (one array when z = w), write w and z
      LaunchScope _ls("fgp2d_block", s, 4.0 * n * (rz == rw ? 7 : 9));
      const FgpBlockArgs A{v, rw, rz, wn, zn, nx, ny, tau, step, mb, ns, nonneg};
      auto launch = [&](auto kern, auto tl) -> cudaError_t {
        using TL = decltype(tl);
        dim3 grid((nx + TL::TX - 1) / TL::TX, (ny + TL::TY - 1) / TL::TY);
        return launch_kernel(kern, grid, dim3(TL::NT), (size_t)TL::SMEM, s, A);
      };
      // tile 0: 32 x 32 or 32 x 27 by fgp_low_tile; 3: 32 x 32; 4: 32 x 27; 1, 2: smaller tiles
      const bool low = tile == 4 || (tile == 0 && fgp_low_tile(nx, ny));
      if (tile == 1) VRPS_CUDA(launch(fgp2d_block<TileWide>, TileWide{}));
      else if (tile == 2) VRPS_CUDA(launch(fgp2d_block<TileSmall>, TileSmall{}));
      else if (low) VRPS_CUDA(launch(fgp2d_block<TileLow>, TileLow{}));
      else VRPS_CUDA(launch(fgp2d_block<TileLarge>, TileLarge{}));
    }
    VRPS_LAUNCHED("fgp2d_block");
    rw = wn;
    rz = zn;
    which ^= 1;
  }
  *w_final = rw;
  return VRPS_OK;
}

int fgp2d_output(const float* v, const float* w, float* wdst, int nx, int ny, float tau, int nonneg,
                 const ProxTail& t, cudaStream_t s) {
  dim3 grid((nx + 31) / 32, (ny + 31) / 32), block(32, 8);
  {
    const double n = (double)nx * ny;
    LaunchScope _ls("fgp2d_out", s, 4.0 * n * (wdst ? 5 : 3) + tail_bytes(t, (size_t)nx * ny));
    const FgpOutArgs A{v, w, wdst, nx, ny, tau, nonneg, t};
    VRPS_CUDA(launch_kernel(fgp2d_out, dim3(grid), dim3(block), (size_t)(0), s, A));
  }
  VRPS_LAUNCHED("fgp_out");
  return VRPS_OK;
}

int fgp_run(const vrps_geom* g, const float* v, float tau, int iters, int nonneg, float* dual,
            const ProxTail& tail, cudaStream_t s) {
  vrps_geom* gm = const_cast<vrps_geom*>(g);
  Workspace& ws = gm->ws;
  if (iters > 0) VRPS_TRY(fgp_prepare(gm));
  // momentum: fgp_momentum (2D blocks) and fgp3_schedule (3D iterations)
  const float step = (float)(1.0 / (4.0 * g->dims * (double)tau));
  const float* w_final = dual;
  if (g->dims == 2) {
    float* pairs[2][2] = {{ws.dual_s1, ws.dual_s2}, {ws.dual_s3, ws.dual_s4}};
    VRPS_TRY(fgp2d_iterate(v, dual, pairs, g->nx, g->ny, tau, iters, nonneg, g->tune_fgp_tile, s, &w_final,
                           ws.fgp_bar, ws.dev_error));
  } else {
    float* buf[3] = {dual, ws.dual_s1, ws.dual_s2};
    const Fgp3Schedule sch = fgp3_schedule(iters);
    Dims3 D{g->nx, g->ny, g->nz, (size_t)g->n};
    const int zc = fgp3_zc(g);
    dim3 grid((g->nx + F3_TX - 1) / F3_TX, (g->ny + F3_TY - 1) / F3_TY, (g->nz + zc - 1) / zc);
    for (int k = 0; k < iters; ++k) {
      const float mk = sch.mom[k];
      {
        // read v, w_k (and w_{k-1} when extrapolating), write w_{k+1}
        LaunchScope _ls("fgp3d_stream", s, 4.0 * g->n * (mk != 0.f ? 10 : 7));
        VRPS_CUDA(launch_kernel(fgp3d_stream, grid, dim3(F3_TX, F3_TY), (size_t)0, s, v, (const float*)buf[sch.cur[k]],
                                (const float*)buf[sch.prev[k]], buf[sch.nxt[k]], D, tau, step, mk, nonneg, zc));
      }
      VRPS_LAUNCHED("fgp_iter");
    }
    w_final = buf[sch.final_buf];
  }
  float* wdst = (w_final != dual) ? dual : nullptr;
  if (g->dims == 2) {
    VRPS_TRY(fgp2d_output(v, w_final, wdst, g->nx, g->ny, tau, nonneg, tail, s));
    return VRPS_OK;
  } else {
    Dims3 D{g->nx, g->ny, g->nz, (size_t)g->n};
    dim3 grid((g->nx + 31) / 32, (g->ny + 7) / 8, g->nz), block(32, 8);
    {
      LaunchScope _ls("fgp3d_out", s, 4.0 * g->n * (wdst ? 7 : 4) + tail_bytes(tail, (size_t)g->n));
      VRPS_CUDA(launch_kernel(fgp3d_out, dim3(grid), dim3(block), (size_t)(0), s, v, w_final, wdst, D, tau, nonneg, tail));
    }
  }
  VRPS_LAUNCHED("fgp_out");
  return VRPS_OK;
}

}  // namespace vrps

// ---------------------------------------------------------------- batched 2D prox
namespace vrps {
namespace {

__device__ __forceinline__ int fgp_batch_job(const int* pre, int n, int item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Launch b of every prox call of the tick: the tiles of all jobs with more than b blocks.
__device__ __forceinline__ int fgp_batch_next(unsigned* counter, int* s_item) {
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) *s_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  return *s_item;
}

__global__ void __launch_bounds__(TileLarge::NT) fgp2d_block_batched_kernel(char* __restrict__ slot, int b) {
  extern __shared__ float smf[];
  __shared__ int pre[BATCH_MAX_JOBS + 1];
  __shared__ int s_item;
  const TickHeader& H = *reinterpret_cast<const TickHeader*>(slot);
  const int n = H.n_prox;
  if (n <= 0) return;
  unsigned* counter = reinterpret_cast<TickHeader*>(slot)->cnt + 3 + b;
  const BatchFgp* jobs = reinterpret_cast<const BatchFgp*>(slot + H.off_fgp);
  const int* src = reinterpret_cast<const int*>(slot + H.off_pfgp) + (size_t)b * (n + 1);
  for (int i = threadIdx.x; i <= n; i += blockDim.x) pre[i] = src[i];
  __syncthreads();
  const int total = pre[n];
  for (int item = fgp_batch_next(counter, &s_item); item < total; item = fgp_batch_next(counter, &s_item)) {
    const int j = fgp_batch_job(pre, n, item);
    const BatchFgp& J = jobs[j];
    const int local = item - pre[j];
    fgp2d_block_item_smem<TileLarge>(J.A[b], local % J.tiles_x, local / J.tiles_x, smf);
  }
}

__global__ void __launch_bounds__(256) fgp2d_out_batched_kernel(char* __restrict__ slot) {
  __shared__ float tile[32][33];
  __shared__ int pre[BATCH_MAX_JOBS + 1];
  __shared__ int s_item;
  const TickHeader& H = *reinterpret_cast<const TickHeader*>(slot);
  const int n = H.n_prox;
  if (n <= 0) return;
  unsigned* counter = reinterpret_cast<TickHeader*>(slot)->cnt + 2;
  const BatchOut* jobs = reinterpret_cast<const BatchOut*>(slot + H.off_out);
  const int* src = reinterpret_cast<const int*>(slot + H.off_pout);
  for (int i = threadIdx.y * blockDim.x + threadIdx.x; i <= n; i += blockDim.x * blockDim.y) pre[i] = src[i];
  __syncthreads();
  const int total = pre[n];
  for (int item = fgp_batch_next(counter, &s_item); item < total; item = fgp_batch_next(counter, &s_item)) {
    const int j = fgp_batch_job(pre, n, item);
    const BatchOut& J = jobs[j];
    const int local = item - pre[j];
    fgp2d_out_item(J.A, local % J.tiles_x, local / J.tiles_x, tile);
  }
}

}  // namespace

int fgp2d_block_batched(char* slot, int b, int grid, cudaStream_t s) {
  VRPS_TRY(smem_opt_in((const void*)fgp2d_block_batched_kernel, BATCHED_FGP_SMEM));
  LaunchScope _ls("fgp2d_block_batched", s);
  VRPS_CUDA(launch_kernel(fgp2d_block_batched_kernel, dim3(grid), dim3(TileLarge::NT), (size_t)BATCHED_FGP_SMEM, s,
                          slot, b));
  return VRPS_OK;
}

int fgp2d_out_batched(char* slot, int grid, cudaStream_t s) {
  LaunchScope _ls("fgp2d_out_batched", s);
  VRPS_CUDA(launch_kernel(fgp2d_out_batched_kernel, dim3(grid), dim3(32, 8), (size_t)0, s, slot));
  return VRPS_OK;
}

int batched_grid(int which, size_t smem, int* grid) {
  if (which <= 1) return batched_grid_2d(which, smem, grid);
  int dev = 0, sms = 0, per = 0;
  VRPS_CUDA(cudaGetDevice(&dev));
  VRPS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (which == 2) {
    VRPS_TRY(smem_opt_in((const void*)fgp2d_block_batched_kernel, BATCHED_FGP_SMEM));
    VRPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fgp2d_block_batched_kernel, TileLarge::NT,
                                                             BATCHED_FGP_SMEM));
  } else {
    VRPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fgp2d_out_batched_kernel, 256, 0));
  }
  *grid = (per < 1 ? 1 : per) * sms;
  return VRPS_OK;
}

}  // namespace vrps

// ---------------------------------------------------------------- batched 3D prox
namespace vrps {
namespace {

__device__ __forceinline__ int f3_next(unsigned* counter, int* s_item) {
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) *s_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  return *s_item;
}

// Iteration `it` of every 3D prox call of the tick (jobs with fewer iterations have no items).
__global__ void __launch_bounds__(F3_TX * F3_TY, 4) fgp3d_iter_batched_kernel(char* __restrict__ slot, int it) {
  __shared__ int pre[BATCH_MAX_JOBS + 1];
  __shared__ int s_item;
  const TickHeader3& H = *reinterpret_cast<const TickHeader3*>(slot);
  const int n = H.n_prox;
  if (n <= 0) return;
  unsigned* counter = reinterpret_cast<TickHeader3*>(slot)->cnt + 4 + it;
  const BatchFgp3* jobs = reinterpret_cast<const BatchFgp3*>(slot + H.off_fgp);
  const int* src = reinterpret_cast<const int*>(slot + H.off_pfgp) + (size_t)it * (n + 1);
  for (int i = threadIdx.y * blockDim.x + threadIdx.x; i <= n; i += blockDim.x * blockDim.y) pre[i] = src[i];
  __syncthreads();
  const int total = pre[n];
  for (int item = f3_next(counter, &s_item); item < total; item = f3_next(counter, &s_item)) {
    const int j = fgp_batch_job(pre, n, item);
    const BatchFgp3& J = jobs[j];
    const int local = item - pre[j];
    const int per = J.tiles_x * J.tiles_y;
    const int bz = local / per, tl = local - bz * per;
    fgp3d_stream_item(J.v, J.buf[J.cur[it]], J.buf[J.prev[it]], J.buf[J.nxt[it]], J.D, J.tau, J.step, J.mom[it],
                      J.nonneg, J.zc, tl % J.tiles_x, tl / J.tiles_x, bz);
  }
}

__global__ void __launch_bounds__(256) fgp3d_out_batched_kernel(char* __restrict__ slot) {
  __shared__ int pre[BATCH_MAX_JOBS + 1];
  __shared__ int s_item;
  const TickHeader3& H = *reinterpret_cast<const TickHeader3*>(slot);
  const int n = H.n_prox;
  if (n <= 0) return;
  unsigned* counter = reinterpret_cast<TickHeader3*>(slot)->cnt + 3;
  const BatchOut3* jobs = reinterpret_cast<const BatchOut3*>(slot + H.off_out);
  const int* src = reinterpret_cast<const int*>(slot + H.off_pout);
  for (int i = threadIdx.y * blockDim.x + threadIdx.x; i <= n; i += blockDim.x * blockDim.y) pre[i] = src[i];
  __syncthreads();
  const int total = pre[n];
  for (int item = f3_next(counter, &s_item); item < total; item = f3_next(counter, &s_item)) {
    const int j = fgp_batch_job(pre, n, item);
    const BatchOut3& J = jobs[j];
    const int local = item - pre[j];
    const int per = J.tiles_x * J.tiles_y;
    const int gz = local / per, tl = local - gz * per;
    fgp3d_out_item(J.v, J.w, J.wdst, J.D, J.tau, J.nonneg, J.t, tl % J.tiles_x, tl / J.tiles_x, gz);
  }
}

}  // namespace

int fgp3d_iter_batched(char* slot, int it, int grid, cudaStream_t s) {
  LaunchScope _ls("fgp3d_iter_batched", s);
  VRPS_CUDA(launch_kernel(fgp3d_iter_batched_kernel, dim3(grid), dim3(F3_TX, F3_TY), (size_t)0, s, slot, it));
  return VRPS_OK;
}

int fgp3d_out_batched(char* slot, int grid, cudaStream_t s) {
  LaunchScope _ls("fgp3d_out_batched", s);
  VRPS_CUDA(launch_kernel(fgp3d_out_batched_kernel, dim3(grid), dim3(32, 8), (size_t)0, s, slot));
  return VRPS_OK;
}

int batched_grid_3d_proj(int which, int* grid);

int fgp3d_batch_entry(vrps_geom* g, const float* v, float tau, int iters, int nonneg, float* dual,
                      const ProxTail& t, BatchFgp3* f, int* f_items, BatchOut3* o, int* o_items) {
  if (iters > BATCH3_MAX_ITERS) return fail(VRPS_ERR_INVALID_ARG, "batched 3D prox takes at most %d iterations",
                                            BATCH3_MAX_ITERS);
  if (iters > 0) VRPS_TRY(fgp_prepare(g));
  Workspace& ws = g->ws;
  const Fgp3Schedule sch = fgp3_schedule(iters);
  std::memset(f, 0, sizeof(*f));
  f->v = v;
  f->buf[0] = dual;
  f->buf[1] = ws.dual_s1;
  f->buf[2] = ws.dual_s2;
  f->D = Dims3{g->nx, g->ny, g->nz, (size_t)g->n};
  f->tau = tau;
  f->step = (float)(1.0 / (4.0 * g->dims * (double)tau));
  f->nonneg = nonneg;
  f->zc = fgp3_zc(g);
  f->iters = iters;
  f->tiles_x = (g->nx + F3_TX - 1) / F3_TX;
  f->tiles_y = (g->ny + F3_TY - 1) / F3_TY;
  f->chunks = (g->nz + f->zc - 1) / f->zc;
  for (int k = 0; k < iters; ++k) {
    f->cur[k] = (unsigned char)sch.cur[k];
    f->prev[k] = (unsigned char)sch.prev[k];
    f->nxt[k] = (unsigned char)sch.nxt[k];
    f->mom[k] = sch.mom[k];
  }
  *f_items = f->tiles_x * f->tiles_y * f->chunks;
  const float* w_final = f->buf[sch.final_buf];
  std::memset(o, 0, sizeof(*o));
  o->v = v;
  o->w = w_final;
  o->wdst = (w_final != dual) ? dual : nullptr;
  o->D = f->D;
  o->tau = tau;
  o->nonneg = nonneg;
  o->t = t;
  o->tiles_x = (g->nx + 31) / 32;
  o->tiles_y = (g->ny + 7) / 8;
  *o_items = o->tiles_x * o->tiles_y * g->nz;
  return VRPS_OK;
}

int batched_grid_3d(int which, int* grid) {
  if (which <= 2) return batched_grid_3d_proj(which, grid);
  int dev = 0, sms = 0, per = 0;
  VRPS_CUDA(cudaGetDevice(&dev));
  VRPS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (which == 3)
    VRPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fgp3d_iter_batched_kernel, F3_TX * F3_TY, 0));
  else
    VRPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fgp3d_out_batched_kernel, 256, 0));
  *grid = (per < 1 ? 1 : per) * sms;
  return VRPS_OK;
}

}  // namespace vrps

extern "C" int vrps_selftest_bounded_wait(unsigned polls, vrps_stream_t stream) {
  using namespace vrps;
  if (polls < 1 || polls > (1u << 24)) return fail(VRPS_ERR_INVALID_ARG, "polls must be in [1, 2^24]");
  const cudaStream_t s = (cudaStream_t)stream;
  char* buf = nullptr;   // [counter (8 bytes)][error word (4 bytes)]
  cudaError_t e = cudaMalloc((void**)&buf, 16);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(self-test)");
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(buf);
  unsigned* err = reinterpret_cast<unsigned*>(buf + 8);
  unsigned word = 0;
  unsigned long long arrived = 0;
  int rc = VRPS_OK;
  if ((e = cudaMemsetAsync(buf, 0, 16, s)) != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync(self-test)");
  if (rc == VRPS_OK) {
    e = launch_kernel(bounded_wait_probe, dim3(1), dim3(32), (size_t)0, s, bar, err, polls);
    if (e != cudaSuccess) rc = launch_fail(e, "bounded_wait_probe", (const void*)bounded_wait_probe, dim3(1), dim3(32), 0);
  }
  if (rc == VRPS_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) rc = cuda_fail(e, "self-test wait");
  if (rc == VRPS_OK && (e = cudaMemcpy(&word, err, sizeof(word), cudaMemcpyDeviceToHost)) != cudaSuccess)
    rc = cuda_fail(e, "self-test read");
  if (rc == VRPS_OK && (e = cudaMemcpy(&arrived, bar, sizeof(arrived), cudaMemcpyDeviceToHost)) != cudaSuccess)
    rc = cuda_fail(e, "self-test read");
  // the context survived the expired wait: a second probe launches, runs and expires the same way
  if (rc == VRPS_OK && (e = cudaMemsetAsync(buf, 0, 16, s)) != cudaSuccess) rc = cuda_fail(e, "cudaMemsetAsync(self-test)");
  unsigned word2 = 1;
  if (rc == VRPS_OK) {
    e = launch_kernel(bounded_wait_probe, dim3(1), dim3(32), (size_t)0, s, bar, err, polls);
    if (e != cudaSuccess) rc = launch_fail(e, "bounded_wait_probe", (const void*)bounded_wait_probe, dim3(1), dim3(32), 0);
  }
  if (rc == VRPS_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) rc = cuda_fail(e, "self-test wait");
  if (rc == VRPS_OK && (e = cudaMemcpy(&word2, err, sizeof(word2), cudaMemcpyDeviceToHost)) != cudaSuccess)
    rc = cuda_fail(e, "self-test read");
  cudaFree(buf);
  if (rc != VRPS_OK) return rc;
  if (!(word & 4u) || arrived != 1ull)
    return fail(VRPS_ERR_INTERNAL, "bounded wait: error word %u, %llu arrivals (expected bit 4 and 1)", word,
                arrived);
  if (!(word2 & 4u)) return fail(VRPS_ERR_INTERNAL, "bounded wait: the second probe did not expire either");
  return VRPS_OK;
}
