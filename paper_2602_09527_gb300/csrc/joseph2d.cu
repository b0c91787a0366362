// 2D parallel-beam Joseph projector: ray-driven forward (gather) with fused residual /
// estimator epilogues, and pixel-driven exact transpose with the fused ProxSkip update.
//
// Forward (Section 1.2, A_i x): a CTA item is (angle, group of bands of dominant-axis lines);
// the band is copied into shared memory by bulk copies (rows of x, or of x^T for angles
// marched along columns, so that adjacent rays read along a row) and every ray of the angle
// is walked through it with exact fixed-point positions; per-group partial ray sums are added
// in a fixed order by the CTA that completes the angle, which runs the estimator epilogue.
//
// Adjoint (A_i^T r): a CTA owns a 16 x 16 or 16 x 32 pixel tile.  For every angle of the
// launch the tile's footprint on the detector (at most fp bins) is staged in shared memory,
// then each pixel sums w_j r_j over the <= nc bins whose ray passes within one interpolation
// cell of its centre, with the Joseph weight of that (ray, pixel) pair.  No atomics.
#include <cstdint>
#include <cstring>

#include "vrps_internal.h"

namespace vrps {
namespace {

constexpr int FWD_LANES = 32;
constexpr int FWD_THREADS = 256;
constexpr int FWD_BAND_BYTES = 64 * 1024;   // shared-memory band of image lines per CTA
constexpr int ADJ_TX = ADJ2D_TILE_X;        // pixel tile: 16 columns (x 16 or 32 rows)
constexpr int ADJ_THREADS = 256;
constexpr int ADJ_CHUNK = 64;
constexpr unsigned WAIT_LIMIT = 1u << 22;   // bounded mbarrier polls before giving up


__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long global_addr(const void* p) {
  unsigned long long g;
  asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(p));
  return g;
}


__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Forward projector, one CTA per (angle row, band of `band` dominant-axis lines).  The band
// -- `band` consecutive rows of x (rows-marched angles) or of x^T (columns-marched angles) --
// is copied row by row into shared memory by TMA bulk copies, with FWD_PAD zero columns on
// both sides of every row so that the taps of any sample whose point lies in (-1, ncols) are
// read without bounds tests.  The CTA's eight warps walk all n_bins rays of the angle through
// the band, 32 bins per warp pass.  Positions: every trip of four lines re-anchors exactly
// from the 64-bit fixed-point walk (u = I + F); the four samples of the trip add A2 k to F
// in float (|F + A2 k| < 5, error ~1e-7 pixel).  Each ray's band sum goes to a partial
// buffer; the CTA that completes a row last adds the bands in band order (deterministic) and
// runs the epilogue.
constexpr int FWD_PAD = 4;   // zero floats left and right of each staged line (16 bytes)

// Estimator epilogue of one ray with value r = (A_i x)_ray (FwdMode).
// Tables keep the stored (rounded) values and the residual handed to the adjoint is formed
// from them, so that the running sums built from the table (SVRG's gbar, SAGA's v-bar) stay
// equal to the sums of the stored rows (no drift from rounding).  Explicitly rounded
// operations: the result does not depend on how the compiler contracts the caller's code.
template <int MODE>
__device__ __forceinline__ void fwd2d_epilogue(const FwdOut& o, size_t idx, float r) {
  if (MODE == FWD_PLAIN) {
    o.y[idx] = r;
  } else if (MODE == FWD_RESID) {
    o.y[idx] = __fsub_rn(r, ld_store(o, o.b, idx));
  } else if (MODE == FWD_SVRG) {
    o.y[idx] = __fsub_rn(r, ld_store(o, o.tab, idx));
  } else if (MODE == FWD_SAGA) {
    const float res = __fsub_rn(r, ld_store(o, o.b, idx));
    const float old = ld_store(o, o.tab, idx);
    o.y[idx] = __fsub_rn(st_store(o, o.tab, idx, res), old);
  } else {  // FWD_SNAP
    o.y[idx] = __fsub_rn(st_store(o, o.tab, idx, r), ld_store(o, o.b, idx));
  }
}

struct FwdShared {
  unsigned long long bar[2];   // mbarriers of the two band buffers (initialised once per CTA)
  unsigned last;               // this CTA completed the angle row
};

constexpr int FWD_RPT = 6;   // most rays per thread held in registers across a band group (nb <= 1536)

// Stages band lines [l0, l0 + nl) of img into buf (zero margins; BULK: bulk copies on bar, the
// caller waits; otherwise plain loads, visible after the caller's barrier).
template <bool BULK>
__device__ __forceinline__ void fwd2d_stage(const float* img, int ncols, int stride, int l0, int nl, float* buf,
                                            unsigned long long* bar) {
  const int tid = threadIdx.x;
  const float* src = img + (size_t)l0 * ncols;
  for (int e = tid; e < nl * 2 * FWD_PAD; e += FWD_THREADS) {
    const int L = e / (2 * FWD_PAD), q = e - L * 2 * FWD_PAD;
    buf[L * stride + (q < FWD_PAD ? q : ncols + q)] = 0.f;
  }
  if (BULK) {
    if (tid == 0) {
      // order earlier generic accesses of the buffer before the async-proxy writes
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const unsigned row_bytes = (unsigned)(ncols * sizeof(float));
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                   "r"(row_bytes * (unsigned)nl)
                   : "memory");
      for (int L = 0; L < nl; ++L)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_addr(buf + L * stride + FWD_PAD)),
            "l"(global_addr(src + (size_t)L * ncols)), "r"(row_bytes), "r"(smem_addr(bar))
            : "memory");
    }
  } else {
    for (int e = tid; e < nl * ncols; e += FWD_THREADS) {
      const int L = e / ncols;
      buf[L * stride + FWD_PAD + (e - L * ncols)] = __ldg(src + e);
    }
  }
}

// Bounded wait for phase `ph` of bar; false (and the error word set) when it gave up.
__device__ __forceinline__ bool fwd2d_wait(unsigned long long* bar, unsigned ph, unsigned* err) {
  unsigned it = 0;
  while (!mbar_try_wait(bar, ph) && ++it < WAIT_LIMIT) {
  }
  if (it < WAIT_LIMIT) return true;
  // record the failure and give the copies in flight a second bounded chance to land in shared
  // memory before the buffer is reused; nothing is computed from it
  if (threadIdx.x == 0) atomicOr(err, 1u);
  unsigned it2 = 0;
  while (!mbar_try_wait(bar, ph) && ++it2 < WAIT_LIMIT) {
  }
  return false;
}

// Fractional part in [0, 1) of a 28-bit fixed-point value, from its top 23 fraction bits.
__device__ __forceinline__ float fix28_frac(int v) {
  return __int_as_float(0x3f800000u | (((unsigned)v << 4) >> 9)) - 1.0f;
}

// Ray j's samples on lines [l0, l0 + nl) of the staged band buf (acc0: even lines of each
// trip of four, acc1: odd ones).  Positions: every trip of four lines re-anchors exactly from
// the 64-bit fixed-point walk (u = I + F); within the trip the fraction is a 32-bit fixed-point
// value (28 fraction bits) stepped by the per-line increment, whose integer part offsets the
// tap and whose top fraction bits give the weight.  Integer and bit operations only: the
// float floor and float-to-int conversions this replaces run at a quarter of the FP32 rate and
// bounded the walk (5.4 instead of 7.3 us of band walking per 512^2 subset forward).
__device__ __forceinline__ void fwd2d_ray(const Fwd2DParams& P, const AngleInfo2D& in, const float* buf, int j,
                                          int l0, int nl, int ncols, int nlines, int stride, float& acc0,
                                          float& acc1) {
  const float uc = 0.5f * (float)(ncols - 1);
  const float lc = 0.5f * (float)(nlines - 1);
  const float u0 = fmaf(in.A1, (float)j - P.jc, uc);   // line-range clipping only
  int lo = l0, hi = l0 + nl - 1;
  if (in.A2 != 0.f) {
    float la = fmaf(-1.f - u0, in.inv_A2, lc);
    float lb = fmaf((float)ncols - u0, in.inv_A2, lc);
    if (la > lb) {
      const float q = la;
      la = lb;
      lb = q;
    }
    la = fminf(fmaxf(la, -2.f), (float)nlines + 1.f);
    lb = fminf(fmaxf(lb, -2.f), (float)nlines + 1.f);
    lo = max(lo, (int)floorf(la) - 1);
    hi = min(hi, (int)ceilf(lb) + 1);
  } else if (!(u0 > -1.f && u0 < (float)ncols)) {
    hi = -1;
  }
  if (lo > hi) return;
  // exact fixed-point walk along the ray: U = u * 2^32; FWD_PAD shifts into the padded row
  long long U = (long long)(ncols - 1 + 2 * FWD_PAD) * 2147483648LL + in.A1H * (long long)(2 * j - (P.nb - 1)) +
                in.A2H * (long long)(2 * lo - (nlines - 1));
  const long long dU4 = 8 * in.A2H;   // four lines
  const int st = (int)((2 * in.A2H) >> 4);   // one line, 28 fraction bits (|A2| <= 1: |st| <= 2^28)
  int rb = (lo - l0) * stride;          // shared-memory offset of the current line
  int l = lo;
  for (; l + 3 <= hi; l += 4) {
    const int I = fix_floor(U) + rb;
    const int p0 = (int)(((unsigned)(unsigned long long)U) >> 4);   // fraction, 28 bits
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int pq = p0 + q * st;   // in (-3, 4) x 2^28: fits 32 bits
      const float* t = buf + (I + q * stride + (pq >> 28));
      const float f = fix28_frac(pq);
      const float a = t[0], b = t[1];
      if (q & 1) acc1 += fmaf(f, b - a, a);
      else acc0 += fmaf(f, b - a, a);
    }
    U += dU4;
    rb += 4 * stride;
  }
  const int I = fix_floor(U) + rb;
  const int p0 = (int)(((unsigned)(unsigned long long)U) >> 4);
  for (int q = 0; l <= hi; ++l, ++q) {
    const int pq = p0 + q * st;
    const float* t = buf + (I + q * stride + (pq >> 28));
    acc0 += fmaf(fix28_frac(pq), t[1] - t[0], t[0]);
  }
}

// Forward projector, one CTA item per (angle row, group of P.group consecutive bands of
// P.band dominant-axis lines).  A band -- lines of x (rows-marched angles) or of x^T
// (columns-marched angles) -- is copied row by row into shared memory by bulk copies, with
// FWD_PAD zero columns on both sides of every row so that the taps of any sample whose point
// lies in (-1, ncols) are read without bounds tests; with groups of several bands the next
// band is copied into the second buffer while the current one is walked, and each thread
// keeps its rays' sums in registers across the group.  Each ray's group sum goes to a partial
// buffer; the CTA that completes a row last adds the groups in order (deterministic) and runs
// the epilogue.  ph[2]: the phases of the CTA's two barriers (flipped on every use).
template <int MODE, bool BULK, int RPT>
__device__ __forceinline__ void fwd2d_item(const Fwd2DParams& P, int cg, int row, float* smem, FwdShared& S,
                                           unsigned* ph) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const AngleInfo2D in = P.ids ? P.ang[P.ids[row]] : P.ang[row];
  const bool tr = in.T != 0;
  const float* __restrict__ img = tr ? P.xT : P.x;
  const int ncols = tr ? P.ny : P.nx;
  const int nlines = tr ? P.nx : P.ny;
  const int stride = ncols + 2 * FWD_PAD;
  const int c0 = cg * P.group;
  const int c1 = min(c0 + P.group, P.nbands);
  const size_t pbase = (size_t)row * P.bands * P.nb + (size_t)cg * P.nb;
  bool ok = true;
  if (RPT == 0 || P.group == 1 || P.nb > RPT * FWD_THREADS) {
    // one band per item: rays written as they finish
    const int l0 = c0 * P.band;
    const int nl = min(P.band, nlines - l0);
    if (nl > 0) {
      fwd2d_stage<BULK>(img, ncols, stride, l0, nl, smem, &S.bar[0]);
      if (BULK) {
        ok = fwd2d_wait(&S.bar[0], ph[0], P.err);
        ph[0] ^= 1u;
      }
      __syncthreads();
    }
    for (int j0 = warp * FWD_LANES; j0 < P.nb; j0 += FWD_THREADS) {
      const int j = j0 + lane;
      float acc0 = 0.f, acc1 = 0.f;
      if (j < P.nb && nl > 0 && ok) fwd2d_ray(P, in, smem, j, l0, nl, ncols, nlines, stride, acc0, acc1);
      if (j < P.nb) P.part[pbase + j] = acc0 + acc1;
    }
  } else {
    const int band_floats = P.band * stride;
    constexpr int NR = RPT > 0 ? RPT : 1;   // rays per thread (RPT = 0: not grouped)
    float acc[NR][2];
#pragma unroll
    for (int k = 0; k < NR; ++k) acc[k][0] = acc[k][1] = 0.f;
    {
      const int nl0 = min(P.band, nlines - c0 * P.band);
      if (nl0 > 0) fwd2d_stage<BULK>(img, ncols, stride, c0 * P.band, nl0, smem, &S.bar[0]);
    }
    for (int c = c0; c < c1; ++c) {
      const int b = (c - c0) & 1;
      const int l0 = c * P.band;
      const int nl = min(P.band, nlines - l0);
      if (nl <= 0) break;   // bands grow along the lines: the rest lie beyond this orientation's image
      const int nl1 = c + 1 < c1 ? min(P.band, nlines - l0 - P.band) : 0;
      if (nl1 > 0) fwd2d_stage<BULK>(img, ncols, stride, l0 + P.band, nl1, smem + (b ^ 1) * band_floats, &S.bar[b ^ 1]);
      if (BULK) {
        ok = fwd2d_wait(&S.bar[b], ph[b], P.err) && ok;
        ph[b] ^= 1u;
      }
      __syncthreads();   // margins, plain loads and bulk data of band c visible
      if (ok) {
        const float* buf = smem + b * band_floats;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          const int j = warp * FWD_LANES + k * FWD_THREADS + lane;
          if (warp * FWD_LANES + k * FWD_THREADS < P.nb && j < P.nb)
            fwd2d_ray(P, in, buf, j, l0, nl, ncols, nlines, stride, acc[k][0], acc[k][1]);
        }
      }
      __syncthreads();   // band c's buffer is free for band c + 2
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const int j = warp * FWD_LANES + k * FWD_THREADS + lane;
      if (j < P.nb) P.part[pbase + j] = acc[k][0] + acc[k][1];
    }
  }
  // the last CTA of this row adds the groups in order and applies the epilogue
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned prev = atomicAdd(P.count + row, 1u);
    S.last = prev == (unsigned)(P.bands - 1) ? 1u : 0u;
    if (S.last) P.count[row] = 0u;
  }
  __syncthreads();
  if (!S.last) return;
  __threadfence();
  const int bands = P.bands, nb = P.nb;
  const float* __restrict__ part = P.part + (size_t)row * bands * nb;
  const size_t obase = (size_t)row * nb;
  if ((nb & 3) == 0) {
    // four rays per thread with 16-byte loads; each ray still adds its groups in order
    const int nb4 = nb >> 2;
    const float4* __restrict__ p4 = reinterpret_cast<const float4*>(part);
    for (int j4 = tid; j4 < nb4; j4 += FWD_THREADS) {
      float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
      for (int q = 0; q < bands; ++q) {
        const float4 v = __ldcg(p4 + (size_t)q * nb4 + j4);
        sum.x += v.x;
        sum.y += v.y;
        sum.z += v.z;
        sum.w += v.w;
      }
      fwd2d_epilogue<MODE>(P.o, obase + 4 * j4 + 0, __fmul_rn(sum.x, in.wgt));
      fwd2d_epilogue<MODE>(P.o, obase + 4 * j4 + 1, __fmul_rn(sum.y, in.wgt));
      fwd2d_epilogue<MODE>(P.o, obase + 4 * j4 + 2, __fmul_rn(sum.z, in.wgt));
      fwd2d_epilogue<MODE>(P.o, obase + 4 * j4 + 3, __fmul_rn(sum.w, in.wgt));
    }
  } else {
    for (int j = tid; j < nb; j += FWD_THREADS) {
      float sum = 0.f;
      for (int q = 0; q < bands; ++q) sum += __ldcg(part + (size_t)q * nb + j);
      fwd2d_epilogue<MODE>(P.o, obase + j, __fmul_rn(sum, in.wgt));
    }
  }
}

__device__ __forceinline__ void fwd2d_init_barrier(FwdShared& S) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.bar[1])) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
}

template <int MODE, bool BULK, int RPT>
__global__ void __launch_bounds__(FWD_THREADS) fwd2d_kernel(Fwd2DParams P) {
  extern __shared__ __align__(128) float band[];
  __shared__ FwdShared S;
  if (BULK) fwd2d_init_barrier(S);
  unsigned ph[2] = {0u, 0u};
  fwd2d_item<MODE, BULK, RPT>(P, blockIdx.x, blockIdx.y, band, S, ph);
}


// Pixel-driven transpose.  Per angle of a chunk, one thread derives the tile's constants: the
// tile origin's fractional bin t0 = J0 + F0 is exact (fixed point), and the footprint
// r[jlo .. jlo+fp) is gathered into shared memory (asynchronous 4-byte copies, bins outside
// [0, nb) zero-filled).  A pixel at tile offset (tx, ty) has t - J0 = F0 + Bx tx + By ty (a
// small float) and receives wgt max(0, 1 - |j - t|/hw) r_j from the bins within hw of t; the
// length factor wgt is folded into the per-angle weight constants.  NC = 2 covers hw <= 1
// (bins not finer than pixels): only bins floor(t) and floor(t) + 1 can be within hw, with
// weights wgt max(0, 1 - phi/hw) and wgt max(0, 1 - (1 - phi)/hw), phi = t - floor(t).  NC = 0
// is the general loop over P.nc candidates from floor(t - hw) + 1 on.
struct AdjShared {
  unsigned last;           // this CTA completed the tile (angle shares)
  float4 par[ADJ_CHUNK];   // Bx, By, F0 (NC = 2) or F0 - hw (NC = 0), wgt/hw
  float2 par2[ADJ_CHUNK];  // NC = 2: wgt, wgt (1 - 1/hw); NC = 0: wgt, hw
  int off[ADJ_CHUNK];      // J0 - jlo
  int jlo[ADJ_CHUNK];
  float tile[32][ADJ_TX + 1];
};

// Asynchronous 4-byte global -> shared copy; ok = false zero-fills the destination instead.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(global_addr(src)),
               "r"(ok ? 4 : 0)
               : "memory");
}

// One pixel tile (bx, by) of the transpose; sm: dynamic shared [chunk][fp].
template <int NC, int PPT>
__device__ __forceinline__ void adj2d_item(const Adj2DParams& P, int bx, int by, float* sm, AdjShared& S,
                                           int part = 0) {
  constexpr int TY = (ADJ_THREADS / ADJ_TX) * PPT;   // tile rows: 16 (one pixel per thread) or 32
  // angle range of this item: part `part` of P.split equal shares of the launch's rows
  const int ra = (int)(((long long)P.rows * part) / P.split);
  const int rz = (int)(((long long)P.rows * (part + 1)) / P.split);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * ADJ_TX + tx;
  const int lane = tid & 31, warp = tid >> 5;
  const int ix0 = bx * ADJ_TX, iy0 = by * TY;
  const float ftx = (float)tx, fty = (float)ty;
  const float half_rows = (float)(TY / 2);
  float acc0 = 0.f, acc1 = 0.f;                  // pixels (tx, ty) and, with PPT = 2, (tx, ty + TY/2)
  for (int r0 = ra; r0 < rz; r0 += P.chunk) {
    const int nr = min(P.chunk, rz - r0);
    if (tid < nr) {
      const AngleInfo2D in = P.ids ? P.ang[P.ids[r0 + tid]] : P.ang[r0 + tid];
      const long long T0 = (long long)(P.nb - 1) * 2147483648LL + in.BxH * (long long)(2 * ix0 - (P.nx - 1)) +
                           in.ByH * (long long)(2 * iy0 - (P.ny - 1));
      const int J0 = fix_floor(T0);
      const float F0 = fix_frac(T0);
      const float tmin = F0 + fminf(0.f, in.Bx * (float)(ADJ_TX - 1)) + fminf(0.f, in.By * (float)(TY - 1));
      const int jlo = J0 + (int)floorf(tmin - in.hw) - 1;
      const float wiw = in.wgt * in.inv_hw;
      if (NC == 2) {
        S.par[tid] = make_float4(in.Bx, in.By, F0, wiw);
        S.par2[tid] = make_float2(in.wgt, in.wgt - wiw);
      } else {
        S.par[tid] = make_float4(in.Bx, in.By, F0 - in.hw, wiw);
        S.par2[tid] = make_float2(in.wgt, in.hw);
      }
      S.off[tid] = J0 - jlo;
      S.jlo[tid] = jlo;
    }
    __syncthreads();
    // footprint gather: warp w copies the rows of angles w, w + 8, ...; every copy is issued
    // before any is waited for
    for (int q = warp; q < nr; q += ADJ_THREADS / 32) {
      const int jl = S.jlo[q];
      const float* __restrict__ rq = P.r + (size_t)(r0 + q) * P.nb;
      float* dq = sm + q * P.fp;
      for (int k = lane; k < P.fp; k += 32) {
        const int j = jl + k;
        const bool ok = j >= 0 && j < P.nb;
        cp_async4(dq + k, rq + (ok ? j : 0), ok);
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    for (int q = 0; q < nr; ++q) {
      const float4 pr = S.par[q];
      const float2 p2 = S.par2[q];
      const float* row = sm + q * P.fp + S.off[q];   // row[k] = bin J0 + k
      const float ua = fmaf(pr.y, fty, fmaf(pr.x, ftx, pr.z));
      const float ub = fmaf(pr.y, half_rows, ua);
      if (NC == 2) {
        {
          const float fl = floorf(ua);
          const float ph = ua - fl;
          const float w0 = fmaxf(0.f, fmaf(-ph, pr.w, p2.x));
          const float w1 = fmaxf(0.f, fmaf(ph, pr.w, p2.y));
          const float* rr = row + (int)fl;
          acc0 = fmaf(w0, rr[0], acc0);
          acc0 = fmaf(w1, rr[1], acc0);
        }
        if (PPT == 2) {
          const float fl = floorf(ub);
          const float ph = ub - fl;
          const float w0 = fmaxf(0.f, fmaf(-ph, pr.w, p2.x));
          const float w1 = fmaxf(0.f, fmaf(ph, pr.w, p2.y));
          const float* rr = row + (int)fl;
          acc1 = fmaf(w0, rr[0], acc1);
          acc1 = fmaf(w1, rr[1], acc1);
        }
      } else {
        const float hw = p2.y;
        const float fa = floorf(ua), fb = floorf(ub);
        const float* ra_ = row + 1 + (int)fa;
        const float* rb_ = row + 1 + (int)fb;
        const float da = fa + 1.f - (ua + hw), db = fb + 1.f - (ub + hw);   // first candidate - t
        for (int c = 0; c < P.nc; ++c) {
          acc0 = fmaf(fmaxf(0.f, fmaf(-fabsf(da + (float)c), pr.w, p2.x)), ra_[c], acc0);
          if (PPT == 2) acc1 = fmaf(fmaxf(0.f, fmaf(-fabsf(db + (float)c), pr.w, p2.x)), rb_[c], acc1);
        }
      }
    }
    __syncthreads();
  }
  const int ix = ix0 + tx, iy = iy0 + ty, iy1 = iy + TY / 2;
  const bool in0 = ix < P.nx && iy < P.ny, in1 = PPT == 2 && ix < P.nx && iy1 < P.ny;
  const size_t p0 = (size_t)iy * P.nx + ix, p1 = (size_t)iy1 * P.nx + ix;
  if (P.split > 1) {
    // angle shares of one tile: partial sums to scratch; the last share to arrive adds them in
    // share order (deterministic) and runs the epilogue
    const size_t n = (size_t)P.nx * P.ny;
    if (in0) P.part[(size_t)part * n + p0] = acc0;
    if (in1) P.part[(size_t)part * n + p1] = acc1;
    __threadfence();
    __syncthreads();
    const int tile = by * P.tiles_x + bx;
    if (tid == 0) {
      const unsigned prev = atomicAdd(P.count + tile, 1u);
      S.last = prev == (unsigned)(P.split - 1) ? 1u : 0u;
      if (S.last) P.count[tile] = 0u;
    }
    __syncthreads();
    if (!S.last) return;
    __threadfence();
    acc0 = 0.f;
    acc1 = 0.f;
    for (int q = 0; q < P.split; ++q) {
      if (in0) acc0 += __ldcg(P.part + (size_t)q * n + p0);
      if (in1) acc1 += __ldcg(P.part + (size_t)q * n + p1);
    }
  }
  const UpdateArgs& u = P.u;
  if (!u.enabled) {
    if (in0) u.out[p0] = acc0;
    if (in1) u.out[p1] = acc1;
    return;
  }
  const float x0 = in0 ? update_pixel(u, p0, acc0) : 0.f;
  const float x1 = in1 ? update_pixel(u, p1, acc1) : 0.f;
  if (!u.theta && u.xT) {
    S.tile[ty][tx] = x0;
    if (PPT == 2) S.tile[ty + TY / 2][tx] = x1;
    __syncthreads();
    for (int e = tid; e < ADJ_TX * TY; e += ADJ_THREADS) {
      const int c = e / TY, r = e - c * TY;
      const int ox = ix0 + c, oy = iy0 + r;
      if (ox < P.nx && oy < P.ny) u.xT[(size_t)ox * P.ny + oy] = S.tile[r][c];
    }
  }
}

template <int NC, int PPT>
__global__ void __launch_bounds__(ADJ_THREADS) adj2d_kernel(Adj2DParams P) {
  extern __shared__ float sm[];
  __shared__ AdjShared S;
  // blockIdx.y = tile row * split + angle share
  adj2d_item<NC, PPT>(P, blockIdx.x, blockIdx.y / P.split, sm, S, blockIdx.y % P.split);
}

__global__ void transpose_kernel(const float* __restrict__ in, float* __restrict__ out, int ny, int nx) {
  __shared__ float t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  in += (size_t)blockIdx.z * nx * ny;   // one [ny][nx] slice per blockIdx.z
  out += (size_t)blockIdx.z * nx * ny;
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

int transpose2d(const float* in, float* out, int ny, int nx, cudaStream_t s, int slices) {
  dim3 grid((nx + 31) / 32, (ny + 31) / 32, slices), block(32, 8);
  { LaunchScope _ls("transpose_kernel", s, 8.0 * nx * ny * slices);
  VRPS_CUDA(launch_kernel(transpose_kernel, dim3(grid), dim3(block), (size_t)(0), s, in, out, ny, nx));
  }
  VRPS_LAUNCHED("transpose2d");
  return VRPS_OK;
}

int fwd2d_setup(const vrps_geom* g, const float* x, const float* xT, const int* ids, int rows, FwdOut o,
                Fwd2DParams* out, size_t* smem, bool* bulk) {
  Fwd2DParams& P = *out;
  P.x = x;
  P.xT = xT;
  // row-indexed angle constants when ids is a subset of one of the geometry's orders
  const AngleInfo2D* rows_tab = angle_rows(g, ids);
  P.ang = rows_tab ? rows_tab : g->ang2d;
  P.ids = rows_tab ? nullptr : ids;
  P.nx = g->nx;
  P.ny = g->ny;
  P.nb = g->n_bins;
  P.jc = 0.5f * (float)(g->n_bins - 1);
  P.o = o;
  const int maxw = g->nx > g->ny ? g->nx : g->ny;   // widest line (row of x or of x^T)
  const int maxl = maxw;
  // all-angle passes take their own tuned shape when there is one
  const bool full = rows >= g->n_angles && g->tune_full_fwd_bytes > 0;
  const int band_bytes = full ? g->tune_full_fwd_bytes : (g->tune_fwd_bytes > 0 ? g->tune_fwd_bytes : FWD_BAND_BYTES);
  const int want_group = full ? g->tune_full_fwd_group : g->tune_fwd_group;
  int band = band_bytes / (int)(sizeof(float) * (maxw + 2 * FWD_PAD));
  if (band < 1) band = 1;
  if (band > maxl) band = maxl;
  P.band = band;
  P.nbands = (maxl + band - 1) / band;
  // the bulk copy needs 16-byte aligned rows: line lengths that are multiples of 4 floats
  *bulk = (g->nx % 4 == 0) && (g->ny % 4 == 0) && (((uintptr_t)x | (uintptr_t)xT) % 16 == 0);
  // band groups: bulk copies only (the plain-load path walks one band per item)
  P.group = *bulk && want_group > 1 && g->n_bins <= FWD_RPT * FWD_THREADS ? want_group : 1;
  if (P.group > P.nbands) P.group = P.nbands;
  P.bands = (P.nbands + P.group - 1) / P.group;
  vrps_geom* gm = const_cast<vrps_geom*>(g);
  Workspace& ws = gm->ws;
  const size_t part_need = (size_t)g->n_angles * P.bands * g->n_bins;
  if (ws.fwd_part_cap < part_need) {
    if (ws.fwd_part) cudaFree(ws.fwd_part);
    ws.fwd_part = nullptr;
    ws.fwd_part_cap = 0;
    VRPS_CUDA(cudaMalloc((void**)&ws.fwd_part, sizeof(float) * part_need));
    ws.fwd_part_cap = part_need;
  }
  if (!ws.fwd_count) {
    VRPS_CUDA(cudaMalloc((void**)&ws.fwd_count, sizeof(unsigned) * (size_t)g->n_angles));
    VRPS_CUDA(cudaMemset(ws.fwd_count, 0, sizeof(unsigned) * (size_t)g->n_angles));
  }
  if (!ws.dev_error) {
    VRPS_CUDA(cudaMalloc((void**)&ws.dev_error, sizeof(unsigned)));
    VRPS_CUDA(cudaMemset(ws.dev_error, 0, sizeof(unsigned)));
  }
  P.part = ws.fwd_part;
  P.count = ws.fwd_count;
  P.err = ws.dev_error;
  *smem = sizeof(float) * (size_t)band * (maxw + 2 * FWD_PAD) * (P.group > 1 ? 2 : 1);
  return VRPS_OK;
}

int fwd2d(const vrps_geom* g, const float* x, const float* xT, const int* ids, int rows, int mode,
          FwdOut o, cudaStream_t s) {
  if (rows <= 0) return VRPS_OK;
  Fwd2DParams P;
  size_t smem = 0;
  bool bulk = false;
  VRPS_TRY(fwd2d_setup(g, x, xT, ids, rows, o, &P, &smem, &bulk));
  dim3 grid(P.bands, rows), block(FWD_THREADS);
  auto launch = [&](auto kern) -> int {
    VRPS_TRY(smem_opt_in((const void*)kern, smem));
    LaunchScope _ls("fwd2d_kernel", s, 4.0 * g->n + fwd_mode_bytes(mode, (size_t)rows * g->n_bins, o.store));
    VRPS_LAUNCH("fwd2d_kernel", kern, dim3(grid), dim3(block), (size_t)(smem), s, P);
    return VRPS_OK;
  };
  const bool grouped = bulk && P.group > 1;
  switch (mode) {
#define VRPS_FWD_CASE(M)                                                                          \
  case M:                                                                                         \
    VRPS_TRY(grouped ? (g->n_bins <= 3 * FWD_THREADS ? launch(fwd2d_kernel<M, true, 3>)            \
                                                      : launch(fwd2d_kernel<M, true, FWD_RPT>))    \
                     : (bulk ? launch(fwd2d_kernel<M, true, 0>) : launch(fwd2d_kernel<M, false, 0>))); \
    break;
    VRPS_FWD_CASE(FWD_PLAIN)
    VRPS_FWD_CASE(FWD_RESID)
    VRPS_FWD_CASE(FWD_SVRG)
    VRPS_FWD_CASE(FWD_SAGA)
    VRPS_FWD_CASE(FWD_SNAP)
#undef VRPS_FWD_CASE
    default: return fail(VRPS_ERR_INVALID_ARG, "bad forward mode %d", mode);
  }
  VRPS_LAUNCHED("fwd2d");
  return VRPS_OK;
}

int adj2d_setup(const vrps_geom* g, const float* r, const int* ids, int rows, const UpdateArgs& u,
                Adj2DParams* out, size_t* smem, int* variant, int* tiles_x, int* tiles_y) {
  Adj2DParams& P = *out;
  P.r = r;
  const AngleInfo2D* rows_tab = angle_rows(g, ids);
  P.ang = rows_tab ? rows_tab : g->ang2d;
  P.ids = rows_tab ? nullptr : ids;
  P.rows = rows;
  P.nx = g->nx;
  P.ny = g->ny;
  P.nb = g->n_bins;
  P.fp = g->adj_fp;
  P.nc = g->adj_nc;
  int chunk = (int)(96 * 1024 / (sizeof(float) * (size_t)g->adj_fp));
  P.chunk = chunk < ADJ_CHUNK ? (chunk < 1 ? 1 : chunk) : ADJ_CHUNK;
  P.u = u;
  *smem = sizeof(float) * (size_t)P.chunk * P.fp;
  // two pixels per thread (shared per-angle parameters) unless the image is very small
  const bool two = g->tune_adj_two >= 0 ? g->tune_adj_two != 0 : (long long)g->nx * g->ny > 512LL * g->sms;
  const int ty = (ADJ_THREADS / ADJ_TX) * (two ? 2 : 1);
  *variant = (g->adj_nc == 2 ? 2 : 0) + (two ? 1 : 0);
  *tiles_x = (g->nx + ADJ_TX - 1) / ADJ_TX;
  *tiles_y = (g->ny + ty - 1) / ty;
  P.tiles_x = *tiles_x;
  // angle shares per tile (at least 4 angles each)
  int split = (rows >= g->n_angles && g->tune_full_adj_split > 0) ? g->tune_full_adj_split
                                                                  : (g->tune_adj_split > 1 ? g->tune_adj_split : 1);
  while (split > 1 && rows / split < 4) --split;
  P.split = split;
  P.part = nullptr;
  P.count = nullptr;
  if (split > 1) {
    vrps_geom* gm = const_cast<vrps_geom*>(g);
    Workspace& ws = gm->ws;
    const size_t need = (size_t)split * (size_t)g->n;
    if (ws.adj_part_cap < need) {
      if (ws.adj_part) cudaFree(ws.adj_part);
      ws.adj_part = nullptr;
      ws.adj_part_cap = 0;
      VRPS_CUDA(cudaMalloc((void**)&ws.adj_part, sizeof(float) * need));
      ws.adj_part_cap = need;
    }
    const size_t tiles = (size_t)(*tiles_x) * (*tiles_y);
    if (ws.adj_count_cap < tiles) {
      if (ws.adj_count) cudaFree(ws.adj_count);
      ws.adj_count = nullptr;
      ws.adj_count_cap = 0;
      VRPS_CUDA(cudaMalloc((void**)&ws.adj_count, sizeof(unsigned) * tiles));
      VRPS_CUDA(cudaMemset(ws.adj_count, 0, sizeof(unsigned) * tiles));
      ws.adj_count_cap = tiles;
    }
    P.part = ws.adj_part;
    P.count = ws.adj_count;
  }
  return VRPS_OK;
}

int adj2d(const vrps_geom* g, const float* r, const int* ids, int rows, const UpdateArgs& u,
          cudaStream_t s) {
  Adj2DParams P;
  size_t smem = 0;
  int variant = 0, tx = 0, ty = 0;
  VRPS_TRY(adj2d_setup(g, r, ids, rows, u, &P, &smem, &variant, &tx, &ty));
  dim3 grid(tx, ty * P.split), block(ADJ_TX, ADJ_THREADS / ADJ_TX);
  auto launch = [&](auto kern) -> int {
    VRPS_TRY(smem_opt_in((const void*)kern, smem));
    LaunchScope _ls("adj2d_kernel", s, 4.0 * rows * g->n_bins + update_bytes(u, (size_t)g->n));
    VRPS_LAUNCH("adj2d_kernel", kern, dim3(grid), dim3(block), (size_t)(smem), s, P);
    return VRPS_OK;
  };
  switch (variant) {
    case 3: VRPS_TRY(launch(adj2d_kernel<2, 2>)); break;
    case 2: VRPS_TRY(launch(adj2d_kernel<2, 1>)); break;
    case 1: VRPS_TRY(launch(adj2d_kernel<0, 2>)); break;
    default: VRPS_TRY(launch(adj2d_kernel<0, 1>)); break;
  }
  VRPS_LAUNCHED("adj2d");
  return VRPS_OK;
}

// ------------------------------------------------------------------ batched launches
namespace {

// Job j of item `item` from the prefix array cached in shared memory (pre[j] <= item < pre[j+1]).
__device__ __forceinline__ int batch_job(const int* pre, int n, int item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void batch_load_prefix(int* dst, const int* src, int n) {
  for (int i = threadIdx.y * blockDim.x + threadIdx.x; i <= n; i += blockDim.x * blockDim.y) dst[i] = src[i];
  __syncthreads();
}

template <bool BULK, int RPT>
__device__ __forceinline__ void fwd2d_item_mode(const BatchFwd& J, int c, int row, float* band, FwdShared& S,
                                                unsigned* ph) {
  switch (J.mode) {
    case FWD_PLAIN: fwd2d_item<FWD_PLAIN, BULK, RPT>(J.P, c, row, band, S, ph); break;
    case FWD_RESID: fwd2d_item<FWD_RESID, BULK, RPT>(J.P, c, row, band, S, ph); break;
    case FWD_SVRG: fwd2d_item<FWD_SVRG, BULK, RPT>(J.P, c, row, band, S, ph); break;
    case FWD_SAGA: fwd2d_item<FWD_SAGA, BULK, RPT>(J.P, c, row, band, S, ph); break;
    default: fwd2d_item<FWD_SNAP, BULK, RPT>(J.P, c, row, band, S, ph); break;
  }
}

// Next item of the launch for the whole CTA: one atomic on the tick's counter (items are
// handed out in order, so the CTAs in flight work on neighbouring tiles of one job).
__device__ __forceinline__ int batch_next(unsigned* counter, int* s_item) {
  __syncthreads();   // everyone has read the previous item
  if (threadIdx.x == 0 && threadIdx.y == 0) *s_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  return *s_item;
}

template <int RPT>
__global__ void __launch_bounds__(FWD_THREADS) fwd2d_batched_kernel(char* __restrict__ slot) {
  extern __shared__ __align__(128) float band[];
  __shared__ FwdShared S;
  __shared__ int pre[BATCH_MAX_JOBS + 1];
  __shared__ int s_item;
  const TickHeader& H = *reinterpret_cast<const TickHeader*>(slot);
  const int n = H.n_fwd;
  if (n <= 0) return;
  unsigned* counter = reinterpret_cast<TickHeader*>(slot)->cnt + 0;
  const BatchFwd* jobs = reinterpret_cast<const BatchFwd*>(slot + H.off_fwd);
  batch_load_prefix(pre, reinterpret_cast<const int*>(slot + H.off_pfwd), n);
  fwd2d_init_barrier(S);
  unsigned ph[2] = {0u, 0u};
  const int total = pre[n];
  for (int item = batch_next(counter, &s_item); item < total; item = batch_next(counter, &s_item)) {
    const int j = batch_job(pre, n, item);
    const BatchFwd& J = jobs[j];
    const int local = item - pre[j];
    const int bands = J.P.bands;
    const int c = local % bands, row = local / bands;
    if (J.bulk) fwd2d_item_mode<true, RPT>(J, c, row, band, S, ph);
    else fwd2d_item_mode<false, 0>(J, c, row, band, S, ph);
  }
}

__global__ void __launch_bounds__(ADJ_THREADS) adj2d_batched_kernel(char* __restrict__ slot) {
  extern __shared__ float sm[];
  __shared__ AdjShared S;
  __shared__ int pre[BATCH_MAX_JOBS + 1];
  __shared__ int s_item;
  const TickHeader& H = *reinterpret_cast<const TickHeader*>(slot);
  const int n = H.n_adj;
  if (n <= 0) return;
  unsigned* counter = reinterpret_cast<TickHeader*>(slot)->cnt + 1;
  const BatchAdj* jobs = reinterpret_cast<const BatchAdj*>(slot + H.off_adj);
  batch_load_prefix(pre, reinterpret_cast<const int*>(slot + H.off_padj), n);
  const int total = pre[n];
  for (int item = batch_next(counter, &s_item); item < total; item = batch_next(counter, &s_item)) {
    const int j = batch_job(pre, n, item);
    const BatchAdj& J = jobs[j];
    const int local = item - pre[j];
    const int sp = J.P.split;
    const int tile = local / sp, part = local - tile * sp;
    const int bx = tile % J.tiles_x, by = tile / J.tiles_x;
    switch (J.variant) {
      case 3: adj2d_item<2, 2>(J.P, bx, by, sm, S, part); break;
      case 2: adj2d_item<2, 1>(J.P, bx, by, sm, S, part); break;
      case 1: adj2d_item<0, 2>(J.P, bx, by, sm, S, part); break;
      default: adj2d_item<0, 1>(J.P, bx, by, sm, S, part); break;
    }
  }
}

}  // namespace

int fwd2d_batched(char* slot, int grid, size_t smem, bool grouped, cudaStream_t s) {
  auto kern = grouped ? fwd2d_batched_kernel<FWD_RPT> : fwd2d_batched_kernel<0>;
  VRPS_TRY(smem_opt_in((const void*)kern, smem));
  LaunchScope _ls("fwd2d_batched", s);
  VRPS_LAUNCH("fwd2d_batched", kern, dim3(grid), dim3(FWD_THREADS), smem, s, slot);
  return VRPS_OK;
}

int adj2d_batched(char* slot, int grid, size_t smem, cudaStream_t s) {
  VRPS_TRY(smem_opt_in((const void*)adj2d_batched_kernel, smem));
  LaunchScope _ls("adj2d_batched", s);
  VRPS_LAUNCH("adj2d_batched", adj2d_batched_kernel, dim3(grid), dim3(ADJ_TX, ADJ_THREADS / ADJ_TX), smem, s, slot);
  return VRPS_OK;
}

int batched_grid_2d(int which, size_t smem, int* grid) {
  int dev = 0, sms = 0, per = 0;
  VRPS_CUDA(cudaGetDevice(&dev));
  VRPS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (which == 0 || which == 4) {
    auto kern = which == 4 ? fwd2d_batched_kernel<FWD_RPT> : fwd2d_batched_kernel<0>;
    VRPS_TRY(smem_opt_in((const void*)kern, smem));
    VRPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, FWD_THREADS, smem));
  } else {
    VRPS_TRY(smem_opt_in((const void*)adj2d_batched_kernel, smem));
    VRPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, adj2d_batched_kernel, ADJ_THREADS, smem));
  }
  *grid = (per < 1 ? 1 : per) * sms;
  return VRPS_OK;
}

}  // namespace vrps
