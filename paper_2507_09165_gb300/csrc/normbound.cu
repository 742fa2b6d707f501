// Norm bound of Sec. 3.4 (Theorem 2, Algorithm 2 steps 1-2) and the scaled
// cast X_0 = X / lam~ (Algorithm 2 step 3).
//
// Lanczos on A = X^2 (Parlett, The Symmetric Eigenvalue Problem, Ch. 13):
// 20 steps, A q = X (X q), Lanczos vectors and all recurrences in FP64 with
// full re-orthogonalisation (classical Gram-Schmidt, two passes), then the
// largest Ritz pair (sigma, q) of the tridiagonal T_m and
//     lam~ = sqrt(sigma + ||X (X q) - sigma q||_2),
// raised to max(lam~, ||X||_F / sqrt(n), max_i |X_ii|) (both lower bounds of
// ||X||_2; they only matter when the start vector misses the top eigenvector).
//
// The mat-vec reads only the upper triangle of the FP32 input, once per
// product (an HBM-bound pass of n^2/2 words), in 128 x 128 tiles: each tile
// adds its rows' dot products (X(i,j) v_j, i <= j) and its columns' dot
// products (X(i,j) v_i, i < j) into per-tile partial sums, reduced afterwards
// in a fixed order (deterministic).  GB300's FP64 pipe is narrow, so the
// element level runs in FP32: each thread forms 8-term FP32 FMA sums, which
// are combined exactly into double-float (FP32 pair) partial sums with the
// TwoSum error-free transformation (Knuth; Ogita, Rump & Oishi, "Accurate sum
// and dot product", SIAM J. Sci. Comput. 2005), converted to FP64 per vector
// element.  A mat-vec is thus accurate to a few FP32 roundings of the 8-term
// runs (~1e-7 relative); every operation on vectors -- the recurrences, dot
// products, re-orthogonalisation and norms -- is FP64 in a fixed order.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "internal.h"
#include "ptx.cuh"
#include "tridiag.cuh"

namespace psd {

namespace {

constexpr uint64_t kSeed = 0x243F6A8885A308D3ull;  // Lanczos start vector seed

// Host-side fault injection (psd_debug_set): a factor applied to lam~ (1.0:
// none; a factor below 1 drives the chain past the composite's basin and
// exercises the overshoot report) and the limit of the grid barriers' waits
// (0: every barrier that is not already complete gives up at once and the
// bound returns PSD_ERR_TIMEOUT).  Read by the kernels at run time, so
// captured graphs see the current values.
__device__ double g_debug_bound_scale = 1.0;
__device__ unsigned long long g_debug_barrier_limit_ns = kWaitLimitNs;
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

// ------------------------------------------------------- double-float helpers
struct F2 {
  float h, l;
};
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return F2{s, __fadd_rn(__fadd_rn(a.l, b.l), e)};
}
__device__ __forceinline__ double f2_to_d(F2 a) { return static_cast<double>(a.h) + static_cast<double>(a.l); }
__device__ __forceinline__ void split_d(double v, float& h, float& l) {
  h = __double2float_rn(v);
  l = __double2float_rn(v - static_cast<double>(h));
}
__device__ __forceinline__ F2 shfl_xor_f2(F2 a, int m) {
  return F2{__shfl_xor_sync(0xffffffffu, a.h, m), __shfl_xor_sync(0xffffffffu, a.l, m)};
}

// --------------------------------------------------------------- SplitMix64
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * kGolden;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// The FP32 estimate (FP64 runs at a small fraction of the FP32 rate on this GPU,
// and every thread of a tile's CTA evaluates this) is corrected exactly by the
// integer loops.
__device__ __forceinline__ void tile_of(int t, int& bi, int& bj) {
  int j = static_cast<int>((sqrtf(8.f * static_cast<float>(t) + 1.f) - 1.f) * 0.5f);
  while ((j + 1) * (j + 2) / 2 <= t) ++j;
  while (j * (j + 1) / 2 > t) --j;
  bj = j;
  bi = t - j * (j + 1) / 2;
}

// ------------------------------------------------------------------ phases
//
// Every phase of the norm bound is a device function over virtual blocks of
// kNT = 256 threads.  It runs either as the body of its own kernel (one CTA
// per virtual block: the multi-launch path, 151 launches per bound) or inside
// one persistent cooperative kernel whose CTAs take virtual blocks
// blockIdx.x, blockIdx.x + gridDim.x, ... between grid-wide barriers.  Both
// execute the same arithmetic in the same order and give the same bits.
// Vectors an earlier phase wrote are read with ld.global.cg (through L2): in
// the persistent kernel they change while it runs, which the non-coherent
// read-only path must not be used for.
constexpr int kNT = 256;
static_assert(kVecThreads == kNT, "vector phases: one element per thread of a 256-thread block");

// Shared memory of one CTA, reused by the phases (each virtual block ends
// with a barrier before the next one writes it again).
struct NBShared {
  union {
    struct {
      float2 red[2][8][kSymvTile];  // two buffers: consecutive tiles of a run alternate
      double fro[8];
    } mv;
    float2 part[8][32];
    struct {
      double h[32];
      double w[8][32];
    } orth;
    struct {
      double y[kMaxSteps];
      float a[kMaxSteps], b[kMaxSteps];
    } tri;
  } u;
  double bs[8];  // block_sum64 (apart from u: a phase may still read u.orth.h when a warp enters it)
  double scalar[2];
};

// Everything the phases read: sizes, the argument block, state and buffers.
struct NBCtx {
  int n, nb, ntiles, nv, npart;
  int64_t npad;
  const DevArgs* args;
  DevState* st;
  double *Qv, *u, *w, *q, *zsave;
  float *vh, *vl;
  float2 *P1, *P2;
  float2 *dots, *dots2;  // per chunk: 32 double-float partials (dot products, slot 31 ||w||^2)
  double* norms;         // per 256-element block: FP64 partial of ||q_0||^2
  float2* norms2;        // per chunk: double-float partial of a squared norm (same storage as norms)
  double* tile_fro;
};

// Block-wide FP64 sum of one value per thread (kNT threads), fixed order;
// every thread receives the sum.
__device__ __forceinline__ double block_sum64(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < kNT / 32; ++k) s += sh[k];
  __syncthreads();
  return s;
}

// Fixed-order warp sum of cnt FP64 values (lane-strided, then a butterfly).
// Each lane's values are loaded 8 at a time before they are added (in order):
// the sums are L2-latency chains otherwise.
__device__ __forceinline__ double warp_sum_array(const double* a, int cnt, int stride) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int c0 = 0; c0 < cnt; c0 += 8 * 32) {
    double t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int c = c0 + 32 * i + lane;
      t[i] = c < cnt ? __ldcg(a + static_cast<int64_t>(c) * stride) : 0.0;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (c0 + 32 * i + lane < cnt) s += t[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Recursive-halving sum of cnt (<= 32) FP64 values over a warp; on return
// lane l holds the warp total of value l.  Values live in v[0..31].
__device__ __forceinline__ double warp_multi_sum(double (&v)[32], int lane) {
#pragma unroll
  for (int half = 16, m = 16; half >= 1; half >>= 1, m >>= 1) {
    const bool upper = (lane & m) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const double send = upper ? v[i] : v[i + half];
      const double keep = upper ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
  }
  return v[0];
}

// One tile of y = X v over the upper triangle (see file comment), in three
// pieces so that the persistent kernel can load the next tile while it
// reduces the current one.  Thread (tr, tc) = (lane & 15, 2 warp + lane / 16)
// owns rows i0 + 8 tr .. +7 and columns j0 + 8 tc .. +7: each column's 128
// rows are read by a half-warp as 512 contiguous bytes.  DIAG tiles mask to
// i <= j (rows) and i < j (columns).  STATS adds the tile's share of
// ||X||_F^2 and max |X_ii|.
struct TileGeom {
  int bi, bj, ib, jb;
  bool diag;
};
__device__ __forceinline__ TileGeom tile_geom(int t) {
  TileGeom g;
  tile_of(t, g.bi, g.bj);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  g.ib = g.bi * kSymvTile + 8 * (lane & 15);
  g.jb = g.bj * kSymvTile + 8 * (2 * warp + (lane >> 4));
  g.diag = g.bi == g.bj;
  return g;
}

// The thread's slices of v (rows and columns) and its 64 elements: 16
// independent 16-byte loads of X in flight.
__device__ __forceinline__ void tile_load(const float* __restrict__ X, int64_t ld, int n, const TileGeom& g,
                                          const float* vh, float (&vi)[8], float (&vj)[8], float (&x)[8][8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    vi[k] = (g.ib + k < n) ? __ldcg(vh + g.ib + k) : 0.f;
    vj[k] = (g.jb + k < n) ? __ldcg(vh + g.jb + k) : 0.f;
  }
  const bool full = (g.ib + 7 < n) && (g.jb + 7 < n);
  const bool vec = full && ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float* col = X + static_cast<int64_t>(g.jb + c) * ld + g.ib;
    if (vec) {
      const float4 a4 = __ldg(reinterpret_cast<const float4*>(col));
      const float4 b4 = __ldg(reinterpret_cast<const float4*>(col + 4));
      x[c][0] = a4.x; x[c][1] = a4.y; x[c][2] = a4.z; x[c][3] = a4.w;
      x[c][4] = b4.x; x[c][5] = b4.y; x[c][6] = b4.z; x[c][7] = b4.w;
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[c][k] = (g.jb + c < n && g.ib + k < n) ? __ldg(col + k) : 0.f;
    }
  }
}

// Per-thread row and column dot products of the 8 x 8 block (8-term FP32 FMA runs).
template <bool STATS, bool DIAG>
__device__ __forceinline__ void tile_fma(int n, const TileGeom& g, const float (&vi)[8], const float (&vj)[8],
                                         const float (&x)[8][8], float (&rsum)[8], float (&csum)[8], float& fro,
                                         unsigned& mdiag) {
  fro = 0.f;
  mdiag = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) rsum[k] = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    csum[c] = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float xr = x[c][k], xc = x[c][k];
      if (DIAG) {
        const int i = g.ib + k, j = g.jb + c;
        xr = (i <= j) ? xr : 0.f;
        xc = (i < j) ? xc : 0.f;
        if (STATS && i == j && i < n) mdiag = max(mdiag, __float_as_uint(fabsf(x[c][k])));
      }
      rsum[k] = fmaf(xr, vj[c], rsum[k]);
      csum[c] = fmaf(xc, vi[k], csum[c]);
      if (STATS) fro = fmaf(xr, xc + xr, fro);  // x^2 on the diagonal, 2 x^2 above it
    }
  }
}

// Combines the threads' sums in a fixed order (double-float) into the tile's
// row partials P1[bj][rows] and column partials P2[bi][columns], through row
// buffer `buf`.  Ends with a CTA barrier unless `sync_after` is false: a run
// of tiles alternates the two buffers instead, since a tile two ahead writes a
// buffer only after every thread has passed the barrier of the tile between
// (and so finished reading it); the run is followed by a CTA barrier.
template <bool STATS>
__device__ __forceinline__ void tile_reduce_store(int n, const TileGeom& g, const float (&rsum)[8],
                                                  const float (&csum)[8], float fro, unsigned mdiag, float2* P1,
                                                  float2* P2, int64_t ps, double* tile_fro, DevState* st,
                                                  NBShared& sh, int tile, int buf = 0,
                                                  bool sync_after = true) {
  float2 (*red)[kSymvTile] = sh.u.mv.red[buf];
  const int i0 = g.bi * kSymvTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tr = lane & 15;
  // rows: the two column groups of a warp (exact TwoSum), then the 8 warps
  F2 rs[8], cs[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float o = __shfl_xor_sync(0xffffffffu, rsum[k], 16);
    float h, e;
    if (lane < 16) two_sum(rsum[k], o, h, e); else two_sum(o, rsum[k], h, e);
    rs[k] = F2{h, e};
    cs[k] = F2{csum[k], 0.f};
  }
  if (lane < 16) {
#pragma unroll
    for (int k = 0; k < 8; ++k) red[warp][8 * tr + k] = make_float2(rs[k].h, rs[k].l);
  }
  // columns: recursive halving over the 16 row groups of a half-warp
#pragma unroll
  for (int half = 4, m = 8; half >= 1; half >>= 1, m >>= 1) {
    const bool upper = (tr & m) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const F2 send = upper ? cs[i] : cs[i + half];
      const F2 keep = upper ? cs[i + half] : cs[i];
      cs[i] = f2_add(keep, shfl_xor_f2(send, m));
    }
  }
  {
    const F2 o = shfl_xor_f2(cs[0], 1);
    cs[0] = (tr & 1) ? f2_add(o, cs[0]) : f2_add(cs[0], o);
    const int j = g.jb + (tr >> 1);
    if ((tr & 1) == 0 && j < n) P2[static_cast<int64_t>(g.bi) * ps + j] = make_float2(cs[0].h, cs[0].l);
  }
  __syncthreads();
  if (threadIdx.x < kSymvTile) {
    const int r = threadIdx.x;
    F2 a{red[0][r].x, red[0][r].y};
#pragma unroll
    for (int w = 1; w < 8; ++w) a = f2_add(a, F2{red[w][r].x, red[w][r].y});
    if (i0 + r < n) P1[static_cast<int64_t>(g.bj) * ps + i0 + r] = make_float2(a.h, a.l);
  }
  if (STATS) {
    double f = static_cast<double>(fro);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0) sh.u.mv.fro[warp] = f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mdiag = max(mdiag, __shfl_xor_sync(0xffffffffu, mdiag, o));
    if (lane == 0 && mdiag) atomicMax(&st->maxdiag_bits, mdiag);
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < 8; ++w) sum += sh.u.mv.fro[w];
      tile_fro[tile] = sum;
    }
  }
  if (sync_after) __syncthreads();
}

// Tile t of a product over X (t in [0, ntiles)), one tile per call.
template <bool STATS>
__device__ __forceinline__ void ph_symv(const NBCtx& c, const float* X, int64_t ld, int t, NBShared& sh) {
  const TileGeom g = tile_geom(t);
  float vi[8], vj[8], x[8][8], rsum[8], csum[8], fro;
  unsigned mdiag;
  tile_load(X, ld, c.n, g, c.vh, vi, vj, x);
  if (g.diag)
    tile_fma<STATS, true>(c.n, g, vi, vj, x, rsum, csum, fro, mdiag);
  else
    tile_fma<STATS, false>(c.n, g, vi, vj, x, rsum, csum, fro, mdiag);
  tile_reduce_store<STATS>(c.n, g, rsum, csum, fro, mdiag, c.P1, c.P2, c.npad, c.tile_fro, c.st, sh, t);
}

// Tiles r = first, first + stride, ... < ntiles of a product (in the
// opposite order of the tile list if `rev`), each loaded while the previous
// one is reduced: the same arithmetic per tile as ph_symv.  The caller ends
// the run with a CTA barrier (the grid barrier after the phase).
template <bool STATS>
__device__ __forceinline__ void ph_symv_run(const NBCtx& c, const float* X, int64_t ld, int first, int stride,
                                            bool rev, NBShared& sh) {
  if (first >= c.ntiles) return;
  auto tile_at = [&](int r) { return rev ? c.ntiles - 1 - r : r; };
  float vi[8], vj[8], x[8][8];
  int r = first;
  int buf = 0;
  TileGeom g = tile_geom(tile_at(r));
  tile_load(X, ld, c.n, g, c.vh, vi, vj, x);
  while (true) {
    float rsum[8], csum[8], fro;
    unsigned mdiag;
    if (g.diag)
      tile_fma<STATS, true>(c.n, g, vi, vj, x, rsum, csum, fro, mdiag);
    else
      tile_fma<STATS, false>(c.n, g, vi, vj, x, rsum, csum, fro, mdiag);
    const int rn = r + stride;
    const TileGeom gn = tile_geom(tile_at(rn < c.ntiles ? rn : r));
    if (rn < c.ntiles) tile_load(X, ld, c.n, gn, c.vh, vi, vj, x);  // in flight during the reduction
    tile_reduce_store<STATS>(c.n, g, rsum, csum, fro, mdiag, c.P1, c.P2, c.npad, c.tile_fro, c.st, sh,
                             tile_at(r), buf, false);
    if (rn >= c.ntiles) break;
    r = rn;
    g = gn;
    buf ^= 1;
  }
}

// State reset and the start vector q_0 (unit SplitMix64 vector, before scaling).
__device__ __forceinline__ void ph_init(const NBCtx& c, int vb, NBShared& sh) {
  const int e = vb * kNT + threadIdx.x;
  double v = 0.0;
  if (e < c.n) {
    const uint64_t z = splitmix64(kSeed, static_cast<uint64_t>(e));
    const double u = static_cast<double>(z >> 11) * 0x1.0p-53;
    v = 2.0 * u - 1.0;
  }
  const double s = block_sum64(v * v, sh.bs);
  if (threadIdx.x == 0) c.norms[vb] = s;
  if (e < c.n) c.Qv[e] = v;  // unnormalised; ph_norm0 scales it
  if (vb == 0 && threadIdx.x == 0) {
    DevState* st = c.st;
    st->m = 0;
    st->done = 0;
    st->status = 0;
    st->maxdiag_bits = 0;
    st->absmax_bits = 0;
    st->sigma = st->resid = st->lambda = st->fro = st->maxdiag = st->inv_lambda = 0.0;
  }
}

// Broadcast of a value computed by warp 0 (slot k of the CTA's scalars).
__device__ __forceinline__ double bcast(double v, NBShared& sh, int k) {
  if (threadIdx.x == 0) sh.scalar[k] = v;
  __syncthreads();
  const double r = sh.scalar[k];
  __syncthreads();
  return r;
}

// q_0 /= ||v||, split.
__device__ __forceinline__ void ph_norm0(const NBCtx& c, int vb, NBShared& sh) {
  double s = 0.0;
  if (threadIdx.x < 32) s = warp_sum_array(c.norms, c.nv, 1);
  if (threadIdx.x == 0) s = 1.0 / sqrt(s);  // FP64 scalar work in one thread
  const double inv = bcast(s, sh, 0);
  const int e = vb * kNT + threadIdx.x;
  if (e < c.n) {
    const double q = __ldcg(c.Qv + e) * inv;
    c.Qv[e] = q;
    split_d(q, c.vh[e], c.vl[e]);
  }
}

// ||X||_F from the per-tile sums of the first product (one warp, fixed order).
__device__ __forceinline__ void ph_fro(const NBCtx& c) {
  const double f = warp_sum_array(c.tile_fro, c.ntiles, 1);
  if (threadIdx.x == 0) c.st->fro = sqrt(f);
}

// The chunk-reducing phases take two chunks per CTA at once, one per half
// of the CTA (warps 0-3 and 4-7): a chunk pair index cp covers chunks 2 cp and
// 2 cp + 1.  With one chunk per CTA, orders just above 32 x the CTA count
// (n = 10,000: 313 chunks, 304 CTAs) left a few CTAs a second chunk and the
// whole phase waiting for them.
__device__ __forceinline__ int chunk_of_half(int cp) { return 2 * cp + static_cast<int>(threadIdx.x >> 7); }
__device__ __forceinline__ bool half_lead_warp() { return (threadIdx.x & 127) < 32; }

// y_e = sum_{bj >= b(e)} P1[bj][e] + sum_{bi <= b(e)} P2[bi][e] for the 32
// elements e of chunk `ch`, by the 4 warps of this thread's half of the CTA:
// warp h (0-3 in the half) adds the blocks congruent to h mod 4 in
// double-float, then the half's first warp combines the 4 warp sums in a fixed
// order.  Returns y_e (FP64) in that warp; other warps return 0.  Both halves
// call it together (CTA barriers).
__device__ __forceinline__ double reduce_partials(const NBCtx& c, int ch, NBShared& sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, hw = w & 3;
  const int e = ch * 32 + lane;
  F2 a{0.f, 0.f}, d{0.f, 0.f};
  if (e < c.n) {
    const int b = e / kSymvTile;
#pragma unroll 4
    for (int bj = b + hw; bj < c.nb; bj += 4) {
      const float2 t = __ldcg(c.P1 + static_cast<int64_t>(bj) * c.npad + e);
      a = f2_add(a, F2{t.x, t.y});
    }
#pragma unroll 4
    for (int bi = hw; bi <= b; bi += 4) {
      const float2 t = __ldcg(c.P2 + static_cast<int64_t>(bi) * c.npad + e);
      d = f2_add(d, F2{t.x, t.y});
    }
  }
  const F2 t = f2_add(a, d);
  sh.u.part[w][lane] = make_float2(t.h, t.l);
  __syncthreads();
  double y = 0.0;
  if (hw == 0) {
    F2 acc{sh.u.part[w][lane].x, sh.u.part[w][lane].y};
#pragma unroll
    for (int q = 1; q < 4; ++q) acc = f2_add(acc, F2{sh.u.part[w + q][lane].x, sh.u.part[w + q][lane].y});
    y = f2_to_d(acc);
  }
  __syncthreads();
  return y;
}

// u = X v (first product of X (X v)); split u for the second product.  Chunk pair cp.
__device__ __forceinline__ void ph_reduce_split(const NBCtx& c, int cp, double* u, NBShared& sh) {
  const int ch = chunk_of_half(cp);
  const double y = reduce_partials(c, ch, sh);
  const int e = ch * 32 + (threadIdx.x & 31);
  if (half_lead_warp() && e < c.n) {
    u[e] = y;
    split_d(y, c.vh[e], c.vl[e]);
  }
}

// ---- Lanczos step j after the second product: Gram-Schmidt and q_{j+1}.
// Element work is done per chunk of 32 elements by one warp (lane =
// element), FP64.  Sums over the chunks (the dot products q_k . w and ||w||^2)
// go through per-chunk partials stored as double-float pairs (FP32 hi + lo,
// about 48 bits): every CTA adds them up itself in FP32 arithmetic, in the same
// order, because this GPU issues FP64 at a small fraction of its FP32 rate.

__device__ __forceinline__ float2 d_to_f2(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - static_cast<double>(h)));
}

// S[k] = sum over the chunks of part[k * nch + ch] (slot-major: a warp's 32
// lanes read 256 contiguous bytes) for the slots k with (want >> k) & 1,
// double-float in a fixed order (lanes stride over the chunks, then a
// butterfly), into shared memory as FP64.  Warp w takes the slots k = w,
// w + 8, ...  The loads of a lane are issued 8 at a time.
__device__ __forceinline__ void chunk_sums(const float2* part, int nch, uint32_t want, double* S) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = w; k < 32; k += kNT / 32) {
    if (!((want >> k) & 1u)) continue;
    F2 acc{0.f, 0.f};
    for (int c0 = 0; c0 < nch; c0 += 8 * 32) {
      float2 t[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int ch = c0 + 32 * i + lane;
        t[i] = ch < nch ? __ldcg(part + static_cast<int64_t>(k) * nch + ch) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) acc = f2_add(acc, F2{t[i].x, t[i].y});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const F2 other = shfl_xor_f2(acc, o);
      acc = (lane & o) ? f2_add(other, acc) : f2_add(acc, other);
    }
    if (lane == 0) S[k] = f2_to_d(acc);
  }
}

// w = X u (the second product, reduced); partial dots q_k . w (k <= j) of the
// chunk into slot k of dots.  Chunk pair cp.
__device__ __forceinline__ void ph_reduce_dots(const NBCtx& c, int cp, int j, NBShared& sh) {
  const int ch = chunk_of_half(cp);
  const double y = reduce_partials(c, ch, sh);
  if (!half_lead_warp() || ch >= c.npart) return;
  const int lane = threadIdx.x & 31;
  const int e = ch * 32 + lane;
  if (e < c.n) c.w[e] = y;
  double v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k)
    v[k] = (k <= j && e < c.n) ? __ldcg(c.Qv + static_cast<int64_t>(k) * c.npad + e) * y : 0.0;
  c.dots[static_cast<int64_t>(lane) * c.npart + ch] = d_to_f2(warp_multi_sum(v, lane));
}

// First Gram-Schmidt pass (every CTA first sums the chunks' dots: h, and
// alpha_j = h_j), then per chunk: w -= sum_k h_k q_k, and the partials of the
// second pass, q_k . w (k <= j) and ||w||^2 (slot 31), into dots2.
// Chunks ch = cta + ncta * warp, ... (warp 0 only while there are no more
// chunks than CTAs: the FP64 work spreads over the SMs).
__device__ __forceinline__ void ph_orth1(const NBCtx& c, int cta, int ncta, int j, NBShared& sh) {
  chunk_sums(c.dots, c.npart, (2u << j) - 1u, sh.u.orth.h);
  __syncthreads();
  if (cta == 0 && threadIdx.x == 0) c.st->alpha[j] = sh.u.orth.h[j];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int ch = cta + ncta * wp; ch < c.npart; ch += ncta * (kNT / 32)) {
    const int e = ch * 32 + lane;
    double qk[kMaxSteps];
#pragma unroll
    for (int k = 0; k < kMaxSteps; ++k)
      qk[k] = (k <= j && e < c.n) ? __ldcg(c.Qv + static_cast<int64_t>(k) * c.npad + e) : 0.0;
    double we = 0.0;
    if (e < c.n) {
      we = __ldcg(c.w + e);
#pragma unroll
      for (int k = 0; k < kMaxSteps; ++k)
        if (k <= j) we -= sh.u.orth.h[k] * qk[k];
      c.w[e] = we;
    }
    double v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = (k < kMaxSteps && k <= j) ? qk[k < kMaxSteps ? k : 0] * we : 0.0;
    v[31] = we * we;
    c.dots2[static_cast<int64_t>(lane) * c.npart + ch] = d_to_f2(warp_multi_sum(v, lane));
  }
  __syncthreads();
}

// Second Gram-Schmidt pass and the next Lanczos vector.  Every CTA sums the
// second pass's dots h2 and ||w||^2; w' = w - Q h2 is orthogonal to Q and
// (Q orthonormal) ||w'||^2 = ||w||^2 - ||h2||^2, so beta_j = ||w'|| needs no
// further reduction (h2 is at the rounding level of w after the first pass:
// no cancellation).  Stops on breakdown (beta_j <= 1e-12 ||X||_F^2) or after
// the last step; otherwise q_{j+1} = w' / beta_j per chunk.  Returns `stop`
// (the same in every CTA) and beta_j.
__device__ __forceinline__ bool ph_orth2_next(const NBCtx& c, int cta, int ncta, int j, NBShared& sh,
                                              double& beta) {
  chunk_sums(c.dots2, c.npart, ((2u << j) - 1u) | 0x80000000u, sh.u.orth.h);
  __syncthreads();
  if (threadIdx.x == 0) {  // FP64 scalar work once per CTA
    double h2 = 0.0;
    for (int k = 0; k <= j; ++k) h2 += sh.u.orth.h[k] * sh.u.orth.h[k];
    const double b = sqrt(fmax(sh.u.orth.h[31] - h2, 0.0));
    sh.scalar[0] = b;
    sh.scalar[1] = 1.0 / b;
  }
  __syncthreads();
  beta = sh.scalar[0];
  const double fro = __ldcg(&c.st->fro);
  const bool stop = !(beta > kBreakdown * (fro * fro)) || j == kMaxSteps - 1;  // also true for NaN
  if (cta == 0 && threadIdx.x == 0) {
    c.st->beta[j] = beta;
    c.st->m = j + 1;
    if (stop) c.st->done = 1;
  }
  if (!stop) {
    const double inv = sh.scalar[1];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int ch = cta + ncta * wp; ch < c.npart; ch += ncta * (kNT / 32)) {
      const int e = ch * 32 + lane;
      if (e >= c.n) continue;
      double qk[kMaxSteps];
#pragma unroll
      for (int k = 0; k < kMaxSteps; ++k)
        qk[k] = k <= j ? __ldcg(c.Qv + static_cast<int64_t>(k) * c.npad + e) : 0.0;
      double we = __ldcg(c.w + e);
#pragma unroll
      for (int k = 0; k < kMaxSteps; ++k)
        if (k <= j) we -= sh.u.orth.h[k] * qk[k];
      const double q = we * inv;
      c.Qv[static_cast<int64_t>(j + 1) * c.npad + e] = q;
      split_d(q, c.vh[e], c.vl[e]);
    }
  }
  __syncthreads();
  return stop;
}

// Largest eigenpair of the Lanczos tridiagonal (tridiag.cuh): sigma and the
// Ritz vector's coordinates y in the Lanczos basis.  One warp.
__device__ __forceinline__ void ph_tridiag(const NBCtx& c, NBShared& sh) {
  DevState* st = c.st;
  // alpha, beta and m were written by thread 0 of this CTA (persistent kernel)
  // or by earlier kernels: plain loads
  const int m = *reinterpret_cast<volatile int*>(&st->m);
  const double sigma = tridiag_top_eig(st->alpha, st->beta, m, sh.u.tri.y, sh.u.tri.a, sh.u.tri.b);
  if (threadIdx.x == 0) {
    st->sigma = sigma;
    for (int k = 0; k < kMaxSteps; ++k) st->y[k] = sh.u.tri.y[k];
  }
}

// q = sum_k y_k q_k per chunk (one warp), partial ||q||^2 into norms[ch] (double-float).
__device__ __forceinline__ void ph_ritz(const NBCtx& c, int cta, int ncta, NBShared& sh) {
  (void)sh;
  const int m = __ldcg(&c.st->m);
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int ch = cta + ncta * wp; ch < c.npart; ch += ncta * (kNT / 32)) {
    const int e = ch * 32 + lane;
    double s = 0.0;
    if (e < c.n) {
      double qk[kMaxSteps], yk[kMaxSteps];
#pragma unroll
      for (int k = 0; k < kMaxSteps; ++k) {
        qk[k] = k < m ? __ldcg(c.Qv + static_cast<int64_t>(k) * c.npad + e) : 0.0;
        yk[k] = k < m ? __ldcg(&c.st->y[k]) : 0.0;
      }
#pragma unroll
      for (int k = 0; k < kMaxSteps; ++k)
        if (k < m) s += yk[k] * qk[k];
      c.q[e] = s;
    }
    F2 t = {__double2float_rn(s * s), 0.f};
    t.l = __double2float_rn(s * s - static_cast<double>(t.h));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const F2 other = shfl_xor_f2(t, o);
      t = (lane & o) ? f2_add(other, t) : f2_add(t, other);
    }
    if (lane == 0) c.norms2[ch] = make_float2(t.h, t.l);
  }
}

// 1 / sqrt of the sum of the chunks' double-float partials norms2[0 .. npart)
// (fixed order; 0 for a zero sum); every thread of the CTA receives it.
__device__ __forceinline__ double inv_norm_of_sum(const NBCtx& c, NBShared& sh) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    F2 acc{0.f, 0.f};
    for (int c0 = 0; c0 < c.npart; c0 += 8 * 32) {
      float2 t[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int ch = c0 + 32 * i + lane;
        t[i] = ch < c.npart ? __ldcg(c.norms2 + ch) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) acc = f2_add(acc, F2{t[i].x, t[i].y});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const F2 other = shfl_xor_f2(acc, o);
      acc = (lane & o) ? f2_add(other, acc) : f2_add(acc, other);
    }
    if (lane == 0) {
      const double s2 = f2_to_d(acc);
      sh.scalar[0] = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
    }
  }
  __syncthreads();
  const double r = sh.scalar[0];
  __syncthreads();
  return r;
}

// q /= ||q|| (inv = 1 / ||q||), split for the residual products.
__device__ __forceinline__ void ph_ritz_norm(const NBCtx& c, int vb, double inv) {
  const int e = vb * kNT + threadIdx.x;
  if (e < c.n) {
    const double v = __ldcg(c.q + e) * inv;
    c.q[e] = v;
    split_d(v, c.vh[e], c.vl[e]);
  }
}

// r = X (X q) - sigma q, partial ||r||^2 of the chunk into norms2[ch].
__device__ __forceinline__ void ph_resid(const NBCtx& c, int cp, NBShared& sh) {
  const int ch = chunk_of_half(cp);
  const double y = reduce_partials(c, ch, sh);
  if (!half_lead_warp() || ch >= c.npart) return;
  const int lane = threadIdx.x & 31;
  const int e = ch * 32 + lane;
  double r = 0.0;
  if (e < c.n) r = y - __ldcg(&c.st->sigma) * __ldcg(c.q + e);
  F2 t = {__double2float_rn(r * r), 0.f};
  t.l = __double2float_rn(r * r - static_cast<double>(t.h));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const F2 other = shfl_xor_f2(t, o);
    t = (lane & o) ? f2_add(other, t) : f2_add(t, other);
  }
  if (lane == 0) c.norms2[ch] = make_float2(t.h, t.l);
}

// lam~ = max(sqrt(sigma + r), ||X||_F / sqrt n, max |X_ii|); report.  One warp.
__device__ __forceinline__ void ph_final(const NBCtx& c) {
  const int lane = threadIdx.x;
  F2 acc{0.f, 0.f};
  for (int ch = lane; ch < c.npart; ch += 32) acc = f2_add(acc, F2{__ldcg(c.norms2 + ch).x, __ldcg(c.norms2 + ch).y});
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const F2 other = shfl_xor_f2(acc, o);
    acc = (lane & o) ? f2_add(other, acc) : f2_add(acc, other);
  }
  const double r2 = f2_to_d(acc);
  if (threadIdx.x != 0) return;
  DevState* st = c.st;
  const double r = sqrt(r2);
  const double fro = __ldcg(&st->fro);
  const double fro2 = fro * fro;
  const double md = static_cast<double>(__uint_as_float(__ldcg(&st->maxdiag_bits)));
  const double sigma = __ldcg(&st->sigma);
  double lam = sqrt(fmax(sigma + r, 0.0));
  lam = fmax(lam, fro / sqrt(static_cast<double>(c.n)));
  lam = fmax(lam, md);
  lam *= g_debug_bound_scale;  // 1.0 unless a test injects a bound that is too small
  st->resid = r;
  st->maxdiag = md;
  const bool finite = isfinite(fro2) && isfinite(lam) && isfinite(sigma);
  if (!finite) {
    atomicCAS(&st->status, 0, PSD_ERR_NONFINITE);
    lam = 0.0;
  }
  st->lambda = lam;
  st->inv_lambda = lam > 0.0 ? 1.0 / lam : 0.0;
  psd_info_t* info = c.args->info;
  if (info) {
    info->lambda_bound = lam;
    info->lanczos_sigma = sigma;
    info->lanczos_resid = r;
    info->fro_X = fro;
    info->max_diag = md;
    info->lanczos_steps = __ldcg(&st->m);
    info->status = __ldcg(&st->status);
    info->compl_resid = __longlong_as_double(0x7ff8000000000000ll);  // set by a projection's last step
  }
}

// ------------------------------------------------- multi-launch kernels
// One CTA per virtual block; `skip` kernels of Lanczos step j >= 1 return at
// once after a breakdown (the state's `done`).
__global__ void __launch_bounds__(kNT) nb_init_kernel(NBCtx c) {
  __shared__ NBShared sh;
  ph_init(c, blockIdx.x, sh);
}
__global__ void __launch_bounds__(kNT) nb_norm0_kernel(NBCtx c) {
  __shared__ NBShared sh;
  ph_norm0(c, blockIdx.x, sh);
}
// `reverse` deals the tiles to the CTAs in the opposite order: consecutive
// products over the same X alternate direction, so each starts on the tiles
// the previous one read last, which are still in L2.  The tile -> partial slot
// mapping does not depend on the order: results are identical.
template <bool STATS>
__global__ void __launch_bounds__(kNT, 2) nb_symv_kernel(NBCtx c, int skip, int reverse) {
  if (skip && c.st->done) return;
  __shared__ NBShared sh;
  const int t = reverse ? c.ntiles - 1 - static_cast<int>(blockIdx.x) : static_cast<int>(blockIdx.x);
  ph_symv<STATS>(c, c.args->X, c.args->ld, t, sh);
}
__global__ void nb_fro_kernel(NBCtx c) { ph_fro(c); }
__global__ void __launch_bounds__(kNT) nb_reduce_split_kernel(NBCtx c, double* u, int skip) {
  if (skip && c.st->done) return;
  __shared__ NBShared sh;
  ph_reduce_split(c, blockIdx.x, u, sh);
}
__global__ void __launch_bounds__(kNT) nb_reduce_dots_kernel(NBCtx c, int j) {
  if (c.st->done) return;
  __shared__ NBShared sh;
  ph_reduce_dots(c, blockIdx.x, j, sh);
}
__global__ void __launch_bounds__(kNT) nb_orth1_kernel(NBCtx c, int j) {
  if (c.st->done) return;
  __shared__ NBShared sh;
  ph_orth1(c, blockIdx.x, gridDim.x, j, sh);
}
__global__ void __launch_bounds__(kNT) nb_orth2_kernel(NBCtx c, int j) {
  if (c.st->done) return;
  __shared__ NBShared sh;
  double beta;
  ph_orth2_next(c, blockIdx.x, gridDim.x, j, sh, beta);
}
__global__ void nb_tridiag_kernel(NBCtx c) {
  __shared__ NBShared sh;
  ph_tridiag(c, sh);
}
__global__ void __launch_bounds__(kNT) nb_ritz_kernel(NBCtx c) {
  __shared__ NBShared sh;
  ph_ritz(c, blockIdx.x, gridDim.x, sh);
}
__global__ void __launch_bounds__(kNT) nb_ritz_norm_kernel(NBCtx c) {
  __shared__ NBShared sh;
  ph_ritz_norm(c, blockIdx.x, inv_norm_of_sum(c, sh));
}
__global__ void __launch_bounds__(kNT) nb_resid_kernel(NBCtx c) {
  __shared__ NBShared sh;
  ph_resid(c, blockIdx.x, sh);
}
__global__ void nb_final_kernel(NBCtx c) { ph_final(c); }

// ----------------------------------------------------- persistent kernel
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch: every CTA adds 1 to sync[0]
// (zeroed before the launch); the k-th barrier is passed when it reaches
// k * gridDim.x.  The wait is bounded: after kWaitLimitNs the CTA raises
// PSD_ERR_TIMEOUT and sync[1], and every CTA that sees sync[1] leaves the
// kernel at its next barrier.  Thread 0 keeps the count of barriers.
struct GridBarrier {
  unsigned* sync;
  unsigned epoch;
  __device__ __forceinline__ bool wait(int* status, volatile int* ok_sh) {
    __syncthreads();
    if (threadIdx.x == 0) {
      ++epoch;
      const unsigned target = epoch * gridDim.x;
      __threadfence();
      atomicAdd(sync, 1u);
      int ok = 1;
      const unsigned long long limit = g_debug_barrier_limit_ns;
      const unsigned long long t0 = globaltimer_ns();
      while (ld_acquire_u32(sync) < target) {
        if (ld_acquire_u32(sync + 1) != 0u) {
          // another CTA gave up; record it too: the first phase resets the
          // status word in CTA 0, which may run after that CTA's record, and
          // every CTA (CTA 0 included) leaves through a barrier after its own
          // first phase
          atomicCAS(status, 0, PSD_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        if (globaltimer_ns() - t0 >= limit) {  // >=: a zero limit gives up on the first poll
          atomicExch(sync + 1, 1u);
          atomicCAS(status, 0, PSD_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
      __threadfence();
      *ok_sh = ok;
    }
    __syncthreads();
    return *ok_sh != 0;
  }
};

// The whole bound in one launch: the phases of the multi-launch path in the
// same order, separated by grid barriers instead of kernel boundaries (about
// 150 of them, each a few microseconds shorter than a kernel boundary, and no
// launch of a small FP64 vector kernel waits on an empty GPU).
__global__ void __launch_bounds__(kNT, 2) nb_persistent_kernel(NBCtx c, unsigned* sync) {
  __shared__ NBShared sh;
  __shared__ volatile int ok_sh;
  GridBarrier gb{sync, 0u};
  int* status = &c.st->status;
  const int G = gridDim.x, b0 = blockIdx.x;
  const int npair = (c.npart + 1) / 2;  // chunk pairs of the reducing phases
  const float* X = c.args->X;
  const int64_t ld = c.args->ld;
#define NB_SYNC()                           \
  do {                                      \
    if (!gb.wait(status, &ok_sh)) return;   \
  } while (0)
  for (int vb = b0; vb < c.nv; vb += G) ph_init(c, vb, sh);
  NB_SYNC();
  for (int vb = b0; vb < c.nv; vb += G) ph_norm0(c, vb, sh);
  NB_SYNC();
  int pass = 0;
  for (int j = 0; j < kMaxSteps; ++j) {
    const bool rev = (pass++ & 1) != 0;
    if (j == 0)
      ph_symv_run<true>(c, X, ld, b0, G, rev, sh);
    else
      ph_symv_run<false>(c, X, ld, b0, G, rev, sh);
    NB_SYNC();
    if (j == 0 && b0 == 0 && threadIdx.x < 32) ph_fro(c);
    double* u = c.zsave ? c.zsave + j * c.npad : c.u;
    for (int cp = b0; cp < npair; cp += G) ph_reduce_split(c, cp, u, sh);
    NB_SYNC();
    ph_symv_run<false>(c, X, ld, b0, G, (pass++ & 1) != 0, sh);
    NB_SYNC();
    for (int cp = b0; cp < npair; cp += G) ph_reduce_dots(c, cp, j, sh);
    NB_SYNC();
    ph_orth1(c, b0, G, j, sh);
    NB_SYNC();
    double beta;
    if (ph_orth2_next(c, b0, G, j, sh, beta)) break;  // the same decision in every CTA
    NB_SYNC();
  }
  __syncthreads();  // thread 0's record of the last step, for warp 0
  if (b0 == 0 && threadIdx.x < 32) ph_tridiag(c, sh);
  NB_SYNC();
  ph_ritz(c, b0, G, sh);
  NB_SYNC();
  {
    const double inv = inv_norm_of_sum(c, sh);
    for (int vb = b0; vb < c.nv; vb += G) ph_ritz_norm(c, vb, inv);
  }
  NB_SYNC();
  ph_symv_run<false>(c, X, ld, b0, G, (pass++ & 1) != 0, sh);
  NB_SYNC();
  for (int cp = b0; cp < npair; cp += G) ph_reduce_split(c, cp, c.u, sh);
  NB_SYNC();
  ph_symv_run<false>(c, X, ld, b0, G, (pass++ & 1) != 0, sh);
  NB_SYNC();
  for (int cp = b0; cp < npair; cp += G) ph_resid(c, cp, sh);
  NB_SYNC();
  if (b0 == 0 && threadIdx.x < 32) ph_final(c);
#undef NB_SYNC
}

// TF32 rounding (10 explicit mantissa bits, nearest, ties away from zero) of a
// finite value; the tensor cores read only these bits of an FP32 operand.
__device__ __forceinline__ float tf32_round(float v) {
  if (!isfinite(v)) return v;
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

// Four consecutive elements (positions pos .. pos+3 of a row) of the output
// matrix in the chain's storage: 16-bit, or TF32 hi/lo pairs.
__device__ __forceinline__ void put16(uint16_t* H, const uint16_t (&u)[4], int valid) {
  if (valid == 4) {
    *reinterpret_cast<uint2*>(H) =
        make_uint2(u[0] | (static_cast<uint32_t>(u[1]) << 16), u[2] | (static_cast<uint32_t>(u[3]) << 16));
  } else {
    for (int k = 0; k < valid; ++k) H[k] = u[k];
  }
}

template <int DT>
__device__ __forceinline__ void store4(void* M, void* M_lo, int64_t pos, const float (&v)[4],
                                       int valid) {
  if (DT == DT_TF32X3) {
    float h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      h[k] = tf32_round(v[k]);
      l[k] = tf32_round(v[k] - h[k]);
    }
    float* Mh = static_cast<float*>(M) + pos;
    float* Ml = static_cast<float*>(M_lo) + pos;
    if (valid == 4) {
      *reinterpret_cast<float4*>(Mh) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4*>(Ml) = make_float4(l[0], l[1], l[2], l[3]);
    } else {
      for (int k = 0; k < valid; ++k) {
        Mh[k] = h[k];
        Ml[k] = l[k];
      }
    }
  } else {
    uint16_t u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      u[k] = DT == DT_BF16 ? __bfloat16_as_ushort(__float2bfloat16_rn(v[k])) : __half_as_ushort(__float2half_rn(v[k]));
    put16(static_cast<uint16_t*>(M) + pos, u, valid);
  }
}

// X_0 = RN(X * (1/lam~)) into a full symmetric matrix (16-bit, or TF32 hi/lo
// pairs), from the upper triangle of X, in 64 x 64 tiles through shared memory.
// Thread (tx, ty): rows i0 + 4 tx .. +3 (one 16-byte load), columns
// j0 + ty + 16 c, c = 0..3.  Both output positions are written with
// row-contiguous vector stores.
template <int DT>
__global__ void __launch_bounds__(256) scale_cast_kernel(const DevArgs* __restrict__ args, int n,
                                                         const DevState* __restrict__ st, void* __restrict__ M,
                                                         void* __restrict__ M_lo,
                                                         int64_t ldm) {
  __shared__ float s[64][65];
  int bi, bj;
  tile_of(blockIdx.x, bi, bj);
  const int i0 = bi * 64, j0 = bj * 64;
  const float* __restrict__ X = args->X;
  const int64_t ld = args->ld;
  const float inv = static_cast<float>(st->inv_lambda);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool diag = bi == bj;
  const bool vec = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
  const int ib = i0 + 4 * tx;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int jj = ty + 16 * c, j = j0 + jj;
    float x[4] = {0.f, 0.f, 0.f, 0.f};
    if (j < n) {
      const float* col = X + static_cast<int64_t>(j) * ld + ib;
      if (vec && ib + 3 < n) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(col));
        x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (ib + k < n) x[k] = __ldg(col + k);
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int ii = 4 * tx + k;
      s[ii][jj] = (!diag || ii <= jj) ? x[k] * inv : 0.f;
    }
  }
  __syncthreads();
  if (diag) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int jj = ty + 16 * c;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int ii = 4 * tx + k;
        if (ii > jj) s[ii][jj] = s[jj][ii];
      }
    }
    __syncthreads();
  }
  const int valid_i = min(4, n - ib);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int jj = ty + 16 * c, j = j0 + jj;
    // position (i + j ldm): memory row j, elements i0 + 4 tx .. +3
    if (j < n && valid_i > 0) {
      const float v[4] = {s[4 * tx][jj], s[4 * tx + 1][jj], s[4 * tx + 2][jj], s[4 * tx + 3][jj]};
      store4<DT>(M, M_lo, static_cast<int64_t>(j) * ldm + ib, v, valid_i);
    }
    // mirrored position (j + i ldm): memory row i = i0 + jj, elements j0 + 4 tx .. +3
    const int i = i0 + jj, jc = j0 + 4 * tx;
    const int valid_j = min(4, n - jc);
    if (!diag && i < n && valid_j > 0) {
      const float v[4] = {s[jj][4 * tx], s[jj][4 * tx + 1], s[jj][4 * tx + 2], s[jj][4 * tx + 3]};
      store4<DT>(M, M_lo, static_cast<int64_t>(i) * ldm + jc, v, valid_j);
    }
  }
}

// Caller pointers of one replay: the argument block, and (single projection)
// the caller-facing fields of the one block record.
__global__ void set_args_kernel(DevArgs* d, DevArgs h, BlockRec* blk) {
  *d = h;
  if (blk) {
    blk->X = h.X;
    blk->ld = h.ld;
    blk->out = h.out;
    blk->ld_out = h.ld_out;
  }
}

__global__ void set_block_kernel(BlockRec* dst, BlockRec v) { *dst = v; }

// Status word and overshoot of the last stage into the report, and the
// complementarity residual from the final product's per-warp shares (256
// threads: strided sums, warp trees, then the 8 warp sums in order).
__global__ void __launch_bounds__(kComplSumThreads)
    finalize_kernel(const DevArgs* args, DevState* st, const double* cres, int ncompl) {
  __shared__ double wsum[kComplSumThreads / 32];
  psd_info_t* info = args->info;
  const double v = compl_cta_sum<kComplSumThreads>(cres, cres ? ncompl : 0, wsum);
  if (threadIdx.x != 0) return;
  finalize_report(st, info);
  if (info) {
    const double f2 = st->fro * st->fro;
    info->compl_resid = !cres ? __longlong_as_double(0x7ff8000000000000ll) : (f2 > 0.0 ? v / f2 : 0.0);
  }
}

}  // namespace

cudaError_t set_norm_bound_debug(int knob, double value) {
  if (knob == 1) return cudaMemcpyToSymbol(g_debug_bound_scale, &value, sizeof(double));
  if (knob == 2) {
    const unsigned long long ns = static_cast<unsigned long long>(value);
    return cudaMemcpyToSymbol(g_debug_barrier_limit_ns, &ns, sizeof(ns));
  }
  return cudaErrorInvalidValue;
}

size_t lanczos_bytes(int64_t n) {
  const int64_t npad = (n + 255) / 256 * 256;
  const int64_t nb = (n + kSymvTile - 1) / kSymvTile;
  const int64_t ntiles = nb * (nb + 1) / 2;
  const int64_t nctas = (n + kVecThreads - 1) / kVecThreads;
  const int64_t npart = (n + 31) / 32;
  size_t b = 0;
  auto add = [&](size_t bytes) { b += (bytes + 255) / 256 * 256; };
  add(sizeof(double) * (kMaxSteps + 1) * npad);  // Qv
  add(sizeof(double) * npad * 3);                // u, w, q
  add(sizeof(float) * npad * 2);                 // vh, vl
  add(sizeof(float2) * nb * npad * 2);           // P1, P2
  add(sizeof(float2) * npart * 32);              // dots
  add(sizeof(float2) * npart * 32);              // dots2
  add(sizeof(double) * std::max(npart, nctas));  // norms
  add(sizeof(double) * ntiles);                  // tile_fro
  add(sizeof(unsigned) * 2);                     // grid barrier of the persistent kernel
  return b;
}

void lanczos_carve(LanczosBufs& L, int64_t n, uint8_t* base) {
  L.zsave = nullptr;
  L.n = n;
  L.npad = (n + 255) / 256 * 256;
  L.nb = static_cast<int>((n + kSymvTile - 1) / kSymvTile);
  L.ntiles = L.nb * (L.nb + 1) / 2;
  L.nvec_ctas = static_cast<int>((n + kVecThreads - 1) / kVecThreads);
  L.npart = static_cast<int>((n + 31) / 32);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    uint8_t* p = base + off;
    off += (bytes + 255) / 256 * 256;
    return p;
  };
  L.Qv = reinterpret_cast<double*>(take(sizeof(double) * (kMaxSteps + 1) * L.npad));
  double* v3 = reinterpret_cast<double*>(take(sizeof(double) * L.npad * 3));
  L.u = v3;
  L.w = v3 + L.npad;
  L.q = v3 + 2 * L.npad;
  float* f2 = reinterpret_cast<float*>(take(sizeof(float) * L.npad * 2));
  L.vh = f2;
  L.vl = f2 + L.npad;
  float2* P = reinterpret_cast<float2*>(take(sizeof(float2) * L.nb * L.npad * 2));
  L.P1 = P;
  L.P2 = P + static_cast<int64_t>(L.nb) * L.npad;
  L.dots = reinterpret_cast<float2*>(take(sizeof(float2) * L.npart * 32));
  L.dots2 = reinterpret_cast<float2*>(take(sizeof(float2) * L.npart * 32));
  L.norms = reinterpret_cast<double*>(take(sizeof(double) * std::max(L.npart, L.nvec_ctas)));
  L.tile_fro = reinterpret_cast<double*>(take(sizeof(double) * L.ntiles));
  L.sync = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * 2));
}

namespace {

NBCtx make_ctx(const LanczosBufs& L, const DevArgs* args, DevState* st) {
  NBCtx c{};
  c.n = static_cast<int>(L.n);
  c.nb = L.nb;
  c.ntiles = L.ntiles;
  c.nv = L.nvec_ctas;
  c.npart = L.npart;
  c.npad = L.npad;
  c.args = args;
  c.st = st;
  c.Qv = L.Qv;
  c.u = L.u;
  c.w = L.w;
  c.q = L.q;
  c.zsave = L.zsave;
  c.vh = L.vh;
  c.vl = L.vl;
  c.P1 = L.P1;
  c.P2 = L.P2;
  c.dots = L.dots;
  c.dots2 = L.dots2;
  c.norms = L.norms;
  c.norms2 = reinterpret_cast<float2*>(L.norms);
  c.tile_fro = L.tile_fro;
  return c;
}

// CTAs of the persistent kernel: as many as can be resident at once (a
// cooperative launch needs every CTA resident), no more than the largest
// phase has virtual blocks.  0 if the device cannot run it.
int persistent_grid(const NBCtx& c) {
  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, nb_persistent_kernel, kNT, 0) != cudaSuccess) return 0;
  const int work = std::max(std::max(c.ntiles, c.npart), c.nv);
  return std::min(occ * sms, std::max(work, 1));
}

}  // namespace

cudaError_t enqueue_norm_bound(const LanczosBufs& L, const DevArgs* args, DevState* st, cudaStream_t s,
                               bool persistent) {
  const NBCtx c = make_ctx(L, args, st);
  if (persistent) {
    const int G = persistent_grid(c);
    if (G > 0) {
      cudaError_t e = cudaMemsetAsync(L.sync, 0, 2 * sizeof(unsigned), s);
      if (e != cudaSuccess) return e;
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(G);
      cfg.blockDim = dim3(kNT);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, nb_persistent_kernel, c, L.sync);
    }
  }
  const int vb = c.nv, rb = c.npart, pb = (c.npart + 1) / 2;  // pb: chunk pairs
  nb_init_kernel<<<vb, kNT, 0, s>>>(c);
  nb_norm0_kernel<<<vb, kNT, 0, s>>>(c);
  int pass = 0;  // products over X so far: odd ones traverse the tiles backwards
  for (int j = 0; j < kMaxSteps; ++j) {
    if (j == 0) {
      nb_symv_kernel<true><<<c.ntiles, kNT, 0, s>>>(c, 0, pass++ & 1);
      nb_fro_kernel<<<1, 32, 0, s>>>(c);
    } else {
      nb_symv_kernel<false><<<c.ntiles, kNT, 0, s>>>(c, 1, pass++ & 1);
    }
    double* u = L.zsave ? L.zsave + j * L.npad : L.u;
    nb_reduce_split_kernel<<<pb, kNT, 0, s>>>(c, u, 1);
    nb_symv_kernel<false><<<c.ntiles, kNT, 0, s>>>(c, 1, pass++ & 1);
    nb_reduce_dots_kernel<<<pb, kNT, 0, s>>>(c, j);
    nb_orth1_kernel<<<rb, kNT, 0, s>>>(c, j);
    nb_orth2_kernel<<<rb, kNT, 0, s>>>(c, j);
  }
  nb_tridiag_kernel<<<1, 32, 0, s>>>(c);
  nb_ritz_kernel<<<rb, kNT, 0, s>>>(c);
  nb_ritz_norm_kernel<<<vb, kNT, 0, s>>>(c);
  // (after a breakdown the remaining steps' products do no work, so these two
  // may not continue the alternation; results do not depend on the direction)
  nb_symv_kernel<false><<<c.ntiles, kNT, 0, s>>>(c, 0, pass++ & 1);
  nb_reduce_split_kernel<<<pb, kNT, 0, s>>>(c, L.u, 0);
  nb_symv_kernel<false><<<c.ntiles, kNT, 0, s>>>(c, 0, pass++ & 1);
  nb_resid_kernel<<<pb, kNT, 0, s>>>(c);
  nb_final_kernel<<<1, 32, 0, s>>>(c);
  return cudaGetLastError();
}


cudaError_t enqueue_scale_cast(int dtype, const DevArgs* args, const DevState* st, int64_t n, void* M,
                               void* M_lo, int64_t ldm, cudaStream_t s) {
  const int nb = static_cast<int>((n + 63) / 64);
  const int tiles = nb * (nb + 1) / 2;
  const int blk = 256;
  const int ni = static_cast<int>(n);
  switch (dtype) {
    case DT_F16: scale_cast_kernel<DT_F16><<<tiles, blk, 0, s>>>(args, ni, st, M, M_lo, ldm); break;
    case DT_BF16: scale_cast_kernel<DT_BF16><<<tiles, blk, 0, s>>>(args, ni, st, M, M_lo, ldm); break;
    case DT_TF32X3: scale_cast_kernel<DT_TF32X3><<<tiles, blk, 0, s>>>(args, ni, st, M, M_lo, ldm); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t enqueue_set_args(DevArgs* d_args, const DevArgs& h, cudaStream_t s, BlockRec* blk) {
  set_args_kernel<<<1, 1, 0, s>>>(d_args, h, blk);
  return cudaGetLastError();
}

cudaError_t enqueue_set_block(BlockRec* d_blk, const BlockRec& v, cudaStream_t s) {
  set_block_kernel<<<1, 1, 0, s>>>(d_blk, v);
  return cudaGetLastError();
}

cudaError_t enqueue_finalize(const DevArgs* args, DevState* st, cudaStream_t s, const double* cres, int ncompl) {
  finalize_kernel<<<1, kComplSumThreads, 0, s>>>(args, st, cres, ncompl);
  return cudaGetLastError();
}

}  // namespace psd
