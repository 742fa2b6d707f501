// Grouped kernels of the batched projection of a block-diagonal cone: the
// norm bound of every block (Sec. 3.4, Theorem 2) in one sequence of launches,
// and the scaled cast of every block into the stacked iterate buffers.
//
// The mat-vec is one launch over the 128 x 128 upper tiles of all blocks
// (same per-tile arithmetic as the single-matrix kernel: 8-term FP32 FMA runs
// combined exactly into double-float partial sums); every vector operation of
// a block -- the Lanczos recurrence with full re-orthogonalisation, the Ritz
// vector, the residual and the bound -- runs in one CTA per block with a fixed
// reduction order, so a block's result does not depend on the other blocks of
// the batch.  The Lanczos vectors and their arithmetic are double-float (an
// FP32 pair hi + lo, about 48 significant bits: Dekker's products and Knuth's
// TwoSum): this GPU issues a warp's FP64 instruction every ~19 cycles per SM,
// and a block's whole step runs on one SM.
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
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr int kBT = 256;  // threads of a per-block CTA
constexpr int kEPT = kMaxBatchOrder / kBT;  // elements per thread
constexpr int kQChunk = 7;  // Lanczos vectors loaded at once in the Ritz vector's sum (21 = 3 x 7)

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
__device__ __forceinline__ F2 shfl_xor_f2(F2 a, int m) {
  return F2{__shfl_xor_sync(0xffffffffu, a.h, m), __shfl_xor_sync(0xffffffffu, a.l, m)};
}
// Normalised double-float arithmetic (hi = RN(hi + lo)).
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return F2{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 df_add(F2 a, F2 b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ F2 df_mul(F2 a, F2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ F2 df_neg(F2 a) { return F2{-a.h, -a.l}; }
__device__ __forceinline__ F2 df_from_d(double v) {
  const float h = __double2float_rn(v);
  return F2{h, __double2float_rn(v - static_cast<double>(h))};
}
// Loads of data written during the bound.  CG (the one-launch form, where
// other CTAs write it while the kernel runs): through L2 (ld.global.cg).
// Otherwise (grouped launches: written by earlier kernels) a plain load, which
// may hit L1 when a thread reads the same element again.
template <bool CG, typename T>
__device__ __forceinline__ T ldv(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}
template <bool CG>
__device__ __forceinline__ F2 ld_f2(const float2* p) {
  const float2 t = ldv<CG>(p);
  return F2{t.x, t.y};
}
__device__ __forceinline__ void st_f2(float2* p, F2 a) { *p = make_float2(a.h, a.l); }
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * kGolden;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Fixed-order sum over the CTA (kBT threads) of one FP64 value per thread.
__device__ __forceinline__ double cta_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kBT / 32; ++k) s += sh[k];
  return s;
}

// Fixed-order double-float sum over the CTA (kBT threads); every thread gets it.
__device__ __forceinline__ F2 cta_sum_df(F2 v, F2* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, shfl_xor_f2(v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  F2 s = sh[0];
#pragma unroll
  for (int k = 1; k < kBT / 32; ++k) s = df_add(s, sh[k]);
  return s;
}

// Per-block views of the batched Lanczos buffers.
struct BView {
  int n, nb;
  float2* Q;   // (kMaxSteps + 1) x n Lanczos vectors, double-float
  double* u;   // n
  double* w;   // n
  double* q;   // n
  float* vh;   // n
  float* vl;   // n
  float2* P1;  // nb x n
  float2* P2;  // nb x n
};
__device__ __forceinline__ BView view_of(const BatchLanczos& L, const BatchBlock& bb) {
  BView v;
  v.n = bb.n;
  v.nb = (bb.n + kSymvTile - 1) / kSymvTile;
  double* base = L.vec64 + bb.voff * (kMaxSteps + 4);
  v.Q = reinterpret_cast<float2*>(base);  // same 8 bytes per element
  v.u = base + static_cast<int64_t>(kMaxSteps + 1) * bb.n;
  v.w = v.u + bb.n;
  v.q = v.w + bb.n;
  v.vh = L.vec32 + bb.voff * 2;
  v.vl = v.vh + bb.n;
  v.P1 = L.part + bb.poff;
  v.P2 = v.P1 + static_cast<int64_t>(v.nb) * bb.n;
  return v;
}
__device__ __forceinline__ BView view(const BatchLanczos& L, int b) { return view_of(L, L.blk[b]); }

// ------------------------------------------------------------ grouped mat-vec
// One 128 x 128 upper tile (bi, bj) of a block: same arithmetic as the
// single-matrix kernel (see normbound.cu), partial sums into the block's
// P1 / P2.  In four pieces so that a loop over tiles can have the next tile's
// loads in flight while the previous one is reduced.

// The thread's 64 elements of the packed tile: column c of the tile at
// T + 128 c, zeros outside n x n (the zeros are not read: small blocks fill a
// few rows of their tile); on a diagonal tile, an 8 x 8 piece wholly below the
// diagonal (tr > tcol) is masked to zero below and not read either (18% of the
// bytes of 512 blocks of orders 16-1024).
// A 16-byte load of packed X with an L2 evict-first policy (the one-launch
// form, STREAM): there the mat-vec tiles stream while other CTAs run Lanczos
// steps, whose reads of the Lanczos vectors the tiles would otherwise push out
// of L2 (measured: the steps' dot products 25-30% faster).  The grouped
// launches keep the default policy: consecutive products read the tiles in
// opposite orders and find part of them in L2.
__device__ __forceinline__ float4 ld_stream4(const float* p) {
  float4 r;
  asm volatile(
      "{\n\t.reg .b64 pol;\n\tcreatepolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
      "ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], pol;\n\t}"
      : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
      : "l"(p));
  return r;
}

template <bool STREAM>
__device__ __forceinline__ void btile_load_x(const float* __restrict__ T, int n, int bi, int bj,
                                             float (&x)[8][8]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tr = lane & 15, tcol = 2 * warp + (lane >> 4);
  const int ib = bi * kSymvTile + 8 * tr;
  const int jb = bj * kSymvTile + 8 * tcol;
  const bool piece = bi != bj || tr <= tcol;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float* col = T + (8 * tcol + c) * kSymvTile + 8 * tr;
    const bool live = jb + c < n && ib < n && piece;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 a4 = !live ? z : STREAM ? ld_stream4(col) : __ldg(reinterpret_cast<const float4*>(col));
    const float4 b4 = !(live && ib + 4 < n) ? z
                      : STREAM              ? ld_stream4(col + 4)
                                            : __ldg(reinterpret_cast<const float4*>(col + 4));
    x[c][0] = a4.x; x[c][1] = a4.y; x[c][2] = a4.z; x[c][3] = a4.w;
    x[c][4] = b4.x; x[c][5] = b4.y; x[c][6] = b4.z; x[c][7] = b4.w;
  }
}

// The thread's slices of the mat-vec input (rows and columns).
template <bool CG>
__device__ __forceinline__ void btile_load_v(const float* vh, int n, int bi, int bj, float (&vi)[8],
                                             float (&vj)[8]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ib = bi * kSymvTile + 8 * (lane & 15);
  const int jb = bj * kSymvTile + 8 * (2 * warp + (lane >> 4));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    vi[k] = (ib + k < n) ? (CG ? __ldcg(vh + ib + k) : __ldg(vh + ib + k)) : 0.f;
    vj[k] = (jb + k < n) ? (CG ? __ldcg(vh + jb + k) : __ldg(vh + jb + k)) : 0.f;
  }
}

// Per-thread row and column dot products of the 8 x 8 piece (8-term FP32 FMA runs).
template <bool STATS, bool DIAG>
__device__ __forceinline__ void btile_fma(int n, int bi, int bj, const float (&vi)[8], const float (&vj)[8],
                                          const float (&x)[8][8], float (&rsum)[8], float (&csum)[8], float& fro,
                                          unsigned& mdiag) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ib = bi * kSymvTile + 8 * (lane & 15);
  const int jb = bj * kSymvTile + 8 * (2 * warp + (lane >> 4));
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
        const int i = ib + k, j = jb + c;
        xr = (i <= j) ? xr : 0.f;
        xc = (i < j) ? xc : 0.f;
        if (STATS && i == j && i < n) mdiag = max(mdiag, __float_as_uint(fabsf(x[c][k])));
      }
      rsum[k] = fmaf(xr, vj[c], rsum[k]);
      csum[c] = fmaf(xc, vi[k], csum[c]);
      if (STATS) fro = fmaf(xr, xc + xr, fro);
    }
  }
}

// Combines the threads' sums in a fixed order (double-float) into the tile's
// row partials P1[bj][rows] and column partials P2[bi][columns]; STATS: the
// tile's share of ||X||_F^2 and max |X_ii|.  `red` is read after its barrier:
// a loop over tiles alternates two buffers, since a tile two ahead writes one
// only after every thread has passed the barrier of the tile between (and so
// finished reading it).
template <bool STATS>
__device__ __forceinline__ void btile_reduce(int n, int bi, int bj, const float (&rsum)[8], const float (&csum)[8],
                                             float fro, unsigned mdiag, float2* __restrict__ P1,
                                             float2* __restrict__ P2, double* __restrict__ tile_fro, int tile_slot,
                                             unsigned* maxdiag, float2 (*red)[kSymvTile], double* fro_sh) {
  const int i0 = bi * kSymvTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tr = lane & 15;
  const int jb = bj * kSymvTile + 8 * (2 * warp + (lane >> 4));
  F2 cs[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float o = __shfl_xor_sync(0xffffffffu, rsum[k], 16);
    float h, e;
    if (lane < 16) two_sum(rsum[k], o, h, e); else two_sum(o, rsum[k], h, e);
    if (lane < 16) red[warp][8 * tr + k] = make_float2(h, e);
    cs[k] = F2{csum[k], 0.f};
  }
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
    const int j = jb + (tr >> 1);
    if ((tr & 1) == 0 && j < n) P2[static_cast<int64_t>(bi) * n + j] = make_float2(cs[0].h, cs[0].l);
  }
  __syncthreads();
  if (threadIdx.x < kSymvTile) {
    const int r = threadIdx.x;
    F2 a{red[0][r].x, red[0][r].y};
#pragma unroll
    for (int w = 1; w < 8; ++w) a = f2_add(a, F2{red[w][r].x, red[w][r].y});
    if (i0 + r < n) P1[static_cast<int64_t>(bj) * n + i0 + r] = make_float2(a.h, a.l);
  }
  if (STATS) {
    double f = static_cast<double>(fro);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0) fro_sh[warp] = f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mdiag = max(mdiag, __shfl_xor_sync(0xffffffffu, mdiag, o));
    if (lane == 0 && mdiag) atomicMax(maxdiag, mdiag);
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < 8; ++w) sum += fro_sh[w];
      tile_fro[tile_slot] = sum;
    }
  }
}


// Copies the 128 x 128 upper tiles of every block out of the caller's
// matrices into L.xt, one contiguous 64 KB tile per mat-vec work item (column
// c of the tile at 128 c; zeros outside the block and below the diagonal of a
// diagonal tile, which the mat-vec masks anyway).  The caller's leading
// dimensions are arbitrary, so this pass reads them with coalesced scalar
// loads once per projection, and the 41 mat-vecs that follow read aligned,
// contiguous tiles with 16-byte loads.
__global__ void __launch_bounds__(256) bpack_kernel(BatchLanczos L, const int4* __restrict__ items) {
  const int4 it = items[blockIdx.x];
  const BatchBlock bb = L.blk[it.x];
  const int i0 = it.y * kSymvTile, j0 = it.z * kSymvTile;
  const bool diag = it.y == it.z;
  float* T = L.xt + static_cast<int64_t>(blockIdx.x) * kSymvTile * kSymvTile;
  const int r = threadIdx.x & (kSymvTile - 1);
  for (int c = threadIdx.x >> 7; c < kSymvTile; c += 2) {
    const int i = i0 + r, j = j0 + c;
    float x = 0.f;
    if (i < bb.n && j < bb.n && (!diag || r <= c)) x = __ldg(bb.X + static_cast<int64_t>(j) * bb.ld + i);
    T[c * kSymvTile + r] = x;
  }
}

// work item: (block, bi, bj, tile slot of the block's tile_fro entries)
// `reverse` deals the items to the CTAs in the opposite order: consecutive
// products alternate direction, so each starts on the packed tiles the
// previous one read last, still in L2 (the packed tiles of a large batch
// exceed L2).  The item -> partial slot mapping does not change: results are
// identical.

// The grouped mat-vec as a persistent launch: CTA c takes the items r = c,
// c + G, ... (in the opposite order of the item list if `reverse`), and each
// next tile's X and input slices are loaded while the previous tile is
// reduced (a CTA per tile waits out every tile's load latency, and the small
// blocks' mostly empty tiles cost as much as full ones).  Same per-tile
// arithmetic and partial-sum slots as one CTA per tile: identical results.
template <bool STATS>
__global__ void __launch_bounds__(256, 2) bsymv_run_kernel(BatchLanczos L, const int4* __restrict__ items, int nitems,
                                                          int reverse) {
  __shared__ float2 red[2][8][kSymvTile];  // consecutive live tiles alternate (btile_reduce)
  __shared__ double fro_sh[8];
  const int G = static_cast<int>(gridDim.x);
  int buf = 0;
  auto item_at = [&](int r) { return reverse ? nitems - 1 - r : r; };
  int r = static_cast<int>(blockIdx.x);
  if (r >= nitems) return;
  int idx = item_at(r);
  int4 it = items[idx];
  BatchBlock bb = L.blk[it.x];
  float x[8][8], vi[8], vj[8];
  btile_load_x<false>(L.xt + static_cast<int64_t>(idx) * kSymvTile * kSymvTile, bb.n, it.y, it.z, x);
  btile_load_v<false>(view_of(L, bb).vh, bb.n, it.y, it.z, vi, vj);
  while (true) {
    const BView v = view_of(L, bb);
    const bool live = STATS || !(L.skip_done && L.st[it.x].done);
    float rsum[8], csum[8], fro;
    unsigned mdiag;
    if (live) {
      if (it.y == it.z)
        btile_fma<STATS, true>(v.n, it.y, it.z, vi, vj, x, rsum, csum, fro, mdiag);
      else
        btile_fma<STATS, false>(v.n, it.y, it.z, vi, vj, x, rsum, csum, fro, mdiag);
    }
    const int rn = r + G;
    const int4 cur = it;
    const int cur_b = it.x;
    if (rn < nitems) {  // in flight during the reduction
      idx = item_at(rn);
      it = items[idx];
      bb = L.blk[it.x];
      btile_load_x<false>(L.xt + static_cast<int64_t>(idx) * kSymvTile * kSymvTile, bb.n, it.y, it.z, x);
      btile_load_v<false>(view_of(L, bb).vh, bb.n, it.y, it.z, vi, vj);
    }
    if (live) {
      btile_reduce<STATS>(v.n, cur.y, cur.z, rsum, csum, fro, mdiag, v.P1, v.P2, L.tile_fro, cur.w,
                          &L.st[cur_b].maxdiag_bits, red[buf], fro_sh);
      buf ^= 1;
    }
    if (rn >= nitems) break;
    r = rn;
  }
}


// y_e of block b from its partial sums (fixed order, double-float, normalised), e < n:
// P1 of the tiles bj = b(e) .. nb - 1, then P2 of bi = 0 .. b(e).  All (at most
// 2 kMaxBatchOrder / 128) loads are issued before the additions.
constexpr int kMaxTileBlocks = kMaxBatchOrder / kSymvTile;
template <bool CG>
__device__ __forceinline__ F2 bred(const BView& v, int e) {
  const int bk = e / kSymvTile;
  float2 p1[kMaxTileBlocks], p2[kMaxTileBlocks];
#pragma unroll
  for (int i = 0; i < kMaxTileBlocks; ++i) {
    const int bj = bk + i, bi = i;
    p1[i] = bj < v.nb ? ldv<CG>(v.P1 + static_cast<int64_t>(bj) * v.n + e) : make_float2(0.f, 0.f);
    p2[i] = bi <= bk ? ldv<CG>(v.P2 + static_cast<int64_t>(bi) * v.n + e) : make_float2(0.f, 0.f);
  }
  F2 a{0.f, 0.f};
#pragma unroll
  for (int i = 0; i < kMaxTileBlocks; ++i)
    if (bk + i < v.nb) a = f2_add(a, F2{p1[i].x, p1[i].y});
#pragma unroll
  for (int i = 0; i < kMaxTileBlocks; ++i)
    if (i <= bk) a = f2_add(a, F2{p2[i].x, p2[i].y});
  return fast_two_sum(a.h, a.l);
}

// Lanczos vectors c0 .. c0 + kQChunk - 1 (those below `cnt`) at the thread's
// elements: every load issued before any is used (zeros elsewhere).
template <bool CG>
__device__ __forceinline__ void load_q_chunk(const BView& v, int c0, int cnt, F2 (&qk)[kEPT][kQChunk]) {
#pragma unroll
  for (int k = 0; k < kEPT; ++k) {
    const int e = threadIdx.x + k * kBT;
#pragma unroll
    for (int i = 0; i < kQChunk; ++i)
      qk[k][i] = (e < v.n && c0 + i < cnt) ? ld_f2<CG>(v.Q + static_cast<int64_t>(c0 + i) * v.n + e) : F2{0.f, 0.f};
  }
}

// ------------------------------------------------------------ per-block CTAs
// Start vector (SplitMix64, normalised), state reset, split for the first product.
__device__ __forceinline__ void ph_binit(const BatchLanczos& L, int b) {
  __shared__ F2 sh[kBT / 32];
  __shared__ double inv_sh;
  const BView v = view(L, b);
  F2 loc[kEPT];
  F2 s{0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kEPT; ++k) {
    const int e = threadIdx.x + k * kBT;
    F2 x{0.f, 0.f};
    if (e < v.n) {
      const uint64_t z = splitmix64(kSeed, static_cast<uint64_t>(e));
      x = df_from_d(2.0 * (static_cast<double>(z >> 11) * 0x1.0p-53) - 1.0);
    }
    loc[k] = x;
    s = df_add(s, df_mul(x, x));
  }
  const F2 nrm2 = cta_sum_df(s, sh);
  if (threadIdx.x == 0) inv_sh = 1.0 / sqrt(static_cast<double>(nrm2.h) + static_cast<double>(nrm2.l));
  __syncthreads();
  const F2 inv = df_from_d(inv_sh);
#pragma unroll
  for (int k = 0; k < kEPT; ++k) {
    const int e = threadIdx.x + k * kBT;
    if (e < v.n) {
      const F2 q = df_mul(loc[k], inv);
      st_f2(v.Q + e, q);
      v.vh[e] = q.h;
      v.vl[e] = q.l;
    }
  }
  if (threadIdx.x == 0) {
    DevState* st = &L.st[b];
    st->m = 0;
    st->done = 0;
    st->status = 0;
    st->maxdiag_bits = 0;
    st->absmax_bits = 0;
    st->sigma = st->resid = st->lambda = st->fro = st->maxdiag = st->inv_lambda = 0.0;
  }
}

// ||X_b||_F from the block's tile sums (after the first product).
// (lanes 0-31 of the CTA)
template <bool CG>
__device__ __forceinline__ void ph_bfro(const BatchLanczos& L, int b) {
  const BatchBlock& bb = L.blk[b];
  double f = 0.0;
  for (int t = threadIdx.x; t < bb.ntiles; t += 32) f += ldv<CG>(L.tile_fro + bb.toff + t);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if (threadIdx.x == 0) L.st[b].fro = sqrt(f);
}

// u = X v: reduce, store, split for the second product.  MODE 1: Ritz pass (no done check).
template <bool CG>
__device__ __forceinline__ void ph_breduce(const BatchLanczos& L, int b, int mode) {
  if (mode == 0 && ldv<CG>(&L.st[b].done)) return;
  const BView v = view(L, b);
  for (int e = threadIdx.x; e < v.n; e += kBT) {
    const F2 y = bred<CG>(v, e);
    v.u[e] = f2_to_d(y);
    v.vh[e] = y.h;
    v.vl[e] = y.l;
  }
}

// Lanczos step j after w = X u: alpha_j, two classical Gram-Schmidt passes
// (all j + 1 projections of a pass reduced together), beta_j, breakdown test,
// q_{j+1} = w / beta_j and its split, in double-float arithmetic.  Warps that
// own no element add zeros without arithmetic, and the cross-lane sum of the
// j + 1 partial dots halves only over V = 2^ceil(log2(j + 1)) values (then a
// plain butterfly), not all 32.  Every reduction has a fixed order that
// depends on j alone, so a block's result does not depend on the rest of the
// batch.

// Sum over the CTA (kBT threads) of v[k], k <= j, into out[k]: recursive
// halving over V values inside each warp (lane l ends with value l mod V,
// summed over its V-lane group), a butterfly over the 32 / V groups, then the
// warp sums of value k added in order by thread k.
__device__ __forceinline__ void cta_multi_sum(const F2 (&v)[kMaxSteps + 1], int j, bool warp_active,
                                              F2 (*sh)[32], F2* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (warp_active) {
    int V = 1;
    while (V < j + 1) V <<= 1;  // uniform across the CTA
    F2 t[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) t[k] = (k <= j && k <= kMaxSteps) ? v[k <= kMaxSteps ? k : 0] : F2{0.f, 0.f};
#pragma unroll
    for (int half = 16, m = 16; half >= 1; half >>= 1, m >>= 1) {
      if (half >= V) continue;  // values >= V are zero: skip the exchange
      const bool upper = (lane & m) != 0;
#pragma unroll
      for (int i = 0; i < half; ++i) {
        const F2 send = upper ? t[i] : t[i + half];
        const F2 keep = upper ? t[i + half] : t[i];
        t[i] = df_add(keep, shfl_xor_f2(send, m));
      }
    }
    // lanes l and l ^ (V, 2V, ...) hold the same value index: butterfly over them
    for (int m = V; m < 32; m <<= 1) t[0] = df_add(t[0], shfl_xor_f2(t[0], m));
    sh[w][lane] = t[0];
  } else {
    sh[w][lane] = F2{0.f, 0.f};
  }
  __syncthreads();
  if (threadIdx.x <= j) {
    F2 s = sh[0][threadIdx.x];
#pragma unroll
    for (int q = 1; q < kBT / 32; ++q) s = df_add(s, sh[q][threadIdx.x]);
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

template <bool CG>
__device__ __forceinline__ void ph_bstep(const BatchLanczos& L, int b, int j) {
  __shared__ F2 sh[kBT / 32][32];
  __shared__ F2 h[32];
  __shared__ F2 shs[kBT / 32];
  __shared__ double beta_sh[2];
  DevState* st = &L.st[b];
  if (ldv<CG>(&st->done)) return;
  const BView v = view(L, b);
  const bool any = (threadIdx.x & ~31) < v.n;  // the warp owns an element
  F2 w[kEPT];
#pragma unroll
  for (int k = 0; k < kEPT; ++k) {
    const int e = threadIdx.x + k * kBT;
    w[k] = e < v.n ? bred<CG>(v, e) : F2{0.f, 0.f};
  }
  for (int pass = 0; pass < 2; ++pass) {
    F2 d[kMaxSteps + 1];
#pragma unroll
    for (int kk = 0; kk <= kMaxSteps; ++kk) d[kk] = F2{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
      const int e = threadIdx.x + k * kBT;
      if (e < v.n) {
#pragma unroll
        for (int kk = 0; kk <= kMaxSteps; ++kk)
          if (kk <= j) d[kk] = df_add(d[kk], df_mul(ld_f2<CG>(v.Q + static_cast<int64_t>(kk) * v.n + e), w[k]));
      }
    }
    cta_multi_sum(d, j, any, sh, h);
    if (pass == 0 && threadIdx.x == 0) st->alpha[j] = f2_to_d(h[j]);
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
      const int e = threadIdx.x + k * kBT;
      if (e < v.n)
        for (int kk = 0; kk <= j; ++kk)
          w[k] = df_add(w[k], df_neg(df_mul(h[kk], ld_f2<CG>(v.Q + static_cast<int64_t>(kk) * v.n + e))));
    }
    __syncthreads();  // h is rewritten by the next pass
  }
  F2 s{0.f, 0.f};
  if (any) {
#pragma unroll
    for (int k = 0; k < kEPT; ++k) s = df_add(s, df_mul(w[k], w[k]));
  }
  const F2 nrm2 = cta_sum_df(s, shs);
  if (threadIdx.x == 0) {  // FP64 scalar work once per block
    const double bt = sqrt(f2_to_d(nrm2));
    beta_sh[0] = bt;
    beta_sh[1] = 1.0 / bt;
  }
  __syncthreads();
  const double beta = beta_sh[0];
  const double fro = ldv<CG>(&st->fro);
  const bool brk = !(beta > kBreakdown * fro * fro);
  if (brk || j == kMaxSteps - 1) {
    if (threadIdx.x == 0) {
      st->beta[j] = beta;
      st->m = j + 1;
      st->done = 1;
    }
    return;
  }
  if (threadIdx.x == 0) {
    st->beta[j] = beta;
    st->m = j + 1;
  }
  const F2 inv = df_from_d(beta_sh[1]);
#pragma unroll
  for (int k = 0; k < kEPT; ++k) {
    const int e = threadIdx.x + k * kBT;
    if (e < v.n) {
      const F2 q = df_mul(w[k], inv);
      st_f2(v.Q + static_cast<int64_t>(j + 1) * v.n + e, q);
      v.vh[e] = q.h;
      v.vl[e] = q.l;
    }
  }
}

// Largest Ritz pair of each block's tridiagonal (one warp per block):
// multisection on the Sturm count, inverse iteration with partial pivoting,
// then q = Q_m y, normalised, split.
template <bool CG>
__device__ __forceinline__ void ph_britz(const BatchLanczos& L, int b) {
  __shared__ double y[kMaxSteps];
  __shared__ float a32[kMaxSteps], b32[kMaxSteps];
  __shared__ F2 sh[kBT / 32];
  __shared__ F2 yf[kMaxSteps];
  __shared__ double inv_sh;
  __shared__ double ab[2][kMaxSteps];
  DevState* st = &L.st[b];
  const int m = ldv<CG>(&st->m);
  if (threadIdx.x < 32) {
    if (threadIdx.x < kMaxSteps) {
      ab[0][threadIdx.x] = ldv<CG>(st->alpha + threadIdx.x);
      ab[1][threadIdx.x] = ldv<CG>(st->beta + threadIdx.x);
    }
    __syncwarp();
    const double sigma = tridiag_top_eig(ab[0], ab[1], m, y, a32, b32);
    if (threadIdx.x == 0) {
      st->sigma = sigma;
      for (int k = 0; k < kMaxSteps; ++k) st->y[k] = y[k];
    }
  }
  if (threadIdx.x < kMaxSteps) yf[threadIdx.x] = df_from_d(y[threadIdx.x]);
  __syncthreads();
  const BView v = view(L, b);
  F2 qv[kEPT];
#pragma unroll
  for (int k = 0; k < kEPT; ++k) qv[k] = F2{0.f, 0.f};
  // qv = sum_k y_k q_k in order k = 0 .. m - 1
#pragma unroll
  for (int c0 = 0; c0 < kMaxSteps; c0 += kQChunk) {
    if (c0 < m) {
      F2 qk[kEPT][kQChunk];
      load_q_chunk<CG>(v, c0, m, qk);
#pragma unroll
      for (int k = 0; k < kEPT; ++k) {
        if (threadIdx.x + k * kBT < v.n) {
#pragma unroll
          for (int i = 0; i < kQChunk; ++i)
            if (c0 + i < m) qv[k] = df_add(qv[k], df_mul(yf[c0 + i], qk[k][i]));
        }
      }
    }
  }
  F2 s{0.f, 0.f};
#pragma unroll
  for (int k = 0; k < kEPT; ++k) s = df_add(s, df_mul(qv[k], qv[k]));
  const F2 nrm2 = cta_sum_df(s, sh);
  if (threadIdx.x == 0) {
    const double n2 = f2_to_d(nrm2);
    inv_sh = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
  }
  __syncthreads();
  const F2 inv = df_from_d(inv_sh);
#pragma unroll
  for (int k = 0; k < kEPT; ++k) {
    const int e = threadIdx.x + k * kBT;
    if (e < v.n) {
      const F2 t = df_mul(qv[k], inv);
      v.q[e] = f2_to_d(t);
      v.vh[e] = t.h;
      v.vl[e] = t.l;
    }
  }
}

// r = ||X (X q) - sigma q||, lam~ = max(sqrt(sigma + r), ||X||_F / sqrt n, max |X_ii|), report.
template <bool CG>
__device__ __forceinline__ void ph_bbound(const BatchLanczos& L, int b) {
  __shared__ double sh[kBT / 32];
  DevState* st = &L.st[b];
  const BView v = view(L, b);
  const double sigma = ldv<CG>(&st->sigma);
  double s = 0.0;
  for (int e = threadIdx.x; e < v.n; e += kBT) {
    const double r = f2_to_d(bred<CG>(v, e)) - sigma * ldv<CG>(v.q + e);
    s += r * r;
  }
  const double r2 = cta_sum(s, sh);
  if (threadIdx.x != 0) return;
  const double r = sqrt(r2);
  const double fro = ldv<CG>(&st->fro);
  const double md = static_cast<double>(__uint_as_float(ldv<CG>(&st->maxdiag_bits)));
  double lam = sqrt(fmax(sigma + r, 0.0));
  lam = fmax(lam, fro / sqrt(static_cast<double>(v.n)));
  lam = fmax(lam, md);
  st->resid = r;
  st->maxdiag = md;
  if (!(isfinite(fro) && isfinite(lam) && isfinite(sigma))) {
    atomicCAS(&st->status, 0, PSD_ERR_NONFINITE);
    lam = 0.0;
  }
  st->lambda = lam;
  st->inv_lambda = lam > 0.0 ? 1.0 / lam : 0.0;
  psd_info_t* info = L.blk[b].info;
  if (info) {
    info->lambda_bound = lam;
    info->lanczos_sigma = sigma;
    info->lanczos_resid = r;
    info->fro_X = fro;
    info->max_diag = md;
    info->lanczos_steps = ldv<CG>(&st->m);
    info->status = ldv<CG>(&st->status);
    info->compl_resid = __longlong_as_double(0x7ff8000000000000ll);  // set by the last step
  }
}

// One CTA per block (block order[blockIdx.x]) for the grouped launches.
__global__ void __launch_bounds__(kBT) binit_kernel(BatchLanczos L) { ph_binit(L, L.order[blockIdx.x]); }
__global__ void bfro_kernel(BatchLanczos L) { ph_bfro<false>(L, L.order[blockIdx.x]); }
__global__ void __launch_bounds__(kBT) breduce_kernel(BatchLanczos L, int mode) {
  ph_breduce<false>(L, L.order[blockIdx.x], mode);
}
__global__ void __launch_bounds__(kBT) bstep_kernel(BatchLanczos L, int j) {
  ph_bstep<false>(L, L.order[blockIdx.x], j);
}
__global__ void __launch_bounds__(kBT) britz_kernel(BatchLanczos L) { ph_britz<false>(L, L.order[blockIdx.x]); }
__global__ void __launch_bounds__(kBT) bbound_kernel(BatchLanczos L) { ph_bbound<false>(L, L.order[blockIdx.x]); }

// ------------------------------------------------------------ one-launch form
// The whole batched bound as ONE launch of resident CTAs that take work items
// from a list in a fixed global order (host-built, see build_flow): a block's
// items are its start vector, then per Lanczos step its mat-vec tiles (up to 4
// per item, pipelined), its reduction, its mat-vec tiles again and its step,
// then the Ritz vector and the residual's two products and reduction, and its
// bound.  Each CTA claims the next item with one atomic add (the claim of item
// k + 1 is issued while item k waits for its inputs), waits until the block's
// counter shows every item the new one depends on done (item.w = the number of
// the block's earlier items; a mat-vec item loads its first tile's X before it
// waits), runs it with the same per-tile and per-block device code as the
// grouped launches, and adds 1 to the counter.  No grid-wide barrier: a block's next phase starts as soon
// as its own previous phase is done, so the Lanczos steps of the large blocks
// overlap the mat-vec tiles of the others.
//
// Progress: items are claimed in list order and an item waits only for items
// of lower index.  The unfinished item of lowest index is therefore claimed by
// a running CTA whose earlier items are all finished, and its inputs are
// ready: it completes, whatever the residency of the other CTAs.  Every wait
// is bounded: after g_flow_limit_ns the CTA raises the abort word, every CTA
// that sees it leaves, and the batch reports PSD_ERR_TIMEOUT.
//
// Results are bit-identical to the grouped launches: each item runs the same
// arithmetic on the same inputs, and every reduction order is fixed per block.
__device__ unsigned long long g_flow_limit_ns = kWaitLimitNs;


__device__ __forceinline__ unsigned ld_acquire_flow(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0: wait until *cnt >= need, or give up (abort word ctl[1]).  The
// acquire load orders thread 0 after the producers' counts; the CTA barrier
// that follows orders the other threads after it, and every read of data
// another item wrote goes through L2 (ld.global.cg), where the producers'
// stores were performed before their counts.
__device__ __forceinline__ bool flow_wait(const unsigned* cnt, unsigned need, unsigned* ctl) {
  if (ld_acquire_flow(cnt) >= need) return true;
  const unsigned long long limit = g_flow_limit_ns;
  const unsigned long long t0 = globaltimer_ns();
  while (ld_acquire_flow(cnt) < need) {
    if (ld_acquire_flow(ctl + 1) != 0u) return false;
    if (globaltimer_ns() - t0 >= limit) {  // >=: a zero limit gives up on the first poll
      atomicExch(ctl + 1, 1u);
      return false;
    }
  }
  return true;
}

// Tile t of a block's upper tiles in their list order (column-major over the
// upper triangle: t = bj (bj + 1) / 2 + bi).
__device__ __forceinline__ void btile_of(int t, int& bi, int& bj) {
  int j = static_cast<int>((sqrtf(8.f * static_cast<float>(t) + 1.f) - 1.f) * 0.5f);
  while ((j + 1) * (j + 2) / 2 <= t) ++j;
  while (j * (j + 1) / 2 > t) --j;
  bj = j;
  bi = t - j * (j + 1) / 2;
}

// Mat-vec item: tiles first .. first + cnt - 1 of block b (consecutive entries
// of the tile list), the packed X of the first already in x; each next tile's
// X and input slices are loaded while the previous tile is reduced.  Per
// tile the same arithmetic as the grouped mat-vec (bsymv_run_kernel).
template <bool STATS>
__device__ __forceinline__ void ph_bsymv_run(const BatchLanczos& L, int b, int first, int cnt, float (&x)[8][8],
                                             float2 (*red)[8][kSymvTile], double* fro_sh) {
  const BatchBlock bb = L.blk[b];
  const BView v = view_of(L, bb);
  int bi, bj;
  btile_of(first - static_cast<int>(bb.toff), bi, bj);
  float vi[8], vj[8];
  btile_load_v<true>(v.vh, v.n, bi, bj, vi, vj);
  for (int k = 0; k < cnt; ++k) {
    float rsum[8], csum[8], fro;
    unsigned mdiag;
    if (bi == bj)
      btile_fma<STATS, true>(v.n, bi, bj, vi, vj, x, rsum, csum, fro, mdiag);
    else
      btile_fma<STATS, false>(v.n, bi, bj, vi, vj, x, rsum, csum, fro, mdiag);
    const int ci = bi, cj = bj;
    if (k + 1 < cnt) {  // in flight during the reduction
      btile_of(first + k + 1 - static_cast<int>(bb.toff), bi, bj);
      btile_load_x<true>(L.xt + static_cast<int64_t>(first + k + 1) * kSymvTile * kSymvTile, v.n, bi, bj, x);
      btile_load_v<true>(v.vh, v.n, bi, bj, vi, vj);
    }
    btile_reduce<STATS>(v.n, ci, cj, rsum, csum, fro, mdiag, v.P1, v.P2, L.tile_fro, first + k,
                        &L.st[b].maxdiag_bits, red[k & 1], fro_sh);
  }
}

__global__ void __launch_bounds__(kBT, 2) bflow_kernel(BatchLanczos L, const int4* __restrict__ flow, int nflow,
                                                      unsigned* ctl, unsigned* cnt) {
  __shared__ float2 red[2][8][kSymvTile];  // tiles of an item alternate (btile_reduce)
  __shared__ double fro_sh[8];
  __shared__ int claim_sh[2];
  __shared__ int ok_sh;
  if (threadIdx.x == 0) claim_sh[0] = static_cast<int>(atomicAdd(ctl, 1u));
  __syncthreads();
  int slot = 0;
  int cur = claim_sh[0];
  int4 fn = cur < nflow ? __ldg(flow + cur) : make_int4(0, 0, 0, 0);
  while (cur < nflow) {
    const int4 f = fn;
    const int kind = f.x & 0xff, j = (f.x >> 8) & 0xff, b = f.y;
    float x[8][8];
    if (kind == FK_MV) {  // X does not change during the bound: load before the wait
      const BatchBlock& bb = L.blk[b];
      int bi, bj;
      btile_of(f.z - static_cast<int>(bb.toff), bi, bj);
      btile_load_x<true>(L.xt + static_cast<int64_t>(f.z) * kSymvTile * kSymvTile, bb.n, bi, bj, x);
    }
    if (threadIdx.x == 0) {
      const unsigned next = atomicAdd(ctl, 1u);  // in flight during the wait
      ok_sh = flow_wait(cnt + b, static_cast<unsigned>(f.w), ctl);
      claim_sh[slot ^ 1] = static_cast<int>(next);
    }
    __syncthreads();
    if (!ok_sh) return;
    // the next item's record, in flight during this one
    const int nxt = claim_sh[slot ^ 1];
    fn = nxt < nflow ? __ldg(flow + nxt) : make_int4(0, 0, 0, 0);
    switch (kind) {
      case FK_INIT: ph_binit(L, b); break;
      case FK_MV: {
        const int ntile = (f.x >> 20) & 0xf;
        if (f.x & FF_STATS)
          ph_bsymv_run<true>(L, b, f.z, ntile, x, red, fro_sh);
        else if (!((f.x & FF_SKIP) && __ldcg(&L.st[b].done)))
          ph_bsymv_run<false>(L, b, f.z, ntile, x, red, fro_sh);
        break;
      }
      case FK_RED:
        if ((f.x & FF_FRO) && threadIdx.x < 32) ph_bfro<true>(L, b);
        ph_breduce<true>(L, b, (f.x & FF_RITZ) ? 1 : 0);
        break;
      case FK_STEP: ph_bstep<true>(L, b, j); break;
      case FK_RITZ: ph_britz<true>(L, b); break;
      default: ph_bbound<true>(L, b); break;
    }
    __syncthreads();  // every thread's stores of the item precede the count
    // the count goes out from another warp: thread 0 goes on to the next claim
    if (threadIdx.x == 32) {
      __threadfence();
      atomicAdd(cnt + b, 1u);
    }
    slot ^= 1;
    cur = claim_sh[slot];
  }
}

// ------------------------------------------------------------ grouped cast
__device__ __forceinline__ void put4_16(uint16_t* H, const uint16_t (&u)[4], int valid) {
  if (valid == 4) {
    *reinterpret_cast<uint2*>(H) =
        make_uint2(u[0] | (static_cast<uint32_t>(u[1]) << 16), u[2] | (static_cast<uint32_t>(u[3]) << 16));
  } else {
    for (int k = 0; k < valid; ++k) H[k] = u[k];
  }
}
__device__ __forceinline__ float tf32_round(float v) {
  if (!isfinite(v)) return v;
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

template <int DT>
__device__ __forceinline__ void bstore4(const BatchCast& c, int64_t pos, const float (&v)[4], int valid) {
  if (DT == DT_TF32X3) {
    float* Mh = static_cast<float*>(c.M) + pos;
    float* Ml = static_cast<float*>(c.M_lo) + pos;
    for (int k = 0; k < valid; ++k) {
      const float h = tf32_round(v[k]);
      Mh[k] = h;
      Ml[k] = tf32_round(v[k] - h);
    }
  } else {
    uint16_t u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      u[k] = DT == DT_BF16 ? __bfloat16_as_ushort(__float2bfloat16_rn(v[k])) : __half_as_ushort(__float2half_rn(v[k]));
    put4_16(static_cast<uint16_t*>(c.M) + pos, u, valid);
  }
}

// X_0 of every block into the stacked buffers (64 x 64 upper tiles, item =
// (block, bi, bj)); same arithmetic as the single-matrix cast.
template <int DT>
__global__ void __launch_bounds__(256) bcast_kernel(BatchCast c, const BatchBlock* __restrict__ blk,
                                                    const DevState* __restrict__ st, const int4* __restrict__ items) {
  __shared__ float s[64][65];
  const int4 it = items[blockIdx.x];
  const BatchBlock& bb = blk[it.x];
  const int n = bb.n;
  const int i0 = it.y * 64, j0 = it.z * 64;
  const float* __restrict__ X = bb.X;
  const int64_t ld = bb.ld;
  const float inv = static_cast<float>(st[it.x].inv_lambda);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const bool diag = it.y == it.z;
  const int ib = i0 + 4 * tx;
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    const int jj = ty + 16 * cc, j = j0 + jj;
    float x[4] = {0.f, 0.f, 0.f, 0.f};
    if (j < n) {
      const float* col = X + static_cast<int64_t>(j) * ld + ib;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (ib + k < n) x[k] = __ldg(col + k);
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
    for (int cc = 0; cc < 4; ++cc) {
      const int jj = ty + 16 * cc;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int ii = 4 * tx + k;
        if (ii > jj) s[ii][jj] = s[jj][ii];
      }
    }
    __syncthreads();
  }
  const int64_t rowbase = bb.off;  // stacked rows of this block
  const int valid_i = min(4, n - ib);
#pragma unroll
  for (int cc = 0; cc < 4; ++cc) {
    const int jj = ty + 16 * cc, j = j0 + jj;
    if (j < n && valid_i > 0) {
      const float v[4] = {s[4 * tx][jj], s[4 * tx + 1][jj], s[4 * tx + 2][jj], s[4 * tx + 3][jj]};
      bstore4<DT>(c, (rowbase + j) * c.ldm + ib, v, valid_i);
    }
    const int i = i0 + jj, jc = j0 + 4 * tx;
    const int valid_j = min(4, n - jc);
    if (!diag && i < n && valid_j > 0) {
      const float v[4] = {s[jj][4 * tx], s[jj][4 * tx + 1], s[jj][4 * tx + 2], s[jj][4 * tx + 3]};
      bstore4<DT>(c, (rowbase + i) * c.ldm + jc, v, valid_j);
    }
  }
}

// Status and overshoot of every block into its report.
// Per block: status and overshoot, and the complementarity residual from the
// shares of the block's final-product tiles, added in the block's own tile
// order (cidx: positions of its tiles in the launch's tile list, range crange[b])
// so that the sum does not depend on the schedule or the rest of the batch.
// A one-launch bound that gave up (abort word set) marks every block: a block
// whose items were not all run may still hold an earlier call's state.
__global__ void bfinalize_kernel(const BatchBlock* __restrict__ blk, DevState* st, int count,
                                 const double* __restrict__ cres, const int* __restrict__ cidx,
                                 const int2* __restrict__ crange, int shares, const unsigned* flow_abort) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  const float amax = __uint_as_float(st[b].absmax_bits);
  int status = st[b].status;
  if (status == 0 && flow_abort && *flow_abort) {
    status = PSD_ERR_TIMEOUT;
    st[b].status = status;
  }
  if (status == 0) {
    if (!(amax == amax) || isinf(amax))
      status = PSD_ERR_NONFINITE;
    else if (amax > kOvershootLimit)
      status = PSD_ERR_BOUND;
    st[b].status = status;
  }
  psd_info_t* info = blk[b].info;
  if (info) {
    info->overshoot_max = static_cast<double>(amax);
    info->status = status;
    double v = 0.0;
    const int2 rg = crange[b];
    for (int k = rg.x; k < rg.x + rg.y; ++k)
      for (int w = 0; w < shares; ++w) v += cres[shares * static_cast<int64_t>(cidx[k]) + w];
    const double f2 = st[b].fro * st[b].fro;
    info->compl_resid = f2 > 0.0 ? v / f2 : 0.0;
  }
}

}  // namespace

cudaError_t enqueue_batch_norm_bound(const BatchLanczos& L, int count, const int4* symv_items, int nsymv,
                                     cudaStream_t s) {
  // resident CTAs per SM of the persistent mat-vec (computed once, thread-safe)
  static const int occ = [] {
    int o = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, bsymv_run_kernel<false>, 256, 0) == cudaSuccess ? o
                                                                                                            : 0;
  }();
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int mv_grid = std::max(1, std::min(occ * num_sms(), nsymv));
  BatchLanczos Lk = L;
  Lk.skip_done = 0;
  bpack_kernel<<<nsymv, 256, 0, s>>>(Lk, symv_items);
  binit_kernel<<<count, kBT, 0, s>>>(Lk);
  int pass = 0;  // products so far: odd ones traverse the items backwards
  for (int j = 0; j < kMaxSteps; ++j) {
    Lk.skip_done = j == 0 ? 0 : 1;
    if (j == 0) {
      bsymv_run_kernel<true><<<mv_grid, 256, 0, s>>>(Lk, symv_items, nsymv, pass++ & 1);
      bfro_kernel<<<count, 32, 0, s>>>(Lk);
    } else {
      bsymv_run_kernel<false><<<mv_grid, 256, 0, s>>>(Lk, symv_items, nsymv, pass++ & 1);
    }
    breduce_kernel<<<count, kBT, 0, s>>>(Lk, 0);
    Lk.skip_done = 1;
    bsymv_run_kernel<false><<<mv_grid, 256, 0, s>>>(Lk, symv_items, nsymv, pass++ & 1);
    bstep_kernel<<<count, kBT, 0, s>>>(Lk, j);
  }
  britz_kernel<<<count, kBT, 0, s>>>(Lk);
  Lk.skip_done = 0;
  bsymv_run_kernel<false><<<mv_grid, 256, 0, s>>>(Lk, symv_items, nsymv, pass++ & 1);
  breduce_kernel<<<count, kBT, 0, s>>>(Lk, 1);
  bsymv_run_kernel<false><<<mv_grid, 256, 0, s>>>(Lk, symv_items, nsymv, pass++ & 1);
  bbound_kernel<<<count, kBT, 0, s>>>(Lk);
  return cudaGetLastError();
}

cudaError_t enqueue_batch_norm_bound_flow(const BatchLanczos& L, const int4* symv_items, int nsymv, const int4* flow,
                                          int nflow, unsigned* ctl, int count, cudaStream_t s) {
  // resident CTAs per SM (the same on every device of a process: one GPU
  // type); computed once, thread-safe (function-local static)
  static const int occ = [] {
    int o = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, bflow_kernel, kBT, 0) == cudaSuccess ? o : 0;
  }();
  if (occ < 1) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(unsigned) * (2 + count), s);
  if (e != cudaSuccess) return e;
  BatchLanczos Lk = L;
  Lk.skip_done = 0;
  bpack_kernel<<<nsymv, 256, 0, s>>>(Lk, symv_items);
  const int grid = std::max(1, std::min(occ * num_sms(), nflow));
  bflow_kernel<<<grid, kBT, 0, s>>>(Lk, flow, nflow, ctl, ctl + 2);
  return cudaGetLastError();
}

cudaError_t set_batch_flow_limit(unsigned long long ns) {
  return cudaMemcpyToSymbol(g_flow_limit_ns, &ns, sizeof(ns));
}

cudaError_t enqueue_batch_cast(int dtype, const BatchCast& c, const BatchBlock* blk, const DevState* st,
                               const int4* items, int nitems, cudaStream_t s) {
  switch (dtype) {
    case DT_F16: bcast_kernel<DT_F16><<<nitems, 256, 0, s>>>(c, blk, st, items); break;
    case DT_BF16: bcast_kernel<DT_BF16><<<nitems, 256, 0, s>>>(c, blk, st, items); break;
    case DT_TF32X3: bcast_kernel<DT_TF32X3><<<nitems, 256, 0, s>>>(c, blk, st, items); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t enqueue_batch_finalize(const BatchBlock* blk, DevState* st, int count, const double* cres,
                                   const int* cidx, const int2* crange, int shares, const unsigned* flow_abort,
                                   cudaStream_t s) {
  bfinalize_kernel<<<(count + 127) / 128, 128, 0, s>>>(blk, st, count, cres, cidx, crange, shares, flow_abort);
  return cudaGetLastError();
}

}  // namespace psd
