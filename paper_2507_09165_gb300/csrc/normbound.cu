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

#include <cmath>

#include "internal.h"
#include "tridiag.cuh"

namespace psd {

namespace {

constexpr uint64_t kSeed = 0x243F6A8885A308D3ull;  // Lanczos start vector seed
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

// ------------------------------------------------------------------ kernels

// Block-wide FP64 sum of one value per thread (kVecThreads threads), fixed order.
__device__ __forceinline__ double block_sum64(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < kVecThreads / 32; ++k) s += sh[k];
  __syncthreads();
  return s;
}

// Fixed-order warp sum of cnt FP64 values (lane-strided, then a butterfly).
__device__ __forceinline__ double warp_sum_array(const double* a, int cnt, int stride) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int c = lane; c < cnt; c += 32) s += a[static_cast<int64_t>(c) * stride];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// State reset + start vector q_0 (unit SplitMix64 vector), split for the first mat-vec.
__global__ void lanczos_init_kernel(int n, int64_t npad, double* Qv, float* vh, float* vl, DevState* st,
                                    double* norms) {
  __shared__ double sh[kVecThreads / 32];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (e < n) {
    const uint64_t z = splitmix64(kSeed, static_cast<uint64_t>(e));
    const double u = static_cast<double>(z >> 11) * 0x1.0p-53;
    v = 2.0 * u - 1.0;
  }
  const double s = block_sum64(v * v, sh);
  if (threadIdx.x == 0) norms[blockIdx.x] = s;
  if (e < n) Qv[e] = v;  // unnormalised; lanczos_norm0 scales it
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->m = 0;
    st->done = 0;
    st->status = 0;
    st->maxdiag_bits = 0;
    st->absmax_bits = 0;
    st->sigma = st->resid = st->lambda = st->fro = st->maxdiag = st->inv_lambda = 0.0;
  }
}

// q_0 /= ||v||, split.
__global__ void lanczos_norm0_kernel(int n, double* Qv, float* vh, float* vl, const double* norms,
                                     int nctas) {
  __shared__ double inv;
  if (threadIdx.x < 32) {
    const double s = warp_sum_array(norms, nctas, 1);
    if (threadIdx.x == 0) inv = 1.0 / sqrt(s);
  }
  __syncthreads();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) {
    const double q = Qv[e] * inv;
    Qv[e] = q;
    split_d(q, vh[e], vl[e]);
  }
}

// One tile of y = X v over the upper triangle (see file comment).  Thread
// (tr, tc) = (lane & 15, 2 warp + lane / 16) owns rows i0 + 8 tr .. +7 and
// columns j0 + 8 tc .. +7: each column's 128 rows are read by a half-warp as
// 512 contiguous bytes.  DIAG tiles mask to i <= j (rows) and i < j
// (columns).  STATS adds the tile's share of ||X||_F^2 and max |X_ii|.
template <bool STATS, bool DIAG>
__device__ __forceinline__ void symv_tile(const float* __restrict__ X, int64_t ld, int n, int bi, int bj,
                                          const float* __restrict__ vh, float2* __restrict__ P1,
                                          float2* __restrict__ P2, int64_t ps, double* __restrict__ tile_fro,
                                          DevState* __restrict__ st, float2 (*red)[kSymvTile], double* fro_sh) {
  const int i0 = bi * kSymvTile, j0 = bj * kSymvTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tr = lane & 15, tcol = 2 * warp + (lane >> 4);
  const int ib = i0 + 8 * tr;
  const int jb = j0 + 8 * tcol;
  const bool full = (ib + 7 < n) && (jb + 7 < n);
  const bool vec = full && ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
  float vi[8], vj[8], x[8][8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    vi[k] = (ib + k < n) ? __ldg(vh + ib + k) : 0.f;
    vj[k] = (jb + k < n) ? __ldg(vh + jb + k) : 0.f;
  }
  // all 64 elements first: 16 independent 16-byte loads in flight per thread
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float* col = X + static_cast<int64_t>(jb + c) * ld + ib;
    if (vec) {
      const float4 a4 = __ldg(reinterpret_cast<const float4*>(col));
      const float4 b4 = __ldg(reinterpret_cast<const float4*>(col + 4));
      x[c][0] = a4.x; x[c][1] = a4.y; x[c][2] = a4.z; x[c][3] = a4.w;
      x[c][4] = b4.x; x[c][5] = b4.y; x[c][6] = b4.z; x[c][7] = b4.w;
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[c][k] = (jb + c < n && ib + k < n) ? __ldg(col + k) : 0.f;
    }
  }
  float rsum[8], csum[8];
  float fro = 0.f;
  unsigned mdiag = 0;
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
      if (STATS) fro = fmaf(xr, xc + xr, fro);  // x^2 on the diagonal, 2 x^2 above it
    }
  }
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
    const int j = jb + (tr >> 1);
    if ((tr & 1) == 0 && j < n) P2[static_cast<int64_t>(bi) * ps + j] = make_float2(cs[0].h, cs[0].l);
  }
  __syncthreads();
  if (threadIdx.x < kSymvTile) {
    const int r = threadIdx.x;
    F2 a{red[0][r].x, red[0][r].y};
#pragma unroll
    for (int w = 1; w < 8; ++w) a = f2_add(a, F2{red[w][r].x, red[w][r].y});
    if (i0 + r < n) P1[static_cast<int64_t>(bj) * ps + i0 + r] = make_float2(a.h, a.l);
  }
  if (STATS) {
    double f = static_cast<double>(fro);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0) fro_sh[warp] = f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mdiag = max(mdiag, __shfl_xor_sync(0xffffffffu, mdiag, o));
    if (lane == 0 && mdiag) atomicMax(&st->maxdiag_bits, mdiag);
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < 8; ++w) sum += fro_sh[w];
      tile_fro[blockIdx.x] = sum;
    }
  }
}

template <bool STATS>
__global__ void __launch_bounds__(256, 2) symv_upper_kernel(const DevArgs* __restrict__ args, int n,
                                                            const float* __restrict__ vh,
                                                            const float* __restrict__ vl,
                                                            float2* __restrict__ P1, float2* __restrict__ P2,
                                                            int64_t ps, double* __restrict__ tile_fro,
                                                            DevState* __restrict__ st, int skip_if_done) {
  if (skip_if_done && st->done) return;
  __shared__ float2 red[8][kSymvTile];
  __shared__ double fro_sh[8];
  (void)vl;
  int bi, bj;
  tile_of(blockIdx.x, bi, bj);
  if (bi == bj)
    symv_tile<STATS, true>(args->X, args->ld, n, bi, bj, vh, P1, P2, ps, tile_fro, st, red, fro_sh);
  else
    symv_tile<STATS, false>(args->X, args->ld, n, bi, bj, vh, P1, P2, ps, tile_fro, st, red, fro_sh);
}

// ||X||_F from the per-tile sums of the first product (one warp, fixed order).
__global__ void fro_kernel(const double* tile_fro, int ntiles, DevState* st) {
  double f = 0.0;
  for (int t = threadIdx.x; t < ntiles; t += 32) f += tile_fro[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if (threadIdx.x == 0) st->fro = sqrt(f);
}

// y_e = sum_{bj >= b(e)} P1[bj][e] + sum_{bi <= b(e)} P2[bi][e] for the 32
// elements e of this CTA (kRedThreads threads): warp w adds the blocks
// congruent to w mod 8 in double-float, then warp 0 combines the 8 warp sums
// in a fixed order.  Returns y_e (FP64) in warp 0; other warps return 0.
constexpr int kRedThreads = 256;
__device__ __forceinline__ double reduce_partials_cta(int n, int nb, const float2* __restrict__ P1,
                                                      const float2* __restrict__ P2, int64_t ps, float2 (*sh)[32]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  F2 a{0.f, 0.f}, c{0.f, 0.f};
  if (e < n) {
    const int b = e / kSymvTile;
#pragma unroll 4
    for (int bj = b + w; bj < nb; bj += 8) {
      const float2 t = __ldg(P1 + static_cast<int64_t>(bj) * ps + e);
      a = f2_add(a, F2{t.x, t.y});
    }
#pragma unroll 4
    for (int bi = w; bi <= b; bi += 8) {
      const float2 t = __ldg(P2 + static_cast<int64_t>(bi) * ps + e);
      c = f2_add(c, F2{t.x, t.y});
    }
  }
  const F2 t = f2_add(a, c);
  sh[w][lane] = make_float2(t.h, t.l);
  __syncthreads();
  double y = 0.0;
  if (w == 0) {
    F2 acc{sh[0][lane].x, sh[0][lane].y};
#pragma unroll
    for (int q = 1; q < kRedThreads / 32; ++q) acc = f2_add(acc, F2{sh[q][lane].x, sh[q][lane].y});
    y = f2_to_d(acc);
  }
  return y;
}

// u = X v (first product of X (X v)); split u for the second product.
__global__ void __launch_bounds__(kRedThreads) reduce_split_kernel(int n, int nb, const float2* P1,
                                                                   const float2* P2, int64_t ps, double* u,
                                                                   float* vh, float* vl, const DevState* st,
                                                                   int skip_if_done) {
  if (skip_if_done && st->done) return;
  __shared__ float2 sh[kRedThreads / 32][32];
  const double y = reduce_partials_cta(n, nb, P1, P2, ps, sh);
  const int e = blockIdx.x * 32 + (threadIdx.x & 31);
  if (threadIdx.x < 32 && e < n) {
    u[e] = y;
    split_d(y, vh[e], vl[e]);
  }
}

// Recursive-halving sum of cnt (<= 32) FP64 values over a warp; on return
// lane l < cnt holds the warp total of value l.  Values live in v[0..31].
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
  // lane l now holds value index bitrev-free: index = lane (bits consumed high to low)
  return v[0];
}

// w = X u; partial dots h_k = q_k . w (k = 0..j) over this CTA's 32 elements.
__global__ void __launch_bounds__(kRedThreads) reduce_dots_kernel(int n, int nb, const float2* P1,
                                                                  const float2* P2, int64_t ps, double* w,
                                                                  const double* Qv, int64_t npad, int j,
                                                                  double* dots, const DevState* st) {
  if (st->done) return;
  __shared__ float2 sh[kRedThreads / 32][32];
  const double y = reduce_partials_cta(n, nb, P1, P2, ps, sh);
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const int e = blockIdx.x * 32 + lane;
  if (e < n) w[e] = y;
  double v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = (k <= j && e < n) ? Qv[static_cast<int64_t>(k) * npad + e] * y : 0.0;
  dots[blockIdx.x * 32 + lane] = warp_multi_sum(v, lane);
}

// Classical Gram-Schmidt pass: h = sum over CTAs of the partial dots (same
// order in every CTA); w -= sum_k h_k q_k; new partial dots (pass 1) or
// partial squared norm (pass 2).  Pass 1 also records alpha_j = h_j.
template <int PASS>
__global__ void orth_kernel(int n, double* w, const double* Qv, int64_t npad, int j, const double* dots_in,
                            int nctas, double* out_partial, DevState* st) {
  if (st->done) return;
  __shared__ double h[32];
  __shared__ double sh[kVecThreads / 32][32];
  // h_k = sum over CTAs of the partial dots; warp w reduces k = w, w + nwarps, ...
  // (every CTA sums the same partials in the same order)
  for (int k = threadIdx.x >> 5; k <= j; k += kVecThreads / 32) {
    const double t = warp_sum_array(dots_in + k, nctas, 32);
    if ((threadIdx.x & 31) == 0) h[k] = t;
  }
  __syncthreads();
  if (PASS == 1 && blockIdx.x == 0 && threadIdx.x == 0) st->alpha[j] = h[j];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  double we = 0.0;
  if (e < n) {
    we = w[e];
    for (int k = 0; k <= j; ++k) we -= h[k] * Qv[static_cast<int64_t>(k) * npad + e];
    w[e] = we;
  }
  if (PASS == 1) {
    double v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = (k <= j && e < n) ? Qv[static_cast<int64_t>(k) * npad + e] * we : 0.0;
    const double s = warp_multi_sum(v, lane);
    sh[wp][lane] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
      double t = 0.0;
      for (int q = 0; q < kVecThreads / 32; ++q) t += sh[q][threadIdx.x];
      out_partial[blockIdx.x * 32 + threadIdx.x] = t;
    }
  } else {
    const double s = block_sum64(we * we, &sh[0][0]);
    if (threadIdx.x == 0) out_partial[blockIdx.x] = s;
  }
}

// beta_j = ||w||; breakdown test; q_{j+1} = w / beta_j and its split.
__global__ void lanczos_next_kernel(int n, const double* w, double* Qv, int64_t npad, int j,
                                    const double* norms, int nctas, float* vh, float* vl, DevState* st) {
  if (st->done) return;
  __shared__ double beta_s, fro2_s;
  if (threadIdx.x < 32) {
    const double s = warp_sum_array(norms, nctas, 1);
    if (threadIdx.x == 0) {
      beta_s = sqrt(s);
      fro2_s = st->fro * st->fro;
    }
  }
  __syncthreads();
  const double beta = beta_s;
  const bool last = (j == kMaxSteps - 1);
  const bool brk = !(beta > kBreakdown * fro2_s);  // also true for NaN
  if (brk || last) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->beta[j] = beta;
      st->m = j + 1;
      st->done = 1;
    }
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->beta[j] = beta;
    st->m = j + 1;
  }
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) {
    const double q = w[e] / beta;
    Qv[static_cast<int64_t>(j + 1) * npad + e] = q;
    split_d(q, vh[e], vl[e]);
  }
}

// Largest eigenpair of the Lanczos tridiagonal (tridiag.cuh): sigma and the
// Ritz vector's coordinates y in the Lanczos basis.
__global__ void tridiag_kernel(DevState* st) {
  __shared__ double y[kMaxSteps];
  __shared__ float a32[kMaxSteps], b32[kMaxSteps];
  const double sigma = tridiag_top_eig(st->alpha, st->beta, st->m, y, a32, b32);
  if (threadIdx.x == 0) {
    st->sigma = sigma;
    for (int k = 0; k < kMaxSteps; ++k) st->y[k] = y[k];
  }
}

// q = sum_k y_k q_k, partial ||q||^2.
__global__ void ritz_kernel(int n, const double* Qv, int64_t npad, double* q, double* norms,
                            const DevState* st) {
  __shared__ double sh[kVecThreads / 32];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = st->m;
  double s = 0.0;
  if (e < n) {
    for (int k = 0; k < m; ++k) s += st->y[k] * Qv[static_cast<int64_t>(k) * npad + e];
    q[e] = s;
  }
  const double t = block_sum64(s * s, sh);
  if (threadIdx.x == 0) norms[blockIdx.x] = t;
}

// q /= ||q||, split for the residual products.
__global__ void ritz_norm_kernel(int n, double* q, const double* norms, int nctas, float* vh, float* vl) {
  __shared__ double inv;
  if (threadIdx.x < 32) {
    const double s = warp_sum_array(norms, nctas, 1);
    if (threadIdx.x == 0) inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  }
  __syncthreads();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) {
    const double v = q[e] * inv;
    q[e] = v;
    split_d(v, vh[e], vl[e]);
  }
}

// r = X (X q) - sigma q, partial ||r||^2 over this CTA's 32 elements.
__global__ void __launch_bounds__(kRedThreads) resid_kernel(int n, int nb, const float2* P1, const float2* P2,
                                                            int64_t ps, const double* q, double* norms,
                                                            const DevState* st) {
  __shared__ float2 sh[kRedThreads / 32][32];
  const double y = reduce_partials_cta(n, nb, P1, P2, ps, sh);
  if (threadIdx.x >= 32) return;
  const int e = blockIdx.x * 32 + threadIdx.x;
  double r = 0.0;
  if (e < n) r = y - st->sigma * q[e];
  double t = r * r;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (threadIdx.x == 0) norms[blockIdx.x] = t;
}

// lam~ = max(sqrt(sigma + r), ||X||_F / sqrt n, max |X_ii|); report.
__global__ void bound_final_kernel(int n, const double* norms, int nctas, DevState* st, const DevArgs* args) {
  const double r2 = warp_sum_array(norms, nctas, 1);
  if (threadIdx.x != 0) return;
  const double r = sqrt(r2);
  const double fro = st->fro;
  const double fro2 = fro * fro;
  const double md = static_cast<double>(__uint_as_float(st->maxdiag_bits));
  const double sigma = st->sigma;
  double lam = sqrt(fmax(sigma + r, 0.0));
  lam = fmax(lam, fro / sqrt(static_cast<double>(n)));
  lam = fmax(lam, md);
  st->resid = r;
  st->maxdiag = md;
  const bool finite = isfinite(fro2) && isfinite(lam) && isfinite(sigma);
  if (!finite) {
    atomicCAS(&st->status, 0, PSD_ERR_NONFINITE);
    lam = 0.0;
  }
  st->lambda = lam;
  st->inv_lambda = lam > 0.0 ? 1.0 / lam : 0.0;
  psd_info_t* info = args->info;
  if (info) {
    info->lambda_bound = lam;
    info->lanczos_sigma = sigma;
    info->lanczos_resid = r;
    info->fro_X = fro;
    info->max_diag = md;
    info->lanczos_steps = st->m;
    info->status = st->status;
    info->compl_resid = __longlong_as_double(0x7ff8000000000000ll);  // set by a projection's last step
  }
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
  add(sizeof(double) * npart * 32);              // dots
  add(sizeof(double) * nctas * 32);              // dots2
  add(sizeof(double) * npart);                   // norms
  add(sizeof(double) * ntiles);                  // tile_fro
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
  L.dots = reinterpret_cast<double*>(take(sizeof(double) * L.npart * 32));
  L.dots2 = reinterpret_cast<double*>(take(sizeof(double) * L.nvec_ctas * 32));
  L.norms = reinterpret_cast<double*>(take(sizeof(double) * L.npart));
  L.tile_fro = reinterpret_cast<double*>(take(sizeof(double) * L.ntiles));
}

cudaError_t enqueue_norm_bound(const LanczosBufs& L, const DevArgs* args, DevState* st, cudaStream_t s) {
  const int n = static_cast<int>(L.n);
  const int vb = L.nvec_ctas, vt = kVecThreads, rb = L.npart, rt = kRedThreads;
  const int64_t ps = L.npad;
  lanczos_init_kernel<<<vb, vt, 0, s>>>(n, L.npad, L.Qv, L.vh, L.vl, st, L.norms);
  lanczos_norm0_kernel<<<vb, vt, 0, s>>>(n, L.Qv, L.vh, L.vl, L.norms, vb);
  for (int j = 0; j < kMaxSteps; ++j) {
    if (j == 0) {
      symv_upper_kernel<true><<<L.ntiles, 256, 0, s>>>(args, n, L.vh, L.vl, L.P1, L.P2, ps, L.tile_fro, st, 0);
      fro_kernel<<<1, 32, 0, s>>>(L.tile_fro, L.ntiles, st);
    } else {
      symv_upper_kernel<false><<<L.ntiles, 256, 0, s>>>(args, n, L.vh, L.vl, L.P1, L.P2, ps, L.tile_fro, st, 1);
    }
    double* u = L.zsave ? L.zsave + j * L.npad : L.u;
    reduce_split_kernel<<<rb, rt, 0, s>>>(n, L.nb, L.P1, L.P2, ps, u, L.vh, L.vl, st, 1);
    symv_upper_kernel<false><<<L.ntiles, 256, 0, s>>>(args, n, L.vh, L.vl, L.P1, L.P2, ps, L.tile_fro, st, 1);
    reduce_dots_kernel<<<rb, rt, 0, s>>>(n, L.nb, L.P1, L.P2, ps, L.w, L.Qv, L.npad, j, L.dots, st);
    orth_kernel<1><<<vb, vt, 0, s>>>(n, L.w, L.Qv, L.npad, j, L.dots, rb, L.dots2, st);
    orth_kernel<2><<<vb, vt, 0, s>>>(n, L.w, L.Qv, L.npad, j, L.dots2, vb, L.norms, st);
    lanczos_next_kernel<<<vb, vt, 0, s>>>(n, L.w, L.Qv, L.npad, j, L.norms, vb, L.vh, L.vl, st);
  }
  tridiag_kernel<<<1, 32, 0, s>>>(st);
  ritz_kernel<<<vb, vt, 0, s>>>(n, L.Qv, L.npad, L.q, L.norms, st);
  ritz_norm_kernel<<<vb, vt, 0, s>>>(n, L.q, L.norms, vb, L.vh, L.vl);
  symv_upper_kernel<false><<<L.ntiles, 256, 0, s>>>(args, n, L.vh, L.vl, L.P1, L.P2, ps, L.tile_fro, st, 0);
  reduce_split_kernel<<<rb, rt, 0, s>>>(n, L.nb, L.P1, L.P2, ps, L.u, L.vh, L.vl, st, 0);
  symv_upper_kernel<false><<<L.ntiles, 256, 0, s>>>(args, n, L.vh, L.vl, L.P1, L.P2, ps, L.tile_fro, st, 0);
  resid_kernel<<<rb, rt, 0, s>>>(n, L.nb, L.P1, L.P2, ps, L.q, L.norms, st);
  bound_final_kernel<<<1, 32, 0, s>>>(n, L.norms, rb, st, args);
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
