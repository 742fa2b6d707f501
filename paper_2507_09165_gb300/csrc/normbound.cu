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
// element-level arithmetic uses the error-free transformations of Ogita,
// Rump & Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 2005,
// algorithm Dot2: TwoProduct by FMA, TwoSum) in FP32, which returns the dot
// product as accurately as if it were computed in twice the working precision;
// v enters as an FP64 value split into two FP32 parts.  Partial sums cross to
// FP64 per tile row/column; every reduction over the vector (dot products,
// norms) is FP64 with a fixed order.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>

#include "internal.h"

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
// acc += x * (vh + vl)   (Dot2 step: TwoProduct + TwoSum, error terms carried in l)
__device__ __forceinline__ void dot2(F2& acc, float x, float vh, float vl) {
  const float p = __fmul_rn(x, vh);
  float e = __fmaf_rn(x, vh, -p);
  e = __fmaf_rn(x, vl, e);
  float s, q;
  two_sum(acc.h, p, s, q);
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(q, e));
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

__device__ __forceinline__ void tile_of(int t, int& bi, int& bj) {
  int j = static_cast<int>((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
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

// One tile of y = X v over the upper triangle (see file comment).  STATS adds
// the tile's share of ||X||_F^2 and max |X_ii| (first product only).
template <bool STATS>
__global__ void __launch_bounds__(256) symv_upper_kernel(const DevArgs* __restrict__ args, int n,
                                                         const float* __restrict__ vh,
                                                         const float* __restrict__ vl,
                                                         float2* __restrict__ P1, float2* __restrict__ P2,
                                                         int64_t ps, double* __restrict__ tile_fro,
                                                         DevState* __restrict__ st, int skip_if_done) {
  if (skip_if_done && st->done) return;
  __shared__ float red_h[8][kSymvTile];
  __shared__ float red_l[8][kSymvTile];
  __shared__ double fro_sh[8];
  const float* __restrict__ X = args->X;
  const int64_t ld = args->ld;
  int bi, bj;
  tile_of(blockIdx.x, bi, bj);
  const int i0 = bi * kSymvTile, j0 = bj * kSymvTile;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ib = i0 + 4 * lane;
  const int jb = j0 + 16 * warp;
  const bool diag = bi == bj;

  float vih[4], vil[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = ib + k;
    vih[k] = i < n ? vh[i] : 0.f;
    vil[k] = i < n ? vl[i] : 0.f;
  }
  F2 rs[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) rs[k] = F2{0.f, 0.f};
  F2 cs[16];
  F2 fro{0.f, 0.f};
  unsigned mdiag = 0;
  const bool vec = ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (ib + 3 < n);
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    cs[c] = F2{0.f, 0.f};
    const int j = jb + c;
    if (j >= n) continue;
    const float* col = X + static_cast<int64_t>(j) * ld;
    float x[4];
    if (vec) {
      const float4 q4 = __ldg(reinterpret_cast<const float4*>(col + ib));
      x[0] = q4.x;
      x[1] = q4.y;
      x[2] = q4.z;
      x[3] = q4.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) x[k] = (ib + k < n) ? __ldg(col + ib + k) : 0.f;
    }
    const float vjh = vh[j], vjl = vl[j];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = ib + k;
      const bool up = (!diag || i <= j) && i < n;
      const bool strict = (!diag || i < j) && i < n;
      const float xu = up ? x[k] : 0.f;
      dot2(rs[k], xu, vjh, vjl);
      if (strict) dot2(cs[c], x[k], vih[k], vil[k]);
      if (STATS) {
        dot2(fro, xu, strict ? 2.f * xu : xu, 0.f);
        if (diag && i == j) mdiag = max(mdiag, __float_as_uint(fabsf(x[k])));
      }
    }
  }
  // rows: reduce over the 8 warps through shared memory
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    red_h[warp][4 * lane + k] = rs[k].h;
    red_l[warp][4 * lane + k] = rs[k].l;
  }
  // columns: recursive halving over the 32 lanes; lanes 2c, 2c+1 end with column c
#pragma unroll
  for (int half = 8, m = 16; half >= 1; half >>= 1, m >>= 1) {
    const bool upper = (lane & m) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const F2 send = upper ? cs[i] : cs[i + half];
      const F2 keep = upper ? cs[i + half] : cs[i];
      cs[i] = f2_add(keep, shfl_xor_f2(send, m));
    }
  }
  cs[0] = f2_add(cs[0], shfl_xor_f2(cs[0], 1));
  {
    const int j = jb + (lane >> 1);
    if ((lane & 1) == 0 && j < n) P2[static_cast<int64_t>(bi) * ps + j] = make_float2(cs[0].h, cs[0].l);
  }
  __syncthreads();
  if (threadIdx.x < kSymvTile) {
    const int r = threadIdx.x;
    F2 a{red_h[0][r], red_l[0][r]};
#pragma unroll
    for (int w = 1; w < 8; ++w) a = f2_add(a, F2{red_h[w][r], red_l[w][r]});
    if (i0 + r < n) P1[static_cast<int64_t>(bj) * ps + i0 + r] = make_float2(a.h, a.l);
  }
  if (STATS) {
    double f = f2_to_d(fro);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (lane == 0) fro_sh[warp] = f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mdiag = max(mdiag, __shfl_xor_sync(0xffffffffu, mdiag, o));
    if (lane == 0 && mdiag) atomicMax(&st->maxdiag_bits, mdiag);
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < 8; ++w) s += fro_sh[w];
      tile_fro[blockIdx.x] = s;
    }
  }
}

// ||X||_F from the per-tile sums of the first product (one warp, fixed order).
__global__ void fro_kernel(const double* tile_fro, int ntiles, DevState* st) {
  double f = 0.0;
  for (int t = threadIdx.x; t < ntiles; t += 32) f += tile_fro[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if (threadIdx.x == 0) st->fro = sqrt(f);
}

// y_e = sum_{bj >= b(e)} P1[bj][e] + sum_{bi <= b(e)} P2[bi][e] in double-float, then FP64.
__device__ __forceinline__ double reduce_partials(int e, int nb, const float2* P1, const float2* P2,
                                                  int64_t ps) {
  const int b = e / kSymvTile;
  F2 a{0.f, 0.f};
  for (int bj = b; bj < nb; ++bj) {
    const float2 t = P1[static_cast<int64_t>(bj) * ps + e];
    a = f2_add(a, F2{t.x, t.y});
  }
  for (int bi = 0; bi <= b; ++bi) {
    const float2 t = P2[static_cast<int64_t>(bi) * ps + e];
    a = f2_add(a, F2{t.x, t.y});
  }
  return f2_to_d(a);
}

// u = X v (first product of X (X v)); split u for the second product.
__global__ void reduce_split_kernel(int n, int nb, const float2* P1, const float2* P2, int64_t ps,
                                    double* u, float* vh, float* vl, const DevState* st,
                                    int skip_if_done) {
  if (skip_if_done && st->done) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double y = reduce_partials(e, nb, P1, P2, ps);
  u[e] = y;
  split_d(y, vh[e], vl[e]);
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

// w = X u; partial dots h_k = q_k . w (k = 0..j) per CTA.
__global__ void reduce_dots_kernel(int n, int nb, const float2* P1, const float2* P2, int64_t ps,
                                   double* w, const double* Qv, int64_t npad, int j, double* dots,
                                   const DevState* st) {
  if (st->done) return;
  __shared__ double sh[kVecThreads / 32][32];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  double y = 0.0;
  if (e < n) {
    y = reduce_partials(e, nb, P1, P2, ps);
    w[e] = y;
  }
  double v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) v[k] = (k <= j && e < n) ? Qv[static_cast<int64_t>(k) * npad + e] * y : 0.0;
  const double s = warp_multi_sum(v, lane);
  sh[wp][lane] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int q = 0; q < kVecThreads / 32; ++q) t += sh[q][threadIdx.x];
    dots[blockIdx.x * 32 + threadIdx.x] = t;
  }
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
  if (threadIdx.x < 32) {
    double t = 0.0;
    if (static_cast<int>(threadIdx.x) <= j)
      for (int c = 0; c < nctas; ++c) t += dots_in[c * 32 + threadIdx.x];
    h[threadIdx.x] = t;
  }
  __syncthreads();  // h_k: every CTA sums the same partials in the same order
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

// Sturm count: number of eigenvalues of T (m x m, diag a, off-diag b) below x.
__device__ int sturm_count(const double* a, const double* b, int m, double x) {
  int cnt = 0;
  double d = a[0] - x;
  if (d < 0.0) ++cnt;
  for (int k = 1; k < m; ++k) {
    if (d == 0.0) d = -1e-300;
    d = (a[k] - x) - b[k - 1] * b[k - 1] / d;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// Largest eigenpair of the Lanczos tridiagonal: multisection on the Sturm
// count (32 points per round), then inverse iteration with partial pivoting.
__global__ void tridiag_kernel(DevState* st) {
  __shared__ double a[kMaxSteps], b[kMaxSteps];
  __shared__ double lo_s, hi_s;
  const int lane = threadIdx.x;
  const int m = st->m;
  if (lane < m) {
    a[lane] = st->alpha[lane];
    b[lane] = lane < m - 1 ? st->beta[lane] : 0.0;
  }
  __syncwarp();
  if (lane == 0) {
    double lo = a[0], hi = a[0];
    for (int k = 0; k < m; ++k) {
      const double r = (k > 0 ? fabs(b[k - 1]) : 0.0) + (k < m - 1 ? fabs(b[k]) : 0.0);
      lo = fmin(lo, a[k] - r);
      hi = fmax(hi, a[k] + r);
    }
    lo_s = lo;
    hi_s = hi;
  }
  __syncwarp();
  for (int round = 0; round < 40; ++round) {
    const double lo = lo_s, hi = hi_s;
    if (!(hi - lo > 4.0 * 2.2e-16 * fmax(fabs(lo), fabs(hi)))) break;
    const double x = lo + (hi - lo) * (lane + 1) / 33.0;
    const int all_below = sturm_count(a, b, m, x) >= m;  // x is above every eigenvalue
    const unsigned mask = __ballot_sync(0xffffffffu, all_below);
    __syncwarp();
    if (lane == 0) {
      const int first = mask ? __ffs(mask) - 1 : 32;  // first x above the top eigenvalue
      const double nlo = first == 0 ? lo : lo + (hi - lo) * first / 33.0;
      const double nhi = first == 32 ? hi : lo + (hi - lo) * (first + 1) / 33.0;
      lo_s = nlo;
      hi_s = nhi;
    }
    __syncwarp();
  }
  if (lane != 0) return;
  const double sigma = 0.5 * (lo_s + hi_s);
  // inverse iteration on (T - sigma I): Gaussian elimination with partial
  // pivoting on the tridiagonal (rows may swap, which creates a second
  // super-diagonal).
  double tnorm = 0.0;
  for (int k = 0; k < m; ++k) tnorm = fmax(tnorm, fabs(a[k]) + (k ? fabs(b[k - 1]) : 0.0) + fabs(b[k]));
  const double tiny = fmax(tnorm, 1e-300) * 1e-15;
  double d[kMaxSteps], du[kMaxSteps], du2[kMaxSteps], dl[kMaxSteps], l[kMaxSteps];
  int piv[kMaxSteps];
  for (int k = 0; k < m; ++k) {
    d[k] = a[k] - sigma;
    du[k] = k < m - 1 ? b[k] : 0.0;
    dl[k] = k < m - 1 ? b[k] : 0.0;
    du2[k] = 0.0;
    piv[k] = 0;
  }
  for (int k = 0; k < m - 1; ++k) {
    if (fabs(d[k]) >= fabs(dl[k])) {
      if (d[k] == 0.0) d[k] = tiny;
      l[k] = dl[k] / d[k];
      d[k + 1] -= l[k] * du[k];
    } else {
      piv[k] = 1;
      l[k] = d[k] / dl[k];
      d[k] = dl[k];
      const double t = d[k + 1];
      d[k + 1] = du[k] - l[k] * t;
      du[k] = t;
      if (k < m - 2) {
        du2[k] = du[k + 1];
        du[k + 1] = -l[k] * du[k + 1];
      }
    }
  }
  if (d[m - 1] == 0.0) d[m - 1] = tiny;
  double y[kMaxSteps];
  for (int k = 0; k < m; ++k) y[k] = 1.0;
  for (int it = 0; it < 3; ++it) {
    // forward: apply L^-1 with the row swaps
    for (int k = 0; k < m - 1; ++k) {
      if (piv[k]) {
        const double t = y[k];
        y[k] = y[k + 1];
        y[k + 1] = t - l[k] * y[k];
      } else {
        y[k + 1] -= l[k] * y[k];
      }
    }
    // backward: U y = rhs
    for (int k = m - 1; k >= 0; --k) {
      double s = y[k];
      if (k + 1 < m) s -= du[k] * y[k + 1];
      if (k + 2 < m) s -= du2[k] * y[k + 2];
      y[k] = s / d[k];
    }
    double nrm = 0.0;
    for (int k = 0; k < m; ++k) nrm += y[k] * y[k];
    nrm = sqrt(nrm);
    if (!(nrm > 0.0)) {
      for (int k = 0; k < m; ++k) y[k] = k == 0 ? 1.0 : 0.0;
      break;
    }
    for (int k = 0; k < m; ++k) y[k] /= nrm;
  }
  st->sigma = sigma;
  for (int k = 0; k < kMaxSteps; ++k) st->y[k] = k < m ? y[k] : 0.0;
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

// r = X (X q) - sigma q, partial ||r||^2.
__global__ void resid_kernel(int n, int nb, const float2* P1, const float2* P2, int64_t ps, const double* q,
                             double* norms, const DevState* st) {
  __shared__ double sh[kVecThreads / 32];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double r = 0.0;
  if (e < n) r = reduce_partials(e, nb, P1, P2, ps) - st->sigma * q[e];
  const double t = block_sum64(r * r, sh);
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
  }
}

// X_0 = RN(X * (1/lam~)) into a full symmetric 16-bit matrix, from the upper
// triangle of X, in 32 x 32 tiles through shared memory.
template <int DT>
__global__ void scale_cast_kernel(const DevArgs* __restrict__ args, int n, const DevState* __restrict__ st,
                                  void* __restrict__ M, void* __restrict__ M_lo, int64_t ldm) {
  __shared__ float s[32][33];
  int bi, bj;
  tile_of(blockIdx.x, bi, bj);
  const int i0 = bi * 32, j0 = bj * 32;
  const float* __restrict__ X = args->X;
  const int64_t ld = args->ld;
  const float inv = static_cast<float>(st->inv_lambda);
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const bool diag = bi == bj;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int jj = ty + 8 * r;
    const int i = i0 + tx, j = j0 + jj;
    float v = 0.f;
    if (i < n && j < n && (!diag || tx <= jj)) v = X[static_cast<int64_t>(j) * ld + i] * inv;
    s[tx][jj] = v;
  }
  __syncthreads();
  if (diag) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int jj = ty + 8 * r;
      if (tx > jj) s[tx][jj] = s[jj][tx];
    }
    __syncthreads();
  }
  // store at (i + j ldm) and mirrored at (j + i ldm); both coalesced along tx
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int jj = ty + 8 * r;
    const int i = i0 + tx, j = j0 + jj;
    if (i < n && j < n) {
      const float v = s[tx][jj];
      const float w = s[jj][tx];
      if (DT == DT_TF32X3) {
        float* Mh = static_cast<float*>(M);
        float* Ml = static_cast<float*>(M_lo);
        // hi = v rounded to TF32 (10 explicit mantissa bits), lo = remainder rounded to TF32
        uint32_t b = __float_as_uint(v);
        uint32_t hb = (b + 0x1000u) & 0xFFFFE000u;
        float hi = __uint_as_float(hb);
        if (!isfinite(v)) hi = v;
        float rem = v - hi;
        uint32_t rb = (__float_as_uint(rem) + 0x1000u) & 0xFFFFE000u;
        Mh[static_cast<int64_t>(j) * ldm + i] = hi;
        Ml[static_cast<int64_t>(j) * ldm + i] = __uint_as_float(rb);
        (void)w;
      } else {
        uint16_t* H = static_cast<uint16_t*>(M);
        H[static_cast<int64_t>(j) * ldm + i] =
            DT == DT_BF16 ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : __half_as_ushort(__float2half_rn(v));
      }
    }
    const int i2 = i0 + jj, j2 = j0 + tx;  // mirrored position, coalesced along tx
    if (!diag && i2 < n && j2 < n) {
      const float v2 = s[jj][tx];
      if (DT == DT_TF32X3) {
        float* Mh = static_cast<float*>(M);
        float* Ml = static_cast<float*>(M_lo);
        uint32_t b = __float_as_uint(v2);
        float hi = __uint_as_float((b + 0x1000u) & 0xFFFFE000u);
        if (!isfinite(v2)) hi = v2;
        float rem = v2 - hi;
        Mh[static_cast<int64_t>(i2) * ldm + j2] = hi;
        Ml[static_cast<int64_t>(i2) * ldm + j2] = __uint_as_float((__float_as_uint(rem) + 0x1000u) & 0xFFFFE000u);
      } else {
        uint16_t* H = static_cast<uint16_t*>(M);
        H[static_cast<int64_t>(i2) * ldm + j2] =
            DT == DT_BF16 ? __bfloat16_as_ushort(__float2bfloat16_rn(v2)) : __half_as_ushort(__float2half_rn(v2));
      }
    }
  }
}

__global__ void set_args_kernel(DevArgs* d, DevArgs h) { *d = h; }

// Status word and overshoot of the last stage into the report.
__global__ void finalize_kernel(const DevArgs* args, DevState* st) {
  const float amax = __uint_as_float(st->absmax_bits);
  int status = st->status;
  if (status == 0) {
    if (!(amax == amax) || isinf(amax))
      status = PSD_ERR_NONFINITE;
    else if (amax > kOvershootLimit)
      status = PSD_ERR_BOUND;
    st->status = status;
  }
  psd_info_t* info = args->info;
  if (info) {
    info->overshoot_max = static_cast<double>(amax);
    info->status = status;
  }
}

}  // namespace

size_t lanczos_bytes(int64_t n) {
  const int64_t npad = (n + 255) / 256 * 256;
  const int64_t nb = (n + kSymvTile - 1) / kSymvTile;
  const int64_t ntiles = nb * (nb + 1) / 2;
  const int64_t nctas = (n + kVecThreads - 1) / kVecThreads;
  size_t b = 0;
  auto add = [&](size_t bytes) { b += (bytes + 255) / 256 * 256; };
  add(sizeof(double) * (kMaxSteps + 1) * npad);  // Qv
  add(sizeof(double) * npad * 3);                // u, w, q
  add(sizeof(float) * npad * 2);                 // vh, vl
  add(sizeof(float2) * nb * npad * 2);           // P1, P2
  add(sizeof(double) * nctas * 32 * 2);          // dots, dots2
  add(sizeof(double) * nctas);                   // norms
  add(sizeof(double) * ntiles);                  // tile_fro
  return b;
}

void lanczos_carve(LanczosBufs& L, int64_t n, uint8_t* base) {
  L.n = n;
  L.npad = (n + 255) / 256 * 256;
  L.nb = static_cast<int>((n + kSymvTile - 1) / kSymvTile);
  L.ntiles = L.nb * (L.nb + 1) / 2;
  L.nvec_ctas = static_cast<int>((n + kVecThreads - 1) / kVecThreads);
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
  double* d2 = reinterpret_cast<double*>(take(sizeof(double) * L.nvec_ctas * 32 * 2));
  L.dots = d2;
  L.dots2 = d2 + L.nvec_ctas * 32;
  L.norms = reinterpret_cast<double*>(take(sizeof(double) * L.nvec_ctas));
  L.tile_fro = reinterpret_cast<double*>(take(sizeof(double) * L.ntiles));
}

cudaError_t enqueue_norm_bound(const LanczosBufs& L, const DevArgs* args, DevState* st, cudaStream_t s) {
  const int n = static_cast<int>(L.n);
  const int vb = L.nvec_ctas, vt = kVecThreads;
  const int64_t ps = L.npad;
  lanczos_init_kernel<<<vb, vt, 0, s>>>(n, L.npad, L.Qv, L.vh, L.vl, st, L.norms);
  lanczos_norm0_kernel<<<vb, vt, 0, s>>>(n, L.Qv, L.vh, L.vl, L.norms, vb);
  for (int j = 0; j < kMaxSteps; ++j) {
    if (j == 0) {
      symv_upper_kernel<true><<<L.ntiles, 256, 0, s>>>(args, n, L.vh, L.vl, L.P1, L.P2, ps, L.tile_fro, st, 0);
      fro_kernel<<<1, 32, 0, s>>>(L.tile_fro, L.ntiles, st);
    } else
      symv_upper_kernel<false><<<L.ntiles, 256, 0, s>>>(args, n, L.vh, L.vl, L.P1, L.P2, ps, L.tile_fro, st, 1);
    reduce_split_kernel<<<vb, vt, 0, s>>>(n, L.nb, L.P1, L.P2, ps, L.u, L.vh, L.vl, st, 1);
    symv_upper_kernel<false><<<L.ntiles, 256, 0, s>>>(args, n, L.vh, L.vl, L.P1, L.P2, ps, L.tile_fro, st, 1);
    reduce_dots_kernel<<<vb, vt, 0, s>>>(n, L.nb, L.P1, L.P2, ps, L.w, L.Qv, L.npad, j, L.dots, st);
    orth_kernel<1><<<vb, vt, 0, s>>>(n, L.w, L.Qv, L.npad, j, L.dots, vb, L.dots2, st);
    orth_kernel<2><<<vb, vt, 0, s>>>(n, L.w, L.Qv, L.npad, j, L.dots2, vb, L.norms, st);
    lanczos_next_kernel<<<vb, vt, 0, s>>>(n, L.w, L.Qv, L.npad, j, L.norms, vb, L.vh, L.vl, st);
  }
  tridiag_kernel<<<1, 32, 0, s>>>(st);
  ritz_kernel<<<vb, vt, 0, s>>>(n, L.Qv, L.npad, L.q, L.norms, st);
  ritz_norm_kernel<<<vb, vt, 0, s>>>(n, L.q, L.norms, vb, L.vh, L.vl);
  symv_upper_kernel<false><<<L.ntiles, 256, 0, s>>>(args, n, L.vh, L.vl, L.P1, L.P2, ps, L.tile_fro, st, 0);
  reduce_split_kernel<<<vb, vt, 0, s>>>(n, L.nb, L.P1, L.P2, ps, L.u, L.vh, L.vl, st, 0);
  symv_upper_kernel<false><<<L.ntiles, 256, 0, s>>>(args, n, L.vh, L.vl, L.P1, L.P2, ps, L.tile_fro, st, 0);
  resid_kernel<<<vb, vt, 0, s>>>(n, L.nb, L.P1, L.P2, ps, L.q, L.norms, st);
  bound_final_kernel<<<1, 32, 0, s>>>(n, L.norms, vb, st, args);
  return cudaGetLastError();
}

cudaError_t enqueue_scale_cast(int dtype, const DevArgs* args, const DevState* st, int64_t n, void* M,
                               void* M_lo, int64_t ldm, cudaStream_t s) {
  const int nb = static_cast<int>((n + 31) / 32);
  const int tiles = nb * (nb + 1) / 2;
  dim3 blk(32, 8);
  if (dtype == DT_F16)
    scale_cast_kernel<DT_F16><<<tiles, blk, 0, s>>>(args, static_cast<int>(n), st, M, M_lo, ldm);
  else if (dtype == DT_BF16)
    scale_cast_kernel<DT_BF16><<<tiles, blk, 0, s>>>(args, static_cast<int>(n), st, M, M_lo, ldm);
  else
    scale_cast_kernel<DT_TF32X3><<<tiles, blk, 0, s>>>(args, static_cast<int>(n), st, M, M_lo, ldm);
  return cudaGetLastError();
}

cudaError_t enqueue_set_args(DevArgs* d_args, const DevArgs& h, cudaStream_t s) {
  set_args_kernel<<<1, 1, 0, s>>>(d_args, h);
  return cudaGetLastError();
}

cudaError_t enqueue_finalize(const DevArgs* args, DevState* st, cudaStream_t s) {
  finalize_kernel<<<1, 1, 0, s>>>(args, st);
  return cudaGetLastError();
}

}  // namespace psd
