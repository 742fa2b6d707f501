// Deflation of the dominant eigenpairs before filtering: the remedy the paper
// names for its failure mode (a few dominant eigenvalues squeeze the rest of
// the spectrum into the region around 0 that the composite cannot resolve;
// Sec. 6, Limitations).  Not part of Algorithm 2.
//
//   1. The norm bound's Lanczos run on X^2 leaves an orthonormal basis
//      Q_m = [q_0 .. q_{m-1}] of the Krylov space K_m(X^2, q_0), which is rich
//      in the eigenvectors of X of largest |lambda|.
//   2. Rayleigh-Ritz with X on span(Q_m): Z = X Q_m (the first mat-vec of
//      each Lanczos step on X^2, kept), H = Q_m^T Z,
//      H = W diag(mu) W^T (cyclic Jacobi); Ritz pairs (mu_j, v_j = Q_m w_j),
//      residuals r_j = Z w_j - mu_j v_j.
//   3. Among the k_max pairs of largest |mu|, those with ||r_j|| <= kDeflateTol
//      lam~ are deflated: out = X - V diag(mu) V^T.
//   4. out <- the composite projection of out (the standard path, in place,
//      with its own norm bound lam~' of the deflated matrix).
//   5. out += V diag(max(mu, 0)) V^T.
// If span(V) is invariant under X, Pi(X) = V max(M, 0) V^T + Pi(X - V M V^T)
// exactly; the residual bound keeps the coupling below kDeflateTol lam~.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"

namespace psd {
namespace {

constexpr int kMaxDeflate = 16;
// ||X v - mu v|| / lam~ of a deflated pair.  The coupling the deflation drops
// is V E^T + E V^T with E = X V - V M, so the result moves by about
// 2 sqrt(k) kDeflateTol lam~ in the Frobenius norm (<= 8e-6 lam~ at k = 16):
// below the FP32 path's 1e-5 relative to ||Pi(X)||_F >= the largest positive
// eigenvalue.  A looser bound deflates more pairs but its coupling then
// dominates the FP32 error (1e-5: 7e-6 on a power-law spectrum of order 700,
// against 6e-7 at 1e-6).
constexpr double kDeflateTol = 1e-6;
constexpr int kM = kMaxSteps;         // Rayleigh-Ritz space at most kM vectors
constexpr int kThr = 256;

struct DeflPlan {
  int64_t n = 0;
  LanczosBufs L{};
  uint8_t* mem = nullptr;
  DevArgs* args = nullptr;
  DevState* st = nullptr;
  double* Z = nullptr;      // kM x npad: X q_a
  double* V = nullptr;      // kMaxDeflate x npad: Ritz vectors
  double* H = nullptr;      // kM x kM
  double* W = nullptr;      // kM x kM, column j = eigenvector j (sorted by |mu| desc)
  double* mu = nullptr;     // kM
  double* parts = nullptr;  // nctas x kMaxDeflate residual partial sums
  int* idx = nullptr;       // kMaxDeflate: rows of V deflated (packed)
  float* cmul = nullptr;    // kMaxDeflate: -mu of the deflated pairs
  float* cadd = nullptr;    // kMaxDeflate: max(mu, 0) of the deflated pairs
  int* kused = nullptr;
  int nctas = 0;
};

std::mutex g_dmu;
std::map<std::tuple<int, cudaStream_t, int64_t>, DeflPlan*> g_dplans;

size_t r256(size_t b) { return (b + 255) / 256 * 256; }

// Block-wide FP64 sum, fixed order (warp trees, then warp 0 over the warp sums).
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) t += sh[i];
  __syncthreads();
  return t;  // valid in thread 0
}

// H[a][b] = q_a . (X q_b), a, b < m.
__global__ void gram_kernel(int n, int64_t npad, const double* __restrict__ Q, const double* __restrict__ Z,
                            double* H, const DevState* st) {
  __shared__ double sh[kThr / 32];
  const int a = blockIdx.x / kM, b = blockIdx.x % kM;
  const int m = st->m;
  if (a >= m || b >= m) return;
  double s = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) s += Q[a * npad + e] * Z[b * npad + e];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) H[a * kM + b] = s;
}

// Symmetric 2 x 2 Schur rotation (Golub & Van Loan, Sec. 8.5): (c, s) with
// [c s; -s c]^T [app apq; apq aqq] [c s; -s c] diagonal.
__device__ void sym_schur2(double app, double apq, double aqq, double& c, double& s) {
  if (apq == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
  const double tau = (aqq - app) / (2.0 * apq);
  const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  c = 1.0 / sqrt(1.0 + t * t);
  s = t * c;
}

// Eigen-decomposition of the m x m Rayleigh quotient: parallel cyclic Jacobi
// with the round-robin ordering (Golub & Van Loan, Sec. 8.5.5): each of the
// M - 1 rounds of a sweep (M = m rounded up to even) rotates M / 2 disjoint
// index pairs at once.  Disjoint rotations leave each other's 2 x 2 blocks
// alone, so a round equals the same rotations applied one by one.  Thread
// (k, i) = (t % 32, t / 32) applies rotation i to row k (the column rotations,
// of A and of V), then to column k (the row rotations).  Eigenpairs sorted by
// |mu| descending.
constexpr int kRrThreads = 32 * (kM / 2);
__global__ void __launch_bounds__(kRrThreads) rr_kernel(const DevState* st, const double* H, double* W, double* mu) {
  __shared__ double A[kM][kM], V[kM][kM];
  __shared__ double cs[kM / 2][2];
  __shared__ int pq[kM / 2][2];
  __shared__ int converged;
  const int m = st->m, t = threadIdx.x, k = t & 31, i = t >> 5;
  const int M = m + (m & 1);
  for (int e = t; e < m * m; e += blockDim.x) {
    const int r = e / m, c = e % m;
    A[r][c] = 0.5 * (H[r * kM + c] + H[c * kM + r]);
    V[r][c] = r == c ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 40 && m > 1; ++sweep) {
    if (i == 0) {
      double off = 0.0, tot = 0.0;
      if (k < m)
        for (int j = 0; j < m; ++j) {
          const double v = A[k][j] * A[k][j];
          tot += v;
          if (j != k) off += v;
        }
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
      }
      if (k == 0) converged = !(off > 1e-30 * tot);  // also on NaN
    }
    __syncthreads();
    if (converged) break;
    for (int r = 0; r < M - 1; ++r) {
      if (t < M / 2) {  // pair t of round r (circle method, player M - 1 fixed)
        int p = t == 0 ? r : (r + t) % (M - 1);
        int q = t == 0 ? M - 1 : (r - t + M - 1) % (M - 1);
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
        double c = 1.0, sn = 0.0;
        if (q < m) sym_schur2(A[p][p], A[p][q], A[q][q], c, sn);
        pq[t][0] = p;
        pq[t][1] = q < m ? q : -1;  // the dummy player of an odd m
        cs[t][0] = c;
        cs[t][1] = sn;
      }
      __syncthreads();
      const bool act = k < m && i < M / 2 && pq[i][1] >= 0;
      const int p = act ? pq[i][0] : 0, q = act ? pq[i][1] : 0;
      const double c = act ? cs[i][0] : 1.0, sn = act ? cs[i][1] : 0.0;
      if (act) {  // columns p, q of row k
        const double akp = A[k][p], akq = A[k][q];
        A[k][p] = c * akp - sn * akq;
        A[k][q] = sn * akp + c * akq;
        const double vkp = V[k][p], vkq = V[k][q];
        V[k][p] = c * vkp - sn * vkq;
        V[k][q] = sn * vkp + c * vkq;
      }
      __syncthreads();
      if (act) {  // rows p, q of column k; the annihilated pair set to 0 exactly
        const double apk = A[p][k], aqk = A[q][k];
        A[p][k] = k == q ? 0.0 : c * apk - sn * aqk;
        A[q][k] = k == p ? 0.0 : sn * apk + c * aqk;
      }
      __syncthreads();
    }
  }
  if (t == 0) {
    int order[kM];
    for (int j = 0; j < m; ++j) order[j] = j;
    for (int x = 1; x < m; ++x) {  // insertion sort by |eigenvalue| descending
      const int o = order[x];
      int y = x;
      while (y > 0 && fabs(A[order[y - 1]][order[y - 1]]) < fabs(A[o][o])) {
        order[y] = order[y - 1];
        --y;
      }
      order[y] = o;
    }
    for (int j = 0; j < m; ++j) {
      mu[j] = A[order[j]][order[j]];
      for (int a = 0; a < m; ++a) W[a * kM + j] = V[a][order[j]];
    }
  }
}

// v_j = Q w_j, r_j = Z w_j - mu_j v_j for j < kmax (and < m); per-CTA partial
// sums of ||r_j||^2.
__global__ void ritz_kernel(int n, int64_t npad, const double* __restrict__ Q, const double* __restrict__ Z,
                            const double* __restrict__ W, const double* __restrict__ mu, int kmax,
                            const DevState* st, double* V, double* parts) {
  __shared__ double sh[kThr / 32][kMaxDeflate];
  const int m = st->m;
  const int k = min(kmax, m);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double r2[kMaxDeflate];
#pragma unroll
  for (int j = 0; j < kMaxDeflate; ++j) r2[j] = 0.0;
  if (e < n) {
    for (int j = 0; j < k; ++j) {
      double v = 0.0, xv = 0.0;
      for (int a = 0; a < m; ++a) {
        const double w = W[a * kM + j];
        v += Q[a * npad + e] * w;
        xv += Z[a * npad + e] * w;
      }
      V[j * npad + e] = v;
      const double r = xv - mu[j] * v;
      r2[j] = r * r;
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < kMaxDeflate; ++j) {
    double v = r2[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) sh[w][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < kMaxDeflate) {
    double t = 0.0;
    for (int i = 0; i < kThr / 32; ++i) t += sh[i][threadIdx.x];
    parts[blockIdx.x * kMaxDeflate + threadIdx.x] = t;
  }
}

// Which pairs to deflate: residual <= kDeflateTol lam~ (lam~ of X).  Writes
// the kept pairs packed: idx[l] (row of V), cmul[l] = -mu (the deflation),
// cadd[l] = max(mu, 0) (the add-back), l < *kused.
__global__ void select_kernel(const double* parts, int nctas, const double* mu, int kmax, const DevState* st,
                              int* idx, float* cmul, float* cadd, int* kused) {
  const int j = threadIdx.x;
  const int m = st->m;
  bool keep = false;
  double muj = 0.0;
  if (j < kMaxDeflate) {
    double r2 = 0.0;
    for (int c = 0; c < nctas; ++c) r2 += parts[c * kMaxDeflate + j];
    muj = j < m ? mu[j] : 0.0;
    keep = j < kmax && j < m && st->status == 0 && muj != 0.0 && sqrt(r2) <= kDeflateTol * st->lambda;
  }
  const unsigned b = __ballot_sync(0xffffffffu, keep);
  if (keep) {
    const int l = __popc(b & ((1u << j) - 1u));
    idx[l] = j;
    cmul[l] = static_cast<float>(-muj);
    cadd[l] = static_cast<float>(fmax(muj, 0.0));
  }
  if (j == 0) *kused = __popc(b);
}

// Upper tile index t -> (bi <= bj) of 64 x 64 tiles (FP32 estimate, exact integer correction).
__device__ void tile64(int t, int& bi, int& bj) {
  int j = static_cast<int>((sqrtf(8.f * static_cast<float>(t) + 1.f) - 1.f) * 0.5f);
  while ((j + 1) * (j + 2) / 2 <= t) ++j;
  while (j * (j + 1) / 2 > t) --j;
  bj = j;
  bi = t - j * (j + 1) / 2;
}

// out(i, j) = in(i, j) + sum_{l < k} coef_l v_l(i) v_l(j) over the whole
// matrix (k = *kused, v_l = row idx[l] of V), from the upper triangle of `in`
// (column-major, in[i + j ld_in], i <= j), written to both triangles of out.
// In place (in == out) is safe: a tile reads only its own upper part, before
// any write.  FP32 arithmetic: each entry's rounding is relative to the
// rank-k term, ~k 2^-24 |mu| |v_l(i) v_l(j)|, below the FP32 path's 1e-5.
__global__ void __launch_bounds__(256) rank_update_kernel(int n, const float* in, int64_t ld_in, float* out,
                                                          int64_t ld_out, const double* __restrict__ V,
                                                          int64_t npad, const int* __restrict__ idx,
                                                          const float* __restrict__ coef,
                                                          const int* __restrict__ kused) {
  __shared__ float s[64][65];
  __shared__ float vi[kMaxDeflate][64], vj[kMaxDeflate][64];
  int bi, bj;
  tile64(blockIdx.x, bi, bj);
  const int i0 = bi * 64, j0 = bj * 64;
  const bool diag = bi == bj;
  const int k = *kused;
  if (k == 0 && in == out && ld_in == ld_out) return;  // nothing to add, out already symmetric
  for (int q = threadIdx.x; q < k * 64; q += blockDim.x) {
    const int l = q / 64, r = q % 64;
    const double* v = V + static_cast<int64_t>(idx[l]) * npad;
    vi[l][r] = i0 + r < n ? static_cast<float>(coef[l] * v[i0 + r]) : 0.f;
    vj[l][r] = j0 + r < n ? static_cast<float>(v[j0 + r]) : 0.f;
  }
  // the upper part: element (i0 + r, j0 + cc), column-major, 64-float runs along r
  for (int q = threadIdx.x; q < 64 * 64; q += blockDim.x) {
    const int cc = q / 64, r = q % 64;
    const int i = i0 + r, j = j0 + cc;
    float x = 0.f;
    if (i < n && j < n && (!diag || r <= cc)) x = in[static_cast<int64_t>(j) * ld_in + i];
    s[r][cc] = x;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 64 * 64; q += blockDim.x) {
    const int cc = q / 64, r = q % 64;
    if (diag && r > cc) continue;
    float acc = s[r][cc];
    for (int l = 0; l < k; ++l) acc = fmaf(vi[l][r], vj[l][cc], acc);
    s[r][cc] = acc;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 64 * 64; q += blockDim.x) {
    const int cc = q / 64, r = q % 64;
    const int i = i0 + r, j = j0 + cc;
    if (i >= n || j >= n) continue;
    out[static_cast<int64_t>(j) * ld_out + i] = (diag && r > cc) ? s[cc][r] : s[r][cc];  // (i, j)
  }
  if (!diag)  // the mirror (j, i): runs along cc of the tile
    for (int q = threadIdx.x; q < 64 * 64; q += blockDim.x) {
      const int r = q / 64, cc = q % 64;
      const int i = i0 + r, j = j0 + cc;
      if (i < n && j < n) out[static_cast<int64_t>(i) * ld_out + j] = s[r][cc];
    }
}

void free_dplan(DeflPlan* p) {
  if (!p) return;
  if (p->mem) cudaFree(p->mem);
  delete p;
}

DeflPlan* get_dplan(int dev, cudaStream_t stream, int64_t n, psd_status_t* st) {
  auto key = std::make_tuple(dev, stream, n);
  auto it = g_dplans.find(key);
  if (it != g_dplans.end()) {
    *st = PSD_OK;
    return it->second;
  }
  DeflPlan* p = new DeflPlan();
  p->n = n;
  const int64_t npad = (n + 255) / 256 * 256;
  p->nctas = static_cast<int>((n + kThr - 1) / kThr);
  const size_t oz = 0;
  const size_t ov = oz + r256(sizeof(double) * kM * npad);
  const size_t oh = ov + r256(sizeof(double) * kMaxDeflate * npad);
  const size_t ow = oh + r256(sizeof(double) * kM * kM);
  const size_t om = ow + r256(sizeof(double) * kM * kM);
  const size_t op = om + r256(sizeof(double) * kM);
  const size_t oc = op + r256(sizeof(double) * p->nctas * kMaxDeflate);
  const size_t oa = oc + r256(sizeof(float) * kMaxDeflate);
  const size_t oi = oa + r256(sizeof(float) * kMaxDeflate);
  const size_t ok = oi + r256(sizeof(int) * kMaxDeflate);
  const size_t orec = ok + 256;
  const size_t ol = orec + 1024;
  const size_t total = ol + lanczos_bytes(n);
  if (cudaMalloc(&p->mem, total) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    *st = PSD_ERR_NO_MEMORY;
    return nullptr;
  }
  cudaMemset(p->mem, 0, total);
  uint8_t* b = p->mem;
  p->Z = reinterpret_cast<double*>(b + oz);
  p->V = reinterpret_cast<double*>(b + ov);
  p->H = reinterpret_cast<double*>(b + oh);
  p->W = reinterpret_cast<double*>(b + ow);
  p->mu = reinterpret_cast<double*>(b + om);
  p->parts = reinterpret_cast<double*>(b + op);
  p->cmul = reinterpret_cast<float*>(b + oc);
  p->cadd = reinterpret_cast<float*>(b + oa);
  p->idx = reinterpret_cast<int*>(b + oi);
  p->kused = reinterpret_cast<int*>(b + ok);
  p->args = reinterpret_cast<DevArgs*>(b + orec);
  p->st = reinterpret_cast<DevState*>(b + orec + 256);
  static_assert(sizeof(DevState) <= 768, "state record");
  lanczos_carve(p->L, n, b + ol);
  p->L.zsave = p->Z;  // the Lanczos run keeps Z = X Q_m
  g_dplans[key] = p;
  *st = PSD_OK;
  return p;
}

bool overlapping(const float* a, const float* b, int64_t n, int64_t lda, int64_t ldb) {
  const char* a0 = reinterpret_cast<const char*>(a);
  const char* a1 = reinterpret_cast<const char*>(a + (n - 1) * lda + n);
  const char* b0 = reinterpret_cast<const char*>(b);
  const char* b1 = reinterpret_cast<const char*>(b + (n - 1) * ldb + n);
  return a0 < b1 && b0 < a1;
}

}  // namespace

void release_deflate_plans() {
  std::lock_guard<std::mutex> lk(g_dmu);
  for (auto& kv : g_dplans) free_dplan(kv.second);
  g_dplans.clear();
}

}  // namespace psd

using namespace psd;

extern "C" psd_status_t psd_project_deflate(int64_t n, const float* X, int64_t ld, float* out, int64_t ld_out,
                                            psd_precision_t precision, int32_t kmax, psd_info_t* d_info,
                                            int32_t* d_kused, psd_stream_t stream) {
  if (n < 0 || n > kMaxOrder || kmax < 0 || kmax > kMaxDeflate) return PSD_ERR_INVALID_ARG;
  if (precision < PSD_PREC_FP32 || precision > PSD_PREC_FP8_LATE) return PSD_ERR_INVALID_ARG;
  if (n == 0) return PSD_OK;
  if (!X || !out || ld < n || ld_out < n) return PSD_ERR_INVALID_ARG;
  if (overlapping(X, out, n, ld, ld_out) && !(static_cast<const void*>(X) == out && ld == ld_out))
    return PSD_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (kmax == 0) {
    if (d_kused && cudaMemsetAsync(d_kused, 0, sizeof(int32_t), s) != cudaSuccess) return PSD_ERR_CUDA;
    return psd_project_ex(n, X, ld, out, ld_out, precision, d_info, nullptr, 0, stream);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PSD_ERR_CUDA;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return PSD_ERR_UNSUPPORTED;
  DeflPlan* p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_dmu);
    psd_status_t st = PSD_OK;
    p = get_dplan(dev, s, n, &st);
    if (!p) return st;
  }
  const int nt = static_cast<int>((n + 63) / 64);
  const int tiles = nt * (nt + 1) / 2;
  const int ni = static_cast<int>(n);
  const int64_t npad = p->L.npad;
  // 1-2: Lanczos on X^2 (the norm bound), Rayleigh-Ritz with X on its basis
  DevArgs h{X, ld, out, ld_out, nullptr};
  if (enqueue_set_args(p->args, h, s) != cudaSuccess) return PSD_ERR_CUDA;
  if (enqueue_norm_bound(p->L, p->args, p->st, s) != cudaSuccess) return PSD_ERR_CUDA;
  gram_kernel<<<kM * kM, kThr, 0, s>>>(ni, npad, p->L.Qv, p->Z, p->H, p->st);
  rr_kernel<<<1, kRrThreads, 0, s>>>(p->st, p->H, p->W, p->mu);
  ritz_kernel<<<p->nctas, kThr, 0, s>>>(ni, npad, p->L.Qv, p->Z, p->W, p->mu, kmax, p->st, p->V, p->parts);
  select_kernel<<<1, 32, 0, s>>>(p->parts, p->nctas, p->mu, kmax, p->st, p->idx, p->cmul, p->cadd, p->kused);
  // 3: out = X - V M V^T
  rank_update_kernel<<<tiles, 256, 0, s>>>(ni, X, ld, out, ld_out, p->V, npad, p->idx, p->cmul, p->kused);
  if (cudaGetLastError() != cudaSuccess) return PSD_ERR_CUDA;
  // 4: the composite projection of the deflated matrix, in place
  psd_status_t r = psd_project_ex(n, out, ld_out, out, ld_out, precision, d_info, nullptr, 0, stream);
  if (r != PSD_OK) return r;
  // 5: add back the positive part of the deflated pairs
  rank_update_kernel<<<tiles, 256, 0, s>>>(ni, out, ld_out, out, ld_out, p->V, npad, p->idx, p->cadd,
                                           p->kused);
  if (cudaGetLastError() != cudaSuccess) return PSD_ERR_CUDA;
  if (d_kused && cudaMemcpyAsync(d_kused, p->kused, sizeof(int32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return PSD_ERR_CUDA;
  return PSD_OK;
}
