// Largest eigenpair of the Lanczos tridiagonal T_m (diagonal alpha, off-diagonal
// beta, order m <= kMaxSteps), for the norm bound of Sec. 3.4 (Theorem 2 uses
// the largest Ritz pair of T_m).  One warp.
//
// GB300's FP64 pipe has a long dependent-operation latency (a 20-step Sturm
// recurrence costs ~18k cycles in FP64), so the search runs in FP32 on T
// scaled to unit size: multisection on the Sturm count (32 points per round,
// Gershgorin bracket), then inverse iteration with partial pivoting at the
// FP32 eigenvalue (Parlett, The Symmetric Eigenvalue Problem, Ch. 4).  The
// eigenvalue returned is the FP64 Rayleigh quotient y^T T y / y^T y of that
// vector, whose error is the square of the vector's (~1e-14 relative); the
// vector itself carries FP32 accuracy, which only loosens the residual term of
// the bound by ~1e-7 relative (the bound stays a bound: the residual is
// evaluated for the vector actually used).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace psd {

// Number of eigenvalues of the unit-scaled T below x: sign changes of the
// leading minors p_k = (a_k - x) p_{k-1} - b_{k-1}^2 p_{k-2} (no divisions;
// rescaled when they grow).
__device__ __forceinline__ int sturm_count32(const float* a, const float* b, int m, float x) {
  float pm = 1.f, p = a[0] - x;
  int cnt = (p < 0.f) ? 1 : 0;
  for (int k = 1; k < m; ++k) {
    const float pn = (a[k] - x) * p - b[k - 1] * b[k - 1] * pm;
    const bool change = (pn == 0.f) ? (p > 0.f) : ((pn < 0.f) != (p < 0.f));
    if (p != 0.f || pn != 0.f) cnt += change ? 1 : 0;
    pm = p;
    p = pn;
    if (fabsf(p) + fabsf(pm) > 1e18f) {
      p *= 1e-18f;
      pm *= 1e-18f;
    }
  }
  return cnt;
}

// Call with the 32 lanes of one warp.  a32, b32: shared scratch of kMaxSteps
// floats each; y: shared, kMaxSteps doubles (y[k] = 0 for k >= m on return).
// Returns the eigenvalue (every lane); y is valid after the call (every lane).
__device__ __forceinline__ double tridiag_top_eig(const double* alpha, const double* beta, int m, double* y,
                                                  float* a32, float* b32) {
  const int lane = threadIdx.x & 31;
  if (m < 1) {
    if (lane < kMaxSteps) y[lane] = 0.0;
    __syncwarp();
    return 0.0;
  }
  // unit scale: the largest Gershgorin radius bound |a_k| + |b_{k-1}| + |b_k|
  double g = 0.0;
  if (lane < m)
    g = fabs(alpha[lane]) + (lane > 0 ? fabs(beta[lane - 1]) : 0.0) + (lane < m - 1 ? fabs(beta[lane]) : 0.0);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g = fmax(g, __shfl_xor_sync(0xffffffffu, g, o));
  const double sc = (g > 0.0 && isfinite(g)) ? g : 1.0;
  const float inv = static_cast<float>(1.0 / sc);
  if (lane < m) {
    a32[lane] = static_cast<float>(alpha[lane]) * inv;
    b32[lane] = lane < m - 1 ? static_cast<float>(beta[lane]) * inv : 0.f;
  }
  __syncwarp();
  // Gershgorin bracket
  float lo = 0.f, hi = 0.f;
  if (lane < m) {
    const float r = (lane > 0 ? fabsf(b32[lane - 1]) : 0.f) + fabsf(b32[lane]);
    lo = a32[lane] - r;
    hi = a32[lane] + r;
  } else {
    lo = a32[0];
    hi = a32[0];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  // multisection for the top eigenvalue: the first of 32 points with all m eigenvalues below it
  for (int round = 0; round < 24; ++round) {
    if (!(hi - lo > 4.f * 1.2e-7f * fmaxf(fabsf(lo), fabsf(hi)))) break;
    const float w = (hi - lo) * (1.f / 33.f);
    const float x = lo + w * static_cast<float>(lane + 1);
    const unsigned mask = __ballot_sync(0xffffffffu, sturm_count32(a32, b32, m, x) >= m);
    const int first = mask ? __ffs(mask) - 1 : 32;
    const float nlo = first == 0 ? lo : lo + w * static_cast<float>(first);
    const float nhi = first == 32 ? hi : lo + w * static_cast<float>(first + 1);
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) {
    // inverse iteration on (T - s I): Gaussian elimination with partial
    // pivoting on the tridiagonal (a row swap adds a second super-diagonal)
    const float s = 0.5f * (lo + hi);
    const float tiny = 1e-30f;
    float d[kMaxSteps], du[kMaxSteps], du2[kMaxSteps], l[kMaxSteps], rd[kMaxSteps], v[kMaxSteps];
    bool piv[kMaxSteps];
    for (int k = 0; k < m; ++k) {
      d[k] = a32[k] - s;
      du[k] = k < m - 1 ? b32[k] : 0.f;
      du2[k] = 0.f;
      piv[k] = false;
    }
    for (int k = 0; k < m - 1; ++k) {
      const float dl = b32[k];
      if (fabsf(d[k]) >= fabsf(dl)) {
        if (d[k] == 0.f) d[k] = tiny;
        l[k] = dl / d[k];
        d[k + 1] -= l[k] * du[k];
      } else {
        piv[k] = true;
        l[k] = d[k] / dl;
        d[k] = dl;
        const float t = d[k + 1];
        d[k + 1] = du[k] - l[k] * t;
        du[k] = t;
        if (k < m - 2) {
          du2[k] = du[k + 1];
          du[k + 1] = -l[k] * du[k + 1];
        }
      }
    }
    if (m > 0 && d[m - 1] == 0.f) d[m - 1] = tiny;
    for (int k = 0; k < m; ++k) rd[k] = 1.f / d[k];
    for (int k = 0; k < m; ++k) v[k] = 1.f;
    for (int it = 0; it < 3; ++it) {
      for (int k = 0; k < m - 1; ++k) {
        if (piv[k]) {
          const float t = v[k];
          v[k] = v[k + 1];
          v[k + 1] = t - l[k] * v[k];
        } else {
          v[k + 1] -= l[k] * v[k];
        }
      }
      for (int k = m - 1; k >= 0; --k) {
        float acc = v[k];
        if (k + 1 < m) acc -= du[k] * v[k + 1];
        if (k + 2 < m) acc -= du2[k] * v[k + 2];
        v[k] = acc * rd[k];
      }
      float mx = 0.f;
      for (int k = 0; k < m; ++k) mx = fmaxf(mx, fabsf(v[k]));
      if (!(mx > 0.f) || !isfinite(mx)) {
        for (int k = 0; k < m; ++k) v[k] = k == 0 ? 1.f : 0.f;
        break;
      }
      const float r = 1.f / mx;  // max-norm scaling keeps the iterate in range
      for (int k = 0; k < m; ++k) v[k] *= r;
    }
    for (int k = 0; k < kMaxSteps; ++k) y[k] = k < m ? static_cast<double>(v[k]) : 0.0;
  }
  __syncwarp();
  // FP64 Rayleigh quotient and normalisation (lane-parallel, fixed order)
  double num = 0.0, den = 0.0;
  if (lane < m) {
    const double yk = y[lane];
    num = alpha[lane] * yk * yk + (lane < m - 1 ? 2.0 * beta[lane] * yk * y[lane + 1] : 0.0);
    den = yk * yk;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  const double rn = den > 0.0 ? 1.0 / sqrt(den) : 0.0;
  __syncwarp();
  if (lane < m) y[lane] *= rn;
  __syncwarp();
  return den > 0.0 ? num / den : alpha[0];
}

}  // namespace psd
