// The stage sequence of Algorithm 2 shared by the single and the batched
// projection: which storage each matrix of a stage uses for a precision,
// workspace slots, and the order of the 3T + 1 products.
//
//   X_0 = RN(X / lam~)                                   (cast)
//   for t = 1..T:  Y = X_{t-1}^2;  P = a_t I + b_t Y + c_t Y^2;  X_t = X_{t-1} P / s_t
//   out = (X + lam~ X_0 X_T) / 2                          (final product)
//
// A path supplies the storage (Mat slots), the cast, the product launches and
// the report through an Ops object:
//   cudaError_t cast(const Mat& X0);
//   cudaError_t gemm(int epi, const Mat& A, const Mat& B, const Mat* out, const Mat* Y,
//                    float a, float b, float c, float s, bool track);   // track: max |X_T|
//   cudaError_t finish();
#pragma once

#include <algorithm>
#include <cmath>

#include "internal.h"

namespace psd {

// Storage of one matrix of the chain (workspace slots of n x ldm 16-bit elements).
enum MatKind : int {
  MK_16 = 0,      // one FP16 or BF16 matrix (Mat::dt16)
  MK_TF32X3 = 2,  // TF32 hi/lo pair in FP32 containers (4 slots)
  MK_E4M3 = 3,    // e4m3 values times Mat::scale (1 slot)
  MK_F16X2 = 4,   // FP16 hi/lo pair (2 slots)
};

struct Mat {
  int kind = MK_16;
  int slot = -1;
  int dt16 = DT_F16;  // element type of an MK_16 matrix
  float scale = 1.f;  // MK_E4M3: stored value = RN_e4m3(value * scale)
};

inline int kind_slots(int kind) {
  return kind == MK_TF32X3 ? 4 : kind == MK_F16X2 ? 2 : 1;
}
inline int kind_dtype(const Mat& m) {
  return m.kind == MK_16 ? m.dt16 : m.kind == MK_E4M3 ? DT_E4M3 : m.kind == MK_F16X2 ? DT_F16X2 : DT_TF32X3;
}
// Slot offset of the lo part of a pair.
inline int kind_lo_step(int kind) { return kind == MK_TF32X3 ? 2 : 1; }
inline bool kind_is_pair(int kind) { return kind == MK_TF32X3 || kind == MK_F16X2; }

// Mixed precision: P of the first kMixedPStages stages as an FP16 pair, and Y
// of stages kMixedYFirst .. kMixedYLast (0-based) too; X_t stays FP16.  The
// rounding model of the chain (CPU) shows the roundings of P and Y in the
// early stages carry the error, those of X_t do not, and stage 1's Y the
// least of them: without its pair the model's error grows from ~7e-4 to
// ~8-9e-4 on spread spectra (and not at all on dominated ones) for one
// pair x pair product less.  A stage with a single Y forms P from it with a
// pair output (4 tensor products instead of 6).
constexpr int kMixedPStages = 4;
constexpr int kMixedYFirst = 1, kMixedYLast = 2;
// FP8_LATE: the last kFp8Stages stages on e4m3 operands.  The first stages
// cannot be: their coefficients (a_1 = 8.29, b_1 = -22.6) amplify the e4m3
// rounding of X^2 (u = 2^-4) beyond the composite's basin.
constexpr int kFp8Stages = 2;
// Power-of-two scales of the e4m3 matrices: |X_t(i,j)|, |Y(i,j)| <= their
// spectral norms <= 1.25 (the filter keeps the spectrum near [-1, 1]), so
// 256 x 1.25 = 320 stays below the e4m3 maximum 448; P's scale comes from
// max |a + b y + c y^2| over y in [0, 1.25].
constexpr float kFp8ScaleX = 256.f;
constexpr float kFp8ScaleY = 256.f;

inline float fp8_poly_scale(const double (&c)[3]) {
  double m = 0.0;
  const double ys[3] = {0.0, 1.25, c[2] != 0.0 ? -c[1] / (2.0 * c[2]) : 0.0};
  for (double y : ys)
    if (y >= 0.0 && y <= 1.25) m = std::max(m, std::fabs(c[0] + c[1] * y + c[2] * y * y));
  double sc = 1.0;
  while (sc * 2.0 * m < 400.0) sc *= 2.0;
  while (sc > 1.0 / 1024 && sc * m >= 400.0) sc *= 0.5;
  return static_cast<float>(sc);
}

// Storage kinds of stage t (0-based) of T: the input iterate, Y, P, X_t.
struct StageKinds {
  int x, y, p, out;
};
inline StageKinds stage_kinds(psd_precision_t prec, int t, int T) {
  auto xk = [&](int s) {
    if (prec == PSD_PREC_FP32) return static_cast<int>(MK_TF32X3);
    if (prec == PSD_PREC_FP8_LATE && s >= T - kFp8Stages) return static_cast<int>(MK_E4M3);
    return static_cast<int>(MK_16);
  };
  StageKinds k{};
  k.x = xk(t);
  if (prec == PSD_PREC_MIXED && t < kMixedPStages) {
    k.y = (t >= kMixedYFirst && t <= kMixedYLast) ? MK_F16X2 : MK_16;
    k.p = MK_F16X2;
  } else {
    k.y = k.p = k.x;
  }
  k.out = prec == PSD_PREC_FP32 ? static_cast<int>(MK_TF32X3) : (t + 1 < T ? xk(t + 1) : static_cast<int>(MK_16));
  return k;
}

// First-fit allocator of workspace slots (contiguous runs for pairs).
struct SlotPool {
  uint32_t used = 0;
  int nslots = 0;
  int high = 0;  // slots touched so far
  int alloc(int k) {
    for (int s = 0; s + k <= nslots; ++s) {
      const uint32_t mask = ((1u << k) - 1u) << s;
      if ((used & mask) == 0) {
        used |= mask;
        high = std::max(high, s + k);
        return s;
      }
    }
    return -1;
  }
  void release(const Mat& m) { used &= ~(((1u << kind_slots(m.kind)) - 1u) << m.slot); }
};

template <class Ops>
cudaError_t run_chain(psd_precision_t prec, const Schedule& sched, int nslots, int dt16, Ops& ops,
                      int* high_water = nullptr) {
  cudaError_t e;
  SlotPool pool;
  pool.nslots = nslots;
  struct HighWater {
    SlotPool& pool;
    int* out;
    ~HighWater() {
      if (out) *out = pool.high;
    }
  } hw{pool, high_water};
  const int T = sched.T;
  auto make = [&](int kind, float scale) {
    Mat m;
    m.kind = kind;
    m.dt16 = dt16;
    m.scale = kind == MK_E4M3 ? scale : 1.f;
    m.slot = pool.alloc(kind_slots(kind));
    return m;
  };
  Mat X0 = make(stage_kinds(prec, 0, T).x, kFp8ScaleX);
  if (X0.slot < 0) return cudaErrorMemoryAllocation;
  if ((e = ops.cast(X0)) != cudaSuccess) return e;
  Mat cur = X0;
  for (int t = 0; t < T; ++t) {
    const StageKinds k = stage_kinds(prec, t, T);
    Mat Y = make(k.y, kFp8ScaleY);
    if (Y.slot < 0) return cudaErrorMemoryAllocation;
    if ((e = ops.gemm(EPI_COPY, cur, cur, &Y, nullptr, 0.f, 0.f, 0.f, 1.f, false)) != cudaSuccess) return e;
    Mat P = make(k.p, fp8_poly_scale(sched.coef[t]));
    if (P.slot < 0) return cudaErrorMemoryAllocation;
    if ((e = ops.gemm(EPI_POLY, Y, Y, &P, &Y, static_cast<float>(sched.coef[t][0]),
                      static_cast<float>(sched.coef[t][1]), static_cast<float>(sched.coef[t][2]), 1.f, false)) !=
        cudaSuccess)
      return e;
    pool.release(Y);
    Mat Xn = make(k.out, kFp8ScaleX);
    if (Xn.slot < 0) return cudaErrorMemoryAllocation;
    if ((e = ops.gemm(EPI_SCALE, cur, P, &Xn, nullptr, 0.f, 0.f, 0.f, static_cast<float>(1.0 / sched.post[t]),
                      t == T - 1)) != cudaSuccess)
      return e;
    pool.release(P);
    if (cur.slot != X0.slot) pool.release(cur);
    cur = Xn;
  }
  if ((e = ops.gemm(EPI_FINAL, X0, cur, nullptr, nullptr, 0.f, 0.f, 0.f, 1.f, false)) != cudaSuccess) return e;
  return ops.finish();
}

// Which kernel forms a product of the given operand kinds:
//   both MK_16 or both MK_E4M3: the 16-bit/e4m3 kernel (symgemm.cu);
//   both pairs of one type:      the split kernel (symgemm_x3.cu), three products;
//   MK_16 A with an MK_F16X2 B:  the split kernel's single-B instance with the
//                                operands exchanged (B A = A B: they commute),
//                                two products.
enum GemmRoute : int { ROUTE_16 = 0, ROUTE_X3 = 1, ROUTE_X2 = 2, ROUTE_NONE = 3 };
inline GemmRoute gemm_route(const Mat& A, const Mat& B) {
  if ((A.kind == MK_16 || A.kind == MK_E4M3) && A.kind == B.kind) return ROUTE_16;
  if (kind_is_pair(A.kind) && A.kind == B.kind) return ROUTE_X3;
  if (A.kind == MK_16 && A.dt16 == DT_F16 && B.kind == MK_F16X2) return ROUTE_X2;
  return ROUTE_NONE;
}

}  // namespace psd

namespace psd {

// Workspace slots the chain of a precision needs: its allocation sequence run
// without launching anything (pairs need contiguous slots, so this is more
// than the number of matrices alive at once).
struct ChainDryRun {
  cudaError_t cast(const Mat&) { return cudaSuccess; }
  cudaError_t gemm(int, const Mat&, const Mat&, const Mat*, const Mat*, float, float, float, float, bool) {
    return cudaSuccess;
  }
  cudaError_t finish() { return cudaSuccess; }
};
inline int chain_slots(psd_precision_t prec) {
  Schedule sched{};
  if (!get_schedule(prec, sched)) return 0;
  ChainDryRun dry;
  int high = 0;
  if (run_chain(prec, sched, 32, DT_F16, dry, &high) != cudaSuccess) return 0;
  return high;
}

}  // namespace psd
