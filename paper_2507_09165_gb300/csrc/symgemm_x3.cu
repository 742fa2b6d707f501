// Split-operand symmetric product: C = A B with each operand stored as a pair
// (hi, lo), hi = RN(v), lo = RN(v - hi), and the product formed on the tensor
// cores as A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated in one FP32 tensor
// memory accumulator (the lo * lo term is below the accumulation error).
//   TF32 pairs (kind::tf32): the FP32 path; three-term TF32 splitting as in
//     Ootomo & Yokota, "Recovering single precision accuracy from Tensor Cores
//     while surpassing the FP32 theoretical peak performance" (IJHPCA 2022).
//   FP16 pairs (kind::f16): about 22 significant bits (fewer where the lo part
//     is subnormal) at three FP16 products; the Y^2 product of the
//     mixed-precision chain's pair stages.
// A variant with a single B operand (B1) forms A_hi B + A_lo B: the P X (= X P,
// the two commute) product of those stages, where only P is a pair; its
// stages (no B_lo) are two thirds the size, so the ring has half again as many.
// Same symmetric tiling, warp roles and fused stage epilogues as the 16-bit
// kernel (symgemm.cu); the output is again a pair, or a single FP16 matrix,
// or the FP32 final result.
//
// Promoted accumulation (TF32 pairs): the tensor cores add into an FP32
// accumulator without rounding to nearest, so over the 3 n / 8 accumulation
// steps of a product the error grows like n.  TF32 products therefore
// accumulate K in chunks of kPromoteK elements in one tensor-memory buffer;
// after each chunk the epilogue warps add it to a running FP32 sum in a
// second buffer (round to nearest, chunks in order) and hand the chunk buffer
// back, so the accumulation error stays that of a kPromoteK-long sum at any n
// (the technique used for the low-precision accumulators of FP8 GEMMs).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "ptx.cuh"

namespace psd {

namespace {

constexpr int kBM = 128;
constexpr int kBN = 256;
constexpr int kThreads = 192;
constexpr int kSW = 33;                                 // staging row stride (words)
constexpr int kEpiWarpBytes = 2 * 32 * kSW * 4;         // values + Y chunk
constexpr int kTmemCols = 512;
constexpr int kPromoteK = 128;  // K elements per promoted chunk (TF32 pairs)

// Pipeline (x3_row_bytes): with a pair B, 4 stages of 48 KB (A_hi | A_lo |
// B_hi | B_lo) of 64-byte rows of K, 64-byte swizzle (3 stages in flight while
// the MMAs read the fourth: three times the lookahead of 2 stages of 128-byte
// rows in the same space); with a single B, 3 stages of 64 KB (A_hi | A_lo |
// B) of kRowBytesX3Single-byte rows (or 6 of 32 KB).
// PAIR (FP16 pairs): the product on SM pairs (tcgen05.mma.cta_group::2,
// M = 256, 256 x 256 tiles): each CTA stages its 128 rows of A_hi and A_lo and
// half of B's rows, so a stage holds 32 KB (pair B) or 48 KB (single B) and
// the ring 6 or 4 stages.
template <bool B1, bool PAIR = false>
struct X3Cfg {
  static constexpr int kRowBytes = B1 ? kRowBytesX3Single : 64;
  static constexpr bool kSW64 = kRowBytes == 64;
  static constexpr int kABytes = kBM * kRowBytes;
  static constexpr int kBBytes = (PAIR ? kBM : kBN) * kRowBytes;
  static constexpr int kStages = PAIR ? (B1 ? 4 : 6) : (B1 ? 3 : 2) * (128 / kRowBytes);
  static constexpr int kStageBytes = B1 ? 2 * kABytes + kBBytes : 2 * kABytes + 2 * kBBytes;
  static constexpr int smem() {
    return 1024 + kStages * kStageBytes + 4 * kEpiWarpBytes + 8 * (2 * kStages + 5) + 16;
  }
};
static_assert(X3Cfg<false>::smem() <= 232448 && X3Cfg<true>::smem() <= 232448 &&
                  X3Cfg<false, true>::smem() <= 232448 && X3Cfg<true, true>::smem() <= 232448,
              "shared memory per CTA");

__device__ __forceinline__ float tf32_rn(float v) {
  if (!isfinite(v)) return v;
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ float f16_rn(float v) { return __half2float(__float2half_rn(v)); }

// 4 consecutive elements of a staged column (col = true: S[t..t+3][j]) or row
// (S[t][j..j+3]) to global memory as FP32, BF16 or FP16, clipped at `valid`.
template <int KIND>  // 0 = FP32 words, 1 = BF16, 2 = FP16
__device__ __forceinline__ void store4(void* base, int64_t pos, const float (&v)[4], int valid, bool vec_ok) {
  if (KIND == 0) {
    float* d = static_cast<float*>(base) + pos;
    if (valid == 4 && vec_ok) {
      *reinterpret_cast<float4*>(d) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
      for (int e = 0; e < valid; ++e) d[e] = v[e];
    }
  } else {
    uint16_t u[4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
      u[e] = KIND == 1 ? __bfloat16_as_ushort(__float2bfloat16_rn(v[e])) : __half_as_ushort(__float2half_rn(v[e]));
    uint16_t* d = static_cast<uint16_t*>(base) + pos;
    if (valid == 4 && vec_ok) {
      *reinterpret_cast<uint2*>(d) = make_uint2(u[0] | (static_cast<uint32_t>(u[1]) << 16),
                                                u[2] | (static_cast<uint32_t>(u[3]) << 16));
    } else {
      for (int e = 0; e < valid; ++e) d[e] = u[e];
    }
  }
}

// Writes the staged 32 x 32 chunk S (S[t][j] = value at (r0 + t, c0 + j)) to
// positions (r, c) -- memory rows c0 + j -- and, unless diagonal, (c, r) --
// memory rows r0 + t.  Lane l handles 4 consecutive elements of memory row
// l / 8 + 4 i.  Vector stores only when the row stride and base allow them
// (the caller's FP32 output may have any leading dimension).
template <int KIND>
__device__ __forceinline__ void store_chunk(void* C, int64_t ldc, int n, int r0, int c0, bool diag,
                                            const float* S, int lane) {
  const int q = lane & 7;
  const int64_t esz = KIND == 0 ? 4 : 2;
  const bool vec_ok = ((ldc * esz) % (4 * esz)) == 0 && (reinterpret_cast<uintptr_t>(C) % (4 * esz)) == 0;
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const int jj = (lane >> 3) + 4 * it;
    const int c = c0 + jj, rs = r0 + 4 * q;
    if (c < n && rs < n) {
      const float v[4] = {S[(4 * q) * kSW + jj], S[(4 * q + 1) * kSW + jj], S[(4 * q + 2) * kSW + jj],
                          S[(4 * q + 3) * kSW + jj]};
      store4<KIND>(C, static_cast<int64_t>(c) * ldc + rs, v, min(4, n - rs), vec_ok);
    }
  }
  if (!diag) {
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const int tt = (lane >> 3) + 4 * it;
      const int r = r0 + tt, cs = c0 + 4 * q;
      if (r < n && cs < n) {
        const float v[4] = {S[tt * kSW + 4 * q], S[tt * kSW + 4 * q + 1], S[tt * kSW + 4 * q + 2],
                            S[tt * kSW + 4 * q + 3]};
        store4<KIND>(C, static_cast<int64_t>(r) * ldc + cs, v, min(4, n - cs), vec_ok);
      }
    }
  }
}

// The Y chunk (r0..r0+31) x (c0..c0+31) of a symmetric pair, value hi + lo
// (FP32 sum of the two parts), into YB[j * kSW + t] = Y(r0 + t, c0 + j); zeros
// outside n.  Read as memory rows c0 + j with 16-byte loads, all of a lane's
// loads issued before any is used (the epilogue of the polynomial stage is
// otherwise bound by the latency of 2-byte loads).  The caller synchronises
// the warp before YB is read.
template <int ET>
__device__ __forceinline__ void load_y_pair_chunk(const void* Yh, const void* Yl, int64_t ldy, int n, int r0, int c0,
                                                  int lane, float* YB) {
  if constexpr (ET == DT_TF32X3) {
    const int q = lane & 7;  // rows r0 + 4 q .. + 3
    const int r = r0 + 4 * q;
    float4 h[8], l[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int c = c0 + (lane >> 3) + 4 * k;
      h[k] = l[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (c < n && r < n) {
        const int64_t idx = static_cast<int64_t>(c) * ldy + r;
        const float* ph = static_cast<const float*>(Yh) + idx;
        const float* pl = static_cast<const float*>(Yl) + idx;
        if (r + 3 < n && ((reinterpret_cast<uintptr_t>(ph) | reinterpret_cast<uintptr_t>(pl)) & 15) == 0) {
          h[k] = __ldg(reinterpret_cast<const float4*>(ph));
          l[k] = __ldg(reinterpret_cast<const float4*>(pl));
        } else {
          float th[4] = {0.f, 0.f, 0.f, 0.f}, tl[4] = {0.f, 0.f, 0.f, 0.f};
          for (int e = 0; e < 4 && r + e < n; ++e) {  // the edge at n, or an unaligned caller buffer
            th[e] = ph[e];
            tl[e] = pl[e];
          }
          h[k] = make_float4(th[0], th[1], th[2], th[3]);
          l[k] = make_float4(tl[0], tl[1], tl[2], tl[3]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      float* d = YB + ((lane >> 3) + 4 * k) * kSW + 4 * q;
      d[0] = h[k].x + l[k].x;
      d[1] = h[k].y + l[k].y;
      d[2] = h[k].z + l[k].z;
      d[3] = h[k].w + l[k].w;
    }
  } else {
    const int q = lane & 3;  // rows r0 + 8 q .. + 7
    const int r = r0 + 8 * q;
    uint4 h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int c = c0 + (lane >> 2) + 8 * k;
      h[k] = l[k] = make_uint4(0u, 0u, 0u, 0u);
      if (c < n && r < n) {
        const int64_t idx = static_cast<int64_t>(c) * ldy + r;
        const uint16_t* ph = static_cast<const uint16_t*>(Yh) + idx;
        const uint16_t* pl = static_cast<const uint16_t*>(Yl) + idx;
        if (r + 7 < n && ((reinterpret_cast<uintptr_t>(ph) | reinterpret_cast<uintptr_t>(pl)) & 15) == 0) {
          h[k] = __ldg(reinterpret_cast<const uint4*>(ph));
          l[k] = __ldg(reinterpret_cast<const uint4*>(pl));
        } else {
          uint32_t th[4] = {0u, 0u, 0u, 0u}, tl[4] = {0u, 0u, 0u, 0u};
          for (int e = 0; e < 8 && r + e < n; ++e) {  // the edge at n, or an unaligned caller buffer
            th[e >> 1] |= static_cast<uint32_t>(ph[e]) << (16 * (e & 1));
            tl[e >> 1] |= static_cast<uint32_t>(pl[e]) << (16 * (e & 1));
          }
          h[k] = make_uint4(th[0], th[1], th[2], th[3]);
          l[k] = make_uint4(tl[0], tl[1], tl[2], tl[3]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float* d = YB + ((lane >> 2) + 8 * k) * kSW + 8 * q;
      const uint32_t wh[4] = {h[k].x, h[k].y, h[k].z, h[k].w};
      const uint32_t wl[4] = {l[k].x, l[k].y, l[k].z, l[k].w};
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const uint16_t uh = static_cast<uint16_t>(wh[e >> 1] >> (16 * (e & 1)));
        const uint16_t ul = static_cast<uint16_t>(wl[e >> 1] >> (16 * (e & 1)));
        d[e] = __half2float(__ushort_as_half(uh)) + __half2float(__ushort_as_half(ul));
      }
    }
  }
}

// OUT: 0 = split pair of the operand kind, 1 = single FP16, 2 = FP32 final output.
template <int ET, int EPI, int OUT>
__device__ __forceinline__ void epilogue_chunk_x3(const GemmParams& p, const BlockRec& br, int r0, int c0,
                                                  const uint32_t (&v)[32], float* S, float* YB, int lane, float lam,
                                                  bool track, unsigned& amax_bits, ComplAcc* cacc_out = nullptr) {
  constexpr bool TF32 = ET == DT_TF32X3;
  const int n = br.n;
  const int64_t off = br.off;
  const bool pb = p.ep.per_block_coef != 0;
  const float ca = pb ? br.ca : p.ep.a, cb = pb ? br.cb : p.ep.b, cc = pb ? br.cc : p.ep.c;
  const float cs = pb ? br.cs : p.ep.s;
  const int64_t esz = OUT == 1 ? 2 : (TF32 ? 4 : 2);  // element size of the iterate output
  void* C = static_cast<uint8_t*>(p.ep.C) + (off + br.dc) * p.ep.ldc * esz;
  void* C_lo = p.ep.C_lo ? static_cast<uint8_t*>(p.ep.C_lo) + (off + br.dc) * p.ep.ldc * esz : nullptr;
  const int64_t ysz = TF32 ? 4 : 2;
  const void* Yh = p.ep.Y ? static_cast<const uint8_t*>(p.ep.Y) + (off + br.dy) * p.ep.ldy * ysz : nullptr;
  const void* Yl = p.ep.Y_lo ? static_cast<const uint8_t*>(p.ep.Y_lo) + (off + br.dy) * p.ep.ldy * ysz : nullptr;
  const int r = r0 + lane;
  const bool diag = (r0 == c0);
  const bool row_ok = r < n;
  float o[32];
  if (EPI == EPI_POLY) {
    load_y_pair_chunk<ET>(Yh, Yl, p.ep.ldy, n, r0, c0, lane, YB);
    __syncwarp();
  }
  const float* X = nullptr;
  int64_t ldx = 0;
  if (EPI == EPI_FINAL) {
    X = br.X;
    ldx = br.ld;
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const float acc = __uint_as_float(v[j]);
    float val;
    if (EPI == EPI_POLY) {
      val = fmaf(cc, acc, cb * YB[j * kSW + lane]);
      if (diag && j == lane) val += ca;
    } else if (EPI == EPI_SCALE) {
      val = acc * cs;
    } else if (EPI == EPI_FINAL) {
      const int c = c0 + j;
      float x = 0.f;
      const bool upper = !diag || j >= lane;
      if (row_ok && c < n && upper) x = X[static_cast<int64_t>(c) * ldx + r];
      val = 0.5f * fmaf(lam, acc, x);
      if (cacc_out && row_ok && c < n && upper) compl_add(*cacc_out, val, x, c == r ? 1.f : 2.f);
    } else {
      val = acc;
    }
    o[j] = val;
  }
  // symmetrise diagonal chunks from their upper part (values before splitting)
#pragma unroll
  for (int j = 0; j < 32; ++j) S[lane * kSW + j] = o[j];
  __syncwarp();
  if (diag) {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < lane) o[j] = S[j * kSW + lane];
    __syncwarp();
  }
  if constexpr (OUT == 2) {
    if (diag) {
#pragma unroll
      for (int j = 0; j < 32; ++j) S[lane * kSW + j] = o[j];
      __syncwarp();
    }
    store_chunk<0>(br.out, br.ld_out, n, r0, c0, diag, S, lane);
    __syncwarp();
  } else if constexpr (OUT == 1) {
    if (track && row_ok) {
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + j < n) amax_bits = max(amax_bits, __float_as_uint(fabsf(__half2float(__float2half_rn(o[j])))));
    }
    if (diag) {
#pragma unroll
      for (int j = 0; j < 32; ++j) S[lane * kSW + j] = o[j];
      __syncwarp();
    }
    store_chunk<2>(C, p.ep.ldc, n, r0, c0, diag, S, lane);
    __syncwarp();
  } else {
  // split pair: hi first, then lo, through the same staging buffer
  float lo[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const float hi = TF32 ? tf32_rn(o[j]) : f16_rn(o[j]);
    lo[j] = TF32 ? tf32_rn(o[j] - hi) : f16_rn(o[j] - hi);
    o[j] = hi;
  }
  if (track && row_ok) {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (c0 + j < n) amax_bits = max(amax_bits, __float_as_uint(fabsf(o[j] + lo[j])));
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) S[lane * kSW + j] = o[j];
  __syncwarp();
  store_chunk<TF32 ? 0 : 2>(C, p.ep.ldc, n, r0, c0, diag, S, lane);
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32; ++j) S[lane * kSW + j] = lo[j];
  __syncwarp();
  store_chunk<TF32 ? 0 : 2>(C_lo, p.ep.ldc, n, r0, c0, diag, S, lane);
  __syncwarp();
  }
}

// A wait that has given up in the pair form leaves copies of this CTA in
// flight, which signal the leader's barrier: they are given this long to land.
constexpr unsigned long long kPairDrainNs = 200000ull;

template <int ET, int EPI, int OUT, bool B1, bool PAIR = false>
__global__ void __launch_bounds__(kThreads, 1)
    symgemm_x3_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                      const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                      const GemmParams p) {
  static_assert(!PAIR || (ET == DT_F16X2 && EPI != EPI_FINAL), "pair form: FP16 pairs, stage products");
  constexpr int kStages = X3Cfg<B1, PAIR>::kStages;
  constexpr int kStageBytes = X3Cfg<B1, PAIR>::kStageBytes;
  constexpr int kABytes = X3Cfg<B1, PAIR>::kABytes;
  constexpr int kBBytes = X3Cfg<B1, PAIR>::kBBytes;
  constexpr bool kSW64 = X3Cfg<B1, PAIR>::kSW64;
  auto desc = [](uint32_t a) { return kSW64 ? sw64_kmajor_desc(a) : sw128_kmajor_desc(a); };
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* stages = smem;
  uint8_t* epi = smem + kStages * kStageBytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(epi + 4 * kEpiWarpBytes);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // pair form: CTA rank in its cluster of two; tiles are dealt to clusters
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
  const bool leader = rank == 0;
  const int cl = PAIR ? static_cast<int>(blockIdx.x >> 1) : static_cast<int>(blockIdx.x);
  const int ncl = PAIR ? static_cast<int>(gridDim.x >> 1) : static_cast<int>(gridDim.x);
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + kStages + s); };
  auto tfull_bar = [&](int a) { return smem_u32(bars + 2 * kStages + a); };
  auto tempty_bar = [&](int a) { return smem_u32(bars + 2 * kStages + 2 + a); };
  const uint32_t drain_bar = smem_u32(bars + 2 * kStages + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), PAIR ? 8 : 4);  // pair: the leader's, 4 epilogue warps of each CTA
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_desc(&tmAh);
    tma_prefetch_desc(&tmAl);
    tma_prefetch_desc(&tmBh);
    if (!B1) tma_prefetch_desc(&tmBl);
  }
  if (warp == 1) {
    if (PAIR) {
      tmem_alloc_pair(smem_u32(tmem_holder), kTmemCols);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(smem_u32(tmem_holder), kTmemCols);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  if (PAIR)
    cluster_sync_all();  // both CTAs' barriers initialised before any arrival crosses the pair
  else
    __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;
  constexpr bool TF32 = ET == DT_TF32X3;
  constexpr int kKElems = X3Cfg<B1>::kRowBytes / (TF32 ? 4 : 2);  // K elements per stage
  constexpr int kKStep = TF32 ? 8 : 16;    // K per MMA instruction (32 bytes)
  constexpr bool kPromote = TF32;

  if (warp == 0) {
    if (lane == 0) {
      int last_parity[kStages];
      for (int s = 0; s < kStages; ++s) last_parity[s] = -1;
      uint32_t s = 0, ph = 0;
      bool ok = true;
      for (TileStream ts(p, cl, ncl); ok && ts.valid(); ts.advance()) {
        ts.prefetch();
        const TileMeta& m = ts.cur();
        const int4 tc = m.tc;
        const int kbn = (m.n + kKElems - 1) / kKElems;
        // pair form: this CTA's 128 rows of A and its N/2 rows of B
        const int ya = static_cast<int>(m.off + tc.x + 128 * static_cast<int>(rank));
        const int yb = static_cast<int>(m.off + m.db + tc.y + (tc.w >> 1) * static_cast<int>(rank));
        for (int kb = 0; kb < kbn; ++kb) {
          if (!wait_bounded(empty_bar(s), ph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          const uint32_t base = smem_u32(stages + s * kStageBytes);
          if (PAIR) {
            if (leader) mbar_arrive_expect_tx(full_bar(s), 2 * kStageBytes);  // both CTAs' copies
            const uint32_t fb = mapa_shared(full_bar(s), 0);
            tma_load_2d_pair(base, &tmAh, kb * kKElems, ya, fb);
            tma_load_2d_pair(base + kABytes, &tmAl, kb * kKElems, ya, fb);
            tma_load_2d_pair(base + 2 * kABytes, &tmBh, kb * kKElems, yb, fb);
            if (!B1) tma_load_2d_pair(base + 2 * kABytes + kBBytes, &tmBl, kb * kKElems, yb, fb);
          } else {
            mbar_arrive_expect_tx(full_bar(s), kStageBytes);
            tma_load_2d(base, &tmAh, kb * kKElems, ya, full_bar(s));
            tma_load_2d(base + kABytes, &tmAl, kb * kKElems, ya, full_bar(s));
            tma_load_2d(base + 2 * kABytes, &tmBh, kb * kKElems, yb, full_bar(s));
            if (!B1) tma_load_2d(base + 2 * kABytes + kBBytes, &tmBl, kb * kKElems, yb, full_bar(s));
          }
          last_parity[s] = static_cast<int>(ph);
          if (++s == kStages) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      if (!ok && PAIR) {
        // the copies in flight signal the leader's barrier: give them time to land
        bool any = false;
        for (int q = 0; q < kStages; ++q) any = any || last_parity[q] >= 0;
        const unsigned long long t0 = globaltimer_ns();
        while (any && globaltimer_ns() - t0 < kPairDrainNs) {
        }
      } else if (!ok) {
        for (int q = 0; q < kStages; ++q)
          if (last_parity[q] >= 0) {
            const unsigned long long t0 = globaltimer_ns();
            while (!mbar_try_wait(full_bar(q), static_cast<uint32_t>(last_parity[q])) &&
                   globaltimer_ns() - t0 < kWaitLimitNs) {
            }
          }
      }
    }
  } else if (warp == 1 && kPromote) {
    // chunk buffer at column 0 (tfull/tempty[0]); the running sum (column kBN)
    // belongs to the epilogue warps
    uint32_t s = 0, ph = 0, cph = 0;
    bool ok = true;
    constexpr int kChunkBlocks = kPromoteK / kKElems;
    for (TileStream ts(p, cl, ncl); ok && ts.valid(); ts.advance()) {
      ts.prefetch();
      const int4 tc = ts.cur().tc;
      const int kbn = (ts.cur().n + kKElems - 1) / kKElems;
      const uint32_t idesc = p.idesc | (static_cast<uint32_t>(tc.w >> 3) << 17);  // N = tile width
      for (int kc = 0; ok && kc < kbn; kc += kChunkBlocks) {
        if (!wait_bounded(tempty_bar(0), cph ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int kend = min(kbn, kc + kChunkBlocks);
        for (int kb = kc; kb < kend; ++kb) {
          if (!wait_bounded(full_bar(s), ph, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          if (lane == 0) {
            const uint32_t ah = smem_u32(stages + s * kStageBytes);
            const uint32_t al = ah + kABytes, bh = ah + 2 * kABytes, bl = bh + kBBytes;
#pragma unroll
            for (int k = 0; k < kKElems / kKStep; ++k) {
              const uint32_t off = 32 * k;
              const uint32_t first = ((kb - kc) | k) == 0 ? 0u : 1u;
              mma_tf32(tmem_base, desc(ah + off), desc(bh + off), idesc, first);
              mma_tf32(tmem_base, desc(ah + off), desc(bl + off), idesc, 1u);
              mma_tf32(tmem_base, desc(al + off), desc(bh + off), idesc, 1u);
            }
            mma_commit(empty_bar(s));
          }
          __syncwarp();
          if (++s == kStages) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
        if (lane == 0) mma_commit(tfull_bar(0));
        __syncwarp();
        cph ^= 1u;
      }
    }
    if (!ok && lane == 0) {
      mma_commit(drain_bar);
      const unsigned long long t0 = globaltimer_ns();
      while (!mbar_try_wait(drain_bar, 0) && globaltimer_ns() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
  } else if (warp == 1 && (!PAIR || leader)) {  // pair form: the leader issues for both CTAs
    uint32_t s = 0, ph = 0, acc = 0, acc_ph = 0;
    bool ok = true;
    for (TileStream ts(p, cl, ncl); ok && ts.valid(); ts.advance()) {
      ts.prefetch();
      const int4 tc = ts.cur().tc;
      const int kbn = (ts.cur().n + kKElems - 1) / kKElems;
      const uint32_t idesc = p.idesc | (static_cast<uint32_t>(tc.w >> 3) << 17);  // N = tile width
      if (!wait_bounded(tempty_bar(acc), acc_ph ^ 1u, abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + acc * kBN;
      for (int kb = 0; kb < kbn; ++kb) {
        if (!wait_bounded(full_bar(s), ph, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (lane == 0) {
          const uint32_t ah = smem_u32(stages + s * kStageBytes);
          const uint32_t al = ah + kABytes, bh = ah + 2 * kABytes, bl = bh + kBBytes;
#pragma unroll
          for (int k = 0; k < kKElems / kKStep; ++k) {
            const uint32_t off = 32 * k;
            const uint32_t first = (kb | k) == 0 ? 0u : 1u;
            if (TF32) {
              mma_tf32(d_tmem, desc(ah + off), desc(bh + off), idesc, first);
              mma_tf32(d_tmem, desc(ah + off), desc(bl + off), idesc, 1u);
              mma_tf32(d_tmem, desc(al + off), desc(bh + off), idesc, 1u);
            } else if (PAIR) {
              mma_f16_pair(d_tmem, desc(ah + off), desc(bh + off), idesc, first);
              if (!B1) mma_f16_pair(d_tmem, desc(ah + off), desc(bl + off), idesc, 1u);
              mma_f16_pair(d_tmem, desc(al + off), desc(bh + off), idesc, 1u);
            } else {
              mma_f16(d_tmem, desc(ah + off), desc(bh + off), idesc, first);
              if (!B1) mma_f16(d_tmem, desc(ah + off), desc(bl + off), idesc, 1u);
              mma_f16(d_tmem, desc(al + off), desc(bh + off), idesc, 1u);
            }
          }
          if (PAIR)
            mma_commit_pair(empty_bar(s), 3);  // frees the stage in both CTAs
          else
            mma_commit(empty_bar(s));
        }
        __syncwarp();
        if (++s == kStages) {
          s = 0;
          ph ^= 1u;
        }
      }
      if (!ok) break;
      if (lane == 0) {
        if (PAIR)
          mma_commit_pair(tfull_bar(acc), 3);
        else
          mma_commit(tfull_bar(acc));
      }
      __syncwarp();
      acc ^= 1u;
      if (acc == 0) acc_ph ^= 1u;
    }
    if (!ok && lane == 0) {
      // the MMAs already issued, before tensor memory is released
      if (PAIR)
        mma_commit_pair(drain_bar, 1);
      else
        mma_commit(drain_bar);
      const unsigned long long t0 = globaltimer_ns();
      while (!mbar_try_wait(drain_bar, 0) && globaltimer_ns() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // pair form, peer CTA: the leader's MMA warp issues for both
  } else {
    const int ew = warp & 3;
    float* S = reinterpret_cast<float*>(epi + ew * kEpiWarpBytes);
    float* YB = S + 32 * kSW;
    uint32_t acc = 0, acc_ph = 0;
    unsigned amax_bits = 0;
    int amax_block = -1;
    const bool track_launch = p.ep.absmax_blocks != 0 || p.ep.absmax != nullptr;
    auto flush_amax = [&](int blk) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) amax_bits = max(amax_bits, __shfl_xor_sync(0xffffffffu, amax_bits, o));
      if (lane == 0 && amax_bits) {
        unsigned* dst = p.ep.absmax ? p.ep.absmax : &p.blocks[blk].st->absmax_bits;
        atomicMax(dst, amax_bits);
      }
      amax_bits = 0;
    };
    // pair form: the peer releases an accumulator through the leader's barrier
    const uint32_t tempty_leader[2] = {PAIR ? mapa_shared(tempty_bar(0), 0) : 0u,
                                       PAIR ? mapa_shared(tempty_bar(1), 0) : 0u};
    for (int t = cl; t < p.num_tiles; t += ncl) {
      const int4 tc = p.tiles[t];
      const BlockRec& br = p.blocks[tc.z];
      const int n = br.n;
      const bool track = track_launch && (p.ep.absmax_blocks != 2 || br.track != 0);
      if (track_launch && amax_block != tc.z) {
        if (amax_block >= 0) flush_amax(amax_block);
        amax_block = tc.z;
      }
      const float lam = EPI == EPI_FINAL ? static_cast<float>(br.st->lambda) : 0.f;
      const int r0 = tc.x + 128 * static_cast<int>(rank) + 32 * ew;
      const int ch_begin = max(0, (r0 - tc.y) >> 5);
      const int ch_end = r0 < n ? min((tc.w + 31) >> 5, (n - tc.y + 31) >> 5) : ch_begin;
      const uint32_t lanes = static_cast<uint32_t>(32 * ew) << 16;
      if constexpr (kPromote) {
        // fold every chunk into the running sum (column kBN), in K order
        const int kbn = (n + kKElems - 1) / kKElems;
        constexpr int kChunkBlocks = kPromoteK / kKElems;
        bool ok = true;
        for (int kc = 0; kc < kbn; kc += kChunkBlocks) {
          if (!wait_bounded(tfull_bar(0), acc_ph, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          // one load round trip per 32 columns: chunk and sum loads issued
          // together, stores left in flight until the end of the fold
#pragma unroll 1
          for (int ch = ch_begin; ch < ch_end; ++ch) {
            uint32_t v[32], w[32];
            tmem_ld32_async(tmem_base + lanes + 32 * ch, v);
            if (kc > 0) {
              tmem_ld32_async(tmem_base + lanes + kBN + 32 * ch, w);
            } else {
#pragma unroll
              for (int j = 0; j < 32; ++j) w[j] = 0u;  // +0.0f: the first chunk is stored as it is
            }
            tmem_wait_ld2(v, w);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = __float_as_uint(__uint_as_float(w[j]) + __uint_as_float(v[j]));
            tmem_st32_async(tmem_base + lanes + kBN + 32 * ch, v);
          }
          tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tempty_bar(0));
          acc_ph ^= 1u;
        }
        if (!ok) break;
        ComplAcc cacc;
        ComplAcc* cap = (EPI == EPI_FINAL && p.ep.cres) ? &cacc : nullptr;
#pragma unroll 1
        for (int ch = ch_begin; ch < ch_end; ++ch) {
          uint32_t v[32];
          tmem_ld32(tmem_base + lanes + kBN + 32 * ch, v);
          epilogue_chunk_x3<ET, EPI, OUT>(p, br, r0, tc.y + 32 * ch, v, S, YB, lane, lam, track, amax_bits, cap);
        }
        if (EPI == EPI_FINAL && p.ep.cres) {
          const double cs = compl_warp_sum(cacc);
          if (lane == 0) p.ep.cres[4 * t + ew] = cs;
        }
      } else {
        if (!wait_bounded(tfull_bar(acc), acc_ph, abort_flag)) break;
        tc_fence_after();
#pragma unroll 1
        for (int ch = ch_begin; ch < ch_end; ++ch) {
          uint32_t v[32];
          tmem_ld32(tmem_base + lanes + acc * kBN + 32 * ch, v);
          epilogue_chunk_x3<ET, EPI, OUT>(p, br, r0, tc.y + 32 * ch, v, S, YB, lane, lam, track, amax_bits);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (!PAIR || leader)
            mbar_arrive(tempty_bar(acc));
          else
            mbar_arrive_remote(tempty_leader[acc]);
        }
        acc ^= 1u;
        if (acc == 0) acc_ph ^= 1u;
      }
    }
    if (track_launch && amax_block >= 0) flush_amax(amax_block);
  }

  // pair form: every operand read, remote arrival and copy of the pair is
  // complete before either CTA releases tensor memory or exits
  tc_fence_before();
  if (PAIR)
    cluster_sync_all();
  else
    __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    if (PAIR)
      tmem_dealloc_pair(tmem_base, kTmemCols);
    else
      tmem_dealloc(tmem_base, kTmemCols);
  }
  if (threadIdx.x == 0 && *abort_flag && p.ep.status) atomicCAS(p.ep.status, 0, PSD_ERR_TIMEOUT);
}

using KernelX3 = void (*)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const CUtensorMap,
                          const GemmParams);

// Instances: TF32 pairs (the FP32 path: pair outputs, the FP32 final output);
// FP16 pairs (pair or FP16 outputs); FP16 pair A with a single FP16 B (P X of
// the mixed precision's pair stages, FP16 output).
KernelX3 pick_pair(bool b1, int epi, int out) {
  if (b1) return (epi == EPI_SCALE && out == 1) ? symgemm_x3_kernel<DT_F16X2, EPI_SCALE, 1, true, true> : nullptr;
  if (out != 0) return nullptr;
  if (epi == EPI_COPY) return symgemm_x3_kernel<DT_F16X2, EPI_COPY, 0, false, true>;
  if (epi == EPI_POLY) return symgemm_x3_kernel<DT_F16X2, EPI_POLY, 0, false, true>;
  if (epi == EPI_SCALE) return symgemm_x3_kernel<DT_F16X2, EPI_SCALE, 0, false, true>;
  return nullptr;
}

KernelX3 pick(int et, bool b1, int epi, int out) {
  if (et == DT_TF32X3) {
    if (b1) return nullptr;
    if (epi == EPI_FINAL) return out == 2 ? symgemm_x3_kernel<DT_TF32X3, EPI_FINAL, 2, false> : nullptr;
    if (out != 0) return nullptr;
    if (epi == EPI_COPY) return symgemm_x3_kernel<DT_TF32X3, EPI_COPY, 0, false>;
    if (epi == EPI_POLY) return symgemm_x3_kernel<DT_TF32X3, EPI_POLY, 0, false>;
    return symgemm_x3_kernel<DT_TF32X3, EPI_SCALE, 0, false>;
  }
  if (et != DT_F16X2 || epi == EPI_FINAL) return nullptr;
  if (b1) return (epi == EPI_SCALE && out == 1) ? symgemm_x3_kernel<DT_F16X2, EPI_SCALE, 1, true> : nullptr;
  if (out == 1) {
    if (epi == EPI_COPY) return symgemm_x3_kernel<DT_F16X2, EPI_COPY, 1, false>;
    if (epi == EPI_POLY) return symgemm_x3_kernel<DT_F16X2, EPI_POLY, 1, false>;
    return symgemm_x3_kernel<DT_F16X2, EPI_SCALE, 1, false>;
  }
  if (epi == EPI_COPY) return symgemm_x3_kernel<DT_F16X2, EPI_COPY, 0, false>;
  if (epi == EPI_POLY) return symgemm_x3_kernel<DT_F16X2, EPI_POLY, 0, false>;
  return symgemm_x3_kernel<DT_F16X2, EPI_SCALE, 0, false>;
}

}  // namespace

// et: DT_TF32X3 or DT_F16X2; b_single: B is one FP16 matrix (tm[3] unused).
// tm: A_hi, A_lo, B_hi, B_lo.  out: 0 = split pair, 1 = FP16 (EPI_FINAL: 2, FP32 to the block's out).
cudaError_t launch_symgemm_x3(int et, bool b_single, int epi, int out, const CUtensorMap* tm, const GemmParams& p,
                              int grid, cudaStream_t stream, bool pair) {
  if (p.num_tiles == 0) return cudaSuccess;
  if (pair && et != DT_F16X2) return cudaErrorNotSupported;
  KernelX3 k = pair ? pick_pair(b_single, epi, out) : pick(et, b_single, epi, out);
  if (!k) return cudaErrorNotSupported;
  const int smem = pair ? (b_single ? X3Cfg<true, true>::smem() : X3Cfg<false, true>::smem())
                        : (b_single ? X3Cfg<true>::smem() : X3Cfg<false>::smem());
  static std::mutex done_mu;  // launches come from callers' threads and the request server's
  static KernelX3 done[32];
  static int ndone = 0;
  {
    std::lock_guard<std::mutex> lk(done_mu);
    bool set = false;
    for (int i = 0; i < ndone; ++i) set = set || done[i] == k;
    if (!set) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      if (ndone < 32) done[ndone++] = k;
    }
  }
  GemmParams q = p;
  const uint32_t fmt = et == DT_TF32X3 ? 2u : 0u;  // kind::tf32, or kind::f16 with FP16 operands
  q.idesc = make_idesc(fmt, pair ? 2 * kBM : kBM, 0);  // N comes from each tile
  if (!pair) {
    const int g = std::max(1, std::min(grid, p.num_tiles));
    k<<<g, kThreads, smem, stream>>>(tm[0], tm[1], tm[2], tm[3], q);
    return cudaGetLastError();
  }
  const int pairs = std::max(1, std::min(grid / 2, p.num_tiles));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(2 * pairs);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, tm[0], tm[1], tm[2], tm[3], q);
}

}  // namespace psd
