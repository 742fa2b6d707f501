// Symmetric matrix product on the sm_103a tensor cores with fused epilogues.
//
// Every product of Algorithm 2 multiplies two polynomials in X, which
// commute, so the exact result is symmetric.  The kernel forms only the
// 128 x 256 output tiles of the upper triangle (256 x 256 blocks (I, J) with
// I <= J, each split into two 128-row tiles), accumulates them in tensor
// memory with tcgen05.mma (operands staged by TMA with the 128-byte swizzle),
// and writes every 32 x 32 chunk twice -- at (r, c) and mirrored at (c, r) --
// so the stored result is exactly symmetric and no separate pass over HBM is
// needed.  The epilogue applies the stage arithmetic of Sec. 3 / Algorithm 2:
//   EPI_COPY   Y   = X_{t-1}^2
//   EPI_POLY   P   = a_t I + b_t Y + c_t Y^2          (the degree-5 stage, Sec. 3.3)
//   EPI_SCALE  X_t = (X_{t-1} P) / s_t               (Sec. 3.4 rescale)
//   EPI_FINAL  out = (X + lam~ X_0 X_T) / 2           (Algorithm 2 return, FP32)
//
// Warp roles (192 threads, one CTA per SM, persistent over a static tile list):
//   warp 0   TMA producer (one lane)
//   warp 1   tensor-memory allocation and MMA issue (one lane)
//   warps 2-5 epilogue; warp w reads TMEM lanes 32 (w % 4) .. +31
// Two 256-column FP32 accumulators in tensor memory let the epilogue of one
// tile overlap the main loop of the next.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "internal.h"
#include "ptx.cuh"

namespace psd {

namespace {

constexpr int kBM = 128;
constexpr int kBN = 256;

// One swizzle row of kRowBytes16 (128) bytes of K per operand row and stage:
// 64 K-elements for 16-bit operands, 128 for e4m3 (the same stage layout in
// bytes); 4 stages of 48 KB.
constexpr int kBK16 = kRowBytes16 / 2;
constexpr int kBK8 = kRowBytes16;
constexpr int kStages16 = 4 * (128 / kRowBytes16);
constexpr int kABytes16 = kBM * kRowBytes16;          // 16 KB
constexpr int kBBytes16 = kBN * kRowBytes16;          // 32 KB
constexpr int kStageBytes16 = kABytes16 + kBBytes16;  // 48 KB

// Epilogue staging per warp.  16-bit outputs: the chunk row-major (S),
// transposed (ST) and the prefetched Y chunk (YB), each 32 x 40 halves (80-byte
// rows keep 16-byte accesses aligned and spread over the banks).  FP32 output:
// 32 x 33 words, in the same space.
constexpr int kStgWords = 33;
constexpr int kH = 40;
constexpr int kEpiWarpBytes = 3 * 32 * kH * 2;  // 7680 >= 32 * 33 * 4

constexpr int kTmemCols = 512;

// Epilogue warps: 4 (one per 32-lane quarter of tensor memory) with a 4-stage
// ring, or 8 (two per quarter, taking alternate 32-column chunks) with a
// 3-stage ring.  The second form is for launches over the small blocks of a
// block-diagonal cone, whose short tiles leave the epilogue, not the main
// loop, as the bound (512 blocks of orders 16-1024: 6.14 -> 5.79 ms); served
// steps, which mix in large requests, lost 12% throughput with it.
__host__ __device__ constexpr int stages16(int ew) { return ew == 4 ? kStages16 : 3; }
__host__ __device__ constexpr int threads16(int ew) { return 64 + 32 * ew; }
__host__ __device__ constexpr int smem_bytes16(int ew = 4) {
  return 1024 /* alignment slack */ + stages16(ew) * kStageBytes16 + ew * kEpiWarpBytes +
         8 * (2 * stages16(ew) + 5) + 16;
}
static_assert(smem_bytes16(4) <= 232448 && smem_bytes16(8) <= 232448, "shared memory per CTA");

__device__ __forceinline__ uint16_t to16(float v, bool bf16) {
  return bf16 ? __bfloat16_as_ushort(__float2bfloat16_rn(v)) : __half_as_ushort(__float2half_rn(v));
}
__device__ __forceinline__ float from16(uint16_t u, bool bf16) {
  return bf16 ? __bfloat162float(__ushort_as_bfloat16(u)) : __half2float(__ushort_as_half(u));
}

__device__ __forceinline__ uint16_t to8(float v) {
  return static_cast<uint16_t>(__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3));
}

__device__ __forceinline__ void raise_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Y chunk (r0..r0+31) x (c0..c0+31) of a symmetric 16-bit matrix, read as
// memory rows c (32 contiguous halves at c * ldy + r0): lane l loads 16 bytes of
// rows c0 + l/4 + 8k, k = 0..3.  Zeros outside n.
__device__ __forceinline__ void load_y_chunk(const uint16_t* __restrict__ Y, int64_t ldy, int n, int r0, int c0,
                                             int lane, uint4 (&y)[4]) {
  const int r = r0 + 8 * (lane & 3);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = c0 + (lane >> 2) + 8 * k;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (c < n && r < n) {
      const uint16_t* p = Y + static_cast<int64_t>(c) * ldy + r;
      if (r + 7 < n) {
        v = __ldg(reinterpret_cast<const uint4*>(p));
      } else {
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        for (int e = 0; e < 8 && r + e < n; ++e) w[e >> 1] |= static_cast<uint32_t>(p[e]) << (16 * (e & 1));
        v = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    y[k] = v;
  }
}

// The same chunk of a symmetric e4m3 matrix (8 bytes per lane and row),
// decoded to FP16 and multiplied by ysc (a power of two: exact).
__device__ __forceinline__ void load_y_chunk8(const uint8_t* __restrict__ Y, int64_t ldy, int n, int r0, int c0,
                                              int lane, __half2 ysc, uint4 (&y)[4]) {
  const int r = r0 + 8 * (lane & 3);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = c0 + (lane >> 2) + 8 * k;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (c < n && r < n) {
      const uint8_t* p = Y + static_cast<int64_t>(c) * ldy + r;
      uint2 raw = make_uint2(0u, 0u);
      if (r + 7 < n) {
        raw = __ldg(reinterpret_cast<const uint2*>(p));
      } else {
        for (int e = 0; e < 8 && r + e < n; ++e) {
          const uint32_t b = p[e];
          if (e < 4)
            raw.x |= b << (8 * e);
          else
            raw.y |= b << (8 * (e - 4));
        }
      }
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t word = q < 2 ? raw.x : raw.y;
        const __nv_fp8x2_storage_t pair = static_cast<__nv_fp8x2_storage_t>((word >> (16 * (q & 1))) & 0xFFFFu);
        __half2 h = __half2(__nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3));
        h = __hmul2(h, ysc);
        w[q] = *reinterpret_cast<uint32_t*>(&h);
      }
      v = make_uint4(w[0], w[1], w[2], w[3]);
    }
    y[k] = v;
  }
}

// 8 e4m3 codes (low bytes of 8 staged 16-bit words) to global memory at dst[0..7], clipped at n.
__device__ __forceinline__ void store8_u8(uint8_t* dst, const uint16_t* src, int first, int n) {
  const uint4 v = *reinterpret_cast<const uint4*>(src);
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
  uint32_t lo = 0u, hi = 0u;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const uint32_t b = (w[e >> 1] >> (16 * (e & 1))) & 0xFFu;
    if (e < 4)
      lo |= b << (8 * e);
    else
      hi |= b << (8 * (e - 4));
  }
  if (first + 7 < n) {
    *reinterpret_cast<uint2*>(dst) = make_uint2(lo, hi);
  } else {
    for (int e = 0; e < 8 && first + e < n; ++e) dst[e] = static_cast<uint8_t>(e < 4 ? lo >> (8 * e) : hi >> (8 * (e - 4)));
  }
}

// 16 bytes (8 halves) of one staged row to global memory at dst[0..7], clipped at `limit`.
__device__ __forceinline__ void store8(uint16_t* dst, const uint16_t* src, int first, int n) {
  const uint4 v = *reinterpret_cast<const uint4*>(src);
  if (first + 7 < n) {
    *reinterpret_cast<uint4*>(dst) = v;
  } else {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    for (int e = 0; e < 8 && first + e < n; ++e) dst[e] = static_cast<uint16_t>(w[e >> 1] >> (16 * (e & 1)));
  }
}

// One 32 x 32 chunk with 16-bit output.  Lane l holds row r0 + l, v[j] is the
// accumulator at column c0 + j.  Diagonal chunks (r0 == c0) are symmetrised
// from their upper part; off-diagonal chunks are written at both positions,
// (r, c) and (c, r), with 16-byte stores from the staged copies.
// Stages a 32 x 32 chunk of 16-bit codes (h[j] = code at (r0 + lane, c0 + j))
// and writes it at (r, c) and, unless diagonal, mirrored at (c, r); diagonal
// chunks are symmetrised from their upper part first (h is updated to the
// symmetric codes).  OUTK 1 writes the low bytes (e4m3 codes).
template <int OUTK>
__device__ __forceinline__ void stage_store16(uint32_t (&h)[32], uint16_t* S, uint16_t* ST, bool diag, void* Cv,
                                              int64_t ldc, int n, int r0, int c0, int lane) {
  uint16_t* row = S + lane * kH;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    *reinterpret_cast<uint4*>(row + 8 * q) =
        make_uint4(h[8 * q] | (h[8 * q + 1] << 16), h[8 * q + 2] | (h[8 * q + 3] << 16),
                   h[8 * q + 4] | (h[8 * q + 5] << 16), h[8 * q + 6] | (h[8 * q + 7] << 16));
  if (diag) {
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < lane) h[j] = S[j * kH + lane];
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 4; ++q)
      *reinterpret_cast<uint4*>(row + 8 * q) =
          make_uint4(h[8 * q] | (h[8 * q + 1] << 16), h[8 * q + 2] | (h[8 * q + 3] << 16),
                     h[8 * q + 4] | (h[8 * q + 5] << 16), h[8 * q + 6] | (h[8 * q + 7] << 16));
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) ST[j * kH + lane] = static_cast<uint16_t>(h[j]);
  }
  __syncwarp();
  const int seg = 8 * (lane & 3);
  // memory rows c0 + j: output column c0 + j over rows r0..r0+31 (ST row j; S row j when symmetric)
  const uint16_t* SA = diag ? S : ST;
  uint16_t* C = static_cast<uint16_t*>(Cv);
  uint8_t* C8 = static_cast<uint8_t*>(Cv);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int jj = (lane >> 2) + 8 * k;
    const int c = c0 + jj;
    if (c < n && r0 + seg < n) {
      if (OUTK == 1)
        store8_u8(C8 + static_cast<int64_t>(c) * ldc + r0 + seg, SA + jj * kH + seg, r0 + seg, n);
      else
        store8(C + static_cast<int64_t>(c) * ldc + r0 + seg, SA + jj * kH + seg, r0 + seg, n);
    }
  }
  if (!diag) {
    // memory rows r0 + t: output row r0 + t over columns c0..c0+31 (S row t)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int tt = (lane >> 2) + 8 * k;
      const int rr = r0 + tt;
      if (rr < n && c0 + seg < n) {
        if (OUTK == 1)
          store8_u8(C8 + static_cast<int64_t>(rr) * ldc + c0 + seg, S + tt * kH + seg, c0 + seg, n);
        else
          store8(C + static_cast<int64_t>(rr) * ldc + c0 + seg, S + tt * kH + seg, c0 + seg, n);
      }
    }
  }
  __syncwarp();
}

// One 32 x 32 chunk with 16-bit (or e4m3, or FP16 hi/lo pair) output.  Lane l
// holds row r0 + l, v[j] is the accumulator at column c0 + j.
//   OUTK 0: 16-bit (FP16 or BF16 by `bf16`), 1: e4m3 (value * out_scale),
//   2: FP16 pair, hi = RN(value) at C, lo = RN(value - hi) at C_lo.
template <int EPI, bool IN8, int OUTK>
__device__ __forceinline__ void epilogue_chunk16(const GemmParams& p, const BlockRec& br, bool bf16, int n,
                                                 void* Cv, void* Cv_lo, int r0, int c0, const uint32_t (&v)[32],
                                                 uint8_t* wbuf, const uint4 (&y)[4], int lane, bool track,
                                                 unsigned& amax_bits) {
  const bool pb = p.ep.per_block_coef != 0;
  const float ca = pb ? br.ca : p.ep.a, cb = pb ? br.cb : p.ep.b, cc = pb ? br.cc : p.ep.c;
  const float cs = pb ? br.cs : p.ep.s;
  uint16_t* S = reinterpret_cast<uint16_t*>(wbuf);  // [32][kH] row t = output row r0 + t
  uint16_t* ST = S + 32 * kH;                        // [32][kH] row j = output column c0 + j
  uint16_t* YB = ST + 32 * kH;                       // [32][kH] row j = Y column c0 + j
  const int r = r0 + lane;
  const bool diag = (r0 == c0);
  if (EPI == EPI_POLY) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      *reinterpret_cast<uint4*>(YB + ((lane >> 2) + 8 * k) * kH + 8 * (lane & 3)) = y[k];
    __syncwarp();
  }
  uint32_t h[32], l[OUTK == 2 ? 32 : 1];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    float acc = __uint_as_float(v[j]);
    if (IN8) acc *= p.ep.in_scale;
    float val;
    if (EPI == EPI_POLY) {
      const float yv = from16(YB[j * kH + lane], IN8 ? false : bf16);
      val = fmaf(cc, acc, cb * yv);
      if (diag && j == lane) val += ca;
    } else if (EPI == EPI_SCALE) {
      val = acc * cs;
    } else {
      val = acc;
    }
    if constexpr (OUTK == 2) {
      h[j] = to16(val, false);
      l[j] = to16(val - from16(static_cast<uint16_t>(h[j]), false), false);
    } else {
      h[j] = OUTK == 1 ? to8(val * p.ep.out_scale) : to16(val, bf16);
    }
  }
  const int64_t ldc = p.ep.ldc;
  stage_store16<OUTK>(h, S, ST, diag, Cv, ldc, n, r0, c0, lane);
  if constexpr (OUTK == 2) stage_store16<0>(l, S, ST, diag, Cv_lo, ldc, n, r0, c0, lane);
  if (OUTK == 0 && track && r < n) {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (c0 + j < n) amax_bits = max(amax_bits, __float_as_uint(fabsf(from16(static_cast<uint16_t>(h[j]), bf16))));
  }
}

// One 32 x 32 chunk of the final output out = (X + lam~ acc) / 2 in FP32,
// reading only the upper triangle of the caller's X (column-major).
__device__ __forceinline__ void epilogue_chunk_final(const BlockRec& br, int r0, int c0,
                                                     const uint32_t (&v)[32], uint8_t* wbuf,
                                                     int lane, float lam, ComplAcc* ca) {
  uint32_t* stg = reinterpret_cast<uint32_t*>(wbuf);
  const int n = br.n;
  const float* X = br.X;
  const int64_t ld = br.ld;
  float* out = br.out;
  const int64_t ldo = br.ld_out;
  const int r = r0 + lane;
  const bool diag = (r0 == c0);
  const bool row_ok = r < n;
  float o[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const int c = c0 + j;
    float x = 0.f;
    const bool upper = !diag || j >= lane;
    if (row_ok && c < n && upper) x = X[static_cast<int64_t>(c) * ld + r];
    o[j] = 0.5f * fmaf(lam, __uint_as_float(v[j]), x);
    if (ca && row_ok && c < n && upper) compl_add(*ca, o[j], x, c == r ? 1.f : 2.f);
  }
  float* sf = reinterpret_cast<float*>(stg);
  if (diag) {
#pragma unroll
    for (int j = 0; j < 32; ++j) sf[lane * kStgWords + j] = o[j];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < lane) o[j] = sf[j * kStgWords + lane];
    __syncwarp();
  }
  if (row_ok) {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (c0 + j < n) out[static_cast<int64_t>(c0 + j) * ldo + r] = o[j];
  }
  if (!diag) {
#pragma unroll
    for (int j = 0; j < 32; ++j) sf[lane * kStgWords + j] = o[j];
    __syncwarp();
    const int c = c0 + lane;
    if (c < n) {
#pragma unroll 4
      for (int rr = 0; rr < 32; ++rr)
        if (r0 + rr < n) out[static_cast<int64_t>(r0 + rr) * ldo + c] = sf[rr * kStgWords + lane];
    }
    __syncwarp();
  }
}

template <int EPI, bool IN8, int OUTK, int EW = 4>
__global__ void __launch_bounds__(threads16(EW), 1)
    symgemm16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const GemmParams p, const int bf16_flag) {
  static_assert(EW == 4 || (EW == 8 && EPI != EPI_FINAL), "8 epilogue warps: stage products only");
  constexpr int kStages16 = stages16(EW);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* stages = smem;
  uint8_t* epi_stg = smem + kStages16 * kStageBytes16;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages16 * kStageBytes16 + EW * kEpiWarpBytes);
  // bars: full[S] | empty[S] | tfull[2] | tempty[2] | drain
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * kStages16 + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const bool bf16 = bf16_flag != 0;
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + kStages16 + s); };
  auto tfull_bar = [&](int a) { return smem_u32(bars + 2 * kStages16 + a); };
  auto tempty_bar = [&](int a) { return smem_u32(bars + 2 * kStages16 + 2 + a); };
  const uint32_t drain_bar = smem_u32(bars + 2 * kStages16 + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages16; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), EW);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_holder), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      int last_parity[kStages16];
      for (int s = 0; s < kStages16; ++s) last_parity[s] = -1;
      uint32_t s = 0, ph = 0;
      bool ok = true;
      for (TileStream ts(p, blockIdx.x, gridDim.x); ok && ts.valid(); ts.advance()) {
        ts.prefetch();
        const TileMeta& m = ts.cur();
        constexpr int kBK = IN8 ? kBK8 : kBK16;
        const int kbn = (m.n + kBK - 1) / kBK;
        const int ya = static_cast<int>(m.off + m.tc.x), yb = static_cast<int>(m.off + m.db + m.tc.y);
        for (int kb = 0; kb < kbn; ++kb) {
          if (!wait_bounded(empty_bar(s), ph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full_bar(s), kStageBytes16);
          const uint32_t a_dst = smem_u32(stages + s * kStageBytes16);
          tma_load_2d(a_dst, &tmA, kb * kBK, ya, full_bar(s));
          tma_load_2d(a_dst + kABytes16, &tmB, kb * kBK, yb, full_bar(s));
          last_parity[s] = static_cast<int>(ph);
          if (++s == kStages16) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      if (!ok) {
        // let the copies already in flight land before the CTA exits
        for (int q = 0; q < kStages16; ++q)
          if (last_parity[q] >= 0) {
            const unsigned long long t0 = globaltimer_ns();
            while (!mbar_try_wait(full_bar(q), static_cast<uint32_t>(last_parity[q])) &&
                   globaltimer_ns() - t0 < kWaitLimitNs) {
            }
          }
      }
    }
  } else if (warp == 1) {
    uint32_t s = 0, ph = 0, acc = 0, acc_ph = 0;
    bool ok = true;
    for (TileStream ts(p, blockIdx.x, gridDim.x); ok && ts.valid(); ts.advance()) {
      ts.prefetch();
      const int4 tc = ts.cur().tc;
      constexpr int kBK = IN8 ? kBK8 : kBK16;
      const int kbn = (ts.cur().n + kBK - 1) / kBK;
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
          const uint32_t a_addr = smem_u32(stages + s * kStageBytes16);
          const uint32_t b_addr = a_addr + kABytes16;
          auto desc = [](uint32_t a) { return kRowBytes16 == 64 ? sw64_kmajor_desc(a) : sw128_kmajor_desc(a); };
#pragma unroll
          for (int k = 0; k < kRowBytes16 / 32; ++k) {  // 32 bytes of K per instruction (16 halves or 32 e4m3)
            if (IN8)
              mma_f8(d_tmem, desc(a_addr + 32 * k), desc(b_addr + 32 * k), idesc, (kb | k) != 0 ? 1u : 0u);
            else
              mma_f16(d_tmem, desc(a_addr + 32 * k), desc(b_addr + 32 * k), idesc, (kb | k) != 0 ? 1u : 0u);
          }
          mma_commit(empty_bar(s));
        }
        __syncwarp();
        if (++s == kStages16) {
          s = 0;
          ph ^= 1u;
        }
      }
      if (!ok) break;
      if (lane == 0) mma_commit(tfull_bar(acc));
      __syncwarp();
      acc ^= 1u;
      if (acc == 0) acc_ph ^= 1u;
    }
    if (!ok && lane == 0) {
      // wait for the MMAs already issued before tensor memory is released
      mma_commit(drain_bar);
      const unsigned long long t0 = globaltimer_ns();
      while (!mbar_try_wait(drain_bar, 0) && globaltimer_ns() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
  } else {
    const int ew = warp & 3;                  // tensor-memory lane quarter (warp % 4)
    const int ewi = warp - 2;                 // epilogue warp 0 .. EW - 1
    constexpr int kChStep = EW / 4;           // chunks of a quarter, dealt to its EW / 4 warps
    const int ch_first = ewi / 4;
    uint8_t* wbuf = epi_stg + ewi * kEpiWarpBytes;
    uint32_t acc = 0, acc_ph = 0;
    unsigned amax_bits = 0;  // max |output| of the current block (absmax_blocks) or of the launch
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
    for (int t = blockIdx.x; t < p.num_tiles; t += gridDim.x) {
      const int4 tc = p.tiles[t];
      const BlockRec& br = p.blocks[tc.z];
      const int n = br.n;
      const int64_t off = br.off;
      void* C = static_cast<uint8_t*>(p.ep.C) + (off + br.dc) * p.ep.ldc * (OUTK == 1 ? 1 : 2);
      void* C_lo = OUTK == 2 ? static_cast<uint8_t*>(p.ep.C_lo) + (off + br.dc) * p.ep.ldc * 2 : nullptr;
      const uint8_t* Yb = static_cast<const uint8_t*>(p.ep.Y) + (off + br.dy) * p.ep.ldy * (IN8 ? 1 : 2);
      const bool track = track_launch && (p.ep.absmax_blocks != 2 || br.track != 0);
      if (track_launch && amax_block != tc.z) {
        if (amax_block >= 0) flush_amax(amax_block);
        amax_block = tc.z;
      }
      const int r0 = tc.x + 32 * ew;
      // chunks of this warp's 32 rows that lie on or above the diagonal and inside n
      const int ch_begin = max(0, (r0 - tc.y) >> 5);
      const int ch_end = r0 < n ? min((tc.w + 31) >> 5, (n - tc.y + 31) >> 5) : ch_begin;
      uint4 ynext[4] = {};
      auto load_y = [&](int c0, uint4 (&dst)[4]) {
        if (IN8)
          load_y_chunk8(Yb, p.ep.ldy, n, r0, c0, lane, __float2half2_rn(p.ep.y_scale), dst);
        else
          load_y_chunk(reinterpret_cast<const uint16_t*>(Yb), p.ep.ldy, n, r0, c0, lane, dst);
      };
      if (EPI == EPI_POLY && ch_begin + ch_first < ch_end) load_y(tc.y + 32 * (ch_begin + ch_first), ynext);
      if (!wait_bounded(tfull_bar(acc), acc_ph, abort_flag)) break;
      tc_fence_after();
      const float lam = EPI == EPI_FINAL ? static_cast<float>(br.st->lambda) : 0.f;
      // shares of <out, X - out>: at the launch position, or at the tile's
      // position in the block's own list (served requests)
      double* cdst = nullptr;
      if (EPI == EPI_FINAL)
        cdst = p.ep.cres ? p.ep.cres + 4 * t : br.cres ? br.cres + 4 * (t + br.cres_shift) : nullptr;
      ComplAcc cacc;
      ComplAcc* cap = cdst ? &cacc : nullptr;
#pragma unroll 1
      for (int ch = ch_begin + ch_first; ch < ch_end; ch += kChStep) {
        const int c0 = tc.y + 32 * ch;
        uint4 ycur[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) ycur[k] = ynext[k];
        if (EPI == EPI_POLY && ch + kChStep < ch_end) load_y(c0 + 32 * kChStep, ynext);
        uint32_t v[32];
        tmem_ld32(tmem_base + (static_cast<uint32_t>(32 * ew) << 16) + acc * kBN + 32 * ch, v);
        if (EPI == EPI_FINAL)
          epilogue_chunk_final(br, r0, c0, v, wbuf, lane, lam, cap);
        else
          epilogue_chunk16<EPI, IN8, OUTK>(p, br, bf16, n, C, C_lo, r0, c0, v, wbuf, ycur, lane, track,
                                           amax_bits);
      }
      if (EPI == EPI_FINAL && cdst) {
        const double cs = compl_warp_sum(cacc);
        if (lane == 0) cdst[ew] = cs;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty_bar(acc));
      acc ^= 1u;
      if (acc == 0) acc_ph ^= 1u;
    }
    if (EPI != EPI_FINAL && track_launch && amax_block >= 0) flush_amax(amax_block);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
  if (threadIdx.x == 0 && *abort_flag) raise_status(p.ep.status, PSD_ERR_TIMEOUT);
}

// ------------------------------------------------------------ 2-SM form
// The same product on CTA pairs (a cluster of two CTAs on two SMs): one
// tcgen05.mma.cta_group::2 of M = 256 covers a 256 x N tile, rows 0-127 in the
// leader's tensor memory and 128-255 in the peer's.  Each CTA stages its own
// 128 rows of A and half of B (N/2 rows), so a stage holds 32 KB instead of
// 48 KB and the ring six stages instead of four (the MMA warp has twice the
// lookahead), and each SM loads half the B operand it used to.  The leader's
// producer counts the bytes of both CTAs on its full barrier (the peer's TMA
// signals it across the pair), its MMA warp issues for both, and its commits
// arrive on the barriers of both CTAs; the peer's epilogue warps release an
// accumulator through the leader's barrier.  Tiles: (m0, n0, block, width),
// 256 x 256 blocks of the upper triangle, diagonal blocks in full (chunks
// below the diagonal are computed but not written).  Epilogues: copy,
// polynomial and scale with a 16-bit or FP16-pair output, and the final
// product (FP32 output; with 4 epilogue warps per CTA, the eight of a pair
// tile write the complementarity shares of the two 128-row tiles of the
// one-SM form, in its order: slots 8 t + 4 rank + warp quarter).
// EW epilogue warps per CTA: 4 with a 6-stage ring (single matrices, long
// K), or 8 with a 5-stage ring (the blocks of a block-diagonal cone: K <=
// 1024, where one warp per 32-lane quarter no longer drains a tile within
// the next tile's main loop); with 8, a quarter's two warps take alternate
// 32-column chunks and FINAL writes 16 shares per pair tile (2 EW t + EW rank
// + warp).
constexpr int kBHalfBytes = kBM * kRowBytes16;          // 16 KB: 128 rows of B
constexpr int kStageBytesP = kABytes16 + kBHalfBytes;  // 32 KB
__host__ __device__ constexpr int stages_pair(int ew) { return ew == 4 ? 6 : 5; }
__host__ __device__ constexpr int smem_bytes_pair(int ew = 4) {
  return 1024 + stages_pair(ew) * kStageBytesP + ew * kEpiWarpBytes + 8 * (2 * stages_pair(ew) + 5) + 16;
}
static_assert(smem_bytes_pair(4) <= 232448 && smem_bytes_pair(8) <= 232448, "shared memory per CTA");
// A wait that has given up leaves copies of this CTA in flight, which signal
// the leader's barrier: they are given this long to land before the CTA exits.
constexpr unsigned long long kPairDrainNs = 200000ull;

template <int EPI, int OUTK, int EW = 4>
__global__ void __launch_bounds__(threads16(EW), 1)
    symgemm16_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                          const GemmParams p, const int bf16_flag) {
  static_assert(OUTK != 1 && (EPI != EPI_FINAL || OUTK == 0), "pair form: 16-bit operands, no e4m3 output");
  static_assert(EW == 4 || EW == 8, "4 or 8 epilogue warps");
  constexpr int kStagesP = stages_pair(EW);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* stages = smem;
  uint8_t* epi_stg = smem + kStagesP * kStageBytesP;
  uint64_t* bars = reinterpret_cast<uint64_t*>(epi_stg + EW * kEpiWarpBytes);
  // bars: full[S] | empty[S] | tfull[2] | tempty[2] | drain
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * kStagesP + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const bool bf16 = bf16_flag != 0;
  const uint32_t rank = cluster_ctarank();
  const bool leader = rank == 0;
  const int cl = static_cast<int>(blockIdx.x >> 1), ncl = static_cast<int>(gridDim.x >> 1);
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + kStagesP + s); };
  auto tfull_bar = [&](int a) { return smem_u32(bars + 2 * kStagesP + a); };
  auto tempty_bar = [&](int a) { return smem_u32(bars + 2 * kStagesP + 2 + a); };
  const uint32_t drain_bar = smem_u32(bars + 2 * kStagesP + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStagesP; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), 2 * EW);  // the leader's: the epilogue warps of both CTAs
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  if (warp == 1) {
    tmem_alloc_pair(smem_u32(tmem_holder), kTmemCols);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  cluster_sync_all();  // both CTAs' barriers initialised before any arrival crosses the pair
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t s = 0, ph = 0;
      bool ok = true, issued = false;
      for (TileStream ts(p, cl, ncl); ok && ts.valid(); ts.advance()) {
        ts.prefetch();
        const TileMeta& m = ts.cur();
        const int4 tc = m.tc;
        const int kbn = (m.n + kBK16 - 1) / kBK16;
        // this CTA's 128 rows of A and its N/2 rows of B
        const int ya = static_cast<int>(m.off + tc.x + 128 * static_cast<int>(rank));
        const int yb = static_cast<int>(m.off + m.db + tc.y + (tc.w >> 1) * static_cast<int>(rank));
        for (int kb = 0; kb < kbn; ++kb) {
          if (!wait_bounded(empty_bar(s), ph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          if (leader) mbar_arrive_expect_tx(full_bar(s), 2 * kStageBytesP);  // both CTAs' copies
          const uint32_t dst = smem_u32(stages + s * kStageBytesP);
          const uint32_t fb = mapa_shared(full_bar(s), 0);
          tma_load_2d_pair(dst, &tmA, kb * kBK16, ya, fb);
          tma_load_2d_pair(dst + kABytes16, &tmB, kb * kBK16, yb, fb);
          issued = true;
          if (++s == kStagesP) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      if (!ok && issued) {
        const unsigned long long t0 = globaltimer_ns();
        while (globaltimer_ns() - t0 < kPairDrainNs) {
        }
      }
    }
  } else if (warp == 1) {
    if (leader) {
      uint32_t s = 0, ph = 0, acc = 0, acc_ph = 0;
      bool ok = true;
      for (TileStream ts(p, cl, ncl); ok && ts.valid(); ts.advance()) {
        ts.prefetch();
        const int4 tc = ts.cur().tc;
        const int kbn = (ts.cur().n + kBK16 - 1) / kBK16;
        const uint32_t idesc = p.idesc | (static_cast<uint32_t>(tc.w >> 3) << 17);  // M = 256, N = tile width
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
            const uint32_t a_addr = smem_u32(stages + s * kStageBytesP);
            const uint32_t b_addr = a_addr + kABytes16;
#pragma unroll
            for (int k = 0; k < kRowBytes16 / 32; ++k)
              mma_f16_pair(d_tmem, sw128_kmajor_desc(a_addr + 32 * k), sw128_kmajor_desc(b_addr + 32 * k), idesc,
                           (kb | k) != 0 ? 1u : 0u);
            mma_commit_pair(empty_bar(s), 3);  // frees the stage in both CTAs
          }
          __syncwarp();
          if (++s == kStagesP) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
        if (lane == 0) mma_commit_pair(tfull_bar(acc), 3);
        __syncwarp();
        acc ^= 1u;
        if (acc == 0) acc_ph ^= 1u;
      }
      if (!ok && lane == 0) {
        mma_commit_pair(drain_bar, 1);  // the MMAs already issued, before tensor memory is released
        const unsigned long long t0 = globaltimer_ns();
        while (!mbar_try_wait(drain_bar, 0) && globaltimer_ns() - t0 < kWaitLimitNs) {
        }
      }
      __syncwarp();
    }
  } else {
    const int ew = warp & 3;         // tensor-memory lane quarter
    const int ewi = warp - 2;        // epilogue warp 0 .. EW - 1
    constexpr int kChStep = EW / 4;  // chunks of a quarter, dealt to its EW / 4 warps
    const int ch_first = ewi / 4;
    uint8_t* wbuf = epi_stg + ewi * kEpiWarpBytes;
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
    const uint32_t tempty_leader[2] = {mapa_shared(tempty_bar(0), 0), mapa_shared(tempty_bar(1), 0)};
    for (int t = cl; t < p.num_tiles; t += ncl) {
      const int4 tc = p.tiles[t];
      const BlockRec& br = p.blocks[tc.z];
      const int n = br.n;
      const int64_t off = br.off;
      void* C = static_cast<uint8_t*>(p.ep.C) + (off + br.dc) * p.ep.ldc * 2;
      void* C_lo = OUTK == 2 ? static_cast<uint8_t*>(p.ep.C_lo) + (off + br.dc) * p.ep.ldc * 2 : nullptr;
      const uint16_t* Yb = EPI == EPI_POLY
                               ? reinterpret_cast<const uint16_t*>(static_cast<const uint8_t*>(p.ep.Y) +
                                                                   (off + br.dy) * p.ep.ldy * 2)
                               : nullptr;
      const bool track = track_launch && (p.ep.absmax_blocks != 2 || br.track != 0);
      if (track_launch && amax_block != tc.z) {
        if (amax_block >= 0) flush_amax(amax_block);
        amax_block = tc.z;
      }
      const int r0 = tc.x + 128 * static_cast<int>(rank) + 32 * ew;
      // chunks of this warp's 32 rows that lie on or above the diagonal and inside n
      const int ch_begin = max(0, (r0 - tc.y) >> 5);
      const int ch_end = r0 < n ? min((tc.w + 31) >> 5, (n - tc.y + 31) >> 5) : ch_begin;
      uint4 ynext[4] = {};
      if (EPI == EPI_POLY && ch_begin + ch_first < ch_end)
        load_y_chunk(Yb, p.ep.ldy, n, r0, tc.y + 32 * (ch_begin + ch_first), lane, ynext);
      if (!wait_bounded(tfull_bar(acc), acc_ph, abort_flag)) break;
      tc_fence_after();
      const float lam = EPI == EPI_FINAL ? static_cast<float>(br.st->lambda) : 0.f;
      // shares at the launch position t, or (a served request) at its tile's
      // position in the request's own list, t + cres_shift
      double* cdst = nullptr;
      if (EPI == EPI_FINAL)
        cdst = p.ep.cres ? p.ep.cres + 2 * EW * static_cast<int64_t>(t) + EW * static_cast<int>(rank)
               : br.cres ? br.cres + 2 * EW * (static_cast<int64_t>(t) + br.cres_shift) + EW * static_cast<int>(rank)
                         : nullptr;
      ComplAcc cacc;
      ComplAcc* cap = cdst ? &cacc : nullptr;
#pragma unroll 1
      for (int ch = ch_begin + ch_first; ch < ch_end; ch += kChStep) {
        const int c0 = tc.y + 32 * ch;
        uint4 ycur[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) ycur[k] = ynext[k];
        if (EPI == EPI_POLY && ch + kChStep < ch_end)
          load_y_chunk(Yb, p.ep.ldy, n, r0, c0 + 32 * kChStep, lane, ynext);
        uint32_t v[32];
        tmem_ld32(tmem_base + (static_cast<uint32_t>(32 * ew) << 16) + acc * kBN + 32 * ch, v);
        if (EPI == EPI_FINAL)
          epilogue_chunk_final(br, r0, c0, v, wbuf, lane, lam, cap);
        else
          epilogue_chunk16<EPI, false, OUTK>(p, br, bf16, n, C, C_lo, r0, c0, v, wbuf, ycur, lane, track,
                                             amax_bits);
      }
      if (EPI == EPI_FINAL && cdst) {
        const double cs = compl_warp_sum(cacc);
        if (lane == 0) cdst[EW == 4 ? ew : ewi] = cs;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (leader)
          mbar_arrive(tempty_bar(acc));
        else
          mbar_arrive_remote(tempty_leader[acc]);
      }
      acc ^= 1u;
      if (acc == 0) acc_ph ^= 1u;
    }
    if (EPI != EPI_FINAL && track_launch && amax_block >= 0) flush_amax(amax_block);
  }

  // every operand read, remote arrival and copy of the pair is complete
  // before either CTA releases tensor memory or exits
  tc_fence_before();
  cluster_sync_all();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc_pair(tmem_base, kTmemCols);
  }
  if (threadIdx.x == 0 && *abort_flag) raise_status(p.ep.status, PSD_ERR_TIMEOUT);
}

// ------------------------------------------------------------ chain form
// All 16-bit products of a block-diagonal cone's chain in one persistent
// launch (launch_symgemm_chain).  Roles, ring and per-tile arithmetic are
// those of symgemm16_kernel with 8 epilogue warps, so every output is
// bit-identical to one launch per product; what changes is that a CTA goes
// on to its tiles of the next product without waiting for the whole grid:
// a block's next product starts as soon as that block's previous product is
// written, so small blocks run ahead while large blocks' tiles are in flight,
// and no launch boundary leaves SMs idle behind the slowest tile.

// Spins until *ctr >= target; false (and *abort raised) after kWaitLimitNs.
__device__ __forceinline__ bool wait_count(const int* ctr, int target, volatile int* abort) {
  if (ld_acquire_gpu(ctr) >= target) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (true) {
    if (ld_acquire_gpu(ctr) >= target) return true;
    if (*abort) return false;
    if (globaltimer_ns() - t0 > kWaitLimitNs) {
      *abort = 1;
      return false;
    }
    __nanosleep(64);
  }
}

template <int EW>
__global__ void __launch_bounds__(threads16(EW), 1)
    symgemm16_chain_kernel(const __grid_constant__ ChainMaps maps, const ChainProduct* __restrict__ prods,
                           const int nprod, const GemmParams p, int* done, const int bf16_flag) {
  constexpr int kStages16 = stages16(EW);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint8_t* stages = smem;
  uint8_t* epi_stg = smem + kStages16 * kStageBytes16;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages16 * kStageBytes16 + EW * kEpiWarpBytes);
  // bars: full[S] | empty[S] | tfull[2] | tempty[2] | drain
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * kStages16 + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const bool bf16 = bf16_flag != 0;
  auto full_bar = [&](int s) { return smem_u32(bars + s); };
  auto empty_bar = [&](int s) { return smem_u32(bars + kStages16 + s); };
  auto tfull_bar = [&](int a) { return smem_u32(bars + 2 * kStages16 + a); };
  auto tempty_bar = [&](int a) { return smem_u32(bars + 2 * kStages16 + 2 + a); };
  const uint32_t drain_bar = smem_u32(bars + 2 * kStages16 + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages16; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), EW);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
    for (int k = 0; k < nprod; ++k) {
      tma_prefetch_desc(&maps.m[prods[k].ma]);
      tma_prefetch_desc(&maps.m[prods[k].mb]);
    }
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_holder), kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {
      int last_parity[kStages16];
      for (int s = 0; s < kStages16; ++s) last_parity[s] = -1;
      uint32_t s = 0, ph = 0;
      bool ok = true;
      for (int k = 0; ok && k < nprod; ++k) {
        const CUtensorMap* tmA = &maps.m[prods[k].ma];
        const CUtensorMap* tmB = &maps.m[prods[k].mb];
        for (int t = blockIdx.x; ok && t < p.num_tiles; t += gridDim.x) {
          const int4 tc = p.tiles[t];
          const BlockRec& bz = p.blocks[tc.z];
          const int kbn = (bz.n + kBK16 - 1) / kBK16;
          const int ya = static_cast<int>(bz.off + tc.x), yb = static_cast<int>(bz.off + bz.db + tc.y);
          if (k > 0) {  // the block's previous product is written (by any CTA)
            if (!wait_count(done + static_cast<int64_t>(tc.z) * nprod + k - 1, tile_count_of_order(bz.n),
                            abort_flag)) {
              ok = false;
              break;
            }
            fence_proxy_async_global();
          }
          for (int kb = 0; kb < kbn; ++kb) {
            if (!wait_bounded(empty_bar(s), ph ^ 1u, abort_flag)) {
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(full_bar(s), kStageBytes16);
            const uint32_t a_dst = smem_u32(stages + s * kStageBytes16);
            tma_load_2d(a_dst, tmA, kb * kBK16, ya, full_bar(s));
            tma_load_2d(a_dst + kABytes16, tmB, kb * kBK16, yb, full_bar(s));
            last_parity[s] = static_cast<int>(ph);
            if (++s == kStages16) {
              s = 0;
              ph ^= 1u;
            }
          }
        }
      }
      if (!ok) {
        for (int q = 0; q < kStages16; ++q)
          if (last_parity[q] >= 0) {
            const unsigned long long t0 = globaltimer_ns();
            while (!mbar_try_wait(full_bar(q), static_cast<uint32_t>(last_parity[q])) &&
                   globaltimer_ns() - t0 < kWaitLimitNs) {
            }
          }
      }
    }
  } else if (warp == 1) {
    uint32_t s = 0, ph = 0, acc = 0, acc_ph = 0;
    bool ok = true;
    for (int k = 0; ok && k < nprod; ++k) {
      for (int t = blockIdx.x; ok && t < p.num_tiles; t += gridDim.x) {
        const int4 tc = p.tiles[t];
        const int kbn = (p.blocks[tc.z].n + kBK16 - 1) / kBK16;
        const uint32_t idesc = p.idesc | (static_cast<uint32_t>(tc.w >> 3) << 17);
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
            const uint32_t a_addr = smem_u32(stages + s * kStageBytes16);
            const uint32_t b_addr = a_addr + kABytes16;
#pragma unroll
            for (int q = 0; q < kRowBytes16 / 32; ++q)
              mma_f16(d_tmem, sw128_kmajor_desc(a_addr + 32 * q), sw128_kmajor_desc(b_addr + 32 * q), idesc,
                      (kb | q) != 0 ? 1u : 0u);
            mma_commit(empty_bar(s));
          }
          __syncwarp();
          if (++s == kStages16) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
        if (lane == 0) mma_commit(tfull_bar(acc));
        __syncwarp();
        acc ^= 1u;
        if (acc == 0) acc_ph ^= 1u;
      }
    }
    if (!ok && lane == 0) {
      mma_commit(drain_bar);
      const unsigned long long t0 = globaltimer_ns();
      while (!mbar_try_wait(drain_bar, 0) && globaltimer_ns() - t0 < kWaitLimitNs) {
      }
    }
    __syncwarp();
  } else {
    const int ew = warp & 3;         // tensor-memory lane quarter
    const int ewi = warp - 2;        // epilogue warp 0 .. EW - 1
    constexpr int kChStep = EW / 4;  // chunks of a quarter, dealt to its EW / 4 warps
    const int ch_first = ewi / 4;
    uint8_t* wbuf = epi_stg + ewi * kEpiWarpBytes;
    uint32_t acc = 0, acc_ph = 0;
    unsigned amax_bits = 0;
    int amax_block = -1;
    auto flush_amax = [&](int blk) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) amax_bits = max(amax_bits, __shfl_xor_sync(0xffffffffu, amax_bits, o));
      if (lane == 0 && amax_bits) atomicMax(&p.blocks[blk].st->absmax_bits, amax_bits);
      amax_bits = 0;
    };
    bool ok = true;
    for (int k = 0; ok && k < nprod; ++k) {
      const ChainProduct cp = prods[k];
      GemmParams q = p;  // the product's coefficients for the shared epilogue code
      q.ep.a = cp.a;
      q.ep.b = cp.b;
      q.ep.c = cp.c;
      q.ep.s = cp.s;
      const bool track = cp.track != 0;
      for (int t = blockIdx.x; t < p.num_tiles; t += gridDim.x) {
        const int4 tc = p.tiles[t];
        const BlockRec& br = p.blocks[tc.z];
        const int n = br.n;
        const int64_t off = br.off;
        void* C = cp.epi == EPI_FINAL ? nullptr : static_cast<uint8_t*>(cp.C) + (off + br.dc) * p.ep.ldc * 2;
        const uint16_t* Yb = cp.epi == EPI_POLY
                                 ? reinterpret_cast<const uint16_t*>(static_cast<const uint8_t*>(cp.Y) +
                                                                     (off + br.dy) * p.ep.ldy * 2)
                                 : nullptr;
        if (track && amax_block != tc.z) {
          if (amax_block >= 0) flush_amax(amax_block);
          amax_block = tc.z;
        }
        const int r0 = tc.x + 32 * ew;
        const int ch_begin = max(0, (r0 - tc.y) >> 5);
        const int ch_end = r0 < n ? min((tc.w + 31) >> 5, (n - tc.y + 31) >> 5) : ch_begin;
        uint4 ynext[4] = {};
        if (cp.epi == EPI_POLY && ch_begin + ch_first < ch_end)
          load_y_chunk(Yb, p.ep.ldy, n, r0, tc.y + 32 * (ch_begin + ch_first), lane, ynext);
        if (!wait_bounded(tfull_bar(acc), acc_ph, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const float lam = cp.epi == EPI_FINAL ? static_cast<float>(br.st->lambda) : 0.f;
        double* cdst = cp.epi == EPI_FINAL && p.ep.cres ? p.ep.cres + 8 * static_cast<int64_t>(t) + ewi : nullptr;
        ComplAcc cacc;
        ComplAcc* cap = cdst ? &cacc : nullptr;
#pragma unroll 1
        for (int ch = ch_begin + ch_first; ch < ch_end; ch += kChStep) {
          const int c0 = tc.y + 32 * ch;
          uint4 ycur[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) ycur[i] = ynext[i];
          if (cp.epi == EPI_POLY && ch + kChStep < ch_end)
            load_y_chunk(Yb, p.ep.ldy, n, r0, c0 + 32 * kChStep, lane, ynext);
          uint32_t v[32];
          tmem_ld32(tmem_base + (static_cast<uint32_t>(32 * ew) << 16) + acc * kBN + 32 * ch, v);
          if (cp.epi == EPI_COPY)
            epilogue_chunk16<EPI_COPY, false, 0>(q, br, bf16, n, C, nullptr, r0, c0, v, wbuf, ycur, lane, track,
                                                 amax_bits);
          else if (cp.epi == EPI_POLY)
            epilogue_chunk16<EPI_POLY, false, 0>(q, br, bf16, n, C, nullptr, r0, c0, v, wbuf, ycur, lane, track,
                                                 amax_bits);
          else if (cp.epi == EPI_SCALE)
            epilogue_chunk16<EPI_SCALE, false, 0>(q, br, bf16, n, C, nullptr, r0, c0, v, wbuf, ycur, lane, track,
                                                  amax_bits);
          else
            epilogue_chunk_final(br, r0, c0, v, wbuf, lane, lam, cap);
        }
        if (cdst) {
          const double cs = compl_warp_sum(cacc);
          if (lane == 0) *cdst = cs;
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty_bar(acc));
        acc ^= 1u;
        if (acc == 0) acc_ph ^= 1u;
        if (k + 1 < nprod) {
          // publish the tile: every epilogue warp's stores, then one increment
          __threadfence();
          fence_proxy_async_global();
          asm volatile("bar.sync 1, %0;" ::"n"(32 * EW) : "memory");
          if (ewi == 0 && lane == 0) red_release_add_gpu(done + static_cast<int64_t>(tc.z) * nprod + k, 1);
        }
      }
      if (track && amax_block >= 0) flush_amax(amax_block);
      amax_block = -1;
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
  if (threadIdx.x == 0 && *abort_flag) raise_status(p.ep.status, PSD_ERR_TIMEOUT);
}

using Kernel16 = void (*)(const CUtensorMap, const CUtensorMap, const GemmParams, const int);

// Instances: 16-bit operands with 16-bit output (every epilogue); e4m3
// operands with e4m3 output (the FP8 stages); e4m3 operands with 16-bit output
// and 16-bit operands with e4m3 output (EPI_SCALE only: the last FP8 stage and
// the stage before the first one); FP16 operands with an FP16 pair output
// (EPI_COPY: Y = X^2 of the mixed precision's pair stages).
// With 8 epilogue warps: 16-bit operands with a 16-bit or FP16-pair output,
// COPY / POLY / SCALE.
Kernel16 kernel16_for8(int epi, int outk) {
  if (outk == 0)
    return epi == EPI_COPY    ? symgemm16_kernel<EPI_COPY, false, 0, 8>
           : epi == EPI_POLY  ? symgemm16_kernel<EPI_POLY, false, 0, 8>
           : epi == EPI_SCALE ? symgemm16_kernel<EPI_SCALE, false, 0, 8>
                              : nullptr;
  if (outk == 2)
    return epi == EPI_COPY ? symgemm16_kernel<EPI_COPY, false, 2, 8>
           : epi == EPI_POLY ? symgemm16_kernel<EPI_POLY, false, 2, 8>
                             : nullptr;
  return nullptr;
}

Kernel16 kernel16_for(int epi, bool in8, int outk) {
  if (!in8 && outk == 0) {
    switch (epi) {
      case EPI_COPY: return symgemm16_kernel<EPI_COPY, false, 0>;
      case EPI_POLY: return symgemm16_kernel<EPI_POLY, false, 0>;
      case EPI_SCALE: return symgemm16_kernel<EPI_SCALE, false, 0>;
      default: return symgemm16_kernel<EPI_FINAL, false, 0>;
    }
  }
  if (in8 && outk == 1) {
    switch (epi) {
      case EPI_COPY: return symgemm16_kernel<EPI_COPY, true, 1>;
      case EPI_POLY: return symgemm16_kernel<EPI_POLY, true, 1>;
      case EPI_SCALE: return symgemm16_kernel<EPI_SCALE, true, 1>;
      default: return nullptr;
    }
  }
  if (!in8 && outk == 2)
    return epi == EPI_COPY ? symgemm16_kernel<EPI_COPY, false, 2>
           : epi == EPI_POLY ? symgemm16_kernel<EPI_POLY, false, 2>
                             : nullptr;
  if (epi != EPI_SCALE) return nullptr;
  return in8 ? symgemm16_kernel<EPI_SCALE, true, 0> : symgemm16_kernel<EPI_SCALE, false, 1>;
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                              CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                              CUtensorMapFloatOOBfill);

// Resolved once (a function-local static: thread-safe initialisation; the
// request server's thread and callers' threads encode maps concurrently).
EncodeFn get_encode() {
  static const EncodeFn fn = [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeFn>(ptr);
    return static_cast<EncodeFn>(nullptr);
  }();
  return fn;
}

}  // namespace

int num_sms() {
  static const int sms = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return sms;
}

// Tensor map of an n x n symmetric operand with row stride ld elements.  The
// box is row_bytes (128 or 64) bytes of K -- one swizzle row, 128- or 64-byte
// swizzle -- by box_rows rows; boxes that reach past n are zero-filled by the
// TMA unit.
bool encode_tmap(CUtensorMap* map, int dtype, const void* base, int64_t n, int64_t ld, int box_rows,
                 int row_bytes) {
  EncodeFn fn = get_encode();
  if (!fn) return false;
  const int esz = dtype == DT_TF32X3 ? 4 : (dtype == DT_E4M3 ? 1 : 2);
  const CUtensorMapDataType dt = (dtype == DT_F16 || dtype == DT_F16X2) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                 : dtype == DT_BF16                     ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                 : dtype == DT_E4M3                     ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  if (row_bytes != 128 && row_bytes != 64) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(n)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * esz};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(row_bytes / esz), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE,
                  row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Tensor map of a stacked buffer of `rows` rows (row stride ld elements) of
// which the first `cols` columns are addressed; same boxes as encode_tmap.
bool encode_tmap_rows(CUtensorMap* map, int dtype, const void* base, int64_t cols, int64_t rows, int64_t ld,
                      int box_rows, int row_bytes) {
  EncodeFn fn = get_encode();
  if (!fn) return false;
  const int esz = dtype == DT_TF32X3 ? 4 : (dtype == DT_E4M3 ? 1 : 2);
  const CUtensorMapDataType dt = (dtype == DT_F16 || dtype == DT_F16X2) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                 : dtype == DT_BF16                     ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                 : dtype == DT_E4M3                     ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  if (row_bytes != 128 && row_bytes != 64) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * esz};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(row_bytes / esz), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Upper-triangle tiles of 256 x 256 blocks, each split into two 128-row
// tiles, in a grouped raster: block rows are taken in groups of `group` (8),
// and inside
// a group the columns advance first so that the tiles resident at one time
// share their operand panels in L2.  The lower tile of a diagonal block only
// needs its right half (columns >= its first row), and every tile is trimmed
// to the columns below n (rounded up to 16, the MMA's N granularity).
std::vector<int4> make_tile_list(int64_t n, int block, int group) {
  std::vector<int4> tiles;
  const int nb = static_cast<int>((n + kBN - 1) / kBN);
  const int G = group > 0 ? group : 8;
  auto width = [&](int n0, int w) { return std::min(w, static_cast<int>((n - n0 + 15) / 16 * 16)); };
  for (int g0 = 0; g0 < nb; g0 += G) {
    for (int J = g0; J < nb; ++J) {
      const int iend = std::min(g0 + G, J + 1);
      for (int I = g0; I < iend; ++I) {
        for (int h = 0; h < 2; ++h) {
          const int m0 = I * kBN + h * kBM;
          if (m0 >= n) continue;
          if (I == J && h == 1)
            tiles.push_back(make_int4(m0, m0, block, width(m0, kBM)));
          else
            tiles.push_back(make_int4(m0, J * kBN, block, width(J * kBN, kBN)));
        }
      }
    }
  }
  return tiles;
}

// Tiles of the pair form: every 256 x 256 upper block (I <= J) as one 256-row
// tile, in the same grouped raster; widths trimmed to the columns below n,
// rounded up to 32 (N/2 rows of B per CTA; the extra columns read zero-filled
// rows and are not written).
std::vector<int4> make_tile_list_pair(int64_t n, int block, int group) {
  std::vector<int4> tiles;
  const int nb = static_cast<int>((n + kBN - 1) / kBN);
  const int G = group > 0 ? group : 8;
  for (int g0 = 0; g0 < nb; g0 += G)
    for (int J = g0; J < nb; ++J) {
      const int iend = std::min(g0 + G, J + 1);
      for (int I = g0; I < iend; ++I)
        tiles.push_back(make_int4(I * kBN, J * kBN, block, std::min(kBN, static_cast<int>((n - J * kBN + 31) / 32 * 32))));
    }
  return tiles;
}

cudaError_t launch_symgemm_pair(int dtype, int epi, const CUtensorMap& tmA, const CUtensorMap& tmB,
                                const GemmParams& p, int grid, cudaStream_t stream, int out_dtype, bool many_small) {
  if (p.num_tiles == 0) return cudaSuccess;
  if (dtype != DT_F16 && dtype != DT_BF16) return cudaErrorNotSupported;
  if (out_dtype < 0) out_dtype = dtype;
  const int outk = out_dtype == DT_F16X2 ? 2 : 0;
  if ((outk == 2 && dtype != DT_F16) || (outk == 0 && out_dtype != dtype)) return cudaErrorNotSupported;
  Kernel16 k = nullptr;
  if (outk == 0)
    k = epi == EPI_COPY    ? symgemm16_pair_kernel<EPI_COPY, 0>
        : epi == EPI_POLY  ? symgemm16_pair_kernel<EPI_POLY, 0>
        : epi == EPI_SCALE ? symgemm16_pair_kernel<EPI_SCALE, 0>
        : epi == EPI_FINAL ? symgemm16_pair_kernel<EPI_FINAL, 0>
                           : nullptr;
  else
    k = epi == EPI_COPY ? symgemm16_pair_kernel<EPI_COPY, 2> : epi == EPI_POLY ? symgemm16_pair_kernel<EPI_POLY, 2> : nullptr;
  const int ew = many_small && outk == 0 ? 8 : 4;
  if (ew == 8)
    k = epi == EPI_COPY    ? symgemm16_pair_kernel<EPI_COPY, 0, 8>
        : epi == EPI_POLY  ? symgemm16_pair_kernel<EPI_POLY, 0, 8>
        : epi == EPI_SCALE ? symgemm16_pair_kernel<EPI_SCALE, 0, 8>
        : epi == EPI_FINAL ? symgemm16_pair_kernel<EPI_FINAL, 0, 8>
                           : nullptr;
  if (!k) return cudaErrorNotSupported;
  static std::mutex attr_mu;
  static Kernel16 attr_done[16] = {};
  {
    std::lock_guard<std::mutex> lk(attr_mu);
    bool set = false;
    for (Kernel16 d : attr_done) set = set || d == k;
    if (!set) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes_pair(ew));
      if (e != cudaSuccess) return e;
      for (Kernel16& d : attr_done)
        if (!d) {
          d = k;
          break;
        }
    }
  }
  const int pairs = std::max(1, std::min(grid / 2, p.num_tiles));
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(2 * pairs);
  cfg.blockDim = dim3(threads16(ew));
  cfg.dynamicSmemBytes = smem_bytes_pair(ew);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, tmA, tmB, p, out_dtype == DT_BF16 ? 1 : 0);
}

cudaError_t launch_symgemm_chain(int dtype, const ChainMaps& maps, const ChainProduct* prods, int nprod,
                                 const GemmParams& p, int* done, int grid, cudaStream_t stream) {
  if (p.num_tiles == 0 || nprod <= 0) return cudaSuccess;
  if (dtype != DT_F16 && dtype != DT_BF16) return cudaErrorNotSupported;
  constexpr int kEW = 8;
  auto k = symgemm16_chain_kernel<kEW>;
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [&] {
    attr_err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes16(kEW));
  });
  if (attr_err != cudaSuccess) return attr_err;
  // one CTA per SM (its shared memory allows no second), all resident: the
  // cooperative launch fails rather than leave a CTA waiting for an SM
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(std::max(1, std::min(grid, p.num_tiles)));
  cfg.blockDim = dim3(threads16(kEW));
  cfg.dynamicSmemBytes = smem_bytes16(kEW);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, maps, prods, nprod, p, done, dtype == DT_BF16 ? 1 : 0);
}

cudaError_t launch_symgemm(int dtype, int epi, const CUtensorMap& tmA, const CUtensorMap& tmB,
                           const GemmParams& p, int grid, cudaStream_t stream, int out_dtype, bool many_small) {
  if (p.num_tiles == 0) return cudaSuccess;
  if (dtype != DT_F16 && dtype != DT_BF16 && dtype != DT_E4M3) return cudaErrorNotSupported;
  if (out_dtype < 0) out_dtype = dtype;
  if (epi < EPI_COPY || epi > EPI_FINAL) return cudaErrorInvalidValue;
  const bool in8 = dtype == DT_E4M3;
  const int outk = epi == EPI_FINAL ? 0 : out_dtype == DT_E4M3 ? 1 : out_dtype == DT_F16X2 ? 2 : 0;
  if (outk == 2 && dtype != DT_F16) return cudaErrorNotSupported;
  // 8 epilogue warps where the launch has one (the final product keeps 4: its
  // per-warp shares of <out, X - out> are four per tile)
  Kernel16 k8 = many_small && !in8 ? kernel16_for8(epi, outk) : nullptr;
  const int ew = k8 ? 8 : 4;
  Kernel16 k = k8 ? k8 : kernel16_for(epi, in8, outk);
  if (!k) return cudaErrorNotSupported;
  static std::mutex attr_mu;  // launches come from callers' threads and the request server's
  static bool attr_set[48] = {};
  const int idx = (epi * 6 + (in8 ? 3 : 0) + outk) * 2 + (ew == 8 ? 1 : 0);
  const int smem = smem_bytes16(ew);
  {
    std::lock_guard<std::mutex> lk(attr_mu);
    if (!attr_set[idx]) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      attr_set[idx] = true;
    }
  }
  const int g = std::max(1, std::min(grid, p.num_tiles));
  k<<<g, threads16(ew), smem, stream>>>(tmA, tmB, p, out_dtype == DT_BF16 ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace psd
