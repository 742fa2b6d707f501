// Internal declarations shared by the translation units of libpsdproj.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "psdproj.h"

namespace psd {

constexpr int kMaxSteps = 20;     // Lanczos steps (Sec. 3.4, Algorithm 2)
constexpr int kMaxStages = 10;    // T <= 10 (Table 1)
constexpr int kSymvTile = 128;    // Lanczos mat-vec tile
constexpr int kVecThreads = 256;  // elements (threads) per block of the Lanczos vector phases
constexpr int64_t kMaxOrder = 131072;
constexpr double kBreakdown = 1e-12;       // beta_j <= 1e-12 ||X||_F^2: invariant subspace
constexpr float kOvershootLimit = 1.01f;   // max |X_T(i,j)| above this: bound too small

// Caller pointers read by the kernels of a captured graph.  A tiny kernel
// launched (with these as parameters) in front of each graph replay writes it.
struct DevArgs {
  const float* X;
  int64_t ld;
  float* out;
  int64_t ld_out;
  psd_info_t* info;
};

struct BlockRec;

// Device-resident state of one projection.
struct DevState {
  double alpha[kMaxSteps];
  double beta[kMaxSteps];
  double y[kMaxSteps];   // Ritz vector in the Lanczos basis
  double sigma;
  double resid;
  double lambda;         // lam~
  double fro;            // ||X||_F
  double maxdiag;
  double inv_lambda;     // 1 / lam~ (0 when lam~ == 0)
  int m;                 // Lanczos steps taken
  int done;              // breakdown reached
  int status;            // first psd_status_t raised on the device
  unsigned maxdiag_bits; // max |X_ii| as float bits (atomicMax)
  unsigned absmax_bits;  // max |X_T(i,j)| as float bits (atomicMax)
  int pad;
};

// Epilogue kinds of the symmetric product (fused into the tensor-core kernel).
enum Epi : int { EPI_COPY = 0, EPI_POLY = 1, EPI_SCALE = 2, EPI_FINAL = 3 };

// Operand storage of the chain: single 16-bit or e4m3 matrices, TF32 hi/lo
// pairs (FP32 containers), FP16 hi/lo pairs.
// Element types; the X2/X3 names are hi/lo pairs (DT_F16X2: FP16 hi + FP16 lo).
enum Dtype : int { DT_F16 = 0, DT_BF16 = 1, DT_TF32X3 = 2, DT_E4M3 = 4, DT_F16X2 = 5 };

// One symmetric matrix of a product launch.  A launch covers one matrix
// (single projection) or many (block-diagonal cone, served requests); the
// iterates of block b occupy rows off .. off + n - 1 of the stacked buffers.
struct BlockRec {
  int64_t off;          // first row in the stacked iterate buffers
  int n;                // order
  int track;            // absmax_blocks == 2: track max |output| of this block
  const float* X;       // EPI_FINAL: caller input (upper triangle), column-major
  int64_t ld;
  float* out;           // EPI_FINAL: caller output
  int64_t ld_out;
  DevState* st;         // lam~, and the max |X_T| of the last stage
  float ca, cb, cc, cs; // per-block stage coefficients (EpiParams::per_block_coef)
  // Row offsets of the B operand, the output C and the EPI_POLY operand Y,
  // relative to `off` (the A operand's first row).  Zero when every operand of
  // the block sits at the same rows of its own buffer.
  int64_t db, dc, dy;
  // EPI_FINAL with EpiParams::cres unset: if set, the shares of <out, X - out>
  // of the tile at launch position t go to cres at the tile's position in the
  // request's own tile list, t + cres_shift (a served request; 4 per 128-row
  // tile, 8 per tile on SM pairs: 4 (2 (t + cres_shift) + rank) + warp).
  double* cres;
  int64_t cres_shift;
};

struct EpiParams {
  void* C;               // output iterate (ld = ldc), hi part of a pair
  int64_t ldc;
  void* C_lo;            // lo part of a pair output
  const void* Y;         // EPI_POLY: the stage's X^2 (same storage as C)
  const void* Y_lo;
  int64_t ldy;
  float a, b, c, s;      // EPI_POLY coefficients, EPI_SCALE factor
  int absmax_blocks;     // 1: atomic max of |output| into blocks[b].st->absmax_bits;
                         // 2: the same for the blocks with a nonzero `track`
  int per_block_coef;    // nonzero: a, b, c, s from each tile's block record
  // e4m3 operands / outputs (the 16-bit kernel's FP8 instances): every e4m3
  // matrix holds its values times a power of two; the accumulator is
  // multiplied by in_scale = 1 / (scale_A scale_B), the EPI_POLY operand Y by
  // y_scale = 1 / scale_Y, and an e4m3 output is rounded from value * out_scale.
  float in_scale, y_scale, out_scale;
  unsigned* absmax;      // if set: atomic max of |output| into this word instead
  int* status;           // device status word for timeouts
  double* cres;         // EPI_FINAL, if set: tile t's epilogue warp w writes its share of
                         // <out, X - out> to cres[4 t + w]
};

// Share of <out, X - out> (whole symmetric matrix) of upper-triangle element
// (r, c) with output o and input x: weight 1 on the diagonal, 2 above it (the
// element stands for (c, r) too).  Per-thread double-float sum: the rounded
// product and its FMA error are added with TwoSum, so the cancellation of the
// total (zero for an exact projection) is resolved far below FP32's rounding.
struct ComplAcc {
  float h = 0.f, l = 0.f;
};
__device__ __forceinline__ void compl_add(ComplAcc& a, float o, float x, float w) {
  const float d = __fsub_rn(x, o);
  const float p = __fmul_rn(o, d);
  const float e = fmaf(o, d, -p);
  const float pw = __fmul_rn(p, w), ew = __fmul_rn(e, w);  // w is 1 or 2: exact
  const float s = __fadd_rn(a.h, pw);
  const float z = __fsub_rn(s, a.h);
  const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, z)), __fsub_rn(pw, z));
  a.h = s;
  a.l = __fadd_rn(a.l, __fadd_rn(err, ew));
}
// Warp sum (fixed order) of the lanes' shares; valid in every lane.
__device__ __forceinline__ double compl_warp_sum(const ComplAcc& a) {
  double v = static_cast<double>(a.h) + static_cast<double>(a.l);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Threads of the CTA that sums a projection's shares of <out, X - out> (the
// single-projection finalize and the request server use the same order, so a
// served request reports the same residual as the direct call).
constexpr int kComplSumThreads = 256;

// Sum of ncompl shares by a CTA of NT threads (fixed order: strided sums per
// thread, warp trees, then the warp sums in order); valid in thread 0.  wsum:
// shared scratch of NT / 32 doubles.
template <int NT>
__device__ __forceinline__ double compl_cta_sum(const double* cres, int ncompl, double* wsum) {
  double v = 0.0;
  for (int i = threadIdx.x; i < ncompl; i += NT) v += cres[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
  __syncthreads();
  v = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) v += wsum[w];
  return v;
}

struct GemmParams {
  int num_tiles;
  const int4* tiles;     // (m0, n0, block, ncols) of each 128-row output tile, upper triangle
  const BlockRec* blocks;
  uint32_t idesc;        // instruction descriptor without its N field
  EpiParams ep;
};

// A tile and the fields of its block that the producer and MMA roles need.
struct TileMeta {
  int4 tc;
  int n;
  int64_t off, db;
};
// The tiles t0, t0 + stride, ... of a persistent role, with their metadata read
// ahead: the tile record two tiles on and the block record of the next tile are
// loaded while the current tile runs (prefetch() before working on cur()).
// Read on demand, the tile record and then its block's record (a dependent
// load) put two global-memory latencies between one tile's last K-step and the
// next tile's first, which tiles with short K loops (a block-diagonal cone's
// blocks) feel at every boundary.
class TileStream {
 public:
  __device__ __forceinline__ TileStream(const GemmParams& p, int t0, int stride)
      : tiles_(p.tiles), blocks_(p.blocks), num_(p.num_tiles), t_(t0), stride_(stride) {
    if (t_ < num_) cur_ = meta(tiles_[t_]);
    if (t_ + stride_ < num_) tc1_ = tiles_[t_ + stride_];
  }
  __device__ __forceinline__ bool valid() const { return t_ < num_; }
  __device__ __forceinline__ int index() const { return t_; }
  __device__ __forceinline__ const TileMeta& cur() const { return cur_; }
  __device__ __forceinline__ void prefetch() {
    if (t_ + 2 * stride_ < num_) tc2_ = tiles_[t_ + 2 * stride_];
    if (t_ + stride_ < num_) nxt_ = meta(tc1_);
  }
  __device__ __forceinline__ void advance() {
    t_ += stride_;
    cur_ = nxt_;
    tc1_ = tc2_;
  }

 private:
  __device__ __forceinline__ TileMeta meta(const int4& tc) const {
    const BlockRec& b = blocks_[tc.z];
    return TileMeta{tc, b.n, b.off, b.db};
  }
  const int4* tiles_;
  const BlockRec* blocks_;
  int num_, t_, stride_;
  TileMeta cur_{}, nxt_{};
  int4 tc1_{}, tc2_{};
};

// Upper-triangle tiles of one order-n matrix: 256 x 256 blocks (I <= J) split
// into two 128-row tiles; the lower-right tile of a diagonal block starts at
// its diagonal (128 columns); tile widths are trimmed at n (multiples of 16).
std::vector<int4> make_tile_list(int64_t n, int block = 0, int group = 8);
// Frees the cached plans of psd_project_batched (device synchronised by the caller).
void release_batched_plans();

// Coefficients of the run-time filter (Tables 1 and 2) and the per-stage
// divisors s_t of Sec. 3.4 for a precision (psdproj.cu).
struct Schedule {
  int T;
  double coef[kMaxStages][3];
  double post[kMaxStages];  // s_t
};
bool get_schedule(psd_precision_t prec, Schedule& s);

// --- host helpers (symgemm.cu) ---
// Bytes of K per operand row in a pipeline stage (one swizzle row) and per
// tensor-map box row, by kernel: the 16-bit / e4m3 product keeps 128-byte
// rows (4 stages of 48 KB; 8 stages of 64-byte rows measured 20% slower); the
// split product with a pair B takes 64-byte rows (4 stages of 48 KB in place
// of 2 of 96 KB: three stages in flight instead of one, 10% faster); with a
// single B, kRowBytesX3Single.
constexpr int kRowBytes16 = 128;
constexpr int kRowBytesX3Single = 128;
inline int x3_row_bytes(bool b_single) { return b_single ? kRowBytesX3Single : 64; }
// row_bytes: bytes of K per box row, 128 (128-byte swizzle) or 64 (64-byte swizzle).
bool encode_tmap(CUtensorMap* map, int dtype, const void* base, int64_t n, int64_t ld, int box_rows,
                 int row_bytes = kRowBytes16);
// dtype: operand type (DT_F16, DT_BF16 or DT_E4M3); out_dtype: type of the
// EPI_COPY/POLY/SCALE output (DT_F16, DT_BF16, DT_E4M3, or DT_F16X2 for an FP16
// pair written to ep.C / ep.C_lo; -1: the operand type).
// many_small: a launch over many small matrices (the blocks of a block-diagonal
// cone, orders <= 1024), run with 8 epilogue warps and a 3-stage ring where an
// instance exists.
cudaError_t launch_symgemm(int dtype, int epi, const CUtensorMap& tmA, const CUtensorMap& tmB,
                           const GemmParams& p, int grid, cudaStream_t stream, int out_dtype = -1,
                           bool many_small = false);
// The same product on CTA pairs (tcgen05.mma.cta_group::2, M = 256): tiles
// from make_tile_list_pair, tmB with 128-row boxes (each CTA loads half of
// B), p.idesc with M = 256; 16-bit operands; EPI_COPY / EPI_POLY / EPI_SCALE
// with a 16-bit (out_dtype = dtype or -1) or FP16-pair output, and EPI_FINAL
// (cres: 8 shares per tile; 16 with many_small).  many_small: 8 epilogue warps
// per CTA and a 5-stage ring (16-bit outputs and EPI_FINAL).
std::vector<int4> make_tile_list_pair(int64_t n, int block = 0, int group = 8);
cudaError_t launch_symgemm_pair(int dtype, int epi, const CUtensorMap& tmA, const CUtensorMap& tmB,
                                const GemmParams& p, int grid, cudaStream_t stream, int out_dtype = -1,
                                bool many_small = false);
// The whole chain of 16-bit products of a block-diagonal cone in ONE
// persistent launch (symgemm.cu): products 0 .. nprod - 1 (prods, device
// memory) over the tile list p.tiles, every CTA taking its tiles of product 0,
// then of product 1, ...  A tile of product k of block b starts loading once
// all tiles of product k - 1 of block b are written: done[b nprod + k - 1]
// counts them (zeroed before the launch), waited on with a bounded spin.  The
// launch is cooperative (all CTAs resident), which with the product-major
// order rules out a wait that never ends.  Each product names its operands
// by tensor map (maps: for slot s, 2 s with 128-row boxes for A and 2 s + 1
// with 256-row boxes for B); EPI_FINAL writes 8 shares per tile position to
// p.ep.cres (8 epilogue warps).
constexpr int kChainMaxSlots = 6;
struct ChainMaps {
  CUtensorMap m[2 * kChainMaxSlots];
};
struct ChainProduct {
  int epi;          // EPI_COPY / POLY / SCALE / FINAL
  int ma, mb;       // tensor maps of A and B
  int track;        // atomic max of |output| per block (absmax_bits)
  void* C;          // 16-bit output slot (stacked rows, ld = p.ep.ldc)
  const void* Y;    // EPI_POLY operand slot
  float a, b, c, s;
};
// Tiles of make_tile_list(n) (any group).
__host__ __device__ inline int tile_count_of_order(int n) {
  const int nb = (n + 255) / 256;
  return nb * (nb + 1) - ((n - (nb - 1) * 256) <= 128 ? 1 : 0);
}
cudaError_t launch_symgemm_chain(int dtype, const ChainMaps& maps, const ChainProduct* prods, int nprod,
                                 const GemmParams& p, int* done, int grid, cudaStream_t stream);
// split-operand product (symgemm_x3.cu); tm = {A_hi, A_lo, B_hi, B_lo};
// out: 0 = split pair, 1 = single FP16, (EPI_FINAL) FP32 to the caller's output.
// Split-operand products: et = DT_TF32X3 (TF32 pairs) or DT_F16X2 (FP16
// pairs); b_single: A is an FP16 pair and B one FP16 matrix.
// pair: FP16 pairs on SM pairs (M = 256; tiles from make_tile_list_pair; every
// tensor map with 128-row boxes), EPI_COPY / POLY / SCALE with a pair output,
// or a single B with EPI_SCALE and an FP16 output.
cudaError_t launch_symgemm_x3(int et, bool b_single, int epi, int out, const CUtensorMap* tm, const GemmParams& p,
                              int grid, cudaStream_t stream, bool pair = false);
int num_sms();

// --- batched projection of a block-diagonal cone (batched_kernels.cu) ---
constexpr int kMaxBatchOrder = 1024;  // largest block order of a batched call

struct BatchBlock {       // per-block record of the batched norm bound and cast
  int n;
  int ntiles;             // mat-vec tiles of the block
  int64_t off;            // first row of the block in the stacked iterate buffers
  int64_t voff;           // element offset of the block's vectors
  int64_t poff;           // float2 offset of the block's partial sums
  int64_t toff;           // offset of the block's per-tile Frobenius sums
  const float* X;         // caller input (upper triangle), column-major
  int64_t ld;
  psd_info_t* info;       // caller report (may be null)
};

struct BatchLanczos {
  const BatchBlock* blk;
  DevState* st;           // one per block
  double* vec64;          // per block: (kMaxSteps + 4) x n  (Lanczos vectors, u, w, q)
  float* vec32;           // per block: 2 x n  (hi / lo of the mat-vec input)
  float2* part;           // per block: 2 x nb x n  (row / column partial sums)
  double* tile_fro;       // per mat-vec tile
  float* xt;              // per mat-vec tile: the block's 128 x 128 tile, packed (64 KB)
  const int* order;       // per-block kernels: CTA i works on block order[i] (largest blocks first,
                          // so that they start in the first wave of CTAs)
  int skip_done;
};

struct BatchCast {
  void* M;                // X_0: stacked iterate buffer (hi part of a pair)
  void* M_lo;
  int64_t ldm;
};

cudaError_t enqueue_batch_norm_bound(const BatchLanczos& L, int count, const int4* symv_items, int nsymv,
                                     cudaStream_t stream);
cudaError_t enqueue_batch_cast(int dtype, const BatchCast& c, const BatchBlock* blk, const DevState* st,
                               const int4* items, int nitems, cudaStream_t stream);
// Work items of the one-launch bound: x = kind | j << 8 | flags.
enum FlowKind : int { FK_INIT = 0, FK_MV = 1, FK_RED = 2, FK_STEP = 3, FK_RITZ = 4, FK_BOUND = 5 };
// FF_STATS: first product (||X||_F, max |X_ii|); FF_SKIP: no work once the
// block broke down; FF_FRO: ||X||_F before the first reduction; FF_RITZ:
// reduction of the residual pass (no done check).
constexpr int FF_STATS = 1 << 16, FF_SKIP = 1 << 17, FF_FRO = 1 << 18, FF_RITZ = 1 << 19;
// The same bound as ONE launch over a list of work items with per-block
// counters (bit-identical): flow = nflow items {kind | j << 8 | flags | tiles
// << 20, block, first symv item (mat-vec items: `tiles` consecutive ones), the
// block's items that must be done first}; ctl = 2 + count words
// (claim counter, abort word, per-block counters), zeroed here.
cudaError_t enqueue_batch_norm_bound_flow(const BatchLanczos& L, const int4* symv_items, int nsymv, const int4* flow,
                                          int nflow, unsigned* ctl, int count, cudaStream_t stream);
// Wait limit of the one-launch bound's dependency waits (psd_debug_set knob 2).
cudaError_t set_batch_flow_limit(unsigned long long ns);
// shares: final-product shares per tile position in cres (4, or 8 from the chain form);
// flow_abort: the one-launch bound's abort word (or null).
cudaError_t enqueue_batch_finalize(const BatchBlock* blk, DevState* st, int count, const double* cres,
                                   const int* cidx, const int2* crange, int shares, const unsigned* flow_abort,
                                   cudaStream_t stream);
bool encode_tmap_rows(CUtensorMap* map, int dtype, const void* base, int64_t cols, int64_t rows, int64_t ld,
                      int box_rows, int row_bytes = kRowBytes16);

// --- norm bound and cast (normbound.cu) ---
// Host-side fault injection (psd_debug_set): knob 1 = factor on lam~, knob 2 =
// grid-barrier wait limit in ns; current device.
cudaError_t set_norm_bound_debug(int knob, double value);
struct LanczosBufs {
  int64_t n, npad;
  int nb;                // 128-blocks
  int ntiles;            // symv tiles nb (nb + 1) / 2
  int nvec_ctas;         // CTAs of the vector kernels (kVecThreads elements each)
  int npart;             // CTAs of the partial-sum reductions (32 elements each)
  double* Qv;            // (kMaxSteps + 1) x npad Lanczos vectors
  double* u;             // npad
  double* w;             // npad
  double* q;             // npad  Ritz vector
  float* vh;             // npad  hi part of the mat-vec input
  float* vl;             // npad  lo part
  float2* P1;            // nb x npad row partials
  float2* P2;            // nb x npad column partials
  float2* dots;          // npart x 32 double-float partial dot products (one chunk of 32 elements each)
  float2* dots2;         // npart x 32 (second Gram-Schmidt pass; slot 31: ||w||^2)
  double* norms;         // max(npart, nvec_ctas) partial squared norms
  double* tile_fro;      // ntiles
  double* zsave = nullptr;  // if set: X q_j of Lanczos step j kept at zsave + j npad (kMaxSteps x npad)
  unsigned* sync;        // 2 words: grid barrier of the persistent kernel (zeroed before each launch)
};
size_t lanczos_bytes(int64_t n);
void lanczos_carve(LanczosBufs& b, int64_t n, uint8_t* base);
// persistent: the whole bound as one cooperative persistent kernel (grid
// barriers between the phases); otherwise 151 launches (kNormBoundLaunches)
// that can share the GPU with other work -- the request server's preparation
// streams run beside product kernels that leave no room for a co-resident
// grid.  Both paths give identical results.
cudaError_t enqueue_norm_bound(const LanczosBufs& b, const DevArgs* args, DevState* st,
                               cudaStream_t stream, bool persistent = true);
// Frees the cached plans of psd_project_deflate (device synchronised by the caller).
void release_deflate_plans();
// X_0 = X / lam~ as `dtype` (DT_F16, DT_BF16, or DT_TF32X3 with M = hi, M_lo = lo).
cudaError_t enqueue_scale_cast(int dtype, const DevArgs* args, const DevState* st, int64_t n,
                               void* M, void* M_lo, int64_t ldm, cudaStream_t stream);
// Argument block of one replay (and the caller fields of a one-block record, if given).
cudaError_t enqueue_set_args(DevArgs* d_args, const DevArgs& h, cudaStream_t stream, BlockRec* blk = nullptr);
cudaError_t enqueue_set_block(BlockRec* d_blk, const BlockRec& v, cudaStream_t stream);
cudaError_t enqueue_state_reset(DevState* st, cudaStream_t stream);
// Status, overshoot and (if cres is set) the complementarity residual from the
// ncompl per-warp shares of the final product.
cudaError_t enqueue_finalize(const DevArgs* args, DevState* st, cudaStream_t stream, const double* cres = nullptr,
                             int ncompl = 0);

// Status and overshoot of the last stage: a non-finite or overshooting X_T
// (max |X_T(i,j)| > kOvershootLimit) turns an OK status into an error; the
// result goes to the state and, if given, the report.
__device__ __forceinline__ void finalize_report(DevState* st, psd_info_t* info) {
  const float amax = __uint_as_float(st->absmax_bits);
  int status = st->status;
  if (status == 0) {
    if (!(amax == amax) || isinf(amax))
      status = PSD_ERR_NONFINITE;
    else if (amax > kOvershootLimit)
      status = PSD_ERR_BOUND;
    st->status = status;
  }
  if (info) {
    info->overshoot_max = static_cast<double>(amax);
    info->status = status;
  }
}

// Kernel launches of one multi-launch enqueue_norm_bound: start vector (2),
// the Lanczos steps (6 each, plus the Frobenius norm in the first), the
// tridiagonal solve, Ritz vector and residual (8).
constexpr int kNormBoundLaunches = 2 + 6 * kMaxSteps + 1 + 8;

}  // namespace psd
