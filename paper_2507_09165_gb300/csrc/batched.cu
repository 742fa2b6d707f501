// Batched projection of a block-diagonal cone: psd_project_batched.
//
// All blocks are projected by one sequence of grouped launches captured in a
// CUDA graph per (device, stream, precision, block orders): the grouped norm
// bound and cast (batched_kernels.cu) and the 3T + 1 tensor-core products,
// each ONE launch over the upper tiles of every block (tiles ordered from the
// largest blocks down).  Iterates are stacked: block b occupies rows
// off_b .. off_b + n_b - 1 of buffers with a common row length ldm =
// round_up(max n_b, 64); the columns n_b .. ldm - 1 of its rows are zeroed once
// and never written, so a tile's K range and its valid outputs only involve
// the block's own entries -- a block's result is bit-identical alone and in
// any batch.
#include <algorithm>
#include <map>
#include <tuple>
#include <mutex>
#include <vector>

#include "chain.h"
#include "internal.h"

namespace psd {
namespace {

struct BatchPlan {
  psd_precision_t prec = PSD_PREC_BF16;
  int count = 0;
  std::vector<int> sizes;
  Schedule sched{};
  int64_t R = 0;     // stacked rows
  int64_t ldm = 0;   // row length of the stacked buffers
  size_t slot_size = 0;
  int nslots = 0;
  uint8_t* ws = nullptr;
  uint8_t* slots = nullptr;
  BatchLanczos L{};
  BlockRec* d_rec = nullptr;
  BatchBlock* d_bb = nullptr;
  DevState* d_st = nullptr;
  int* d_status = nullptr;
  int4* d_tiles = nullptr;
  int ntiles = 0;
  // 256 x 256 tiles on SM pairs (FP16 / BF16 plans), chosen by the autotuner
  // when faster than every schedule of the 128-row tiles
  int4* d_tiles_pair = nullptr;
  int ntiles_pair = 0;
  bool pair = false;
  int4* d_symv = nullptr;
  int nsymv = 0;
  int4* d_cast = nullptr;
  int ncast = 0;
  double* d_cres = nullptr;  // 4 per tile position: shares of <out, X - out> (final product)
  int* d_cidx = nullptr;     // per block, in its own tile order: positions in the tile list
  int2* d_crange = nullptr;  // per block: (first entry of d_cidx, count)
  uint8_t* small = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_tried = false;
  // The chain form (FP16 / BF16): every product of the chain in one persistent
  // launch over the same tile list (launch_symgemm_chain).
  bool chain = false;
  ChainMaps cmaps{};
  ChainProduct* d_prods = nullptr;  // in `small`
  int nprod = 0;
  int* d_done = nullptr;            // count x nprod tile counters, in `small`
  Mat x0{};                         // the cast's output (the chain's X_0)
  // The norm bound as one launch over a work-item list (the default), or as
  // grouped launches (psd_batched_force_bound(0)).
  bool flow = false;
  int4* d_flow = nullptr;           // in `small`
  int nflow = 0;
  unsigned* d_flowctl = nullptr;    // 2 + count words, in `small`
};

std::mutex g_bmu;
std::map<std::tuple<int, cudaStream_t, int, std::vector<int>>, BatchPlan*> g_bplans;

int64_t rup(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

int nslots_for(psd_precision_t prec) { return chain_slots(prec); }

int dt16_for(psd_precision_t prec) { return prec == PSD_PREC_BF16 ? DT_BF16 : DT_F16; }

__global__ void batch_args_kernel(const psd_block_desc_t* __restrict__ d, BlockRec* rec, BatchBlock* bb,
                                  int count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  const psd_block_desc_t x = d[b];
  rec[b].X = x.X;
  rec[b].ld = x.ld;
  rec[b].out = x.out;
  rec[b].ld_out = x.ld_out;
  bb[b].X = x.X;
  bb[b].ld = x.ld;
  bb[b].info = x.info;
}

void free_bplan(BatchPlan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->ws) cudaFree(p->ws);
  if (p->small) cudaFree(p->small);
  delete p;
}

// Schedules of the grouped products: the order in which their tiles are dealt
// to the persistent CTAs (tile t goes to CTA t mod grid).  None changes a
// tile's arithmetic, so every schedule gives bit-identical results; they
// differ in load balance and L2 reuse, which the autotuner measures.
//   order 0: blocks largest first, each block's tiles in its grouped raster;
//   order 1: all tiles by estimated cost (K-steps x width, plus a fixed
//            epilogue share), dealt in boustrophedon rounds of `grid` tiles.
// Index = 3 order + g, raster group kTileGroups[g].
constexpr int kTileGroups[3] = {4, 8, 16};
constexpr int kNumSchedules = 6;

std::vector<int4> schedule_tiles(const std::vector<int>& sizes, int cand, int grid) {
  const int count = static_cast<int>(sizes.size());
  const int order = cand / 3, group = kTileGroups[cand % 3];
  std::vector<int> blocks(count);
  for (int b = 0; b < count; ++b) blocks[b] = b;
  std::stable_sort(blocks.begin(), blocks.end(), [&](int x, int y) { return sizes[x] > sizes[y]; });
  std::vector<int4> tiles;
  for (int b : blocks) {
    std::vector<int4> tl = make_tile_list(sizes[b], b, group);
    tiles.insert(tiles.end(), tl.begin(), tl.end());
  }
  if (order == 0 || grid <= 1) return tiles;
  auto cost = [&](const int4& t) {
    const int64_t k = (sizes[t.z] + 63) / 64;
    return (k + 4) * static_cast<int64_t>(t.w);
  };
  std::stable_sort(tiles.begin(), tiles.end(), [&](const int4& x, const int4& y) { return cost(x) > cost(y); });
  std::vector<int4> out(tiles.size());
  const int64_t T = static_cast<int64_t>(tiles.size());
  for (int64_t r0 = 0, k = 0; r0 < T; r0 += grid, ++k) {
    const int64_t len = std::min<int64_t>(grid, T - r0);
    for (int64_t c = 0; c < len; ++c) out[r0 + c] = tiles[r0 + ((k & 1) ? len - 1 - c : c)];
  }
  return out;
}

// Pair-form tiles: blocks largest first, each block's 256 x 256 tiles in its
// grouped raster (make_tile_list_pair).
std::vector<int4> pair_tiles(const std::vector<int>& sizes) {
  std::vector<int> blocks(sizes.size());
  for (size_t b = 0; b < sizes.size(); ++b) blocks[b] = static_cast<int>(b);
  std::stable_sort(blocks.begin(), blocks.end(), [&](int x, int y) { return sizes[x] > sizes[y]; });
  std::vector<int4> tiles;
  for (int b : blocks) {
    std::vector<int4> tl = make_tile_list_pair(sizes[b], b, 8);
    tiles.insert(tiles.end(), tl.begin(), tl.end());
  }
  return tiles;
}
constexpr int kPairCandidate = kNumSchedules;  // autotune candidate index of the pair form

struct TuneReport {
  int chosen = -1;
  int ncand = 0;
  float ms[kNumSchedules + 1] = {};
};
int g_force_schedule = -1;                                  // for plans built next; -1: autotune
int g_force_form = -1;  // for plans built next: -1 / 0 one launch per product, 1 chain form where it applies
int g_force_bound = -1;  // for plans built next: -1 / 0 grouped launches, 1 the bound in one launch
std::map<std::pair<int, std::vector<int>>, int> g_tuned;   // (precision, order buckets) -> schedule

// Tuning key: the precision and the number of blocks per order bucket
// (n in (2^(k-1), 2^k]), so that batches with the same size profile share a
// choice (every schedule gives the same results, so sharing is always safe).
std::pair<int, std::vector<int>> tune_key(const BatchPlan* p) {
  std::vector<int> hist(12, 0);
  for (int n : p->sizes) {
    int k = 0;
    while ((1 << k) < n && k < 11) ++k;
    ++hist[k];
  }
  return std::make_pair(static_cast<int>(p->prec), hist);
}
TuneReport g_last_tune;

// Work items of the one-launch bound in their global order (the order in which
// CTAs claim them).  Per block: start vector; per Lanczos step j its mat-vec
// tiles, reduction, mat-vec tiles and step; the Ritz vector; the residual's
// tiles, reduction and tiles; the bound.  item.w counts the block's items in
// earlier phases: the new item starts when the block's counter reaches it.
// Within a phase the single-item kinds take the blocks largest first (the
// longest items start first) and the mat-vecs smallest first, so that a large
// block's tiles are claimed last, when its step (claimed first in the phase
// before) is most likely done.
constexpr int kFlowTiles = 4;
std::vector<int4> build_flow(const std::vector<int>& sizes, const std::vector<BatchBlock>& bb,
                             const std::vector<int>& big_first) {
  const int count = static_cast<int>(sizes.size());
  std::vector<int> big_last(big_first.rbegin(), big_first.rend());
  std::vector<int4> flow;
  std::vector<int> done(count, 0);
  auto single = [&](int op) {
    for (int b : big_first) flow.push_back(make_int4(op, b, 0, done[b]));
    for (int b = 0; b < count; ++b) done[b] += 1;
  };
  // mat-vec items: up to kFlowTiles consecutive tiles of a block each
  auto products = [&](int op) {
    for (int b : big_last)
      for (int t = 0; t < bb[b].ntiles; t += kFlowTiles) {
        const int k = std::min(kFlowTiles, bb[b].ntiles - t);
        flow.push_back(make_int4(op | (k << 20), b, static_cast<int>(bb[b].toff) + t, done[b]));
      }
    for (int b = 0; b < count; ++b) done[b] += (bb[b].ntiles + kFlowTiles - 1) / kFlowTiles;
  };
  single(FK_INIT);
  for (int j = 0; j < kMaxSteps; ++j) {
    products(FK_MV | (j << 8) | (j == 0 ? FF_STATS : FF_SKIP));
    single(FK_RED | (j << 8) | (j == 0 ? FF_FRO : 0));
    products(FK_MV | (j << 8) | FF_SKIP);
    single(FK_STEP | (j << 8));
  }
  single(FK_RITZ);
  products(FK_MV);
  single(FK_RED | FF_RITZ);
  products(FK_MV);
  single(FK_BOUND);
  return flow;
}

psd_status_t build_bplan(BatchPlan* p) {
  if (!get_schedule(p->prec, p->sched)) return PSD_ERR_INVALID_ARG;
  const int count = p->count;
  int maxn = 1;
  for (int n : p->sizes) maxn = std::max(maxn, n);
  p->ldm = rup(maxn, 64);
  // host records
  std::vector<BlockRec> rec(count);
  std::vector<BatchBlock> bb(count);
  int64_t off = 0, voff = 0, poff = 0, toff = 0;
  std::vector<int4> symv, cast;
  for (int b = 0; b < count; ++b) {
    const int n = p->sizes[b];
    const int nb = (n + kSymvTile - 1) / kSymvTile;
    rec[b] = BlockRec{};
    rec[b].off = off;
    rec[b].n = n;
    bb[b] = BatchBlock{};
    bb[b].n = n;
    bb[b].ntiles = nb * (nb + 1) / 2;
    bb[b].off = off;
    bb[b].voff = voff;
    bb[b].poff = poff;
    bb[b].toff = toff;
    int t = 0;
    for (int j = 0; j < nb; ++j)
      for (int i = 0; i <= j; ++i) symv.push_back(make_int4(b, i, j, static_cast<int>(toff + t++)));
    const int nc = (n + 63) / 64;
    for (int j = 0; j < nc; ++j)
      for (int i = 0; i <= j; ++i) cast.push_back(make_int4(b, i, j, 0));
    off += n;
    voff += n;
    poff += 2LL * nb * n;
    toff += bb[b].ntiles;
  }
  p->R = off;
  // product tiles of all blocks in the default schedule (the autotuner may reorder them)
  std::vector<int4> tiles = schedule_tiles(p->sizes, 0, num_sms());
  std::vector<int4> tiles_pair = pair_tiles(p->sizes);
  p->ntiles_pair = static_cast<int>(tiles_pair.size());
  p->ntiles = static_cast<int>(tiles.size());
  p->nsymv = static_cast<int>(symv.size());
  p->ncast = static_cast<int>(cast.size());
  // device memory: stacked slots + Lanczos vectors (one allocation, zeroed once)
  p->slot_size = static_cast<size_t>(rup(p->R * p->ldm * 2, 1024));
  p->nslots = nslots_for(p->prec);
  const size_t b_slots = p->nslots * p->slot_size;
  const size_t b_vec64 = rup(sizeof(double) * (kMaxSteps + 4) * voff, 256);
  const size_t b_vec32 = rup(sizeof(float) * 2 * voff, 256);
  const size_t b_part = rup(sizeof(float2) * poff, 256);
  const size_t b_fro = rup(sizeof(double) * std::max<int64_t>(toff, 1), 256);
  const size_t b_xt = sizeof(float) * kSymvTile * kSymvTile * symv.size();
  const size_t total = 1024 + b_slots + b_vec64 + b_vec32 + b_part + b_fro + b_xt;
  if (cudaMalloc(&p->ws, total) != cudaSuccess) {
    cudaGetLastError();
    p->ws = nullptr;
    return PSD_ERR_NO_MEMORY;
  }
  if (cudaMemset(p->ws, 0, total) != cudaSuccess) return PSD_ERR_CUDA;
  uint8_t* base = reinterpret_cast<uint8_t*>(rup(reinterpret_cast<int64_t>(p->ws), 1024));
  p->slots = base;
  uint8_t* q = base + b_slots;
  p->L.vec64 = reinterpret_cast<double*>(q);
  q += b_vec64;
  p->L.vec32 = reinterpret_cast<float*>(q);
  q += b_vec32;
  p->L.part = reinterpret_cast<float2*>(q);
  q += b_part;
  p->L.tile_fro = reinterpret_cast<double*>(q);
  q += b_fro;
  p->L.xt = reinterpret_cast<float*>(q);
  // small records: BlockRec | BatchBlock | DevState | status | tiles | symv items | cast items
  const size_t o_bb = rup(sizeof(BlockRec) * count, 256);
  const size_t o_st = o_bb + rup(sizeof(BatchBlock) * count, 256);
  const size_t o_status = o_st + rup(sizeof(DevState) * count, 256);
  const size_t o_tiles = o_status + 256;
  const size_t o_symv = o_tiles + rup(sizeof(int4) * tiles.size(), 256);
  const size_t o_cast = o_symv + rup(sizeof(int4) * symv.size(), 256);
  const size_t o_cres = o_cast + rup(sizeof(int4) * cast.size(), 256);
  // final-product shares: 4 per tile position (one launch per product), 8 (chain form),
  // 16 per pair tile
  const size_t ncres = std::max<size_t>(std::max(8 * tiles.size(), 16 * tiles_pair.size()), 1);
  const size_t o_cidx = o_cres + rup(sizeof(double) * ncres, 256);
  const size_t o_crange = o_cidx + rup(sizeof(int) * std::max<size_t>(tiles.size(), 1), 256);
  const size_t o_order = o_crange + rup(sizeof(int2) * count, 256);
  constexpr int kMaxProducts = 3 * kMaxStages + 1;
  const size_t o_prods = o_order + rup(sizeof(int) * count, 256);
  const size_t o_done = o_prods + rup(sizeof(ChainProduct) * kMaxProducts, 256);
  const size_t o_tpair = o_done + rup(sizeof(int) * kMaxProducts * count, 256);
  // per-block kernels take the blocks largest first (the longest CTAs start first)
  std::vector<int> order(count);
  for (int b = 0; b < count; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return p->sizes[x] > p->sizes[y]; });
  p->flow = g_force_bound == 1;
  const std::vector<int4> flow = p->flow ? build_flow(p->sizes, bb, order) : std::vector<int4>();
  p->nflow = static_cast<int>(flow.size());
  const size_t o_flow = o_tpair + rup(sizeof(int4) * std::max<size_t>(tiles_pair.size(), 1), 256);
  const size_t o_flowctl = o_flow + rup(sizeof(int4) * std::max<size_t>(flow.size(), 1), 256);
  const size_t smallb = o_flowctl + rup(sizeof(unsigned) * (2 + count), 256);
  if (cudaMalloc(&p->small, smallb) != cudaSuccess) {
    cudaGetLastError();
    p->small = nullptr;
    return PSD_ERR_NO_MEMORY;
  }
  cudaMemset(p->small, 0, smallb);
  p->d_rec = reinterpret_cast<BlockRec*>(p->small);
  p->d_bb = reinterpret_cast<BatchBlock*>(p->small + o_bb);
  p->d_st = reinterpret_cast<DevState*>(p->small + o_st);
  p->d_status = reinterpret_cast<int*>(p->small + o_status);
  p->d_tiles = reinterpret_cast<int4*>(p->small + o_tiles);
  p->d_symv = reinterpret_cast<int4*>(p->small + o_symv);
  p->d_cast = reinterpret_cast<int4*>(p->small + o_cast);
  p->d_cres = reinterpret_cast<double*>(p->small + o_cres);
  p->d_cidx = reinterpret_cast<int*>(p->small + o_cidx);
  p->d_crange = reinterpret_cast<int2*>(p->small + o_crange);
  int* d_order = reinterpret_cast<int*>(p->small + o_order);
  p->d_prods = reinterpret_cast<ChainProduct*>(p->small + o_prods);
  p->d_done = reinterpret_cast<int*>(p->small + o_done);
  p->d_tiles_pair = reinterpret_cast<int4*>(p->small + o_tpair);
  p->d_flow = reinterpret_cast<int4*>(p->small + o_flow);
  p->d_flowctl = reinterpret_cast<unsigned*>(p->small + o_flowctl);
  for (int b = 0; b < count; ++b) rec[b].st = p->d_st + b;
  bool ok = cudaMemcpy(p->d_rec, rec.data(), sizeof(BlockRec) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(p->d_bb, bb.data(), sizeof(BatchBlock) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(p->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice) ==
                cudaSuccess &&
            cudaMemcpy(p->d_symv, symv.data(), sizeof(int4) * symv.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(p->d_cast, cast.data(), sizeof(int4) * cast.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(p->d_tiles_pair, tiles_pair.data(), sizeof(int4) * tiles_pair.size(),
                       cudaMemcpyHostToDevice) == cudaSuccess &&
            (flow.empty() ||
             cudaMemcpy(p->d_flow, flow.data(), sizeof(int4) * flow.size(), cudaMemcpyHostToDevice) == cudaSuccess);
  if (!ok) return PSD_ERR_CUDA;
  p->L.order = d_order;
  p->L.blk = p->d_bb;
  p->L.st = p->d_st;
  p->L.skip_done = 0;
  return PSD_OK;
}

void* bpart(const BatchPlan* p, const Mat& m, int part) {
  return p->slots + (static_cast<size_t>(m.slot) + static_cast<size_t>(part * kind_lo_step(m.kind))) * p->slot_size;
}

// The chain form: run_chain's sequence recorded without launching anything
// (the cast's output and, per product, its epilogue, operands by tensor map,
// output and coefficients).  Applies when every product is a 16-bit product
// with a 16-bit output (FP16, BF16).
struct ChainRecorder {
  BatchPlan* p;
  std::vector<ChainProduct> prods;
  uint32_t encoded = 0;
  bool ok = true;
  Mat x0{};
  int map_of(const Mat& m, int role) {  // role 0: A (128-row boxes), 1: B (256-row boxes)
    if (m.slot < 0 || m.slot >= kChainMaxSlots || m.kind != MK_16) {
      ok = false;
      return 0;
    }
    const int idx = 2 * m.slot + role;
    if (!(encoded & (1u << idx))) {
      if (!encode_tmap_rows(&p->cmaps.m[idx], m.dt16, bpart(p, m, 0), p->ldm, p->R, p->ldm, role ? 256 : 128))
        ok = false;
      encoded |= 1u << idx;
    }
    return idx;
  }
  cudaError_t cast(const Mat& X0) {
    x0 = X0;
    return cudaSuccess;
  }
  cudaError_t gemm(int epi, const Mat& A, const Mat& B, const Mat* out, const Mat* Y, float a, float b, float c,
                   float sc, bool track) {
    if (gemm_route(A, B) != ROUTE_16 || A.kind != MK_16 || (out && out->kind != MK_16) || (Y && Y->kind != MK_16))
      ok = false;
    ChainProduct cp{};
    cp.epi = epi;
    cp.ma = map_of(A, 0);
    cp.mb = map_of(B, 1);
    cp.track = track ? 1 : 0;
    cp.C = out ? bpart(p, *out, 0) : nullptr;
    cp.Y = Y ? bpart(p, *Y, 0) : nullptr;
    cp.a = a;
    cp.b = b;
    cp.c = c;
    cp.s = sc;
    prods.push_back(cp);
    return cudaSuccess;
  }
  cudaError_t finish() { return cudaSuccess; }
};

// Decides the plan's form and, for the chain form, stores the product table.
psd_status_t prepare_chain(BatchPlan* p) {
  p->chain = false;
  if (g_force_form != 1 || p->pair || (p->prec != PSD_PREC_FP16 && p->prec != PSD_PREC_BF16)) return PSD_OK;
  ChainRecorder rec{p};
  if (run_chain(p->prec, p->sched, p->nslots, dt16_for(p->prec), rec) != cudaSuccess || !rec.ok ||
      rec.prods.empty() || rec.prods.size() > static_cast<size_t>(3 * kMaxStages + 1))
    return PSD_OK;  // one launch per product
  for (int b = 0; b < p->count; ++b)  // the counters' targets
    if (static_cast<int>(make_tile_list(p->sizes[b], b, 8).size()) != tile_count_of_order(p->sizes[b]))
      return PSD_OK;
  if (cudaMemcpy(p->d_prods, rec.prods.data(), sizeof(ChainProduct) * rec.prods.size(), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return PSD_ERR_CUDA;
  p->nprod = static_cast<int>(rec.prods.size());
  p->x0 = rec.x0;
  p->chain = true;
  return PSD_OK;
}

// One grouped product over every block's tiles (routes: chain.h gemm_route).
cudaError_t bgemm(BatchPlan* p, int epi, const Mat& A, const Mat& B, const Mat* out, const Mat* Y, float a,
                  float b, float c, float sc, bool track, cudaStream_t s) {
  GemmParams g{};
  g.num_tiles = p->ntiles;
  g.tiles = p->d_tiles;
  g.blocks = p->d_rec;
  g.ep.status = p->d_status;
  g.ep.a = a;
  g.ep.b = b;
  g.ep.c = c;
  g.ep.s = sc;
  g.ep.absmax_blocks = track ? 1 : 0;
  if (epi != EPI_FINAL) {
    g.ep.C = bpart(p, *out, 0);
    g.ep.C_lo = kind_is_pair(out->kind) ? bpart(p, *out, 1) : nullptr;
    g.ep.ldc = p->ldm;
  }
  if (epi == EPI_POLY) {
    g.ep.Y = bpart(p, *Y, 0);
    g.ep.Y_lo = kind_is_pair(Y->kind) ? bpart(p, *Y, 1) : nullptr;
    g.ep.ldy = p->ldm;
  }
  g.ep.in_scale = g.ep.y_scale = g.ep.out_scale = 1.f;
  if (epi == EPI_FINAL) g.ep.cres = p->d_cres;
  const int grid = num_sms();
  const int64_t cols = p->ldm, rows = p->R;
  const GemmRoute route = gemm_route(A, B);
  if (route == ROUTE_16) {
    const int dt = kind_dtype(A);
    CUtensorMap ta, tb;
    if (p->pair && (dt == DT_F16 || dt == DT_BF16) && (epi == EPI_FINAL || kind_dtype(*out) == dt)) {
      // 256 x 256 tiles on SM pairs: each CTA stages 128 rows of A and half of B
      if (!encode_tmap_rows(&ta, dt, bpart(p, A, 0), cols, rows, p->ldm, 128) ||
          !encode_tmap_rows(&tb, dt, bpart(p, B, 0), cols, rows, p->ldm, 128))
        return cudaErrorInvalidValue;
      g.num_tiles = p->ntiles_pair;
      g.tiles = p->d_tiles_pair;
      const uint32_t fmt = dt == DT_BF16 ? 1u : 0u;
      g.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (16u << 24);  // M = 256; N per tile
      return launch_symgemm_pair(dt, epi, ta, tb, g, grid, s, -1, /*many_small=*/true);
    }
    if (!encode_tmap_rows(&ta, dt, bpart(p, A, 0), cols, rows, p->ldm, 128) ||
        !encode_tmap_rows(&tb, dt, bpart(p, B, 0), cols, rows, p->ldm, 256))
      return cudaErrorInvalidValue;
    const uint32_t fmt = dt == DT_BF16 ? 1u : 0u;
    g.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (8u << 24);
    return launch_symgemm(dt, epi, ta, tb, g, grid, s, out ? kind_dtype(*out) : -1, /*many_small=*/true);
  }
  if (route == ROUTE_NONE) return cudaErrorNotSupported;
  const bool b1 = route == ROUTE_X2;
  const Mat& PA = b1 ? B : A;  // the pair operand goes first
  const Mat& PB = b1 ? A : B;
  const int dt = kind_dtype(PA);
  CUtensorMap tm[4];
  const int rb = x3_row_bytes(b1);
  if (!encode_tmap_rows(&tm[0], dt, bpart(p, PA, 0), cols, rows, p->ldm, 128, rb) ||
      !encode_tmap_rows(&tm[1], dt, bpart(p, PA, 1), cols, rows, p->ldm, 128, rb) ||
      !encode_tmap_rows(&tm[2], dt, bpart(p, PB, 0), cols, rows, p->ldm, 256, rb) ||
      !encode_tmap_rows(&tm[3], dt, bpart(p, PB, b1 ? 0 : 1), cols, rows, p->ldm, 256, rb))
    return cudaErrorInvalidValue;
  const int out_mode = epi == EPI_FINAL ? 2 : (kind_is_pair(out->kind) ? 0 : 1);
  return launch_symgemm_x3(dt, b1, epi, out_mode, tm, g, grid, s);
}

struct BatchOps {
  BatchPlan* p;
  cudaStream_t s;
  cudaError_t cast(const Mat& X0) {
    BatchCast bc{bpart(p, X0, 0), kind_is_pair(X0.kind) ? bpart(p, X0, 1) : nullptr, p->ldm};
    return enqueue_batch_cast(kind_dtype(X0), bc, p->d_bb, p->d_st, p->d_cast, p->ncast, s);
  }
  cudaError_t gemm(int epi, const Mat& A, const Mat& B, const Mat* out, const Mat* Y, float a, float b, float c,
                   float sc, bool track) {
    return bgemm(p, epi, A, B, out, Y, a, b, c, sc, track, s);
  }
  cudaError_t finish() {
    return enqueue_batch_finalize(p->d_bb, p->d_st, p->count, p->d_cres, p->d_cidx, p->d_crange, p->pair ? 16 : 4,
                                  p->flow ? p->d_flowctl + 1 : nullptr,
                                  s);
  }
};

cudaError_t enqueue_batch(BatchPlan* p, cudaStream_t s) {
  cudaError_t e;
  e = p->flow ? enqueue_batch_norm_bound_flow(p->L, p->d_symv, p->nsymv, p->d_flow, p->nflow, p->d_flowctl, p->count, s)
              : enqueue_batch_norm_bound(p->L, p->count, p->d_symv, p->nsymv, s);
  if (e != cudaSuccess) return e;
  if (!p->chain) {
    BatchOps ops{p, s};
    return run_chain(p->prec, p->sched, p->nslots, dt16_for(p->prec), ops);
  }
  BatchOps ops{p, s};
  if ((e = ops.cast(p->x0)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(p->d_done, 0, sizeof(int) * p->nprod * p->count, s)) != cudaSuccess) return e;
  GemmParams g{};
  g.num_tiles = p->ntiles;
  g.tiles = p->d_tiles;
  g.blocks = p->d_rec;
  g.ep.status = p->d_status;
  g.ep.ldc = p->ldm;
  g.ep.ldy = p->ldm;
  g.ep.in_scale = g.ep.y_scale = g.ep.out_scale = 1.f;
  g.ep.cres = p->d_cres;
  const uint32_t fmt = dt16_for(p->prec) == DT_BF16 ? 1u : 0u;
  g.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (8u << 24);  // M = 128; N per tile
  if ((e = launch_symgemm_chain(dt16_for(p->prec), p->cmaps, p->d_prods, p->nprod, g, p->d_done, num_sms(), s)) !=
      cudaSuccess)
    return e;
  return enqueue_batch_finalize(p->d_bb, p->d_st, p->count, p->d_cres, p->d_cidx, p->d_crange, 8,
                                p->flow ? p->d_flowctl + 1 : nullptr, s);
}

// Picks the plan's product schedule: the forced one, the one tuned earlier for
// the same (precision, block orders), or the fastest of all candidates on one
// product of the chain's first stage (median of 3 after a warm-up, on a
// private stream; the slots hold zeros, which leaves the timing unchanged).
psd_status_t tune_bplan(BatchPlan* p) {
  const int grid = std::max(1, std::min(num_sms(), p->ntiles));
  const auto key = tune_key(p);
  // the pair form: FP16 / BF16 plans (every product a 16-bit product), not with the chain form
  const bool pair_ok = (p->prec == PSD_PREC_FP16 || p->prec == PSD_PREC_BF16) && g_force_form != 1;
  TuneReport rep;
  rep.ncand = kNumSchedules + (pair_ok ? 1 : 0);
  int chosen = 0;
  if (g_force_schedule >= 0 && g_force_schedule < rep.ncand) {
    chosen = g_force_schedule;
  } else if (g_tuned.count(key) && g_tuned[key] < rep.ncand) {
    chosen = g_tuned[key];
  } else {
    cudaStream_t ts;
    if (cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) != cudaSuccess) return PSD_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const StageKinds k = stage_kinds(p->prec, 0, p->sched.T);
    Mat A, Y;
    A.kind = k.x;
    A.slot = 0;
    A.dt16 = dt16_for(p->prec);
    Y.kind = k.y;
    Y.slot = kind_slots(k.x);
    Y.dt16 = A.dt16;
    float best = 0.f;
    bool ok = true;
    for (int c = 0; c < rep.ncand && ok; ++c) {
      p->pair = c == kPairCandidate;
      if (!p->pair) {
        const std::vector<int4> t = schedule_tiles(p->sizes, c, grid);
        ok = cudaMemcpyAsync(p->d_tiles, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice, ts) ==
             cudaSuccess;
      }
      float ms[3] = {};
      for (int r = -1; r < 3 && ok; ++r) {
        cudaEventRecord(e0, ts);
        ok = bgemm(p, EPI_COPY, A, A, &Y, nullptr, 0.f, 0.f, 0.f, 1.f, false, ts) == cudaSuccess;
        cudaEventRecord(e1, ts);
        ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
        if (ok && r >= 0) cudaEventElapsedTime(&ms[r], e0, e1);
      }
      std::sort(ms, ms + 3);
      rep.ms[c] = ms[1];
      if (ok && (c == 0 || ms[1] < best)) {
        best = ms[1];
        chosen = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(ts);
    if (!ok) return PSD_ERR_CUDA;
    g_tuned[key] = chosen;
  }
  p->pair = chosen == kPairCandidate;
  const std::vector<int4> t = schedule_tiles(p->sizes, p->pair ? 0 : chosen, grid);
  if (cudaMemcpy(p->d_tiles, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return PSD_ERR_CUDA;
  // each block's final-product shares, in the block's own tile order (schedule-independent
  // sums), positions in the tile list the final product runs over
  const std::vector<int4> tf = p->pair ? pair_tiles(p->sizes) : t;
  std::map<std::tuple<int, int, int>, int> pos;
  for (int i = 0; i < static_cast<int>(tf.size()); ++i) pos[std::make_tuple(tf[i].z, tf[i].x, tf[i].y)] = i;
  std::vector<int> cidx;
  std::vector<int2> crange(p->count);
  for (int b = 0; b < p->count; ++b) {
    crange[b].x = static_cast<int>(cidx.size());
    const std::vector<int4> own = p->pair ? make_tile_list_pair(p->sizes[b], b, 8) : make_tile_list(p->sizes[b], b, 8);
    for (const int4& c : own) cidx.push_back(pos.at(std::make_tuple(b, c.x, c.y)));
    crange[b].y = static_cast<int>(cidx.size()) - crange[b].x;
  }
  if (cudaMemcpy(p->d_cidx, cidx.data(), sizeof(int) * cidx.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_crange, crange.data(), sizeof(int2) * crange.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return PSD_ERR_CUDA;
  rep.chosen = chosen;
  g_last_tune = rep;
  return PSD_OK;
}

void ensure_bgraph(BatchPlan* p) {
  if (p->graph_tried) return;
  p->graph_tried = true;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    cudaError_t e = enqueue_batch(p, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess && e2 == cudaSuccess && graph) {
      if (cudaGraphInstantiate(&p->exec, graph, 0) != cudaSuccess) p->exec = nullptr;
    }
    if (graph) cudaGraphDestroy(graph);
  }
  cudaGetLastError();
  cudaStreamDestroy(cs);
}

}  // namespace

void release_batched_plans() {
  std::lock_guard<std::mutex> lk(g_bmu);
  for (auto& kv : g_bplans) free_bplan(kv.second);
  g_bplans.clear();
}

}  // namespace psd

using namespace psd;

extern "C" int32_t psd_batched_force_schedule(int32_t index) {
  std::lock_guard<std::mutex> lk(g_bmu);
  const int prev = g_force_schedule;
  g_force_schedule = (index >= 0 && index <= kPairCandidate) ? index : -1;
  return prev;
}

extern "C" int32_t psd_batched_force_form(int32_t form) {
  std::lock_guard<std::mutex> lk(g_bmu);
  const int prev = g_force_form;
  g_force_form = (form == 0 || form == 1) ? form : -1;
  return prev;
}

extern "C" int32_t psd_batched_force_bound(int32_t form) {
  std::lock_guard<std::mutex> lk(g_bmu);
  const int prev = g_force_bound;
  g_force_bound = (form == 0 || form == 1) ? form : -1;
  return prev;
}

extern "C" psd_status_t psd_batched_last_tuning(int32_t* chosen, int32_t* candidates, float* ms) {
  std::lock_guard<std::mutex> lk(g_bmu);
  if (g_last_tune.chosen < 0) return PSD_ERR_INVALID_ARG;
  if (chosen) *chosen = g_last_tune.chosen;
  if (candidates) *candidates = g_last_tune.ncand;
  if (ms)
    for (int c = 0; c < g_last_tune.ncand; ++c) ms[c] = g_last_tune.ms[c];
  return PSD_OK;
}

extern "C" psd_status_t psd_project_batched(int32_t count, const psd_block_desc_t* d_descs,
                                            psd_precision_t precision, psd_stream_t stream) {
  if (count < 0 || (count > 0 && !d_descs)) return PSD_ERR_INVALID_ARG;
  if (precision != PSD_PREC_FP16 && precision != PSD_PREC_BF16 && precision != PSD_PREC_FP32 &&
      precision != PSD_PREC_MIXED)
    return (precision == PSD_PREC_FP8_EARLY || precision == PSD_PREC_FP8_LATE) ? PSD_ERR_UNSUPPORTED
                                                                               : PSD_ERR_INVALID_ARG;
  if (count == 0) return PSD_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PSD_ERR_CUDA;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return PSD_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<psd_block_desc_t> h(static_cast<size_t>(count));
  if (cudaMemcpyAsync(h.data(), d_descs, sizeof(psd_block_desc_t) * h.size(), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PSD_ERR_CUDA;
  std::vector<int> sizes(static_cast<size_t>(count));
  for (int b = 0; b < count; ++b) {
    const psd_block_desc_t& d = h[b];
    if (d.n < 1 || d.n > kMaxBatchOrder || !d.X || !d.out || d.ld < d.n || d.ld_out < d.n)
      return PSD_ERR_INVALID_ARG;
    const char* x0 = reinterpret_cast<const char*>(d.X);
    const char* x1 = reinterpret_cast<const char*>(d.X + (d.n - 1) * d.ld + d.n);
    const char* o0 = reinterpret_cast<const char*>(d.out);
    const char* o1 = reinterpret_cast<const char*>(d.out + (d.n - 1) * d.ld_out + d.n);
    if (x0 < o1 && o0 < x1 && !(x0 == o0 && d.ld == d.ld_out)) return PSD_ERR_INVALID_ARG;
    sizes[b] = static_cast<int>(d.n);
  }
  std::lock_guard<std::mutex> lk(g_bmu);
  auto key = std::make_tuple(dev, s, 4 * static_cast<int>(precision) + g_force_form + 1 + 64 * (g_force_bound == 1),
                             sizes);
  BatchPlan* p = nullptr;
  auto it = g_bplans.find(key);
  if (it != g_bplans.end()) {
    p = it->second;
  } else {
    p = new BatchPlan();
    p->prec = precision;
    p->count = count;
    p->sizes = sizes;
    psd_status_t st = build_bplan(p);
    if (st == PSD_OK) st = tune_bplan(p);
    if (st == PSD_OK) st = prepare_chain(p);
    if (st != PSD_OK) {
      free_bplan(p);
      return st;
    }
    g_bplans[key] = p;
  }
  ensure_bgraph(p);
  batch_args_kernel<<<(count + 127) / 128, 128, 0, s>>>(d_descs, p->d_rec, p->d_bb, count);
  if (cudaGetLastError() != cudaSuccess) return PSD_ERR_CUDA;
  cudaError_t e = p->exec ? cudaGraphLaunch(p->exec, s) : enqueue_batch(p, s);
  return e == cudaSuccess ? PSD_OK : PSD_ERR_CUDA;
}
