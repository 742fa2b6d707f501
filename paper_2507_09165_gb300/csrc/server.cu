// Request server: stage-level continuous batching of projections (a serving
// layer around Algorithm 2; the paper itself projects one matrix at a time).
//
// Device memory (one allocation of the caller's HBM budget):
//   [launch status | records | lane scratch x kLanes | staging x kRing | arena]
//   record (per admitted request): DevArgs | DevState | psd_info_t
//   lane scratch: DevArgs | DevState | Lanczos buffers of order max_order
//   staging: the block tables and tile lists of one scheduler step
//   arena: rows of ldm 16-bit elements; a request of order n holds the 4 n
//          rows [row, row + 4n): X_0, R1, P, R3 (X_0, the two rotating
//          iterates, the stage polynomial), then the rows that hold the
//          per-warp shares of <out, X - out> of its final product (4 doubles
//          per tile, at the tile's position in the request's tile list).
//
// Stage t of a request (cur: X_{t-1}; R1/R3 alternate):
//   cur = X_0 (t = 0), R1 (t odd), R3 (t even > 0);  Y = R1 (t even), R3 (t odd)
//   Y = cur cur;  P = a_t I + b_t Y + c_t Y Y;  Y <- cur P / s_t   (X_t overwrites Y)
// and after the last stage out = (X + lam~ X_0 X_T) / 2.  The products are the
// 16-bit symmetric tensor-core kernels of symgemm.cu over a block table with
// per-block row offsets and coefficients, so one launch covers every running
// request whatever its stage; a step spreads large products over several
// launches under a work budget (enqueue_step).  The norm bound runs on a preparation stream
// ("lane") with the single-projection kernels, replayed from a CUDA graph per
// (lane, n); its result is copied into the request's record.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace psd {
namespace {

constexpr int kLanes = 2;            // preparation streams
constexpr int kRing = 2;             // scheduler steps in flight
constexpr size_t kRecBytes = 1280;   // DevArgs (256) | DevState (768) | psd_info_t (256)
constexpr size_t kLaneHead = 1024;   // DevArgs (256) | DevState (768)
constexpr int kMaxGraphsPerLane = 32;
constexpr int kMaxBatchLimit = 1024;
constexpr int64_t kMaxArenaRows = (int64_t{1} << 31) - 1024;  // TMA row coordinates are 32-bit
// Work budget of one scheduler step in tile-K-blocks (one 128 x 256 output
// tile over 64 K: 4.2 MFLOP; at ~1.3 PFLOP/s about 3 ns of the whole GPU), so a
// step lasts about 0.5 ms however large the running requests are (measured on
// the mixed ADMM stream: 1 ms steps gave n = 500 requests 14 / 24 ms p50 / p99,
// 0.5 ms steps 10 / 14 ms, at 1.7% less throughput).
constexpr int64_t kStepBudget = 150000;
constexpr int64_t kQuantumDiv = 8;

using Clock = std::chrono::steady_clock;

size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

enum ReqState : int { RQ_QUEUED = 0, RQ_PREP = 1, RQ_RUN = 2, RQ_DONE = 3 };

struct Request {
  uint64_t id = 0;
  int64_t n = 0;
  const float* X = nullptr;
  int64_t ld = 0;
  float* out = nullptr;
  int64_t ld_out = 0;
  int dt = DT_F16;
  cudaEvent_t ready = nullptr;
  int state = RQ_QUEUED;
  int slot = -1;     // record slot
  int64_t row = -1;  // first arena row
  int lane = 0;
  int stage = 0;
  int g = 0;         // product of the stage in progress: 0 Y, 1 P, 2 X_t, 3 final
  int k = 0;         // tiles of that product done
  int ntiles = 0;    // bound on the tile count (admission)
  std::vector<int4> tl;  // tile list of order n: 256 x 256 tiles on SM pairs (make_tile_list_pair)
  double* cres = nullptr;  // shares of <out, X - out>, 8 per tile of tl in the one-SM order (arena rows
                           // after the matrices)
  Clock::time_point t_submit;
  double latency_ms = 0.0;
  psd_info_t info{};
};

// First-fit allocator of arena rows with coalescing.
struct RowAllocator {
  std::map<int64_t, int64_t> free_;  // start -> length
  int64_t used = 0, peak = 0;
  void init(int64_t rows) {
    free_.clear();
    free_[0] = rows;
  }
  int64_t alloc(int64_t len) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < len) continue;
      const int64_t start = it->first, rest = it->second - len;
      free_.erase(it);
      if (rest > 0) free_[start + len] = rest;
      used += len;
      peak = std::max(peak, used);
      return start;
    }
    return -1;
  }
  void release(int64_t start, int64_t len) {
    used -= len;
    auto next = free_.lower_bound(start);
    if (next != free_.end() && start + len == next->first) {
      len += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == start) {
        prev->second += len;
        return;
      }
    }
    free_[start] = len;
  }
};

// Tiles of one request of order n (two 128-row tiles per upper 256 x 256 block).
int64_t tiles_of(int64_t n) {
  const int64_t nb = (n + 255) / 256;
  return nb * (nb + 1);
}

// Arena rows of a request of order n: its four matrices, then its shares of
// <out, X - out> (8 doubles per 256 x 256 tile, 4 per 128-row half: tiles_of(n)
// halves) in whole rows of ldm 16-bit elements.
int64_t rows_of(int64_t ldm, int64_t n) {
  const int64_t share_bytes = 4 * static_cast<int64_t>(sizeof(double)) * tiles_of(n);
  return 4 * n + (share_bytes + 2 * ldm - 1) / (2 * ldm);
}

struct StepDone;

}  // namespace
}  // namespace psd

struct psd_server {
  int device = 0;
  int64_t max_order = 0, ldm = 0, rows = 0;
  int max_batch = 0;
  int64_t tile_cap = 0;
  psd::Schedule sched{};
  // device memory
  uint8_t* mem = nullptr;
  int* d_launch_status = nullptr;
  uint8_t* recs = nullptr;
  uint8_t* lane_mem[psd::kLanes] = {};
  uint8_t* d_stage[psd::kRing] = {};
  uint8_t* h_stage[psd::kRing] = {};
  size_t stage_bytes = 0;
  uint16_t* arena = nullptr;
  CUtensorMap tmA[2], tmB[2];  // [0] FP16, [1] BF16 views of the arena (128-row boxes: the pair form)
  // streams and events
  cudaStream_t main = nullptr;
  cudaStream_t lane[psd::kLanes] = {};
  cudaEvent_t step_ev[psd::kRing] = {};
  bool ring_busy[psd::kRing] = {};
  int ring_next = 0;
  std::vector<cudaEvent_t> prep_ev;  // per record slot
  std::map<int64_t, cudaGraphExec_t> nb_graph[psd::kLanes];
  std::deque<int64_t> nb_order[psd::kLanes];
  int lane_next = 0;
  // scheduler state (guarded by mu)
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<psd::Request*> queue;
  std::vector<psd::Request*> prep, run;
  std::unordered_map<uint64_t, psd::Request*> tickets;
  std::vector<int> free_slots;
  psd::RowAllocator rows_alloc;
  int64_t tiles_held = 0;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread th;
  // statistics (guarded by mu)
  uint64_t submitted = 0, completed = 0, canceled = 0, steps = 0, launches = 0;
  int max_running = 0;
  std::vector<double> lat;
  int64_t peak_rows = 0;
};

namespace psd {
namespace {

DevArgs* rec_args(psd_server* s, int slot) { return reinterpret_cast<DevArgs*>(s->recs + slot * kRecBytes); }
DevState* rec_state(psd_server* s, int slot) {
  return reinterpret_cast<DevState*>(s->recs + slot * kRecBytes + 256);
}
psd_info_t* rec_info(psd_server* s, int slot) {
  return reinterpret_cast<psd_info_t*>(s->recs + slot * kRecBytes + 1024);
}

// Copies the lane's argument block and norm-bound state into a request record.
__global__ void adopt_kernel(DevArgs* dst_args, DevState* dst_st, const DevArgs* src_args, const DevState* src_st) {
  *dst_args = *src_args;
  *dst_st = *src_st;
}

// A request that finishes in a step: its record slot and its shares of
// <out, X - out> (ncompl = 4 per tile).
struct FinRec {
  int slot;
  int ncompl;
  const double* cres;
};

// Report of every request that finished in a step (one CTA each): status and
// overshoot (finalize_report), with a timed-out launch of the step as the
// status of an otherwise clean request, and the complementarity residual
// summed in the order of the single-projection finalize; copied into the
// step's report array.
__global__ void __launch_bounds__(kComplSumThreads)
    server_finalize_kernel(uint8_t* recs, const FinRec* fin, const int* launch_status, psd_info_t* out) {
  __shared__ double wsum[kComplSumThreads / 32];
  const FinRec f = fin[blockIdx.x];
  const double v = compl_cta_sum<kComplSumThreads>(f.cres, f.ncompl, wsum);
  if (threadIdx.x != 0) return;
  uint8_t* r = recs + static_cast<size_t>(f.slot) * kRecBytes;
  DevState* st = reinterpret_cast<DevState*>(r + 256);
  psd_info_t* info = reinterpret_cast<psd_info_t*>(r + 1024);
  if (st->status == 0 && *launch_status != 0) st->status = *launch_status;
  finalize_report(st, info);
  const double f2 = st->fro * st->fro;
  info->compl_resid = f2 > 0.0 ? v / f2 : 0.0;
  out[blockIdx.x] = *info;
}

// Staging layout of one step (host and device copies are identical):
//   BlockRec blocks[4][max_batch]   GEMM 1, 2, 3 and the final product
//   FinRec fin[max_batch]           the requests that finish (slot, shares)
//   int4 tiles[4 tile_cap]          tile lists of the step's launches
//   psd_info_t infos[max_batch]     reports of the finishing requests (device -> host)
struct StageLayout {
  size_t blocks, fin, tiles, infos, total;
};
StageLayout stage_layout(int max_batch, int64_t tile_cap) {
  StageLayout L{};
  L.blocks = 0;
  L.fin = round_up(4 * sizeof(BlockRec) * max_batch, 256);
  L.tiles = L.fin + round_up(sizeof(FinRec) * max_batch, 256);
  L.infos = L.tiles + round_up(sizeof(int4) * 4 * tile_cap, 256);  // up to 4 product slots per request
  L.total = L.infos + round_up(sizeof(psd_info_t) * max_batch, 256);
  return L;
}

struct StepDone {
  psd_server* s;
  std::vector<uint64_t> ids;
  const psd_info_t* infos;  // pinned staging, valid until the step's event completes
};

// Host callback after a step's last kernel: completes the finished tickets
// and returns their rows and records.  Runs on a CUDA runtime thread and must
// make no CUDA call.
void CUDART_CB on_step_done(void* arg) {
  StepDone* d = static_cast<StepDone*>(arg);
  psd_server* s = d->s;
  const auto now = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t k = 0; k < d->ids.size(); ++k) {
      auto it = s->tickets.find(d->ids[k]);
      if (it == s->tickets.end()) continue;
      Request* r = it->second;
      r->info = d->infos[k];
      r->latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
      r->state = RQ_DONE;
      s->rows_alloc.release(r->row, rows_of(s->ldm, r->n));
      s->tiles_held -= r->ntiles;
      s->free_slots.push_back(r->slot);
      s->lat.push_back(r->latency_ms);
      ++s->completed;
    }
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();
  delete d;
}

cudaGraphExec_t norm_bound_graph(psd_server* s, int lane, int64_t n) {
  auto& cache = s->nb_graph[lane];
  auto it = cache.find(n);
  if (it != cache.end()) return it->second;
  if (static_cast<int>(cache.size()) >= kMaxGraphsPerLane) {
    const int64_t old = s->nb_order[lane].front();
    s->nb_order[lane].pop_front();
    cudaGraphExecDestroy(cache[old]);
    cache.erase(old);
  }
  uint8_t* base = s->lane_mem[lane];
  DevArgs* args = reinterpret_cast<DevArgs*>(base);
  DevState* st = reinterpret_cast<DevState*>(base + 256);
  LanczosBufs L;
  lanczos_carve(L, n, base + kLaneHead);
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    // the multi-launch form: these lanes run beside the step's product kernels,
    // which leave no room for a co-resident persistent grid
    const cudaError_t e = enqueue_norm_bound(L, args, st, cs, false);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess && e2 == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess)
      exec = nullptr;
    if (g) cudaGraphDestroy(g);
  }
  cudaGetLastError();
  cudaStreamDestroy(cs);
  if (exec) {
    cache[n] = exec;
    s->nb_order[lane].push_back(n);
  }
  return exec;
}

// Preparation of an admitted request on its lane: zero the K-padding columns
// [n, round_up(n, 64)) of its rows (the products read whole 64-column blocks),
// norm bound, X_0 = RN(X / lam~) into its first n rows.
bool enqueue_prep(psd_server* s, Request* r, int& launches) {
  const int lane = r->lane;
  cudaStream_t ls = s->lane[lane];
  const int64_t n = r->n;
  if (r->ready && cudaStreamWaitEvent(ls, r->ready, 0) != cudaSuccess) return false;
  const int64_t kpad = (n + 63) / 64 * 64;
  uint16_t* base = s->arena + r->row * s->ldm;
  if (kpad > n &&
      cudaMemset2DAsync(base + n, s->ldm * 2, 0, static_cast<size_t>(kpad - n) * 2, static_cast<size_t>(4 * n), ls) !=
          cudaSuccess)
    return false;
  cudaGraphExec_t g = norm_bound_graph(s, lane, n);
  if (!g) return false;
  uint8_t* lb = s->lane_mem[lane];
  DevArgs* largs = reinterpret_cast<DevArgs*>(lb);
  DevState* lst = reinterpret_cast<DevState*>(lb + 256);
  DevArgs h{r->X, r->ld, r->out, r->ld_out, rec_info(s, r->slot)};
  if (enqueue_set_args(largs, h, ls) != cudaSuccess) return false;
  if (cudaGraphLaunch(g, ls) != cudaSuccess) return false;
  adopt_kernel<<<1, 1, 0, ls>>>(rec_args(s, r->slot), rec_state(s, r->slot), largs, lst);
  if (enqueue_scale_cast(r->dt, rec_args(s, r->slot), rec_state(s, r->slot), n, base, nullptr, s->ldm,
                         ls) != cudaSuccess)
    return false;
  if (cudaEventRecord(s->prep_ev[r->slot], ls) != cudaSuccess) return false;
  launches += 4 + kNormBoundLaunches;  // set_args, graph kernels, adopt, cast (+ memset)
  return true;
}

// One grouped product launch over the tiles [t0, t1) of the staging tile list.
cudaError_t step_gemm(psd_server* s, int dti, int epi, const BlockRec* d_blocks, const int4* d_tiles, int ntiles,
                      int& launches) {
  if (ntiles == 0) return cudaSuccess;
  GemmParams g{};
  g.num_tiles = ntiles;
  g.tiles = d_tiles;
  g.blocks = d_blocks;
  g.ep.status = s->d_launch_status;
  g.ep.C = s->arena;
  g.ep.ldc = s->ldm;
  g.ep.Y = s->arena;
  g.ep.ldy = s->ldm;
  g.ep.per_block_coef = 1;
  g.ep.absmax_blocks = epi == EPI_SCALE ? 2 : 0;
  const uint32_t fmt = dti == 1 ? 1u : 0u;
  g.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (16u << 24);  // M = 256: tiles on SM pairs
  ++launches;
  // SM pairs with 4 epilogue warps per CTA: served steps mix large requests,
  // whose long main loops want the 6-stage ring
  return launch_symgemm_pair(dti == 1 ? DT_BF16 : DT_F16, epi, s->tmA[dti], s->tmB[dti], g, num_sms(), s->main);
}

// Builds and enqueues one scheduler step over `run`.  A step is one grouped
// launch per product slot (Y = X^2, the polynomial, X P / s_t, the final
// product) and operand type.  Each request keeps a cursor (stage, product,
// tiles done) and takes the next tiles of its current product; a request that
// completes a product continues with the next slot in the same step, so a
// small request runs a whole stage per step.  Requests are visited smallest
// first against a work budget of kStepBudget tile-K-blocks, which bounds the
// step's duration; a request the budget does not reach still gets
// kStepBudget / kQuantumDiv worth of tiles, so large requests always progress.
// Every tile's arithmetic is the same whichever launch computes it.
// Between building the step and enqueueing its GPU work the running set moves
// on, so that the completion callback never sees a request that is still
// listed as running.
bool enqueue_step(psd_server* s, const std::vector<Request*>& run, int& launches) {
  const int slot = s->ring_next;
  s->ring_next = (s->ring_next + 1) % kRing;
  if (s->ring_busy[slot] && cudaEventSynchronize(s->step_ev[slot]) != cudaSuccess) return false;
  const StageLayout SL = stage_layout(s->max_batch, s->tile_cap);
  uint8_t* h = s->h_stage[slot];
  uint8_t* d = s->d_stage[slot];
  BlockRec* hb = reinterpret_cast<BlockRec*>(h + SL.blocks);
  FinRec* hfin = reinterpret_cast<FinRec*>(h + SL.fin);
  int4* ht = reinterpret_cast<int4*>(h + SL.tiles);
  const int T = s->sched.T;
  const int mb = s->max_batch;
  const int nrun = static_cast<int>(run.size());
  // block records of every running request for every product slot
  for (int i = 0; i < nrun; ++i) {
    Request* r = run[i];
    const int t = r->stage;
    const int64_t n = r->n;
    const int64_t x0 = r->row, r1 = r->row + n, rp = r->row + 2 * n, r3 = r->row + 3 * n;
    const int64_t cur = t == 0 ? x0 : ((t & 1) ? r1 : r3);
    const int64_t ry = (t & 1) ? r3 : r1;
    DevState* st = rec_state(s, r->slot);
    BlockRec b{};
    b.n = static_cast<int>(n);
    b.st = st;
    // Y = cur cur
    b.off = cur;
    b.dc = ry - cur;
    hb[0 * mb + i] = b;
    // P = a I + b Y + c Y Y
    b.off = ry;
    b.dc = rp - ry;
    b.ca = static_cast<float>(s->sched.coef[t][0]);
    b.cb = static_cast<float>(s->sched.coef[t][1]);
    b.cc = static_cast<float>(s->sched.coef[t][2]);
    hb[1 * mb + i] = b;
    // X_t = cur P / s_t into Y's rows; max |X_T| tracked at the last stage
    b.off = cur;
    b.db = rp - cur;
    b.dc = ry - cur;
    b.ca = b.cb = b.cc = 0.f;
    b.cs = static_cast<float>(1.0 / s->sched.post[t]);
    b.track = t == T - 1 ? 1 : 0;
    hb[2 * mb + i] = b;
    // out = (X + lam~ X_0 X_T) / 2
    BlockRec f{};
    f.n = static_cast<int>(n);
    f.st = st;
    f.off = x0;
    f.db = ry - x0;
    f.X = r->X;
    f.ld = r->ld;
    f.out = r->out;
    f.ld_out = r->ld_out;
    f.cres = r->cres;  // cres_shift: set with the tile list below
    hb[3 * mb + i] = f;
  }
  // tile allotment, smallest requests first
  struct Part {
    int req, begin, end;
  };
  std::vector<Part> parts[4];
  struct Cursor {
    int stage, g, k;
    bool done;
  };
  std::vector<Cursor> next(nrun);
  std::vector<int> order(nrun);
  for (int i = 0; i < nrun; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return run[a]->n < run[b]->n; });
  int64_t budget = kStepBudget;
  for (int i : order) {
    Request* r = run[i];
    const int nt = static_cast<int>(r->tl.size());
    const int64_t cost = 2 * ((r->n + 63) / 64);  // K-blocks of 64 per 256-row tile (two 128-row tiles)
    Cursor c{r->stage, r->g, r->k, false};
    bool any = false;
    for (;;) {
      const int rem = nt - c.k;
      int64_t m = std::min<int64_t>(rem, std::max<int64_t>(budget, 0) / cost);
      if (m <= 0 && !any) m = std::min<int64_t>(rem, std::max<int64_t>(1, kStepBudget / kQuantumDiv / cost));
      if (m <= 0) break;
      parts[c.g].push_back({i, c.k, c.k + static_cast<int>(m)});
      any = true;
      budget -= m * cost;
      c.k += static_cast<int>(m);
      if (c.k < nt) break;  // the product continues in the next step
      c.k = 0;
      if (c.g == 3) {
        c.done = true;
        break;
      }
      if (c.g == 2) {
        if (c.stage == T - 1) {
          c.g = 3;  // the final product follows in this step
        } else {
          c.g = 0;  // the next stage starts with the next step
          ++c.stage;
          break;
        }
      } else {
        ++c.g;
      }
    }
    next[i] = c;
  }
  // tile lists per slot and operand type, largest orders first (long tiles lead)
  int cnt[4][2] = {};
  int64_t nt_all = 0;
  for (int g = 0; g < 4; ++g) {
    for (int dti = 0; dti < 2; ++dti) {
      const int64_t start = nt_all;
      for (auto it = parts[g].rbegin(); it != parts[g].rend(); ++it) {
        const Request* r = run[it->req];
        if ((r->dt == DT_BF16 ? 1 : 0) != dti) continue;
        // final product: tile q of the request sits at launch position q - cres_shift
        if (g == 3) hb[3 * mb + it->req].cres_shift = it->begin - (nt_all - start);
        for (int q = it->begin; q < it->end; ++q) {
          int4 tc = r->tl[q];
          tc.z = it->req;
          ht[nt_all++] = tc;
        }
      }
      cnt[g][dti] = static_cast<int>(nt_all - start);
    }
  }
  std::vector<uint64_t> fin_ids;
  int nf = 0;
  for (int i = 0; i < nrun; ++i)
    if (next[i].done) {
      hfin[nf++] = FinRec{run[i]->slot, 8 * static_cast<int>(run[i]->tl.size()), run[i]->cres};
      fin_ids.push_back(run[i]->id);
    }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    ++s->steps;
    s->max_running = std::max(s->max_running, nrun);
    std::vector<Request*> keep;
    for (int i = 0; i < nrun; ++i) {
      Request* r = run[i];
      if (next[i].done) continue;  // completes in on_step_done
      r->stage = next[i].stage;
      r->g = next[i].g;
      r->k = next[i].k;
      keep.push_back(r);
    }
    s->run.swap(keep);  // only this thread changes the running set: s->run == run here
  }
  cudaStream_t ms = s->main;
  const size_t upload = SL.tiles + sizeof(int4) * static_cast<size_t>(nt_all);
  if (cudaMemcpyAsync(d, h, upload, cudaMemcpyHostToDevice, ms) != cudaSuccess) return false;
  const BlockRec* db = reinterpret_cast<const BlockRec*>(d + SL.blocks);
  const int4* dt = reinterpret_cast<const int4*>(d + SL.tiles);
  const int epis[4] = {EPI_COPY, EPI_POLY, EPI_SCALE, EPI_FINAL};
  int64_t off = 0;
  for (int g = 0; g < 4; ++g)
    for (int dti = 0; dti < 2; ++dti) {
      if (step_gemm(s, dti, epis[g], db + g * mb, dt + off, cnt[g][dti], launches) != cudaSuccess) return false;
      off += cnt[g][dti];
    }
  if (nf > 0) {
    server_finalize_kernel<<<nf, kComplSumThreads, 0, ms>>>(s->recs, reinterpret_cast<const FinRec*>(d + SL.fin),
                                                            s->d_launch_status,
                                                            reinterpret_cast<psd_info_t*>(d + SL.infos));
    ++launches;
    if (cudaGetLastError() != cudaSuccess) return false;
    if (cudaMemcpyAsync(h + SL.infos, d + SL.infos, sizeof(psd_info_t) * nf, cudaMemcpyDeviceToHost, ms) !=
        cudaSuccess)
      return false;
    StepDone* done = new StepDone{s, std::move(fin_ids), reinterpret_cast<const psd_info_t*>(h + SL.infos)};
    if (cudaLaunchHostFunc(ms, on_step_done, done) != cudaSuccess) {
      delete done;
      return false;
    }
  }
  if (cudaEventRecord(s->step_ev[slot], ms) != cudaSuccess) return false;
  s->ring_busy[slot] = true;
  return true;
}

// Marks every admitted request failed (a CUDA call of the server failed) and
// stops the scheduler; the GPU work already enqueued is drained first.
void fail_all(psd_server* s) {
  cudaStreamSynchronize(s->main);
  for (int l = 0; l < kLanes; ++l) cudaStreamSynchronize(s->lane[l]);
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto* v : {&s->prep, &s->run})
    for (Request* r : *v) {
      r->info.status = PSD_ERR_CUDA;
      r->state = RQ_DONE;
      s->rows_alloc.release(r->row, rows_of(s->ldm, r->n));
      s->tiles_held -= r->ntiles;
      s->free_slots.push_back(r->slot);
    }
  s->prep.clear();
  s->run.clear();
  for (Request* r : s->queue) {
    r->info.status = PSD_ERR_CUDA;
    r->state = RQ_DONE;
  }
  s->queue.clear();
  s->stop = true;
}

void scheduler(psd_server* s) {
  cudaSetDevice(s->device);
  std::vector<Request*> admitted, run_now;
  for (;;) {
    admitted.clear();
    bool wait_first = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        // admission in arrival order
        while (!s->queue.empty()) {
          Request* r = s->queue.front();
          if (s->free_slots.empty() || s->tiles_held + r->ntiles > s->tile_cap) break;
          const int64_t row = s->rows_alloc.alloc(rows_of(s->ldm, r->n));
          if (row < 0) break;
          s->peak_rows = std::max(s->peak_rows, s->rows_alloc.used);
          r->row = row;
          r->cres = reinterpret_cast<double*>(s->arena + (row + 4 * r->n) * s->ldm);
          r->slot = s->free_slots.back();
          s->free_slots.pop_back();
          s->tiles_held += r->ntiles;
          r->lane = s->lane_next;
          s->lane_next = (s->lane_next + 1) % kLanes;
          r->state = RQ_PREP;
          s->queue.pop_front();
          admitted.push_back(r);
        }
        if (!admitted.empty() || !s->run.empty() || !s->prep.empty()) break;
        if (s->stop && s->queue.empty()) return;
        s->cv_work.wait(lk);
      }
    }
    int launches = 0;
    bool ok = true;
    for (Request* r : admitted) ok = ok && enqueue_prep(s, r, launches);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (Request* r : admitted) s->prep.push_back(r);
    }
    // join at this stage boundary: prepared requests; with nothing running,
    // the oldest one too (the step then waits for it on the device)
    // (only this thread changes prep and run, so they are read here without
    // the lock; no CUDA call is made while the lock is held)
    std::vector<char> is_ready(s->prep.size());
    for (size_t k = 0; k < s->prep.size(); ++k) {
      is_ready[k] = cudaEventQuery(s->prep_ev[s->prep[k]->slot]) == cudaSuccess;
      if (!is_ready[k]) cudaGetLastError();  // cudaErrorNotReady is not an error here
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      std::vector<Request*> still;
      for (size_t k = 0; k < s->prep.size(); ++k) {
        Request* r = s->prep[k];
        const bool ready = is_ready[k] != 0;
        const bool first = k == 0 && s->run.empty();
        if (ready || first) {
          if (!ready) wait_first = true;
          r->state = RQ_RUN;
          r->stage = 0;
          r->g = 0;
          r->k = 0;
          s->run.push_back(r);
          if (!ready) run_now.push_back(r);
        } else {
          still.push_back(r);
        }
      }
      s->prep.swap(still);
    }
    if (wait_first) {
      for (Request* r : run_now) ok = ok && cudaStreamWaitEvent(s->main, s->prep_ev[r->slot], 0) == cudaSuccess;
      run_now.clear();
    }
    std::vector<Request*> run_copy;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      run_copy = s->run;
    }
    if (ok && !run_copy.empty()) ok = enqueue_step(s, run_copy, launches);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->launches += launches;
    }
    if (!ok) {
      fail_all(s);
      s->cv_done.notify_all();
      return;
    }
  }
}

psd_status_t check_sm103(int device) {
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess) {
    cudaGetLastError();
    return PSD_ERR_CUDA;
  }
  return (major == 10 && minor == 3) ? PSD_OK : PSD_ERR_UNSUPPORTED;
}

void destroy_resources(psd_server* s) {
  for (int l = 0; l < kLanes; ++l) {
    for (auto& kv : s->nb_graph[l]) cudaGraphExecDestroy(kv.second);
    if (s->lane[l]) cudaStreamDestroy(s->lane[l]);
  }
  for (int k = 0; k < kRing; ++k) {
    if (s->step_ev[k]) cudaEventDestroy(s->step_ev[k]);
    if (s->h_stage[k]) cudaFreeHost(s->h_stage[k]);
  }
  for (cudaEvent_t e : s->prep_ev)
    if (e) cudaEventDestroy(e);
  if (s->main) cudaStreamDestroy(s->main);
  if (s->mem) cudaFree(s->mem);
  for (auto& kv : s->tickets) delete kv.second;
  delete s;
}

bool ranges_overlap(const float* a, const float* b, int64_t n, int64_t lda, int64_t ldb) {
  const char* a0 = reinterpret_cast<const char*>(a);
  const char* a1 = reinterpret_cast<const char*>(a + (n - 1) * lda + n);
  const char* b0 = reinterpret_cast<const char*>(b);
  const char* b1 = reinterpret_cast<const char*>(b + (n - 1) * ldb + n);
  return a0 < b1 && b0 < a1;
}

// Takes a completed ticket out of the table (caller holds mu).
void retire(psd_server* s, Request* r, psd_info_t* host_info, double* latency_ms) {
  if (host_info) *host_info = r->info;
  if (latency_ms) *latency_ms = r->latency_ms;
  s->tickets.erase(r->id);
  delete r;
}

}  // namespace
}  // namespace psd

using namespace psd;

extern "C" psd_status_t psd_server_create(size_t hbm_budget_bytes, int32_t device, int64_t max_order,
                                          int32_t max_batch, psd_server_t** server) {
  if (!server || max_order < 1 || max_order > kMaxOrder || max_batch < 1 || max_batch > kMaxBatchLimit)
    return PSD_ERR_INVALID_ARG;
  *server = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return PSD_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return PSD_ERR_INVALID_ARG;
  psd_status_t st = check_sm103(device);
  if (st != PSD_OK) return st;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return PSD_ERR_CUDA;
  psd_server* s = new psd_server();
  s->device = device;
  s->max_order = max_order;
  s->max_batch = max_batch;
  s->ldm = (max_order + 63) / 64 * 64;
  get_schedule(PSD_PREC_FP16, s->sched);
  const size_t row_bytes = static_cast<size_t>(s->ldm) * 2;
  const size_t lane_bytes = round_up(kLaneHead + lanczos_bytes(max_order), 1024);
  const size_t recs_bytes = round_up(kRecBytes * max_batch, 1024);
  // tile capacity: sum over requests of tiles_of(n) <= (max_order/256 + 3) rows/1024 + 2 max_batch
  auto fixed_for = [&](int64_t tile_cap) {
    return 1024 + recs_bytes + kLanes * lane_bytes + kRing * round_up(stage_layout(max_batch, tile_cap).total, 1024);
  };
  int64_t rows = 0;
  int64_t tile_cap = 2 * max_batch;
  for (int it = 0; it < 3; ++it) {  // rows and tile capacity depend on each other; settle them
    const size_t fixed = fixed_for(tile_cap);
    rows = hbm_budget_bytes > fixed ? static_cast<int64_t>((hbm_budget_bytes - fixed) / row_bytes) : 0;
    rows = std::min(rows, kMaxArenaRows);
    tile_cap = 2 * static_cast<int64_t>(max_batch) + (max_order / 256 + 3) * (rows / 1024 + 1);
  }
  while (rows > 0 && fixed_for(tile_cap) + static_cast<size_t>(rows) * row_bytes > hbm_budget_bytes) --rows;
  if (rows < rows_of(s->ldm, max_order)) {
    delete s;
    cudaSetDevice(prev);
    return PSD_ERR_NO_MEMORY;
  }
  s->rows = rows;
  s->tile_cap = tile_cap;
  s->stage_bytes = round_up(stage_layout(max_batch, tile_cap).total, 1024);
  const size_t total = fixed_for(tile_cap) + static_cast<size_t>(rows) * row_bytes;
  if (cudaMalloc(&s->mem, total) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    cudaSetDevice(prev);
    return PSD_ERR_NO_MEMORY;
  }
  bool ok = cudaMemset(s->mem, 0, total) == cudaSuccess;
  uint8_t* p = s->mem;
  s->d_launch_status = reinterpret_cast<int*>(p);
  p += 1024;
  s->recs = p;
  p += recs_bytes;
  for (int l = 0; l < kLanes; ++l, p += lane_bytes) s->lane_mem[l] = p;
  for (int k = 0; k < kRing; ++k, p += s->stage_bytes) s->d_stage[k] = p;
  s->arena = reinterpret_cast<uint16_t*>(p);
  for (int k = 0; ok && k < kRing; ++k) ok = cudaMallocHost(&s->h_stage[k], s->stage_bytes) == cudaSuccess;
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  ok = ok && cudaStreamCreateWithPriority(&s->main, cudaStreamNonBlocking, lo) == cudaSuccess;
  for (int l = 0; ok && l < kLanes; ++l)
    ok = cudaStreamCreateWithPriority(&s->lane[l], cudaStreamNonBlocking, hi) == cudaSuccess;
  for (int k = 0; ok && k < kRing; ++k)
    ok = cudaEventCreateWithFlags(&s->step_ev[k], cudaEventDisableTiming) == cudaSuccess;
  s->prep_ev.assign(max_batch, nullptr);
  for (int k = 0; ok && k < max_batch; ++k)
    ok = cudaEventCreateWithFlags(&s->prep_ev[k], cudaEventDisableTiming) == cudaSuccess;
  for (int d = 0; ok && d < 2; ++d)
    ok = encode_tmap_rows(&s->tmA[d], d ? DT_BF16 : DT_F16, s->arena, s->ldm, rows, s->ldm, 128) &&
         encode_tmap_rows(&s->tmB[d], d ? DT_BF16 : DT_F16, s->arena, s->ldm, rows, s->ldm, 128);
  ok = ok && cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    destroy_resources(s);
    cudaSetDevice(prev);
    return PSD_ERR_CUDA;
  }
  s->rows_alloc.init(rows);
  for (int k = max_batch - 1; k >= 0; --k) s->free_slots.push_back(k);
  s->th = std::thread(scheduler, s);
  cudaSetDevice(prev);
  *server = s;
  return PSD_OK;
}

extern "C" psd_status_t psd_server_submit(psd_server_t* s, int64_t n, const float* X, int64_t ld, float* out,
                                          int64_t ld_out, psd_precision_t precision, psd_event_t ready,
                                          uint64_t* ticket) {
  if (!s || !ticket) return PSD_ERR_INVALID_ARG;
  if (precision < PSD_PREC_FP32 || precision > PSD_PREC_FP8_LATE) return PSD_ERR_INVALID_ARG;
  if (n < 0 || n > s->max_order) return PSD_ERR_INVALID_ARG;
  if (n > 0) {
    if (!X || !out || ld < n || ld_out < n) return PSD_ERR_INVALID_ARG;
    if (ranges_overlap(X, out, n, ld, ld_out) && !(static_cast<const void*>(X) == out && ld == ld_out))
      return PSD_ERR_INVALID_ARG;
  }
  if (precision != PSD_PREC_FP16 && precision != PSD_PREC_BF16) return PSD_ERR_UNSUPPORTED;
  Request* r = new Request();
  r->n = n;
  r->X = X;
  r->ld = ld;
  r->out = out;
  r->ld_out = ld_out;
  r->dt = precision == PSD_PREC_BF16 ? DT_BF16 : DT_F16;
  r->ready = reinterpret_cast<cudaEvent_t>(ready);
  r->ntiles = static_cast<int>(tiles_of(n));
  if (n > 0) r->tl = make_tile_list_pair(n, 0);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete r;
      return PSD_ERR_INVALID_ARG;
    }
    r->id = s->next_id++;
    s->tickets[r->id] = r;
    ++s->submitted;
    if (n == 0) {
      r->state = RQ_DONE;
      ++s->completed;
      s->lat.push_back(0.0);
    } else {
      s->queue.push_back(r);
    }
    *ticket = r->id;
  }
  s->cv_work.notify_all();
  return PSD_OK;
}

extern "C" psd_status_t psd_server_poll(psd_server_t* s, uint64_t ticket, int32_t* done, psd_info_t* host_info,
                                        double* latency_ms) {
  if (!s || !done) return PSD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return PSD_ERR_INVALID_ARG;
  *done = it->second->state == RQ_DONE ? 1 : 0;
  if (*done) retire(s, it->second, host_info, latency_ms);
  return PSD_OK;
}

extern "C" psd_status_t psd_server_wait(psd_server_t* s, uint64_t ticket, int64_t timeout_ms, psd_info_t* host_info,
                                        double* latency_ms) {
  if (!s) return PSD_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return PSD_ERR_INVALID_ARG;
  Request* r = it->second;
  auto is_done = [&] { return r->state == RQ_DONE; };
  if (timeout_ms > 0) {
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), is_done)) return PSD_ERR_TIMEOUT;
  } else {
    s->cv_done.wait(lk, is_done);
  }
  retire(s, r, host_info, latency_ms);
  return PSD_OK;
}

extern "C" psd_status_t psd_server_cancel(psd_server_t* s, uint64_t ticket) {
  if (!s) return PSD_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return PSD_ERR_INVALID_ARG;
    Request* r = it->second;
    if (r->state == RQ_DONE) return PSD_OK;
    if (r->state != RQ_QUEUED) return PSD_ERR_UNSUPPORTED;
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
    r->state = RQ_DONE;
    r->info = psd_info_t{};
    r->info.status = PSD_ERR_CANCELED;
    r->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
    ++s->canceled;
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();
  return PSD_OK;
}

extern "C" psd_status_t psd_server_stats(psd_server_t* s, psd_server_stats_t* out) {
  if (!s || !out) return PSD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  psd_server_stats_t v{};
  v.submitted = s->submitted;
  v.completed = s->completed;
  v.canceled = s->canceled;
  v.steps = s->steps;
  v.kernel_launches = s->launches;
  v.queued = static_cast<int32_t>(s->queue.size());
  v.admitted = static_cast<int32_t>(s->prep.size() + s->run.size());
  v.max_running = s->max_running;
  std::vector<double> l = s->lat;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) {  // nearest rank
      size_t k = static_cast<size_t>(q * static_cast<double>(l.size()) + 0.999999999);
      k = std::min(std::max<size_t>(k, 1), l.size());
      return l[k - 1];
    };
    v.p50_ms = pct(0.50);
    v.p99_ms = pct(0.99);
    v.max_ms = l.back();
  }
  v.arena_rows = s->rows;
  v.peak_rows = s->peak_rows;
  *out = v;
  return PSD_OK;
}

extern "C" psd_status_t psd_server_destroy(psd_server_t* s) {
  if (!s) return PSD_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Request* r : s->queue) {
      r->state = RQ_DONE;
      r->info.status = PSD_ERR_CANCELED;
      ++s->canceled;
    }
    s->queue.clear();
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->main);  // host callbacks of the last steps have run after this
  for (int l = 0; l < kLanes; ++l) cudaStreamSynchronize(s->lane[l]);
  destroy_resources(s);
  cudaSetDevice(prev);
  return PSD_OK;
}
