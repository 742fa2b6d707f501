// Host side of libpsdproj: argument checks, plans (workspace carve-up, tensor
// maps, tile list), CUDA-graph capture of the whole projection, and the C ABI
// of include/psdproj.h.
//
// One projection enqueues (Algorithm 2):
//   norm bound: 20-step Lanczos on X^2 + Theorem 2          (normbound.cu)
//   X_0 = RN(X / lam~), full symmetric 16-bit matrix          (normbound.cu)
//   for t = 1..T: Y = X^2; P = a I + b Y + c Y^2; X_t = X P / s_t   (symgemm.cu)
//   out = (X + lam~ X_0 X_T) / 2                               (symgemm.cu)
//   status / overshoot report
// The sequence is captured once per (device, stream, n, precision, workspace)
// into a CUDA graph; the caller's pointers reach the graph through a small
// device argument block written by a one-thread kernel in front of each replay.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "chain.h"
#include "internal.h"

namespace psd {

namespace {

// Table 2 of the paper, column f~*_half (T = 7).
const double kHalfCoef[7][3] = {
    {8.2885332412, -22.5927099246, 15.8201383114}, {4.1666196466, -2.9679004036, 0.5307623217},
    {4.0611848147, -2.9698947955, 0.5492133813},   {3.6678301399, -2.7561018955, 0.5421513305},
    {2.7632556383, -2.0607754898, 0.4695405857},   {2.0527445797, -1.4345145882, 0.4070669182},
    {1.8804816691, -1.2583997294, 0.3779501813},
};
// Table 1 of the paper, column f~*_single (T = 10).
const double kSingleCoef[10][3] = {
    {8.3119043343, -23.0739115930, 16.4664144722}, {4.1439360087, -2.9176674704, 0.5246212487},
    {4.0257813209, -2.9025002398, 0.5334261214},   {3.5118574347, -2.5740236523, 0.5050097282},
    {2.4398158400, -1.7586675341, 0.4191290613},   {1.9779835097, -1.3337358510, 0.3772169049},
    {1.9559726949, -1.3091355170, 0.3746734515},   {1.9282822454, -1.2823649693, 0.3704626545},
    {1.9220135179, -1.2812524618, 0.3707011753},   {1.8942192942, -1.2613293407, 0.3676616051},
};

}  // namespace

// Sec. 3.4: half divides the iterate by 1.01 after every stage but the last;
// single divides by 1.001 after each of the first eight stages.
bool get_schedule(psd_precision_t prec, Schedule& s) {
  switch (prec) {
    case PSD_PREC_FP16:
    case PSD_PREC_BF16:
    case PSD_PREC_MIXED:
    case PSD_PREC_FP8_LATE:
      s.T = 7;
      for (int t = 0; t < 7; ++t) {
        for (int k = 0; k < 3; ++k) s.coef[t][k] = kHalfCoef[t][k];
        s.post[t] = t < 6 ? 1.01 : 1.0;
      }
      return true;
    case PSD_PREC_FP32:
      s.T = 10;
      for (int t = 0; t < 10; ++t) {
        for (int k = 0; k < 3; ++k) s.coef[t][k] = kSingleCoef[t][k];
        s.post[t] = t < 8 ? 1.001 : 1.0;
      }
      return true;
    default:
      return false;
  }
}

namespace {

int dtype16_of(psd_precision_t prec) { return prec == PSD_PREC_BF16 ? DT_BF16 : DT_F16; }

bool prec_built(psd_precision_t prec) {
  return prec == PSD_PREC_FP16 || prec == PSD_PREC_BF16 || prec == PSD_PREC_FP32 || prec == PSD_PREC_MIXED ||
         prec == PSD_PREC_FP8_LATE;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Leading dimension of the internal iterates: a multiple of 64 elements (128 B rows).
int64_t internal_ld(int64_t n) { return round_up(std::max<int64_t>(n, 1), 64); }

// Workspace is carved into slots of one n x ldm 16-bit matrix: a 16-bit
// matrix takes 1 slot, an FP16 pair 2, a TF32 pair 4.
size_t slot_bytes(int64_t n) {
  return static_cast<size_t>(round_up(static_cast<int64_t>(internal_ld(n)) * n * 2, 1024));
}

int slots_needed(psd_precision_t prec) { return chain_slots(prec); }

size_t total_ws_bytes(int64_t n, psd_precision_t prec) {
  return slots_needed(prec) * slot_bytes(n) + lanczos_bytes(n) + 1024;
}

psd_status_t check_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PSD_ERR_CUDA;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return PSD_ERR_UNSUPPORTED;
  return PSD_OK;
}

struct Plan {
  int device = 0;
  cudaStream_t stream = nullptr;
  int64_t n = 0;
  psd_precision_t prec = PSD_PREC_FP16;
  Schedule sched{};
  uint8_t* ws = nullptr;
  size_t ws_bytes = 0;
  bool owns_ws = false;
  uint8_t* slots = nullptr;  // slot 0 base
  size_t slot_size = 0;
  int nslots = 0;
  int64_t ldm = 0;
  LanczosBufs L{};
  DevArgs* d_args = nullptr;
  DevState* d_state = nullptr;
  psd_info_t* d_info = nullptr;  // default report
  BlockRec* d_block = nullptr;   // the one block of a single projection
  int4* d_tiles = nullptr;
  int ntiles = 0;
  int4* d_tiles_pair = nullptr;  // 256-row tiles of the CTA-pair form of the 16-bit stage products
  int ntiles_pair = 0;
  int ncompl = 0;  // complementarity shares the final product writes (4 per one-SM tile, 8 per pair tile)
  double* d_compl = nullptr;  // 4 per tile: shares of <out, X - out> from the final product
  cudaGraphExec_t exec = nullptr;
  bool graph_tried = false;
  int launches = 0;  // kernel launches of one projection (graph nodes + argument block)
};

using PlanKey = std::tuple<int, cudaStream_t, int64_t, int, void*>;
std::mutex g_mu;
std::map<PlanKey, Plan*> g_plans;
std::map<std::pair<int, cudaStream_t>, Plan*> g_last;  // last default-report plan per stream

void free_plan(Plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->owns_ws && p->ws) cudaFree(p->ws);
  if (p->d_args) cudaFree(p->d_args);  // one allocation: args | state | info | tiles
  delete p;
}

psd_status_t build_plan(Plan* p, void* user_ws, size_t user_bytes) {
  const int64_t n = p->n;
  if (!get_schedule(p->prec, p->sched)) return PSD_ERR_INVALID_ARG;
  p->ldm = internal_ld(n);
  p->ws_bytes = total_ws_bytes(n, p->prec);
  if (user_ws) {
    if (user_bytes < p->ws_bytes) return PSD_ERR_NO_MEMORY;
    p->ws = static_cast<uint8_t*>(user_ws);
    p->owns_ws = false;
  } else {
    if (cudaMalloc(&p->ws, p->ws_bytes) != cudaSuccess) {
      cudaGetLastError();
      p->ws = nullptr;
      return PSD_ERR_NO_MEMORY;
    }
    p->owns_ws = true;
  }
  uint8_t* base = reinterpret_cast<uint8_t*>(round_up(reinterpret_cast<int64_t>(p->ws), 1024));
  p->slot_size = slot_bytes(n);
  p->nslots = slots_needed(p->prec);
  p->slots = base;
  lanczos_carve(p->L, n, base + p->nslots * p->slot_size);

  // small library-owned records: args | state | info | tiles
  std::vector<int4> tiles = make_tile_list(n);
  p->ntiles = static_cast<int>(tiles.size());
  const size_t o_state = round_up(sizeof(DevArgs), 256);
  const size_t o_info = o_state + round_up(sizeof(DevState), 256);
  const size_t o_block = o_info + round_up(sizeof(psd_info_t), 256);
  const size_t o_tiles = o_block + round_up(sizeof(BlockRec), 256);
  std::vector<int4> tiles_pair = make_tile_list_pair(n);
  p->ntiles_pair = static_cast<int>(tiles_pair.size());
  const size_t o_compl = o_tiles + round_up(sizeof(int4) * std::max<size_t>(tiles.size(), 1), 256);
  const size_t ncompl_max = std::max<size_t>(std::max(4 * tiles.size(), 8 * tiles_pair.size()), 1);
  const size_t o_pair = o_compl + round_up(sizeof(double) * ncompl_max, 256);
  const size_t small = o_pair + sizeof(int4) * std::max<size_t>(tiles_pair.size(), 1);
  uint8_t* sm = nullptr;
  if (cudaMalloc(&sm, small) != cudaSuccess) {
    cudaGetLastError();
    return PSD_ERR_NO_MEMORY;
  }
  cudaMemset(sm, 0, small);
  p->d_args = reinterpret_cast<DevArgs*>(sm);
  p->d_state = reinterpret_cast<DevState*>(sm + o_state);
  p->d_info = reinterpret_cast<psd_info_t*>(sm + o_info);
  p->d_block = reinterpret_cast<BlockRec*>(sm + o_block);
  p->d_tiles = reinterpret_cast<int4*>(sm + o_tiles);
  p->d_compl = reinterpret_cast<double*>(sm + o_compl);
  p->d_tiles_pair = reinterpret_cast<int4*>(sm + o_pair);
  if (!tiles.empty() &&
      cudaMemcpy(p->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return PSD_ERR_CUDA;
  if (!tiles_pair.empty() && cudaMemcpy(p->d_tiles_pair, tiles_pair.data(), sizeof(int4) * tiles_pair.size(),
                                        cudaMemcpyHostToDevice) != cudaSuccess)
    return PSD_ERR_CUDA;
  BlockRec br{};
  br.off = 0;
  br.n = static_cast<int>(n);
  br.st = p->d_state;
  if (cudaMemcpy(p->d_block, &br, sizeof(br), cudaMemcpyHostToDevice) != cudaSuccess) return PSD_ERR_CUDA;
  return PSD_OK;
}

void* part_ptr(const Plan* p, const Mat& m, int part) {
  return p->slots + (static_cast<size_t>(m.slot) + static_cast<size_t>(part * kind_lo_step(m.kind))) * p->slot_size;
}

GemmParams base_params(const Plan* p) {
  GemmParams g{};
  g.num_tiles = p->ntiles;
  g.tiles = p->d_tiles;
  g.blocks = p->d_block;
  g.ep.status = &p->d_state->status;
  return g;
}

// One product C = epi(A * B) (routes: chain.h gemm_route); `out` is the
// output matrix (ignored for EPI_FINAL), `Y` the EPI_POLY operand.
cudaError_t gemm(Plan* p, int epi, const Mat& A, const Mat& B, const Mat* out, const Mat* Y, float a, float b,
                 float c, float sc, unsigned* absmax, cudaStream_t s) {
  GemmParams g = base_params(p);
  const int64_t n = p->n, ldm = p->ldm;
  g.ep.a = a;
  g.ep.b = b;
  g.ep.c = c;
  g.ep.s = sc;
  g.ep.absmax = absmax;
  if (epi != EPI_FINAL) {
    g.ep.C = part_ptr(p, *out, 0);
    g.ep.C_lo = kind_is_pair(out->kind) ? part_ptr(p, *out, 1) : nullptr;
    g.ep.ldc = ldm;
  }
  if (epi == EPI_POLY) {
    g.ep.Y = part_ptr(p, *Y, 0);
    g.ep.Y_lo = kind_is_pair(Y->kind) ? part_ptr(p, *Y, 1) : nullptr;
    g.ep.ldy = ldm;
  }
  if (epi == EPI_FINAL) {
    g.ep.cres = p->d_compl;
    p->ncompl = 4 * p->ntiles;
  }
  g.ep.in_scale = 1.f / (A.scale * B.scale);
  g.ep.y_scale = Y ? 1.f / Y->scale : 1.f;
  g.ep.out_scale = out ? out->scale : 1.f;
  const int grid = num_sms();
  const GemmRoute route = gemm_route(A, B);
  if (route == ROUTE_16) {
    const int dt = kind_dtype(A);
    const int odt = out ? kind_dtype(*out) : -1;
    if ((dt == DT_F16 || dt == DT_BF16) &&
        (epi == EPI_FINAL || odt == dt || (odt == DT_F16X2 && dt == DT_F16))) {
      // 16-bit products on CTA pairs: M = 256, half of B in each CTA (128-row boxes)
      CUtensorMap ta, tb;
      if (!encode_tmap(&ta, dt, part_ptr(p, A, 0), n, ldm, 128) || !encode_tmap(&tb, dt, part_ptr(p, B, 0), n, ldm, 128))
        return cudaErrorInvalidValue;
      const uint32_t fmt = dt == DT_BF16 ? 1u : 0u;
      g.num_tiles = p->ntiles_pair;
      g.tiles = p->d_tiles_pair;
      g.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (16u << 24);  // M = 256; N per tile
      if (epi == EPI_FINAL) p->ncompl = 8 * p->ntiles_pair;
      return launch_symgemm_pair(dt, epi, ta, tb, g, grid, s, epi == EPI_FINAL ? -1 : odt);
    }
    CUtensorMap ta, tb;
    if (!encode_tmap(&ta, dt, part_ptr(p, A, 0), n, ldm, 128) || !encode_tmap(&tb, dt, part_ptr(p, B, 0), n, ldm, 256))
      return cudaErrorInvalidValue;
    const uint32_t fmt = dt == DT_BF16 ? 1u : 0u;  // F16 and E4M3 are both format 0 in their MMA kinds
    g.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (8u << 24);  // M = 128; N per tile
    return launch_symgemm(dt, epi, ta, tb, g, grid, s, out ? kind_dtype(*out) : -1);
  }
  if (route == ROUTE_NONE) return cudaErrorNotSupported;
  const bool b1 = route == ROUTE_X2;
  const Mat& PA = b1 ? B : A;  // the pair operand goes first
  const Mat& PB = b1 ? A : B;
  const int dt = kind_dtype(PA);
  CUtensorMap tm[4];
  const int rb = x3_row_bytes(b1);
  const int out_mode = epi == EPI_FINAL ? 2 : (kind_is_pair(out->kind) ? 0 : 1);
  // FP16-pair stage products on CTA pairs (M = 256, half of B in each CTA)
  const bool pair = dt == DT_F16X2 && epi != EPI_FINAL &&
                    (b1 ? (epi == EPI_SCALE && out_mode == 1) : out_mode == 0);
  const int brows = pair ? 128 : 256;
  if (!encode_tmap(&tm[0], dt, part_ptr(p, PA, 0), n, ldm, 128, rb) ||
      !encode_tmap(&tm[1], dt, part_ptr(p, PA, 1), n, ldm, 128, rb) ||
      !encode_tmap(&tm[2], dt, part_ptr(p, PB, 0), n, ldm, brows, rb) ||
      !encode_tmap(&tm[3], dt, part_ptr(p, PB, b1 ? 0 : 1), n, ldm, brows, rb))
    return cudaErrorInvalidValue;
  if (pair) {
    g.num_tiles = p->ntiles_pair;
    g.tiles = p->d_tiles_pair;
  }
  return launch_symgemm_x3(dt, b1, epi, out_mode, tm, g, grid, s, pair);
}

struct PlanOps {
  Plan* p;
  cudaStream_t s;
  cudaError_t cast(const Mat& X0) {
    return enqueue_scale_cast(kind_dtype(X0), p->d_args, p->d_state, p->n, part_ptr(p, X0, 0),
                              kind_is_pair(X0.kind) ? part_ptr(p, X0, 1) : nullptr, p->ldm, s);
  }
  cudaError_t gemm(int epi, const Mat& A, const Mat& B, const Mat* out, const Mat* Y, float a, float b, float c,
                   float sc, bool track) {
    return psd::gemm(p, epi, A, B, out, Y, a, b, c, sc, track ? &p->d_state->absmax_bits : nullptr, s);
  }
  cudaError_t finish() { return enqueue_finalize(p->d_args, p->d_state, s, p->d_compl, p->ncompl); }
};

// Enqueue the whole projection (used for graph capture and for direct launch).
cudaError_t enqueue_projection(Plan* p, cudaStream_t s) {
  cudaError_t e;
  if ((e = enqueue_norm_bound(p->L, p->d_args, p->d_state, s)) != cudaSuccess) return e;
  PlanOps ops{p, s};
  return run_chain(p->prec, p->sched, p->nslots, dtype16_of(p->prec), ops);
}

Plan* get_plan(int dev, cudaStream_t stream, int64_t n, psd_precision_t prec, void* user_ws, size_t user_bytes,
               psd_status_t* st) {
  PlanKey key{dev, stream, n, static_cast<int>(prec), user_ws};
  auto it = g_plans.find(key);
  if (it != g_plans.end()) {
    *st = PSD_OK;
    return it->second;
  }
  Plan* p = new Plan();
  p->device = dev;
  p->stream = stream;
  p->n = n;
  p->prec = prec;
  *st = build_plan(p, user_ws, user_bytes);
  if (*st != PSD_OK) {
    free_plan(p);
    return nullptr;
  }
  g_plans[key] = p;
  return p;
}

// Capture the projection into a graph on a private stream (once per plan).
void ensure_graph(Plan* p) {
  if (p->graph_tried) return;
  p->graph_tried = true;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    cudaError_t e = enqueue_projection(p, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess && e2 == cudaSuccess && graph) {
      size_t nodes = 0;
      cudaGraphGetNodes(graph, nullptr, &nodes);
      p->launches = static_cast<int>(nodes) + 1;
      if (cudaGraphInstantiate(&p->exec, graph, 0) != cudaSuccess) p->exec = nullptr;
    }
    if (graph) cudaGraphDestroy(graph);
  }
  cudaGetLastError();
  cudaStreamDestroy(cs);
}

bool ranges_overlap(const float* a, const float* b, int64_t n, int64_t lda, int64_t ldb) {
  const char* a0 = reinterpret_cast<const char*>(a);
  const char* a1 = reinterpret_cast<const char*>(a + (n - 1) * lda + n);
  const char* b0 = reinterpret_cast<const char*>(b);
  const char* b1 = reinterpret_cast<const char*>(b + (n - 1) * ldb + n);
  return a0 < b1 && b0 < a1;
}

psd_status_t project_impl(int64_t n, const float* X, int64_t ld, float* out, int64_t ld_out,
                          psd_precision_t prec, psd_info_t* d_info, void* ws, size_t ws_bytes,
                          cudaStream_t stream) {
  if (n < 0 || n > kMaxOrder) return PSD_ERR_INVALID_ARG;
  if (prec < PSD_PREC_FP32 || prec > PSD_PREC_FP8_LATE) return PSD_ERR_INVALID_ARG;
  if (n == 0) return PSD_OK;
  if (!X || !out || ld < n || ld_out < n) return PSD_ERR_INVALID_ARG;
  if (ranges_overlap(X, out, n, ld, ld_out) && !(static_cast<const void*>(X) == out && ld == ld_out))
    return PSD_ERR_INVALID_ARG;
  if (!prec_built(prec)) return PSD_ERR_UNSUPPORTED;
  psd_status_t st = check_device();
  if (st != PSD_OK) return st;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  Plan* p = get_plan(dev, stream, n, prec, ws, ws_bytes, &st);
  if (!p) return st;
  ensure_graph(p);
  DevArgs h{X, ld, out, ld_out, d_info ? d_info : p->d_info};
  if (enqueue_set_args(p->d_args, h, stream, p->d_block) != cudaSuccess) return PSD_ERR_CUDA;
  cudaError_t e = p->exec ? cudaGraphLaunch(p->exec, stream) : enqueue_projection(p, stream);
  if (e != cudaSuccess) return PSD_ERR_CUDA;
  if (!d_info) g_last[{dev, stream}] = p;
  return PSD_OK;
}

// --- scratch for the building-block entry point
struct ProductScratch {
  DevArgs* d_args = nullptr;
  DevState* d_state = nullptr;
  BlockRec* d_block = nullptr;
  std::map<int64_t, int4*> tiles;
  std::map<int64_t, int> ntiles;
};
std::map<int, ProductScratch> g_prod;

__global__ void set_lambda_kernel(DevState* st, double lam) {
  st->lambda = lam;
  st->status = 0;
}

}  // namespace
}  // namespace psd

using namespace psd;

extern "C" {

psd_status_t psd_project(int64_t n, const float* X, int64_t ld, float* out, psd_precision_t precision,
                         psd_stream_t stream) {
  return project_impl(n, X, ld, out, ld, precision, nullptr, nullptr, 0,
                      reinterpret_cast<cudaStream_t>(stream));
}

psd_status_t psd_project_ex(int64_t n, const float* X, int64_t ld, float* out, int64_t ld_out,
                            psd_precision_t precision, psd_info_t* d_info, void* workspace, size_t ws_bytes,
                            psd_stream_t stream) {
  if (workspace && ws_bytes == 0) return PSD_ERR_INVALID_ARG;
  return project_impl(n, X, ld, out, ld_out, precision, d_info, workspace, ws_bytes,
                      reinterpret_cast<cudaStream_t>(stream));
}

size_t psd_workspace_size(int64_t n, psd_precision_t precision) {
  if (n <= 0 || n > kMaxOrder || precision < PSD_PREC_FP32 || precision > PSD_PREC_FP8_LATE) return 0;
  return total_ws_bytes(n, precision);
}

psd_status_t psd_last_info(psd_stream_t stream, psd_info_t* host_info) {
  if (!host_info) return PSD_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PSD_ERR_CUDA;
  Plan* p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_last.find({dev, reinterpret_cast<cudaStream_t>(stream)});
    if (it == g_last.end()) return PSD_ERR_INVALID_ARG;
    p = it->second;
  }
  if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return PSD_ERR_CUDA;
  if (cudaMemcpy(host_info, p->d_info, sizeof(psd_info_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PSD_ERR_CUDA;
  return PSD_OK;
}

psd_status_t psd_release_workspaces(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaDeviceSynchronize();
  for (auto& kv : g_plans) free_plan(kv.second);
  g_plans.clear();
  g_last.clear();
  for (auto& kv : g_prod) {
    if (kv.second.d_args) cudaFree(kv.second.d_args);
    for (auto& t : kv.second.tiles) cudaFree(t.second);
  }
  g_prod.clear();
  release_deflate_plans();
  release_batched_plans();
  return PSD_OK;
}

psd_status_t psd_norm_bound(int64_t n, const float* X, int64_t ld, psd_info_t* d_info, psd_stream_t stream) {
  if (n <= 0 || n > kMaxOrder || !X || ld < n || !d_info) return PSD_ERR_INVALID_ARG;
  psd_status_t st = check_device();
  if (st != PSD_OK) return st;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(g_mu);
  Plan* p = get_plan(dev, s, n, PSD_PREC_FP16, nullptr, 0, &st);
  if (!p) return st;
  DevArgs h{X, ld, nullptr, 0, d_info};
  if (enqueue_set_args(p->d_args, h, s) != cudaSuccess) return PSD_ERR_CUDA;
  if (enqueue_norm_bound(p->L, p->d_args, p->d_state, s) != cudaSuccess) return PSD_ERR_CUDA;
  return PSD_OK;
}

psd_status_t psd_symm_product(int64_t n, const void* A, const void* B, int64_t ld, void* C, int64_t ld_out,
                              psd_precision_t precision, int32_t epi, const double* params, const void* aux,
                              int64_t ld_aux, float* d_absmax, psd_stream_t stream) {
  if (n <= 0 || n > kMaxOrder || !A || !B || !C || ld < n || (ld % 8) != 0) return PSD_ERR_INVALID_ARG;
  const bool split = precision == PSD_PREC_MIXED || precision == PSD_PREC_FP32;
  const bool f8 = precision == PSD_PREC_FP8_LATE;
  if (precision != PSD_PREC_FP16 && precision != PSD_PREC_BF16 && !split && !f8) return PSD_ERR_INVALID_ARG;
  const int flags = epi & ~0xFF;
  epi &= 0xFF;
  const bool grouped = (flags & PSD_EPI_GROUPED) != 0, pair_out = (flags & PSD_EPI_F16_PAIR_OUT) != 0;
  const bool cta_pair = (flags & PSD_EPI_CTA_PAIR) != 0;
  if (flags & ~(PSD_EPI_GROUPED | PSD_EPI_F16_PAIR_OUT | PSD_EPI_CTA_PAIR)) return PSD_ERR_INVALID_ARG;
  if ((grouped || pair_out) && (split || f8 || epi == 3)) return PSD_ERR_INVALID_ARG;
  if (cta_pair && (f8 || precision == PSD_PREC_FP32)) return PSD_ERR_INVALID_ARG;
  if (grouped && cta_pair) return PSD_ERR_INVALID_ARG;
  if (pair_out && (precision != PSD_PREC_FP16 || epi == 2)) return PSD_ERR_INVALID_ARG;
  if (epi < 0 || epi > 3) return PSD_ERR_INVALID_ARG;
  if (f8 && (epi == 3 || (ld % 16) != 0 || !params)) return PSD_ERR_INVALID_ARG;
  if (precision == PSD_PREC_MIXED && epi == 3) return PSD_ERR_INVALID_ARG;  // FP16 pairs: epi 0-2
  if ((epi == 1 || epi == 2 || epi == 3) && !params) return PSD_ERR_INVALID_ARG;
  if ((epi == 1 || epi == 3) && !aux) return PSD_ERR_INVALID_ARG;
  if (epi == 3 && (ld_aux < n || ld_out < n)) return PSD_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15) ||
      (reinterpret_cast<uintptr_t>(C) & 15))
    return PSD_ERR_INVALID_ARG;
  psd_status_t st = check_device();
  if (st != PSD_OK) return st;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(g_mu);
  ProductScratch& ps = g_prod[dev];
  if (!ps.d_args) {
    const size_t o_state = round_up(sizeof(DevArgs), 256);
    const size_t o_block = o_state + round_up(sizeof(DevState), 256);
    const size_t bytes = o_block + round_up(sizeof(BlockRec), 256);
    uint8_t* sm = nullptr;
    if (cudaMalloc(&sm, bytes) != cudaSuccess) return PSD_ERR_NO_MEMORY;
    cudaMemset(sm, 0, bytes);
    ps.d_args = reinterpret_cast<DevArgs*>(sm);
    ps.d_state = reinterpret_cast<DevState*>(sm + o_state);
    ps.d_block = reinterpret_cast<BlockRec*>(sm + o_block);
  }
  const int64_t tkey = cta_pair ? -n : n;  // the pair form's 256-row tiles under -n
  if (!ps.tiles.count(tkey)) {
    std::vector<int4> tl = cta_pair ? make_tile_list_pair(n) : make_tile_list(n);
    int4* d = nullptr;
    if (cudaMalloc(&d, sizeof(int4) * tl.size()) != cudaSuccess) return PSD_ERR_NO_MEMORY;
    cudaMemcpy(d, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice);
    ps.tiles[tkey] = d;
    ps.ntiles[tkey] = static_cast<int>(tl.size());
  }
  const int dtype = precision == PSD_PREC_BF16    ? DT_BF16
                    : precision == PSD_PREC_MIXED ? DT_F16X2
                    : precision == PSD_PREC_FP32  ? DT_TF32X3
                    : f8                          ? DT_E4M3
                                                  : DT_F16;
  const size_t esz = dtype == DT_TF32X3 ? 4 : (f8 ? 1 : 2);
  const size_t pair = static_cast<size_t>(n) * static_cast<size_t>(ld) * esz;  // byte offset of the lo part
  GemmParams g{};
  g.num_tiles = ps.ntiles[tkey];
  g.tiles = ps.tiles[tkey];
  g.blocks = ps.d_block;
  g.ep.C = C;
  g.ep.C_lo = (split || pair_out) ? static_cast<uint8_t*>(C) + pair : nullptr;
  g.ep.ldc = ld;
  g.ep.status = &ps.d_state->status;
  g.ep.absmax = reinterpret_cast<unsigned*>(d_absmax);
  if (epi == 1) {
    g.ep.Y = aux;
    g.ep.Y_lo = split ? static_cast<const uint8_t*>(aux) + pair : nullptr;
    g.ep.ldy = ld;
    g.ep.a = static_cast<float>(params[0]);
    g.ep.b = static_cast<float>(params[1]);
    g.ep.c = static_cast<float>(params[2]);
  } else if (epi == 2) {
    g.ep.s = static_cast<float>(params[0]);
  } else if (epi == 3) {
    set_lambda_kernel<<<1, 1, 0, s>>>(ps.d_state, params[0]);
    g.ep.absmax = nullptr;
  }
  if (f8) {
    const double* sc = params + (epi == 0 ? 0 : epi == 1 ? 3 : 1);
    g.ep.in_scale = static_cast<float>(sc[0]);
    g.ep.y_scale = static_cast<float>(sc[1]);
    g.ep.out_scale = static_cast<float>(sc[2]);
    g.ep.absmax = nullptr;
  }
  BlockRec br{};
  br.off = 0;
  br.n = static_cast<int>(n);
  br.st = ps.d_state;
  if (epi == 3) {
    br.X = static_cast<const float*>(aux);
    br.ld = ld_aux;
    br.out = static_cast<float*>(C);
    br.ld_out = ld_out;
  }
  if (enqueue_set_block(ps.d_block, br, s) != cudaSuccess) return PSD_ERR_CUDA;
  cudaError_t e;
  if (cta_pair && !split) {
    CUtensorMap ta, tb;
    if (!encode_tmap(&ta, dtype, A, n, ld, 128) || !encode_tmap(&tb, dtype, B, n, ld, 128)) return PSD_ERR_CUDA;
    const uint32_t fmt = dtype == DT_BF16 ? 1u : 0u;
    g.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (16u << 24);  // M = 256; N per tile
    e = launch_symgemm_pair(dtype, epi, ta, tb, g, num_sms(), s, pair_out ? DT_F16X2 : -1);
  } else if (!split) {
    CUtensorMap ta, tb;
    if (!encode_tmap(&ta, dtype, A, n, ld, 128) || !encode_tmap(&tb, dtype, B, n, ld, 256)) return PSD_ERR_CUDA;
    const uint32_t fmt = dtype == DT_BF16 ? 1u : 0u;
    g.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (8u << 24);  // M = 128; N per tile
    e = launch_symgemm(dtype, epi, ta, tb, g, num_sms(), s, pair_out ? DT_F16X2 : -1, grouped);
  } else {
    CUtensorMap tm[4];
    const uint8_t* a8 = static_cast<const uint8_t*>(A);
    const uint8_t* b8 = static_cast<const uint8_t*>(B);
    const int rb = x3_row_bytes(false);
    const int brows = cta_pair ? 128 : 256;
    if (!encode_tmap(&tm[0], dtype, a8, n, ld, 128, rb) || !encode_tmap(&tm[1], dtype, a8 + pair, n, ld, 128, rb) ||
        !encode_tmap(&tm[2], dtype, b8, n, ld, brows, rb) || !encode_tmap(&tm[3], dtype, b8 + pair, n, ld, brows, rb))
      return PSD_ERR_CUDA;
    e = launch_symgemm_x3(dtype, false, epi, epi == 3 ? 2 : 0, tm, g, num_sms(), s, cta_pair);
  }
  return e == cudaSuccess ? PSD_OK : PSD_ERR_CUDA;
}

psd_status_t psd_debug_set(int32_t knob, double value) {
  if (knob == PSD_DEBUG_BOUND_SCALE) {
    if (!(value > 0.0) || !std::isfinite(value)) return PSD_ERR_INVALID_ARG;
  } else if (knob == PSD_DEBUG_BARRIER_LIMIT_NS) {
    if (!(value >= 0.0) || !(value <= 6.0e10)) return PSD_ERR_INVALID_ARG;  // at most a minute
  } else {
    return PSD_ERR_INVALID_ARG;
  }
  psd_status_t st = check_device();
  if (st != PSD_OK) return st;
  if (set_norm_bound_debug(knob, value) != cudaSuccess) return PSD_ERR_CUDA;
  if (knob == PSD_DEBUG_BARRIER_LIMIT_NS &&
      set_batch_flow_limit(static_cast<unsigned long long>(value)) != cudaSuccess)
    return PSD_ERR_CUDA;
  return PSD_OK;
}

const char* psd_status_string(psd_status_t status) {
  switch (status) {
    case PSD_OK: return "ok";
    case PSD_ERR_INVALID_ARG: return "invalid argument";
    case PSD_ERR_CUDA: return "CUDA runtime error";
    case PSD_ERR_NO_MEMORY: return "out of device memory or workspace too small";
    case PSD_ERR_NONFINITE: return "non-finite value in the input or an iterate";
    case PSD_ERR_BOUND: return "norm bound below ||X||_2: the filter diverged";
    case PSD_ERR_TIMEOUT: return "a bounded device wait timed out";
    case PSD_ERR_UNSUPPORTED: return "unsupported device or precision";
    case PSD_ERR_CANCELED: return "request canceled before it ran";
    default: return "unknown status";
  }
}

psd_status_t psd_schedule(psd_precision_t precision, int32_t* T, double* coef, double* post_scale) {
  Schedule s;
  if (!T || !coef || !post_scale || !get_schedule(precision, s)) return PSD_ERR_INVALID_ARG;
  *T = s.T;
  for (int t = 0; t < s.T; ++t) {
    for (int k = 0; k < 3; ++k) coef[3 * t + k] = s.coef[t][k];
    post_scale[t] = s.post[t];
  }
  return PSD_OK;
}

int32_t psd_kernel_launches(int64_t n, psd_precision_t precision, psd_stream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_plans.find(PlanKey{dev, reinterpret_cast<cudaStream_t>(stream), n, static_cast<int>(precision), nullptr});
  return it == g_plans.end() ? 0 : it->second->launches;
}

int32_t psd_gemm_count(psd_precision_t precision) {
  Schedule s;
  if (!get_schedule(precision, s)) return 0;
  return 3 * s.T + 1;
}

const char* psd_version(void) { return "psdproj 0.1 (sm_103a)"; }

}  // extern "C"
