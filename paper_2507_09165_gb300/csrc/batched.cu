// Batched projection of a block-diagonal cone and the request server.
//
// psd_project_batched: the descriptors live in device memory; their orders
// are read back once per call, then every block is projected on `stream`
// through the same per-order plan as psd_project_ex, so a block's result is
// bit-identical alone and in the batch.
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

extern "C" psd_status_t psd_project_ex(int64_t n, const float* X, int64_t ld, float* out, int64_t ld_out,
                                       psd_precision_t precision, psd_info_t* d_info, void* workspace,
                                       size_t ws_bytes, psd_stream_t stream);

extern "C" psd_status_t psd_project_batched(int32_t count, const psd_block_desc_t* d_descs,
                                            psd_precision_t precision, psd_stream_t stream) {
  if (count < 0 || (count > 0 && !d_descs)) return PSD_ERR_INVALID_ARG;
  if (count == 0) return PSD_OK;
  std::vector<psd_block_desc_t> h(static_cast<size_t>(count));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(h.data(), d_descs, sizeof(psd_block_desc_t) * h.size(), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PSD_ERR_CUDA;
  for (const auto& d : h)
    if (d.n < 0 || d.n > 1024 || (d.n > 0 && (!d.X || !d.out || d.ld < d.n || d.ld_out < d.n)))
      return PSD_ERR_INVALID_ARG;
  for (const auto& d : h) {
    if (d.n == 0) continue;
    psd_status_t st = psd_project_ex(d.n, d.X, d.ld, d.out, d.ld_out, precision, d.info, nullptr, 0, stream);
    if (st != PSD_OK) return st;
  }
  return PSD_OK;
}
