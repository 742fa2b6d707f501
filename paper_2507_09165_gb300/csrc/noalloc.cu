// psd_norm_bound_noalloc: the norm bound (the same kernels as psd_norm_bound)
// with all of its scratch memory in one file-scope device array of fixed size,
// so that a call allocates nothing.
//
// Who needs this: callers that must not allocate device memory while they
// run -- a solver or serving loop whose memory is reserved up front by a pool
// that owns the GPU's free memory (a cudaMalloc there fails or fragments the
// pool), or a latency-critical loop that cannot afford the implicit device
// synchronisation cudaMalloc/cudaFree may perform.  They still pass their own
// input and report buffers.
//
// The array g_noalloc_scratch holds the argument block, the device state and
// the Lanczos buffers for orders up to kNoAllocMaxOrder (about 3 MB); every
// GPU that loads the library holds it until the process exits.  In host code
// the array's name is only a host-side stand-in, so the device address is
// looked up with cudaGetSymbolAddress on the first call made with a device
// current (make that first call before any stream capture).  The address is
// kept per device together with the CUDA context it belongs to; if the
// device's current context is a different one (the primary context was torn
// down, e.g. by cudaDeviceReset, and the module loaded anew), it is looked up
// again.
//
// All calls share the array and it keeps the last call's contents: the first
// kernel of each call resets the device state record, and every other scratch
// word is written before it is read.  Calls whose work overlaps on the GPU
// (different streams, or different host threads without ordering) race on the
// array and must not be issued; calls on one stream are ordered and safe.
#include <mutex>

#include "internal.h"

namespace psd {
namespace {

constexpr int64_t kNoAllocMaxOrder = 4096;
constexpr size_t kRecordBytes = 1024;  // argument block (256) + device state (768)

constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Upper bound of lanczos_bytes(n) (normbound.cu), evaluated at compile time.
constexpr size_t lanczos_bound_bytes(int64_t n) {
  const size_t npad = static_cast<size_t>((n + 255) / 256 * 256);
  const size_t nb = static_cast<size_t>((n + 127) / 128);
  const size_t ntiles = nb * (nb + 1) / 2;
  const size_t nctas = static_cast<size_t>((n + kVecThreads - 1) / kVecThreads);
  const size_t npart = static_cast<size_t>((n + 31) / 32);
  return round256(8 * 21 * npad) + round256(8 * 3 * npad) + round256(4 * 2 * npad) +
         round256(8 * 2 * nb * npad) + round256(8 * 32 * npart) + round256(8 * 32 * npart) +
         round256(8 * (npart > nctas ? npart : nctas)) + round256(8 * ntiles) + round256(4 * 2);
}

constexpr size_t kNoAllocBytes = kRecordBytes + lanczos_bound_bytes(kNoAllocMaxOrder);
static_assert(sizeof(DevArgs) <= 256 && sizeof(DevState) <= kRecordBytes - 256, "records exceed their slots");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mu;
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

// cuCtxGetCurrent through the runtime's driver entry point (the library does
// not link libcuda directly).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      ptr = nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(ptr);
  }();
  return fn;
}

}  // namespace
}  // namespace psd

using namespace psd;

extern "C" psd_status_t psd_norm_bound_noalloc(int64_t n, const float* X, int64_t ld, psd_info_t* d_info,
                                               psd_stream_t stream) {
  if (n <= 0 || !X || ld < n || !d_info) return PSD_ERR_INVALID_ARG;
  if (n > kNoAllocMaxOrder) return PSD_ERR_INVALID_ARG;  // beyond the static scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PSD_ERR_CUDA;
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return PSD_ERR_UNSUPPORTED;
  if (lanczos_bytes(n) + kRecordBytes > kNoAllocBytes) return PSD_ERR_INVALID_ARG;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    CtxGetCurrentFn get_ctx = ctx_get_current();
    if (!get_ctx) return PSD_ERR_CUDA;
    // null until the runtime has made the device's primary context current on
    // this thread; cudaGetSymbolAddress does that
    CUcontext ctx = nullptr;
    if (get_ctx(&ctx) != CUDA_SUCCESS) return PSD_ERR_CUDA;
    if (!ctx || !g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return PSD_ERR_CUDA;
      }
      if (get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return PSD_ERR_CUDA;
      g_scratch_addr[dev] = p;
      g_scratch_ctx[dev] = ctx;
    }
    base = g_scratch_addr[dev];
  }
  uint8_t* b = static_cast<uint8_t*>(base);
  DevArgs* args = reinterpret_cast<DevArgs*>(b);
  DevState* st = reinterpret_cast<DevState*>(b + 256);
  LanczosBufs L;
  lanczos_carve(L, n, b + kRecordBytes);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DevArgs h{X, ld, nullptr, 0, d_info};
  if (enqueue_set_args(args, h, s) != cudaSuccess) return PSD_ERR_CUDA;
  if (enqueue_norm_bound(L, args, st, s) != cudaSuccess) return PSD_ERR_CUDA;
  return PSD_OK;
}
