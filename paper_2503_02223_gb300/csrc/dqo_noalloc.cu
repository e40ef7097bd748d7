// dqo_depth_order_noalloc: the depth radix sort of the rasterizer for callers that must
// not allocate device memory.
//
// Some hosts of this library cannot call cudaMalloc once they are running: a real-time
// mapping loop where an allocation's implicit device synchronisation would stall the
// frame, a plugin whose host framework owns all device memory through its own pool, or
// an embedded deployment that reserves its memory budget up front.  This entry point
// runs the same stable radix sort the forward render uses for its depth ordering, with
// all scratch memory in a fixed array that lives in the library image.
//
// The scratch array below is a static __device__ array: every GPU that loads this
// library holds it (about 16 MiB) until the process exits.  In host code its name is
// only a host-side stand-in, so the device address is fetched once per device with
// cudaGetSymbolAddress (done by the first call on that device, which may also load the
// library's device code onto that GPU) and passed to the kernels.  All calls share the
// one array and it keeps the last call's contents, so calls that overlap on the GPU (on
// different streams, or from different host threads) race with each other and must be
// serialised by the caller.  A word of the array records whether a look-back wait of the
// sort gave up; each call clears it first and copies it to the caller's status word.
#include <mutex>

#include "dqo_internal.cuh"

namespace dqo {
namespace {

constexpr int64_t kNoAllocMaxKeys = int64_t(1) << 20;
// a radix pass takes at least 2048 keys per CTA (4096 once every SM has a CTA): at most
// 2^20 / 2048 = 512 CTAs on any GPU
constexpr int64_t kNoAllocMaxBlocks = kNoAllocMaxKeys / 2048;
// layout: keys_a | keys_b | vals_b (uint32 each) | sort scratch (histograms, look-back status
// of up to 8 passes, counters) | error word (256 bytes reserved)
constexpr size_t kKeysBytes = sizeof(uint32_t) * kNoAllocMaxKeys;
constexpr size_t kHistWords = onesweep_scratch_words(kNoAllocMaxBlocks, kMaxRadixPasses);
constexpr size_t kHistBytes = (sizeof(uint32_t) * kHistWords + 255) / 256 * 256;
constexpr size_t kErrBytes = 256;
constexpr size_t kScratchBytes = 3 * kKeysBytes + kHistBytes + kErrBytes;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, fetched once per device.
cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Copies the caller's keys into scratch (the sort ping-pongs in place) and seeds the
// value array with the identity permutation.
__global__ void k_seed_order(const uint32_t* __restrict__ keys_in, uint32_t* __restrict__ keys,
                             uint32_t* __restrict__ order, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    keys[i] = keys_in[i];
    order[i] = (uint32_t)i;
  }
}

// The caller's status word: the sort's error word (0: the order is valid, 1: a look-back
// wait gave up).
__global__ void k_report_status(const uint32_t* __restrict__ err, uint32_t* __restrict__ status) {
  *status = *err;
}

}  // namespace
}  // namespace dqo

extern "C" dqo_status dqo_depth_order_noalloc(const uint32_t* depth_keys, int64_t n, uint32_t* order,
                                              uint32_t* status, dqo_stream stream_) {
  using namespace dqo;
  if (n < 0 || n > kNoAllocMaxKeys) return DQO_EINVAL;
  if (n > 0 && (!depth_keys || !order)) return DQO_EINVAL;
  if (n > 0 && radix_scratch_words(n) > kHistWords) return DQO_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
  if (n == 0) {
    if (status && cudaMemsetAsync(status, 0, sizeof(uint32_t), s) != cudaSuccess) return DQO_ECUDA;
    return DQO_OK;
  }
  unsigned char* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return DQO_ECUDA;
  uint32_t* keys_a = reinterpret_cast<uint32_t*>(base);
  uint32_t* keys_b = reinterpret_cast<uint32_t*>(base + kKeysBytes);
  uint32_t* vals_b = reinterpret_cast<uint32_t*>(base + 2 * kKeysBytes);
  uint32_t* hist = reinterpret_cast<uint32_t*>(base + 3 * kKeysBytes);
  uint32_t* err = reinterpret_cast<uint32_t*>(base + 3 * kKeysBytes + kHistBytes);
  // the previous call's error word stays in the array: clear it before this sort
  if (cudaMemsetAsync(err, 0, sizeof(uint32_t), s) != cudaSuccess) return DQO_ECUDA;
  k_seed_order<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(depth_keys, keys_a, order, n);
  if (cudaGetLastError() != cudaSuccess) return DQO_ECUDA;
  // 32-bit keys take an even number of 8-bit passes, so the sorted indices end in `order`
  int sel = 0;
  if (radix_sort_u32(keys_a, keys_b, order, vals_b, n, 32, hist, &sel, s, nullptr, err) != cudaSuccess)
    return DQO_ECUDA;
  if (sel != 0) return DQO_ECUDA;
  if (status) {
    k_report_status<<<1, 1, 0, s>>>(err, status);
    if (cudaGetLastError() != cudaSuccess) return DQO_ECUDA;
  }
  return DQO_OK;
}
