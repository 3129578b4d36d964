// sar_backproject_noalloc: backprojection whose only scratch (the partial
// sums of pixel tiles that several CTAs share) lives in a static device array
// of this library instead of memory the plan allocates.
//
// Who needs it: callers that cannot allocate device memory while they image
// frames -- embedded or safety-certified automotive processes that allocate
// only at start-up, or hosts whose device memory is reserved in advance by
// another allocator.  The call itself issues no cudaMalloc, cudaFree or other
// allocating call; the array below exists on every GPU that loads the
// library, for the lifetime of the process.
#include <mutex>

#include "sar_internal.h"

namespace {

// Maximum scratch: 16 MiB (2 Mi complex64 partial sums, 2048 tile slots of
// 1024 points).
constexpr size_t kScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_bp_scratch[kScratchBytes / sizeof(float2)];

std::mutex g_setup_mutex;
float2 *g_scratch_addr[kMaxDevices] = {};

// Device address of g_bp_scratch on `dev` (which must be current).  Looked up
// once per device, on the first call there.  In host code the name
// g_bp_scratch is only a host-side handle, never a device address.
int scratch_address(int dev, float2 **out) {
    if (dev < 0 || dev >= kMaxDevices) return SAR_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bp_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return SAR_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<float2 *>(p);
    }
    *out = g_scratch_addr[dev];
    return SAR_OK;
}

}  // namespace

extern "C" int sar_backproject_noalloc(sar_plan *plan, const void *prof_dev, int32_t M, const double *q_tx_dev,
                                       const double *q_rx_dev, const float *fdopp_idx_dev, void *image_dev,
                                       int32_t accumulate, void *stream) {
    if (!plan || !prof_dev || !q_tx_dev || !q_rx_dev || !image_dev || M < 1) return SAR_EINVAL;
    const auto aligned = [](const void *p, size_t a) { return ((uintptr_t)p % a) == 0; };
    if (!aligned(prof_dev, 256) || !aligned(q_tx_dev, 16) || !aligned(q_rx_dev, 16) || !aligned(image_dev, 8) ||
        (fdopp_idx_dev && !aligned(fdopp_idx_dev, 4)))
        return SAR_EINVAL;
    const int dev = sar::plan_device(plan);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return SAR_ECUDA;
    if (cur != dev && cudaSetDevice(dev) != cudaSuccess) return SAR_ECUDA;
    float2 *scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc == SAR_OK)
        rc = sar::backproject_with_scratch(plan, prof_dev, M, q_tx_dev, q_rx_dev, fdopp_idx_dev, image_dev,
                                           accumulate, scratch, kScratchBytes, (cudaStream_t)stream);
    if (cur != dev) cudaSetDevice(cur);
    return rc;
}
