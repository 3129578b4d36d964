// sar_backproject_noalloc: backprojection whose only scratch (the partial
// sums of pixel tiles that several CTAs share) lives in a static device array
// of this library instead of memory the plan allocates.
//
// Who needs it: callers that cannot allocate device memory while they image
// frames -- embedded or safety-certified automotive processes that allocate
// only at start-up, or hosts whose device memory is reserved in advance by
// another allocator.  The call itself issues no cudaMalloc, cudaFree or other
// allocating call; the array below exists on every GPU where a plan was
// created, for the lifetime of the process.
//
// This file is its own CUDA module, holding only the array.  Under lazy module
// loading the driver loads it -- and reserves its 16 MiB of device memory --
// at the first symbol lookup on a device.  That lookup is done by
// sar_plan_create (set-up time), never by the imaging call.
#include <mutex>

#include "sar_internal.h"

namespace {

// Maximum scratch: 16 MiB = 2048 partial-sum slots of 8 KB (one slot holds the
// 1024 complex64 partial sums of one pixel tile).  A launch needs G x seg_max
// slots: G persistent CTAs times the tiles one CTA's range can touch, i.e.
// floor((ceil(units / G) - 1) / blocks_per_tile) + 2 per CTA.  Example: a
// 1024 x 1024 image (1024 tiles) at 2048 chirps on 152 SMs x 2 CTAs uses
// 304 x 5 = 1520 slots (12.5 MB).
constexpr size_t kScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_bp_scratch[kScratchBytes / sizeof(float2)];

std::mutex g_setup_mutex;
float2 *g_scratch_addr[kMaxDevices] = {};

}  // namespace

namespace sar {

// Set-up of `dev` (which must be current), once per device: look up the
// device address of g_bp_scratch.  In host code the name g_bp_scratch is only
// a host-side handle, never a device address.  Called by sar_plan_create.
int noalloc_setup(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return SAR_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_addr[dev]) return SAR_OK;
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_bp_scratch);
    if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SAR_ENOMEM : SAR_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<float2 *>(p);
    return SAR_OK;
}

}  // namespace sar

extern "C" int sar_backproject_noalloc(sar_plan *plan, const void *prof_dev, int32_t M, const double *q_tx_dev,
                                       const double *q_rx_dev, const float *fdopp_idx_dev, void *image_dev,
                                       int32_t accumulate, void *stream) {
    if (!plan || !prof_dev || !q_tx_dev || !q_rx_dev || !image_dev || M < 1) return SAR_EINVAL;
    const auto aligned = [](const void *p, size_t a) { return ((uintptr_t)p % a) == 0; };
    if (!aligned(prof_dev, 256) || !aligned(q_tx_dev, 16) || !aligned(q_rx_dev, 16) || !aligned(image_dev, 8) ||
        (fdopp_idx_dev && !aligned(fdopp_idx_dev, 4)))
        return SAR_EINVAL;
    const int dev = sar::plan_device(plan);
    if (dev < 0 || dev >= kMaxDevices) return SAR_EINVAL;
    float2 *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        scratch = g_scratch_addr[dev];  // set when the plan was created
    }
    if (!scratch) return SAR_ECUDA;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return SAR_ECUDA;
    if (cur != dev && cudaSetDevice(dev) != cudaSuccess) return SAR_ECUDA;
    const int rc = sar::backproject_with_scratch(plan, prof_dev, M, q_tx_dev, q_rx_dev, fdopp_idx_dev, image_dev,
                                                 accumulate, scratch, kScratchBytes, (cudaStream_t)stream);
    if (cur != dev) cudaSetDevice(cur);
    return rc;
}
