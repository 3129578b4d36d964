// Internal declarations shared by the host API (api.cpp) and the CUDA
// kernels (range_compress.cu, backproject.cu).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sar.h"

namespace sar {

// Backprojection tiling: 1024 reconstruction points per tile, 256 threads,
// 4 points per thread.
constexpr int kTilePx = 1024;
constexpr int kBpThreads = 256;
constexpr int kPxPerThread = kTilePx / kBpThreads;
// Bins of guard band on each side of a staged window.
constexpr int kGuardBins = 2;
// Absolute distances beyond this (m) are treated as invalid geometry.
constexpr double kMaxRange = 1.0e6;
// Bits of the device error flag (any bit set: SAR_EBOUNDS).
constexpr int kErrGeometry = 1;      // non-finite or out-of-range antenna geometry
constexpr int kErrDopplerBound = 2;  // |f_doppler(p)| beyond the plan's bound, or not finite

// Range compression output modes.
enum RcMode { kRcProfileF32 = 0, kRcProfileF16 = 1, kRcSpectrum = 2 };

struct RcArgs {
    const float2 *beat;      // [rows][N]
    const float *w_r;        // [N] range window
    const float2 *tw;        // [n_fft] exp(sign j 2 pi i / n_fft)
    const float2 *rot;       // [n_bins] exp(sign j 2 pi frac(k beta)), k = crop_lo + i
    const float *w_az;       // [M] or null
    void *out;               // profile samples or spectrum
    float *scales;           // [rows] (FP16 profiles)
    long long rows;          // M * R
    int R;
    int N;
    int n_fft;
    int log2n;
    int crop_lo;
    int n_bins;
};

cudaError_t launch_range_compress(const RcArgs &a, int sign, int mode, cudaStream_t s);

// Split-transform range compression (N = 32 N2 samples, N2 in {8, 16, 32},
// N2 os <= 256): tables built by the plan.  CTAs of kSplitThreads threads
// handle kSplitThreads / (N2 os) rows at a time (a row group).
constexpr int kSplitThreads = 256;
struct RcSplitArgs {
    const float2 *beat;  // [rows][N]
    const float2 *pre;   // [os][N]: w_r[n] exp(SGN j 2 pi n s / N_fft), input rotation of sub-transform s
    const float2 *twd;   // [32][N2]: W_N^(j k1) at [k1][j]
    const float2 *rot;   // [n_bins]: per-bin rotation of the stored profile
    const float *w_az;   // [M] or null
    void *out;           // profile samples
    float *scales;       // [rows] (FP16 profiles)
    long long rows;
    int R, N2, os;
    int crop_lo, crop_hi, n_bins;
};
// Batched form: several jobs with the same N, os, convention and storage in
// one launch; job j owns row groups [group_begin[j], group_begin[j + 1]).
struct RcSplitBatch {
    const RcSplitArgs *jobs;
    const long long *group_begin;  // [n_jobs + 1]
    int n_jobs;
};
bool rc_split_supported(int n_samples, int os);
// tab == null: the single job a; otherwise a gives N2 and os of the table's
// jobs and groups is the table's total row-group count.
cudaError_t launch_range_compress_split(const RcSplitArgs &a, int sign, int mode, cudaStream_t s,
                                        const RcSplitBatch *tab = nullptr, long long groups = 0);
// Fills the split-kernel job of range compression of M chirps on `plan`;
// false when the plan's shape needs the general kernel.
bool fill_rc_split(const sar_plan *plan, const void *beat, int M, const float *w_az, void *prof, RcSplitArgs *out,
                   int *sign, int *mode);

// Per-tile data: reference point (x, y), radius rho (max distance of the
// tile's points from the reference), number of valid points, and two
// plan-dependent constants of the expansion loop: o_allow, the largest Rx
// offset (m) the common window absorbs, and klo_off = a1 (2 rho + o_allow) +
// fd_max, so that a pulse's window starts at floor(2 a1 R_tx - klo_off) - G.
struct TileInfo {
    double x, y, rho;
    float o_allow, klo_off;
    int32_t n_valid;
    int32_t pad;
};

struct BpArgs {
    const void *prof;          // profile samples (float2 or half2)
    const float *prof_scale;   // [M][R] FP16 scales, or null
    const double *q_tx;        // [M][2]
    const double *q_rx;        // [M][R][2]
    const float *fdopp;        // [n_pixels] or null
    float2 *image;             // [n_pixels]
    float2 *image_out;         // second destination of the result (null: none); may be mapped host memory
    float2 *partial;           // [G * seg_max][kTilePx]
    int *err;                  // device error flags
    const float2 *pix;         // [n_tiles][kTilePx] (dx, dy) from the tile reference
    const int *out_idx;        // [n_tiles][kTilePx] image index or -1
    const TileInfo *tiles;     // [n_tiles]
    long long units;           // n_tiles * blocks_per_tile
    int G;                     // persistent CTAs
    int blocks_per_tile;       // ceil(M / Mb)
    int seg_max;               // partial slots per CTA
    int M, R, n_tiles, Mb, L;
    int n_bins, crop_lo, crop_hi;
    int accumulate;
    double a1;                 // bins per metre
    float a1f;
    float kappa;               // sign * 2 pi beta' (radians per bin), 22 significant bits;
                               // beta' = cycles per bin at the transform's time origin
    float kappa_magic;         // kappa * 1.5 * 2^23 (exact)
    float inv_kappa;           // 1 / kappa
    float beta;                // beta' (cycles per bin at the time origin)
    float sign;
    float2 cb_k;               // exp(-sign j 2 pi beta') / kappa
    float fd_max;              // bound on |f_doppler|
    unsigned long long div_nq; // ceil(2^32 / (L / 4)): division by the groups per window
    unsigned long long div_r;  // ceil(2^32 / R)
    int fp16;                  // profile storage (batched form)
    int rg;                    // Rx group of the inner loop (batched form)
};

// Batched form: several requests (each a BpArgs with its own plan data)
// backprojected by one persistent launch.  Requests are grouped into classes
// (Rx group, storage); class c owns CTAs [cta_begin, cta_begin + G) and tiles
// [tile_base, tile_base + tiles) of the fix-up.
struct BpClassArgs {
    const BpArgs *jobs;          // [n_jobs]
    const long long *unit_begin; // [n_jobs + 1] prefix sums of (tile, pulse block) units
    const int *tile_begin;       // [n_jobs + 1] prefix sums of tiles
    long long units;
    int n_jobs;
    int G;                       // CTAs of the class
    int cta_begin;               // first CTA of the class in the grid
    int tile_base;               // first fix-up CTA of the class
    int rg;                      // Rx group of the inner loop
    int fp16;                    // profile storage
};
constexpr int kBatchClasses = 8;  // Rx group 1..4 x storage
// Classes of up to kParamJobs requests get their job arguments as a kernel
// parameter (constant bank, like a single request's); larger ones read the
// device table.
constexpr int kParamJobs = 128;
struct BpJobTable {
    BpArgs jobs[kParamJobs];
};
static_assert(sizeof(BpJobTable) + sizeof(BpClassArgs) + 64 <= 32764, "kernel parameter limit");
struct BpMultiArgs {
    BpClassArgs cls[kBatchClasses];
    int n_classes;
};
// Partial-sum scratch of a batch and the checks of its kernels.
struct BpCheck {
    float2 *scratch;             // [CTAs * 2][kTilePx] partial sums
    long long scratch_slots;     // capacity of scratch in kTilePx slots
    unsigned smem_bytes;         // dynamic shared memory of the launch
    int *err;                    // [4]: check code, then three values of the first failed check
};

struct BpLaunch {
    int rg;       // Rx group size of the inner loop (1, 2, 3 or 4)
    bool fp16;
    size_t smem;  // dynamic shared memory bytes
    int minb;     // CTAs per SM the kernel's registers are sized for (2 or 3)
};

size_t bp_smem_bytes(int Mb, int R, int L, bool fp16);
cudaError_t bp_prepare(bool fp16, int rg, size_t smem);  // sets function attributes
int bp_occupancy(bool fp16, int rg, size_t smem, int minb, int *ctas_per_sm);
cudaError_t launch_backproject(const BpArgs &a, const BpLaunch &l, cudaStream_t s);
cudaError_t bp_batch_prepare(int rg, bool fp16, size_t smem, int *ctas_per_sm);
// host_jobs: the class's jobs in host memory (the same as c.jobs), passed as
// parameters when there are at most kParamJobs; null to read c.jobs.
cudaError_t launch_backproject_class(const BpClassArgs &c, const BpCheck &chk, size_t smem, cudaStream_t s,
                                     const BpArgs *host_jobs);
cudaError_t launch_batch_fixup(const BpMultiArgs &m, const BpCheck &chk, int total_tiles, cudaStream_t s);

// Per-pixel Doppler offsets (doppler.cu).
struct DopplerArgs {
    const double *q_tx, *q_rx, *vel;  // [M][2], [M][R][2], [M][2]
    int M, R;
    const TileInfo *tiles;
    const float2 *pix;
    const int *out_idx;
    int n_tiles;
    double *means;  // [6] device scratch of the plan
    double scale;   // f0 / c * N_fft / fs: bins per (m/s) of path rate
    float *fd;      // [n_pixels] output in image order
};
cudaError_t launch_doppler_offsets(const DopplerArgs &a, cudaStream_t s);

// Used by the server (serve.cpp).
int batch_add_rows(sar_batch *b, sar_plan *plan, const void *samples, const float *scales, int32_t M,
                   const double *q_tx, const double *q_rx, void *image, int32_t accumulate,
                   void *image_out = nullptr);
int plan_geometry(const sar_plan *pl, int *n_rx, int *n_samples, int *n_bins, int *fp16, int64_t *n_pixels,
                  int *max_pulses);
int fill_bp_args(const sar_plan *pl, const void *prof, int M, const double *q_tx, const double *q_rx,
                 void *image, int accumulate, BpArgs *out, size_t *smem);

// Used by sar_backproject_noalloc (noalloc.cu).
int plan_device(const sar_plan *pl);
int noalloc_setup(int dev);  // once per device, at plan creation (device current)
int backproject_with_scratch(sar_plan *pl, const void *prof, int M, const double *q_tx, const double *q_rx,
                             const float *fd, void *image, int accumulate, float2 *scratch, size_t scratch_bytes,
                             cudaStream_t s);

}  // namespace sar
