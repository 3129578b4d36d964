/*
 * sar.h -- C ABI of the GB300-native automotive FMCW SAR imaging library
 * (range compression + time-domain backprojection, after "Implementation of
 * Real-Time Automotive SAR Imaging", arXiv 2306.09784).
 *
 * General rules
 *  - Every call returns an int status (enum sar_status); no C++ exception
 *    crosses this boundary.
 *  - Pointers named *_dev are CUDA device pointers on the plan's device;
 *    pointers named *_host are host pointers (pinned memory gives the fastest
 *    copies).  The caller owns every buffer it passes in; the plan owns only
 *    its tables and scratch.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls that take a stream are asynchronous: they validate their
 *    arguments on the host, enqueue kernels and return.  Errors raised inside
 *    kernels are reported by sar_plan_check_errors() after the work finished.
 *  - Units are SI (metres, seconds, hertz).  Geometry is 2-D (x, y): the
 *    paper computes 2-D distances (Alg. 1, Sec. II).
 *  - Complex values are interleaved (re, im) pairs: complex64 = 2 x float.
 *  - Calls on one plan must not overlap in time from several host threads.
 */
#ifndef SAR_H
#define SAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum sar_status {
    SAR_OK = 0,
    SAR_EINVAL = 1,    /* invalid argument (null pointer, size, parameter) */
    SAR_ENOMEM = 2,    /* device allocation failed or HBM budget exceeded */
    SAR_EAGAIN = 3,    /* not ready yet (poll) or admission queue full */
    SAR_ETIMEOUT = 4,  /* a bounded wait ran out */
    SAR_ECUDA = 5,     /* a CUDA runtime call failed */
    SAR_EBOUNDS = 6,   /* a kernel saw invalid geometry (non-finite or out of range) */
    SAR_ENOTFOUND = 7, /* unknown ticket */
    SAR_ESCRATCH = 8   /* sar_backproject_noalloc: the call needs more than its static scratch */
};

enum sar_window { SAR_WINDOW_RECT = 0, SAR_WINDOW_HANN = 1, SAR_WINDOW_KAISER = 2 };

/* Time origin of the range transform (the instant whose frequency is the
 * phase correction's carrier, Sec. II). */
enum sar_time_origin {
    SAR_ORIGIN_FIRST_SAMPLE = 0,  /* sample 0: carrier f0 (Alg. 1 / Alg. 2 as printed) */
    SAR_ORIGIN_CHIRP_CENTRE = 1   /* sample (N - 1) / 2: carrier f0 + slope (N - 1) / (2 fs) */
};

/* Storage of the range profiles between the two stages. */
enum sar_precision {
    SAR_PREC_FP32 = 0,  /* complex64 samples */
    SAR_PREC_FP16 = 1   /* half-precision complex samples with one FP32 scale per (chirp, Rx) */
};

/*
 * Radar and processing parameters (paper Table I, Sec. II, Sec. III-C).
 *  f0          frequency at the range transform's time origin (sample 0), Hz
 *  slope       chirp slope mu = B / T_P, Hz/s
 *  fs          beat-signal sample rate, Hz
 *  c           propagation speed, m/s
 *  n_samples   N, samples per chirp and Rx
 *  os          zero-padding factor; N_fft = N * os must be a power of two
 *              between 64 and 16384
 *  n_rx        R, Rx channels per chirp (1..64)
 *  max_pulses  capacity in chirps per call (sizes the plan's scratch)
 *  range_window    enum sar_window applied to each chirp before the transform
 *  kaiser_beta     beta of the Kaiser window
 *  precision   enum sar_precision of the range profiles
 *  phase_sign  +1: range transform kernel exp(+j 2 pi n k / N_fft) and phase
 *              correction exp(+j 2 pi f0 d / c) (beat taken as Rx conj(Tx));
 *              -1: the conjugate convention (forward transform, exp(-j ...))
 *  crop_lo, crop_hi  interpolation base bins kept, [crop_lo, crop_hi);
 *              terms whose base bin falls outside contribute nothing.
 *              0, 0 selects the full valid range [0, N_fft - 1).
 *  time_origin enum sar_time_origin.  SAR_ORIGIN_CHIRP_CENTRE evaluates the
 *              transform over the centred time index n - (N - 1) / 2 and the
 *              phase correction at the carrier of that instant; the spectrum's
 *              phase is then flat across a target's main lobe, so linear
 *              interpolation between bins loses less (at os = 4 the image is
 *              about 9 times closer to the exact matched filter).  The
 *              limit as os grows is the same image for both origins; the
 *              kernels' work is the same.
 *  max_doppler_bins  bound on |f_doppler(p)| (in bins) of the Doppler
 *              offsets passed to sar_backproject; the staged bin windows are
 *              widened by it (0..64).  A pixel whose offset lies beyond the
 *              bound (or is not finite) is left out of that call and the call
 *              is flagged SAR_EBOUNDS (see sar_backproject).
 * The derived phase rate beta = f0 / (c a1) cycles per bin, a1 = slope N_fft
 * / (c fs) bins per metre, must lie in [1e-9, 1e9] (f0 / (B os) for a chirp
 * of bandwidth B; about 19 at 77 GHz, 1 GHz, os 4); sar_plan_create rejects
 * other parameters with SAR_EINVAL.
 */
typedef struct sar_radar_params {
    double f0;
    double slope;
    double fs;
    double c;
    int32_t n_samples;
    int32_t os;
    int32_t n_rx;
    int32_t max_pulses;
    int32_t range_window;
    int32_t precision;
    double kaiser_beta;
    int32_t phase_sign;
    int32_t crop_lo;
    int32_t crop_hi;
    int32_t time_origin;
    double max_doppler_bins;
} sar_radar_params;

/*
 * Reconstruction points (paper Sec. III-E: Cartesian reference grid or any
 * other set of points, e.g. a polar grid).
 *  pixels_xy == NULL: Cartesian grid, pixel (ix, iy) at
 *      (x0 + ix dx, y0 + iy dy), image stored [ny][nx] with x fastest;
 *  pixels_xy != NULL: host array [n_pixels][2] of (x, y) points, image
 *      stored [n_pixels] in the caller's order; x0..ny are ignored.
 * The plan copies what it needs; the caller may free pixels_xy afterwards.
 */
typedef struct sar_grid {
    double x0, y0, dx, dy;
    int32_t nx, ny;
    const double *pixels_xy;
    int64_t n_pixels;
} sar_grid;

typedef struct sar_plan sar_plan;

/*
 * Polar reconstruction grid (paper Sec. III-E, Fig. 2), a point list for
 * sar_grid.pixels_xy.  The grid originates in the centre of the synthetic
 * aperture and is `factor` times finer than the radar's resolution in range
 * and azimuth (the paper: 2.5, "larger than 2 to depict point targets").  The
 * paper's point-spread function is not printed; the textbook resolutions
 * stand in for it: range c / (2 B), B = |slope| n_samples / fs, and azimuth
 * lambda r / (2 L) at range r, i.e. the angle lambda / (2 L), with lambda =
 * c / (f0 + slope n_samples / (2 fs)) and L = |q_tx(M-1) - q_tx(0)|.  With
 * o = (q_tx(0) + q_tx(M-1)) / 2, u the unit vector from q_tx(0) to
 * q_tx(M-1) and v = u turned +90 degrees, the points are
 *     o + (k Dr) (cos(j Dphi) u + sin(j Dphi) v),
 *     Dr = c / (2 B) / factor,  Dphi = lambda / (2 L) / factor,
 * for integers k >= 1 and j with j Dphi in [-pi, pi), kept where they fall in
 * the box [x_min, x_max] x [y_min, y_max] (borders included), listed by k then
 * j, both ascending.
 */
typedef struct sar_polar_spec {
    double x_min, x_max, y_min, y_max;  /* region of interest, m */
    double factor;                      /* resolution / spacing (> 0) */
} sar_polar_spec;

/*
 *  params     f0, slope, fs, c and n_samples are used
 *  q_tx_host  double [M][2] Tx positions of the aperture (M >= 2, host)
 *  xy_host    double [capacity][2] output (host), or NULL to count only
 *  n_points   receives the number of grid points in the box
 * Host-only (no device work).  SAR_EINVAL for invalid parameters, a
 * zero-length aperture, an empty or non-finite box, or capacity below the
 * count (then nothing beyond capacity is written; *n_points is the count).
 */
int sar_polar_grid(const sar_radar_params *params, const double *q_tx_host, int32_t M,
                   const sar_polar_spec *spec, double *xy_host, int64_t capacity, int64_t *n_points);

/* Sizes derived by a plan (all read-only). */
typedef struct sar_plan_info {
    int32_t n_fft;              /* N * os */
    int32_t n_bins;             /* samples per stored range profile = crop_hi - crop_lo + 1 */
    int32_t crop_lo, crop_hi;
    int64_t n_pixels;           /* image size in complex64 values */
    int32_t n_tiles;            /* pixel tiles of 1024 reconstruction points (slots) */
    int32_t window_bins;        /* bins staged per (tile, chirp, Rx) */
    int32_t pulses_per_block;   /* chirps staged per pipeline step */
    int32_t bp_ctas;            /* persistent backprojection grid size */
    double bins_per_metre;      /* a1 = mu N_fft / (c fs) */
    double cycles_per_bin;      /* f0 / (c a1) */
    size_t device_bytes;        /* device memory the plan owns */
    int32_t rx_group;           /* Rx channels per inner-loop group of the launch shape */
    int32_t regs_ctas_per_sm;   /* CTAs per SM the launch's registers are sized for */
    int32_t tile_w, tile_h;     /* pixel tile of a Cartesian plan (0, 0: point list) */
} sar_plan_info;

/*
 * Create a plan on the current CUDA device.  Validates the parameters,
 * builds the FP64 tables (range window, transform twiddles, per-bin phase
 * rotation, pixel tiles) and allocates the plan's device memory.
 * hbm_budget_bytes bounds that memory (0 = no bound): SAR_ENOMEM if it
 * would be exceeded.  *out receives the plan (NULL on error).  SAR_EINVAL,
 * before any CUDA call, for invalid parameters, a null or empty grid (nx or
 * ny < 1, n_pixels < 1 for a point list), more than 2^30 points or a
 * non-finite Cartesian origin or spacing; non-finite listed points give
 * SAR_EINVAL too.  The first plan on a device also sets up the static scratch
 * of sar_backproject_noalloc there (16 MiB of device memory, outside the
 * budget, held until exit; SAR_ENOMEM if the device cannot provide it).
 */
int sar_plan_create(const sar_radar_params *params, const sar_grid *grid,
                    size_t hbm_budget_bytes, sar_plan **out);

/* Release a plan and its device memory (synchronises its device). NULL is a no-op. */
void sar_plan_destroy(sar_plan *plan);

int sar_plan_get_info(const sar_plan *plan, sar_plan_info *info);

/* Bytes of the range-profile buffer that sar_range_compress fills for M chirps. */
int sar_profile_bytes(const sar_plan *plan, int32_t M, size_t *bytes);

/*
 * Range compression (paper: the beat spectrum s(f, m, n_rx) that Alg. 1
 * and Alg. 2 interpolate at f_hyp / f_ind; its equidistant beat-frequency
 * axis, Sec. III-C).  For every chirp m < M and Rx r:
 *     S[m][r][k] = sum_{n<N} w_r[n] beat[m][r][n] exp(sign j 2 pi n k / N_fft)
 * and the stored profile, for bins k = crop_lo .. crop_hi, is
 *     prof[m][r][k - crop_lo] = w_sar[m] exp(sign j 2 pi frac(k f0 / (c a1))) S[m][r][k]
 * i.e. the spectrum with the window w_sar (Sec. III-B, NULL = ones) and the
 * per-bin part of the phase correction exp(sign j 2 pi f0 d / c) folded in
 * (d = index / a1 on the bin axis, so the correction splits into a per-bin
 * factor and a factor of the fractional index).
 *  beat_dev   complex64 [M][R][N]
 *  w_az_dev   float [M] or NULL
 *  prof_dev   sar_profile_bytes(M) bytes, 256-byte aligned.  Layout:
 *             FP32: complex64 [M][R][n_bins];
 *             FP16: float scale[M][R], padded to a 256-byte multiple, then
 *                   half2 [M][R][n_bins] with value = scale * half.
 * Errors: SAR_EINVAL (null pointers, M < 1 or M > max_pulses, misalignment).
 */
int sar_range_compress(sar_plan *plan, const void *beat_dev, int32_t M,
                       const float *w_az_dev, void *prof_dev, void *stream);

/*
 * The plain windowed, zero-padded range transform S[m][r][k] for all
 * k < N_fft as complex64 [M][R][N_fft] (same kernel as sar_range_compress,
 * without window w_sar, rotation or crop).  For inspection and parity checks.
 */
int sar_range_spectrum(sar_plan *plan, const void *beat_dev, int32_t M,
                       void *spec_dev, void *stream);

/*
 * Backprojection, paper Alg. 2 (Sec. IV): for every reconstruction point p
 *     P(p) = sum_{m<M} sum_{r<R} exp(sign j 2 pi f0 d / c) s(a1 d + f_doppler(p), m, r)
 * with d = ||p - q_tx(m)|| + ||p - q_rx(m, r)|| and s(., m, r) the linear
 * interpolation of the stored profile (w_sar already folded in).
 *  prof_dev        output of sar_range_compress for these M chirps
 *  q_tx_dev        double [M][2] Tx positions
 *  q_rx_dev        double [M][R][2] Rx positions
 *  fdopp_idx_dev   float [n_pixels] Doppler index offsets f_doppler(p) in bins
 *                  (f_doppler of Alg. 2, e.g. from sar_doppler_offsets), or
 *                  NULL for none; needs a plan with max_doppler_bins > 0
 *  image_dev       complex64 [n_pixels]; written (accumulate = 0) or added to
 *                  (accumulate = 1, for sub-aperture accumulation)
 * Errors: SAR_EINVAL; non-finite or absurd geometry (beyond 1e6 m) is
 * skipped and flagged for sar_plan_check_errors (SAR_EBOUNDS).  A pixel
 * whose |f_doppler(p)| exceeds the plan's max_doppler_bins, or is not finite,
 * gets no contribution from the call (its value is written as 0, or left
 * unchanged when accumulating) and the call is flagged SAR_EBOUNDS too: its
 * interpolation index would leave the staged bin window.
 */
int sar_backproject(sar_plan *plan, const void *prof_dev, int32_t M,
                    const double *q_tx_dev, const double *q_rx_dev,
                    const float *fdopp_idx_dev, void *image_dev,
                    int32_t accumulate, void *stream);

/*
 * Per-pixel Doppler index offsets f_doppler(p) of Alg. 2 (paper Sec. III-D):
 * the velocity terms of Alg. 1 (lines 5, 8, 9 and the f0 v / c term of line
 * 11) computed once per reconstruction point from the average vehicle
 * velocity over the chirp sequence:
 *     vbar = mean_m vel(m),  qt = mean_m q_tx(m),  qr = mean_{m,r} q_rx(m, r),
 *     f_doppler(p) = -(f0' / c) (<p - qt, vbar> / |p - qt| + <p - qr, vbar> / |p - qr|) N_fft / fs
 * in bins, f0' the carrier at the transform's time origin.  The bracket is
 * minus the rate of change of the two-way path for a platform moving with
 * vbar (a platform closing on p lowers the beat frequency under the beat
 * model Rx conj(Tx); the same offset holds for the conjugate convention).
 *  q_tx_dev   double [M][2], q_rx_dev double [M][R][2] (the frame's trajectory)
 *  vel_dev    double [M][2] platform velocity per chirp (m/s)
 *  fdopp_idx_dev  float [n_pixels] output in image order, ready for
 *             sar_backproject; |f_doppler| <= 2 f0' |vbar| N_fft / (c fs), so a
 *             plan with max_doppler_bins at least that takes every pixel
 * Asynchronous on `stream` (two kernels, device memory only).  SAR_EINVAL for
 * null or misaligned pointers or M outside 1..max_pulses.
 */
int sar_doppler_offsets(sar_plan *plan, const double *q_tx_dev, const double *q_rx_dev,
                        const double *vel_dev, int32_t M, float *fdopp_idx_dev, void *stream);

/*
 * sar_backproject without any device allocation on the library's side, for
 * callers that cannot allocate device memory when they image a frame: an
 * embedded or safety-certified automotive process that allocates only at
 * start-up, or a caller whose device memory is reserved up front by another
 * allocator.  (The paper has no counterpart; this is an interface matter.)
 *
 * Same arguments, result and errors as sar_backproject.  The plan's
 * read-only tables are still used; only the scratch for tiles that several
 * CTAs share (partial sums) comes from one static 16 MiB device array in the
 * library: 2048 slots of 8 KB, one slot per pixel tile a CTA covers in part.
 *  - sar_plan_create sets the array up on the plan's device: the first plan
 *    on a device looks up its address, and that lookup makes the driver load
 *    the library module holding it, which reserves its 16 MiB of device
 *    memory (outside the plan's HBM budget) until the process exits.  The
 *    imaging call itself makes no cudaMalloc, cudaFree or other allocating
 *    call.  After a cudaDeviceReset, plans made before it must not be used
 *    (their own device memory is gone as well) and this call is unsupported.
 *  - A launch needs G x seg_max slots (G persistent CTAs, seg_max tiles per
 *    CTA range); a call needing more than 2048 returns SAR_ESCRATCH and
 *    enqueues nothing.  Example: a 1024 x 1024 image at 2048 chirps on 152 SMs
 *    x 2 CTAs uses 304 x 5 = 1520 slots (12.5 MB).
 *  - Every call on a device shares the one array and finds the previous
 *    call's contents there; nothing in it needs to start at zero (each slot
 *    read is written earlier in the same call).  Calls whose work overlaps on
 *    the GPU (several streams, several host threads) race on it: serialise
 *    them.
 */
int sar_backproject_noalloc(sar_plan *plan, const void *prof_dev, int32_t M,
                            const double *q_tx_dev, const double *q_rx_dev,
                            const float *fdopp_idx_dev, void *image_dev,
                            int32_t accumulate, void *stream);

/*
 * Batched backprojection (Alg. 2 for several requests in a few launches).
 * Requests of uneven sizes -- each with its own plan (radar parameters,
 * reconstruction points, FP32 or FP16 profiles), profiles, trajectory and
 * image -- are packed as (request, pixel tile, pulse block) work units and
 * grouped into classes that share an Rx group and a profile storage (at most
 * 8; the pixel loop is specialised per class).  Each class is one persistent
 * launch over the whole GPU that splits the units of all its requests evenly
 * over the CTAs; the classes run back to back and one fix-up kernel then sums
 * the tiles that two CTAs shared.  Each request's image equals
 * sar_backproject's up to FP32 summation order.
 *
 * Use: sar_batch_clear, sar_batch_add per request, sar_batch_commit (groups
 * the requests by class and uploads the request table on `stream`), then
 * sar_batch_launch (one kernel per class and the fix-up on `stream`; a class
 * of up to 128 requests gets their kernel arguments as launch parameters,
 * larger ones read the uploaded table; it can be captured in a CUDA graph,
 * which keeps the parameters of the committed batch, and replayed while the
 * batch is not committed again and the request buffers stay unchanged).
 * sar_batch_autotune picks each class's pulse block and argument source.
 * All plans of a batch must be on the batch's device; the batch owns its
 * request table (pinned host + device) and
 * partial sums of 16 KB per CTA and class (39 MB on 152 SMs).
 * Requests of one batch must not write the same image.
 */
typedef struct sar_batch sar_batch;

/* Create a batch for up to max_jobs requests on the current device. */
int sar_batch_create(int32_t max_jobs, sar_batch **out);
void sar_batch_destroy(sar_batch *batch);
/* Forget all requests (waits for a pending table upload).  Launch choices
 * made by sar_batch_autotune are kept. */
int sar_batch_clear(sar_batch *batch);
/* Append one request: arguments as sar_backproject (no Doppler offsets). */
int sar_batch_add(sar_batch *batch, sar_plan *plan, const void *prof_dev, int32_t M,
                  const double *q_tx_dev, const double *q_rx_dev, void *image_dev,
                  int32_t accumulate);
/*
 * Append one frame: its range compression (as sar_range_compress of beat_dev
 * and w_az_dev into prof_dev) and its backprojection (as sar_batch_add of
 * prof_dev).  sar_batch_launch then range-compresses the batch's frames
 * first: frames of the same transform shape (samples, zero padding,
 * convention, storage) in one packed launch of the split-transform kernel
 * when it supports the shape, each frame in its own launch otherwise.
 *  beat_dev  complex64 [M][R][N] (8-byte aligned);  w_az_dev float [M] or NULL;
 *  prof_dev  sar_profile_bytes(M) bytes (256-byte aligned), written by the launch.
 */
int sar_batch_add_frame(sar_batch *batch, sar_plan *plan, const void *beat_dev, const float *w_az_dev,
                        void *prof_dev, int32_t M, const double *q_tx_dev, const double *q_rx_dev,
                        void *image_dev, int32_t accumulate);
/* Upload the request table asynchronously on `stream`. */
int sar_batch_commit(sar_batch *batch, void *stream);
/* Launch the range compressions of the frames added with sar_batch_add_frame,
 * then the persistent backprojection of every class and the fix-up. */
int sar_batch_launch(sar_batch *batch, void *stream);
/* Requests, work units and the largest class launch's grid (CTAs) of the
 * committed batch (any pointer may be NULL). */
int sar_batch_get_info(const sar_batch *batch, int32_t *n_jobs, int64_t *units, int32_t *ctas);

/*
 * Autotuner of the batched launch (no counterpart in the paper): it times
 * every class's launch with chirps per pipeline block from {each request's
 * plan's own, the largest that fits two CTAs per SM for every request of the
 * class, 2/3 and 1/2 of that} and keeps each class's fastest; at that block
 * it then times a class of up to 128 requests with its arguments read from
 * the device table instead of passed as launch parameters, and keeps the
 * faster source (the two give identical images).  Needs a
 * committed batch; re-commits it on `stream` and blocks until the timing runs
 * finish.  The requests' images are overwritten (and accumulating requests
 * accumulate repeatedly): their contents are undefined afterwards.  The
 * choices persist across sar_batch_clear.
 */
int sar_batch_autotune(sar_batch *batch, void *stream);

/* One class of the committed batch (see sar_batch_num_classes). */
typedef struct sar_batch_class {
    int32_t rx_group;          /* Rx channels per inner-loop group */
    int32_t fp16;              /* profile storage: 1 = FP16 */
    int32_t n_jobs;            /* requests in the class */
    int32_t pulses_per_block;  /* chirps per pipeline block; 0 = each request's plan's own */
    int32_t ctas;              /* CTAs of the class's launch */
    int32_t regs_ctas_per_sm;  /* CTAs per SM the launch's registers are sized for (2) */
    int64_t units;             /* (tile, pulse block) work units */
    double updates;            /* pixel slots x chirps x Rx */
    double tuned_ms;           /* the class launch (with its fix-up) at the chosen block, as timed by
                                  sar_batch_autotune; 0 before it runs */
    int32_t param_args;        /* 1: the requests' kernel arguments travel as launch parameters (classes
                                  of up to 128 requests), 0: the kernel reads them from the batch's
                                  device table */
    int32_t reserved;
} sar_batch_class;

int sar_batch_num_classes(const sar_batch *batch, int32_t *n_classes);
/* Waits for the device and reports (then clears) the batched kernels' checks
 * of their work decomposition: SAR_OK, or SAR_EBOUNDS when a check failed (the
 * work it guarded was skipped); detail (may be NULL) receives [4]: the check's
 * code and three values.  Geometry errors are reported per plan by
 * sar_plan_check_errors. */
int sar_batch_check_errors(sar_batch *batch, int32_t *detail);
int sar_batch_get_class(const sar_batch *batch, int32_t index, sar_batch_class *out);

/*
 * Served form: continuous batching of imaging requests from several radars.
 * A server owns one worker thread and three CUDA streams on the device that
 * is current at creation.  Each request is one frame (sar_request): its beat
 * cube, w_sar and trajectory are copied to the device when it is admitted,
 * range-compressed, then backprojected in rounds: every round is one batched
 * launch (sar_batch_launch) over the next chunk of every active request --
 * chunk_pulses chirps, or fewer when quantum_mupdates bounds each request's
 * work per round -- accumulated into the request's device-resident image.
 * Requests that arrive while a round runs join the first round launched after
 * their upload and range compression have completed; finished ones leave.
 * Larger chunks mean fewer rounds (less per-round cost), but a newcomer waits
 * for the round in flight: chunk_pulses and quantum_mupdates trade throughput
 * against the latency tail.  Admission is bounded by max_inflight and by an
 * HBM budget (one device pool allocated at creation and sub-allocated per
 * request); a request
 * waits in arrival order until its buffers fit.  A request's image equals its
 * stand-alone sar_range_compress + sar_backproject result up to FP32
 * summation order.
 *
 * The caller keeps the plan and the host buffers of a request alive and
 * unchanged until the request is DONE, FAILED or released.  Host buffers
 * should be pinned (cudaHostAlloc) for asynchronous copies.
 */
enum sar_request_state {
    SAR_REQ_QUEUED = 0,   /* waiting for admission */
    SAR_REQ_RUNNING = 1,  /* on the device */
    SAR_REQ_DONE = 2,     /* image complete (and copied to image_host if given) */
    SAR_REQ_FAILED = 3    /* a CUDA error stopped the server */
};

typedef struct sar_server_config {
    size_t hbm_budget_bytes;  /* device pool for request buffers (>= 1 MiB) */
    int32_t max_inflight;     /* requests on the device at once (1..4096) */
    int32_t queue_capacity;   /* submitted, not yet admitted (SAR_EAGAIN beyond) */
    int32_t chunk_pulses;     /* chirps per request per round (at most) */
    int32_t quantum_mupdates; /* 0, or a work quantum per request and round in millions of
                                 pixel x chirp x Rx updates: a request advances by at most
                                 ceil(quantum / (pixels x Rx)) chirps per round, so frames
                                 smaller than the quantum finish in their first round while
                                 larger ones share the following rounds with newcomers */
} sar_server_config;

typedef struct sar_request {
    sar_plan *plan;           /* radar parameters and reconstruction points */
    const void *beat_host;    /* complex64 [M][R][N] */
    int32_t M;                /* chirps (1..plan max_pulses) */
    const float *w_az_host;   /* float [M] or NULL */
    const double *q_tx_host;  /* double [M][2] */
    const double *q_rx_host;  /* double [M][R][2] */
    void *image_host;         /* complex64 [n_pixels] destination, or NULL (device only); a
                                 page-locked, mapped one is written by the final round's kernels,
                                 any other by a copy after them */
} sar_request;

typedef struct sar_server_stats {
    int32_t queued, active;
    int64_t rounds, completed;
    size_t pool_bytes;
} sar_server_stats;

typedef struct sar_server sar_server;

int sar_server_create(const sar_server_config *cfg, sar_server **out);
/* Stops the worker (after its queued GPU work drains) and frees everything. */
void sar_server_destroy(sar_server *server);
/* Queue a request.  SAR_EAGAIN: queue full; SAR_ENOMEM: it can never fit the
 * budget; SAR_EINVAL: bad request.  *ticket identifies it afterwards. */
int sar_submit(sar_server *server, const sar_request *req, uint64_t *ticket);
/* Non-blocking: SAR_OK when done (image_dev valid until sar_release,
 * latency_ms = submit to image ready), SAR_EAGAIN while queued or running,
 * the failure status if failed, SAR_ENOTFOUND for an unknown ticket. */
int sar_poll(sar_server *server, uint64_t ticket, int32_t *state, const void **image_dev,
             double *latency_ms);
/* Block until done or failed; SAR_ETIMEOUT after timeout_ms. */
int sar_wait(sar_server *server, uint64_t ticket, double timeout_ms);
/* Forget a request: frees its device image.  A queued request is dropped; a
 * running one is cancelled and freed once its GPU work has drained. */
int sar_release(sar_server *server, uint64_t ticket);
int sar_server_get_stats(sar_server *server, sar_server_stats *stats);

/*
 * Whole frame from host memory: copy beat, w_sar and trajectory to the
 * plan's device staging buffers, range-compress, backproject and copy the
 * image back to image_host; returns after the image is in host memory (the
 * call synchronises `stream`).  The uploads run on a copy stream of the plan
 * in two chunks of chirps, ordered after the work already queued on
 * `stream`; the kernels run on `stream`, the first chunk's while the second
 * chunk is still being copied.  A page-locked, mapped image_host (cudaHostAlloc
 * memory under unified addressing) is written by the last kernels directly;
 * any other image_host gets a device-to-host copy.  Frames whose upload is short are not split;
 * a split frame's image equals sar_backproject's up to FP32 summation order
 * (the second chunk accumulates onto the first).  Staging buffers are allocated on first use
 * for max_pulses chirps (counted in the HBM budget).  Calls on one plan must
 * not overlap.
 *  beat_host  complex64 [M][R][N];  w_az_host float [M] or NULL;
 *  q_tx_host  double [M][2];  q_rx_host double [M][R][2];
 *  image_host complex64 [n_pixels].
 */
int sar_form_image_host(sar_plan *plan, const void *beat_host, int32_t M,
                        const float *w_az_host, const double *q_tx_host,
                        const double *q_rx_host, void *image_host, void *stream);

/*
 * Autotuner of the backprojection launch shape (no counterpart in the paper):
 * times sar_backproject on these inputs for each candidate shape (pixel
 * tile, Cartesian grids only: 32 x 32, 64 x 16 and 16 x 64 pixels, see
 * sar_plan_set_tile_shape; then per tiling the Rx group: the plan's default
 * and the next smaller divisor of n_rx; CTAs per SM the registers are sized
 * for: 2 or 3; chirps per pipeline block: the largest that fits that many
 * CTAs' shared memory, 2/3 and 1/2 of it) and keeps the fastest in the plan
 * (see sar_plan_get_info); another tile shape than the plan's current one is
 * taken only if it is at least 2 % faster (its longer staged windows also
 * size the pulse block of any batch class the plan joins).  The choice is also remembered for the process,
 * keyed by device, Rx count, the staged window length and tile count of the
 * plan's first tiling (tile count and max_pulses rounded up to powers of
 * two) and profile storage: plans created later with the same key start
 * from it.  image_dev is overwritten.  Blocks until the timing runs on
 * `stream` finish.  Results of later calls do not depend on the choice
 * beyond FP32 rounding (summation order, and pixel offsets taken from
 * another tile reference).
 */
int sar_plan_autotune(sar_plan *plan, const void *prof_dev, int32_t M, const double *q_tx_dev,
                      const double *q_rx_dev, void *image_dev, void *stream);

/*
 * Set the backprojection launch shape explicitly, e.g. one saved from
 * sar_plan_get_info after sar_plan_autotune:
 *  rx_group          Rx channels per inner-loop group: 1..4, dividing n_rx
 *  regs_ctas_per_sm  2 or 3 (register budget of the kernel variant)
 *  pulses_per_block  chirps staged per pipeline step, 1..32
 * SAR_EINVAL if the shape is out of range or its shared memory does not
 * allow one CTA per SM; the plan keeps its previous shape then.  Results do
 * not depend on the shape beyond FP32 summation order.  Not thread-safe
 * against calls that use the plan.
 */
int sar_plan_set_launch(sar_plan *plan, int32_t rx_group, int32_t regs_ctas_per_sm, int32_t pulses_per_block);

/*
 * Pixel tile shape of a Cartesian plan: tiles of tile_w x (1024 / tile_w)
 * pixels, tile_w = 16, 32 (the default) or 64.  The backprojection stages,
 * per (tile, chirp, Rx), the bins the tile can reach (Alg. 2's
 * interpolation window), sized by the tile's circumradius: a square tile
 * needs the shortest window for its 1024 points, an elongated one can fit a
 * narrow grid with fewer empty slots.  The first use of a width builds and
 * uploads its tiling (tile offsets, output indices, split-tile partial sums:
 * about 20 bytes per grid pixel plus 8 KB per tile and 48 KB per SM, within
 * the plan's HBM budget); every tiling a plan has built stays allocated until
 * sar_plan_destroy, so launches and batches that captured an earlier tiling
 * remain valid.  The launch shape keeps its Rx group and register budget
 * where they fit and takes the largest pulse block that fits two CTAs per SM.
 * SAR_EINVAL for a point-list plan (its tiles are 1024 Morton-ordered points)
 * or another width; SAR_ENOMEM if the tiling does not fit the budget.  On
 * error the plan is unchanged.  Not thread-safe against calls that use the
 * plan.
 */
int sar_plan_set_tile_shape(sar_plan *plan, int32_t tile_w);

/*
 * Waits for the plan's device work and reports (then clears) kernel-side
 * error flags: SAR_OK or SAR_EBOUNDS.
 */
int sar_plan_check_errors(sar_plan *plan);

/*
 * Measured throughput of the two pipes that bound the backprojection, on the
 * current device (no counterpart in the paper; used to check the kernel's
 * ALU roofline against measured rates).  Runs three ~1 ms microbenchmark
 * kernels, each over 4 CTAs of 256 threads per SM with 8 independent
 * dependency chains per thread, and reports the best of three timed
 * launches: FP32 FMA lane-ops/s with scalar FFMA, with packed FFMA2 (2 lane
 * ops each) and MUFU operations/s (sin.approx).  Synchronous; allocates and
 * frees a small device buffer.  Errors: SAR_EINVAL (null pointers),
 * SAR_ENOMEM, SAR_ECUDA.
 */
int sar_alu_peaks(double *fma_lane_ops_per_s, double *ffma2_lane_ops_per_s, double *mufu_ops_per_s);

/* Static text for a status code. */
const char *sar_status_string(int status);

/* Library version (major * 10000 + minor * 100 + patch). */
int sar_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SAR_H */
