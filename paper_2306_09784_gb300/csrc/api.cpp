// Host side of the C ABI declared in include/sar.h: parameter validation,
// FP64 tables, pixel tiling, device memory and kernel launches.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <numeric>
#include <vector>

#include "sar_internal.h"

using namespace sar;

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr size_t kBpSmemTarget = 110 * 1024;  // two CTAs per SM
constexpr size_t kBpSmemMax = 227 * 1024;
constexpr int kMaxPulsesPerBlock = 32;

}  // namespace

struct sar_plan {
    sar_radar_params p{};
    int device = 0;
    int n_fft = 0, log2n = 0, crop_lo = 0, crop_hi = 0, n_bins = 0;
    double a1 = 0, beta = 0;
    double beta_frac = 0;  // cycles per bin of the interpolated fraction (beta at the time origin)
    int sign = 1;
    bool fp16 = false;
    int64_t n_pixels = 0;
    int n_tiles = 0;
    int L = 0, Mb = 0, rg = 1;
    size_t bp_smem = 0;
    int num_sms = 0, ctas_per_sm = 0, G = 0, minb = 2;
    size_t partial_slots = 0;  // partial-sum tile slots allocated
    float fd_max = 0.f;
    // device memory owned by the plan
    float *d_wr = nullptr;
    float2 *d_tw = nullptr;
    float2 *d_rot = nullptr;
    float2 *d_pix = nullptr;
    int *d_out = nullptr;
    TileInfo *d_tiles = nullptr;
    float2 *d_partial = nullptr;
    int *d_err = nullptr;
    double *d_means = nullptr;  // sar_doppler_offsets: mean positions and velocity
    // tables of the split-transform range compression (when supported)
    bool rc_split = false;
    float2 *d_rc_pre = nullptr, *d_rc_twd = nullptr;
    // staging buffers of sar_form_image_host
    void *s_beat = nullptr;
    float *s_waz = nullptr;
    double *s_qtx = nullptr, *s_qrx = nullptr;
    void *s_prof = nullptr, *s_img = nullptr;
    // its copy stream and events (created on first use)
    cudaStream_t s_copy = nullptr;
    cudaEvent_t ev_start = nullptr, ev_chunk[2] = {nullptr, nullptr}, ev_traj = nullptr;
    size_t budget = 0, used = 0;
    std::vector<void *> allocs;
    // Pixel tilings built so far; the current one is mirrored in n_tiles, L,
    // d_pix, d_out, d_tiles, d_partial and partial_slots.  A Cartesian grid
    // can be tiled 16 x 64, 32 x 32 or 64 x 16 (tile width tw); a point list
    // has its one Morton tiling (tw = 0).  Buffers of every tiling live until
    // the plan is destroyed, so launches in flight and batches that captured
    // an earlier tiling stay valid.
    struct Tiling {
        int tw = 0, n_tiles = 0, L = 0;
        size_t partial_slots = 0;
        float2 *d_pix = nullptr;
        int *d_out = nullptr;
        TileInfo *d_tiles = nullptr;
        float2 *d_partial = nullptr;
    };
    std::vector<Tiling> tilings;
    int tile_w = 0;
    sar_grid grid{};  // the Cartesian grid (pixels_xy = null), for re-tiling
    int key_L = 0, key_tiles = 0;  // window and tile count of the first tiling (remembered-shape key)
};

// Requests of a batch are grouped into classes with the same Rx group and
// profile storage (the pixel loop is specialised on both); one persistent
// launch runs every class, each on its share of the CTAs.
struct BatchClass {
    int rg = 0;
    bool fp16 = false;
    int j0 = 0, n = 0;       // jobs [j0, j0 + n) of the sorted table
    int off = 0;             // first entry of its prefix sums (j0 + class index)
    long long units = 0;
    double updates = 0;      // pixel slots x chirps x Rx of its jobs
    int tiles = 0, G = 0, cta_begin = 0, tile_base = 0;
    size_t smem = 0;
};

// Launch choice per class key (storage x Rx group): chirps per pipeline block
// (0 = each request's plan's own).
struct ClassShape {
    int mb = 0;
    bool param = true;  // job arguments as kernel parameters (classes of up to kParamJobs requests)
    float ms = 0.f;     // its launch time as measured by sar_batch_autotune (0: not tuned)
};

struct sar_batch {
    int device = 0;
    int max_jobs = 0, n_jobs = 0;
    int num_sms = 0, g_cap = 0, G = 0;
    long long units = 0;
    int tiles = 0;
    bool committed = false, upload_pending = false;
    BpArgs *h_jobs = nullptr;    // in the order added, each with its plan's own block size
    // One pinned upload blob and its device copy, [ub | tb | sorted jobs], so
    // that a commit is a single host-to-device copy:
    unsigned char *h_blob = nullptr, *d_blob = nullptr;
    size_t jobs_off = 0;
    BpArgs *h_sorted = nullptr;  // grouped by class (upload source)
    long long *h_ub = nullptr;   // per-class prefix sums of units
    int *h_tb = nullptr;         // per-class prefix sums of tiles
    BpArgs *d_jobs = nullptr;
    long long *d_ub = nullptr;
    int *d_tb = nullptr;
    float2 *d_scratch = nullptr;
    int *d_err = nullptr;        // [4] checks of the batched kernels
    cudaEvent_t uploaded = nullptr;
    int n_classes = 0;
    BatchClass cls[kBatchClasses];
    ClassShape shape[kBatchClasses];
    // occupancy of each class key's kernel, cached for its shared-memory size
    size_t occ_smem[kBatchClasses] = {};
    int occ_ctas[kBatchClasses] = {};
    size_t scratch_slots = 0;    // partial-sum slots: two per CTA of every class
    // range compressions of frames added with sar_batch_add_frame: jobs of the
    // split kernel grouped into one launch per (N, os, convention, storage)
    // class; frames whose shape needs the general kernel get their own launch
    struct RcJob {
        RcSplitArgs a;
        int sign = 1, mode = 0;
        bool split = false;
        sar_plan *plan = nullptr;
        const void *beat = nullptr;
        const float *w_az = nullptr;
        void *prof = nullptr;
        int M = 0;
    };
    std::vector<RcJob> rc;
    struct RcClass {
        RcSplitArgs a;           // shape (N2, os) of its jobs
        int sign = 1, mode = 0;
        int j0 = 0, n = 0, off = 0;
        long long groups = 0;
    };
    RcClass rcc[kBatchClasses];
    int n_rcc = 0;
    size_t rc_off = 0, rc_jobs_off = 0;  // blob offsets of the group prefix sums and the jobs
    long long *h_rgb = nullptr, *d_rgb = nullptr;
    RcSplitArgs *h_rjobs = nullptr, *d_rjobs = nullptr;
};

namespace {

struct DeviceGuard {
    int old = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&old) != cudaSuccess) {
            ok = false;
            return;
        }
        if (old != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (old >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != old) cudaSetDevice(old);
    }
};

int dev_alloc(sar_plan *pl, size_t bytes, void **out) {
    *out = nullptr;
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    if (pl->budget && pl->used + bytes > pl->budget) return SAR_ENOMEM;
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SAR_ENOMEM;
    }
    pl->used += bytes;
    pl->allocs.push_back(p);
    *out = p;
    return SAR_OK;
}

template <class T>
int upload(sar_plan *pl, const std::vector<T> &h, T **out) {
    void *p = nullptr;
    int rc = dev_alloc(pl, h.size() * sizeof(T), &p);
    if (rc) return rc;
    if (!h.empty() && cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return SAR_ECUDA;
    *out = static_cast<T *>(p);
    return SAR_OK;
}

void free_plan(sar_plan *pl) {
    if (!pl) return;
    DeviceGuard g(pl->device);
    cudaDeviceSynchronize();
    for (void *p : pl->allocs) cudaFree(p);
    if (pl->s_copy) cudaStreamDestroy(pl->s_copy);
    for (cudaEvent_t e : {pl->ev_start, pl->ev_chunk[0], pl->ev_chunk[1], pl->ev_traj})
        if (e) cudaEventDestroy(e);
    delete pl;
}

// Largest of 4, 3, 2, 1 that divides the Rx count.
int default_rx_group(int R) { return (R % 4 == 0) ? 4 : (R % 3 == 0) ? 3 : (R % 2 == 0) ? 2 : 1; }

// Validate and install a backprojection launch shape; the plan is unchanged
// on failure.
int apply_launch(sar_plan *pl, int rg, int minb, int Mb) {
    if (rg < 1 || rg > 4 || pl->p.n_rx % rg != 0 || minb < 2 || minb > 3 || Mb < 1 || Mb > kMaxPulsesPerBlock)
        return SAR_EINVAL;
    const size_t smem = bp_smem_bytes(Mb, pl->p.n_rx, pl->L, pl->fp16);
    if (smem > kBpSmemMax) return SAR_EINVAL;
    if (bp_prepare(pl->fp16, rg, smem) != cudaSuccess) {
        cudaGetLastError();
        return SAR_EINVAL;
    }
    int occ = 0;
    if (bp_occupancy(pl->fp16, rg, smem, minb, &occ) != 0 || occ < 1) {
        cudaGetLastError();
        return SAR_EINVAL;
    }
    occ = std::min(occ, minb);
    const int G = pl->num_sms * occ;
    // split-tile slots of the worst case (one pulse block per tile)
    if ((size_t)G * (size_t)(pl->n_tiles / G + 2) > pl->partial_slots) return SAR_EINVAL;
    pl->rg = rg;
    pl->minb = minb;
    pl->Mb = Mb;
    pl->bp_smem = smem;
    pl->ctas_per_sm = occ;
    pl->G = G;
    return SAR_OK;
}

// Launch shapes chosen by sar_plan_autotune, remembered for the process and
// keyed by what the shape depends on: device, Rx count, window length,
// storage, and max_pulses and tile count rounded up to powers of two.
using ShapeKey = std::tuple<int, int, int, int, int, int>;
struct Shape {
    int rg, minb, Mb, tw;
};
std::mutex g_shape_mu;
std::map<ShapeKey, Shape> g_shapes;

int pow2_ceil(long long v) {
    int e = 0;
    while ((1ll << e) < v && e < 62) ++e;
    return e;
}

// Keyed by the plan's first tiling, whatever tiling it uses now.
ShapeKey shape_key(const sar_plan *pl) {
    return ShapeKey{pl->device, pl->p.n_rx, pl->key_L, pl->fp16 ? 1 : 0, pow2_ceil(pl->p.max_pulses),
                    pow2_ceil(pl->key_tiles)};
}

void remember_shape(const sar_plan *pl) {
    std::lock_guard<std::mutex> g(g_shape_mu);
    g_shapes[shape_key(pl)] = Shape{pl->rg, pl->minb, pl->Mb, pl->tile_w};
}

int plan_retile(sar_plan *pl, int tw);

// Start a new plan from a remembered shape, if there is one that fits.
void recall_shape(sar_plan *pl) {
    Shape sh{};
    {
        std::lock_guard<std::mutex> g(g_shape_mu);
        auto it = g_shapes.find(shape_key(pl));
        if (it == g_shapes.end()) return;
        sh = it->second;
    }
    // the plan keeps its default tiling and shape where these fail
    if (sh.tw != pl->tile_w && plan_retile(pl, sh.tw) != SAR_OK) return;
    apply_launch(pl, sh.rg, sh.minb, sh.Mb);
}

// Modified Bessel I0 from its power series.
double i0_series(double x) {
    double term = 1.0, sum = 1.0;
    const double h = x / 2.0;
    for (int k = 1; k < 1000; ++k) {
        term *= h / k;
        const double t2 = term * term;
        sum += t2;
        if (t2 <= sum * 1e-17) break;
    }
    return sum;
}

std::vector<float> range_window(int kind, int N, double beta) {
    std::vector<float> w(N, 1.0f);
    if (N == 1 || kind == SAR_WINDOW_RECT) return w;
    for (int n = 0; n < N; ++n) {
        double v = 1.0;
        if (kind == SAR_WINDOW_HANN) {
            v = 0.5 * (1.0 - std::cos(2.0 * kPi * n / (N - 1)));
        } else {
            const double t = 2.0 * n / (N - 1) - 1.0;
            v = i0_series(beta * std::sqrt(std::max(0.0, 1.0 - t * t))) / i0_series(beta);
        }
        w[n] = (float)v;
    }
    return w;
}

int ilog2_exact(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return (1 << l) == n ? l : -1;
}

uint32_t spread_bits(uint32_t v) {
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

struct HostTiles {
    std::vector<float2> pix;
    std::vector<int> out;
    std::vector<TileInfo> tiles;
    double rho_max = 0;
};

void finish_tile(HostTiles &ht, int t, const std::vector<double> &xs, const std::vector<double> &ys,
                 const std::vector<int> &oi) {
    TileInfo ti{};
    if (xs.empty()) {
        ht.tiles[t] = ti;
        return;
    }
    const double xl = *std::min_element(xs.begin(), xs.end()), xh = *std::max_element(xs.begin(), xs.end());
    const double yl = *std::min_element(ys.begin(), ys.end()), yh = *std::max_element(ys.begin(), ys.end());
    ti.x = 0.5 * (xl + xh);
    ti.y = 0.5 * (yl + yh);
    double rho = 0;
    for (size_t i = 0; i < xs.size(); ++i) rho = std::max(rho, std::hypot(xs[i] - ti.x, ys[i] - ti.y));
    ti.rho = rho * (1.0 + 1e-9) + 1e-9;
    ti.n_valid = (int)xs.size();
    ht.tiles[t] = ti;
    ht.rho_max = std::max(ht.rho_max, ti.rho);
    for (size_t i = 0; i < xs.size(); ++i) {
        // slot i of the tile
        const size_t s = (size_t)t * kTilePx + i;
        ht.pix[s] = make_float2((float)(xs[i] - ti.x), (float)(ys[i] - ti.y));
        ht.out[s] = oi[i];
    }
}

// Tiles of kTilePx reconstruction points.  Cartesian grid: rectangles of
// tw x (kTilePx / tw) pixels, row-major over the grid; slot = ly tw + lx, so
// thread t of a CTA owns slots t + kBpThreads j.  Point list: Morton order,
// kTilePx consecutive points per tile (tw is ignored).
int build_tiles(const sar_grid *g, HostTiles &ht, int64_t *n_pixels, int tw) {
    if (g->pixels_xy == nullptr) {
        if (g->nx <= 0 || g->ny <= 0 || !std::isfinite(g->x0) || !std::isfinite(g->y0) ||
            !std::isfinite(g->dx) || !std::isfinite(g->dy))
            return SAR_EINVAL;
        if (tw <= 0 || kTilePx % tw != 0) return SAR_EINVAL;
        const int th = kTilePx / tw;
        const int64_t np = (int64_t)g->nx * g->ny;
        if (np > (int64_t)1 << 30) return SAR_EINVAL;
        *n_pixels = np;
        const int ntx = (g->nx + tw - 1) / tw, nty = (g->ny + th - 1) / th;
        const int T = ntx * nty;
        ht.pix.assign((size_t)T * kTilePx, make_float2(0.f, 0.f));
        ht.out.assign((size_t)T * kTilePx, -1);
        ht.tiles.assign(T, TileInfo{});
        ht.rho_max = 0;
        std::vector<double> xs, ys;
        std::vector<int> oi;
        for (int ty = 0; ty < nty; ++ty)
            for (int tx = 0; tx < ntx; ++tx) {
                const int t = ty * ntx + tx;
                xs.clear();
                ys.clear();
                oi.clear();
                for (int ly = 0; ly < th; ++ly)
                    for (int lx = 0; lx < tw; ++lx) {
                        const int ix = tx * tw + lx, iy = ty * th + ly;
                        const bool v = ix < g->nx && iy < g->ny;
                        xs.push_back(v ? g->x0 + ix * g->dx : 0.0);
                        ys.push_back(v ? g->y0 + iy * g->dy : 0.0);
                        oi.push_back(v ? iy * g->nx + ix : -1);
                    }
                // reference and radius from the valid points only
                std::vector<double> vx, vy;
                std::vector<int> vo;
                for (size_t i = 0; i < oi.size(); ++i)
                    if (oi[i] >= 0) {
                        vx.push_back(xs[i]);
                        vy.push_back(ys[i]);
                        vo.push_back(oi[i]);
                    }
                finish_tile(ht, t, vx, vy, vo);
                // place points at their 2-D slots (finish_tile packed them)
                const TileInfo &ti = ht.tiles[t];
                for (int s = 0; s < kTilePx; ++s) {
                    const size_t d = (size_t)t * kTilePx + s;
                    if (oi[s] >= 0) {
                        ht.pix[d] = make_float2((float)(xs[s] - ti.x), (float)(ys[s] - ti.y));
                        ht.out[d] = oi[s];
                    } else {
                        ht.pix[d] = make_float2(0.f, 0.f);
                        ht.out[d] = -1;
                    }
                }
            }
        return SAR_OK;
    }
    // explicit point list: Morton order, 1024 consecutive points per tile
    const int64_t np = g->n_pixels;
    if (np <= 0 || np > (int64_t)1 << 30) return SAR_EINVAL;
    *n_pixels = np;
    const double *xy = g->pixels_xy;
    double xl = INFINITY, xh = -INFINITY, yl = INFINITY, yh = -INFINITY;
    for (int64_t i = 0; i < np; ++i) {
        const double x = xy[2 * i], y = xy[2 * i + 1];
        if (!std::isfinite(x) || !std::isfinite(y)) return SAR_EINVAL;
        xl = std::min(xl, x);
        xh = std::max(xh, x);
        yl = std::min(yl, y);
        yh = std::max(yh, y);
    }
    const double sx = xh > xl ? 65535.0 / (xh - xl) : 0.0;
    const double sy = yh > yl ? 65535.0 / (yh - yl) : 0.0;
    std::vector<uint32_t> code(np);
    for (int64_t i = 0; i < np; ++i) {
        const uint32_t qx = (uint32_t)std::lround((xy[2 * i] - xl) * sx);
        const uint32_t qy = (uint32_t)std::lround((xy[2 * i + 1] - yl) * sy);
        code[i] = spread_bits(qx) | (spread_bits(qy) << 1);
    }
    std::vector<int64_t> order(np);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return code[a] < code[b]; });
    const int T = (int)((np + kTilePx - 1) / kTilePx);
    ht.pix.assign((size_t)T * kTilePx, make_float2(0.f, 0.f));
    ht.out.assign((size_t)T * kTilePx, -1);
    ht.tiles.assign(T, TileInfo{});
    std::vector<double> xs, ys;
    std::vector<int> oi;
    for (int t = 0; t < T; ++t) {
        xs.clear();
        ys.clear();
        oi.clear();
        for (int64_t k = (int64_t)t * kTilePx; k < std::min(np, (int64_t)(t + 1) * kTilePx); ++k) {
            xs.push_back(xy[2 * order[k]]);
            ys.push_back(xy[2 * order[k] + 1]);
            oi.push_back((int)order[k]);
        }
        finish_tile(ht, t, xs, ys, oi);
    }
    return SAR_OK;
}

int validate_params(const sar_radar_params *p) {
    if (!p) return SAR_EINVAL;
    if (!(p->f0 > 0) || !(p->slope != 0) || !(p->fs > 0) || !(p->c > 0)) return SAR_EINVAL;
    if (!std::isfinite(p->f0) || !std::isfinite(p->slope) || !std::isfinite(p->fs) || !std::isfinite(p->c))
        return SAR_EINVAL;
    if (p->n_samples < 1 || p->os < 1 || p->n_rx < 1 || p->n_rx > 64 || p->max_pulses < 1) return SAR_EINVAL;
    const long long nfft = (long long)p->n_samples * p->os;
    if (nfft < 64 || nfft > 16384 || ilog2_exact((int)nfft) < 0) return SAR_EINVAL;
    if (p->range_window < 0 || p->range_window > 2) return SAR_EINVAL;
    if (p->precision != SAR_PREC_FP32 && p->precision != SAR_PREC_FP16) return SAR_EINVAL;
    if (p->phase_sign != 1 && p->phase_sign != -1) return SAR_EINVAL;
    if (p->crop_lo < 0 || p->crop_hi < 0) return SAR_EINVAL;
    if (!(p->crop_lo == 0 && p->crop_hi == 0)) {
        if (p->crop_lo >= p->crop_hi || p->crop_hi > nfft - 1) return SAR_EINVAL;
    }
    if (!(p->max_doppler_bins >= 0) || p->max_doppler_bins > 64) return SAR_EINVAL;
    if (p->time_origin != SAR_ORIGIN_FIRST_SAMPLE && p->time_origin != SAR_ORIGIN_CHIRP_CENTRE)
        return SAR_EINVAL;
    if (p->range_window == SAR_WINDOW_KAISER && !(p->kaiser_beta >= 0 && p->kaiser_beta < 100)) return SAR_EINVAL;
    // bins per metre a1 and phase cycles per bin beta (the kernels scale by
    // 2 pi beta and by its inverse)
    const double a1 = p->slope * (double)nfft / (p->c * p->fs);
    if (!(a1 > 0)) return SAR_EINVAL;
    const double beta = p->f0 / (p->c * a1);
    if (!(beta >= 1e-9 && beta <= 1e9)) return SAR_EINVAL;
    return SAR_OK;
}

// Shape checks of the reconstruction points that need no device (the point
// values are checked while the tiles are built).
int validate_grid(const sar_grid *g) {
    if (!g) return SAR_EINVAL;
    if (g->pixels_xy == nullptr) {
        if (g->nx <= 0 || g->ny <= 0 || (int64_t)g->nx * g->ny > (int64_t)1 << 30) return SAR_EINVAL;
        if (!std::isfinite(g->x0) || !std::isfinite(g->y0) || !std::isfinite(g->dx) || !std::isfinite(g->dy))
            return SAR_EINVAL;
        return SAR_OK;
    }
    return (g->n_pixels <= 0 || g->n_pixels > (int64_t)1 << 30) ? SAR_EINVAL : SAR_OK;
}

// Staged window length of a tiling: it covers a1 (d0 -+ 2 rho) -+ fd_max
// plus guards for every tile (two-way range spread of a disc of radius rho),
// and the per-tile window constants that depend on it.
int window_length(const sar_plan *pl, HostTiles &ht) {
    const double span = 4.0 * ht.rho_max * pl->a1 + 2.0 * std::ceil((double)pl->fd_max);
    int L = (int)std::ceil(span) + 2 * kGuardBins + 4;
    L = (L + 3) & ~3;
    for (TileInfo &ti : ht.tiles) {
        const double o_allow = ((double)(L - 3 - 2 * kGuardBins) - 2.0 * pl->fd_max - 4.0 * ti.rho * pl->a1) /
                               (2.0 * pl->a1);
        ti.o_allow = (float)o_allow;
        ti.klo_off = (float)(pl->a1 * (2.0 * ti.rho + o_allow) + pl->fd_max);
    }
    return L;
}

// Largest pulse block whose shared memory fits two CTAs per SM.
int default_block(const sar_plan *pl, int L) {
    const int R = pl->p.n_rx;
    const size_t per_pulse = bp_smem_bytes(1, R, L, pl->fp16);
    int Mb = (int)std::min<size_t>(kMaxPulsesPerBlock, std::max<size_t>(1, kBpSmemTarget / per_pulse));
    while (Mb > 1 && bp_smem_bytes(Mb, R, L, pl->fp16) > kBpSmemTarget) --Mb;
    return Mb;
}

// Upload a tiling and its split-tile partial sums, and make it current.  The
// partial sums cover any persistent grid G of 1 to 3 CTAs per SM: a launch
// needs G seg_max slots with seg_max <= n_tiles / G + 2.
int install_tiling(sar_plan *pl, const HostTiles &ht, int tw, int L) {
    sar_plan::Tiling t;
    t.tw = tw;
    t.L = L;
    t.n_tiles = (int)ht.tiles.size();
    t.partial_slots = (size_t)t.n_tiles + 6u * (size_t)pl->num_sms;
    int rc = upload(pl, ht.pix, &t.d_pix);
    if (!rc) rc = upload(pl, ht.out, &t.d_out);
    if (!rc) rc = upload(pl, ht.tiles, &t.d_tiles);
    if (!rc) {
        void *q = nullptr;
        rc = dev_alloc(pl, t.partial_slots * kTilePx * sizeof(float2), &q);
        t.d_partial = (float2 *)q;
    }
    if (rc) return rc;  // what was allocated is freed with the plan
    pl->tilings.push_back(t);
    return SAR_OK;
}

void use_tiling(sar_plan *pl, const sar_plan::Tiling &t) {
    pl->tile_w = t.tw;
    pl->n_tiles = t.n_tiles;
    pl->L = t.L;
    pl->partial_slots = t.partial_slots;
    pl->d_pix = t.d_pix;
    pl->d_out = t.d_out;
    pl->d_tiles = t.d_tiles;
    pl->d_partial = t.d_partial;
}

// Switch a Cartesian plan to tiles tw pixels wide (16, 32 or 64), building
// the tiling on first use.  The launch shape keeps its Rx group and register
// budget where they fit; the pulse block becomes the largest that fits two
// CTAs per SM.  On failure the plan is unchanged.
int plan_retile(sar_plan *pl, int tw) {
    if (pl->tile_w == 0) return SAR_EINVAL;  // point list: one Morton tiling
    if (tw != 16 && tw != 32 && tw != 64) return SAR_EINVAL;
    if (tw == pl->tile_w) return SAR_OK;
    sar_plan::Tiling prev = pl->tilings[0];
    for (const sar_plan::Tiling &t : pl->tilings)
        if (t.tw == pl->tile_w) prev = t;
    const int rg = pl->rg, minb = pl->minb, Mb0 = pl->Mb;
    int idx = -1;
    for (size_t i = 0; i < pl->tilings.size(); ++i)
        if (pl->tilings[i].tw == tw) idx = (int)i;
    if (idx < 0) {
        HostTiles ht;
        int64_t np = 0;
        int rc = build_tiles(&pl->grid, ht, &np, tw);
        if (rc) return rc;
        const int L = window_length(pl, ht);
        if (bp_smem_bytes(1, pl->p.n_rx, L, pl->fp16) > kBpSmemMax) return SAR_EINVAL;
        rc = install_tiling(pl, ht, tw, L);
        if (rc) return rc;
        idx = (int)pl->tilings.size() - 1;
    }
    use_tiling(pl, pl->tilings[idx]);
    const int Mb = default_block(pl, pl->L);
    if (apply_launch(pl, rg, minb, Mb) == SAR_OK || apply_launch(pl, rg, 2, Mb) == SAR_OK ||
        apply_launch(pl, default_rx_group(pl->p.n_rx), 2, Mb) == SAR_OK)
        return SAR_OK;
    use_tiling(pl, prev);
    apply_launch(pl, rg, minb, Mb0);
    return SAR_EINVAL;
}

int plan_create(const sar_radar_params *params, const sar_grid *grid, size_t budget, sar_plan **out) {
    int rc = validate_params(params);
    if (rc) return rc;
    rc = validate_grid(grid);
    if (rc) return rc;
    sar_plan *pl = new (std::nothrow) sar_plan();
    if (!pl) return SAR_ENOMEM;
    pl->p = *params;
    pl->budget = budget;
    if (cudaGetDevice(&pl->device) != cudaSuccess) {
        delete pl;
        return SAR_ECUDA;
    }
    const sar_radar_params &p = pl->p;
    pl->n_fft = p.n_samples * p.os;
    pl->log2n = ilog2_exact(pl->n_fft);
    pl->crop_lo = (p.crop_lo == 0 && p.crop_hi == 0) ? 0 : p.crop_lo;
    pl->crop_hi = (p.crop_lo == 0 && p.crop_hi == 0) ? pl->n_fft - 1 : p.crop_hi;
    pl->n_bins = pl->crop_hi - pl->crop_lo + 1;
    pl->sign = p.phase_sign;
    pl->fp16 = p.precision == SAR_PREC_FP16;
    pl->a1 = p.slope * pl->n_fft / (p.c * p.fs);  // validated positive
    pl->beta = p.f0 / (p.c * pl->a1);              // validated in [1e-9, 1e9]
    // A transform whose time origin is sample t0 has the carrier f0 + slope
    // t0 / fs, i.e. beta + t0 / N_fft cycles per bin, and its bin k equals the
    // first-sample transform's times exp(-sign j 2 pi t0 k / N_fft).  That
    // rotation and the one by beta combine into the per-bin rotation by beta
    // the range compression already stores, so only the backprojection's
    // fractional-phase rate changes.
    pl->beta_frac = pl->beta;
    if (p.time_origin == SAR_ORIGIN_CHIRP_CENTRE)
        pl->beta_frac += 0.5 * (double)(p.n_samples - 1) / (double)pl->n_fft;
    pl->fd_max = (float)p.max_doppler_bins;

    HostTiles ht;
    const int tw0 = grid->pixels_xy == nullptr ? 32 : 0;
    rc = build_tiles(grid, ht, &pl->n_pixels, tw0);
    if (rc) {
        delete pl;
        return rc;
    }
    if (tw0) {
        pl->grid = *grid;
        pl->grid.pixels_xy = nullptr;
    }
    pl->tile_w = tw0;
    pl->n_tiles = (int)ht.tiles.size();
    pl->L = window_length(pl, ht);
    pl->key_L = pl->L;
    pl->key_tiles = pl->n_tiles;
    pl->rg = default_rx_group(p.n_rx);
    pl->Mb = default_block(pl, pl->L);
    pl->bp_smem = bp_smem_bytes(pl->Mb, p.n_rx, pl->L, pl->fp16);
    if (pl->bp_smem > kBpSmemMax) {
        delete pl;
        return SAR_EINVAL;  // reconstruction points too spread out for one tile window
    }

    DeviceGuard dg(pl->device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, pl->device) != cudaSuccess) {
        delete pl;
        return SAR_ECUDA;
    }
    pl->num_sms = prop.multiProcessorCount;
    // set-up of sar_backproject_noalloc's static scratch on this device (its
    // module load reserves 16 MiB here, never in the imaging call)
    rc = noalloc_setup(pl->device);
    if (rc) {
        delete pl;
        return rc;
    }
    if (bp_prepare(pl->fp16, pl->rg, pl->bp_smem) != cudaSuccess ||
        bp_occupancy(pl->fp16, pl->rg, pl->bp_smem, pl->minb, &pl->ctas_per_sm) != 0 || pl->ctas_per_sm < 1) {
        cudaGetLastError();
        delete pl;
        return SAR_ECUDA;
    }
    pl->G = pl->num_sms * pl->ctas_per_sm;

    // FP64 tables
    std::vector<float> wr = range_window(p.range_window, p.n_samples, p.kaiser_beta);
    std::vector<float2> tw(pl->n_fft);
    for (int i = 0; i < pl->n_fft; ++i) {
        const double ang = pl->sign * 2.0 * kPi * (double)i / pl->n_fft;
        tw[i] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    std::vector<float2> rot(pl->n_bins);
    for (int i = 0; i < pl->n_bins; ++i) {
        const double k = (double)(pl->crop_lo + i);
        double cyc = k * pl->beta;
        cyc -= std::floor(cyc);
        const double ang = pl->sign * 2.0 * kPi * cyc;
        rot[i] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }

    // split-transform range compression: input rotations with the window
    // folded in, and the inter-pass twiddles (FP64, stored FP32)
    std::vector<float2> rc_pre, rc_twd;
    pl->rc_split = rc_split_supported(p.n_samples, p.os);
    if (pl->rc_split) {
        const int N = p.n_samples, n2 = N / 32, nf = pl->n_fft;
        auto ang = [&](long long num, long long den) { return pl->sign * 2.0 * kPi * (double)(num % den) / den; };
        rc_pre.resize((size_t)p.os * N);
        for (int q = 0; q < p.os; ++q)
            for (int n = 0; n < N; ++n) {
                const double w = wr[n], t = ang((long long)n * q, nf);
                rc_pre[(size_t)q * N + n] = make_float2((float)(w * std::cos(t)), (float)(w * std::sin(t)));
            }
        rc_twd.resize((size_t)n2 * 32);
        for (int j = 0; j < n2; ++j)
            for (int k1 = 0; k1 < 32; ++k1) {
                const double t = ang((long long)j * k1, N);
                rc_twd[(size_t)k1 * n2 + j] = make_float2((float)std::cos(t), (float)std::sin(t));
            }
    }

    rc = upload(pl, wr, &pl->d_wr);
    if (!rc && pl->rc_split) rc = upload(pl, rc_pre, &pl->d_rc_pre);
    if (!rc && pl->rc_split) rc = upload(pl, rc_twd, &pl->d_rc_twd);
    if (!rc) rc = upload(pl, tw, &pl->d_tw);
    if (!rc) rc = upload(pl, rot, &pl->d_rot);
    if (!rc) rc = install_tiling(pl, ht, tw0, pl->L);
    if (!rc) use_tiling(pl, pl->tilings.back());
    if (!rc) {
        void *q = nullptr;
        rc = dev_alloc(pl, sizeof(int) * 4, &q);
        pl->d_err = (int *)q;
        if (!rc && cudaMemset(q, 0, sizeof(int) * 4) != cudaSuccess) rc = SAR_ECUDA;
    }
    if (!rc) {
        void *q = nullptr;
        rc = dev_alloc(pl, sizeof(double) * 8, &q);
        pl->d_means = (double *)q;
    }
    if (rc) {
        free_plan(pl);
        return rc;
    }
    recall_shape(pl);
    *out = pl;
    return SAR_OK;
}

size_t profile_bytes(const sar_plan *pl, int M) {
    const size_t rows = (size_t)M * pl->p.n_rx;
    if (pl->fp16) return ((rows * 4 + 255) & ~size_t(255)) + rows * pl->n_bins * 4;
    return rows * pl->n_bins * 8;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }


// Split-kernel job from the general kernel's arguments and the plan's tables.
void split_args(const sar_plan *pl, const RcArgs &a, RcSplitArgs *b) {
    b->beat = a.beat;
    b->pre = pl->d_rc_pre;
    b->twd = pl->d_rc_twd;
    b->rot = pl->d_rot;
    b->w_az = a.w_az;
    b->out = a.out;
    b->scales = a.scales;
    b->rows = a.rows;
    b->R = a.R;
    b->N2 = pl->p.n_samples / 32;
    b->os = pl->p.os;
    b->crop_lo = pl->crop_lo;
    b->crop_hi = pl->crop_hi;
    b->n_bins = pl->n_bins;
}

// General-kernel arguments of range compression of pulses [m0, m0 + M) of a
// profile buffer laid out for M_tot pulses; `beat` and `w_az` point at pulse m0.
RcArgs rc_args(const sar_plan *pl, const void *beat, int m0, int M, int M_tot, const float *w_az, void *out,
               int mode) {
    RcArgs a{};
    a.beat = (const float2 *)beat;
    a.w_r = pl->d_wr;
    a.tw = pl->d_tw;
    a.rot = pl->d_rot;
    a.w_az = w_az;
    a.rows = (long long)M * pl->p.n_rx;
    a.R = pl->p.n_rx;
    a.N = pl->p.n_samples;
    a.n_fft = pl->n_fft;
    a.log2n = pl->log2n;
    a.crop_lo = pl->crop_lo;
    a.n_bins = pl->n_bins;
    const size_t r0 = (size_t)m0 * pl->p.n_rx;
    if (mode == kRcProfileF16) {
        const size_t rows = (size_t)M_tot * pl->p.n_rx;
        a.scales = (float *)out + r0;
        a.out = (unsigned char *)out + ((rows * 4 + 255) & ~size_t(255)) + r0 * pl->n_bins * 4;
    } else if (mode == kRcProfileF32) {
        a.out = (float2 *)out + r0 * pl->n_bins;
    } else {
        a.out = (float2 *)out + r0 * pl->n_fft;
    }
    return a;
}

// Range compression of pulses [m0, m0 + M) of a profile buffer laid out for
// M_tot pulses; `beat` and `w_az` point at pulse m0.
int rc_launch_part(sar_plan *pl, const void *beat, int m0, int M, int M_tot, const float *w_az, void *out,
                   int mode, cudaStream_t s) {
    const RcArgs a = rc_args(pl, beat, m0, M, M_tot, w_az, out, mode);
    DeviceGuard dg(pl->device);
    if (!dg.ok) return SAR_ECUDA;
    if (pl->rc_split && mode != kRcSpectrum) {
        RcSplitArgs b{};
        split_args(pl, a, &b);
        return launch_range_compress_split(b, pl->sign, mode, s) == cudaSuccess ? SAR_OK : SAR_ECUDA;
    }
    return launch_range_compress(a, pl->sign, mode, s) == cudaSuccess ? SAR_OK : SAR_ECUDA;
}

int rc_launch(sar_plan *pl, const void *beat, int M, const float *w_az, void *out, int mode, cudaStream_t s) {
    return rc_launch_part(pl, beat, 0, M, M, w_az, out, mode, s);
}

// Kernel arguments common to every backprojection launch of a plan: the
// profile layout, geometry tables and phase constants.  The launch fields
// (G, seg_max, partial) are left for the caller.
// With M_tot > 0, the call covers pulses [m0, m0 + M) of a profile buffer
// laid out for M_tot pulses, and q_tx, q_rx point at pulse m0.
BpArgs common_bp_args(const sar_plan *pl, const void *prof, int M, const double *q_tx, const double *q_rx,
                      const float *fd, void *image, int accumulate, int m0 = 0, int M_tot = 0) {
    BpArgs a{};
    if (M_tot <= 0) M_tot = M;
    const size_t rows = (size_t)M_tot * pl->p.n_rx, r0 = (size_t)m0 * pl->p.n_rx;
    if (pl->fp16) {
        a.prof_scale = (const float *)prof + r0;
        a.prof = (const unsigned char *)prof + ((rows * 4 + 255) & ~size_t(255)) + r0 * pl->n_bins * 4;
    } else {
        a.prof = (const float2 *)prof + r0 * pl->n_bins;
        a.prof_scale = nullptr;
    }
    a.q_tx = q_tx;
    a.q_rx = q_rx;
    a.fdopp = fd;
    a.image = (float2 *)image;
    a.partial = nullptr;
    a.err = pl->d_err;
    a.pix = pl->d_pix;
    a.out_idx = pl->d_out;
    a.tiles = pl->d_tiles;
    a.M = M;
    a.R = pl->p.n_rx;
    a.n_tiles = pl->n_tiles;
    a.Mb = pl->Mb;
    a.L = pl->L;
    a.blocks_per_tile = (M + pl->Mb - 1) / pl->Mb;
    a.units = (long long)pl->n_tiles * a.blocks_per_tile;
    a.n_bins = pl->n_bins;
    a.crop_lo = pl->crop_lo;
    a.crop_hi = pl->crop_hi;
    a.accumulate = accumulate ? 1 : 0;
    a.a1 = pl->a1;
    a.a1f = (float)pl->a1;
    // kappa = sign 2 pi beta_frac rounded to 22 significant bits, so that
    // kappa * 1.5 * 2^23 is exact in FP32 (the kernel's fractional-phase step
    // relies on it); the relative change is below 2.4e-7.
    int ex = 0;
    const double mant = std::frexp(pl->sign * 2.0 * kPi * pl->beta_frac, &ex);
    const float kap = (float)std::ldexp(std::nearbyint(std::ldexp(mant, 22)), ex - 22);
    a.kappa = kap;
    a.kappa_magic = (float)((double)kap * 12582912.0);
    a.beta = (float)pl->beta_frac;
    a.sign = (float)pl->sign;
    const double cb = -pl->sign * 2.0 * kPi * (pl->beta_frac - std::floor(pl->beta_frac));
    a.cb_k = make_float2((float)(std::cos(cb) / kap), (float)(std::sin(cb) / kap));
    a.inv_kappa = (float)(1.0 / kap);
    a.fd_max = pl->fd_max;
    a.div_nq = ((1ull << 32) + (unsigned)(pl->L / 4) - 1) / (unsigned)(pl->L / 4);
    a.div_r = ((1ull << 32) + (unsigned)pl->p.n_rx - 1) / (unsigned)pl->p.n_rx;
    a.fp16 = pl->fp16 ? 1 : 0;
    a.rg = pl->rg;
    return a;
}

// Persistent grid and split-tile slots of one launch over `slots` partial
// sums.  Returns false when the decomposition needs more slots.
bool set_launch(const sar_plan *pl, BpArgs &a, float2 *partial, size_t slots) {
    a.G = (int)std::min<long long>(pl->G, a.units);
    const long long per = (a.units + a.G - 1) / a.G;
    a.seg_max = (int)((per - 1) / a.blocks_per_tile) + 2;
    a.partial = partial;
    return (size_t)a.G * (size_t)a.seg_max <= slots;
}

int bp_launch(sar_plan *pl, const void *prof, int M, const double *q_tx, const double *q_rx, const float *fd,
              void *image, int accumulate, cudaStream_t s, int m0 = 0, int M_tot = 0,
              void *image_out = nullptr) {
    BpArgs a = common_bp_args(pl, prof, M, q_tx, q_rx, fd, image, accumulate, m0, M_tot);
    a.image_out = (float2 *)image_out;
    if (!set_launch(pl, a, pl->d_partial, pl->partial_slots)) return SAR_EINVAL;  // cannot happen
    BpLaunch l{pl->rg, pl->fp16, pl->bp_smem, pl->minb};
    DeviceGuard dg(pl->device);
    if (!dg.ok) return SAR_ECUDA;
    return launch_backproject(a, l, s) == cudaSuccess ? SAR_OK : SAR_ECUDA;
}

}  // namespace

namespace sar {

int plan_device(const sar_plan *pl) { return pl->device; }

bool fill_rc_split(const sar_plan *pl, const void *beat, int M, const float *w_az, void *prof, RcSplitArgs *out,
                   int *sign, int *mode) {
    if (!pl->rc_split) return false;
    *mode = pl->fp16 ? kRcProfileF16 : kRcProfileF32;
    *sign = pl->sign;
    split_args(pl, rc_args(pl, beat, 0, M, M, w_az, prof, *mode), out);
    return true;
}

// Kernel arguments of one backprojection request (no scratch; the batched
// form supplies its own).
int fill_bp_args(const sar_plan *pl, const void *prof, int M, const double *q_tx, const double *q_rx,
                 void *image, int accumulate, BpArgs *out, size_t *smem) {
    if (!pl || !prof || !q_tx || !q_rx || !image || M < 1 || M > pl->p.max_pulses) return SAR_EINVAL;
    if (!aligned(prof, 256) || !aligned(q_tx, 16) || !aligned(q_rx, 16) || !aligned(image, 8)) return SAR_EINVAL;
    *out = common_bp_args(pl, prof, M, q_tx, q_rx, nullptr, image, accumulate);
    *smem = pl->bp_smem;
    return SAR_OK;
}

// The launch of sar_backproject with the split-tile partial sums in
// `scratch` (scratch_bytes long) instead of the plan's own buffer.  Returns
// SAR_ESCRATCH when this call's decomposition needs more than scratch_bytes.
int backproject_with_scratch(sar_plan *pl, const void *prof, int M, const double *q_tx, const double *q_rx,
                             const float *fd, void *image, int accumulate, float2 *scratch, size_t scratch_bytes,
                             cudaStream_t s) {
    if (!pl || M < 1 || M > pl->p.max_pulses) return SAR_EINVAL;
    if (fd && !(pl->fd_max > 0)) return SAR_EINVAL;
    BpArgs a = common_bp_args(pl, prof, M, q_tx, q_rx, fd, image, accumulate);
    if (!set_launch(pl, a, scratch, scratch_bytes / (kTilePx * sizeof(float2)))) return SAR_ESCRATCH;
    BpLaunch l{pl->rg, pl->fp16, pl->bp_smem, pl->minb};
    DeviceGuard dg(pl->device);
    if (!dg.ok) return SAR_ECUDA;
    return launch_backproject(a, l, s) == cudaSuccess ? SAR_OK : SAR_ECUDA;
}

}  // namespace sar

extern "C" {

int sar_version(void) { return 100; }

const char *sar_status_string(int st) {
    switch (st) {
        case SAR_OK: return "ok";
        case SAR_EINVAL: return "invalid argument";
        case SAR_ENOMEM: return "out of device memory or HBM budget";
        case SAR_EAGAIN: return "not ready";
        case SAR_ETIMEOUT: return "timed out";
        case SAR_ECUDA: return "CUDA error";
        case SAR_EBOUNDS: return "invalid geometry skipped";
        case SAR_ENOTFOUND: return "unknown ticket";
        case SAR_ESCRATCH: return "work needs more than the 16 MiB static scratch of sar_backproject_noalloc";
        default: return "unknown status";
    }
}

int sar_plan_create(const sar_radar_params *params, const sar_grid *grid, size_t hbm_budget_bytes,
                    sar_plan **out) {
    if (!out) return SAR_EINVAL;
    *out = nullptr;
    try {
        return plan_create(params, grid, hbm_budget_bytes, out);
    } catch (const std::bad_alloc &) {
        return SAR_ENOMEM;
    } catch (...) {
        return SAR_EINVAL;
    }
}

void sar_plan_destroy(sar_plan *plan) { free_plan(plan); }

int sar_plan_get_info(const sar_plan *pl, sar_plan_info *info) {
    if (!pl || !info) return SAR_EINVAL;
    sar_plan_info i{};
    i.n_fft = pl->n_fft;
    i.n_bins = pl->n_bins;
    i.crop_lo = pl->crop_lo;
    i.crop_hi = pl->crop_hi;
    i.n_pixels = pl->n_pixels;
    i.n_tiles = pl->n_tiles;
    i.window_bins = pl->L;
    i.pulses_per_block = pl->Mb;
    i.bp_ctas = pl->G;
    i.bins_per_metre = pl->a1;
    i.cycles_per_bin = pl->beta;
    i.device_bytes = pl->used;
    i.rx_group = pl->rg;
    i.regs_ctas_per_sm = pl->minb;
    i.tile_w = pl->tile_w;
    i.tile_h = pl->tile_w ? kTilePx / pl->tile_w : 0;
    *info = i;
    return SAR_OK;
}

int sar_profile_bytes(const sar_plan *pl, int32_t M, size_t *bytes) {
    if (!pl || !bytes || M < 1 || M > pl->p.max_pulses) return SAR_EINVAL;
    *bytes = profile_bytes(pl, M);
    return SAR_OK;
}

int sar_range_compress(sar_plan *pl, const void *beat_dev, int32_t M, const float *w_az_dev, void *prof_dev,
                       void *stream) {
    if (!pl || !beat_dev || !prof_dev || M < 1 || M > pl->p.max_pulses) return SAR_EINVAL;
    if (!aligned(beat_dev, 8) || !aligned(prof_dev, 256) || (w_az_dev && !aligned(w_az_dev, 4))) return SAR_EINVAL;
    return rc_launch(pl, beat_dev, M, w_az_dev, prof_dev, pl->fp16 ? kRcProfileF16 : kRcProfileF32,
                     (cudaStream_t)stream);
}

int sar_range_spectrum(sar_plan *pl, const void *beat_dev, int32_t M, void *spec_dev, void *stream) {
    if (!pl || !beat_dev || !spec_dev || M < 1 || M > pl->p.max_pulses) return SAR_EINVAL;
    if (!aligned(beat_dev, 8) || !aligned(spec_dev, 8)) return SAR_EINVAL;
    return rc_launch(pl, beat_dev, M, nullptr, spec_dev, kRcSpectrum, (cudaStream_t)stream);
}

int sar_backproject(sar_plan *pl, const void *prof_dev, int32_t M, const double *q_tx_dev,
                    const double *q_rx_dev, const float *fdopp_idx_dev, void *image_dev, int32_t accumulate,
                    void *stream) {
    if (!pl || !prof_dev || !q_tx_dev || !q_rx_dev || !image_dev || M < 1 || M > pl->p.max_pulses)
        return SAR_EINVAL;
    if (!aligned(prof_dev, 256) || !aligned(q_tx_dev, 16) || !aligned(q_rx_dev, 16) || !aligned(image_dev, 8) ||
        (fdopp_idx_dev && !aligned(fdopp_idx_dev, 4)))
        return SAR_EINVAL;
    if (fdopp_idx_dev && !(pl->fd_max > 0)) return SAR_EINVAL;
    return bp_launch(pl, prof_dev, M, q_tx_dev, q_rx_dev, fdopp_idx_dev, image_dev, accumulate,
                     (cudaStream_t)stream);
}

int sar_doppler_offsets(sar_plan *pl, const double *q_tx_dev, const double *q_rx_dev, const double *vel_dev,
                        int32_t M, float *fdopp_idx_dev, void *stream) {
    if (!pl || !q_tx_dev || !q_rx_dev || !vel_dev || !fdopp_idx_dev || M < 1 || M > pl->p.max_pulses)
        return SAR_EINVAL;
    if (!aligned(q_tx_dev, 8) || !aligned(q_rx_dev, 8) || !aligned(vel_dev, 8) || !aligned(fdopp_idx_dev, 4))
        return SAR_EINVAL;
    DopplerArgs a{};
    a.q_tx = q_tx_dev;
    a.q_rx = q_rx_dev;
    a.vel = vel_dev;
    a.M = M;
    a.R = pl->p.n_rx;
    a.tiles = pl->d_tiles;
    a.pix = pl->d_pix;
    a.out_idx = pl->d_out;
    a.n_tiles = pl->n_tiles;
    a.means = pl->d_means;
    // f0 at the transform's time origin (the carrier the phase correction uses)
    const double f0 = pl->beta_frac * pl->p.c * pl->a1;
    a.scale = f0 / pl->p.c * (double)pl->n_fft / pl->p.fs;
    a.fd = fdopp_idx_dev;
    DeviceGuard dg(pl->device);
    if (!dg.ok) return SAR_ECUDA;
    return launch_doppler_offsets(a, (cudaStream_t)stream) == cudaSuccess ? SAR_OK : SAR_ECUDA;
}

int sar_form_image_host(sar_plan *pl, const void *beat_host, int32_t M, const float *w_az_host,
                        const double *q_tx_host, const double *q_rx_host, void *image_host, void *stream) {
    if (!pl || !beat_host || !q_tx_host || !q_rx_host || !image_host || M < 1 || M > pl->p.max_pulses)
        return SAR_EINVAL;
    DeviceGuard dg(pl->device);
    if (!dg.ok) return SAR_ECUDA;
    const int R = pl->p.n_rx, N = pl->p.n_samples, Mc = pl->p.max_pulses;
    int rc = SAR_OK;
    if (!pl->s_beat) {
        void *q;
        rc = dev_alloc(pl, (size_t)Mc * R * N * 8, &q);
        if (!rc) pl->s_beat = q;
        if (!rc) rc = dev_alloc(pl, (size_t)Mc * 4, &q), pl->s_waz = (float *)q;
        if (!rc) rc = dev_alloc(pl, (size_t)Mc * 16, &q), pl->s_qtx = (double *)q;
        if (!rc) rc = dev_alloc(pl, (size_t)Mc * R * 16, &q), pl->s_qrx = (double *)q;
        if (!rc) rc = dev_alloc(pl, profile_bytes(pl, Mc), &q), pl->s_prof = q;
        if (!rc) rc = dev_alloc(pl, (size_t)pl->n_pixels * 8, &q), pl->s_img = q;
        if (rc) {
            pl->s_beat = nullptr;  // partially allocated buffers stay owned by the plan
            return rc;
        }
    }
    if (!pl->s_copy) {
        if (cudaStreamCreateWithFlags(&pl->s_copy, cudaStreamNonBlocking) != cudaSuccess) {
            pl->s_copy = nullptr;
            return SAR_ECUDA;
        }
        for (cudaEvent_t *e : {&pl->ev_start, &pl->ev_chunk[0], &pl->ev_chunk[1], &pl->ev_traj})
            if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) return SAR_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // Two-chunk pipeline.  The copy stream uploads w_sar and the first chunk
    // of chirps (whole pulse blocks), then the trajectory, then the rest; the
    // caller's stream range-compresses the first chunk while the trajectory
    // is in flight, backprojects it while the rest is, then the rest
    // (accumulating into the image).  The first chunk is the smallest whose
    // backprojection should outlast the upload of the rest, from a model of
    // the kernel's update rate (~1.3e12 updates/s) and of pinned host-to-device
    // bandwidth (~200 GB/s): only its upload is exposed.  Frames whose whole
    // upload takes less than ~40 us are not split (a second range compression
    // and backprojection launch would cost about as much).
    const size_t row_bytes = (size_t)R * N * 8;
    const double t_bp = (double)pl->n_pixels * R / 1.3e12, t_up = (double)row_bytes / 2.0e11;
    int cut = (int)std::ceil(M * t_up / (t_bp + t_up) / pl->Mb) * pl->Mb;
    cut = std::max(cut, pl->Mb);
    if (cut >= M || M * t_up < 4.0e-5) cut = M;
    const int bounds[3] = {0, cut, M};
    const int n_chunks = cut < M ? 2 : 1;
    bool ok = cudaEventRecord(pl->ev_start, s) == cudaSuccess &&
              cudaStreamWaitEvent(pl->s_copy, pl->ev_start, 0) == cudaSuccess;
    if (w_az_host)
        ok = ok &&
             cudaMemcpyAsync(pl->s_waz, w_az_host, (size_t)M * 4, cudaMemcpyHostToDevice, pl->s_copy) == cudaSuccess;
    for (int c = 0; c < n_chunks && ok; ++c) {
        const size_t off = (size_t)bounds[c] * row_bytes, bytes = (size_t)(bounds[c + 1] - bounds[c]) * row_bytes;
        ok = cudaMemcpyAsync((unsigned char *)pl->s_beat + off, (const unsigned char *)beat_host + off, bytes,
                             cudaMemcpyHostToDevice, pl->s_copy) == cudaSuccess &&
             cudaEventRecord(pl->ev_chunk[c], pl->s_copy) == cudaSuccess;
        if (c == 0) {
            ok = ok &&
                 cudaMemcpyAsync(pl->s_qtx, q_tx_host, (size_t)M * 16, cudaMemcpyHostToDevice, pl->s_copy) ==
                     cudaSuccess &&
                 cudaMemcpyAsync(pl->s_qrx, q_rx_host, (size_t)M * R * 16, cudaMemcpyHostToDevice, pl->s_copy) ==
                     cudaSuccess &&
                 cudaEventRecord(pl->ev_traj, pl->s_copy) == cudaSuccess;
        }
    }
    if (!ok) return SAR_ECUDA;
    // A page-locked, mapped image_host (e.g. cudaHostAlloc memory under
    // unified addressing) is written by the last chunk's kernels directly
    // (next to the device image), tile by tile while they run, instead of by
    // one copy after them.
    void *img_dev = nullptr;
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, image_host) == cudaSuccess) {
        if (pa.type == cudaMemoryTypeHost && pa.devicePointer && aligned(pa.devicePointer, 8)) img_dev = pa.devicePointer;
    } else {
        cudaGetLastError();
    }
    const int mode = pl->fp16 ? kRcProfileF16 : kRcProfileF32;
    for (int c = 0; c < n_chunks; ++c) {
        const int m0 = bounds[c], Mc = bounds[c + 1] - bounds[c];
        if (cudaStreamWaitEvent(s, pl->ev_chunk[c], 0) != cudaSuccess) return SAR_ECUDA;
        rc = rc_launch_part(pl, (const unsigned char *)pl->s_beat + (size_t)m0 * row_bytes, m0, Mc, M,
                            w_az_host ? pl->s_waz + m0 : nullptr, pl->s_prof, mode, s);
        if (rc) return rc;
        if (c == 0 && cudaStreamWaitEvent(s, pl->ev_traj, 0) != cudaSuccess) return SAR_ECUDA;
        rc = bp_launch(pl, pl->s_prof, Mc, pl->s_qtx + 2 * (size_t)m0, pl->s_qrx + 2 * (size_t)m0 * R, nullptr,
                       pl->s_img, c > 0, s, m0, M, c == n_chunks - 1 ? img_dev : nullptr);
        if (rc) return rc;
    }
    if (!img_dev &&
        cudaMemcpyAsync(image_host, pl->s_img, (size_t)pl->n_pixels * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SAR_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? SAR_OK : SAR_ECUDA;
}

int sar_batch_create(int32_t max_jobs, sar_batch **out) {
    if (!out || max_jobs < 1 || max_jobs > (1 << 20)) return SAR_EINVAL;
    *out = nullptr;
    sar_batch *b = new (std::nothrow) sar_batch();
    if (!b) return SAR_ENOMEM;
    b->max_jobs = max_jobs;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return SAR_ECUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, b->device) != cudaSuccess) {
        delete b;
        return SAR_ECUDA;
    }
    b->num_sms = prop.multiProcessorCount;
    b->g_cap = b->num_sms * 2;  // CTAs of one class's launch (two per SM)
    const size_t n_pref = (size_t)max_jobs + kBatchClasses;
    const size_t tb_off = sizeof(long long) * n_pref;
    b->jobs_off = (tb_off + sizeof(int) * n_pref + 15) & ~size_t(15);
    b->rc_off = (b->jobs_off + sizeof(BpArgs) * max_jobs + 15) & ~size_t(15);
    b->rc_jobs_off = (b->rc_off + sizeof(long long) * n_pref + 15) & ~size_t(15);
    const size_t blob = b->rc_jobs_off + sizeof(RcSplitArgs) * max_jobs;
    b->scratch_slots = (size_t)kBatchClasses * b->g_cap * 2;
    bool ok = cudaMallocHost((void **)&b->h_jobs, sizeof(BpArgs) * max_jobs) == cudaSuccess &&
              cudaMalloc((void **)&b->d_scratch, sizeof(float2) * kTilePx * b->scratch_slots) == cudaSuccess &&
              cudaMallocHost((void **)&b->h_blob, blob) == cudaSuccess &&
              cudaMalloc((void **)&b->d_blob, blob) == cudaSuccess &&

              cudaMalloc((void **)&b->d_err, sizeof(int) * 4) == cudaSuccess &&
              cudaMemset(b->d_err, 0, sizeof(int) * 4) == cudaSuccess &&

              cudaEventCreateWithFlags(&b->uploaded, cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
        b->h_ub = reinterpret_cast<long long *>(b->h_blob);
        b->h_tb = reinterpret_cast<int *>(b->h_blob + tb_off);
        b->h_sorted = reinterpret_cast<BpArgs *>(b->h_blob + b->jobs_off);
        b->d_ub = reinterpret_cast<long long *>(b->d_blob);
        b->d_tb = reinterpret_cast<int *>(b->d_blob + tb_off);
        b->d_jobs = reinterpret_cast<BpArgs *>(b->d_blob + b->jobs_off);
        b->h_rgb = reinterpret_cast<long long *>(b->h_blob + b->rc_off);
        b->d_rgb = reinterpret_cast<long long *>(b->d_blob + b->rc_off);
        b->h_rjobs = reinterpret_cast<RcSplitArgs *>(b->h_blob + b->rc_jobs_off);
        b->d_rjobs = reinterpret_cast<RcSplitArgs *>(b->d_blob + b->rc_jobs_off);
    }
    if (!ok) {
        cudaGetLastError();
        sar_batch_destroy(b);
        return SAR_ENOMEM;
    }
    *out = b;
    return SAR_OK;
}

void sar_batch_destroy(sar_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->h_jobs) cudaFreeHost(b->h_jobs);
    if (b->h_blob) cudaFreeHost(b->h_blob);
    if (b->d_blob) cudaFree(b->d_blob);
    if (b->d_scratch) cudaFree(b->d_scratch);
    if (b->d_err) cudaFree(b->d_err);

    if (b->uploaded) cudaEventDestroy(b->uploaded);
    delete b;
}

int sar_batch_clear(sar_batch *b) {
    if (!b) return SAR_EINVAL;
    // the host descriptor table may still be read by an upload in flight
    if (b->upload_pending && cudaEventSynchronize(b->uploaded) != cudaSuccess) return SAR_ECUDA;
    b->upload_pending = false;
    b->n_jobs = 0;
    b->units = 0;
    b->tiles = 0;
    b->n_classes = 0;
    b->rc.clear();
    b->n_rcc = 0;
    b->committed = false;
    return SAR_OK;
}

int sar_batch_add_frame(sar_batch *b, sar_plan *plan, const void *beat_dev, const float *w_az_dev, void *prof_dev,
                        int32_t M, const double *q_tx_dev, const double *q_rx_dev, void *image_dev,
                        int32_t accumulate) {
    if (!b || !plan || !beat_dev || !aligned(beat_dev, 8) || (w_az_dev && !aligned(w_az_dev, 4))) return SAR_EINVAL;
    const int rc = sar_batch_add(b, plan, prof_dev, M, q_tx_dev, q_rx_dev, image_dev, accumulate);
    if (rc) return rc;
    try {
        sar_batch::RcJob j;
        j.plan = plan;
        j.beat = beat_dev;
        j.w_az = w_az_dev;
        j.prof = prof_dev;
        j.M = M;
        j.mode = plan->fp16 ? kRcProfileF16 : kRcProfileF32;
        j.sign = plan->sign;
        j.split = fill_rc_split(plan, beat_dev, M, w_az_dev, prof_dev, &j.a, &j.sign, &j.mode);
        b->rc.push_back(j);
    } catch (...) {
        b->n_jobs -= 1;  // undo the backprojection request
        return SAR_ENOMEM;
    }
    return SAR_OK;
}

int sar_batch_add(sar_batch *b, sar_plan *plan, const void *prof_dev, int32_t M, const double *q_tx_dev,
                  const double *q_rx_dev, void *image_dev, int32_t accumulate) {
    if (!b || !plan) return SAR_EINVAL;
    if (b->n_jobs >= b->max_jobs || plan->device != b->device) return SAR_EINVAL;
    if (b->upload_pending) {
        if (cudaEventSynchronize(b->uploaded) != cudaSuccess) return SAR_ECUDA;
        b->upload_pending = false;
    }
    BpArgs a;
    size_t smem = 0;
    const int rc = fill_bp_args(plan, prof_dev, M, q_tx_dev, q_rx_dev, image_dev, accumulate, &a, &smem);
    if (rc) return rc;
    (void)smem;
    b->h_jobs[b->n_jobs] = a;
    b->units += a.units;
    b->tiles += a.n_tiles;
    b->n_jobs += 1;
    b->committed = false;
    return SAR_OK;
}

int sar_batch_commit(sar_batch *b, void *stream) {
    if (!b) return SAR_EINVAL;
    if (b->n_jobs == 0) {
        b->committed = true;
        return SAR_OK;
    }
    DeviceGuard dg(b->device);
    if (!dg.ok) return SAR_ECUDA;
    if (b->upload_pending) {  // the upload blob is about to be rewritten
        if (cudaEventSynchronize(b->uploaded) != cudaSuccess) return SAR_ECUDA;
        b->upload_pending = false;
    }
    // group the jobs by class, keeping their order within a class; apply the
    // class's block size (if set) to each job's unit decomposition
    int count[kBatchClasses] = {0};
    auto key = [](const BpArgs &a) { return (a.fp16 ? 4 : 0) + a.rg - 1; };
    for (int j = 0; j < b->n_jobs; ++j) ++count[key(b->h_jobs[j])];
    int fill[kBatchClasses];
    int cls_of_key[kBatchClasses];
    b->n_classes = 0;
    for (int k = 0, j0 = 0; k < kBatchClasses; ++k) {
        fill[k] = j0;
        cls_of_key[k] = -1;
        if (count[k]) {
            BatchClass &c = b->cls[b->n_classes];
            c = BatchClass{};
            c.rg = k % 4 + 1;
            c.fp16 = k >= 4;
            c.j0 = j0;
            c.n = count[k];
            c.off = j0 + b->n_classes;
            cls_of_key[k] = b->n_classes;
            ++b->n_classes;
        }
        j0 += count[k];
    }
    for (int j = 0; j < b->n_jobs; ++j) {
        BpArgs a = b->h_jobs[j];
        const int k = key(a);
        if (b->shape[k].mb > 0) {
            a.Mb = b->shape[k].mb;
            a.blocks_per_tile = (a.M + a.Mb - 1) / a.Mb;
            a.units = (long long)a.n_tiles * a.blocks_per_tile;
        }
        b->h_sorted[fill[k]++] = a;
    }
    // per-class prefix sums, shared memory and estimated time
    b->units = 0;
    b->tiles = 0;
    for (int ci = 0; ci < b->n_classes; ++ci) {
        BatchClass &c = b->cls[ci];
        for (int i = 0; i < c.n; ++i) {
            const BpArgs &a = b->h_sorted[c.j0 + i];
            b->h_ub[c.off + i] = c.units;
            b->h_tb[c.off + i] = c.tiles;
            c.units += a.units;
            c.tiles += a.n_tiles;
            c.updates += (double)a.n_tiles * kTilePx * a.M * a.R;
            c.smem = std::max(c.smem, bp_smem_bytes(a.Mb, a.R, a.L, c.fp16));
        }
        b->h_ub[c.off + c.n] = c.units;
        b->h_tb[c.off + c.n] = c.tiles;
        if (c.smem > kBpSmemMax) return SAR_EINVAL;
        b->units += c.units;
    }
    // the classes run one after another, each on the whole grid (two CTAs
    // per SM, stream-K over its units); each class has its own partial-sum
    // slots so that one fix-up after the last class serves all of them
    for (int ci = 0; ci < b->n_classes; ++ci) {
        BatchClass &c = b->cls[ci];
        const int k = (c.fp16 ? 4 : 0) + c.rg - 1;
        if (b->occ_smem[k] != c.smem || b->occ_ctas[k] < 1) {
            int occ = 0;
            const cudaError_t e = bp_batch_prepare(c.rg, c.fp16, c.smem, &occ);
            if (e == cudaErrorInvalidValue) {  // the class's shared memory exceeds what a CTA can have
                cudaGetLastError();
                return SAR_EINVAL;
            }
            if (e != cudaSuccess || occ < 1) {
                cudaGetLastError();
                return SAR_ECUDA;
            }
            b->occ_smem[k] = c.smem;
            b->occ_ctas[k] = occ;
        }
        c.G = (int)std::min<long long>(b->num_sms * std::min(b->occ_ctas[k], 2), c.units);
    }
    b->G = 0;
    int ctas = 0;
    for (int ci = 0; ci < b->n_classes; ++ci) {
        BatchClass &c = b->cls[ci];
        c.cta_begin = ctas;
        c.tile_base = b->tiles;
        ctas += c.G;
        b->G = std::max(b->G, c.G);
        b->tiles += c.tiles;
    }
    if ((size_t)ctas * 2 > b->scratch_slots) return SAR_EINVAL;  // sized for every class at creation
    // range-compression classes: split-kernel jobs of the same shape share a
    // launch; each job owns ceil(rows / rows per CTA group) row groups
    b->n_rcc = 0;
    {
        int placed = 0;
        std::vector<char> done(b->rc.size(), 0);
        for (size_t i = 0; i < b->rc.size(); ++i) {
            const sar_batch::RcJob &ji = b->rc[i];
            if (!ji.split || done[i] || b->n_rcc == kBatchClasses) continue;
            sar_batch::RcClass &c = b->rcc[b->n_rcc];
            c.a = ji.a;
            c.sign = ji.sign;
            c.mode = ji.mode;
            c.j0 = placed;
            c.n = 0;
            c.off = placed + b->n_rcc;
            c.groups = 0;
            const int rpc = kSplitThreads / (ji.a.N2 * ji.a.os);
            for (size_t q = i; q < b->rc.size(); ++q) {
                const sar_batch::RcJob &jq = b->rc[q];
                if (!jq.split || done[q] || jq.sign != ji.sign || jq.mode != ji.mode || jq.a.N2 != ji.a.N2 ||
                    jq.a.os != ji.a.os)
                    continue;
                done[q] = 1;
                b->h_rjobs[placed] = jq.a;
                b->h_rgb[c.off + c.n] = c.groups;
                c.groups += (jq.a.rows + rpc - 1) / rpc;
                ++c.n;
                ++placed;
            }
            b->h_rgb[c.off + c.n] = c.groups;
            ++b->n_rcc;
        }
        for (size_t i = 0; i < b->rc.size(); ++i) b->rc[i].split = b->rc[i].split && done[i];
    }
    (void)cls_of_key;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t up = b->rc.empty() ? b->jobs_off + sizeof(BpArgs) * b->n_jobs
                                    : b->rc_jobs_off + sizeof(RcSplitArgs) * b->rc.size();
    bool ok = cudaMemcpyAsync(b->d_blob, b->h_blob, up, cudaMemcpyHostToDevice, s) == cudaSuccess &&
              cudaEventRecord(b->uploaded, s) == cudaSuccess;
    if (!ok) return SAR_ECUDA;
    b->upload_pending = true;
    b->committed = true;
    return SAR_OK;
}

namespace {

// Kernel arguments of class ci of the committed batch, on G CTAs (0: its
// share) numbered from cta_begin, and of all classes for the fix-up.
BpClassArgs class_args(const sar_batch *b, int ci, int G, int cta_begin) {
    const BatchClass &c = b->cls[ci];
    BpClassArgs a{};
    a.jobs = b->d_jobs + c.j0;
    a.unit_begin = b->d_ub + c.off;
    a.tile_begin = b->d_tb + c.off;
    a.units = c.units;
    a.n_jobs = c.n;
    a.G = G > 0 ? (int)std::min<long long>(G, c.units) : c.G;
    a.cta_begin = cta_begin;
    a.tile_base = c.tile_base;
    a.rg = c.rg;
    a.fp16 = c.fp16 ? 1 : 0;
    return a;
}

BpCheck batch_check(const sar_batch *b, size_t smem) {
    BpCheck k{};
    k.scratch = b->d_scratch;
    k.scratch_slots = (long long)b->scratch_slots;
    k.smem_bytes = (unsigned)smem;
    k.err = b->d_err;
    return k;
}

// Class ci alone (autotuning), with its fix-up.
int batch_launch_class(const sar_batch *b, int ci, cudaStream_t s) {
    const BatchClass &c = b->cls[ci];
    const BpClassArgs a = class_args(b, ci, 0, c.cta_begin);
    BpMultiArgs m{};
    m.cls[0] = a;
    m.cls[0].tile_base = 0;
    m.n_classes = 1;
    const BpCheck chk = batch_check(b, c.smem);
    const int k = (c.fp16 ? 4 : 0) + c.rg - 1;
    const BpArgs *host_jobs = b->shape[k].param ? b->h_sorted + c.j0 : nullptr;
    if (launch_backproject_class(a, chk, c.smem, s, host_jobs) != cudaSuccess) return SAR_ECUDA;
    return launch_batch_fixup(m, chk, c.tiles, s) == cudaSuccess ? SAR_OK : SAR_ECUDA;
}

}  // namespace

int sar_batch_launch(sar_batch *b, void *stream) {
    if (!b || !b->committed) return SAR_EINVAL;
    if (b->n_jobs == 0) return SAR_OK;
    DeviceGuard dg(b->device);
    if (!dg.ok) return SAR_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // range compressions of frames added with sar_batch_add_frame: one launch
    // per class, and the general kernel for the other shapes
    for (int ci = 0; ci < b->n_rcc; ++ci) {
        const sar_batch::RcClass &c = b->rcc[ci];
        const RcSplitBatch tab{b->d_rjobs + c.j0, b->d_rgb + c.off, c.n};
        if (launch_range_compress_split(c.a, c.sign, c.mode, s, &tab, c.groups) != cudaSuccess) return SAR_ECUDA;
    }
    for (const sar_batch::RcJob &j : b->rc)
        if (!j.split) {
            const int rc = rc_launch(j.plan, j.beat, j.M, j.w_az, j.prof, j.mode, s);
            if (rc) return rc;
        }
    BpMultiArgs m{};
    m.n_classes = b->n_classes;
    size_t smem_max = 0;
    for (int ci = 0; ci < b->n_classes; ++ci) {
        m.cls[ci] = class_args(b, ci, 0, b->cls[ci].cta_begin);
        smem_max = std::max(smem_max, b->cls[ci].smem);
        const int k = (b->cls[ci].fp16 ? 4 : 0) + b->cls[ci].rg - 1;
        const BpArgs *host_jobs = b->shape[k].param ? b->h_sorted + b->cls[ci].j0 : nullptr;
        if (launch_backproject_class(m.cls[ci], batch_check(b, b->cls[ci].smem), b->cls[ci].smem, s, host_jobs) !=
            cudaSuccess)
            return SAR_ECUDA;
    }
    // one fix-up over the tiles of every class
    return launch_batch_fixup(m, batch_check(b, smem_max), b->tiles, s) == cudaSuccess ? SAR_OK : SAR_ECUDA;
}

}  // extern "C"

namespace sar {

// Append a sub-aperture request whose profile samples (and FP16 scales) start
// at the given rows; used by the server.  Same checks as sar_batch_add except
// the 256-byte alignment of the profile block (rows keep their sample
// alignment).
int batch_add_rows(sar_batch *b, sar_plan *plan, const void *samples, const float *scales, int32_t M,
                   const double *q_tx, const double *q_rx, void *image, int32_t accumulate, void *image_out) {
    if (!b || !plan || !samples || (plan->fp16 && !scales)) return SAR_EINVAL;
    if (b->n_jobs >= b->max_jobs || plan->device != b->device) return SAR_EINVAL;
    if (!q_tx || !q_rx || !image || M < 1 || M > plan->p.max_pulses) return SAR_EINVAL;
    if (b->upload_pending) {
        if (cudaEventSynchronize(b->uploaded) != cudaSuccess) return SAR_ECUDA;
        b->upload_pending = false;
    }
    BpArgs a;
    size_t smem = 0;
    // fill from a dummy aligned base, then point at the given rows
    int rc = fill_bp_args(plan, (const void *)256, M, q_tx, q_rx, image, accumulate, &a, &smem);
    if (rc) return rc;
    a.prof = samples;
    a.prof_scale = plan->fp16 ? scales : nullptr;
    a.image_out = (float2 *)image_out;
    (void)smem;
    b->h_jobs[b->n_jobs] = a;
    b->units += a.units;
    b->tiles += a.n_tiles;
    b->n_jobs += 1;
    b->committed = false;
    return SAR_OK;
}

int plan_geometry(const sar_plan *pl, int *n_rx, int *n_samples, int *n_bins, int *fp16, int64_t *n_pixels,
                  int *max_pulses) {
    if (!pl) return SAR_EINVAL;
    *n_rx = pl->p.n_rx;
    *n_samples = pl->p.n_samples;
    *n_bins = pl->n_bins;
    *fp16 = pl->fp16 ? 1 : 0;
    *n_pixels = pl->n_pixels;
    *max_pulses = pl->p.max_pulses;
    return SAR_OK;
}

}  // namespace sar

extern "C" {

int sar_batch_get_info(const sar_batch *b, int32_t *n_jobs, int64_t *units, int32_t *ctas) {
    if (!b) return SAR_EINVAL;
    if (n_jobs) *n_jobs = b->n_jobs;
    if (units) *units = b->units;
    if (ctas) *ctas = b->G;
    return SAR_OK;
}

int sar_batch_check_errors(sar_batch *b, int32_t *detail) {
    if (!b) return SAR_EINVAL;
    DeviceGuard dg(b->device);
    if (cudaDeviceSynchronize() != cudaSuccess) return SAR_ECUDA;
    int h[4] = {0, 0, 0, 0};
    if (cudaMemcpy(h, b->d_err, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return SAR_ECUDA;
    if (cudaMemset(b->d_err, 0, sizeof(h)) != cudaSuccess) return SAR_ECUDA;
    if (detail)
        for (int i = 0; i < 4; ++i) detail[i] = h[i];
    return h[0] ? SAR_EBOUNDS : SAR_OK;
}

int sar_batch_num_classes(const sar_batch *b, int32_t *n_classes) {
    if (!b || !n_classes) return SAR_EINVAL;
    *n_classes = b->committed ? b->n_classes : 0;
    return SAR_OK;
}

int sar_plan_autotune(sar_plan *pl, const void *prof_dev, int32_t M, const double *q_tx_dev,
                      const double *q_rx_dev, void *image_dev, void *stream) {
    if (!pl || !prof_dev || !q_tx_dev || !q_rx_dev || !image_dev || M < 1 || M > pl->p.max_pulses)
        return SAR_EINVAL;
    DeviceGuard dg(pl->device);
    if (!dg.ok) return SAR_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    struct Cfg {
        int tw, rg, minb, Mb;
    };
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SAR_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SAR_ECUDA;
    }
    const Cfg saved{pl->tile_w, pl->rg, pl->minb, pl->Mb};
    // best per tiling: the plan's tiling on entry (square tiles unless the
    // caller chose another) and the others; another tiling must be faster by
    // 2 % to be taken
    // (its longer staged windows cost every batch the plan joins: a batch
    // class sizes its pulse block for the longest window of its requests)
    constexpr float kTileMargin = 0.98f;
    float best = 1e30f, best_other = 1e30f;
    Cfg best_c = saved, best_other_c = saved;
    int rc = SAR_OK;
    // tile shapes (Cartesian grids), then per tiling the Rx group, register
    // budget and pulse block
    std::vector<int> tws{pl->tile_w};
    if (pl->tile_w)
        for (int tw : {32, 64, 16})
            if (tw != pl->tile_w) tws.push_back(tw);
    for (int tw : tws) {
        if (rc) break;
        if (tw != pl->tile_w && plan_retile(pl, tw) != SAR_OK) continue;  // does not fit: skip
        std::vector<Cfg> cands;
        const int R = pl->p.n_rx;
        const int rg0 = default_rx_group(R);
        int rg1 = 0;
        for (int g = rg0 - 1; g >= 1 && !rg1; --g)
            if (R % g == 0) rg1 = g;
        const size_t budgets[2] = {kBpSmemTarget, 73 * 1024};
        for (int rg : {rg0, rg1}) {
            if (rg < 1) continue;
            for (int minb = 2; minb <= 3; ++minb) {
                int mb_max = 0;
                for (int mb = kMaxPulsesPerBlock; mb >= 1; --mb)
                    if (bp_smem_bytes(mb, R, pl->L, pl->fp16) <= budgets[minb - 2]) {
                        mb_max = mb;
                        break;
                    }
                if (mb_max == 0) continue;
                for (int mb : {mb_max, std::max(1, (mb_max * 2) / 3), std::max(1, mb_max / 2)}) {
                    bool dup = false;
                    for (const Cfg &d : cands) dup |= (d.rg == rg && d.minb == minb && d.Mb == mb);
                    if (!dup) cands.push_back(Cfg{tw, rg, minb, mb});
                }
            }
        }
        for (const Cfg &c : cands) {
            if (apply_launch(pl, c.rg, c.minb, c.Mb) != SAR_OK) continue;  // does not fit: skip
            float times[3];
            for (int rep = -1; rep < 3 && rc == SAR_OK; ++rep) {
                if (rep >= 0 && cudaEventRecord(e0, s) != cudaSuccess) rc = SAR_ECUDA;
                if (!rc) rc = bp_launch(pl, prof_dev, M, q_tx_dev, q_rx_dev, nullptr, image_dev, 0, s);
                if (!rc && rep >= 0) {
                    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&times[rep], e0, e1) != cudaSuccess)
                        rc = SAR_ECUDA;
                }
            }
            if (rc) break;
            std::sort(times, times + 3);
            float &b = (c.tw == tws[0]) ? best : best_other;
            if (times[1] < b) {
                b = times[1];
                (c.tw == tws[0] ? best_c : best_other_c) = c;
            }
        }
    }
    if (best_other < kTileMargin * best) best_c = best_other_c;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const Cfg fin = rc ? saved : best_c;
    if ((fin.tw != pl->tile_w && plan_retile(pl, fin.tw) != SAR_OK) ||
        apply_launch(pl, fin.rg, fin.minb, fin.Mb) != SAR_OK)
        if (!rc) rc = SAR_ECUDA;
    if (!rc) remember_shape(pl);
    return rc;
}

int sar_batch_autotune(sar_batch *b, void *stream) {
    if (!b || !b->committed) return SAR_EINVAL;
    if (b->n_jobs == 0) return SAR_OK;
    DeviceGuard dg(b->device);
    if (!dg.ok) return SAR_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SAR_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SAR_ECUDA;
    }
    int rc = SAR_OK;
    // median of three timed launches after one untimed: class ci alone on
    // the whole grid of its storage's launch
    auto time_class = [&](int ci, float *ms) {
        float t[3] = {0, 0, 0};
        for (int rep = -1; rep < 3 && rc == SAR_OK; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess || batch_launch_class(b, ci, s) != SAR_OK ||
                cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = SAR_ECUDA;
                break;
            }
            if (rep >= 0 && cudaEventElapsedTime(&t[rep], e0, e1) != cudaSuccess) rc = SAR_ECUDA;
        }
        std::sort(t, t + 3);
        *ms = t[1];
    };
    ClassShape saved[kBatchClasses];
    std::copy(b->shape, b->shape + kBatchClasses, saved);
    for (int k = 0; k < kBatchClasses; ++k) b->shape[k] = ClassShape{};
    rc = sar_batch_commit(b, stream);
    for (int ci = 0; ci < b->n_classes && rc == SAR_OK; ++ci) {
        const BatchClass c0 = b->cls[ci];
        const int k = (c0.fp16 ? 4 : 0) + c0.rg - 1;
        // largest block whose staging fits two CTAs per SM for every request
        // of the class
        int fit = 0;
        for (int mb = kMaxPulsesPerBlock; mb >= 1 && !fit; --mb) {
            bool ok = true;
            for (int i = 0; i < c0.n && ok; ++i) {
                const BpArgs &a = b->h_sorted[c0.j0 + i];
                ok = bp_smem_bytes(mb, a.R, a.L, c0.fp16) <= kBpSmemTarget;
            }
            if (ok) fit = mb;
        }
        const int cand[4] = {0, fit, std::max(1, fit * 2 / 3), std::max(1, fit / 2)};
        float t_best = 1e30f;
        int mb_best = 0;
        for (int q = 0; q < 4 && rc == SAR_OK; ++q) {
            if (q > 0 && (cand[q] == 0 || cand[q] == cand[q - 1])) continue;
            b->shape[k].mb = cand[q];
            rc = sar_batch_commit(b, stream);
            float t = 0;
            if (rc == SAR_OK) time_class(ci, &t);
            if (rc == SAR_OK && t < t_best) {
                t_best = t;
                mb_best = cand[q];
            }
        }
        b->shape[k].mb = mb_best;
        // then the job arguments' source at that block: kernel parameters
        // (the default) or the device table
        if (rc == SAR_OK && c0.n <= kParamJobs) {
            b->shape[k].param = false;
            rc = sar_batch_commit(b, stream);
            float t = 0;
            if (rc == SAR_OK) time_class(ci, &t);
            if (rc == SAR_OK && t < t_best)
                t_best = t;
            else
                b->shape[k].param = true;
        }
        b->shape[k].ms = t_best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        std::copy(saved, saved + kBatchClasses, b->shape);
        sar_batch_commit(b, stream);
        return rc;
    }
    return sar_batch_commit(b, stream);
}

int sar_batch_get_class(const sar_batch *b, int32_t index, sar_batch_class *out) {
    if (!b || !out || index < 0 || index >= b->n_classes || !b->committed) return SAR_EINVAL;
    const BatchClass &c = b->cls[index];
    const int k = (c.fp16 ? 4 : 0) + c.rg - 1;
    sar_batch_class r{};
    r.rx_group = c.rg;
    r.fp16 = c.fp16 ? 1 : 0;
    r.n_jobs = c.n;
    r.pulses_per_block = b->shape[k].mb;
    r.ctas = c.G;
    r.regs_ctas_per_sm = 2;
    r.units = c.units;
    r.updates = c.updates;
    r.tuned_ms = b->shape[k].ms;
    r.param_args = (b->shape[k].param && c.n <= kParamJobs) ? 1 : 0;
    *out = r;
    return SAR_OK;
}

int sar_plan_set_launch(sar_plan *pl, int32_t rx_group, int32_t regs_ctas_per_sm, int32_t pulses_per_block) {
    if (!pl) return SAR_EINVAL;
    DeviceGuard dg(pl->device);
    if (!dg.ok) return SAR_ECUDA;
    return apply_launch(pl, rx_group, regs_ctas_per_sm, pulses_per_block);
}

int sar_plan_set_tile_shape(sar_plan *pl, int32_t tile_w) {
    if (!pl) return SAR_EINVAL;
    DeviceGuard dg(pl->device);
    if (!dg.ok) return SAR_ECUDA;
    try {
        return plan_retile(pl, tile_w);
    } catch (const std::bad_alloc &) {
        return SAR_ENOMEM;
    }
}

int sar_plan_check_errors(sar_plan *pl) {
    if (!pl) return SAR_EINVAL;
    DeviceGuard dg(pl->device);
    if (cudaDeviceSynchronize() != cudaSuccess) return SAR_ECUDA;
    int h[4] = {0, 0, 0, 0};
    if (cudaMemcpy(h, pl->d_err, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return SAR_ECUDA;
    if (cudaMemset(pl->d_err, 0, sizeof(h)) != cudaSuccess) return SAR_ECUDA;
    return h[0] ? SAR_EBOUNDS : SAR_OK;
}

}  // extern "C"
