// Per-pixel Doppler index offsets f_doppler(p) of Alg. 2 (paper Sec. III-D):
// the velocity terms of Alg. 1 (lines 5, 8, 9 and the f0 v / c part of line
// 11), evaluated once per reconstruction point from the average vehicle
// velocity over the chirp sequence instead of per (chirp, antenna):
//   vbar = mean_m vel(m),  qt = mean_m q_tx(m),  qr = mean_{m,n} q_rx(m, n),
//   f_doppler(p) = -(f0 / c) (<p - qt, vbar> / |p - qt| + <p - qr, vbar> / |p - qr|) N_fft / fs,
// the rate of change of the two-way path (a platform closing on p shortens
// it) times f0 / c, in bins of the range transform.
//
// Two kernels: one CTA reduces the means in FP64; then one thread per pixel
// slot of the plan's tiles (positions = FP64 tile reference + FP32 offset)
// writes its offset at the pixel's image index.  Both read device memory only
// (graph-capturable).
#include "sar_internal.h"

namespace sar {
namespace {

constexpr int kMeanThreads = 256;

// means[0..5] = (qt.x, qt.y, qr.x, qr.y, vbar.x, vbar.y)
__global__ void __launch_bounds__(kMeanThreads) doppler_means_kernel(const double *__restrict__ q_tx,
                                                                     const double *__restrict__ q_rx,
                                                                     const double *__restrict__ vel, int M, int R,
                                                                     double *__restrict__ means) {
    __shared__ double part[6][kMeanThreads / 32];
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        s[0] += q_tx[2 * m];
        s[1] += q_tx[2 * m + 1];
        s[4] += vel[2 * m];
        s[5] += vel[2 * m + 1];
    }
    const long long nr = (long long)M * R;
    for (long long i = threadIdx.x; i < nr; i += blockDim.x) {
        s[2] += q_rx[2 * i];
        s[3] += q_rx[2 * i + 1];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        double v = s[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) part[c][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = 0;
        for (int w = 0; w < kMeanThreads / 32; ++w) v += part[threadIdx.x][w];
        const int c = threadIdx.x;
        means[c] = v / ((c == 2 || c == 3) ? (double)nr : (double)M);
    }
}

__global__ void __launch_bounds__(256) doppler_offsets_kernel(const TileInfo *__restrict__ tiles,
                                                               const float2 *__restrict__ pix,
                                                               const int *__restrict__ out_idx, long long slots,
                                                               const double *__restrict__ means, double scale,
                                                               float *__restrict__ fd) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= slots) return;
    const int o = out_idx[s];
    if (o < 0) return;
    const TileInfo ti = tiles[s / kTilePx];
    const float2 d = pix[s];
    const double x = ti.x + (double)d.x, y = ti.y + (double)d.y;
    const double ex = x - means[0], ey = y - means[1];
    const double gx = x - means[2], gy = y - means[3];
    const double vx = means[4], vy = means[5];
    // a pixel on an antenna's mean position has no radial direction: 0 there
    const double nt = hypot(ex, ey), nr = hypot(gx, gy);
    const double v_tx = nt > 0 ? (ex * vx + ey * vy) / nt : 0.0;
    const double v_rx = nr > 0 ? (gx * vx + gy * vy) / nr : 0.0;
    fd[o] = (float)(-(v_tx + v_rx) * scale);
}

}  // namespace

cudaError_t launch_doppler_offsets(const DopplerArgs &a, cudaStream_t s) {
    doppler_means_kernel<<<1, kMeanThreads, 0, s>>>(a.q_tx, a.q_rx, a.vel, a.M, a.R, a.means);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long slots = (long long)a.n_tiles * kTilePx;
    if (slots == 0) return cudaSuccess;
    doppler_offsets_kernel<<<(unsigned)((slots + 255) / 256), 256, 0, s>>>(a.tiles, a.pix, a.out_idx, slots,
                                                                            a.means, a.scale, a.fd);
    return cudaGetLastError();
}

}  // namespace sar
