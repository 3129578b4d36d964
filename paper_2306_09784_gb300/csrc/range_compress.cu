// Range compression: window, zero-padded range transform and profile store
// for every (chirp, Rx) row of the FMCW beat cube.
//
// The paper interpolates the beat spectrum on an equidistant beat-frequency
// axis (s(f_hyp) in Alg. 1, s(f_ind) in Alg. 2, Sec. III-C) but does not say how it is
// produced; here it is the windowed, zero-padded DFT of each chirp,
//     S[k] = sum_{n<N} w_r[n] beat[n] exp(sign j 2 pi n k / N_fft).
//
// One CTA transforms 4096 / N_fft rows (one row when N_fft >= 4096) in shared
// memory.  Each thread keeps 16 values in registers; log2(N_fft) / 4 radix-16
// Stockham passes (plus one radix-2/4/8 pass for the remainder) exchange
// through one shared buffer.  The first pass reads the beat samples straight
// from global memory with the range window fused into the load (zero padding
// costs no loads).  The store stage folds w_sar[m] and the per-bin phase
// rotation into the profile (see sar.h) and writes only the cropped bins.
#include <cuda_fp16.h>

#include <algorithm>

#include "sar_internal.h"

namespace sar {
namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// exp(SGN j 2 pi t / 16), t in [0, 8): exact values of cos/sin at multiples of pi/8.
template <int SGN>
__device__ __forceinline__ float2 w16(int t) {
    constexpr float c1 = 0.923879532511286756f;  // cos(pi/8)
    constexpr float s1 = 0.382683432365089772f;  // sin(pi/8)
    constexpr float h = 0.707106781186547524f;   // cos(pi/4)
    float c, s;
    switch (t) {
        case 0: c = 1.f; s = 0.f; break;
        case 1: c = c1; s = s1; break;
        case 2: c = h; s = h; break;
        case 3: c = s1; s = c1; break;
        case 4: c = 0.f; s = 1.f; break;
        case 5: c = -s1; s = c1; break;
        case 6: c = -h; s = h; break;
        default: c = -c1; s = s1; break;
    }
    return make_float2(c, SGN > 0 ? s : -s);
}

template <int SGN>
__device__ __forceinline__ float2 twiddle_const(float2 v, int t) {
    if (t == 0) return v;
    if (t == 4) return SGN > 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    return cmul(v, w16<SGN>(t));
}

__host__ __device__ constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// Shared-memory index with one spare element after every 16: the
// stride-16 stores of the first passes then spread over all banks.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

template <int RAD>
__host__ __device__ constexpr int ilog2(int) {
    return RAD == 2 ? 1 : RAD == 4 ? 2 : RAD == 8 ? 3 : 4;
}

// In-register DFT of RAD points, v[k] <- sum_n v[n] exp(SGN j 2 pi n k / RAD),
// natural order in and out (radix-2 decimation in time).  ZR < RAD: only
// v[0..ZR) may be nonzero.  After the bit reversal those sit at multiples of
// RAD / ZR, and the first log2(RAD / ZR) butterfly stages pair each of them
// with zeros only, which copies it across its block: those stages become
// register copies.
template <int RAD, int SGN, int ZR = RAD>
__device__ __forceinline__ void dft_reg(float2 *v) {
    constexpr int bits = ilog2<RAD>(0);
    constexpr int H0 = RAD / ZR;
#pragma unroll
    for (int i = 0; i < RAD; ++i) {
        const int j = bitrev(i, bits);
        if (i < j) {
            float2 t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
    if (H0 > 1) {
#pragma unroll
        for (int p = 0; p < RAD; p += H0)
#pragma unroll
            for (int i = 1; i < H0; ++i) v[p + i] = v[p];
    }
#pragma unroll
    for (int h = H0; h < RAD; h <<= 1) {
#pragma unroll
        for (int s = 0; s < RAD; s += 2 * h) {
#pragma unroll
            for (int t = 0; t < h; ++t) {
                const float2 a = v[s + t];
                const float2 b = twiddle_const<SGN>(v[s + t + h], t * (8 / h));
                v[s + t] = cadd(a, b);
                v[s + t + h] = csub(a, b);
            }
        }
    }
}

// One Stockham pass of radix RAD over an n-point row held in shared memory X
// (Ns = product of the radices of the earlier passes).  Each of the T = n/16
// threads of the row owns 16 values: 16/RAD butterflies j = tid + g T.
// FIRST: the pass reads the windowed beat samples from global memory.
// STAGED: the beat row, the window and the twiddles are in shared memory;
// there tw is this pass's own table: for each power 2^i < RAD the Ns
// twiddles exp(SGN j 2 pi k 2^i / (Ns RAD)), k < Ns (consecutive threads read
// consecutive entries).  Otherwise tw is the full N_fft-point table.
// ZR (first pass): N_fft / N = 16 / ZR, so only the first ZR of a thread's
// 16 inputs lie inside the chirp; the rest are the zero padding.
template <int RAD, int SGN, bool FIRST, bool STAGED = false, int ZR = RAD>
__device__ __forceinline__ void stockham_pass(float2 *X, int n, int log2n, int Ns, int tid, int T,
                                              bool active, const float2 *__restrict__ tw,
                                              const float2 *__restrict__ beat_row,
                                              const float *__restrict__ w_r, int N) {
    constexpr int G = 16 / RAD;
    const int stride = n / RAD;
    float2 v[16];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = tid + g * T;
#pragma unroll
        for (int r = 0; r < RAD; ++r) {
            const int idx = j + r * stride;
            if (FIRST) {
                float2 x = make_float2(0.f, 0.f);
                if (active && r < ZR && (ZR < RAD || idx < N)) {
                    const float2 b = STAGED ? beat_row[idx] : __ldg(beat_row + idx);
                    const float w = STAGED ? w_r[idx] : __ldg(w_r + idx);
                    x = make_float2(w * b.x, w * b.y);
                }
                v[g * RAD + r] = x;
            } else {
                v[g * RAD + r] = X[pad16(idx)];
            }
        }
    }
    if (!FIRST) __syncthreads();
    // log2(n / (Ns * RAD)): shift from the twiddle exponent k r to the table index
    const int tw_shift = log2n - (31 - __clz(Ns)) - ilog2<RAD>(0);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int j = tid + g * T;
        const int k = j & (Ns - 1);
        if (Ns > 1) {
            // w^r for r < RAD from the loaded powers w, w^2, w^4, w^8 (at most
            // three complex products deep: ~4e-7 relative error)
            float2 wp[16];
            if (STAGED) {
                wp[1] = tw[k];
                if (RAD > 2) wp[2] = tw[Ns + k];
                if (RAD > 4) wp[4] = tw[2 * Ns + k];
                if (RAD > 8) wp[8] = tw[3 * Ns + k];
            } else {
                const int t1 = k << tw_shift;
                wp[1] = __ldg(tw + t1);
                if (RAD > 2) wp[2] = __ldg(tw + 2 * t1);
                if (RAD > 4) wp[4] = __ldg(tw + 4 * t1);
                if (RAD > 8) wp[8] = __ldg(tw + 8 * t1);
            }
            if (RAD > 2) wp[3] = cmul(wp[1], wp[2]);
            if (RAD > 4) {
                wp[5] = cmul(wp[4], wp[1]);
                wp[6] = cmul(wp[4], wp[2]);
                wp[7] = cmul(wp[4], wp[3]);
            }
            if (RAD > 8) {
#pragma unroll
                for (int r = 9; r < 16; ++r) wp[r] = cmul(wp[8], wp[r - 8]);
            }
#pragma unroll
            for (int r = 1; r < RAD; ++r) v[g * RAD + r] = cmul(v[g * RAD + r], wp[r]);
        }
        dft_reg<RAD, SGN, FIRST ? ZR : RAD>(v + g * RAD);
        const int base = (j - k) * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) X[pad16(base + r * Ns)] = v[g * RAD + r];
    }
    __syncthreads();
}

// BIG: N_fft of 8192 or 16384 (512 or 1024 threads per row); otherwise at
// most 256 threads per CTA and registers to spare for the 16 values in flight.
template <int SGN, int MODE, bool BIG>
__global__ void __launch_bounds__(BIG ? 1024 : 256, BIG ? 1 : 3) range_compress_kernel(RcArgs a) {
    extern __shared__ float2 smem_rc[];
    __shared__ int row_max[64];  // rows per CTA <= 4096 / 64
    const int n = a.n_fft;
    const int T = n >> 4;
    const int rows_per_cta = blockDim.x / T;
    const int lrow = threadIdx.x / T;
    const int tid = threadIdx.x - lrow * T;
    const long long row = (long long)blockIdx.x * rows_per_cta + lrow;
    const bool active = row < a.rows;
    float2 *X = smem_rc + (size_t)lrow * (n + n / 16);
    const float2 *beat_row = a.beat + (active ? row : 0) * (long long)a.N;

    if (MODE == kRcProfileF16 && threadIdx.x < 64) row_max[threadIdx.x] = 0;

    // radix-16 passes, then the remainder radix
    const int n16 = a.log2n >> 2;
    const int rem = a.log2n & 3;
    int Ns = 1;
    for (int p = 0; p < n16; ++p) {
        if (p == 0)
            stockham_pass<16, SGN, true>(X, n, a.log2n, Ns, tid, T, active, a.tw, beat_row, a.w_r, a.N);
        else
            stockham_pass<16, SGN, false>(X, n, a.log2n, Ns, tid, T, active, a.tw, beat_row, a.w_r, a.N);
        Ns <<= 4;
    }
    if (rem == 1) stockham_pass<2, SGN, false>(X, n, a.log2n, Ns, tid, T, active, a.tw, beat_row, a.w_r, a.N);
    if (rem == 2) stockham_pass<4, SGN, false>(X, n, a.log2n, Ns, tid, T, active, a.tw, beat_row, a.w_r, a.N);
    if (rem == 3) stockham_pass<8, SGN, false>(X, n, a.log2n, Ns, tid, T, active, a.tw, beat_row, a.w_r, a.N);

    if (MODE == kRcSpectrum) {
        if (!active) return;
        float2 *out = reinterpret_cast<float2 *>(a.out) + row * (long long)n;
        for (int k = tid; k < n; k += T) out[k] = X[pad16(k)];
        return;
    }

    const float g = (a.w_az != nullptr && active) ? __ldg(a.w_az + row / a.R) : 1.f;
    if (MODE == kRcProfileF32) {
        if (!active) return;
        float2 *out = reinterpret_cast<float2 *>(a.out) + row * (long long)a.n_bins;
        for (int i = tid; i < a.n_bins; i += T) {
            const float2 v = cmul(X[pad16(a.crop_lo + i)], __ldg(a.rot + i));
            out[i] = make_float2(g * v.x, g * v.y);
        }
        return;
    }

    // FP16 profile: per-row max |component| sets the scale (max maps to 2^14)
    float mx = 0.f;
    if (active) {
        for (int i = tid; i < a.n_bins; i += T) {
            const float2 v = cmul(X[pad16(a.crop_lo + i)], __ldg(a.rot + i));
            mx = fmaxf(mx, fmaxf(fabsf(g * v.x), fabsf(g * v.y)));
        }
    }
    atomicMax(&row_max[lrow], __float_as_int(mx));
    __syncthreads();
    if (!active) return;
    const float rmax = __int_as_float(row_max[lrow]);
    const float scale = rmax > 0.f ? rmax * (1.0f / 16384.0f) : 1.0f;
    const float inv = 1.0f / scale;
    if (tid == 0) a.scales[row] = scale;
    __half2 *out = reinterpret_cast<__half2 *>(a.out) + row * (long long)a.n_bins;
    for (int i = tid; i < a.n_bins; i += T) {
        const float2 v = cmul(X[pad16(a.crop_lo + i)], __ldg(a.rot + i));
        out[i] = __floats2half2_rn(g * v.x * inv, g * v.y * inv);
    }
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}

// Output stage shared by both kernels: spectrum, FP32 profile or FP16
// profile (scale = row max / 2^14) of the row held in X.
template <int MODE>
__device__ __forceinline__ void store_row(const RcArgs &a, const float2 *X, long long row, bool active, int tid,
                                          int T, int lrow, int *row_max) {
    const int n = a.n_fft;
    if (MODE == kRcSpectrum) {
        if (!active) return;
        float2 *out = reinterpret_cast<float2 *>(a.out) + row * (long long)n;
        for (int k = tid; k < n; k += T) out[k] = X[pad16(k)];
        return;
    }
    const float g = (a.w_az != nullptr && active) ? __ldg(a.w_az + row / a.R) : 1.f;
    if (MODE == kRcProfileF32) {
        if (!active) return;
        float2 *out = reinterpret_cast<float2 *>(a.out) + row * (long long)a.n_bins;
        for (int i = tid; i < a.n_bins; i += T) {
            const float2 v = cmul(X[pad16(a.crop_lo + i)], __ldg(a.rot + i));
            out[i] = make_float2(g * v.x, g * v.y);
        }
        return;
    }
    float mx = 0.f;
    if (active) {
        for (int i = tid; i < a.n_bins; i += T) {
            const float2 v = cmul(X[pad16(a.crop_lo + i)], __ldg(a.rot + i));
            mx = fmaxf(mx, fmaxf(fabsf(g * v.x), fabsf(g * v.y)));
        }
    }
    atomicMax(&row_max[lrow], __float_as_int(mx));
    __syncthreads();
    if (!active) return;
    const float rmax = __int_as_float(row_max[lrow]);
    const float scale = rmax > 0.f ? rmax * (1.0f / 16384.0f) : 1.0f;
    const float inv = 1.0f / scale;
    if (tid == 0) a.scales[row] = scale;
    __half2 *out = reinterpret_cast<__half2 *>(a.out) + row * (long long)a.n_bins;
    for (int i = tid; i < a.n_bins; i += T) {
        const float2 v = cmul(X[pad16(a.crop_lo + i)], __ldg(a.rot + i));
        out[i] = __floats2half2_rn(g * v.x * inv, g * v.y * inv);
    }
}

// Start of the twiddle table of the pass with Ns = 16^q (q >= 1) in the
// per-pass tables of the persistent kernel: 4 (16 + 256 + ... + 16^(q-1)).
__host__ __device__ constexpr int pass_table_offset(int q) { return 4 * (((1 << (4 * q)) - 16) / 15); }

// Persistent form for N_fft <= 4096 (256 threads, 4096 / N_fft rows per
// group).  Per-pass twiddle tables and the window sit in shared memory for
// the CTA's lifetime; the beat samples of the next row group are copied in
// with cp.async while the current group is transformed.  LOGN > 0: N_fft =
// 2^LOGN fixed at compile time (index and twiddle arithmetic folds into
// constants); 0: any size.  ZR < 16: N_fft = 16 N / ZR, and the first pass
// skips the zero padding.
template <int SGN, int MODE, int LOGN, int ZR>
__global__ void __launch_bounds__(256, 2) range_compress_persistent(RcArgs a, long long n_groups) {
    extern __shared__ float2 smem_rcp[];
    __shared__ int row_max[64];
    const int n = LOGN ? (1 << LOGN) : a.n_fft, N = a.N;
    const int log2n = LOGN ? LOGN : a.log2n;
    const int T = n >> 4;
    const int rows_per = 256 / T;  // launched with 256 threads
    const int lrow = threadIdx.x / T;
    const int tid = threadIdx.x - lrow * T;
    float2 *X = smem_rcp + (size_t)lrow * (n + n / 16);
    float2 *tw = smem_rcp + (size_t)rows_per * (n + n / 16);
    float2 *stage = tw + n;  // [2][rows_per][N]
    float *wr = reinterpret_cast<float *>(stage + 2 * rows_per * N);
    // per-pass twiddle tables (at most N_fft / 2 entries): the pass with Ns
    // and radix RAD holds tw[(k << i) N_fft / (Ns RAD)] at i Ns + k
    {
        const int n16 = log2n >> 2, rem = log2n & 3;
        for (int q = 1; q <= n16; ++q) {
            const int lns = 4 * q, Ns = 1 << lns;
            const int lrad = q < n16 ? 4 : rem;
            if (lrad == 0) break;
            const int step = n >> (lns + lrad);
            float2 *dst = tw + pass_table_offset(q);
            for (int i = threadIdx.x; i < lrad * Ns; i += blockDim.x)
                dst[i] = __ldg(a.tw + (((i & (Ns - 1)) << (i >> lns)) * step));
        }
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) wr[i] = __ldg(a.w_r + i);
    const uint32_t stage_addr = (uint32_t)__cvta_generic_to_shared(stage);
    const int per_group = rows_per * N;

    // 16-byte copies of two samples when the beat cube is 16-byte aligned (N
    // is a power of two >= 4, so every row and the staging buffer are too);
    // 8-byte copies otherwise
    const bool a16 = (reinterpret_cast<uintptr_t>(a.beat) & 15u) == 0;
    auto issue = [&](long long g, int buf) {
        if (a16) {
            for (int e = 2 * threadIdx.x; e < per_group; e += 2 * blockDim.x) {
                const int lr = rows_per == 1 ? 0 : e / N;
                const int k = e - lr * N;
                const long long row = g * rows_per + lr;
                const bool ok = row < a.rows;
                const void *src = ok ? (const void *)(a.beat + row * (long long)N + k) : (const void *)a.beat;
                cp_async16(stage_addr + (uint32_t)(buf * per_group + e) * 8u, src, ok ? 16u : 0u);
            }
        } else {
            for (int i = threadIdx.x; i < per_group; i += blockDim.x) {
                const int lr = rows_per == 1 ? 0 : i / N;
                const int k = i - lr * N;
                const long long row = g * rows_per + lr;
                const bool ok = row < a.rows;
                const void *src = ok ? (const void *)(a.beat + row * (long long)N + k) : (const void *)a.beat;
                cp_async8(stage_addr + (uint32_t)(buf * per_group + i) * 8u, src, ok ? 8u : 0u);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    long long g = blockIdx.x;
    if (g < n_groups) issue(g, 0);
    for (int it = 0; g < n_groups; g += gridDim.x, ++it) {
        const long long gn = g + gridDim.x;
        if (gn < n_groups) {
            issue(gn, (it + 1) & 1);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        if (MODE == kRcProfileF16 && threadIdx.x < 64) row_max[threadIdx.x] = 0;
        __syncthreads();  // staged samples, twiddles and window visible
        const long long row = g * rows_per + lrow;
        const bool active = row < a.rows;
        const float2 *src = stage + (size_t)((it & 1) * rows_per + lrow) * N;
        const int n16 = log2n >> 2;
        const int rem = log2n & 3;
        stockham_pass<16, SGN, true, true, ZR>(X, n, log2n, 1, tid, T, active, tw, src, wr, N);
        if (LOGN) {
#pragma unroll
            for (int p = 1; p < (LOGN >> 2); ++p) {
                stockham_pass<16, SGN, false, true>(X, n, log2n, 1 << (4 * p), tid, T, active,
                                                    tw + pass_table_offset(p), src, wr, N);
            }
        } else {
            for (int p = 1; p < n16; ++p)
                stockham_pass<16, SGN, false, true>(X, n, log2n, 1 << (4 * p), tid, T, active,
                                                    tw + pass_table_offset(p), src, wr, N);
        }
        const int Ns = 1 << (4 * n16);
        const float2 *twr = tw + pass_table_offset(n16);
        if (rem == 1) stockham_pass<2, SGN, false, true>(X, n, log2n, Ns, tid, T, active, twr, src, wr, N);
        if (rem == 2) stockham_pass<4, SGN, false, true>(X, n, log2n, Ns, tid, T, active, twr, src, wr, N);
        if (rem == 3) stockham_pass<8, SGN, false, true>(X, n, log2n, Ns, tid, T, active, twr, src, wr, N);
        store_row<MODE>(a, X, row, active, tid, T, lrow, row_max);
        __syncthreads();  // X and this group's stage buffer are reused next
    }
}

// ---------------------------------------------------------------------------
// Split-transform kernel (the common case: N = 32 N2 samples, N2 in {8, 16,
// 32}, N2 os <= 256).  With bins k = os q + s (q < N, s < os) the
// zero-padded transform splits into os N-point transforms
//     S[os q + s] = sum_{n<N} (w_r[n] x[n] W^{n s}) W_N^{n q},  W = exp(SGN j 2 pi / N_fft),
// so the zero padding costs only the input rotations W^{n s} (a table with
// the window folded in).  One thread group of N2 threads runs each N-point
// transform as 32 x N2: a pass of 32-point DFTs over n1 (n = N2 n1 + j for
// thread j, 32 complex values in registers), the twiddles W_N^{j k1}, one
// exchange through shared memory inside the warp (XOR-swizzled, no CTA
// barrier) and a pass of N2-point DFTs.  Thread j then holds X[k1 + 32 k2]
// for its k1 = j (32 / N2) + i and all k2; only the cropped bins are rotated,
// scaled and stored.  Complex values are (re, im) float2: additions are single
// packed FP32 instructions.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as a fused multiply-add by -1 (exact, one instruction)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

// cos(k pi / 16), k = 0..16
__device__ __forceinline__ constexpr float cos_pi16(int k) {
    constexpr float t[17] = {1.0f,
                             0.98078528040323044913f,
                             0.92387953251128675613f,
                             0.83146961230254523708f,
                             0.70710678118654752440f,
                             0.55557023301960222474f,
                             0.38268343236508977173f,
                             0.19509032201612826785f,
                             0.0f,
                             -0.19509032201612826785f,
                             -0.38268343236508977173f,
                             -0.55557023301960222474f,
                             -0.70710678118654752440f,
                             -0.83146961230254523708f,
                             -0.92387953251128675613f,
                             -0.98078528040323044913f,
                             -1.0f};
    return t[k];
}

// One radix-2 butterfly of a decimation-in-time stage: a + w b, a - w b with
// w = exp(SGN j pi E / 16), E in [0, 16).  Quarter turns are swaps.
template <int SGN, int E>
__device__ __forceinline__ void bfly(float2 &a, float2 &b) {
    float2 wb = b;
    if (E == 8) {
        wb = SGN > 0 ? make_float2(-b.y, b.x) : make_float2(b.y, -b.x);
    } else if (E != 0) {
        constexpr float c = cos_pi16(E);
        constexpr float sn = (SGN > 0 ? 1.0f : -1.0f) * (E <= 8 ? cos_pi16(8 - E) : cos_pi16(E - 8));
        wb = make_float2(fmaf(b.x, c, -b.y * sn), fmaf(b.x, sn, b.y * c));
    }
    const float2 x = a;
    a = add2(x, wb);
    b = sub2(x, wb);
}

// Stage of span H of an R-point DIT transform (R <= 32): butterflies
// (s + t, s + t + H) with w = exp(SGN j 2 pi t / (2 H)) = exp(SGN j pi e / 16),
// e = t * 16 / H.
template <int R, int SGN, int H, int T = 0>
__device__ __forceinline__ void stage_t(float2 *v) {
    if constexpr (T < H) {
#pragma unroll
        for (int s = 0; s < R; s += 2 * H) bfly<SGN, T * 16 / H>(v[s + T], v[s + T + H]);
        stage_t<R, SGN, H, T + 1>(v);
    }
}

// In-register R-point DFT (R = 8, 16, 32), natural order in and out:
//   v[k] <- sum_n v[n] exp(SGN j 2 pi n k / R).
template <int R, int SGN>
__device__ __forceinline__ void dft_small(float2 *v) {
    constexpr int bits = R == 8 ? 3 : R == 16 ? 4 : 5;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int j = bitrev(i, bits);
        if (i < j) {
            const float2 t = v[i];
            v[i] = v[j];
            v[j] = t;
        }
    }
    stage_t<R, SGN, 1>(v);
    stage_t<R, SGN, 2>(v);
    stage_t<R, SGN, 4>(v);
    if constexpr (R >= 16) stage_t<R, SGN, 8>(v);
    if constexpr (R >= 32) stage_t<R, SGN, 16>(v);
}

// Exchange / output region per sub-transform: at least N + N2 float2 (the
// padded transpose layout needs N + N2 - 1; the outputs use the first N),
// rounded so that the stride is 16 / os modulo 16 elements: the output stage
// reads bins k, k + 1, ... from the os regions in turn (k mod os), and that
// stride puts the 16 lanes of a half-warp on 16 different bank pairs.
__host__ __device__ constexpr int split_region(int n2, int os) {
    const int base = 32 * n2 + n2;
    const int want = os >= 16 ? 1 : 16 / os;
    return base + (((want - base) % 16) + 16) % 16;
}

// Batched form: the job of the table whose row groups
// [group_begin[j], group_begin[j + 1]) hold g, with g made local to it.
__device__ __forceinline__ int split_job(const RcSplitBatch &t, long long &g) {
    int lo = 0, hi = t.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.group_begin[mid] <= g) lo = mid; else hi = mid - 1;
    }
    g -= t.group_begin[lo];
    return lo;
}

// BATCH: jobs from the table (fields loaded per row group); otherwise the
// single job a0, whose fields stay kernel parameters (constant bank).
template <int SGN, int MODE, int N2, bool BATCH>
__global__ void __launch_bounds__(kSplitThreads, 2) range_compress_split(RcSplitArgs a0, RcSplitBatch tab,
                                                                         long long n_groups) {
    constexpr int N = 32 * N2;
    constexpr int C = 32 / N2;  // pass-2 transforms per thread
    extern __shared__ __align__(16) float2 xbuf[];  // [sub-transforms of the CTA][REG]
    __shared__ float row_max[kSplitThreads / 32];
    const int os = a0.os;  // the same for every job of a launch
    const int REG = split_region(N2, os);  // float2 per region
    const int RT = N2 * os;               // threads per row
    const int RPC = kSplitThreads / RT;   // rows per CTA
    const int lrow = threadIdx.x / RT;
    const int rem = threadIdx.x - lrow * RT;
    const int s = rem / N2;               // sub-transform: bins os q + s
    const int j = rem - s * N2;           // thread within the sub-transform
    float2 *xb = xbuf + (threadIdx.x / N2) * REG;   // this sub-transform's region
    float2 *xrow = xbuf + lrow * os * REG;          // the row's first region
    const int sh_os = 31 - __clz(os);

    // one row group of job a (gl: the group's index within the job)
    auto group = [&](const RcSplitArgs &a, long long gl) {
        const float2 *pre = a.pre + (size_t)s * N + j;  // w_r[n] W^(n s) at n = N2 n1 + j
        const float2 *twd = a.twd + j;                   // W_N^(j k1) at [k1][j]
        const long long row = gl * RPC + lrow;
        const bool active = row < a.rows;
        const float2 *x = a.beat + (active ? row : 0) * (long long)N;
        float2 v[32];
#pragma unroll
        for (int n1 = 0; n1 < 32; ++n1) {
            const float2 xv = active ? __ldg(x + N2 * n1 + j) : make_float2(0.f, 0.f);
            const float2 t = __ldg(pre + N2 * n1);
            v[n1] = make_float2(fmaf(xv.x, t.x, -xv.y * t.y), fmaf(xv.x, t.y, xv.y * t.x));
        }
        dft_small<32, SGN>(v);
#pragma unroll
        for (int k1 = 1; k1 < 32; ++k1) {
            const float2 w = __ldg(twd + k1 * N2);
            const float2 b = v[k1];
            v[k1] = make_float2(fmaf(b.x, w.x, -b.y * w.y), fmaf(b.x, w.y, b.y * w.x));
        }
        // exchange A[j][k1] -> thread owning k1: element (k1, jj) sits at
        // k1 N2 + k1 / C + jj.  Writes of one k1 are consecutive; thread j
        // reads its k1 = j C + i at j (C N2 + 1) + i N2 + jj, a stride of
        // C N2 + 1 = 33 elements between threads (16 bank pairs per half-warp).
        // Every address is a per-thread base plus a constant.
#pragma unroll
        for (int k1 = 0; k1 < 32; ++k1) xb[k1 * N2 + k1 / C + j] = v[k1];
        __syncwarp();
        {
            const float2 *rd = xb + j * (C * N2 + 1);
#pragma unroll
            for (int i = 0; i < C; ++i)
#pragma unroll
                for (int jj = 0; jj < N2; ++jj) v[i * N2 + jj] = rd[i * N2 + jj];
        }
#pragma unroll
        for (int i = 0; i < C; ++i) dft_small<N2, SGN>(v + i * N2);
        // X[q] with q = k1 + 32 k2 (k1 = j C + i) back into the region, by q
        __syncwarp();
#pragma unroll
        for (int i = 0; i < C; ++i)
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) xb[j * C + i + 32 * k2] = v[i * N2 + k2];
        __syncthreads();

        // cropped bins k in [crop_lo, crop_hi], RT consecutive bins per step
        // across the row's threads: X = sub-transform k mod os at q = k / os,
        // times the per-bin rotation and w_sar
        const float g_az = (a.w_az != nullptr && active) ? __ldg(a.w_az + row / a.R) : 1.f;
        if (MODE == kRcProfileF32) {
            if (active) {
                float2 *out = reinterpret_cast<float2 *>(a.out) + row * (long long)a.n_bins - a.crop_lo;
                for (int k = a.crop_lo + rem; k <= a.crop_hi; k += RT) {
                    const float2 b = xrow[(k & (os - 1)) * REG + (k >> sh_os)];
                    const float2 r = __ldg(a.rot + (k - a.crop_lo));
                    out[k] = make_float2(g_az * fmaf(b.x, r.x, -b.y * r.y), g_az * fmaf(b.x, r.y, b.y * r.x));
                }
            }
            __syncthreads();  // the regions are rewritten by the next row
        } else {
            float mx = 0.f;
            if (active) {
                for (int k = a.crop_lo + rem; k <= a.crop_hi; k += RT) {
                    const float2 b = xrow[(k & (os - 1)) * REG + (k >> sh_os)];
                    const float2 r = __ldg(a.rot + (k - a.crop_lo));
                    mx = fmaxf(mx, fmaxf(fabsf(g_az * fmaf(b.x, r.x, -b.y * r.y)),
                                         fabsf(g_az * fmaf(b.x, r.y, b.y * r.x))));
                }
            }
            // row maximum: within the warp's lanes of the row, then across the
            // row's warps (RT >= 32) through shared memory
            const int span = RT < 32 ? RT : 32;
            for (int o = span >> 1; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (RT > 32) {
                if ((threadIdx.x & 31) == 0) row_max[threadIdx.x >> 5] = mx;
                __syncthreads();
                const int w0 = (lrow * RT) >> 5;
                for (int w = 0; w < (RT >> 5); ++w) mx = fmaxf(mx, row_max[w0 + w]);
            }
            if (active) {
                const float scale = mx > 0.f ? mx * (1.0f / 16384.0f) : 1.0f;
                const float inv = g_az / scale;
                if (rem == 0) a.scales[row] = scale;
                __half2 *out = reinterpret_cast<__half2 *>(a.out) + row * (long long)a.n_bins - a.crop_lo;
                for (int k = a.crop_lo + rem; k <= a.crop_hi; k += RT) {
                    const float2 b = xrow[(k & (os - 1)) * REG + (k >> sh_os)];
                    const float2 r = __ldg(a.rot + (k - a.crop_lo));
                    out[k] = __floats2half2_rn(inv * fmaf(b.x, r.x, -b.y * r.y), inv * fmaf(b.x, r.y, b.y * r.x));
                }
            }
            __syncthreads();  // the regions and row_max are rewritten by the next row
        }
    };

    for (long long g = blockIdx.x; g < n_groups; g += gridDim.x) {
        // L2 prefetch of the row this thread group handles next (one 128-byte
        // line per thread)
        const long long gn = g + gridDim.x;
        if constexpr (BATCH) {
            if (gn < n_groups) {
                long long gnl = gn;
                const RcSplitArgs &an = tab.jobs[split_job(tab, gnl)];
                const long long nrow = gnl * RPC + lrow;
                if (nrow < an.rows && rem * 16 < N)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(an.beat + nrow * (long long)N + rem * 16));
            }
            long long gl = g;
            const RcSplitArgs aj = tab.jobs[split_job(tab, gl)];
            group(aj, gl);
        } else {
            const long long nrow = gn * RPC + lrow;
            if (nrow < a0.rows && rem * 16 < N)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(a0.beat + nrow * (long long)N + rem * 16));
            group(a0, g);
        }
    }
}

template <int SGN, int MODE>
cudaError_t launch_rc(const RcArgs &a, cudaStream_t s) {
    const int n = a.n_fft;
    if (n <= 4096) {
        const int rows_per = 4096 / n;
        const long long n_groups = (a.rows + rows_per - 1) / rows_per;
        if (n_groups == 0) return cudaSuccess;
        const size_t smem = ((size_t)rows_per * (n + n / 16) + n + 2 * (size_t)rows_per * a.N) * sizeof(float2) +
                            (size_t)a.N * sizeof(float);
        const bool os4 = n == 4 * a.N;
        auto kern = n == 4096   ? (os4 ? range_compress_persistent<SGN, MODE, 12, 4>
                                       : range_compress_persistent<SGN, MODE, 12, 16>)
                    : n == 2048 ? (os4 ? range_compress_persistent<SGN, MODE, 11, 4>
                                       : range_compress_persistent<SGN, MODE, 11, 16>)
                                : range_compress_persistent<SGN, MODE, 0, 16>;
        int dev = 0, sms = 0, optin = 0, occ = 0;
        cudaFuncAttributes fa;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, kern) != cudaSuccess)
            return cudaErrorInvalidConfiguration;
        // process-wide attribute: the largest dynamic size the device allows
        // next to the kernel's static shared memory
        const int max_dyn = optin - (int)fa.sharedSizeBytes;
        if ((int)smem > max_dyn) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn);
        if (e != cudaSuccess) return e;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem) != cudaSuccess || occ < 1)
            return cudaErrorInvalidConfiguration;
        const long long grid = std::min<long long>(n_groups, (long long)sms * occ);
        kern<<<(unsigned)grid, 256, smem, s>>>(a, n_groups);
        return cudaGetLastError();
    }
    const int T = n / 16;
    const int rows_per_cta = n >= 4096 ? 1 : 4096 / n;
    const int threads = T * rows_per_cta;
    const size_t smem = (size_t)rows_per_cta * (n + n / 16) * sizeof(float2);
    auto kern = n > 4096 ? range_compress_kernel<SGN, MODE, true> : range_compress_kernel<SGN, MODE, false>;
    // process-wide attribute shared by all plans: the largest row size
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(16384 * 17 / 16 * sizeof(float2)));
    if (e != cudaSuccess) return e;
    const long long blocks = (a.rows + rows_per_cta - 1) / rows_per_cta;
    if (blocks == 0) return cudaSuccess;
    kern<<<(unsigned)blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int SGN, int MODE>
cudaError_t launch_split(const RcSplitArgs &a, const RcSplitBatch &tab, long long groups, cudaStream_t s) {
    auto kern = tab.jobs ? (a.N2 == 32   ? range_compress_split<SGN, MODE, 32, true>
                            : a.N2 == 16 ? range_compress_split<SGN, MODE, 16, true>
                                         : range_compress_split<SGN, MODE, 8, true>)
                         : (a.N2 == 32   ? range_compress_split<SGN, MODE, 32, false>
                            : a.N2 == 16 ? range_compress_split<SGN, MODE, 16, false>
                                         : range_compress_split<SGN, MODE, 8, false>);
    const int rpc = kSplitThreads / (a.N2 * a.os);
    const long long n_groups = tab.jobs ? groups : (a.rows + rpc - 1) / rpc;
    if (n_groups == 0) return cudaSuccess;
    // one region per sub-transform of the CTA (66 KB at N2 = 32)
    const size_t smem = (size_t)(kSplitThreads / a.N2) * split_region(a.N2, a.os) * sizeof(float2);
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kSplitThreads, smem) != cudaSuccess || occ < 1)
        return cudaErrorInvalidConfiguration;
    const long long grid = std::min<long long>(n_groups, (long long)sms * occ);
    kern<<<(unsigned)grid, kSplitThreads, smem, s>>>(a, tab, n_groups);
    return cudaGetLastError();
}

}  // namespace

bool rc_split_supported(int n_samples, int os) {
    if (os < 1 || os > 16 || (os & (os - 1)) != 0) return false;
    const int n2 = n_samples / 32;
    if (n_samples != 32 * n2 || (n2 != 8 && n2 != 16 && n2 != 32)) return false;
    return n2 * os <= kSplitThreads;
}

cudaError_t launch_range_compress_split(const RcSplitArgs &a, int sign, int mode, cudaStream_t s,
                                        const RcSplitBatch *tab, long long groups) {
    if (mode == kRcSpectrum || !rc_split_supported(32 * a.N2, a.os)) return cudaErrorInvalidValue;
    const RcSplitBatch t = tab ? *tab : RcSplitBatch{};
    if (sign > 0)
        return mode == kRcProfileF16 ? launch_split<1, kRcProfileF16>(a, t, groups, s)
                                     : launch_split<1, kRcProfileF32>(a, t, groups, s);
    return mode == kRcProfileF16 ? launch_split<-1, kRcProfileF16>(a, t, groups, s)
                                 : launch_split<-1, kRcProfileF32>(a, t, groups, s);
}

cudaError_t launch_range_compress(const RcArgs &a, int sign, int mode, cudaStream_t s) {
    if (sign > 0) {
        if (mode == kRcProfileF32) return launch_rc<1, kRcProfileF32>(a, s);
        if (mode == kRcProfileF16) return launch_rc<1, kRcProfileF16>(a, s);
        return launch_rc<1, kRcSpectrum>(a, s);
    }
    if (mode == kRcProfileF32) return launch_rc<-1, kRcProfileF32>(a, s);
    if (mode == kRcProfileF16) return launch_rc<-1, kRcProfileF16>(a, s);
    return launch_rc<-1, kRcSpectrum>(a, s);
}

}  // namespace sar
