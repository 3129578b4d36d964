// Time-domain backprojection, paper Alg. 2 (Sec. IV):
//   P(p) = sum_m sum_r exp(sign j 2 pi f0 d / c) s(a1 d + f_doppler(p), m, r),
//   d = ||p - q_tx(m)|| + ||p - q_rx(m, r)||,
// with s the linear interpolation of the stored range profile (Sec. III-C).
//
// GB300 design:
//  * Persistent grid of (SMs x resident CTAs).  The work units (pixel tile,
//    pulse block) are split into equal contiguous ranges, one per CTA
//    ("stream-K"): every CTA does the same number of pulse blocks.  A tile
//    split across CTAs is summed by bp_fixup_kernel in CTA order, so results
//    are deterministic for a given grid.
//  * Each thread keeps 4 pixels in registers: offsets (dx, dy) from the tile
//    reference point and the complex accumulators.
//  * Per (tile, pulse, antenna) the reference range R0 to the tile reference
//    is computed in FP64 (the only FP64 in the path).  Per pixel the FP32
//    differential range d - R0 comes from one rsqrt and a Newton correction
//    that never forms the cancelling difference of two large ranges.
//  * Because both the bin index and the phase are linear in d, the phase
//    correction exp(sign j 2 pi f0 d / c) = exp(sign j 2 pi beta idx) splits
//    into a per-bin rotation (folded into the stored profile at range
//    compression) and exp(sign j 2 pi beta f) of the fractional index f.
//  * The bins a tile can touch for one (pulse, Rx) form a short window
//    (a few tens of bins).  Windows of a block of pulses are staged in shared
//    memory as (A_k, D_k) = rot_k (S_k, S_{k+1} - S_k) pairs, so one 16-byte
//    shared load feeds an update: v = A + f D.
//  * Three-stage software pipeline per pulse block: FP64 reference ranges two
//    blocks ahead, cp.async copies of the raw samples one block ahead, the
//    pixel loop on the current block; one barrier per block.
#include <cuda_fp16.h>

#include "sar_internal.h"

namespace sar {
namespace {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: adding it (rounding down) floors to an integer
constexpr uint32_t kMagicBits = 0x4B400000u;

struct Layout {
    uint32_t table, raw, txr, rxr, pair, total;
};

__host__ __device__ inline Layout bp_layout(int Mb, int R, int L, bool fp16) {
    Layout s;
    uint32_t off = 0;
    s.table = off;
    off += 2u * Mb * R * L * 16u;
    s.raw = off;
    off += (uint32_t)Mb * R * (L / 4) * 5u * (fp16 ? 4u : 8u);
    off = (off + 15u) & ~15u;
    s.txr = off;
    off += 3u * Mb * 16u;
    s.rxr = off;
    off += 3u * Mb * R * 16u;
    s.pair = off;
    off += 3u * Mb * R * 16u;
    s.total = off;
    return s;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(dst), "l"(src), "n"(BYTES),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ float4 lds128(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

// Differential range d - R for a point at offset (dx, dy) from the tile
// reference, given w = (reference - antenna).xy, R ~ |w| and R^2 in
// w4 = (wx, wy, R, R^2).  Exact identity: d^2 = R^2 + 2 num with
// num = w.delta + |delta|^2 / 2.  With y = rsqrt(s), s = R^2 + 2 num, the first
// guess e = s y - R is refined by one Newton step on the residual
// r = num - e (R + e / 2) = (d^2 - (R + e)^2) / 2, giving e + r y.  Relative
// FP32 error of each term, never an absolute error of order ulp(R).
__device__ __forceinline__ float range_delta(float4 w, float dx, float dy, float hd2) {
    const float num = fmaf(w.x, dx, fmaf(w.y, dy, hd2));
    const float s = fmaf(2.0f, num, w.w);
    const float y = rsqrtf(s);
    const float e = fmaf(s, y, -w.z);
    const float t = fmaf(0.5f, e, w.z);
    const float r = fmaf(-e, t, num);
    return fmaf(r, y, e);
}

struct Smem {
    unsigned char *base;
    uint32_t base_addr;
    Layout lay;
    __device__ float4 *txr(int slot, int Mb) const { return reinterpret_cast<float4 *>(base + lay.txr) + slot * Mb; }
    __device__ float4 *rxr(int slot, int MbR) const {
        return reinterpret_cast<float4 *>(base + lay.rxr) + slot * MbR;
    }
    __device__ int4 *pair(int slot, int MbR) const { return reinterpret_cast<int4 *>(base + lay.pair) + slot * MbR; }
    __device__ float4 *table(int slot, int MbRL) const {
        return reinterpret_cast<float4 *>(base + lay.table) + (size_t)slot * MbRL;
    }
};

// FP64 reference ranges of one pulse block into constant slot `cslot`, with
// the shared-memory address constants pointing at table slot `tslot`.
__device__ __forceinline__ void prep_block(const BpArgs &a, const Smem &sm, const TileInfo &ti, int b,
                                           int cslot, int tslot) {
    const int R = a.R, Mb = a.Mb, MbR = Mb * R;
    const int m0 = b * Mb;
    const int np = min(Mb, a.M - m0);
    float4 *txr = sm.txr(cslot, Mb);
    float4 *rxr = sm.rxr(cslot, MbR);
    int4 *pr = sm.pair(cslot, MbR);
    const uint32_t table_addr = sm.base_addr + sm.lay.table + (uint32_t)tslot * (uint32_t)(MbR * a.L) * 16u;
    for (int task = threadIdx.x; task < np * R; task += blockDim.x) {
        const int p = task / R;
        const int r = task - p * R;
        const int m = m0 + p;
        const double2 qt = reinterpret_cast<const double2 *>(a.q_tx)[m];
        const double2 qr = reinterpret_cast<const double2 *>(a.q_rx)[(long long)m * R + r];
        const double wtx = ti.x - qt.x, wty = ti.y - qt.y;
        const double wrx = ti.x - qr.x, wry = ti.y - qr.y;
        const double r_tx = sqrt(wtx * wtx + wty * wty);
        const double r_rx = sqrt(wrx * wrx + wry * wry);
        const double d0 = r_tx + r_rx;
        const uint32_t addr_c = table_addr + (uint32_t)(task * a.L) * 16u - kMagicBits * 16u;
        // invalid geometry contributes nothing: finite stand-in distances and a
        // window far outside every profile (all staged samples zero)
        const float4 dummy = make_float4(0.f, 0.f, 1.f, 1.f);
        const bool ok_tx = isfinite(r_tx) && r_tx < kMaxRange;
        const bool ok_rx = isfinite(r_rx) && r_rx < kMaxRange;
        const float4 t4 = ok_tx ? make_float4((float)wtx, (float)wty, (float)r_tx, (float)(r_tx * r_tx)) : dummy;
        const float4 r4 = ok_rx ? make_float4((float)wrx, (float)wry, (float)r_rx, (float)(r_rx * r_rx)) : dummy;
        int4 q;
        if (ok_tx && ok_rx) {
            const double lo = a.a1 * (d0 - 2.0 * ti.rho) - (double)a.fd_max;
            const int k_lo = (int)floor(lo) - kGuardBins;
            const float idx0 = (float)(a.a1 * d0 - (double)k_lo);
            q = make_int4(__float_as_int(idx0), (int)addr_c, k_lo, 1);
        } else {
            q = make_int4(__float_as_int((float)kGuardBins), (int)addr_c, -(1 << 30), 0);
            atomicOr(a.err, 1);
        }
        if (r == 0) txr[p] = t4;
        rxr[task] = r4;
        pr[task] = q;
    }
}

// Issue cp.async copies of the raw profile samples of one pulse block.  Item
// = (window w, group q of 4 entries) = samples k_lo + 4q .. k_lo + 4q + 4.
// Samples outside [crop_lo, crop_hi] are zero-filled.
template <bool FP16>
__device__ __forceinline__ void stage_block(const BpArgs &a, const Smem &sm, int b, int cslot) {
    constexpr int SB = FP16 ? 4 : 8;
    const int R = a.R, Mb = a.Mb, MbR = Mb * R;
    const int np = min(Mb, a.M - b * Mb);
    const int nq = a.L >> 2;
    const int4 *pr = sm.pair(cslot, MbR);
    const unsigned char *prof = reinterpret_cast<const unsigned char *>(a.prof);
    const uint32_t raw = sm.base_addr + sm.lay.raw;
    const int n_items = np * R * nq;
    for (int it = threadIdx.x; it < n_items; it += blockDim.x) {
        const int w = it / nq;
        const int q = it - w * nq;
        const int p = w / R;
        const int r = w - p * R;
        const long long row = (long long)(b * Mb + p) * R + r;
        const unsigned char *rowp = prof + row * a.n_bins * SB;
        const int k0 = pr[w].z + 4 * q;
        const uint32_t dst = raw + (uint32_t)it * 5u * SB;
#pragma unroll
        for (int e = 0; e < 5; ++e) {
            const int k = k0 + e;
            const bool ok = (k >= a.crop_lo) && (k <= a.crop_hi);
            const void *src = ok ? (const void *)(rowp + (long long)(k - a.crop_lo) * SB) : a.prof;
            cp_async<SB>(dst + e * SB, src, ok ? SB : 0);
        }
    }
}

// Convert this thread's staged raw samples into (A, D) table entries.
template <bool FP16>
__device__ __forceinline__ void convert_block(const BpArgs &a, const Smem &sm, int b, int cslot, int tslot) {
    constexpr int SB = FP16 ? 4 : 8;
    const int R = a.R, Mb = a.Mb, MbR = Mb * R;
    const int np = min(Mb, a.M - b * Mb);
    const int nq = a.L >> 2;
    const int4 *pr = sm.pair(cslot, MbR);
    float4 *table = sm.table(tslot, MbR * a.L);
    const unsigned char *raw = sm.base + sm.lay.raw;
    const int n_items = np * R * nq;
    for (int it = threadIdx.x; it < n_items; it += blockDim.x) {
        const int w = it / nq;
        const int q = it - w * nq;
        const int k0 = pr[w].z + 4 * q;
        float2 s[5];
        if (FP16) {
            const int p = w / R;
            const int r = w - p * R;
            const float sc = __ldg(a.prof_scale + (long long)(b * Mb + p) * R + r);
            const __half2 *h = reinterpret_cast<const __half2 *>(raw + (size_t)it * 5 * SB);
#pragma unroll
            for (int e = 0; e < 5; ++e) {
                const float2 f = __half22float2(h[e]);
                s[e] = make_float2(f.x * sc, f.y * sc);
            }
        } else {
            const float2 *f = reinterpret_cast<const float2 *>(raw + (size_t)it * 5 * SB);
#pragma unroll
            for (int e = 0; e < 5; ++e) s[e] = f[e];
        }
        float4 *dst = table + w * a.L + 4 * q;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = k0 + e;
            const bool valid = (k >= a.crop_lo) && (k < a.crop_hi);
            const float2 nb = cmul(s[e + 1], a.cb);
            const float4 ent = make_float4(s[e].x, s[e].y, nb.x - s[e].x, nb.y - s[e].y);
            dst[e] = valid ? ent : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

template <int RG, bool FD>
__device__ __forceinline__ void compute_block(const BpArgs &a, const Smem &sm, int b, int cslot,
                                              const float (&dx)[kPxPerThread], const float (&dy)[kPxPerThread],
                                              const float (&hd2)[kPxPerThread], const float (&fdm)[kPxPerThread],
                                              float (&acc_re)[kPxPerThread], float (&acc_im)[kPxPerThread]) {
    const int R = a.R, Mb = a.Mb, MbR = Mb * R;
    const int np = min(Mb, a.M - b * Mb);
    const float4 *txr = sm.txr(cslot, Mb);
    const float4 *rxr = sm.rxr(cslot, MbR);
    const int4 *pr = sm.pair(cslot, MbR);
    const float a1 = a.a1f;
    const float k2pb = a.two_pi_beta;
    const float lmax = (float)(a.L - 2);
    for (int p = 0; p < np; ++p) {
        const float4 t4 = txr[p];
        float dt[kPxPerThread];
#pragma unroll
        for (int j = 0; j < kPxPerThread; ++j) {
            dt[j] = range_delta(t4, dx[j], dy[j], hd2[j]);
            if (FD) dt[j] += fdm[j];
        }
        for (int r0 = 0; r0 < R; r0 += RG) {
#pragma unroll
            for (int rr = 0; rr < RG; ++rr) {
                const int w = p * R + r0 + rr;
                const float4 q4 = rxr[w];
                const int4 pq = pr[w];
                const float idx0 = __int_as_float(pq.x);
                const uint32_t ac = (uint32_t)pq.y;
#pragma unroll
                for (int j = 0; j < kPxPerThread; ++j) {
                    const float drx = range_delta(q4, dx[j], dy[j], hd2[j]);
                    float idx = fmaf(a1, dt[j] + drx, idx0);
                    idx = fminf(fmaxf(idx, 0.0f), lmax);
                    const float tm = __fadd_rd(idx, kMagic);
                    const float f = idx - (tm - kMagic);
                    const float4 e = lds128((__float_as_uint(tm) << 4) + ac);
                    const float vre = fmaf(f, e.z, e.x);
                    const float vim = fmaf(f, e.w, e.y);
                    float sn, cs;
                    __sincosf(f * k2pb, &sn, &cs);
                    acc_re[j] = fmaf(vre, cs, acc_re[j]);
                    acc_im[j] = fmaf(vre, sn, acc_im[j]);
                    acc_re[j] = fmaf(-vim, sn, acc_re[j]);
                    acc_im[j] = fmaf(vim, cs, acc_im[j]);
                }
            }
        }
    }
}

template <int RG, bool FP16, bool FD>
__global__ void __launch_bounds__(kBpThreads, 2) backproject_kernel(BpArgs a) {
    extern __shared__ __align__(16) unsigned char smem_bp[];
    Smem sm;
    sm.base = smem_bp;
    sm.base_addr = (uint32_t)__cvta_generic_to_shared(smem_bp);
    sm.lay = bp_layout(a.Mb, a.R, a.L, FP16);

    const long long u0 = (long long)blockIdx.x * a.units / a.G;
    const long long u1 = (long long)(blockIdx.x + 1) * a.units / a.G;
    const int PB = a.blocks_per_tile;
    const int t_first = (int)(u0 / PB);

    long long u = u0;
    while (u < u1) {
        const int tile = (int)(u / PB);
        const int b0 = (int)(u - (long long)tile * PB);
        const int b1 = (int)min((long long)PB, (long long)b0 + (u1 - u));
        const TileInfo ti = a.tiles[tile];

        float dx[kPxPerThread], dy[kPxPerThread], hd2[kPxPerThread], fdm[kPxPerThread];
        float fdc[kPxPerThread];
        int oi[kPxPerThread];
        float acc_re[kPxPerThread], acc_im[kPxPerThread];
#pragma unroll
        for (int j = 0; j < kPxPerThread; ++j) {
            const long long slot = (long long)tile * kTilePx + threadIdx.x + j * kBpThreads;
            const float2 d = a.pix[slot];
            oi[j] = a.out_idx[slot];
            dx[j] = d.x;
            dy[j] = d.y;
            hd2[j] = 0.5f * fmaf(d.x, d.x, d.y * d.y);
            fdm[j] = 0.f;
            fdc[j] = 0.f;
            if (FD && oi[j] >= 0) {
                const float fd = fminf(fmaxf(a.fdopp[oi[j]], -a.fd_max), a.fd_max);
                fdm[j] = fd / a.a1f;  // in metres of d, added to the Tx delta
                fdc[j] = fd;
            }
            acc_re[j] = 0.f;
            acc_im[j] = 0.f;
        }

        // pipeline prologue
        prep_block(a, sm, ti, b0, 0, 0);
        if (b0 + 1 < b1) prep_block(a, sm, ti, b0 + 1, 1, 1);
        __syncthreads();
        stage_block<FP16>(a, sm, b0, 0);
        cp_async_commit();
        cp_async_wait_all();
        convert_block<FP16>(a, sm, b0, 0, 0);
        __syncthreads();

        for (int b = b0; b < b1; ++b) {
            const int k = b - b0;
            if (b + 2 < b1) prep_block(a, sm, ti, b + 2, (k + 2) % 3, (k + 2) & 1);
            if (b + 1 < b1) stage_block<FP16>(a, sm, b + 1, (k + 1) % 3);
            cp_async_commit();
            compute_block<RG, FD>(a, sm, b, k % 3, dx, dy, hd2, fdm, acc_re, acc_im);
            cp_async_wait_all();
            if (b + 1 < b1) convert_block<FP16>(a, sm, b + 1, (k + 1) % 3, (k + 1) & 1);
            __syncthreads();
        }

        if (FD) {
            // the Doppler offset moved the index, not the phase: undo its share
            // exp(sign j 2 pi beta f_doppler) of the per-index phase
#pragma unroll
            for (int j = 0; j < kPxPerThread; ++j) {
                float cyc = a.beta * fdc[j];
                cyc -= rintf(cyc);
                float sn, cs;
                sincospif(-2.0f * a.sign * cyc, &sn, &cs);
                const float re = acc_re[j] * cs - acc_im[j] * sn;
                const float im = acc_re[j] * sn + acc_im[j] * cs;
                acc_re[j] = re;
                acc_im[j] = im;
            }
        }

        if (b0 == 0 && b1 == PB) {
#pragma unroll
            for (int j = 0; j < kPxPerThread; ++j) {
                if (oi[j] < 0) continue;
                float2 v = make_float2(acc_re[j], acc_im[j]);
                if (a.accumulate) {
                    const float2 o = a.image[oi[j]];
                    v.x += o.x;
                    v.y += o.y;
                }
                a.image[oi[j]] = v;
            }
        } else {
            const long long slot = (long long)blockIdx.x * a.seg_max + (tile - t_first);
            float2 *dst = a.partial + slot * kTilePx;
#pragma unroll
            for (int j = 0; j < kPxPerThread; ++j)
                dst[threadIdx.x + j * kBpThreads] = make_float2(acc_re[j], acc_im[j]);
        }
        u += b1 - b0;
    }
}

// Sums, in CTA order, the partial sums of tiles that were split across CTAs.
__global__ void __launch_bounds__(256) bp_fixup_kernel(BpArgs a) {
    const int tile = blockIdx.x;
    const long long PB = a.blocks_per_tile;
    const long long ua = (long long)tile * PB;
    const long long ub = ua + PB - 1;
    const int ia = (int)(((ua + 1) * a.G - 1) / a.units);
    const int ib = (int)(((ub + 1) * a.G - 1) / a.units);
    if (ia == ib) return;
    for (int s = threadIdx.x; s < kTilePx; s += blockDim.x) {
        const int o = a.out_idx[(long long)tile * kTilePx + s];
        if (o < 0) continue;
        float2 acc = make_float2(0.f, 0.f);
        for (int i = ia; i <= ib; ++i) {
            const long long ui0 = (long long)i * a.units / a.G;
            const long long slot = (long long)i * a.seg_max + (tile - (int)(ui0 / PB));
            const float2 v = a.partial[slot * kTilePx + s];
            acc.x += v.x;
            acc.y += v.y;
        }
        if (a.accumulate) {
            const float2 old = a.image[o];
            acc.x += old.x;
            acc.y += old.y;
        }
        a.image[o] = acc;
    }
}

template <int RG, bool FP16, bool FD>
void *kernel_ptr() {
    return (void *)backproject_kernel<RG, FP16, FD>;
}

void *select_kernel(int rg, bool fp16, bool fd) {
#define SAR_SEL(RGV)                                                              \
    if (rg == RGV) {                                                              \
        if (fp16) return fd ? kernel_ptr<RGV, true, true>() : kernel_ptr<RGV, true, false>();   \
        return fd ? kernel_ptr<RGV, false, true>() : kernel_ptr<RGV, false, false>();           \
    }
    SAR_SEL(1)
    SAR_SEL(2)
    SAR_SEL(4)
#undef SAR_SEL
    return nullptr;
}

}  // namespace

size_t bp_smem_bytes(int Mb, int R, int L, bool fp16) { return bp_layout(Mb, R, L, fp16).total; }

cudaError_t bp_prepare(bool fp16, int rg, size_t smem) {
    for (int fd = 0; fd < 2; ++fd) {
        void *k = select_kernel(rg, fp16, fd != 0);
        if (!k) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int bp_occupancy(bool fp16, int rg, size_t smem, int *ctas_per_sm) {
    void *k = select_kernel(rg, fp16, false);
    if (!k) return -1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kBpThreads, smem) != cudaSuccess) return -1;
    *ctas_per_sm = n;
    return 0;
}

cudaError_t launch_backproject(const BpArgs &a, const BpLaunch &l, cudaStream_t s) {
    void *k = select_kernel(l.rg, l.fp16, a.fdopp != nullptr);
    if (!k) return cudaErrorInvalidValue;
    if (a.units == 0) return cudaSuccess;
    BpArgs args = a;
    void *params[] = {&args};
    cudaError_t e = cudaLaunchKernel(k, dim3(a.G), dim3(kBpThreads), params, l.smem, s);
    if (e != cudaSuccess) return e;
    bp_fixup_kernel<<<a.n_tiles, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sar
