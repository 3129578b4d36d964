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
//    memory as (A_k, D_k) = rot_k (S_k, (S_{k+1} - S_k) / kappa) pairs,
//    kappa = sign 2 pi beta, so one 16-byte shared load feeds an update:
//    with g = kappa f the phase, v = A + g D.  g comes from the index in two
//    FMAs (kappa has 22 significant bits, so kappa floor(idx) is formed
//    exactly from the magic-number floor).
//  * Two inner loops, chosen per (tile, pulse block) by the FP64 stage:
//    - expansion loop (the common case): Rx antennas lie millimetres from the
//      Tx antenna, so with o = q_rx - q_tx and a = |o|^2 / 2 - (p - q_tx).o,
//      d_rx = sqrt(d_tx^2 + 2 a) = d_tx + a / d_tx - a^2 / (2 d_tx^3) + e3,
//      |e3| <= |o|^3 / (2 d_tx^2).  It reuses the Tx rsqrt (no MUFU per Rx)
//      and is taken only where a1 |o|^3 / (2 (R0_tx - rho)^2) <= 2e-6 bins
//      and the common window of the pulse's Rx channels fits;
//    - exact loop: every distance with its own rsqrt and Newton step, and
//      the index clamped into the window (near field, large arrays, invalid
//      geometry).
//  * Three-stage software pipeline per pulse block: FP64 reference ranges two
//    blocks ahead, cp.async copies of the raw samples one block ahead, the
//    pixel loop on the current block; one barrier per block, which also
//    reduces the per-block loop choice.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>

#include "sar_internal.h"

namespace sar {
namespace {

// Fix-up kernels: threads per CTA and pixels per thread of one tile.
constexpr int kFixupThreads = 256;
constexpr int kFixupPx = kTilePx / kFixupThreads;

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: adding it (rounding down) floors to an integer
constexpr uint32_t kMagicBits = 0x4B400000u;
// Truncation bound of the expansion loop, in bins of the index.
constexpr double kExpansionTolBins = 2e-6;

// Shared memory per CTA: two (A, D) table slots, one raw staging buffer and
// three slots of per-pulse constants.
struct Layout {
    uint32_t table, raw, txr, txc, rxr, rxt, pair, flags, total;
};

// Per-block loop choice, OR-reduced over the CTA's FP64 tasks.
constexpr int kFlagExact = 1;    // the expansion loop cannot take the block
constexpr int kFlagOffAxis = 2;  // some Rx offset has a y component

__host__ __device__ inline Layout bp_layout(int Mb, int R, int L, bool fp16) {
    Layout s;
    uint32_t off = 0;
    s.table = off;
    off += 2u * Mb * R * L * 16u;
    s.raw = off;
    off += (uint32_t)Mb * R * (L / 4) * 5u * (fp16 ? 4u : 8u);
    off = (off + 15u) & ~15u;
    s.txr = off;  // float4 (wx, wy, R, R^2) of the Tx antenna
    off += 3u * Mb * 16u;
    s.txc = off;  // int4 (c = 2 a1 R0_tx - k_lo, k_lo, 0, 0) for the expansion loop
    off += 3u * Mb * 16u;
    s.rxr = off;  // float4 (wx, wy, R, R^2) of each Rx antenna (exact loop)
    off += 3u * Mb * R * 16u;
    s.rxt = off;  // float4 (-o_x, -o_y, |o|^2/2 - w_tx.o, table address constant)
    off += 3u * Mb * R * 16u;
    s.pair = off;  // int4 (idx0 bits, table address constant, k_lo, FP16 scale bits)
    off += 3u * Mb * R * 16u;
    s.flags = off;  // int per constant slot: loop choice of the block (kFlag*)
    off += 16u;
    s.total = off;
    return s;
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

// Single MUFU operations (flush-to-zero, no special-case fix-up sequences).
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void sincos_approx(float x, float &s, float &c) {
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(x));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(x));
}

// FP64 square root of x >= 0 from an FP32 reciprocal-square-root seed and one
// Newton step on the residual x - r^2 (relative error ~1e-14, below what the
// index and phase need).  Non-finite or negative x gives NaN.
__device__ __forceinline__ double sqrt_fp64(double x) {
    // outside the seed's range: tiny -> 0, huge stays huge (rejected later as
    // beyond the maximum range), negative or NaN -> NaN
    const float xf = (float)x;
    if (!(xf >= 1e-30f && xf <= 1e30f))
        return x >= 0.0 ? (x < 1e-30 ? 0.0 : x) : __longlong_as_double(0x7ff8000000000000ll);
    const double y = (double)rsqrt_approx(xf);
    const double r = x * y;
    return fma(0.5 * y, fma(-r, r, x), r);
}

// Differential range d - R for a point at offset (dx, dy) from the tile
// reference, given w = (reference - antenna).xy, R ~ |w| and R^2 in
// w4 = (wx, wy, R, R^2).  Exact identity: d^2 = R^2 + 2 num with
// num = w.delta + |delta|^2 / 2.  With y = rsqrt(s), s = R^2 + 2 num, the first
// guess e = s y - R is refined by one Newton step on the residual
// r = num - e (R + e / 2) = (d^2 - (R + e)^2) / 2, giving e + r y.  Relative
// FP32 error of each term, never an absolute error of order ulp(R).
// `y` returns the reciprocal distance.
__device__ __forceinline__ float range_delta(float4 w, float dx, float dy, float hd2, float &y) {
    const float num = fmaf(w.x, dx, fmaf(w.y, dy, hd2));
    const float s = fmaf(2.0f, num, w.w);
    y = rsqrt_approx(s);
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
    __device__ int4 *txc(int slot, int Mb) const { return reinterpret_cast<int4 *>(base + lay.txc) + slot * Mb; }
    __device__ float4 *rxr(int slot, int MbR) const {
        return reinterpret_cast<float4 *>(base + lay.rxr) + slot * MbR;
    }
    __device__ float4 *rxt(int slot, int MbR) const {
        return reinterpret_cast<float4 *>(base + lay.rxt) + slot * MbR;
    }
    __device__ int4 *pair(int slot, int MbR) const { return reinterpret_cast<int4 *>(base + lay.pair) + slot * MbR; }
    __device__ int *flags() const { return reinterpret_cast<int *>(base + lay.flags); }
    __device__ float4 *table(int slot, int MbRL) const {
        return reinterpret_cast<float4 *>(base + lay.table) + (size_t)slot * MbRL;
    }
};

// OR of the threads' flag bits into a shared slot (one atomic per warp).
__device__ __forceinline__ void or_flags(int *slot, int bits) {
    const int w = (int)__reduce_or_sync(0xffffffffu, (unsigned)bits);
    if ((threadIdx.x & 31) == 0 && w) atomicOr(slot, w);
}

// FP64 stage for one pulse block into constant slot `cslot`, with the
// table address constants pointing at table slot `tslot`: the Tx records of
// both loops and the Rx records of the expansion loop.  Tx tasks run on the
// first warp(s), Rx tasks on the others.  Returns nonzero if one of this
// thread's tasks rules out the expansion loop for the block: near field (an
// antenna within 2 rho + 1 mm of the tile reference), invalid geometry, an
// Rx offset beyond the window allowance, or the truncation bound.
__device__ __forceinline__ int prep_block(const BpArgs &a, const Smem &sm, const TileInfo &ti, int b,
                                          int cslot, int tslot) {
    int exact = 0;
    const int R = a.R, Mb = a.Mb, MbR = Mb * R;
    const int m0 = b * Mb;
    const int np = min(Mb, a.M - m0);
    const int rx_base = ((Mb + 31) >> 5) << 5;
    const int t = threadIdx.x;
    if (t < rx_base) {
        float4 *txr = sm.txr(cslot, Mb);
        int4 *txc = sm.txc(cslot, Mb);
        for (int p = t; p < np; p += rx_base) {
            // FP64 where FP32 would lose the index: the differences, the
            // range, the window start and 2 a1 R_tx - k_lo
            const double2 qt = reinterpret_cast<const double2 *>(a.q_tx)[m0 + p];
            const double wx = ti.x - qt.x, wy = ti.y - qt.y;
            const double r2 = fma(wx, wx, wy * wy);
            const double r_tx = sqrt_fp64(r2);
            const float r_f = (float)r_tx;
            const bool ok = r_f < (float)kMaxRange;  // false for NaN and inf
            float4 t4 = make_float4(0.f, 0.f, 1.f, 1.f);
            int4 c = make_int4(0, -(1 << 30), 0, 0);
            if (ok) {
                t4 = make_float4((float)wx, (float)wy, r_f, (float)r2);
                const int k_lo = __double2int_rd(fma(2.0 * a.a1, r_tx, -(double)ti.klo_off)) - kGuardBins;
                c = make_int4(__float_as_int((float)fma(2.0 * a.a1, r_tx, -(double)k_lo)), k_lo, 0, 0);
            } else {
                exact = kFlagExact;
            }
            txr[p] = t4;
            txc[p] = c;
        }
    } else {
        float4 *rxt = sm.rxt(cslot, MbR);
        int4 *pr = sm.pair(cslot, MbR);
        const uint32_t table_addr =
            sm.base_addr + sm.lay.table + (uint32_t)tslot * (uint32_t)(MbR * a.L) * 16u;
        const float rho = (float)ti.rho;
        const float tol2 = (float)(kExpansionTolBins * 2.0 / a.a1);
        for (int task = t - rx_base; task < np * R; task += blockDim.x - rx_base) {
            const int p = task / R;
            const int r = task - p * R;
            const int m = m0 + p;
            const double2 qt = reinterpret_cast<const double2 *>(a.q_tx)[m];
            const double2 qr = reinterpret_cast<const double2 *>(a.q_rx)[(long long)m * R + r];
            // differences in FP64, the rest in FP32: the a / d term carries a
            // relative error of a few 1e-7, i.e. ~1e-7 bins
            const float wx = (float)(ti.x - qt.x), wy = (float)(ti.y - qt.y);
            const float ox = (float)(qr.x - qt.x), oy = (float)(qr.y - qt.y);
            const float o2 = fmaf(ox, ox, oy * oy);
            const float cexp = fmaf(0.5f, o2, -fmaf(wx, ox, wy * oy));
            const uint32_t addr_c = table_addr + (uint32_t)(task * a.L) * 16u - kMagicBits * 16u;
            // halved so that the pixel loop gets a / 2 directly
            rxt[task] = make_float4(-0.5f * ox, -0.5f * oy, 0.5f * cexp, __uint_as_float(addr_c));
            if (!(fabsf(oy) <= 1e-9f)) exact |= kFlagOffAxis;
            const float scale = a.prof_scale ? __ldg(a.prof_scale + (long long)m * R + r) : 1.0f;
            pr[task].w = __float_as_int(scale);
            // path criteria (FP32 is plenty; non-finite input fails them)
            const float rt = hypotf(wx, wy);
            const float oa = sqrtf(o2);
            const float dmin = rt - rho;
            const bool expand = rt > 2.0f * rho + oa + 1e-3f && rt < (float)kMaxRange &&
                                oa <= ti.o_allow && (float)o2 * oa <= tol2 * dmin * dmin;
            exact |= expand ? 0 : kFlagExact;
        }
    }
    return exact;
}

// FP64 records of the exact loop for one pulse block (blocks the expansion
// loop cannot take): per (pulse, Rx) the Rx reference range, the window start
// of this Rx and the reference index.  Invalid geometry is flagged and given
// a window outside every profile.
__device__ __forceinline__ void prep_exact(const BpArgs &a, const Smem &sm, const TileInfo &ti, int b,
                                           int cslot, int tslot) {
    const int R = a.R, Mb = a.Mb, MbR = Mb * R;
    const int m0 = b * Mb;
    const int np = min(Mb, a.M - m0);
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
        const double r_tx = sqrt_fp64(wtx * wtx + wty * wty);
        const double r_rx = sqrt_fp64(wrx * wrx + wry * wry);
        const double d0 = r_tx + r_rx;
        const uint32_t addr_c = table_addr + (uint32_t)(task * a.L) * 16u - kMagicBits * 16u;
        const bool ok_tx = isfinite(r_tx) && r_tx < kMaxRange;
        const bool ok_rx = isfinite(r_rx) && r_rx < kMaxRange;
        rxr[task] = ok_rx ? make_float4((float)wrx, (float)wry, (float)r_rx, (float)(r_rx * r_rx))
                          : make_float4(0.f, 0.f, 1.f, 1.f);
        int4 q = pr[task];
        if (ok_tx && ok_rx) {
            const int k_lo = (int)floor(a.a1 * (d0 - 2.0 * ti.rho) - (double)a.fd_max) - kGuardBins;
            q.x = __float_as_int((float)(a.a1 * d0 - (double)k_lo));
            q.z = k_lo;
        } else {
            q.x = __float_as_int((float)kGuardBins);
            q.z = -(1 << 30);
            atomicOr(a.err, kErrGeometry);
        }
        q.y = (int)addr_c;
        pr[task] = q;
    }
}

// Window start of (pulse p, Rx r): per Rx in the exact loop, per pulse in
// the expansion loop.
__device__ __forceinline__ int window_start(const Smem &sm, int cslot, int Mb, int MbR, int w, int p,
                                            bool exact) {
    return exact ? sm.pair(cslot, MbR)[w].z : sm.txc(cslot, Mb)[p].y;
}

// floor(n / d) for 0 <= n, n d < 2^32, from mul = ceil(2^32 / d).
__device__ __forceinline__ int fast_div(int n, unsigned long long mul) {
    return (int)(((unsigned long long)(unsigned)n * mul) >> 32);
}

// Issue cp.async copies of the raw profile samples of one pulse block.  Item
// = (window w, group q of 4 entries) = samples k_lo + 4q .. k_lo + 4q + 4.
// Samples outside [crop_lo, crop_hi] are zero-filled.
template <bool FP16>
__device__ __forceinline__ void stage_block(const BpArgs &a, const Smem &sm, int b, int cslot, bool exact) {
    constexpr int SB = FP16 ? 4 : 8;
    const int R = a.R, Mb = a.Mb, MbR = Mb * R;
    const int np = min(Mb, a.M - b * Mb);
    const int nq = a.L >> 2;
    const unsigned char *prof = reinterpret_cast<const unsigned char *>(a.prof);
    const uint32_t raw = sm.base_addr + sm.lay.raw;
    const int n_items = np * R * nq;
    const long long row0 = (long long)b * MbR;  // window w reads profile row row0 + w
    // loop invariants as locals: the copies' asm statements clobber memory,
    // which would otherwise reload them every item
    const unsigned long long div_nq = a.div_nq, div_r = a.div_r;
    const int n_bins = a.n_bins, crop_lo = a.crop_lo, crop_hi = a.crop_hi;
    for (int it = threadIdx.x; it < n_items; it += blockDim.x) {
        const int w = fast_div(it, div_nq);
        const int q = it - w * nq;
        const int p = exact ? 0 : fast_div(w, div_r);
        const int k0 = window_start(sm, cslot, Mb, MbR, w, p, exact) + 4 * q;
        // sample k of this row sits at prof + (base + k) * SB
        const long long base = (row0 + w) * n_bins - crop_lo;
        const uint32_t dst = raw + (uint32_t)it * 5u * SB;
        if (k0 >= crop_lo && k0 + 4 <= crop_hi) {
            const unsigned char *src = prof + (base + k0) * SB;
#pragma unroll
            for (int e = 0; e < 5; ++e) cp_async<SB>(dst + e * SB, src + e * SB, SB);
        } else {
#pragma unroll
            for (int e = 0; e < 5; ++e) {
                const int k = k0 + e;
                const bool ok = (k >= crop_lo) && (k <= crop_hi);
                const void *src = ok ? (const void *)(prof + (base + k) * SB) : (const void *)prof;
                cp_async<SB>(dst + e * SB, src, ok ? SB : 0);
            }
        }
    }
}

// Convert this thread's staged raw samples into (A, D) table entries:
// A = S_k, D = (S_{k+1} exp(-sign j 2 pi beta) - S_k) / kappa (the stored
// samples carry the per-bin rotation already).  Entries whose base bin lies
// outside [crop_lo, crop_hi) are zero.
template <bool FP16>
__device__ __forceinline__ void convert_block(const BpArgs &a, const Smem &sm, int b, int cslot, int tslot,
                                              bool exact) {
    constexpr int SB = FP16 ? 4 : 8;
    const int R = a.R, Mb = a.Mb, MbR = Mb * R;
    const int np = min(Mb, a.M - b * Mb);
    const int nq = a.L >> 2;
    const int4 *pr = sm.pair(cslot, MbR);
    const int L = a.L;
    float4 *table = sm.table(tslot, MbR * L);
    const unsigned char *raw = sm.base + sm.lay.raw;
    const int n_items = np * R * nq;
    const unsigned long long div_nq = a.div_nq, div_r = a.div_r;
    const int crop_lo = a.crop_lo, crop_hi = a.crop_hi;
    const float2 cbk = a.cb_k;
    const float ik = a.inv_kappa;
    for (int it = threadIdx.x; it < n_items; it += blockDim.x) {
        const int w = fast_div(it, div_nq);
        const int q = it - w * nq;
        const int p = exact ? 0 : fast_div(w, div_r);
        const int k0 = window_start(sm, cslot, Mb, MbR, w, p, exact) + 4 * q;
        float2 s[5];
        if (FP16) {
            const float sc = __int_as_float(pr[w].w);
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
        float4 *dst = table + w * L + 4 * q;
        const bool inside = k0 >= crop_lo && k0 + 3 < crop_hi;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = k0 + e;
            const bool valid = inside || ((k >= crop_lo) && (k < crop_hi));
            const float dre = fmaf(s[e + 1].x, cbk.x, fmaf(-s[e + 1].y, cbk.y, -s[e].x * ik));
            const float dim = fmaf(s[e + 1].x, cbk.y, fmaf(s[e + 1].y, cbk.x, -s[e].y * ik));
            const float4 ent = make_float4(s[e].x, s[e].y, dre, dim);
            dst[e] = valid ? ent : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// One update: with f the fractional part of idx and g = kappa f, interpolate
// entry (A, D) as A + g D and accumulate it times exp(j g).  tm = 1.5 2^23 +
// floor(idx) exactly; kapm = kappa 1.5 2^23 is exact, so fma(-kappa, tm, kapm)
// = -kappa floor(idx) with one rounding, and g = fma(idx, kappa, that) with
// one more (absolute error ~ ulp(kappa L), a few 1e-4 rad at most).
__device__ __forceinline__ void accumulate(float idx, uint32_t ac, float kap, float kapm, float &acc_re,
                                           float &acc_im) {
    const float tm = __fadd_rd(idx, kMagic);
    const float g = fmaf(idx, kap, fmaf(-kap, tm, kapm));
    const float4 e = lds128((__float_as_uint(tm) << 4) + ac);
    const float vre = fmaf(g, e.z, e.x);
    const float vim = fmaf(g, e.w, e.y);
    float sn, cs;
    sincos_approx(g, sn, cs);
    acc_re = fmaf(vre, cs, acc_re);
    acc_im = fmaf(vre, sn, acc_im);
    acc_re = fmaf(-vim, sn, acc_re);
    acc_im = fmaf(vim, cs, acc_im);
}

// Blackwell's packed FP32 pairs: one instruction issues two FP32 operations,
// each rounded as its scalar form.  Pixels 2h and 2h + 1 of a thread share
// each pair, which cuts the pixel loop's instruction count by a fifth (the
// loop is issue-bound; the FMA pipe does the same work).
__device__ __forceinline__ float2 ffma2(float2 x, float2 y, float2 z) { return __ffma2_rn(x, y, z); }
__device__ __forceinline__ float2 fmul2(float2 x, float2 y) { return __fmul2_rn(x, y); }
__device__ __forceinline__ float2 bcast(float v) { return make_float2(v, v); }

// accumulate() for the pixel pair (2h, 2h + 1) of one pulse and Rx.  The
// imaginary part is kept as two sums, sum vre sn in acc_im and
// sum (-vim) cs in acc_imb (subtracted by the caller), so that every packed
// product has operands of the sign they are computed with; -vim itself comes
// from one scalar FMA with negated operands.
__device__ __forceinline__ void accumulate2(float2 idx, uint32_t ac, float2 kap, float2 nkap, float2 kapm,
                                            float (&acc_re)[kPxPerThread], float (&acc_im)[kPxPerThread],
                                            float (&acc_imb)[kPxPerThread], int h) {
    const float2 tm = __fadd2_rd(idx, bcast(kMagic));
    const float2 g = ffma2(idx, kap, ffma2(nkap, tm, kapm));
    const float4 e0 = lds128((__float_as_uint(tm.x) << 4) + ac);
    const float4 e1 = lds128((__float_as_uint(tm.y) << 4) + ac);
    const float2 vre = make_float2(fmaf(g.x, e0.z, e0.x), fmaf(g.y, e1.z, e1.x));
    const float2 vimn = make_float2(fmaf(-g.x, e0.w, -e0.y), fmaf(-g.y, e1.w, -e1.y));
    float2 sn, cs;
    sincos_approx(g.x, sn.x, cs.x);
    sincos_approx(g.y, sn.y, cs.y);
    float2 re = make_float2(acc_re[2 * h], acc_re[2 * h + 1]);
    float2 im = make_float2(acc_im[2 * h], acc_im[2 * h + 1]);
    float2 imb = make_float2(acc_imb[2 * h], acc_imb[2 * h + 1]);
    re = ffma2(vre, cs, re);
    im = ffma2(vre, sn, im);
    re = ffma2(vimn, sn, re);
    imb = ffma2(vimn, cs, imb);
    acc_re[2 * h] = re.x;
    acc_re[2 * h + 1] = re.y;
    acc_im[2 * h] = im.x;
    acc_im[2 * h + 1] = im.y;
    acc_imb[2 * h] = imb.x;
    acc_imb[2 * h + 1] = imb.y;
}

// PU consecutive pulses of the expansion loop, unrolled together so that
// RG x PU x 4 updates per thread are independent (latency hiding for small
// Rx counts).
template <int RG, int PU, bool FD, bool AXIS>
__device__ __forceinline__ void expand_pulses(const BpArgs &a, const float4 *txr, const int4 *txc,
                                              const float4 *rxt, int p,
                                              const float (&dx)[kPxPerThread],
                                              const float (&dy)[kPxPerThread],
                                              const float (&hd2)[kPxPerThread],
                                              const float (&fdi)[kPxPerThread],
                                              float (&acc_re)[kPxPerThread],
                                              float (&acc_im)[kPxPerThread]) {
    constexpr int H = kPxPerThread / 2;
    const int R = a.R;
    const float two_a1 = 2.0f * a.a1f;
    const float2 kap = bcast(a.kappa), nkap = bcast(-a.kappa), kapm = bcast(a.kappa_magic);
    float2 u[PU][H], ay[PU][H], nkk[PU][H];
    float acc_imb[kPxPerThread];
#pragma unroll
    for (int j = 0; j < kPxPerThread; ++j) acc_imb[j] = 0.f;
#pragma unroll
    for (int q = 0; q < PU; ++q) {
        const float4 t4 = txr[p + q];
        const float cidx = __int_as_float(txc[p + q].x);
#pragma unroll
        for (int h = 0; h < H; ++h) {
            float2 y;
            const float2 dt = make_float2(range_delta(t4, dx[2 * h], dy[2 * h], hd2[2 * h], y.x),
                                          range_delta(t4, dx[2 * h + 1], dy[2 * h + 1], hd2[2 * h + 1], y.y));
            // index of the Tx part (twice the Tx range) and, with w = a / 2,
            // a1 (d_rx - d_tx) = w (2 a1 / d - w 2 a1 / d^3)
            const float2 c2 = FD ? make_float2(cidx + fdi[2 * h], cidx + fdi[2 * h + 1]) : bcast(cidx);
            u[q][h] = ffma2(bcast(two_a1), dt, c2);
            ay[q][h] = fmul2(bcast(two_a1), y);
            nkk[q][h] = fmul2(fmul2(bcast(-two_a1), y), fmul2(y, y));
        }
    }
    for (int r0 = 0; r0 < R; r0 += RG) {
#pragma unroll
        for (int q = 0; q < PU; ++q) {
#pragma unroll
            for (int rr = 0; rr < RG; ++rr) {
                const float4 o4 = rxt[(p + q) * R + r0 + rr];
                const uint32_t ac = __float_as_uint(o4.w);
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    // w = a / 2 = (|o|^2/2 - (p - q_tx).o) / 2 (rxt holds halved constants)
                    const float2 dx2 = make_float2(dx[2 * h], dx[2 * h + 1]);
                    const float2 w = AXIS ? ffma2(bcast(o4.x), dx2, bcast(o4.z))
                                          : ffma2(bcast(o4.x), dx2,
                                                  ffma2(bcast(o4.y), make_float2(dy[2 * h], dy[2 * h + 1]),
                                                        bcast(o4.z)));
                    const float2 m1 = ffma2(w, nkk[q][h], ay[q][h]);
                    const float2 idx = ffma2(w, m1, u[q][h]);
                    accumulate2(idx, ac, kap, nkap, kapm, acc_re, acc_im, acc_imb, h);
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kPxPerThread; ++j) acc_im[j] -= acc_imb[j];  // once per PU pulses
}

// Expansion loop over one pulse block (far field, small Rx offsets).  When
// all Rx channels of a pulse fit one group (R == RG), 4 / RG pulses (2 for
// RG >= 3) are processed together; the per-pixel summation order stays pulse
// by pulse.
template <int RG, bool FD, bool AXIS>
__device__ __forceinline__ void compute_block_expand(const BpArgs &a, const Smem &sm, int b, int cslot,
                                                     const float (&dx)[kPxPerThread],
                                                     const float (&dy)[kPxPerThread],
                                                     const float (&hd2)[kPxPerThread],
                                                     const float (&fdi)[kPxPerThread],
                                                     float (&acc_re)[kPxPerThread],
                                                     float (&acc_im)[kPxPerThread]) {
    constexpr int PU = RG >= 3 ? 2 : 4 / RG;
    const int R = a.R, Mb = a.Mb, MbR = Mb * R;
    const int np = min(Mb, a.M - b * Mb);
    const float4 *txr = sm.txr(cslot, Mb);
    const int4 *txc = sm.txc(cslot, Mb);
    const float4 *rxt = sm.rxt(cslot, MbR);
    int p = 0;
    if (PU > 1 && R == RG) {
        for (; p + PU <= np; p += PU)
            expand_pulses<RG, PU, FD, AXIS>(a, txr, txc, rxt, p, dx, dy, hd2, fdi, acc_re, acc_im);
    }
    for (; p < np; ++p)
        expand_pulses<RG, 1, FD, AXIS>(a, txr, txc, rxt, p, dx, dy, hd2, fdi, acc_re, acc_im);
}

// Exact loop over one pulse block: every distance from its own rsqrt and
// Newton step, the index clamped into the staged window.
template <int RG, bool FD>
__device__ __forceinline__ void compute_block_exact(const BpArgs &a, const Smem &sm, int b, int cslot,
                                                    const float (&dx)[kPxPerThread],
                                                    const float (&dy)[kPxPerThread],
                                                    const float (&hd2)[kPxPerThread],
                                                    const float (&fdi)[kPxPerThread],
                                                    float (&acc_re)[kPxPerThread],
                                                    float (&acc_im)[kPxPerThread]) {
    const int R = a.R, Mb = a.Mb, MbR = Mb * R;
    const int np = min(Mb, a.M - b * Mb);
    const float4 *txr = sm.txr(cslot, Mb);
    const float4 *rxr = sm.rxr(cslot, MbR);
    const int4 *pr = sm.pair(cslot, MbR);
    const float a1 = a.a1f;
    const float kap = a.kappa, kapm = a.kappa_magic;
    const float lmax = (float)(a.L - 2);
    for (int p = 0; p < np; ++p) {
        const float4 t4 = txr[p];
        float dt[kPxPerThread];
#pragma unroll
        for (int j = 0; j < kPxPerThread; ++j) {
            float y;
            dt[j] = range_delta(t4, dx[j], dy[j], hd2[j], y);
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
                    float y;
                    const float drx = range_delta(q4, dx[j], dy[j], hd2[j], y);
                    float idx = fmaf(a1, dt[j] + drx, idx0);
                    if (FD) idx += fdi[j];
                    idx = fminf(fmaxf(idx, 0.0f), lmax);
                    accumulate(idx, ac, kap, kapm, acc_re[j], acc_im[j]);
                }
            }
        }
    }
}

// One segment of a CTA's work: pulse blocks [b0, b1) of one tile, from the
// pixel load through the pipeline to the output write.  partial_dst == null:
// the segment covers the whole tile and writes (or adds to) the image;
// otherwise it writes its partial sums there for the fix-up kernel.
// REREAD: the tile record and the output indices are read where they are
// used (the FP64 stage of each block, the output stage) instead of being held
// in registers through the pixel loop (per-request kernel 0.6 % faster, the
// batched class kernel 0.8 % slower on the same frame).
template <int RG, bool FP16, bool FD, bool REREAD = true>
__device__ __forceinline__ void process_segment(const BpArgs &a, const Smem &sm, int tile, int b0, int b1,
                                                float2 *partial_dst) {
    const TileInfo ti_held = REREAD ? TileInfo{} : a.tiles[tile];
    const TileInfo &ti = REREAD ? a.tiles[tile] : ti_held;
    const int *oidx = a.out_idx + (long long)tile * kTilePx + threadIdx.x;
    int oi[kPxPerThread];
#pragma unroll
    for (int j = 0; j < kPxPerThread; ++j) oi[j] = REREAD ? 0 : oidx[j * kBpThreads];
    auto out_index = [&](int j) { return REREAD ? oidx[j * kBpThreads] : oi[j]; };

    float dx[kPxPerThread], dy[kPxPerThread], hd2[kPxPerThread], fdi[kPxPerThread];
    float acc_re[kPxPerThread], acc_im[kPxPerThread];
#pragma unroll
    for (int j = 0; j < kPxPerThread; ++j) {
        const long long slot = (long long)tile * kTilePx + threadIdx.x + j * kBpThreads;
        const float2 d = a.pix[slot];
        dx[j] = d.x;
        dy[j] = d.y;
        hd2[j] = 0.5f * fmaf(d.x, d.x, d.y * d.y);
        fdi[j] = 0.f;
        const int o = FD ? out_index(j) : -1;
        if (FD && o >= 0) {
            // an offset beyond the plan's bound (or not finite) would index
            // outside the staged window: the pixel is left out of this call
            // (its sum is zeroed below) and the call is flagged
            const float f = a.fdopp[o];
            if (fabsf(f) <= a.fd_max)
                fdi[j] = f;
            else
                atomicOr(a.err, kErrDopplerBound);
        }
        acc_re[j] = 0.f;
        acc_im[j] = 0.f;
    }

    // pipeline prologue.  The loop choice of each block (kFlag* bits) is
    // OR-reduced into a shared slot per constant slot and read after the
    // next barrier; slot j is cleared at the end of the iteration that
    // computes its block, before the block three ahead reuses it.
    int *bfl = sm.flags();
    if (threadIdx.x < 3) bfl[threadIdx.x] = 0;
    __syncthreads();
    or_flags(bfl + 0, prep_block(a, sm, ti, b0, 0, 0));
    if (b0 + 1 < b1) or_flags(bfl + 1, prep_block(a, sm, ti, b0 + 1, 1, 1));
    __syncthreads();
    int f_cur = bfl[0];
    int f_next = (b0 + 1 < b1) ? bfl[1] : 0;
    if (f_cur & kFlagExact) {
        prep_exact(a, sm, ti, b0, 0, 0);
        __syncthreads();
    }
    stage_block<FP16>(a, sm, b0, 0, f_cur & kFlagExact);
    cp_async_commit();
    cp_async_wait_all();
    convert_block<FP16>(a, sm, b0, 0, 0, f_cur & kFlagExact);
    __syncthreads();

    for (int b = b0; b < b1; ++b) {
        const int k = b - b0;
        if (b + 2 < b1) or_flags(bfl + (k + 2) % 3, prep_block(a, sm, ti, b + 2, (k + 2) % 3, (k + 2) & 1));
        if (b + 1 < b1 && (f_next & kFlagExact)) {  // block-uniform
            prep_exact(a, sm, ti, b + 1, (k + 1) % 3, (k + 1) & 1);
            __syncthreads();
        }
        if (b + 1 < b1) stage_block<FP16>(a, sm, b + 1, (k + 1) % 3, f_next & kFlagExact);
        cp_async_commit();
        if (f_cur & kFlagExact)
            compute_block_exact<RG, FD>(a, sm, b, k % 3, dx, dy, hd2, fdi, acc_re, acc_im);
        else if (f_cur & kFlagOffAxis)
            compute_block_expand<RG, FD, false>(a, sm, b, k % 3, dx, dy, hd2, fdi, acc_re, acc_im);
        else
            compute_block_expand<RG, FD, true>(a, sm, b, k % 3, dx, dy, hd2, fdi, acc_re, acc_im);
        cp_async_wait_all();
        if (b + 1 < b1) convert_block<FP16>(a, sm, b + 1, (k + 1) % 3, (k + 1) & 1, f_next & kFlagExact);
        if (threadIdx.x == 0) bfl[k % 3] = 0;  // block b's slot, free for block b + 3
        __syncthreads();
        f_cur = f_next;
        f_next = (b + 2 < b1) ? bfl[(k + 2) % 3] : 0;
    }

    if (FD) {
        // the Doppler offset moved the index, not the phase: undo its share
        // exp(sign j 2 pi beta f_doppler) of the per-index phase
#pragma unroll
        for (int j = 0; j < kPxPerThread; ++j) {
            float cyc = a.beta * fdi[j];
            cyc -= rintf(cyc);
            float sn, cs;
            sincospif(-2.0f * a.sign * cyc, &sn, &cs);
            float re = acc_re[j] * cs - acc_im[j] * sn;
            float im = acc_re[j] * sn + acc_im[j] * cs;
            // out-of-bound offset (re-read rather than kept in a register
            // through the pulse loop): no contribution from this call
            const int o = out_index(j);
            if (o >= 0 && !(fabsf(a.fdopp[o]) <= a.fd_max)) re = im = 0.f;
            acc_re[j] = re;
            acc_im[j] = im;
        }
    }

    if (partial_dst == nullptr) {
#pragma unroll
        for (int j = 0; j < kPxPerThread; ++j) {
            const int o = out_index(j);
            if (o < 0) continue;
            float2 v = make_float2(acc_re[j], acc_im[j]);
            if (a.accumulate) {
                const float2 prev = a.image[o];
                v.x += prev.x;
                v.y += prev.y;
            }
            a.image[o] = v;
            if (a.image_out) a.image_out[o] = v;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kPxPerThread; ++j)
            partial_dst[threadIdx.x + j * kBpThreads] = make_float2(acc_re[j], acc_im[j]);
    }
}

// MINB: CTAs per SM the register budget is sized for (2: 128 registers and
// more independent updates per thread; 3: 80 registers and more warps).
template <int RG, bool FP16, bool FD, int MINB>
__global__ void __launch_bounds__(kBpThreads, MINB) backproject_kernel(BpArgs a) {
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
        float2 *dst = nullptr;
        if (!(b0 == 0 && b1 == PB))
            dst = a.partial + ((long long)blockIdx.x * a.seg_max + (tile - t_first)) * kTilePx;
        process_segment<RG, FP16, FD>(a, sm, tile, b0, b1, dst);
        u += b1 - b0;
    }
}

// Batched form: the (request, tile, pulse block) units of several requests,
// each with its own plan, profiles, trajectory and image.  The requests are
// grouped into classes that share an Rx group and a profile storage (the
// pixel loop is specialised on both); ONE persistent launch runs every class:
// CTAs [cta_begin, cta_begin + G) of the grid belong to class c and split its
// concatenated units into equal contiguous ranges.  Only the first and the
// last segment of a CTA's range can cover part of a tile, so each CTA owns two
// partial-sum slots (0: first segment, 1: last segment).
// Records the first failed check of a batched launch (code and three values);
// the caller then skips the access.  Conditions are CTA-uniform.
__device__ __forceinline__ void batch_fail(int *err, int code, long long x, long long y, long long z) {
    if (threadIdx.x == 0 && err && atomicCAS(err, 0, code) == 0) {
        err[1] = (int)x;
        err[2] = (int)y;
        err[3] = (int)z;
    }
}

// PARAM: `jobs` points into the kernel's parameter table (read in place from
// the constant bank, as a single request's arguments are); otherwise at the
// device table (each segment takes a private copy).
template <int RG, bool FP16, bool PARAM>
__device__ __forceinline__ void run_class(const BpCheck &M, const BpClassArgs &B, const BpArgs *jobs, int cta,
                                          float2 *scratch, uint32_t smem_addr, unsigned char *smem_base) {
    Smem sm;
    sm.base = smem_base;
    sm.base_addr = smem_addr;
    if (!(cta >= 0 && cta < B.G && B.units > 0 && B.n_jobs > 0 && (!PARAM || B.n_jobs <= kParamJobs))) {
        batch_fail(M.err, 1, cta, B.G, B.units);
        return;
    }
    const long long u0 = (long long)cta * B.units / B.G;
    const long long u1 = (long long)(cta + 1) * B.units / B.G;
    // job holding u0: the last j with unit_begin[j] <= u0
    int lo = 0, hi = B.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.unit_begin[mid] <= u0) lo = mid; else hi = mid - 1;
    }
    int j = lo;
    long long u = u0;
    // units [u, ...) of job j with arguments a: one segment; returns the units
    // processed, -1 after a failed check
    auto segment = [&](const BpArgs &a) -> long long {
        sm.lay = bp_layout(a.Mb, a.R, a.L, FP16);
        if (!(a.Mb >= 1 && a.Mb <= 32 && sm.lay.total <= M.smem_bytes && a.R == B.rg * (a.R / B.rg) &&
              a.fp16 == (FP16 ? 1 : 0))) {
            batch_fail(M.err, 3, a.Mb, sm.lay.total, M.smem_bytes);
            return -1;
        }
        const long long v = u - B.unit_begin[j];
        const int PB = a.blocks_per_tile;
        const int tile = (int)(v / PB);
        const int b0 = (int)(v - (long long)tile * PB);
        const int b1 = (int)min((long long)PB, (long long)b0 + (u1 - u));
        if (!(PB == (a.M + a.Mb - 1) / a.Mb && tile >= 0 && tile < a.n_tiles && b0 >= 0 && b0 < b1 && b1 <= PB)) {
            batch_fail(M.err, 4, tile, b0, b1);
            return -1;
        }
        float2 *dst = nullptr;
        if (!(b0 == 0 && b1 == PB)) {
            if (!((long long)(B.cta_begin + cta) * 2 + 1 < M.scratch_slots)) {
                batch_fail(M.err, 5, B.cta_begin + cta, M.scratch_slots, 0);
                return -1;
            }
            dst = scratch + (u == u0 ? 0 : kTilePx);
        }
        process_segment<RG, FP16, false, false>(a, sm, tile, b0, b1, dst);
        return (long long)(b1 - b0);
    };
    while (u < u1) {
        while (j + 1 < B.n_jobs && u >= B.unit_begin[j + 1]) ++j;
        if (!(u >= B.unit_begin[j] && u < B.unit_begin[j + 1])) {
            batch_fail(M.err, 2, u, j, B.n_jobs);
            return;
        }
        long long done;
        if constexpr (PARAM) {
            done = segment(jobs[j]);
        } else {
            // a private copy of the job's arguments (a few bytes of it spill).
            // Read in place from global or shared memory instead, every field
            // access after a copy's or load's memory clobber becomes a load:
            // 3-10 % slower per class through a restricted global reference,
            // 2-11 % from a shared-memory copy.
            const BpArgs a = jobs[j];
            done = segment(a);
        }
        if (done < 0) return;
        u += done;
    }
}

// One class of the batch: its own specialised kernel on the whole grid; the
// batch launches its classes one after another.  CTA i of the class owns
// partial-sum slots 2 (cta_begin + i) and 2 (cta_begin + i) + 1.
template <int RG, bool FP16>
__global__ void __launch_bounds__(kBpThreads, 2) backproject_class_kernel(BpClassArgs B, BpCheck chk) {
    extern __shared__ __align__(16) unsigned char smem_bp[];
    const uint32_t smem_addr = (uint32_t)__cvta_generic_to_shared(smem_bp);
    float2 *scratch = chk.scratch + ((long long)B.cta_begin + blockIdx.x) * 2 * kTilePx;
    run_class<RG, FP16, false>(chk, B, B.jobs, (int)blockIdx.x, scratch, smem_addr, smem_bp);
}

// The same with the class's jobs (at most kParamJobs) as a kernel parameter.
template <int RG, bool FP16>
__global__ void __launch_bounds__(kBpThreads, 2)
    backproject_class_param_kernel(BpClassArgs B, BpCheck chk, const __grid_constant__ BpJobTable T) {
    extern __shared__ __align__(16) unsigned char smem_bp[];
    const uint32_t smem_addr = (uint32_t)__cvta_generic_to_shared(smem_bp);
    float2 *scratch = chk.scratch + ((long long)B.cta_begin + blockIdx.x) * 2 * kTilePx;
    run_class<RG, FP16, true>(chk, B, T.jobs, (int)blockIdx.x, scratch, smem_addr, smem_bp);
}

// Fix-up of the batched form: one CTA per tile of every request of every
// class; the split tile's partial sums are added in CTA order.
__global__ void __launch_bounds__(kFixupThreads) bp_batch_fixup_kernel(BpMultiArgs M, BpCheck chk) {
    const int gt = blockIdx.x;
    int c = 0;
    while (c + 1 < M.n_classes && gt >= M.cls[c + 1].tile_base) ++c;
    const BpClassArgs &B = M.cls[c];
    const int ct = gt - B.tile_base;
    int lo = 0, hi = B.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (B.tile_begin[mid] <= ct) lo = mid; else hi = mid - 1;
    }
    const BpArgs &a = B.jobs[lo];
    const int tile = ct - B.tile_begin[lo];
    const long long PB = a.blocks_per_tile;
    const long long tb = B.unit_begin[lo] + (long long)tile * PB;
    const long long te = tb + PB;
    if (!(ct >= 0 && ct < B.tile_begin[B.n_jobs] && tile >= 0 && tile < a.n_tiles && te <= B.unit_begin[lo + 1])) {
        batch_fail(chk.err, 6, ct, lo, tile);
        return;
    }
    const int ia = (int)(((tb + 1) * B.G - 1) / B.units);
    const int ib = (int)((te * B.G - 1) / B.units);
    if (ia == ib) return;
    if (!(ia >= 0 && ib < B.G && ((long long)B.cta_begin + ib) * 2 + 1 < chk.scratch_slots)) {
        batch_fail(chk.err, 7, ia, ib, B.cta_begin);
        return;
    }
    float2 acc[kFixupPx];
#pragma unroll
    for (int k = 0; k < kFixupPx; ++k) acc[k] = make_float2(0.f, 0.f);
    for (int i = ia; i <= ib; ++i) {  // CTA order; one slot lookup per CTA
        const long long ui0 = (long long)i * B.units / B.G;
        const float2 *part = chk.scratch + ((long long)(B.cta_begin + i) * 2 + (ui0 >= tb ? 0 : 1)) * kTilePx;
#pragma unroll
        for (int k = 0; k < kFixupPx; ++k) {
            const float2 v = part[threadIdx.x + k * kFixupThreads];
            acc[k].x += v.x;
            acc[k].y += v.y;
        }
    }
#pragma unroll
    for (int k = 0; k < kFixupPx; ++k) {
        const int o = a.out_idx[(long long)tile * kTilePx + threadIdx.x + k * kFixupThreads];
        if (o < 0) continue;
        float2 v = acc[k];
        if (a.accumulate) {
            const float2 old = a.image[o];
            v.x += old.x;
            v.y += old.y;
        }
        a.image[o] = v;
        if (a.image_out) a.image_out[o] = v;
    }
}

// Sums, in CTA order, the partial sums of tiles that were split across CTAs.
__global__ void __launch_bounds__(kFixupThreads) bp_fixup_kernel(BpArgs a) {
    const int tile = blockIdx.x;
    const long long PB = a.blocks_per_tile;
    const long long ua = (long long)tile * PB;
    const long long ub = ua + PB - 1;
    const int ia = (int)(((ua + 1) * a.G - 1) / a.units);
    const int ib = (int)(((ub + 1) * a.G - 1) / a.units);
    if (ia == ib) return;
    float2 acc[kFixupPx];
#pragma unroll
    for (int k = 0; k < kFixupPx; ++k) acc[k] = make_float2(0.f, 0.f);
    for (int i = ia; i <= ib; ++i) {  // CTA order; one slot lookup per CTA
        const long long ui0 = (long long)i * a.units / a.G;
        const float2 *part = a.partial + ((long long)i * a.seg_max + (tile - (int)(ui0 / PB))) * kTilePx;
#pragma unroll
        for (int k = 0; k < kFixupPx; ++k) {
            const float2 v = part[threadIdx.x + k * kFixupThreads];
            acc[k].x += v.x;
            acc[k].y += v.y;
        }
    }
#pragma unroll
    for (int k = 0; k < kFixupPx; ++k) {
        const int o = a.out_idx[(long long)tile * kTilePx + threadIdx.x + k * kFixupThreads];
        if (o < 0) continue;
        float2 v = acc[k];
        if (a.accumulate) {
            const float2 old = a.image[o];
            v.x += old.x;
            v.y += old.y;
        }
        a.image[o] = v;
        if (a.image_out) a.image_out[o] = v;
    }
}

template <int RG, bool FP16, bool FD>
void *kernel_ptr(int minb) {
    return minb == 3 ? (void *)backproject_kernel<RG, FP16, FD, 3> : (void *)backproject_kernel<RG, FP16, FD, 2>;
}

void *select_kernel(int rg, bool fp16, bool fd, int minb) {
#define SAR_SEL(RGV)                                                                                    \
    if (rg == RGV) {                                                                                    \
        if (fp16) return fd ? kernel_ptr<RGV, true, true>(minb) : kernel_ptr<RGV, true, false>(minb); \
        return fd ? kernel_ptr<RGV, false, true>(minb) : kernel_ptr<RGV, false, false>(minb);         \
    }
    SAR_SEL(1)
    SAR_SEL(2)
    SAR_SEL(3)
    SAR_SEL(4)
#undef SAR_SEL
    return nullptr;
}

}  // namespace

size_t bp_smem_bytes(int Mb, int R, int L, bool fp16) { return bp_layout(Mb, R, L, fp16).total; }

// The dynamic shared-memory limit is a per-kernel, process-wide attribute:
// plans (and batches) of different sizes share the kernels, so it is raised
// once to the largest size any of them may use, never lowered: 227 KB less
// the kernel's static shared memory.
constexpr int kSmemLimit = 227 * 1024;

// Raise kernel k's dynamic shared-memory limit; *max_dyn receives it.
cudaError_t raise_smem_limit(const void *k, size_t *max_dyn) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    if (fa.sharedSizeBytes >= (size_t)kSmemLimit) return cudaErrorInvalidValue;
    *max_dyn = (size_t)kSmemLimit - fa.sharedSizeBytes;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*max_dyn);
}

cudaError_t bp_prepare(bool fp16, int rg, size_t smem) {
    if (smem > (size_t)kSmemLimit) return cudaErrorInvalidValue;
    for (int fd = 0; fd < 2; ++fd)
        for (int minb = 2; minb <= 3; ++minb) {
            void *k = select_kernel(rg, fp16, fd != 0, minb);
            if (!k) return cudaErrorInvalidValue;
            size_t max_dyn = 0;
            cudaError_t e = raise_smem_limit(k, &max_dyn);
            if (e != cudaSuccess) return e;
            if (smem > max_dyn) return cudaErrorInvalidValue;
        }
    return cudaSuccess;
}

int bp_occupancy(bool fp16, int rg, size_t smem, int minb, int *ctas_per_sm) {
    void *k = select_kernel(rg, fp16, false, minb);
    if (!k) return -1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kBpThreads, smem) != cudaSuccess) return -1;
    *ctas_per_sm = n;
    return 0;
}

namespace {

void *select_class_kernel(int rg, bool fp16, bool param) {
#define SAR_SELB(RGV)                                                                      \
    if (rg == RGV) {                                                                       \
        if (param)                                                                         \
            return fp16 ? (void *)backproject_class_param_kernel<RGV, true>                \
                        : (void *)backproject_class_param_kernel<RGV, false>;              \
        return fp16 ? (void *)backproject_class_kernel<RGV, true>                          \
                    : (void *)backproject_class_kernel<RGV, false>;                        \
    }
    SAR_SELB(1)
    SAR_SELB(2)
    SAR_SELB(3)
    SAR_SELB(4)
#undef SAR_SELB
    return nullptr;
}

}  // namespace

// Both variants of the class kernel (job arguments from the device table or
// from the parameters); the occupancy reported is the lower of the two.
cudaError_t bp_batch_prepare(int rg, bool fp16, size_t smem, int *ctas_per_sm) {
    if (smem > (size_t)kSmemLimit) return cudaErrorInvalidValue;
    int occ = 1 << 30;
    for (int param = 0; param < 2; ++param) {
        void *k = select_class_kernel(rg, fp16, param != 0);
        if (!k) return cudaErrorInvalidValue;
        size_t max_dyn = 0;
        cudaError_t e = raise_smem_limit(k, &max_dyn);
        if (e != cudaSuccess) return e;
        if (smem > max_dyn) return cudaErrorInvalidValue;
        int n = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kBpThreads, smem);
        if (e != cudaSuccess) return e;
        occ = std::min(occ, n);
    }
    *ctas_per_sm = occ;
    return cudaSuccess;
}

cudaError_t launch_backproject_class(const BpClassArgs &c, const BpCheck &chk, size_t smem, cudaStream_t s,
                                     const BpArgs *host_jobs) {
    if (c.G == 0 || c.units == 0) return cudaSuccess;
    const bool param = host_jobs != nullptr && c.n_jobs >= 1 && c.n_jobs <= kParamJobs;
    void *k = select_class_kernel(c.rg, c.fp16 != 0, param);
    if (!k) return cudaErrorInvalidValue;
    BpClassArgs a = c;
    BpCheck b = chk;
    if (!param) {
        void *params[] = {&a, &b};
        return cudaLaunchKernel(k, dim3(c.G), dim3(kBpThreads), params, smem, s);
    }
    // the parameter block is copied at launch (and into a captured graph)
    static thread_local BpJobTable table;
    std::memset(&table, 0, sizeof(table));
    std::memcpy(table.jobs, host_jobs, sizeof(BpArgs) * (size_t)c.n_jobs);
    void *params[] = {&a, &b, &table};
    return cudaLaunchKernel(k, dim3(c.G), dim3(kBpThreads), params, smem, s);
}

cudaError_t launch_batch_fixup(const BpMultiArgs &m, const BpCheck &chk, int total_tiles, cudaStream_t s) {
    if (m.n_classes == 0 || total_tiles == 0) return cudaSuccess;
    bp_batch_fixup_kernel<<<total_tiles, kFixupThreads, 0, s>>>(m, chk);
    return cudaGetLastError();
}

cudaError_t launch_backproject(const BpArgs &a, const BpLaunch &l, cudaStream_t s) {
    void *k = select_kernel(l.rg, l.fp16, a.fdopp != nullptr, l.minb);
    if (!k) return cudaErrorInvalidValue;
    if (a.units == 0) return cudaSuccess;
    BpArgs args = a;
    void *params[] = {&args};
    cudaError_t e = cudaLaunchKernel(k, dim3(a.G), dim3(kBpThreads), params, l.smem, s);
    if (e != cudaSuccess) return e;
    bp_fixup_kernel<<<a.n_tiles, kFixupThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace sar
