/*
 * FP64 CPU oracle for FMCW range compression and time-domain backprojection
 * ("Implementation of Real-Time Automotive SAR Imaging", arXiv 2306.09784).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct reference code.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
 * reference legs may load or call it.  The CUDA library never does, and this
 * file shares no code, header, table or constant with it.
 *
 * Conventions (readings where the paper is silent or garbled):
 *  - complex arrays are interleaved (re, im) doubles;
 *  - 2-D geometry (Sec. II: "2D distance"); positions are (x, y) pairs;
 *  - `sign` = +1 selects the +j range-transform kernel and the phase
 *    correction exp(+j 2 pi f0 d / c); -1 gives the conjugate convention;
 *  - a backprojection term whose interpolation base bin i0 = floor(index)
 *    lies outside [crop_lo, crop_hi) contributes nothing (the default range
 *    is [0, N_fft - 1), i.e. both interpolation samples must exist).
 *
 * Every function below is pinned by the -m "not gpu" tests (closed forms,
 * brute force, invariants, planted mutations).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define API __attribute__((visibility("default")))

static const double PI = 3.14159265358979323846264338327950288;

API int oracle_version(void) { return 1; }

API int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void set_threads(int threads) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
}

/* Modified Bessel function I0 by its power series sum_k ((x/2)^k / k!)^2. */
static double bessel_i0(double x) {
    double term = 1.0, sum = 1.0, h = 0.5 * x;
    for (int k = 1; k < 500; ++k) {
        term *= h / k;
        double t2 = term * term;
        sum += t2;
        if (t2 < 1e-18 * sum) break;
    }
    return sum;
}

/*
 * Window weights of length L.  kind 0: rectangular; 1: symmetric Hann
 * 0.5 - 0.5 cos(2 pi n / (L - 1)) (Sec. II names Hann for w_sar);
 * 2: Kaiser I0(beta sqrt(1 - (2n/(L-1) - 1)^2)) / I0(beta) (Sec. III-B).
 */
API int oracle_window(int kind, int L, double beta, double *w) {
    if (L <= 0 || !w) return -1;
    for (int n = 0; n < L; ++n) {
        if (kind == 0 || L == 1) {
            w[n] = 1.0;
        } else if (kind == 1) {
            w[n] = 0.5 - 0.5 * cos(2.0 * PI * n / (L - 1));
        } else if (kind == 2) {
            double r = 2.0 * n / (L - 1) - 1.0;
            double a = 1.0 - r * r;
            w[n] = bessel_i0(beta * sqrt(a > 0 ? a : 0.0)) / bessel_i0(beta);
        } else {
            return -1;
        }
    }
    return 0;
}

/* Textbook DFT: X[k] = sum_{n < n_in} x[n] exp(sign j 2 pi n k / n_out). */
API int oracle_dft(int n_in, const double *x, int n_out, int sign, double *X) {
    if (n_in <= 0 || n_out <= 0) return -1;
    for (int k = 0; k < n_out; ++k) {
        double sr = 0.0, si = 0.0;
        for (int n = 0; n < n_in; ++n) {
            /* reduce n k modulo n_out exactly in integers before the angle */
            long long nk = ((long long)n * k) % n_out;
            double ang = sign * 2.0 * PI * (double)nk / n_out;
            double c = cos(ang), s = sin(ang);
            double xr = x[2 * n], xi = x[2 * n + 1];
            sr += xr * c - xi * s;
            si += xr * s + xi * c;
        }
        X[2 * k] = sr;
        X[2 * k + 1] = si;
    }
    return 0;
}

/*
 * In-place iterative radix-2 FFT (bit-reversal permutation, then log2(n)
 * butterfly stages), X[k] = sum_n x[n] exp(sign j 2 pi n k / n); n a power
 * of two.  Twiddles come from cos/sin of 2 pi t / n directly.
 */
API int oracle_fft(int n, double *x, int sign) {
    if (n <= 0 || (n & (n - 1))) return -1;
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double tr = x[2 * i], ti = x[2 * i + 1];
            x[2 * i] = x[2 * j]; x[2 * i + 1] = x[2 * j + 1];
            x[2 * j] = tr; x[2 * j + 1] = ti;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int t = 0; t < half; ++t) {
            double ang = sign * 2.0 * PI * t / len;
            double wr = cos(ang), wi = sin(ang);
            for (int s = 0; s < n; s += len) {
                int a = s + t, b = s + t + half;
                double br = x[2 * b] * wr - x[2 * b + 1] * wi;
                double bi = x[2 * b] * wi + x[2 * b + 1] * wr;
                x[2 * b] = x[2 * a] - br; x[2 * b + 1] = x[2 * a + 1] - bi;
                x[2 * a] += br; x[2 * a + 1] += bi;
            }
        }
    }
    return 0;
}

/*
 * Range compression of every (chirp m, Rx r) row of the beat cube
 * beat[M][R][N]: window by w_r[n], zero-pad to N_fft = os * N and transform,
 * S[m][r][k] = sum_{n < N} w_r[n] beat[m][r][n] exp(sign j 2 pi (n - t0) k / N_fft)
 * for k < N_fft.  The paper interpolates the beat spectrum "at f_hyp"
 * (Alg. 1) on an equidistant beat-frequency axis (Sec. III-C) without saying
 * how it is made; this is the windowed, zero-padded DFT of each chirp.
 * t0 is the transform's time origin in samples: 0 (the chirp's first sample,
 * the default reading of Sec. II's f0) or (N - 1) / 2 (the chirp centre).
 * The transform is computed for n and then moved to n - t0 by the shift
 * theorem, one rotation exp(-sign j 2 pi t0 k / N_fft) per bin.
 */
API int oracle_range_compress(int N, int os, int M, int R, const double *beat,
                              const double *w_r, int sign, double t0, double *S,
                              int threads) {
    if (N <= 0 || os <= 0 || M < 0 || R <= 0) return -1;
    int nfft = N * os;
    if (nfft & (nfft - 1)) return -1;
    set_threads(threads);
    long long rows = (long long)M * R;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : err)
    for (long long row = 0; row < rows; ++row) {
        double *out = S + 2LL * nfft * row;
        const double *in = beat + 2LL * N * row;
        memset(out, 0, sizeof(double) * 2 * (size_t)nfft);
        for (int n = 0; n < N; ++n) {
            out[2 * n] = w_r[n] * in[2 * n];
            out[2 * n + 1] = w_r[n] * in[2 * n + 1];
        }
        err |= oracle_fft(nfft, out, sign);
        if (t0 != 0.0) {
            for (int k = 0; k < nfft; ++k) {
                const double ang = -sign * 2.0 * PI * t0 * k / nfft;
                const double cr = cos(ang), ci = sin(ang);
                const double re = out[2 * k], im = out[2 * k + 1];
                out[2 * k] = re * cr - im * ci;
                out[2 * k + 1] = re * ci + im * cr;
            }
        }
    }
    return err ? -1 : 0;
}

/*
 * Linear interpolation of the spectrum row `s` (n_fft bins) at fractional
 * bin `index` (Sec. III-C: the beat-frequency axis is equidistant, so the
 * index is computed directly).  Returns 0 and leaves v untouched when the base
 * bin is outside [crop_lo, crop_hi).
 */
static int interp(const double *s, double index, int crop_lo, int crop_hi,
                  double *vr, double *vi) {
    double fl = floor(index);
    if (!(fl >= crop_lo && fl < crop_hi)) return 0;
    long long i0 = (long long)fl;
    double f = index - fl;
    *vr = (1.0 - f) * s[2 * i0] + f * s[2 * i0 + 2];
    *vi = (1.0 - f) * s[2 * i0 + 1] + f * s[2 * i0 + 3];
    return 1;
}

/*
 * Optimised backprojection, Alg. 2 (Sec. IV), for the pixel list px[P][2]:
 *   for every pixel p, chirp m:  d_tx = ||p - q_tx(m)||
 *     for every Rx n:  d_rx = ||p - q_rx(m, n)||,  d_hyp = d_tx + d_rx
 *       f_ind = a1 d_hyp + f_doppler(p)          a1 = mu N_fft / (c fs)
 *       s_hyp = exp(a2 d_hyp)                     a2 = sign j 2 pi f0 / c
 *       P(p) += s_hyp * s(f_ind, m, n) * w_sar(m)
 * s(., m, n) is row (m, n) of S[M][R][n_fft], linearly interpolated.
 * fd_idx may be NULL (f_doppler = 0); w_az may be NULL (all ones).
 * out[P] is complex (interleaved).
 */
API int oracle_backproject(double f0, double slope, double fs, double c, int n_fft,
                           int sign, int crop_lo, int crop_hi, int M, int R,
                           const double *S, const double *q_tx, const double *q_rx,
                           const double *w_az, const double *fd_idx, int P,
                           const double *px, double *out, int threads) {
    if (n_fft <= 1 || M < 0 || R <= 0 || P < 0) return -1;
    if (crop_lo < 0) crop_lo = 0;
    if (crop_hi > n_fft - 1) crop_hi = n_fft - 1;
    const double a1 = slope * n_fft / (c * fs);
    const double a2 = sign * 2.0 * PI * f0 / c;
    set_threads(threads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int p = 0; p < P; ++p) {
        const double x = px[2 * p], y = px[2 * p + 1];
        const double fd = fd_idx ? fd_idx[p] : 0.0;
        double ar = 0.0, ai = 0.0;
        for (int m = 0; m < M; ++m) {
            const double d_tx = hypot(x - q_tx[2 * m], y - q_tx[2 * m + 1]);
            const double w = w_az ? w_az[m] : 1.0;
            for (int n = 0; n < R; ++n) {
                const double *qr = q_rx + 2 * ((long long)m * R + n);
                const double d_rx = hypot(x - qr[0], y - qr[1]);
                const double d_hyp = d_tx + d_rx;
                const double f_ind = a1 * d_hyp + fd;
                double vr, vi;
                const double *row = S + 2LL * n_fft * ((long long)m * R + n);
                if (!interp(row, f_ind, crop_lo, crop_hi, &vr, &vi)) continue;
                const double ph = a2 * d_hyp;
                const double hr = cos(ph), hi = sin(ph);
                ar += w * (hr * vr - hi * vi);
                ai += w * (hr * vi + hi * vr);
            }
        }
        out[2 * p] = ar;
        out[2 * p + 1] = ai;
    }
    return 0;
}

/*
 * Standard backprojection, Alg. 1 (Sec. II), with per-chirp velocity vel[M][2]
 * (NULL = zero velocity):
 *   v_tx = <p - q_tx, v(m)> / d_tx,  v_rx = <p - q_rx, v(m)> / d_rx
 *   tau  = (d_tx + d_rx) / c
 *   f_hyp = mu tau + f0 (v_tx + v_rx) / c
 *   s_hyp = exp(sign j 2 pi f0 tau)       (the printed s_hyp lacks f0;
 *                                           the phase of a delay tau is 2 pi f0 tau)
 *   P(p) += s_hyp * s(f_hyp) * w_sar(m)
 * The spectrum is sampled on the beat-frequency axis f_k = k fs / N_fft, so
 * s(f_hyp) is the linear interpolation at bin f_hyp N_fft / fs.
 */
API int oracle_backproject_alg1(double f0, double slope, double fs, double c, int n_fft,
                                int sign, int crop_lo, int crop_hi, int M, int R,
                                const double *S, const double *q_tx, const double *q_rx,
                                const double *vel, const double *w_az, int P,
                                const double *px, double *out, int threads) {
    if (n_fft <= 1 || M < 0 || R <= 0 || P < 0) return -1;
    if (crop_lo < 0) crop_lo = 0;
    if (crop_hi > n_fft - 1) crop_hi = n_fft - 1;
    set_threads(threads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int p = 0; p < P; ++p) {
        const double x = px[2 * p], y = px[2 * p + 1];
        double ar = 0.0, ai = 0.0;
        for (int m = 0; m < M; ++m) {
            const double ex = x - q_tx[2 * m], ey = y - q_tx[2 * m + 1];
            const double d_tx = hypot(ex, ey);
            const double vx = vel ? vel[2 * m] : 0.0, vy = vel ? vel[2 * m + 1] : 0.0;
            const double v_tx = (ex * vx + ey * vy) / d_tx;
            const double w = w_az ? w_az[m] : 1.0;
            for (int n = 0; n < R; ++n) {
                const double *qr = q_rx + 2 * ((long long)m * R + n);
                const double rx = x - qr[0], ry = y - qr[1];
                const double d_rx = hypot(rx, ry);
                const double v_rx = (rx * vx + ry * vy) / d_rx;
                const double tau = (d_tx + d_rx) / c;
                const double f_hyp = slope * tau + f0 * (v_tx + v_rx) / c;
                const double bin = f_hyp * n_fft / fs;
                double vr, vi;
                const double *row = S + 2LL * n_fft * ((long long)m * R + n);
                if (!interp(row, bin, crop_lo, crop_hi, &vr, &vi)) continue;
                const double ph = sign * 2.0 * PI * f0 * tau;
                const double hr = cos(ph), hi = sin(ph);
                ar += w * (hr * vr - hi * vi);
                ai += w * (hr * vi + hi * vr);
            }
        }
        out[2 * p] = ar;
        out[2 * p + 1] = ai;
    }
    return 0;
}

/*
 * Brute-force matched filter: the band-limited limit of "range transform +
 * linear interpolation".  The windowed beat row is correlated directly at the
 * pixel's fractional beat frequency mu d_hyp / c (no transform, no
 * interpolation):
 *   P_bf(p) = sum_m sum_n w_sar(m) exp(sign j 2 pi f0 d/c)
 *             sum_k w_r[k] beat[m][n][k] exp(sign j 2 pi mu d k / (c fs))
 */
API int oracle_matched_filter(double f0, double slope, double fs, double c, int sign,
                              int N, int M, int R, const double *beat, const double *w_r,
                              const double *q_tx, const double *q_rx, const double *w_az,
                              int P, const double *px, double *out, int threads) {
    if (N <= 0 || M < 0 || R <= 0 || P < 0) return -1;
    set_threads(threads);
#pragma omp parallel for schedule(dynamic, 4)
    for (int p = 0; p < P; ++p) {
        const double x = px[2 * p], y = px[2 * p + 1];
        double ar = 0.0, ai = 0.0;
        for (int m = 0; m < M; ++m) {
            const double d_tx = hypot(x - q_tx[2 * m], y - q_tx[2 * m + 1]);
            const double w = w_az ? w_az[m] : 1.0;
            for (int n = 0; n < R; ++n) {
                const double *qr = q_rx + 2 * ((long long)m * R + n);
                const double d = d_tx + hypot(x - qr[0], y - qr[1]);
                const double *row = beat + 2LL * N * ((long long)m * R + n);
                const double cyc = slope * d / (c * fs); /* cycles per sample */
                double sr = 0.0, si = 0.0;
                for (int k = 0; k < N; ++k) {
                    double t = cyc * k;
                    t -= floor(t);
                    const double ang = sign * 2.0 * PI * t;
                    const double cr = cos(ang), ci = sin(ang);
                    const double br = w_r[k] * row[2 * k], bi = w_r[k] * row[2 * k + 1];
                    sr += br * cr - bi * ci;
                    si += br * ci + bi * cr;
                }
                double ph = f0 * d / c;
                ph -= floor(ph);
                ph *= sign * 2.0 * PI;
                const double hr = cos(ph), hi = sin(ph);
                ar += w * (hr * sr - hi * si);
                ai += w * (hr * si + hi * sr);
            }
        }
        out[2 * p] = ar;
        out[2 * p + 1] = ai;
    }
    return 0;
}

/*
 * Polar reconstruction grid (Sec. III-E, Fig. 2).  The grid originates in the
 * centre of the synthetic aperture; its spacing is the radar's resolution
 * divided by `factor` (the paper uses 2.5).  The paper takes the resolution
 * from a point spread function it does not print; the textbook values stand
 * in for it:
 *   range:   dr = c / (2 B), B = |slope| N / fs the swept bandwidth;
 *   azimuth: lambda r / (2 L) at range r, i.e. the angle dphi = lambda / (2 L),
 *            lambda = c / f_c at the sweep's centre frequency
 *            f_c = f0 + slope N / (2 fs), L = |q_tx(M-1) - q_tx(0)|.
 * With centre o = (q_tx(0) + q_tx(M-1)) / 2, along-track unit vector
 * u = (q_tx(M-1) - q_tx(0)) / L and its left normal v = (-u_y, u_x), the
 * grid points are
 *   o + (k Dr) (cos(j Dphi) u + sin(j Dphi) v),  Dr = dr / factor,
 *   Dphi = dphi / factor,  integers k >= 1 and j with j Dphi in [-pi, pi),
 * and the ones kept lie in the box [x_min, x_max] x [y_min, y_max] (borders
 * included), listed by ring k, then by angle j, both ascending.
 * Every (k, j) pair is visited (plain enumeration).  out_xy may be NULL (count
 * only); otherwise at most `capacity` points are written.  *n_out receives
 * the number of grid points in the box.  Returns -1 for invalid input.
 */
API int oracle_polar_grid(double f0, double slope, double fs, double c, int N, int M,
                          const double *q_tx, double x_min, double x_max, double y_min,
                          double y_max, double factor, long long capacity, double *out_xy,
                          long long *n_out) {
    if (N <= 0 || M < 2 || !(factor > 0) || !(x_max >= x_min) || !(y_max >= y_min) || !n_out)
        return -1;
    const double ax = q_tx[2 * (M - 1)] - q_tx[0], ay = q_tx[2 * (M - 1) + 1] - q_tx[1];
    const double L = hypot(ax, ay);
    if (!(L > 0)) return -1;
    const double ux = ax / L, uy = ay / L;
    const double vx = -uy, vy = ux;
    const double ox = 0.5 * (q_tx[0] + q_tx[2 * (M - 1)]);
    const double oy = 0.5 * (q_tx[1] + q_tx[2 * (M - 1) + 1]);
    const double B = fabs(slope) * N / fs;
    const double fc = f0 + slope * N / (2.0 * fs);
    const double dr = c / (2.0 * B) / factor;
    const double dphi = (c / fc) / (2.0 * L) / factor;
    /* the farthest box corner bounds the rings */
    double rmax = 0.0;
    const double cx[4] = {x_min, x_max, x_min, x_max}, cy[4] = {y_min, y_min, y_max, y_max};
    for (int i = 0; i < 4; ++i) {
        const double d = hypot(cx[i] - ox, cy[i] - oy);
        if (d > rmax) rmax = d;
    }
    const long long kmax = (long long)floor(rmax / dr) + 1;
    const long long jlo = (long long)ceil(-PI / dphi), jhi = (long long)ceil(PI / dphi) - 1;
    long long n = 0;
    for (long long k = 1; k <= kmax; ++k) {
        const double r = k * dr;
        for (long long j = jlo; j <= jhi; ++j) {
            const double phi = j * dphi;
            const double cs = cos(phi), sn = sin(phi);
            const double x = ox + r * (cs * ux + sn * vx);
            const double y = oy + r * (cs * uy + sn * vy);
            if (x >= x_min && x <= x_max && y >= y_min && y <= y_max) {
                if (out_xy && n < capacity) {
                    out_xy[2 * n] = x;
                    out_xy[2 * n + 1] = y;
                }
                ++n;
            }
        }
    }
    *n_out = n;
    return 0;
}

/*
 * Per-pixel Doppler index offsets f_doppler(p) of Alg. 2 (Sec. III-D): the
 * radial velocity terms of Alg. 1 (lines 5, 8, 9, 11) evaluated once per pixel
 * with the average vehicle velocity and the aperture's mean antenna
 * positions instead of per chirp and antenna:
 *   vbar = mean_m vel(m),  qt = mean_m q_tx(m),  qr = mean_{m,n} q_rx(m, n),
 *   ddot(p) = -( <p - qt, vbar> / ||p - qt|| + <p - qr, vbar> / ||p - qr|| ),
 *   f_doppler(p) = f0 ddot(p) / c * n_fft / fs   [bins].
 * ddot is the rate of change of the two-way path d_tx + d_rx for a platform
 * moving with vbar; under the beat model Rx conj(Tx) with the +j transform
 * (the reading this oracle follows throughout) it shifts a target's beat
 * frequency by f0 ddot / c, which is Alg. 1's f0 v / c with v the scene's
 * velocity relative to the radar.  f0 is the carrier at the transform's time
 * origin.  vel is the platform velocity per chirp [M][2].
 */
API int oracle_doppler_offsets(double f0, double fs, double c, int n_fft, int M, int R,
                               const double *q_tx, const double *q_rx, const double *vel,
                               int P, const double *px, double *out) {
    if (M <= 0 || R <= 0 || P < 0 || n_fft <= 0) return -1;
    double tx = 0, ty = 0, rx = 0, ry = 0, vx = 0, vy = 0;
    for (int m = 0; m < M; ++m) {
        tx += q_tx[2 * m];
        ty += q_tx[2 * m + 1];
        vx += vel[2 * m];
        vy += vel[2 * m + 1];
        for (int n = 0; n < R; ++n) {
            rx += q_rx[2 * ((long long)m * R + n)];
            ry += q_rx[2 * ((long long)m * R + n) + 1];
        }
    }
    tx /= M; ty /= M; vx /= M; vy /= M;
    rx /= (double)M * R; ry /= (double)M * R;
    for (int p = 0; p < P; ++p) {
        const double ex = px[2 * p] - tx, ey = px[2 * p + 1] - ty;
        const double gx = px[2 * p] - rx, gy = px[2 * p + 1] - ry;
        const double v_tx = (ex * vx + ey * vy) / hypot(ex, ey);
        const double v_rx = (gx * vx + gy * vy) / hypot(gx, gy);
        out[p] = f0 * (-(v_tx + v_rx)) / c * n_fft / fs;
    }
    return 0;
}
