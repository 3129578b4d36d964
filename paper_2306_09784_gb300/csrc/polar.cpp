// Polar reconstruction grid, paper Sec. III-E (Fig. 2): a grid that originates
// in the centre of the synthetic aperture, with range and azimuth spacings a
// fixed factor finer than the radar's range and azimuth resolution (the paper
// uses 2.5).  The paper takes the resolutions from a point spread function it
// does not print; the textbook values stand in for it:
//   range    dr   = c / (2 B),        B = |slope| N / fs (swept bandwidth)
//   azimuth  dphi = lambda / (2 L),   lambda r / (2 L) at range r; lambda at
//                                     the sweep's centre frequency, L the
//                                     aperture length |q_tx(M-1) - q_tx(0)|
// Points: o + (k Dr) (cos(j Dphi) u + sin(j Dphi) v) for integers k >= 1 and
// j with j Dphi in [-pi, pi), Dr = dr / factor, Dphi = dphi / factor, o the
// aperture centre, u the along-track unit vector, v its left normal; those in
// the region of interest are kept, ring by ring (k ascending), then by angle.
//
// This is plan set-up (a point list for sar_plan_create), not per-frame work:
// it runs on the host.  Only the rings and angles that can reach the box are
// visited.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "sar_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

struct JRange {
    long long lo, hi;  // inclusive; empty when lo > hi
};

}  // namespace

extern "C" int sar_polar_grid(const sar_radar_params *p, const double *q_tx, int32_t M, const sar_polar_spec *spec,
                              double *xy, int64_t capacity, int64_t *n_points) {
    if (!p || !q_tx || !spec || !n_points || M < 2 || p->n_samples < 1) return SAR_EINVAL;
    *n_points = 0;
    if (!(p->fs > 0) || !(p->c > 0) || !(p->f0 > 0) || !(p->slope != 0) || !std::isfinite(p->slope) ||
        !std::isfinite(p->f0) || !std::isfinite(p->fs) || !std::isfinite(p->c))
        return SAR_EINVAL;
    const double x0 = spec->x_min, x1 = spec->x_max, y0 = spec->y_min, y1 = spec->y_max;
    if (!(spec->factor > 0) || !std::isfinite(spec->factor) || !(x1 >= x0) || !(y1 >= y0) || !std::isfinite(x0) ||
        !std::isfinite(x1) || !std::isfinite(y0) || !std::isfinite(y1))
        return SAR_EINVAL;
    if (xy && capacity < 0) return SAR_EINVAL;
    const double ax = q_tx[2 * (M - 1)] - q_tx[0], ay = q_tx[2 * (M - 1) + 1] - q_tx[1];
    const double L = std::hypot(ax, ay);
    if (!(L > 0) || !std::isfinite(L)) return SAR_EINVAL;
    const double ux = ax / L, uy = ay / L, vx = -uy, vy = ux;
    const double ox = 0.5 * (q_tx[0] + q_tx[2 * (M - 1)]);
    const double oy = 0.5 * (q_tx[1] + q_tx[2 * (M - 1) + 1]);
    const double B = std::fabs(p->slope) * p->n_samples / p->fs;
    const double fc = p->f0 + p->slope * p->n_samples / (2.0 * p->fs);
    if (!(fc > 0)) return SAR_EINVAL;
    const double dr = p->c / (2.0 * B) / spec->factor;
    const double dphi = (p->c / fc) / (2.0 * L) / spec->factor;
    if (!(dr > 0) || !(dphi > 0) || !std::isfinite(dr) || !std::isfinite(dphi)) return SAR_EINVAL;

    // rings that can meet the box: from the box's nearest point to its
    // farthest corner
    const double cx = std::min(std::max(ox, x0), x1), cy = std::min(std::max(oy, y0), y1);
    const double rmin = std::hypot(cx - ox, cy - oy);
    double rmax = 0.0;
    const double kx[4] = {x0, x1, x0, x1}, ky[4] = {y0, y0, y1, y1};
    for (int i = 0; i < 4; ++i) rmax = std::max(rmax, std::hypot(kx[i] - ox, ky[i] - oy));
    const long long k_lo = std::max(1ll, (long long)std::floor(rmin / dr) - 1);
    const long long k_hi = (long long)std::floor(rmax / dr) + 1;
    if ((double)(k_hi - k_lo) * (2.0 * kPi / dphi) > 4e12) return SAR_EINVAL;  // absurd density

    // lattice angles in [-pi, pi), restricted to the sector the box spans as
    // seen from o (angles in the (u, v) frame, widened by a small margin);
    // the whole circle when o lies in or next to the box
    const long long jmin = (long long)std::ceil(-kPi / dphi), jmax = (long long)std::ceil(kPi / dphi) - 1;
    JRange rng[2] = {{jmin, jmax}, {1, 0}};
    if (rmin > 1e-6 * (rmax + 1.0)) {
        // direction to the box centre, then the corners' angles relative to it
        const double bx = 0.5 * (x0 + x1) - ox, by = 0.5 * (y0 + y1) - oy;
        const double a0 = std::atan2(bx * vx + by * vy, bx * ux + by * uy);
        double lo = 0.0, hi = 0.0;
        for (int i = 0; i < 4; ++i) {
            const double ex = kx[i] - ox, ey = ky[i] - oy;
            double a = std::atan2(ex * vx + ey * vy, ex * ux + ey * uy) - a0;
            a -= 2.0 * kPi * std::floor((a + kPi) / (2.0 * kPi));  // into [-pi, pi)
            lo = std::min(lo, a);
            hi = std::max(hi, a);
        }
        const double margin = 1e-9 + 4.0 * dphi;
        lo = a0 + lo - margin;
        hi = a0 + hi + margin;
        if (hi - lo < 2.0 * kPi) {
            // [lo, hi] may reach past -pi or pi: split it on the circle
            auto jr = [&](double a, double b) {
                return JRange{std::max(jmin, (long long)std::ceil(a / dphi)),
                              std::min(jmax, (long long)std::floor(b / dphi))};
            };
            if (lo < -kPi) {
                rng[0] = jr(-kPi, hi);
                rng[1] = jr(lo + 2.0 * kPi, kPi);
            } else if (hi >= kPi) {
                rng[0] = jr(-kPi, hi - 2.0 * kPi);
                rng[1] = jr(lo, kPi);
            } else {
                rng[0] = jr(lo, hi);
            }
        }
    }

    long long n = 0;
    for (long long k = k_lo; k <= k_hi; ++k) {
        const double r = (double)k * dr;
        for (const JRange &jr : rng) {
            for (long long j = jr.lo; j <= jr.hi; ++j) {
                const double phi = (double)j * dphi;
                const double cs = std::cos(phi), sn = std::sin(phi);
                const double x = ox + r * (cs * ux + sn * vx);
                const double y = oy + r * (cs * uy + sn * vy);
                if (x >= x0 && x <= x1 && y >= y0 && y <= y1) {
                    if (xy && n < capacity) {
                        xy[2 * n] = x;
                        xy[2 * n + 1] = y;
                    }
                    ++n;
                }
            }
        }
    }
    *n_points = n;
    return (xy && n > capacity) ? SAR_EINVAL : SAR_OK;
}
