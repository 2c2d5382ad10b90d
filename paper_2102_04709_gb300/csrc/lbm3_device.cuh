// lbm3_device.cuh -- device helpers shared by the step kernels and the adjoint kernels:
// thresholds of the readings of Section II.B, compensated (float-float) sums, the fraction C_k
// of a pulled node, and the characteristic-line march.
#pragma once

#include <cfloat>
#include <cmath>

#include "lbm3_common.cuh"

namespace lbm3k {
namespace {

constexpr float kG2Eps = 1e-24f;   // |G|^2 at or below which n_kl = 0 and the stress vanishes
constexpr double kRayEps = 1e-6;   // crossings this close to a node are node hits
constexpr double kPhiSnap = 1e-6;  // |90 - theta_k| below this (deg): both lines along n_s
constexpr double kRayTmax = 16.0;  // the characteristic-line search stops beyond this length

// ---- compensated (float-float) phase fields ----
// Near a contact line the colour gradient of a well-mixed node can be 1e-3 while C ~ 0.5, so
// the normal n_kl = G_kl/|G_kl| of Eq.(13) and the stress of Eq.(10) need C to more bits than a
// float holds.  C_k is kept as an unevaluated pair hi + lo: the populations are summed with
// error-free transformations (Knuth's TwoSum), the division carries its exact FMA residual,
// and the Eq.(12) stencil is applied to hi and lo separately (hi differences of close values
// are exact).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// sum of the 9 populations q[0..8] as hi + lo
__device__ __forceinline__ void sum9_df(const float* q, float& hi, float& lo)
{
    float s = q[0], e = 0.0f;
#pragma unroll
    for (int a = 1; a < kQ; a++) {
        float t;
        two_sum(s, q[a], s, t);
        e += t;
    }
    two_sum(s, e, hi, lo);
}

// (nh + nl) / (dh + dl) as hi + lo
__device__ __forceinline__ void div_df(float nh, float nl, float dh, float dl, float& qh, float& ql)
{
    qh = nh / dh;
    const float r = fmaf(-qh, dh, nh) + nl - qh * dl;
    ql = r / dh;
}

// ------------------------------------------------------------------------------------------
// wetting: characteristic lines (Section II.B)
// ------------------------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ bool node_is_fluid(const Params& P, const uint8_t* __restrict__ type,
                                              int X, int Y)
{
    Loc L = locate(P, X, Y);
    if (L.kind != 0) return false;  // solid beyond a wall side, or beyond an open side
    return !(__ldg(type + L.idx) & 2);
}

// C_k at the fluid node at unwrapped (X, Y), in the frame of the home domain.  The populations
// are summed with error-free transformations and divided in float-float arithmetic (div_df), so
// the value is the fraction of the stored FP32 populations to about 44 bits (a node holding one
// fluid gives exactly 0 or 1) without a double-precision division, which is slow on this GPU.
// (kept out of line: the wetting pass calls it up to ten times per lane, and inlining each call
// made that kernel wait on its instruction cache)
template <class S>
__device__ __noinline__ double node_C(const Params& P, const S& st, const uint8_t* __restrict__ type, int X,
                         int Y, int k)
{
    float q[27];
    pull_global(P, st, type, X, Y, q);
    float rh[kNF], rl[kNF];
#pragma unroll
    for (int j = 0; j < kNF; j++) sum9_df(q + 9 * j, rh[j], rl[j]);
    float th, tl, sh, sl, dh;
    two_sum(rh[0], rh[1], th, tl);
    two_sum(th, rh[2], sh, sl);
    const float dl = (tl + sl) + ((rl[0] + rl[1]) + rl[2]);
    two_sum(sh, dl, dh, sl);
    const float nh = k == 0 ? rh[0] : (k == 1 ? rh[1] : rh[2]);
    const float nl = k == 0 ? rl[0] : (k == 1 ? rl[1] : rl[2]);
    float qh, ql;
    div_df(nh, nl, dh, sl, qh, ql);
    return (double)qh + (double)ql;
}

template <class S>
__device__ double neighbour_mean(const Params& P, const S& st, const uint8_t* __restrict__ type,
                                 int px, int py, int k)
{
    double s = 0.0, ws = 0.0;
#pragma unroll 1
    for (int a = 1; a < kQ; a++) {
        if (node_is_fluid<S>(P, type, px + ex(a), py + ey(a))) {
            const double w = a < 5 ? 1.0 / 9.0 : 1.0 / 36.0;
            s += w * node_C(P, st, type, px + ex(a), py + ey(a), k);
            ws += w;
        }
    }
    return ws > 0.0 ? s / ws : 0.0;
}

// Where a characteristic line from the C_SB node (px, py) along (dx, dy) picks up its value:
// kind 0 = no valid crossing within the search length, 1 = a node hit (node a),
// 2 = a crossing between the fluid nodes a and b at fraction fr from a.
struct Crossing {
    int kind, ax, ay, bx, by;
    double fr;
};

template <class S>
__device__ Crossing characteristic_line(const Params& P, const uint8_t* __restrict__ type, int px,
                                        int py, double dx, double dy)
{
    Crossing c{0, 0, 0, 0, 0, 0.0};
    const int sx = dx > 0.0 ? 1 : -1;
    const int sy = dy > 0.0 ? 1 : -1;
    int X = px + sx;  // next vertical grid line
    int Y = py + sy;  // next horizontal grid line
    double tX = fabs(dx) > 1e-14 ? (double)(X - px) / dx : HUGE_VAL;
    double tY = fabs(dy) > 1e-14 ? (double)(Y - py) / dy : HUGE_VAL;
#pragma unroll 1
    for (int it = 0; it < 64; it++) {
        const double t = fmin(tX, tY);
        if (!(t <= kRayTmax)) return c;
        const bool onX = (tX - t) <= kRayEps;
        const bool onY = (tY - t) <= kRayEps;
        if (onX && onY) {
            if (node_is_fluid<S>(P, type, X, Y)) {
                c.kind = 1;
                c.ax = X;
                c.ay = Y;
                return c;
            }
        } else {
            // position along the crossed line, without fused multiply-add so that the node-hit
            // test sees the same value as a plain double evaluation
            const double s = onX ? __dadd_rn((double)py, __dmul_rn(t, dy))
                                 : __dadd_rn((double)px, __dmul_rn(t, dx));
            const double sr = floor(s + 0.5);
            if (fabs(s - sr) < kRayEps) {
                const int hx = onX ? X : (int)sr, hy = onX ? (int)sr : Y;
                if (node_is_fluid<S>(P, type, hx, hy)) {
                    c.kind = 1;
                    c.ax = hx;
                    c.ay = hy;
                    return c;
                }
            } else {
                const int s0 = (int)floor(s);
                const int ax = onX ? X : s0, ay = onX ? s0 : Y;
                const int bx = onX ? X : s0 + 1, by = onX ? s0 + 1 : Y;
                if (node_is_fluid<S>(P, type, ax, ay) && node_is_fluid<S>(P, type, bx, by)) {
                    c.kind = 2;
                    c.ax = ax;
                    c.ay = ay;
                    c.bx = bx;
                    c.by = by;
                    c.fr = s - (double)s0;
                    return c;
                }
            }
        }
        if (onX) {
            X += sx;
            tX = (double)(X - px) / dx;
        }
        if (onY) {
            Y += sy;
            tY = (double)(Y - py) / dy;
        }
    }
    return c;
}

// Eq.(21) for one fluid k with the other two fractions w_m, w_l and angles t_m, t_l: the paper's
// (w_m t_m + w_l t_l) / (1 - C_k) with 1 - C_k = w_m + w_l, written as the convex combination
// t_l + w_m / (w_m + w_l) (t_m - t_l); the mean of the two angles when both weights vanish
__device__ __forceinline__ double local_angle(double wm, double tm, double wl, double tl)
{
    return wm + wl < 1e-12 ? 0.5 * (tm + tl) : tl + wm / (wm + wl) * (tm - tl);
}


// accumulate sigma A (|G|^2 I - G G)/|G| of one fluid pair into (Txx, Txy, Tyy)
template <typename R>
__device__ __forceinline__ void pair_stress(R sig, R ck, R cl, R gkx, R gky, R glx, R gly, R rho2,
                                            R& Txx, R& Txy, R& Tyy)
{
    const R Gx = cl * gkx - ck * glx;
    const R Gy = cl * gky - ck * gly;
    const R G2 = Gx * Gx + Gy * Gy;
    if (G2 > kG2Eps) {
        // A_kl lies in [0, 1]; the clamp at 0 matters only for the reduced storage, where an
        // absent fluid can reconstruct to a density of -1e-5 that 1e6 would amplify
        const R A = fmin(fmax(R(1e6) * ck * cl * rho2, R(0.0)), R(1.0));
        const R s = sig * A * rsqrt(G2);
        Txx += s * Gy * Gy;
        Txy -= s * Gx * Gy;
        Tyy += s * Gx * Gx;
    }
}

}  // namespace
}  // namespace lbm3k
