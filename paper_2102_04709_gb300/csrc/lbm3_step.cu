// lbm3_step.cu -- sm_103a kernels of one timestep of the three-phase MRT colour-gradient
// lattice Boltzmann model with the characteristic-line wetting condition
// (arXiv:2102.04709, Section II).
//
//   k_wet      Eq.(21)-(22) and the characteristic lines of Section II.B, one thread per
//              solid boundary node (C_SB), FP64 ray geometry
//   k_step     fused Eq.(1)-(16): pull-streaming with halfway bounce-back (and the x boundary),
//              densities and phase fields, isotropic gradients (Eq.12), the surface-stress
//              tensor and its divergence (Eq.10), MRT collision with forcing (Eq.1-9, 11),
//              recolouring (Eq.13-15); one CTA per TX x TY tile, halo staged in shared memory
//   k_init     rest-equilibrium initial state written as the pre-image of a pull
//   k_fields   post-streaming densities
//   k_diag     FP64 block partials of mass, centroid, max|u|, min rho, non-finite count
#include <cfloat>
#include <cmath>

#include "lbm3_common.cuh"
#include "lbm3_device.cuh"

namespace lbm3k {

namespace {

// Four lanes per C_SB node: lane = 2 * k + side, for the wetted fluids k = 0, 1 and the two
// characteristic lines (rotated by +phi and -phi from n_s).  Each lane marches its line over the
// class bytes, then gathers C at the one or two nodes it found; Eq.(22) combines the two lines
// of a fluid with a shuffle, and lane 0 writes the wall values (and, when Cw_prev is given, the
// lagged ones it started from, which the adjoint keeps for every step).
template <class S>
__global__ void __launch_bounds__(128) k_wet(const Params P, const int nw, const int* __restrict__ widx,
                                             const double* __restrict__ wnrm,
                                             const float* __restrict__ wang, const S st,
                                             const uint8_t* __restrict__ type, double* __restrict__ Cw,
                                             WetCache* __restrict__ cache, double* __restrict__ Cw_prev)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = g >> 2;
    const int k = (g >> 1) & 1, side = g & 1;
    const bool valid = w < nw;
    int i = 0, px = 0, py = 0;
    double th = 90.0;
    Crossing cr{0, 0, 0, 0, 0, 0.0};
    if (valid) {
        i = widx[w];
        px = i % P.nx;
        py = i / P.nx;
        // Eq.(21) with the wall values of the previous step
        const double Cr = Cw[i], Cg = Cw[P.N + i], Cb = Cw[2 * P.N + i];
        if (Cw_prev && (g & 3) == 0) {
            Cw_prev[i] = Cr;
            Cw_prev[P.N + i] = Cg;
            Cw_prev[2 * P.N + i] = Cb;
        }
        const double wm = Cb, wl = k == 0 ? Cg : Cr;  // the weights of Eq.(21) for fluid k
        const WetCache c = cache[g];
        if (c.wm == wm && c.wl == wl) {
            // the same wall values as last time: the same angle, line and crossing
            th = c.th;
            cr = Crossing{c.kind, c.ax, c.ay, c.bx, c.by, c.fr};
        } else {
            const double t_rg = wang[3 * w], t_br = wang[3 * w + 1], t_gb = wang[3 * w + 2];
            th = k == 0 ? local_angle(wm, 180.0 - t_br, wl, t_rg) : local_angle(wm, t_gb, wl, 180.0 - t_rg);
            if (c.th == th) {
                // the same angle as when this lane last marched: the same line, the same crossing
                cr = Crossing{c.kind, c.ax, c.ay, c.bx, c.by, c.fr};
            } else {
                const double nx_ = wnrm[2 * w], ny_ = wnrm[2 * w + 1];
                const double dev = fabs(90.0 - th);
                const double phi = dev < kPhiSnap ? 0.0 : dev * (M_PI / 180.0);
                double sn, cs;
                sincos(phi, &sn, &cs);
                if (side) sn = -sn;
                // the line makes the angle phi with n_s (tangent (-n_y, n_x))
                cr = characteristic_line<S>(P, type, px, py, cs * nx_ - sn * ny_, cs * ny_ + sn * nx_);
            }
            cache[g] = WetCache{th, cr.fr, wm, wl, cr.kind, cr.ax, cr.ay, cr.bx, cr.by, 0};
        }
    }
    double ca = 0.0, cb = 0.0;
    if (valid && cr.kind >= 1) ca = node_C(P, st, type, cr.ax, cr.ay, k);
    if (valid && cr.kind == 2) cb = node_C(P, st, type, cr.bx, cr.by, k);
    if (valid && cr.kind == 0) ca = neighbour_mean(P, st, type, px, py, k);
    const double cd = cr.kind == 2 ? ca + cr.fr * (cb - ca) : ca;
    // Eq.(22): max of the two lines for theta_k <= 90 deg, min otherwise
    const double other = __shfl_xor_sync(0xffffffffu, cd, 1);
    const double cp = th <= 90.0 ? fmax(cd, other) : fmin(cd, other);
    const double cg = __shfl_xor_sync(0xffffffffu, cp, 2);
    if (valid && (g & 3) == 0) {
        // fractions stay in [0, 1] (a no-op unless 16-bit storage rounded a density below 0)
        double c0 = fmin(fmax(cp, 0.0), 1.0), c1 = fmin(fmax(cg, 0.0), 1.0);
        const double s = c0 + c1;
        if (s > 1.0) {
            c0 /= s;
            c1 /= s;
        }
        Cw[i] = c0;
        Cw[P.N + i] = c1;
        Cw[2 * P.N + i] = fmax(0.0, 1.0 - c0 - c1);
    }
}

// initial wall values: w-weighted mean of the fluid neighbours, for each fluid
template <class S>
__global__ void k_wet_init(const Params P, const int nw, const int* __restrict__ widx, const S st,
                           const uint8_t* __restrict__ type, double* __restrict__ Cw)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    const int i = widx[w];
    const int px = i % P.nx, py = i / P.nx;
    for (int k = 0; k < kNF; k++) Cw[k * P.N + i] = neighbour_mean(P, st, type, px, py, k);
}

// ------------------------------------------------------------------------------------------
// fused step
// ------------------------------------------------------------------------------------------
// Rest populations of unit density as R constants, and the FP64 residuals of the rounded
// constants in the density and energy moments: sum_a fl(w_a) = 1 + kDRho, energy row
// M_1 . fl(w) = -2 + kDE, M_2 . fl(w) = 1 + kDEps (row weights -4 + 3|e|^2 and
// 4 - 21/2 |e|^2 + 9/2 |e|^4).  Moments are taken of f - fl(w), which is exact for
// populations within a factor 2 of fl(w_a) and small otherwise, so that the equilibrium
// deviations e - e_eq and eps - eps_eq carry no O(1) cancellation.
constexpr float kW0 = 4.0f / 9.0f, kW1 = 1.0f / 9.0f, kW5 = 1.0f / 36.0f;
constexpr double kDRho = (double)kW0 + 4.0 * (double)kW1 + 4.0 * (double)kW5 - 1.0;
constexpr double kDE = -4.0 * (double)kW0 - 4.0 * (double)kW1 + 8.0 * (double)kW5 + 2.0;
constexpr double kDEps = 4.0 * (double)kW0 - 8.0 * (double)kW1 + 4.0 * (double)kW5 - 1.0;

// MRT collision with forcing in moment space (the rows of M in Eq.4; M^-1 = M^T diag(1/|row|^2)).
// f: totals f_a; F: interfacial force; returns f_dag in f and the velocity of Eq.(11).  The
// update is applied as f_dag = f + M^-1 dm with dm = -S (m - m_eq) + (I - S/2) M Ftilde, so that
// the rounded constants 1/9, 1/36 ... only scale the small non-equilibrium change (dm_0 = 0).
template <typename R>
__device__ __forceinline__ void collide_mrt(R f[kQ], R rho, R Fx, R Fy, R s1, R& ux, R& uy)
{
    const R d0 = f[0] - kW0;
    const R d1 = f[1] - kW1, d2 = f[2] - kW1, d3 = f[3] - kW1, d4 = f[4] - kW1;
    const R d5 = f[5] - kW5, d6 = f[6] - kW5, d7 = f[7] - kW5, d8 = f[8] - kW5;
    const R b14 = (d1 + d3) + (d2 + d4);
    const R b58 = (d5 + d7) + (d6 + d8);
    const R drho = (d0 + b14) + b58 + (R)kDRho;          // rho - 1
    const R de = (-R(4.0) * d0 - b14 + R(2.0) * b58) + (R)kDE;   // e + 2
    const R deps = (R(4.0) * d0 - R(2.0) * b14 + b58) + (R)kDEps; // eps - 1
    const R jx = (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
    const R qx = -R(2.0) * (f[1] - f[3]) + (f[5] - f[7]) + (f[8] - f[6]);
    const R jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
    const R qy = -R(2.0) * (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
    const R pxx = (f[1] - f[2]) + (f[3] - f[4]);
    const R pxy = (f[5] - f[6]) + (f[7] - f[8]);
    const R irho = __fdividef(R(1.0), rho);  // rounding here only perturbs u by ~1 ulp
    ux = (jx + R(0.5) * Fx) * irho;  // Eq.(11)
    uy = (jy + R(0.5) * Fy) * irho;
    const R u2 = ux * ux + uy * uy;
    const R uF = ux * Fx + uy * Fy;
    // relaxation rates, Eq.(5)-(6) (s1 = 1/tau from the caller)
    const R s4 = __fdividef(R(8.0) * (R(2.0) - s1), R(8.0) - s1);
    const R h1 = R(1.0) - R(0.5) * s1, h4 = R(1.0) - R(0.5) * s4;
    // moment changes: relaxation towards the Eq.(3) equilibrium moments
    // e_eq = rho(-2 + 3u^2), eps_eq = rho(1 - 3u^2), q_eq = -rho u, p_eq = rho(ux^2 - uy^2), rho ux uy,
    // plus the moments of the Eq.(9) forcing vector
    // (0, 6uF, -6uF, Fx, -Fx, Fy, -Fy, 2(uxFx - uyFy), uxFy + uyFx)
    const R dE = -s1 * (de + R(2.0) * drho - R(3.0) * rho * u2) + h1 * R(6.0) * uF;
    const R dEps = -s1 * (deps - drho + R(3.0) * rho * u2) - h1 * R(6.0) * uF;
    const R djx = Fx, djy = Fy;
    const R dqx = -s4 * (qx + rho * ux) - h4 * Fx;
    const R dqy = -s4 * (qy + rho * uy) - h4 * Fy;
    const R dpxx = -s1 * (pxx - rho * (ux * ux - uy * uy)) + h1 * R(2.0) * (ux * Fx - uy * Fy);
    const R dpxy = -s1 * (pxy - rho * ux * uy) + h1 * (ux * Fy + uy * Fx);
    // back to populations
    const R c0 = (R(1.0) / R(9.0)) * (dEps - dE);
    const R ca = -(R(1.0) / R(36.0)) * dE - (R(1.0) / R(18.0)) * dEps;
    const R cd = (R(1.0) / R(18.0)) * dE + (R(1.0) / R(36.0)) * dEps;
    const R X1 = (R(1.0) / R(6.0)) * (djx - dqx), Y1 = (R(1.0) / R(6.0)) * (djy - dqy);
    const R X2 = (R(1.0) / R(6.0)) * djx + (R(1.0) / R(12.0)) * dqx;
    const R Y2 = (R(1.0) / R(6.0)) * djy + (R(1.0) / R(12.0)) * dqy;
    const R P4 = R(0.25) * dpxx, Q4 = R(0.25) * dpxy;
    f[0] += c0;
    f[1] += ca + X1 + P4;
    f[2] += ca + Y1 - P4;
    f[3] += ca - X1 + P4;
    f[4] += ca - Y1 - P4;
    f[5] += cd + X2 + Y2 + Q4;
    f[6] += cd - X2 + Y2 - Q4;
    f[7] += cd - X2 - Y2 + Q4;
    f[8] += cd + X2 - Y2 - Q4;
}

// unit normal of one pair (0 if |G| vanishes)
template <typename R>
__device__ __forceinline__ void pair_normal(R ck, R cl, R gkx, R gky, R glx, R gly, R& nx_, R& ny_)
{
    const R Gx = cl * gkx - ck * glx;
    const R Gy = cl * gky - ck * gly;
    const R G2 = Gx * Gx + Gy * Gy;
    if (G2 > kG2Eps) {
        const R r = rsqrt(G2);
        nx_ = Gx * r;
        ny_ = Gy * r;
    } else {
        nx_ = ny_ = R(0.0);
    }
}

// Eq.(12) derivative weights: d_x psi = (psi_1 - psi_3)/3 + (psi_5 - psi_6 - psi_7 + psi_8)/12
template <int W, typename R>
__device__ __forceinline__ void grad9_df(const float (*h)[W], const float (*l)[W], int cx, int cy,
                                         R& gx, R& gy)
{
    R hx, hy, lx_, ly_;
    {
        const R c1 = h[cy][cx + 1], c3 = h[cy][cx - 1], c2 = h[cy + 1][cx], c4 = h[cy - 1][cx];
        const R c5 = h[cy + 1][cx + 1], c6 = h[cy + 1][cx - 1], c7 = h[cy - 1][cx - 1], c8 = h[cy - 1][cx + 1];
        hx = (R(1.0) / R(3.0)) * (c1 - c3) + (R(1.0) / R(12.0)) * ((c5 - c7) + (c8 - c6));
        hy = (R(1.0) / R(3.0)) * (c2 - c4) + (R(1.0) / R(12.0)) * ((c5 - c7) + (c6 - c8));
    }
    {
        const R c1 = l[cy][cx + 1], c3 = l[cy][cx - 1], c2 = l[cy + 1][cx], c4 = l[cy - 1][cx];
        const R c5 = l[cy + 1][cx + 1], c6 = l[cy + 1][cx - 1], c7 = l[cy - 1][cx - 1], c8 = l[cy - 1][cx + 1];
        lx_ = (R(1.0) / R(3.0)) * (c1 - c3) + (R(1.0) / R(12.0)) * ((c5 - c7) + (c8 - c6));
        ly_ = (R(1.0) / R(3.0)) * (c2 - c4) + (R(1.0) / R(12.0)) * ((c5 - c7) + (c6 - c8));
    }
    gx = hx + lx_;
    gy = hy + ly_;
}

// ---- tensor memory accelerator (bulk tensor copies) and mbarrier, inline PTX ----
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// 3-D tiled load of a box at (x, y, z) into shared memory, completing on the mbarrier; x times
// the element size must be a multiple of 16 bytes
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, uint32_t src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map),
                 "r"(x), "r"(y), "r"(z), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until the committed bulk stores have read their shared-memory source
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// make this thread's shared-memory writes visible to the bulk copy engine
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// polls of an mbarrier before a block gives up draining its bulk copies after a timeout (each
// poll may suspend the thread for a short time; a completed copy takes a few microseconds); the
// first wait for a tile's copies polls Params::wait_polls times (kWaitLimit unless lowered to
// test the timeout path)
constexpr int kWaitLimit = 1 << 22;

// A C_SB node whose wall values are not all within kMixEps of one pure fluid: a fluid-fluid
// interface reaches the wall there (a contact line, or one within a few nodes of it), where the
// lagged wetting feedback amplifies the rounding of single-precision phase fields.  Away from
// such nodes the phase fields near walls are those of one fluid and a float suffices.
constexpr double kMixEps = 1e-6;
__device__ __forceinline__ bool mixed_wall(const double* __restrict__ Cw, long long N, long long i)
{
    const double m = fmax(fmax(Cw[i], Cw[N + i]), Cw[2 * N + i]);
    return m < 1.0 - kMixEps;
}

// Eq.(12) derivative of a float field held in shared memory
template <int W>
__device__ __forceinline__ void grad9_f(const float (*c)[W], int cx, int cy, float& gx, float& gy)
{
    const float c1 = c[cy][cx + 1], c3 = c[cy][cx - 1], c2 = c[cy + 1][cx], c4 = c[cy - 1][cx];
    const float c5 = c[cy + 1][cx + 1], c6 = c[cy + 1][cx - 1], c7 = c[cy - 1][cx - 1], c8 = c[cy - 1][cx + 1];
    gx = (1.0f / 3.0f) * (c1 - c3) + (1.0f / 12.0f) * ((c5 - c7) + (c8 - c6));
    gy = (1.0f / 3.0f) * (c2 - c4) + (1.0f / 12.0f) * ((c5 - c7) + (c6 - c8));
}

// Block-wide barrier that also reports how many of the three fluids occur in the block's
// phase-field region (present: bit k set where a node holds rho_k != 0).  Where only one fluid
// occurs, the two absent fluids have C_l = 0 exactly at every node, so every pair
// G_kl = C_l grad C_k - C_k grad C_l of Eq.(10) and (13) vanishes: no stress, no force and no
// recolouring term, and skipping the stress phase leaves every bit of the result unchanged.
__device__ __forceinline__ int single_fluid_or(int present)
{
    const int f0 = __syncthreads_or(present & 1);
    const int f1 = __syncthreads_or(present & 2);
    const int f2 = __syncthreads_or(present & 4);
    return (f0 != 0) + (f1 != 0) + (f2 != 0);
}

// The same count with one barrier, for the persistent kernels: each warp ORs its lanes' bits
// into the shared word flags[j & 1] of tile iteration j, the barrier publishes them, and thread 0
// clears the word of the next iteration (nobody writes it before the next tile's barriers).
__device__ __forceinline__ int fluids_present(int present, int* flags, int j, int tid)
{
    const int w = __reduce_or_sync(0xffffffffu, present);
    if ((tid & 31) == 0 && w) atomicOr(&flags[j & 1], w);
    __syncthreads();
    const int v = flags[j & 1];
    if (tid == 0) flags[(j + 1) & 1] = 0;
    return __popc(v & 7);
}

// F_s = div T at (rx, ry) of the stress region: Eq.(10) with the Eq.(12) derivative
template <int RX>
__device__ __forceinline__ void div_stress(const float (*txx)[RX], const float (*txy)[RX],
                                           const float (*tyy)[RX], int rx, int ry, float& Fx, float& Fy)
{
    Fx = (1.0f / 3.0f) * (txx[ry][rx + 1] - txx[ry][rx - 1]) +
         (1.0f / 12.0f) * ((txx[ry + 1][rx + 1] - txx[ry - 1][rx - 1]) + (txx[ry - 1][rx + 1] - txx[ry + 1][rx - 1])) +
         (1.0f / 3.0f) * (txy[ry + 1][rx] - txy[ry - 1][rx]) +
         (1.0f / 12.0f) * ((txy[ry + 1][rx + 1] - txy[ry - 1][rx - 1]) + (txy[ry + 1][rx - 1] - txy[ry - 1][rx + 1]));
    Fy = (1.0f / 3.0f) * (txy[ry][rx + 1] - txy[ry][rx - 1]) +
         (1.0f / 12.0f) * ((txy[ry + 1][rx + 1] - txy[ry - 1][rx - 1]) + (txy[ry - 1][rx + 1] - txy[ry + 1][rx - 1])) +
         (1.0f / 3.0f) * (tyy[ry + 1][rx] - tyy[ry - 1][rx]) +
         (1.0f / 12.0f) * ((tyy[ry + 1][rx + 1] - tyy[ry - 1][rx - 1]) + (tyy[ry + 1][rx - 1] - tyy[ry - 1][rx + 1]));
}

// the recoloured post-collision populations of one node are C_k f_a + w_a (Vx_k e_ax + Vy_k e_ay)
struct Recolour {
    float C[kNF], Vx[kNF], Vy[kNF];
};

// One node: velocity (Eq.11), mixture relaxation (Eq.7), MRT collision with forcing (Eq.1-9)
// applied in place to the 9 post-streaming totals f, and the recolouring coefficients of
// Eq.(13)-(15) from the fluid densities r0..r2 and the colour gradients g = (d C_k / dx, dy).
__device__ __forceinline__ Recolour collide_node(const Params& P, float f[kQ], float r0, float r1, float r2,
                                                 float Fx, float Fy, const float g[6], float& ux, float& uy)
{
    const float rho = (r0 + r1) + r2;
    const float ir = __fdividef(1.0f, rho);
    // fractions as the quotient corrected by its exact FMA residual: a node that holds one fluid
    // gets exactly C = 1, so the recolouring leaves its mass unscaled (r * fl(1/r) can round
    // below 1 every step)
    auto frac = [&](float r) {
        const float q = r * ir;
        return fmaf(fmaf(-q, rho, r), ir, q);
    };
    const float c0 = frac(r0), c1 = frac(r1), c2 = frac(r2);
    float n01x, n01y, n02x, n02y, n12x, n12y;
    pair_normal(c0, c1, g[0], g[1], g[2], g[3], n01x, n01y);
    pair_normal(c0, c2, g[0], g[1], g[4], g[5], n02x, n02y);
    pair_normal(c1, c2, g[2], g[3], g[4], g[5], n12x, n12y);
    // tau = 1/2 + 3 / sum(rho_k / nu_k), so 1/tau = D / (D/2 + 3)
    const float D = (r0 * P.inv_nu0 + r1 * P.inv_nu1) + r2 * P.inv_nu2;
    const float s1 = __fdividef(D, 0.5f * D + 3.0f);
    collide_mrt(f, rho, Fx, Fy, s1, ux, uy);
    const float trip = fminf(35.0f * r0 * r1 * r2 * ir * ir * ir, 1.0f);
    const float b01 = P.beta0 * (1.0f + trip * P.g01) * r0 * r1 * ir;
    const float b02 = P.beta0 * (1.0f + trip * P.g02) * r0 * r2 * ir;
    const float b12 = P.beta0 * (1.0f + trip * P.g12) * r1 * r2 * ir;
    Recolour rc;
    rc.C[0] = c0;
    rc.C[1] = c1;
    rc.C[2] = c2;
    rc.Vx[0] = b01 * n01x + b02 * n02x;
    rc.Vy[0] = b01 * n01y + b02 * n02y;
    rc.Vx[1] = -b01 * n01x + b12 * n12x;
    rc.Vy[1] = -b01 * n01y + b12 * n12y;
    rc.Vx[2] = -b02 * n02x - b12 * n12x;
    rc.Vy[2] = -b02 * n02y - b12 * n12y;
    return rc;
}

// Densities and phase fields of position (cx, cy) of a tile's phase-field region from its 27
// post-streaming populations q; returns which fluids occur there (bit k: rho_k != 0; all three
// for float-float fields, which are never skipped).  df: C_k as hi + lo (TwoSum sums, division
// with its FMA residual), else a float quotient.
template <int CX, int CY>
__device__ __forceinline__ int phase_fields(bool df, const float q[27], float (*ch)[CY][CX], float (*cl)[CY][CX],
                                            float (*rh)[CX], int cx, int cy)
{
    if (df) {
        float rhi[kNF], rlo[kNF];
#pragma unroll
        for (int k = 0; k < kNF; k++) sum9_df(q + 9 * k, rhi[k], rlo[k]);
        float th, tl, sh, sl;
        two_sum(rhi[0], rhi[1], th, tl);
        two_sum(th, rhi[2], sh, sl);
        const float dl = (tl + sl) + ((rlo[0] + rlo[1]) + rlo[2]);
        float dh;
        two_sum(sh, dl, dh, sl);  // rho = dh + sl
#pragma unroll
        for (int k = 0; k < kNF; k++) div_df(rhi[k], rlo[k], dh, sl, ch[k][cy][cx], cl[k][cy][cx]);
        rh[cy][cx] = dh;
        return 7;
    }
    float r[kNF];
#pragma unroll
    for (int k = 0; k < kNF; k++) {
        const float* qk = q + 9 * k;
        r[k] = ((qk[0] + (qk[1] + qk[3])) + (qk[2] + qk[4])) + ((qk[5] + qk[7]) + (qk[6] + qk[8]));
    }
    const float rho = (r[0] + r[1]) + r[2];
    const float ir = __fdividef(1.0f, rho);
#pragma unroll
    for (int k = 0; k < kNF; k++) ch[k][cy][cx] = r[k] * ir;
    rh[cy][cx] = rho;
    return (r[0] != 0.0f ? 1 : 0) | (r[1] != 0.0f ? 2 : 0) | (r[2] != 0.0f ? 4 : 0);
}

// Wall values of a C_SB node at (cx, cy) of the phase-field region (FP64 from the wetting pass,
// split into hi + lo; labels relabelled across a modified periodic seam when par); rho := 1 at
// solid nodes.  Returns the fluids with a nonzero wall value.
template <int CX, int CY>
__device__ __forceinline__ int wall_fields(const double* __restrict__ Cw, long long N, int in, bool par,
                                           float (*ch)[CY][CX], float (*cl)[CY][CX], float (*rh)[CX], int cx,
                                           int cy)
{
    int present = 0;
#pragma unroll
    for (int k = 0; k < kNF; k++) {
        const double c = Cw[(long long)relabel(k, par) * N + in];
        const float h = (float)c;
        ch[k][cy][cx] = h;
        cl[k][cy][cx] = (float)(c - (double)h);
        if (c != 0.0) present |= 1 << k;
    }
    rh[cy][cx] = 1.0f;
    return present;
}

// Eq.(12) gradients (gxk, gyk) and the Eq.(10) stress of position (rx, ry) of the stress region
// of a tile with solids: class bytes t of the geometry region (halo 3), phase fields of the
// phase-field region (halo 2).  At a C_SB centre a neighbour without a value of its own takes
// the extrapolation 2 C(P) - C(P - e_a) (its rounding error carried in the lo word), or C(P)
// when P - e_a has none either; lo words exist only in float-float (df) tiles.
template <int HX, int CX, int CY>
__device__ __forceinline__ void stress_at(const Params& P, const uint8_t (*t)[HX], const float (*ch)[CY][CX],
                                          const float (*cl)[CY][CX], const float (*rh)[CX], bool df, int rx,
                                          int ry, float gxk[kNF], float gyk[kNF], float& Txx, float& Txy,
                                          float& Tyy)
{
    const int cx = rx + 1, cy = ry + 1, hx = rx + 2, hy = ry + 2;
    Txx = Txy = Tyy = 0.f;
    const uint8_t tc = t[hy][hx];
    if ((tc & 3) == kSI) {
#pragma unroll
        for (int k = 0; k < kNF; k++) gxk[k] = gyk[k] = 0.0f;
        return;
    }
    const float rho = rh[cy][cx];
    float c[kNF];
#pragma unroll
    for (int k = 0; k < kNF; k++) c[k] = ch[k][cy][cx];
    if ((tc & 3) == kSB) {
#pragma unroll
        for (int k = 0; k < kNF; k++) {
            float v[kQ], vl[kQ];
            const float h0 = ch[k][cy][cx], l0 = df ? cl[k][cy][cx] : 0.0f;
#pragma unroll
            for (int a = 1; a < kQ; a++) {
                if ((t[hy + ey(a)][hx + ex(a)] & 3) != kSI) {
                    v[a] = ch[k][cy + ey(a)][cx + ex(a)];
                    vl[a] = df ? cl[k][cy + ey(a)][cx + ex(a)] : 0.0f;
                } else if ((t[hy - ey(a)][hx - ex(a)] & 3) == kSI) {
                    v[a] = h0;
                    vl[a] = l0;
                } else {
                    const float oh = ch[k][cy - ey(a)][cx - ex(a)];
                    const float ol = df ? cl[k][cy - ey(a)][cx - ex(a)] : 0.0f;
                    float e;
                    two_sum(2.0f * h0, -oh, v[a], e);
                    vl[a] = (2.0f * l0 - ol) + e;
                }
            }
            gxk[k] = (1.0f / 3.0f) * (v[1] - v[3]) + (1.0f / 12.0f) * ((v[5] - v[7]) + (v[8] - v[6])) +
                     ((1.0f / 3.0f) * (vl[1] - vl[3]) + (1.0f / 12.0f) * ((vl[5] - vl[7]) + (vl[8] - vl[6])));
            gyk[k] = (1.0f / 3.0f) * (v[2] - v[4]) + (1.0f / 12.0f) * ((v[5] - v[7]) + (v[6] - v[8])) +
                     ((1.0f / 3.0f) * (vl[2] - vl[4]) + (1.0f / 12.0f) * ((vl[5] - vl[7]) + (vl[6] - vl[8])));
        }
    } else if (df) {
#pragma unroll
        for (int k = 0; k < kNF; k++) grad9_df<CX>(ch[k], cl[k], cx, cy, gxk[k], gyk[k]);
    } else {
#pragma unroll
        for (int k = 0; k < kNF; k++) grad9_f<CX>(ch[k], cx, cy, gxk[k], gyk[k]);
    }
    const float rho2 = rho * rho;
    pair_stress(P.sig01, c[0], c[1], gxk[0], gyk[0], gxk[1], gyk[1], rho2, Txx, Txy, Tyy);
    pair_stress(P.sig02, c[0], c[2], gxk[0], gyk[0], gxk[2], gyk[2], rho2, Txx, Txy, Tyy);
    pair_stress(P.sig12, c[1], c[2], gxk[1], gyk[1], gxk[2], gyk[2], rho2, Txx, Txy, Tyy);
}

// resident blocks per SM the wall-tile specialisation of the one-tile-per-block step kernel is
// compiled for (registers capped at 65536 / (256 x this)); the others for four
#ifndef LBM3_STEP_BLOCKS_PER_SM
#define LBM3_STEP_BLOCKS_PER_SM 5
#endif
constexpr int kStepBlocksPerSm = LBM3_STEP_BLOCKS_PER_SM;

// One CTA per TX x TY tile of interior nodes.
//   phase 0: class bytes (and, for tiles touching the domain edge, storage indices and seam
//            parities) of the halo-3 region into shared memory
//   phase 1: pull-streaming of every fluid node of the halo-2 region, densities rho_k and the
//            phase fields C_k; the tile's own nodes keep their 9 post-streaming totals and 3
//            densities in registers
//   phase 2: the Eq.(10) stress tensor on the halo-1 region
//   phase 3: force, velocity, MRT collision with forcing, recolouring, 27 stores per node
// Tiles whose halo-3 region stays inside the domain take arithmetic source indices and skip the
// bounce-back tests at C_FI nodes; only tiles whose halo-2 region holds a C_SB node with mixed
// wall values (a contact line at or near it) carry the float-float phase fields, decided anew
// every step from the wall values of this step's wetting pass.
template <int TX, int TY, bool PURE, bool INNER, int STORE>
__global__ void __launch_bounds__(TX* TY, (INNER && !PURE) ? kStepBlocksPerSm : 4) k_step(const Params P, const int* __restrict__ tiles,
                                                  const Pop fin, const Pop fout,
                                                  const uint8_t* __restrict__ type,
                                                  const double* __restrict__ Cw,
                                                  float* __restrict__ uout,
                                                  const uint64_t* __restrict__ pres_in,
                                                  uint64_t* __restrict__ pres_out)
{
    constexpr int NT = TX * TY;
    constexpr int HX = TX + 6, HY = TY + 6;  // geometry region (halo 3)
    constexpr int CX = TX + 4, CY = TY + 4;  // phase-field region (halo 2)
    constexpr int RX = TX + 2, RY = TY + 2;  // stress region (halo 1)
    __shared__ int s_idx[HY][HX];            // storage index (tiles at the domain edge only)
    __shared__ uint8_t s_t[HY][HX];          // class bits 0-1; bit 3: ghost beyond an open side
    __shared__ uint8_t s_par[HX];
    __shared__ float s_ch[kNF][CY][CX], s_cl[kNF][CY][CX];  // C_k = hi (+ lo in wall tiles)
    __shared__ float s_rho[CY][CX];
    __shared__ float s_txx[RY][RX], s_txy[RY][RX], s_tyy[RY][RX];
    __shared__ float s_g[2 * kNF][TY][TX];   // colour gradients of the tile's own nodes
    __shared__ int s_flags[2];                // fluids present (wall and edge tiles)
    // wall tiles: fluids stored in the 3 x 3 tiles around (one word each), and the fluids with a
    // nonzero wall value at the C_SB nodes of the phase-field region (one word per warp)
    __shared__ uint64_t s_nb[9];
    __shared__ int s_wp[TX * TY / 32];

    const int tid = threadIdx.x + TX * threadIdx.y;
    if (!PURE && tid == 0) s_flags[0] = 0;  // published by the phase-0 barrier
    const int ntx = (P.nx + TX - 1) / TX;
    const int tile = tiles[blockIdx.x];
    const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
    const int nx = P.nx;
    const int N = (int)P.N;
    // halo-3 region inside the domain: no wrap, no ghost, no seam (INNER: every listed tile).
    // A PURE tile is also free of solid nodes in that region (every node it touches is in C_FI).
    const bool inner = PURE || INNER || (x0 >= 3 && y0 >= 3 && x0 + TX + 3 <= P.nx && y0 + TY + 3 <= P.ny);

    // ---- phase 0: geometry of the halo-3 region ----
    int wall = 0, wp = 0;
    if (PURE) {
    } else if (inner) {
        if constexpr (INNER) {
            if (tid < 9) s_nb[tid] = pres_in[tile + (tid / 3 - 1) * ntx + (tid % 3 - 1)];
        }
        for (int j = tid; j < HX * HY; j += NT) {
            const int hx = j % HX, hy = j / HX;
            const uint8_t t = __ldg(type + (y0 + hy - 3) * nx + (x0 + hx - 3));
            s_t[hy][hx] = t;
            if ((t & 3) == kSB && hx >= 1 && hx <= CX && hy >= 1 && hy <= CY) {
                const long long in = (long long)(y0 + hy - 3) * nx + (x0 + hx - 3);
                const double c0 = Cw[in], c1 = Cw[P.N + in], c2 = Cw[2 * P.N + in];
                if (fmax(fmax(c0, c1), c2) < 1.0 - kMixEps) wall = 1;  // mixed_wall
                wp |= (c0 != 0.0 ? 1 : 0) | (c1 != 0.0 ? 2 : 0) | (c2 != 0.0 ? 4 : 0);
            }
        }
        if constexpr (INNER) {
            const int w = __reduce_or_sync(0xffffffffu, wp);
            if ((tid & 31) == 0) s_wp[tid >> 5] = w;
        }
    } else {
        for (int j = tid; j < HX * HY; j += NT) {
            const int hx = j % HX, hy = j / HX;
            const int X = x0 + hx - 3, Y = y0 + hy - 3;
            const Loc L = locate(P, X, Y);
            uint8_t t = kSI;
            if (L.kind != 1) {
                t = __ldg(type + L.idx);
                if (L.kind == 2) t |= 8;
            }
            s_t[hy][hx] = t;
            s_idx[hy][hx] = L.idx;
            if (hy == 0) s_par[hx] = parity_x(P, X);
            if ((t & 3) == kSB && hx >= 1 && hx <= CX && hy >= 1 && hy <= CY && mixed_wall(Cw, P.N, L.idx))
                wall = 1;
        }
    }
    const bool df = PURE ? false : __syncthreads_or(wall);
    // A wall tile whose 3 x 3 tiles stored one fluid, and whose C_SB nodes in the phase-field
    // region have wall values of that fluid only, holds that fluid alone in the region after
    // the pull: it is not mixed, and its halo's phase fields, which only the mixed path reads,
    // are skipped (same results).  The plain float path only (no float-float words).
    bool single = false;
    if constexpr (INNER && !PURE) {
        if (!df) {
            uint64_t nb = 0;
#pragma unroll
            for (int t = 0; t < 9; t++) nb |= s_nb[t];
            nb |= nb >> 32;
            nb |= nb >> 16;
            nb |= nb >> 8;
            int bits = (int)(nb & 7u);
#pragma unroll
            for (int w = 0; w < TX * TY / 32; w++) bits |= s_wp[w];
            single = __popc(bits) == 1;
        }
    }

    // ---- phase 1: post-streaming populations, densities and phase fields ----
    // pull of the fluid node at (hx, hy) of the geometry region into q[27]
    auto pull = [&](int hx, int hy, float q[27]) {
        const uint8_t t = PURE ? (uint8_t)kFI : s_t[hy][hx];
        if (inner) {
            const int i = (y0 + hy - 3) * nx + (x0 + hx - 3);
            const bool fi = PURE || (t & 3) == kFI;
            if constexpr (STORE == kStoreF32) {
                const float* b = fin.f + i;
                if (fi) {
#pragma unroll
                    for (int a = 0; a < kQ; a++)
#pragma unroll
                        for (int k = 0; k < kNF; k++) q[9 * k + a] = __ldg(b + P.off_pull[k * kQ + a]);
                } else {
#pragma unroll
                    for (int a = 0; a < kQ; a++) {
                        const bool bb = s_t[hy - ey(a)][hx - ex(a)] & 2;
#pragma unroll
                        for (int k = 0; k < kNF; k++)
                            q[9 * k + a] = __ldg(b + (bb ? P.off_plane[k * kQ + opp(a)] : P.off_pull[k * kQ + a]));
                    }
                }
            } else {
                // own node: rho_k and the 8 offsets (the rest population and any bounce-back)
                const float* rb = fin.rho + i;
                const unsigned short* ob = fin.off + i;
#pragma unroll
                for (int k = 0; k < kNF; k++) {
                    const float rk = __ldg(rb + k * N);
                    float d[kQ];
#pragma unroll
                    for (int a = 1; a < kQ; a++) d[a] = dec16<STORE>(__ldg(ob + (8 * k + a - 1) * N));
                    q[9 * k] = wq(0) * rk - sum_offsets(d);
#pragma unroll
                    for (int a = 1; a < kQ; a++) {
                        const bool bb = !fi && (s_t[hy - ey(a)][hx - ex(a)] & 2);
                        if (bb) {
                            q[9 * k + a] = wq(opp(a)) * rk + d[opp(a)];
                        } else {
                            const int o = P.off_pull16[k * kQ + a];
                            q[9 * k + a] = wq(a) * __ldg(fin.rho + i + o) +
                                           dec16<STORE>(__ldg(ob + P.off_pull16o[k * kQ + a]));
                        }
                    }
                }
            }
            return;
        }
        if (t & 8) {
            // ghost beyond an open side: copy of the boundary-column node (zero gradient)
            const Store<STORE> st(fin, P.N);
            pull_global(P, st, type, x0 + hx - 3, y0 + hy - 3, q);
            return;
        }
        const Store<STORE> st(fin, P.N);
        const bool pn = s_par[hx];
        const int in = s_idx[hy][hx];
        bool inl = false, outl = false;
#pragma unroll
        for (int a = 0; a < kQ; a++) {
            const int sx = hx - ex(a), sy = hy - ey(a);
            const uint8_t ts = s_t[sy][sx];
            if (ts & 8) {
                if (x0 + hx - 3 == 0) inl = true; else outl = true;
#pragma unroll
                for (int k = 0; k < kNF; k++) q[9 * k + a] = 0.0f;
            } else if (ts & 2) {
#pragma unroll
                for (int k = 0; k < kNF; k++) q[9 * k + a] = st.get(relabel(k, pn), opp(a), in);
            } else {
                const bool ps = s_par[sx];
                const int is = s_idx[sy][sx];
#pragma unroll
                for (int k = 0; k < kNF; k++) q[9 * k + a] = st.get(relabel(k, ps), a, is);
            }
        }
        if (inl) zou_he(P, q, true);
        if (outl) zou_he(P, q, false);
    };
    // densities / phase fields of the position (cx, cy) of the phase-field region from q, and which
    // fluids occur in the region (bit k: some rho_k != 0, or a wall value C_k != 0 at a C_SB node)
    int present = 0;
    auto store_phase = [&](int cx, int cy, const float q[27]) {
        present |= phase_fields<CX, CY>(df, q, s_ch, s_cl, s_rho, cx, cy);
    };
    auto fill = [&](int cx, int cy, float q[27]) -> bool {
        const int hx = cx + 1, hy = cy + 1;
        const uint8_t t = PURE ? (uint8_t)kFI : s_t[hy][hx];
        if (!(t & 2)) {
            pull(hx, hy, q);
            store_phase(cx, cy, q);
            return true;
        }
        if ((t & 3) == kSB) {
            // wall value from the wetting pass (FP64, split into hi + lo); rho := 1 at solid nodes
            const int in = inner ? (y0 + hy - 3) * nx + (x0 + hx - 3) : s_idx[hy][hx];
            const bool pr = inner ? false : s_par[hx];
            present |= wall_fields<CX, CY>(Cw, P.N, in, pr, s_ch, s_cl, s_rho, cx, cy);
        } else {
#pragma unroll
            for (int k = 0; k < kNF; k++) s_ch[k][cy][cx] = s_cl[k][cy][cx] = 0.0f;
            s_rho[cy][cx] = 0.0f;
        }
        return false;
    };

    if (!single) {
        // ring of the halo-2 region: rows 0, 1, CY-2, CY-1 and columns 0, 1, CX-2, CX-1
        constexpr int NRING = CX * CY - TX * TY;
        for (int j = tid; j < NRING; j += NT) {
            int cx, cy;
            if (j < 2 * CX) {
                cx = j % CX;
                cy = j / CX;
            } else if (j < 4 * CX) {
                cx = (j - 2 * CX) % CX;
                cy = CY - 2 + (j - 2 * CX) / CX;
            } else {
                const int r = j - 4 * CX;  // 4 * TY side nodes
                const int side = r / (2 * TY), rr = r % (2 * TY);
                cy = 2 + rr / 2;
                cx = side == 0 ? (rr & 1) : CX - 2 + (rr & 1);
            }
            float q[27];
            fill(cx, cy, q);
        }
    }
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int gx = x0 + lx, gy = y0 + ly;
    // own node: keep the 9 post-streaming totals and the 3 densities
    float f[kQ], r0, r1, r2;
    bool own_fluid;
    {
        float q[27];
        if (single) {
            own_fluid = !(s_t[ly + 3][lx + 3] & 2);
            if (own_fluid) pull(lx + 3, ly + 3, q);
        } else {
            own_fluid = fill(lx + 2, ly + 2, q);
        }
#pragma unroll
        for (int a = 0; a < kQ; a++) f[a] = (q[a] + q[9 + a]) + q[18 + a];
        r0 = ((q[0] + (q[1] + q[3])) + (q[2] + q[4])) + ((q[5] + q[7]) + (q[6] + q[8]));
        r1 = ((q[9] + (q[10] + q[12])) + (q[11] + q[13])) + ((q[14] + q[16]) + (q[15] + q[17]));
        r2 = ((q[18] + (q[19] + q[21])) + (q[20] + q[22])) + ((q[23] + q[25]) + (q[24] + q[26]));
    }
    if constexpr (INNER && !PURE) {
        // the fluids this warp's fluid nodes hold, for the tiles around this one in the next step
        const int own = own_fluid ? (r0 != 0.0f ? 1 : 0) | (r1 != 0.0f ? 2 : 0) | (r2 != 0.0f ? 4 : 0) : 0;
        const int w = __reduce_or_sync(0xffffffffu, own);
        if ((tid & 31) == 0) reinterpret_cast<uint8_t*>(pres_out + tile)[tid >> 5] = (uint8_t)w;
    }
    // fluids present in the phase-field region: one barrier for tiles that had one already (the
    // word was cleared before the phase-0 barrier), three for the pure tiles of the plain path
    const bool mixed =
        single ? false : (PURE ? single_fluid_or(present) : fluids_present(present, s_flags, 0, tid)) != 1;

    // ---- phase 2: stress tensor of Eq.(10) on the halo-1 region ----
    for (int j = mixed ? tid : RX * RY; j < RX * RY; j += NT) {
        const int rx = j % RX, ry = j / RX;
        float Txx = 0.f, Txy = 0.f, Tyy = 0.f;
        float gxk[kNF], gyk[kNF];
        if (PURE) {
            const float rho = s_rho[ry + 1][rx + 1];
            float c[kNF];
#pragma unroll
            for (int k = 0; k < kNF; k++) {
                c[k] = s_ch[k][ry + 1][rx + 1];
                grad9_f<CX>(s_ch[k], rx + 1, ry + 1, gxk[k], gyk[k]);
            }
            const float rho2 = rho * rho;
            pair_stress(P.sig01, c[0], c[1], gxk[0], gyk[0], gxk[1], gyk[1], rho2, Txx, Txy, Tyy);
            pair_stress(P.sig02, c[0], c[2], gxk[0], gyk[0], gxk[2], gyk[2], rho2, Txx, Txy, Tyy);
            pair_stress(P.sig12, c[1], c[2], gxk[1], gyk[1], gxk[2], gyk[2], rho2, Txx, Txy, Tyy);
        } else {
            stress_at<HX, CX, CY>(P, s_t, s_ch, s_cl, s_rho, df, rx, ry, gxk, gyk, Txx, Txy, Tyy);
        }
        if (rx >= 1 && rx <= TX && ry >= 1 && ry <= TY) {
#pragma unroll
            for (int k = 0; k < kNF; k++) {
                s_g[2 * k][ry - 1][rx - 1] = gxk[k];
                s_g[2 * k + 1][ry - 1][rx - 1] = gyk[k];
            }
        }
        s_txx[ry][rx] = Txx;
        s_txy[ry][rx] = Txy;
        s_tyy[ry][rx] = Tyy;
    }
    if (!single) __syncthreads();

    if (!own_fluid || gx >= P.nx || gy >= P.ny) return;

    // ---- interfacial force F_s = div T (Eq.10 with Eq.12) ----
    float Fx = 0.0f, Fy = 0.0f, g[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (mixed) {
        div_stress<RX>(s_txx, s_txy, s_tyy, lx + 1, ly + 1, Fx, Fy);
        // own colour gradients from phase 2
#pragma unroll
        for (int k = 0; k < 6; k++) g[k] = s_g[k][ly][lx];
    }
    // ---- velocity, MRT collision with forcing, recolouring coefficients ----
    float ux, uy;
    const Recolour rc = collide_node(P, f, r0, r1, r2, Fx, Fy, g, ux, uy);
    const int i = gy * nx + gx;
    if (uout) {
        uout[i] = ux;
        uout[N + i] = uy;
    }
    const float* Cs = rc.C;
    const float* Vx = rc.Vx;
    const float* Vy = rc.Vy;
    if constexpr (STORE == kStoreF32) {
        float* o = fout.f + i;
#pragma unroll
        for (int k = 0; k < kNF; k++) {
#pragma unroll
            for (int a = 0; a < kQ; a++) {
                const float v = Cs[k] * f[a] + wq(a) * (Vx[k] * (float)ex(a) + Vy[k] * (float)ey(a));
                o[P.off_plane[k * kQ + a]] = v;
            }
        }
    } else {
        float v[27];
#pragma unroll
        for (int k = 0; k < kNF; k++)
#pragma unroll
            for (int a = 0; a < kQ; a++)
                v[9 * k + a] = Cs[k] * f[a] + wq(a) * (Vx[k] * (float)ex(a) + Vy[k] * (float)ey(a));
        store_node<STORE>(fout, P.N, i, v);
    }
}



// Eq.(10) stress on the halo-1 region of a pure tile from the phase fields of its halo-2 region
// (float path: no solid, no float-float words)
template <int TX, int TY>
__device__ __forceinline__ void stress_halo1(const Params& P, const float (*s_ch)[TY + 4][TX + 4],
                                             const float (*s_rho)[TX + 4], float (*s_txx)[TX + 2],
                                             float (*s_txy)[TX + 2], float (*s_tyy)[TX + 2], int tid)
{
    constexpr int CX = TX + 4, RX = TX + 2, RY = TY + 2;
    for (int r = tid; r < RX * RY; r += TX * TY) {
        const int rx = r % RX, ry = r / RX;
        const int cx = rx + 1, cy = ry + 1;
        const float rho = s_rho[cy][cx];
        float c[kNF], gxk[kNF], gyk[kNF];
#pragma unroll
        for (int k = 0; k < kNF; k++) {
            c[k] = s_ch[k][cy][cx];
            grad9_f<CX>(s_ch[k], cx, cy, gxk[k], gyk[k]);
        }
        float Txx = 0.f, Txy = 0.f, Tyy = 0.f;
        const float rho2 = rho * rho;
        pair_stress(P.sig01, c[0], c[1], gxk[0], gyk[0], gxk[1], gyk[1], rho2, Txx, Txy, Tyy);
        pair_stress(P.sig02, c[0], c[2], gxk[0], gyk[0], gxk[2], gyk[2], rho2, Txx, Txy, Tyy);
        pair_stress(P.sig12, c[1], c[2], gxk[1], gyk[1], gxk[2], gyk[2], rho2, Txx, Txy, Tyy);
        s_txx[ry][rx] = Txx;
        s_txy[ry][rx] = Txy;
        s_tyy[ry][rx] = Tyy;
    }
}

// Pure FP32 tiles through the tensor memory accelerator, persistent: block b handles tiles
// b, b + gridDim.x, ...  For each tile the 27 pull-source planes over the (TX + 8) x (TY + 6)
// box starting at (x0 - 4, y0 - 3) -- x rounded down to a 16-byte boundary -- arrive by one bulk
// tensor copy completing on an mbarrier, and the pulls read them at compile-time offsets.  The
// box is needed only for the pulls: as soon as they are done the copy of the next tile's box is
// issued, so it lands while this tile computes its stress, force, collision and recolouring.
// The 27 output planes are written directly (STAGE = false: 72 KB of shared memory per block)
// or staged in shared memory and written by one bulk tensor store per tile (STAGE = true,
// 100 KB).  kTmaBlocksPerSm = 2 blocks per SM: three (the most that fit) measured slower.
// Same arithmetic as k_step<PURE>, so the two give identical results.
template <int TX, int TY, bool STAGE>
__global__ void __launch_bounds__(TX* TY, kTmaBlocksPerSm) k_step_tma(const Params P, const int* __restrict__ tiles,
                                                        const int ntiles, float* __restrict__ fout,
                                                        float* __restrict__ uout,
                                                        const __grid_constant__ CUtensorMap tm_in_a,
                                                        const __grid_constant__ CUtensorMap tm_in_b,
                                                        const __grid_constant__ CUtensorMap tm_out)
{
    constexpr int NT = TX * TY;
    constexpr int CX = TX + 4, CY = TY + 4;  // phase-field region (halo 2)
    constexpr int RX = TX + 2, RY = TY + 2;  // stress region (halo 1)
    constexpr int BX = TX + 8, BY = TY + 6;  // pull-source box
    constexpr int NBOX = kQ * kNF * BY * BX;
    constexpr int NBOXP = (NBOX + 31) / 32 * 32;  // keeps the staging buffer 128-byte aligned
    constexpr int NRING = CX * CY - TX * TY;      // halo-2 ring: one node per thread at most
    static_assert(NRING <= NT, "the ring of the halo-2 region must not exceed one node per thread");
    static_assert((kTmaPlanesA * BY * BX * 4) % 128 == 0, "second copy must start 128-byte aligned");
    __shared__ float s_ch[kNF][CY][CX];
    __shared__ float s_rho[CY][CX];
    __shared__ float s_txx[RY][RX], s_txy[RY][RX], s_tyy[RY][RX];
    __shared__ __align__(8) uint64_t s_bar[2];  // completion of copy A (planes 0..13) and B (14..26)
    __shared__ int s_flags[2];                  // fluids present in the tile, by iteration parity
    extern __shared__ unsigned char dsm[];
    float* box = reinterpret_cast<float*>(dsm + ((128u - (smem_u32(dsm) & 127u)) & 127u));  // [27][BY][BX]
    float* outb = box + NBOXP;                                                              // [27][TY][TX]

    const int tid = threadIdx.x + TX * threadIdx.y;
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int ntx = (P.nx + TX - 1) / TX;
    const uint32_t bar_a = smem_u32(&s_bar[0]), bar_b = smem_u32(&s_bar[1]);
    if ((int)blockIdx.x >= ntiles) return;
    auto issue_a = [&](int tile) {
        const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
        mbar_arrive_expect_tx(bar_a, (uint32_t)(kTmaPlanesA * BY * BX) * 4u);
        tma_load_3d(smem_u32(box), &tm_in_a, x0 - 4, y0 - 3, 0, bar_a);
    };
    auto issue_b = [&](int tile) {
        const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
        mbar_arrive_expect_tx(bar_b, (uint32_t)((kQ * kNF - kTmaPlanesA) * BY * BX) * 4u);
        tma_load_3d(smem_u32(box + kTmaPlanesA * BY * BX), &tm_in_b, x0 - 4, y0 - 3, kTmaPlanesA, bar_b);
    };
    int tile = tiles[blockIdx.x];
    int last_a = 0, last_b = 0;  // tile iteration of the latest copy into each part (thread 0)
    if (tid == 0) {
        mbar_init(bar_a, 1);
        mbar_init(bar_b, 1);
        fence_mbar_init();
        issue_a(tile);
        issue_b(tile);
        s_flags[0] = s_flags[1] = 0;
    }
    __syncthreads();

    // bounded wait for one part of iteration j's box, with the same outcome in every thread; on
    // a timeout the error bit is set and thread 0 gives the copies it issued a second bounded
    // wait, so that none lands in a later block's shared memory
    auto wait_part = [&](uint32_t bar, int j) -> bool {
        bool ok = false;
        for (int it = 0; it < P.wait_polls && !ok; it++) ok = mbar_try_wait(bar, j & 1);
        if (!__syncthreads_or(!ok)) return true;
        if (tid == 0) {
            atomicOr(P.err, 1);
            for (int it = 0; it < kWaitLimit && !mbar_try_wait(bar_a, last_a & 1); it++) {
            }
            for (int it = 0; it < kWaitLimit && !mbar_try_wait(bar_b, last_b & 1); it++) {
            }
            bulk_wait_read0();
        }
        return false;
    };
    // pulls of the node at (cx, cy) of the phase-field region from the planes p of the box with
    // P0 <= p < P1 (q[p], p = 9 k + a)
    auto pull = [&](int cx, int cy, float q[27], int p0, int p1) {
#pragma unroll
        for (int p = 0; p < kQ * kNF; p++) {
            const int a = p % kQ;
            if (p >= p0 && p < p1) q[p] = box[(p * BY + cy + 1 - ey(a)) * BX + cx + 2 - ex(a)];
        }
    };
    // densities and phase fields of one node; returns which fluids it holds (bit k: rho_k != 0)
    auto store_phase = [&](int cx, int cy, float r0, float r1, float r2) {
        const float rho = (r0 + r1) + r2;
        const float ir = __fdividef(1.0f, rho);
        s_ch[0][cy][cx] = r0 * ir;
        s_ch[1][cy][cx] = r1 * ir;
        s_ch[2][cy][cx] = r2 * ir;
        s_rho[cy][cx] = rho;
        return (r0 != 0.0f ? 1 : 0) | (r1 != 0.0f ? 2 : 0) | (r2 != 0.0f ? 4 : 0);
    };

    // the ring node of this thread (a fixed position in every tile)
    const bool ring = tid < NRING;
    int rcx = 0, rcy = 0;
    if (ring) {
        if (tid < 2 * CX) {
            rcx = tid % CX;
            rcy = tid / CX;
        } else if (tid < 4 * CX) {
            rcx = (tid - 2 * CX) % CX;
            rcy = CY - 2 + (tid - 2 * CX) / CX;
        } else {
            const int rr0 = tid - 4 * CX;  // 4 * TY side nodes
            const int side = rr0 / (2 * TY), rr = rr0 % (2 * TY);
            rcy = 2 + rr / 2;
            rcx = side == 0 ? (rr & 1) : CX - 2 + (rr & 1);
        }
    }

    int j = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, j++) {
        // the next tile's index is read now and used after the pulls
        const bool more = t + (int)gridDim.x < ntiles;
        const int next = more ? tiles[t + gridDim.x] : 0;
        const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;

        // ---- phase 1: pulls, densities and phase fields of the halo-2 region, in two passes
        // over the two parts of the box (the sums keep the order of the one-pass kernel) ----
        if (!wait_part(bar_a, j)) return;
        float q[27];
        float ra0 = 0.0f, ra1 = 0.0f;  // ring node: rho_0 and the planes 9..13 part of rho_1
        if (ring) {
            pull(rcx, rcy, q, 0, kTmaPlanesA);
            ra0 = ((q[0] + (q[1] + q[3])) + (q[2] + q[4])) + ((q[5] + q[7]) + (q[6] + q[8]));
            ra1 = (q[9] + (q[10] + q[12])) + (q[11] + q[13]);
        }
        float f[kQ], r0, r1, r2;
        pull(lx + 2, ly + 2, q, 0, kTmaPlanesA);
#pragma unroll
        for (int a = 0; a < kQ; a++) f[a] = a < 5 ? q[a] + q[9 + a] : q[a];
        r0 = ((q[0] + (q[1] + q[3])) + (q[2] + q[4])) + ((q[5] + q[7]) + (q[6] + q[8]));
        r1 = (q[9] + (q[10] + q[12])) + (q[11] + q[13]);
        // the wait for part B is a barrier: past it every thread has pulled from part A, which
        // is then free for the next tile's copy while part B is pulled and this tile computes
        if (!wait_part(bar_b, j)) return;
        if (tid == 0 && more) {
            issue_a(next);
            last_a = j + 1;
        }
        int present = 0;
        if (ring) {
            pull(rcx, rcy, q, kTmaPlanesA, kQ * kNF);
            const float rb1 = ra1 + ((q[14] + q[16]) + (q[15] + q[17]));
            const float rb2 = ((q[18] + (q[19] + q[21])) + (q[20] + q[22])) + ((q[23] + q[25]) + (q[24] + q[26]));
            present |= store_phase(rcx, rcy, ra0, rb1, rb2);
        }
        pull(lx + 2, ly + 2, q, kTmaPlanesA, kQ * kNF);
#pragma unroll
        for (int a = 0; a < kQ; a++) f[a] = (a < 5 ? f[a] : f[a] + q[9 + a]) + q[18 + a];
        r1 = r1 + ((q[14] + q[16]) + (q[15] + q[17]));
        r2 = ((q[18] + (q[19] + q[21])) + (q[20] + q[22])) + ((q[23] + q[25]) + (q[24] + q[26]));
        present |= store_phase(lx + 2, ly + 2, r0, r1, r2);
        const bool mixed = fluids_present(present, s_flags, j, tid) != 1;
        if (tid == 0 && more) {
            issue_b(next);
            last_b = j + 1;
        }

        // ---- phase 2: stress tensor of Eq.(10) on the halo-1 region ----
        if (mixed) stress_halo1<TX, TY>(P, s_ch, s_rho, s_txx, s_txy, s_tyy, tid);
        // the previous tile's bulk store must have read the staging buffer before it is refilled
        if (STAGE && tid == 0) bulk_wait_read0();
        __syncthreads();

        // ---- phase 3: force, collision, recolouring into the staging buffer ----
        float Fx = 0.0f, Fy = 0.0f, g[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (mixed) {
            div_stress<RX>(s_txx, s_txy, s_tyy, lx + 1, ly + 1, Fx, Fy);
            // own colour gradients, the same stencil as phase 2 on the same phase fields (the
            // next tile overwrites them only after the barrier at the top of the loop)
#pragma unroll
            for (int k = 0; k < kNF; k++) grad9_f<CX>(s_ch[k], lx + 2, ly + 2, g[2 * k], g[2 * k + 1]);
        }
        float ux, uy;
        const Recolour rc = collide_node(P, f, r0, r1, r2, Fx, Fy, g, ux, uy);
        if (uout) {
            const int i = (y0 + ly) * P.nx + x0 + lx;
            uout[i] = ux;
            uout[P.N + i] = uy;
        }
        tile = next;
        if constexpr (STAGE) {
            float* o = outb + ly * TX + lx;
#pragma unroll
            for (int k = 0; k < kNF; k++)
#pragma unroll
                for (int a = 0; a < kQ; a++)
                    o[(k * kQ + a) * TY * TX] =
                        rc.C[k] * f[a] + wq(a) * (rc.Vx[k] * (float)ex(a) + rc.Vy[k] * (float)ey(a));
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                tma_store_3d(&tm_out, x0, y0, 0, smem_u32(outb));
                bulk_commit();
            }
        } else {
            float* o = fout + (y0 + ly) * P.nx + x0 + lx;
#pragma unroll
            for (int k = 0; k < kNF; k++)
#pragma unroll
                for (int a = 0; a < kQ; a++)
                    o[P.off_plane[k * kQ + a]] =
                        rc.C[k] * f[a] + wq(a) * (rc.Vx[k] * (float)ex(a) + rc.Vy[k] * (float)ey(a));
        }
    }
    if (STAGE && tid == 0) bulk_wait_read0();
}

// ---- named barriers of one consumer group and a plain mbarrier arrival ----
__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// barrier of the group that also ORs a predicate over its threads
__device__ __forceinline__ bool group_or(bool v, int id, int nthreads)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Pure FP32 tiles through a ring of bulk tensor copies, warp-specialised: one producer warp and
// two consumer groups of TX x TY threads per block, one block per SM (persistent).  Tile j of the
// block (tiles[blockIdx.x + j gridDim.x]) lands in ring buffer j % 3 -- its 27-plane pull box,
// (TX + 8) x (TY + 6) nodes from (x0 - 4, y0 - 3), by one copy -- and is computed by group j % 2.
// A group releases its buffer as soon as its pulls are done (one arrival per warp on the buffer's
// "empty" barrier), and the producer refills it at once with tile j + 3, so up to three boxes are
// in flight or waiting while the groups compute their force, collision and recolouring.  The
// "full" barrier of tile j is full[j % 6]: its tiles j, j + 6, ... are consumed in order by the
// same group, so a wait never meets a phase two behind (no parity aliasing).  Every wait is
// bounded: a consumer that gives up sets the error bit and its group returns; the producer gives
// up on a buffer that is never released, and before exiting it waits (full limit) for every copy
// it issued, so no copy lands in the shared memory of a later block.  The arithmetic is that of
// k_step_tma and k_step<PURE>, so the results are identical.
// Each warp also records the fluids its nodes hold (one byte of pres_out[tile] per warp); when
// the 3 x 3 tiles around a tile held one fluid in the step's input (pres_in, read by the
// producer), the tile is single-fluid after the pull, and its consumers skip the halo's phase
// fields and the presence barrier, which only decide that (same results, fewer instructions).
constexpr int kRingBufs = 3;
template <int TX, int TY>
__global__ void __launch_bounds__(2 * TX * TY + 32, 1) k_step_ring(const Params P, const int* __restrict__ tiles,
                                                                    const int ntiles, float* __restrict__ fout,
                                                                    float* __restrict__ uout,
                                                                    const __grid_constant__ CUtensorMap tm_in,
                                                                    const uint64_t* __restrict__ pres_in,
                                                                    uint64_t* __restrict__ pres_out)
{
    constexpr int NT = TX * TY;               // threads of a consumer group
    constexpr int NW = NT / 32;               // warps of a consumer group
    constexpr int CX = TX + 4, CY = TY + 4;  // phase-field region (halo 2)
    constexpr int RX = TX + 2, RY = TY + 2;  // stress region (halo 1)
    constexpr int BX = TX + 8, BY = TY + 6;  // pull-source box
    constexpr int NBOX = kQ * kNF * BY * BX;
    constexpr int NBOXP = (NBOX + 31) / 32 * 32;  // keeps every buffer 128-byte aligned
    constexpr int NRING = CX * CY - TX * TY;
    static_assert(NRING <= NT, "the ring of the halo-2 region must not exceed one node per thread");
    static_assert(NT % 32 == 0, "whole warps per group");
    __shared__ float s_ch[2][kNF][CY][CX];
    __shared__ float s_rho[2][CY][CX];
    __shared__ float s_txx[2][RY][RX], s_txy[2][RY][RX], s_tyy[2][RY][RX];
    __shared__ __align__(8) uint64_t s_full[2 * kRingBufs], s_empty[kRingBufs];
    __shared__ int s_flags[2][2];
    __shared__ int s_single[2 * kRingBufs];  // by full-barrier slot: the tile's 3 x 3 tiles hold one fluid
    __shared__ int s_tile[2 * kRingBufs];    // by full-barrier slot: the tile
    extern __shared__ unsigned char dsm[];
    float* ring = reinterpret_cast<float*>(dsm + ((128u - (smem_u32(dsm) & 127u)) & 127u));  // [3][27][BY][BX]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntx = (P.nx + TX - 1) / TX;
    if ((int)blockIdx.x >= ntiles) return;
    const int njobs = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    if (threadIdx.x == 0) {
        for (int m = 0; m < 2 * kRingBufs; m++) mbar_init(smem_u32(&s_full[m]), 1);
        for (int b = 0; b < kRingBufs; b++) mbar_init(smem_u32(&s_empty[b]), NW);
        fence_mbar_init();
        s_flags[0][0] = s_flags[0][1] = s_flags[1][0] = s_flags[1][1] = 0;
    }
    __syncthreads();

    // ---------------- producer warp ----------------
    if (warp == 2 * NW) {
        if (lane != 0) return;
        // fluids stored in the 3 x 3 tiles around a tile (a pure tile is inner, so they exist)
        auto around = [&](int t) {
            uint64_t nb = 0;
#pragma unroll
            for (int dy = -1; dy <= 1; dy++)
#pragma unroll
                for (int dx = -1; dx <= 1; dx++) nb |= pres_in[t + dy * ntx + dx];
            nb |= nb >> 32;
            nb |= nb >> 16;
            nb |= nb >> 8;
            return (int)(nb & 7u);
        };
        // tile indices are loaded two tiles ahead and the fluids around a tile one tile ahead, so
        // that no load waits on another within a tile and their latency passes while the
        // producer waits for a free buffer
        auto tile_at = [&](int jj) { return jj < njobs ? tiles[blockIdx.x + jj * gridDim.x] : 0; };
        int tile_n = tile_at(0), tile_nn = tile_at(1);
        int around_n = around(tile_n);
        int issued = 0;
        for (int j = 0; j < njobs; j++) {
            const int b = j % kRingBufs;
            if (j >= kRingBufs) {
                // buffer b is free once the group that computed tile j - 3 has pulled from it
                bool ok = false;
                const uint32_t par = (uint32_t)((j / kRingBufs - 1) & 1);
                for (int it = 0; it < P.wait_polls && !ok; it++) ok = mbar_try_wait(smem_u32(&s_empty[b]), par);
                if (!ok) {
                    atomicOr(P.err, 1);
                    break;
                }
            }
            const int tile = tile_n;
            const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
            // written before the arrive, whose release the consumers' wait acquires
            s_single[j % (2 * kRingBufs)] = __popc((unsigned)around_n) == 1;
            s_tile[j % (2 * kRingBufs)] = tile;
            const uint32_t full = smem_u32(&s_full[j % (2 * kRingBufs)]);
            mbar_arrive_expect_tx(full, (uint32_t)NBOX * 4u);
            tma_load_3d(smem_u32(ring + b * NBOXP), &tm_in, x0 - 4, y0 - 3, 0, full);
            issued = j + 1;
            tile_n = tile_nn;
            tile_nn = tile_at(j + 2);
            if (j + 1 < njobs) around_n = around(tile_n);
        }
        // every copy issued has landed before the block may exit
        for (int m = 0; m < 2 * kRingBufs; m++) {
            int last = -1;
            for (int j = issued - 1; j >= 0 && j >= issued - 2 * kRingBufs; j--)
                if (j % (2 * kRingBufs) == m) {
                    last = j;
                    break;
                }
            if (last < 0) continue;
            const uint32_t par = (uint32_t)((last / (2 * kRingBufs)) & 1);
            for (int it = 0; it < kWaitLimit && !mbar_try_wait(smem_u32(&s_full[m]), par); it++) {
            }
        }
        return;
    }

    // ---------------- consumer groups ----------------
    const int g = warp / NW;
    const int bar_id = 1 + g;  // named barrier of the group (0 is the block-wide one)
    const int tid = threadIdx.x - g * NT;
    const int lx = tid % TX, ly = tid / TX;
    float(*ch)[CY][CX] = s_ch[g];
    float(*rh)[CX] = s_rho[g];
    int* flags = s_flags[g];
    const bool ring_node = tid < NRING;
    int rcx = 0, rcy = 0;
    if (ring_node) {
        if (tid < 2 * CX) {
            rcx = tid % CX;
            rcy = tid / CX;
        } else if (tid < 4 * CX) {
            rcx = (tid - 2 * CX) % CX;
            rcy = CY - 2 + (tid - 2 * CX) / CX;
        } else {
            const int rr0 = tid - 4 * CX;  // 4 * TY side nodes
            const int side = rr0 / (2 * TY), rr = rr0 % (2 * TY);
            rcy = 2 + rr / 2;
            rcx = side == 0 ? (rr & 1) : CX - 2 + (rr & 1);
        }
    }
    auto store_phase = [&](int cx, int cy, float r0, float r1, float r2) {
        const float rho = (r0 + r1) + r2;
        const float ir = __fdividef(1.0f, rho);
        ch[0][cy][cx] = r0 * ir;
        ch[1][cy][cx] = r1 * ir;
        ch[2][cy][cx] = r2 * ir;
        rh[cy][cx] = rho;
        return (r0 != 0.0f ? 1 : 0) | (r1 != 0.0f ? 2 : 0) | (r2 != 0.0f ? 4 : 0);
    };

    for (int j = g, jj = 0; j < njobs; j += 2, jj++) {
        const float* box = ring + (j % kRingBufs) * NBOXP;
        {
            bool ok = false;
            const uint32_t full = smem_u32(&s_full[j % (2 * kRingBufs)]);
            const uint32_t par = (uint32_t)((j / (2 * kRingBufs)) & 1);
            for (int it = 0; it < P.wait_polls && !ok; it++) ok = mbar_try_wait(full, par);
            if (group_or(!ok, bar_id, NT)) {
                if (tid == 0) atomicOr(P.err, 1);
                return;
            }
        }
        const int tile = s_tile[j % (2 * kRingBufs)];
        const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
        // One fluid in the 3 x 3 tiles around: every node of the halo-2 region holds that fluid
        // alone after the pull (a fluid absent from a node's sources stays absent), so the tile
        // is not mixed, and its phase fields, which only the mixed path reads, are skipped.
        const bool single = s_single[j % (2 * kRingBufs)];
        if (single && tid == 0) flags[(jj + 1) & 1] = 0;  // all threads are past the last tile
        // ---- phase 1: pulls, densities and phase fields of the halo-2 region ----
        auto pull = [&](int cx, int cy, float q[27]) {
#pragma unroll
            for (int p = 0; p < kQ * kNF; p++) {
                const int a = p % kQ;
                q[p] = box[(p * BY + cy + 1 - ey(a)) * BX + cx + 2 - ex(a)];
            }
        };
        int present = 0;
        float q[27];
        if (ring_node && !single) {
            pull(rcx, rcy, q);
            const float a0 = ((q[0] + (q[1] + q[3])) + (q[2] + q[4])) + ((q[5] + q[7]) + (q[6] + q[8]));
            const float a1 = ((q[9] + (q[10] + q[12])) + (q[11] + q[13])) + ((q[14] + q[16]) + (q[15] + q[17]));
            const float a2 = ((q[18] + (q[19] + q[21])) + (q[20] + q[22])) + ((q[23] + q[25]) + (q[24] + q[26]));
            present |= store_phase(rcx, rcy, a0, a1, a2);
        }
        float f[kQ], r0, r1, r2;
        pull(lx + 2, ly + 2, q);
        // the box is not read again: release it to the producer (all lanes of the warp are done)
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&s_empty[j % kRingBufs]));
#pragma unroll
        for (int a = 0; a < kQ; a++) f[a] = (q[a] + q[9 + a]) + q[18 + a];
        r0 = ((q[0] + (q[1] + q[3])) + (q[2] + q[4])) + ((q[5] + q[7]) + (q[6] + q[8]));
        r1 = ((q[9] + (q[10] + q[12])) + (q[11] + q[13])) + ((q[14] + q[16]) + (q[15] + q[17]));
        r2 = ((q[18] + (q[19] + q[21])) + (q[20] + q[22])) + ((q[23] + q[25]) + (q[24] + q[26]));
        // the fluids this warp's nodes hold, for the tiles around this one in the next step
        {
            const int own = (r0 != 0.0f ? 1 : 0) | (r1 != 0.0f ? 2 : 0) | (r2 != 0.0f ? 4 : 0);
            const int w = __reduce_or_sync(0xffffffffu, own);
            if (lane == 0) reinterpret_cast<uint8_t*>(pres_out + tile)[tid >> 5] = (uint8_t)w;
        }
        bool mixed = false;
        if (!single) {
            present |= store_phase(lx + 2, ly + 2, r0, r1, r2);
            // fluids present in the group's phase-field region (one barrier; see fluids_present)
            int cnt;
            {
                const int w = __reduce_or_sync(0xffffffffu, present);
                if (lane == 0 && w) atomicOr(&flags[jj & 1], w);
                group_sync(bar_id, NT);
                const int v = flags[jj & 1];
                if (tid == 0) flags[(jj + 1) & 1] = 0;
                cnt = __popc(v & 7);
            }
            mixed = cnt != 1;

            // ---- phase 2: stress tensor of Eq.(10) on the halo-1 region ----
            if (mixed) stress_halo1<TX, TY>(P, ch, rh, s_txx[g], s_txy[g], s_tyy[g], tid);
            group_sync(bar_id, NT);
        }

        // ---- phase 3: force, collision, recolouring, 27 stores per node ----
        float Fx = 0.0f, Fy = 0.0f, gr[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (mixed) {
            div_stress<RX>(s_txx[g], s_txy[g], s_tyy[g], lx + 1, ly + 1, Fx, Fy);
#pragma unroll
            for (int k = 0; k < kNF; k++) grad9_f<CX>(ch[k], lx + 2, ly + 2, gr[2 * k], gr[2 * k + 1]);
        }
        float ux, uy;
        const Recolour rc = collide_node(P, f, r0, r1, r2, Fx, Fy, gr, ux, uy);
        if (uout) {
            const int i = (y0 + ly) * P.nx + x0 + lx;
            uout[i] = ux;
            uout[P.N + i] = uy;
        }
        float* o = fout + (y0 + ly) * P.nx + x0 + lx;
#pragma unroll
        for (int k = 0; k < kNF; k++)
#pragma unroll
            for (int a = 0; a < kQ; a++)
                o[P.off_plane[k * kQ + a]] =
                    rc.C[k] * f[a] + wq(a) * (rc.Vx[k] * (float)ex(a) + rc.Vy[k] * (float)ey(a));
        // the next tile's phase fields overwrite ch / rh only after its own barriers; the stress
        // arrays after its phase-1 barrier, by which time every thread here has read them
    }
}

// ------------------------------------------------------------------------------------------
// initial state, fields, diagnostics
// ------------------------------------------------------------------------------------------
// Stored populations whose pull gives f_ak(x) = w_a rho_k(x): population a of node y is
// w_a rho_k at its destination y + e_a (or at y itself when the destination is solid).
template <int STORE>
__global__ void k_init(const Params P, const double* __restrict__ rho,
                       const uint8_t* __restrict__ type, const Pop f)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int x = i % P.nx, y = i / P.nx;
    const bool solid = type[i] & 2;
    float v[27];
#pragma unroll
    for (int a = 0; a < kQ; a++) {
        const Loc d = locate(P, x + ex(a), y + ey(a));
#pragma unroll
        for (int k = 0; k < kNF; k++) {
            float val = 0.0f;
            if (!solid) {
                if (d.kind == 1 || (d.kind == 0 && (type[d.idx] & 2)))
                    val = wq(a) * (float)rho[(long long)k * P.N + i];
                else if (d.kind == 0)
                    val = wq(a) * (float)rho[(long long)relabel(k, d.par) * P.N + d.idx];
            }
            v[9 * k + a] = val;
        }
    }
    store_node<STORE>(f, P.N, i, v);
}

template <class S>
__global__ void k_fields(const Params P, const S st, const uint8_t* __restrict__ type,
                         float* __restrict__ rho_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    float r[kNF] = {0.f, 0.f, 0.f};
    if (!(type[i] & 2)) {
        float p[27];
        pull_global(P, st, type, i % P.nx, i / P.nx, p);
#pragma unroll
        for (int k = 0; k < kNF; k++)
#pragma unroll
            for (int a = 0; a < kQ; a++) r[k] += p[9 * k + a];
    }
#pragma unroll
    for (int k = 0; k < kNF; k++) rho_out[(long long)k * P.N + i] = r[k];
}

// post-streaming populations of every fluid node (0 at solid nodes)
template <class S>
__global__ void k_get_state(const Params P, const S st, const uint8_t* __restrict__ type,
                            float* __restrict__ post)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    float p[27];
    if (!(type[i] & 2)) {
        pull_global(P, st, type, i % P.nx, i / P.nx, p);
    } else {
#pragma unroll
        for (int j = 0; j < 27; j++) p[j] = 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 27; j++) post[(long long)j * P.N + i] = p[j];
}

// stored populations whose pull reproduces the post-streaming state `post`: population a of
// node y is post_a at its destination y + e_a, or post_opp(a) at y when that destination is solid
template <int STORE>
__global__ void k_set_state(const Params P, const double* __restrict__ post,
                            const uint8_t* __restrict__ type, const Pop f)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int x = i % P.nx, y = i / P.nx;
    const bool solid = type[i] & 2;
    float v[27];
#pragma unroll
    for (int a = 0; a < kQ; a++) {
        const Loc d = locate(P, x + ex(a), y + ey(a));
#pragma unroll
        for (int k = 0; k < kNF; k++) {
            float val = 0.0f;
            if (!solid) {
                if (d.kind == 1 || (d.kind == 0 && (type[d.idx] & 2)))
                    val = (float)post[(long long)(k * kQ + opp(a)) * P.N + i];
                else if (d.kind == 0)
                    val = (float)post[(long long)(relabel(k, d.par) * kQ + a) * P.N + d.idx];
            }
            v[9 * k + a] = val;
        }
    }
    store_node<STORE>(f, P.N, i, v);
}

constexpr int kDiagThreads = 256;

// out per block: [0..2] sum rho_k, [3] sum x rho_0, [4] sum y rho_0, [5] max|u|, [6] min rho,
// [7] non-finite count
template <class S>
__global__ void __launch_bounds__(kDiagThreads) k_diag(const Params P, const S st,
                                                       const uint8_t* __restrict__ type,
                                                       const float* __restrict__ u,
                                                       double* __restrict__ partials)
{
    double acc[8] = {0, 0, 0, 0, 0, 0, DBL_MAX, 0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < P.N;
         i += (long long)gridDim.x * blockDim.x) {
        if (type[i] & 2) continue;
        const int x = (int)(i % P.nx), y = (int)(i / P.nx);
        float p[27];
        pull_global(P, st, type, x, y, p);
        double r[kNF];
#pragma unroll
        for (int k = 0; k < kNF; k++) {
            float s = 0.f;
#pragma unroll
            for (int a = 0; a < kQ; a++) s += p[9 * k + a];
            r[k] = s;
            acc[k] += s;
            if (!isfinite(s)) acc[7] += 1.0;
        }
        acc[3] += x * r[0];
        acc[4] += y * r[0];
        const double um = sqrt((double)u[i] * u[i] + (double)u[P.N + i] * u[P.N + i]);
        acc[5] = fmax(acc[5], um);
        acc[6] = fmin(acc[6], r[0] + r[1] + r[2]);
    }
    __shared__ double sh[8][kDiagThreads];
#pragma unroll
    for (int j = 0; j < 8; j++) sh[j][threadIdx.x] = acc[j];
    __syncthreads();
    for (int s = kDiagThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
#pragma unroll
            for (int j = 0; j < 5; j++) sh[j][threadIdx.x] += sh[j][threadIdx.x + s];
            sh[5][threadIdx.x] = fmax(sh[5][threadIdx.x], sh[5][threadIdx.x + s]);
            sh[6][threadIdx.x] = fmin(sh[6][threadIdx.x], sh[6][threadIdx.x + s]);
            sh[7][threadIdx.x] += sh[7][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x < 8) partials[blockIdx.x * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

// one warp: lane j strides over the block partials, then a shuffle reduction
__global__ void k_diag_final(const int nb, const double* __restrict__ partials, double* __restrict__ out)
{
    double acc[8] = {0, 0, 0, 0, 0, 0, DBL_MAX, 0};
    for (int b = threadIdx.x; b < nb; b += 32) {
        const double* q = partials + 8 * b;
#pragma unroll
        for (int j = 0; j < 5; j++) acc[j] += q[j];
        acc[5] = fmax(acc[5], q[5]);
        acc[6] = fmin(acc[6], q[6]);
        acc[7] += q[7];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int j = 0; j < 5; j++) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
        acc[5] = fmax(acc[5], __shfl_xor_sync(0xffffffffu, acc[5], o));
        acc[6] = fmin(acc[6], __shfl_xor_sync(0xffffffffu, acc[6], o));
        acc[7] += __shfl_xor_sync(0xffffffffu, acc[7], o);
    }
    if (threadIdx.x == 0)
        for (int j = 0; j < 8; j++) out[j] = acc[j];
}

}  // namespace

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
// call fn with the Store type of the storage format
template <class Fn>
void with_store(int store, const Pop& p, long long N, Fn fn)
{
    if (store == kStoreF32)
        fn(Store<kStoreF32>(p, N));
    else if (store == kStoreF16)
        fn(Store<kStoreF16>(p, N));
    else
        fn(Store<kStoreBF16>(p, N));
}

void launch_wet(int store, const Params& P, int nw, const int* widx, const double* wnrm,
                const float* wang, const Pop& f, const uint8_t* type, double* Cw, WetCache* cache,
                cudaStream_t s, double* Cw_prev)
{
    if (nw <= 0) return;
    const long long threads = 4LL * nw;
    with_store(store, f, P.N, [&](auto st) {
        k_wet<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(P, nw, widx, wnrm, wang, st, type, Cw, cache, Cw_prev);
    });
}

__global__ void k_wet_cache_reset(WetCache* cache, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);  // never equal
        cache[i].th = nan;
        cache[i].wm = nan;
        cache[i].wl = nan;
    }
}

void reset_wet_cache(WetCache* cache, int nw, cudaStream_t s)
{
    if (nw <= 0) return;
    const int n = 4 * nw;
    k_wet_cache_reset<<<(n + 255) / 256, 256, 0, s>>>(cache, n);
}

void launch_wet_init(int store, const Params& P, int nw, const int* widx, const Pop& f,
                     const uint8_t* type, double* Cw, cudaStream_t s)
{
    if (nw <= 0) return;
    with_store(store, f, P.N, [&](auto st) {
        k_wet_init<<<(nw + 127) / 128, 128, 0, s>>>(P, nw, widx, st, type, Cw);
    });
}

template <int STORE>
static void launch_step_t(const Params& P, const int* tiles, int ntiles, int kind, const Pop& fin,
                          const Pop& fout, const uint8_t* type, const double* Cw, float* u,
                          const uint64_t* pres_in, uint64_t* pres_out, cudaStream_t s)
{
    if (kind == kTilesPure)
        k_step<kTX, kTY, true, true, STORE>
            <<<ntiles, dim3(kTX, kTY), 0, s>>>(P, tiles, fin, fout, type, Cw, u, pres_in, pres_out);
    else if (kind == kTilesWall)
        k_step<kTX, kTY, false, true, STORE>
            <<<ntiles, dim3(kTX, kTY), 0, s>>>(P, tiles, fin, fout, type, Cw, u, pres_in, pres_out);
    else
        k_step<kTX, kTY, false, false, STORE>
            <<<ntiles, dim3(kTX, kTY), 0, s>>>(P, tiles, fin, fout, type, Cw, u, pres_in, pres_out);
}

void launch_step(int store, const Params& P, const int* tiles, int ntiles, int kind, const Pop& fin,
                 const Pop& fout, const uint8_t* type, const double* Cw, float* u, const uint64_t* pres_in,
                 uint64_t* pres_out, cudaStream_t s)
{
    if (ntiles <= 0) return;
    if (store == kStoreF32)
        launch_step_t<kStoreF32>(P, tiles, ntiles, kind, fin, fout, type, Cw, u, pres_in, pres_out, s);
    else if (store == kStoreF16)
        launch_step_t<kStoreF16>(P, tiles, ntiles, kind, fin, fout, type, Cw, u, pres_in, pres_out, s);
    else
        launch_step_t<kStoreBF16>(P, tiles, ntiles, kind, fin, fout, type, Cw, u, pres_in, pres_out, s);
}

// Pure tiles of the 16-bit storage through the tensor memory accelerator, persistent, with the
// tile loop of k_step_tma: per tile one bulk copy of the FP32 densities (box (TX + 8) x (TY + 6)
// x 3 from (x0 - 4, y0 - 3)) and one of the 24 planes of 16-bit offsets (box (TX + 16) x (TY + 6)
// x 24 from (x0 - 8, y0 - 3): a 16-bit box must start on a 16-byte boundary) complete on an
// mbarrier; a pull rebuilds w_a rho_k + offset at its source, the rest population from the
// node's own offsets, exactly as the plain kernel does from global memory.  A warp's reads of
// one plane are consecutive 16-bit words (no bank conflicts).  The next tile's boxes are fetched
// as soon as the pulls are done.
template <int TX, int TY, int STORE>
__global__ void __launch_bounds__(TX* TY, kTma16BlocksPerSm) k_step_tma16(const Params P, const int* __restrict__ tiles,
                                                            const int ntiles, const Pop fout,
                                                            float* __restrict__ uout,
                                                            const __grid_constant__ CUtensorMap tm_rho,
                                                            const __grid_constant__ CUtensorMap tm_off,
                                                            const uint64_t* __restrict__ pres_in,
                                                            uint64_t* __restrict__ pres_out)
{
    constexpr int NT = TX * TY;
    constexpr int CX = TX + 4, CY = TY + 4;
    constexpr int RX = TX + 2, RY = TY + 2;
    constexpr int BX = TX + 8, BY = TY + 6;          // density box
    constexpr int OX = TX + 16;                      // width of the offset box
    constexpr int NR = kNF * BY * BX;                // floats of the density box
    constexpr int NRP = (NR + 31) / 32 * 32;         // keeps the offset box 128-byte aligned
    constexpr int PO = BY * OX;                      // 16-bit words of one offset plane
    constexpr uint32_t kBytes = NR * 4u + 24u * PO * 2u;  // both copies
    __shared__ float s_ch[kNF][CY][CX];
    __shared__ float s_rho[CY][CX];
    __shared__ float s_txx[RY][RX], s_txy[RY][RX], s_tyy[RY][RX];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_flags[2];   // fluids present in the tile, by iteration parity
    __shared__ int s_single[2];  // by iteration parity: the tile's 3 x 3 tiles hold one fluid
    extern __shared__ unsigned char dsm[];
    float* rbox = reinterpret_cast<float*>(dsm + ((128u - (smem_u32(dsm) & 127u)) & 127u));  // [3][BY][BX]
    const unsigned short* obox = reinterpret_cast<const unsigned short*>(rbox + NRP);          // [24][BY][OX]

    const int tid = threadIdx.x + TX * threadIdx.y;
    const int lx = threadIdx.x, ly = threadIdx.y;
    const int ntx = (P.nx + TX - 1) / TX;
    const uint32_t bar = smem_u32(&s_bar);
    if ((int)blockIdx.x >= ntiles) return;
    auto issue = [&](int tile) {
        const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
        mbar_arrive_expect_tx(bar, kBytes);
        tma_load_3d(smem_u32(rbox), &tm_rho, x0 - 4, y0 - 3, 0, bar);
        tma_load_3d(smem_u32(obox), &tm_off, x0 - 8, y0 - 3, 0, bar);
    };
    // fluids stored in the 3 x 3 tiles around a tile (a pure tile is inner, so they exist): one
    // fluid means the tile holds it alone after the pull (as in k_step_ring)
    auto single_around = [&](int t) {
        uint64_t nb = 0;
#pragma unroll
        for (int dy = -1; dy <= 1; dy++)
#pragma unroll
            for (int dx = -1; dx <= 1; dx++) nb |= pres_in[t + dy * ntx + dx];
        nb |= nb >> 32;
        nb |= nb >> 16;
        nb |= nb >> 8;
        return __popc((unsigned)(nb & 7u)) == 1 ? 1 : 0;
    };
    int tile = tiles[blockIdx.x];
    int last = 0;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        issue(tile);
        s_flags[0] = s_flags[1] = 0;
        s_single[0] = single_around(tile);
    }
    __syncthreads();

    // pull of the node at (cx, cy) of the phase-field region from the boxes
    auto pull = [&](int cx, int cy, float q[27]) {
        const int own = (cy + 1) * BX + cx + 2, owno = (cy + 1) * OX + cx + 6;
#pragma unroll
        for (int k = 0; k < kNF; k++) {
            const float rk = rbox[k * BY * BX + own];
            float d[kQ];
#pragma unroll
            for (int a = 1; a < kQ; a++) d[a] = dec16<STORE>(obox[(8 * k + a - 1) * PO + owno]);
            q[9 * k] = wq(0) * rk - sum_offsets(d);
#pragma unroll
            for (int a = 1; a < kQ; a++) {
                const int src = k * BY * BX + (cy + 1 - ey(a)) * BX + cx + 2 - ex(a);
                const int srco = (8 * k + a - 1) * PO + (cy + 1 - ey(a)) * OX + cx + 6 - ex(a);
                q[9 * k + a] = wq(a) * rbox[src] + dec16<STORE>(obox[srco]);
            }
        }
    };
    auto store_phase = [&](int cx, int cy, const float q[27]) {
        float r[kNF];
#pragma unroll
        for (int k = 0; k < kNF; k++) {
            const float* qk = q + 9 * k;
            r[k] = ((qk[0] + (qk[1] + qk[3])) + (qk[2] + qk[4])) + ((qk[5] + qk[7]) + (qk[6] + qk[8]));
        }
        const float rho = (r[0] + r[1]) + r[2];
        const float ir = __fdividef(1.0f, rho);
#pragma unroll
        for (int k = 0; k < kNF; k++) s_ch[k][cy][cx] = r[k] * ir;
        s_rho[cy][cx] = rho;
        return (r[0] != 0.0f ? 1 : 0) | (r[1] != 0.0f ? 2 : 0) | (r[2] != 0.0f ? 4 : 0);
    };

    int j = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, j++) {
        const bool more = t + (int)gridDim.x < ntiles;
        const int next = more ? tiles[t + gridDim.x] : 0;
        const int x0 = (tile % ntx) * TX, y0 = (tile / ntx) * TY;
        bool ok = false;
        for (int it = 0; it < P.wait_polls && !ok; it++) ok = mbar_try_wait(bar, j & 1);
        if (__syncthreads_or(!ok)) {
            // the copies did not complete in time: record it, give them a second bounded wait
            // so that they do not land in a later block's shared memory, and stop
            if (tid == 0) {
                atomicOr(P.err, 1);
                for (int it = 0; it < kWaitLimit && !mbar_try_wait(bar, last & 1); it++) {
                }
            }
            return;
        }

        const bool single = s_single[j & 1];
        int single_next = 0;  // thread 0: for the next tile, written once this one is computed
        // ---- phase 1: pulls, densities and phase fields of the halo-2 region ----
        int present = 0;
        if (!single) {
            constexpr int NRING = CX * CY - TX * TY;
            for (int r = tid; r < NRING; r += NT) {
                int cx, cy;
                if (r < 2 * CX) {
                    cx = r % CX;
                    cy = r / CX;
                } else if (r < 4 * CX) {
                    cx = (r - 2 * CX) % CX;
                    cy = CY - 2 + (r - 2 * CX) / CX;
                } else {
                    const int rr0 = r - 4 * CX;  // 4 * TY side nodes
                    const int side = rr0 / (2 * TY), rr = rr0 % (2 * TY);
                    cy = 2 + rr / 2;
                    cx = side == 0 ? (rr & 1) : CX - 2 + (rr & 1);
                }
                float q[27];
                pull(cx, cy, q);
                present |= store_phase(cx, cy, q);
            }
        }
        float f[kQ], r0, r1, r2;
        {
            float q[27];
            pull(lx + 2, ly + 2, q);
            if (!single) present |= store_phase(lx + 2, ly + 2, q);
#pragma unroll
            for (int a = 0; a < kQ; a++) f[a] = (q[a] + q[9 + a]) + q[18 + a];
            r0 = ((q[0] + (q[1] + q[3])) + (q[2] + q[4])) + ((q[5] + q[7]) + (q[6] + q[8]));
            r1 = ((q[9] + (q[10] + q[12])) + (q[11] + q[13])) + ((q[14] + q[16]) + (q[15] + q[17]));
            r2 = ((q[18] + (q[19] + q[21])) + (q[20] + q[22])) + ((q[23] + q[25]) + (q[24] + q[26]));
        }
        // the fluids this warp's nodes hold, for the tiles around this one in the next step
        {
            const int own = (r0 != 0.0f ? 1 : 0) | (r1 != 0.0f ? 2 : 0) | (r2 != 0.0f ? 4 : 0);
            const int w = __reduce_or_sync(0xffffffffu, own);
            if ((tid & 31) == 0) reinterpret_cast<uint8_t*>(pres_out + tile)[tid >> 5] = (uint8_t)w;
        }
        bool mixed = false;
        if (single) {
            __syncthreads();  // every pull is done before the boxes are refilled
            if (tid == 0) s_flags[(j + 1) & 1] = 0;
        } else {
            mixed = fluids_present(present, s_flags, j, tid) != 1;
        }
        // the boxes are free: fetch the next tile's while this one computes
        if (tid == 0 && more) {
            issue(next);
            last = j + 1;
            single_next = single_around(next);
        }

        // ---- phase 2: stress tensor of Eq.(10) on the halo-1 region ----
        if (!single) {
            if (mixed) stress_halo1<TX, TY>(P, s_ch, s_rho, s_txx, s_txy, s_tyy, tid);
            __syncthreads();
        }

        // ---- phase 3: force, collision, recolouring, 16-bit stores ----
        float Fx = 0.0f, Fy = 0.0f, g[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (mixed) {
            div_stress<RX>(s_txx, s_txy, s_tyy, lx + 1, ly + 1, Fx, Fy);
#pragma unroll
            for (int k = 0; k < kNF; k++) grad9_f<CX>(s_ch[k], lx + 2, ly + 2, g[2 * k], g[2 * k + 1]);
        }
        float ux, uy;
        const Recolour rc = collide_node(P, f, r0, r1, r2, Fx, Fy, g, ux, uy);
        const int i = (y0 + ly) * P.nx + x0 + lx;
        if (uout) {
            uout[i] = ux;
            uout[P.N + i] = uy;
        }
        tile = next;
        float v[27];
#pragma unroll
        for (int k = 0; k < kNF; k++)
#pragma unroll
            for (int a = 0; a < kQ; a++)
                v[9 * k + a] = rc.C[k] * f[a] + wq(a) * (rc.Vx[k] * (float)ex(a) + rc.Vy[k] * (float)ey(a));
        store_node<STORE>(fout, P.N, i, v);
        // read by every thread after the next tile's first barrier
        if (tid == 0) s_single[(j + 1) & 1] = single_next;
    }
}

// output path of the TMA kernel: staged in shared memory and written by one bulk tensor store per
// tile, or written directly (a smaller shared-memory footprint leaves room on each SM for blocks
// of the wall-tile kernel, which runs concurrently)
constexpr bool kTmaStage = false;

size_t step_tma_smem_bytes()
{
    const size_t nbox = ((size_t)kQ * kNF * (kTY + 6) * (kTX + 8) + 31) / 32 * 32;
    return (nbox + (kTmaStage ? (size_t)kQ * kNF * kTY * kTX : 0)) * sizeof(float) + 128u;
}

cudaError_t step_tma_prepare()
{
    return cudaFuncSetAttribute(k_step_tma<kTX, kTY, kTmaStage>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)step_tma_smem_bytes());
}

void launch_step_tma(const Params& P, const int* tiles, int ntiles, int nblocks, const Pop& fout, float* u,
                     const CUtensorMap& tin_a, const CUtensorMap& tin_b, const CUtensorMap& tout, cudaStream_t s)
{
    if (ntiles <= 0) return;
    const int nb = nblocks < ntiles ? nblocks : ntiles;
    k_step_tma<kTX, kTY, kTmaStage>
        <<<nb, dim3(kTX, kTY), step_tma_smem_bytes(), s>>>(P, tiles, ntiles, fout.f, u, tin_a, tin_b, tout);
}

size_t step_ring_smem_bytes()
{
    const size_t nbox = ((size_t)kQ * kNF * (kTY + 6) * (kTX + 8) + 31) / 32 * 32;
    return (size_t)kRingBufs * nbox * sizeof(float) + 128u;
}

cudaError_t step_ring_prepare()
{
    return cudaFuncSetAttribute(k_step_ring<kTX, kTY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)step_ring_smem_bytes());
}

void launch_step_ring(const Params& P, const int* tiles, int ntiles, int nblocks, const Pop& fout, float* u,
                      const CUtensorMap& tin, const uint64_t* pres_in, uint64_t* pres_out, cudaStream_t s)
{
    if (ntiles <= 0) return;
    const int nb = nblocks < ntiles ? nblocks : ntiles;
    k_step_ring<kTX, kTY><<<nb, 2 * kTX * kTY + 32, step_ring_smem_bytes(), s>>>(P, tiles, ntiles, fout.f, u, tin,
                                                                                 pres_in, pres_out);
}

size_t step_tma16_smem_bytes()
{
    const size_t nr = ((size_t)kNF * (kTY + 6) * (kTX + 8) + 31) / 32 * 32;
    return nr * sizeof(float) + (size_t)24 * (kTY + 6) * (kTX + 16) * sizeof(unsigned short) + 128u;
}

// the 16-bit offset box takes the block past the 48 KB of shared memory a kernel gets without
// opting in
cudaError_t step_tma16_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(k_step_tma16<kTX, kTY, kStoreF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_tma16_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step_tma16<kTX, kTY, kStoreBF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)step_tma16_smem_bytes());
    return e;
}

void launch_step_tma16(int store, const Params& P, const int* tiles, int ntiles, int nblocks, const Pop& fout,
                       float* u, const CUtensorMap& trho, const CUtensorMap& toff, const uint64_t* pres_in,
                       uint64_t* pres_out, cudaStream_t s)
{
    if (ntiles <= 0) return;
    const int nb = nblocks < ntiles ? nblocks : ntiles;
    if (store == kStoreF16)
        k_step_tma16<kTX, kTY, kStoreF16><<<nb, dim3(kTX, kTY), step_tma16_smem_bytes(), s>>>(
            P, tiles, ntiles, fout, u, trho, toff, pres_in, pres_out);
    else
        k_step_tma16<kTX, kTY, kStoreBF16><<<nb, dim3(kTX, kTY), step_tma16_smem_bytes(), s>>>(
            P, tiles, ntiles, fout, u, trho, toff, pres_in, pres_out);
}

void launch_init(int store, const Params& P, const double* rho, const uint8_t* type, const Pop& f,
                 cudaStream_t s)
{
    const unsigned nb = (unsigned)((P.N + 255) / 256);
    if (store == kStoreF32)
        k_init<kStoreF32><<<nb, 256, 0, s>>>(P, rho, type, f);
    else if (store == kStoreF16)
        k_init<kStoreF16><<<nb, 256, 0, s>>>(P, rho, type, f);
    else
        k_init<kStoreBF16><<<nb, 256, 0, s>>>(P, rho, type, f);
}

void launch_fields(int store, const Params& P, const Pop& f, const uint8_t* type, float* rho_out,
                   cudaStream_t s)
{
    with_store(store, f, P.N, [&](auto st) {
        k_fields<<<(unsigned)((P.N + 255) / 256), 256, 0, s>>>(P, st, type, rho_out);
    });
}

void launch_get_state(int store, const Params& P, const Pop& f, const uint8_t* type, float* post,
                      cudaStream_t s)
{
    with_store(store, f, P.N, [&](auto st) {
        k_get_state<<<(unsigned)((P.N + 255) / 256), 256, 0, s>>>(P, st, type, post);
    });
}

void launch_set_state(int store, const Params& P, const double* post, const uint8_t* type,
                      const Pop& f, cudaStream_t s)
{
    const unsigned nb = (unsigned)((P.N + 255) / 256);
    if (store == kStoreF32)
        k_set_state<kStoreF32><<<nb, 256, 0, s>>>(P, post, type, f);
    else if (store == kStoreF16)
        k_set_state<kStoreF16><<<nb, 256, 0, s>>>(P, post, type, f);
    else
        k_set_state<kStoreBF16><<<nb, 256, 0, s>>>(P, post, type, f);
}

int diag_blocks(const Params& P)
{
    long long b = (P.N + kDiagThreads - 1) / kDiagThreads;
    return (int)(b < 1216 ? b : 1216);
}

void launch_diag(int store, const Params& P, const Pop& f, const uint8_t* type, const float* u,
                 double* partials, double* out, cudaStream_t s)
{
    const int nb = diag_blocks(P);
    with_store(store, f, P.N, [&](auto st) {
        k_diag<<<nb, kDiagThreads, 0, s>>>(P, st, type, u, partials);
    });
    k_diag_final<<<1, 32, 0, s>>>(nb, partials, out);
}

}  // namespace lbm3k
