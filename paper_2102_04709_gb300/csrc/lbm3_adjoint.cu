// lbm3_adjoint.cu -- reverse-mode (adjoint) kernels of one timestep of the three-phase MRT
// colour-gradient step with characteristic-line wetting (arXiv:2102.04709, Section II), for the
// gradient of an objective of the final state with respect to the wall-angle triples of
// Eq.(17)/(21) and the Zou-He inflow velocity.
//
// The forward state of each step (stored populations + lagged wall values) comes from the
// production kernels.  The adjoint first recomputes the intermediates of that step, unfused, into
// global arrays (post-streaming populations, phase fields, wall values with the decisions of the
// characteristic lines, gradients, stress, force), then applies the vector-Jacobian products in
// reverse order:  collision + recolouring (Eq.1-15), divergence (Eq.10, 12), stress (Eq.10),
// gradients (Eq.12), wetting (Eq.21, 22, characteristic lines), fractions, pull-streaming with
// halfway bounce-back and Zou-He (Eq.16).  All in FP32, gradient accumulators in FP64.
// Supported: periodic, wall and Zou-He x boundaries (not the modified periodic seam).
//
// Padded arrays carry one ghost column on each side of the grid (index y * (nx + 2) + x + 1),
// used for the zero-gradient copies beyond the open Zou-He columns.
#include <cmath>
#include <utility>

#include "lbm3_common.cuh"
#include "lbm3_device.cuh"

namespace lbm3k {

namespace {

// the last march of a wetting lane: the same angle gives the same line, crossing and derivative
struct AdjLine {
    double th, fr, dfr;
    int kind, ax, ay, bx, by, pad;
};

struct Adj {
    int nxp;  // nx + 2
    // forward intermediates
    float* fpost;  // [27][N]
    float* C;      // [3][NP]
    float* rho;    // [NP]
    float* g;      // [6][NP]   (dC0/dx, dC0/dy, dC1/dx, ...)
    float* T;      // [3][NP]
    float* F;      // [2][N]
    AdjLine* wline;  // [4 Nw] by lane 4 w + 2 k + side
    // wetting decisions, lane = 2 k + side
    int* wkind;    // [4][Nw]
    int* wa;       // [4][Nw] in-domain node index of the first bracketing node
    int* wb;       // [4][Nw]
    float* wfr;    // [4][Nw]
    float* wdfr;   // [4][Nw] d fr / d theta_k (deg)
    float* wraw;   // [2][Nw] C_P of fluid k before the normalisation
    int* wsel;     // [2][Nw] side chosen by Eq.(22)
    // adjoint fields
    float* l_fpost;  // [27][N]
    float* l_F;      // [2][N]
    float* l_g;      // [6][NP]  (written at fluid positions only; zero elsewhere)
    float* l_C;      // [3][NP]
    float* l_rho;    // [NP]
    float* l_fs;     // [27][N] adjoint of the stored populations
    float* l_cw;     // [3][N]  adjoint of the lagged wall values (input, from the next step)
    float* l_cw2;    // [3][N]  adjoint of the lagged wall values (output, for the previous step)
    double* l_th;    // [2][Nw] adjoint of the local angle theta_k of Eq.(21)
    double* d_ang;   // [3][Nw] dJ/d(theta_01, theta_20, theta_12)
    double* d_u;     // [1] dJ/dU
};

__device__ __forceinline__ int pad(const Adj& A, int x, int y) { return y * A.nxp + x + 1; }

// The lattice position (X, Y), unwrapped, brought into the domain in place, as locate() does but
// without dividing its index back into coordinates: 0 inside, 1 solid beyond a wall side (X, Y
// then meaningless), 2 beyond an open x side (X clamped to the boundary column).  (The adjoint
// has no modified-periodic seam.)
__device__ __forceinline__ int wrap_xy(const Params& P, int& X, int& Y)
{
    if (Y < 0 || Y >= P.ny) {
        if (!P.per_y) return 1;
        Y -= floordiv_i(Y, P.ny) * P.ny;
    }
    if (X < 0 || X >= P.nx) {
        if (P.bc_x == kWalls) return 1;
        if (P.bc_x == kZouHe) {
            X = X < 0 ? 0 : P.nx - 1;
            return 2;
        }
        X -= floordiv_i(X, P.nx) * P.nx;
    }
    return 0;
}

// position of C / rho seen from an unwrapped lattice position: kind 0 = an in-domain node
// (padded index), 1 = solid beyond a wall side; beyond an open side: the boundary-column node
__device__ __forceinline__ int cpos(const Params& P, const Adj& A, int X, int Y, int& kind)
{
    kind = wrap_xy(P, X, Y) == 1;
    return kind ? 0 : pad(A, X, Y);
}

// position of T seen from an unwrapped lattice position: the ghost columns are their own slots
__device__ __forceinline__ int tpos(const Params& P, const Adj& A, int X, int Y)
{
    if (P.bc_x == kZouHe && (X == -1 || X == P.nx)) {
        int x0 = 0;
        if (wrap_xy(P, x0, Y) == 1) Y = 0;
        return pad(A, X, Y);
    }
    if (wrap_xy(P, X, Y) == 1) return pad(A, 0, 0);
    return pad(A, X, Y);
}

// ------------------------------------------------------------------------------------------
// forward intermediates
// ------------------------------------------------------------------------------------------
// A1: post-streaming populations, densities and fractions (fluid nodes and ghost columns); also
// clears the step's adjoint accumulators lambda_C, lambda_rho at every padded position
__global__ void a_dens(const Params P, const Adj A, const float* __restrict__ fs,
                       const uint8_t* __restrict__ type)
{
    const int gx = blockIdx.x * blockDim.x + threadIdx.x - 1, y = blockIdx.y;
    if (gx > P.nx || y >= P.ny) return;
    const int p = pad(A, gx, y);
    {
        const int NP = P.ny * A.nxp;
        for (int k = 0; k < kNF; k++) A.l_C[k * NP + p] = 0.0f;
        A.l_rho[p] = 0.0f;
    }
    const bool ghost = gx < 0 || gx >= P.nx;
    if (ghost && P.bc_x != kZouHe) return;
    const int x = gx < 0 ? 0 : (gx >= P.nx ? P.nx - 1 : gx);
    const int i = y * P.nx + x;
    const uint8_t t = type[i];
    if (t & 2) {
        A.rho[p] = (t & 3) == kSB ? 1.0f : 0.0f;
        if ((t & 3) == kSI)
            for (int k = 0; k < kNF; k++) A.C[k * (P.ny * A.nxp) + p] = 0.0f;
        return;
    }
    float q[27];
    const Store<kStoreF32> st(fs, P.N);
    pull_global(P, st, type, x, y, q);
    float r[kNF];
    for (int k = 0; k < kNF; k++) {
        float s = 0.f;
        for (int a = 0; a < kQ; a++) s += q[9 * k + a];
        r[k] = s;
    }
    const float rho = r[0] + r[1] + r[2];
    for (int k = 0; k < kNF; k++) A.C[k * (P.ny * A.nxp) + p] = r[k] / rho;
    A.rho[p] = rho;
    if (!ghost)
        for (int j = 0; j < 27; j++) A.fpost[(long long)j * P.N + i] = q[j];
}

// A2: wetting with its decisions, 4 lanes per C_SB node (the same computation as k_wet)
__global__ void a_wet(const Params P, const Adj A, int nw, const int* __restrict__ widx,
                      const double* __restrict__ wnrm, const float* __restrict__ wang,
                      const float* __restrict__ fs, const uint8_t* __restrict__ type,
                      const double* __restrict__ cw_lag)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int w = g >> 2, lane = g & 3;
    const int k = lane >> 1, side = lane & 1;
    const bool valid = w < nw;
    const Store<kStoreF32> st(fs, P.N);
    int i = 0, px = 0, py = 0;
    double th = 90.0, dfr = 0.0;
    Crossing cr{0, 0, 0, 0, 0, 0.0};
    if (valid) {
        i = widx[w];
        px = i % P.nx;
        py = i / P.nx;
        const double Cr = cw_lag[i], Cg = cw_lag[P.N + i], Cb = cw_lag[2 * P.N + i];
        const double t_rg = wang[3 * w], t_br = wang[3 * w + 1], t_gb = wang[3 * w + 2];
        th = k == 0 ? local_angle(Cb, 180.0 - t_br, Cg, t_rg) : local_angle(Cb, t_gb, Cr, 180.0 - t_rg);
        const AdjLine c = A.wline[g];
        if (c.th == th) {
            cr = Crossing{c.kind, c.ax, c.ay, c.bx, c.by, c.fr};
            dfr = c.dfr;
        } else {
            const double nx_ = wnrm[2 * w], ny_ = wnrm[2 * w + 1];
            const double dev = fabs(90.0 - th);
            const double phi = dev < kPhiSnap ? 0.0 : dev * (M_PI / 180.0);
            const double sg = side ? -1.0 : 1.0;
            double sn, cs;
            sincos(phi, &sn, &cs);
            const double dx = cs * nx_ - sg * sn * ny_, dy = cs * ny_ + sg * sn * nx_;
            cr = characteristic_line<Store<kStoreF32>>(P, type, px, py, dx, dy);
            if (cr.kind == 2 && dev >= kPhiSnap) {
                // d(position along the crossed line)/d phi, then d phi / d theta_k
                const double ddx = -sn * nx_ - sg * cs * ny_, ddy = -sn * ny_ + sg * cs * nx_;
                double ds;
                if (cr.ax == cr.bx)
                    ds = (double)(cr.ax - px) * (ddy * dx - dy * ddx) / (dx * dx);
                else
                    ds = (double)(cr.ay - py) * (ddx * dy - dx * ddy) / (dy * dy);
                dfr = ds * (90.0 - th > 0 ? -1.0 : 1.0) * (M_PI / 180.0);
            }
            A.wline[g] = AdjLine{th, cr.fr, dfr, cr.kind, cr.ax, cr.ay, cr.bx, cr.by, 0};
        }
    }
    double ca = 0.0, cb = 0.0;
    if (valid && cr.kind >= 1) ca = node_C(P, st, type, cr.ax, cr.ay, k);
    if (valid && cr.kind == 2) cb = node_C(P, st, type, cr.bx, cr.by, k);
    if (valid && cr.kind == 0) ca = neighbour_mean(P, st, type, px, py, k);
    const double cd = cr.kind == 2 ? ca + cr.fr * (cb - ca) : ca;
    const double other = __shfl_xor_sync(0xffffffffu, cd, 1);
    const bool takes_max = th <= 90.0;
    const double cp = takes_max ? fmax(cd, other) : fmin(cd, other);
    // the chosen side (ties: side 0)
    const int sel = (takes_max ? (cd > other || (cd == other && side == 0)) : (cd < other || (cd == other && side == 0))) ? side : 1 - side;
    const double cg = __shfl_xor_sync(0xffffffffu, cp, 2);
    if (valid) {
        const int j = lane * nw + w;
        A.wkind[j] = cr.kind;
        int kk;
        A.wa[j] = cr.kind >= 1 ? cpos(P, A, cr.ax, cr.ay, kk) : 0;
        A.wb[j] = cr.kind == 2 ? cpos(P, A, cr.bx, cr.by, kk) : 0;
        A.wfr[j] = (float)cr.fr;
        A.wdfr[j] = (float)dfr;
        if (side == 0) {
            A.wraw[k * nw + w] = (float)cp;
            A.wsel[k * nw + w] = sel;
        }
        if (lane == 0) {
            double c0 = fmin(fmax(cp, 0.0), 1.0), c1 = fmin(fmax(cg, 0.0), 1.0);
            const double s = c0 + c1;
            if (s > 1.0) {
                c0 /= s;
                c1 /= s;
            }
            const int p = pad(A, px, py);
            const int NP = P.ny * A.nxp;
            A.C[p] = (float)c0;
            A.C[NP + p] = (float)c1;
            A.C[2 * NP + p] = (float)fmax(0.0, 1.0 - c0 - c1);
        }
    }
}

__device__ __forceinline__ bool is_active(const Params& P, const Adj& A, const uint8_t* type, int gx,
                                          int y, int& cls)
{
    // fluid or C_SB node in the domain, or a ghost column of an open side
    if (gx < 0 || gx >= P.nx) {
        cls = kFI;
        return P.bc_x == kZouHe;
    }
    cls = type[y * P.nx + gx] & 3;
    return cls != kSI;
}

// The 9-point stencil of C around the position (gx, gy) (in-domain or ghost), the same for every
// fluid: value a is m[a] C[src[a]] - C[src2[a]], the second term only where src2[a] >= 0.  At a
// C_SB centre a neighbour without a value of its own (C_SI, or solid beyond a wall side) is the
// extrapolation 2 C(centre) - C(opposite neighbour), or C(centre) when the opposite neighbour
// has no value either.
__device__ __forceinline__ void stencil_geom(const Params& P, const Adj& A, const uint8_t* type, int gx,
                                             int gy, int cls, int src[kQ], int src2[kQ], float m[kQ])
{
    int kind;
    const int pc = cpos(P, A, gx, gy, kind);
    // kd == 1: solid beyond a wall side; otherwise the class of the node (or of the boundary
    // column node a ghost copies)
    auto no_value = [&](int kd, int X, int Y) { return kd == 1 || (type[Y * P.nx + X] & 3) == kSI; };
    for (int a = 0; a < kQ; a++) {
        int X = gx + ex(a), Y = gy + ey(a);
        const int kd = wrap_xy(P, X, Y);
        int q = kd == 1 ? 0 : pad(A, X, Y);
        int q2 = -1;
        float mm = 1.0f;
        if (cls == kSB && a > 0 && no_value(kd, X, Y)) {
            int Xo = gx - ex(a), Yo = gy - ey(a);
            const int kd2 = wrap_xy(P, Xo, Yo);
            q = pc;
            if (!no_value(kd2, Xo, Yo)) {
                q2 = pad(A, Xo, Yo);
                mm = 2.0f;
            }
        }
        src[a] = q;
        src2[a] = q2;
        m[a] = mm;
    }
}

// values of the stencil for fluid k
__device__ __forceinline__ void stencil_C(const Params& P, const Adj& A, int k, const int src[kQ],
                                          const int src2[kQ], const float m[kQ], float v[kQ])
{
    const float* C = A.C + k * (P.ny * A.nxp);
    for (int a = 0; a < kQ; a++) v[a] = src2[a] < 0 ? C[src[a]] : m[a] * C[src[a]] - C[src2[a]];
}

// A3: gradients (Eq.12) and the Eq.(10) stress at fluid, C_SB and ghost positions
__global__ void a_grad_stress(const Params P, const Adj A, const uint8_t* __restrict__ type,
                              const float sig01, const float sig02, const float sig12)
{
    const int gx = blockIdx.x * blockDim.x + threadIdx.x - 1, y = blockIdx.y;
    if (gx > P.nx || y >= P.ny) return;
    int cls;
    if (!is_active(P, A, type, gx, y, cls)) return;
    const int NP = P.ny * A.nxp;
    const int p = pad(A, gx, y);
    float c[kNF], gxk[kNF], gyk[kNF], m[kQ];
    int src[kQ], src2[kQ];
    stencil_geom(P, A, type, gx, y, cls, src, src2, m);
    for (int k = 0; k < kNF; k++) {
        float v[kQ];
        stencil_C(P, A, k, src, src2, m, v);
        c[k] = v[0];
        gxk[k] = (1.0f / 3.0f) * (v[1] - v[3]) + (1.0f / 12.0f) * ((v[5] - v[7]) + (v[8] - v[6]));
        gyk[k] = (1.0f / 3.0f) * (v[2] - v[4]) + (1.0f / 12.0f) * ((v[5] - v[7]) + (v[6] - v[8]));
        A.g[(2 * k) * NP + p] = gxk[k];
        A.g[(2 * k + 1) * NP + p] = gyk[k];
    }
    const float rho = A.rho[p];
    float Txx = 0.f, Txy = 0.f, Tyy = 0.f;
    const float rho2 = rho * rho;
    pair_stress(sig01, c[0], c[1], gxk[0], gyk[0], gxk[1], gyk[1], rho2, Txx, Txy, Tyy);
    pair_stress(sig02, c[0], c[2], gxk[0], gyk[0], gxk[2], gyk[2], rho2, Txx, Txy, Tyy);
    pair_stress(sig12, c[1], c[2], gxk[1], gyk[1], gxk[2], gyk[2], rho2, Txx, Txy, Tyy);
    A.T[p] = Txx;
    A.T[NP + p] = Txy;
    A.T[2 * NP + p] = Tyy;
}

// A4: force F = div T (Eq.10) at the fluid nodes, from the stress of their neighbours
__global__ void a_force(const Params P, const Adj A, const uint8_t* __restrict__ type)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const int i = y * P.nx + x;
    if (type[i] & 2) return;
    const int NP = P.ny * A.nxp;
    float Fx = 0.f, Fy = 0.f;
    for (int a = 1; a < kQ; a++) {
        const int q = tpos(P, A, x + ex(a), y + ey(a));
        const float c = 3.0f * wq(a);
        Fx += c * (A.T[q] * ex(a) + A.T[NP + q] * ey(a));
        Fy += c * (A.T[NP + q] * ex(a) + A.T[2 * NP + q] * ey(a));
    }
    A.F[i] = Fx;
    A.F[P.N + i] = Fy;
}

// ------------------------------------------------------------------------------------------
// reverse
// ------------------------------------------------------------------------------------------
// B1: VJP of the MRT collision with forcing and the recolouring at a fluid node
__global__ void b_collide(const Params P, const Adj A, const uint8_t* __restrict__ type)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const int i = y * P.nx + x;
    if (type[i] & 2) return;
    const int NP = P.ny * A.nxp;
    const int p = pad(A, x, y);
    // ---- forward recompute ----
    float q[27], f[kQ], r[kNF];
    for (int j = 0; j < 27; j++) q[j] = A.fpost[(long long)j * P.N + i];
    for (int k = 0; k < kNF; k++) {
        float s = 0.f;
        for (int a = 0; a < kQ; a++) s += q[9 * k + a];
        r[k] = s;
    }
    for (int a = 0; a < kQ; a++) f[a] = q[a] + q[9 + a] + q[18 + a];
    const float rho = r[0] + r[1] + r[2];
    const float irho = 1.f / rho;  // one division; every other quotient by rho is a product
    const float Fx = A.F[i], Fy = A.F[P.N + i];
    float g[6];
    for (int j = 0; j < 6; j++) g[j] = A.g[j * NP + p];
    float C[kNF];
    for (int k = 0; k < kNF; k++) C[k] = r[k] * irho;
    // moments
    const float e = -4.f * f[0] - (f[1] + f[2] + f[3] + f[4]) + 2.f * (f[5] + f[6] + f[7] + f[8]);
    const float eps = 4.f * f[0] - 2.f * (f[1] + f[2] + f[3] + f[4]) + (f[5] + f[6] + f[7] + f[8]);
    const float jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    const float qx = -2.f * (f[1] - f[3]) + f[5] - f[6] - f[7] + f[8];
    const float jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    const float qy = -2.f * (f[2] - f[4]) + f[5] + f[6] - f[7] - f[8];
    const float pxx = f[1] - f[2] + f[3] - f[4];
    const float pxy = f[5] - f[6] + f[7] - f[8];
    const float ux = (jx + 0.5f * Fx) * irho, uy = (jy + 0.5f * Fy) * irho;
    const float u2 = ux * ux + uy * uy, uF = ux * Fx + uy * Fy;
    const float D = r[0] * P.inv_nu0 + r[1] * P.inv_nu1 + r[2] * P.inv_nu2;
    const float s1 = D / (0.5f * D + 3.0f);
    const float s4 = 8.0f * (2.0f - s1) / (8.0f - s1);
    const float h1 = 1.0f - 0.5f * s1, h4 = 1.0f - 0.5f * s4;
    const float XE = e + 2.f * rho - 3.f * rho * u2, XEps = eps - rho + 3.f * rho * u2;
    const float Xqx = qx + rho * ux, Xqy = qy + rho * uy;
    const float Xpxx = pxx - rho * (ux * ux - uy * uy), Xpxy = pxy - rho * ux * uy;
    const float dE = -s1 * XE + h1 * 6.f * uF, dEps = -s1 * XEps - h1 * 6.f * uF;
    const float dqx = -s4 * Xqx - h4 * Fx, dqy = -s4 * Xqy - h4 * Fy;
    const float dpxx = -s1 * Xpxx + h1 * 2.f * (ux * Fx - uy * Fy);
    const float dpxy = -s1 * Xpxy + h1 * (ux * Fy + uy * Fx);
    // f_dag = f + M^-1 dm
    float fd[kQ];
    {
        const float c0 = (dEps - dE) * (1.f / 9.f);
        const float ca = -dE * (1.f / 36.f) - dEps * (1.f / 18.f), cd = dE * (1.f / 18.f) + dEps * (1.f / 36.f);
        const float X1 = (Fx - dqx) * (1.f / 6.f), Y1 = (Fy - dqy) * (1.f / 6.f);
        const float X2 = Fx * (1.f / 6.f) + dqx * (1.f / 12.f), Y2 = Fy * (1.f / 6.f) + dqy * (1.f / 12.f);
        const float P4 = 0.25f * dpxx, Q4 = 0.25f * dpxy;
        fd[0] = f[0] + c0;
        fd[1] = f[1] + ca + X1 + P4;
        fd[2] = f[2] + ca + Y1 - P4;
        fd[3] = f[3] + ca - X1 + P4;
        fd[4] = f[4] + ca - Y1 - P4;
        fd[5] = f[5] + cd + X2 + Y2 + Q4;
        fd[6] = f[6] + cd - X2 + Y2 - Q4;
        fd[7] = f[7] + cd - X2 - Y2 + Q4;
        fd[8] = f[8] + cd + X2 - Y2 - Q4;
    }
    // normals
    const float gg[3][2] = {{g[0], g[1]}, {g[2], g[3]}, {g[4], g[5]}};
    const int pk[3] = {0, 0, 1}, pl[3] = {1, 2, 2};
    float nxp_[3], nyp_[3], Gx[3], Gy[3], rGn[3];
    bool act[3];
    for (int m = 0; m < 3; m++) {
        const int k = pk[m], l = pl[m];
        Gx[m] = C[l] * gg[k][0] - C[k] * gg[l][0];
        Gy[m] = C[l] * gg[k][1] - C[k] * gg[l][1];
        const float G2 = Gx[m] * Gx[m] + Gy[m] * Gy[m];
        act[m] = G2 > 1e-24f;
        rGn[m] = act[m] ? rsqrtf(G2) : 1.f;  // 1 / |G|
        nxp_[m] = act[m] ? Gx[m] * rGn[m] : 0.f;
        nyp_[m] = act[m] ? Gy[m] * rGn[m] : 0.f;
    }
    const float gX[3] = {P.g01, P.g02, P.g12};
    const float irho3 = irho * irho * irho;
    const float T3 = 35.f * r[0] * r[1] * r[2] * irho3;
    const float trip = fminf(T3, 1.0f);
    float b[3];
    for (int m = 0; m < 3; m++) b[m] = P.beta0 * (1.f + trip * gX[m]) * r[pk[m]] * r[pl[m]] * irho;

    // ---- reverse ----
    float lo[27];
    for (int j = 0; j < 27; j++) lo[j] = A.l_fs[(long long)j * P.N + i];
    float lC[kNF] = {0, 0, 0}, lfd[kQ] = {0}, lV[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    for (int k = 0; k < kNF; k++)
        for (int a = 0; a < kQ; a++) {
            const float l = lo[9 * k + a];
            lC[k] += l * fd[a];
            lfd[a] += l * C[k];
            lV[k][0] += l * wq(a) * ex(a);
            lV[k][1] += l * wq(a) * ey(a);
        }
    // V0 = b01 n01 + b02 n02, V1 = -b01 n01 + b12 n12, V2 = -b02 n02 - b12 n12
    const float dV[3][2] = {{lV[0][0] - lV[1][0], lV[0][1] - lV[1][1]},
                            {lV[0][0] - lV[2][0], lV[0][1] - lV[2][1]},
                            {lV[1][0] - lV[2][0], lV[1][1] - lV[2][1]}};
    float lb[3], lg[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    for (int m = 0; m < 3; m++) {
        lb[m] = dV[m][0] * nxp_[m] + dV[m][1] * nyp_[m];
        if (!act[m]) continue;
        const float lnx = b[m] * dV[m][0], lny = b[m] * dV[m][1];
        const float dot = nxp_[m] * lnx + nyp_[m] * lny;
        const float lGx = (lnx - nxp_[m] * dot) * rGn[m], lGy = (lny - nyp_[m] * dot) * rGn[m];
        const int k = pk[m], l = pl[m];
        lg[k][0] += C[l] * lGx;
        lg[k][1] += C[l] * lGy;
        lg[l][0] -= C[k] * lGx;
        lg[l][1] -= C[k] * lGy;
        lC[l] += gg[k][0] * lGx + gg[k][1] * lGy;
        lC[k] -= gg[l][0] * lGx + gg[l][1] * lGy;
    }
    // b_m = beta0 (1 + trip g_m) r_k r_l / rho
    float lr[kNF] = {0, 0, 0}, lrho = 0.f, ltrip = 0.f;
    for (int m = 0; m < 3; m++) {
        const int k = pk[m], l = pl[m];
        const float base = P.beta0 * (1.f + trip * gX[m]);
        ltrip += lb[m] * P.beta0 * gX[m] * r[k] * r[l] * irho;
        lr[k] += lb[m] * base * r[l] * irho;
        lr[l] += lb[m] * base * r[k] * irho;
        lrho -= lb[m] * b[m] * irho;
    }
    if (T3 < 1.0f) {
        lr[0] += ltrip * 35.f * r[1] * r[2] * irho3;
        lr[1] += ltrip * 35.f * r[0] * r[2] * irho3;
        lr[2] += ltrip * 35.f * r[0] * r[1] * irho3;
        lrho -= ltrip * 3.f * T3 * irho;
    }
    // collision: f_dag = f + M^-1 dm
    float lf[kQ];
    for (int a = 0; a < kQ; a++) lf[a] = lfd[a];
    // lambda of the moment changes = (M^-1)^T lfd
    const float ldE = (-lfd[0] * (1.f / 9.f)) + (-(lfd[1] + lfd[2] + lfd[3] + lfd[4]) * (1.f / 36.f)) +
                      ((lfd[5] + lfd[6] + lfd[7] + lfd[8]) * (1.f / 18.f));
    const float ldEps = (lfd[0] * (1.f / 9.f)) + (-(lfd[1] + lfd[2] + lfd[3] + lfd[4]) * (1.f / 18.f)) +
                        ((lfd[5] + lfd[6] + lfd[7] + lfd[8]) * (1.f / 36.f));
    const float lX1 = (lfd[1] - lfd[3]) * (1.f / 6.f), lY1 = (lfd[2] - lfd[4]) * (1.f / 6.f);
    const float lX2 = (lfd[5] - lfd[6] - lfd[7] + lfd[8]), lY2 = (lfd[5] + lfd[6] - lfd[7] - lfd[8]);
    // X1 = (Fx - dqx)/6, X2 = Fx/6 + dqx/12
    const float ldqx = -lX1 + lX2 * (1.f / 12.f), ldqy = -lY1 + lY2 * (1.f / 12.f);
    float lFx = lX1 + lX2 * (1.f / 6.f), lFy = lY1 + lY2 * (1.f / 6.f);
    const float ldpxx = 0.25f * (lfd[1] - lfd[2] + lfd[3] - lfd[4]);
    const float ldpxy = 0.25f * (lfd[5] - lfd[6] + lfd[7] - lfd[8]);
    // moment changes -> moments, rho, u, F, s1, s4
    const float le = -s1 * ldE, leps = -s1 * ldEps, lqx = -s4 * ldqx, lqy = -s4 * ldqy;
    const float lpxx = -s1 * ldpxx, lpxy = -s1 * ldpxy;
    lrho += -s1 * (2.f - 3.f * u2) * ldE - s1 * (-1.f + 3.f * u2) * ldEps - s4 * ux * ldqx - s4 * uy * ldqy +
            s1 * (ux * ux - uy * uy) * ldpxx + s1 * ux * uy * ldpxy;
    float lux = (6.f * s1 * rho * ux + 6.f * h1 * Fx) * ldE + (-6.f * s1 * rho * ux - 6.f * h1 * Fx) * ldEps -
                s4 * rho * ldqx + (2.f * s1 * rho * ux + 2.f * h1 * Fx) * ldpxx + (s1 * rho * uy + h1 * Fy) * ldpxy;
    float luy = (6.f * s1 * rho * uy + 6.f * h1 * Fy) * ldE + (-6.f * s1 * rho * uy - 6.f * h1 * Fy) * ldEps -
                s4 * rho * ldqy + (-2.f * s1 * rho * uy - 2.f * h1 * Fy) * ldpxx + (s1 * rho * ux + h1 * Fx) * ldpxy;
    lFx += 6.f * h1 * ux * ldE - 6.f * h1 * ux * ldEps - h4 * ldqx + 2.f * h1 * ux * ldpxx + h1 * uy * ldpxy;
    lFy += 6.f * h1 * uy * ldE - 6.f * h1 * uy * ldEps - h4 * ldqy - 2.f * h1 * uy * ldpxx + h1 * ux * ldpxy;
    float ls1 = (-XE - 3.f * uF) * ldE + (-XEps + 3.f * uF) * ldEps + (-Xpxx - (ux * Fx - uy * Fy)) * ldpxx +
                (-Xpxy - 0.5f * (ux * Fy + uy * Fx)) * ldpxy;
    const float ls4 = (-Xqx + 0.5f * Fx) * ldqx + (-Xqy + 0.5f * Fy) * ldqy;
    ls1 += ls4 * (-48.f / ((8.f - s1) * (8.f - s1)));
    const float lD = ls1 * 3.f / ((0.5f * D + 3.f) * (0.5f * D + 3.f));
    lr[0] += lD * P.inv_nu0;
    lr[1] += lD * P.inv_nu1;
    lr[2] += lD * P.inv_nu2;
    // u = (j + F/2)/rho
    const float ljx = lux * irho, ljy = luy * irho;
    lFx += 0.5f * lux * irho;
    lFy += 0.5f * luy * irho;
    lrho -= (lux * ux + luy * uy) * irho;
    // moments -> populations (rows of M)
    for (int a = 0; a < kQ; a++) {
        const int e2 = ex(a) * ex(a) + ey(a) * ey(a);
        const float me = (float)(-4 + 3 * e2);
        const float meps = e2 == 0 ? 4.f : (e2 == 1 ? -2.f : 1.f);
        const float mqx = (float)(ex(a) * (3 * e2 - 5)), mqy = (float)(ey(a) * (3 * e2 - 5));
        const float mpxx = (float)(ex(a) * ex(a) - ey(a) * ey(a)), mpxy = (float)(ex(a) * ey(a));
        lf[a] += le * me + leps * meps + ljx * ex(a) + lqx * mqx + ljy * ey(a) + lqy * mqy + lpxx * mpxx +
                 lpxy * mpxy + lrho;
    }
    // C_k = r_k / rho
    float sc = 0.f;
    for (int k = 0; k < kNF; k++) sc += lC[k] * C[k];
    for (int k = 0; k < kNF; k++) lr[k] += (lC[k] - sc) * irho;
    for (int k = 0; k < kNF; k++)
        for (int a = 0; a < kQ; a++) A.l_fpost[(long long)(9 * k + a) * P.N + i] = lf[a] + lr[k];
    A.l_F[i] = lFx;
    A.l_F[P.N + i] = lFy;
    for (int k = 0; k < kNF; k++) {
        A.l_g[(2 * k) * NP + p] = lg[k][0];
        A.l_g[(2 * k + 1) * NP + p] = lg[k][1];
    }
}

// adjoint of the divergence: lambda_T at the fluid / C_SB / ghost position (gx, y) with padded
// index p, gathered from the fluid nodes whose force read T there
__device__ __forceinline__ void div_adjoint(const Params& P, const Adj& A, const uint8_t* type, int gx,
                                            int y, int p, float lT[3])
{
    float lxx = 0.f, lxy = 0.f, lyy = 0.f;
    for (int a = 1; a < kQ; a++) {
        // the fluid node q = p - e_a looked up T at p in direction a
        int qx = gx - ex(a), qy = y - ey(a);
        if (wrap_xy(P, qx, qy) != 0) continue;
        const int qi = qy * P.nx + qx;
        if (type[qi] & 2) continue;
        if (tpos(P, A, qx + ex(a), qy + ey(a)) != p) continue;
        const float c = 3.0f * wq(a);
        const float lFx = A.l_F[qi], lFy = A.l_F[P.N + qi];
        lxx += c * ex(a) * lFx;
        lxy += c * (ey(a) * lFx + ex(a) * lFy);
        lyy += c * ey(a) * lFy;
    }
    lT[0] = lxx;
    lT[1] = lxy;
    lT[2] = lyy;
}

// VJP of one pair's stress sigma A (|G|^2 I - G G)/|G|
__device__ __forceinline__ void pair_stress_vjp(float sig, float ck, float cl, float gkx, float gky,
                                                float glx, float gly, float rho, const float lT[3],
                                                float& lck, float& lcl, float lgk[2], float lgl[2],
                                                float& lrho)
{
    const float Gx = cl * gkx - ck * glx, Gy = cl * gky - ck * gly;
    const float G2 = Gx * Gx + Gy * Gy;
    if (!(G2 > 1e-24f)) return;
    const float Gn = sqrtf(G2), iG = 1.0f / Gn, iG3 = iG * iG * iG;
    const float Ar = 1e6f * ck * cl * rho * rho;
    const float A = fminf(fmaxf(Ar, 0.0f), 1.0f);
    const float sA = sig * A;
    // T = sA (Gy^2, -Gx Gy, Gx^2) / |G|
    const float dTxx_dGx = -sA * Gy * Gy * Gx * iG3, dTxx_dGy = sA * (2.f * Gy * iG - Gy * Gy * Gy * iG3);
    const float dTxy_dGx = -sA * (Gy * iG - Gx * Gx * Gy * iG3), dTxy_dGy = -sA * (Gx * iG - Gx * Gy * Gy * iG3);
    const float dTyy_dGx = sA * (2.f * Gx * iG - Gx * Gx * Gx * iG3), dTyy_dGy = -sA * Gx * Gx * Gy * iG3;
    const float lGx = lT[0] * dTxx_dGx + lT[1] * dTxy_dGx + lT[2] * dTyy_dGx;
    const float lGy = lT[0] * dTxx_dGy + lT[1] * dTxy_dGy + lT[2] * dTyy_dGy;
    if (Ar > 0.0f && Ar < 1.0f) {
        const float lA = sig * (Gy * Gy * lT[0] - Gx * Gy * lT[1] + Gx * Gx * lT[2]) * iG;
        lck += lA * 1e6f * cl * rho * rho;
        lcl += lA * 1e6f * ck * rho * rho;
        lrho += lA * 2e6f * ck * cl * rho;
    }
    lgk[0] += cl * lGx;
    lgk[1] += cl * lGy;
    lgl[0] -= ck * lGx;
    lgl[1] -= ck * lGy;
    lcl += gkx * lGx + gky * lGy;
    lck -= glx * lGx + gly * lGy;
}

// B2: adjoint of the divergence, of the stress (local part) and of the gradient stencil (scatter
// into lambda_C)
__global__ void b_stress_grad(const Params P, const Adj A, const uint8_t* __restrict__ type,
                              const float sig01, const float sig02, const float sig12)
{
    const int gx = blockIdx.x * blockDim.x + threadIdx.x - 1, y = blockIdx.y;
    if (gx > P.nx || y >= P.ny) return;
    int cls;
    if (!is_active(P, A, type, gx, y, cls)) return;
    const int NP = P.ny * A.nxp;
    const int p = pad(A, gx, y);
    int kind;
    const int pc = cpos(P, A, gx, y, kind);  // where this position's own C lives
    float c[kNF], g[kNF][2], lc[kNF] = {0, 0, 0}, lg[kNF][2];
    for (int k = 0; k < kNF; k++) {
        c[k] = A.C[k * NP + pc];
        g[k][0] = A.g[(2 * k) * NP + p];
        g[k][1] = A.g[(2 * k + 1) * NP + p];
        lg[k][0] = A.l_g[(2 * k) * NP + p];
        lg[k][1] = A.l_g[(2 * k + 1) * NP + p];
    }
    float lT[3];
    div_adjoint(P, A, type, gx, y, p, lT);
    float lrho = 0.f;
    const float rho = A.rho[pc];
    pair_stress_vjp(sig01, c[0], c[1], g[0][0], g[0][1], g[1][0], g[1][1], rho, lT, lc[0], lc[1], lg[0], lg[1], lrho);
    pair_stress_vjp(sig02, c[0], c[2], g[0][0], g[0][1], g[2][0], g[2][1], rho, lT, lc[0], lc[2], lg[0], lg[2], lrho);
    pair_stress_vjp(sig12, c[1], c[2], g[1][0], g[1][1], g[2][0], g[2][1], rho, lT, lc[1], lc[2], lg[1], lg[2], lrho);
    float m[kQ];
    int src[kQ], src2[kQ];
    stencil_geom(P, A, type, gx, y, cls, src, src2, m);
    for (int k = 0; k < kNF; k++) {
        if (lc[k] != 0.f) atomicAdd(&A.l_C[k * NP + pc], lc[k]);
        // gradient stencil transpose
        for (int a = 1; a < kQ; a++) {
            const float w = 3.0f * wq(a) * (ex(a) * lg[k][0] + ey(a) * lg[k][1]);
            if (w != 0.f) {
                atomicAdd(&A.l_C[k * NP + src[a]], m[a] * w);
                if (src2[a] >= 0) atomicAdd(&A.l_C[k * NP + src2[a]], -w);
            }
        }
    }
    // rho is 1 at C_SB nodes (no dependence); at fluid and ghost positions it is the pulled total
    if (cls != kSB && lrho != 0.f) atomicAdd(&A.l_rho[pc], lrho);
}

// B3: adjoint of the wetting pass, one thread per C_SB node: the wall values' adjoint goes to the
// fluid nodes they were read from (lambda_C), and the local angles' adjoint to l_th
__global__ void b_wet(const Params P, const Adj A, int nw, const int* __restrict__ widx,
                      const uint8_t* __restrict__ type)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    const int NP = P.ny * A.nxp;
    const int i = widx[w];
    const int px = i % P.nx, py = i / P.nx;
    const int p = pad(A, px, py);
    // adjoint of the wall values: from this step's stress and gradients, and from Eq.(21) of the
    // next step
    float l0 = A.l_C[p] + A.l_cw[i], l1 = A.l_C[NP + p] + A.l_cw[P.N + i], l2 = A.l_C[2 * NP + p] + A.l_cw[2 * P.N + i];
    const float c0r = A.wraw[w], c1r = A.wraw[nw + w];
    float c0 = fminf(fmaxf(c0r, 0.f), 1.f), c1 = fminf(fmaxf(c1r, 0.f), 1.f);
    const float s = c0 + c1;
    if (1.f - (s > 1.f ? 1.f : s) > 0.f) {  // c2 = 1 - c0 - c1 > 0
        l0 -= l2;
        l1 -= l2;
    }
    float lc0 = l0, lc1 = l1;
    if (s > 1.f) {
        lc0 = l0 * (1.f / s - c0 / (s * s)) + l1 * (-c1 / (s * s));
        lc1 = l0 * (-c0 / (s * s)) + l1 * (1.f / s - c1 / (s * s));
    }
    if (!(c0r >= 0.f && c0r <= 1.f)) lc0 = 0.f;
    if (!(c1r >= 0.f && c1r <= 1.f)) lc1 = 0.f;
    const float lk[2] = {lc0, lc1};
    for (int k = 0; k < 2; k++) {
        double lth = 0.0;
        if (lk[k] != 0.f) {
            const int j = (2 * k + A.wsel[k * nw + w]) * nw + w;
            const int kind = A.wkind[j];
            if (kind == 1) {
                atomicAdd(&A.l_C[k * NP + A.wa[j]], lk[k]);
            } else if (kind == 2) {
                const float fr = A.wfr[j];
                atomicAdd(&A.l_C[k * NP + A.wa[j]], (1.f - fr) * lk[k]);
                atomicAdd(&A.l_C[k * NP + A.wb[j]], fr * lk[k]);
                const float ca = A.C[k * NP + A.wa[j]], cb = A.C[k * NP + A.wb[j]];
                lth = (double)lk[k] * (cb - ca) * A.wdfr[j];
            } else {
                // w-weighted mean of the fluid neighbours
                double ws = 0.0;
                for (int a = 1; a < kQ; a++)
                    if (node_is_fluid<Store<kStoreF32>>(P, type, px + ex(a), py + ey(a))) ws += a < 5 ? 1.0 / 9.0 : 1.0 / 36.0;
                for (int a = 1; a < kQ; a++) {
                    if (!node_is_fluid<Store<kStoreF32>>(P, type, px + ex(a), py + ey(a))) continue;
                    int kd;
                    const int q = cpos(P, A, px + ex(a), py + ey(a), kd);
                    atomicAdd(&A.l_C[k * NP + q], (float)((a < 5 ? 1.0 / 9.0 : 1.0 / 36.0) / ws * lk[k]));
                }
            }
        }
        A.l_th[k * nw + w] = lth;
    }
}

// B3b: adjoint of Eq.(21), one thread per C_SB node: from the local angles' adjoint to the
// wall-angle triple (accumulated over the steps) and to the lagged wall values of the previous
// step.  Nothing in the reverse chain of this step needs it, so it runs beside it.
__global__ void b_wet_angles(const Params P, const Adj A, int nw, const int* __restrict__ widx,
                             const float* __restrict__ wang, const double* __restrict__ cw_lag)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    const int i = widx[w];
    const double t_rg = wang[3 * w], t_br = wang[3 * w + 1], t_gb = wang[3 * w + 2];
    const double Cr = cw_lag[i], Cg = cw_lag[P.N + i], Cb = cw_lag[2 * P.N + i];
    double l_rg = 0.0, l_br = 0.0, l_gb = 0.0, lCr = 0.0, lCg = 0.0, lCb = 0.0;
    for (int k = 0; k < 2; k++) {
        const double lth = A.l_th[k * nw + w];
        if (lth == 0.0) continue;
        // Eq.(21) in the convex-combination form
        if (k == 0) {
            // theta_r = t_rg + r (t_rb - t_rg), r = Cb / (Cb + Cg), t_rb = 180 - t_br
            const double den = Cb + Cg;
            if (den < 1e-12) {
                l_rg += 0.5 * lth;
                l_br -= 0.5 * lth;
            } else {
                const double r = Cb / den, t_rb = 180.0 - t_br;
                l_rg += (1.0 - r) * lth;
                l_br -= r * lth;
                lCb += lth * (t_rb - t_rg) * Cg / (den * den);
                lCg -= lth * (t_rb - t_rg) * Cb / (den * den);
            }
        } else {
            // theta_g = t_gr + r (t_gb - t_gr), r = Cb / (Cb + Cr), t_gr = 180 - t_rg
            const double den = Cb + Cr;
            if (den < 1e-12) {
                l_gb += 0.5 * lth;
                l_rg -= 0.5 * lth;
            } else {
                const double r = Cb / den, t_gr = 180.0 - t_rg;
                l_rg -= (1.0 - r) * lth;
                l_gb += r * lth;
                lCb += lth * (t_gb - t_gr) * Cr / (den * den);
                lCr -= lth * (t_gb - t_gr) * Cb / (den * den);
            }
        }
    }
    A.d_ang[w] += l_rg;
    A.d_ang[nw + w] += l_br;
    A.d_ang[2 * nw + w] += l_gb;
    A.l_cw2[i] = (float)lCr;
    A.l_cw2[P.N + i] = (float)lCg;
    A.l_cw2[2 * P.N + i] = (float)lCb;
}

// adjoint of rho_k, C_k at the fluid node (x, y) (the ghost-column copies already sent theirs to
// it): lr[k] is added to lambda of each of the node's nine post-streaming populations of fluid k
__device__ __forceinline__ void frac_adjoint(const Params& P, const Adj& A, int x, int y, float lr[kNF])
{
    const int NP = P.ny * A.nxp;
    const int p = pad(A, x, y);
    float lC[kNF], C[kNF];
    for (int k = 0; k < kNF; k++) {
        lC[k] = A.l_C[k * NP + p];
        C[k] = A.C[k * NP + p];
    }
    const float lrho = A.l_rho[p];
    const float rho = A.rho[p];
    float sc = 0.f;
    for (int k = 0; k < kNF; k++) sc += lC[k] * C[k];
    for (int k = 0; k < kNF; k++) lr[k] = (lC[k] - sc) / rho + lrho;
}

// adjoint of the Zou-He completion at the fluid node i of an open column: lk (lambda of the
// node's post-streaming populations, fractions included) becomes lambda of the populations before
// the completion (the unknown ones end there: 0); returns this node's share of dJ/dU
__device__ __forceinline__ double zouhe_adjoint(const Params& P, const Adj& A, bool inlet, int i, float lk[27])
{
    float fk[27];
#pragma unroll
    for (int j = 0; j < 27; j++) fk[j] = A.fpost[(long long)j * P.N + i];
    float f[kQ];
#pragma unroll
    for (int a = 0; a < kQ; a++) f[a] = fk[a] + fk[9 + a] + fk[18 + a];
    float lf[kQ] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, lpart[kNF] = {0, 0, 0};
    double lU = 0.0;
    if (inlet) {
        // inlet x = 0: unknown a = 1, 5, 8 (fluid 2)
        const float U = P.u_in;
        const float rho = (f[0] + f[2] + f[4] + 2.f * (f[3] + f[6] + f[7])) / (1.f - U);
        const float L1 = lk[18 + 1], L5 = lk[18 + 5], L8 = lk[18 + 8];
        const float lrho = (2.f / 3.f) * U * L1 + (U / 6.f) * (L5 + L8);
        lf[3] += L1;
        lf[7] += L5;
        lf[6] += L8;
        lf[2] += -0.5f * L5 + 0.5f * L8;
        lf[4] += 0.5f * L5 - 0.5f * L8;
        const float ir = 1.f / (1.f - U);
        lf[0] += lrho * ir;
        lf[2] += lrho * ir;
        lf[4] += lrho * ir;
        lf[3] += 2.f * lrho * ir;
        lf[6] += 2.f * lrho * ir;
        lf[7] += 2.f * lrho * ir;
        lU = (double)L1 * (2.0 / 3.0) * rho + (double)(L5 + L8) * rho / 6.0 + (double)lrho * rho / (1.0 - U);
    } else {
        // outlet x = nx-1: unknown a = 3, 6, 7, split by the known fractions
        float part[kNF], tot = 0.f;
#pragma unroll
        for (int k = 0; k < kNF; k++) {
            const float* q = fk + 9 * k;
            part[k] = q[0] + q[1] + q[2] + q[4] + q[5] + q[8];
            tot += part[k];
        }
        const float ro = P.rho_out;
        const float S = f[0] + f[2] + f[4] + 2.f * (f[1] + f[5] + f[8]);
        const float h3 = f[1] - (2.f / 3.f) * (S - ro);
        const float h7 = f[5] + 0.5f * (f[2] - f[4]) - (S - ro) / 6.f;
        const float h6 = f[8] - 0.5f * (f[2] - f[4]) - (S - ro) / 6.f;
        float lh3 = 0.f, lh6 = 0.f, lh7 = 0.f, acc = 0.f;
#pragma unroll
        for (int k = 0; k < kNF; k++) {
            const float a3 = lk[9 * k + 3], a6 = lk[9 * k + 6], a7 = lk[9 * k + 7];
            lh3 += a3 * part[k] / tot;
            lh6 += a6 * part[k] / tot;
            lh7 += a7 * part[k] / tot;
            lpart[k] = (a3 * h3 + a6 * h6 + a7 * h7) / tot;
            acc += lpart[k] * part[k] / tot;
        }
#pragma unroll
        for (int k = 0; k < kNF; k++) lpart[k] -= acc;
        // h3 = f1 - (2/3)(S - ro), h7 = f5 + (f2 - f4)/2 - (S - ro)/6, h6 = f8 - (f2 - f4)/2 - (S - ro)/6
        lf[1] += lh3 * (1.f - 4.f / 3.f);
        lf[0] += lh3 * (-2.f / 3.f);
        lf[2] += lh3 * (-2.f / 3.f);
        lf[4] += lh3 * (-2.f / 3.f);
        lf[5] += lh3 * (-4.f / 3.f);
        lf[8] += lh3 * (-4.f / 3.f);
        lf[5] += lh7 * (1.f - 1.f / 3.f);
        lf[2] += lh7 * (0.5f - 1.f / 6.f);
        lf[4] += lh7 * (-0.5f - 1.f / 6.f);
        lf[0] += lh7 * (-1.f / 6.f);
        lf[1] += lh7 * (-1.f / 3.f);
        lf[8] += lh7 * (-1.f / 3.f);
        lf[8] += lh6 * (1.f - 1.f / 3.f);
        lf[2] += lh6 * (-0.5f - 1.f / 6.f);
        lf[4] += lh6 * (0.5f - 1.f / 6.f);
        lf[0] += lh6 * (-1.f / 6.f);
        lf[1] += lh6 * (-1.f / 3.f);
        lf[5] += lh6 * (-1.f / 3.f);
    }
#pragma unroll
    for (int k = 0; k < kNF; k++)
#pragma unroll
        for (int a = 0; a < kQ; a++) {
            const bool unknown = inlet ? (a == 1 || a == 5 || a == 8) : (a == 3 || a == 6 || a == 7);
            lk[9 * k + a] = unknown ? 0.f : lk[9 * k + a] + (lf[a] + lpart[k]);
        }
    return lU;
}

// B4: adjoint of the fractions, of the Zou-He completion and of the pull, pushed back from the
// puller.  The post-streaming population (d, a) of the fluid node d came from the stored
// population (d - e_a, a), or, where d - e_a is solid or beyond a wall side, from its own
// (d, opp a) by the halfway bounce-back; its lambda, with the adjoint of d's fractions added (and,
// at an open column, taken through the adjoint of the Zou-He completion), goes back there.
// Every stored population of a fluid node has exactly one puller, except those that leave
// through an open side, which nobody reads (lambda 0).  Solid nodes' lambda is never read.
__global__ void b_pull(const Params P, const Adj A, const uint8_t* __restrict__ type)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const int i = y * P.nx + x;
    if (type[i] & 2) return;
    const bool zh = P.bc_x == kZouHe;
    const bool zcol = zh && (x == 0 || x == P.nx - 1);
    float lr[kNF];
    frac_adjoint(P, A, x, y, lr);
    float lk[27];
#pragma unroll
    for (int j = 0; j < 27; j++) lk[j] = A.l_fpost[(long long)j * P.N + i] + lr[j / 9];
    if (zcol) {
        const double lU = zouhe_adjoint(P, A, x == 0, i, lk);
        if (lU != 0.0) atomicAdd(A.d_u, lU);
    }
#pragma unroll
    for (int a = 0; a < kQ; a++) {
        int X = x - ex(a), Y = y - ey(a);
        const int sk = wrap_xy(P, X, Y);
        int dst = i, dir = opp(a);
        if (sk == 2) continue;  // entered through an open side: a Zou-He unknown, no stored source
        if (sk == 0 && !(type[Y * P.nx + X] & 2)) {
            dst = Y * P.nx + X;
            dir = a;
        }
        for (int k = 0; k < kNF; k++) A.l_fs[(long long)(9 * k + dir) * P.N + dst] = lk[9 * k + a];
    }
    if (zcol)
        for (int a = 1; a < kQ; a++) {
            int X = x + ex(a), Y = y + ey(a);
            if (wrap_xy(P, X, Y) != 2) continue;
            for (int k = 0; k < kNF; k++) A.l_fs[(long long)(9 * k + a) * P.N + i] = 0.f;
        }
}

// objective: x-centroid of fluid 0, J = sum x rho_0 / sum rho_0 over the post-streaming state,
// from the diagnostics of the final state (diag[0] = sum rho_0, diag[3] = sum x rho_0, so that
// no value passes through the host); seed lambda_fpost = dJ/dfpost
__global__ void b_seed(const Params P, const Adj A, const uint8_t* __restrict__ type,
                       const double* __restrict__ diag)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const double M0 = diag[0], J = diag[3] / M0;
    const int i = y * P.nx + x;
    const bool fluid = !(type[i] & 2);
    for (int k = 0; k < kNF; k++)
        for (int a = 0; a < kQ; a++)
            A.l_fpost[(long long)(9 * k + a) * P.N + i] = (fluid && k == 0) ? (float)(((double)x - J) / M0) : 0.f;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// host-side driver
// ------------------------------------------------------------------------------------------
// The forward intermediates of a step depend only on its stored state, not on the adjoint, so
// they are computed on a stream of their own one step ahead of the reverse chain, into the
// buffer set of the step's parity: the two views A[0], A[1] share the adjoint arrays that the
// reverse chain carries from step to step and differ in the intermediates and in lambda_C,
// lambda_rho (cleared by a_dens).  The adjoint of Eq.(21) (b_wet_angles) runs on a third stream
// beside the rest of the step's reverse chain; the next step's b_wet waits for it.
struct AdjointWork {
    Adj A[2];
    size_t bytes = 0;
    cudaStream_t side = nullptr, side_w = nullptr;
    cudaEvent_t ev_a[2] = {nullptr, nullptr};  // intermediates of the parity ready
    cudaEvent_t ev_b[2] = {nullptr, nullptr};  // reverse of the parity done with them
    cudaEvent_t ev_sync = nullptr, ev_wet = nullptr, ev_ang = nullptr;
    bool ang_recorded = false;  // ev_ang was recorded in this sweep (no wait on an older record)
};

static cudaError_t amalloc(void** p, size_t b, size_t& tot)
{
    tot += b;
    return cudaMalloc(p, b ? b : 16);
}

cudaError_t adjoint_alloc(const Params& P, int nw, AdjointWork** out)
{
    AdjointWork* W = new AdjointWork();
    *out = W;
    const size_t N = (size_t)P.N, NP = (size_t)P.ny * (P.nx + 2);
    const size_t nwz = nw > 0 ? (size_t)nw : 1;
    size_t& t = W->bytes;
    cudaError_t e = cudaSuccess;
    auto M = [&](void** p, size_t b) {
        if (e == cudaSuccess) e = amalloc(p, b, t);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, b ? b : 16);
    };
    Adj& S = W->A[0];
    S.nxp = P.nx + 2;
    // shared by both views
    M((void**)&S.wline, 4 * nwz * sizeof(AdjLine));
    if (e == cudaSuccess) e = cudaMemset(S.wline, 0xff, 4 * nwz * sizeof(AdjLine));  // th = NaN: march
    M((void**)&S.l_fpost, 27 * N * 4);
    M((void**)&S.l_F, 2 * N * 4);
    M((void**)&S.l_g, 6 * NP * 4);
    M((void**)&S.l_fs, 27 * N * 4);
    M((void**)&S.l_cw, 3 * N * 4);
    M((void**)&S.l_cw2, 3 * N * 4);
    M((void**)&S.l_th, 2 * nwz * 8);
    M((void**)&S.d_ang, 3 * nwz * 8);
    M((void**)&S.d_u, 8);
    W->A[1] = S;
    // one set per parity
    for (Adj& A : W->A) {
        M((void**)&A.fpost, 27 * N * 4);
        M((void**)&A.C, 3 * NP * 4);
        M((void**)&A.rho, NP * 4);
        M((void**)&A.g, 6 * NP * 4);
        M((void**)&A.T, 3 * NP * 4);
        M((void**)&A.F, 2 * N * 4);
        M((void**)&A.wkind, 4 * nwz * 4);
        M((void**)&A.wa, 4 * nwz * 4);
        M((void**)&A.wb, 4 * nwz * 4);
        M((void**)&A.wfr, 4 * nwz * 4);
        M((void**)&A.wdfr, 4 * nwz * 4);
        M((void**)&A.wraw, 2 * nwz * 4);
        M((void**)&A.wsel, 2 * nwz * 4);
        M((void**)&A.l_C, 3 * NP * 4);
        M((void**)&A.l_rho, NP * 4);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&W->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&W->side_w, cudaStreamNonBlocking);
    for (int c = 0; c < 2; c++) {
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&W->ev_a[c], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&W->ev_b[c], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&W->ev_sync, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&W->ev_wet, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&W->ev_ang, cudaEventDisableTiming);
    return e;
}

void adjoint_free(AdjointWork* W)
{
    if (!W) return;
    const Adj& S = W->A[0];
    void* shared[] = {S.wline, S.l_fpost, S.l_F, S.l_g, S.l_fs, S.l_cw, S.l_cw2, S.l_th, S.d_ang, S.d_u};
    for (void* p : shared)
        if (p) cudaFree(p);
    for (const Adj& A : W->A) {
        void* own[] = {A.fpost, A.C, A.rho, A.g, A.T, A.F, A.wkind, A.wa, A.wb, A.wfr, A.wdfr, A.wraw, A.wsel, A.l_C, A.l_rho};
        for (void* p : own)
            if (p) cudaFree(p);
    }
    if (W->side) cudaStreamDestroy(W->side);
    if (W->side_w) cudaStreamDestroy(W->side_w);
    cudaEvent_t evs[] = {W->ev_a[0], W->ev_a[1], W->ev_b[0], W->ev_b[1], W->ev_sync, W->ev_wet, W->ev_ang};
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    delete W;
}

size_t adjoint_bytes(const AdjointWork* W) { return W ? W->bytes : 0; }

double* adjoint_dang(AdjointWork* W) { return W->A[0].d_ang; }
double* adjoint_du(AdjointWork* W) { return W->A[0].d_u; }

// seed the adjoint from the final stored populations: lambda_fs = pull^T (dJ/dfpost)
void adjoint_seed(const Params& P, AdjointWork* W, const float* fs, const uint8_t* type, const double* diag,
                  cudaStream_t s)
{
    Adj& A = W->A[0];
    const dim3 gn((P.nx + 127) / 128, P.ny), gp((P.nx + 2 + 127) / 128, P.ny);
    a_dens<<<gp, 128, 0, s>>>(P, A, fs, type);
    b_seed<<<gn, 128, 0, s>>>(P, A, type, diag);
    b_pull<<<gn, 128, 0, s>>>(P, A, type);
    cudaMemsetAsync(A.l_cw, 0, sizeof(float) * 3 * (size_t)P.N, s);
    W->ang_recorded = false;
}

cudaError_t adjoint_sync(AdjointWork* W, cudaStream_t s)
{
    cudaError_t e = cudaEventRecord(W->ev_sync, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(W->side, W->ev_sync, 0);
    return e;
}

cudaError_t adjoint_join(AdjointWork* W, cudaStream_t s)
{
    return W->ang_recorded ? cudaStreamWaitEvent(s, W->ev_ang, 0) : cudaSuccess;
}

cudaStream_t adjoint_side_stream(AdjointWork* W) { return W->side; }

// forward intermediates of step t from its stored populations fs and lagged wall values cw_lag,
// on the side stream; wait_reverse: first wait until the reverse of step t + 2 (the same buffer
// set) is done with them
cudaError_t adjoint_prepare(const Params& P, AdjointWork* W, int t, bool wait_reverse, int nw,
                            const int* widx, const double* wnrm, const float* wang, const float* fs,
                            const double* cw_lag, const uint8_t* type)
{
    const int c = t & 1;
    const Adj& A = W->A[c];
    cudaStream_t s = W->side;
    cudaError_t e = wait_reverse ? cudaStreamWaitEvent(s, W->ev_b[c], 0) : cudaSuccess;
    if (e != cudaSuccess) return e;
    const dim3 gp((P.nx + 2 + 127) / 128, P.ny);
    a_dens<<<gp, 128, 0, s>>>(P, A, fs, type);
    if (nw > 0)
        a_wet<<<(unsigned)((4LL * nw + 127) / 128), 128, 0, s>>>(P, A, nw, widx, wnrm, wang, fs, type, cw_lag);
    a_grad_stress<<<gp, 128, 0, s>>>(P, A, type, P.sig01, P.sig02, P.sig12);
    a_force<<<dim3((P.nx + 127) / 128, P.ny), 128, 0, s>>>(P, A, type);
    return cudaEventRecord(W->ev_a[c], s);
}

// the reverse of step t on s, once its intermediates are ready: on entry lambda_fs and
// lambda_cw hold the adjoint of the step's outputs, on exit of its inputs
cudaError_t adjoint_reverse(const Params& P, AdjointWork* W, int t, int nw, const int* widx,
                            const float* wang, const double* cw_lag, const uint8_t* type, cudaStream_t s)
{
    const int c = t & 1;
    const Adj& A = W->A[c];
    cudaError_t e = cudaStreamWaitEvent(s, W->ev_a[c], 0);
    if (e != cudaSuccess) return e;
    const dim3 gn((P.nx + 127) / 128, P.ny), gp((P.nx + 2 + 127) / 128, P.ny);
    b_collide<<<gn, 128, 0, s>>>(P, A, type);
    b_stress_grad<<<gp, 128, 0, s>>>(P, A, type, P.sig01, P.sig02, P.sig12);
    if (nw > 0) {
        // lambda_cw and l_th: b_wet_angles of the step after this one is done with them
        if (W->ang_recorded && (e = cudaStreamWaitEvent(s, W->ev_ang, 0)) != cudaSuccess) return e;
        b_wet<<<(nw + 127) / 128, 128, 0, s>>>(P, A, nw, widx, type);
        if ((e = cudaEventRecord(W->ev_wet, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(W->side_w, W->ev_wet, 0)) != cudaSuccess) return e;
        b_wet_angles<<<(nw + 127) / 128, 128, 0, W->side_w>>>(P, A, nw, widx, wang, cw_lag);
        if ((e = cudaEventRecord(W->ev_ang, W->side_w)) != cudaSuccess) return e;
        W->ang_recorded = true;
    }
    b_pull<<<gn, 128, 0, s>>>(P, A, type);
    for (Adj& V : W->A) std::swap(V.l_cw, V.l_cw2);
    return cudaEventRecord(W->ev_b[c], s);
}

}  // namespace lbm3k
