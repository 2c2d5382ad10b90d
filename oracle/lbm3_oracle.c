/*
 * lbm3_oracle.c -- plain, slow FP64 CPU oracle of one timestep of the three-phase
 * MRT colour-gradient lattice Boltzmann model with the characteristic-line wetting
 * condition (arXiv:2102.04709, Section II).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference legs may load this library.  The GPU product path never
 * links, loads or calls it, and it shares no code, header, table or helper with the
 * CUDA sources: every constant below is written out again from the paper.
 *
 * The step follows the paper's order and notation:
 *   O1  Eq.(16) last sentence: rho_k = sum_a f_ak, rho = sum_k rho_k, C_k = rho_k/rho
 *   O2  Eq.(21): weighted local contact angles theta_r, theta_g at every C_SB node
 *   O3  Section II.B (text after Eq.21): two characteristic lines l1, l2 per fluid,
 *       march to the first grid-line crossing whose two bracketing nodes are in C_F,
 *       linear interpolation
 *   O4  Eq.(22): C_P = max/min(C_D1, C_D2); C_b = 1 - C_r - C_g
 *   O5  Eq.(12): isotropic gradients of C_k (C_SB values enter the stencil)
 *   O6  Eq.(10)-(11): G_kl, n_kl, A_kl, F_s = divergence of the surface-stress tensor
 *   O7  Eq.(11), (7), (3): velocity with half force, mixture relaxation time, f^eq
 *   O8  Eq.(1), (2), (4)-(6), (8), (9): MRT collision with forcing, literal 9x9 matrices
 *   O9  Eq.(13)-(15): recolouring with segregation parameters beta_kl
 *   O10 Eq.(16): streaming with halfway bounce-back, periodic / modified periodic
 *       (Section III.C) and Zou-He velocity inlet / pressure outlet (Section III.D)
 *
 * Readings of points the paper leaves open (each one also listed in the design notes):
 *   - weights of directions 5-8 are 1/36 (the text prints "5-6"; the weights must sum to 1)
 *   - Eq.(10) sums ordered pairs with a factor 1/2, i.e. each unordered pair once
 *   - n_kl = 0 and no stress contribution when |G_kl|^2 <= 1e-24
  *   - the stress tensor is also evaluated at C_SB nodes; a neighbour in that stencil with no
 *     C of its own (C_SI, or solid beyond a wall side) takes the linear extrapolation
 *     2 C(P) - C(P - e_a) through the C_SB node P, or C(P) when P - e_a has no C either
 *     (this reading reproduces the angles of Table I; C(P) alone biased them towards 90 deg)
 *   - at C_SB nodes rho := 1, so rho_k = C_k for A_kl
 *   - "in contact with" means any of the 8 D2Q9 neighbours
 *   - n_s of Eq.(19) points into the solid; the characteristic lines use -n_s
 *   - Eq.(21) uses the C_SB values of the previous step (initially the w-weighted mean
 *     of the fluid neighbours), evaluated with 1 - C_r = C_b + C_g as the convex combination
 *     theta_r = theta_rg + C_b/(C_b + C_g) (theta_rb - theta_rg) (and likewise for green);
 *     when both weights are below 1e-12 theta_k is the mean of its two angles
 *   - |pi/2 - theta_k| below 1e-6 deg is taken as 0 (both lines along n_s)
 *   - ray march: crossings within 1e-6 of a node are node hits; search stops at t > 16;
 *     if no valid crossing exists, C_D is the w-weighted mean of the fluid neighbours
 *   - Eq.(22) tie theta_k = 90 deg takes the max branch; if C_r + C_g > 1 both are
 *     rescaled to sum to 1, and C_b = max(0, 1 - C_r - C_g)
 *   - modified periodic: every population or C value that crosses the x seam swaps the
 *     labels of fluids 0 and 2 (requires sigma_01 == sigma_12 so the stress is unchanged)
 *   - Zou-He: velocity inlet at x = 0 (incoming populations belong to fluid 2), pressure
 *     outlet at x = nx-1 (incoming populations split by the known populations' fractions);
 *     C beyond the open columns is a copy of the boundary column (zero gradient)
 *
 * Fluid indices 0, 1, 2 are the paper's red, green, blue.
 *
 * Threads: the per-node loops of a step may run on several OpenMP threads (ora_set_threads,
 * default 1).  Every iteration writes only its own node's values (push streaming: each
 * destination population has exactly one source), and no loop reduces across nodes, so the
 * result is bit-identical for any thread count.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define Q 9
#define NF 3

/* Scalar type of every quantity that depends on the state or on the differentiated parameters
 * (wall angles, inflow velocity): double here.  The reference tape (lbm3_oracle_tape.cpp)
 * compiles this same file with a reverse-mode recording type in its place, so that its
 * gradients are those of exactly these operations.  VAL() reads a value out of either. */
#ifndef ORA_TAPE
typedef double real;
#define VAL(x) (x)
#endif

/* ---- D2Q9 lattice, Section II.A (text below Eq.3) ---- */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WQ[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2 with dx = dt = 1 */

/* ---- transformation matrix, Eq.(4) ---- */
static const double MMAT[Q][Q] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},         {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},     {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},      {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},      {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

enum { BC_PERIODIC = 0, BC_MODPER = 1, BC_ZOUHE = 2, BC_WALLS = 3 };
enum { CL_FI = 0, CL_FB = 1, CL_SB = 2, CL_SI = 3 };
enum { LOC_IN = 0, LOC_SOLID = 1, LOC_GHOST = 2 };

#define G2_EPS 1e-24
#define RAY_TMAX 16.0
#define RAY_EPS 1e-6
#define PHI_SNAP 1e-6

typedef struct ora {
    int nx, ny, n;
    int per_y, bc_x;
    real u_in;
    double rho_out;
    double sigma[NF][NF]; /* symmetric interfacial tensions, Eq.(10) */
    double nu[NF];        /* kinematic viscosities; mu_k = rho_k^0 nu_k with rho_k^0 = 1 */
    double rho0[NF];      /* pure-fluid densities (all 1: the method assumes equal densities) */
    double beta0;
    double gX[NF][NF];    /* g(X_kl), Eq.(15) */
    double Minv[Q][Q];
    int opp[Q];
    unsigned char *solid, *cls;
    real *theta;          /* per node: theta_01, theta_20, theta_12 (deg) = theta_rg, theta_br, theta_gb */
    double *ns;           /* outward unit normal at C_SB nodes (minus Eq.19) */
    real   *f, *fnew;     /* [k][a][node] post-streaming populations */
    real   *rho;          /* [k][node] */
    real   *C;            /* [k][node]: fluid nodes from O1, C_SB nodes from O4 */
    real   *Cw;           /* [k][node]: C_SB values of the previous step (Eq.21 input) */
    real   *T;            /* [3][node]: Txx, Txy, Tyy at C_F and C_SB nodes */
    real   *Fs;           /* [2][node] */
    real   *u;            /* [2][node]: velocity of the last collision, Eq.(11) */
    long steps;
    int threads;          /* OpenMP threads of the per-node loops (1 unless set) */
} ora_t;

/* ------------------------------------------------------------------------- */
/* small helpers                                                              */
/* ------------------------------------------------------------------------- */
static int swapk(int k) { return k == 1 ? 1 : 2 - k; }

static int floordiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

/* Where does lattice position (X, Y) live?  Periodic directions wrap (the x seam of the
 * modified periodic boundary swaps fluids 0 and 2 once per crossing); wall directions are
 * solid outside the domain; the open x direction has ghost copies of the boundary column. */
static int locate(const ora_t* o, int X, int Y, int* idx, int* swap)
{
    *swap = 0;
    if (Y < 0 || Y >= o->ny) {
        if (!o->per_y) return LOC_SOLID;
        Y -= floordiv(Y, o->ny) * o->ny;
    }
    if (X < 0 || X >= o->nx) {
        if (o->bc_x == BC_PERIODIC || o->bc_x == BC_MODPER) {
            int q = floordiv(X, o->nx);
            X -= q * o->nx;
            if (o->bc_x == BC_MODPER && (q & 1)) *swap = 1;
        } else if (o->bc_x == BC_WALLS) {
            return LOC_SOLID;
        } else {
            X = X < 0 ? 0 : o->nx - 1;
            *idx = Y * o->nx + X;
            return LOC_GHOST;
        }
    }
    *idx = Y * o->nx + X;
    return LOC_IN;
}

static int is_solid_at(const ora_t* o, int X, int Y)
{
    int idx, sw;
    int loc = locate(o, X, Y, &idx, &sw);
    if (loc == LOC_SOLID) return 1;
    if (loc == LOC_GHOST) return 0;
    return o->solid[idx];
}

/* C_k at a located position, seen in the frame of the caller */
static real c_at(const ora_t* o, int idx, int sw, int k)
{
    return o->C[(size_t)(sw ? swapk(k) : k) * o->n + idx];
}

/* Gauss-Jordan inverse with partial pivoting (used once for M^-1) */
static int invert9(const double A[Q][Q], double R[Q][Q])
{
    double a[Q][2 * Q];
    for (int i = 0; i < Q; i++)
        for (int j = 0; j < 2 * Q; j++) a[i][j] = j < Q ? A[i][j] : (j - Q == i ? 1.0 : 0.0);
    for (int c = 0; c < Q; c++) {
        int p = c;
        for (int r = c + 1; r < Q; r++)
            if (fabs(a[r][c]) > fabs(a[p][c])) p = r;
        if (fabs(a[p][c]) < 1e-14) return -1;
        if (p != c)
            for (int j = 0; j < 2 * Q; j++) {
                double t = a[c][j];
                a[c][j] = a[p][j];
                a[p][j] = t;
            }
        double d = a[c][c];
        for (int j = 0; j < 2 * Q; j++) a[c][j] /= d;
        for (int r = 0; r < Q; r++) {
            if (r == c) continue;
            double m = a[r][c];
            if (m != 0.0)
                for (int j = 0; j < 2 * Q; j++) a[r][j] -= m * a[c][j];
        }
    }
    for (int i = 0; i < Q; i++)
        for (int j = 0; j < Q; j++) R[i][j] = a[i][Q + j];
    return 0;
}

/* Eq.(15) */
double ora_gfun(double X)
{
    if (X < -1.0) return 1.0;
    if (X < 0.0) return 1.0 - sin(acos(X));
    if (X <= 1.0) return sin(acos(X)) - 1.0;
    return -1.0;
}

/* ------------------------------------------------------------------------- */
/* Eq.(1)-(9), (11): MRT collision with the forcing term at one node          */
/* ------------------------------------------------------------------------- */
static void matvec(const double A[Q][Q], const real* x, real* y)
{
    for (int i = 0; i < Q; i++) {
        real s = 0.0;
        for (int j = 0; j < Q; j++) s += A[i][j] * x[j];
        y[i] = s;
    }
}

static void collide_node(const double Minv[Q][Q], const real f[Q], const real Fs[2],
                         real tau, real fdag[Q], real u[2])
{
    real rho = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < Q; a++) {
        rho += f[a];
        jx += f[a] * EX[a];
        jy += f[a] * EY[a];
    }
    /* Eq.(11) */
    u[0] = (jx + 0.5 * Fs[0]) / rho;
    u[1] = (jy + 0.5 * Fs[1]) / rho;
    real uu = u[0] * u[0] + u[1] * u[1];
    real feq[Q], Ft[Q], d[Q], m[Q], om[Q], mF[Q], Fbar[Q];
    for (int a = 0; a < Q; a++) {
        real eu = EX[a] * u[0] + EY[a] * u[1];
        /* Eq.(3) */
        feq[a] = rho * WQ[a] * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
        /* Eq.(9) */
        real cx = (EX[a] - u[0]) / CS2 + eu * EX[a] / (CS2 * CS2);
        real cy = (EY[a] - u[1]) / CS2 + eu * EY[a] / (CS2 * CS2);
        Ft[a] = WQ[a] * (cx * Fs[0] + cy * Fs[1]);
        d[a] = f[a] - feq[a];
    }
    /* Eq.(5)-(6) */
    real s1 = 1.0 / tau;
    real s4 = 8.0 * (2.0 - s1) / (8.0 - s1);
    real S[Q] = {0.0, s1, s1, 0.0, s4, 0.0, s4, s1, s1};
    /* Eq.(2): Omega = -M^-1 S M (f - f^eq) */
    matvec(MMAT, d, m);
    for (int i = 0; i < Q; i++) m[i] *= S[i];
    matvec(Minv, m, om);
    /* Eq.(8): Fbar = M^-1 (I - S/2) M Ftilde */
    matvec(MMAT, Ft, mF);
    for (int i = 0; i < Q; i++) mF[i] *= (1.0 - 0.5 * S[i]);
    matvec(Minv, mF, Fbar);
    /* Eq.(1) */
    for (int a = 0; a < Q; a++) fdag[a] = f[a] - om[a] + Fbar[a];
}

/* Eq.(7): rho/mu = sum_k rho_k/mu_k, mu = (tau - 1/2) rho c_s^2 */
static real mixture_tau(const ora_t* o, const real rk[NF])
{
    real rho = rk[0] + rk[1] + rk[2];
    real inv = 0.0;
    for (int k = 0; k < NF; k++) inv += rk[k] / (o->rho0[k] * o->nu[k]);
    real mu = rho / inv;
    return mu / (rho * CS2) + 0.5;
}

/* ------------------------------------------------------------------------- */
/* Eq.(12) gradients and the Eq.(10) stress tensor at a position              */
/* ------------------------------------------------------------------------- */
/* C_k (frame of the caller) and rho_k at position (X, Y) that is a fluid node, a C_SB
 * node or a ghost of the open boundary */
static void state_at(const ora_t* o, int X, int Y, real c[NF], real rk[NF])
{
    int idx, sw;
    int loc = locate(o, X, Y, &idx, &sw);
    for (int k = 0; k < NF; k++) c[k] = c_at(o, idx, sw, k);
    if (loc == LOC_IN && o->solid[idx]) {
        for (int k = 0; k < NF; k++) rk[k] = c[k] * 1.0; /* rho := 1 at C_SB nodes */
    } else {
        for (int k = 0; k < NF; k++) rk[k] = o->rho[(size_t)(sw ? swapk(k) : k) * o->n + idx];
    }
}

/* Eq.(12) on the 9 values v[a] = psi(x + e_a): g = sum_a w_a psi(x + e_a) e_a / c_s^2 (the
 * step's gradients and the ora_gradient_periodic accessor both use it) */
static void eq12(const real v[Q], real g[2])
{
    g[0] = g[1] = 0.0;
    for (int a = 0; a < Q; a++) {
        g[0] += WQ[a] * v[a] * EX[a] / CS2;
        g[1] += WQ[a] * v[a] * EY[a] / CS2;
    }
}

/* a position whose C is never defined: solid beyond a wall side, a C_SI node, or the ghost
 * copy of a C_SI node beyond an open side */
static int no_value(const ora_t* o, int loc, int idx)
{
    return loc == LOC_SOLID || o->cls[idx] == CL_SI;
}

/* grad C_k at (X, Y) by Eq.(12).  Only a C_SB centre has neighbours without a value; such a
 * neighbour P + e_a takes the value on the straight line through the opposite neighbour and
 * the centre, 2 C(P) - C(P - e_a) (the centre's own value when P - e_a has none either) */
static void grad_at(const ora_t* o, int X, int Y, real g[NF][2])
{
    real c0[NF], r0[NF];
    state_at(o, X, Y, c0, r0);
    real v[NF][Q];
    for (int k = 0; k < NF; k++) v[k][0] = c0[k];
    for (int a = 1; a < Q; a++) {
        int idx, sw;
        int loc = locate(o, X + EX[a], Y + EY[a], &idx, &sw);
        if (no_value(o, loc, idx)) {
            int idx2, sw2;
            int loc2 = locate(o, X - EX[a], Y - EY[a], &idx2, &sw2);
            if (no_value(o, loc2, idx2)) {
                for (int k = 0; k < NF; k++) v[k][a] = c0[k];
            } else {
                for (int k = 0; k < NF; k++) v[k][a] = 2.0 * c0[k] - c_at(o, idx2, sw2, k);
            }
        } else {
            for (int k = 0; k < NF; k++) v[k][a] = c_at(o, idx, sw, k);
        }
    }
    for (int k = 0; k < NF; k++) eq12(v[k], g[k]);
}

/* Eq.(10) tensor sum_k sum_{l!=k} (sigma_kl A_kl / 2) |G_kl| (I - n_kl n_kl) at (X, Y) */
static void tensor_at(const ora_t* o, int X, int Y, real T[3])
{
    real c[NF], rk[NF], g[NF][2];
    state_at(o, X, Y, c, rk);
    grad_at(o, X, Y, g);
    T[0] = T[1] = T[2] = 0.0;
    for (int k = 0; k < NF; k++)
        for (int l = 0; l < NF; l++) {
            if (l == k) continue;
            real Gx = c[l] * g[k][0] - c[k] * g[l][0];
            real Gy = c[l] * g[k][1] - c[k] * g[l][1];
            real G2 = Gx * Gx + Gy * Gy;
            if (G2 <= G2_EPS) continue;
            real Gn = sqrt(G2);
            real nx = Gx / Gn, ny = Gy / Gn;
            real A = fmin(1e6 * rk[k] * rk[l] / (o->rho0[k] * o->rho0[l]), 1.0);
            real s = 0.5 * o->sigma[k][l] * A * Gn;
            T[0] += s * (1.0 - nx * nx);
            T[1] += s * (0.0 - nx * ny);
            T[2] += s * (1.0 - ny * ny);
        }
}

/* ------------------------------------------------------------------------- */
/* Section II.B: characteristic lines                                         */
/* ------------------------------------------------------------------------- */
static int fluid_at(const ora_t* o, int X, int Y, int* idx, int* sw)
{
    int loc = locate(o, X, Y, idx, sw);
    if (loc == LOC_SOLID) return 0;
    if (loc == LOC_GHOST) return 0; /* a characteristic line stops at an open boundary */
    return !o->solid[*idx];
}

/* w-weighted mean of C_k over the fluid D2Q9 neighbours of node (px, py) */
static real neighbour_mean(const ora_t* o, int px, int py, int k)
{
    real s = 0.0;
    double ws = 0.0;
    for (int a = 1; a < Q; a++) {
        int idx, sw;
        if (fluid_at(o, px + EX[a], py + EY[a], &idx, &sw)) {
            s += WQ[a] * c_at(o, idx, sw, k);
            ws += WQ[a];
        }
    }
    return ws > 0.0 ? s / ws : 0.0;
}

/* March P + t d (t > 0) across the grid lines; return 1 and C_D at the first crossing whose
 * bracketing nodes are both in C_F. */
static int march(const ora_t* o, int px, int py, real dx, real dy, int k, real* CD)
{
    int sx = dx > 0 ? 1 : -1, sy = dy > 0 ? 1 : -1;
    int useX = fabs(dx) > 1e-14, useY = fabs(dy) > 1e-14;
    int Xn = px + sx, Yn = py + sy;
    real tv = useX ? (Xn - px) / dx : INFINITY;
    real th = useY ? (Yn - py) / dy : INFINITY;
    for (;;) {
        real t = fmin(tv, th);
        if (!(t <= RAY_TMAX)) return 0;
        int hitV = (tv - t) <= RAY_EPS, hitH = (th - t) <= RAY_EPS;
        int idx, sw, idx2, sw2;
        if (hitV && hitH) {
            /* passes through the node (Xn, Yn) */
            if (fluid_at(o, Xn, Yn, &idx, &sw)) {
                *CD = c_at(o, idx, sw, k);
                return 1;
            }
        } else if (hitV) {
            /* vertical grid line x = Xn: interpolate between the lower and upper node */
            real ys = py + t * dy;
            double Yr = floor(ys + 0.5);
            if (fabs(ys - Yr) < RAY_EPS) {
                if (fluid_at(o, Xn, (int)Yr, &idx, &sw)) {
                    *CD = c_at(o, idx, sw, k);
                    return 1;
                }
            } else {
                int Y0 = (int)floor(ys);
                real fr = ys - Y0;
                if (fluid_at(o, Xn, Y0, &idx, &sw) && fluid_at(o, Xn, Y0 + 1, &idx2, &sw2)) {
                    real Clow = c_at(o, idx, sw, k), Cup = c_at(o, idx2, sw2, k);
                    *CD = Clow + fr * (Cup - Clow);
                    return 1;
                }
            }
        } else {
            /* horizontal grid line y = Yn: interpolate between the left and right node */
            real xs = px + t * dx;
            double Xr = floor(xs + 0.5);
            if (fabs(xs - Xr) < RAY_EPS) {
                if (fluid_at(o, (int)Xr, Yn, &idx, &sw)) {
                    *CD = c_at(o, idx, sw, k);
                    return 1;
                }
            } else {
                int X0 = (int)floor(xs);
                real fr = xs - X0;
                if (fluid_at(o, X0, Yn, &idx, &sw) && fluid_at(o, X0 + 1, Yn, &idx2, &sw2)) {
                    real Clef = c_at(o, idx, sw, k), Crig = c_at(o, idx2, sw2, k);
                    *CD = Clef + fr * (Crig - Clef);
                    return 1;
                }
            }
        }
        if (hitV) {
            Xn += sx;
            tv = (Xn - px) / dx;
        }
        if (hitH) {
            Yn += sy;
            th = (Yn - py) / dy;
        }
    }
}

/* C_P for fluid k with local contact angle theta_k (deg) at C_SB node p; Eq.(22) */
static real wet_value(const ora_t* o, int p, int k, real theta_k, real* CD1, real* CD2)
{
    int px = p % o->nx, py = p / o->nx;
    double nx = o->ns[2 * (size_t)p], ny = o->ns[2 * (size_t)p + 1];
    double tx = -ny, ty = nx; /* tangent */
    /* |pi/2 - theta_k|; within 1e-6 deg of 90 both lines run along n_s */
    real phi = fabs(90.0 - theta_k) < PHI_SNAP ? 0.0 : fabs(90.0 - theta_k) * (M_PI / 180.0);
    real cphi = cos(phi), sphi = sin(phi);
    real d1x = cphi * nx + sphi * tx, d1y = cphi * ny + sphi * ty;
    real d2x = cphi * nx - sphi * tx, d2y = cphi * ny - sphi * ty;
    real c1, c2;
    if (!march(o, px, py, d1x, d1y, k, &c1)) c1 = neighbour_mean(o, px, py, k);
    if (!march(o, px, py, d2x, d2y, k, &c2)) c2 = neighbour_mean(o, px, py, k);
    if (CD1) *CD1 = c1;
    if (CD2) *CD2 = c2;
    return theta_k <= 90.0 ? fmax(c1, c2) : fmin(c1, c2);
}

/* Eq.(21) with the previous C_SB values at node p */
static void local_angles(const ora_t* o, int p, real th[2])
{
    size_t n = o->n;
    real Cr = o->Cw[p], Cg = o->Cw[n + p], Cb = o->Cw[2 * n + p];
    real t_rg = o->theta[3 * (size_t)p + 0];
    real t_br = o->theta[3 * (size_t)p + 1];
    real t_gb = o->theta[3 * (size_t)p + 2];
    real t_rb = 180.0 - t_br, t_gr = 180.0 - t_rg; /* theta_lk = pi - theta_kl */
    /* Eq.(21) with 1 - C_r = C_b + C_g (the fractions sum to 1), written as a convex combination
     * so that it is exact when one of the two weights vanishes; both weights below 1e-12 (the
     * 0/0 of a wall node filled by fluid k): the mean of the two angles */
    if (Cb + Cg < 1e-12)
        th[0] = 0.5 * (t_rb + t_rg);
    else
        th[0] = t_rg + Cb / (Cb + Cg) * (t_rb - t_rg);
    if (Cb + Cr < 1e-12)
        th[1] = 0.5 * (t_gb + t_gr);
    else
        th[1] = t_gr + Cb / (Cb + Cr) * (t_gb - t_gr);
}

/* O2-O4 for every C_SB node */
static void wetting(ora_t* o)
{
    size_t n = o->n;
    /* each C_SB node writes only its own values and reads C at fluid nodes */
#pragma omp parallel for num_threads(o->threads) schedule(dynamic, 64) if (o->threads > 1)
    for (int p = 0; p < o->n; p++) {
        if (o->cls[p] != CL_SB) continue;
        real th[2];
        local_angles(o, p, th);
        real cr = wet_value(o, p, 0, th[0], NULL, NULL);
        real cg = wet_value(o, p, 1, th[1], NULL, NULL);
        real s = cr + cg;
        if (s > 1.0) {
            cr /= s;
            cg /= s;
        }
        real cb = fmax(0.0, 1.0 - cr - cg);
        o->C[p] = cr;
        o->C[n + p] = cg;
        o->C[2 * n + p] = cb;
        o->Cw[p] = cr;
        o->Cw[n + p] = cg;
        o->Cw[2 * n + p] = cb;
    }
}

/* ------------------------------------------------------------------------- */
/* set-up: node classes (Section II.B, Fig.1) and solid normals (Eq.19-20)    */
/* ------------------------------------------------------------------------- */
static void classify(ora_t* o)
{
    for (int y = 0; y < o->ny; y++)
        for (int x = 0; x < o->nx; x++) {
            int i = y * o->nx + x, touch = 0;
            for (int a = 1; a < Q; a++) {
                int s = is_solid_at(o, x + EX[a], y + EY[a]);
                if (o->solid[i] ? !s : s) touch = 1;
            }
            if (o->solid[i])
                o->cls[i] = touch ? CL_SB : CL_SI;
            else
                o->cls[i] = touch ? CL_FB : CL_FI;
        }
}

/* eighth-order weight function, Eq.(20) */
static double w8(int c2)
{
    switch (c2) {
        case 1: return 4.0 / 21.0;
        case 2: return 4.0 / 45.0;
        case 4: return 1.0 / 60.0;
        case 5: return 2.0 / 315.0;
        case 8: return 1.0 / 5040.0;
        default: return 0.0;
    }
}

static void normals(ora_t* o)
{
    for (int y = 0; y < o->ny; y++)
        for (int x = 0; x < o->nx; x++) {
            int i = y * o->nx + x;
            o->ns[2 * (size_t)i] = o->ns[2 * (size_t)i + 1] = 0.0;
            if (o->cls[i] != CL_SB) continue;
            double sx = 0.0, sy = 0.0;
            for (int cy = -2; cy <= 2; cy++)
                for (int cx = -2; cx <= 2; cx++) {
                    double w = w8(cx * cx + cy * cy);
                    if (w == 0.0) continue;
                    double s = is_solid_at(o, x + cx, y + cy);
                    sx += w * s * cx;
                    sy += w * s * cy;
                }
            double nrm = sqrt(sx * sx + sy * sy);
            if (nrm < 1e-12) {
                /* symmetric neighbourhood: fall back to the D2Q9 fluid directions */
                sx = sy = 0.0;
                for (int a = 1; a < Q; a++) {
                    double s = is_solid_at(o, x + EX[a], y + EY[a]);
                    sx += WQ[a] * s * EX[a];
                    sy += WQ[a] * s * EY[a];
                }
                nrm = sqrt(sx * sx + sy * sy);
                if (nrm < 1e-12) {
                    sx = 0.0;
                    sy = -1.0;
                    nrm = 1.0;
                }
            }
            /* Eq.(19) points into the solid; the characteristic lines start outward */
            o->ns[2 * (size_t)i] = -sx / nrm;
            o->ns[2 * (size_t)i + 1] = -sy / nrm;
        }
}

/* ------------------------------------------------------------------------- */
/* public API                                                                 */
/* ------------------------------------------------------------------------- */
ora_t* ora_create(int nx, int ny, int per_y, int bc_x, double u_in, double rho_out,
                  const unsigned char* solid, const double* angles_deg, const double* sigma,
                  const double* nu, double beta0)
{
    ora_t* o = (ora_t*)calloc(1, sizeof(ora_t));
    size_t n = (size_t)nx * ny;
    o->nx = nx;
    o->ny = ny;
    o->n = (int)n;
    o->per_y = per_y;
    o->bc_x = bc_x;
    o->u_in = u_in;
    o->rho_out = rho_out;
    o->beta0 = beta0;
    /* sigma = (sigma_01, sigma_02, sigma_12) */
    o->sigma[0][1] = o->sigma[1][0] = sigma[0];
    o->sigma[0][2] = o->sigma[2][0] = sigma[1];
    o->sigma[1][2] = o->sigma[2][1] = sigma[2];
    for (int k = 0; k < NF; k++) {
        o->nu[k] = nu[k];
        o->rho0[k] = 1.0;
    }
    /* X_kl = (sigma_mk^2 + sigma_ml^2 - sigma_kl^2) / (2 sigma_mk sigma_ml), m the third fluid */
    for (int k = 0; k < NF; k++)
        for (int l = 0; l < NF; l++) {
            if (k == l) continue;
            int m = 3 - k - l;
            double X = (o->sigma[m][k] * o->sigma[m][k] + o->sigma[m][l] * o->sigma[m][l] -
                        o->sigma[k][l] * o->sigma[k][l]) /
                       (2.0 * o->sigma[m][k] * o->sigma[m][l]);
            o->gX[k][l] = ora_gfun(X);
        }
    invert9(MMAT, o->Minv);
    for (int a = 0; a < Q; a++)
        for (int b = 0; b < Q; b++)
            if (EX[b] == -EX[a] && EY[b] == -EY[a]) o->opp[a] = b;
    o->solid = (unsigned char*)malloc(n);
    o->cls = (unsigned char*)malloc(n);
    memcpy(o->solid, solid, n);
    o->theta = (real*)malloc(3 * n * sizeof(real));
    for (size_t j = 0; j < 3 * n; j++) o->theta[j] = angles_deg[j];
    o->ns = (double*)calloc(2 * n, sizeof(double));
    o->f = (real*)calloc((size_t)NF * Q * n, sizeof(real));
    o->fnew = (real*)calloc((size_t)NF * Q * n, sizeof(real));
    o->rho = (real*)calloc(NF * n, sizeof(real));
    o->C = (real*)calloc(NF * n, sizeof(real));
    o->Cw = (real*)calloc(NF * n, sizeof(real));
    o->T = (real*)calloc(3 * n, sizeof(real));
    o->Fs = (real*)calloc(2 * n, sizeof(real));
    o->u = (real*)calloc(2 * n, sizeof(real));
    o->threads = 1;
    classify(o);
    normals(o);
    return o;
}

void ora_destroy(ora_t* o)
{
    if (!o) return;
    free(o->solid); free(o->cls); free(o->theta); free(o->ns); free(o->f); free(o->fnew);
    free(o->rho); free(o->C); free(o->Cw); free(o->T); free(o->Fs); free(o->u);
    free(o);
}

/* O1 */
static void densities(ora_t* o)
{
    size_t n = o->n;
#pragma omp parallel for num_threads(o->threads) schedule(static) if (o->threads > 1)
    for (size_t i = 0; i < n; i++) {
        if (o->solid[i]) continue;
        real r = 0.0;
        for (int k = 0; k < NF; k++) {
            real s = 0.0;
            for (int a = 0; a < Q; a++) s += o->f[((size_t)k * Q + a) * n + i];
            o->rho[k * n + i] = s;
            r += s;
        }
        for (int k = 0; k < NF; k++) o->C[k * n + i] = o->rho[k * n + i] / r;
    }
}

static void zou_he(ora_t* o, real* F);

/* rest equilibrium f_ak = w_a rho_k, taken as a post-streaming state (so the open-boundary
 * populations are completed by Zou-He as after any streaming step); lagged C_SB values =
 * w-weighted fluid-neighbour mean */
void ora_set_fields(ora_t* o, const double* rho_in)
{
    size_t n = o->n;
    memset(o->f, 0, sizeof(real) * NF * Q * n);
    memset(o->u, 0, sizeof(real) * 2 * n);
    for (size_t i = 0; i < n; i++) {
        if (o->solid[i]) continue;
        for (int k = 0; k < NF; k++)
            for (int a = 0; a < Q; a++) o->f[((size_t)k * Q + a) * n + i] = WQ[a] * rho_in[k * n + i];
    }
    if (o->bc_x == BC_ZOUHE) zou_he(o, o->f);
    densities(o);
    for (int p = 0; p < o->n; p++) {
        if (o->cls[p] != CL_SB) continue;
        for (int k = 0; k < NF; k++) o->Cw[k * n + p] = neighbour_mean(o, p % o->nx, p / o->nx, k);
    }
    for (int p = 0; p < o->n; p++)
        if (o->cls[p] == CL_SB)
            for (int k = 0; k < NF; k++) o->C[k * n + p] = o->Cw[k * n + p];
    o->steps = 0;
}

/* O10 tail: Zou-He non-equilibrium bounce-back on the open columns of the post-streaming
 * populations F */
static void zou_he(ora_t* o, real* F)
{
    size_t n = o->n;
    for (int y = 0; y < o->ny; y++) {
        /* velocity inlet, x = 0: unknown a = 1, 5, 8 */
        size_t i = (size_t)y * o->nx;
        real f[Q];
        for (int a = 0; a < Q; a++) f[a] = F[(0 * Q + a) * n + i] + F[(1 * Q + a) * n + i] + F[(2 * Q + a) * n + i];
        real U = o->u_in;
        real rho = (f[0] + f[2] + f[4] + 2.0 * (f[3] + f[6] + f[7])) / (1.0 - U);
        real g1 = f[3] + 2.0 / 3.0 * rho * U;
        real g5 = f[7] - 0.5 * (f[2] - f[4]) + 1.0 / 6.0 * rho * U;
        real g8 = f[6] + 0.5 * (f[2] - f[4]) + 1.0 / 6.0 * rho * U;
        int un[3] = {1, 5, 8};
        real gv[3] = {g1, g5, g8};
        for (int j = 0; j < 3; j++) {
            F[(0 * Q + un[j]) * n + i] = 0.0;
            F[(1 * Q + un[j]) * n + i] = 0.0;
            F[(2 * Q + un[j]) * n + i] = gv[j];
        }
        /* pressure outlet, x = nx - 1: unknown a = 3, 6, 7 */
        i = (size_t)y * o->nx + (o->nx - 1);
        for (int a = 0; a < Q; a++) f[a] = F[(0 * Q + a) * n + i] + F[(1 * Q + a) * n + i] + F[(2 * Q + a) * n + i];
        double ro = o->rho_out;
        real ux = -1.0 + (f[0] + f[2] + f[4] + 2.0 * (f[1] + f[5] + f[8])) / ro;
        real h3 = f[1] - 2.0 / 3.0 * ro * ux;
        real h7 = f[5] + 0.5 * (f[2] - f[4]) - 1.0 / 6.0 * ro * ux;
        real h6 = f[8] - 0.5 * (f[2] - f[4]) - 1.0 / 6.0 * ro * ux;
        int kn[6] = {0, 1, 2, 4, 5, 8};
        real part[NF], tot = 0.0;
        for (int k = 0; k < NF; k++) {
            part[k] = 0.0;
            for (int j = 0; j < 6; j++) part[k] += F[((size_t)k * Q + kn[j]) * n + i];
            tot += part[k];
        }
        int uo[3] = {3, 6, 7};
        real hv[3] = {h3, h6, h7};
        for (int j = 0; j < 3; j++)
            for (int k = 0; k < NF; k++) F[((size_t)k * Q + uo[j]) * n + i] = hv[j] * part[k] / tot;
    }
}

/* Eq.(14): segregation parameters beta_kl of a node with densities rho_k (beta_kk = 0); the
 * recolouring of the step and the ora_beta accessor both take them from here */
static void segregation(const ora_t* o, const real rk[NF], real beta[NF][NF])
{
    real rho = rk[0] + rk[1] + rk[2];
    real trip = fmin(35.0 * rk[0] * rk[1] * rk[2] / (rho * rho * rho), 1.0);
    for (int k = 0; k < NF; k++)
        for (int l = 0; l < NF; l++) beta[k][l] = (k == l) ? 0.0 : o->beta0 + o->beta0 * trip * o->gX[k][l];
}

static void one_step(ora_t* o)
{
    size_t n = o->n;
    /* O1 */
    densities(o);
    /* O2-O4 */
    wetting(o);
    /* O5-O6: stress tensor at C_F and C_SB nodes, then its divergence at C_F */
#pragma omp parallel for num_threads(o->threads) schedule(static) if (o->threads > 1)
    for (int y = 0; y < o->ny; y++)
        for (int x = 0; x < o->nx; x++) {
            int i = y * o->nx + x;
            if (o->cls[i] == CL_SI) continue;
            real T[3];
            tensor_at(o, x, y, T);
            for (int c = 0; c < 3; c++) o->T[c * n + i] = T[c];
        }
#pragma omp parallel for num_threads(o->threads) schedule(static) if (o->threads > 1)
    for (int y = 0; y < o->ny; y++)
        for (int x = 0; x < o->nx; x++) {
            int i = y * o->nx + x;
            if (o->solid[i]) continue;
            real Fx = 0.0, Fy = 0.0;
            for (int a = 1; a < Q; a++) {
                int idx, sw;
                int loc = locate(o, x + EX[a], y + EY[a], &idx, &sw);
                real T[3];
                if (loc == LOC_GHOST) {
                    tensor_at(o, x + EX[a], y + EY[a], T);
                } else {
                    for (int c = 0; c < 3; c++) T[c] = o->T[c * n + idx];
                }
                /* F_i = sum_j d_j T_ij, derivatives by Eq.(12) */
                Fx += WQ[a] * (T[0] * EX[a] + T[1] * EY[a]) / CS2;
                Fy += WQ[a] * (T[1] * EX[a] + T[2] * EY[a]) / CS2;
            }
            o->Fs[i] = Fx;
            o->Fs[n + i] = Fy;
        }
    /* O7-O9 per fluid node: collision, then recolouring; results into fnew in place of
     * the post-collision populations of the node (streamed below) */
    real* fdd = (real*)malloc(sizeof(real) * NF * Q * n);
#pragma omp parallel for num_threads(o->threads) schedule(static) if (o->threads > 1)
    for (int y = 0; y < o->ny; y++)
        for (int x = 0; x < o->nx; x++) {
            int i = y * o->nx + x;
            if (o->solid[i]) continue;
            real f[Q], rk[NF], rho = 0.0;
            for (int a = 0; a < Q; a++) {
                f[a] = 0.0;
                for (int k = 0; k < NF; k++) f[a] += o->f[((size_t)k * Q + a) * n + i];
            }
            for (int k = 0; k < NF; k++) {
                rk[k] = o->rho[k * n + i];
                rho += rk[k];
            }
            real Fs[2] = {o->Fs[i], o->Fs[n + i]}, u[2], fdag[Q];
            real tau = mixture_tau(o, rk);
            collide_node(o->Minv, f, Fs, tau, fdag, u);
            o->u[i] = u[0];
            o->u[n + i] = u[1];
            /* Eq.(13)-(15) */
            real g[NF][2], c[NF];
            grad_at(o, x, y, g);
            for (int k = 0; k < NF; k++) c[k] = o->C[k * n + i];
            real nkl[NF][NF][2];
            for (int k = 0; k < NF; k++)
                for (int l = 0; l < NF; l++) {
                    nkl[k][l][0] = nkl[k][l][1] = 0.0;
                    if (k == l) continue;
                    real Gx = c[l] * g[k][0] - c[k] * g[l][0];
                    real Gy = c[l] * g[k][1] - c[k] * g[l][1];
                    real G2 = Gx * Gx + Gy * Gy;
                    if (G2 <= G2_EPS) continue;
                    real Gn = sqrt(G2);
                    nkl[k][l][0] = Gx / Gn;
                    nkl[k][l][1] = Gy / Gn;
                }
            real beta_kl[NF][NF];
            segregation(o, rk, beta_kl);
            for (int k = 0; k < NF; k++)
                for (int a = 0; a < Q; a++) {
                    real v = rk[k] / rho * fdag[a];
                    for (int l = 0; l < NF; l++) {
                        if (l == k) continue;
                        real beta = beta_kl[k][l];
                        real ne = nkl[k][l][0] * EX[a] + nkl[k][l][1] * EY[a];
                        v += beta * WQ[a] * rk[k] * rk[l] / rho * ne;
                    }
                    fdd[((size_t)k * Q + a) * n + i] = v;
                }
        }
    /* O10: streaming, Eq.(16) */
    memset(o->fnew, 0, sizeof(real) * NF * Q * n);
#pragma omp parallel for num_threads(o->threads) schedule(static) if (o->threads > 1)
    for (int y = 0; y < o->ny; y++)
        for (int x = 0; x < o->nx; x++) {
            int i = y * o->nx + x;
            if (o->solid[i]) continue;
            for (int a = 0; a < Q; a++) {
                int idx, sw;
                int loc = locate(o, x + EX[a], y + EY[a], &idx, &sw);
                for (int k = 0; k < NF; k++) {
                    real v = fdd[((size_t)k * Q + a) * n + i];
                    if (loc == LOC_SOLID || (loc == LOC_IN && o->solid[idx])) {
                        /* halfway bounce-back */
                        o->fnew[((size_t)k * Q + o->opp[a]) * n + i] = v;
                    } else if (loc == LOC_IN) {
                        int kk = sw ? swapk(k) : k;
                        o->fnew[((size_t)kk * Q + a) * n + idx] = v;
                    } /* LOC_GHOST: leaves through the open boundary */
                }
            }
        }
    if (o->bc_x == BC_ZOUHE) zou_he(o, o->fnew);
    free(fdd);
    real* t = o->f;
    o->f = o->fnew;
    o->fnew = t;
    o->steps++;
}

/* OpenMP threads of the per-node loops (results do not depend on it); n < 1 means 1 */
void ora_set_threads(ora_t* o, int n) { o->threads = n < 1 ? 1 : n; }

void ora_step(ora_t* o, int nsteps)
{
    for (int s = 0; s < nsteps; s++) one_step(o);
}

/* rho_k of the current (post-streaming) state; u of the last collision */
void ora_fields(ora_t* o, double* rho_out, double* u_out)
{
    size_t n = o->n;
    densities(o);
    for (size_t i = 0; i < n; i++)
        for (int k = 0; k < NF; k++) rho_out[k * n + i] = o->solid[i] ? 0.0 : VAL(o->rho[k * n + i]);
    if (u_out)
        for (size_t i = 0; i < 2 * n; i++) u_out[i] = VAL(o->u[i]);
}

/* masses, x- and y-moments of fluid 0, max|u|, min rho, non-finite count */
void ora_diag(ora_t* o, double out[8])
{
    size_t n = o->n;
    densities(o);
    for (int j = 0; j < 8; j++) out[j] = 0.0;
    out[6] = INFINITY;
    for (size_t i = 0; i < n; i++) {
        if (o->solid[i]) continue;
        double r = 0.0;
        for (int k = 0; k < NF; k++) {
            double v = VAL(o->rho[k * n + i]);
            out[k] += v;
            r += v;
            if (!isfinite(v)) out[7] += 1.0;
        }
        out[3] += (double)(i % o->nx) * VAL(o->rho[i]);
        out[4] += (double)(i / o->nx) * VAL(o->rho[i]);
        double ux = VAL(o->u[i]), uy = VAL(o->u[n + i]);
        double um = sqrt(ux * ux + uy * uy);
        if (um > out[5]) out[5] = um;
        if (r < out[6]) out[6] = r;
    }
}

/* 0 if the configuration satisfies the oracle's preconditions, else a code:
 * 1 a fluid node touches an out-of-domain wall (non-periodic side without a solid layer),
 * 2 open x boundary without periodic y or with solid within 4 columns of it,
 * 3 modified periodic boundary with sigma_01 != sigma_12,
 * 4 a non-positive viscosity */
int ora_check(ora_t* o)
{
    for (int y = 0; y < o->ny; y++)
        for (int x = 0; x < o->nx; x++) {
            if (o->solid[y * o->nx + x]) continue;
            for (int a = 1; a < Q; a++) {
                int idx, sw;
                if (locate(o, x + EX[a], y + EY[a], &idx, &sw) == LOC_SOLID) return 1;
            }
        }
    if (o->bc_x == BC_ZOUHE) {
        if (!o->per_y) return 2;
        for (int y = 0; y < o->ny; y++)
            for (int j = 0; j < 4; j++)
                if (o->solid[y * o->nx + j] || o->solid[y * o->nx + o->nx - 1 - j]) return 2;
    }
    if (o->bc_x == BC_MODPER && o->sigma[0][1] != o->sigma[1][2]) return 3;
    for (int k = 0; k < NF; k++)
        if (!(o->nu[k] > 0.0)) return 4;
    return 0;
}

#ifndef ORA_TAPE
/* ---- accessors used by the pinning tests ---- */
void ora_get_f(ora_t* o, double* out) { memcpy(out, o->f, sizeof(double) * NF * Q * o->n); }
void ora_set_f(ora_t* o, const double* in) { memcpy(o->f, in, sizeof(double) * NF * Q * o->n); }
void ora_get_classes(ora_t* o, unsigned char* out) { memcpy(out, o->cls, o->n); }
void ora_get_normals(ora_t* o, double* out) { memcpy(out, o->ns, sizeof(double) * 2 * o->n); }
void ora_get_wallC(ora_t* o, double* out) { memcpy(out, o->Cw, sizeof(double) * NF * o->n); }
void ora_get_force(ora_t* o, double* out) { memcpy(out, o->Fs, sizeof(double) * 2 * o->n); }

void ora_lattice(int* ex, int* ey, double* w, double* M, double* Minv)
{
    double R[Q][Q];
    invert9(MMAT, R);
    for (int a = 0; a < Q; a++) {
        ex[a] = EX[a];
        ey[a] = EY[a];
        w[a] = WQ[a];
        for (int b = 0; b < Q; b++) {
            M[a * Q + b] = MMAT[a][b];
            Minv[a * Q + b] = R[a][b];
        }
    }
}

/* one collision (Eq.1-9, 11) on a 9-vector of totals, for unit pins */
void ora_collide(const double* f, const double* Fs, double tau, double* fdag, double* u)
{
    double R[Q][Q];
    invert9(MMAT, R);
    collide_node(R, f, Fs, tau, fdag, u);
}

/* Eq.(12) applied to a periodic scalar field psi[ny][nx]; out[2][ny][nx] */
void ora_gradient_periodic(int nx, int ny, const double* psi, double* out)
{
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            double v[Q], g[2];
            for (int a = 0; a < Q; a++) v[a] = psi[((y + EY[a] + ny) % ny) * nx + (x + EX[a] + nx) % nx];
            eq12(v, g);
            out[y * nx + x] = g[0];
            out[nx * ny + y * nx + x] = g[1];
        }
}

/* beta_kl table of Eq.(14) for given rho_k; out[3][3] */
void ora_beta(ora_t* o, const double* rk, double* out)
{
    double b[NF][NF];
    segregation(o, rk, b);
    for (int k = 0; k < NF; k++)
        for (int l = 0; l < NF; l++) out[k * NF + l] = b[k][l];
}

/* Characteristic lines at one C_SB node against a caller-supplied C field (3n, C_F values
 * used); out = {C_D1, C_D2, C_P} */
void ora_wet_probe(ora_t* o, int p, int k, double theta_k, const double* Cfield, double* out)
{
    memcpy(o->C, Cfield, sizeof(double) * NF * o->n);
    out[2] = wet_value(o, p, k, theta_k, &out[0], &out[1]);
}

/* Eq.(21) at node p with caller-supplied lagged C (3 values) */
void ora_local_angles(ora_t* o, int p, const double* Cp, double* th)
{
    size_t n = o->n;
    for (int k = 0; k < NF; k++) o->Cw[k * n + p] = Cp[k];
    local_angles(o, p, th);
}

/* Eq.(12) gradients of C_0..C_2 at node (x, y), the step's own grad_at, against a
 * caller-supplied C field (3n values: fluid nodes and C_SB wall values); g = 6 values
 * (dC_k/dx, dC_k/dy for k = 0, 1, 2) */
void ora_gradient_at(ora_t* o, const double* Cfield, int x, int y, double* g)
{
    double gg[NF][2];
    memcpy(o->C, Cfield, sizeof(double) * NF * o->n);
    grad_at(o, x, y, gg);
    for (int k = 0; k < NF; k++) {
        g[2 * k] = gg[k][0];
        g[2 * k + 1] = gg[k][1];
    }
}
#endif /* ORA_TAPE */
