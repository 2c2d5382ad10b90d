// lbm3_oracle_tape.cpp -- reverse-mode reference tape of the FP64 oracle: the gradient of the
// fluid-0 x-centroid after n steps with respect to the wall angles of every C_SB node and the
// Zou-He inflow velocity, obtained by running the oracle's own step (lbm3_oracle.c, compiled
// here a second time with a recording scalar type) and sweeping each step's record backwards.
//
// TEST INFRASTRUCTURE ONLY, like the oracle itself: only tests/ load it.  It shares nothing with
// the CUDA sources; the gradient it returns is that of exactly the oracle's operations, in the
// oracle's order (every branch -- Eq.22's max/min, the ray-march decisions, the A_kl and beta_kl
// clamps -- is taken as the forward run takes it and differentiated on that branch).
//
// Scheme: the forward run stores the state (populations f and lagged wall values Cw) before
// every step.  The objective J = sum_x x rho_0 / sum_x rho_0 over the fluid nodes of the final
// state is recorded and swept to give dJ/d(final state).  Then, from the last step to the first,
// the step is recorded again from its stored state with fresh input variables (state, wall
// angles, inflow velocity), its outputs are seeded with the adjoint of the next state, and the
// backward sweep gives the adjoint of this step's state and adds this step's share of dJ/dtheta
// and dJ/dU.  Last, the initial state itself (rest populations completed by Zou-He, which reads
// the inflow velocity) is recorded and swept for its share of dJ/dU.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace tape {

// one recorded operation: value = op(parent a, parent b); da, db = partial derivatives.  Node 0
// stands for every constant (no parents); its adjoint is discarded.
struct Node {
    int a, b;
    double da, db;
};
static std::vector<Node> nodes(1, Node{0, 0, 0.0, 0.0});

inline int rec(int a, double da, int b, double db)
{
    if (a == 0 && b == 0) return 0;  // a function of constants is a constant
    nodes.push_back(Node{a, b, da, db});
    return (int)nodes.size() - 1;
}

// a recorded scalar: value and node index (0 = constant).  Trivially copyable, and all-zero bytes
// are the constant 0, so arrays of it may be calloc'ed, memset and memcpy'ed like doubles.
struct var {
    double v;
    int i;
    var() = default;
    var(double x) : v(x), i(0) {}
    var(double x, int idx) : v(x), i(idx) {}
    var& operator+=(const var& o) { return *this = var(v + o.v, rec(i, 1.0, o.i, 1.0)); }
    var& operator-=(const var& o) { return *this = var(v - o.v, rec(i, 1.0, o.i, -1.0)); }
    var& operator*=(const var& o) { return *this = var(v * o.v, rec(i, o.v, o.i, v)); }
    var& operator/=(const var& o) { return *this = var(v / o.v, rec(i, 1.0 / o.v, o.i, -v / (o.v * o.v))); }
};

inline var input(double x)
{
    nodes.push_back(Node{0, 0, 0.0, 0.0});
    return var(x, (int)nodes.size() - 1);
}

inline var operator+(const var& a, const var& b) { return var(a.v + b.v, rec(a.i, 1.0, b.i, 1.0)); }
inline var operator-(const var& a, const var& b) { return var(a.v - b.v, rec(a.i, 1.0, b.i, -1.0)); }
inline var operator*(const var& a, const var& b) { return var(a.v * b.v, rec(a.i, b.v, b.i, a.v)); }
inline var operator/(const var& a, const var& b)
{
    return var(a.v / b.v, rec(a.i, 1.0 / b.v, b.i, -a.v / (b.v * b.v)));
}
inline var operator+(const var& a, double b) { return var(a.v + b, rec(a.i, 1.0, 0, 0.0)); }
inline var operator+(double a, const var& b) { return var(a + b.v, rec(0, 0.0, b.i, 1.0)); }
inline var operator-(const var& a, double b) { return var(a.v - b, rec(a.i, 1.0, 0, 0.0)); }
inline var operator-(double a, const var& b) { return var(a - b.v, rec(0, 0.0, b.i, -1.0)); }
inline var operator*(const var& a, double b) { return var(a.v * b, rec(a.i, b, 0, 0.0)); }
inline var operator*(double a, const var& b) { return var(a * b.v, rec(0, 0.0, b.i, a)); }
inline var operator/(const var& a, double b) { return var(a.v / b, rec(a.i, 1.0 / b, 0, 0.0)); }
inline var operator/(double a, const var& b) { return var(a / b.v, rec(0, 0.0, b.i, -a / (b.v * b.v))); }
inline var operator-(const var& a) { return var(-a.v, rec(a.i, -1.0, 0, 0.0)); }

inline bool operator<(const var& a, const var& b) { return a.v < b.v; }
inline bool operator<=(const var& a, const var& b) { return a.v <= b.v; }
inline bool operator>(const var& a, const var& b) { return a.v > b.v; }
inline bool operator>=(const var& a, const var& b) { return a.v >= b.v; }
inline bool operator<(const var& a, double b) { return a.v < b; }
inline bool operator<=(const var& a, double b) { return a.v <= b; }
inline bool operator>(const var& a, double b) { return a.v > b; }
inline bool operator>=(const var& a, double b) { return a.v >= b; }
inline bool operator<(double a, const var& b) { return a < b.v; }
inline bool operator>(double a, const var& b) { return a > b.v; }

inline var sqrt(const var& a)
{
    const double s = std::sqrt(a.v);
    return var(s, rec(a.i, 0.5 / s, 0, 0.0));
}
inline var sin(const var& a) { return var(std::sin(a.v), rec(a.i, std::cos(a.v), 0, 0.0)); }
inline var cos(const var& a) { return var(std::cos(a.v), rec(a.i, -std::sin(a.v), 0, 0.0)); }
inline var fabs(const var& a) { return a.v < 0.0 ? -a : a; }
// the selected operand carries the derivative (the oracle's branch)
inline var fmin(const var& a, const var& b) { return b.v < a.v ? b : a; }
inline var fmax(const var& a, const var& b) { return b.v > a.v ? b : a; }
inline var fmin(const var& a, double b) { return b < a.v ? var(b) : a; }
inline var fmax(double a, const var& b) { return b.v > a ? b : var(a); }
// piecewise constant: no derivative
inline double floor(const var& a) { return std::floor(a.v); }

}  // namespace tape

using tape::var;
using std::acos;
using std::floor;
using std::sqrt;

#define ORA_TAPE 1
typedef tape::var real;
#define VAL(x) ((x).v)
using tape::cos;
using tape::fabs;
using tape::fmax;
using tape::fmin;
using tape::sin;
using tape::sqrt;
using tape::floor;

#include "lbm3_oracle.c"

namespace {

// backward sweep of the current record from the given seeds
std::vector<double> sweep(const std::vector<std::pair<int, double>>& seeds)
{
    std::vector<double> adj(tape::nodes.size(), 0.0);
    for (const auto& s : seeds) adj[s.first] += s.second;
    for (size_t j = tape::nodes.size() - 1; j > 0; j--) {
        const double g = adj[j];
        if (g == 0.0) continue;
        const tape::Node& nd = tape::nodes[j];
        adj[nd.a] += nd.da * g;
        adj[nd.b] += nd.db * g;
    }
    return adj;
}

void reset() { tape::nodes.resize(1); }

}  // namespace

extern "C" {

// Gradient of J = sum_x x rho_0 / sum_x rho_0 (fluid nodes, final post-streaming state) after
// nsteps oracle steps from the rest state rho_init (host [3][ny][nx]), with respect to the wall
// angles (out dJ_dangles [ny][nx][3], nonzero at C_SB nodes only) and the inflow velocity.
// Arguments as ora_create.  Returns 0, or -1 if the configuration fails the oracle's checks.
int tape_centroid_gradient(int nx, int ny, int per_y, int bc_x, double u_in, double rho_out,
                           const unsigned char* solid, const double* angles_deg, const double* sigma,
                           const double* nu, double beta0, const double* rho_init, int nsteps,
                           double* J_out, double* dJ_dangles, double* dJ_du)
{
    reset();
    ora_t* o = ora_create(nx, ny, per_y, bc_x, u_in, rho_out, solid, angles_deg, sigma, nu, beta0);
    if (ora_check(o) != 0) {
        ora_destroy(o);
        return -1;
    }
    const size_t n = (size_t)nx * ny, nf = (size_t)NF * Q * n, nc = (size_t)NF * n;
    // forward run: values only, the record cleared after every step
    ora_set_fields(o, rho_init);
    std::vector<double> S((size_t)(nsteps + 1) * (nf + nc));
    auto save = [&](int t) {
        double* s = &S[(size_t)t * (nf + nc)];
        for (size_t j = 0; j < nf; j++) s[j] = o->f[j].v;
        for (size_t j = 0; j < nc; j++) s[nf + j] = o->Cw[j].v;
    };
    auto load = [&](int t, std::vector<var>* fin, std::vector<var>* cin) {
        const double* s = &S[(size_t)t * (nf + nc)];
        for (size_t j = 0; j < nf; j++) o->f[j] = fin ? ((*fin)[j] = tape::input(s[j])) : var(s[j]);
        for (size_t j = 0; j < nc; j++) o->Cw[j] = cin ? ((*cin)[j] = tape::input(s[nf + j])) : var(s[nf + j]);
    };
    for (size_t j = 0; j < 3 * n; j++) o->theta[j] = var(angles_deg[j]);
    o->u_in = var(u_in);
    save(0);
    reset();
    for (int t = 0; t < nsteps; t++) {
        load(t, nullptr, nullptr);
        one_step(o);
        save(t + 1);
        reset();
    }
    // J of the final state and its adjoint
    std::vector<var> fin(nf), cin(nc);
    load(nsteps, &fin, nullptr);
    densities(o);
    var m0 = 0.0, mx = 0.0;
    for (size_t i = 0; i < n; i++) {
        if (o->solid[i]) continue;
        m0 += o->rho[i];
        mx += (double)(i % (size_t)nx) * o->rho[i];
    }
    const var J = mx / m0;
    *J_out = J.v;
    std::vector<double> adj = sweep({{J.i, 1.0}});
    std::vector<double> lf(nf), lc(nc, 0.0);
    for (size_t j = 0; j < nf; j++) lf[j] = adj[fin[j].i];
    reset();
    // reverse over the steps
    std::vector<double> dang(3 * n, 0.0);
    double du = 0.0;
    std::vector<var> th(3 * n);
    for (int t = nsteps - 1; t >= 0; t--) {
        load(t, &fin, &cin);
        for (size_t j = 0; j < 3 * n; j++) o->theta[j] = th[j] = tape::input(angles_deg[j]);
        const var U = tape::input(u_in);
        o->u_in = U;
        one_step(o);
        std::vector<std::pair<int, double>> seeds;
        seeds.reserve(nf + nc);
        for (size_t j = 0; j < nf; j++)
            if (lf[j] != 0.0) seeds.push_back({o->f[j].i, lf[j]});
        for (size_t j = 0; j < nc; j++)
            if (lc[j] != 0.0) seeds.push_back({o->Cw[j].i, lc[j]});
        adj = sweep(seeds);
        for (size_t j = 0; j < nf; j++) lf[j] = adj[fin[j].i];
        for (size_t j = 0; j < nc; j++) lc[j] = adj[cin[j].i];
        for (size_t j = 0; j < 3 * n; j++) dang[j] += adj[th[j].i];
        du += adj[U.i];
        reset();
    }
    // the initial state: rest populations of rho_init completed by Zou-He with the inflow U, and
    // the lagged wall values of its fluid neighbours
    {
        const var U = tape::input(u_in);
        o->u_in = U;
        ora_set_fields(o, rho_init);
        std::vector<std::pair<int, double>> seeds;
        for (size_t j = 0; j < nf; j++)
            if (lf[j] != 0.0) seeds.push_back({o->f[j].i, lf[j]});
        for (size_t j = 0; j < nc; j++)
            if (lc[j] != 0.0) seeds.push_back({o->Cw[j].i, lc[j]});
        adj = sweep(seeds);
        du += adj[U.i];
        reset();
    }
    for (size_t j = 0; j < 3 * n; j++) dJ_dangles[j] = dang[j];
    *dJ_du = bc_x == BC_ZOUHE ? du : 0.0;
    ora_destroy(o);
    return 0;
}

}  // extern "C"
