// lbm3_common.cuh -- lattice constants, parameters and device helpers shared by the
// kernels of the three-phase colour-gradient step (arXiv:2102.04709, Section II).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbm3k {

constexpr int kQ = 9;   // D2Q9
constexpr int kNF = 3;  // fluids r, g, b -> 0, 1, 2

// node classes of Section II.B (Fig.1); bit 1 set = solid
enum : uint8_t { kFI = 0, kFB = 1, kSB = 2, kSI = 3 };
// x boundary kinds
enum : int { kPeriodic = 0, kModPer = 1, kZouHe = 2, kWalls = 3 };
// population storage
enum : int { kStoreF32 = 0, kStoreF16 = 1, kStoreBF16 = 2 };

// D2Q9 velocities e_0..e_8 = (0,0), (1,0), (0,1), (-1,0), (0,-1), (1,1), (-1,1), (-1,-1), (1,-1)
__host__ __device__ constexpr int ex(int a)
{
    return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey(int a)
{
    return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}
// weights 4/9, 1/9 (axes), 1/36 (diagonals)
__host__ __device__ constexpr float wq(int a)
{
    return a == 0 ? 4.0f / 9.0f : (a < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
// opposite direction
__host__ __device__ constexpr int opp(int a)
{
    return a == 0 ? 0 : (a < 5 ? ((a + 1) % 4) + 1 : ((a - 3) % 4) + 5);
}
// label of fluid k after crossing the modified periodic seam an odd number of times
__host__ __device__ constexpr int relabel(int k, bool swapped) { return (swapped && k != 1) ? 2 - k : k; }

struct Params {
    int nx, ny;
    long long N;          // nx * ny
    int per_y, bc_x;
    float u_in, rho_out;
    float sig01, sig02, sig12;
    float inv_nu0, inv_nu1, inv_nu2;
    float beta0;
    float g01, g02, g12;  // g(X_kl) of Eq.(15), constant per pair
    // element offsets of the 27 population planes (k * 9 + a) * N, and of the pull sources
    // (k * 9 + a) * N - e_ax - e_ay * nx, for the step kernel's interior tiles
    int off_plane[27];
    int off_pull[27];
    // reduced storage: element offsets k * N - e_ax - e_ay * nx of the pull sources in the rho
    // planes
    int off_pull16[27];
    // reduced storage: element offsets (8 k + a - 1) * N - e_ax - e_ay * nx of the pull sources in
    // the 16-bit offset planes (a >= 1; entry a = 0 unused)
    int off_pull16o[27];
    // device word of error bits set by kernels (bit 0: a bulk tensor copy did not complete)
    int* err;
    // polls of an mbarrier before a block gives up waiting for its tile's bulk copies (the wait
    // that then drains the copies in flight always uses the full limit kWaitLimit)
    int wait_polls;
};

// One population buffer.  FP32 storage: f[27][N], plane k*9+a, the post-collision populations
// f''_ak.  Reduced storage (FP16 / BF16 offsets): rho[3][N] = sum_a f''_ak in FP32 and
// off[3][8][N] = 24 planes of 16-bit words, plane 8k + a - 1 holding the offsets
// f''_ak - w_a rho_k (a = 1..8); the rest population is w_0 rho_k - sum of the offsets, so the
// stored mass of every fluid is exact whatever the 16-bit rounding.  Planes (rather than one
// 16-byte record per node) keep the 16-bit reads of a warp contiguous, in global and in shared
// memory.
struct Pop {
    float* f;
    float* rho;
    unsigned short* off;
};

template <int STORE>
__device__ __forceinline__ float dec16(unsigned short u)
{
    if constexpr (STORE == kStoreF16)
        return __half2float(__ushort_as_half(u));
    else
        return __uint_as_float((unsigned)u << 16);
}

template <int STORE>
__device__ __forceinline__ unsigned short enc16(float v)
{
    if constexpr (STORE == kStoreF16)
        return __half_as_ushort(__float2half_rn(v));
    else
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// sum of the 8 decoded offsets d[1..8] of one node and fluid, in the one order every kernel uses
// for the rest population w_0 rho_k - sum
__device__ __forceinline__ float sum_offsets(const float d[kQ])
{
    return ((d[1] + d[3]) + (d[2] + d[4])) + ((d[5] + d[7]) + (d[6] + d[8]));
}

__host__ __device__ inline int floordiv_i(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Where an unwrapped lattice position lives.  kind: 0 inside, 1 solid outside a wall side,
// 2 ghost beyond an open x side (idx = nearest boundary-column node).  par: the position lies
// an odd number of modified-periodic seams away from the home domain.
struct Loc {
    int idx;
    int kind;
    bool par;
};

__device__ __forceinline__ Loc locate(const Params& P, int X, int Y)
{
    Loc L;
    L.par = false;
    L.kind = 0;
    L.idx = 0;
    if (Y < 0 || Y >= P.ny) {
        if (!P.per_y) {
            L.kind = 1;
            return L;
        }
        Y -= floordiv_i(Y, P.ny) * P.ny;
    }
    if (X < 0 || X >= P.nx) {
        if (P.bc_x == kPeriodic || P.bc_x == kModPer) {
            int q = floordiv_i(X, P.nx);
            X -= q * P.nx;
            L.par = (P.bc_x == kModPer) && (q & 1);
        } else if (P.bc_x == kWalls) {
            L.kind = 1;
            return L;
        } else {
            X = X < 0 ? 0 : P.nx - 1;
            L.kind = 2;
        }
    }
    L.idx = Y * P.nx + X;
    return L;
}

__device__ __forceinline__ bool parity_x(const Params& P, int X)
{
    return P.bc_x == kModPer && (floordiv_i(X, P.nx) & 1);
}

// Zou-He completion of the populations p[k*9+a] of a node in an open column
// (inlet: x = 0, unknown a = 1, 5, 8; outlet: x = nx-1, unknown a = 3, 6, 7).
__device__ __forceinline__ void zou_he(const Params& P, float p[27], bool inlet)
{
    float f[kQ];
#pragma unroll
    for (int a = 0; a < kQ; a++) f[a] = p[a] + p[9 + a] + p[18 + a];
    if (inlet) {
        const float U = P.u_in;
        const float rho = (f[0] + f[2] + f[4] + 2.0f * (f[3] + f[6] + f[7])) / (1.0f - U);
        const float half = 0.5f * (f[2] - f[4]);
        const float g1 = f[3] + (2.0f / 3.0f) * rho * U;
        const float g5 = f[7] - half + (1.0f / 6.0f) * rho * U;
        const float g8 = f[6] + half + (1.0f / 6.0f) * rho * U;
        // the inlet reservoir holds the carrier fluid 2
        p[1] = p[5] = p[8] = 0.0f;
        p[10] = p[14] = p[17] = 0.0f;
        p[19] = g1;
        p[23] = g5;
        p[26] = g8;
    } else {
        const float ro = P.rho_out;
        const float ux = -1.0f + (f[0] + f[2] + f[4] + 2.0f * (f[1] + f[5] + f[8])) / ro;
        const float half = 0.5f * (f[2] - f[4]);
        const float h3 = f[1] - (2.0f / 3.0f) * ro * ux;
        const float h7 = f[5] + half - (1.0f / 6.0f) * ro * ux;
        const float h6 = f[8] - half - (1.0f / 6.0f) * ro * ux;
        float part[kNF], tot = 0.0f;
#pragma unroll
        for (int k = 0; k < kNF; k++) {
            const float* q = p + 9 * k;
            part[k] = q[0] + q[1] + q[2] + q[4] + q[5] + q[8];
            tot += part[k];
        }
        const float it = 1.0f / tot;
#pragma unroll
        for (int k = 0; k < kNF; k++) {
            p[9 * k + 3] = h3 * part[k] * it;
            p[9 * k + 6] = h6 * part[k] * it;
            p[9 * k + 7] = h7 * part[k] * it;
        }
    }
}

// Post-streaming populations of fluid k for the pull from a stored buffer.
template <int STORE>
struct Store;

template <>
struct Store<kStoreF32> {
    const float* f;  // [27][N] post-collision, pre-streaming populations
    long long N;
    __host__ __device__ Store(const Pop& p, long long n) : f(p.f), N(n) {}
    __host__ __device__ Store(const float* p, long long n) : f(p), N(n) {}
    // population a of (storage) fluid k stored at node idx
    __device__ __forceinline__ float get(int k, int a, int idx) const
    {
        return __ldg(f + (long long)(k * kQ + a) * N + idx);
    }
};

template <int STORE>
struct Store16 {
    const float* rho;
    const unsigned short* off;
    long long N;
    __host__ __device__ Store16(const Pop& p, long long n) : rho(p.rho), off(p.off), N(n) {}
    // offset of population a >= 1 of fluid k at node idx
    __device__ __forceinline__ float offset(int k, int a, int idx) const
    {
        return dec16<STORE>(__ldg(off + (long long)(8 * k + a - 1) * N + idx));
    }
    __device__ __forceinline__ float get(int k, int a, int idx) const
    {
        const float r = __ldg(rho + (long long)k * N + idx);
        if (a > 0) return wq(a) * r + offset(k, a, idx);
        float d[kQ];
#pragma unroll
        for (int b = 1; b < kQ; b++) d[b] = offset(k, b, idx);
        return wq(0) * r - sum_offsets(d);
    }
};
template <>
struct Store<kStoreF16> : Store16<kStoreF16> {
    using Store16<kStoreF16>::Store16;
};
template <>
struct Store<kStoreBF16> : Store16<kStoreBF16> {
    using Store16<kStoreBF16>::Store16;
};

// write the 27 post-collision populations v[k*9+a] of node i into an output buffer
template <int STORE>
__device__ __forceinline__ void store_node(const Pop& out, long long N, int i, const float v[27])
{
    if constexpr (STORE == kStoreF32) {
#pragma unroll
        for (int j = 0; j < 27; j++) out.f[(long long)j * N + i] = v[j];
    } else {
#pragma unroll
        for (int k = 0; k < kNF; k++) {
            const float* q = v + 9 * k;
            const float r = ((q[0] + (q[1] + q[3])) + (q[2] + q[4])) + ((q[5] + q[7]) + (q[6] + q[8]));
            out.rho[(long long)k * N + i] = r;
#pragma unroll
            for (int a = 1; a < kQ; a++) out.off[(long long)(8 * k + a - 1) * N + i] = enc16<STORE>(q[a] - wq(a) * r);
        }
    }
}

// Pull the post-streaming populations of the fluid node at unwrapped (X, Y) from global
// memory (labels in the frame of that unwrapped position), Eq.(16) with halfway bounce-back,
// periodic / modified periodic wrap and Zou-He on open columns.  A ghost position beyond an
// open side returns the populations of the nearest boundary-column node.
template <class S>
__device__ void pull_global(const Params& P, const S& st, const uint8_t* __restrict__ type,
                            int X, int Y, float p[27])
{
    Loc n = locate(P, X, Y);
    int nX = X;
    if (n.kind == 2) nX = X < 0 ? 0 : P.nx - 1;
    bool inlet = false, outlet = false;
#pragma unroll
    for (int a = 0; a < kQ; a++) {
        Loc s = locate(P, nX - ex(a), Y - ey(a));
        if (s.kind == 2) {
            if (nX == 0) inlet = true; else outlet = true;
#pragma unroll
            for (int k = 0; k < kNF; k++) p[9 * k + a] = 0.0f;
        } else if (s.kind == 1 || (__ldg(type + s.idx) & 2)) {
#pragma unroll
            for (int k = 0; k < kNF; k++) p[9 * k + a] = st.get(relabel(k, n.par), opp(a), n.idx);
        } else {
#pragma unroll
            for (int k = 0; k < kNF; k++) p[9 * k + a] = st.get(relabel(k, s.par), a, s.idx);
        }
    }
    if (inlet) zou_he(P, p, true);
    if (outlet) zou_he(P, p, false);
}

// Where the characteristic line of one lane of the wetting pass (C_SB node, wetted fluid, side)
// met the fluid for the local contact angle th of Eq.(21) it was marched with: the line depends
// on th and the fixed geometry only, so while a node's th repeats bit for bit (every node away
// from a moving contact line) the march is skipped and its crossing reused.  th itself is kept
// with the two wall values (wm, wl) of Eq.(21) it came from, so that while those repeat it is
// not recomputed either (the wall angles are fixed between resets of the cache).  th, wm, wl =
// NaN: none yet.
struct WetCache {
    double th, fr, wm, wl;
    int kind, ax, ay, bx, by, pad;
};

// ---- kernel launchers (lbm3_step.cu); `store` is kStoreF32 / kStoreF16 / kStoreBF16 ----
// Cw_prev (or nullptr): where the wetting pass also stores the lagged wall values it reads
void launch_wet(int store, const Params& P, int nw, const int* widx, const double* wnrm,
                const float* wang, const Pop& f, const uint8_t* type, double* Cw, WetCache* cache,
                cudaStream_t s, double* Cw_prev = nullptr);
void reset_wet_cache(WetCache* cache, int nw, cudaStream_t s);
void launch_wet_init(int store, const Params& P, int nw, const int* widx, const Pop& f,
                     const uint8_t* type, double* Cw, cudaStream_t s);
// tile of the fused step kernel (interior nodes per CTA)
constexpr int kTX = 32, kTY = 8;
// tiles: list of tile indices ty * ceil(nx / kTX) + tx; pure = every listed tile is free of solid
// nodes within 3 nodes of it and away from the domain edges
// pure FP32 tiles through bulk tensor copies (persistent, nblocks blocks): the dynamic shared
// memory they need, the one-time attribute set-up, and the launch with tensor maps of fin
// (boxes (kTX + 8, kTY + 6, kTmaPlanesA) and (kTX + 8, kTY + 6, 27 - kTmaPlanesA)) and fout
// (box (kTX, kTY, 27)) over the [27][ny][nx] buffers
constexpr int kTmaBlocksPerSm = 2;  // resident blocks of the persistent pure-tile kernel per SM
constexpr int kTmaPlanesA = 14;     // planes of a pull box in its first copy (the rest in the second)
constexpr int kTma16BlocksPerSm = 4;  // the same for the pure tiles of the 16-bit storage (3: 16.2k, 2: 15.7k MLUPS)
size_t step_tma_smem_bytes();
cudaError_t step_tma_prepare();
cudaError_t step_tma16_prepare();
void launch_step_tma(const Params& P, const int* tiles, int ntiles, int nblocks, const Pop& fout, float* u,
                     const CUtensorMap& tin_a, const CUtensorMap& tin_b, const CUtensorMap& tout, cudaStream_t s);
// pure FP32 tiles through a ring of three bulk-copy buffers, one producer warp and two consumer
// groups per block, one block per SM (nblocks blocks): tensor map of fin with the whole pull box
// (kTX + 8, kTY + 6, 27) over the [27][ny][nx] buffer
size_t step_ring_smem_bytes();
cudaError_t step_ring_prepare();
// pres_in / pres_out: fluids present per tile in the step's input / output (see k_step_ring)
void launch_step_ring(const Params& P, const int* tiles, int ntiles, int nblocks, const Pop& fout, float* u,
                      const CUtensorMap& tin, const uint64_t* pres_in, uint64_t* pres_out, cudaStream_t s);
// pure tiles of the 16-bit storage through bulk tensor copies (persistent, nblocks blocks): tensor
// maps of the densities (box (kTX + 8, kTY + 6, 3) of [3][ny][nx] FP32) and of the offset planes
// (box (kTX + 16, kTY + 6, 24) of [24][ny][nx] 16-bit words)
size_t step_tma16_smem_bytes();
void launch_step_tma16(int store, const Params& P, const int* tiles, int ntiles, int nblocks, const Pop& fout,
                       float* u, const CUtensorMap& trho, const CUtensorMap& toff, const uint64_t* pres_in,
                       uint64_t* pres_out, cudaStream_t s);
// tile lists of the fused step: pure tiles (no solid within 3 nodes, away from the domain
// edge), wall tiles (solids near, halo inside the domain) and edge tiles (halo crossing the
// domain edge: wrap, ghost columns, seam)
constexpr int kTilesPure = 0, kTilesWall = 1, kTilesEdge = 2;
// pres_in / pres_out: fluids present per tile in the step's input / output; the wall tiles read
// and write them (see k_step), the other kinds ignore them
void launch_step(int store, const Params& P, const int* tiles, int ntiles, int kind, const Pop& fin,
                 const Pop& fout, const uint8_t* type, const double* Cw, float* u, const uint64_t* pres_in,
                 uint64_t* pres_out, cudaStream_t s);
void launch_init(int store, const Params& P, const double* rho, const uint8_t* type, const Pop& f,
                 cudaStream_t s);
void launch_fields(int store, const Params& P, const Pop& f, const uint8_t* type, float* rho_out,
                   cudaStream_t s);
void launch_get_state(int store, const Params& P, const Pop& f, const uint8_t* type, float* post,
                      cudaStream_t s);
void launch_set_state(int store, const Params& P, const double* post, const uint8_t* type,
                      const Pop& f, cudaStream_t s);
int diag_blocks(const Params& P);
// adjoint (lbm3_adjoint.cu)
struct AdjointWork;
cudaError_t adjoint_alloc(const Params& P, int nw, AdjointWork** out);
void adjoint_free(AdjointWork* W);
size_t adjoint_bytes(const AdjointWork* W);
double* adjoint_dang(AdjointWork* W);
double* adjoint_du(AdjointWork* W);
// diag: the device diagnostics of the final state (sum rho_0 and sum x rho_0 give J)
void adjoint_seed(const Params& P, AdjointWork* W, const float* fs, const uint8_t* type, const double* diag,
                  cudaStream_t s);
// the stream of the forward intermediates (idle outside the reverse sweep)
cudaStream_t adjoint_side_stream(AdjointWork* W);
// the side stream waits for the work enqueued on s so far
cudaError_t adjoint_sync(AdjointWork* W, cudaStream_t s);
// forward intermediates of step t (stored state fs, lagged wall values cw_lag) on the side stream
cudaError_t adjoint_prepare(const Params& P, AdjointWork* W, int t, bool wait_reverse, int nw,
                            const int* widx, const double* wnrm, const float* wang, const float* fs,
                            const double* cw_lag, const uint8_t* type);
// s waits for the adjoint of Eq.(21) of the last reversed step (before its lagged wall values
// are overwritten, and before the angle gradient is read)
cudaError_t adjoint_join(AdjointWork* W, cudaStream_t s);
// reverse of step t on s, after its intermediates
cudaError_t adjoint_reverse(const Params& P, AdjointWork* W, int t, int nw, const int* widx,
                            const float* wang, const double* cw_lag, const uint8_t* type, cudaStream_t s);
void launch_diag(int store, const Params& P, const Pop& f, const uint8_t* type, const float* u,
                 double* partials, double* out, cudaStream_t s);

}  // namespace lbm3k
