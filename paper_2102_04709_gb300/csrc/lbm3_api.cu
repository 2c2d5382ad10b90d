// lbm3_api.cu -- host side of the C ABI declared in include/lbm3.h: argument checks, node
// classification (Section II.B), eighth-order solid normals (Eq.19-20), the compact wall list,
// device buffers and the per-step launch sequence.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/lbm3.h"
#include "lbm3_common.cuh"

using namespace lbm3k;

struct lbm3 {
    Params P{};
    int precision = 0;
    cudaStream_t stream = nullptr;
    // device buffers: two population buffers (FP32 planes, or FP32 densities + 16-bit offset
    // planes), the node classes, wall values, velocity, scratch
    Pop pop[2] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    uint8_t* type = nullptr;
    double* Cw = nullptr;          // [3][N] wall values (written at C_SB nodes only)
    float* u = nullptr;
    float* scratch = nullptr;      // 3N floats for fields
    double* partials = nullptr;    // diagnostics block partials
    double* dout = nullptr;        // 8 doubles
    int* err_flag = nullptr;       // error bits set by kernels (Params::err)
    // bulk-tensor-copy path of the pure tiles (nx a multiple of 4): tensor maps of each
    // population buffer, FP32 storage: the two parts of the source box and the destination tile;
    // 16-bit storage: the density box (tm_in_a) and the offset-plane box (tm_in_b)
    bool tma = false;
    int tma_blocks = 0;  // persistent blocks of that kernel: kTmaBlocksPerSm per SM
    CUtensorMap tm_in_a[2], tm_in_b[2], tm_out[2];
    // FP32 pure tiles through the ring kernel (one producer warp, two consumer groups, one block
    // per SM): tensor maps of each buffer with the whole pull box, and its block count
    bool ring = false;
    int ring_blocks = 0;
    CUtensorMap tm_box[2];
    int* widx = nullptr;
    double* wnrm = nullptr;
    float* wang = nullptr;
    WetCache* wcache = nullptr;  // [4 nw] characteristic-line crossings of the wetting lanes
    double* cw_keep = nullptr;   // set by the adjoint for one step: the wetting pass stores there
                                 // the lagged wall values it reads
    // set by the adjoint for one step: the step reads io_in (through the tensor map io_box on the
    // ring path) and writes io_out instead of the two population buffers, whose turn is kept
    const Pop* io_in = nullptr;
    const Pop* io_out = nullptr;
    const CUtensorMap* io_box = nullptr;
    // the timing events of enqueue_step are recorded into a graph being captured (as nodes that
    // record them when the graph runs)
    bool ev_external = false;
    int nw = 0;
    long long n_fluid = 0;
    // tiles of the fused step kernel: pure tiles (no solid within 3 nodes, away from the domain
    // edge) run on the main stream and do not wait for the wetting pass; the other tiles run
    // after the wetting pass on a higher-priority side stream
    int* tiles_pure = nullptr;
    int* tiles_gen = nullptr;
    int n_pure = 0, n_gen = 0;
    int n_walltiles = 0;  // tiles_gen lists the inner wall tiles first, then the edge tiles
    int n_edgewall = 0;   // of the edge tiles, those with a solid node within 3 nodes come first;
                          // the others read no wall value and need not wait for the wetting pass
    long long pure_fluid = 0;
    // fluids present per tile (one byte per warp of the ring kernel's group, so no byte needs an
    // atomic or a clearing): pres[pp] describes the current state, the ring kernel writes the
    // next one's for the pure tiles; every other tile keeps 0x07 (all fluids), and so does every
    // tile after the state is replaced from outside.  pp turns with cur (and alone in the
    // adjoint's slot-to-slot steps).
    uint64_t* pres[2] = {nullptr, nullptr};
    size_t pres_bytes = 0;
    int pp = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the edge tiles run on a second side stream once the wetting pass is done, concurrently with
    // the wall tiles (the two sets are independent)
    cudaStream_t side2 = nullptr;
    cudaEvent_t ev_wet = nullptr, ev_join2 = nullptr;
    // CUDA graphs of kGraphSteps consecutive steps (an even count: a graph starts and ends on the
    // same population buffer), one per starting buffer, captured on the internal stream gcap
    // when lbm3_step first needs them and replayed on the caller's stream; dropped when a
    // captured launch argument changes (lbm3_set_inflow).  graph_off: a capture failed, so steps
    // are launched one by one (the same kernels, the same results).
    cudaStream_t gcap = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    bool graph_off = false;
    size_t bytes = 0;
    int cur = 0;
    bool ready = false;
    std::vector<int> wall_host;
    std::string err;
    // device memory of lbm3_adjoint_centroid, kept for later calls that need no more of it: the
    // checkpoints (nck states), the segment's states (nsg), the final state, the work arrays,
    // and two events that order the state copies; released by lbm3_adjoint_release or
    // lbm3_destroy
    struct AdjStore {
        float *ck_f = nullptr, *sg_f = nullptr, *fin_f = nullptr;
        double *ck_c = nullptr, *sg_c = nullptr, *fin_c = nullptr;
        int nck = 0, nsg = 0;
        AdjointWork* W = nullptr;
        cudaEvent_t ev_in = nullptr, ev_saved = nullptr;
        std::vector<CUtensorMap> box;  // ring path: the tensor map of every segment slot
        // the sweep as a graph, for nsteps / K from state buffer g_cur
        cudaGraphExec_t gexec = nullptr;
        int g_nsteps = 0, g_K = 0, g_cur = 0;
    } adj;
};

namespace {

std::string g_create_error;

int fail(lbm3* h, int code, const std::string& msg)
{
    if (h) h->err = msg; else g_create_error = msg;
    return code;
}

#define CUDA_TRY(h, call)                                                              \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail(h, e_ == cudaErrorMemoryAllocation ? LBM3_ERR_OOM : LBM3_ERR_CUDA, \
                        std::string(#call) + ": " + cudaGetErrorString(e_));           \
    } while (0)

// Solid indicator s(x) of Eq.(19) at an unwrapped position: periodic sides wrap, wall sides
// are solid beyond the domain, open sides are fluid beyond the domain.
struct Indicator {
    int nx, ny, per_y, bc_x;
    const uint8_t* m;
    int operator()(int X, int Y) const
    {
        if (Y < 0 || Y >= ny) {
            if (!per_y) return 1;
            Y = ((Y % ny) + ny) % ny;
        }
        if (X < 0 || X >= nx) {
            if (bc_x == kWalls) return 1;
            if (bc_x == kZouHe) return 0;
            X = ((X % nx) + nx) % nx;
        }
        return m[(size_t)Y * nx + X] ? 1 : 0;
    }
    bool outside_solid(int X, int Y) const
    {
        if ((Y < 0 || Y >= ny) && !per_y) return true;
        if ((X < 0 || X >= nx) && bc_x == kWalls) return true;
        return false;
    }
};

// g(X) of Eq.(15)
double seg_g(double X)
{
    if (X < -1.0) return 1.0;
    if (X > 1.0) return -1.0;
    const double s = std::sqrt(std::max(0.0, 1.0 - X * X));  // sin(arccos X)
    return X < 0.0 ? 1.0 - s : s - 1.0;
}

size_t tally(lbm3* h, size_t b)
{
    h->bytes += b;
    return b;
}

void adj_release(lbm3* h)
{
    lbm3::AdjStore& a = h->adj;
    void* ptrs[] = {a.ck_f, a.sg_f, a.fin_f, a.ck_c, a.sg_c, a.fin_c};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (a.gexec) cudaGraphExecDestroy(a.gexec);
    adjoint_free(a.W);
    if (a.ev_in) cudaEventDestroy(a.ev_in);
    if (a.ev_saved) cudaEventDestroy(a.ev_saved);
    a = lbm3::AdjStore{};
}

void release(lbm3* h)
{
    adj_release(h);
    void* ptrs[] = {h->pop[0].f, h->pop[1].f, h->pop[0].rho, h->pop[1].rho, h->pop[0].off,
                    h->pop[1].off, h->type, h->Cw, h->u, h->scratch, h->partials, h->dout,
                    h->widx, h->wnrm, h->wang, h->tiles_pure, h->tiles_gen, h->err_flag, h->wcache,
                    h->pres[0], h->pres[1]};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    h->pop[0] = h->pop[1] = Pop{nullptr, nullptr, nullptr};
    for (int c = 0; c < 2; c++)
        if (h->gexec[c]) cudaGraphExecDestroy(h->gexec[c]);
    if (h->gcap) cudaStreamDestroy(h->gcap);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_wet) cudaEventDestroy(h->ev_wet);
    if (h->ev_join2) cudaEventDestroy(h->ev_join2);
    if (h->side2) cudaStreamDestroy(h->side2);
    if (h->side) cudaStreamDestroy(h->side);
}

// Tensor maps of one [27][ny][nx] FP32 population buffer: as the two parts of the pull-source box
// of a pure tile, (kTX + 8) x (kTY + 6) x kTmaPlanesA and x (27 - kTmaPlanesA) planes, and as its
// destination tile kTX x kTY x 27.  false if the driver has no encoder or refuses the layout (the
// plain kernel is used then).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return nullptr;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    return encode;
}

// Tensor map of one [27][ny][nx] FP32 population buffer with the whole pull box of a pure tile,
// (kTX + 8) x (kTY + 6) x 27, for the ring kernel.
bool make_box_map(const Params& P, float* f, CUtensorMap* box)
{
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny, 27};
    const cuuint64_t strides[2] = {(cuuint64_t)P.nx * sizeof(float), (cuuint64_t)P.N * sizeof(float)};
    const cuuint32_t bx[3] = {kTX + 8, kTY + 6, 27};
    const cuuint32_t unit[3] = {1, 1, 1};
    return encode(box, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, f, dims, strides, bx, unit, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_tensor_maps(const Params& P, float* f, CUtensorMap* in_a, CUtensorMap* in_b, CUtensorMap* out)
{
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny, 27};
    const cuuint64_t strides[2] = {(cuuint64_t)P.nx * sizeof(float), (cuuint64_t)P.N * sizeof(float)};
    const cuuint32_t box_a[3] = {kTX + 8, kTY + 6, kTmaPlanesA};
    const cuuint32_t box_b[3] = {kTX + 8, kTY + 6, 27 - kTmaPlanesA};
    const cuuint32_t box_out[3] = {kTX, kTY, 27};
    const cuuint32_t unit[3] = {1, 1, 1};
    auto enc = [&](CUtensorMap* m, const cuuint32_t* box) {
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, f, dims, strides, box, unit,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    return enc(in_a, box_a) && enc(in_b, box_b) && enc(out, box_out);
}

// Tensor maps of one 16-bit-storage population buffer: the densities rho[3][ny][nx] (FP32, box
// (kTX + 8) x (kTY + 6) x 3) and the offset planes off[24][ny][nx] (16-bit words, box
// (kTX + 16) x (kTY + 6) x 24; its row pitch 2 nx bytes must be a multiple of 16).
bool make_tensor_maps16(const Params& P, const Pop& p, CUtensorMap* trho, CUtensorMap* toff)
{
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return false;
    const cuuint64_t rdims[3] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny, 3};
    const cuuint64_t rstrides[2] = {(cuuint64_t)P.nx * sizeof(float), (cuuint64_t)P.N * sizeof(float)};
    const cuuint32_t rbox[3] = {kTX + 8, kTY + 6, 3}, unit[3] = {1, 1, 1};
    const cuuint64_t odims[3] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny, 24};
    const cuuint64_t ostrides[2] = {(cuuint64_t)P.nx * 2, (cuuint64_t)P.N * 2};
    const cuuint32_t obox[3] = {kTX + 16, kTY + 6, 24};
    return encode(trho, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p.rho, rdims, rstrides, rbox, unit,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS &&
           encode(toff, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, p.off, odims, ostrides, obox, unit,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One timestep: fork the side streams off the main stream, run the pure tiles on the main stream
// while the side stream runs the wetting pass and then the wall tiles, and the second side stream
// the edge tiles (at once those without a solid node near them, after the wetting pass the
// others), join.  With ev != NULL the launches are bracketed by the events ev[0..6] (main: 0-1
// pure tiles; side: 2-3 wetting pass, 3-4 wall tiles; second side stream: 5-6 edge tiles).
// a timing event of enqueue_step (a record node when captured into a graph)
void record_timing(lbm3* h, cudaEvent_t ev, cudaStream_t s)
{
    if (h->ev_external)
        cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    else
        cudaEventRecord(ev, s);
}

cudaError_t enqueue_step(lbm3* h, bool last, cudaEvent_t* ev)
{
    cudaError_t e;
    const bool io = h->io_in != nullptr;
    const Pop& fin = io ? *h->io_in : h->pop[h->cur];
    const Pop& fo = io ? *h->io_out : h->pop[1 - h->cur];
    float* u = last ? h->u : nullptr;
    const uint64_t* pin = h->pres[h->pp];
    uint64_t* pout = h->pres[1 - h->pp];
    if ((e = cudaEventRecord(h->ev_fork, h->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(h->side, h->ev_fork, 0)) != cudaSuccess) return e;
    if (ev) record_timing(h, ev[0], h->stream);
    if (h->ring)
        launch_step_ring(h->P, h->tiles_pure, h->n_pure, h->ring_blocks, fo, u, io ? *h->io_box : h->tm_box[h->cur],
                         pin, pout, h->stream);
    else if (h->tma && h->precision == LBM3_FP32)
        launch_step_tma(h->P, h->tiles_pure, h->n_pure, h->tma_blocks, fo, u, h->tm_in_a[h->cur],
                        h->tm_in_b[h->cur], h->tm_out[1 - h->cur], h->stream);
    else if (h->tma)
        launch_step_tma16(h->precision, h->P, h->tiles_pure, h->n_pure, h->tma_blocks, fo, u, h->tm_in_a[h->cur],
                          h->tm_in_b[h->cur], pin, pout, h->stream);
    else
        launch_step(h->precision, h->P, h->tiles_pure, h->n_pure, kTilesPure, fin, fo, h->type, h->Cw, u,
                    pin, pout, h->stream);
    if (ev) record_timing(h, ev[1], h->stream);
    if (ev) record_timing(h, ev[2], h->side);
    launch_wet(h->precision, h->P, h->nw, h->widx, h->wnrm, h->wang, fin, h->type, h->Cw, h->wcache, h->side,
               h->cw_keep);
    if (ev) record_timing(h, ev[3], h->side);
    // edge tiles: those without a solid node near them start at once, the others after the
    // wetting pass
    const int n_edge = h->n_gen - h->n_walltiles, n_edge_free = n_edge - h->n_edgewall;
    const int* tiles_edge = h->tiles_gen + h->n_walltiles;
    const bool edges = n_edge > 0;
    if (edges) {
        if ((e = cudaStreamWaitEvent(h->side2, h->ev_fork, 0)) != cudaSuccess) return e;
        if (ev) record_timing(h, ev[5], h->side2);
        launch_step(h->precision, h->P, tiles_edge + h->n_edgewall, n_edge_free, kTilesEdge, fin, fo, h->type,
                    h->Cw, u, pin, pout, h->side2);
        if (h->n_edgewall > 0) {
            if ((e = cudaEventRecord(h->ev_wet, h->side)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(h->side2, h->ev_wet, 0)) != cudaSuccess) return e;
        }
    }
    launch_step(h->precision, h->P, h->tiles_gen, h->n_walltiles, kTilesWall, fin, fo, h->type, h->Cw, u, pin,
                pout, h->side);
    if (ev) record_timing(h, ev[4], h->side);
    if (edges) {
        launch_step(h->precision, h->P, tiles_edge, h->n_edgewall, kTilesEdge, fin, fo, h->type, h->Cw, u, pin,
                    pout, h->side2);
        if (ev) record_timing(h, ev[6], h->side2);
        if ((e = cudaEventRecord(h->ev_join2, h->side2)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(h->stream, h->ev_join2, 0)) != cudaSuccess) return e;
    } else if (ev) {
        record_timing(h, ev[5], h->side);
        record_timing(h, ev[6], h->side);
    }
    if ((e = cudaEventRecord(h->ev_join, h->side)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(h->stream, h->ev_join, 0)) != cudaSuccess) return e;
    if (!io) h->cur = 1 - h->cur;
    h->pp = 1 - h->pp;
    return cudaGetLastError();
}

constexpr int kGraphSteps = 8;
// polls of an mbarrier before a step kernel gives up on a tile's bulk copies (a completed copy
// takes a few microseconds; this is seconds of polling)
constexpr int kCopyWaitPolls = 1 << 22;

// Error bits that the kernels set (bit 0: a bulk tensor copy outlived its wait), read after the
// stream has been synchronised and cleared once read, so that each timeout is reported once.
int take_kernel_error(lbm3* h, int* bits)
{
    *bits = 0;
    cudaError_t e = cudaMemcpyAsync(bits, h->err_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess && *bits) e = cudaMemsetAsync(h->err_flag, 0, sizeof(int), h->stream);
    return e == cudaSuccess ? LBM3_OK : fail(h, LBM3_ERR_CUDA, std::string("error bits: ") + cudaGetErrorString(e));
}

// the state was replaced from outside: every tile may hold every fluid
cudaError_t pres_reset(lbm3* h)
{
    h->pp = h->cur;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; b++) e = cudaMemsetAsync(h->pres[b], 0x07, h->pres_bytes, h->stream);
    return e;
}

void drop_graphs(lbm3* h)
{
    for (int c = 0; c < 2; c++) {
        if (h->gexec[c]) cudaGraphExecDestroy(h->gexec[c]);
        h->gexec[c] = nullptr;
    }
    if (h->adj.gexec) cudaGraphExecDestroy(h->adj.gexec);
    h->adj.gexec = nullptr;
}

// kGraphSteps steps from the current buffer, none of them the last of an lbm3_step call (no
// velocity output): replay of the captured graph, captured first if needed.  Capturing only
// records the launches (nothing runs), on the internal stream, so the caller's stream may be any
// stream, the legacy default one included.
cudaError_t graph_block(lbm3* h)
{
    const int c = h->cur, pc = h->pp;
    if (!h->gexec[c] && !h->graph_off) {
        cudaStream_t user = h->stream;
        h->stream = h->gcap;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->gcap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = cudaSuccess;
            for (int s = 0; s < kGraphSteps && el == cudaSuccess; s++) el = enqueue_step(h, false, nullptr);
            e = cudaStreamEndCapture(h->gcap, &g);
            if (el != cudaSuccess) e = el;
        }
        h->stream = user;
        h->cur = c;
        h->pp = pc;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec[c], g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->gexec[c] = nullptr;
            h->graph_off = true;
            cudaGetLastError();  // a failed capture leaves no sticky error; clear the last one
        }
    }
    if (!h->gexec[c]) {
        for (int s = 0; s < kGraphSteps; s++) {
            const cudaError_t e = enqueue_step(h, false, nullptr);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    return cudaGraphLaunch(h->gexec[c], h->stream);  // ends on buffer c again
}

}  // namespace

extern "C" {

int lbm3_create(lbm3** out, const lbm3_grid* g, const uint8_t* solid, const double* angles,
                const double sigma[3], const double nu[3], double beta0, void* stream)
{
    if (!out) return fail(nullptr, LBM3_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!g || !solid || !angles || !sigma || !nu)
        return fail(nullptr, LBM3_ERR_INVALID, "NULL argument");
    // the step kernel addresses the 27 population planes with 32-bit offsets
    if (g->nx < 8 || g->ny < 8 || 27LL * g->nx * g->ny >= (1LL << 31))
        return fail(nullptr, LBM3_ERR_INVALID, "grid must be at least 8x8 with 27 * nx * ny < 2^31");
    if (g->bc_x < 0 || g->bc_x > 3) return fail(nullptr, LBM3_ERR_INVALID, "bad bc_x");
    if (g->precision != LBM3_FP32 && g->precision != LBM3_FP16 && g->precision != LBM3_BF16)
        return fail(nullptr, LBM3_ERR_INVALID, "precision must be LBM3_FP32, LBM3_FP16 or LBM3_BF16");
    for (int j = 0; j < 3; j++) {
        if (!(sigma[j] > 0.0) || !std::isfinite(sigma[j]))
            return fail(nullptr, LBM3_ERR_INVALID, "sigma must be positive");
        if (!(nu[j] > 0.0) || !std::isfinite(nu[j]))
            return fail(nullptr, LBM3_ERR_INVALID, "nu must be positive");
    }
    if (!(beta0 >= 0.0)) return fail(nullptr, LBM3_ERR_INVALID, "beta0 must be >= 0");
    if (g->bc_x == kZouHe && (!(std::fabs(g->u_in) < 0.3) || !(g->rho_out > 0.0)))
        return fail(nullptr, LBM3_ERR_INVALID, "Zou-He needs |u_in| < 0.3 and rho_out > 0");
    if (g->bc_x == kModPer && sigma[0] != sigma[2])
        return fail(nullptr, LBM3_ERR_INVALID, "modified periodic boundary needs sigma_01 == sigma_12");

    const int nx = g->nx, ny = g->ny;
    const size_t N = (size_t)nx * ny;
    const Indicator S{nx, ny, g->periodic_y ? 1 : 0, g->bc_x, solid};

    // ---- node classes: a node is a boundary node when any D2Q9 neighbour is of the other kind
    std::vector<uint8_t> cls(N);
    long long n_fluid = 0;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            const int me = S(x, y);
            bool touch = false;
            for (int a = 1; a < kQ; a++) {
                if (!me && S.outside_solid(x + ex(a), y + ey(a)))
                    return fail(nullptr, LBM3_ERR_INVALID,
                                "a fluid node touches a wall side: make the boundary rows/columns solid");
                if (S(x + ex(a), y + ey(a)) != me) touch = true;
            }
            cls[(size_t)y * nx + x] = me ? (touch ? kSB : kSI) : (touch ? kFB : kFI);
            n_fluid += !me;
        }
    if (g->bc_x == kZouHe) {
        if (!g->periodic_y) return fail(nullptr, LBM3_ERR_INVALID, "Zou-He boundary needs periodic y");
        for (int y = 0; y < ny; y++)
            for (int j = 0; j < 4; j++)
                if (solid[(size_t)y * nx + j] || solid[(size_t)y * nx + nx - 1 - j])
                    return fail(nullptr, LBM3_ERR_INVALID, "no solid node allowed within 4 columns of an open side");
    }

    // ---- wall list: C_SB nodes, outward normals by the eighth-order stencil, angle triples
    std::vector<int> widx;
    std::vector<double> wnrm;
    std::vector<float> wang;
    double young = 0.0;
    for (size_t i = 0; i < N; i++) {
        if (cls[i] != kSB) continue;
        const int x = (int)(i % nx), y = (int)(i / nx);
        double sx = 0.0, sy = 0.0;
        // eighth-order weights of Eq.(20) by |c|^2 (index = |c|^2)
        static const double w8[9] = {0.0, 4.0 / 21.0, 4.0 / 45.0, 0.0, 1.0 / 60.0, 2.0 / 315.0, 0.0, 0.0, 1.0 / 5040.0};
        for (int cy = -2; cy <= 2; cy++)
            for (int cx = -2; cx <= 2; cx++) {
                const int c2 = cx * cx + cy * cy;
                if (c2 == 0 || w8[c2] == 0.0) continue;
                if (S(x + cx, y + cy)) {
                    sx += w8[c2] * cx;
                    sy += w8[c2] * cy;
                }
            }
        double len = std::sqrt(sx * sx + sy * sy);
        if (len < 1e-12) {
            sx = sy = 0.0;
            for (int a = 1; a < kQ; a++)
                if (S(x + ex(a), y + ey(a))) {
                    const double w = a < 5 ? 1.0 / 9.0 : 1.0 / 36.0;
                    sx += w * ex(a);
                    sy += w * ey(a);
                }
            len = std::sqrt(sx * sx + sy * sy);
            if (len < 1e-12) {
                sx = 0.0;
                sy = -1.0;
                len = 1.0;
            }
        }
        widx.push_back((int)i);
        // Eq.(19) points into the solid; the characteristic lines leave along -n_s
        wnrm.push_back(-sx / len);
        wnrm.push_back(-sy / len);
        double th[3];
        for (int j = 0; j < 3; j++) {
            th[j] = angles[3 * i + j];
            if (!(th[j] > 0.0 && th[j] < 180.0))
                return fail(nullptr, LBM3_ERR_INVALID, "wall angles must lie in (0, 180) degrees");
            wang.push_back((float)th[j]);
        }
        const double d2r = M_PI / 180.0;
        const double r = sigma[0] * std::cos(th[0] * d2r) + sigma[1] * std::cos(th[1] * d2r) +
                         sigma[2] * std::cos(th[2] * d2r);
        young = std::max(young, std::fabs(r));
    }

    // ---- tiles of the fused step kernel (2-D prefix sums of the solid mask)
    std::vector<int> tp, tg, te, tf;
    long long pure_fluid = 0;
    {
        std::vector<long long> ps((size_t)(nx + 1) * (ny + 1), 0);
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++)
                ps[(size_t)(y + 1) * (nx + 1) + x + 1] = ps[(size_t)y * (nx + 1) + x + 1] +
                                                         ps[(size_t)(y + 1) * (nx + 1) + x] -
                                                         ps[(size_t)y * (nx + 1) + x] +
                                                         (solid[(size_t)y * nx + x] ? 1 : 0);
        auto box = [&](int xa, int ya, int xb, int yb) {  // solids in [xa, xb) x [ya, yb)
            return ps[(size_t)yb * (nx + 1) + xb] - ps[(size_t)ya * (nx + 1) + xb] -
                   ps[(size_t)yb * (nx + 1) + xa] + ps[(size_t)ya * (nx + 1) + xa];
        };
        const int ntx = (nx + kTX - 1) / kTX, nty = (ny + kTY - 1) / kTY;
        for (int ty = 0; ty < nty; ty++)
            for (int tx = 0; tx < ntx; tx++) {
                const int x0 = tx * kTX, y0 = ty * kTY;
                const int x1 = std::min(nx, x0 + kTX), y1 = std::min(ny, y0 + kTY);
                // a tile without a fluid node has nothing to update (solid nodes are never
                // written and their populations never read): no block is launched for it
                if (box(x0, y0, x1, y1) == (long long)(x1 - x0) * (y1 - y0)) continue;
                const bool inner = x0 >= 3 && y0 >= 3 && x0 + kTX + 3 <= nx && y0 + kTY + 3 <= ny;
                if (inner && box(x0 - 3, y0 - 3, x0 + kTX + 3, y0 + kTY + 3) == 0) {
                    tp.push_back(ty * ntx + tx);
                    pure_fluid += (long long)kTX * kTY;
                } else if (inner) {
                    tg.push_back(ty * ntx + tx);
                } else {
                    // an edge tile: any solid node within 3 nodes, across a periodic side too?
                    bool near_solid = false;
                    for (int y = y0 - 3; y < y0 + kTY + 3 && !near_solid; y++) {
                        int yy = y;
                        if (yy < 0 || yy >= ny) {
                            if (!g->periodic_y) continue;
                            yy = (yy % ny + ny) % ny;
                        }
                        for (int x = x0 - 3; x < x0 + kTX + 3; x++) {
                            int xx = x;
                            if (xx < 0 || xx >= nx) {
                                if (g->bc_x != kPeriodic && g->bc_x != kModPer) continue;
                                xx = (xx % nx + nx) % nx;
                            }
                            if (solid[(size_t)yy * nx + xx]) {
                                near_solid = true;
                                break;
                            }
                        }
                    }
                    (near_solid ? te : tf).push_back(ty * ntx + tx);
                }
            }
    }
    const int n_wall_tiles = (int)tg.size();
    const int n_edge_wall = (int)te.size();
    tg.insert(tg.end(), te.begin(), te.end());
    tg.insert(tg.end(), tf.begin(), tf.end());

    // ---- parameters
    lbm3* h = new lbm3();
    h->stream = (cudaStream_t)stream;
    h->precision = g->precision;
    Params& P = h->P;
    P.nx = nx;
    P.ny = ny;
    P.N = (long long)N;
    P.per_y = g->periodic_y ? 1 : 0;
    P.bc_x = g->bc_x;
    P.u_in = (float)g->u_in;
    P.rho_out = (float)g->rho_out;
    P.sig01 = (float)sigma[0];
    P.sig02 = (float)sigma[1];
    P.sig12 = (float)sigma[2];
    P.inv_nu0 = (float)(1.0 / nu[0]);
    P.inv_nu1 = (float)(1.0 / nu[1]);
    P.inv_nu2 = (float)(1.0 / nu[2]);
    P.beta0 = (float)beta0;
    // X_kl = (sigma_mk^2 + sigma_ml^2 - sigma_kl^2) / (2 sigma_mk sigma_ml), m = the third fluid
    const double s01 = sigma[0], s02 = sigma[1], s12 = sigma[2];
    P.g01 = (float)seg_g((s02 * s02 + s12 * s12 - s01 * s01) / (2.0 * s02 * s12));
    P.g02 = (float)seg_g((s01 * s01 + s12 * s12 - s02 * s02) / (2.0 * s01 * s12));
    P.g12 = (float)seg_g((s01 * s01 + s02 * s02 - s12 * s12) / (2.0 * s01 * s02));
    for (int k = 0; k < kNF; k++)
        for (int a = 0; a < kQ; a++) {
            P.off_plane[k * kQ + a] = (k * kQ + a) * (int)N;
            P.off_pull[k * kQ + a] = (k * kQ + a) * (int)N - ex(a) - ey(a) * nx;
            P.off_pull16[k * kQ + a] = k * (int)N - ex(a) - ey(a) * nx;
            P.off_pull16o[k * kQ + a] = a > 0 ? (8 * k + a - 1) * (int)N - ex(a) - ey(a) * nx : 0;
        }
    h->nw = (int)widx.size();
    h->n_fluid = n_fluid;
    h->n_pure = (int)tp.size();
    h->n_gen = (int)tg.size();
    h->n_walltiles = n_wall_tiles;
    h->n_edgewall = n_edge_wall;
    h->pure_fluid = pure_fluid;
    h->wall_host = widx;

    // ---- device buffers
    auto dmalloc = [&](void** p, size_t b) -> cudaError_t {
        cudaError_t e = cudaMalloc(p, b ? b : 16);
        if (e == cudaSuccess) tally(h, b);
        return e;
    };
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2; b++) {
        if (g->precision == LBM3_FP32) {
            if (e == cudaSuccess) e = dmalloc((void**)&h->pop[b].f, (size_t)27 * N * sizeof(float));
        } else {
            if (e == cudaSuccess) e = dmalloc((void**)&h->pop[b].rho, (size_t)3 * N * sizeof(float));
            if (e == cudaSuccess) e = dmalloc((void**)&h->pop[b].off, (size_t)24 * N * sizeof(unsigned short));
        }
    }
    if (e == cudaSuccess) e = dmalloc((void**)&h->type, N);
    if (e == cudaSuccess) e = dmalloc((void**)&h->Cw, 3 * N * sizeof(double));
    if (e == cudaSuccess) e = dmalloc((void**)&h->u, 2 * N * sizeof(float));
    if (e == cudaSuccess) e = dmalloc((void**)&h->scratch, 3 * N * sizeof(float));
    if (e == cudaSuccess) e = dmalloc((void**)&h->partials, (size_t)diag_blocks(P) * 8 * sizeof(double));
    if (e == cudaSuccess) e = dmalloc((void**)&h->dout, 8 * sizeof(double));
    if (e == cudaSuccess) e = dmalloc((void**)&h->err_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->err_flag, 0, sizeof(int));
    P.err = h->err_flag;
    P.wait_polls = kCopyWaitPolls;
    if (e == cudaSuccess) e = dmalloc((void**)&h->widx, widx.size() * sizeof(int));
    if (e == cudaSuccess) e = dmalloc((void**)&h->wnrm, wnrm.size() * sizeof(double));
    if (e == cudaSuccess) e = dmalloc((void**)&h->wang, wang.size() * sizeof(float));
    if (e == cudaSuccess) e = dmalloc((void**)&h->wcache, 4 * widx.size() * sizeof(WetCache));
    if (e == cudaSuccess) {
        reset_wet_cache(h->wcache, (int)widx.size(), nullptr);
        e = cudaGetLastError();
    }
    h->pres_bytes = (size_t)((nx + kTX - 1) / kTX) * ((ny + kTY - 1) / kTY) * sizeof(uint64_t);
    for (int b = 0; b < 2; b++) {
        if (e == cudaSuccess) e = dmalloc((void**)&h->pres[b], h->pres_bytes);
        if (e == cudaSuccess) e = cudaMemset(h->pres[b], 0x07, h->pres_bytes);
    }
    if (e == cudaSuccess) e = dmalloc((void**)&h->tiles_pure, tp.size() * sizeof(int));
    if (e == cudaSuccess) e = dmalloc((void**)&h->tiles_gen, tg.size() * sizeof(int));
    if (e == cudaSuccess && !tp.empty()) e = cudaMemcpy(h->tiles_pure, tp.data(), tp.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !tg.empty()) e = cudaMemcpy(h->tiles_gen, tg.data(), tg.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        int lo = 0, hi = 0;
        e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->side2, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->gcap, cudaStreamNonBlocking);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_wet, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join2, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemcpy(h->type, cls.data(), N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !widx.empty()) e = cudaMemcpy(h->widx, widx.data(), widx.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !wnrm.empty()) e = cudaMemcpy(h->wnrm, wnrm.data(), wnrm.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !wang.empty()) e = cudaMemcpy(h->wang, wang.data(), wang.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->Cw, 0, 3 * N * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(h->u, 0, 2 * N * sizeof(float));
    // pure tiles through bulk tensor copies where the layout allows them (row pitch a multiple of
    // 16 bytes: nx % 4 == 0 for FP32 populations, nx % 8 == 0 for 16-bit offset planes);
    // LBM3_DISABLE_TMA=1 in the environment keeps the plain kernel
    if (e == cudaSuccess && nx % (g->precision == LBM3_FP32 ? 4 : 8) == 0 && h->n_pure > 0) {
        const char* off = std::getenv("LBM3_DISABLE_TMA");
        const bool f32 = g->precision == LBM3_FP32;
        bool maps = !(off && off[0] == '1');
        for (int b = 0; b < 2 && maps; b++)
            maps = f32 ? make_tensor_maps(P, h->pop[b].f, &h->tm_in_a[b], &h->tm_in_b[b], &h->tm_out[b])
                       : make_tensor_maps16(P, h->pop[b], &h->tm_in_a[b], &h->tm_in_b[b]);
        if (maps) {
            int dev = 0, sms = 0;
            e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            // a kernel that cannot get the shared memory it needs leaves the pure tiles on the plain
            // kernel (the same results), as when the tensor maps cannot be encoded
            cudaError_t ep = cudaSuccess;
            if (e == cudaSuccess) {
                ep = f32 ? step_tma_prepare() : step_tma16_prepare();
                if (ep != cudaSuccess) cudaGetLastError();
            }
            // SMs left free for the wetting pass and the wall / edge tiles, which run on the side
            // stream while the persistent pure-tile kernel holds its SMs: their share of the step's
            // work, in units of a pure tile's SM time as measured on the 4096 x 2048 pillars (a
            // wall or edge tile 1.8, the wetting pass 0.038 per C_SB node: 30 of 152 SMs there).
            // LBM3_SPARE_SMS=<n> in the environment at lbm3_create sets the count instead.
            const double wg = 1.8 * h->n_gen + 0.038 * h->nw;
            int spare = std::min(sms / 2, (int)std::lround(sms * wg / (wg + h->n_pure)));
            if (const char* ov = std::getenv("LBM3_SPARE_SMS"))
                spare = std::max(0, std::min(sms - 1, std::atoi(ov)));
            h->tma_blocks = (f32 ? kTmaBlocksPerSm : kTma16BlocksPerSm) * (sms - spare);
            h->tma = e == cudaSuccess && ep == cudaSuccess && sms > 0;
            // FP32: the warp-specialised ring kernel, unless LBM3_PURE_KERNEL=tma asks for the
            // two-blocks-per-SM kernel (both give the same results)
            const char* pk = std::getenv("LBM3_PURE_KERNEL");
            if (h->tma && f32 && !(pk && std::strcmp(pk, "tma") == 0)) {
                bool rm = true;
                for (int b = 0; b < 2 && rm; b++) rm = make_box_map(P, h->pop[b].f, &h->tm_box[b]);
                if (rm && step_ring_prepare() == cudaSuccess) {
                    h->ring = true;
                    h->ring_blocks = sms - spare;
                } else {
                    cudaGetLastError();
                }
            }
        }
    }
    if (e != cudaSuccess) {
        const int code = e == cudaErrorMemoryAllocation ? LBM3_ERR_OOM : LBM3_ERR_CUDA;
        release(h);
        delete h;
        return fail(nullptr, code, std::string("device set-up failed: ") + cudaGetErrorString(e));
    }
    *out = h;
    if (young > 1e-6) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "wall angles violate Eq.(18): max |sum sigma cos theta| = %.3g", young);
        h->err = buf;
        return LBM3_WARN_YOUNG;
    }
    h->err.clear();
    return LBM3_OK;
}

int lbm3_set_fields(lbm3* h, const double* rho)
{
    if (!h || !rho) return fail(h, LBM3_ERR_INVALID, "NULL argument");
    const size_t N = (size_t)h->P.N;
    double* drho = nullptr;
    CUDA_TRY(h, cudaMallocAsync((void**)&drho, 3 * N * sizeof(double), h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(drho, rho, 3 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    h->cur = 0;
    CUDA_TRY(h, pres_reset(h));
    CUDA_TRY(h, cudaMemsetAsync(h->err_flag, 0, sizeof(int), h->stream));
    launch_init(h->precision, h->P, drho, h->type, h->pop[0], h->stream);
    launch_wet_init(h->precision, h->P, h->nw, h->widx, h->pop[0], h->type, h->Cw, h->stream);
    CUDA_TRY(h, cudaMemsetAsync(h->u, 0, 2 * N * sizeof(float), h->stream));
    CUDA_TRY(h, cudaFreeAsync(drho, h->stream));
    CUDA_TRY(h, cudaGetLastError());
    h->ready = true;
    return LBM3_OK;
}

int lbm3_step(lbm3* h, int32_t nsteps)
{
    if (!h) return fail(h, LBM3_ERR_INVALID, "NULL handle");
    if (nsteps < 0) return fail(h, LBM3_ERR_INVALID, "nsteps < 0");
    if (!h->ready) return fail(h, LBM3_ERR_STATE, "lbm3_set_fields has not been called");
    // blocks of kGraphSteps steps through the graphs while at least one step remains after them;
    // the rest, and the last step (it writes the velocity), one by one
    int s = 0;
    for (; s + kGraphSteps < nsteps; s += kGraphSteps) CUDA_TRY(h, graph_block(h));
    for (; s < nsteps; s++) CUDA_TRY(h, enqueue_step(h, s == nsteps - 1, nullptr));
    return LBM3_OK;
}

int lbm3_step_timed_detail(lbm3* h, int32_t nsteps, double ms_out[5])
{
    if (!h || !ms_out) return fail(h, LBM3_ERR_INVALID, "NULL argument");
    if (nsteps < 0) return fail(h, LBM3_ERR_INVALID, "nsteps < 0");
    if (!h->ready) return fail(h, LBM3_ERR_STATE, "lbm3_set_fields has not been called");
    for (int j = 0; j < 5; j++) ms_out[j] = 0.0;
    std::vector<cudaEvent_t> ev(7 * (size_t)nsteps + 1);  // 7 per step, and the end of the run
    for (auto& e : ev) CUDA_TRY(h, cudaEventCreate(&e));
    // The steps are captured into one graph with the events as record nodes, so that they run
    // as lbm3_step runs them (replayed graphs) rather than launched one by one; launched one by
    // one if the capture fails.
    bool ran = false;
    if (nsteps > 0 && !h->graph_off) {
        const int c0 = h->cur, p0 = h->pp;
        cudaStream_t user = h->stream;
        h->stream = h->gcap;
        h->ev_external = true;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        cudaError_t ec = cudaStreamBeginCapture(h->gcap, cudaStreamCaptureModeThreadLocal);
        if (ec == cudaSuccess) {
            cudaError_t el = cudaSuccess;
            for (int s = 0; s < nsteps && el == cudaSuccess; s++) el = enqueue_step(h, s == nsteps - 1, &ev[7 * (size_t)s]);
            if (el == cudaSuccess) el = cudaEventRecordWithFlags(ev.back(), h->gcap, cudaEventRecordExternal);
            ec = cudaStreamEndCapture(h->gcap, &g);
            if (el != cudaSuccess) ec = el;
        }
        h->ev_external = false;
        h->stream = user;
        if (ec == cudaSuccess) ec = cudaGraphInstantiate(&x, g, 0);
        if (g) cudaGraphDestroy(g);
        if (ec == cudaSuccess) {
            // cur and pp turned during the capture as the steps turn them
            cudaError_t er = cudaGraphLaunch(x, h->stream);
            if (er == cudaSuccess) er = cudaStreamSynchronize(h->stream);
            cudaGraphExecDestroy(x);
            CUDA_TRY(h, er);
            ran = true;
        } else {
            h->cur = c0;
            h->pp = p0;
            cudaGetLastError();  // a failed capture leaves no sticky error; clear the last one
        }
    }
    if (!ran) {
        for (int s = 0; s < nsteps; s++) CUDA_TRY(h, enqueue_step(h, s == nsteps - 1, &ev[7 * (size_t)s]));
        CUDA_TRY(h, cudaEventRecord(ev.back(), h->stream));  // after the last step's joins
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    }
    if (nsteps > 0) {
        float t = 0.f;
        CUDA_TRY(h, cudaEventElapsedTime(&t, ev[0], ev.back()));
        ms_out[4] = t;
    }
    for (int s = 0; s < nsteps; s++) {
        const cudaEvent_t* E = &ev[7 * (size_t)s];
        const int from[4] = {2, 0, 3, 5}, to[4] = {3, 1, 4, 6};
        for (int j = 0; j < 4; j++) {
            float t = 0.f;
            CUDA_TRY(h, cudaEventElapsedTime(&t, E[from[j]], E[to[j]]));
            ms_out[j] += t;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return LBM3_OK;
}

int lbm3_step_timed(lbm3* h, int32_t nsteps, double ms_out[3])
{
    if (!ms_out) return fail(h, LBM3_ERR_INVALID, "NULL argument");
    double d[5];
    const int rc = lbm3_step_timed_detail(h, nsteps, d);
    if (rc != LBM3_OK) return rc;
    ms_out[0] = d[0];
    ms_out[1] = d[1];
    ms_out[2] = d[2] + d[3];
    return LBM3_OK;
}

int lbm3_fields(lbm3* h, double* rho_out, double* u_out)
{
    if (!h || !rho_out) return fail(h, LBM3_ERR_INVALID, "NULL argument");
    if (!h->ready) return fail(h, LBM3_ERR_STATE, "lbm3_set_fields has not been called");
    const size_t N = (size_t)h->P.N;
    launch_fields(h->precision, h->P, h->pop[h->cur], h->type, h->scratch, h->stream);
    CUDA_TRY(h, cudaGetLastError());
    std::vector<float> tmp(3 * N);
    CUDA_TRY(h, cudaMemcpyAsync(tmp.data(), h->scratch, 3 * N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    std::vector<float> tu;
    if (u_out) {
        tu.resize(2 * N);
        CUDA_TRY(h, cudaMemcpyAsync(tu.data(), h->u, 2 * N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < 3 * N; i++) rho_out[i] = tmp[i];
    if (u_out)
        for (size_t i = 0; i < 2 * N; i++) u_out[i] = tu[i];
    int bits = 0;
    if (int rc = take_kernel_error(h, &bits)) return rc;
    if (bits & 1) return fail(h, LBM3_ERR_CUDA, "a bulk tensor copy of the step kernel did not complete in time");
    return LBM3_OK;
}

int lbm3_diag(lbm3* h, double out[8])
{
    if (!h || !out) return fail(h, LBM3_ERR_INVALID, "NULL argument");
    if (!h->ready) return fail(h, LBM3_ERR_STATE, "lbm3_set_fields has not been called");
    launch_diag(h->precision, h->P, h->pop[h->cur], h->type, h->u, h->partials, h->dout, h->stream);
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaMemcpyAsync(out, h->dout, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    int bits = 0;
    if (int rc = take_kernel_error(h, &bits)) return rc;
    if (bits & 1) return fail(h, LBM3_ERR_CUDA, "a bulk tensor copy of the step kernel did not complete in time");
    if (out[7] > 0.0 || !(out[6] > 0.0)) return fail(h, LBM3_ERR_DIVERGED, "non-finite or non-positive density");
    return LBM3_OK;
}

int lbm3_n_wall(const lbm3* h) { return h ? h->nw : LBM3_ERR_INVALID; }

int lbm3_wall_nodes(const lbm3* h, int32_t* idx, int32_t cap)
{
    if (!h || (!idx && cap > 0)) return LBM3_ERR_INVALID;
    const int n = std::min<int>(cap, h->nw);
    for (int j = 0; j < n; j++) idx[j] = h->wall_host[j];
    return h->nw;
}

int lbm3_wall_values(lbm3* h, double* c, int32_t cap)
{
    if (!h || (!c && cap > 0)) return fail(h, LBM3_ERR_INVALID, "NULL argument");
    if (!h->ready) return fail(h, LBM3_ERR_STATE, "lbm3_set_fields has not been called");
    const size_t N = (size_t)h->P.N;
    std::vector<double> cw(3 * N);
    CUDA_TRY(h, cudaMemcpyAsync(cw.data(), h->Cw, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    const int n = std::min<int>(cap, h->nw);
    for (int j = 0; j < n; j++) {
        const size_t i = (size_t)h->wall_host[j];
        for (int k = 0; k < 3; k++) c[3 * j + k] = cw[k * N + i];
    }
    return h->nw;
}

int lbm3_get_state(lbm3* h, double* f_post, double* wall_c)
{
    if (!h || !f_post) return fail(h, LBM3_ERR_INVALID, "NULL argument");
    if (!h->ready) return fail(h, LBM3_ERR_STATE, "lbm3_set_fields has not been called");
    const size_t N = (size_t)h->P.N;
    float* post = nullptr;
    CUDA_TRY(h, cudaMallocAsync((void**)&post, 27 * N * sizeof(float), h->stream));
    launch_get_state(h->precision, h->P, h->pop[h->cur], h->type, post, h->stream);
    CUDA_TRY(h, cudaGetLastError());
    std::vector<float> tmp(27 * N);
    CUDA_TRY(h, cudaMemcpyAsync(tmp.data(), post, 27 * N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaFreeAsync(post, h->stream));
    std::vector<double> cw;
    if (wall_c) {
        cw.resize(3 * N);
        CUDA_TRY(h, cudaMemcpyAsync(cw.data(), h->Cw, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < 27 * N; i++) f_post[i] = tmp[i];
    if (wall_c) std::memcpy(wall_c, cw.data(), 3 * N * sizeof(double));
    return LBM3_OK;
}

int lbm3_set_state(lbm3* h, const double* f_post, const double* wall_c)
{
    if (!h || !f_post || !wall_c) return fail(h, LBM3_ERR_INVALID, "NULL argument");
    const size_t N = (size_t)h->P.N;
    double* dpost = nullptr;
    CUDA_TRY(h, cudaMallocAsync((void**)&dpost, 27 * N * sizeof(double), h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(dpost, f_post, 27 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    h->cur = 0;
    CUDA_TRY(h, pres_reset(h));
    CUDA_TRY(h, cudaMemsetAsync(h->err_flag, 0, sizeof(int), h->stream));
    launch_set_state(h->precision, h->P, dpost, h->type, h->pop[0], h->stream);
    CUDA_TRY(h, cudaMemcpyAsync(h->Cw, wall_c, 3 * N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->u, 0, 2 * N * sizeof(float), h->stream));
    CUDA_TRY(h, cudaFreeAsync(dpost, h->stream));
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->ready = true;
    return LBM3_OK;
}

int lbm3_set_wall_angles(lbm3* h, const double* angles)
{
    if (!h || (!angles && h->nw > 0)) return fail(h, LBM3_ERR_INVALID, "NULL argument");
    std::vector<float> a(3 * (size_t)h->nw);
    for (size_t j = 0; j < a.size(); j++) {
        if (!(angles[j] > 0.0 && angles[j] < 180.0))
            return fail(h, LBM3_ERR_INVALID, "wall angles must lie in (0, 180) degrees");
        a[j] = (float)angles[j];
    }
    if (!a.empty())
        CUDA_TRY(h, cudaMemcpyAsync(h->wang, a.data(), a.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    // the wetting pass keeps each lane's angle with the wall values it came from: forget them
    reset_wet_cache(h->wcache, h->nw, h->stream);
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return LBM3_OK;
}

int lbm3_set_inflow(lbm3* h, double u_in)
{
    if (!h) return fail(h, LBM3_ERR_INVALID, "NULL handle");
    if (h->P.bc_x != kZouHe) return fail(h, LBM3_ERR_INVALID, "no Zou-He inlet");
    if (!(std::fabs(u_in) < 0.3)) return fail(h, LBM3_ERR_INVALID, "|u_in| must be < 0.3");
    if ((float)u_in == h->P.u_in) return LBM3_OK;  // the captured graphs stay valid
    h->P.u_in = (float)u_in;
    drop_graphs(h);  // the graphs hold the old Params
    return LBM3_OK;
}

int lbm3_adjoint_centroid(lbm3* h, int32_t nsteps, int32_t K, double* J_out, double* dJ_dangles,
                          double* dJ_du)
{
    if (!h || !J_out || !dJ_du || (!dJ_dangles && h->nw > 0)) return fail(h, LBM3_ERR_INVALID, "NULL argument");
    if (nsteps < 1 || K < 1) return fail(h, LBM3_ERR_INVALID, "nsteps and checkpoint_every must be >= 1");
    if (!h->ready) return fail(h, LBM3_ERR_STATE, "lbm3_set_fields has not been called");
    if (h->precision != LBM3_FP32) return fail(h, LBM3_ERR_INVALID, "the adjoint needs FP32 storage");
    if (h->P.bc_x == kModPer) return fail(h, LBM3_ERR_INVALID, "the adjoint does not support the modified periodic boundary");
    const size_t N = (size_t)h->P.N;
    const size_t fb = 27 * N * sizeof(float), cb = 3 * N * sizeof(double);
    const int nseg = (nsteps + K - 1) / K;
    const int seglen = std::min(K, nsteps);
    const int nck = std::max(nseg - 1, 1);
    lbm3::AdjStore& st = h->adj;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess && st.W && (st.nck < nck || st.nsg < seglen)) adj_release(h);
    if (e == cudaSuccess && !st.W) {
        if (e == cudaSuccess) e = cudaMalloc((void**)&st.ck_f, fb * nck);
        if (e == cudaSuccess) e = cudaMalloc((void**)&st.ck_c, cb * nck);
        if (e == cudaSuccess) e = cudaMalloc((void**)&st.sg_f, fb * seglen);
        if (e == cudaSuccess) e = cudaMalloc((void**)&st.sg_c, cb * seglen);
        if (e == cudaSuccess) e = cudaMalloc((void**)&st.fin_f, fb);
        if (e == cudaSuccess) e = cudaMalloc((void**)&st.fin_c, cb);
        // the wetting pass stores only the C_SB nodes' wall values into a state's slot; the rest
        // stays 0, as in the handle's own array
        if (e == cudaSuccess) e = cudaMemset(st.ck_c, 0, cb * nck);
        if (e == cudaSuccess) e = cudaMemset(st.sg_c, 0, cb * seglen);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st.ev_in, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st.ev_saved, cudaEventDisableTiming);
        if (e == cudaSuccess) e = adjoint_alloc(h->P, h->nw, &st.W);
        if (e == cudaSuccess && h->ring) {
            st.box.resize(seglen);
            for (int j = 0; j < seglen && e == cudaSuccess; j++)
                if (!make_box_map(h->P, st.sg_f + (size_t)j * 27 * N, &st.box[j])) e = cudaErrorInvalidValue;
        }
        st.nck = nck;
        st.nsg = seglen;
    }
    if (e != cudaSuccess) {
        adj_release(h);
        return fail(h, e == cudaErrorMemoryAllocation ? LBM3_ERR_OOM : LBM3_ERR_CUDA,
                    std::string("adjoint set-up: ") + cudaGetErrorString(e));
    }
    float *ck_f = st.ck_f, *sg_f = st.sg_f, *fin_f = st.fin_f;
    double *ck_c = st.ck_c, *sg_c = st.sg_c, *fin_c = st.fin_c;
    AdjointWork* W = st.W;
    auto cleanup = [&]() {
        if (e != cudaSuccess) adj_release(h);
    };
    cudaStream_t s = h->stream;
    // A state is saved while the next step runs, which only reads its populations: they are
    // copied on the adjoint's side stream, which the step after next waits for, as it overwrites
    // them; that step's wetting pass stores the wall values it starts from (saved_step).  A save
    // that no step follows (the final state) copies the wall values itself.
    cudaStream_t cs = adjoint_side_stream(W);
    bool copying = false;
    auto save_wait = [&]() {
        if (copying) cudaStreamWaitEvent(s, st.ev_saved, 0);
        copying = false;
    };
    auto save = [&](float* df, double* dc, bool stepped) {
        save_wait();
        cudaEventRecord(st.ev_in, s);
        cudaStreamWaitEvent(cs, st.ev_in, 0);
        cudaMemcpyAsync(df, h->pop[h->cur].f, fb, cudaMemcpyDeviceToDevice, cs);
        cudaEventRecord(st.ev_saved, cs);
        copying = true;
        if (!stepped || h->nw == 0) cudaMemcpyAsync(dc, h->Cw, cb, cudaMemcpyDeviceToDevice, s);
    };
    // one step whose lagged wall values go to dc (or nowhere)
    auto saved_step = [&](double* dc, bool last) {
        h->cw_keep = h->nw > 0 ? dc : nullptr;
        const cudaError_t r = enqueue_step(h, last, nullptr);
        h->cw_keep = nullptr;
        return r;
    };
    // Where the step kernels can read any buffer (the ring path, through the slot's tensor map, or
    // the plain kernels), a segment's steps go from slot to slot of the store and its states need
    // no copy: one step from slot j to `out`, its lagged wall values to slot j's
    const bool direct = h->ring || !h->tma;
    auto slot = [&](int j) { return Pop{sg_f + (size_t)j * 27 * N, nullptr, nullptr}; };
    auto slot_step = [&](int j, const Pop& out, bool last) {
        const Pop in = slot(j);
        h->io_in = &in;
        h->io_out = &out;
        h->io_box = h->ring ? &st.box[j] : nullptr;
        const cudaError_t r = saved_step(sg_c + (size_t)j * 3 * N, last);
        h->io_in = h->io_out = nullptr;
        h->io_box = nullptr;
        return r;
    };
    auto restore = [&](const float* df, const double* dc) {
        save_wait();
        h->cur = 0;
        pres_reset(h);
        cudaMemcpyAsync(h->pop[0].f, df, fb, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(h->Cw, dc, cb, cudaMemcpyDeviceToDevice, s);
    };
    // The whole sweep, enqueued without a host round trip (the seed reads J from the device
    // diagnostics): the forward pass with checkpoints, whose last segment's states go straight to
    // the segment store (with K >= nsteps: every state, no recompute at all), then the reverse
    // over the segments, each other segment recomputed from its checkpoint, then the final state
    // back into the handle.  capturing: recorded into a graph (no host waits allowed).
    auto enqueue_all = [&](bool capturing) -> cudaError_t {
        cudaError_t r = cudaSuccess;
        const int t_last = (nseg - 1) * K;
        for (int t = 0; t < nsteps && r == cudaSuccess; t++) {
            double* dc = nullptr;
            if (t >= t_last && direct) {
                if (t == t_last) {
                    save_wait();
                    cudaMemcpyAsync(sg_f, h->pop[h->cur].f, fb, cudaMemcpyDeviceToDevice, s);
                }
                const int j = t - t_last;
                if (t + 1 < nsteps) {
                    r = slot_step(j, slot(j + 1), false);
                } else {
                    r = slot_step(j, h->pop[1 - h->cur], true);  // the final state in the handle's buffer
                    h->cur = 1 - h->cur;
                    if (h->pp != h->cur) pres_reset(h);
                }
                continue;
            }
            if (t >= t_last) {
                dc = sg_c + (size_t)(t - t_last) * 3 * N;
                save(sg_f + (size_t)(t - t_last) * 27 * N, dc, true);
            } else if (t % K == 0) {
                dc = ck_c + (size_t)(t / K) * 3 * N;
                save(ck_f + (size_t)(t / K) * 27 * N, dc, true);
            } else {
                save_wait();  // the copy of the previous state is done before this step overwrites it
            }
            r = saved_step(dc, t == nsteps - 1);
        }
        save_wait();
        if (r != cudaSuccess) return r;
        launch_diag(h->precision, h->P, h->pop[h->cur], h->type, h->u, h->partials, h->dout, s);
        save(fin_f, fin_c, false);
        save_wait();
        cudaMemsetAsync(adjoint_dang(W), 0, sizeof(double) * 3 * (size_t)std::max(h->nw, 1), s);
        cudaMemsetAsync(adjoint_du(W), 0, sizeof(double), s);
        adjoint_seed(h->P, W, h->pop[h->cur].f, h->type, h->dout, s);
        for (int seg = nseg - 1; seg >= 0 && r == cudaSuccess; seg--) {
            const int t0 = seg * K, t1 = std::min(nsteps, t0 + K);
            if (seg < nseg - 1 && direct) {
                // the checkpoint into slot 0 and the wall values into the handle, then slot to slot
                pres_reset(h);
                cudaMemcpyAsync(sg_f, ck_f + (size_t)seg * 27 * N, fb, cudaMemcpyDeviceToDevice, s);
                cudaMemcpyAsync(h->Cw, ck_c + (size_t)seg * 3 * N, cb, cudaMemcpyDeviceToDevice, s);
                for (int t = t0; t < t1 - 1 && r == cudaSuccess; t++) r = slot_step(t - t0, slot(t - t0 + 1), false);
                cudaMemcpyAsync(sg_c + (size_t)(t1 - 1 - t0) * 3 * N, h->Cw, cb, cudaMemcpyDeviceToDevice, s);
            } else if (seg < nseg - 1) {
                restore(ck_f + (size_t)seg * 27 * N, ck_c + (size_t)seg * 3 * N);
                for (int t = t0; t < t1; t++) {
                    double* dc = sg_c + (size_t)(t - t0) * 3 * N;
                    save(sg_f + (size_t)(t - t0) * 27 * N, dc, t < t1 - 1);
                    if (t < t1 - 1 && (r = saved_step(dc, false)) != cudaSuccess) break;
                }
                save_wait();
            }
            // the intermediates of step t - 1 are prepared on the adjoint's side stream while the
            // reverse of step t runs
            auto prepare = [&](int t, bool wait) {
                return adjoint_prepare(h->P, W, t, wait, h->nw, h->widx, h->wnrm, h->wang,
                                       sg_f + (size_t)(t - t0) * 27 * N, sg_c + (size_t)(t - t0) * 3 * N, h->type);
            };
            if (r == cudaSuccess) r = adjoint_sync(W, s);
            if (r == cudaSuccess) r = prepare(t1 - 1, false);
            for (int t = t1 - 1; t >= t0 && r == cudaSuccess; t--) {
                if (t > t0) r = prepare(t - 1, t + 1 < t1);
                if (r == cudaSuccess)
                    r = adjoint_reverse(h->P, W, t, h->nw, h->widx, h->wang, sg_c + (size_t)(t - t0) * 3 * N, h->type, s);
                if (r == cudaSuccess) r = cudaGetLastError();
            }
            // the segment's stored states are recomputed for the next segment; launched one by
            // one, the host waits for this segment's reverse before it enqueues that (running
            // further ahead made the sweep slower)
            if (r == cudaSuccess) r = adjoint_join(W, s);
            if (r == cudaSuccess && seg > 0 && !capturing) r = cudaStreamSynchronize(s);
        }
        restore(fin_f, fin_c);
        return r;
    };
    // Replayed as one CUDA graph, captured by the first call of a size (the graph holds the
    // store's addresses, so it lives as long as the store) and dropped with the handle's other
    // graphs when a captured parameter changes; launched one by one if the capture fails.
    if (st.gexec && (st.g_nsteps != nsteps || st.g_K != K || st.g_cur != h->cur)) {
        cudaGraphExecDestroy(st.gexec);
        st.gexec = nullptr;
    }
    if (!st.gexec && !h->graph_off) {
        const int cur0 = h->cur;
        cudaStream_t user = h->stream;
        h->stream = h->gcap;
        s = h->gcap;
        cudaGraph_t g = nullptr;
        cudaError_t ec = cudaStreamBeginCapture(h->gcap, cudaStreamCaptureModeThreadLocal);
        if (ec == cudaSuccess) {
            const cudaError_t el = enqueue_all(true);
            ec = cudaStreamEndCapture(h->gcap, &g);
            if (el != cudaSuccess) ec = el;
        }
        if (ec == cudaSuccess) ec = cudaGraphInstantiate(&st.gexec, g, 0);
        if (g) cudaGraphDestroy(g);
        h->stream = user;
        s = user;
        if (ec == cudaSuccess) {
            st.g_nsteps = nsteps;
            st.g_K = K;
            st.g_cur = cur0;
        } else {
            st.gexec = nullptr;
            cudaGetLastError();  // a failed capture leaves no sticky error; clear the last one
        }
        h->cur = cur0;  // the capture ran nothing
        h->pp = cur0;
        copying = false;
    }
    if (st.gexec) {
        e = cudaGraphLaunch(st.gexec, s);
        h->cur = 0;  // where the sweep leaves the state (restore of the final state)
        h->pp = 0;
    } else {
        e = enqueue_all(false);
    }
    double d[8];
    std::vector<double> dang(3 * (size_t)std::max(h->nw, 1));
    double du = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, h->dout, sizeof d, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dang.data(), adjoint_dang(W), sizeof(double) * dang.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&du, adjoint_du(W), sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return fail(h, LBM3_ERR_CUDA, std::string("adjoint: ") + cudaGetErrorString(e));
    int bits = 0;
    if (int rc = take_kernel_error(h, &bits)) return rc;
    if (bits & 1) return fail(h, LBM3_ERR_CUDA, "a bulk tensor copy of the step kernel did not complete in time");
    *J_out = d[3] / d[0];
    for (int w = 0; w < h->nw; w++)
        for (int j = 0; j < 3; j++) dJ_dangles[3 * w + j] = dang[(size_t)j * h->nw + w];
    *dJ_du = h->P.bc_x == kZouHe ? du : 0.0;
    return LBM3_OK;
}

int lbm3_info(const lbm3* h, int64_t out[9])
{
    if (!h || !out) return LBM3_ERR_INVALID;
    for (int j = 0; j < 9; j++) out[j] = 0;
    out[0] = h->n_fluid;
    out[1] = h->nw;
    // populations read and written per fluid node: 27 FP32 (216 B), or per fluid an FP32 density
    // and 8 16-bit offsets (120 B); plus one class byte per node
    const long long per = h->precision == LBM3_FP32 ? 216 : 120;
    out[2] = h->n_fluid * per + h->P.N;
    out[3] = (h->n_pure > 0) + (h->n_walltiles > 0) + (h->n_edgewall > 0) +
             (h->n_gen - h->n_walltiles - h->n_edgewall > 0);
    out[4] = h->nw > 0 ? 1 : 0;
    out[5] = (int64_t)h->bytes;
    // the pure-tile launch reads and writes 27 FP32 populations per node and no class bytes
    out[6] = h->pure_fluid * per;
    out[7] = h->pure_fluid;
    out[8] = h->ring ? 2 : (h->tma ? 1 : 0);
    return LBM3_OK;
}

int lbm3_set_stream(lbm3* h, void* stream)
{
    if (!h) return LBM3_ERR_INVALID;
    const cudaStream_t next = (cudaStream_t)stream;
    if (next != h->stream) {
        // work already queued on the old stream (and the side stream, joined to it at the end of
        // every step) comes before anything later enqueued on the new one
        CUDA_TRY(h, cudaEventRecord(h->ev_fork, h->stream));
        CUDA_TRY(h, cudaStreamWaitEvent(next, h->ev_fork, 0));
    }
    h->stream = next;
    return LBM3_OK;
}

int lbm3_set_copy_wait_limit(lbm3* h, int32_t polls)
{
    if (!h) return LBM3_ERR_INVALID;
    h->P.wait_polls = polls < 0 ? kCopyWaitPolls : polls;
    drop_graphs(h);  // the graphs hold the old Params
    return LBM3_OK;
}

int lbm3_sync(lbm3* h)
{
    if (!h) return LBM3_ERR_INVALID;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return LBM3_OK;
}

int lbm3_adjoint_release(lbm3* h)
{
    if (!h) return fail(h, LBM3_ERR_INVALID, "NULL handle");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    adj_release(h);
    return e == cudaSuccess ? LBM3_OK : fail(h, LBM3_ERR_CUDA, std::string("adjoint release: ") + cudaGetErrorString(e));
}

void lbm3_destroy(lbm3* h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
}

const char* lbm3_last_error(const lbm3* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
