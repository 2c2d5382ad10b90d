// lbm3_noalloc.cu -- lbm3_diag_fields: the diagnostics reduction of lbm3_diag applied to
// caller-owned device fields, without allocating.  Its block partials live in a fixed
// file-scope device array; the only set-up is a one-time lookup of that array's address on
// each device.  Nothing here depends on the rest of the library.
#include <cfloat>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/lbm3.h"

namespace {

constexpr int kThreads = 256;
// partials of at most this many blocks (8 doubles each: 64 KiB in all); the reduction strides
// over the grid, so any grid within LBM3_DIAG_FIELDS_MAX_NODES fits
constexpr int kMaxBlocks = LBM3_DIAG_FIELDS_MAX_BLOCKS;
constexpr int kMaxDevices = 64;

// scratch of the reduction: every block writes its 8 partials before the final pass reads them,
// so nothing in it has to start at zero
static __device__ __align__(256) double g_partials[kMaxBlocks * 8];

std::mutex g_mutex;
double* g_scratch[kMaxDevices] = {};

// per block: [0..2] sum rho_k, [3] sum x rho_0, [4] sum y rho_0, [5] max |u|, [6] min rho,
// [7] non-finite count, over fluid nodes
__global__ void __launch_bounds__(kThreads) k_diag_fields(const float* __restrict__ rho,
                                                          const float* __restrict__ u,
                                                          const uint8_t* __restrict__ solid,
                                                          int nx, long long N,
                                                          double* __restrict__ partials)
{
    double acc[8] = {0, 0, 0, 0, 0, 0, DBL_MAX, 0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        if (solid[i]) continue;
        const double r0 = rho[i], r1 = rho[N + i], r2 = rho[2 * N + i];
        acc[0] += r0;
        acc[1] += r1;
        acc[2] += r2;
        acc[7] += (double)!isfinite(r0) + (double)!isfinite(r1) + (double)!isfinite(r2);
        acc[3] += (double)(i % nx) * r0;
        acc[4] += (double)(i / nx) * r0;
        const double ux = u[i], uy = u[N + i];
        acc[5] = fmax(acc[5], sqrt(ux * ux + uy * uy));
        acc[6] = fmin(acc[6], r0 + r1 + r2);
    }
    __shared__ double sh[8][kThreads];
#pragma unroll
    for (int j = 0; j < 8; j++) sh[j][threadIdx.x] = acc[j];
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
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

// one warp: lane j strides over the blocks' partials, then a shuffle reduction
__global__ void k_diag_fields_final(int nb, const double* __restrict__ partials,
                                    double* __restrict__ out)
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

// the scratch address on the current device, looked up once per device
int scratch_address(double** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LBM3_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return LBM3_ERR_INVALID;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return LBM3_ERR_CUDA;
        g_scratch[dev] = static_cast<double*>(p);
    }
    *out = g_scratch[dev];
    return LBM3_OK;
}

}  // namespace

extern "C" int lbm3_diag_fields(const float* rho, const float* u, const uint8_t* solid,
                                int32_t nx, int32_t ny, double* out, void* stream)
{
    if (!rho || !u || !solid || !out) return LBM3_ERR_INVALID;
    if (nx <= 0 || ny <= 0) return LBM3_ERR_INVALID;
    const long long N = (long long)nx * ny;
    if (N > LBM3_DIAG_FIELDS_MAX_NODES) return LBM3_ERR_TOO_LARGE;
    double* partials = nullptr;
    const int rc = scratch_address(&partials);
    if (rc != LBM3_OK) return rc;
    const long long want = (N + kThreads - 1) / kThreads;
    const int nb = (int)(want < kMaxBlocks ? want : kMaxBlocks);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_diag_fields<<<nb, kThreads, 0, s>>>(rho, u, solid, nx, N, partials);
    k_diag_fields_final<<<1, 32, 0, s>>>(nb, partials, out);
    return cudaGetLastError() == cudaSuccess ? LBM3_OK : LBM3_ERR_CUDA;
}
