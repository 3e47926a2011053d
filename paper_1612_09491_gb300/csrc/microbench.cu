// microbench.cu -- the peaks the deposit kernel's roofline is measured against, taken on
// the GPU it runs on: the FP32 FMA issue rate (independent FMA chains in every lane) and
// the throughput of FP64 reductions to global memory scattered over a large array (the
// deposit's accumulation pattern).  The FP32 and FP64-reduction peaks of this part are
// not published as measured figures, so the bench measures them beside the deposit.
#include <cstdint>

#include "../../include/pse.h"
#include "internal.h"

namespace pse {
namespace {

constexpr int kChains = 8;

// kChains independent FMA chains per thread, `iters` steps each: 2 * kChains * iters FLOP
__global__ void __launch_bounds__(256) k_fma_peak(float *out, int64_t iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

// each thread adds `per_thread` values to cells of grid[n] chosen by a multiplicative hash
__global__ void __launch_bounds__(256) k_red_peak(double *grid, int64_t n, int64_t per_thread)
{
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t h = tid * 0x9E3779B97F4A7C15ull + 1;
    for (int64_t i = 0; i < per_thread; ++i) {
        h = h * 6364136223846793005ull + 1442695040888963407ull;
        atomicAdd(grid + (int64_t)((h >> 17) % (uint64_t)n), 1.0);
    }
}

}  // namespace
}  // namespace pse

extern "C" {

int pse_microbench_fma(float *d_out, int64_t blocks, int64_t iters, void *stream)
{
    if (!d_out || blocks < 1 || iters < 1) return PSE_ERR_INVALID_ARG;
    pse::k_fma_peak<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_out, iters, 0.999999f,
                                                                                     1e-6f);
    return cudaGetLastError() == cudaSuccess ? PSE_OK : PSE_ERR_CUDA;
}

int pse_microbench_red(double *d_grid, int64_t n_cells, int64_t blocks, int64_t per_thread, void *stream)
{
    if (!d_grid || n_cells < 1 || blocks < 1 || per_thread < 1) return PSE_ERR_INVALID_ARG;
    pse::k_red_peak<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_grid, n_cells, per_thread);
    return cudaGetLastError() == cudaSuccess ? PSE_OK : PSE_ERR_CUDA;
}

}  // extern "C"
