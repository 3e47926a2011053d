// costmodel.cu -- the learned cost model of the binned schedule.
//
// The paper balances the deposit by estimated work per tetrahedron (Sec. 5) and notes
// how unevenly the work falls across tetrahedra (Sec. 6.2).  This file holds a small
// learned estimate of that work:
//  * 16 geometric features per tetrahedron (tet_features);
//  * an MLP 16 -> 64 -> 64 -> 2 with ReLU, predicting log(1 + overlapped cells) and
//    log(1 + partial clips).  Inference runs on the tensor cores (mma.sync m16n8k16,
//    BF16 operands, FP32 accumulation), 32 tetrahedra per warp;
//  * training on the GPU: a forward/backward kernel (BF16-rounded operands, FP32
//    arithmetic, per-block gradient reduction in shared memory) and an Adam kernel;
//  * the labels: per-tetrahedron counts produced by the exact FP32 deposit itself
//    (k_tet_counts).
// The model only steers scheduling (which tetrahedra are split across warps); it never
// touches a deposited value.
#include <cuda_bf16.h>

#include "common.cuh"
#include "costmodel.cuh"

namespace pse {
namespace {

// ---------------------------------------------------------------------------
// labels: overlapped cells and partial clips of every tetrahedron, from the same
// classification and FP32 clip (with the FP64 guard) as the deposit.  A cell counts as
// overlapped when its overlap exceeds 1e-6 of the cell volume: FP32 rounding leaves
// cells that only touch the tetrahedron with overlaps of that order instead of 0.
// ---------------------------------------------------------------------------
constexpr double kOverlapFloor = 1e-6;

__global__ void __launch_bounds__(128) k_tet_counts(const DepositParams P, int32_t *__restrict__ counts)
{
    const int64_t n_tets = 6 * P.n_units;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tets;
         t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i, j, k;
        int n_ov = 0, n_clip = 0;
        if (cube_of_unit(P, t / 6, i, j, k)) {
            P3<float> v[4], res[4];
            int base[3];
            lattice_tet<float>(P, i, j, k, (int)(t % 6), v, base, res);
            TetSetup<float> ts;
            if (tet_setup<float>(v, ts)) swap12(res);
            const int64_t ncell = (int64_t)ts.dim[0] * ts.dim[1] * ts.dim[2];
            if (!tet_ok(base, ts) || ts.vol6 == 0.0 || ncell == 1) {
                n_ov = 1;
            } else if (ncell <= (int64_t)(1 << 25)) {
                const bool g64 = !(ts.kappa <= P.kappa_max);
                for (int iz = 0; iz < ts.dim[2]; ++iz)
                    for (int iy = 0; iy < ts.dim[1]; ++iy)
                        for (int ix = 0; ix < ts.dim[0]; ++ix) {
                            const int cx = ts.lo[0] + ix, cy = ts.lo[1] + iy, cz = ts.lo[2] + iz;
                            const int cls = classify_cell<float>(ts.n, ts.e, ts.pos, ts.neg, (float)cx, (float)cy,
                                                                 (float)cz);
                            if (cls == CELL_INSIDE) {
                                ++n_ov;
                            } else if (cls == CELL_PARTIAL) {
                                ++n_clip;
                                double vol;
                                if (g64) {
                                    P3<double> pd[4];
                                    exact_vertices(ts.v, res, cx, cy, cz, pd);
                                    vol = overlap_volume_fp64(pd);
                                } else {
                                    P3<float> p[4];
#pragma unroll
                                    for (int q = 0; q < 4; ++q)
                                        p[q] = mk<float>(ts.v[q].x - cx, ts.v[q].y - cy, ts.v[q].z - cz);
                                    float err;
                                    vol = (double)overlap_volume_ax<float>(p, ts.n, ts.axis, ts.lx, ts.ly, err);
                                }
                                if (vol > kOverlapFloor) ++n_ov;
                            }
                        }
            }
        }
        counts[2 * t] = n_ov;
        counts[2 * t + 1] = n_clip;
    }
}

__global__ void __launch_bounds__(128) k_features(const DepositParams P, float *__restrict__ feat)
{
    const int64_t n_tets = 6 * P.n_units;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tets;
         t += (int64_t)gridDim.x * blockDim.x) {
        float f[kNFeat];
        int64_t i, j, k;
        if (cube_of_unit(P, t / 6, i, j, k)) {
            P3<float> v[4];
            int base[3];
            lattice_tet<float>(P, i, j, k, (int)(t % 6), v, base);
            TetSetup<float> ts;
            tet_setup<float>(v, ts);
            tet_features(ts, f);
        } else {
#pragma unroll
            for (int q = 0; q < kNFeat; ++q) f[q] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < kNFeat; ++q) feat[kNFeat * t + q] = f[q];
    }
}

// one thread per 32 rows: predictions through the warp MLP
__global__ void __launch_bounds__(256) k_predict(const CostModelDev *__restrict__ M, const float *__restrict__ feat,
                                                 int64_t n, float *__restrict__ out)
{
    __shared__ MlpSmem sm[8];
    MlpSmem &S = sm[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w * 32 < n; w += warps) {
        const int64_t r = w * 32 + lane;
        float f[kNFeat];
#pragma unroll
        for (int q = 0; q < kNFeat; ++q) f[q] = (r < n) ? feat[kNFeat * r + q] : 0.f;
        float y[kNOut];
        mlp_warp(M, S, lane, f, y);
        if (r < n) {
            out[kNOut * r] = y[0];
            out[kNOut * r + 1] = y[1];
        }
    }
}

// ---------------------------------------------------------------------------
// training: forward and backward of the mean squared error, one sample per thread;
// gradients reduced per block in shared memory, then added to M->g
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rb(float x, bool round)
{
    return round ? __bfloat162float(__float2bfloat16_rn(x)) : x;
}

__global__ void __launch_bounds__(128) k_train_fwd_bwd(CostModelDev *__restrict__ M, const float *__restrict__ feat,
                                                       const float *__restrict__ target,
                                                       const int64_t *__restrict__ index, int64_t batch, int fp32,
                                                       double *__restrict__ loss)
{
    extern __shared__ float gs[];  // [kNPar - kOffW1] gradient of the weights and biases
    const int ng = kNPar - kOffW1;
    for (int i = threadIdx.x; i < ng; i += blockDim.x) gs[i] = 0.f;
    __syncthreads();
    const bool bf = fp32 == 0;
    const float *p = M->p;
    const float inv_b = 1.0f / (float)batch;
    double lsum = 0.0;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < batch; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = index ? index[b] : b;
        float z[kNFeat];
#pragma unroll
        for (int q = 0; q < kNFeat; ++q) z[q] = rb((feat[kNFeat * s + q] - p[kOffMu + q]) / p[kOffSigma + q], bf);
        float a1[kNHid], h1[kNHid], a2[kNHid], h2[kNHid];
        for (int o = 0; o < kNHid; ++o) {
            float acc = p[kOffB1 + o];
#pragma unroll
            for (int q = 0; q < kNFeat; ++q) acc = fmaf(rb(p[kOffW1 + o * kNFeat + q], bf), z[q], acc);
            a1[o] = acc;
            h1[o] = rb(fmaxf(acc, 0.f), bf);
        }
        for (int o = 0; o < kNHid; ++o) {
            float acc = p[kOffB2 + o];
            for (int q = 0; q < kNHid; ++q) acc = fmaf(rb(p[kOffW2 + o * kNHid + q], bf), h1[q], acc);
            a2[o] = acc;
            h2[o] = rb(fmaxf(acc, 0.f), bf);
        }
        float dy[kNOut];
#pragma unroll
        for (int o = 0; o < kNOut; ++o) {
            float acc = p[kOffB3 + o];
            for (int q = 0; q < kNHid; ++q) acc = fmaf(rb(p[kOffW3 + o * kNHid + q], bf), h2[q], acc);
            const float d = acc - target[kNOut * s + o];
            lsum += 0.5 * (double)d * d;
            dy[o] = d * inv_b;
        }
        // layer 3
#pragma unroll
        for (int o = 0; o < kNOut; ++o) {
            atomicAdd(&gs[kOffB3 - kOffW1 + o], dy[o]);
            for (int q = 0; q < kNHid; ++q) atomicAdd(&gs[kOffW3 - kOffW1 + o * kNHid + q], dy[o] * h2[q]);
        }
        // layer 2 (a2 is reused for dL/da2)
        for (int q = 0; q < kNHid; ++q) {
            float d = 0.f;
#pragma unroll
            for (int o = 0; o < kNOut; ++o) d = fmaf(dy[o], rb(p[kOffW3 + o * kNHid + q], bf), d);
            a2[q] = (a2[q] > 0.f) ? d : 0.f;
        }
        for (int o = 0; o < kNHid; ++o) {
            const float d = a2[o];
            if (d == 0.f) continue;
            atomicAdd(&gs[kOffB2 - kOffW1 + o], d);
            for (int q = 0; q < kNHid; ++q) atomicAdd(&gs[kOffW2 - kOffW1 + o * kNHid + q], d * h1[q]);
        }
        // layer 1 (a1 is reused for dL/da1)
        for (int q = 0; q < kNHid; ++q) {
            float d = 0.f;
            for (int o = 0; o < kNHid; ++o) d = fmaf(a2[o], rb(p[kOffW2 + o * kNHid + q], bf), d);
            a1[q] = (a1[q] > 0.f) ? d : 0.f;
        }
        for (int o = 0; o < kNHid; ++o) {
            const float d = a1[o];
            if (d == 0.f) continue;
            atomicAdd(&gs[kOffB1 - kOffW1 + o], d);
#pragma unroll
            for (int q = 0; q < kNFeat; ++q) atomicAdd(&gs[o * kNFeat + q], d * z[q]);
        }
    }
    // block totals
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(kFull, lsum, o);
    if ((threadIdx.x & 31) == 0 && lsum != 0.0) atomicAdd(loss, lsum / (double)batch);
    __syncthreads();
    for (int i = threadIdx.x; i < ng; i += blockDim.x)
        if (gs[i] != 0.f) atomicAdd(&M->g[kOffW1 + i], gs[i]);
}

__global__ void k_adam(CostModelDev *__restrict__ M, float lr)
{
    const long long step = M->step + 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    for (int i = kOffW1 + blockIdx.x * blockDim.x + threadIdx.x; i < kNPar; i += gridDim.x * blockDim.x) {
        const float g = M->g[i];
        const float m = b1 * M->m[i] + (1.0f - b1) * g;
        const float v = b2 * M->v[i] + (1.0f - b2) * g * g;
        M->m[i] = m;
        M->v[i] = v;
        M->p[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

// BF16 copies of the weights (W3 padded to 8 rows with zeros) and the step counter
__global__ void k_refresh(CostModelDev *__restrict__ M, int bump)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNHid * kNHid; i += gridDim.x * blockDim.x) {
        M->w2[i] = __float2bfloat16_rn(M->p[kOffW2 + i]);
        if (i < kNHid * kNFeat) M->w1[i] = __float2bfloat16_rn(M->p[kOffW1 + i]);
        if (i < 8 * kNHid) M->w3[i] = __float2bfloat16_rn(i < kNOut * kNHid ? M->p[kOffW3 + i] : 0.f);
    }
    if (bump && blockIdx.x == 0 && threadIdx.x == 0) M->step += 1;
}

}  // namespace

size_t costmodel_bytes() { return sizeof(CostModelDev); }

cudaError_t costmodel_set(CostModelDev *m, const float *h_params, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(m, 0, sizeof(CostModelDev), st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(m->p, h_params, sizeof(float) * kNPar, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = launch_refresh(m, false, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

cudaError_t costmodel_get(const CostModelDev *m, float *h_params, float *h_grad, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    if (h_params) e = cudaMemcpyAsync(h_params, m->p, sizeof(float) * kNPar, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && h_grad) e = cudaMemcpyAsync(h_grad, m->g, sizeof(float) * kNPar, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

cudaError_t launch_tet_counts(const DepositParams &p, int32_t *counts, cudaStream_t st)
{
    const int64_t n = 6 * p.n_units;
    int64_t blocks = (n + 127) / 128;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    k_tet_counts<<<(unsigned)blocks, 128, 0, st>>>(p, counts);
    return cudaGetLastError();
}

cudaError_t launch_features(const DepositParams &p, float *feat, cudaStream_t st)
{
    const int64_t n = 6 * p.n_units;
    int64_t blocks = (n + 127) / 128;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    k_features<<<(unsigned)blocks, 128, 0, st>>>(p, feat);
    return cudaGetLastError();
}

cudaError_t launch_predict(const CostModelDev *m, const float *feat, int64_t n, float *out, cudaStream_t st)
{
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_predict<<<(unsigned)blocks, 256, 0, st>>>(m, feat, n, out);
    return cudaGetLastError();
}

cudaError_t launch_refresh(CostModelDev *m, bool bump, cudaStream_t st)
{
    k_refresh<<<16, 256, 0, st>>>(m, bump ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_train_step(CostModelDev *m, const float *feat, const float *target, const int64_t *index,
                              int64_t batch, float lr, bool fp32, bool update, double *loss, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(m->g, 0, sizeof(m->g), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(loss, 0, sizeof(double), st);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(float) * (kNPar - kOffW1);
    e = cudaFuncSetAttribute((const void *)k_train_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t blocks = (batch + 127) / 128;
    if (blocks > 152 * 2) blocks = 152 * 2;
    if (blocks < 1) blocks = 1;
    k_train_fwd_bwd<<<(unsigned)blocks, 128, smem, st>>>(m, feat, target, index, batch, fp32 ? 1 : 0, loss);
    e = cudaGetLastError();
    if (e != cudaSuccess || !update) return e;
    k_adam<<<(kNPar + 255) / 256, 256, 0, st>>>(m, lr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_refresh(m, true, st);
}

}  // namespace pse
