// costmodel.cuh -- layout of the cost model and the device functions that evaluate it
// (features of a tetrahedron, the warp-level MLP on the tensor cores).  Included by
// costmodel.cu (training, prediction, labels) and deposit.cu (the binned schedule's
// bin pass).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace pse {

constexpr int kNFeat = 16, kNHid = 64, kNOut = 2;
// flat parameter vector: mu[16], sigma[16] (feature standardisation), W1[64][16], b1[64],
// W2[64][64], b2[64], W3[2][64], b3[2]; weights row-major [out][in]
constexpr int kOffMu = 0, kOffSigma = 16, kOffW1 = 32;
constexpr int kOffB1 = kOffW1 + kNHid * kNFeat;
constexpr int kOffW2 = kOffB1 + kNHid;
constexpr int kOffB2 = kOffW2 + kNHid * kNHid;
constexpr int kOffW3 = kOffB2 + kNHid;
constexpr int kOffB3 = kOffW3 + kNOut * kNHid;
constexpr int kNPar = kOffB3 + kNOut;  // 5410

// The device-resident model (pse_costmodel_bytes() bytes, caller-owned).
struct CostModelDev {
    float p[kNPar];  // FP32 master parameters
    float m[kNPar];  // Adam first moments
    float v[kNPar];  // Adam second moments
    float g[kNPar];  // gradient of the last training step
    __nv_bfloat16 w1[kNHid * kNFeat];  // BF16 copies used by the forward passes
    __nv_bfloat16 w2[kNHid * kNHid];
    __nv_bfloat16 w3[8 * kNHid];       // W3 padded to the 8 columns of an mma tile
    long long step;                    // Adam steps taken
};

namespace {

// 16 features of a tetrahedron (grid units); tests restate them in float64.
__device__ __forceinline__ void tet_features(const TetSetup<float> &ts, float (&f)[kNFeat])
{
    float lo[3], hi[3];
    lo[0] = fminf(fminf(ts.v[0].x, ts.v[1].x), fminf(ts.v[2].x, ts.v[3].x));
    hi[0] = fmaxf(fmaxf(ts.v[0].x, ts.v[1].x), fmaxf(ts.v[2].x, ts.v[3].x));
    lo[1] = fminf(fminf(ts.v[0].y, ts.v[1].y), fminf(ts.v[2].y, ts.v[3].y));
    hi[1] = fmaxf(fmaxf(ts.v[0].y, ts.v[1].y), fmaxf(ts.v[2].y, ts.v[3].y));
    lo[2] = fminf(fminf(ts.v[0].z, ts.v[1].z), fminf(ts.v[2].z, ts.v[3].z));
    hi[2] = fmaxf(fmaxf(ts.v[0].z, ts.v[1].z), fmaxf(ts.v[2].z, ts.v[3].z));
    float ncell = 1.f, box = 1.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f[a] = hi[a] - lo[a];
        f[3 + a] = lo[a] - floorf(lo[a]);
        ncell *= (float)ts.dim[a];
        box *= f[a];
    }
    const float vol = (float)(ts.vol6 / 6.0);
    float area2 = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) area2 += sqrtf(dot(ts.n[q], ts.n[q]));
    float lmax = 0.f, lmin = 3.0e38f, lsum = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i + 1; j < 4; ++j) {
            const P3<float> d = sub(ts.v[j], ts.v[i]);
            const float l = sqrtf(dot(d, d));
            lmax = fmaxf(lmax, l);
            lmin = fminf(lmin, l);
            lsum += l;
        }
    const float lmean = lsum * (1.0f / 6.0f);
    f[6] = log2f(ncell);
    f[7] = log2f(fmaxf(vol, 1e-30f));
    f[8] = log2f(fmaxf(0.5f * area2, 1e-30f));
    f[9] = lmax;
    f[10] = lmin;
    f[11] = lmean;
    f[12] = (ts.vol6 > 0.0) ? log2f(fmaxf(ts.kappa, 1.f)) : 128.f;
    f[13] = box > 0.f ? vol / box : 0.f;
    f[14] = log2f(lmax / fmaxf(lmin, 1e-30f));
    f[15] = lmean > 0.f ? cbrtf(vol) / lmean : 0.f;
}

struct MlpSmem {
    __nv_bfloat16 x[32][kNFeat + 8];  // standardised features of the warp's 32 rows
    __nv_bfloat16 h[32][kNHid + 8];   // hidden activations
    float y[32][kNOut];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 t = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&t);
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const uint32_t *>(p);
}

// D = A (16x16, row) * B (16x8, col) + D, BF16 operands, FP32 accumulation
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// A fragment of rows [r0, r0 + 16), columns [c0, c0 + 16) of a row-major bf16 tile
template <int LD>
__device__ __forceinline__ void load_a(const __nv_bfloat16 (*m)[LD], int r0, int c0, int lane, uint32_t (&a)[4])
{
    const int g = lane >> 2, t = lane & 3;
    a[0] = ld32(&m[r0 + g][c0 + 2 * t]);
    a[1] = ld32(&m[r0 + g + 8][c0 + 2 * t]);
    a[2] = ld32(&m[r0 + g][c0 + 2 * t + 8]);
    a[3] = ld32(&m[r0 + g + 8][c0 + 2 * t + 8]);
}

// B fragment: B[k][n] = W[n][k] for n in [n0, n0 + 8), k in [k0, k0 + 16); W row-major [out][IN]
template <int IN>
__device__ __forceinline__ void load_b(const __nv_bfloat16 *__restrict__ w, int n0, int k0, int lane, uint32_t &b0,
                                       uint32_t &b1)
{
    const int g = lane >> 2, t = lane & 3;
    b0 = ld32(w + (n0 + g) * IN + k0 + 2 * t);
    b1 = ld32(w + (n0 + g) * IN + k0 + 2 * t + 8);
}

// bias + ReLU of a 32 x 64 accumulator tile, written to S.h as bf16
__device__ __forceinline__ void relu_store(MlpSmem &S, const float (&acc)[2][8][4], const float *__restrict__ bias,
                                           int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int c = nt * 8 + 2 * t;
            const float b0 = bias[c], b1 = bias[c + 1];
            *reinterpret_cast<uint32_t *>(&S.h[mt * 16 + g][c]) =
                pack_bf16(fmaxf(acc[mt][nt][0] + b0, 0.f), fmaxf(acc[mt][nt][1] + b1, 0.f));
            *reinterpret_cast<uint32_t *>(&S.h[mt * 16 + g + 8][c]) =
                pack_bf16(fmaxf(acc[mt][nt][2] + b0, 0.f), fmaxf(acc[mt][nt][3] + b1, 0.f));
        }
}

// The MLP on the warp's 32 rows (one per lane): f = raw features of this lane's row,
// y = its two outputs.  Every lane of the warp must call it.
__device__ __forceinline__ void mlp_warp(const CostModelDev *__restrict__ M, MlpSmem &S, int lane,
                                         const float (&f)[kNFeat], float (&y)[kNOut])
{
    const float *p = M->p;
#pragma unroll
    for (int q = 0; q < kNFeat; q += 2) {
        const float z0 = (f[q] - p[kOffMu + q]) / p[kOffSigma + q];
        const float z1 = (f[q + 1] - p[kOffMu + q + 1]) / p[kOffSigma + q + 1];
        *reinterpret_cast<uint32_t *>(&S.x[lane][q]) = pack_bf16(z0, z1);
    }
    __syncwarp();
    float acc[2][8][4];
    // layer 1: [32 x 16] x [16 x 64]
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        uint32_t a[4];
        load_a<kNFeat + 8>(S.x, mt * 16, 0, lane, a);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.f;
            uint32_t b0, b1;
            load_b<kNFeat>(M->w1, nt * 8, 0, lane, b0, b1);
            mma_bf16(acc[mt][nt], a[0], a[1], a[2], a[3], b0, b1);
        }
    }
    relu_store(S, acc, p + kOffB1, lane);
    __syncwarp();
    // layer 2: [32 x 64] x [64 x 64]
    uint32_t a2[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) load_a<kNHid + 8>(S.h, mt * 16, ks * 16, lane, a2[mt][ks]);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            uint32_t b0, b1;
            load_b<kNHid>(M->w2, nt * 8, ks * 16, lane, b0, b1);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
                mma_bf16(acc[mt][nt], a2[mt][ks][0], a2[mt][ks][1], a2[mt][ks][2], a2[mt][ks][3], b0, b1);
        }
    __syncwarp();
    relu_store(S, acc, p + kOffB2, lane);
    __syncwarp();
    // layer 3: [32 x 64] x [64 x 8] (outputs 0, 1; the rest is zero padding)
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            uint32_t a[4], b0, b1;
            load_a<kNHid + 8>(S.h, mt * 16, ks * 16, lane, a);
            load_b<kNHid>(M->w3, 0, ks * 16, lane, b0, b1);
            mma_bf16(o, a[0], a[1], a[2], a[3], b0, b1);
        }
        if (t == 0) {
            S.y[mt * 16 + g][0] = o[0] + p[kOffB3];
            S.y[mt * 16 + g][1] = o[1] + p[kOffB3 + 1];
            S.y[mt * 16 + g + 8][0] = o[2] + p[kOffB3];
            S.y[mt * 16 + g + 8][1] = o[3] + p[kOffB3 + 1];
        }
    }
    __syncwarp();
    y[0] = S.y[lane][0];
    y[1] = S.y[lane][1];
    __syncwarp();
}

}  // namespace
}  // namespace pse
