// Kernels shared by the tensor-core and the plain FP32 dense samplers: the per-replica
// scale c0 ("Simulated Bifurcation with Gaussian noise"), the start state with its phi, and
// the read-out of the packed signs (and optional final state) from the padded state arrays.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "sb_common.cuh"

namespace moq {
namespace {

// c0_r = 1 / max_i |sum_j J(c)_ij| (fallback 1 / max_i sum_j |J(c)_ij|, then 1); one block per replica.
__global__ void k_dense_c0(const int64_t* __restrict__ rowsum, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ wn,
                           int64_t nnz, int32_t n, int32_t K, const float* __restrict__ lambda, int32_t R, float* c0)
{
    __shared__ unsigned red[2];
    const int r = blockIdx.x;
    if (r >= R) return;
    float lam[kMaxK];
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) lam[k] = k < K ? lambda[(int64_t)r * K + k] : 0.0f;
    if (threadIdx.x == 0) red[0] = red[1] = 0u;
    __syncthreads();
    float mx = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < kMaxK; ++k)
            if (k < K) s = fmaf(lam[k], (float)rowsum[(int64_t)i * K + k], s);
        mx = fmaxf(mx, fabsf(s));
    }
    atomicMax(&red[0], __float_as_uint(mx));
    __syncthreads();
    float m = __uint_as_float(red[0]);
    if (m == 0.0f) {  // every row sum vanishes: the rare fallback walks the rows
        float ma = 0.0f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            float s = 0.0f;
            for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                float v = 0.0f;
                for (int k = 0; k < K; ++k) v = fmaf(lam[k], (float)wn[(int64_t)k * nnz + p], v);
                s += fabsf(v);
            }
            ma = fmaxf(ma, s);
        }
        atomicMax(&red[1], __float_as_uint(ma));
        __syncthreads();
        m = __uint_as_float(red[1]);
    }
    if (threadIdx.x == 0) c0[r] = m > 0.0f ? 1.0f / m : 1.0f;
}

__device__ __forceinline__ void store_phi(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void store_phi(float* p, float v) { *p = v; }
__device__ __forceinline__ void store_phi(__nv_fp8_e4m3* p, float v) { *p = __nv_fp8_e4m3(v); }

// Start state (Philox or the caller's arrays) and its phi; PhiT = BF16 or E4M3 (tensor-core
// sampler) or float (CUDA-core FP32 sampler).
template <int VARIANT, typename PhiT>
__global__ void k_dense_init(int32_t n, int32_t np, int32_t R, int32_t R_pad, float init_amp, const float* __restrict__ x_init,
                             const float* __restrict__ y_init, uint32_t key0, uint32_t key1, uint32_t round32, float* x, float* y,
                             PhiT* phi)
{
    const int64_t total = (int64_t)R_pad * np;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(q / np), i = (int)(q - (int64_t)r * np);
        float xv = 0.0f, yv = 0.0f;
        if (r < R && i < n) {
            if (x_init) {
                xv = x_init[(int64_t)r * n + i] + 0.0f;
                yv = y_init ? y_init[(int64_t)r * n + i] : 0.0f;
            } else {
                const uint4 o = Philox4x32::block(make_uint4(0xFFFFFFFFu, (uint32_t)i, (uint32_t)r, round32), key0, key1);
                xv = __fmul_rn(init_amp, signed_unit(o.x)) + 0.0f;
                yv = __fmul_rn(init_amp, signed_unit(o.y));
            }
        }
        x[q] = xv;
        y[q] = yv;
        store_phi(phi + q, (r < R && i < n) ? phi_of<VARIANT>(xv) : 0.0f);
    }
}

__global__ void k_dense_readout(int32_t n, int32_t np, int32_t R, int32_t W, const float* __restrict__ x, const float* __restrict__ y,
                                uint64_t* bits, float* x_out, float* y_out)
{
    const int r = blockIdx.x;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        uint64_t word = 0;
        for (int b = 0; b < 64 && w * 64 + b < n; ++b)
            if (x[(int64_t)r * np + w * 64 + b] < 0.0f) word |= 1ull << b;
        bits[(int64_t)r * W + w] = word;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if (x_out) x_out[(int64_t)r * n + i] = x[(int64_t)r * np + i];
        if (y_out) y_out[(int64_t)r * n + i] = y[(int64_t)r * np + i];
    }
}

}  // namespace
}  // namespace moq
