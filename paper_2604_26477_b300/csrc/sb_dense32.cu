// Dense NI-SB in plain FP32 on the CUDA cores (SB equations and Eq. NI-SB): the force
// c0 sum_k c_k (J^(k) Phi)_i with J^(k) and phi in FP32 and every product and sum in FP32,
// the full-precision comparison for the tensor-core sampler. Start state, noise counters,
// force combination and update are those of the tensor-core sampler.
#include <algorithm>

#include "dense_common.cuh"

// Plain FP32 form of the dense sampler: the same replica state on the CUDA cores, with the
// couplings and phi in FP32 (every product and sum in FP32).
struct moq_dense_fp32 {
    int32_t n = 0, K = 0, n_pad = 0, max_R = 0, R_pad = 0;
    const moq_instance* inst = nullptr;
    float* J = nullptr;                  // K x n_pad x n_pad, row-major, zero-padded
    float* x = nullptr;                  // R_pad x n_pad
    float* y = nullptr;                  // R_pad x n_pad
    float* phi[2] = {nullptr, nullptr};  // R_pad x n_pad
    float* c0 = nullptr;                 // R_pad
};

namespace moq {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---- plain FP32 step on the CUDA cores ------------------------------------------------
// The dynamics of the tensor-core step with every product in FP32: G_k = J^(k) Phi for a tile
// of 64 spins x 128 replicas by a register-tiled FMA loop. Thread (ti, tr) of 256 holds spins
// i0 + ti + 16 s (s < 4) of the replica octet r0 + 8 tr.., i.e. 4 x 8 accumulators per
// objective. The spin dimension j is walked in chunks of 32: J^(k)[i0:+64, j0:+32] and
// Phi[r0:+128, j0:+32] go from L2 to shared memory by 16-byte cp.async into three stages
// (rows as in memory, padded to 36 floats, plus 4 floats per replica octet, so that the
// 16-byte reads of a warp fall on distinct bank groups). Measured at n = 2000, K = 3,
// R = 8192 (bSB, same call): chunks of 16 took 4.57 ms per step, 32 4.29 ms; unrolling the
// inner loop over j (254 registers) gained nothing at 32. The epilogue combines the force,
// draws the noise and updates the state exactly as the tensor-core epilogue does, so for
// dSB with integer couplings whose row sums of |J| stay below 2^24 this form gives the bits
// of the split-precision tensor-core form (|J| <= 65408) and of the BF16 form (|J| <= 256):
// every G_k is then the same exact integer.
constexpr int kF32M = 64, kF32N = 128, kF32K = 32, kF32Threads = 256, kF32Stages = 3;
constexpr int kF32Row = kF32K + 4;  // staged operand row (floats)

__host__ __device__ constexpr int f32_b_offset(int row) { return row * kF32Row + (row >> 3) * 4; }
__host__ __device__ constexpr int f32_stage_floats(int K) { return K * kF32M * kF32Row + f32_b_offset(kF32N); }
size_t f32_smem_bytes(int K) { return sizeof(float) * (size_t)kF32Stages * f32_stage_floats(K); }

struct Dense32Args {
    const float* J;  // K x n_pad x n_pad
    const float* phi_in;
    float* phi_out;
    float* x;
    float* y;
    const float* lambda;  // R x K
    const float* c0;
    int32_t n, n_pad, R, m;
    float cm;  // a_m - a0 (when schedule is NULL)
    const float* schedule;
    float a0, dt, kappa, dta0;
    uint32_t key0, key1, round32;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int VARIANT, int KOBJ, bool NOISE>
__global__ void __launch_bounds__(kF32Threads, 1) k_dense32_step(Dense32Args a)
{
    extern __shared__ __align__(16) float sm32[];
    const int tid = threadIdx.x, ti = tid & 15, tr = tid >> 4;
    const int i0 = blockIdx.x * kF32M, r0 = blockIdx.y * kF32N;
    const int np = a.n_pad, nchunks = np / kF32K;
    auto issue = [&](int c) {
        const int j0 = c * kF32K;
        float* st = sm32 + (c % kF32Stages) * f32_stage_floats(KOBJ);
        constexpr int Q = kF32K / 4;  // 16-byte pieces per staged row
#pragma unroll
        for (int e = tid; e < KOBJ * kF32M * Q; e += kF32Threads) {
            const int row = e / Q, c4 = (e % Q) * 4, k = row / kF32M, ir = row % kF32M;
            cp_async16(smem_u32(st + row * kF32Row + c4), a.J + ((int64_t)k * np + i0 + ir) * np + j0 + c4);
        }
        float* bs = st + KOBJ * kF32M * kF32Row;
#pragma unroll
        for (int e = tid; e < kF32N * Q; e += kF32Threads) {
            const int row = e / Q, c4 = (e % Q) * 4;
            cp_async16(smem_u32(bs + f32_b_offset(row) + c4), a.phi_in + (int64_t)(r0 + row) * np + j0 + c4);
        }
        cp_async_commit();
    };
    float acc[KOBJ][4][8];
#pragma unroll
    for (int k = 0; k < KOBJ; ++k)
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[k][s][q] = 0.0f;
    issue(0);
    if (nchunks > 1) issue(1);
    else cp_async_commit();
#pragma unroll 1
    for (int c = 0; c < nchunks; ++c) {
        if (c + 2 < nchunks) issue(c + 2);
        else cp_async_commit();  // an empty group keeps "all but the two newest" = chunk c
        asm volatile("cp.async.wait_group 2;" ::: "memory");
        __syncthreads();
        const float* st = sm32 + (c % kF32Stages) * f32_stage_floats(KOBJ);
        const float* bs = st + KOBJ * kF32M * kF32Row;
#pragma unroll 1
        for (int j4 = 0; j4 < kF32K; j4 += 4) {
            float4 b[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) b[q] = *reinterpret_cast<const float4*>(bs + f32_b_offset(tr * 8 + q) + j4);
#pragma unroll
            for (int k = 0; k < KOBJ; ++k)
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const float4 av = *reinterpret_cast<const float4*>(st + (k * kF32M + ti + 16 * s) * kF32Row + j4);
                    // j in order for every accumulator; the eight replicas interleave the chains
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[k][s][q] = fmaf(av.x, b[q].x, acc[k][s][q]);
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[k][s][q] = fmaf(av.y, b[q].y, acc[k][s][q]);
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[k][s][q] = fmaf(av.z, b[q].z, acc[k][s][q]);
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[k][s][q] = fmaf(av.w, b[q].w, acc[k][s][q]);
                }
        }
        __syncthreads();  // stage c % 3 is refilled by the next iteration's copies
    }
    // f = -c0_r sum_k c_rk G_k, combined in the tensor-core epilogue's order
    const int rb = r0 + tr * 8;
    float f[4][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int r = rb + q;
        float lam[KOBJ], c0 = 0.0f;
#pragma unroll
        for (int k = 0; k < KOBJ; ++k) lam[k] = r < a.R ? a.lambda[(int64_t)r * KOBJ + k] : 0.0f;
        if (r < a.R) c0 = a.c0[r];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            float v = 0.0f;
#pragma unroll
            for (int k = 0; k < KOBJ; ++k) v = fmaf(lam[k], acc[k][s][q], v);
            f[s][q] = v * -c0;  // the force acts on the negated coupling
        }
    }
    const float cm = a.schedule ? (__ldg(a.schedule + a.m) - a.a0) : a.cm;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int i = i0 + ti + 16 * s;
        if (i >= a.n) continue;
        float eta[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) eta[q] = 0.0f;
        if (NOISE) {
            const uint4 o = Philox4x32::block(make_uint4((uint32_t)a.m, (uint32_t)i, 0x40000000u + (uint32_t)(rb >> 3), a.round32),
                                              a.key0, a.key1);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const float2 pr = box_muller16(word_of(o, w));
                eta[2 * w] = pr.x;
                eta[2 * w + 1] = pr.y;
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int r = rb + q;
            if (r < a.R) {
                const int64_t at = (int64_t)r * np + i;
                float xv = a.x[at], yv = a.y[at];
                sb_update<NOISE>(f[s][q], cm, eta[q], a.dt, a.kappa, a.dta0, xv, yv);
                a.x[at] = xv;
                a.y[at] = yv;
                a.phi_out[at] = phi_of<VARIANT>(xv);
            }
        }
    }
}

__global__ void k_dense32_fill(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const int32_t* __restrict__ wn,
                               int64_t nnz, int32_t n, int32_t K, int32_t np, float* J)
{
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
        for (int32_t p = rowptr[i] + threadIdx.x; p < rowptr[i + 1]; p += blockDim.x)
            for (int k = 0; k < K; ++k) J[((int64_t)k * np + i) * np + col[p]] = (float)wn[(int64_t)k * nnz + p];
}

template <int VARIANT, int KOBJ, bool NOISE>
cudaError_t launch_step32(const Dense32Args& a, dim3 grid, cudaStream_t st)
{
    auto k = k_dense32_step<VARIANT, KOBJ, NOISE>;
    const size_t smem = f32_smem_bytes(KOBJ);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kF32Threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int VARIANT, bool NOISE>
cudaError_t launch_step32_k(int K, const Dense32Args& a, dim3 grid, cudaStream_t st)
{
    switch (K) {
    case 2: return launch_step32<VARIANT, 2, NOISE>(a, grid, st);
    case 3: return launch_step32<VARIANT, 3, NOISE>(a, grid, st);
    default: return launch_step32<VARIANT, 4, NOISE>(a, grid, st);
    }
}

void free_dense32(moq_dense_fp32* d)
{
    if (!d) return;
    cudaFree(d->J);
    cudaFree(d->x);
    cudaFree(d->y);
    cudaFree(d->phi[0]);
    cudaFree(d->phi[1]);
    cudaFree(d->c0);
    delete d;
}

}  // namespace
}  // namespace moq

extern "C" {

int moq_dense_fp32_create(const moq_instance* inst, int32_t max_replicas, moq_dense_fp32** out)
{
    using namespace moq;
    if (!out) return fail(MOQ_ERR_ARG, "moq_dense_fp32_create: out is NULL");
    *out = nullptr;
    if (!inst || max_replicas < 1) return fail(MOQ_ERR_ARG, "moq_dense_fp32_create: NULL instance or max_replicas < 1");
    if (inst->K > 4) return fail(MOQ_ERR_UNSUPPORTED, "moq_dense_fp32_create: K=%d > 4", inst->K);
    if (inst->n > 16384) return fail(MOQ_ERR_UNSUPPORTED, "moq_dense_fp32_create: n=%d > 16384", inst->n);
    moq_dense_fp32* d = new moq_dense_fp32();
    d->n = inst->n;
    d->K = inst->K;
    d->inst = inst;
    d->n_pad = (int)ceil_div(inst->n, kF32M) * kF32M;
    d->max_R = max_replicas;
    d->R_pad = (int)ceil_div(max_replicas, kF32N) * kF32N;
    const size_t cells = (size_t)d->R_pad * d->n_pad;
    const size_t jbytes = sizeof(float) * (size_t)d->K * d->n_pad * d->n_pad;
    cudaError_t e = cudaMalloc((void**)&d->J, jbytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->x, sizeof(float) * cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->y, sizeof(float) * cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->phi[0], sizeof(float) * cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->phi[1], sizeof(float) * cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->c0, sizeof(float) * d->R_pad);
    if (e == cudaSuccess) e = cudaMemset(d->J, 0, jbytes);
    if (e == cudaSuccess) {
        k_dense32_fill<<<std::min(d->n, 148 * 8), 128>>>(inst->rowptr, inst->col, inst->wn, inst->nnz, d->n, d->K, d->n_pad, d->J);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_dense32(d);
        return cuda_fail(e, "moq_dense_fp32_create");
    }
    *out = d;
    return MOQ_OK;
}

void moq_dense_fp32_destroy(moq_dense_fp32* d) { moq::free_dense32(d); }

int moq_sample_dense_fp32(moq_dense_fp32* d, const float* lambda, int32_t R, const moq_sample_params* p, uint64_t seed,
                          uint64_t round, uint64_t* bits, void* stream)
{
    using namespace moq;
    if (!d || !p) return fail(MOQ_ERR_ARG, "moq_sample_dense_fp32: NULL handle or params");
    if (R < 0 || R > d->max_R) return fail(MOQ_ERR_ARG, "moq_sample_dense_fp32: R=%d outside [0, max_replicas=%d]", R, d->max_R);
    if (p->steps < 0 || (p->variant != MOQ_DSB && p->variant != MOQ_BSB))
        return fail(MOQ_ERR_ARG, "moq_sample_dense_fp32: bad steps or variant");
    if (R == 0) return MOQ_OK;
    if (!lambda || !bits) return fail(MOQ_ERR_ARG, "moq_sample_dense_fp32: NULL lambda or bits");
    if (p->replica_offset != 0) return fail(MOQ_ERR_UNSUPPORTED, "moq_sample_dense_fp32: replica_offset must be 0");
    if (p->precision != MOQ_PREC_FP32) return fail(MOQ_ERR_UNSUPPORTED, "moq_sample_dense_fp32: p->precision must be MOQ_PREC_FP32");
    cudaStream_t st = as_stream(stream);
    const moq_instance* h = d->inst;
    const int np = d->n_pad, Rp = (int)ceil_div(R, kF32N) * kF32N;
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32), rnd = (uint32_t)round;
    k_dense_c0<<<R, 256, 0, st>>>(h->rowsum, h->rowptr, h->wn, h->nnz, d->n, d->K, lambda, R, d->c0);
    const int gi = (int)std::min<int64_t>(ceil_div((int64_t)Rp * np, 256), 148 * 32);
    if (p->variant == MOQ_DSB)
        k_dense_init<MOQ_DSB, float><<<gi, 256, 0, st>>>(d->n, np, R, Rp, p->init_amp, p->x_init, p->y_init, key0, key1, rnd, d->x, d->y,
                                                         d->phi[0]);
    else
        k_dense_init<MOQ_BSB, float><<<gi, 256, 0, st>>>(d->n, np, R, Rp, p->init_amp, p->x_init, p->y_init, key0, key1, rnd, d->x, d->y,
                                                         d->phi[0]);
    MOQ_CUDA_TRY(cudaMemsetAsync(d->phi[1], 0, sizeof(float) * (size_t)Rp * np, st));  // padded entries stay 0
    MOQ_LAUNCH_CHECK("moq_sample_dense_fp32 prologue");
    Dense32Args a{};
    a.J = d->J;
    a.x = d->x;
    a.y = d->y;
    a.lambda = lambda;
    a.c0 = d->c0;
    a.n = d->n;
    a.n_pad = np;
    a.R = R;
    a.schedule = p->schedule;
    a.a0 = p->a0;
    a.dt = p->dt;
    a.kappa = (p->noise_sqrt_dt ? sqrtf(p->dt) : p->dt) * p->alpha;
    a.dta0 = p->dt * p->a0;
    a.key0 = key0;
    a.key1 = key1;
    a.round32 = rnd;
    const float a0inv = p->steps > 1 ? p->a0 / (float)(p->steps - 1) : 0.0f;
    const dim3 grid(np / kF32M, Rp / kF32N);
    const bool noise = p->alpha != 0.0f;
    for (int m = 0; m < p->steps; ++m) {
        a.m = m;
        a.cm = fmaf(a0inv, (float)m, -p->a0);
        a.phi_in = d->phi[m & 1];
        a.phi_out = d->phi[(m + 1) & 1];
        cudaError_t e;
        if (p->variant == MOQ_DSB)
            e = noise ? launch_step32_k<MOQ_DSB, true>(d->K, a, grid, st) : launch_step32_k<MOQ_DSB, false>(d->K, a, grid, st);
        else
            e = noise ? launch_step32_k<MOQ_BSB, true>(d->K, a, grid, st) : launch_step32_k<MOQ_BSB, false>(d->K, a, grid, st);
        if (e != cudaSuccess) return cuda_fail(e, "moq_sample_dense_fp32 step launch");
    }
    k_dense_readout<<<R, 128, 0, st>>>(d->n, np, R, h->words, d->x, d->y, bits, p->x_out, p->y_out);
    MOQ_LAUNCH_CHECK("moq_sample_dense_fp32 readout");
    return MOQ_OK;
}

}  // extern "C"
