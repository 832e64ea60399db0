// a2..a5: noise-injected simulated bifurcation on sparse graphs ("Simulated Bifurcation
// with Gaussian noise", SB equations and Eq. NI-SB), the whole trajectory on-chip.
//
// A block owns Rb replicas of one instance for all T steps. Thread t handles spin
// i = t / Rb of replica t % Rb (spin-major), so the 32 threads of a warp read the
// same neighbour columns of different replicas: phi(x_j) lives in shared memory as
// phi[j * Rb + replica] and a warp's gathers hit consecutive words (no bank conflicts).
// Each thread keeps x_i, y_i and its row of -c0 * J(c) (at most DMAX entries) in
// registers; the only per-step traffic is the shared-memory gather and one barrier.
// The state never touches HBM: the kernel reads the CSR row and lambda once and writes
// the packed signs once.
#include <algorithm>
#include <stdlib.h>

#include "moq_common.cuh"

namespace moq {
namespace {

struct SbArgs {
    int32_t n, K, R, Rb, T, W;
    int64_t nnz;
    const int32_t* rowptr;
    const int32_t* col;
    const int32_t* wn;
    const int64_t* rowsum;
    const float* lambda;
    float dt, a0, alpha, init_amp, inv_Tm1, sqrt_dt;
    int32_t noise_sqrt_dt;
    const float* schedule;
    const float* x_init;
    const float* y_init;
    float* x_out;
    float* y_out;
    uint32_t key0, key1, round32;
    uint64_t* bits;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline size_t sb_smem_bytes(int n, int Rb, int W)
{
    return align_up(sizeof(float) * 2 * (size_t)n * Rb + sizeof(unsigned) * 2 * Rb, 16) + sizeof(unsigned long long) * (size_t)Rb * W;
}

template <int VARIANT, int DMAX, bool NOISE>
__global__ void __launch_bounds__(1024) k_sb_sparse(const SbArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n, Rb = a.Rb;
    const int nt = n * Rb;  // == blockDim.x
    float* phi_a = reinterpret_cast<float*>(smem_raw);
    float* phi_b = phi_a + nt;
    unsigned* red = reinterpret_cast<unsigned*>(phi_b + nt);  // 2 * Rb
    unsigned long long* wb = reinterpret_cast<unsigned long long*>(smem_raw + align_up(sizeof(float) * 2 * nt + sizeof(unsigned) * 2 * Rb, 16));

    const int tid = threadIdx.x;
    const int i = tid / Rb;       // spin
    const int lr = tid - i * Rb;  // replica within the block
    const int r = blockIdx.x * Rb + lr;
    const bool active = r < a.R;
    const int rs = active ? r : 0;

    // weight vector c = lambda_r (Eq. H_total)
    float lam[kMaxK];
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) lam[k] = (k < a.K) ? a.lambda[(int64_t)rs * a.K + k] : 0.0f;

    // row i of J(c) = sum_k c_k J^(k), kept in registers
    const int p0 = a.rowptr[i];
    const int deg = a.rowptr[i + 1] - p0;
    float jc[DMAX];
    int nb[DMAX];
    float sabs = 0.0f;
#pragma unroll
    for (int d = 0; d < DMAX; ++d) {
        float v = 0.0f;
        int c = i;
        if (d < deg) {
            const int p = p0 + d;
            c = a.col[p];
            for (int k = 0; k < a.K; ++k) v = fmaf(lam[k], (float)a.wn[(int64_t)k * a.nnz + p], v);
        }
        jc[d] = v;
        nb[d] = c * Rb + lr;
        sabs += fabsf(v);
    }
    float srow = 0.0f;
    for (int k = 0; k < a.K; ++k) srow = fmaf(lam[k], (float)a.rowsum[(int64_t)i * a.K + k], srow);

    // c0 = 1 / max_i |sum_j J(c)_ij| per replica (fallbacks: sum |J(c)_ij|, then 1);
    // non-negative floats order like their bit patterns, so an integer max reduces them
    if (tid < 2 * Rb) red[tid] = 0u;
    __syncthreads();
    atomicMax(&red[lr], __float_as_uint(fabsf(srow)));
    atomicMax(&red[Rb + lr], __float_as_uint(sabs));
    __syncthreads();
    const float mx = __uint_as_float(red[lr]), mxa = __uint_as_float(red[Rb + lr]);
    const float c0 = mx > 0.0f ? 1.0f / mx : (mxa > 0.0f ? 1.0f / mxa : 1.0f);
#pragma unroll
    for (int d = 0; d < DMAX; ++d) jc[d] *= -c0;  // the force acts on the negated coupling

    // start state
    float x, y;
    if (a.x_init) {
        x = active ? a.x_init[(int64_t)r * n + i] : 0.0f;
        y = (active && a.y_init) ? a.y_init[(int64_t)r * n + i] : 0.0f;
    } else {
        const uint4 o = Philox4x32::block(make_uint4(0xFFFFFFFFu, (uint32_t)i, (uint32_t)r, a.round32), a.key0, a.key1);
        x = __fmul_rn(a.init_amp, signed_unit(o.x));
        y = __fmul_rn(a.init_amp, signed_unit(o.y));
    }

    float* cur = phi_a;
    float* nxt = phi_b;
    cur[tid] = (VARIANT == MOQ_DSB) ? (x >= 0.0f ? 1.0f : -1.0f) : x;
    __syncthreads();

    const float dta0 = a.dt * a.a0;
    float z0 = 0.0f, z1 = 0.0f, z2 = 0.0f, z3 = 0.0f;
    for (int m = 0; m < a.T; ++m) {
        if (NOISE) {
            if ((m & 3) == 0) {
                const uint4 o = Philox4x32::block(make_uint4((uint32_t)(m >> 2), (uint32_t)i, (uint32_t)r, a.round32), a.key0, a.key1);
                const float2 p = box_muller(o.x, o.y), q = box_muller(o.z, o.w);
                z0 = p.x; z1 = p.y; z2 = q.x; z3 = q.y;
            } else {
                z0 = z1; z1 = z2; z2 = z3;
            }
        }
        const float am = a.schedule ? __ldg(a.schedule + m) : a.a0 * (float)m * a.inv_Tm1;
        float f = 0.0f;
#pragma unroll
        for (int d = 0; d < DMAX; ++d)
            if (d < deg) f = fmaf(jc[d], cur[nb[d]], f);
        const float drift = fmaf(-(a.a0 - am), x, f);
        if (NOISE) {
            const float nz = a.alpha * z0;
            y = a.noise_sqrt_dt ? fmaf(a.sqrt_dt, nz, fmaf(a.dt, drift, y)) : fmaf(a.dt, drift + nz, y);
        } else {
            y = fmaf(a.dt, drift, y);
        }
        x = fmaf(dta0, y, x);
        if (fabsf(x) > 1.0f) {  // inelastic wall
            x = copysignf(1.0f, x);
            y = 0.0f;
        }
        nxt[tid] = (VARIANT == MOQ_DSB) ? (x >= 0.0f ? 1.0f : -1.0f) : x;
        __syncthreads();
        float* t = cur;
        cur = nxt;
        nxt = t;
    }

    // readout s_i = sgn(x_i), sgn(0) = +1; bit set for s_i = -1
    const int W = a.W;
    for (int t = tid; t < Rb * W; t += blockDim.x) wb[t] = 0ull;
    __syncthreads();
    if (x < 0.0f) atomicOr(&wb[lr * W + (i >> 6)], 1ull << (i & 63));
    __syncthreads();
    for (int t = tid; t < Rb * W; t += blockDim.x) {
        const int r2 = blockIdx.x * Rb + t / W;
        if (r2 < a.R) a.bits[(int64_t)r2 * W + (t % W)] = wb[t];
    }
    if (active) {
        if (a.x_out) a.x_out[(int64_t)r * n + i] = x;
        if (a.y_out) a.y_out[(int64_t)r * n + i] = y;
    }
}

template <int VARIANT, int DMAX>
cudaError_t launch_noise(const SbArgs& a, bool noise, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    if (noise) {
        auto k = k_sb_sparse<VARIANT, DMAX, true>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, block, smem, st>>>(a);
    } else {
        auto k = k_sb_sparse<VARIANT, DMAX, false>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, block, smem, st>>>(a);
    }
    return cudaGetLastError();
}

template <int VARIANT>
cudaError_t launch_variant(const SbArgs& a, int dmax, bool noise, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    switch (dmax) {
    case 4: return launch_noise<VARIANT, 4>(a, noise, grid, block, smem, st);
    case 8: return launch_noise<VARIANT, 8>(a, noise, grid, block, smem, st);
    default: return launch_noise<VARIANT, 16>(a, noise, grid, block, smem, st);
    }
}

// Replicas per block: the spin-major layout wants whole warps of one spin (Rb up to 32)
// but also enough blocks to cover the 148 SMs when R is small.
int choose_rb(int n, int R)
{
    int rb = std::max(1, std::min(32, 1024 / n));
    if (const char* env = getenv("MOQ_SB_RB")) {
        int v = atoi(env);
        if (v >= 1) rb = std::min(v, 1024 / n);
    }
    const int spread = (int)std::max<int64_t>(1, ceil_div(R, 148));
    rb = std::max(1, std::min(rb, spread));
    return rb;
}

}  // namespace
}  // namespace moq

extern "C" int moq_sample(const moq_instance* inst, const float* lambda, int32_t R, const moq_sample_params* p,
                          uint64_t seed, uint64_t round, uint64_t* bits, void* stream)
{
    using namespace moq;
    if (!inst || !p) return fail(MOQ_ERR_ARG, "moq_sample: NULL instance or params");
    if (R < 0) return fail(MOQ_ERR_ARG, "moq_sample: R < 0");
    if (p->steps < 0) return fail(MOQ_ERR_ARG, "moq_sample: steps < 0");
    if (p->variant != MOQ_DSB && p->variant != MOQ_BSB) return fail(MOQ_ERR_ARG, "moq_sample: unknown variant %d", p->variant);
    if (R == 0) return MOQ_OK;
    if (!lambda || !bits) return fail(MOQ_ERR_ARG, "moq_sample: NULL lambda or bits");
    if (inst->n > 1024) return fail(MOQ_ERR_UNSUPPORTED, "moq_sample: n=%d > 1024 is not supported by the on-chip sampler", inst->n);
    if (inst->max_degree > 16) return fail(MOQ_ERR_UNSUPPORTED, "moq_sample: max degree %d > 16", inst->max_degree);

    SbArgs a{};
    a.n = inst->n;
    a.K = inst->K;
    a.R = R;
    a.T = p->steps;
    a.W = inst->words;
    a.nnz = inst->nnz;
    a.rowptr = inst->rowptr;
    a.col = inst->col;
    a.wn = inst->wn;
    a.rowsum = inst->rowsum;
    a.lambda = lambda;
    a.dt = p->dt;
    a.a0 = p->a0;
    a.alpha = p->alpha;
    a.init_amp = p->init_amp;
    a.inv_Tm1 = p->steps > 1 ? 1.0f / (float)(p->steps - 1) : 0.0f;
    a.sqrt_dt = sqrtf(p->dt);
    a.noise_sqrt_dt = p->noise_sqrt_dt;
    a.schedule = p->schedule;
    a.x_init = p->x_init;
    a.y_init = p->y_init;
    a.x_out = p->x_out;
    a.y_out = p->y_out;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.round32 = (uint32_t)round;
    a.bits = bits;
    a.Rb = choose_rb(a.n, R);
    const int dmax = inst->max_degree <= 4 ? 4 : (inst->max_degree <= 8 ? 8 : 16);
    const dim3 block(a.n * a.Rb), grid((unsigned)ceil_div(R, a.Rb));
    const size_t smem = sb_smem_bytes(a.n, a.Rb, a.W);
    const bool noise = p->alpha != 0.0f;
    cudaError_t e = (p->variant == MOQ_DSB) ? launch_variant<MOQ_DSB>(a, dmax, noise, grid, block, smem, as_stream(stream))
                                            : launch_variant<MOQ_BSB>(a, dmax, noise, grid, block, smem, as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, "moq_sample launch");
    return MOQ_OK;
}
