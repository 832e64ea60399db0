// a2..a5: noise-injected simulated bifurcation on sparse graphs ("Simulated Bifurcation
// with Gaussian noise", SB equations and Eq. NI-SB), the whole trajectory on-chip.
//
// A block owns Rb replicas of one instance for all T steps. Thread t handles spin
// i = t / Rb of replica t % Rb (spin-major), so the threads of a warp read the same
// neighbour columns of different replicas: phi(x_j) lives in shared memory as
// phi[j * Rb + replica] and a warp's gathers hit consecutive words. Each thread keeps
// x_i, y_i and its row of -c0 * J(c) (DMAX entries, zero-padded) in registers; per step
// the only memory traffic is the shared-memory gather, one store and one barrier.
// The step loop is unrolled by eight: one Philox4x32-10 block gives the eight Gaussians
// of eight consecutive steps (two per word), and the two phi buffers alternate at a fixed
// offset.
// HBM sees the CSR rows and lambda once (in) and the packed signs once (out).
#include <algorithm>
#include <stdlib.h>

#include <cuda_fp16.h>

#include "gather_layout.cuh"
#include "sb_common.cuh"

namespace moq {
namespace {

constexpr int kPhiStride = 1024;  // floats per phi buffer (a block has at most 1024 threads)

struct SbArgs {
    int32_t n, K, R, Rb, T, W;
    int64_t nnz;
    const int32_t* rowptr;
    const int32_t* col;
    const int32_t* slot_spin;  // slot -> spin (gather_layout.cuh)
    const int32_t* spin_slot;  // spin -> slot
    const int32_t* wn;
    const int64_t* rowsum;
    const float* lambda;
    float dt, a0, init_amp;
    float kappa;  // coefficient of eta in the y update: dt*alpha (Euler) or sqrt(dt)*alpha
    float a0inv;  // a0 / (T - 1): the linear pump gives a_m - a0 = a0inv * m - a0
    const float* schedule;
    const float* x_init;
    const float* y_init;
    float* x_out;
    float* y_out;
    uint32_t key0, key1, round32, rep_off;
    uint64_t* bits;
    uint32_t rk0[10], rk1[10];  // Philox round keys: key0 + r * W0, key1 + r * W1
};

// The noise block of the samplers' step loops: Philox4x32-10 with the round keys taken from
// the kernel parameters (constant operands) instead of bumped per round; the same words as
// Philox4x32::block(c, key0, key1)
__device__ __forceinline__ uint4 philox_rk(uint4 c, const SbArgs& a)
{
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        const uint64_t p0 = (uint64_t)Philox4x32::kM0 * c.x;
        const uint64_t p1 = (uint64_t)Philox4x32::kM1 * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ a.rk0[rnd], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ a.rk1[rnd], (uint32_t)p0);
    }
    return c;
}

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Pump: 0 = caller's schedule array, 1 = linear pump computed per step, 2 = linear pump
// read from a per-block table of the T values (one shared-memory load per step instead of
// a multiply-add and a counter update; the same single-rounding formula fills it)
constexpr int kPumpSchedule = 0, kPumpInline = 1, kPumpTable = 2;
// The pair and FP16 kernels also come register-capped for two resident blocks of up to 640
// threads (a pump code + 3; the table pump only serves blocks of up to 256 threads): where the
// 60-register build fits one such block per SM, the capped build fits two, which hides the
// per-step barrier (FP16, n = 600: 4.16 against 4.70 ms per launch); the host takes it only where
// the occupancy API says it keeps more threads resident (n = 450 fits two blocks either way, and
// the capped build's spills then cost 4 %).
constexpr int kPumpScheduleCap = 3, kPumpInlineCap = 4;
__host__ __device__ constexpr int pump_base(int p) { return p >= 3 ? p - 3 : p; }
constexpr int kCapThreads = 640;
constexpr int kPumpTableMax = 8192;
constexpr int kPumpTableMaxThreads = 256;

__host__ __device__ inline size_t sb_smem_bytes(int Rb, int W, int pump_table_steps)
{
    return sizeof(float) * 2 * kPhiStride + align_up(sizeof(unsigned) * 2 * Rb, 16) +
           align_up(sizeof(unsigned long long) * (size_t)Rb * W, 16) + sizeof(float) * (size_t)pump_table_steps;
}

// One Euler step of one spin: force from the shared-memory phi buffer `rd`, symplectic
// update, inelastic wall, phi into `wr`, then the block barrier.
template <int VARIANT, int DMAX, bool NOISE>
__device__ __forceinline__ void sb_step(const float* rd, float* wr, int tid, const float (&jc)[DMAX],
                                        const int (&nb)[DMAX], float cm, float eta, float dt, float kappa, float dta0,
                                        float& x, float& y)
{
    float f = 0.0f;  // c0 sum_j (-J(c)_ij) phi(x_j)
#pragma unroll
    for (int d = 0; d < DMAX; ++d) f = fmaf(jc[d], rd[nb[d]], f);
    sb_update<NOISE>(f, cm, eta, dt, kappa, dta0, x, y);
    wr[tid] = phi_of<VARIANT>(x);
    __syncthreads();
}

template <int VARIANT, int DMAX, bool NOISE, int PUMP>
__global__ void __launch_bounds__(1024) k_sb_sparse(const SbArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n, Rb = a.Rb;
    float* phiA = reinterpret_cast<float*>(smem_raw);
    float* phiB = phiA + kPhiStride;
    unsigned* red = reinterpret_cast<unsigned*>(phiB + kPhiStride);  // 2 * Rb
    unsigned long long* wb = reinterpret_cast<unsigned long long*>(smem_raw + sizeof(float) * 2 * kPhiStride +
                                                                   align_up(sizeof(unsigned) * 2 * Rb, 16));
    float* pump_t = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(wb) +
                                             align_up(sizeof(unsigned long long) * (size_t)Rb * a.W, 16));

    const int tid = threadIdx.x;
    const int slot = tid / Rb;         // spins sit in slots by decreasing degree
    const int lr = tid - slot * Rb;    // replica within the block
    const int i = a.slot_spin[slot];   // spin
    const int r = blockIdx.x * Rb + lr;
    const bool active = r < a.R;
    const int rs = active ? r : 0;

    // weight vector c = lambda_r (Eq. H_total)
    float lam[kMaxK];
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) lam[k] = (k < a.K) ? a.lambda[(int64_t)rs * a.K + k] : 0.0f;

    // row i of J(c) = sum_k c_k J^(k) in registers, zero-padded to DMAX entries
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
#pragma unroll
            for (int k = 0; k < kMaxK; ++k)  // constant indices keep lam in registers
                if (k < a.K) v = fmaf(lam[k], (float)a.wn[(int64_t)k * a.nnz + p], v);
        }
        jc[d] = v;
        nb[d] = a.spin_slot[c] * Rb + lr;
        sabs += fabsf(v);
    }
    float srow = 0.0f;
#pragma unroll
    for (int k = 0; k < kMaxK; ++k)
        if (k < a.K) srow = fmaf(lam[k], (float)a.rowsum[(int64_t)i * a.K + k], srow);

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

    // start state (+0.0f turns a caller's -0 into +0, which phi_of relies on)
    float x, y;
    if (a.x_init) {
        x = (active ? a.x_init[(int64_t)r * n + i] : 0.0f) + 0.0f;
        y = (active && a.y_init) ? a.y_init[(int64_t)r * n + i] : 0.0f;
    } else {
        const uint4 o = Philox4x32::block(make_uint4(0xFFFFFFFFu, (uint32_t)i, a.rep_off + (uint32_t)r, a.round32), a.key0, a.key1);
        x = __fmul_rn(a.init_amp, signed_unit(o.x)) + 0.0f;
        y = __fmul_rn(a.init_amp, signed_unit(o.y));
    }
    phiA[tid] = phi_of<VARIANT>(x);
    __syncthreads();

    const float dt = a.dt, kappa = a.kappa, dta0 = a.dt * a.a0, a0 = a.a0, a0inv = a.a0inv;
    const float* sched = a.schedule;
    const int T = a.T;
    if (PUMP == kPumpTable) {
        for (int q = tid; q < T; q += blockDim.x) pump_t[q] = fmaf(a0inv, (float)q, -a0);
        __syncthreads();
    }
    auto cm_at = [&](int m, float mf) -> float {
        return PUMP == kPumpTable ? pump_t[m] : (PUMP == kPumpInline ? fmaf(a0inv, mf, -a0) : (__ldg(sched + m) - a0));
    };
    // one Philox4x32-10 block per eight steps: word q gives the Gaussians of steps 2q, 2q+1
    auto block8 = [&](int m) -> uint4 {
        return NOISE ? philox_rk(make_uint4((uint32_t)(m >> 3), (uint32_t)i, a.rep_off + (uint32_t)r, a.round32), a)
                     : make_uint4(0u, 0u, 0u, 0u);
    };
    // the Gaussians of four consecutive steps from two words
    auto noise4 = [&](uint32_t wa, uint32_t wb, float& e0, float& e1, float& e2, float& e3) {
        if (NOISE) {
            const float2 p = box_muller16(wa), q = box_muller16(wb);
            e0 = p.x; e1 = p.y; e2 = q.x; e3 = q.y;
        }
    };
    auto four_steps = [&](int m, float mf, float e0, float e1, float e2, float e3) {
        sb_step<VARIANT, DMAX, NOISE>(phiA, phiB, tid, jc, nb, cm_at(m, mf), e0, dt, kappa, dta0, x, y);
        sb_step<VARIANT, DMAX, NOISE>(phiB, phiA, tid, jc, nb, cm_at(m + 1, mf + 1.0f), e1, dt, kappa, dta0, x, y);
        sb_step<VARIANT, DMAX, NOISE>(phiA, phiB, tid, jc, nb, cm_at(m + 2, mf + 2.0f), e2, dt, kappa, dta0, x, y);
        sb_step<VARIANT, DMAX, NOISE>(phiB, phiA, tid, jc, nb, cm_at(m + 3, mf + 3.0f), e3, dt, kappa, dta0, x, y);
    };
    // the Gaussians of steps m..m+3 (m a multiple of 4): words (x, y) or (z, w) of the block
    auto noise_at = [&](int m, float& e0, float& e1, float& e2, float& e3) {
        if (NOISE) {
            const uint4 o = block8(m);
            noise4((m & 4) ? o.z : o.x, (m & 4) ? o.w : o.y, e0, e1, e2, e3);
        }
    };
    int m = 0;
    float mf = 0.0f;
    if (NOISE) {
        for (; m + 8 <= T; m += 8) {
            const uint4 o = block8(m);
            float e0, e1, e2, e3;
            noise4(o.x, o.y, e0, e1, e2, e3);
            four_steps(m, mf, e0, e1, e2, e3);
            noise4(o.z, o.w, e0, e1, e2, e3);
            four_steps(m + 4, mf + 4.0f, e0, e1, e2, e3);
            mf += 8.0f;
        }
    }
    // without noise the whole run; with noise at most one pass (T mod 8 >= 4)
    for (; m + 4 <= T; m += 4) {
        float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f, e3 = 0.0f;
        noise_at(m, e0, e1, e2, e3);
        four_steps(m, mf, e0, e1, e2, e3);
        mf += 4.0f;
    }
    if (m < T) {  // the last T mod 4 steps (uniform over the block)
        float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f, e3 = 0.0f;
        noise_at(m, e0, e1, e2, e3);
        sb_step<VARIANT, DMAX, NOISE>(phiA, phiB, tid, jc, nb, cm_at(m, mf), e0, dt, kappa, dta0, x, y);
        if (m + 1 < T) sb_step<VARIANT, DMAX, NOISE>(phiB, phiA, tid, jc, nb, cm_at(m + 1, mf + 1.0f), e1, dt, kappa, dta0, x, y);
        if (m + 2 < T) sb_step<VARIANT, DMAX, NOISE>(phiA, phiB, tid, jc, nb, cm_at(m + 2, mf + 2.0f), e2, dt, kappa, dta0, x, y);
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

template <int VARIANT, int DMAX, bool NOISE, int PUMP>
cudaError_t launch_one(const SbArgs& a, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    auto k = k_sb_sparse<VARIANT, DMAX, NOISE, PUMP>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <int VARIANT, int DMAX, bool NOISE>
cudaError_t launch_pump(const SbArgs& a, int pump, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    switch (pump) {
    case kPumpTable: return launch_one<VARIANT, DMAX, NOISE, kPumpTable>(a, grid, block, smem, st);
    case kPumpInline: return launch_one<VARIANT, DMAX, NOISE, kPumpInline>(a, grid, block, smem, st);
    default: return launch_one<VARIANT, DMAX, NOISE, kPumpSchedule>(a, grid, block, smem, st);
    }
}

template <int VARIANT, int DMAX>
cudaError_t launch_flags(const SbArgs& a, bool noise, int pump, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    return noise ? launch_pump<VARIANT, DMAX, true>(a, pump, grid, block, smem, st)
                 : launch_pump<VARIANT, DMAX, false>(a, pump, grid, block, smem, st);
}

template <int VARIANT>
cudaError_t launch_variant(const SbArgs& a, int dmax, bool noise, int pump, dim3 grid, dim3 block, size_t smem,
                           cudaStream_t st)
{
    switch (dmax) {
    case 3: return launch_flags<VARIANT, 3>(a, noise, pump, grid, block, smem, st);
    case 4: return launch_flags<VARIANT, 4>(a, noise, pump, grid, block, smem, st);
    case 8: return launch_flags<VARIANT, 8>(a, noise, pump, grid, block, smem, st);
    default: return launch_flags<VARIANT, 16>(a, noise, pump, grid, block, smem, st);
    }
}


// ---- two replicas per thread ------------------------------------------------------------
// The same dynamics with each thread running spin i of two replicas (2q, 2q + 1) of its
// block: the neighbour gathers fetch both replicas' phi in one 8-byte load (phi is stored
// as a float2 per slot and pair), and the pump value, the barrier and the loop control are
// shared by two updates. Each replica's arithmetic and noise counters are those of
// k_sb_sparse, so both kernels give the same bits; the host takes this form when it keeps
// more replicas in flight per SM (register and block limits, from the occupancy API).
// Both replicas' arithmetic runs in packed two-lane FP32 instructions (jc[d] holds the
// pair's couplings of neighbour d, x and y the pair's states), lane by lane the scalar
// arithmetic of k_sb_sparse. (Measured at n = 42, R = 16384, T = 2000: 1.55 against 1.63 ms
// per launch for the scalar pair; packing the Box-Muller pairs as well, with the pump value
// stored twice, measured 1.58 ms.)
template <int VARIANT, int DMAX, bool NOISE>
__device__ __forceinline__ void sb_step2(const float2* rd, float2* wr, int tid, const float2 (&jc)[DMAX], const int (&nb)[DMAX],
                                         float cm, float e0, float e1, float2 dt, float2 kappa, float2 dta0, float2& x, float2& y)
{
    float2 f = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int d = 0; d < DMAX; ++d) f = __ffma2_rn(jc[d], rd[nb[d]], f);
    sb_update2<NOISE>(f, make_float2(cm, cm), make_float2(e0, e1), dt, kappa, dta0, x, y);
    wr[tid] = make_float2(phi_of<VARIANT>(x.x), phi_of<VARIANT>(x.y));
    __syncthreads();
}

__host__ __device__ inline size_t sb_smem_bytes2(int Rb, int W, int pump_table_steps)
{
    return sizeof(float) * 4 * kPhiStride + align_up(sizeof(unsigned) * 2 * Rb, 16) +
           align_up(sizeof(unsigned long long) * (size_t)Rb * W, 16) + sizeof(float) * (size_t)pump_table_steps;
}

// Rows of J(c) of spin i for the replica pair (r0, r0 + 1), before the c0 scaling: the
// couplings of its neighbours (zero past its degree), their phi indices spin_slot[c] * Rp + lp,
// and the sums that c0 is reduced from (sabs = sum_d |J(c)_id|, srow = sum_j J(c)_ij).
template <int DMAX>
__device__ __forceinline__ void pair_rows(const SbArgs& a, int i, int lp, int Rp, int r0, float (&jc0)[DMAX], float (&jc1)[DMAX],
                                          int (&nb)[DMAX], float& sabs0, float& sabs1, float& srow0, float& srow1)
{
    const int r1 = r0 + 1;
    const int rs0 = r0 < a.R ? r0 : 0, rs1 = r1 < a.R ? r1 : 0;
    float lam0[kMaxK], lam1[kMaxK];
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
        lam0[k] = (k < a.K) ? a.lambda[(int64_t)rs0 * a.K + k] : 0.0f;
        lam1[k] = (k < a.K) ? a.lambda[(int64_t)rs1 * a.K + k] : 0.0f;
    }
    const int p0 = a.rowptr[i];
    const int deg = a.rowptr[i + 1] - p0;
    sabs0 = 0.0f;
    sabs1 = 0.0f;
#pragma unroll
    for (int d = 0; d < DMAX; ++d) {
        float v0 = 0.0f, v1 = 0.0f;
        int c = i;
        if (d < deg) {
            const int p = p0 + d;
            c = a.col[p];
#pragma unroll
            for (int k = 0; k < kMaxK; ++k)
                if (k < a.K) {
                    const float w = (float)a.wn[(int64_t)k * a.nnz + p];
                    v0 = fmaf(lam0[k], w, v0);
                    v1 = fmaf(lam1[k], w, v1);
                }
        }
        jc0[d] = v0;
        jc1[d] = v1;
        nb[d] = a.spin_slot[c] * Rp + lp;
        sabs0 += fabsf(v0);
        sabs1 += fabsf(v1);
    }
    srow0 = 0.0f;
    srow1 = 0.0f;
#pragma unroll
    for (int k = 0; k < kMaxK; ++k)
        if (k < a.K) {
            const float w = (float)a.rowsum[(int64_t)i * a.K + k];
            srow0 = fmaf(lam0[k], w, srow0);
            srow1 = fmaf(lam1[k], w, srow1);
        }
}

// c0 of a replica from its block maxima of |srow| and sabs, and the rows scaled by -c0
__device__ __forceinline__ float c0_of(float mx, float mxa) { return mx > 0.0f ? 1.0f / mx : (mxa > 0.0f ? 1.0f / mxa : 1.0f); }

// Start state of spin i for the pair: the given one, or init_amp times uniforms on [-1, 1)
__device__ __forceinline__ void pair_start(const SbArgs& a, int i, int r0, float& x0, float& y0, float& x1, float& y1)
{
    const int n = a.n, r1 = r0 + 1;
    const bool act0 = r0 < a.R, act1 = r1 < a.R;
    if (a.x_init) {
        x0 = (act0 ? a.x_init[(int64_t)r0 * n + i] : 0.0f) + 0.0f;
        y0 = (act0 && a.y_init) ? a.y_init[(int64_t)r0 * n + i] : 0.0f;
        x1 = (act1 ? a.x_init[(int64_t)r1 * n + i] : 0.0f) + 0.0f;
        y1 = (act1 && a.y_init) ? a.y_init[(int64_t)r1 * n + i] : 0.0f;
    } else {
        const uint4 o0 = Philox4x32::block(make_uint4(0xFFFFFFFFu, (uint32_t)i, a.rep_off + (uint32_t)r0, a.round32), a.key0, a.key1);
        const uint4 o1 = Philox4x32::block(make_uint4(0xFFFFFFFFu, (uint32_t)i, a.rep_off + (uint32_t)r1, a.round32), a.key0, a.key1);
        x0 = __fmul_rn(a.init_amp, signed_unit(o0.x)) + 0.0f;
        y0 = __fmul_rn(a.init_amp, signed_unit(o0.y));
        x1 = __fmul_rn(a.init_amp, signed_unit(o1.x)) + 0.0f;
        y1 = __fmul_rn(a.init_amp, signed_unit(o1.y));
    }
}

// Set-up of the replica pair (r0, r0 + 1) on spin i, shared by the FP32 and FP16 pair
// kernels: both rows of -c0 J(c) in FP32 (c0 reduced over the block's replicas in red[]:
// 4 * Rp words), the neighbours' phi indices and the start state. Contains two block barriers.
template <int DMAX>
__device__ __forceinline__ void pair_setup(const SbArgs& a, int tid, int i, int lp, int Rp, int r0, unsigned* red,
                                           float (&jc0)[DMAX], float (&jc1)[DMAX], int (&nb)[DMAX], float& x0, float& y0,
                                           float& x1, float& y1)
{
    const int Rb = 2 * Rp;
    float sabs0, sabs1, srow0, srow1;
    pair_rows<DMAX>(a, i, lp, Rp, r0, jc0, jc1, nb, sabs0, sabs1, srow0, srow1);
    for (int q = tid; q < 2 * Rb; q += blockDim.x) red[q] = 0u;  // 2 Rb = 4 Rp may exceed n Rp threads (n < 4)
    __syncthreads();
    atomicMax(&red[2 * lp], __float_as_uint(fabsf(srow0)));
    atomicMax(&red[2 * lp + 1], __float_as_uint(fabsf(srow1)));
    atomicMax(&red[Rb + 2 * lp], __float_as_uint(sabs0));
    atomicMax(&red[Rb + 2 * lp + 1], __float_as_uint(sabs1));
    __syncthreads();
    const float c00 = c0_of(__uint_as_float(red[2 * lp]), __uint_as_float(red[Rb + 2 * lp]));
    const float c01 = c0_of(__uint_as_float(red[2 * lp + 1]), __uint_as_float(red[Rb + 2 * lp + 1]));
#pragma unroll
    for (int d = 0; d < DMAX; ++d) {
        jc0[d] *= -c00;
        jc1[d] *= -c01;
    }
    pair_start(a, i, r0, x0, y0, x1, y1);
}

template <int VARIANT, int DMAX, bool NOISE, int PUMP>
__global__ void __launch_bounds__(PUMP >= 3 ? kCapThreads : 1024, PUMP >= 3 ? 2 : 1) k_sb_sparse2(const SbArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n, Rb = a.Rb, Rp = a.Rb >> 1;
    float2* phiA = reinterpret_cast<float2*>(smem_raw);
    float2* phiB = phiA + kPhiStride;
    unsigned* red = reinterpret_cast<unsigned*>(phiB + kPhiStride);  // 2 * Rb
    unsigned long long* wb = reinterpret_cast<unsigned long long*>(smem_raw + sizeof(float) * 4 * kPhiStride +
                                                                   align_up(sizeof(unsigned) * 2 * Rb, 16));
    float* pump_t = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(wb) +
                                             align_up(sizeof(unsigned long long) * (size_t)Rb * a.W, 16));
    const int tid = threadIdx.x;
    const int slot = tid / Rp;
    const int lp = tid - slot * Rp;
    const int i = a.slot_spin[slot];
    const int r0 = blockIdx.x * Rb + 2 * lp, r1 = r0 + 1;
    const bool act0 = r0 < a.R, act1 = r1 < a.R;
    float jc0[DMAX], jc1[DMAX];
    int nb[DMAX];
    float x0, y0, x1, y1;
    pair_setup<DMAX>(a, tid, i, lp, Rp, r0, red, jc0, jc1, nb, x0, y0, x1, y1);
    float2 jc[DMAX];
#pragma unroll
    for (int d = 0; d < DMAX; ++d) jc[d] = make_float2(jc0[d], jc1[d]);
    phiA[tid] = make_float2(phi_of<VARIANT>(x0), phi_of<VARIANT>(x1));
    __syncthreads();
    float2 xs = make_float2(x0, x1), ys = make_float2(y0, y1);
    const float2 dt2 = make_float2(a.dt, a.dt), kappa2 = make_float2(a.kappa, a.kappa);
    const float2 dta02 = make_float2(a.dt * a.a0, a.dt * a.a0);
    const float a0 = a.a0, a0inv = a.a0inv;
    const float* sched = a.schedule;
    const int T = a.T;
    if (pump_base(PUMP) == kPumpTable) {
        for (int q = tid; q < T; q += blockDim.x) pump_t[q] = fmaf(a0inv, (float)q, -a0);
        __syncthreads();
    }
    auto cm_at = [&](int m, float mf) -> float {
        return pump_base(PUMP) == kPumpTable ? pump_t[m] : (pump_base(PUMP) == kPumpInline ? fmaf(a0inv, mf, -a0) : (__ldg(sched + m) - a0));
    };
    auto block8 = [&](int m, int r) -> uint4 {
        return NOISE ? philox_rk(make_uint4((uint32_t)(m >> 3), (uint32_t)i, a.rep_off + (uint32_t)r, a.round32), a)
                     : make_uint4(0u, 0u, 0u, 0u);
    };
    auto noise4 = [&](uint32_t wa, uint32_t wbb, float (&e)[4]) {
        if (NOISE) {
            const float2 p = box_muller16(wa), q = box_muller16(wbb);
            e[0] = p.x; e[1] = p.y; e[2] = q.x; e[3] = q.y;
        }
    };
    auto step = [&](const float2* rd, float2* wr, float cm, float e0, float e1) {
        sb_step2<VARIANT, DMAX, NOISE>(rd, wr, tid, jc, nb, cm, e0, e1, dt2, kappa2, dta02, xs, ys);
    };
    auto four_steps = [&](int m, float mf, const float (&e)[4], const float (&g)[4]) {
        step(phiA, phiB, cm_at(m, mf), e[0], g[0]);
        step(phiB, phiA, cm_at(m + 1, mf + 1.0f), e[1], g[1]);
        step(phiA, phiB, cm_at(m + 2, mf + 2.0f), e[2], g[2]);
        step(phiB, phiA, cm_at(m + 3, mf + 3.0f), e[3], g[3]);
    };
    auto noise_at = [&](int m, float (&e)[4], float (&g)[4]) {
        if (NOISE) {
            const uint4 o = block8(m, r0), q = block8(m, r1);
            noise4((m & 4) ? o.z : o.x, (m & 4) ? o.w : o.y, e);
            noise4((m & 4) ? q.z : q.x, (m & 4) ? q.w : q.y, g);
        }
    };
    int m = 0;
    float mf = 0.0f;
    if (NOISE && PUMP < 3) {
        // the Gaussians two steps at a time (one Box-Muller pair per replica; measured 1.526
        // against 1.530 ms per launch at n = 42 for four steps at a time; the register-capped
        // builds keep four at a time, 4.69 against 4.72 ms at n = 600)
        auto two_steps = [&](int mm, float mmf, uint32_t wa, uint32_t wbb) {
            const float2 pa = box_muller16(wa), pb = box_muller16(wbb);
            step(phiA, phiB, cm_at(mm, mmf), pa.x, pb.x);
            step(phiB, phiA, cm_at(mm + 1, mmf + 1.0f), pa.y, pb.y);
        };
        for (; m + 8 <= T; m += 8) {
            const uint4 o = block8(m, r0), q = block8(m, r1);
            two_steps(m, mf, o.x, q.x);
            two_steps(m + 2, mf + 2.0f, o.y, q.y);
            two_steps(m + 4, mf + 4.0f, o.z, q.z);
            two_steps(m + 6, mf + 6.0f, o.w, q.w);
            mf += 8.0f;
        }
    } else if (NOISE) {
        for (; m + 8 <= T; m += 8) {
            const uint4 o = block8(m, r0), q = block8(m, r1);
            float e[4], g[4];
            noise4(o.x, o.y, e);
            noise4(q.x, q.y, g);
            four_steps(m, mf, e, g);
            noise4(o.z, o.w, e);
            noise4(q.z, q.w, g);
            four_steps(m + 4, mf + 4.0f, e, g);
            mf += 8.0f;
        }
    }
    for (; m + 4 <= T; m += 4) {
        float e[4] = {0.0f, 0.0f, 0.0f, 0.0f}, g[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        noise_at(m, e, g);
        four_steps(m, mf, e, g);
        mf += 4.0f;
    }
    if (m < T) {
        float e[4] = {0.0f, 0.0f, 0.0f, 0.0f}, g[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        noise_at(m, e, g);
        step(phiA, phiB, cm_at(m, mf), e[0], g[0]);
        if (m + 1 < T) step(phiB, phiA, cm_at(m + 1, mf + 1.0f), e[1], g[1]);
        if (m + 2 < T) step(phiA, phiB, cm_at(m + 2, mf + 2.0f), e[2], g[2]);
    }
    x0 = xs.x;
    x1 = xs.y;
    y0 = ys.x;
    y1 = ys.y;
    const int W = a.W;
    for (int t = tid; t < Rb * W; t += blockDim.x) wb[t] = 0ull;
    __syncthreads();
    if (x0 < 0.0f) atomicOr(&wb[(2 * lp) * W + (i >> 6)], 1ull << (i & 63));
    if (x1 < 0.0f) atomicOr(&wb[(2 * lp + 1) * W + (i >> 6)], 1ull << (i & 63));
    __syncthreads();
    for (int t = tid; t < Rb * W; t += blockDim.x) {
        const int r2 = blockIdx.x * Rb + t / W;
        if (r2 < a.R) a.bits[(int64_t)r2 * W + (t % W)] = wb[t];
    }
    if (act0) {
        if (a.x_out) a.x_out[(int64_t)r0 * n + i] = x0;
        if (a.y_out) a.y_out[(int64_t)r0 * n + i] = y0;
    }
    if (act1) {
        if (a.x_out) a.x_out[(int64_t)r1 * n + i] = x1;
        if (a.y_out) a.y_out[(int64_t)r1 * n + i] = y1;
    }
}

template <int VARIANT, int DMAX, bool NOISE, int PUMP>
cudaError_t launch_one2(const SbArgs& a, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    auto k = k_sb_sparse2<VARIANT, DMAX, NOISE, PUMP>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <int VARIANT, int DMAX, bool NOISE>
cudaError_t launch_pump2(const SbArgs& a, int pump, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    switch (pump) {
    case kPumpTable: return launch_one2<VARIANT, DMAX, NOISE, kPumpTable>(a, grid, block, smem, st);
    case kPumpInline: return launch_one2<VARIANT, DMAX, NOISE, kPumpInline>(a, grid, block, smem, st);
    case kPumpInlineCap: return launch_one2<VARIANT, DMAX, NOISE, kPumpInlineCap>(a, grid, block, smem, st);
    case kPumpScheduleCap: return launch_one2<VARIANT, DMAX, NOISE, kPumpScheduleCap>(a, grid, block, smem, st);
    default: return launch_one2<VARIANT, DMAX, NOISE, kPumpSchedule>(a, grid, block, smem, st);
    }
}

// ---- two spins per thread -------------------------------------------------------------
// For large graphs the pair form's blocks (n threads, one per spin) leave one block per SM,
// whose every step ends in a barrier over all of it. This form runs one replica pair per block
// with S = n / 2 rounded up to whole warps threads, thread t holding slots t and S + t (the
// second idle past n): blocks of at most 512 threads, two resident per SM, and two independent
// force chains per thread between barriers. phi keeps the pair form's layout (one float2 per
// slot), so both gathers of a thread follow the slot order's bank plan. Each replica's
// arithmetic and noise counters are those of k_sb_sparse2 (and k_sb_sparse): the same bits.
constexpr int kTwoSpinThreads = 512;
constexpr int kTwoSpinThreadsSmall = 448;  // up to 896 spins: 72 registers a thread at two blocks per SM

inline int two_spin_threads(int n) { return (int)(ceil_div((n + 1) / 2, 32) * 32); }

template <int VARIANT, int DMAX, bool NOISE, int PUMP, int MAXT>
__global__ void __launch_bounds__(MAXT, 2) k_sb_sparse2s(const SbArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n, S = blockDim.x;
    float2* phiA = reinterpret_cast<float2*>(smem_raw);
    float2* phiB = phiA + kPhiStride;
    unsigned* red = reinterpret_cast<unsigned*>(phiB + kPhiStride);  // 4 words
    unsigned long long* wb = reinterpret_cast<unsigned long long*>(smem_raw + sizeof(float) * 4 * kPhiStride + align_up(sizeof(unsigned) * 4, 16));
    const int tid = threadIdx.x;
    const bool hasB = S + tid < n;
    const int iA = a.slot_spin[tid];
    const int iB = hasB ? a.slot_spin[S + tid] : iA;  // idle half: spin A again (harmless in the maxima)
    const int r0 = 2 * blockIdx.x, r1 = r0 + 1;
    float jA0[DMAX], jA1[DMAX], jB0[DMAX], jB1[DMAX];
    int nbA[DMAX], nbB[DMAX];
    float sA0, sA1, wA0, wA1, sB0, sB1, wB0, wB1;
    pair_rows<DMAX>(a, iA, 0, 1, r0, jA0, jA1, nbA, sA0, sA1, wA0, wA1);
    pair_rows<DMAX>(a, iB, 0, 1, r0, jB0, jB1, nbB, sB0, sB1, wB0, wB1);
    if (tid < 4) red[tid] = 0u;
    __syncthreads();
    atomicMax(&red[0], __float_as_uint(fmaxf(fabsf(wA0), fabsf(wB0))));
    atomicMax(&red[1], __float_as_uint(fmaxf(fabsf(wA1), fabsf(wB1))));
    atomicMax(&red[2], __float_as_uint(fmaxf(sA0, sB0)));
    atomicMax(&red[3], __float_as_uint(fmaxf(sA1, sB1)));
    __syncthreads();
    float2 jA[DMAX], jB[DMAX];
    {
        const float c00 = c0_of(__uint_as_float(red[0]), __uint_as_float(red[2]));
        const float c01 = c0_of(__uint_as_float(red[1]), __uint_as_float(red[3]));
#pragma unroll
        for (int d = 0; d < DMAX; ++d) {
            jA[d] = make_float2(jA0[d] * -c00, jA1[d] * -c01);
            jB[d] = make_float2(jB0[d] * -c00, jB1[d] * -c01);
        }
    }
    float2 xA, yA, xB, yB;
    pair_start(a, iA, r0, xA.x, yA.x, xA.y, yA.y);
    pair_start(a, iB, r0, xB.x, yB.x, xB.y, yB.y);
    phiA[tid] = make_float2(phi_of<VARIANT>(xA.x), phi_of<VARIANT>(xA.y));
    if (hasB) phiA[S + tid] = make_float2(phi_of<VARIANT>(xB.x), phi_of<VARIANT>(xB.y));
    __syncthreads();
    const float2 dt2 = make_float2(a.dt, a.dt), kappa2 = make_float2(a.kappa, a.kappa);
    const float2 dta02 = make_float2(a.dt * a.a0, a.dt * a.a0);
    const float a0 = a.a0, a0inv = a.a0inv;
    const float* sched = a.schedule;
    const int T = a.T;
    auto cm_at = [&](int m, float mf) -> float {
        return pump_base(PUMP) == kPumpInline ? fmaf(a0inv, mf, -a0) : (__ldg(sched + m) - a0);
    };
    auto block8 = [&](int m, int i, int r) -> uint4 {
        return NOISE ? philox_rk(make_uint4((uint32_t)(m >> 3), (uint32_t)i, a.rep_off + (uint32_t)r, a.round32), a)
                     : make_uint4(0u, 0u, 0u, 0u);
    };
    auto noise4 = [&](uint32_t wa, uint32_t wbb, float (&e)[4]) {
        if (NOISE) {
            const float2 p = box_muller16(wa), q = box_muller16(wbb);
            e[0] = p.x; e[1] = p.y; e[2] = q.x; e[3] = q.y;
        }
    };
    // one step of both spins: gathers, packed updates, phi written, barrier
    auto step = [&](const float2* rd, float2* wr, float cm, float ea0, float ea1, float eb0, float eb1) {
        float2 fA = make_float2(0.0f, 0.0f), fB = fA;
#pragma unroll
        for (int d = 0; d < DMAX; ++d) {
            fA = __ffma2_rn(jA[d], rd[nbA[d]], fA);
            fB = __ffma2_rn(jB[d], rd[nbB[d]], fB);
        }
        sb_update2<NOISE>(fA, make_float2(cm, cm), make_float2(ea0, ea1), dt2, kappa2, dta02, xA, yA);
        sb_update2<NOISE>(fB, make_float2(cm, cm), make_float2(eb0, eb1), dt2, kappa2, dta02, xB, yB);
        wr[tid] = make_float2(phi_of<VARIANT>(xA.x), phi_of<VARIANT>(xA.y));
        if (hasB) wr[S + tid] = make_float2(phi_of<VARIANT>(xB.x), phi_of<VARIANT>(xB.y));
        __syncthreads();
    };
    auto four_steps = [&](int m, float mf, const float (&e)[4], const float (&g)[4], const float (&u)[4], const float (&v)[4]) {
        step(phiA, phiB, cm_at(m, mf), e[0], g[0], u[0], v[0]);
        step(phiB, phiA, cm_at(m + 1, mf + 1.0f), e[1], g[1], u[1], v[1]);
        step(phiA, phiB, cm_at(m + 2, mf + 2.0f), e[2], g[2], u[2], v[2]);
        step(phiB, phiA, cm_at(m + 3, mf + 3.0f), e[3], g[3], u[3], v[3]);
    };
    auto noise_at = [&](int m, float (&e)[4], float (&g)[4], float (&u)[4], float (&v)[4]) {
        if (NOISE) {
            const bool hi = (m & 4) != 0;
            const uint4 o = block8(m, iA, r0), q = block8(m, iA, r1), ob = block8(m, iB, r0), qb = block8(m, iB, r1);
            noise4(hi ? o.z : o.x, hi ? o.w : o.y, e);
            noise4(hi ? q.z : q.x, hi ? q.w : q.y, g);
            noise4(hi ? ob.z : ob.x, hi ? ob.w : ob.y, u);
            noise4(hi ? qb.z : qb.x, hi ? qb.w : qb.y, v);
        }
    };
    int m = 0;
    float mf = 0.0f;
    if (NOISE) {
        // the Gaussians two steps at a time (one Philox word per replica and spin), which keeps
        // fewer of them live than four at a time
        auto two_steps = [&](int mm, float mmf, uint32_t wa, uint32_t wbb, uint32_t wc, uint32_t wd) {
            const float2 pa = box_muller16(wa), pb = box_muller16(wbb), pc = box_muller16(wc), pd = box_muller16(wd);
            step(phiA, phiB, cm_at(mm, mmf), pa.x, pb.x, pc.x, pd.x);
            step(phiB, phiA, cm_at(mm + 1, mmf + 1.0f), pa.y, pb.y, pc.y, pd.y);
        };
        for (; m + 8 <= T; m += 8) {
            const uint4 o = block8(m, iA, r0), q = block8(m, iA, r1), ob = block8(m, iB, r0), qb = block8(m, iB, r1);
            two_steps(m, mf, o.x, q.x, ob.x, qb.x);
            two_steps(m + 2, mf + 2.0f, o.y, q.y, ob.y, qb.y);
            two_steps(m + 4, mf + 4.0f, o.z, q.z, ob.z, qb.z);
            two_steps(m + 6, mf + 6.0f, o.w, q.w, ob.w, qb.w);
            mf += 8.0f;
        }
    }
    for (; m + 4 <= T; m += 4) {
        float e[4] = {0.0f, 0.0f, 0.0f, 0.0f}, g[4] = {0.0f, 0.0f, 0.0f, 0.0f}, u[4] = {0.0f, 0.0f, 0.0f, 0.0f},
              v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        noise_at(m, e, g, u, v);
        four_steps(m, mf, e, g, u, v);
        mf += 4.0f;
    }
    if (m < T) {
        float e[4] = {0.0f, 0.0f, 0.0f, 0.0f}, g[4] = {0.0f, 0.0f, 0.0f, 0.0f}, u[4] = {0.0f, 0.0f, 0.0f, 0.0f},
              v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        noise_at(m, e, g, u, v);
        step(phiA, phiB, cm_at(m, mf), e[0], g[0], u[0], v[0]);
        if (m + 1 < T) step(phiB, phiA, cm_at(m + 1, mf + 1.0f), e[1], g[1], u[1], v[1]);
        if (m + 2 < T) step(phiA, phiB, cm_at(m + 2, mf + 2.0f), e[2], g[2], u[2], v[2]);
    }
    const int W = a.W;
    for (int t = tid; t < 2 * W; t += blockDim.x) wb[t] = 0ull;
    __syncthreads();
    if (xA.x < 0.0f) atomicOr(&wb[iA >> 6], 1ull << (iA & 63));
    if (xA.y < 0.0f) atomicOr(&wb[W + (iA >> 6)], 1ull << (iA & 63));
    if (hasB && xB.x < 0.0f) atomicOr(&wb[iB >> 6], 1ull << (iB & 63));
    if (hasB && xB.y < 0.0f) atomicOr(&wb[W + (iB >> 6)], 1ull << (iB & 63));
    __syncthreads();
    for (int t = tid; t < 2 * W; t += blockDim.x) {
        const int r2 = r0 + t / W;
        if (r2 < a.R) a.bits[(int64_t)r2 * W + (t % W)] = wb[t];
    }
    auto out = [&](int i, float2 x, float2 y) {
        if (r0 < a.R) {
            if (a.x_out) a.x_out[(int64_t)r0 * n + i] = x.x;
            if (a.y_out) a.y_out[(int64_t)r0 * n + i] = y.x;
        }
        if (r1 < a.R) {
            if (a.x_out) a.x_out[(int64_t)r1 * n + i] = x.y;
            if (a.y_out) a.y_out[(int64_t)r1 * n + i] = y.y;
        }
    };
    out(iA, xA, yA);
    if (hasB) out(iB, xB, yB);
}

__host__ __device__ inline size_t sb_smem_bytes2s(int W) { return sizeof(float) * 4 * kPhiStride + 16 + align_up(sizeof(unsigned long long) * 2 * (size_t)W, 16); }

template <int VARIANT, int DMAX, bool NOISE, int PUMP>
cudaError_t launch_one2s(const SbArgs& a, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    // blocks of up to 448 threads take the build bounded for them (72 registers instead of
    // 64, fewer spills): 2-3 % faster at 660-896 spins, the same bits
    auto k = block.x <= (unsigned)kTwoSpinThreadsSmall ? k_sb_sparse2s<VARIANT, DMAX, NOISE, PUMP, kTwoSpinThreadsSmall>
                                                       : k_sb_sparse2s<VARIANT, DMAX, NOISE, PUMP, kTwoSpinThreads>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

// degree bounds 3 and 4; the pump from the schedule or inline
template <int VARIANT>
cudaError_t launch_variant2s(const SbArgs& a, int dmax, bool noise, bool schedule, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
#define MOQ_2S(D, N) (schedule ? launch_one2s<VARIANT, D, N, kPumpSchedule>(a, grid, block, smem, st) \
                               : launch_one2s<VARIANT, D, N, kPumpInline>(a, grid, block, smem, st))
    switch (dmax) {
    case 3: return noise ? MOQ_2S(3, true) : MOQ_2S(3, false);
    case 4: return noise ? MOQ_2S(4, true) : MOQ_2S(4, false);
    default: return cudaErrorInvalidValue;
    }
#undef MOQ_2S
}

// ---- float16 state: the paper's precision ---------------------------------------------
// The paper runs SB in float16. This form keeps the state and does the step's arithmetic in
// FP16: each thread runs spin i of two replicas with x, y, its two rows of -c0 J(c) and phi
// as packed half2 (lane 0: replica r0, lane 1: r0 + 1), the force sum and the Euler update
// as two-lane FP16 multiply-adds (one rounding each), the wall and dSB's sign on the bit
// patterns. c0 and the couplings are formed in FP32 (as the FP32 form does) and rounded once
// to FP16, the start state is the FP32 form's rounded to FP16, and eta is the FP32 form's
// Gaussian (same Philox counters) rounded to FP16; the pump value a_m - a0 is rounded to FP16.
// phi takes 4 bytes per pair of replicas in shared memory (half the FP32 pair form's).
__device__ __forceinline__ uint32_t h2_bits(__half2 v) { return *reinterpret_cast<uint32_t*>(&v); }
__device__ __forceinline__ __half2 bits_h2(uint32_t u) { return *reinterpret_cast<__half2*>(&u); }

__host__ __device__ inline size_t sb_smem_bytes_h(int Rb, int W, int pump_table_steps)
{
    return sizeof(__half2) * 2 * kPhiStride + align_up(sizeof(unsigned) * 2 * Rb, 16) +
           align_up(sizeof(unsigned long long) * (size_t)Rb * W, 16) + sizeof(__half2) * (size_t)pump_table_steps;
}

// The FP16 Euler step of a replica pair on its force f, lane by lane: update, then the wall
// (lanes with |x| > 1 take x = sgn(x), the dSB phi of x, and y = 0). Returns sgn(x) as +-1 halves.
template <bool NOISE>
__device__ __forceinline__ uint32_t h2_update(__half2 f, __half2 cm, __half2 eta, __half2 dt, __half2 kappa, __half2 dta0, __half2& x,
                                              __half2& y)
{
    y = __hfma2(dt, __hfma2(cm, x, f), y);
    if (NOISE) y = __hfma2(kappa, eta, y);
    x = __hfma2(dta0, y, x);
    const uint32_t xb = h2_bits(x);
    const uint32_t sg = (xb & 0x80008000u) | 0x3C003C00u;
    const uint32_t over = __hgt2_mask(__habs2(x), __float2half2_rn(1.0f));
    x = bits_h2((over & sg) | (~over & xb));
    y = bits_h2(~over & h2_bits(y));
    return sg;
}

template <int VARIANT, int DMAX, bool NOISE>
__device__ __forceinline__ void sb_step_h(const __half2* rd, __half2* wr, int tid, const __half2 (&jc)[DMAX], const int (&nb)[DMAX],
                                          __half2 cm, __half2 eta, __half2 dt, __half2 kappa, __half2 dta0, __half2& x, __half2& y)
{
    __half2 f = __float2half2_rn(0.0f);
#pragma unroll
    for (int d = 0; d < DMAX; ++d) f = __hfma2(jc[d], rd[nb[d]], f);
    const uint32_t sg = h2_update<NOISE>(f, cm, eta, dt, kappa, dta0, x, y);
    wr[tid] = VARIANT == MOQ_DSB ? bits_h2(sg) : x;
    __syncthreads();
}

template <int VARIANT, int DMAX, bool NOISE, int PUMP>
__global__ void __launch_bounds__(PUMP >= 3 ? kCapThreads : 1024, PUMP >= 3 ? 2 : 1) k_sb_sparse_h(const SbArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n, Rb = a.Rb, Rp = a.Rb >> 1;
    __half2* phiA = reinterpret_cast<__half2*>(smem_raw);
    __half2* phiB = phiA + kPhiStride;
    unsigned* red = reinterpret_cast<unsigned*>(phiB + kPhiStride);  // 2 * Rb
    unsigned long long* wb = reinterpret_cast<unsigned long long*>(smem_raw + sizeof(__half2) * 2 * kPhiStride +
                                                                   align_up(sizeof(unsigned) * 2 * Rb, 16));
    __half2* pump_t = reinterpret_cast<__half2*>(reinterpret_cast<unsigned char*>(wb) +
                                                 align_up(sizeof(unsigned long long) * (size_t)Rb * a.W, 16));
    const int tid = threadIdx.x;
    const int slot = tid / Rp;
    const int lp = tid - slot * Rp;
    const int i = a.slot_spin[slot];
    const int r0 = blockIdx.x * Rb + 2 * lp, r1 = r0 + 1;
    const bool act0 = r0 < a.R, act1 = r1 < a.R;
    float jc0[DMAX], jc1[DMAX];
    int nb[DMAX];
    float x0, y0, x1, y1;
    pair_setup<DMAX>(a, tid, i, lp, Rp, r0, red, jc0, jc1, nb, x0, y0, x1, y1);
    __half2 jc[DMAX];
#pragma unroll
    for (int d = 0; d < DMAX; ++d) jc[d] = __floats2half2_rn(jc0[d], jc1[d]);
    __half2 xs = __floats2half2_rn(x0, x1), ys = __floats2half2_rn(y0, y1);
    phiA[tid] = VARIANT == MOQ_DSB ? bits_h2((h2_bits(xs) & 0x80008000u) | 0x3C003C00u) : xs;
    __syncthreads();
    const __half2 dt2 = __float2half2_rn(a.dt), kappa2 = __float2half2_rn(a.kappa), dta02 = __float2half2_rn(a.dt * a.a0);
    const float a0 = a.a0, a0inv = a.a0inv;
    const float* sched = a.schedule;
    const int T = a.T;
    if (pump_base(PUMP) == kPumpTable) {
        for (int q = tid; q < T; q += blockDim.x) pump_t[q] = __float2half2_rn(fmaf(a0inv, (float)q, -a0));
        __syncthreads();
    }
    auto cm_at = [&](int m, float mf) -> __half2 {
        if (pump_base(PUMP) == kPumpTable) return pump_t[m];
        return __float2half2_rn(pump_base(PUMP) == kPumpInline ? fmaf(a0inv, mf, -a0) : (__ldg(sched + m) - a0));
    };
    auto block8 = [&](int m, int r) -> uint4 {
        return NOISE ? philox_rk(make_uint4((uint32_t)(m >> 3), (uint32_t)i, a.rep_off + (uint32_t)r, a.round32), a)
                     : make_uint4(0u, 0u, 0u, 0u);
    };
    // the Gaussians of four steps of both replicas, rounded to FP16 (lane 0: r0, lane 1: r1)
    auto noise4 = [&](uint32_t wa, uint32_t wbb, uint32_t va, uint32_t vb, __half2 (&eg)[4]) {
        if (NOISE) {
            const float2 p = box_muller16(wa), q = box_muller16(wbb), u = box_muller16(va), v = box_muller16(vb);
            eg[0] = __floats2half2_rn(p.x, u.x);
            eg[1] = __floats2half2_rn(p.y, u.y);
            eg[2] = __floats2half2_rn(q.x, v.x);
            eg[3] = __floats2half2_rn(q.y, v.y);
        }
    };
    auto step = [&](const __half2* rd, __half2* wr, __half2 cm, __half2 eta) {
        sb_step_h<VARIANT, DMAX, NOISE>(rd, wr, tid, jc, nb, cm, eta, dt2, kappa2, dta02, xs, ys);
    };
    auto four_steps = [&](int m, float mf, const __half2 (&eg)[4]) {
        step(phiA, phiB, cm_at(m, mf), eg[0]);
        step(phiB, phiA, cm_at(m + 1, mf + 1.0f), eg[1]);
        step(phiA, phiB, cm_at(m + 2, mf + 2.0f), eg[2]);
        step(phiB, phiA, cm_at(m + 3, mf + 3.0f), eg[3]);
    };
    auto noise_at = [&](int m, __half2 (&eg)[4]) {
        if (NOISE) {
            const uint4 o = block8(m, r0), q = block8(m, r1);
            noise4((m & 4) ? o.z : o.x, (m & 4) ? o.w : o.y, (m & 4) ? q.z : q.x, (m & 4) ? q.w : q.y, eg);
        }
    };
    const __half2 zero2 = __float2half2_rn(0.0f);
    int m = 0;
    float mf = 0.0f;
    if (NOISE) {
        for (; m + 8 <= T; m += 8) {
            const uint4 o = block8(m, r0), q = block8(m, r1);
            __half2 eg[4];
            noise4(o.x, o.y, q.x, q.y, eg);
            four_steps(m, mf, eg);
            noise4(o.z, o.w, q.z, q.w, eg);
            four_steps(m + 4, mf + 4.0f, eg);
            mf += 8.0f;
        }
    }
    for (; m + 4 <= T; m += 4) {
        __half2 eg[4] = {zero2, zero2, zero2, zero2};
        noise_at(m, eg);
        four_steps(m, mf, eg);
        mf += 4.0f;
    }
    if (m < T) {
        __half2 eg[4] = {zero2, zero2, zero2, zero2};
        noise_at(m, eg);
        step(phiA, phiB, cm_at(m, mf), eg[0]);
        if (m + 1 < T) step(phiB, phiA, cm_at(m + 1, mf + 1.0f), eg[1]);
        if (m + 2 < T) step(phiA, phiB, cm_at(m + 2, mf + 2.0f), eg[2]);
    }
    const float2 xf = __half22float2(xs), yf = __half22float2(ys);
    const int W = a.W;
    for (int t = tid; t < Rb * W; t += blockDim.x) wb[t] = 0ull;
    __syncthreads();
    if (xf.x < 0.0f) atomicOr(&wb[(2 * lp) * W + (i >> 6)], 1ull << (i & 63));
    if (xf.y < 0.0f) atomicOr(&wb[(2 * lp + 1) * W + (i >> 6)], 1ull << (i & 63));
    __syncthreads();
    for (int t = tid; t < Rb * W; t += blockDim.x) {
        const int r2 = blockIdx.x * Rb + t / W;
        if (r2 < a.R) a.bits[(int64_t)r2 * W + (t % W)] = wb[t];
    }
    if (act0) {
        if (a.x_out) a.x_out[(int64_t)r0 * n + i] = xf.x;
        if (a.y_out) a.y_out[(int64_t)r0 * n + i] = yf.x;
    }
    if (act1) {
        if (a.x_out) a.x_out[(int64_t)r1 * n + i] = xf.y;
        if (a.y_out) a.y_out[(int64_t)r1 * n + i] = yf.y;
    }
}

// Four replicas per thread (two half2 pairs, A = (r0, r0 + 1), B = (r0 + 2, r0 + 3)) for large
// graphs, where one block of n threads fills an SM: one 8-byte gather brings a neighbour's phi of
// all four replicas, and the barrier, pump value and loop control serve four updates. Each
// replica's arithmetic and counters are those of k_sb_sparse_h, so both give the same bits.
__host__ __device__ inline size_t sb_smem_bytes_h4(int Rb, int W, int pump_table_steps)
{
    return sizeof(uint2) * 2 * kPhiStride + align_up(sizeof(unsigned) * 2 * Rb, 16) +
           align_up(sizeof(unsigned long long) * (size_t)Rb * W, 16) + sizeof(__half2) * (size_t)pump_table_steps;
}

template <int VARIANT, int DMAX, bool NOISE>
__device__ __forceinline__ void sb_step_h4(const uint2* rd, uint2* wr, int tid, const __half2 (&ja)[DMAX], const __half2 (&jb)[DMAX],
                                           const int (&nb)[DMAX], __half2 cm, __half2 ea, __half2 eb, __half2 dt, __half2 kappa,
                                           __half2 dta0, __half2& xa, __half2& ya, __half2& xb, __half2& yb)
{
    __half2 fa = __float2half2_rn(0.0f), fb = fa;
#pragma unroll
    for (int d = 0; d < DMAX; ++d) {
        const uint2 ph = rd[nb[d]];
        fa = __hfma2(ja[d], bits_h2(ph.x), fa);
        fb = __hfma2(jb[d], bits_h2(ph.y), fb);
    }
    const uint32_t sa = h2_update<NOISE>(fa, cm, ea, dt, kappa, dta0, xa, ya);
    const uint32_t sg = h2_update<NOISE>(fb, cm, eb, dt, kappa, dta0, xb, yb);
    wr[tid] = VARIANT == MOQ_DSB ? make_uint2(sa, sg) : make_uint2(h2_bits(xa), h2_bits(xb));
    __syncthreads();
}

template <int VARIANT, int DMAX, bool NOISE, int PUMP>
__global__ void __launch_bounds__(1024) k_sb_sparse_h4(const SbArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n, Rb = a.Rb, Rq = a.Rb >> 2;
    uint2* phiA = reinterpret_cast<uint2*>(smem_raw);
    uint2* phiB = phiA + kPhiStride;
    unsigned* red = reinterpret_cast<unsigned*>(phiB + kPhiStride);  // 2 * Rb
    unsigned long long* wb = reinterpret_cast<unsigned long long*>(smem_raw + sizeof(uint2) * 2 * kPhiStride +
                                                                   align_up(sizeof(unsigned) * 2 * Rb, 16));
    __half2* pump_t = reinterpret_cast<__half2*>(reinterpret_cast<unsigned char*>(wb) +
                                                 align_up(sizeof(unsigned long long) * (size_t)Rb * a.W, 16));
    const int tid = threadIdx.x;
    const int slot = tid / Rq;
    const int lq = tid - slot * Rq;
    const int i = a.slot_spin[slot];
    const int r0 = blockIdx.x * Rb + 4 * lq;
    // both pairs set up as pairs 2 lq and 2 lq + 1 of a block of 2 Rq pairs
    float j0[DMAX], j1[DMAX];
    int nb[DMAX];
    float x0, y0, x1, y1;
    __half2 ja[DMAX], jb[DMAX];
    pair_setup<DMAX>(a, tid, i, 2 * lq, 2 * Rq, r0, red, j0, j1, nb, x0, y0, x1, y1);
#pragma unroll
    for (int d = 0; d < DMAX; ++d) ja[d] = __floats2half2_rn(j0[d], j1[d]);
    __half2 xa = __floats2half2_rn(x0, x1), ya = __floats2half2_rn(y0, y1);
    __syncthreads();  // the reduction words are reused by the second pair
    pair_setup<DMAX>(a, tid, i, 2 * lq + 1, 2 * Rq, r0 + 2, red, j0, j1, nb, x0, y0, x1, y1);
#pragma unroll
    for (int d = 0; d < DMAX; ++d) {
        jb[d] = __floats2half2_rn(j0[d], j1[d]);
        nb[d] >>= 1;  // pair index 2 (slot Rq + lq) + 1 -> quad index slot Rq + lq
    }
    __half2 xb = __floats2half2_rn(x0, x1), yb = __floats2half2_rn(y0, y1);
    phiA[tid] = VARIANT == MOQ_DSB ? make_uint2((h2_bits(xa) & 0x80008000u) | 0x3C003C00u, (h2_bits(xb) & 0x80008000u) | 0x3C003C00u)
                                   : make_uint2(h2_bits(xa), h2_bits(xb));
    __syncthreads();
    const __half2 dt2 = __float2half2_rn(a.dt), kappa2 = __float2half2_rn(a.kappa), dta02 = __float2half2_rn(a.dt * a.a0);
    const float a0 = a.a0, a0inv = a.a0inv;
    const float* sched = a.schedule;
    const int T = a.T;
    if (pump_base(PUMP) == kPumpTable) {
        for (int q = tid; q < T; q += blockDim.x) pump_t[q] = __float2half2_rn(fmaf(a0inv, (float)q, -a0));
        __syncthreads();
    }
    auto cm_at = [&](int m, float mf) -> __half2 {
        if (pump_base(PUMP) == kPumpTable) return pump_t[m];
        return __float2half2_rn(pump_base(PUMP) == kPumpInline ? fmaf(a0inv, mf, -a0) : (__ldg(sched + m) - a0));
    };
    auto block8 = [&](int m, int r) -> uint4 {
        return NOISE ? philox_rk(make_uint4((uint32_t)(m >> 3), (uint32_t)i, a.rep_off + (uint32_t)r, a.round32), a)
                     : make_uint4(0u, 0u, 0u, 0u);
    };
    auto noise4 = [&](uint32_t wa, uint32_t wbb, uint32_t va, uint32_t vb, __half2 (&eg)[4]) {
        if (NOISE) {
            const float2 p = box_muller16(wa), q = box_muller16(wbb), u = box_muller16(va), v = box_muller16(vb);
            eg[0] = __floats2half2_rn(p.x, u.x);
            eg[1] = __floats2half2_rn(p.y, u.y);
            eg[2] = __floats2half2_rn(q.x, v.x);
            eg[3] = __floats2half2_rn(q.y, v.y);
        }
    };
    auto step = [&](const uint2* rd, uint2* wr, __half2 cm, __half2 ea, __half2 eb) {
        sb_step_h4<VARIANT, DMAX, NOISE>(rd, wr, tid, ja, jb, nb, cm, ea, eb, dt2, kappa2, dta02, xa, ya, xb, yb);
    };
    auto four_steps = [&](int m, float mf, const __half2 (&ga)[4], const __half2 (&gb)[4]) {
        step(phiA, phiB, cm_at(m, mf), ga[0], gb[0]);
        step(phiB, phiA, cm_at(m + 1, mf + 1.0f), ga[1], gb[1]);
        step(phiA, phiB, cm_at(m + 2, mf + 2.0f), ga[2], gb[2]);
        step(phiB, phiA, cm_at(m + 3, mf + 3.0f), ga[3], gb[3]);
    };
    auto noise_at = [&](int m, __half2 (&ga)[4], __half2 (&gb)[4]) {
        if (NOISE) {
            const uint4 o0 = block8(m, r0), o1 = block8(m, r0 + 1), o2 = block8(m, r0 + 2), o3 = block8(m, r0 + 3);
            const bool hi = (m & 4) != 0;
            noise4(hi ? o0.z : o0.x, hi ? o0.w : o0.y, hi ? o1.z : o1.x, hi ? o1.w : o1.y, ga);
            noise4(hi ? o2.z : o2.x, hi ? o2.w : o2.y, hi ? o3.z : o3.x, hi ? o3.w : o3.y, gb);
        }
    };
    const __half2 zero2 = __float2half2_rn(0.0f);
    int m = 0;
    float mf = 0.0f;
    if (NOISE) {
        for (; m + 8 <= T; m += 8) {
            const uint4 o0 = block8(m, r0), o1 = block8(m, r0 + 1), o2 = block8(m, r0 + 2), o3 = block8(m, r0 + 3);
            __half2 ga[4], gb[4];
            noise4(o0.x, o0.y, o1.x, o1.y, ga);
            noise4(o2.x, o2.y, o3.x, o3.y, gb);
            four_steps(m, mf, ga, gb);
            noise4(o0.z, o0.w, o1.z, o1.w, ga);
            noise4(o2.z, o2.w, o3.z, o3.w, gb);
            four_steps(m + 4, mf + 4.0f, ga, gb);
            mf += 8.0f;
        }
    }
    for (; m + 4 <= T; m += 4) {
        __half2 ga[4] = {zero2, zero2, zero2, zero2}, gb[4] = {zero2, zero2, zero2, zero2};
        noise_at(m, ga, gb);
        four_steps(m, mf, ga, gb);
        mf += 4.0f;
    }
    if (m < T) {
        __half2 ga[4] = {zero2, zero2, zero2, zero2}, gb[4] = {zero2, zero2, zero2, zero2};
        noise_at(m, ga, gb);
        step(phiA, phiB, cm_at(m, mf), ga[0], gb[0]);
        if (m + 1 < T) step(phiB, phiA, cm_at(m + 1, mf + 1.0f), ga[1], gb[1]);
        if (m + 2 < T) step(phiA, phiB, cm_at(m + 2, mf + 2.0f), ga[2], gb[2]);
    }
    const float2 xfa = __half22float2(xa), yfa = __half22float2(ya), xfb = __half22float2(xb), yfb = __half22float2(yb);
    const float xf[4] = {xfa.x, xfa.y, xfb.x, xfb.y}, yf[4] = {yfa.x, yfa.y, yfb.x, yfb.y};
    const int W = a.W;
    for (int t = tid; t < Rb * W; t += blockDim.x) wb[t] = 0ull;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (xf[q] < 0.0f) atomicOr(&wb[(4 * lq + q) * W + (i >> 6)], 1ull << (i & 63));
    __syncthreads();
    for (int t = tid; t < Rb * W; t += blockDim.x) {
        const int r2 = blockIdx.x * Rb + t / W;
        if (r2 < a.R) a.bits[(int64_t)r2 * W + (t % W)] = wb[t];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (r0 + q < a.R) {
            if (a.x_out) a.x_out[(int64_t)(r0 + q) * n + i] = xf[q];
            if (a.y_out) a.y_out[(int64_t)(r0 + q) * n + i] = yf[q];
        }
}

template <int VARIANT, int DMAX, bool NOISE, int PUMP>
cudaError_t launch_one_h4(const SbArgs& a, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    auto k = k_sb_sparse_h4<VARIANT, DMAX, NOISE, PUMP>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <int VARIANT, int DMAX, bool NOISE>
cudaError_t launch_pump_h4(const SbArgs& a, int pump, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    switch (pump) {
    case kPumpTable: return launch_one_h4<VARIANT, DMAX, NOISE, kPumpTable>(a, grid, block, smem, st);
    case kPumpInline: return launch_one_h4<VARIANT, DMAX, NOISE, kPumpInline>(a, grid, block, smem, st);
    default: return launch_one_h4<VARIANT, DMAX, NOISE, kPumpSchedule>(a, grid, block, smem, st);
    }
}

// quads for degree bounds 3 and 4
template <int VARIANT>
cudaError_t launch_variant_h4(const SbArgs& a, int dmax, bool noise, int pump, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    switch (dmax) {
    case 3: return noise ? launch_pump_h4<VARIANT, 3, true>(a, pump, grid, block, smem, st) : launch_pump_h4<VARIANT, 3, false>(a, pump, grid, block, smem, st);
    case 4: return noise ? launch_pump_h4<VARIANT, 4, true>(a, pump, grid, block, smem, st) : launch_pump_h4<VARIANT, 4, false>(a, pump, grid, block, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int VARIANT, int DMAX, bool NOISE, int PUMP>
cudaError_t launch_one_h(const SbArgs& a, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    auto k = k_sb_sparse_h<VARIANT, DMAX, NOISE, PUMP>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <int VARIANT, int DMAX, bool NOISE>
cudaError_t launch_pump_h(const SbArgs& a, int pump, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    switch (pump) {
    case kPumpTable: return launch_one_h<VARIANT, DMAX, NOISE, kPumpTable>(a, grid, block, smem, st);
    case kPumpInline: return launch_one_h<VARIANT, DMAX, NOISE, kPumpInline>(a, grid, block, smem, st);
    case kPumpInlineCap: return launch_one_h<VARIANT, DMAX, NOISE, kPumpInlineCap>(a, grid, block, smem, st);
    case kPumpScheduleCap: return launch_one_h<VARIANT, DMAX, NOISE, kPumpScheduleCap>(a, grid, block, smem, st);
    default: return launch_one_h<VARIANT, DMAX, NOISE, kPumpSchedule>(a, grid, block, smem, st);
    }
}

// the FP16 form for degree bounds 3, 4 and 8 (two rows of half2 couplings fit in registers)
template <int VARIANT>
cudaError_t launch_variant_h(const SbArgs& a, int dmax, bool noise, int pump, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    switch (dmax) {
    case 3: return noise ? launch_pump_h<VARIANT, 3, true>(a, pump, grid, block, smem, st) : launch_pump_h<VARIANT, 3, false>(a, pump, grid, block, smem, st);
    case 4: return noise ? launch_pump_h<VARIANT, 4, true>(a, pump, grid, block, smem, st) : launch_pump_h<VARIANT, 4, false>(a, pump, grid, block, smem, st);
    case 8: return noise ? launch_pump_h<VARIANT, 8, true>(a, pump, grid, block, smem, st) : launch_pump_h<VARIANT, 8, false>(a, pump, grid, block, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

// pairs for degree bounds 3 and 4 only: from 8 up, two rows of J(c) no longer fit in registers
template <int VARIANT>
cudaError_t launch_variant2(const SbArgs& a, int dmax, bool noise, int pump, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    switch (dmax) {
    case 3: return noise ? launch_pump2<VARIANT, 3, true>(a, pump, grid, block, smem, st) : launch_pump2<VARIANT, 3, false>(a, pump, grid, block, smem, st);
    case 4: return noise ? launch_pump2<VARIANT, 4, true>(a, pump, grid, block, smem, st) : launch_pump2<VARIANT, 4, false>(a, pump, grid, block, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

// the kernel instance a launch would use (for the occupancy query)
template <int VARIANT, int DMAX, bool NOISE>
const void* kernel_of(bool pair, int pump)
{
    if (DMAX <= 4 && pair) {
        switch (pump) {
        case kPumpTable: return (const void*)k_sb_sparse2<VARIANT, (DMAX <= 4 ? DMAX : 4), NOISE, kPumpTable>;
        case kPumpInline: return (const void*)k_sb_sparse2<VARIANT, (DMAX <= 4 ? DMAX : 4), NOISE, kPumpInline>;
        case kPumpInlineCap: return (const void*)k_sb_sparse2<VARIANT, (DMAX <= 4 ? DMAX : 4), NOISE, kPumpInlineCap>;
        case kPumpScheduleCap: return (const void*)k_sb_sparse2<VARIANT, (DMAX <= 4 ? DMAX : 4), NOISE, kPumpScheduleCap>;
        default: return (const void*)k_sb_sparse2<VARIANT, (DMAX <= 4 ? DMAX : 4), NOISE, kPumpSchedule>;
        }
    }
    switch (pump) {
    case kPumpTable: return (const void*)k_sb_sparse<VARIANT, DMAX, NOISE, kPumpTable>;
    case kPumpInline: return (const void*)k_sb_sparse<VARIANT, DMAX, NOISE, kPumpInline>;
    default: return (const void*)k_sb_sparse<VARIANT, DMAX, NOISE, kPumpSchedule>;
    }
}

template <int VARIANT, int DMAX, bool NOISE>
const void* kernel_of_h(int pump)
{
    switch (pump) {
    case kPumpTable: return (const void*)k_sb_sparse_h<VARIANT, DMAX, NOISE, kPumpTable>;
    case kPumpInline: return (const void*)k_sb_sparse_h<VARIANT, DMAX, NOISE, kPumpInline>;
    case kPumpInlineCap: return (const void*)k_sb_sparse_h<VARIANT, DMAX, NOISE, kPumpInlineCap>;
    case kPumpScheduleCap: return (const void*)k_sb_sparse_h<VARIANT, DMAX, NOISE, kPumpScheduleCap>;
    default: return (const void*)k_sb_sparse_h<VARIANT, DMAX, NOISE, kPumpSchedule>;
    }
}

template <int VARIANT>
const void* kernel_of_variant_h(int dmax, bool noise, int pump)
{
    switch (dmax) {
    case 3: return noise ? kernel_of_h<VARIANT, 3, true>(pump) : kernel_of_h<VARIANT, 3, false>(pump);
    case 4: return noise ? kernel_of_h<VARIANT, 4, true>(pump) : kernel_of_h<VARIANT, 4, false>(pump);
    default: return noise ? kernel_of_h<VARIANT, 8, true>(pump) : kernel_of_h<VARIANT, 8, false>(pump);
    }
}

// the register-capped build where it keeps more blocks resident; MOQ_SB_CAP = 0 / 1 forces the
// choice (for blocks of at most 640 threads without the pump table)
bool cap_choice(bool more_resident)
{
    if (const char* env = getenv("MOQ_SB_CAP")) return atoi(env) != 0;
    return more_resident;
}

// resident blocks per SM of a kernel instance at the given block shape (0 if the query fails)
int resident_blocks(const void* k, int threads, size_t smem)
{
    int blocks = 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, threads, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return blocks;
}

template <int VARIANT>
const void* kernel_of_variant(int dmax, bool noise, bool pair, int pump)
{
    switch (dmax) {
    case 3: return noise ? kernel_of<VARIANT, 3, true>(pair, pump) : kernel_of<VARIANT, 3, false>(pair, pump);
    case 4: return noise ? kernel_of<VARIANT, 4, true>(pair, pump) : kernel_of<VARIANT, 4, false>(pair, pump);
    case 8: return noise ? kernel_of<VARIANT, 8, true>(pair, pump) : kernel_of<VARIANT, 8, false>(pair, pump);
    default: return noise ? kernel_of<VARIANT, 16, true>(pair, pump) : kernel_of<VARIANT, 16, false>(pair, pump);
    }
}


// Replicas per block: among blocks of up to about 256 threads, the one whose warps are
// fullest (n * Rb close to a multiple of 32), the smaller block on ties -- small blocks hide
// each other's step barriers (measured at n = 42: 126-thread blocks 1.76 ms, 252-thread
// 1.84 ms, 294-thread 2.05 ms per launch); at most 32 replicas, and enough blocks to cover
// the 148 SMs when R is small.
int choose_rb(int n, int R)
{
    int rb = fullest_warp_rb(n);
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
    if (p->precision != MOQ_PREC_FP32 && p->precision != MOQ_PREC_FP16)
        return fail(MOQ_ERR_ARG, "moq_sample: unknown precision %d", p->precision);
    if (p->precision == MOQ_PREC_FP16 && inst->max_degree > 8)
        return fail(MOQ_ERR_UNSUPPORTED, "moq_sample: the FP16 form runs degree bounds up to 8 (max degree %d)", inst->max_degree);

    SbArgs a{};
    a.n = inst->n;
    a.K = inst->K;
    a.R = R;
    a.T = p->steps;
    a.W = inst->words;
    a.nnz = inst->nnz;
    a.rowptr = inst->rowptr;
    a.slot_spin = inst->slot_spin;
    a.spin_slot = inst->spin_slot;
    a.col = inst->col;
    a.wn = inst->wn;
    a.rowsum = inst->rowsum;
    a.lambda = lambda;
    a.dt = p->dt;
    a.a0 = p->a0;
    a.init_amp = p->init_amp;
    a.kappa = (p->noise_sqrt_dt ? sqrtf(p->dt) : p->dt) * p->alpha;
    a.a0inv = p->steps > 1 ? p->a0 / (float)(p->steps - 1) : 0.0f;
    a.schedule = p->schedule;
    a.x_init = p->x_init;
    a.y_init = p->y_init;
    a.x_out = p->x_out;
    a.y_out = p->y_out;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        a.rk0[r] = a.key0 + (uint32_t)r * Philox4x32::kW0;
        a.rk1[r] = a.key1 + (uint32_t)r * Philox4x32::kW1;
    }
    a.round32 = (uint32_t)round;
    a.rep_off = p->replica_offset;
    a.bits = bits;
    const int md = inst->max_degree;
    const int dmax = md <= 3 ? 3 : (md <= 4 ? 4 : (md <= 8 ? 8 : 16));
    const bool noise = p->alpha != 0.0f;
    if (p->precision == MOQ_PREC_FP16) {
        // large graphs (one block of more than 640 threads per SM): four replicas per thread when
        // the grid still covers the GPU (MOQ_SB_QUAD = 0 / 1 forces the choice)
        {
            const int Rq = choose_rb(a.n, (R + 3) / 4);
            bool quad = dmax <= 4 && a.n * choose_rb(a.n, (R + 1) / 2) > kCapThreads && ceil_div(R, 4 * Rq) >= 148;
            if (const char* env = getenv("MOQ_SB_QUAD")) quad = atoi(env) != 0 && dmax <= 4;
            if (quad) {
                a.Rb = 4 * Rq;
                const int threads = a.n * Rq;
                const int pump = p->schedule ? kPumpSchedule : (a.T <= kPumpTableMax && threads <= kPumpTableMaxThreads ? kPumpTable : kPumpInline);
                const size_t smem = sb_smem_bytes_h4(a.Rb, a.W, pump == kPumpTable ? a.T : 0);
                const dim3 block(threads), grid((unsigned)ceil_div(R, a.Rb));
                const cudaError_t e = (p->variant == MOQ_DSB) ? launch_variant_h4<MOQ_DSB>(a, dmax, noise, pump, grid, block, smem, as_stream(stream))
                                                              : launch_variant_h4<MOQ_BSB>(a, dmax, noise, pump, grid, block, smem, as_stream(stream));
                if (e != cudaSuccess) return cuda_fail(e, "moq_sample launch (FP16, four replicas per thread)");
                return MOQ_OK;
            }
        }
        // pairs of replicas per thread, replicas per block as for the FP32 pair form
        const int Rp = choose_rb(a.n, (R + 1) / 2);
        a.Rb = 2 * Rp;
        const int threads = a.n * Rp;
        int pump = p->schedule ? kPumpSchedule : (a.T <= kPumpTableMax && threads <= kPumpTableMaxThreads ? kPumpTable : kPumpInline);
        const size_t smem = sb_smem_bytes_h(a.Rb, a.W, pump == kPumpTable ? a.T : 0);
        if (pump != kPumpTable && threads <= kCapThreads) {
            auto kof = [&](int pu) {
                return p->variant == MOQ_DSB ? kernel_of_variant_h<MOQ_DSB>(dmax, noise, pu) : kernel_of_variant_h<MOQ_BSB>(dmax, noise, pu);
            };
            if (cap_choice(resident_blocks(kof(pump + 3), threads, smem) > resident_blocks(kof(pump), threads, smem))) pump += 3;
        }
        const dim3 block(threads), grid((unsigned)ceil_div(R, a.Rb));
        const cudaError_t e = (p->variant == MOQ_DSB) ? launch_variant_h<MOQ_DSB>(a, dmax, noise, pump, grid, block, smem, as_stream(stream))
                                                      : launch_variant_h<MOQ_BSB>(a, dmax, noise, pump, grid, block, smem, as_stream(stream));
        if (e != cudaSuccess) return cuda_fail(e, "moq_sample launch (FP16)");
        return MOQ_OK;
    }
    // Block shape of either form: replicas per block, threads, pump source, shared memory.
    // The table trades a multiply-add for a shared-memory load: a gain for small blocks, a
    // loss for blocks of more than 256 threads, whose gathers already keep the shared-memory
    // pipe busy (measured: n = 42..150 3-5 % faster, n = 300..1024 2-5 % slower).
    struct Shape {
        int Rb, threads, pump;
        size_t smem;
    };
    auto shape_of = [&](bool pair) {
        Shape sh;
        if (pair) {
            const int Rp = choose_rb(a.n, (R + 1) / 2);
            sh.Rb = 2 * Rp;
            sh.threads = a.n * Rp;
        } else {
            sh.Rb = choose_rb(a.n, R);
            sh.threads = a.n * sh.Rb;
        }
        sh.pump = p->schedule ? kPumpSchedule : (a.T <= kPumpTableMax && sh.threads <= kPumpTableMaxThreads ? kPumpTable : kPumpInline);
        sh.smem = pair ? sb_smem_bytes2(sh.Rb, a.W, sh.pump == kPumpTable ? a.T : 0) : sb_smem_bytes(sh.Rb, a.W, sh.pump == kPumpTable ? a.T : 0);
        return sh;
    };
    const Shape one = shape_of(false);
    Shape two = shape_of(true);
    if (dmax <= 4 && two.pump != kPumpTable && two.threads <= kCapThreads) {
        auto kof = [&](int pu) {
            return p->variant == MOQ_DSB ? kernel_of_variant<MOQ_DSB>(dmax, noise, true, pu) : kernel_of_variant<MOQ_BSB>(dmax, noise, true, pu);
        };
        if (cap_choice(resident_blocks(kof(two.pump + 3), two.threads, two.smem) > resident_blocks(kof(two.pump), two.threads, two.smem)))
            two.pump += 3;
    }
    // two replicas per thread (degree bound <= 4) when that keeps more replicas in flight per
    // SM (n = 42: 8 blocks of 6 against 10 of 3; n = 1024: one block either way; n = 600: 2
    // against 2, where the one-replica form hides latency with twice the warps) and its grid
    // fills at least two waves: below that the per-block latency decides and the shorter
    // one-replica blocks finish first (n = 42, R = 1024: 0.100 against 0.120 ms; n = 300,
    // R = 1024: 0.48 against 0.55 ms); MOQ_SB_PAIR = 0 / 1 forces a form
    bool pair = false;
    {
        auto blocks_per_sm = [&](bool pr, const Shape& sh) -> int {
            const void* k = p->variant == MOQ_DSB ? kernel_of_variant<MOQ_DSB>(dmax, noise, pr, sh.pump)
                                                  : kernel_of_variant<MOQ_BSB>(dmax, noise, pr, sh.pump);
            int blocks = 0;
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, sh.threads, sh.smem) != cudaSuccess) {
                (void)cudaGetLastError();
                return 0;
            }
            return blocks;
        };
        if (R > 1 && dmax <= 4) {
            int dev = 0, sms = 0;
            if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                sms = 148;
            const int b1 = blocks_per_sm(false, one), b2 = blocks_per_sm(true, two);
            const int64_t grid2 = ceil_div(R, two.Rb);
            pair = (int64_t)b2 * two.Rb > (int64_t)b1 * one.Rb && grid2 >= 2 * (int64_t)sms * b2;
        }
        if (const char* env = getenv("MOQ_SB_PAIR")) {
            const int v = atoi(env);
            if (v == 0) pair = false;
            if (v == 1 && dmax <= 4) pair = true;
        }
    }
    // graphs of more than 640 spins (one pair-form block per SM): two spins per thread when the
    // grid of replica pairs still fills two waves (MOQ_SB_TWOSPIN = 0 / 1 forces the choice)
    {
        bool two_spin = dmax <= 4 && a.n > kCapThreads && ceil_div(R, 2) >= 4 * 148;
        if (const char* env = getenv("MOQ_SB_TWOSPIN")) two_spin = atoi(env) != 0 && dmax <= 4 && a.n > 32;
        if (two_spin) {
            a.Rb = 2;
            const dim3 block2((unsigned)two_spin_threads(a.n)), grid2((unsigned)ceil_div(R, 2));
            const size_t smem2 = sb_smem_bytes2s(a.W);
            const bool sched = p->schedule != nullptr;
            const cudaError_t e2 = (p->variant == MOQ_DSB) ? launch_variant2s<MOQ_DSB>(a, dmax, noise, sched, grid2, block2, smem2, as_stream(stream))
                                                           : launch_variant2s<MOQ_BSB>(a, dmax, noise, sched, grid2, block2, smem2, as_stream(stream));
            if (e2 != cudaSuccess) return cuda_fail(e2, "moq_sample launch (two spins per thread)");
            return MOQ_OK;
        }
    }
    const Shape& sh = pair ? two : one;
    a.Rb = sh.Rb;
    const dim3 block(sh.threads), grid((unsigned)ceil_div(R, sh.Rb));
    cudaError_t e;
    if (pair)
        e = (p->variant == MOQ_DSB) ? launch_variant2<MOQ_DSB>(a, dmax, noise, sh.pump, grid, block, sh.smem, as_stream(stream))
                                    : launch_variant2<MOQ_BSB>(a, dmax, noise, sh.pump, grid, block, sh.smem, as_stream(stream));
    else
        e = (p->variant == MOQ_DSB) ? launch_variant<MOQ_DSB>(a, dmax, noise, sh.pump, grid, block, sh.smem, as_stream(stream))
                                    : launch_variant<MOQ_BSB>(a, dmax, noise, sh.pump, grid, block, sh.smem, as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, "moq_sample launch");
    return MOQ_OK;
}
