// Dense NI-SB on the 5th-generation tensor cores (SB equations and Eq. NI-SB,
// "Simulated Bifurcation with Gaussian noise"): for dense couplings the force
// c0 sum_j J(c)_ij phi(x_j) = c0 sum_k c_k (J^(k) Phi)_i is a matrix product, so every
// step computes G_k = J^(k) Phi for all K objectives with tcgen05.mma and applies the
// symplectic update, the wall and the next phi in the epilogue.
//
// Step kernel, tiles of 128 spins (M) x 128 replicas (N), one persistent CTA per SM:
//  - the K-dimension (spins j) is walked in chunks of 64. A producer thread loads the
//    chunk's operands with TMA into the 128-byte-swizzled K-major layout the tensor core
//    reads: J^(k)[i0:+128, j0:+64] of every objective and Phi[r0:+128, j0:+64]. Three
//    stages for K <= 3, two for K = 4;
//  - an MMA thread waits for a stage's "full" barrier (its bytes landed), issues
//    tcgen05.mma (BF16 x BF16 -> FP32, M=128, N=128, K=16) into one TMEM accumulator per
//    objective (K x 128 of the 512 columns), and tcgen05.commit arrives on the stage's
//    "empty" barrier, after which the producer refills it;
//  - the epilogue (16 warps; warp w reads TMEM lanes 32*(w%4).. of columns 32*(w/4)..) forms
//    f = -c0_r sum_k c_rk G_k[i, r], updates x, y (FP32, in HBM), applies the wall and
//    writes phi(x) as BF16 for the next step.
// Every wait on an mbarrier is bounded in time (globaltimer); on time-out the kernel records
// an error flag, waits (bounded) for the products it issued, frees its TMEM and returns.
//
// Exactness: J^(k) is rounded to BF16 (integers |J| <= 256 are exact); with dSB phi = +-1
// is exact, so G_k is an exact integer sum below 2^24 for |J| <= 256; bSB rounds x to BF16.
// Noise: Gaussian number (r & 7) of Philox4x32-10(key = seed, counter = (m, i, 2^30 +
// (r >> 3), round)) -- word (r & 7) >> 1, cosine for even r, sine for odd r, Box-Muller on
// 16-bit halves -- i.e. the eight replicas of an aligned octet share one block per step.
// Start state: the same counter (0xFFFFFFFF, i, r, round) as the sparse sampler.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <stdlib.h>

#include "dense_common.cuh"

struct moq_dense {
    int32_t n = 0, K = 0, n_pad = 0, max_R = 0, R_pad = 0;
    const moq_instance* inst = nullptr;
    __nv_bfloat16* J = nullptr;                  // K x n_pad x n_pad, row-major, zero-padded
    float* x = nullptr;                          // R_pad x n_pad
    float* y = nullptr;                          // R_pad x n_pad
    __nv_bfloat16* phi[2] = {nullptr, nullptr};  // R_pad x n_pad
    float* c0 = nullptr;                         // R_pad
    __nv_bfloat16* J_hi = nullptr;               // J = 256 J_hi + J_lo, both exact in BF16 (|J| <= kSplitMax)
    __nv_bfloat16* J_lo = nullptr;
    unsigned long long* acc = nullptr;           // R_pad x K: s^T J_k s of the configurations being evaluated
    int32_t* maxabs = nullptr;                   // max |J| (device), read back at create
    int32_t max_abs_weight = 0;
    CUtensorMap tm_J;                            // K x n_pad x n_pad, box 64 x 128 x 1
    CUtensorMap tm_Jhi, tm_Jlo;                  // the two halves, box 64 x 128 x 1
    bool resident = false;                       // all steps in one launch (n_pad = 128, K <= 3)
    CUtensorMap tm_phi[2];                       // R_pad x n_pad, box 64 x 128
    int32_t sms = 148;                           // persistent step kernel: one CTA per SM
    int32_t* status = nullptr;                   // device error flags
    int32_t* h_status = nullptr;                 // pinned
    // FP8 (e4m3) operands of the dSB step: J^(k)_ij = rowscale_k(i) * J8, phi = +-1 exact
    __nv_fp8_e4m3* J8 = nullptr;                 // K x n_pad x n_pad
    float* rowscale = nullptr;                   // K x n_pad, powers of two
    __nv_fp8_e4m3* phi8[2] = {nullptr, nullptr}; // R_pad x n_pad
    CUtensorMap tm_J8;                           // box 128 x 128 x 1 (128 bytes per row, as BF16)
    CUtensorMap tm_phi8[2];                      // box 128 x 128
    // split-precision operands (moq_sample_dense_split): J = BF16(J) + J_res with the residual
    // exact in BF16 (|J| <= kSplitMax), and for bSB phi = phi_hi + phi_lo (two BF16 parts)
    __nv_bfloat16* J_res = nullptr;              // K x n_pad x n_pad
    __nv_bfloat16* phi_lo[2] = {nullptr, nullptr};  // R_pad x n_pad
    CUtensorMap tm_Jres;                         // box 64 x 128 x 1
    CUtensorMap tm_philo[2];                     // box 64 x 128
};

namespace moq {
namespace {

constexpr int kTileM = 128, kTileN = 128, kChunkK = 64;
constexpr int kTileBytes = kTileM * kChunkK * 2;  // 16 KB per operand tile
constexpr int kThreads = 512;
// three operand stages (prefetch distance 2) when they fit in shared memory, else two
__host__ __device__ constexpr int dense_stages(int K) { return K <= 3 ? 3 : 2; }
constexpr uint64_t kWaitNs = 2000000000ull;        // bound of every mbarrier wait (2 s)
constexpr int32_t kSplitMax = 65408;               // |J| bound of the exact two-part split (256 * 255 + 128)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B
// apart (stride byte offset), descriptor version 1 (bits 46-47), layout type 2 (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
           ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9, 10-12 = 1),
// both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);

// kind::f8f6f4 with A = B = E4M3 (format 0 in bits 7-9 and 10-12), D = F32, both K-major.
constexpr uint32_t kIdescE4m3 = (1u << 4) | ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
// one K-chunk is 128 bytes of a row in either precision: 64 BF16 or 128 E4M3 elements, and one
// MMA consumes 32 bytes of it (K = 16 BF16 or K = 32 E4M3)
template <bool F8>
__host__ __device__ constexpr int chunk_elems() { return F8 ? 128 : kChunkK; }
// operand forms of the step kernel
constexpr int kPrecBf16 = 0, kPrecE4m3 = 1, kPrecSplit = 2;
// products per K-chunk: one, or for the split form (J_main + J_res) phi (dSB: phi = +-1 is
// exact in BF16) and J_main phi_hi + J_res phi_hi + J_main phi_lo (bSB; J_res phi_lo is below
// 2^-17 of the product and left out)
template <int PREC, int VARIANT>
__host__ __device__ constexpr int prec_passes() { return PREC == kPrecSplit ? (VARIANT == MOQ_DSB ? 2 : 3) : 1; }

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase of the given parity: gives up after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
                 "l"(da), "l"(db), "r"(kIdescBf16), "r"(accumulate)
                 : "memory");
}

__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
                 "l"(da), "l"(db), "r"(kIdescE4m3), "r"(accumulate)
                 : "memory");
}

// TMA tiled loads into this CTA's shared memory, completing bytes on an mbarrier.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2, uint32_t mbar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, uint32_t mbar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]), "=r"(u[9]),
          "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(u[q]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t u[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(u[q]);
}

struct DenseStepArgs {
    __nv_bfloat16* phi_out;
    __nv_fp8_e4m3* phi8_out;   // FP8 form
    __nv_bfloat16* philo_out;  // split form, bSB: BF16(x - BF16(x))
    const float* rowscale;     // FP8 form: K x n_pad scales of the J8 rows
    float* x;
    float* y;
    const float* lambda;  // R x K
    const float* c0;
    int32_t n, n_pad, R, K, m;
    float cm;  // a_m - a0 (when schedule is NULL)
    const float* schedule;
    float a0, dt, kappa, dta0;
    uint32_t key0, key1, round32;
    int32_t* status;
};

// The products G_k = A_k B^T of one 128 x 128 tile for every objective k, accumulated in
// TMEM columns k * 128.. (the exact cut evaluation): thread 0 is the TMA producer, thread 32
// issues the MMAs and releases each stage; `done` flips once all products are complete.
// Returns false on a timed-out wait (role threads only).
template <int KOBJ>
__device__ __forceinline__ bool dense_products(const CUtensorMap* tmA, const CUtensorMap* tmB, uint32_t base, uint64_t* full,
                                               uint64_t* empty, uint64_t* done, uint32_t tmem, int i0, int r0, int nchunks)
{
    constexpr int kStageBytes = (KOBJ + 1) * kTileBytes;
    constexpr int S = dense_stages(KOBJ);
    const int tid = threadIdx.x;
    bool ok = true;
    if (tid == 0) {
        // producer: chunk c goes to stage c % S once the products of chunk c - S released it
        for (int c = 0; c < nchunks && ok; ++c) {
            const int st = c % S;
            if (c >= S && !mbar_wait(smem_u32(&empty[st]), (uint32_t)(((c - S) / S) & 1))) {
                ok = false;
                break;
            }
            const uint32_t stage = base + st * kStageBytes, fb = smem_u32(&full[st]);
            mbar_expect_tx(fb, (uint32_t)kStageBytes);
            const int j0 = c * kChunkK;
#pragma unroll
            for (int k = 0; k < KOBJ; ++k) tma_load_3d(stage + k * kTileBytes, tmA, j0, i0, k, fb);
            tma_load_2d(stage + KOBJ * kTileBytes, tmB, j0, r0, fb);
        }
        // the last release of every stage has arrived before this CTA may leave
        for (int st = 0; st < S && st < nchunks && ok; ++st) {
            const int c_last = st + ((nchunks - 1 - st) / S) * S;
            if (!mbar_wait(smem_u32(&empty[st]), (uint32_t)((c_last / S) & 1))) ok = false;
        }
    } else if (tid == 32) {
        // MMA issuer
        for (int c = 0; c < nchunks; ++c) {
            const int st = c % S;
            if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((c / S) & 1))) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t stage = base + st * kStageBytes;
#pragma unroll
            for (int k = 0; k < KOBJ; ++k)
#pragma unroll
                for (int ks = 0; ks < kChunkK / 16; ++ks)
                    mma_bf16(tmem + k * kTileN, sw128_desc(stage + k * kTileBytes + ks * 32),
                             sw128_desc(stage + KOBJ * kTileBytes + ks * 32), (c > 0 || ks > 0) ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&empty[st]))
                         : "memory");
        }
        // the products of this CTA are complete once `done` flips
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(done)) : "memory");
    }
    __syncwarp();  // lanes 1-31 of warps 0 and 1 wait for their role thread before any block barrier
    return ok;
}

// ---- one SB step over all tiles: persistent and warp-specialised ---------------------
// Tiles of 128 spins x 128 replicas. One CTA per SM walks its tiles b, b + G, ...; warp 0 is
// the TMA producer, warp 1 issues the MMAs, warps 2..17 run the epilogue. The epilogue reads
// the K accumulators of a tile, combines them into the force (32 values per thread, in
// registers) and releases TMEM at once, so the products of the next tile run on the tensor
// cores while the same warps stream the state update (x, y in, x, y, phi out) through HBM.
constexpr int kWsEpiWarps = 16;
constexpr int kWsThreads = 32 * (2 + kWsEpiWarps);

// F8: the operands are E4M3 (J8 rows with a power-of-two scale per row and objective, phi = +-1
// exact for dSB) multiplied by kind::f8f6f4 MMAs; a K-chunk is then 128 spins (the same 128
// bytes per row, so the stages, swizzle and descriptors are those of BF16), and the epilogue
// applies the row scale to each accumulator before the force combination.
//
// Split (PREC = kPrecSplit): every K-chunk is multiplied in P passes into the same FP32
// accumulator, each pass a full stage: (J_main, phi) and (J_res, phi) for dSB -- exact integer
// products, the FP32 force -- and (J_main, phi_hi), (J_res, phi_hi), (J_main, phi_lo) for bSB.
template <int VARIANT, int KOBJ, bool NOISE, int PREC>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_dense_step_ws(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmPhi,
                    const __grid_constant__ CUtensorMap tmJ2, const __grid_constant__ CUtensorMap tmPhi2, const DenseStepArgs a,
                    int32_t n_ib, int32_t n_groups)
{
    constexpr bool F8 = PREC == kPrecE4m3;
    constexpr int P = prec_passes<PREC, VARIANT>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - raw);
    constexpr int kStageBytes = (KOBJ + 1) * kTileBytes;
    constexpr int S = dense_stages(KOBJ);
    uint64_t* full = reinterpret_cast<uint64_t*>(gbase + S * kStageBytes);  // S
    uint64_t* empty = full + S;                                             // S
    uint64_t* tfull = empty + S;     // products of a tile complete (MMA -> epilogue)
    uint64_t* tempty = tfull + 1;    // accumulators read (epilogue -> MMA), one arrival per epilogue warp
    uint64_t* drained = tempty + 1;  // every issued product complete (teardown)
    uint64_t* lready = drained + 1;  // 2: lambda / c0 buffer filled, one arrival per epilogue warp
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(lready + 2);
    float* lam_s = reinterpret_cast<float*>(gbase + S * kStageBytes + 128);  // 2 x kTileN x KOBJ
    float* c0_s = lam_s + 2 * kTileN * KOBJ;                                 // 2 x kTileN

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int kCk = chunk_elems<F8>();
    const int np = a.n_pad, nchunks = np / kCk;
    const int cid = blockIdx.x, nctas = gridDim.x;
    // Tile g: replica block by replica block over all spin blocks; the split form (J and J_res,
    // 50 MB at n = 2048) walks the spin blocks in two halves (when their count is even), so that
    // a wave of 148 tiles reads half of J and J_res with the phi rows of about 18 replica blocks,
    // a working set the L2 keeps across the waves of that half (DRAM reads per step 505 -> 382
    // MB); the one-operand forms keep the plain order, whose J the L2 already keeps (halves
    // would read phi twice: 197 -> 223 MB)
    const int halves = (PREC == kPrecSplit && n_ib % 2 == 0 && n_ib >= 4) ? 2 : 1;
    const int ib_h = n_ib / halves;
    const int per_half = n_groups / halves;
    auto tile_of = [&](int g, int& i0, int& r0) {
        const int h = g / per_half, rem = g - h * per_half;
        i0 = (h * ib_h + rem % ib_h) * kTileM;
        r0 = (rem / ib_h) * kTileN;
    };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 32) {
        for (int st = 0; st < S; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[st])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[st])), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(tfull)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(tempty)), "r"(kWsEpiWarps));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(drained)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&lready[0])), "r"(kWsEpiWarps));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&lready[1])), "r"(kWsEpiWarps));
        asm volatile("fence.mbarrier_init.release.cluster;");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmJ)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmPhi)) : "memory");
        if (P > 1) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmJ2)) : "memory");
        if (P > 2) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmPhi2)) : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {  // producer
            int gc = 0;
            for (int g = cid; g < n_groups && ok; g += nctas) {
                int i0, r0;
                tile_of(g, i0, r0);
                for (int vc = 0; vc < nchunks * P; ++vc, ++gc) {  // chunk vc / P, pass vc % P
                    const int st = gc % S;
                    if (gc >= S && !mbar_wait(smem_u32(&empty[st]), (uint32_t)(((gc - S) / S) & 1))) {
                        ok = false;
                        break;
                    }
                    const uint32_t stage = base + st * kStageBytes, fb = smem_u32(&full[st]);
                    mbar_expect_tx(fb, (uint32_t)kStageBytes);
                    const int j0 = (vc / P) * kCk, pass = vc % P;
                    const CUtensorMap* tA = (P > 1 && pass == 1) ? &tmJ2 : &tmJ;
                    const CUtensorMap* tB = (P > 2 && pass == 2) ? &tmPhi2 : &tmPhi;
#pragma unroll
                    for (int k = 0; k < KOBJ; ++k) tma_load_3d(stage + k * kTileBytes, tA, j0, i0, k, fb);
                    tma_load_2d(stage + KOBJ * kTileBytes, tB, j0, r0, fb);
                }
            }
            // no copy into this CTA is still in flight when it leaves (gc chunks were issued)
            for (int st = 0; st < S && st < gc; ++st) {
                const int c_last = st + ((gc - 1 - st) / S) * S;
                if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((c_last / S) & 1))) ok = false;
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int gc = 0, lt = 0;
            for (int g = cid; g < n_groups && ok; g += nctas, ++lt) {
                // the epilogue has read the previous tile's accumulators
                if (lt > 0 && !mbar_wait(smem_u32(tempty), (uint32_t)((lt - 1) & 1))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                for (int vc = 0; vc < nchunks * P; ++vc, ++gc) {
                    const int st = gc % S;
                    if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((gc / S) & 1))) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t stage = base + st * kStageBytes;
#pragma unroll
                    for (int k = 0; k < KOBJ; ++k)
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {  // 4 x 32 bytes of the 128-byte chunk
                            if (F8)
                                mma_e4m3(tmem + k * kTileN, sw128_desc(stage + k * kTileBytes + ks * 32),
                                         sw128_desc(stage + KOBJ * kTileBytes + ks * 32), (vc > 0 || ks > 0) ? 1u : 0u);
                            else
                                mma_bf16(tmem + k * kTileN, sw128_desc(stage + k * kTileBytes + ks * 32),
                                         sw128_desc(stage + KOBJ * kTileBytes + ks * 32), (vc > 0 || ks > 0) ? 1u : 0u);
                        }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&empty[st]))
                                 : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(tfull))
                             : "memory");
            }
            // teardown: everything issued is complete before TMEM is freed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(drained))
                         : "memory");
            if (!mbar_wait(smem_u32(drained), 0u)) ok = false;
        }
        __syncwarp();
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4).. (its spins) and columns 32 part..
        const int quarter = warp & 3, part = (warp - 2) >> 2;
        const float cm = a.schedule ? (__ldg(a.schedule + a.m) - a.a0) : a.cm;
        // lambda and c0 of a tile's replicas go to shared memory one tile ahead (buffer lt & 1);
        // buffer reuse is ordered by the TMEM hand-off: a warp fills buffer b for tile lt + 2
        // only after the products of tile lt + 1, which wait for every warp to read tile lt
        const int e = tid - 64;
        auto stage_lambda = [&](int g, int b) {
            int i0_unused, r0;
            tile_of(g, i0_unused, r0);
            for (int q = e; q < kTileN * (KOBJ + 1); q += 32 * kWsEpiWarps) {
                const int rl = q / (KOBJ + 1), k = q - rl * (KOBJ + 1), r = r0 + rl;
                const float v = r < a.R ? (k < KOBJ ? a.lambda[(int64_t)r * KOBJ + k] : a.c0[r]) : 0.0f;
                if (k < KOBJ) lam_s[b * kTileN * KOBJ + rl * KOBJ + k] = v;
                else c0_s[b * kTileN + rl] = v;
            }
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&lready[b])) : "memory");
        };
        stage_lambda(cid, 0);
        int lt = 0;
        for (int g = cid; g < n_groups; g += nctas, ++lt) {
            int i0, r0;
            tile_of(g, i0, r0);
            const int i = i0 + quarter * 32 + lane;
            const int b = lt & 1;
            const bool got = __all_sync(0xffffffffu, mbar_wait(smem_u32(tfull), (uint32_t)(lt & 1)) &&
                                                         mbar_wait(smem_u32(&lready[b]), (uint32_t)((lt >> 1) & 1)));
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (!got) {
                ok = false;
                break;
            }
            const float* lam_t = lam_s + b * kTileN * KOBJ;
            const float* c0_t = c0_s + b * kTileN;
            // the force of the warp's 32 replica columns, 8 at a time (registers stay under the
            // limit 18 warps per SM leave)
            float f[32];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int col0 = part * 32 + cc * 8;
                float g[KOBJ][8];
#pragma unroll
                for (int k = 0; k < KOBJ; ++k) tmem_ld8(tmem + ((uint32_t)(quarter * 32) << 16) + k * kTileN + col0, g[k]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (F8) {  // the scale of this spin's J8 row per objective
#pragma unroll
                    for (int k = 0; k < KOBJ; ++k) {
                        const float sc = __ldg(a.rowscale + (int64_t)k * np + i);
#pragma unroll
                        for (int q = 0; q < 8; ++q) g[k][q] *= sc;
                    }
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int rl = col0 + q;
                    float v = 0.0f;
#pragma unroll
                    for (int k = 0; k < KOBJ; ++k) v = fmaf(lam_t[rl * KOBJ + k], g[k][q], v);
                    f[cc * 8 + q] = v * -c0_t[rl];  // the force acts on the negated coupling
                }
            }
            // accumulators free: the next tile's products start while the state streams
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tempty)) : "memory");
            if (g + nctas < n_groups) stage_lambda(g + nctas, b ^ 1);
            if (i < a.n) {
                // one octet of columns per pass; the force of the next octet moves to f[0..7]
#pragma unroll 1
                for (int cc = 0; cc < 4; ++cc) {
                    const int col0 = part * 32 + cc * 8;  // one noise octet
                    float xs[8], ys[8], eta[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int r = r0 + col0 + q;
                        const bool v = r < a.R;
                        // x and y stream through once per step: loads and stores marked
                        // evict-first, so that L2 keeps the operand tiles (J, phi) instead
                        xs[q] = v ? __ldcs(a.x + (int64_t)r * np + i) : 0.0f;
                        ys[q] = v ? __ldcs(a.y + (int64_t)r * np + i) : 0.0f;
                        eta[q] = 0.0f;
                    }
                    if (NOISE) {
                        const uint32_t octet = (uint32_t)((r0 + col0) >> 3);
                        const uint4 o =
                            Philox4x32::block(make_uint4((uint32_t)a.m, (uint32_t)i, 0x40000000u + octet, a.round32), a.key0, a.key1);
#pragma unroll
                        for (int w = 0; w < 4; ++w) {
                            const float2 pr = box_muller16(word_of(o, w));
                            eta[2 * w] = pr.x;
                            eta[2 * w + 1] = pr.y;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int r = r0 + col0 + q;
                        if (r < a.R) {
                            const int64_t at = (int64_t)r * np + i;
                            float xv = xs[q], yv = ys[q];
                            sb_update<NOISE>(f[q], cm, eta[q], a.dt, a.kappa, a.dta0, xv, yv);
                            __stcs(a.x + at, xv);
                            __stcs(a.y + at, yv);
                            if (F8) {
                                a.phi8_out[at] = __nv_fp8_e4m3(phi_of<VARIANT>(xv));
                            } else {
                                const __nv_bfloat16 hi = __float2bfloat16_rn(phi_of<VARIANT>(xv));
                                a.phi_out[at] = hi;
                                if (P > 2) a.philo_out[at] = __float2bfloat16_rn(phi_of<VARIANT>(xv) - __bfloat162float(hi));
                            }
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 24; ++q) f[q] = f[q + 8];
                }
            }
        }
    }
    if (!ok) atomicOr(a.status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// operand stages, 128 B of barriers (2S + 5) and the TMEM slot, then two lambda / c0 buffers
size_t ws_smem_bytes(int K) { return 1024 + dense_stages(K) * (size_t)(K + 1) * kTileBytes + 128 + 2 * sizeof(float) * kTileN * (K + 1); }

// ---- the whole trajectory in one CTA: dense graphs of at most 128 spins ----------------
// With n_pad = 128 a CTA holds everything a block of 128 replicas needs for all T steps:
// J^(k) (K x 128 x 128 BF16) and the phi tile (128 replicas x 128 spins BF16) in shared
// memory in the operand layout, y in shared memory, x in the TMEM columns the K
// accumulators leave free (384..511 for K <= 3). Every step is: one thread issues the K
// products into TMEM, the 16 warps read G_k and x from TMEM, update x, y, write x back to
// TMEM and phi into the operand tile, then a block barrier -- no HBM traffic between the
// first load and the final state. The arithmetic and the noise counters are those of the
// step kernel, so both give the same bits.
struct ResidentArgs {
    float* x;
    float* y;
    const float* lambda;  // R x K
    const float* c0;
    int32_t n, n_pad, R, K, T;
    const float* schedule;
    float a0, a0inv, dt, kappa, dta0;
    uint32_t key0, key1, round32;
    int32_t* status;
};

constexpr int kResidentStateCol = 384;  // first TMEM column of x

__host__ __device__ constexpr size_t resident_smem_bytes(int K)
{
    return 1024 + (size_t)K * 2 * kTileBytes + 2 * kTileBytes + sizeof(float) * kTileM * kTileN + sizeof(float) * kTileN * (K + 1) + 64;
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}

// byte offset of element (row r, column j) in a 128-row x 128-column BF16 operand tile stored
// as two 64-column chunks in the 128-byte-swizzled K-major layout
__device__ __forceinline__ uint32_t sw128_offset(int r, int j)
{
    const int c = j >> 6, jj = j & 63;
    return (uint32_t)(c * kTileBytes + (r >> 3) * 1024 + (r & 7) * 128 + (((jj >> 3) ^ (r & 7)) << 4) + (jj & 7) * 2);
}

template <int VARIANT, int KOBJ, bool NOISE>
__global__ void __launch_bounds__(kThreads, 1)
    k_dense_resident(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmPhi, const ResidentArgs a)
{
    static_assert(KOBJ * kTileN <= kResidentStateCol, "x needs the TMEM columns after the accumulators");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - raw);
    const uint32_t sJ = base, sPhi = base + KOBJ * 2 * kTileBytes;
    unsigned char* phi_tile = gbase + KOBJ * 2 * kTileBytes;
    float* y_s = reinterpret_cast<float*>(gbase + (KOBJ + 1) * 2 * kTileBytes);  // [replica][spin]
    float* lam_s = y_s + kTileM * kTileN;                                          // kTileN x KOBJ
    float* c0_s = lam_s + kTileN * KOBJ;                                           // kTileN
    uint64_t* bars = reinterpret_cast<uint64_t*>(c0_s + kTileN);                   // load, mma (8-aligned)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.x * kTileN;
    const int quarter = warp & 3, part = warp >> 2;
    const int i = quarter * 32 + lane;  // spin (n_pad = 128)
    const int np = a.n_pad;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[0])), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[1])), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    for (int q = tid; q < kTileN; q += kThreads) {
        const int r = r0 + q;
        c0_s[q] = r < a.R ? a.c0[r] : 0.0f;
#pragma unroll
        for (int k = 0; k < KOBJ; ++k) lam_s[q * KOBJ + k] = r < a.R ? a.lambda[(int64_t)r * KOBJ + k] : 0.0f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);

    // operands (J^(k) and the start phi) by TMA, state (x into TMEM, y into shared memory)
    if (tid == 0) {
        const uint32_t lb = smem_u32(&bars[0]);
        mbar_expect_tx(lb, (uint32_t)((KOBJ + 1) * 2 * kTileBytes));
#pragma unroll
        for (int k = 0; k < KOBJ; ++k)
            for (int c = 0; c < 2; ++c) tma_load_3d(sJ + (k * 2 + c) * kTileBytes, &tmJ, c * kChunkK, 0, k, lb);
        for (int c = 0; c < 2; ++c) tma_load_2d(sPhi + c * kTileBytes, &tmPhi, c * kChunkK, r0, lb);
    }
    __syncwarp();  // warp 0 converges before the warp-wide TMEM stores
#pragma unroll 1
    for (int cc = 0; cc < 2; ++cc) {
        const int col0 = part * 32 + cc * 16;
        float xs[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int64_t at = (int64_t)(r0 + col0 + q) * np + i;
            xs[q] = a.x[at];
            y_s[(col0 + q) * kTileM + i] = a.y[at];
        }
        tmem_st16(lane_addr + kResidentStateCol + col0, xs);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    bool ok = mbar_wait(smem_u32(&bars[0]), 0u);
    asm volatile("tcgen05.fence::before_thread_sync;");
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;");

#pragma unroll 1
    for (int m = 0; m < a.T && ok; ++m) {
        if (tid == 0) {
#pragma unroll
            for (int k = 0; k < KOBJ; ++k)
#pragma unroll
                for (int c = 0; c < 2; ++c)
#pragma unroll
                    for (int ks = 0; ks < kChunkK / 16; ++ks)
                        mma_bf16(tmem + k * kTileN, sw128_desc(sJ + (k * 2 + c) * kTileBytes + ks * 32),
                                 sw128_desc(sPhi + c * kTileBytes + ks * 32), (c > 0 || ks > 0) ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&bars[1]))
                         : "memory");
        }
        // warp-uniform outcome: the TMEM loads and stores below are warp-wide
        const bool step_ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&bars[1]), (uint32_t)(m & 1)));
        asm volatile("tcgen05.fence::after_thread_sync;");
        const float cm = a.schedule ? (__ldg(a.schedule + m) - a.a0) : fmaf(a.a0inv, (float)m, -a.a0);
        if (step_ok && quarter * 32 < a.n) {  // warps of padding spins only (warp-uniform) have nothing to do
#pragma unroll 1
            for (int cc = 0; cc < 2; ++cc) {
                const int col0 = part * 32 + cc * 16;
                float g[KOBJ][16], xs[16];
#pragma unroll
                for (int k = 0; k < KOBJ; ++k) tmem_ld16(lane_addr + k * kTileN + col0, g[k]);
                tmem_ld16(lane_addr + kResidentStateCol + col0, xs);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float eta[16];
#pragma unroll
                for (int q8 = 0; q8 < 2; ++q8) {
#pragma unroll
                    for (int t = 0; t < 8; ++t) eta[8 * q8 + t] = 0.0f;
                    if (NOISE) {
                        const uint32_t octet = (uint32_t)((r0 + col0) >> 3) + q8;
                        const uint4 o = Philox4x32::block(make_uint4((uint32_t)m, (uint32_t)i, 0x40000000u + octet, a.round32),
                                                          a.key0, a.key1);
#pragma unroll
                        for (int w = 0; w < 4; ++w) {
                            const float2 p = box_muller16(word_of(o, w));
                            eta[8 * q8 + 2 * w] = p.x;
                            eta[8 * q8 + 2 * w + 1] = p.y;
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int rl = col0 + q, r = r0 + rl;
                    if (i < a.n && r < a.R) {
                        float f = 0.0f;
#pragma unroll
                        for (int k = 0; k < KOBJ; ++k) f = fmaf(lam_s[rl * KOBJ + k], g[k][q], f);
                        f *= -c0_s[rl];  // the force acts on the negated coupling
                        float xv = xs[q], yv = y_s[rl * kTileM + i];
                        sb_update<NOISE>(f, cm, eta[q], a.dt, a.kappa, a.dta0, xv, yv);
                        xs[q] = xv;
                        y_s[rl * kTileM + i] = yv;
                        *reinterpret_cast<__nv_bfloat16*>(phi_tile + sw128_offset(rl, i)) =
                            __float2bfloat16_rn(phi_of<VARIANT>(xv));
                    }
                }
                tmem_st16(lane_addr + kResidentStateCol + col0, xs);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        // phi written through the generic proxy is read by the next products (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        ok = __syncthreads_and(step_ok);
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (ok) {  // the final state back to HBM for the readout
#pragma unroll 1
        for (int cc = 0; cc < 2; ++cc) {
            const int col0 = part * 32 + cc * 16;
            float xs[16];
            tmem_ld16(lane_addr + kResidentStateCol + col0, xs);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int r = r0 + col0 + q;
                if (r < a.R) {
                    const int64_t at = (int64_t)r * np + i;
                    a.x[at] = xs[q];
                    a.y[at] = y_s[(col0 + q) * kTileM + i];
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(a.status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---- exact cut values on the tensor cores (Eq. single_obj) ----------------------------
// For a configuration s (+-1 per spin) and a symmetric J_k with zero diagonal,
// s^T J_k s = 2 sum_E J_e s_i s_j, so C_k(s) = 1/2 sum_E J_e (1 - s_i s_j) = (2 W_k - s^T J_k s) / 4.
// With J_k = 256 J_hi + J_lo (both parts integers exactly representable in BF16) and S the
// +-1 matrix of the configurations, the tiles G = J_part S^T are sums of at most n_pad
// products of magnitude <= 256, so the FP32 accumulators hold them exactly (below 2^24).
// The epilogue multiplies each row i of G by s_i (integer arithmetic), sums the 128 spins of
// the tile and adds it, scaled by 256 for J_hi, into a 64-bit accumulator per (sample, k).

// S[r][j] = +-1 (BF16) for r < M, j < n; 0 in the padding.
__global__ void k_dense_signs(const uint64_t* __restrict__ bits, int32_t M, int32_t W, int32_t n, int32_t np, int32_t Rp,
                              __nv_bfloat16* S)
{
    const int64_t total = (int64_t)Rp * np;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(q / np), j = (int)(q - (int64_t)r * np);
        float v = 0.0f;
        if (r < M && j < n) v = ((bits[(int64_t)r * W + (j >> 6)] >> (j & 63)) & 1ull) ? -1.0f : 1.0f;
        S[q] = __float2bfloat16_rn(v);
    }
}

template <int KOBJ>
__global__ void __launch_bounds__(kThreads, 1)
    k_dense_cuts(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmS, const uint64_t* __restrict__ bits,
                 int32_t M, int32_t W, int32_t n, int32_t np, int64_t scale, unsigned long long* acc, int32_t* status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - raw);
    constexpr int kStageBytes = (KOBJ + 1) * kTileBytes;
    constexpr int S = dense_stages(KOBJ);
    uint64_t* full = reinterpret_cast<uint64_t*>(gbase + S * kStageBytes + (size_t)kTileN * (KOBJ + 1) * 4);
    uint64_t* empty = full + S;
    uint64_t* done = empty + S;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.x * kTileM, r0 = blockIdx.y * kTileN;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int st = 0; st < S; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[st])), "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[st])), "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(done)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    bool ok = dense_products<KOBJ>(&tmA, &tmS, base, full, empty, done, tmem, i0, r0, np / kChunkK);
    const bool products = mbar_wait(smem_u32(done), 0u);
    ok = __syncthreads_and(ok && products);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        const int quarter = warp & 3, part = warp >> 2;
        const int i = i0 + quarter * 32 + lane;
#pragma unroll 1
        for (int cc = 0; cc < 2; ++cc) {
            const int col0 = part * 32 + cc * 16;
            float g[KOBJ][16];
#pragma unroll
            for (int k = 0; k < KOBJ; ++k) tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + k * kTileN + col0, g[k]);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int r = r0 + col0 + q;
                int sgn = 0;
                if (i < n && r < M) sgn = ((bits[(int64_t)r * W + (i >> 6)] >> (i & 63)) & 1ull) ? -1 : 1;
#pragma unroll
                for (int k = 0; k < KOBJ; ++k) {
                    const int v = __reduce_add_sync(0xffffffffu, sgn * __float2int_rn(g[k][q]));
                    if (lane == 0 && r < M) atomicAdd(&acc[(int64_t)r * KOBJ + k], (unsigned long long)(scale * (int64_t)v));
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

struct WeightSums {
    int64_t w[4];
};

// C_k = (2 W_k - s^T J_k s) / 4, exact in 64-bit integers.
__global__ void k_dense_cuts_finish(const unsigned long long* __restrict__ acc, int32_t M, int32_t K, WeightSums ws, int64_t* cuts)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= (int64_t)M * K) return;
    const int k = (int)(q % K);
    cuts[q] = (2 * ws.w[k] - (int64_t)acc[q]) / 4;
}

// J^(k) rows from the CSR, rounded to BF16, into the zero-padded dense matrices.
__global__ void k_dense_fill(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const int32_t* __restrict__ wn,
                             int64_t nnz, int32_t n, int32_t K, int32_t np, __nv_bfloat16* J, __nv_bfloat16* J_hi,
                             __nv_bfloat16* J_lo, __nv_bfloat16* J_res, int32_t* maxabs)
{
    int32_t mx = 0;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
        for (int32_t p = rowptr[i] + threadIdx.x; p < rowptr[i + 1]; p += blockDim.x)
            for (int k = 0; k < K; ++k) {
                const int32_t w = wn[(int64_t)k * nnz + p];
                const int64_t at = ((int64_t)k * np + i) * np + col[p];
                const __nv_bfloat16 jm = __float2bfloat16_rn((float)w);
                J[at] = jm;
                // J - BF16(J): at most half a BF16 ulp of |J|, an integer <= 128 (exact) when
                // |J| <= kSplitMax
                J_res[at] = __float2bfloat16_rn((float)w - __bfloat162float(jm));
                // J = 256 hi + lo with lo in [-128, 127]: both are integers of magnitude <= 256
                // (exact in BF16) whenever |J| <= kSplitMax
                const int32_t hi = (int32_t)(((int64_t)w + 128) >> 8);  // floor((w + 128) / 256)
                J_hi[at] = __float2bfloat16_rn((float)hi);
                J_lo[at] = __float2bfloat16_rn((float)(w - 256 * hi));
                mx = max(mx, abs(w));
            }
    if (mx > 0) atomicMax(maxabs, mx);
}

// FP8 operands of the dSB step: per row i and objective k the power-of-two scale 2^e
// (smallest e >= 0 with max_j |J^(k)_ij| <= 448 2^e, 448 the largest E4M3 value) and
// J8_ij = E4M3(J^(k)_ij / 2^e) (round to nearest even; integers |J| <= 16 are exact). One
// block per row.
__global__ void k_dense_fill8(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const int32_t* __restrict__ wn,
                              int64_t nnz, int32_t n, int32_t K, int32_t np, __nv_fp8_e4m3* J8, float* rowscale)
{
    __shared__ int32_t red;
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x)
        for (int k = 0; k < K; ++k) {
            if (threadIdx.x == 0) red = 0;
            __syncthreads();
            int32_t mx = 0;
            for (int32_t p = rowptr[i] + threadIdx.x; p < rowptr[i + 1]; p += blockDim.x)
                mx = max(mx, abs(wn[(int64_t)k * nnz + p]));
            atomicMax(&red, mx);
            __syncthreads();
            int e = 0;
            while ((double)red > 448.0 * (double)(1ll << e)) ++e;
            const float inv = ldexpf(1.0f, -e);
            for (int32_t p = rowptr[i] + threadIdx.x; p < rowptr[i + 1]; p += blockDim.x)
                J8[((int64_t)k * np + i) * np + col[p]] = __nv_fp8_e4m3((float)wn[(int64_t)k * nnz + p] * inv);
            if (threadIdx.x == 0) rowscale[(int64_t)k * np + i] = ldexpf(1.0f, e);
            __syncthreads();
        }
}

// phi_lo = BF16(x - BF16(x)) of the start state (split form, bSB); 0 on the padding
__global__ void k_dense_philo(int32_t n, int32_t np, int32_t R, int32_t R_pad, const float* __restrict__ x,
                              const __nv_bfloat16* __restrict__ phi, __nv_bfloat16* phi_lo)
{
    const int64_t total = (int64_t)R_pad * np;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(q / np), i = (int)(q - (int64_t)r * np);
        phi_lo[q] = __float2bfloat16_rn((r < R && i < n) ? x[q] - __bfloat162float(phi[q]) : 0.0f);
    }
}

size_t dense_smem_bytes(int K) { return 1024 + dense_stages(K) * (size_t)(K + 1) * kTileBytes + (size_t)kTileN * (K + 1) * 4 + 64; }

// grid: one CTA per SM, at most one per tile; `grid` carries the spin-block and
// replica-block counts
template <int VARIANT, int KOBJ, bool NOISE, int PREC>
cudaError_t launch_step(const moq_dense* d, const CUtensorMap& tm_phi, const CUtensorMap& tm_phi2, const DenseStepArgs& a, dim3 grid,
                        cudaStream_t st)
{
    auto k = k_dense_step_ws<VARIANT, KOBJ, NOISE, PREC>;
    const size_t smem = ws_smem_bytes(KOBJ);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int n_tiles = (int)(grid.x * grid.y);
    const int ctas = std::max(1, std::min(d->sms, n_tiles));
    k<<<ctas, kWsThreads, smem, st>>>(PREC == kPrecE4m3 ? d->tm_J8 : d->tm_J, tm_phi, d->tm_Jres, tm_phi2, a, (int32_t)grid.x,
                                      (int32_t)n_tiles);
    return cudaGetLastError();
}

template <int VARIANT, bool NOISE, int PREC>
cudaError_t launch_step_k(const moq_dense* d, const CUtensorMap& tm_phi, const CUtensorMap& tm_phi2, const DenseStepArgs& a, dim3 grid,
                          cudaStream_t st)
{
    switch (a.K) {
    case 2: return launch_step<VARIANT, 2, NOISE, PREC>(d, tm_phi, tm_phi2, a, grid, st);
    case 3: return launch_step<VARIANT, 3, NOISE, PREC>(d, tm_phi, tm_phi2, a, grid, st);
    default: return launch_step<VARIANT, 4, NOISE, PREC>(d, tm_phi, tm_phi2, a, grid, st);
    }
}

// variant x noise dispatch of one step of the given operand form
template <int PREC>
cudaError_t launch_step_form(const moq_dense* d, int variant, bool noise, const CUtensorMap& tm_phi, const CUtensorMap& tm_phi2,
                             const DenseStepArgs& a, dim3 grid, cudaStream_t st)
{
    if (variant == MOQ_DSB)
        return noise ? launch_step_k<MOQ_DSB, true, PREC>(d, tm_phi, tm_phi2, a, grid, st)
                     : launch_step_k<MOQ_DSB, false, PREC>(d, tm_phi, tm_phi2, a, grid, st);
    if constexpr (PREC == kPrecE4m3) {
        return cudaErrorInvalidValue;  // E4M3 phi serves dSB only (checked by the caller)
    } else {
        return noise ? launch_step_k<MOQ_BSB, true, PREC>(d, tm_phi, tm_phi2, a, grid, st)
                     : launch_step_k<MOQ_BSB, false, PREC>(d, tm_phi, tm_phi2, a, grid, st);
    }
}

template <int VARIANT, int KOBJ, bool NOISE>
cudaError_t launch_resident(const moq_dense* d, const ResidentArgs& a, int tiles, cudaStream_t st)
{
    auto k = k_dense_resident<VARIANT, KOBJ, NOISE>;
    const size_t smem = resident_smem_bytes(KOBJ);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<tiles, kThreads, smem, st>>>(d->tm_J, d->tm_phi[0], a);
    return cudaGetLastError();
}

template <int VARIANT, bool NOISE>
cudaError_t launch_resident_k(const moq_dense* d, const ResidentArgs& a, int tiles, cudaStream_t st)
{
    return a.K == 2 ? launch_resident<VARIANT, 2, NOISE>(d, a, tiles, st) : launch_resident<VARIANT, 3, NOISE>(d, a, tiles, st);
}

// Tensor maps of the J tiles (3-D: j, i, objective) and of the two Phi buffers (2-D: j, r),
// BF16, 128-byte swizzle (the layout of the MMA operands), built once per handle.
int encode_maps(moq_dense* d)
{
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    MOQ_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) return fail(MOQ_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const cuuint64_t np = (cuuint64_t)d->n_pad;
    const cuuint32_t one[3] = {1, 1, 1};
    {
        const cuuint64_t dims[3] = {np, np, (cuuint64_t)d->K};
        const cuuint64_t strides[2] = {np * 2, np * np * 2};
        const cuuint32_t box[3] = {(cuuint32_t)kChunkK, (cuuint32_t)kTileM, 1};
        CUresult r = encode(&d->tm_J, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, d->J, dims, strides, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(MOQ_ERR_CUDA, "cuTensorMapEncodeTiled(J) failed: %d", (int)r);
    }
    for (int h = 0; h < 2; ++h) {
        const cuuint64_t dims[3] = {np, np, (cuuint64_t)d->K};
        const cuuint64_t strides[2] = {np * 2, np * np * 2};
        const cuuint32_t box[3] = {(cuuint32_t)kChunkK, (cuuint32_t)kTileM, 1};
        CUresult r = encode(h ? &d->tm_Jlo : &d->tm_Jhi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, h ? d->J_lo : d->J_hi, dims, strides,
                            box, one, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(MOQ_ERR_CUDA, "cuTensorMapEncodeTiled(J split) failed: %d", (int)r);
    }
    for (int b = 0; b < 2; ++b) {
        const cuuint64_t dims[2] = {np, (cuuint64_t)d->R_pad};
        const cuuint64_t strides[1] = {np * 2};
        const cuuint32_t box[2] = {(cuuint32_t)kChunkK, (cuuint32_t)kTileN};
        CUresult r = encode(&d->tm_phi[b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, d->phi[b], dims, strides, box, one,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(MOQ_ERR_CUDA, "cuTensorMapEncodeTiled(phi) failed: %d", (int)r);
    }
    {  // the residual of the split form: as J
        const cuuint64_t dims[3] = {np, np, (cuuint64_t)d->K};
        const cuuint64_t strides[2] = {np * 2, np * np * 2};
        const cuuint32_t box[3] = {(cuuint32_t)kChunkK, (cuuint32_t)kTileM, 1};
        CUresult r = encode(&d->tm_Jres, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, d->J_res, dims, strides, box, one,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(MOQ_ERR_CUDA, "cuTensorMapEncodeTiled(J_res) failed: %d", (int)r);
    }
    for (int b = 0; b < 2; ++b) {
        const cuuint64_t dims[2] = {np, (cuuint64_t)d->R_pad};
        const cuuint64_t strides[1] = {np * 2};
        const cuuint32_t box[2] = {(cuuint32_t)kChunkK, (cuuint32_t)kTileN};
        CUresult r = encode(&d->tm_philo[b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, d->phi_lo[b], dims, strides, box, one,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(MOQ_ERR_CUDA, "cuTensorMapEncodeTiled(phi_lo) failed: %d", (int)r);
    }
    {  // FP8 operands: the same 128-byte rows, 128 E4M3 elements per chunk
        const cuuint64_t dims[3] = {np, np, (cuuint64_t)d->K};
        const cuuint64_t strides[2] = {np, np * np};
        const cuuint32_t box[3] = {128u, (cuuint32_t)kTileM, 1};
        CUresult r = encode(&d->tm_J8, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, d->J8, dims, strides, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(MOQ_ERR_CUDA, "cuTensorMapEncodeTiled(J8) failed: %d", (int)r);
    }
    for (int b = 0; b < 2; ++b) {
        const cuuint64_t dims[2] = {np, (cuuint64_t)d->R_pad};
        const cuuint64_t strides[1] = {np};
        const cuuint32_t box[2] = {128u, (cuuint32_t)kTileN};
        CUresult r = encode(&d->tm_phi8[b], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, d->phi8[b], dims, strides, box, one,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(MOQ_ERR_CUDA, "cuTensorMapEncodeTiled(phi8) failed: %d", (int)r);
    }
    return MOQ_OK;
}

void free_dense(moq_dense* d)
{
    if (!d) return;
    cudaFree(d->J);
    cudaFree(d->J_hi);
    cudaFree(d->J_lo);
    cudaFree(d->acc);
    cudaFree(d->maxabs);
    cudaFree(d->x);
    cudaFree(d->y);
    cudaFree(d->phi[0]);
    cudaFree(d->phi[1]);
    cudaFree(d->c0);
    cudaFree(d->status);
    cudaFree(d->J8);
    cudaFree(d->rowscale);
    cudaFree(d->phi8[0]);
    cudaFree(d->phi8[1]);
    cudaFree(d->J_res);
    cudaFree(d->phi_lo[0]);
    cudaFree(d->phi_lo[1]);
    if (d->h_status) cudaFreeHost(d->h_status);
    delete d;
}

// moq_sample_dense (BF16 operands) and moq_sample_dense_fp8 (E4M3 operands, dSB)
int sample_dense_impl(moq_dense* d, const float* lambda, int32_t R, const moq_sample_params* p, uint64_t seed, uint64_t round,
                      uint64_t* bits, void* stream, int prec)
{
    const bool f8 = prec == kPrecE4m3, split = prec == kPrecSplit;
    if (!d || !p) return fail(MOQ_ERR_ARG, "moq_sample_dense: NULL handle or params");
    if (R < 0 || R > d->max_R) return fail(MOQ_ERR_ARG, "moq_sample_dense: R=%d outside [0, max_replicas=%d]", R, d->max_R);
    if (p->steps < 0 || (p->variant != MOQ_DSB && p->variant != MOQ_BSB)) return fail(MOQ_ERR_ARG, "moq_sample_dense: bad steps or variant");
    if (R == 0) return MOQ_OK;
    if (!lambda || !bits) return fail(MOQ_ERR_ARG, "moq_sample_dense: NULL lambda or bits");
    if (p->replica_offset != 0) return fail(MOQ_ERR_UNSUPPORTED, "moq_sample_dense: replica_offset must be 0");
    if (p->precision != MOQ_PREC_FP32)
        return fail(MOQ_ERR_UNSUPPORTED, "moq_sample_dense: the dense forms take their operand precision from the entry point "
                                         "(state in FP32); p->precision must be MOQ_PREC_FP32");
    if (f8 && p->variant != MOQ_DSB)
        return fail(MOQ_ERR_UNSUPPORTED, "moq_sample_dense_fp8: E4M3 phi is exact for dSB only (bSB: use moq_sample_dense)");
    if (split && d->max_abs_weight > kSplitMax)
        return fail(MOQ_ERR_UNSUPPORTED, "moq_sample_dense_split: |J| = %d > %d (the residual J - BF16(J) is not exact in BF16)",
                    d->max_abs_weight, kSplitMax);
    cudaStream_t st = as_stream(stream);
    const moq_instance* h = d->inst;
    // replicas come in whole tiles (the padded replicas compute on zero weights and are never
    // written)
    const int np = d->n_pad, Rp = (int)ceil_div(R, kTileN) * kTileN;
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32), rnd = (uint32_t)round;
    k_dense_c0<<<R, 256, 0, st>>>(h->rowsum, h->rowptr, h->wn, h->nnz, d->n, d->K, lambda, R, d->c0);
    const int gi = (int)std::min<int64_t>(ceil_div((int64_t)Rp * np, 256), 148 * 32);
    if (f8) {
        k_dense_init<MOQ_DSB, __nv_fp8_e4m3><<<gi, 256, 0, st>>>(d->n, np, R, Rp, p->init_amp, p->x_init, p->y_init, key0, key1, rnd, d->x,
                                                                 d->y, d->phi8[0]);
        MOQ_CUDA_TRY(cudaMemsetAsync(d->phi8[1], 0, (size_t)Rp * np, st));  // padded entries stay 0
    } else {
        if (p->variant == MOQ_DSB)
            k_dense_init<MOQ_DSB, __nv_bfloat16><<<gi, 256, 0, st>>>(d->n, np, R, Rp, p->init_amp, p->x_init, p->y_init, key0, key1, rnd,
                                                                     d->x, d->y, d->phi[0]);
        else
            k_dense_init<MOQ_BSB, __nv_bfloat16><<<gi, 256, 0, st>>>(d->n, np, R, Rp, p->init_amp, p->x_init, p->y_init, key0, key1, rnd,
                                                                     d->x, d->y, d->phi[0]);
        MOQ_CUDA_TRY(cudaMemsetAsync(d->phi[1], 0, sizeof(__nv_bfloat16) * (size_t)Rp * np, st));  // padded entries stay 0
        if (split && p->variant == MOQ_BSB) {
            k_dense_philo<<<gi, 256, 0, st>>>(d->n, np, R, Rp, d->x, d->phi[0], d->phi_lo[0]);
            MOQ_CUDA_TRY(cudaMemsetAsync(d->phi_lo[1], 0, sizeof(__nv_bfloat16) * (size_t)Rp * np, st));
        }
    }
    MOQ_LAUNCH_CHECK("moq_sample_dense prologue");
    DenseStepArgs a{};
    a.x = d->x;
    a.y = d->y;
    a.lambda = lambda;
    a.c0 = d->c0;
    a.n = d->n;
    a.n_pad = np;
    a.R = R;
    a.K = d->K;
    a.schedule = p->schedule;
    a.a0 = p->a0;
    a.dt = p->dt;
    a.kappa = (p->noise_sqrt_dt ? sqrtf(p->dt) : p->dt) * p->alpha;
    a.dta0 = p->dt * p->a0;
    a.key0 = key0;
    a.key1 = key1;
    a.round32 = rnd;
    a.status = d->status;
    a.rowscale = d->rowscale;
    const float a0inv = p->steps > 1 ? p->a0 / (float)(p->steps - 1) : 0.0f;
    const dim3 grid(np / kTileM, Rp / kTileN);
    const bool noise = p->alpha != 0.0f;
    if (d->resident && prec == kPrecBf16 && p->steps > 0) {
        // one launch runs every step (n_pad = 128, K <= 3): same arithmetic, same bits
        ResidentArgs ra{};
        ra.x = d->x;
        ra.y = d->y;
        ra.lambda = lambda;
        ra.c0 = d->c0;
        ra.n = d->n;
        ra.n_pad = np;
        ra.R = R;
        ra.K = d->K;
        ra.T = p->steps;
        ra.schedule = p->schedule;
        ra.a0 = a.a0;
        ra.a0inv = a0inv;
        ra.dt = a.dt;
        ra.kappa = a.kappa;
        ra.dta0 = a.dta0;
        ra.key0 = key0;
        ra.key1 = key1;
        ra.round32 = rnd;
        ra.status = d->status;
        const int tiles = (int)ceil_div(R, kTileN);
        cudaError_t e;
        if (p->variant == MOQ_DSB)
            e = noise ? launch_resident_k<MOQ_DSB, true>(d, ra, tiles, st) : launch_resident_k<MOQ_DSB, false>(d, ra, tiles, st);
        else
            e = noise ? launch_resident_k<MOQ_BSB, true>(d, ra, tiles, st) : launch_resident_k<MOQ_BSB, false>(d, ra, tiles, st);
        if (e != cudaSuccess) return cuda_fail(e, "moq_sample_dense resident launch");
        k_dense_readout<<<R, 128, 0, st>>>(d->n, np, R, h->words, d->x, d->y, bits, p->x_out, p->y_out);
        MOQ_LAUNCH_CHECK("moq_sample_dense readout");
        return MOQ_OK;
    }
    for (int m = 0; m < p->steps; ++m) {
        a.m = m;
        a.cm = fmaf(a0inv, (float)m, -p->a0);
        const CUtensorMap& tm_in = f8 ? d->tm_phi8[m & 1] : d->tm_phi[m & 1];
        const CUtensorMap& tm_in2 = d->tm_philo[m & 1];
        a.phi_out = d->phi[(m + 1) & 1];
        a.phi8_out = d->phi8[(m + 1) & 1];
        a.philo_out = d->phi_lo[(m + 1) & 1];
        cudaError_t e;
        if (f8)
            e = launch_step_form<kPrecE4m3>(d, p->variant, noise, tm_in, tm_in2, a, grid, st);
        else if (split)
            e = launch_step_form<kPrecSplit>(d, p->variant, noise, tm_in, tm_in2, a, grid, st);
        else
            e = launch_step_form<kPrecBf16>(d, p->variant, noise, tm_in, tm_in2, a, grid, st);
        if (e != cudaSuccess) return cuda_fail(e, "moq_sample_dense step launch");
    }
    k_dense_readout<<<R, 128, 0, st>>>(d->n, np, R, h->words, d->x, d->y, bits, p->x_out, p->y_out);
    MOQ_LAUNCH_CHECK("moq_sample_dense readout");
    return MOQ_OK;
}

}  // namespace
}  // namespace moq

extern "C" {

int moq_dense_create(const moq_instance* inst, int32_t max_replicas, moq_dense** out)
{
    using namespace moq;
    if (!out) return fail(MOQ_ERR_ARG, "moq_dense_create: out is NULL");
    *out = nullptr;
    if (!inst || max_replicas < 1) return fail(MOQ_ERR_ARG, "moq_dense_create: NULL instance or max_replicas < 1");
    if (inst->K > 4) return fail(MOQ_ERR_UNSUPPORTED, "moq_dense_create: K=%d > 4 (one TMEM accumulator per objective)", inst->K);
    if (inst->n > 16384) return fail(MOQ_ERR_UNSUPPORTED, "moq_dense_create: n=%d > 16384", inst->n);
    moq_dense* d = new moq_dense();
    d->n = inst->n;
    d->K = inst->K;
    d->inst = inst;
    d->n_pad = (int)ceil_div(inst->n, kTileM) * kTileM;
    d->max_R = max_replicas;
    d->R_pad = (int)ceil_div(max_replicas, kTileN) * kTileN;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            sms > 0)
            d->sms = sms;
    }
    // graphs of at most 128 spins with K <= 3 run all steps in one launch from shared
    // memory and TMEM (MOQ_DENSE_RESIDENT=0 keeps the per-step kernel)
    d->resident = d->n_pad == kTileM && (d->K == 2 || d->K == 3);
    if (const char* env = getenv("MOQ_DENSE_RESIDENT"))
        if (atoi(env) == 0) d->resident = false;
    const size_t cells = (size_t)d->R_pad * d->n_pad;
    const size_t jbytes = sizeof(__nv_bfloat16) * (size_t)d->K * d->n_pad * d->n_pad;
    cudaError_t e = cudaMalloc((void**)&d->J, jbytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->J_hi, jbytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->J_lo, jbytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->acc, sizeof(unsigned long long) * (size_t)d->R_pad * d->K);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->maxabs, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->x, sizeof(float) * cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->y, sizeof(float) * cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->phi[0], sizeof(__nv_bfloat16) * cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->phi[1], sizeof(__nv_bfloat16) * cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->c0, sizeof(float) * d->R_pad);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&d->h_status, sizeof(int32_t));
    const size_t j8bytes = (size_t)d->K * d->n_pad * d->n_pad;
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->J8, j8bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->rowscale, sizeof(float) * (size_t)d->K * d->n_pad);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->phi8[0], cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->phi8[1], cells);
    if (e == cudaSuccess) e = cudaMemset(d->J8, 0, j8bytes);
    if (e == cudaSuccess) e = cudaMemset(d->rowscale, 0, sizeof(float) * (size_t)d->K * d->n_pad);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->J_res, jbytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->phi_lo[0], sizeof(__nv_bfloat16) * cells);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d->phi_lo[1], sizeof(__nv_bfloat16) * cells);
    if (e == cudaSuccess) e = cudaMemset(d->J_res, 0, jbytes);
    if (e == cudaSuccess) e = cudaMemset(d->J, 0, jbytes);
    if (e == cudaSuccess) e = cudaMemset(d->J_hi, 0, jbytes);
    if (e == cudaSuccess) e = cudaMemset(d->J_lo, 0, jbytes);
    if (e == cudaSuccess) e = cudaMemset(d->maxabs, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(d->status, 0, sizeof(int32_t));
    if (e == cudaSuccess) {
        k_dense_fill<<<std::min(d->n, 148 * 8), 128>>>(inst->rowptr, inst->col, inst->wn, inst->nnz, d->n, d->K, d->n_pad, d->J,
                                                       d->J_hi, d->J_lo, d->J_res, d->maxabs);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_dense_fill8<<<std::min(d->n, 148 * 8), 128>>>(inst->rowptr, inst->col, inst->wn, inst->nnz, d->n, d->K, d->n_pad, d->J8,
                                                        d->rowscale);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&d->max_abs_weight, d->maxabs, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        free_dense(d);
        return cuda_fail(e, "moq_dense_create");
    }
    const int rc = encode_maps(d);
    if (rc != MOQ_OK) {
        free_dense(d);
        return rc;
    }
    *out = d;
    return MOQ_OK;
}

void moq_dense_destroy(moq_dense* d) { moq::free_dense(d); }

int moq_sample_dense(moq_dense* d, const float* lambda, int32_t R, const moq_sample_params* p, uint64_t seed, uint64_t round,
                     uint64_t* bits, void* stream)
{
    return moq::sample_dense_impl(d, lambda, R, p, seed, round, bits, stream, moq::kPrecBf16);
}

int moq_sample_dense_fp8(moq_dense* d, const float* lambda, int32_t R, const moq_sample_params* p, uint64_t seed, uint64_t round,
                         uint64_t* bits, void* stream)
{
    return moq::sample_dense_impl(d, lambda, R, p, seed, round, bits, stream, moq::kPrecE4m3);
}

int moq_sample_dense_split(moq_dense* d, const float* lambda, int32_t R, const moq_sample_params* p, uint64_t seed, uint64_t round,
                           uint64_t* bits, void* stream)
{
    return moq::sample_dense_impl(d, lambda, R, p, seed, round, bits, stream, moq::kPrecSplit);
}

int moq_dense_evaluate_cuts(moq_dense* d, const uint64_t* bits, int32_t M, int64_t* cuts, void* stream)
{
    using namespace moq;
    if (!d) return fail(MOQ_ERR_ARG, "moq_dense_evaluate_cuts: NULL handle");
    if (M < 0 || M > d->max_R) return fail(MOQ_ERR_ARG, "moq_dense_evaluate_cuts: M=%d outside [0, max_replicas=%d]", M, d->max_R);
    if (M == 0) return MOQ_OK;
    if (!bits || !cuts) return fail(MOQ_ERR_ARG, "moq_dense_evaluate_cuts: NULL bits or cuts");
    if (d->max_abs_weight > kSplitMax)
        return fail(MOQ_ERR_UNSUPPORTED, "moq_dense_evaluate_cuts: max |J| = %d exceeds the exact split bound %d (use moq_evaluate_cuts)",
                    d->max_abs_weight, kSplitMax);
    cudaStream_t st = as_stream(stream);
    const moq_instance* h = d->inst;
    const int np = d->n_pad, Rp = (int)ceil_div(M, kTileN) * kTileN, W = h->words;
    MOQ_CUDA_TRY(cudaMemsetAsync(d->acc, 0, sizeof(unsigned long long) * (size_t)M * d->K, st));
    const int gi = (int)std::min<int64_t>(ceil_div((int64_t)Rp * np, 256), 148 * 32);
    k_dense_signs<<<gi, 256, 0, st>>>(bits, M, W, d->n, np, Rp, d->phi[0]);
    MOQ_LAUNCH_CHECK("moq_dense_evaluate_cuts signs");
    const dim3 grid(np / kTileM, Rp / kTileN);
    const size_t smem = dense_smem_bytes(d->K);
    // the high part floor((J + 128) / 256) is all zero when every |J| <= 127
    for (int part = (d->max_abs_weight > 127 ? 0 : 1); part < 2; ++part) {
        const CUtensorMap& tmA = part == 0 ? d->tm_Jhi : d->tm_Jlo;
        const int64_t scale = part == 0 ? 256 : 1;
        cudaError_t e = cudaSuccess;
        switch (d->K) {
        case 2:
            e = cudaFuncSetAttribute(k_dense_cuts<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                k_dense_cuts<2><<<grid, kThreads, smem, st>>>(tmA, d->tm_phi[0], bits, M, W, d->n, np, scale, d->acc, d->status);
            break;
        case 3:
            e = cudaFuncSetAttribute(k_dense_cuts<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                k_dense_cuts<3><<<grid, kThreads, smem, st>>>(tmA, d->tm_phi[0], bits, M, W, d->n, np, scale, d->acc, d->status);
            break;
        default:
            e = cudaFuncSetAttribute(k_dense_cuts<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                k_dense_cuts<4><<<grid, kThreads, smem, st>>>(tmA, d->tm_phi[0], bits, M, W, d->n, np, scale, d->acc, d->status);
            break;
        }
        if (e != cudaSuccess) return cuda_fail(e, "moq_dense_evaluate_cuts attribute");
        MOQ_LAUNCH_CHECK("moq_dense_evaluate_cuts products");
    }
    WeightSums ws{};
    for (int k = 0; k < d->K; ++k) ws.w[k] = h->info.weight_sum[k];
    k_dense_cuts_finish<<<(unsigned)ceil_div((int64_t)M * d->K, 256), 256, 0, st>>>(d->acc, M, d->K, ws, cuts);
    MOQ_LAUNCH_CHECK("moq_dense_evaluate_cuts finish");
    return MOQ_OK;
}

int moq_dense_status(moq_dense* d, void* stream)
{
    using namespace moq;
    if (!d) return fail(MOQ_ERR_ARG, "moq_dense_status: NULL handle");
    cudaStream_t st = as_stream(stream);
    MOQ_CUDA_TRY(cudaMemcpyAsync(d->h_status, d->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MOQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (*d->h_status) {
        MOQ_CUDA_TRY(cudaMemsetAsync(d->status, 0, sizeof(int32_t), st));
        return fail(MOQ_ERR_TIMEOUT, "moq_sample_dense: a tensor-core wait ran out of its budget");
    }
    return MOQ_OK;
}


}  // extern "C"
