// a6: exact cut values, Eq. (single_obj): C_k(s) = sum over edges with s_i != s_j of
// J^(k)_ij (the 1/2 (1 - s_i s_j) factor is 1 on a cut edge and 0 otherwise).
//
// Two forms, the same exact sums:
//  - one thread per sample (many samples): the block stages a chunk of the edge list
//    (endpoints and the K weights) in shared memory; every thread then walks the same edges
//    in lockstep, so the edge reads are broadcasts. A sample's packed spins sit in a register
//    (n <= 64) or in a transposed shared-memory tile (word q of thread t at [q][t]);
//  - one warp per sample (few samples, many edges): the block stages edge chunks the same
//    way, each warp takes one sample and its lanes split the chunk's edges; the lanes' int64
//    partial sums meet in a shuffle reduction.
// The XOR of the two endpoint bits selects the weight; accumulation is in int64, exact.
#include <algorithm>
#include <stdlib.h>
#include <string.h>

#include "moq_common.cuh"

namespace moq {
namespace {

constexpr int kEdgeChunk = 512;

enum BitsMode { kOneWord = 0, kSmemWords = 1, kGlobalWords = 2 };

template <int KT, int MODE>
__global__ void __launch_bounds__(256) k_cuts(int32_t W, int64_t E, const int32_t* __restrict__ ei,
                                              const int32_t* __restrict__ ej, const int32_t* __restrict__ w, int64_t M,
                                              const uint64_t* __restrict__ bits, int64_t* __restrict__ cuts)
{
    __shared__ int32_t s_i[kEdgeChunk], s_j[kEdgeChunk];
    __shared__ int32_t s_w[KT][kEdgeChunk];
    extern __shared__ uint64_t s_bits[];
    const int tid = threadIdx.x, bd = blockDim.x;
    const int64_t m = blockIdx.x * (int64_t)bd + tid;
    const bool act = m < M;

    uint64_t word0 = 0;
    if (MODE == kOneWord) {
        word0 = act ? bits[m] : 0ull;
    } else if (MODE == kSmemWords) {
        for (int q = 0; q < W; ++q) s_bits[q * bd + tid] = act ? bits[m * W + q] : 0ull;
    }
    int64_t acc[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) acc[k] = 0;

    for (int64_t e0 = 0; e0 < E; e0 += kEdgeChunk) {
        const int cnt = (int)std::min<int64_t>(kEdgeChunk, E - e0);
        __syncthreads();
        for (int t = tid; t < cnt; t += bd) {
            s_i[t] = ei[e0 + t];
            s_j[t] = ej[e0 + t];
#pragma unroll
            for (int k = 0; k < KT; ++k) s_w[k][t] = w[k * E + e0 + t];
        }
        __syncthreads();
        for (int t = 0; t < cnt; ++t) {
            const int a = s_i[t], b = s_j[t];
            uint64_t wa, wb;
            if (MODE == kOneWord) {
                wa = word0;
                wb = word0;
            } else if (MODE == kSmemWords) {
                wa = s_bits[(a >> 6) * bd + tid];
                wb = s_bits[(b >> 6) * bd + tid];
            } else {
                wa = act ? bits[m * W + (a >> 6)] : 0ull;
                wb = act ? bits[m * W + (b >> 6)] : 0ull;
            }
            const bool cut = ((wa >> (a & 63)) ^ (wb >> (b & 63))) & 1ull;
#pragma unroll
            for (int k = 0; k < KT; ++k) acc[k] += cut ? (int64_t)s_w[k][t] : 0;
        }
    }
    if (act) {
#pragma unroll
        for (int k = 0; k < KT; ++k) cuts[m * KT + k] = acc[k];
    }
}

// One warp per sample, kWarpsPerBlock samples per block; the sample's words in shared memory.
constexpr int kWarpsPerBlock = 8;
constexpr int kMaxWordsWarp = 64;  // n <= 4096

template <int KT>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) k_cuts_warp(int32_t W, int64_t E, const int32_t* __restrict__ ei,
                                                                   const int32_t* __restrict__ ej, const int32_t* __restrict__ w,
                                                                   int64_t M, const uint64_t* __restrict__ bits,
                                                                   int64_t* __restrict__ cuts)
{
    __shared__ int32_t s_i[kEdgeChunk], s_j[kEdgeChunk];
    __shared__ int32_t s_w[KT][kEdgeChunk];
    __shared__ uint64_t s_bits[kWarpsPerBlock][kMaxWordsWarp];
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    const int64_t m = blockIdx.x * (int64_t)kWarpsPerBlock + wp;
    const bool act = m < M;
    for (int q = lane; q < W; q += 32) s_bits[wp][q] = act ? bits[m * W + q] : 0ull;
    int64_t acc[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) acc[k] = 0;
    for (int64_t e0 = 0; e0 < E; e0 += kEdgeChunk) {
        const int cnt = (int)std::min<int64_t>(kEdgeChunk, E - e0);
        __syncthreads();
        for (int t = tid; t < cnt; t += blockDim.x) {
            s_i[t] = ei[e0 + t];
            s_j[t] = ej[e0 + t];
#pragma unroll
            for (int k = 0; k < KT; ++k) s_w[k][t] = w[k * E + e0 + t];
        }
        __syncthreads();
        for (int t = lane; t < cnt; t += 32) {
            const int a = s_i[t], b = s_j[t];
            const bool cut = ((s_bits[wp][a >> 6] >> (a & 63)) ^ (s_bits[wp][b >> 6] >> (b & 63))) & 1ull;
#pragma unroll
            for (int k = 0; k < KT; ++k) acc[k] += cut ? (int64_t)s_w[k][t] : 0;
        }
    }
#pragma unroll
    for (int k = 0; k < KT; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
    if (act && lane < KT) {
#pragma unroll
        for (int k = 0; k < KT; ++k)
            if (lane == k) cuts[m * KT + k] = acc[k];
    }
}

// The warp form unless the batch alone fills the GPU with threads and the edge loop is short.
// Measured (B300, CUDA events, same call): heavy-hex n=42 E=50 M=16384 11.5 vs 12.3 us (warp vs
// thread); 3-regular n=1024 E=1536 M=4096 14.2 vs 52.5 us; Appendix E n=200 E=19900 M=8192 207 vs
// 610 us; G(1000, 0.05) E=24773 M=256 69 vs 752 us; n=100 E=2505 M=100000 305 vs 304 us (a tie).
// MOQ_CUTS_FORM = thread / warp forces a form.
bool use_warp_form(int64_t M, int64_t E, int W)
{
    if (W > kMaxWordsWarp) return false;
    if (const char* env = getenv("MOQ_CUTS_FORM")) {
        if (!strcmp(env, "warp")) return true;
        if (!strcmp(env, "thread")) return false;
    }
    return M <= 65536 || E >= 4096;
}

template <int KT>
cudaError_t launch_cuts(const moq_instance* h, const uint64_t* bits, int64_t M, int64_t* cuts, cudaStream_t st)
{
    const int W = h->words;
    if (use_warp_form(M, h->E, W)) {
        k_cuts_warp<KT><<<(unsigned)ceil_div(M, kWarpsPerBlock), 32 * kWarpsPerBlock, 0, st>>>(W, h->E, h->ei, h->ej, h->w, M, bits, cuts);
        return cudaGetLastError();
    }
    if (W == 1) {
        const int bd = 256;
        k_cuts<KT, kOneWord><<<(unsigned)ceil_div(M, bd), bd, 0, st>>>(W, h->E, h->ei, h->ej, h->w, M, bits, cuts);
    } else if (W <= 48) {
        const int bd = 128;
        const size_t smem = sizeof(uint64_t) * (size_t)W * bd;
        auto k = k_cuts<KT, kSmemWords>;
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<(unsigned)ceil_div(M, bd), bd, smem, st>>>(W, h->E, h->ei, h->ej, h->w, M, bits, cuts);
    } else {
        const int bd = 128;
        k_cuts<KT, kGlobalWords><<<(unsigned)ceil_div(M, bd), bd, 0, st>>>(W, h->E, h->ei, h->ej, h->w, M, bits, cuts);
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace moq

extern "C" int moq_evaluate_cuts(const moq_instance* inst, const uint64_t* bits, int64_t M, int64_t* cuts, void* stream)
{
    using namespace moq;
    if (!inst) return fail(MOQ_ERR_ARG, "moq_evaluate_cuts: NULL instance");
    if (M < 0) return fail(MOQ_ERR_ARG, "moq_evaluate_cuts: M < 0");
    if (M == 0) return MOQ_OK;
    if (!bits || !cuts) return fail(MOQ_ERR_ARG, "moq_evaluate_cuts: NULL bits or cuts");
    cudaStream_t st = as_stream(stream);
    cudaError_t e;
    switch (inst->K) {
    case 2: e = launch_cuts<2>(inst, bits, M, cuts, st); break;
    case 3: e = launch_cuts<3>(inst, bits, M, cuts, st); break;
    case 4: e = launch_cuts<4>(inst, bits, M, cuts, st); break;
    case 5: e = launch_cuts<5>(inst, bits, M, cuts, st); break;
    case 6: e = launch_cuts<6>(inst, bits, M, cuts, st); break;
    case 7: e = launch_cuts<7>(inst, bits, M, cuts, st); break;
    default: e = launch_cuts<8>(inst, bits, M, cuts, st); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "moq_evaluate_cuts launch (or its shared-memory attribute)");
    return MOQ_OK;
}
