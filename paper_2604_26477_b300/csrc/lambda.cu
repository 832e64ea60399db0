// a2: weight vectors for the weighted-sum scalarisation ("Scalarization via the weighted
// sum method" and Appendix B): the Das-Dennis simplex lattice (optionally interior
// points only, as the paper uses) and uniform vectors on the simplex (Dirichlet(1..1)).
#include "moq_common.cuh"

namespace moq {
namespace {

// Number of compositions of `total` into `parts` parts, each >= lo.
__host__ __device__ int64_t compositions(int parts, int total, int lo)
{
    const int free_units = total - parts * lo;
    if (parts <= 0 || free_units < 0) return 0;
    // C(free_units + parts - 1, parts - 1), exact by the multiplicative recurrence
    int64_t c = 1;
    const int a = free_units + parts - 1, b = parts - 1;
    for (int q = 1; q <= b; ++q) c = c * (a - b + q) / q;
    return c;
}

// Lattice point number idx in lexicographically ascending (m_1..m_K) order.
__global__ void k_das_dennis(int K, int H, int lo, int64_t count, float* lambda)
{
    const int64_t idx0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx0 >= count) return;
    int64_t idx = idx0;
    int left = H;
    const float invH = 1.0f / (float)H;
    for (int k = 0; k < K - 1; ++k) {
        int v = lo;
        for (; v <= left; ++v) {
            const int64_t c = compositions(K - k - 1, left - v, lo);
            if (idx < c) break;
            idx -= c;
        }
        lambda[idx0 * K + k] = (float)v * invH;
        left -= v;
    }
    lambda[idx0 * K + K - 1] = (float)left * invH;
}

// c_k = e_k / sum e, e_k = -ln u_k with u_k in (0, 1] from Philox (r, k >> 2, 'LAMB', round).
__global__ void k_dirichlet(int K, int R, uint32_t key0, uint32_t key1, uint32_t round32, float* lambda)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    float e[kMaxK];
    float sum = 0.0f;
    uint4 o = make_uint4(0, 0, 0, 0);
    for (int k = 0; k < K; ++k) {
        if ((k & 3) == 0) o = Philox4x32::block(make_uint4((uint32_t)r, (uint32_t)(k >> 2), 0x4C414D42u, round32), key0, key1);
        const uint32_t word = (k & 3) == 0 ? o.x : (k & 3) == 1 ? o.y : (k & 3) == 2 ? o.z : o.w;
        const float u = (float)((word >> 8) + 1u) * 0x1p-24f;
        e[k] = -logf(u);
        sum += e[k];
    }
    for (int k = 0; k < K; ++k) lambda[(int64_t)r * K + k] = e[k] / sum;
}

}  // namespace
}  // namespace moq

extern "C" {

int moq_lambda_das_dennis(int32_t K, int32_t H, int32_t interior, float* lambda, int64_t capacity, int64_t* count_out,
                          void* stream)
{
    using namespace moq;
    if (K < 2 || K > kMaxK || H < 1 || H > 4096 || !count_out) return fail(MOQ_ERR_ARG, "moq_lambda_das_dennis: bad K=%d or H=%d", K, H);
    const int lo = interior ? 1 : 0;
    const int64_t count = compositions(K, H, lo);
    *count_out = count;
    if (count > capacity) return fail(MOQ_ERR_CAPACITY, "moq_lambda_das_dennis: %lld points > capacity %lld", (long long)count, (long long)capacity);
    if (count == 0) return MOQ_OK;
    if (!lambda) return fail(MOQ_ERR_ARG, "moq_lambda_das_dennis: NULL lambda");
    k_das_dennis<<<(unsigned)ceil_div(count, 256), 256, 0, as_stream(stream)>>>(K, H, lo, count, lambda);
    MOQ_LAUNCH_CHECK("moq_lambda_das_dennis launch");
    return MOQ_OK;
}

int moq_lambda_dirichlet(int32_t K, int32_t R, uint64_t seed, uint64_t round, float* lambda, void* stream)
{
    using namespace moq;
    if (K < 2 || K > kMaxK || R < 0) return fail(MOQ_ERR_ARG, "moq_lambda_dirichlet: bad K=%d or R=%d", K, R);
    if (R == 0) return MOQ_OK;
    if (!lambda) return fail(MOQ_ERR_ARG, "moq_lambda_dirichlet: NULL lambda");
    k_dirichlet<<<(unsigned)ceil_div(R, 256), 256, 0, as_stream(stream)>>>(K, R, (uint32_t)seed, (uint32_t)(seed >> 32),
                                                                        (uint32_t)round, lambda);
    MOQ_LAUNCH_CHECK("moq_lambda_dirichlet launch");
    return MOQ_OK;
}

}  // extern "C"
