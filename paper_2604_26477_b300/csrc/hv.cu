// a8: exact hypervolume ("Hamiltonian formulation" Eq. HV and Appendix A): the measure
// of the union of boxes prod_k [r_k, y_k] over a point set (maximisation), in 128-bit
// integers, for K = 2, 3, 4.
//
// Slicing: with the points ranked by y_{K-1} descending, the slab between the t-th and
// the (t+1)-th value is covered, in the first K-1 objectives, by exactly the points of
// rank <= t, so HV = sum_t (y_{K-1}[t] - y_{K-1}[t+1]) * HV_{K-1}(rank <= t). Every slab
// is independent, which is what the GPU parallelises:
//   K = 2: one thread per slab; its length is a prefix maximum of y_0.
//   K = 3: one thread per slab; its area is the 2-D staircase over the points sorted by
//          y_0 descending, restricted to rank_2 <= t. All threads walk the same sorted
//          sequence in lockstep from shared memory (broadcast reads).
//   K = 4: one block per slab of y_3 and one thread per sub-slab of y_2; the area walk is
//          the same staircase restricted to rank_3 <= t and rank_2 <= s.
// Ranks come from counting (O(F^2) comparisons, deterministic), ties broken by index.
// Slab contributions are reduced per block in int128 and summed by a final block.
// Points with some y_k < r_k span an empty box and are left out.
#include <algorithm>

#include "moq_common.cuh"

namespace moq {
namespace {

typedef __int128 i128;
constexpr int kThreads = 256;
constexpr int kChunk = 1024;

struct HvWs {
    int32_t* rank;   // K x F, -1 for left-out points
    int32_t* order;  // K x F, order[d*F + rank] = point
    i128* partial;   // one per block of the slab kernels
    // K = 4: the points laid out in y_0 order (y_0, y_1, rank_2, rank_3) and in y_2 order
    // (y_2, rank_2, rank_3), so the slab kernels read them contiguously
    int64_t *o0_y0, *o0_y1, *o2_y2;
    int32_t *o0_r2, *o0_r3, *o2_r2, *o2_r3;
    int32_t* fv;     // number of points kept
    int32_t* wide;   // K = 4: set when some kept point has y_k - r_k >= 2^32 (k < 3)
    i128* result;
    int32_t* flags;
};

__host__ __device__ inline size_t al256(size_t v) { return (v + 255) / 256 * 256; }

__host__ __device__ inline HvWs carve(void* base, int64_t F, int K)
{
    if (F < 1) F = 1;
    unsigned char* p = static_cast<unsigned char*>(base);
    HvWs w;
    w.rank = reinterpret_cast<int32_t*>(p);
    p += al256(sizeof(int32_t) * (size_t)K * F);
    w.order = reinterpret_cast<int32_t*>(p);
    p += al256(sizeof(int32_t) * (size_t)K * F);
    w.partial = reinterpret_cast<i128*>(p);
    p += al256(sizeof(i128) * (size_t)F);
    w.o0_y0 = reinterpret_cast<int64_t*>(p);
    w.o0_y1 = w.o0_y0 + F;
    w.o2_y2 = w.o0_y1 + F;
    w.o0_r2 = reinterpret_cast<int32_t*>(w.o2_y2 + F);
    w.o0_r3 = w.o0_r2 + F;
    w.o2_r2 = w.o0_r3 + F;
    w.o2_r3 = w.o2_r2 + F;
    p += al256(40 * (size_t)F);
    w.fv = reinterpret_cast<int32_t*>(p);
    w.wide = reinterpret_cast<int32_t*>(p + 4);
    w.result = reinterpret_cast<i128*>(p + 16);
    w.flags = reinterpret_cast<int32_t*>(p + 32);
    return w;
}

struct Ref4 {
    int64_t r[4];
};

// Ranks by counting, split over a 2-D grid so that every SM takes part: block (x, y)
// compares the kRankTile points of tile x with the kRankChunk points of chunk y and adds
// its counts to the (zeroed) rank array; integer sums, so the result does not depend on
// the order of the additions.
constexpr int kRankTile = 128;
constexpr int kRankChunk = 256;

template <int KT>
__device__ __forceinline__ bool hv_valid(const int64_t* u, const Ref4& ref)
{
    bool v = true;
#pragma unroll
    for (int k = 0; k < KT; ++k) v &= u[k] >= ref.r[k];
    return v;
}

template <int KT>
__global__ void __launch_bounds__(kRankTile) k_hv_rank_count(const int64_t* __restrict__ pts, int64_t F, Ref4 ref,
                                                             HvWs ws)
{
    __shared__ int64_t tile[kRankChunk][KT];
    __shared__ int32_t tvalid[kRankChunk];
    const int tid = threadIdx.x;
    const int64_t p = blockIdx.x * (int64_t)kRankTile + tid;
    int64_t u[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) u[k] = p < F ? pts[p * KT + k] : 0;
    const bool valid = p < F && hv_valid<KT>(u, ref);
    int32_t rank[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) rank[k] = 0;
    // grid.y is capped at 65535; the chunks beyond it are taken in strides
    for (int64_t chunk = blockIdx.y; chunk * kRankChunk < F; chunk += gridDim.y) {
        const int64_t base = chunk * kRankChunk;
        const int cnt = (int)min((int64_t)kRankChunk, F - base);
        __syncthreads();
        for (int q = tid; q < cnt; q += kRankTile) {
            int64_t v[KT];
#pragma unroll
            for (int k = 0; k < KT; ++k) v[k] = tile[q][k] = pts[(base + q) * KT + k];
            tvalid[q] = hv_valid<KT>(v, ref);
        }
        __syncthreads();
        if (!valid) continue;
        for (int t = 0; t < cnt; ++t) {
            if (!tvalid[t]) continue;
            const int64_t q = base + t;
#pragma unroll
            for (int k = 0; k < KT; ++k) rank[k] += (tile[t][k] > u[k]) || (tile[t][k] == u[k] && q < p);
        }
    }
    if (!valid) return;
#pragma unroll
    for (int k = 0; k < KT; ++k)
        if (rank[k]) atomicAdd(&ws.rank[k * F + p], rank[k]);
}

// Ranks of the kept points are a permutation of 0..Fv-1 in every objective: invert them
// into the orders, mark left-out points with -1 and count the kept ones.
template <int KT>
__global__ void __launch_bounds__(kThreads) k_hv_rank_order(const int64_t* __restrict__ pts, int64_t F, Ref4 ref,
                                                            HvWs ws)
{
    const int64_t p = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    if (p >= F) return;
    int64_t u[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) u[k] = pts[p * KT + k];
    const bool valid = hv_valid<KT>(u, ref);
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        if (valid)
            ws.order[k * F + ws.rank[k * F + p]] = (int32_t)p;
        else
            ws.rank[k * F + p] = -1;
    }
    if (valid) atomicAdd(ws.fv, 1);
}

__device__ i128 block_sum(i128 v, i128* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const i128 out = red[0];
    __syncthreads();
    return out;
}

__device__ __forceinline__ i128 shfl_down_i128(i128 v, int o)
{
    const uint64_t lo = __shfl_down_sync(0xffffffffu, (uint64_t)v, o);
    const uint64_t hi = __shfl_down_sync(0xffffffffu, (uint64_t)((unsigned __int128)v >> 64), o);
    return (i128)(((unsigned __int128)hi << 64) | lo);
}

// The block's sum (integer: independent of the order of the additions) in thread 0 only:
// warp shuffles, one barrier, and thread 0 adds the warp sums.
__device__ i128 block_sum_to0(i128 v, i128* warp_red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_down_i128(v, o);
    if ((threadIdx.x & 31) == 0) warp_red[threadIdx.x >> 5] = v;
    __syncthreads();
    i128 s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += warp_red[w];
    return s;
}

// K = 2: slab t along y_1 (order_1); length = max of y_0 over ranks <= t.
__global__ void __launch_bounds__(kThreads) k_hv2(const int64_t* __restrict__ pts, int64_t F, Ref4 ref, HvWs ws)
{
    __shared__ int64_t s_u0[kChunk];
    __shared__ i128 red[kThreads];
    const int Fv = *ws.fv;
    const int64_t t = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    const int32_t* ord1 = ws.order + F;
    int64_t h = 0;
    if (t < Fv) {
        const int64_t top = pts[(int64_t)ord1[t] * 2 + 1];
        const int64_t below = (t + 1 < Fv) ? pts[(int64_t)ord1[t + 1] * 2 + 1] : ref.r[1];
        h = top - below;
    }
    int64_t best = ref.r[0];
    const int64_t lim = min((int64_t)Fv, blockIdx.x * (int64_t)kThreads + kThreads);
    for (int64_t base = 0; base < lim; base += kChunk) {
        const int cnt = (int)min((int64_t)kChunk, lim - base);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt; q += kThreads) s_u0[q] = pts[(int64_t)ord1[base + q] * 2];
        __syncthreads();
        if (h > 0) {
            const int upto = (int)min((int64_t)cnt, t - base + 1);
            for (int q = 0; q < upto; ++q) best = max(best, s_u0[q]);
        }
    }
    const i128 c = (h > 0) ? (i128)h * (i128)(best - ref.r[0]) : (i128)0;
    const i128 s = block_sum(c, red);
    if (threadIdx.x == 0) ws.partial[blockIdx.x] = s;
}

// K = 3: slab t along y_2 (order_2); area = staircase over order_0 restricted to rank_2 <= t.
// kSlab3Threads slabs per block: each block stages the whole y_0 order once, so small
// blocks spread the slabs over more SMs at the price of more (cheap, L2-resident) staging.
constexpr int kSlab3Threads = 64;

__global__ void __launch_bounds__(kSlab3Threads) k_hv3(const int64_t* __restrict__ pts, int64_t F, Ref4 ref, HvWs ws)
{
    __shared__ int64_t s_u0[kChunk], s_u1[kChunk];
    __shared__ int32_t s_r2[kChunk];
    __shared__ i128 red[kSlab3Threads];
    const int Fv = *ws.fv;
    const int64_t t = blockIdx.x * (int64_t)kSlab3Threads + threadIdx.x;
    const int32_t* ord0 = ws.order;
    const int32_t* ord2 = ws.order + 2 * F;
    const int32_t* rank2 = ws.rank + 2 * F;
    int64_t h = 0;
    if (t < Fv) {
        const int64_t top = pts[(int64_t)ord2[t] * 3 + 2];
        const int64_t below = (t + 1 < Fv) ? pts[(int64_t)ord2[t + 1] * 3 + 2] : ref.r[2];
        h = top - below;
    }
    i128 area = 0;
    int64_t best1 = ref.r[1];
    const bool any = __syncthreads_or(h > 0);
    if (any) {
        for (int64_t base = 0; base < Fv; base += kChunk) {
            const int cnt = (int)min((int64_t)kChunk, Fv - base);
            __syncthreads();
            for (int q = threadIdx.x; q < cnt; q += kSlab3Threads) {
                const int64_t p = ord0[base + q];
                s_u0[q] = pts[p * 3];
                s_u1[q] = pts[p * 3 + 1];
                s_r2[q] = rank2[p];
            }
            __syncthreads();
            if (h > 0) {
                for (int q = 0; q < cnt; ++q) {
                    if (s_r2[q] <= t && s_u1[q] > best1) {
                        area += (i128)(s_u0[q] - ref.r[0]) * (i128)(s_u1[q] - best1);
                        best1 = s_u1[q];
                    }
                }
            }
        }
    }
    const i128 c = (h > 0) ? (i128)h * area : (i128)0;
    const i128 s = block_sum(c, red);
    if (threadIdx.x == 0) ws.partial[blockIdx.x] = s;
}

__device__ __forceinline__ int block_excl_scan_int(int v, int* warp_sums, int* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    const int res = incl - v + (wid > 0 ? warp_sums[wid - 1] : 0);
    *total = warp_sums[nw - 1];
    __syncthreads();
    return res;
}

// The K = 4 point data in y_0 order and in y_2 order (positions past the kept count unused),
// and the flag that sends the slabs to the 128-bit walk: some kept point lies 2^32 or more
// above the reference point in y_0, y_1 or y_2 (kept points lie at or above it, so the
// differences, taken modulo 2^64, are exact).
__global__ void __launch_bounds__(kThreads) k_hv_permute4(const int64_t* __restrict__ pts, int64_t F, Ref4 ref, HvWs ws)
{
    const int64_t q = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    if (q >= *ws.fv) return;
    const int32_t p0 = ws.order[q], p2 = ws.order[2 * F + q];
    const int64_t y0 = pts[(int64_t)p0 * 4], y1 = pts[(int64_t)p0 * 4 + 1], y2 = pts[(int64_t)p2 * 4 + 2];
    ws.o0_y0[q] = y0;
    ws.o0_y1[q] = y1;
    ws.o0_r2[q] = ws.rank[2 * F + p0];
    ws.o0_r3[q] = ws.rank[3 * F + p0];
    ws.o2_y2[q] = y2;
    ws.o2_r2[q] = ws.rank[2 * F + p2];
    ws.o2_r3[q] = ws.rank[3 * F + p2];
    constexpr uint64_t kMax32 = 0xFFFFFFFFull;
    if ((uint64_t)y0 - (uint64_t)ref.r[0] > kMax32 || (uint64_t)y1 - (uint64_t)ref.r[1] > kMax32 ||
        (uint64_t)y2 - (uint64_t)ref.r[2] > kMax32)
        atomicOr(ws.wide, 1);
}

// K = 4 with the slab's points compacted: block b takes slab t = F-1-b (the largest slabs
// first, so the long blocks start in the first wave) and gathers the t+1 points of
// rank_3 <= t into shared memory twice -- in y_0 order (the staircase walk) and in y_2
// order (the sub-slabs). The sub-slabs of non-zero height (one per distinct y_2 value)
// are then packed to the front of the y_2 arrays, so consecutive threads take
// consecutive non-empty sub-slabs and every warp walks with all its lanes busy.
// Shared memory: 32 B per point.
constexpr int kHv4CompactMax = 6144;

__global__ void __launch_bounds__(kThreads) k_hv4_compact(const int64_t* __restrict__ pts, int64_t F, Ref4 ref, HvWs ws)
{
    if (*ws.wide == 0) return;  // k_hv4_narrow takes every slab
    extern __shared__ __align__(16) unsigned char sm[];
    int64_t* s_u0 = reinterpret_cast<int64_t*>(sm);
    int64_t* s_u1 = s_u0 + F;
    int64_t* s_v2 = s_u1 + F;  // y_2 values; after packing, the sub-slab heights
    int32_t* s_r2 = reinterpret_cast<int32_t*>(s_v2 + F);
    int32_t* s_q2 = s_r2 + F;  // rank_2 of the y_2-ordered points; after packing, per sub-slab
    __shared__ i128 red[kThreads];
    __shared__ int warp_sums[kThreads / 32];
    const int Fv = *ws.fv;
    const int64_t t = F - 1 - (int64_t)blockIdx.x;
    const int32_t* ord3 = ws.order + 3 * F;
    int64_t h4 = 0;
    if (t < Fv) {
        const int64_t top = pts[(int64_t)ord3[t] * 4 + 3];
        const int64_t below = (t + 1 < Fv) ? pts[(int64_t)ord3[t + 1] * 4 + 3] : ref.r[3];
        h4 = top - below;
    }
    if (h4 <= 0) {  // uniform over the block
        if (threadIdx.x == 0) ws.partial[t] = 0;
        return;
    }
    // gather the points of rank_3 <= t in both orders: warp w owns a contiguous segment of
    // positions; it counts its kept points (ballots), the segment offsets come from the
    // eight counts, then it writes its points in order -- reads are contiguous and only two
    // barriers are needed
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kThreads / 32;
    const int seg = ((Fv + kWarps - 1) / kWarps + 31) & ~31;
    const int lo = wid * seg, hi = min(Fv, lo + seg);
    __shared__ int wc0[kWarps], wc2[kWarps];
    int n0 = 0, n2 = 0;
    for (int q = lo + lane; q < lo + seg; q += 32) {
        const bool f0 = q < hi && ws.o0_r3[q] <= t, f2 = q < hi && ws.o2_r3[q] <= t;
        n0 += __popc(__ballot_sync(0xffffffffu, f0));
        n2 += __popc(__ballot_sync(0xffffffffu, f2));
    }
    if (lane == 0) {
        wc0[wid] = n0;
        wc2[wid] = n2;
    }
    __syncthreads();
    int pos0 = 0, pos2 = 0, cnt0 = 0;
    for (int w = 0; w < kWarps; ++w) {
        if (w < wid) {
            pos0 += wc0[w];
            pos2 += wc2[w];
        }
        cnt0 += wc0[w];
    }
    const unsigned below = (1u << lane) - 1u;
    for (int q = lo + lane; q < lo + seg; q += 32) {
        const bool f0 = q < hi && ws.o0_r3[q] <= t, f2 = q < hi && ws.o2_r3[q] <= t;
        const unsigned b0 = __ballot_sync(0xffffffffu, f0), b2 = __ballot_sync(0xffffffffu, f2);
        if (f0) {
            const int at = pos0 + __popc(b0 & below);
            s_u0[at] = ws.o0_y0[q];
            s_u1[at] = ws.o0_y1[q];
            s_r2[at] = ws.o0_r2[q];
        }
        if (f2) {
            const int at = pos2 + __popc(b2 & below);
            s_v2[at] = ws.o2_y2[q];
            s_q2[at] = ws.o2_r2[q];
        }
        pos0 += __popc(b0);
        pos2 += __popc(b2);
    }
    __syncthreads();
    const int c = cnt0;  // == t + 1
    // pack the non-empty sub-slabs in place: chunk j reads positions [j*256, j*256+256]
    // before the scan's barriers and writes positions below its own index afterwards, so no
    // write lands on a position another thread has still to read
    int nsub = 0;
    for (int base = 0; base < c; base += kThreads) {
        const int s = base + threadIdx.x;
        int64_t h3 = 0;
        int32_t rs = 0;
        if (s < c) {
            h3 = s_v2[s] - (s + 1 < c ? s_v2[s + 1] : ref.r[2]);
            rs = s_q2[s];
        }
        int tot;
        const int pos = nsub + block_excl_scan_int(h3 > 0 ? 1 : 0, warp_sums, &tot);
        if (h3 > 0) {
            s_v2[pos] = h3;
            s_q2[pos] = rs;
        }
        nsub += tot;
    }
    __syncthreads();
    i128 acc = 0;
    for (int j = threadIdx.x; j < nsub; j += kThreads) {
        const int64_t h3 = s_v2[j];
        const int32_t rs = s_q2[j];
        i128 area = 0;
        int64_t best1 = ref.r[1];
        for (int q = 0; q < c; ++q) {
            const int64_t u1 = s_u1[q];
            if (s_r2[q] <= rs && u1 > best1) {
                area += (i128)(s_u0[q] - ref.r[0]) * (i128)(u1 - best1);
                best1 = u1;
            }
        }
        acc += (i128)h3 * area;
    }
    const i128 sum = block_sum(acc, red);
    if (threadIdx.x == 0) ws.partial[t] = (i128)h4 * sum;
}

// K = 4 with every kept point less than 2^32 above the reference point in y_0, y_1 and y_2 (the
// flag k_hv_permute4 leaves clear): k_hv4_compact's slabs, sub-slabs and sums, on 32-bit
// offsets from the reference point. A staircase area is at most the product of its two
// largest offsets, below 2^64, so the walk adds unsigned 64-bit products; each sub-slab's
// height times its area, and the slab's sum, are 128-bit as before. 20 B of shared memory per
// point instead of 32 (more resident blocks: the walk is latency-bound) and a shorter step.
__global__ void __launch_bounds__(kThreads) k_hv4_narrow(const int64_t* __restrict__ pts, int64_t F, Ref4 ref, HvWs ws)
{
    if (*ws.wide != 0) return;  // k_hv4_compact takes every slab
    extern __shared__ __align__(16) unsigned char sm[];
    uint2* s_w = reinterpret_cast<uint2*>(sm);               // (y_1 - r_1, rank_2) in y_0 order
    uint32_t* s_u0 = reinterpret_cast<uint32_t*>(s_w + F);  // y_0 - r_0 in y_0 order
    uint32_t* s_v2 = s_u0 + F;  // y_2 - r_2 in y_2 order; after packing, the sub-slab heights
    int32_t* s_q2 = reinterpret_cast<int32_t*>(s_v2 + F);  // rank_2 in y_2 order; after packing, per sub-slab
    __shared__ i128 red[kThreads / 32];
    __shared__ int warp_sums[kThreads / 32];
    const int Fv = *ws.fv;
    const int64_t t = F - 1 - (int64_t)blockIdx.x;
    const int32_t* ord3 = ws.order + 3 * F;
    int64_t h4 = 0;
    if (t < Fv) {
        const int64_t top = pts[(int64_t)ord3[t] * 4 + 3];
        const int64_t below = (t + 1 < Fv) ? pts[(int64_t)ord3[t + 1] * 4 + 3] : ref.r[3];
        h4 = top - below;
    }
    if (h4 <= 0) {  // uniform over the block
        if (threadIdx.x == 0) ws.partial[t] = 0;
        return;
    }
    // the points of rank_3 <= t in both orders, as in k_hv4_compact
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kThreads / 32;
    const int seg = ((Fv + kWarps - 1) / kWarps + 31) & ~31;
    const int lo = wid * seg, hi = min(Fv, lo + seg);
    __shared__ int wc0[kWarps], wc2[kWarps];
    // four chunks of 32 positions per round, their loads issued together (the scan is
    // latency-bound: every slab reads the whole rank_3 column of both orders)
    constexpr int kU = 4;
    int n0 = 0, n2 = 0;
    for (int base = lo; base < hi; base += 32 * kU) {  // warp-uniform trip count (ballots below)
        int a0[kU], a2[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int q = base + 32 * u + lane;
            a0[u] = q < hi ? ws.o0_r3[q] : 0x7fffffff;
            a2[u] = q < hi ? ws.o2_r3[q] : 0x7fffffff;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            n0 += __popc(__ballot_sync(0xffffffffu, a0[u] <= t));
            n2 += __popc(__ballot_sync(0xffffffffu, a2[u] <= t));
        }
    }
    if (lane == 0) {
        wc0[wid] = n0;
        wc2[wid] = n2;
    }
    __syncthreads();
    int pos0 = 0, pos2 = 0, cnt0 = 0;
    for (int w = 0; w < kWarps; ++w) {
        if (w < wid) {
            pos0 += wc0[w];
            pos2 += wc2[w];
        }
        cnt0 += wc0[w];
    }
    const unsigned below = (1u << lane) - 1u;
    for (int base = lo; base < hi; base += 32 * kU) {
        bool f0[kU], f2[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int q = base + 32 * u + lane;
            f0[u] = q < hi && ws.o0_r3[q] <= t;
            f2[u] = q < hi && ws.o2_r3[q] <= t;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int q = base + 32 * u + lane;
            const unsigned b0 = __ballot_sync(0xffffffffu, f0[u]), b2 = __ballot_sync(0xffffffffu, f2[u]);
            if (f0[u]) {
                const int at = pos0 + __popc(b0 & below);
                s_w[at] = make_uint2((uint32_t)((uint64_t)ws.o0_y1[q] - (uint64_t)ref.r[1]), (uint32_t)ws.o0_r2[q]);
                s_u0[at] = (uint32_t)((uint64_t)ws.o0_y0[q] - (uint64_t)ref.r[0]);
            }
            if (f2[u]) {
                const int at = pos2 + __popc(b2 & below);
                s_v2[at] = (uint32_t)((uint64_t)ws.o2_y2[q] - (uint64_t)ref.r[2]);
                s_q2[at] = ws.o2_r2[q];
            }
            pos0 += __popc(b0);
            pos2 += __popc(b2);
        }
    }
    __syncthreads();
    const int c = cnt0;  // == t + 1
    // non-empty sub-slabs packed in place (the order of reads and writes of k_hv4_compact)
    int nsub = 0;
    for (int base = 0; base < c; base += kThreads) {
        const int s = base + threadIdx.x;
        uint32_t h3 = 0;
        int32_t rs = 0;
        if (s < c) {
            h3 = s_v2[s] - (s + 1 < c ? s_v2[s + 1] : 0u);
            rs = s_q2[s];
        }
        int tot;
        const int pos = nsub + block_excl_scan_int(h3 > 0 ? 1 : 0, warp_sums, &tot);
        if (h3 > 0) {
            s_v2[pos] = h3;
            s_q2[pos] = rs;
        }
        nsub += tot;
    }
    __syncthreads();
    i128 acc = 0;
    for (int j = threadIdx.x; j < nsub; j += kThreads) {
        const uint32_t h3 = s_v2[j];
        const uint32_t rs = (uint32_t)s_q2[j];
        uint64_t area = 0;
        uint32_t best1 = 0;
#pragma unroll 4
        for (int q = 0; q < c; ++q) {
            const uint2 w = s_w[q];
            if (w.y <= rs && w.x > best1) {
                area += (uint64_t)s_u0[q] * (uint64_t)(w.x - best1);
                best1 = w.x;
            }
        }
        acc += (i128)h3 * (i128)area;
    }
    const i128 sum = block_sum_to0(acc, red);
    if (threadIdx.x == 0) ws.partial[t] = (i128)h4 * sum;
}

// K = 4 for fronts beyond the shared-memory form: block b takes slab t = F-1-b and streams
// the points twice, in chunks of kChunk, keeping only those of rank_3 <= t:
//  - in y_2 order, to find the non-empty sub-slabs (the last point of every run of equal
//    y_2 values; its successor may sit in the next chunk, so the last kept point of a chunk
//    is carried over), which are collected in batches of up to kSubBatch;
//  - for every batch, in y_0 order, where each thread walks the staircases of its
//    kSubPerThread sub-slabs together over the shared chunk.
constexpr int kSubPerThread = 8;
constexpr int kSubBatch = kThreads * kSubPerThread;

__global__ void __launch_bounds__(kThreads) k_hv4_stream(const int64_t* __restrict__ pts, int64_t F, Ref4 ref, HvWs ws)
{
    __shared__ int64_t s_sub_h[kSubBatch];
    __shared__ int32_t s_sub_r[kSubBatch];
    __shared__ int64_t s_a[kChunk + 1], s_b[kChunk];  // y_2 (+ carry) / y_0, and y_1
    __shared__ int32_t s_r[kChunk + 1];                // rank_2
    __shared__ i128 red[kThreads];
    __shared__ int warp_sums[kThreads / 32];
    const int Fv = *ws.fv;
    const int64_t t = F - 1 - (int64_t)blockIdx.x;
    const int32_t* ord0 = ws.order;
    const int32_t* ord2 = ws.order + 2 * F;
    const int32_t* ord3 = ws.order + 3 * F;
    const int32_t* rank2 = ws.rank + 2 * F;
    const int32_t* rank3 = ws.rank + 3 * F;
    int64_t h4 = 0;
    if (t < Fv) {
        const int64_t top = pts[(int64_t)ord3[t] * 4 + 3];
        const int64_t below = (t + 1 < Fv) ? pts[(int64_t)ord3[t + 1] * 4 + 3] : ref.r[3];
        h4 = top - below;
    }
    if (h4 <= 0) {  // uniform over the block
        if (threadIdx.x == 0) ws.partial[t] = 0;
        return;
    }
    i128 acc = 0;
    int nsub = 0;  // sub-slabs collected in the current batch

    // walk all kept points in y_0 order for the batch of nsub sub-slabs
    auto walk_batch = [&]() {
        int64_t h3[kSubPerThread], best1[kSubPerThread];
        int32_t rs[kSubPerThread];
        i128 area[kSubPerThread];
#pragma unroll
        for (int q = 0; q < kSubPerThread; ++q) {
            const int j = threadIdx.x + q * kThreads;
            h3[q] = j < nsub ? s_sub_h[j] : 0;
            rs[q] = j < nsub ? s_sub_r[j] : -1;
            best1[q] = ref.r[1];
            area[q] = 0;
        }
        for (int base = 0; base < Fv; base += kChunk) {
            __syncthreads();  // the previous chunk is consumed
            int cnt = 0;
            for (int sub = 0; sub < kChunk; sub += kThreads) {
                const int q = base + sub + threadIdx.x;
                const int p = q < Fv ? ord0[q] : 0;
                const int f = (q < Fv && rank3[p] <= t) ? 1 : 0;
                int tot;
                const int pos = cnt + block_excl_scan_int(f, warp_sums, &tot);
                if (f) {
                    s_a[pos] = pts[(int64_t)p * 4];
                    s_b[pos] = pts[(int64_t)p * 4 + 1];
                    s_r[pos] = rank2[p];
                }
                cnt += tot;
            }
            __syncthreads();
            for (int q = 0; q < cnt; ++q) {
                const int64_t u0 = s_a[q], u1 = s_b[q];
                const int32_t r2 = s_r[q];
#pragma unroll
                for (int k = 0; k < kSubPerThread; ++k) {
                    if (r2 <= rs[k] && u1 > best1[k]) {
                        area[k] += (i128)(u0 - ref.r[0]) * (i128)(u1 - best1[k]);
                        best1[k] = u1;
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kSubPerThread; ++k) acc += (i128)h3[k] * area[k];
        __syncthreads();  // the batch list is consumed
        nsub = 0;
    };

    // y_2 order: a kept point closes a non-empty sub-slab when the next kept point has a
    // smaller y_2 (or it is the last one: the sub-slab reaches r_2)
    int carry = 0;  // s_a[0] / s_r[0] hold the carried point when 1
    for (int base = 0; base < Fv; base += kChunk) {
        int cnt = carry;
        for (int sub = 0; sub < kChunk; sub += kThreads) {
            const int q = base + sub + threadIdx.x;
            const int p = q < Fv ? ord2[q] : 0;
            const int f = (q < Fv && rank3[p] <= t) ? 1 : 0;
            int tot;
            const int pos = cnt + block_excl_scan_int(f, warp_sums, &tot);
            if (f) {
                s_a[pos] = pts[(int64_t)p * 4 + 2];
                s_r[pos] = rank2[p];
            }
            cnt += tot;
        }
        __syncthreads();
        const bool last_chunk = base + kChunk >= Fv;
        const int closed = last_chunk ? cnt : cnt - 1;  // points whose successor is known
        for (int sub = 0; sub < closed; sub += kThreads) {
            const int q = sub + threadIdx.x;
            int64_t h3 = 0;
            int32_t rq = 0;
            if (q < closed) {
                h3 = s_a[q] - (q + 1 < cnt ? s_a[q + 1] : ref.r[2]);
                rq = s_r[q];
            }
            int tot;
            const int pos = nsub + block_excl_scan_int(h3 > 0 ? 1 : 0, warp_sums, &tot);
            if (h3 > 0) {
                s_sub_h[pos] = h3;
                s_sub_r[pos] = rq;
            }
            nsub += tot;
        }
        __syncthreads();
        if (!last_chunk && cnt > 0) {  // carry the last kept point to the front
            int64_t ca = 0;
            int32_t cr = 0;
            if (threadIdx.x == 0) {
                ca = s_a[cnt - 1];
                cr = s_r[cnt - 1];
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                s_a[0] = ca;
                s_r[0] = cr;
            }
            carry = 1;
        } else {
            carry = 0;
        }
        // a full chunk adds at most kChunk sub-slabs: walk once the batch could overflow
        if (nsub > kSubBatch - kChunk || (last_chunk && nsub > 0)) {
            // the carried y_2 point is restored after the walk reuses the chunk buffers
            int64_t ca = 0;
            int32_t cr = 0;
            if (carry) {
                ca = s_a[0];
                cr = s_r[0];
            }
            __syncthreads();
            walk_batch();
            if (carry && threadIdx.x == 0) {
                s_a[0] = ca;
                s_r[0] = cr;
            }
        }
        __syncthreads();
    }
    const i128 sum = block_sum(acc, red);
    if (threadIdx.x == 0) ws.partial[t] = (i128)h4 * sum;
}

// Sum of the block partials; flags bit 0 = the side-length product reaches 2^125.
__global__ void __launch_bounds__(kThreads) k_hv_final(const int64_t* __restrict__ pts, int64_t F, int K, Ref4 ref,
                                                       int64_t nparts, HvWs ws)
{
    __shared__ i128 red[kThreads];
    i128 acc = 0;
    for (int64_t q = threadIdx.x; q < nparts; q += kThreads) acc += ws.partial[q];
    const i128 s = block_sum(acc, red);
    if (threadIdx.x == 0) {
        const int Fv = *ws.fv;
        int32_t flags = 0;
        if (Fv > 0) {
            double prod = 1.0;
            for (int k = 0; k < K; ++k) prod *= (double)(pts[(int64_t)ws.order[k * F] * K + k] - ref.r[k]);
            if (prod >= 0x1p125) flags |= 1;
        }
        *ws.result = s;
        *ws.flags = flags;
    }
}

}  // namespace
}  // namespace moq

extern "C" {

int64_t moq_hypervolume_workspace_size(int64_t F, int32_t K)
{
    using namespace moq;
    if (F < 1) F = 1;
    if (K < 1) K = 1;
    return (int64_t)(al256(sizeof(int32_t) * (size_t)K * F) * 2 + al256(16 * (size_t)F) + al256(40 * (size_t)F) + 256);
}

}  // extern "C"

namespace moq {
// The hypervolume of F points in the caller's workspace. With pinned_readback the result
// words come back through a pinned buffer leased from the library's kept pinned pages (the
// process's first leases allocate a page); without it they land in this stack frame, so the
// call allocates nothing on the host or the device.
// Queues the whole hypervolume computation of F > 0 points (2 <= K <= 4) on `st`: the
// 128-bit result lands in ws.result and the overflow flag in ws.flags of the returned
// workspace view. No synchronisation.
int hv_launch(const int64_t* pts, int64_t F, int32_t K, const int64_t* ref, void* workspace, cudaStream_t st, HvWs& ws)
{
    ws = carve(workspace, F, K);
    Ref4 r{};
    for (int k = 0; k < K; ++k) r.r[k] = ref[k];
    MOQ_CUDA_TRY(cudaMemsetAsync(ws.fv, 0, 2 * sizeof(int32_t), st));  // fv and wide
    MOQ_CUDA_TRY(cudaMemsetAsync(ws.rank, 0, sizeof(int32_t) * (size_t)K * F, st));
    const unsigned gF = (unsigned)ceil_div(F, kThreads);
    const dim3 gRank((unsigned)ceil_div(F, kRankTile), (unsigned)std::min<int64_t>(ceil_div(F, kRankChunk), 65535));
    int64_t nparts = 0;
    switch (K) {
    case 2:
        k_hv_rank_count<2><<<gRank, kRankTile, 0, st>>>(pts, F, r, ws);
        k_hv_rank_order<2><<<gF, kThreads, 0, st>>>(pts, F, r, ws);
        k_hv2<<<gF, kThreads, 0, st>>>(pts, F, r, ws);
        nparts = gF;
        break;
    case 3:
        k_hv_rank_count<3><<<gRank, kRankTile, 0, st>>>(pts, F, r, ws);
        k_hv_rank_order<3><<<gF, kThreads, 0, st>>>(pts, F, r, ws);
        nparts = ceil_div(F, kSlab3Threads);
        k_hv3<<<(unsigned)nparts, kSlab3Threads, 0, st>>>(pts, F, r, ws);
        break;
    default:
        k_hv_rank_count<4><<<gRank, kRankTile, 0, st>>>(pts, F, r, ws);
        k_hv_rank_order<4><<<gF, kThreads, 0, st>>>(pts, F, r, ws);
        k_hv_permute4<<<gF, kThreads, 0, st>>>(pts, F, r, ws);
        if (F <= kHv4CompactMax) {
            // both launched; the flag k_hv_permute4 leaves decides which one does the slabs
            const size_t smem_n = (size_t)20 * F, smem_w = (size_t)32 * F;
            MOQ_CUDA_TRY(cudaFuncSetAttribute(k_hv4_narrow, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_n));
            MOQ_CUDA_TRY(cudaFuncSetAttribute(k_hv4_compact, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_w));
            k_hv4_narrow<<<(unsigned)F, kThreads, smem_n, st>>>(pts, F, r, ws);
            k_hv4_compact<<<(unsigned)F, kThreads, smem_w, st>>>(pts, F, r, ws);
        } else {
            k_hv4_stream<<<(unsigned)F, kThreads, 0, st>>>(pts, F, r, ws);
        }
        nparts = F;
        break;
    }
    k_hv_final<<<1, kThreads, 0, st>>>(pts, F, K, r, nparts, ws);
    MOQ_LAUNCH_CHECK("moq_hypervolume launch");
    return MOQ_OK;
}

int hv_points_impl(const int64_t* pts, int64_t F, int32_t K, const int64_t* ref, void* workspace, moq_hv* out, void* stream,
                   bool pinned_readback)
{
    if (!ref || !out || !workspace) return fail(MOQ_ERR_ARG, "moq_hypervolume_points: NULL argument");
    if (F < 0 || F >= ((int64_t)1 << 31)) return fail(MOQ_ERR_ARG, "moq_hypervolume_points: F out of range");
    if (K < 2) return fail(MOQ_ERR_ARG, "moq_hypervolume_points: K=%d < 2", K);
    if (K > 4) return fail(MOQ_ERR_UNSUPPORTED, "moq_hypervolume_points: K=%d > 4", K);
    if (F > 0 && !pts) return fail(MOQ_ERR_ARG, "moq_hypervolume_points: NULL points");
    if (((uintptr_t)workspace) % 256) return fail(MOQ_ERR_ARG, "moq_hypervolume_points: workspace not 256-byte aligned");
    out->lo = out->hi = 0;
    out->approx = 0.0;
    if (F == 0) return MOQ_OK;
    cudaStream_t st = as_stream(stream);
    HvWs ws;
    const int rc = hv_launch(pts, F, K, ref, workspace, st, ws);
    if (rc != MOQ_OK) return rc;
    struct Result {
        i128 v;
        int32_t flags;
    } local;
    PinnedLease lease(sizeof(Result), pinned_readback);
    lease.arm(st);
    Result& host = lease.p ? *static_cast<Result*>(lease.p) : local;
    MOQ_CUDA_TRY(cudaMemcpyAsync(&host.v, ws.result, sizeof(i128), cudaMemcpyDeviceToHost, st));
    MOQ_CUDA_TRY(cudaMemcpyAsync(&host.flags, ws.flags, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MOQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (host.flags & 1) return fail(MOQ_ERR_OVERFLOW, "moq_hypervolume: side-length product reaches 2^125");
    out->lo = (int64_t)(uint64_t)host.v;
    out->hi = (int64_t)(host.v >> 64);
    out->approx = (double)host.v;
    return MOQ_OK;
}
}  // namespace moq

extern "C" {

int moq_hypervolume_points(const int64_t* pts, int64_t F, int32_t K, const int64_t* ref, void* workspace, moq_hv* out,
                           void* stream)
{
    return moq::hv_points_impl(pts, F, K, ref, workspace, out, stream, true);
}

int moq_hypervolume(const moq_archive* a, const int64_t* ref, moq_hv* out, void* stream)
{
    using namespace moq;
    if (!a || !ref || !out) return fail(MOQ_ERR_ARG, "moq_hypervolume: NULL argument");
    if (a->K > 4) return fail(MOQ_ERR_UNSUPPORTED, "moq_hypervolume: K=%d > 4", a->K);
    int64_t F = 0;
    int rc = moq_archive_size(a, &F, stream);
    if (rc != MOQ_OK) return rc;
    return moq_hypervolume_points(a->cuts[a->cur], F, a->K, ref, a->hv_ws, out, stream);
}

int moq_hypervolume_many(const moq_archive* const* archives, const int64_t* refs, int32_t count, moq_hv* out, void* stream)
{
    using namespace moq;
    if (count < 0) return fail(MOQ_ERR_ARG, "moq_hypervolume_many: count=%d < 0", count);
    if (count == 0) return MOQ_OK;
    if (!archives || !refs || !out) return fail(MOQ_ERR_ARG, "moq_hypervolume_many: NULL argument");
    for (int32_t i = 0; i < count; ++i) {
        if (!archives[i]) return fail(MOQ_ERR_ARG, "moq_hypervolume_many: archive %d is NULL", i);
        if (archives[i]->K != archives[0]->K) return fail(MOQ_ERR_ARG, "moq_hypervolume_many: archives of different K");
    }
    const int K = archives[0]->K;
    if (K > 4) return fail(MOQ_ERR_UNSUPPORTED, "moq_hypervolume_many: K=%d > 4", K);
    for (int32_t i = 0; i < count; ++i) {
        out[i].lo = out[i].hi = 0;
        out[i].approx = 0.0;
    }
    cudaStream_t st = as_stream(stream);
    // per archive: front size and status, then the result and its overflow flag, in one
    // leased pinned buffer; chunks of kPer archives per lease
    struct Slot {
        int64_t size;
        int32_t status;
        int32_t flags;
        i128 v;
    };
    constexpr int32_t kPer = 4096 / sizeof(Slot);
    Slot fallback[kPer];
    PinnedLease lease(sizeof(Slot) * kPer);
    lease.arm(st);
    Slot* slot = lease.p ? static_cast<Slot*>(lease.p) : fallback;
    for (int32_t c0 = 0; c0 < count; c0 += kPer) {
        const int32_t c1 = std::min(count, c0 + kPer);
        for (int32_t i = c0; i < c1; ++i) {
            MOQ_CUDA_TRY(cudaMemcpyAsync(&slot[i - c0].size, archives[i]->d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            MOQ_CUDA_TRY(cudaMemcpyAsync(&slot[i - c0].status, archives[i]->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        }
        MOQ_CUDA_TRY(cudaStreamSynchronize(st));
        int32_t full = -1;
        for (int32_t i = c0; i < c1; ++i)
            if (slot[i - c0].status & kStatusCapacity) {
                // as moq_archive_size: report the capacity error once and clear the latch
                MOQ_CUDA_TRY(cudaMemsetAsync(archives[i]->d_status, 0, sizeof(int32_t), st));
                if (full < 0) full = i;
            }
        if (full >= 0) {
            MOQ_CUDA_TRY(cudaStreamSynchronize(st));
            return fail(MOQ_ERR_CAPACITY, "moq_hypervolume_many: archive %d: capacity %lld exceeded; the archive was left unchanged",
                        full, (long long)archives[full]->cap);
        }
        int32_t queued = 0;
        for (int32_t i = c0; i < c1; ++i) {
            const moq_archive* a = archives[i];
            const int64_t F = slot[i - c0].size;
            slot[i - c0].flags = 0;
            if (F <= 0) continue;
            if (F >= ((int64_t)1 << 31)) return fail(MOQ_ERR_ARG, "moq_hypervolume_many: archive %d: front too large", i);
            HvWs ws;
            const int rc = hv_launch(a->cuts[a->cur], F, K, refs + (int64_t)i * K, a->hv_ws, st, ws);
            if (rc != MOQ_OK) return rc;
            MOQ_CUDA_TRY(cudaMemcpyAsync(&slot[i - c0].v, ws.result, sizeof(i128), cudaMemcpyDeviceToHost, st));
            MOQ_CUDA_TRY(cudaMemcpyAsync(&slot[i - c0].flags, ws.flags, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            ++queued;
        }
        if (queued) MOQ_CUDA_TRY(cudaStreamSynchronize(st));
        for (int32_t i = c0; i < c1; ++i) {
            if (slot[i - c0].size <= 0) continue;
            if (slot[i - c0].flags & 1)
                return fail(MOQ_ERR_OVERFLOW, "moq_hypervolume_many: archive %d: side-length product reaches 2^125", i);
            const i128 v = slot[i - c0].v;
            out[i].lo = (int64_t)(uint64_t)v;
            out[i].hi = (int64_t)(v >> 64);
            out[i].approx = (double)v;
        }
    }
    return MOQ_OK;
}

}  // extern "C"

// ---- hypervolume without any device allocation --------------------------------------
// Some callers cannot allocate device memory at the point where they need a
// hypervolume: code running under an external allocator that owns the whole device
// budget, latency-critical loops where cudaMalloc/cudaFree would synchronise the
// device, or hosts that forbid allocation after start-up. For them the scratch lives
// in a fixed array of this library's own device memory, reserved when the library is
// loaded (every GPU that loads it holds the array until the process exits).
namespace moq {
namespace {

constexpr int64_t kNoAllocMaxPoints = 16384;
constexpr size_t round256(size_t v) { return (v + 255) / 256 * 256; }
// the workspace layout of moq_hypervolume_points for kNoAllocMaxPoints points, K = 4
constexpr size_t kNoAllocBytes = 2 * round256(sizeof(int32_t) * 4 * kNoAllocMaxPoints) + round256(16 * kNoAllocMaxPoints) +
                                 round256(40 * kNoAllocMaxPoints) + 256;

static __device__ __align__(256) unsigned char g_hv_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array on the current device. The symbol's host-side name is
// only a stand-in, so the address is looked up, with the device current, on every call
// (cheap next to the call's own synchronisation): a cudaDeviceReset, or any teardown of the
// device's primary context, reloads the module and can move the array.
int noalloc_scratch(void** out)
{
    void* p = nullptr;
    MOQ_CUDA_TRY(cudaGetSymbolAddress(&p, g_hv_noalloc_scratch));
    *out = p;
    return MOQ_OK;
}

}  // namespace
}  // namespace moq

extern "C" {

int64_t moq_hypervolume_noalloc_max_points(void) { return moq::kNoAllocMaxPoints; }

int moq_hypervolume_points_noalloc(const int64_t* pts, int64_t F, int32_t K, const int64_t* ref, moq_hv* out,
                                   void* stream)
{
    using namespace moq;
    if (F > kNoAllocMaxPoints)
        return fail(MOQ_ERR_CAPACITY, "moq_hypervolume_points_noalloc: %lld points exceed the fixed scratch limit of %lld",
                    (long long)F, (long long)kNoAllocMaxPoints);
    if (K > 4) return fail(MOQ_ERR_UNSUPPORTED, "moq_hypervolume_points_noalloc: K=%d > 4", K);
    void* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != MOQ_OK) return rc;
    // the path of the allocating entry point, handed the fixed array as its workspace (it
    // clears the counter and the rank array that must start at zero and overwrites the rest
    // before reading it), with the 20 result bytes read back into this call's stack frame
    // instead of a pinned host buffer
    return hv_points_impl(pts, F, K, ref, scratch, out, stream, false);
}

}  // extern "C"
