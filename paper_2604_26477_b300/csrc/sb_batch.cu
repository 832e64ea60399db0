// Batched sampling of many instances of uneven size in one persistent launch (the same
// NI-SB dynamics as sb_sparse.cu: SB equations and Eq. NI-SB, "Simulated Bifurcation
// with Gaussian noise"; the paper runs all weight vectors and replicas "in parallel in a
// single run").
//
// Work items are (instance, block of Rb replicas); a block of `bd` threads covers
// bd * SPT spin slots (slot s = spin s / Rb of replica s % Rb, spin-major as in the
// single-instance kernel), and Rb = min(32, bd * SPT / n) per instance. Items are sorted
// longest first and handed out through a device queue (one atomic per item), so large
// and small instances share the GPU without a tail. Each item runs its whole trajectory
// on-chip; the tile shape (bd, SPT) comes from the project's autotuner.
//
// Noise and start state use Philox with replica counter = the instance's replica offset in
// the batch + r, so a batch reproduces, bit for bit, single-instance calls that pass the
// same offsets.
#include <algorithm>
#include <numeric>
#include <stdlib.h>
#include <vector>

#include "sb_common.cuh"

namespace moq {
namespace {

constexpr int kSlots = 2048;    // most spin slots per block (bd * SPT)
constexpr int kMaxRb = 32;      // most replicas per item
constexpr int kWbWords = 128;   // packed-sign staging (Rb * W <= kSlots/64 + kMaxRb)

struct BatchInst {
    int32_t n, K, W, R;
    int64_t nnz;
    const int32_t* rowptr;
    const int32_t* col;
    const int32_t* wn;
    const int64_t* rowsum;
    int64_t rep_off;   // first replica of this instance in lambda_all / the replica counter
    int64_t bits_off;  // first word of this instance in bits_all
};

struct BatchItem {
    int32_t inst, r0, Rb, pad;
};

struct BatchArgs {
    const BatchInst* insts;
    const BatchItem* items;
    int32_t nitems;
    int32_t* queue;
    const float* lambda;
    uint64_t* bits;
    int32_t T;
    float dt, a0, init_amp, kappa, a0inv;
    const float* schedule;
    uint32_t key0, key1, round32;
};

size_t batch_smem_bytes() { return sizeof(float) * 2 * kSlots + sizeof(unsigned) * 2 * kMaxRb + sizeof(unsigned long long) * kWbWords; }

template <int VARIANT, int DMAX, bool NOISE, bool LINEAR, int SPT>
__global__ void __launch_bounds__(SPT >= 2 ? 512 : 1024) k_sb_batch(const BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* phiA = reinterpret_cast<float*>(smem_raw);
    float* phiB = phiA + kSlots;
    unsigned* red = reinterpret_cast<unsigned*>(phiB + kSlots);  // 2 * kMaxRb
    unsigned long long* wb = reinterpret_cast<unsigned long long*>(red + 2 * kMaxRb);
    __shared__ int s_item;
    const int tid = threadIdx.x, bd = blockDim.x;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= a.nitems) return;  // uniform: every thread read the same item
        const BatchItem item = a.items[it];
        const BatchInst in = a.insts[item.inst];
        const int n = in.n, Rb = item.Rb, ns = n * Rb, K = in.K;

        int sl[SPT], ii[SPT], lrr[SPT];
        uint32_t rc[SPT];
        bool act[SPT], ract[SPT];
        float x[SPT], y[SPT], jc[SPT][DMAX], sabs[SPT], srow[SPT];
        int nb[SPT][DMAX];
#pragma unroll
        for (int q = 0; q < SPT; ++q) {
            const int s = tid + q * bd;
            sl[q] = s;
            act[q] = s < ns;
            const int i = act[q] ? s / Rb : 0;
            const int lr = act[q] ? s - i * Rb : 0;
            ii[q] = i;
            lrr[q] = lr;
            const int r = item.r0 + lr;
            ract[q] = act[q] && r < in.R;
            rc[q] = (uint32_t)(in.rep_off + r);
            const int64_t rs = in.rep_off + (ract[q] ? r : 0);
            float lam[kMaxK];
#pragma unroll
            for (int k = 0; k < kMaxK; ++k) lam[k] = (k < K) ? a.lambda[rs * K + k] : 0.0f;
            const int p0 = act[q] ? in.rowptr[i] : 0;
            const int deg = act[q] ? in.rowptr[i + 1] - p0 : 0;
            sabs[q] = 0.0f;
#pragma unroll
            for (int d = 0; d < DMAX; ++d) {
                float v = 0.0f;
                int c = i;
                if (d < deg) {
                    const int p = p0 + d;
                    c = in.col[p];
#pragma unroll
                    for (int k = 0; k < kMaxK; ++k)
                        if (k < K) v = fmaf(lam[k], (float)in.wn[(int64_t)k * in.nnz + p], v);
                }
                jc[q][d] = v;
                nb[q][d] = c * Rb + lr;
                sabs[q] += fabsf(v);
            }
            srow[q] = 0.0f;
            if (act[q])
#pragma unroll
                for (int k = 0; k < kMaxK; ++k)
                    if (k < K) srow[q] = fmaf(lam[k], (float)in.rowsum[(int64_t)i * K + k], srow[q]);
        }
        // c0 = 1 / max_i |sum_j J(c)_ij| per replica (fallbacks: sum |J(c)_ij|, then 1)
        if (tid < 2 * kMaxRb) red[tid] = 0u;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < SPT; ++q)
            if (act[q]) {
                atomicMax(&red[lrr[q]], __float_as_uint(fabsf(srow[q])));
                atomicMax(&red[kMaxRb + lrr[q]], __float_as_uint(sabs[q]));
            }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < SPT; ++q) {
            const float mx = __uint_as_float(red[lrr[q]]), mxa = __uint_as_float(red[kMaxRb + lrr[q]]);
            const float c0 = mx > 0.0f ? 1.0f / mx : (mxa > 0.0f ? 1.0f / mxa : 1.0f);
#pragma unroll
            for (int d = 0; d < DMAX; ++d) jc[q][d] *= -c0;
            const uint4 o = Philox4x32::block(make_uint4(0xFFFFFFFFu, (uint32_t)ii[q], rc[q], a.round32), a.key0, a.key1);
            x[q] = __fmul_rn(a.init_amp, signed_unit(o.x)) + 0.0f;
            y[q] = __fmul_rn(a.init_amp, signed_unit(o.y));
            if (act[q]) phiA[sl[q]] = phi_of<VARIANT>(x[q]);
        }
        __syncthreads();

        const float dt = a.dt, kappa = a.kappa, dta0 = a.dt * a.a0, a0 = a.a0, a0inv = a.a0inv;
        const int T = a.T;
        // one Philox4x32-10 block per slot and eight steps: word q gives the Gaussians of
        // steps 2q and 2q+1 (the single-instance sampler's layout)
        uint4 blk[SPT];
        float e[SPT][2];
        auto block8 = [&](int m) {
#pragma unroll
            for (int q = 0; q < SPT; ++q)
                blk[q] = NOISE ? Philox4x32::block(make_uint4((uint32_t)(m >> 3), (uint32_t)ii[q], rc[q], a.round32), a.key0, a.key1)
                               : make_uint4(0u, 0u, 0u, 0u);
        };
        auto pairs = [&](int w) {
#pragma unroll
            for (int q = 0; q < SPT; ++q) {
                const float2 p = NOISE ? box_muller16(word_of(blk[q], w)) : make_float2(0.0f, 0.0f);
                e[q][0] = p.x;
                e[q][1] = p.y;
            }
        };
        auto step = [&](const float* rd, float* wr, int m, float mf, int j) {
            const float cm = LINEAR ? fmaf(a0inv, mf, -a0) : (__ldg(a.schedule + m) - a0);
#pragma unroll
            for (int q = 0; q < SPT; ++q) {
                if (act[q]) {
                    float f = 0.0f;
#pragma unroll
                    for (int d = 0; d < DMAX; ++d) f = fmaf(jc[q][d], rd[nb[q][d]], f);
                    sb_update<NOISE>(f, cm, e[q][j], dt, kappa, dta0, x[q], y[q]);
                    wr[sl[q]] = phi_of<VARIANT>(x[q]);
                }
            }
            __syncthreads();
        };
        int m = 0;
        float mf = 0.0f;
        for (; m + 8 <= T; m += 8) {
            block8(m);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                pairs(w);
                step(phiA, phiB, m + 2 * w, mf, 0);
                step(phiB, phiA, m + 2 * w + 1, mf + 1.0f, 1);
                mf += 2.0f;
            }
        }
        if (m < T) {  // the last T mod 8 steps (uniform over the block)
            block8(m);
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                if (m + 2 * w < T) {
                    pairs(w);
                    step(phiA, phiB, m + 2 * w, mf, 0);
                    if (m + 2 * w + 1 < T) step(phiB, phiA, m + 2 * w + 1, mf + 1.0f, 1);
                    mf += 2.0f;
                }
            }
        }

        // readout s_i = sgn(x_i), bit set for s_i = -1
        const int W = in.W;
        for (int t = tid; t < Rb * W; t += bd) wb[t] = 0ull;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < SPT; ++q)
            if (ract[q] && x[q] < 0.0f) atomicOr(&wb[lrr[q] * W + (ii[q] >> 6)], 1ull << (ii[q] & 63));
        __syncthreads();
        for (int t = tid; t < Rb * W; t += bd) {
            const int r = item.r0 + t / W;
            if (r < in.R) a.bits[in.bits_off + (int64_t)r * W + (t % W)] = wb[t];
        }
        __syncthreads();  // shared memory and s_item are reused by the next item
    }
}

// Cut values of every sample of every instance: blockIdx.y = instance, one thread per
// sample, the instance's edges staged through shared memory (as in cuts.cu).
__global__ void __launch_bounds__(256) k_cuts_batch(const BatchInst* __restrict__ insts, const int32_t* const* __restrict__ ei,
                                                    const int32_t* const* __restrict__ ej, const int32_t* const* __restrict__ w,
                                                    const int64_t* __restrict__ E, const uint64_t* __restrict__ bits,
                                                    int64_t* __restrict__ cuts, int32_t Kall)
{
    constexpr int kChunk = 256;
    __shared__ int32_t s_i[kChunk], s_j[kChunk], s_w[kMaxK][kChunk];
    const int b = blockIdx.y;
    const BatchInst in = insts[b];
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (blockIdx.x * (int64_t)blockDim.x >= in.R) return;  // uniform
    const bool act = m < in.R;
    const uint64_t* sb = bits + in.bits_off + m * in.W;
    int64_t acc[kMaxK];
    for (int k = 0; k < kMaxK; ++k) acc[k] = 0;
    const int64_t Eb = E[b];
    for (int64_t e0 = 0; e0 < Eb; e0 += kChunk) {
        const int cnt = (int)min((int64_t)kChunk, Eb - e0);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            s_i[t] = ei[b][e0 + t];
            s_j[t] = ej[b][e0 + t];
            for (int k = 0; k < Kall; ++k) s_w[k][t] = w[b][k * Eb + e0 + t];
        }
        __syncthreads();
        if (act) {
            for (int t = 0; t < cnt; ++t) {
                const int p = s_i[t], q = s_j[t];
                const bool cut = ((sb[p >> 6] >> (p & 63)) ^ (sb[q >> 6] >> (q & 63))) & 1ull;
                if (cut)
                    for (int k = 0; k < Kall; ++k) acc[k] += s_w[k][t];
            }
        }
    }
    if (act)
        for (int k = 0; k < Kall; ++k) cuts[(in.rep_off + m) * Kall + k] = acc[k];
}

}  // namespace
}  // namespace moq

struct moq_batch {
    int32_t count = 0, K = 0, max_degree = 0, max_n = 0;
    int64_t total_R = 0, total_words = 0;
    int32_t bd = 1024, spt = 1;
    int32_t nitems = 0;
    std::vector<moq::BatchInst> h_insts;
    std::vector<int32_t> h_created_R;            // replicas per instance at creation (the layout)
    std::vector<int64_t> h_E;
    std::vector<const moq_instance*> h_handles;  // for the per-instance mode (bd == 0)
    // per-instance mode: launches fan out over these streams (one instance's tail overlaps
    // the next one's start) and join back into the caller's stream
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> lane_done;
    cudaEvent_t fork = nullptr;
    moq::BatchInst* d_insts = nullptr;
    moq::BatchItem* d_items = nullptr;
    int64_t items_cap = 0;
    int32_t* d_queue = nullptr;
    const int32_t** d_ei = nullptr;
    const int32_t** d_ej = nullptr;
    const int32_t** d_w = nullptr;
    int64_t* d_E = nullptr;
    void* slab = nullptr;  // the one device allocation the arrays above live in
};

namespace moq {
namespace {

void free_batch(moq_batch* b)
{
    if (!b) return;
    slab_free(b->slab);
    for (cudaStream_t s : b->lanes) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->lane_done) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

// Items for tile shape (bd, spt): Rb_b = min(32, R_b, bd*spt / n_b), longest first.
int build_items(moq_batch* b)
{
    std::vector<BatchItem> items;
    for (int i = 0; i < b->count; ++i) {
        const BatchInst& in = b->h_insts[i];
        const int rb = std::max(1, std::min({kMaxRb, in.R, b->bd * b->spt / in.n}));
        for (int r0 = 0; r0 < in.R; r0 += rb) items.push_back({i, r0, rb, 0});
    }
    std::stable_sort(items.begin(), items.end(), [&](const BatchItem& p, const BatchItem& q) {
        return (int64_t)b->h_insts[p.inst].n * p.Rb > (int64_t)b->h_insts[q.inst].n * q.Rb;
    });
    if ((int64_t)items.size() > b->items_cap) return fail(MOQ_ERR_CAPACITY, "batch: %zu work items exceed %lld", items.size(), (long long)b->items_cap);
    MOQ_CUDA_TRY(cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice));
    b->nitems = (int32_t)items.size();
    return MOQ_OK;
}

template <int VARIANT, int DMAX, bool NOISE, bool LINEAR, int SPT>
cudaError_t launch_batch(const BatchArgs& a, int bd, cudaStream_t st)
{
    auto k = k_sb_batch<VARIANT, DMAX, NOISE, LINEAR, SPT>;
    const size_t smem = batch_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, bd, smem);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(a.nitems, std::max(1, per_sm) * sms));
    k<<<grid, bd, smem, st>>>(a);
    return cudaGetLastError();
}

template <int VARIANT, int DMAX, bool NOISE, bool LINEAR>
cudaError_t launch_spt(const BatchArgs& a, int bd, int spt, cudaStream_t st)
{
    switch (spt) {
    case 4: return launch_batch<VARIANT, DMAX, NOISE, LINEAR, 4>(a, bd, st);
    case 2: return launch_batch<VARIANT, DMAX, NOISE, LINEAR, 2>(a, bd, st);
    default: return launch_batch<VARIANT, DMAX, NOISE, LINEAR, 1>(a, bd, st);
    }
}

template <int VARIANT, int DMAX>
cudaError_t launch_flags_b(const BatchArgs& a, bool noise, bool linear, int bd, int spt, cudaStream_t st)
{
    if (noise) return linear ? launch_spt<VARIANT, DMAX, true, true>(a, bd, spt, st) : launch_spt<VARIANT, DMAX, true, false>(a, bd, spt, st);
    return linear ? launch_spt<VARIANT, DMAX, false, true>(a, bd, spt, st) : launch_spt<VARIANT, DMAX, false, false>(a, bd, spt, st);
}

template <int VARIANT>
cudaError_t launch_variant_b(const BatchArgs& a, int dmax, bool noise, bool linear, int bd, int spt, cudaStream_t st)
{
    switch (dmax) {
    case 3: return launch_flags_b<VARIANT, 3>(a, noise, linear, bd, spt, st);
    case 4: return launch_flags_b<VARIANT, 4>(a, noise, linear, bd, spt, st);
    default: return launch_flags_b<VARIANT, 8>(a, noise, linear, bd, spt, st);
    }
}

}  // namespace
}  // namespace moq

extern "C" {

int moq_batch_create(const moq_instance* const* insts, int32_t count, const int32_t* replicas, moq_batch** out)
{
    using namespace moq;
    if (!out) return fail(MOQ_ERR_ARG, "moq_batch_create: out is NULL");
    *out = nullptr;
    if (count < 1 || !insts || !replicas) return fail(MOQ_ERR_ARG, "moq_batch_create: need count >= 1 instances and replica counts");
    moq_batch* b = new moq_batch();
    b->count = count;
    b->K = insts[0]->K;
    int64_t rep = 0, words = 0, items_cap = 0;
    for (int i = 0; i < count; ++i) {
        const moq_instance* h = insts[i];
        if (!h || h->K != b->K || replicas[i] < 1) {
            free_batch(b);
            return fail(MOQ_ERR_ARG, "moq_batch_create: instance %d is NULL, has another K, or no replicas", i);
        }
        if (h->n > 1024) {
            free_batch(b);
            return fail(MOQ_ERR_UNSUPPORTED, "moq_batch_create: n=%d > 1024", h->n);
        }
        if (h->max_degree > 8) {
            free_batch(b);
            return fail(MOQ_ERR_UNSUPPORTED, "moq_batch_create: max degree %d > 8", h->max_degree);
        }
        BatchInst in{};
        in.n = h->n;
        in.K = h->K;
        in.W = h->words;
        in.R = replicas[i];
        in.nnz = h->nnz;
        in.rowptr = h->rowptr;
        in.col = h->col;
        in.wn = h->wn;
        in.rowsum = h->rowsum;
        in.rep_off = rep;
        in.bits_off = words;
        rep += in.R;
        words += (int64_t)in.R * in.W;
        items_cap += in.R;  // at most one item per replica
        b->h_insts.push_back(in);
        b->h_created_R.push_back(in.R);
        b->h_E.push_back(h->E);
        b->h_handles.push_back(h);
        b->max_degree = std::max(b->max_degree, h->max_degree);
        b->max_n = std::max(b->max_n, h->n);
    }
    if (rep >= ((int64_t)1 << 32)) {
        free_batch(b);
        return fail(MOQ_ERR_ARG, "moq_batch_create: more than 2^32 replicas");
    }
    b->total_R = rep;
    b->total_words = words;
    b->items_cap = items_cap;
    std::vector<const int32_t*> ei(count), ej(count), w(count);
    for (int i = 0; i < count; ++i) {
        ei[i] = insts[i]->ei;
        ej[i] = insts[i]->ej;
        w[i] = insts[i]->w;
    }
    // one slab from the library's memory pool for the handle's device arrays, filled on the
    // legacy stream and synchronised once
    const std::pair<void**, size_t> parts[] = {
        {(void**)&b->d_insts, sizeof(BatchInst) * count}, {(void**)&b->d_items, sizeof(BatchItem) * items_cap},
        {(void**)&b->d_queue, sizeof(int32_t)}, {(void**)&b->d_ei, sizeof(void*) * count},
        {(void**)&b->d_ej, sizeof(void*) * count}, {(void**)&b->d_w, sizeof(void*) * count},
        {(void**)&b->d_E, sizeof(int64_t) * count}};
    size_t total = 0;
    for (const auto& pr : parts) total += slab_align(pr.second);
    const cudaStream_t st0 = cudaStreamLegacy;
    cudaError_t e = slab_alloc(&b->slab, total, st0);
    if (e == cudaSuccess) {
        size_t off = 0;
        for (const auto& pr : parts) {
            *pr.first = static_cast<char*>(b->slab) + off;
            off += slab_align(pr.second);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_insts, b->h_insts.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice, st0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_ei, ei.data(), sizeof(void*) * count, cudaMemcpyHostToDevice, st0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_ej, ej.data(), sizeof(void*) * count, cudaMemcpyHostToDevice, st0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_w, w.data(), sizeof(void*) * count, cudaMemcpyHostToDevice, st0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_E, b->h_E.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice, st0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st0);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "moq_batch_create");
    }
    b->bd = b->max_n > 512 ? 1024 : (b->max_n > 256 ? 512 : 256);
    b->spt = 1;
    int rc = build_items(b);
    if (rc != MOQ_OK) {
        free_batch(b);
        return rc;
    }
    *out = b;
    return MOQ_OK;
}

void moq_batch_destroy(moq_batch* b) { moq::free_batch(b); }

int moq_batch_layout(const moq_batch* b, int64_t* replica_offsets, int64_t* word_offsets)
{
    using namespace moq;
    if (!b) return fail(MOQ_ERR_ARG, "moq_batch_layout: NULL batch");
    for (int i = 0; i < b->count; ++i) {
        if (replica_offsets) replica_offsets[i] = b->h_insts[i].rep_off;
        if (word_offsets) word_offsets[i] = b->h_insts[i].bits_off;
    }
    if (replica_offsets) replica_offsets[b->count] = b->total_R;
    if (word_offsets) word_offsets[b->count] = b->total_words;
    return MOQ_OK;
}

int moq_batch_set_tiles(moq_batch* b, int32_t block_threads, int32_t slots_per_thread, int32_t* items_out)
{
    using namespace moq;
    if (!b) return fail(MOQ_ERR_ARG, "moq_batch_set_tiles: NULL batch");
    if (block_threads == 0 && slots_per_thread == 0) {  // per-instance launches of the single-instance sampler
        if (b->lanes.empty()) {
            int nl = 4;
            if (const char* env = getenv("MOQ_BATCH_STREAMS")) nl = std::max(1, std::min(16, atoi(env)));
            MOQ_CUDA_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
            for (int l = 0; l < nl; ++l) {
                cudaStream_t s = nullptr;
                cudaEvent_t e = nullptr;
                MOQ_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
                b->lanes.push_back(s);
                MOQ_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                b->lane_done.push_back(e);
            }
        }
        b->bd = 0;
        b->spt = 0;
        if (items_out) *items_out = b->count;
        return MOQ_OK;
    }
    if ((block_threads != 256 && block_threads != 512 && block_threads != 1024) ||
        (slots_per_thread != 1 && slots_per_thread != 2 && slots_per_thread != 4))
        return fail(MOQ_ERR_ARG, "moq_batch_set_tiles: block_threads in {256, 512, 1024}, slots_per_thread in {1, 2, 4} (or 0, 0)");
    if (slots_per_thread >= 2 && block_threads > 512)
        return fail(MOQ_ERR_ARG, "moq_batch_set_tiles: two or four slots per thread need block_threads <= 512");
    if (block_threads * slots_per_thread < b->max_n)
        return fail(MOQ_ERR_ARG, "moq_batch_set_tiles: %d x %d slots cannot hold n=%d", block_threads, slots_per_thread, b->max_n);
    b->bd = block_threads;
    b->spt = slots_per_thread;
    int rc = build_items(b);
    if (items_out) *items_out = b->nitems;
    return rc;
}

int moq_batch_set_replicas(moq_batch* b, const int32_t* replicas)
{
    using namespace moq;
    if (!b || !replicas) return fail(MOQ_ERR_ARG, "moq_batch_set_replicas: NULL argument");
    for (int i = 0; i < b->count; ++i)
        if (replicas[i] < 0 || replicas[i] > b->h_created_R[i])
            return fail(MOQ_ERR_ARG, "moq_batch_set_replicas: instance %d: %d replicas outside [0, %d]", i, replicas[i],
                        b->h_created_R[i]);
    for (int i = 0; i < b->count; ++i) b->h_insts[i].R = replicas[i];
    MOQ_CUDA_TRY(cudaMemcpy(b->d_insts, b->h_insts.data(), sizeof(BatchInst) * b->count, cudaMemcpyHostToDevice));
    if (b->bd == 0) return MOQ_OK;  // per-instance launches read the counts on the host
    return build_items(b);
}

int moq_sample_batch(moq_batch* b, const float* lambda_all, const moq_sample_params* p, uint64_t seed, uint64_t round,
                     uint64_t* bits_all, void* stream)
{
    using namespace moq;
    if (!b || !p || !lambda_all || !bits_all) return fail(MOQ_ERR_ARG, "moq_sample_batch: NULL argument");
    if (p->steps < 0 || (p->variant != MOQ_DSB && p->variant != MOQ_BSB)) return fail(MOQ_ERR_ARG, "moq_sample_batch: bad steps or variant");
    if (p->x_init || p->y_init || p->x_out || p->y_out) return fail(MOQ_ERR_UNSUPPORTED, "moq_sample_batch: state arrays are single-instance only");
    cudaStream_t st = as_stream(stream);
    if (b->bd == 0) {
        // one launch of the single-instance sampler per instance, largest first; replica
        // counters start at the instance's offset, as in the persistent kernel
        std::vector<int> order(b->count);
        for (int i = 0; i < b->count; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->h_insts[x].n > b->h_insts[y].n; });
        const int nl = (int)b->lanes.size();
        MOQ_CUDA_TRY(cudaEventRecord(b->fork, st));
        for (int l = 0; l < nl; ++l) MOQ_CUDA_TRY(cudaStreamWaitEvent(b->lanes[l], b->fork, 0));
        int rc = MOQ_OK;
        for (int q = 0; q < b->count && rc == MOQ_OK; ++q) {
            const int i = order[q];
            const BatchInst& in = b->h_insts[i];
            moq_sample_params pi = *p;
            pi.replica_offset = (uint32_t)in.rep_off;
            rc = moq_sample(b->h_handles[i], lambda_all + in.rep_off * b->K, in.R, &pi, seed, round, bits_all + in.bits_off,
                            nl ? (void*)b->lanes[q % nl] : stream);
        }
        // the caller's stream waits for every lane, also after a failed launch
        for (int l = 0; l < nl; ++l) {
            MOQ_CUDA_TRY(cudaEventRecord(b->lane_done[l], b->lanes[l]));
            MOQ_CUDA_TRY(cudaStreamWaitEvent(st, b->lane_done[l], 0));
        }
        return rc;
    }
    if (p->precision != MOQ_PREC_FP32)
        return fail(MOQ_ERR_UNSUPPORTED, "moq_sample_batch: the persistent kernel runs FP32 (per-instance mode runs FP16)");
    MOQ_CUDA_TRY(cudaMemsetAsync(b->d_queue, 0, sizeof(int32_t), st));
    BatchArgs a{};
    a.insts = b->d_insts;
    a.items = b->d_items;
    a.nitems = b->nitems;
    a.queue = b->d_queue;
    a.lambda = lambda_all;
    a.bits = bits_all;
    a.T = p->steps;
    a.dt = p->dt;
    a.a0 = p->a0;
    a.init_amp = p->init_amp;
    a.kappa = (p->noise_sqrt_dt ? sqrtf(p->dt) : p->dt) * p->alpha;
    a.a0inv = p->steps > 1 ? p->a0 / (float)(p->steps - 1) : 0.0f;
    a.schedule = p->schedule;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.round32 = (uint32_t)round;
    const int md = b->max_degree;
    const int dmax = md <= 3 ? 3 : (md <= 4 ? 4 : 8);
    const bool noise = p->alpha != 0.0f, linear = p->schedule == nullptr;
    cudaError_t e = p->variant == MOQ_DSB ? launch_variant_b<MOQ_DSB>(a, dmax, noise, linear, b->bd, b->spt, st)
                                          : launch_variant_b<MOQ_BSB>(a, dmax, noise, linear, b->bd, b->spt, st);
    if (e != cudaSuccess) return cuda_fail(e, "moq_sample_batch launch");
    return MOQ_OK;
}

int moq_evaluate_cuts_batch(const moq_batch* b, const uint64_t* bits_all, int64_t* cuts_all, void* stream)
{
    using namespace moq;
    if (!b || !bits_all || !cuts_all) return fail(MOQ_ERR_ARG, "moq_evaluate_cuts_batch: NULL argument");
    int maxR = 0;
    for (const BatchInst& in : b->h_insts) maxR = std::max(maxR, in.R);
    if (maxR == 0) return MOQ_OK;  // no instance has an active replica: nothing to evaluate
    const dim3 grid((unsigned)ceil_div(maxR, 256), (unsigned)b->count);
    k_cuts_batch<<<grid, 256, 0, as_stream(stream)>>>(b->d_insts, b->d_ei, b->d_ej, b->d_w, b->d_E, bits_all, cuts_all, b->K);
    MOQ_LAUNCH_CHECK("moq_evaluate_cuts_batch launch");
    return MOQ_OK;
}

}  // extern "C"
