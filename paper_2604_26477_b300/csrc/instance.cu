// a1: instance build ("Hamiltonian formulation of multi-objective MaxCut").
// The edge list and K integer weight sets are copied to the device and turned into a
// both-direction CSR (rows sorted by column) with per-entry weights, integer row sums
// sum_j J^(k)_ij (used for c0 of every weight vector), and the per-objective sums
// W_k, sum |J^(k)| and r_k = sum min(0, J^(k)).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>
#include <cmath>

#include "gather_layout.cuh"
#include "moq_common.cuh"

namespace moq {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__global__ void k_degree(const int32_t* __restrict__ ei, const int32_t* __restrict__ ej, int64_t E, int32_t n,
                         int32_t* deg, int32_t* status)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = ei[e], b = ej[e];
        if (a < 0 || b >= n || a >= b) {
            atomicOr(status, kStatusBadEdge);
            continue;
        }
        atomicAdd(&deg[a], 1);
        atomicAdd(&deg[b], 1);
    }
}

// rowptr[0] = 0, rowptr[i+1] = deg[0] + .. + deg[i]; one block of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_rowptr(const int32_t* __restrict__ deg, int32_t n, int32_t* rowptr)
{
    __shared__ int32_t warp_sums[32];
    __shared__ int32_t carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        carry = 0;
        rowptr[0] = 0;
    }
    __syncthreads();
    for (int32_t base = 0; base < n; base += 1024) {
        const int32_t i = base + threadIdx.x;
        int32_t v = i < n ? deg[i] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) warp_sums[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int32_t s = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t t = __shfl_up_sync(kFull, s, o);
                if (lane >= o) s += t;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const int32_t incl = v + (wid > 0 ? warp_sums[wid - 1] : 0) + carry;
        if (i < n) rowptr[i + 1] = incl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = incl;
        __syncthreads();
    }
}

__global__ void k_fill(const int32_t* __restrict__ ei, const int32_t* __restrict__ ej, int64_t E, int32_t n,
                       const int32_t* __restrict__ rowptr, int32_t* cursor, int32_t* col_tmp, int32_t* eid_tmp)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = ei[e], b = ej[e];
        if (a < 0 || b >= n || a >= b) continue;
        const int32_t pa = rowptr[a] + atomicAdd(&cursor[a], 1);
        col_tmp[pa] = b;
        eid_tmp[pa] = (int32_t)e;
        const int32_t pb = rowptr[b] + atomicAdd(&cursor[b], 1);
        col_tmp[pb] = a;
        eid_tmp[pb] = (int32_t)e;
    }
}

// One warp per row: each entry's rank is the number of row entries with a smaller column
// (deterministic, whatever order the atomics filled the row in); it lands at position rank of
// the row, or at remap[p0 + rank] when a gather order is given. Equal columns mean a repeated
// edge.
__global__ void k_sort_rows(int32_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col_tmp,
                            const int32_t* __restrict__ eid_tmp, const int32_t* __restrict__ remap, int32_t* col, int32_t* eid,
                            int32_t* status)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = warp; row < n; row += nwarps) {
        const int32_t p0 = rowptr[row], p1 = rowptr[row + 1];
        for (int32_t p = p0 + lane; p < p1; p += 32) {
            const int32_t c = col_tmp[p];
            int32_t rank = 0;
            bool dup = false;
            for (int32_t q = p0; q < p1; ++q) {
                const int32_t cq = col_tmp[q];
                rank += (cq < c);
                dup |= (cq == c) && (q != p);
            }
            const int32_t at = remap ? remap[p0 + rank] : rank;
            col[p0 + at] = c;
            eid[p0 + at] = eid_tmp[p];
            if (dup) atomicOr(status, kStatusDuplicateEdge);
        }
    }
}

__global__ void k_entry_weights(int32_t K, int64_t nnz, int64_t E, const int32_t* __restrict__ eid,
                                const int32_t* __restrict__ w, int32_t* wn)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = eid[p];
        for (int k = 0; k < K; ++k) wn[k * nnz + p] = w[k * E + e];
    }
}

__global__ void k_row_sums(int32_t n, int32_t K, int64_t nnz, const int32_t* __restrict__ rowptr,
                           const int32_t* __restrict__ wn, int64_t* rowsum, int32_t* maxdeg)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p0 = rowptr[i], p1 = rowptr[i + 1];
        for (int k = 0; k < K; ++k) {
            int64_t s = 0;
            for (int32_t p = p0; p < p1; ++p) s += wn[k * nnz + p];
            rowsum[i * K + k] = s;
        }
        atomicMax(maxdeg, p1 - p0);
    }
}

// sums[0..K): sum J, sums[K..2K): sum |J|, sums[2K..3K): sum min(0, J). Two's complement
// addition of the unsigned atomics gives the exact signed sums.
__global__ void k_weight_sums(int32_t K, int64_t E, const int32_t* __restrict__ w, unsigned long long* sums)
{
    int64_t s[kMaxK], a[kMaxK], m[kMaxK];
    for (int k = 0; k < K; ++k) s[k] = a[k] = m[k] = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        for (int k = 0; k < K; ++k) {
            const int64_t v = w[k * E + e];
            s[k] += v;
            a[k] += v < 0 ? -v : v;
            m[k] += v < 0 ? v : 0;
        }
    }
    for (int k = 0; k < K; ++k) {
        atomicAdd(&sums[k], (unsigned long long)s[k]);
        atomicAdd(&sums[K + k], (unsigned long long)a[k]);
        atomicAdd(&sums[2 * K + k], (unsigned long long)m[k]);
    }
}

// Integer weight moments for the graph statistics: per k: sum w^2, #(w > 0); per pair k < l:
// sum w_k w_l (exact in 64-bit atomics, so the result does not depend on the order).
__global__ void k_weight_moments(int32_t K, int64_t E, const int32_t* __restrict__ w, unsigned long long* acc)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        int q = 2 * K;
        for (int k = 0; k < K; ++k) {
            const int64_t v = w[k * E + e];
            atomicAdd(&acc[2 * k], (unsigned long long)(v * v));
            atomicAdd(&acc[2 * k + 1], (unsigned long long)(v > 0));
            for (int l = k + 1; l < K; ++l) atomicAdd(&acc[q++], (unsigned long long)(v * (int64_t)w[l * E + e]));
        }
    }
}

// The 8 graph statistics of the learned proposal's input: log n, mean degree / 10, mean over
// objectives of mean|w|/rms(w) and of std(w)/rms(w), the fraction of positive weights, and
// the mean, min and max pairwise Pearson correlation of the objectives' weight vectors.
void graph_features(int n, int K, int64_t E, const long long* sums, const long long* mom, float* out)
{
    const double e = (double)std::max<int64_t>(E, 1);
    double shape = 0.0, spread = 0.0, pos = 0.0;
    double mean[kMaxK], sd[kMaxK];
    for (int k = 0; k < K; ++k) {
        mean[k] = (double)sums[k] / e;
        const double ms = (double)mom[2 * k] / e, rms = std::sqrt(std::max(ms, 1e-300));
        sd[k] = std::sqrt(std::max(ms - mean[k] * mean[k], 0.0));
        shape += ((double)sums[K + k] / e) / rms / K;
        spread += sd[k] / rms / K;
        pos += (double)mom[2 * k + 1] / e / K;
    }
    double cmean = 0.0, cmin = 1.0, cmax = -1.0;
    int q = 2 * K, pairs = 0;
    for (int k = 0; k < K; ++k)
        for (int l = k + 1; l < K; ++l, ++q, ++pairs) {
            const double cov = (double)mom[q] / e - mean[k] * mean[l];
            const double c = (sd[k] > 0 && sd[l] > 0) ? cov / (sd[k] * sd[l]) : 0.0;
            cmean += c;
            cmin = std::min(cmin, c);
            cmax = std::max(cmax, c);
        }
    cmean /= std::max(pairs, 1);
    const double f[8] = {std::log((double)n), 2.0 * (double)E / n / 10.0, shape, spread, pos, cmean, cmin, cmax};
    for (int k = 0; k < 8; ++k) out[k] = (float)f[k];
}

void free_instance(moq_instance* h)
{
    if (!h) return;
    slab_free(h->slab);
    delete h;
}

// Offsets of the arrays of one slab, rounded to 256 bytes; place() fills the pointers once the
// slab exists.
struct SlabPlan {
    std::vector<std::pair<void**, size_t>> parts;
    template <class T>
    void add(T** p, int64_t count) { parts.emplace_back((void**)p, sizeof(T) * (size_t)std::max<int64_t>(count, 1)); }
    size_t bytes() const
    {
        size_t t = 0;
        for (auto& pr : parts) t += slab_align(pr.second);
        return t;
    }
    void place(void* slab) const
    {
        size_t off = 0;
        for (auto& pr : parts) {
            *pr.first = static_cast<char*>(slab) + off;
            off += slab_align(pr.second);
        }
    }
};

// MOQ_SB_LAYOUT_EFFORT = m > 0: the longer layout search (read on every call)
int64_t layout_effort_from_env()
{
    const char* env = getenv("MOQ_SB_LAYOUT_EFFORT");
    return env ? std::max(0, atoi(env)) : 0;
}

// moq_create_instance's layout from the environment: MOQ_SB_LAYOUT=0 keeps the plain layout,
// else the planner with MOQ_SB_LAYOUT_EFFORT's longer search
int32_t layout_from_env()
{
    const char* env = getenv("MOQ_SB_LAYOUT");
    if (env && atoi(env) == 0) return MOQ_LAYOUT_PLAIN;
    return (int32_t)std::min<int64_t>(layout_effort_from_env(), INT32_MAX);
}

int create_instance_impl(int32_t n, int32_t K, int64_t E, const int32_t* ei, const int32_t* ej, const int32_t* w,
                         int32_t layout, void* stream, moq_instance** out);

}  // namespace
}  // namespace moq

extern "C" {

int moq_plan_gather_layout(int32_t n, int64_t E, const int32_t* ei, const int32_t* ej, int32_t* slot_spin, int32_t* gather,
                           int64_t* passes)
{
    using namespace moq;
    if (!ei || !ej || !slot_spin || !gather) return fail(MOQ_ERR_ARG, "moq_plan_gather_layout: NULL pointer");
    std::vector<int32_t> order, remap;
    if (!plan_gather_layout(n, E, ei, ej, order, remap, passes, layout_effort_from_env()))
        return fail(MOQ_ERR_UNSUPPORTED, "moq_plan_gather_layout: graph outside the sparse samplers' range (n=%d, E=%lld)", n,
                    (long long)E);
    std::copy(order.begin(), order.end(), slot_spin);
    // rows by spin, neighbours by column, then placed by remap
    std::vector<int32_t> deg(n, 0), rowptr(n + 1, 0), sorted((size_t)2 * E);
    for (int64_t e = 0; e < E; ++e) {
        ++deg[ei[e]];
        ++deg[ej[e]];
    }
    for (int i = 0; i < n; ++i) rowptr[i + 1] = rowptr[i] + deg[i];
    std::vector<int32_t> fill(rowptr.begin(), rowptr.end() - 1);
    for (int64_t e = 0; e < E; ++e) {
        sorted[fill[ei[e]]++] = ej[e];
        sorted[fill[ej[e]]++] = ei[e];
    }
    for (int i = 0; i < n; ++i) {
        std::sort(sorted.begin() + rowptr[i], sorted.begin() + rowptr[i + 1]);
        for (int r = 0; r < deg[i]; ++r) gather[rowptr[i] + remap[rowptr[i] + r]] = sorted[rowptr[i] + r];
    }
    return MOQ_OK;
}


int moq_create_instance(int32_t n, int32_t K, int64_t E, const int32_t* ei, const int32_t* ej, const int32_t* w,
                        void* stream, moq_instance** out)
{
    return moq::create_instance_impl(n, K, E, ei, ej, w, moq::layout_from_env(), stream, out);
}

int moq_create_instance_layout(int32_t n, int32_t K, int64_t E, const int32_t* ei, const int32_t* ej, const int32_t* w,
                               int32_t layout, void* stream, moq_instance** out)
{
    if (out) *out = nullptr;
    if (layout < MOQ_LAYOUT_PLAIN)
        return moq::fail(MOQ_ERR_ARG, "moq_create_instance_layout: layout=%d below MOQ_LAYOUT_PLAIN", layout);
    return moq::create_instance_impl(n, K, E, ei, ej, w, layout, stream, out);
}

}  // extern "C"

namespace moq {
namespace {
int create_instance_impl(int32_t n, int32_t K, int64_t E, const int32_t* ei, const int32_t* ej, const int32_t* w,
                         int32_t layout, void* stream, moq_instance** out)
{
    if (!out) return fail(MOQ_ERR_ARG, "moq_create_instance: out is NULL");
    *out = nullptr;
    if (n < 2 || n > (1 << 24)) return fail(MOQ_ERR_ARG, "moq_create_instance: n=%d outside [2, 2^24]", n);
    if (K < 2 || K > kMaxK) return fail(MOQ_ERR_ARG, "moq_create_instance: K=%d outside [2, %d]", K, kMaxK);
    if (E < 0 || E >= ((int64_t)1 << 30)) return fail(MOQ_ERR_ARG, "moq_create_instance: E=%lld outside [0, 2^30)", (long long)E);
    if (E > 0 && (!ei || !ej || !w)) return fail(MOQ_ERR_ARG, "moq_create_instance: NULL edge or weight array");
    cudaStream_t st = as_stream(stream);

    moq_instance* h = new moq_instance();
    h->n = n;
    h->K = K;
    h->E = E;
    h->nnz = 2 * E;
    h->words = (n + 63) / 64;
    cudaGetDevice(&h->device);

    int32_t *deg = nullptr, *cursor = nullptr, *col_tmp = nullptr, *eid_tmp = nullptr, *eid = nullptr, *status = nullptr,
            *remap_d = nullptr;
    unsigned long long* sums = nullptr;
    void* tmp_slab = nullptr;
    int rc = MOQ_OK;
    auto cleanup_tmp = [&]() { slab_free_async(tmp_slab, st); };
#define MOQ_STEP(x) do { rc = (x); if (rc != MOQ_OK) { cleanup_tmp(); free_instance(h); return rc; } } while (0)
    // sampler slots in order of decreasing degree (stable), so that warps of the on-chip
    // sampler hold spins of equal degree where the graph allows it (host side, from the
    // edge list; validated on the device below)
    // For graphs the on-chip sampler takes (n <= 1024, degrees <= 8) the slots and the gather
    // order of each CSR row come from plan_gather_layout (against shared-memory bank conflicts;
    // layout = MOQ_LAYOUT_PLAIN keeps the plain layout below, rows by column; m > 0 adds the
    // longer search with m exchanges per spin).
    std::vector<int32_t> order(n), inv(n), remap;
    {
        std::vector<int32_t> dgr(n, 0);
        for (int64_t e = 0; e < E; ++e) {
            if (ei[e] >= 0 && ei[e] < n) ++dgr[ei[e]];
            if (ej[e] >= 0 && ej[e] < n) ++dgr[ej[e]];
        }
        for (int32_t i = 0; i < n; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return dgr[a] > dgr[b]; });
        if (layout != MOQ_LAYOUT_PLAIN) {
            std::vector<int32_t> planned;
            if (plan_gather_layout(n, E, ei, ej, planned, remap, nullptr, layout)) order.swap(planned);
        }
        for (int32_t q = 0; q < n; ++q) inv[order[q]] = q;
    }
    const int nmom = 2 * K + K * (K - 1) / 2;  // weight moments after the 3K sums
    SlabPlan keep, tmp;
    keep.add(&h->ei, E);
    keep.add(&h->ej, E);
    keep.add(&h->w, K * E);
    keep.add(&h->rowptr, n + 1);
    keep.add(&h->col, h->nnz);
    keep.add(&h->wn, K * h->nnz);
    keep.add(&h->rowsum, (int64_t)n * K);
    keep.add(&h->slot_spin, n);
    keep.add(&h->spin_slot, n);
    tmp.add(&deg, n + 1);
    tmp.add(&cursor, n);
    tmp.add(&col_tmp, h->nnz);
    tmp.add(&eid_tmp, h->nnz);
    tmp.add(&eid, h->nnz);
    if (!remap.empty()) tmp.add(&remap_d, h->nnz);
    tmp.add(&status, 2);
    tmp.add(&sums, 3 * K + nmom);
    {
        cudaError_t e = slab_alloc(&h->slab, keep.bytes(), st);
        if (e != cudaSuccess) MOQ_STEP(cuda_fail(e, "moq_create_instance"));
        keep.place(h->slab);
        e = slab_alloc(&tmp_slab, tmp.bytes(), st);
        if (e != cudaSuccess) MOQ_STEP(cuda_fail(e, "moq_create_instance"));
        tmp.place(tmp_slab);
    }

    auto cu = [&](cudaError_t e, const char* what) { return e == cudaSuccess ? MOQ_OK : cuda_fail(e, what); };
    if (E > 0) {
        MOQ_STEP(cu(cudaMemcpyAsync(h->ei, ei, sizeof(int32_t) * E, cudaMemcpyHostToDevice, st), "copy ei"));
        MOQ_STEP(cu(cudaMemcpyAsync(h->ej, ej, sizeof(int32_t) * E, cudaMemcpyHostToDevice, st), "copy ej"));
        MOQ_STEP(cu(cudaMemcpyAsync(h->w, w, sizeof(int32_t) * K * E, cudaMemcpyHostToDevice, st), "copy w"));
    }
    MOQ_STEP(cu(cudaMemcpyAsync(h->slot_spin, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st), "copy slot order"));
    MOQ_STEP(cu(cudaMemcpyAsync(h->spin_slot, inv.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st), "copy slot order"));
    if (remap_d)
        MOQ_STEP(cu(cudaMemcpyAsync(remap_d, remap.data(), sizeof(int32_t) * h->nnz, cudaMemcpyHostToDevice, st), "copy gather order"));
    MOQ_STEP(cu(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (n + 1), st), "memset"));
    MOQ_STEP(cu(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * n, st), "memset"));
    MOQ_STEP(cu(cudaMemsetAsync(status, 0, sizeof(int32_t) * 2, st), "memset"));
    MOQ_STEP(cu(cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * (3 * K + nmom), st), "memset"));

    const int tb = 256;
    const int gE = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(E, tb), 148 * 16));
    const int gN = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, tb), 148 * 16));
    const int gNNZ = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(h->nnz, tb), 148 * 16));
    k_degree<<<gE, tb, 0, st>>>(h->ei, h->ej, E, n, deg, status);
    k_scan_rowptr<<<1, 1024, 0, st>>>(deg, n, h->rowptr);
    k_fill<<<gE, tb, 0, st>>>(h->ei, h->ej, E, n, h->rowptr, cursor, col_tmp, eid_tmp);
    const int gRows = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div((int64_t)n * 32, tb), 148 * 16));
    k_sort_rows<<<gRows, tb, 0, st>>>(n, h->rowptr, col_tmp, eid_tmp, remap_d, h->col, eid, status);
    k_entry_weights<<<gNNZ, tb, 0, st>>>(K, h->nnz, E, eid, h->w, h->wn);
    k_row_sums<<<gN, tb, 0, st>>>(n, K, h->nnz, h->rowptr, h->wn, h->rowsum, status + 1);
    k_weight_sums<<<gE, tb, 0, st>>>(K, E, h->w, sums);
    k_weight_moments<<<gE, tb, 0, st>>>(K, E, h->w, sums + 3 * K);
    {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) MOQ_STEP(cuda_fail(e, "instance build launch"));
    }
    struct ReadBack {
        long long sums[3 * kMaxK + 2 * kMaxK + kMaxK * (kMaxK - 1) / 2];
        int32_t status[2];
    } local;
    PinnedLease lease(sizeof(ReadBack));
    lease.arm(st);
    ReadBack& rb = lease.p ? *static_cast<ReadBack*>(lease.p) : local;
    int32_t* hstatus = rb.status;
    long long* hsums = rb.sums;
    MOQ_STEP(cu(cudaMemcpyAsync(hstatus, status, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, st), "read status"));
    MOQ_STEP(cu(cudaMemcpyAsync(hsums, sums, sizeof(long long) * (3 * K + nmom), cudaMemcpyDeviceToHost, st), "read sums"));
    MOQ_STEP(cu(cudaStreamSynchronize(st), "instance build"));
    if (hstatus[0] & kStatusBadEdge) MOQ_STEP(fail(MOQ_ERR_ARG, "moq_create_instance: an edge has i >= j or an endpoint outside [0, n)"));
    if (hstatus[0] & kStatusDuplicateEdge) MOQ_STEP(fail(MOQ_ERR_ARG, "moq_create_instance: repeated edge"));
    cleanup_tmp();
#undef MOQ_STEP
    h->max_degree = hstatus[1];
    moq_instance_info& inf = h->info;
    memset(&inf, 0, sizeof(inf));
    inf.n = n;
    inf.K = K;
    inf.E = E;
    inf.max_degree = h->max_degree;
    inf.words = h->words;
    for (int k = 0; k < K; ++k) {
        inf.weight_sum[k] = hsums[k];
        inf.abs_sum[k] = hsums[K + k];
        inf.ref_point[k] = hsums[2 * K + k];
    }
    graph_features(n, K, E, hsums, hsums + 3 * K, inf.features);
    *out = h;
    return MOQ_OK;
}
}  // namespace
}  // namespace moq

extern "C" {

void moq_destroy_instance(moq_instance* inst) { moq::free_instance(inst); }

int moq_instance_get_info(const moq_instance* inst, moq_instance_info* out)
{
    if (!inst || !out) return moq::fail(MOQ_ERR_ARG, "moq_instance_get_info: NULL argument");
    *out = inst->info;
    return MOQ_OK;
}

int moq_create_instance_dense(int32_t n, int32_t K, const int32_t* J_upper, void* stream, moq_instance** out)
{
    using namespace moq;
    if (!out) return fail(MOQ_ERR_ARG, "moq_create_instance_dense: out is NULL");
    *out = nullptr;
    if (n < 2 || n > (1 << 16)) return fail(MOQ_ERR_ARG, "moq_create_instance_dense: n=%d outside [2, 65536]", n);
    if (K < 2 || K > kMaxK) return fail(MOQ_ERR_ARG, "moq_create_instance_dense: K=%d outside [2, %d]", K, kMaxK);
    if (!J_upper) return fail(MOQ_ERR_ARG, "moq_create_instance_dense: NULL weights");
    // pairs (i, j), i < j, row by row: the edges are the pairs with a non-zero weight in
    // some objective, in that order
    const int64_t P = (int64_t)n * (n - 1) / 2;
    std::vector<int32_t> ei, ej;
    std::vector<int64_t> at;
    int64_t q = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = i + 1; j < n; ++j, ++q) {
            bool any = false;
            for (int k = 0; k < K && !any; ++k) any = J_upper[(int64_t)k * P + q] != 0;
            if (any) {
                ei.push_back(i);
                ej.push_back(j);
                at.push_back(q);
            }
        }
    const int64_t E = (int64_t)ei.size();
    std::vector<int32_t> w((size_t)K * E);
    for (int k = 0; k < K; ++k)
        for (int64_t e = 0; e < E; ++e) w[(size_t)k * E + e] = J_upper[(int64_t)k * P + at[e]];
    return moq_create_instance(n, K, E, ei.data(), ej.data(), w.data(), stream, out);
}

}  // extern "C"
