// a7: deduplication + Pareto filter merged into a device archive ("Pareto filtering").
//
// Maximisation order: u dominates v iff u_k >= v_k for all k and u_j > v_j for some j.
// The archive A holds the distinct non-dominated vectors of every earlier call, each with
// its lowest global sample index. For a batch X of M candidates:
//  - candidate u survives iff no member of A weakly dominates it (>= everywhere: either
//    it dominates u or equals u and has a lower index), no candidate dominates it, and no
//    equal candidate has a lower index;
//  - member a survives iff no candidate dominates it (a dominated member is dominated by
//    some surviving vector too, since domination is transitive and the sets are finite).
// The tests run either one warp per tested vector (k_dominated_warp, the default) or, as below,
// all-pairs over shared-memory tiles on a 2-D grid (a tile of vectors x a
// chunk of the vectors they are compared with, so even one tile of candidates fills the
// GPU), with a block-wide early exit once every thread's vector is known to be dominated;
// blocks only ever set "dominated" flags (zeroed per call). Survivors are compacted in order --
// old members first, then candidates by index -- into the second buffer of the archive
// by a block scan, so the result is deterministic. Candidate representatives are
// canonicalised to s_0 = +1 (C(s) = C(-s)).
// Packed comparisons: when every objective spans fewer than 2^15 values over the archive
// and the batch (one reduction per call decides, on the device), the candidate test
// shifts each vector by the per-objective minimum and packs it into 16-bit lanes, four
// objectives per 64-bit word. With the top bit of every lane of t set, (t | H) - u has
// the top bit of lane k set iff t_k >= u_k and no borrow crosses a lane, so one
// subtract and one mask test compare four objectives at once. Same decisions, fewer
// instructions.
#include <algorithm>
#include <stdlib.h>

#include <vector>

#include "moq_common.cuh"

namespace moq {
namespace {

constexpr int kTile = 256;
constexpr int kScanBlock = 1024;
constexpr unsigned kFull = 0xffffffffu;

constexpr int kChunk = 1024;   // candidates compared by one block of the 2-D grid
constexpr int64_t kLargeBatch = 1 << 13;  // batches from this size take the dedup / survivor path (MOQ_LARGE_BATCH)
constexpr int kArchChunks = 8; // archive slices per candidate tile

// Dominance of one candidate u (registers) by any vector of a shared-memory tile.
template <int KT, bool ARCHIVE>
__device__ __forceinline__ bool tile_dominates(const int64_t (*tile)[KT], int cnt, const int64_t (&u)[KT], int64_t tile_base,
                                               int64_t c)
{
    for (int t = 0; t < cnt; ++t) {
        bool ge = true, gt = false;
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            ge &= tile[t][k] >= u[k];
            gt |= tile[t][k] > u[k];
        }
        // archive members win ties (lower global index); among candidates the lower index wins
        if (ge && (ARCHIVE || gt || tile_base + t < c)) return true;
    }
    return false;
}

// ---- 16-bit packed vectors ------------------------------------------------------
constexpr uint64_t kLaneHigh = 0x8000800080008000ull;
constexpr unsigned long long kSignBit = 0x8000000000000000ull;
constexpr unsigned long long kPackSpan = 1ull << 15;

template <int KT>
struct Packed {
    static constexpr int NW = (KT + 3) / 4;
    uint64_t w[NW];
};

// Per-objective minimum and maximum over the archive and the batch, as order-preserving
// unsigned keys (v ^ sign bit) so that 64-bit unsigned atomics order signed values;
// range[0..K) holds the minima (preset to all ones), range[K..2K) the maxima (preset 0).
template <int KT>
__global__ void __launch_bounds__(kTile) k_value_range(const int64_t* __restrict__ arch, const int64_t* __restrict__ d_count,
                                                       const int64_t* __restrict__ cand, int64_t M,
                                                       unsigned long long* range)
{
    const int64_t F = *d_count, total = F + M;
    unsigned long long lo[KT], hi[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        lo[k] = ~0ull;
        hi[k] = 0;
    }
    for (int64_t i = blockIdx.x * (int64_t)kTile + threadIdx.x; i < total; i += (int64_t)gridDim.x * kTile) {
        const int64_t* v = i < F ? arch + i * KT : cand + (i - F) * KT;
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const unsigned long long key = (unsigned long long)v[k] ^ kSignBit;
            lo[k] = min(lo[k], key);
            hi[k] = max(hi[k], key);
        }
    }
#pragma unroll
    for (int k = 0; k < KT; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = min(lo[k], __shfl_xor_sync(kFull, lo[k], o));
            hi[k] = max(hi[k], __shfl_xor_sync(kFull, hi[k], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&range[k], lo[k]);
            atomicMax(&range[KT + k], hi[k]);
        }
    }
}

// True (uniformly over the grid) when every objective spans fewer than 2^15 values; lo
// receives the per-objective minima.
template <int KT>
__device__ __forceinline__ bool packable(const unsigned long long* __restrict__ range, int64_t (&lo)[KT])
{
    bool ok = true;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const unsigned long long a = range[k], b = range[KT + k];
        lo[k] = (int64_t)(a ^ kSignBit);
        ok &= a <= b && b - a < kPackSpan;
    }
    return ok;
}

template <int KT>
__device__ __forceinline__ Packed<KT> pack(const int64_t (&v)[KT], const int64_t (&lo)[KT])
{
    Packed<KT> p;
#pragma unroll
    for (int w = 0; w < Packed<KT>::NW; ++w) p.w[w] = 0;
#pragma unroll
    for (int k = 0; k < KT; ++k) p.w[k >> 2] |= (uint64_t)(v[k] - lo[k]) << (16 * (k & 3));
    return p;
}

// t_k >= u_k for every k, four lanes per subtract
template <int KT>
__device__ __forceinline__ bool packed_ge(const Packed<KT>& t, const Packed<KT>& u)
{
    bool ge = true;
#pragma unroll
    for (int w = 0; w < Packed<KT>::NW; ++w) ge &= ((~((t.w[w] | kLaneHigh) - u.w[w])) & kLaneHigh) == 0;
    return ge;
}

template <int KT>
__device__ __forceinline__ bool packed_eq(const Packed<KT>& t, const Packed<KT>& u)
{
    bool eq = true;
#pragma unroll
    for (int w = 0; w < Packed<KT>::NW; ++w) eq &= t.w[w] == u.w[w];
    return eq;
}

template <int KT, bool ARCHIVE>
__device__ __forceinline__ bool tile_dominates_packed(const Packed<KT>* tile, int cnt, const Packed<KT>& u,
                                                      int64_t tile_base, int64_t c)
{
    for (int t = 0; t < cnt; ++t) {
        const Packed<KT> v = tile[t];
        if (packed_ge<KT>(v, u) && (ARCHIVE || tile_base + t < c || !packed_eq<KT>(v, u))) return true;
    }
    return false;
}

// Candidates: blockIdx.x = tile of 256 candidates, blockIdx.y = what they are compared
// with: y < kArchChunks strides over archive tiles, y >= kArchChunks takes candidate
// chunk y - kArchChunks. Any block that finds a dominator sets dom_cand (zeroed per call).
template <int KT>
__global__ void __launch_bounds__(kTile) k_dominated_candidates(const int64_t* __restrict__ arch, const int64_t* __restrict__ d_count,
                                                                const int64_t* __restrict__ cand, int64_t M, int32_t* dom_cand,
                                                                const unsigned long long* __restrict__ range, int arch_chunks,
                                                                const int64_t* __restrict__ d_m)
{
    if (d_m) M = min(M, *d_m);  // the compacted survivors of the large-batch path
    if (blockIdx.x * (int64_t)kTile >= M) return;
    __shared__ int64_t tile[kTile][KT];
    Packed<KT>* ptile = reinterpret_cast<Packed<KT>*>(&tile[0][0]);  // NW <= KT words per row
    const int tid = threadIdx.x;
    const int64_t c = blockIdx.x * (int64_t)kTile + tid;
    const bool act = c < M;
    int64_t u[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) u[k] = act ? cand[c * KT + k] : 0;
    int64_t lo[KT];
    const bool pk = packable<KT>(range, lo);
    const Packed<KT> up = pack<KT>(u, lo);
    bool dropped = !act || dom_cand[c];
    const bool was = dropped;
    const bool vs_archive = (int)blockIdx.y < arch_chunks;
    const int64_t lo_i = vs_archive ? (int64_t)blockIdx.y * kTile : (int64_t)(blockIdx.y - arch_chunks) * kChunk;
    const int64_t hi_i = vs_archive ? *d_count : min(M, lo_i + kChunk);
    const int64_t stride = vs_archive ? (int64_t)arch_chunks * kTile : kTile;
    const int64_t* src = vs_archive ? arch : cand;
    for (int64_t base = lo_i; base < hi_i; base += stride) {
        if (__syncthreads_and(dropped)) break;
        const int cnt = (int)min((int64_t)kTile, hi_i - base);
        if (tid < cnt) {
            int64_t v[KT];
#pragma unroll
            for (int k = 0; k < KT; ++k) v[k] = src[(base + tid) * KT + k];
            if (pk) {
                ptile[tid] = pack<KT>(v, lo);
            } else {
#pragma unroll
                for (int k = 0; k < KT; ++k) tile[tid][k] = v[k];
            }
        }
        __syncthreads();
        if (!dropped) {
            if (pk)
                dropped = vs_archive ? tile_dominates_packed<KT, true>(ptile, cnt, up, base, c)
                                     : tile_dominates_packed<KT, false>(ptile, cnt, up, base, c);
            else
                dropped = vs_archive ? tile_dominates<KT, true>(tile, cnt, u, base, c)
                                     : tile_dominates<KT, false>(tile, cnt, u, base, c);
        }
    }
    if (act && dropped && !was) dom_cand[c] = 1;
}

// Archive members: blockIdx.x strides over archive tiles, blockIdx.y = candidate chunk;
// a member is dropped when a candidate dominates it strictly.
template <int KT>
__global__ void __launch_bounds__(kTile) k_dominated_archive(const int64_t* __restrict__ arch, const int64_t* __restrict__ d_count,
                                                             const int64_t* __restrict__ cand, int64_t M, int32_t* dom_arch,
                                                             const int64_t* __restrict__ d_m)
{
    __shared__ int64_t tile[kTile][KT];
    const int tid = threadIdx.x;
    const int64_t F = *d_count;
    if (d_m) M = min(M, *d_m);
    const int64_t lo = (int64_t)blockIdx.y * kChunk, hi = min(M, lo + kChunk);
    for (int64_t blk = blockIdx.x; blk * kTile < F; blk += gridDim.x) {
        const int64_t a = blk * kTile + tid;
        const bool act = a < F;
        int64_t u[KT];
#pragma unroll
        for (int k = 0; k < KT; ++k) u[k] = act ? arch[a * KT + k] : 0;
        bool dropped = !act || dom_arch[a];
        const bool was = dropped;
        for (int64_t base = lo; base < hi; base += kTile) {
            if (__syncthreads_and(dropped)) break;
            const int cnt = (int)min((int64_t)kTile, hi - base);
            if (tid < cnt) {
#pragma unroll
                for (int k = 0; k < KT; ++k) tile[tid][k] = cand[(base + tid) * KT + k];
            }
            __syncthreads();
            if (!dropped) {
                for (int t = 0; t < cnt; ++t) {
                    bool ge = true, gt = false;
#pragma unroll
                    for (int k = 0; k < KT; ++k) {
                        ge &= tile[t][k] >= u[k];
                        gt |= tile[t][k] > u[k];
                    }
                    if (ge && gt) {
                        dropped = true;
                        break;
                    }
                }
            }
        }
        if (act && dropped && !was) dom_arch[a] = 1;
        __syncthreads();
    }
}

// ---- one warp per tested vector ----------------------------------------------------
// The same tests with one warp per tested vector: its lanes take 128 comparators at a time,
// read straight from global memory (coalesced; the eight warps of a block read the same
// comparators, which L1 keeps), and the warp stops after the first 128 that hold a dominator
// (a vote), so a vector dominated early costs a few chunks where the tile form keeps a whole
// warp scanning until its last vector is decided.
//   MODE 0: a candidate against the archive (>= everywhere: dominated, or an equal member,
//           whose index is lower);
//   MODE 1: a candidate against the candidates (dominated, or equal with a lower index);
//   MODE 2: an archive member against the candidates (strictly dominated).
// Counts may live on the device (the archive size, the compacted survivors); flags already
// set are skipped and only ever set.
// K int64 values of one vector, in 16-byte loads when K is even and the array is 16-byte
// aligned (then every row is)
template <int KT>
__device__ __forceinline__ void load_vec(const int64_t* __restrict__ p, int64_t (&v)[KT], bool vec16)
{
    if (KT % 2 == 0 && vec16) {
#pragma unroll
        for (int k = 0; k < KT; k += 2) {
            const longlong2 w = __ldg(reinterpret_cast<const longlong2*>(p + k));
            v[k] = w.x;
            v[k + 1] = w.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < KT; ++k) v[k] = __ldg(p + k);
    }
}

template <int KT, int MODE>
__global__ void __launch_bounds__(kTile) k_dominated_warp(const int64_t* __restrict__ vecs, int64_t n_vecs,
                                                          const int64_t* __restrict__ n_vecs_dev, const int64_t* __restrict__ cmp,
                                                          int64_t n_cmp, const int64_t* __restrict__ n_cmp_dev, int32_t* flag,
                                                          bool vec16)
{
    const int lane = threadIdx.x & 31;
    const int64_t nv = n_vecs_dev ? min(n_vecs, *n_vecs_dev) : n_vecs;
    const int64_t nc = n_cmp_dev ? min(n_cmp, *n_cmp_dev) : n_cmp;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < nv; c += nw) {
        if (flag[c]) continue;  // the same word for every lane
        int64_t u[KT];
#pragma unroll
        for (int k = 0; k < KT; ++k) u[k] = vecs[c * KT + k];
        // four chunks of 32 per vote: their loads are in flight together (the test is bound
        // by the latency of the comparator loads, not by the comparisons)
        bool dom = false;
        for (int64_t base = 0; base < nc && !dom; base += 4 * 32) {
            bool d = false;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t j = base + 32 * q + lane;
                if (j < nc) {
                    int64_t v[KT];
                    load_vec<KT>(cmp + j * KT, v, vec16);
                    bool ge = true, gt = false;
#pragma unroll
                    for (int k = 0; k < KT; ++k) {
                        ge &= v[k] >= u[k];
                        gt |= v[k] > u[k];
                    }
                    d |= ge && (MODE == 0 || gt || (MODE == 1 && j < c));
                }
            }
            dom = __any_sync(kFull, d);
        }
        if (dom && lane == 0) flag[c] = 1;
    }
}

// The filter form: one warp per tested vector (default) or a thread per vector over
// shared-memory tiles (MOQ_FILTER_FORM=thread)
bool warp_filter()
{
    const char* env = getenv("MOQ_FILTER_FORM");
    return !(env && env[0] == 't');
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

unsigned warp_grid(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kTile / 32), 148 * 16)); }

// ---- large batches: deduplication and survivors ----------------------------------
// A batch of many samples holds few distinct cut vectors and, once the archive has grown,
// few that the archive does not already cover. Before the all-pairs test, (1) an open-
// addressing hash table keeps, for every distinct vector, its lowest candidate index
// (later copies are flagged), (2) the candidates are tested against the archive alone,
// and (3) the survivors are compacted, so the candidate-candidate test runs on distinct,
// uncovered vectors only. Among distinct vectors dominance does not depend on order, so
// the compaction may be unordered; flags go back to the original positions.
constexpr int32_t kEmptySlot = -1;

template <int KT>
__device__ __forceinline__ uint64_t vec_hash(const int64_t* v)
{
    uint64_t h = 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        uint64_t z = (uint64_t)v[k] + h + 0x9E3779B97F4A7C15ull * (k + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        h = z ^ (z >> 31);
    }
    return h;
}

template <int KT>
__device__ __forceinline__ bool vec_eq(const int64_t* a, const int64_t* b)
{
    bool eq = true;
#pragma unroll
    for (int k = 0; k < KT; ++k) eq &= a[k] == b[k];
    return eq;
}

// Insert every candidate; a slot ends holding the lowest index of its vector. Probing is
// linear and bounded by the table size (the table has at least twice the batch's slots).
template <int KT>
__global__ void k_dedup_insert(const int64_t* __restrict__ cand, int64_t M, int32_t* table, uint32_t mask)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= M) return;
    const int64_t* v = cand + c * KT;
    uint32_t slot = (uint32_t)vec_hash<KT>(v) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe, slot = (slot + 1) & mask) {
        int32_t cur = table[slot];
        if (cur == kEmptySlot) {
            cur = atomicCAS(&table[slot], kEmptySlot, (int32_t)c);
            if (cur == kEmptySlot) return;
        }
        if (vec_eq<KT>(cand + (int64_t)cur * KT, v)) {
            atomicMin(&table[slot], (int32_t)c);
            return;
        }
    }
}

// Flag every candidate whose vector's slot holds a lower index.
template <int KT>
__global__ void k_dedup_mark(const int64_t* __restrict__ cand, int64_t M, const int32_t* __restrict__ table, uint32_t mask,
                             int32_t* dom_cand)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= M) return;
    const int64_t* v = cand + c * KT;
    uint32_t slot = (uint32_t)vec_hash<KT>(v) & mask;
    for (uint32_t probe = 0; probe <= mask; ++probe, slot = (slot + 1) & mask) {
        const int32_t cur = table[slot];
        if (cur == kEmptySlot) return;  // not reachable: every candidate was inserted
        if (vec_eq<KT>(cand + (int64_t)cur * KT, v)) {
            if (cur != (int32_t)c) dom_cand[c] = 1;
            return;
        }
    }
}

// Survivors (unflagged candidates) into a compact buffer, in any order; *d_m counts them.
template <int KT>
__global__ void k_compact_survivors(const int64_t* __restrict__ cand, int64_t M, const int32_t* __restrict__ dom_cand,
                                    int64_t* ccuts, int32_t* cidx, unsigned long long* d_m)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool keep = c < M && !dom_cand[c];
    const unsigned ballot = __ballot_sync(kFull, keep);
    if (!ballot) return;
    const int lane = threadIdx.x & 31, leader = __ffs(ballot) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(d_m, (unsigned long long)__popc(ballot));
    base = __shfl_sync(kFull, base, leader);
    if (!keep) return;
    const int64_t pos = (int64_t)base + __popc(ballot & ((1u << lane) - 1u));
#pragma unroll
    for (int k = 0; k < KT; ++k) ccuts[pos * KT + k] = cand[c * KT + k];
    cidx[pos] = (int32_t)c;
}

__global__ void k_survivor_flags_back(const int64_t* __restrict__ d_m, const int32_t* __restrict__ cflag,
                                      const int32_t* __restrict__ cidx, int32_t* dom_cand)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q < *d_m && cflag[q]) dom_cand[cidx[q]] = 1;
}

// Flag of virtual position b*1024+t: blocks [0, nbA) cover archive slots, blocks
// [nbA, nbA+nbC) cover candidates.
__device__ __forceinline__ int32_t flag_at(int64_t b, int t, int64_t nbA, int64_t F, int64_t M,
                                           const int32_t* flag_arch, const int32_t* flag_cand)
{
    if (b < nbA) {
        const int64_t q = b * kScanBlock + t;
        return q < F ? 1 - flag_arch[q] : 0;
    }
    const int64_t c = (b - nbA) * kScanBlock + t;
    return c < M ? 1 - flag_cand[c] : 0;
}

__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t* warp_sums, int32_t* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[wid] = incl;
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
    const int32_t res = incl - v + (wid > 0 ? warp_sums[wid - 1] : 0);
    *total = warp_sums[31];
    return res;
}

__global__ void __launch_bounds__(kScanBlock) k_count_flags(int64_t nbA, int64_t M, const int64_t* __restrict__ d_count,
                                                           const int32_t* __restrict__ flag_arch, const int32_t* __restrict__ flag_cand,
                                                           int64_t* blocksum)
{
    __shared__ int32_t warp_sums[32];
    const int64_t F = *d_count;
    const int64_t b = blockIdx.x;
    if (b < nbA && b * kScanBlock >= F) {
        if (threadIdx.x == 0) blocksum[b] = 0;
        return;
    }
    const int32_t v = flag_at(b, threadIdx.x, nbA, F, M, flag_arch, flag_cand);
    int32_t total;
    block_excl_scan(v, warp_sums, &total);
    if (threadIdx.x == 0) blocksum[b] = total;
}

// Exclusive scan of nb block sums in place; blocksum[nb] receives the total.
__global__ void __launch_bounds__(kScanBlock) k_scan_blocksums(int64_t nb, int64_t* blocksum)
{
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < nb ? blocksum[i] : 0;
        int64_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sums[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int64_t s = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t t = __shfl_up_sync(kFull, s, o);
                if (lane >= o) s += t;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const int64_t excl = incl - v + (wid > 0 ? warp_sums[wid - 1] : 0) + carry;
        if (i < nb) blocksum[i] = excl;
        __syncthreads();
        if (threadIdx.x == kScanBlock - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) blocksum[nb] = carry;
}

struct ScatterArgs {
    int32_t K, W, n;
    int64_t cap, nbA, M, index_base;
    const int64_t* d_count;
    const int32_t* flag_arch;
    const int32_t* flag_cand;
    const int64_t* blockoff;  // nb + 1
    int64_t nb;
    const int64_t* old_cuts;
    const uint64_t* old_bits;
    const int64_t* old_index;
    const int64_t* cand_cuts;
    const uint64_t* cand_bits;
    const int64_t* cand_index;  // NULL: candidate c has index index_base + c
    int64_t* new_cuts;
    uint64_t* new_bits;
    int64_t* new_index;
    int32_t* status;
};

__global__ void __launch_bounds__(kScanBlock) k_scatter(const ScatterArgs s)
{
    __shared__ int32_t warp_sums[32];
    const int64_t F = *s.d_count;
    const int64_t b = blockIdx.x;
    const int64_t total = s.blockoff[s.nb];
    const bool overflow = total > s.cap;
    if (b < s.nbA && b * kScanBlock >= F) {  // empty archive slots
        // block 0 latches an overflow here too, when the archive is empty
        if (b == 0 && threadIdx.x == 0 && overflow) atomicOr(s.status, kStatusCapacity);
        return;
    }
    if (overflow) {
        // keep the archive as it was: copy members to the same slots
        if (b == 0 && threadIdx.x == 0) atomicOr(s.status, kStatusCapacity);
        if (b >= s.nbA) return;
        const int64_t q = b * kScanBlock + threadIdx.x;
        if (q < F) {
            for (int k = 0; k < s.K; ++k) s.new_cuts[q * s.K + k] = s.old_cuts[q * s.K + k];
            for (int w = 0; w < s.W; ++w) s.new_bits[q * s.W + w] = s.old_bits[q * s.W + w];
            s.new_index[q] = s.old_index[q];
        }
        return;
    }
    const int32_t v = flag_at(b, threadIdx.x, s.nbA, F, s.M, s.flag_arch, s.flag_cand);
    int32_t tot;
    const int32_t local = block_excl_scan(v, warp_sums, &tot);
    if (!v) return;
    const int64_t pos = s.blockoff[b] + local;
    if (b < s.nbA) {
        const int64_t q = b * kScanBlock + threadIdx.x;
        for (int k = 0; k < s.K; ++k) s.new_cuts[pos * s.K + k] = s.old_cuts[q * s.K + k];
        for (int w = 0; w < s.W; ++w) s.new_bits[pos * s.W + w] = s.old_bits[q * s.W + w];
        s.new_index[pos] = s.old_index[q];
    } else {
        const int64_t c = (b - s.nbA) * kScanBlock + threadIdx.x;
        for (int k = 0; k < s.K; ++k) s.new_cuts[pos * s.K + k] = s.cand_cuts[c * s.K + k];
        const bool flip = s.cand_bits[c * s.W] & 1ull;  // s_0 = -1 -> store -s
        for (int w = 0; w < s.W; ++w) {
            uint64_t word = s.cand_bits[c * s.W + w];
            if (flip) {
                const int lo = w * 64;
                const int nbits = min(64, s.n - lo);
                const uint64_t mask = nbits >= 64 ? ~0ull : ((1ull << nbits) - 1ull);
                word ^= mask;
            }
            s.new_bits[pos * s.W + w] = word;
        }
        s.new_index[pos] = s.cand_index ? s.cand_index[c] : s.index_base + c;
    }
}

__global__ void k_set_count(int64_t cap, int64_t nb, const int64_t* blockoff, int64_t* d_count)
{
    const int64_t total = blockoff[nb];
    if (total <= cap) *d_count = total;
}

template <int KT>
cudaError_t launch_filters(moq_archive* a, const int64_t* cuts, int64_t M, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(a->flag_arch, 0, sizeof(int32_t) * a->cap, st);
    if (e == cudaSuccess && M > 0) e = cudaMemsetAsync(a->flag_cand, 0, sizeof(int32_t) * M, st);
    if (e != cudaSuccess) return e;
    if (M > 0) {
        const bool wf = warp_filter();
        if (!wf) {  // the value range decides the tile form's packed comparisons
            e = cudaMemsetAsync(a->range, 0xff, sizeof(unsigned long long) * KT, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(a->range + KT, 0, sizeof(unsigned long long) * KT, st);
            if (e != cudaSuccess) return e;
            k_value_range<KT><<<148, kTile, 0, st>>>(a->cuts[a->cur], a->d_count, cuts, M, a->range);
        }
        const unsigned nchunks = (unsigned)ceil_div(M, kChunk), gtiles = (unsigned)ceil_div(M, kTile);
        const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(a->cap, kTile), 32));
        if (M < a->large_min) {
            if (wf) {
                k_dominated_warp<KT, 0><<<warp_grid(M), kTile, 0, st>>>(cuts, M, nullptr, a->cuts[a->cur], a->cap, a->d_count,
                                                                         a->flag_cand, aligned16(a->cuts[a->cur]));
                k_dominated_warp<KT, 1><<<warp_grid(M), kTile, 0, st>>>(cuts, M, nullptr, cuts, M, nullptr, a->flag_cand,
                                                                         aligned16(cuts));
                k_dominated_warp<KT, 2><<<warp_grid(a->cap), kTile, 0, st>>>(a->cuts[a->cur], a->cap, a->d_count, cuts, M, nullptr,
                                                                              a->flag_arch, aligned16(cuts));
            } else {
                k_dominated_candidates<KT><<<dim3(gtiles, kArchChunks + nchunks), kTile, 0, st>>>(
                    a->cuts[a->cur], a->d_count, cuts, M, a->flag_cand, a->range, kArchChunks, nullptr);
                k_dominated_archive<KT><<<dim3(gx, nchunks), kTile, 0, st>>>(a->cuts[a->cur], a->d_count, cuts, M, a->flag_arch,
                                                                              nullptr);
            }
        } else {
            const unsigned g256 = (unsigned)ceil_div(M, 256);
            e = cudaMemsetAsync(a->table, 0xff, sizeof(int32_t) * ((size_t)a->table_mask + 1), st);
            if (e == cudaSuccess) e = cudaMemsetAsync(a->d_m, 0, sizeof(int64_t), st);
            if (e == cudaSuccess) e = cudaMemsetAsync(a->cflag, 0, sizeof(int32_t) * M, st);
            if (e != cudaSuccess) return e;
            k_dedup_insert<KT><<<g256, 256, 0, st>>>(cuts, M, a->table, a->table_mask);
            k_dedup_mark<KT><<<g256, 256, 0, st>>>(cuts, M, a->table, a->table_mask, a->flag_cand);
            if (wf)
                k_dominated_warp<KT, 0><<<warp_grid(M), kTile, 0, st>>>(cuts, M, nullptr, a->cuts[a->cur], a->cap, a->d_count,
                                                                         a->flag_cand, aligned16(a->cuts[a->cur]));
            else
                k_dominated_candidates<KT><<<dim3(gtiles, kArchChunks), kTile, 0, st>>>(a->cuts[a->cur], a->d_count, cuts, M,
                                                                                       a->flag_cand, a->range, kArchChunks, nullptr);
            k_compact_survivors<KT><<<g256, 256, 0, st>>>(cuts, M, a->flag_cand, a->ccuts, a->cidx,
                                                          reinterpret_cast<unsigned long long*>(a->d_m));
            if (wf) {
                k_dominated_warp<KT, 1><<<warp_grid(M), kTile, 0, st>>>(a->ccuts, M, a->d_m, a->ccuts, M, a->d_m, a->cflag,
                                                                         aligned16(a->ccuts));
                k_dominated_warp<KT, 2><<<warp_grid(a->cap), kTile, 0, st>>>(a->cuts[a->cur], a->cap, a->d_count, a->ccuts, M, a->d_m,
                                                                              a->flag_arch, aligned16(a->ccuts));
            } else {
                k_dominated_candidates<KT><<<dim3(gtiles, nchunks), kTile, 0, st>>>(a->cuts[a->cur], a->d_count, a->ccuts, M,
                                                                                   a->cflag, a->range, 0, a->d_m);
                k_dominated_archive<KT><<<dim3(gx, nchunks), kTile, 0, st>>>(a->cuts[a->cur], a->d_count, a->ccuts, M, a->flag_arch,
                                                                             a->d_m);
            }
            k_survivor_flags_back<<<g256, 256, 0, st>>>(a->d_m, a->cflag, a->cidx, a->flag_cand);
        }
    }
    return cudaGetLastError();
}

int read_status(const moq_archive* a, cudaStream_t st, int64_t* size_out)
{
    MOQ_CUDA_TRY(cudaMemcpyAsync(a->h_pinned, a->d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    MOQ_CUDA_TRY(cudaMemcpyAsync(a->h_pinned + 1, a->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MOQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (size_out) *size_out = a->h_pinned[0];
    const int32_t status = (int32_t)a->h_pinned[1];
    if (status & kStatusCapacity) {
        MOQ_CUDA_TRY(cudaMemsetAsync(a->d_status, 0, sizeof(int32_t), st));
        return fail(MOQ_ERR_CAPACITY, "archive capacity %lld exceeded; the archive was left unchanged", (long long)a->cap);
    }
    return MOQ_OK;
}

}  // namespace

void free_archive(moq_archive* a)
{
    if (!a) return;
    slab_free(a->slab);
    pinned_slot_free(a->h_pinned);
    delete a;
}

}  // namespace moq

extern "C" {

int moq_archive_create(int32_t n, int32_t K, int64_t capacity, int64_t max_batch, moq_archive** out)
{
    using namespace moq;
    if (!out) return fail(MOQ_ERR_ARG, "moq_archive_create: out is NULL");
    *out = nullptr;
    if (n < 2 || n > (1 << 24) || K < 2 || K > kMaxK) return fail(MOQ_ERR_ARG, "moq_archive_create: bad n=%d or K=%d", n, K);
    if (capacity < 1 || capacity > ((int64_t)1 << 30) || max_batch < 1 || max_batch > ((int64_t)1 << 30))
        return fail(MOQ_ERR_ARG, "moq_archive_create: capacity and max_batch must be in [1, 2^30]");
    moq_archive* a = new moq_archive();
    a->n = n;
    a->K = K;
    a->W = (n + 63) / 64;
    a->cap = capacity;
    a->max_batch = max_batch;
    cudaGetDevice(&a->device);
    a->n_blocksum = ceil_div(capacity, kScanBlock) + ceil_div(max_batch, kScanBlock) + 1;
    // every device array in one slab: the offsets first, then one allocation
    std::vector<std::pair<void**, size_t>> parts;
    auto al = [&](void** p, size_t bytes) { parts.emplace_back(p, bytes); };
    for (int b = 0; b < 2; ++b) {
        al((void**)&a->cuts[b], sizeof(int64_t) * capacity * K);
        al((void**)&a->bits[b], sizeof(uint64_t) * capacity * a->W);
        al((void**)&a->index[b], sizeof(int64_t) * capacity);
    }
    al((void**)&a->d_count, sizeof(int64_t));
    al((void**)&a->d_status, sizeof(int32_t));
    al((void**)&a->flag_arch, sizeof(int32_t) * capacity);
    al((void**)&a->flag_cand, sizeof(int32_t) * max_batch);
    al((void**)&a->blocksum, sizeof(int64_t) * a->n_blocksum);
    al((void**)&a->range, sizeof(unsigned long long) * 2 * kMaxK);
    a->large_min = kLargeBatch;
    if (const char* env = getenv("MOQ_LARGE_BATCH")) a->large_min = std::max<int64_t>(1, atoll(env));
    if (max_batch >= a->large_min) {
        uint32_t slots = 1;
        while (slots < 2 * (uint64_t)max_batch) slots <<= 1;
        a->table_mask = slots - 1;
        al((void**)&a->table, sizeof(int32_t) * (size_t)slots);
        al((void**)&a->ccuts, sizeof(int64_t) * (size_t)max_batch * K);
        al((void**)&a->cidx, sizeof(int32_t) * (size_t)max_batch);
        al((void**)&a->cflag, sizeof(int32_t) * (size_t)max_batch);
        al((void**)&a->d_m, sizeof(int64_t));
    }
    al(&a->hv_ws, (size_t)moq_hypervolume_workspace_size(capacity, K));
    size_t total = 0;
    for (auto& pr : parts) total += slab_align(pr.second);
    const cudaStream_t st = cudaStreamLegacy;
    cudaError_t e = slab_alloc(&a->slab, total, st);
    if (e == cudaSuccess) {
        size_t off = 0;
        for (auto& pr : parts) {
            *pr.first = static_cast<char*>(a->slab) + off;
            off += slab_align(pr.second);
        }
        e = pinned_slot_alloc((void**)&a->h_pinned);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(a->d_count, 0, sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a->d_status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        free_archive(a);
        return cuda_fail(e, "moq_archive_create");
    }
    *out = a;
    return MOQ_OK;
}

void moq_archive_destroy(moq_archive* a) { moq::free_archive(a); }

int moq_archive_reset(moq_archive* a, void* stream)
{
    using namespace moq;
    if (!a) return fail(MOQ_ERR_ARG, "moq_archive_reset: NULL archive");
    MOQ_CUDA_TRY(cudaMemsetAsync(a->d_count, 0, sizeof(int64_t), as_stream(stream)));
    MOQ_CUDA_TRY(cudaMemsetAsync(a->d_status, 0, sizeof(int32_t), as_stream(stream)));
    return MOQ_OK;
}

static int pareto_merge(moq_archive* a, const int64_t* cuts, const uint64_t* bits, int64_t M, int64_t index_base,
                        const int64_t* cand_index, int64_t* front_size_out, void* stream)
{
    using namespace moq;
    if (!a) return fail(MOQ_ERR_ARG, "moq_pareto_front: NULL archive");
    if (M < 0 || M > a->max_batch) return fail(MOQ_ERR_ARG, "moq_pareto_front: M=%lld outside [0, max_batch=%lld]", (long long)M, (long long)a->max_batch);
    if (M > 0 && (!cuts || !bits)) return fail(MOQ_ERR_ARG, "moq_pareto_front: NULL cuts or bits");
    cudaStream_t st = as_stream(stream);
    cudaError_t e;
    switch (a->K) {
    case 2: e = launch_filters<2>(a, cuts, M, st); break;
    case 3: e = launch_filters<3>(a, cuts, M, st); break;
    case 4: e = launch_filters<4>(a, cuts, M, st); break;
    case 5: e = launch_filters<5>(a, cuts, M, st); break;
    case 6: e = launch_filters<6>(a, cuts, M, st); break;
    case 7: e = launch_filters<7>(a, cuts, M, st); break;
    default: e = launch_filters<8>(a, cuts, M, st); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "moq_pareto_front filter launch");
    const int64_t nbA = ceil_div(a->cap, kScanBlock), nbC = ceil_div(M, kScanBlock), nb = nbA + nbC;
    k_count_flags<<<(unsigned)nb, kScanBlock, 0, st>>>(nbA, M, a->d_count, a->flag_arch, a->flag_cand, a->blocksum);
    k_scan_blocksums<<<1, kScanBlock, 0, st>>>(nb, a->blocksum);
    ScatterArgs s{};
    s.K = a->K;
    s.W = a->W;
    s.n = a->n;
    s.cap = a->cap;
    s.nbA = nbA;
    s.M = M;
    s.index_base = index_base;
    s.cand_index = cand_index;
    s.d_count = a->d_count;
    s.flag_arch = a->flag_arch;
    s.flag_cand = a->flag_cand;
    s.blockoff = a->blocksum;
    s.nb = nb;
    s.old_cuts = a->cuts[a->cur];
    s.old_bits = a->bits[a->cur];
    s.old_index = a->index[a->cur];
    s.cand_cuts = cuts;
    s.cand_bits = bits;
    s.new_cuts = a->cuts[1 - a->cur];
    s.new_bits = a->bits[1 - a->cur];
    s.new_index = a->index[1 - a->cur];
    s.status = a->d_status;
    k_scatter<<<(unsigned)nb, kScanBlock, 0, st>>>(s);
    k_set_count<<<1, 1, 0, st>>>(a->cap, nb, a->blocksum, a->d_count);
    MOQ_LAUNCH_CHECK("moq_pareto_front launch");
    a->cur = 1 - a->cur;
    if (front_size_out) return read_status(a, st, front_size_out);
    return MOQ_OK;
}

int moq_pareto_front(moq_archive* a, const int64_t* cuts, const uint64_t* bits, int64_t M, int64_t index_base,
                     int64_t* front_size_out, void* stream)
{
    return pareto_merge(a, cuts, bits, M, index_base, nullptr, front_size_out, stream);
}

int moq_archive_merge(moq_archive* dst, const moq_archive* src, void* stream)
{
    using namespace moq;
    if (!dst || !src || dst == src) return fail(MOQ_ERR_ARG, "moq_archive_merge: NULL archive or dst == src");
    if (dst->K != src->K || dst->n != src->n)
        return fail(MOQ_ERR_ARG, "moq_archive_merge: archives of different n or K (%d, %d vs %d, %d)", dst->n, dst->K, src->n, src->K);
    cudaStream_t st = as_stream(stream);
    int64_t F = 0;
    int rc = read_status(src, st, &F);
    if (rc != MOQ_OK) return rc;
    // src's members are distinct and mutually non-dominated, so they can enter in batches
    for (int64_t off = 0; off < F; off += dst->max_batch) {
        const int64_t m = std::min<int64_t>(dst->max_batch, F - off);
        rc = pareto_merge(dst, src->cuts[src->cur] + off * src->K, src->bits[src->cur] + off * src->W, m, 0, src->index[src->cur] + off,
                          nullptr, stream);
        if (rc != MOQ_OK) return rc;
    }
    return MOQ_OK;
}

int moq_archive_size(const moq_archive* a, int64_t* size_out, void* stream)
{
    using namespace moq;
    if (!a || !size_out) return fail(MOQ_ERR_ARG, "moq_archive_size: NULL argument");
    return read_status(a, as_stream(stream), size_out);
}

int moq_archive_copy_out(const moq_archive* a, int64_t* cuts_host, uint64_t* bits_host, int64_t* index_host, int64_t cap,
                         int64_t* n_out, void* stream)
{
    using namespace moq;
    if (!a || !n_out) return fail(MOQ_ERR_ARG, "moq_archive_copy_out: NULL argument");
    cudaStream_t st = as_stream(stream);
    int64_t F = 0;
    int rc = read_status(a, st, &F);
    if (rc != MOQ_OK) return rc;
    *n_out = F;
    const int64_t m = std::min(F, cap);
    if (m > 0) {
        if (cuts_host) MOQ_CUDA_TRY(cudaMemcpyAsync(cuts_host, a->cuts[a->cur], sizeof(int64_t) * m * a->K, cudaMemcpyDeviceToHost, st));
        if (bits_host) MOQ_CUDA_TRY(cudaMemcpyAsync(bits_host, a->bits[a->cur], sizeof(uint64_t) * m * a->W, cudaMemcpyDeviceToHost, st));
        if (index_host) MOQ_CUDA_TRY(cudaMemcpyAsync(index_host, a->index[a->cur], sizeof(int64_t) * m, cudaMemcpyDeviceToHost, st));
        MOQ_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return MOQ_OK;
}

int moq_archive_device_view(const moq_archive* a, const int64_t** cuts, const uint64_t** bits, const int64_t** index,
                            const int64_t** size_dev)
{
    if (!a) return moq::fail(MOQ_ERR_ARG, "moq_archive_device_view: NULL archive");
    if (cuts) *cuts = a->cuts[a->cur];
    if (bits) *bits = a->bits[a->cur];
    if (index) *index = a->index[a->cur];
    if (size_dev) *size_dev = a->d_count;
    return MOQ_OK;
}

}  // extern "C"
