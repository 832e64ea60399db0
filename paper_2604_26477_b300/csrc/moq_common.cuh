// Internal definitions shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "moqaia.h"

namespace moq {

constexpr int kMaxK = 8;

// ---- error plumbing ----------------------------------------------------------------
// Records a per-thread message and returns `code`, so call sites read
// `return fail(MOQ_ERR_ARG, "...")`.
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t err, const char* what);

#define MOQ_CUDA_TRY(expr)                                 \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return ::moq::cuda_fail(_e, #expr); \
    } while (0)

#define MOQ_LAUNCH_CHECK(what)                             \
    do {                                                   \
        cudaError_t _e = cudaGetLastError();               \
        if (_e != cudaSuccess) return ::moq::cuda_fail(_e, what); \
    } while (0)

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// ---- handle memory (pool.cu) ----------------------------------------------------------
// One device slab per handle and lifetime class from a library-owned memory pool that keeps
// freed memory; slab_alloc is ordered on `st`; slab_free waits for the device first,
// slab_free_async frees in the order of `st` (a slab only `st` used). Pinned
// 64-byte host slots for the read-backs of a handle. Offsets inside a slab are rounded up with slab_align.
size_t slab_align(size_t bytes);
cudaError_t slab_alloc(void** p, size_t bytes, cudaStream_t st);
void slab_free(void* p);
void slab_free_async(void* p, cudaStream_t st);  // once everything queued on st before it is done
cudaError_t pinned_slot_alloc(void** p);
void pinned_slot_free(void* p);
// Pinned read-back buffer of up to 4 KB for the length of one synchronising call (NULL if
// bytes is larger or pinning fails); PinnedLease returns it on scope exit, after waiting for
// the stream it was armed with, so no copy queued into it can outlive the lease.
void* pinned_lease_acquire(size_t bytes);
void pinned_lease_release(void* p);
struct PinnedLease {
    void* p;
    cudaStream_t st = nullptr;
    bool armed = false;
    explicit PinnedLease(size_t bytes, bool want = true) : p(want ? pinned_lease_acquire(bytes) : nullptr) {}
    void arm(cudaStream_t s) { st = s; armed = true; }
    ~PinnedLease()
    {
        if (p && armed) cudaStreamSynchronize(st);
        pinned_lease_release(p);
    }
    PinnedLease(const PinnedLease&) = delete;
    PinnedLease& operator=(const PinnedLease&) = delete;
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Device status bits latched by kernels and read back by synchronising calls.
enum : int32_t {
    kStatusDuplicateEdge = 1,
    kStatusBadEdge = 2,
    kStatusCapacity = 4,
    kStatusOverflow = 8,
};

// ---- counter-based RNG --------------------------------------------------------------
// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): per round the two
// products M0*c0 and M1*c2 are split into high and low halves; the high halves are
// XORed with the other two counter words and the key, the words are permuted, and the
// key advances by the Weyl increments before every round after the first.
struct Philox4x32 {
    static constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
    static constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;

    __device__ __forceinline__ static uint4 block(uint4 c, uint32_t k0, uint32_t k1)
    {
#pragma unroll
        for (int rnd = 0; rnd < 10; ++rnd) {
            // one 32x32 -> 64-bit multiply per product gives both halves
            const uint64_t p0 = (uint64_t)kM0 * c.x;
            const uint64_t p1 = (uint64_t)kM1 * c.z;
            c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
            k0 += kW0;
            k1 += kW1;
        }
        return c;
    }
};

// Uniform in [-1, 1): (word >> 8 - 2^23) * 2^-23, exact in float.
__device__ __forceinline__ float signed_unit(uint32_t word)
{
    return (float)((int32_t)(word >> 8) - 8388608) * 0x1p-23f;
}

__device__ __forceinline__ float sqrt_approx(float v)
{
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Word q (0..3) of a Philox block; a chain of selects, so no local array is needed when
// q is not a compile-time constant.
__device__ __forceinline__ uint32_t word_of(const uint4& o, int q)
{
    return q == 0 ? o.x : (q == 1 ? o.y : (q == 2 ? o.z : o.w));
}

// Two standard normals from one 32-bit word by Box-Muller on its 16-bit halves:
// u1 = (low + 1) 2^-16 in (0, 1], u2 = high 2^-16 in [0, 1), rho = sqrt(-2 ln u1),
// theta = 2 pi u2 -> (rho cos theta, rho sin theta). Each uniform is built exactly from
// the bits of 1 + h 2^-16 (no integer conversion). The angle is evaluated as
// 2 pi (u2 - 1/2) + pi, so the fast sine/cosine see [-pi, pi): one multiply-add on
// f = 1 + u2, f 2 pi - 3 pi. The radius uses ln u1 = ln 2 log2 u1, one multiply by -2 ln 2.
__device__ __forceinline__ float2 box_muller16(uint32_t w)
{
    constexpr float kTwoPi = 6.2831853071795864f, kThreePi = 9.4247779607693797f;
    constexpr float kMinus2Ln2 = -1.3862943611198906f;
    const float u1 = __uint_as_float(0x3F800000u | ((w & 0xFFFFu) << 7)) - (1.0f - 0x1p-16f);
    const float f2 = __uint_as_float(0x3F800000u | ((w >> 9) & 0x7FFF80u));
    const float rho = sqrt_approx(kMinus2Ln2 * __log2f(u1));
    float s, c;
    __sincosf(fmaf(f2, kTwoPi, -kThreePi), &s, &c);
    return make_float2(-rho * c, -rho * s);
}

}  // namespace moq

// ---- handles ---------------------------------------------------------------------------
struct moq_instance {
    int32_t n = 0, K = 0;
    int64_t E = 0;
    int64_t nnz = 0;
    int32_t max_degree = 0;
    int32_t words = 0;
    int device = 0;
    int32_t* ei = nullptr;      // E
    int32_t* ej = nullptr;      // E
    int32_t* w = nullptr;       // K x E (objective-major)
    int32_t* rowptr = nullptr;  // n + 1
    int32_t* col = nullptr;     // nnz, rows sorted by column
    int32_t* wn = nullptr;      // K x nnz weights of the CSR entries (objective-major)
    int64_t* rowsum = nullptr;  // n x K integer row sums sum_j J^(k)_ij
    int32_t* slot_spin = nullptr;  // sampler slot -> spin (gather_layout.cuh)
    int32_t* spin_slot = nullptr;  // spin -> sampler slot
    void* slab = nullptr;          // the one device allocation the arrays above live in
    moq_instance_info info{};
};

struct moq_archive {
    int32_t n = 0, K = 0, W = 0;
    int64_t cap = 0, max_batch = 0;
    int device = 0;
    int cur = 0;                   // which of the double buffers holds the archive
    int64_t* cuts[2] = {nullptr, nullptr};   // cap x K
    uint64_t* bits[2] = {nullptr, nullptr};  // cap x W
    int64_t* index[2] = {nullptr, nullptr};  // cap
    int64_t* d_count = nullptr;    // archive size (device)
    int32_t* d_status = nullptr;   // latched status bits (device)
    int32_t* flag_arch = nullptr;  // cap
    int32_t* flag_cand = nullptr;  // max_batch
    int64_t* blocksum = nullptr;   // scan partials
    unsigned long long* range = nullptr;  // 2 x kMaxK per-objective min / max keys of a merge
    int32_t* table = nullptr;      // large batches: hash table of lowest indices (power of two slots)
    uint32_t table_mask = 0;
    int64_t* ccuts = nullptr;      // large batches: compacted survivors (max_batch x K)
    int32_t* cidx = nullptr;       // their candidate indices
    int32_t* cflag = nullptr;      // their "dominated" flags
    int64_t* d_m = nullptr;        // number of survivors (device)
    int64_t large_min = 0;         // batches from this size take the dedup / survivor path
    int64_t n_blocksum = 0;
    void* hv_ws = nullptr;         // hypervolume workspace sized for cap
    int64_t* h_pinned = nullptr;   // pinned host words for read-backs (one 64-byte slot)
    void* slab = nullptr;          // the one device allocation all arrays above live in
};
