// Memory for the library's handles: device slabs from a library-owned CUDA memory pool per
// device and small pinned host slots.
//
// Creating an archive or an instance needs a dozen device arrays and a few bytes of pinned
// host memory for read-backs. With cudaMalloc / cudaMallocHost per array that costs about a
// millisecond per handle (and as much again to free), which dominates short end-to-end runs
// such as a time-to-target measurement. Here a handle takes one slab per lifetime class from
// a memory pool that keeps what is freed (release threshold: unlimited), so after the first
// handle of a size the allocation is a pool lookup; pinned read-back words come from 64-byte
// slots (one per archive) or 4 KB leases (one per synchronising call) carved out of 64 KB
// pinned pages that are kept for the life of the process.
#include <mutex>
#include <vector>

#include "moq_common.cuh"

namespace moq {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[kMaxDevices] = {};

cudaError_t pool_of(int device, cudaMemPool_t* out)
{
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool = nullptr;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = ~0ull;  // never hand freed memory back to the driver
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pools[device] = pool;
    }
    *out = g_pools[device];
    return cudaSuccess;
}

constexpr size_t kSlotBytes = 64, kPageBytes = 64 * 1024, kLeaseBytes = 4096;
std::mutex g_slot_mutex;
std::vector<void*> g_free_slots;
std::mutex g_lease_mutex;
std::vector<void*> g_free_leases;

}  // namespace

size_t slab_align(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

cudaError_t slab_alloc(void** p, size_t bytes, cudaStream_t st)
{
    *p = nullptr;
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    cudaMemPool_t pool = nullptr;
    if (e == cudaSuccess) e = pool_of(device, &pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 256, pool, st);
    if (e != cudaSuccess) *p = nullptr;
    return e;
}

void slab_free(void* p)
{
    if (!p) return;
    // work queued on any stream may still use the slab: wait for the device, then return
    // it to the pool at once
    cudaDeviceSynchronize();
    cudaFreeAsync(p, cudaStreamLegacy);
    cudaStreamSynchronize(cudaStreamLegacy);
}

void slab_free_async(void* p, cudaStream_t st)
{
    if (p) cudaFreeAsync(p, st);
}

cudaError_t pinned_slot_alloc(void** p)
{
    std::lock_guard<std::mutex> lock(g_slot_mutex);
    if (g_free_slots.empty()) {
        void* page = nullptr;
        cudaError_t e = cudaMallocHost(&page, kPageBytes);
        if (e != cudaSuccess) return e;
        for (size_t off = kPageBytes; off > 0; off -= kSlotBytes) g_free_slots.push_back(static_cast<char*>(page) + off - kSlotBytes);
    }
    *p = g_free_slots.back();
    g_free_slots.pop_back();
    return cudaSuccess;
}

void pinned_slot_free(void* p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_slot_mutex);
    g_free_slots.push_back(p);
}

void* pinned_lease_acquire(size_t bytes)
{
    // buffers of kLeaseBytes carved from pinned pages that are kept for the life of the
    // process, shared by all host threads: a thread's first read-back costs no page-locked
    // allocation (each cudaMallocHost takes about a millisecond, serialised across threads)
    // and a thread that exits leaves nothing behind
    if (bytes > kLeaseBytes) return nullptr;
    std::lock_guard<std::mutex> lock(g_lease_mutex);
    if (g_free_leases.empty()) {
        void* page = nullptr;
        if (cudaMallocHost(&page, kPageBytes) != cudaSuccess) return nullptr;
        for (size_t off = kPageBytes; off > 0; off -= kLeaseBytes) g_free_leases.push_back(static_cast<char*>(page) + off - kLeaseBytes);
    }
    void* p = g_free_leases.back();
    g_free_leases.pop_back();
    return p;
}

void pinned_lease_release(void* p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_lease_mutex);
    g_free_leases.push_back(p);
}

}  // namespace moq

extern "C" int moq_release_cached_memory(void)
{
    using namespace moq;
    int device = 0;
    MOQ_CUDA_TRY(cudaGetDevice(&device));
    if (device < 0 || device >= kMaxDevices) return MOQ_OK;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_pool_mutex);
        pool = g_pools[device];
    }
    if (!pool) return MOQ_OK;
    MOQ_CUDA_TRY(cudaDeviceSynchronize());
    MOQ_CUDA_TRY(cudaMemPoolTrimTo(pool, 0));
    return MOQ_OK;
}
