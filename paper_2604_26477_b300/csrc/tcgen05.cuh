// tcgen05 / mbarrier plumbing for the surrogate's tensor-core kernels: shared-memory matrix
// descriptors for 128-byte-swizzled tiles, the BF16 MMA with FP32 accumulation in TMEM, its
// commit to an mbarrier, bounded mbarrier waits and TMEM loads.
//
// Tile layout used throughout: a row-major matrix of `rows` rows is stored as chunk tiles of
// 64 BF16 columns (128 bytes per row), each chunk tile rows x 128 bytes with 16-byte unit u of
// row r at unit u ^ (r & 7) (the 128-byte swizzle; 8-row atoms of 1024 bytes). The same tile is
// a K-major operand when its columns run along K (rows = M or N) and an MN-major operand when
// its rows run along K (columns = M or N).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace moq {
namespace tc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, col) in a swizzled tile of `rows` rows
__device__ __forceinline__ uint32_t tile_offset(int row, int col, int rows)
{
    const int chunk = col >> 6, c = col & 63;
    return (uint32_t)(chunk * rows * 128 + row * 128 + ((((c >> 3) ^ (row & 7)) & 7) << 4) + ((c & 7) << 1));
}

// Shared-memory matrix descriptor, 128-byte swizzle (layout type 2, descriptor version 1):
// start address, leading byte offset (MN-major: the stride between 64-element blocks along
// M or N; unused for K-major) and stride byte offset (the stride between 8-row atoms: 1024).
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D: bits 4-5 D format (1 = F32),
// 7-9 / 10-12 A / B format (1 = BF16), 15 / 16 A / B MN-major, 17-22 N >> 3, 24-28 M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn, bool b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accumulate)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
                 "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
                 : "memory");
}

// every MMA issued by this thread so far arrives on `bar` once complete
__device__ __forceinline__ void commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the phase of the given parity, giving up after `limit_ns`
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns)
{
    const uint32_t a = smem_addr(bar);
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (ok) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape: warp w reads lanes 32w..)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]), "=r"(u[9]),
          "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(u[q]);
}

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor core's (async proxy) reads
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&p);
}

// 16 consecutive columns (col0 a multiple of 16) of row `row` as BF16 into a swizzled tile
__device__ __forceinline__ void store_row16(unsigned char* tile, int rows, int row, int col0, const float (&v)[16])
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint4 u = make_uint4(pack_bf16(v[8 * h], v[8 * h + 1]), pack_bf16(v[8 * h + 2], v[8 * h + 3]),
                                   pack_bf16(v[8 * h + 4], v[8 * h + 5]), pack_bf16(v[8 * h + 6], v[8 * h + 7]));
        *reinterpret_cast<uint4*>(tile + tile_offset(row, col0 + 8 * h, rows)) = u;
    }
}

}  // namespace tc
}  // namespace moq
