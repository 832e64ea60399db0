// The surrogate MLP of the learned proposal (not in the paper) on the 5th-generation tensor
// cores: every matrix product of the forward pass and of backpropagation is a tcgen05.mma with
// BF16 operands from shared memory and an FP32 accumulator in TMEM.
//
//   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3,  L = 1/(B D_out) sum (y - t)^2
//
// One CTA of 128 threads takes a tile of 128 rows (thread r owns row r and TMEM lane r). The
// BF16 weights sit in shared memory once per CTA; each activation is written once, as BF16,
// into a row-major 128-byte-swizzled tile, which serves as a K-major operand for the next
// layer's product and as an MN-major operand for the weight gradient (no transposed copies):
//   L1  a1  = X W1^T                 (M 128 rows, N 128, K 16)
//   L2  a2  = H1 W2^T                (M 128, N 128, K 128)
//   L3  y   = H2 W3^T                (M 128, N 16,  K 128)
//   B1  d2' = DY W3                  (M 128, N 2 x 64, K 16)   dW3^T = H2^T DY  (M 128, N 64, K 128 rows)
//   B2  d1' = D2 W2                  (M 128, N 2 x 64, K 128)  dW2   = D2^T H1  (M 128, N 2 x 64, K 128 rows)
//   B3  dW1 = D1^T X                 (M 128, N 64, K 128 rows)
// with the epilogues in between: bias + relu into H1, H2; dy = 2 (y - t) / (B D_out) into DY;
// d2 = d2' [a2 > 0] into D2; d1 = d1' [a1 > 0] into D1. Operands are rounded to BF16 once, when
// they are written; sums, relu masks, the loss and the bias gradients (column sums of dy, d2,
// d1, deterministic butterfly reductions) stay in FP32. Each CTA writes its gradient to its own
// slot; the caller sums the slots in CTA order (deterministic).
//
// TMEM columns: a1 0-127 (kept for the relu mask of d1), a2 128-255 (then d1'), d2' 256-383
// (then dW2), y 384-399 (then dW3^T 384-447), dW1 448-511.
// Every mbarrier wait is bounded (2 s); on time-out the kernel latches a status bit and stops
// issuing, waits (bounded) for what it issued, frees TMEM and returns.
#include <cuda_bf16.h>

#include "mlp_tc.cuh"
#include "moq_common.cuh"
#include "tcgen05.cuh"

namespace moq {

namespace {

using namespace tc;

constexpr int kRowsT = kMlpTcRows, kThreadsT = 128, kHid = 128;
constexpr uint64_t kWaitLimit = 2000000000ull;
// shared-memory regions (bytes from a 1024-aligned base)
constexpr uint32_t kOffW1 = 0;                       // 128 x 64 (din <= 16 used)
constexpr uint32_t kOffW2 = kOffW1 + 16384;          // 128 x 128
constexpr uint32_t kOffW3 = kOffW2 + 32768;          // 16 x 128 (dout <= 8 used)
constexpr uint32_t kOffX = kOffW3 + 4096;            // 128 x 64
constexpr uint32_t kOffH1 = kOffX + 16384;           // 128 x 128, then D1
constexpr uint32_t kOffH2 = kOffH1 + 32768;          // 128 x 128, then D2
constexpr uint32_t kOffDY = kOffH2 + 32768;          // 128 x 64
constexpr uint32_t kOffMisc = kOffDY + 16384;
constexpr uint32_t kMiscBytes = 4 * (4 * kHid + 2 * 16) + 4 * 4 * kHid + 64;  // biases, bias grads, reductions, barrier
constexpr size_t kSmemTc = 1024 + kOffMisc + kMiscBytes;
constexpr uint32_t kTileA = 16384;                   // one 64-column chunk of a 128-row tile

constexpr uint32_t kIdL = idesc_bf16(128, 128, false, false);
constexpr uint32_t kIdL3 = idesc_bf16(128, 16, false, false);
constexpr uint32_t kIdB64 = idesc_bf16(128, 64, false, true);   // K-major A, MN-major B, N = 64
constexpr uint32_t kIdW64 = idesc_bf16(128, 64, true, true);    // both MN-major (weight gradients)

// K-major operand: 8-row atoms 1024 B apart (the leading offset is not used)
__device__ __forceinline__ uint64_t kmaj(uint32_t a) { return desc_sw128(a, 16, 1024); }
// MN-major operand of 64 columns (one chunk) and of 128 columns (two chunks 16 KB apart)
__device__ __forceinline__ uint64_t mn64(uint32_t a) { return desc_sw128(a, 1024, 1024); }
__device__ __forceinline__ uint64_t mn128(uint32_t a) { return desc_sw128(a, kTileA, 1024); }

// Column sums over the 128 rows of 16 values per thread (v is consumed): a butterfly within
// each warp (fixed pattern), then the four warps' partials in order. out[col0 + q] receives
// the sum of column q; red holds 4 x 128 floats.
__device__ __forceinline__ void column_sums16(float (&v)[16], float* red, int col0, float* out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int half = 8 >> s, off = 16 >> s;
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int q = 0; q < half; ++q) {
            const float send = upper ? v[q] : v[q + half];
            const float keep = upper ? v[q + half] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    const int col = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
    if ((lane & 1) == 0) red[warp * kHid + col0 + col] = v[0];
    __syncthreads();
    if (threadIdx.x < 16) {
        const int c = col0 + threadIdx.x;
        out[c] = ((red[c] + red[kHid + c]) + red[2 * kHid + c]) + red[3 * kHid + c];
    }
    __syncthreads();
}

template <bool TRAIN>
__global__ void __launch_bounds__(kThreadsT, 1) k_mlp_tc(const MlpTcArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    const uint32_t sb = smem_addr(base);
    float* b1 = reinterpret_cast<float*>(base + kOffMisc);
    float* b2 = b1 + kHid;
    float* b3 = b2 + kHid;             // 16
    float* db1 = b3 + 16;              // 128
    float* db2 = db1 + kHid;           // 128
    float* db3 = db2 + kHid;           // 16
    float* red = db3 + 16;             // 4 x 128
    uint64_t* bar = reinterpret_cast<uint64_t*>(red + 4 * kHid);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
    float* lred = reinterpret_cast<float*>(tmem_slot + 1);  // 4

    const int tid = threadIdx.x, warp = tid >> 5;
    const int din = a.din, dout = a.dout;
    const int64_t row0 = (int64_t)blockIdx.x * kRowsT;
    const int nr = (int)min((int64_t)kRowsT, a.B - row0);
    const bool live = tid < nr;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // weights into their tiles: W2 (16-byte units straight from the flat BF16 vector), W1 and
    // W3 zero-padded to 16 columns / rows, biases as FP32
    {
        // every global load of the thread is issued before its first shared-memory store
        const uint4* w4 = reinterpret_cast<const uint4*>(a.w + a.oW2);
        constexpr int kW2Units = kHid * kHid / 8 / kThreadsT;  // 16
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        uint4 u2[kW2Units], u3[2];
#pragma unroll
        for (int t = 0; t < kW2Units; ++t) u2[t] = __ldg(w4 + tid + t * kThreadsT);
#pragma unroll
        for (int t = 0; t < 2; ++t) {  // W3: 16 rows x 16 units
            const int u = tid + t * kThreadsT, k = u >> 4, i0 = (u & 15) * 8;
            u3[t] = k < dout ? __ldg(reinterpret_cast<const uint4*>(a.w + a.oW3 + (int64_t)k * kHid + i0)) : z;
        }
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = i < din ? __bfloat162float(a.w[a.oW1 + (int64_t)tid * din + i]) : 0.0f;
#pragma unroll
        for (int t = 0; t < kW2Units; ++t) {
            const int u = tid + t * kThreadsT, j = u >> 4, i0 = (u & 15) * 8;
            *reinterpret_cast<uint4*>(base + kOffW2 + tile_offset(j, i0, 128)) = u2[t];
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int u = tid + t * kThreadsT, k = u >> 4, i0 = (u & 15) * 8;
            *reinterpret_cast<uint4*>(base + kOffW3 + tile_offset(k, i0, 16)) = u3[t];
        }
        store_row16(base + kOffW1, 128, tid, 0, v);  // row j = tid
        for (int c = 16; c < 64; c += 8) {  // W1, X and DY columns 16..63 stay zero
            *reinterpret_cast<uint4*>(base + kOffW1 + tile_offset(tid, c, 128)) = z;
            *reinterpret_cast<uint4*>(base + kOffX + tile_offset(tid, c, 128)) = z;
            if (TRAIN) *reinterpret_cast<uint4*>(base + kOffDY + tile_offset(tid, c, 128)) = z;
        }
        b1[tid] = __bfloat162float(a.w[a.ob1 + tid]);
        b2[tid] = __bfloat162float(a.w[a.ob2 + tid]);
        if (tid < 16) b3[tid] = tid < dout ? __bfloat162float(a.w[a.ob3 + tid]) : 0.0f;
        // the tile's inputs, rounded to BF16 (rows past the batch are zero)
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = (live && i < din) ? a.X[(row0 + tid) * din + i] : 0.0f;
        store_row16(base + kOffX, 128, tid, 0, v);
    }
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    bool ok = true;
    uint32_t phase = 0;
    int issued = 0;  // MMA groups committed

    // thread 0 issues a group of products and commits it; everyone waits for it
    auto run = [&](auto&& issue) {
        if (tid == 0 && ok) {
            fence_after_sync();
            issue();
            commit(bar);
        }
        if (ok) ++issued;
        const bool got = ok ? mbar_wait(bar, phase & 1u, kWaitLimit) : false;
        ++phase;
        ok = __syncthreads_and(got ? 1 : 0) != 0;
        fence_after_sync();
    };
    // this thread's epilogue writes are done: make them visible to the next products
    auto publish = [&]() {
        fence_proxy_async();
        fence_before_sync();
        __syncthreads();
    };

    // L1: a1 = X W1^T
    run([&] { mma_bf16(tmem + 0, kmaj(sb + kOffX), kmaj(sb + kOffW1), kIdL, 0u); });
    float v[16];
    if (ok) {
#pragma unroll 1
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            tmem_ld16(lane_base + 0 + c0, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = fmaxf(v[q] + b1[c0 + q], 0.0f);
            store_row16(base + kOffH1, 128, tid, c0, v);
        }
    }
    publish();
    // L2: a2 = H1 W2^T
    run([&] {
#pragma unroll
        for (int ks = 0; ks < 8; ++ks) {
            const uint32_t o = (ks >> 2) * kTileA + (ks & 3) * 32;
            mma_bf16(tmem + 128, kmaj(sb + kOffH1 + o), kmaj(sb + kOffW2 + o), kIdL, ks > 0 ? 1u : 0u);
        }
    });
    if (ok) {
#pragma unroll 1
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            tmem_ld16(lane_base + 128 + c0, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = fmaxf(v[q] + b2[c0 + q], 0.0f);
            store_row16(base + kOffH2, 128, tid, c0, v);
        }
    }
    publish();
    // L3: y = H2 W3^T
    run([&] {
#pragma unroll
        for (int ks = 0; ks < 8; ++ks)
            mma_bf16(tmem + 384, kmaj(sb + kOffH2 + (ks >> 2) * kTileA + (ks & 3) * 32),
                     kmaj(sb + kOffW3 + (ks >> 2) * 2048 + (ks & 3) * 32), kIdL3, ks > 0 ? 1u : 0u);
    });
    float tgt[8] = {};  // this row's targets, loaded while the forward products run
    if (TRAIN && live) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < dout) tgt[k] = a.T[(row0 + tid) * dout + k];
    }
    float y[16] = {};
    if (ok) tmem_ld16(lane_base + 384, y);
#pragma unroll
    for (int k = 0; k < 16; ++k) y[k] += b3[k];
    if (!TRAIN) {
        if (ok && live)
            for (int k = 0; k < dout; ++k) a.Y[(row0 + tid) * dout + k] = y[k];
    } else {
        // dy = 2 (y - t) / (B D_out); rows past the batch contribute nothing
        const float scale = 1.0f / ((float)a.B * (float)dout);
        float lsum = 0.0f;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float e = 0.0f;
            if (live && k < dout) e = y[k] - tgt[k & 7];
            lsum += e * e * scale;
            y[k] = 2.0f * e * scale;  // dy
        }
        store_row16(base + kOffDY, 128, tid, 0, y);
        // loss: butterfly within the warp, then the warps in order
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
        if ((tid & 31) == 0) lred[warp] = lsum;
        publish();
        column_sums16(y, red, 0, db3);
        // B1: d2' = DY W3 (N in two halves), dW3^T = H2^T DY
        run([&] {
            for (int h = 0; h < 2; ++h)
                mma_bf16(tmem + 256 + 64 * h, kmaj(sb + kOffDY), mn64(sb + kOffW3 + h * 2048), kIdB64, 0u);
#pragma unroll
            for (int ks = 0; ks < 8; ++ks)
                mma_bf16(tmem + 384, mn128(sb + kOffH2 + ks * 2048), mn64(sb + kOffDY + ks * 2048), kIdW64, ks > 0 ? 1u : 0u);
        });
        // d2 = d2' [a2 > 0] into D2 (over H2, read by now); db2
        if (ok) {
#pragma unroll 1
            for (int c0 = 0; c0 < kHid; c0 += 16) {
                float m[16];
                tmem_ld16(lane_base + 128 + c0, m);
                tmem_ld16(lane_base + 256 + c0, v);
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = (m[q] + b2[c0 + q] > 0.0f) ? v[q] : 0.0f;
                store_row16(base + kOffH2, 128, tid, c0, v);
                column_sums16(v, red, c0, db2);
            }
        }
        publish();
        // B2: d1' = D2 W2 (N in two halves), dW2 = D2^T H1 (N in two halves)
        run([&] {
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int ks = 0; ks < 8; ++ks)
                    mma_bf16(tmem + 128 + 64 * h, kmaj(sb + kOffH2 + (ks >> 2) * kTileA + (ks & 3) * 32),
                             mn64(sb + kOffW2 + h * kTileA + ks * 2048), kIdB64, ks > 0 ? 1u : 0u);
#pragma unroll
                for (int ks = 0; ks < 8; ++ks)
                    mma_bf16(tmem + 256 + 64 * h, mn128(sb + kOffH2 + ks * 2048), mn64(sb + kOffH1 + h * kTileA + ks * 2048),
                             kIdW64, ks > 0 ? 1u : 0u);
            }
        });
        // d1 = d1' [a1 > 0] into D1 (over H1, read by now); db1
        if (ok) {
#pragma unroll 1
            for (int c0 = 0; c0 < kHid; c0 += 16) {
                float m[16];
                tmem_ld16(lane_base + 0 + c0, m);
                tmem_ld16(lane_base + 128 + c0, v);
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = (m[q] + b1[c0 + q] > 0.0f) ? v[q] : 0.0f;
                store_row16(base + kOffH1, 128, tid, c0, v);
                column_sums16(v, red, c0, db1);
            }
        }
        publish();
        // B3: dW1 = D1^T X
        run([&] {
#pragma unroll
            for (int ks = 0; ks < 8; ++ks)
                mma_bf16(tmem + 448, mn128(sb + kOffH1 + ks * 2048), mn64(sb + kOffX + ks * 2048), kIdW64, ks > 0 ? 1u : 0u);
        });
        // the CTA's gradient slot: the rows of dW2 and dW1 (one per thread in TMEM) pass through
        // shared memory (X, H1 and H2 are free now) so that the global stores are coalesced
        if (ok) {
            float* g = a.partial + (int64_t)blockIdx.x * a.P;
            float* stage = reinterpret_cast<float*>(base + kOffX);
            constexpr int kLdS = kHid + 4;  // 16-byte rows, 4-bank skew
#pragma unroll 1
            for (int c0 = 0; c0 < kHid; c0 += 16) {  // dW2[j][i], j = tid
                tmem_ld16(lane_base + 256 + c0, v);
#pragma unroll
                for (int q = 0; q < 16; q += 4)
                    *reinterpret_cast<float4*>(stage + tid * kLdS + c0 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
            }
            float w1g[16];
            tmem_ld16(lane_base + 448, w1g);  // dW1[j][i], j = tid
            tmem_ld16(lane_base + 384, v);    // dW3[k][i] = (dW3^T)[i][k], i = tid: coalesced as is
            for (int k = 0; k < dout; ++k) g[a.oW3 + (int64_t)k * kHid + tid] = v[k];
            __syncthreads();
#pragma unroll 4
            for (int q = tid; q < kHid * kHid; q += kThreadsT) g[a.oW2 + q] = stage[(q >> 7) * kLdS + (q & 127)];
            __syncthreads();
            for (int i = 0; i < din; ++i) stage[tid * 17 + i] = w1g[i];  // odd stride: conflict-free
            __syncthreads();
            for (int q = tid; q < kHid * din; q += kThreadsT) g[a.oW1 + q] = stage[(q / din) * 17 + q % din];
            g[a.ob1 + tid] = db1[tid];
            g[a.ob2 + tid] = db2[tid];
            if (tid < dout) g[a.ob3 + tid] = db3[tid];
            if (tid == 0) a.loss_part[blockIdx.x] = ((lred[0] + lred[1]) + lred[2]) + lred[3];
        }
    }
    if (!ok && tid == 0) {
        atomicOr(a.status, 1);
        // nothing may still write TMEM when it is freed: groups complete in order, so the last
        // committed one arriving (bounded wait) covers them all
        if (issued > 0) (void)mbar_wait(bar, (uint32_t)(issued - 1) & 1u, kWaitLimit);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

}  // namespace

// grid: one CTA per 128-row tile
cudaError_t launch_mlp_tc(const MlpTcArgs& a, bool train, cudaStream_t st)
{
    if (a.B <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)ceil_div(a.B, kRowsT);
    cudaError_t e;
    if (train) {
        e = cudaFuncSetAttribute(k_mlp_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTc);
        if (e != cudaSuccess) return e;
        k_mlp_tc<true><<<grid, kThreadsT, kSmemTc, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_mlp_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTc);
        if (e != cudaSuccess) return e;
        k_mlp_tc<false><<<grid, kThreadsT, kSmemTc, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace moq
