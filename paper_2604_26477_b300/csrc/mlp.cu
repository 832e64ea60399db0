// Learned weight-vector proposal (not in the paper): a small surrogate MLP maps a weight
// vector plus graph statistics to the expected normalised cut vector of an SB sample,
// is trained on the (lambda, cut) pairs the sampler produces, and proposes the candidate
// weight vectors whose predicted cuts lie furthest beyond the current front.
//
//   h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3      (H = 128 hidden units)
//   L  = 1 / (B D_out) sum (y - t)^2
// Parameters: one flat FP32 master vector (W1, b1, W2, b2, W3, b3, row-major) for the
// optimiser and its BF16 copy, which is what every kernel computes with (accumulation in
// FP32). The fused training kernel takes a tile of 32 rows per block, keeps the weights
// (converted from BF16) and the tile's activations in shared memory (rows padded by one
// word against bank conflicts), runs the forward pass and backpropagation, and writes the
// block's gradient to its own slot; a second kernel sums the slots in a fixed order, so the
// gradient is deterministic.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <stdlib.h>
#include <vector>

#include "mlp_tc.cuh"
#include "moq_common.cuh"

namespace moq {
namespace {

constexpr int kH = 128;       // hidden width
constexpr int kMaxIn = 16;    // D_in <= 16
constexpr int kMaxOut = 8;    // D_out <= 8
constexpr int kRows = 32;     // rows per block
constexpr int kThreads = 256;
constexpr int kLd = kH + 4;   // padded row stride of H-wide smem matrices (16-byte rows, 4-bank skew)

struct MlpShape {
    int din, dout;
    int64_t oW1, ob1, oW2, ob2, oW3, ob3, P;
};

__host__ __device__ inline MlpShape mlp_shape(int din, int dout)
{
    MlpShape s;
    s.din = din;
    s.dout = dout;
    s.oW1 = 0;
    s.ob1 = s.oW1 + (int64_t)kH * din;
    s.oW2 = s.ob1 + kH;
    s.ob2 = s.oW2 + (int64_t)kH * kH;
    s.oW3 = s.ob2 + kH;
    s.ob3 = s.oW3 + (int64_t)dout * kH;
    s.P = s.ob3 + dout;
    return s;
}

// shared-memory layout (floats) of the fused kernels
struct MlpSmem {
    float* W1;  // kH x (kMaxIn + 1)
    float* b1;
    float* W2;  // kH x kLd
    float* b2;
    float* W3;  // kMaxOut x kLd
    float* b3;
    float* x;   // kRows x (kMaxIn + 1)
    float* a1;  // kRows x kLd (activation 1, relu applied)
    float* a2;  // kRows x kLd (activation 2, relu applied)
    float* d1;  // kRows x kLd
    float* d2;  // kRows x kLd
    float* dy;  // kRows x kMaxOut
};

__host__ __device__ inline size_t mlp_smem_floats()
{
    return (size_t)kH * (kMaxIn + 1) + kH + (size_t)kH * kLd + kH + (size_t)kMaxOut * kLd + kMaxOut + (size_t)kRows * (kMaxIn + 1) +
           4 * (size_t)kRows * kLd + (size_t)kRows * kMaxOut;
}

__device__ MlpSmem carve_mlp(float* s)
{
    MlpSmem m;
    m.W1 = s; s += kH * (kMaxIn + 1);
    m.b1 = s; s += kH;
    m.W2 = s; s += kH * kLd;
    m.b2 = s; s += kH;
    m.W3 = s; s += kMaxOut * kLd;
    m.b3 = s; s += kMaxOut;
    m.x = s; s += kRows * (kMaxIn + 1);
    m.a1 = s; s += kRows * kLd;
    m.a2 = s; s += kRows * kLd;
    m.d1 = s; s += kRows * kLd;
    m.d2 = s; s += kRows * kLd;
    m.dy = s;
    return m;
}

// BF16 weights -> FP32 shared memory, eight values per 16-byte load (every block of the
// flat vector starts on a 16-byte boundary: its offsets are multiples of 128 elements),
// all loads of a thread issued before the first store
__device__ __forceinline__ void unpack8(const uint4& u, float (&v)[8])
{
    const uint32_t wd[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        v[2 * e] = __uint_as_float(wd[e] << 16);
        v[2 * e + 1] = __uint_as_float(wd[e] & 0xFFFF0000u);
    }
}

__device__ void load_weights(const __nv_bfloat16* __restrict__ w, const MlpShape& sh, MlpSmem& m)
{
    const uint4* w4 = reinterpret_cast<const uint4*>(w);
    constexpr int kW2Vec = kH * kH / 8;
    uint4 u2[kW2Vec / kThreads];
#pragma unroll
    for (int t = 0; t < kW2Vec / kThreads; ++t) u2[t] = __ldg(w4 + (sh.oW2 >> 3) + threadIdx.x + t * kThreads);
    const int n1 = kH * sh.din / 8, n3 = sh.dout * kH / 8;  // <= 256, <= 128 vectors
    uint4 u1 = make_uint4(0, 0, 0, 0), u3 = u1, ub = u1;
    if ((int)threadIdx.x < n1) u1 = __ldg(w4 + (sh.oW1 >> 3) + threadIdx.x);
    if ((int)threadIdx.x < n3) u3 = __ldg(w4 + (sh.oW3 >> 3) + threadIdx.x);
    if (threadIdx.x < 32) ub = __ldg(w4 + ((threadIdx.x < 16 ? sh.ob1 : sh.ob2 - 128) >> 3) + threadIdx.x);
#pragma unroll
    for (int t = 0; t < kW2Vec / kThreads; ++t) {
        const int q = (threadIdx.x + t * kThreads) * 8;
        float v[8];
        unpack8(u2[t], v);
#pragma unroll
        for (int e = 0; e < 8; ++e) m.W2[(q >> 7) * kLd + (q & 127) + e] = v[e];
    }
    float v[8];
    if ((int)threadIdx.x < n1) {
        unpack8(u1, v);
        for (int e = 0; e < 8; ++e) {
            const int q = threadIdx.x * 8 + e;
            m.W1[(q / sh.din) * (kMaxIn + 1) + q % sh.din] = v[e];
        }
    }
    if ((int)threadIdx.x < n3) {
        unpack8(u3, v);
        for (int e = 0; e < 8; ++e) {
            const int q = threadIdx.x * 8 + e;
            m.W3[(q >> 7) * kLd + (q & 127)] = v[e];
        }
    }
    if (threadIdx.x < 32) {
        unpack8(ub, v);
        float* dst = threadIdx.x < 16 ? m.b1 + threadIdx.x * 8 : m.b2 + (threadIdx.x - 16) * 8;
        for (int e = 0; e < 8; ++e) dst[e] = v[e];
    }
    for (int q = threadIdx.x; q < sh.dout; q += blockDim.x) m.b3[q] = __bfloat162float(w[sh.ob3 + q]);
}

// Thread tiles of the H-wide products: warp w, lane l own rows w + 8a and columns l + 32b
// (a, b = 0..3), so every step of a dot product loads 4 + 4 values for 16 FMAs (the weight
// loads run along a padded row: conflict-free; the activation loads are warp broadcasts).
// Each output keeps its own FMA chain in index order, so the sums are those of the plain loops.
constexpr int kTileRows = kRows / 8;
constexpr int kTileCols = kH / 32;

// forward pass of the rows [row0, row0 + nr) into m.a1, m.a2 (activations after relu) and y (out)
__device__ void forward_tile(const MlpShape& sh, MlpSmem& m, const float* __restrict__ X, int64_t row0, int nr, float* Yout,
                             float* ysm)
{
    for (int q = threadIdx.x; q < kRows * sh.din; q += blockDim.x) {
        const int r = q / sh.din, i = q % sh.din;
        m.x[r * (kMaxIn + 1) + i] = r < nr ? X[(row0 + r) * sh.din + i] : 0.0f;
    }
    __syncthreads();
    const int w8 = threadIdx.x >> 5, l = threadIdx.x & 31;
    {  // layer 1
        float acc[kTileRows][kTileCols];
#pragma unroll
        for (int a = 0; a < kTileRows; ++a)
#pragma unroll
            for (int b = 0; b < kTileCols; ++b) acc[a][b] = m.b1[l + 32 * b];
        for (int i = 0; i < sh.din; ++i) {
            float wv[kTileCols], xv[kTileRows];
#pragma unroll
            for (int b = 0; b < kTileCols; ++b) wv[b] = m.W1[(l + 32 * b) * (kMaxIn + 1) + i];
#pragma unroll
            for (int a = 0; a < kTileRows; ++a) xv[a] = m.x[(w8 + 8 * a) * (kMaxIn + 1) + i];
#pragma unroll
            for (int a = 0; a < kTileRows; ++a)
#pragma unroll
                for (int b = 0; b < kTileCols; ++b) acc[a][b] = fmaf(wv[b], xv[a], acc[a][b]);
        }
#pragma unroll
        for (int a = 0; a < kTileRows; ++a)
#pragma unroll
            for (int b = 0; b < kTileCols; ++b) m.a1[(w8 + 8 * a) * kLd + l + 32 * b] = fmaxf(acc[a][b], 0.0f);
    }
    __syncthreads();
    {  // layer 2
        float acc[kTileRows][kTileCols];
#pragma unroll
        for (int a = 0; a < kTileRows; ++a)
#pragma unroll
            for (int b = 0; b < kTileCols; ++b) acc[a][b] = m.b2[l + 32 * b];
#pragma unroll 2
        for (int i = 0; i < kH; i += 4) {  // four steps per 16-byte load
            float4 wv[kTileCols], hv[kTileRows];
#pragma unroll
            for (int b = 0; b < kTileCols; ++b) wv[b] = *reinterpret_cast<const float4*>(m.W2 + (l + 32 * b) * kLd + i);
#pragma unroll
            for (int a = 0; a < kTileRows; ++a) hv[a] = *reinterpret_cast<const float4*>(m.a1 + (w8 + 8 * a) * kLd + i);
#pragma unroll
            for (int a = 0; a < kTileRows; ++a)
#pragma unroll
                for (int b = 0; b < kTileCols; ++b) {
                    acc[a][b] = fmaf(wv[b].x, hv[a].x, acc[a][b]);
                    acc[a][b] = fmaf(wv[b].y, hv[a].y, acc[a][b]);
                    acc[a][b] = fmaf(wv[b].z, hv[a].z, acc[a][b]);
                    acc[a][b] = fmaf(wv[b].w, hv[a].w, acc[a][b]);
                }
        }
#pragma unroll
        for (int a = 0; a < kTileRows; ++a)
#pragma unroll
            for (int b = 0; b < kTileCols; ++b) m.a2[(w8 + 8 * a) * kLd + l + 32 * b] = fmaxf(acc[a][b], 0.0f);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kRows * sh.dout; q += blockDim.x) {  // layer 3
        const int r = q / sh.dout, k = q % sh.dout;
        float s = m.b3[k];
        const float* w = m.W3 + k * kLd;
        const float* a = m.a2 + r * kLd;
        for (int i = 0; i < kH; ++i) s = fmaf(w[i], a[i], s);
        if (ysm) ysm[r * kMaxOut + k] = s;
        if (Yout && r < nr) Yout[(row0 + r) * sh.dout + k] = s;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_mlp_forward(const __nv_bfloat16* __restrict__ w, int din, int dout, const float* __restrict__ X,
                                                          int64_t B, float* Y)
{
    extern __shared__ float smem_f[];
    const MlpShape sh = mlp_shape(din, dout);
    MlpSmem m = carve_mlp(smem_f);
    load_weights(w, sh, m);
    __syncthreads();
    for (int64_t row0 = (int64_t)blockIdx.x * kRows; row0 < B; row0 += (int64_t)gridDim.x * kRows)
        forward_tile(sh, m, X, row0, (int)std::min<int64_t>(kRows, B - row0), Y, nullptr);
}

// Forward + backward of one tile per block; partial[block][P] gets the block's gradient,
// loss_part[block] its share of the loss.
__global__ void __launch_bounds__(kThreads) k_mlp_grad(const __nv_bfloat16* __restrict__ w, int din, int dout, const float* __restrict__ X,
                                                       const float* __restrict__ T, int64_t B, float* partial, float* loss_part)
{
    extern __shared__ float smem_f[];
    __shared__ float red[kThreads];
    const MlpShape sh = mlp_shape(din, dout);
    MlpSmem m = carve_mlp(smem_f);
    load_weights(w, sh, m);
    __syncthreads();
    const int64_t row0 = (int64_t)blockIdx.x * kRows;
    const int nr = (int)std::min<int64_t>(kRows, B - row0);
    forward_tile(sh, m, X, row0, nr, nullptr, m.dy);
    // dy = 2 (y - t) / (B D_out); rows beyond the batch contribute nothing
    const float scale = 1.0f / ((float)B * dout);
    float lsum = 0.0f;
    for (int q = threadIdx.x; q < kRows * dout; q += blockDim.x) {
        const int r = q / dout, k = q % dout;
        float e = 0.0f;
        if (r < nr) e = m.dy[r * kMaxOut + k] - T[(row0 + r) * dout + k];
        lsum += e * e * scale;
        m.dy[r * kMaxOut + k] = 2.0f * e * scale;
    }
    red[threadIdx.x] = lsum;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
    const int w8 = threadIdx.x >> 5, l = threadIdx.x & 31;
    // d2 = (W3^T dy) * [a2 > 0]
    for (int q = threadIdx.x; q < kRows * kH; q += blockDim.x) {
        const int r = q / kH, i = q % kH;
        float s = 0.0f;
        for (int k = 0; k < dout; ++k) s = fmaf(m.W3[k * kLd + i], m.dy[r * kMaxOut + k], s);
        m.d2[r * kLd + i] = m.a2[r * kLd + i] > 0.0f ? s : 0.0f;
    }
    __syncthreads();
    {  // d1 = (W2^T d2) * [a1 > 0]: rows w + 8a, columns 4l..4l+3 (one 16-byte load of a W2 row)
        float acc[kTileRows][4];
#pragma unroll
        for (int a = 0; a < kTileRows; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = 0.0f;
#pragma unroll 2
        for (int j = 0; j < kH; j += 4) {
            float4 dv[kTileRows];
#pragma unroll
            for (int a = 0; a < kTileRows; ++a) dv[a] = *reinterpret_cast<const float4*>(m.d2 + (w8 + 8 * a) * kLd + j);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const float4 wv = *reinterpret_cast<const float4*>(m.W2 + (j + jj) * kLd + 4 * l);
#pragma unroll
                for (int a = 0; a < kTileRows; ++a) {
                    const float d = jj == 0 ? dv[a].x : (jj == 1 ? dv[a].y : (jj == 2 ? dv[a].z : dv[a].w));
                    acc[a][0] = fmaf(wv.x, d, acc[a][0]);
                    acc[a][1] = fmaf(wv.y, d, acc[a][1]);
                    acc[a][2] = fmaf(wv.z, d, acc[a][2]);
                    acc[a][3] = fmaf(wv.w, d, acc[a][3]);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < kTileRows; ++a) {
            const int at = (w8 + 8 * a) * kLd + 4 * l;
            const float4 h = *reinterpret_cast<const float4*>(m.a1 + at);
            *reinterpret_cast<float4*>(m.d1 + at) =
                make_float4(h.x > 0.0f ? acc[a][0] : 0.0f, h.y > 0.0f ? acc[a][1] : 0.0f, h.z > 0.0f ? acc[a][2] : 0.0f,
                            h.w > 0.0f ? acc[a][3] : 0.0f);
        }
    }
    __syncthreads();
    float* g = partial + (int64_t)blockIdx.x * sh.P;
    // layer 3: dW3[k][i] = sum_r dy[r][k] h2[r][i]; db3
    for (int q = threadIdx.x; q < dout * kH; q += blockDim.x) {
        const int k = q / kH, i = q % kH;
        float s = 0.0f;
        for (int r = 0; r < kRows; ++r) s = fmaf(m.dy[r * kMaxOut + k], m.a2[r * kLd + i], s);
        g[sh.oW3 + q] = s;
    }
    for (int k = threadIdx.x; k < dout; k += blockDim.x) {
        float s = 0.0f;
        for (int r = 0; r < kRows; ++r) s += m.dy[r * kMaxOut + k];
        g[sh.ob3 + k] = s;
    }
    // layer 2: dW2[j][i] = sum_r d2[r][j] h1[r][i] (thread tile: j = 16w + b, i = 4l + c: per row
    // one 16-byte load of h1 and four broadcast 16-byte loads of d2); db2
    {
        constexpr int kJ = kH / 8;
        float acc[kJ][4];
#pragma unroll
        for (int b = 0; b < kJ; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[b][c] = 0.0f;
#pragma unroll 2
        for (int r = 0; r < kRows; ++r) {
            const float4 hv = *reinterpret_cast<const float4*>(m.a1 + r * kLd + 4 * l);
#pragma unroll
            for (int b4 = 0; b4 < kJ / 4; ++b4) {
                const float4 dv = *reinterpret_cast<const float4*>(m.d2 + r * kLd + kJ * w8 + 4 * b4);
                const float d[4] = {dv.x, dv.y, dv.z, dv.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float* ac = acc[4 * b4 + e];
                    ac[0] = fmaf(d[e], hv.x, ac[0]);
                    ac[1] = fmaf(d[e], hv.y, ac[1]);
                    ac[2] = fmaf(d[e], hv.z, ac[2]);
                    ac[3] = fmaf(d[e], hv.w, ac[3]);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < kJ; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) g[sh.oW2 + (kJ * w8 + b) * kH + 4 * l + c] = acc[b][c];
    }
    for (int j = threadIdx.x; j < kH; j += blockDim.x) {
        float s2 = 0.0f, s1 = 0.0f;
        for (int r = 0; r < kRows; ++r) {
            s2 += m.d2[r * kLd + j];
            s1 += m.d1[r * kLd + j];
        }
        g[sh.ob2 + j] = s2;
        g[sh.ob1 + j] = s1;
    }
    // layer 1: dW1[j][i] = sum_r d1[r][j] x[r][i]
    for (int q = threadIdx.x; q < kH * din; q += blockDim.x) {
        const int j = q / din, i = q % din;
        float s = 0.0f;
        for (int r = 0; r < kRows; ++r) s = fmaf(m.d1[r * kLd + j], m.x[r * (kMaxIn + 1) + i], s);
        g[sh.oW1 + q] = s;
    }
}

// grad[q] = sum over blocks (fixed order) of partial[b][q]; loss = sum of loss_part
__global__ void k_mlp_reduce(const float* __restrict__ partial, const float* __restrict__ loss_part, int nblocks, int64_t P, float* grad,
                             float* loss)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
#pragma unroll 8
        for (int b = 0; b < nblocks; ++b) s += partial[(int64_t)b * P + q];  // loads in flight together, sum in block order
        grad[q] = s;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
        float s = 0.0f;
        for (int b = 0; b < nblocks; ++b) s += loss_part[b];
        *loss = s;
    }
}

// Adam (Kingma & Ba): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
// p -= lr_t m / (sqrt(v) + eps) with the bias corrections folded into lr_t; BF16 copy refreshed.
__global__ void k_mlp_adam(float* p, float* mo, float* ve, const float* __restrict__ g, int64_t P, float lr_t, float b1, float b2, float eps,
                           __nv_bfloat16* w)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * mo[q] + (1.0f - b1) * gq;
        const float vq = b2 * ve[q] + (1.0f - b2) * gq * gq;
        mo[q] = mq;
        ve[q] = vq;
        const float pq = p[q] - lr_t * mq / (sqrtf(vq) + eps);
        p[q] = pq;
        w[q] = __float2bfloat16_rn(pq);
    }
}

// k_mlp_reduce and k_mlp_adam in one pass: the same gradient sums, then the same update.
__global__ void k_mlp_reduce_adam(const float* __restrict__ partial, const float* __restrict__ loss_part, int nblocks, int64_t P,
                                  float* grad, float* loss, float* p, float* mo, float* ve, float lr_t, float b1, float b2, float eps,
                                  __nv_bfloat16* w)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) {
        float gq = 0.0f;
#pragma unroll 16
        for (int b = 0; b < nblocks; ++b) gq += partial[(int64_t)b * P + q];  // loads in flight together, sum in block order
        grad[q] = gq;
        const float mq = b1 * mo[q] + (1.0f - b1) * gq;
        const float vq = b2 * ve[q] + (1.0f - b2) * gq * gq;
        mo[q] = mq;
        ve[q] = vq;
        const float pq = p[q] - lr_t * mq / (sqrtf(vq) + eps);
        p[q] = pq;
        w[q] = __float2bfloat16_rn(pq);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
        float sl = 0.0f;
        for (int b = 0; b < nblocks; ++b) sl += loss_part[b];
        *loss = sl;
    }
}

// He-uniform start: W ~ U(-s, s), s = sqrt(6 / fan_in), from Philox; biases 0.
__global__ void k_mlp_init(float* p, __nv_bfloat16* w, int din, int dout, uint32_t key0, uint32_t key1)
{
    const MlpShape sh = mlp_shape(din, dout);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < sh.P; q += (int64_t)gridDim.x * blockDim.x) {
        float fan = 0.0f;
        if (q < sh.ob1) fan = (float)din;
        else if (q >= sh.oW2 && q < sh.ob2) fan = (float)kH;
        else if (q >= sh.oW3 && q < sh.ob3) fan = (float)kH;
        float v = 0.0f;
        if (fan > 0.0f) {
            const uint4 o = Philox4x32::block(make_uint4((uint32_t)q, 0x4D4C5031u, 0u, 0u), key0, key1);
            v = signed_unit(o.x) * sqrtf(6.0f / fan);
        }
        p[q] = v;
        w[q] = __float2bfloat16_rn(v);
    }
}

__global__ void k_refresh_bf16(const float* __restrict__ p, int64_t P, __nv_bfloat16* w)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) w[q] = __float2bfloat16_rn(p[q]);
}

// Training rows from samples: X = [lambda (K), features], T_k = (C_k - offset_k) / scale_k.
struct RowConsts {
    float feat[kMaxIn];
    float offset[kMaxOut];
    float inv_scale[kMaxOut];
};

__global__ void k_mlp_rows(const float* __restrict__ lam, const int64_t* __restrict__ cuts, int64_t Mrows, int K, int din,
                           const RowConsts c, float* X, float* T)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Mrows * din; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = q / din;
        const int i = (int)(q - r * din);
        X[q] = i < K ? lam[r * K + i] : c.feat[i - K];
        if (i < K) T[r * K + i] = ((float)cuts[r * K + i] - c.offset[i]) * c.inv_scale[i];
    }
}

// ---- proposal ----------------------------------------------------------------------------
// inputs of the candidates: [lambda (K), features (din - K)]
__global__ void k_mlp_inputs(const float* __restrict__ lam, int K, int din, const float* __restrict__ feat, int C, float* X)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < C * din; q += gridDim.x * blockDim.x) {
        const int c = q / din, i = q % din;
        X[q] = i < K ? lam[(int64_t)c * K + i] : feat[i - K];
    }
}

// gap(p) = min over front members f of max_k (p_k - fhat_k), fhat = (f - offset) * inv_scale:
// how far the predicted point reaches beyond the nearest front member (> 0: undominated).
// Block (x, y) takes 256 candidates and the front chunks y, y + gridDim.y, ... of 256
// members; the minima meet in `key` through atomicMin on an order-preserving integer image of
// the float (min is exact, so the result does not depend on the split).
__device__ __forceinline__ uint32_t order_key(float v)
{
    const uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float from_order_key(uint32_t k) { return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k); }

constexpr uint32_t kKeyInf = 0xFF800000u;  // order_key(+inf)
constexpr int kGapSplits = 64;

__global__ void k_gap_init(uint32_t* key, int C)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) key[c] = kKeyInf;
}

__global__ void __launch_bounds__(256) k_front_gap(const float* __restrict__ pred, int C, int K, const int64_t* __restrict__ front,
                                                   const int64_t* __restrict__ d_count, const float* __restrict__ offset,
                                                   const float* __restrict__ inv_scale, uint32_t* key)
{
    __shared__ float tile[256][kMaxOut];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    float p[kMaxOut];
    for (int k = 0; k < kMaxOut; ++k) p[k] = (c < C && k < K) ? pred[(int64_t)c * K + k] : 0.0f;
    const int64_t F = *d_count;
    float gap = INFINITY;
    for (int64_t base = (int64_t)blockIdx.y * 256; base < F; base += (int64_t)gridDim.y * 256) {
        const int cnt = (int)min((int64_t)256, F - base);
        __syncthreads();
        if (threadIdx.x < cnt)
            for (int k = 0; k < K; ++k) tile[threadIdx.x][k] = ((float)front[(base + threadIdx.x) * K + k] - offset[k]) * inv_scale[k];
        __syncthreads();
        for (int t = 0; t < cnt; ++t) {
            float mx = -INFINITY;
            for (int k = 0; k < K; ++k) mx = fmaxf(mx, p[k] - tile[t][k]);
            gap = fminf(gap, mx);
        }
    }
    if (c < C && gap < INFINITY) atomicMin(key + c, order_key(gap));
}

// score = the gap (NaN -> -inf); rank = number of candidates with a higher score (ties: lower
// index first); the R best go out in rank order. Scores pass through shared memory in chunks.
__global__ void __launch_bounds__(64) k_top_r(const uint32_t* __restrict__ key, const float* __restrict__ lam, int C, int K, int R,
                                              float* out)
{
    __shared__ float sc[1024];
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    auto score_of = [&](int q) {
        const float g = from_order_key(key[q]);
        return isnan(g) ? -INFINITY : g;
    };
    const float s = c < C ? score_of(c) : 0.0f;
    int rank = 0;
    for (int base = 0; base < C; base += 1024) {
        const int cnt = min(1024, C - base);
        __syncthreads();
        for (int q = threadIdx.x; q < cnt; q += blockDim.x) sc[q] = score_of(base + q);
        __syncthreads();
        for (int q = 0; q < cnt; ++q) {
            const float t = sc[q];
            rank += (t > s) || (t == s && base + q < c);
        }
    }
    if (c < C && rank < R)
        for (int k = 0; k < K; ++k) out[(int64_t)rank * K + k] = lam[(int64_t)c * K + k];
}

}  // namespace
}  // namespace moq

struct moq_mlp {
    int din = 0, dout = 0, max_batch = 0, max_cand = 0, max_blocks = 0;
    int engine = MOQ_MLP_CUDA_CORES;    // which kernels run the products
    int32_t* status = nullptr;          // tensor-core engine: latched wait time-outs
    int64_t P = 0, step = 0;
    float* master = nullptr;
    __nv_bfloat16* w16 = nullptr;
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* partial = nullptr;
    float* loss_part = nullptr;
    float* cand = nullptr;  // candidate lambda, inputs, predictions, scores, feature/normalisation constants
    float* cand_in = nullptr;
    float* cand_pred = nullptr;
    float* cand_score = nullptr;
    float* consts = nullptr;
    void* slab = nullptr;  // the one device allocation the arrays above live in
};

namespace moq {
namespace {

void free_mlp(moq_mlp* m)
{
    if (!m) return;
    slab_free(m->slab);
    delete m;
}

size_t mlp_smem_bytes() { return sizeof(float) * mlp_smem_floats(); }

MlpTcArgs tc_args(const moq_mlp* m, const float* X, const float* T, int64_t B, float* Y)
{
    const MlpShape sh = mlp_shape(m->din, m->dout);
    MlpTcArgs a{};
    a.w = m->w16;
    a.din = m->din;
    a.dout = m->dout;
    a.oW1 = sh.oW1;
    a.ob1 = sh.ob1;
    a.oW2 = sh.oW2;
    a.ob2 = sh.ob2;
    a.oW3 = sh.oW3;
    a.ob3 = sh.ob3;
    a.P = sh.P;
    a.X = X;
    a.T = T;
    a.B = B;
    a.Y = Y;
    a.partial = m->partial;
    a.loss_part = m->loss_part;
    a.status = m->status;
    return a;
}

}  // namespace
}  // namespace moq

extern "C" {

int moq_mlp_create(int32_t d_in, int32_t d_out, int32_t max_batch, int32_t max_candidates, uint64_t seed, moq_mlp** out)
{
    using namespace moq;
    if (!out) return fail(MOQ_ERR_ARG, "moq_mlp_create: out is NULL");
    *out = nullptr;
    if (d_in < 1 || d_in > kMaxIn || d_out < 1 || d_out > kMaxOut || max_batch < 1 || max_candidates < 1)
        return fail(MOQ_ERR_ARG, "moq_mlp_create: need 1 <= d_in <= %d, 1 <= d_out <= %d, max_batch, max_candidates >= 1", kMaxIn, kMaxOut);
    moq_mlp* m = new moq_mlp();
    m->din = d_in;
    m->dout = d_out;
    m->max_batch = max_batch;
    m->max_cand = max_candidates;
    m->max_blocks = (int)ceil_div(max_batch, kRows);
    m->P = mlp_shape(d_in, d_out).P;
    // one slab from the library's memory pool for all arrays (ordered on the legacy stream;
    // with a cudaMalloc per array a handle cost about a millisecond to create and as much to
    // free, inside every learned time-to-target clock)
    std::vector<std::pair<void**, size_t>> parts = {
        {(void**)&m->master, sizeof(float) * m->P}, {(void**)&m->w16, sizeof(__nv_bfloat16) * m->P},
        {(void**)&m->grad, sizeof(float) * m->P}, {(void**)&m->adam_m, sizeof(float) * m->P},
        {(void**)&m->adam_v, sizeof(float) * m->P}, {(void**)&m->partial, sizeof(float) * m->P * m->max_blocks},
        {(void**)&m->loss_part, sizeof(float) * (m->max_blocks + 1)}, {(void**)&m->cand, sizeof(float) * max_candidates * d_out},
        {(void**)&m->cand_in, sizeof(float) * max_candidates * d_in}, {(void**)&m->cand_pred, sizeof(float) * max_candidates * d_out},
        {(void**)&m->cand_score, sizeof(float) * max_candidates}, {(void**)&m->consts, sizeof(float) * 64},
        {(void**)&m->status, sizeof(int32_t)}};
    size_t total = 0;
    for (auto& pr : parts) total += slab_align(pr.second);
    const cudaStream_t st0 = cudaStreamLegacy;
    cudaError_t e = slab_alloc(&m->slab, total, st0);
    if (e == cudaSuccess) {
        size_t off = 0;
        for (auto& pr : parts) {
            *pr.first = static_cast<char*>(m->slab) + off;
            off += slab_align(pr.second);
        }
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(m->status, 0, sizeof(int32_t), st0);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->adam_m, 0, sizeof(float) * m->P, st0);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->adam_v, 0, sizeof(float) * m->P, st0);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->grad, 0, sizeof(float) * m->P, st0);
    if (e == cudaSuccess) {
        k_mlp_init<<<64, 256, 0, st0>>>(m->master, m->w16, d_in, d_out, (uint32_t)seed, (uint32_t)(seed >> 32));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem_bytes());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem_bytes());
    if (e == cudaSuccess) e = cudaStreamSynchronize(st0);  // ready for any stream
    if (e != cudaSuccess) {
        free_mlp(m);
        return cuda_fail(e, "moq_mlp_create");
    }
    *out = m;
    return MOQ_OK;
}

void moq_mlp_destroy(moq_mlp* m) { moq::free_mlp(m); }

int64_t moq_mlp_param_count(const moq_mlp* m) { return m ? m->P : 0; }

int moq_mlp_set_params(moq_mlp* m, const float* params_host)
{
    using namespace moq;
    if (!m || !params_host) return fail(MOQ_ERR_ARG, "moq_mlp_set_params: NULL argument");
    MOQ_CUDA_TRY(cudaMemcpy(m->master, params_host, sizeof(float) * m->P, cudaMemcpyHostToDevice));
    k_refresh_bf16<<<64, 256>>>(m->master, m->P, m->w16);
    MOQ_LAUNCH_CHECK("moq_mlp_set_params");
    MOQ_CUDA_TRY(cudaDeviceSynchronize());
    return MOQ_OK;
}

int moq_mlp_get_params(const moq_mlp* m, float* params_host, int32_t bf16_rounded)
{
    using namespace moq;
    if (!m || !params_host) return fail(MOQ_ERR_ARG, "moq_mlp_get_params: NULL argument");
    if (!bf16_rounded) {
        MOQ_CUDA_TRY(cudaMemcpy(params_host, m->master, sizeof(float) * m->P, cudaMemcpyDeviceToHost));
        return MOQ_OK;
    }
    std::vector<__nv_bfloat16> tmp(m->P);
    MOQ_CUDA_TRY(cudaMemcpy(tmp.data(), m->w16, sizeof(__nv_bfloat16) * m->P, cudaMemcpyDeviceToHost));
    for (int64_t q = 0; q < m->P; ++q) params_host[q] = __bfloat162float(tmp[q]);
    return MOQ_OK;
}

int moq_mlp_forward(const moq_mlp* m, const float* X, int32_t B, float* Y, void* stream)
{
    using namespace moq;
    if (!m || B < 0 || (B > 0 && (!X || !Y))) return fail(MOQ_ERR_ARG, "moq_mlp_forward: bad argument");
    if (B == 0) return MOQ_OK;
    if (m->engine == MOQ_MLP_TENSOR_CORES) {
        const cudaError_t e = launch_mlp_tc(tc_args(m, X, nullptr, B, Y), false, as_stream(stream));
        if (e != cudaSuccess) return cuda_fail(e, "moq_mlp_forward (tensor cores)");
        return MOQ_OK;
    }
    const int grid = (int)std::min<int64_t>(ceil_div(B, kRows), 148 * 2);
    k_mlp_forward<<<grid, kThreads, mlp_smem_bytes(), as_stream(stream)>>>(m->w16, m->din, m->dout, X, B, Y);
    MOQ_LAUNCH_CHECK("moq_mlp_forward");
    return MOQ_OK;
}

int moq_mlp_gradient(moq_mlp* m, const float* X, const float* T, int32_t B, float* grad_out, float* loss_out, void* stream)
{
    using namespace moq;
    if (!m || B < 1 || B > m->max_batch || !X || !T) return fail(MOQ_ERR_ARG, "moq_mlp_gradient: need 1 <= B <= max_batch and inputs");
    cudaStream_t st = as_stream(stream);
    int nb;
    if (m->engine == MOQ_MLP_TENSOR_CORES) {
        nb = (int)ceil_div(B, kMlpTcRows);
        const cudaError_t e = launch_mlp_tc(tc_args(m, X, T, B, nullptr), true, st);
        if (e != cudaSuccess) return cuda_fail(e, "moq_mlp_gradient (tensor cores)");
    } else {
        nb = (int)ceil_div(B, kRows);
        k_mlp_grad<<<nb, kThreads, mlp_smem_bytes(), st>>>(m->w16, m->din, m->dout, X, T, B, m->partial, m->loss_part);
    }
    k_mlp_reduce<<<(unsigned)std::min<int64_t>(ceil_div(m->P, 256), 148), 256, 0, st>>>(m->partial, m->loss_part, nb, m->P, m->grad,
                                                                                       loss_out ? loss_out : m->loss_part + m->max_blocks);
    MOQ_LAUNCH_CHECK("moq_mlp_gradient");
    if (grad_out) MOQ_CUDA_TRY(cudaMemcpyAsync(grad_out, m->grad, sizeof(float) * m->P, cudaMemcpyDeviceToDevice, st));
    return MOQ_OK;
}

int moq_mlp_adam_step(moq_mlp* m, float lr, void* stream)
{
    using namespace moq;
    if (!m || !(lr > 0.0f)) return fail(MOQ_ERR_ARG, "moq_mlp_adam_step: bad argument");
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    m->step += 1;
    const double t = (double)m->step;
    const float lr_t = (float)(lr * std::sqrt(1.0 - std::pow(b2, t)) / (1.0 - std::pow(b1, t)));
    k_mlp_adam<<<(unsigned)std::min<int64_t>(ceil_div(m->P, 256), 148), 256, 0, as_stream(stream)>>>(m->master, m->adam_m, m->adam_v, m->grad,
                                                                                                       m->P, lr_t, b1, b2, eps, m->w16);
    MOQ_LAUNCH_CHECK("moq_mlp_adam_step");
    return MOQ_OK;
}

int moq_mlp_train_step(moq_mlp* m, const float* X, const float* T, int32_t B, float lr, float* loss_out, void* stream)
{
    using namespace moq;
    if (!m || B < 1 || B > m->max_batch || !X || !T || !(lr > 0.0f))
        return fail(MOQ_ERR_ARG, "moq_mlp_train_step: need 1 <= B <= max_batch, inputs and lr > 0");
    cudaStream_t st = as_stream(stream);
    int nb;
    if (m->engine == MOQ_MLP_TENSOR_CORES) {
        nb = (int)ceil_div(B, kMlpTcRows);
        const cudaError_t e = launch_mlp_tc(tc_args(m, X, T, B, nullptr), true, st);
        if (e != cudaSuccess) return cuda_fail(e, "moq_mlp_train_step (tensor cores)");
    } else {
        nb = (int)ceil_div(B, kRows);
        k_mlp_grad<<<nb, kThreads, mlp_smem_bytes(), st>>>(m->w16, m->din, m->dout, X, T, B, m->partial, m->loss_part);
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    m->step += 1;
    const double t = (double)m->step;
    const float lr_t = (float)(lr * std::sqrt(1.0 - std::pow(b2, t)) / (1.0 - std::pow(b1, t)));
    k_mlp_reduce_adam<<<(unsigned)std::min<int64_t>(ceil_div(m->P, 256), 148), 256, 0, st>>>(
        m->partial, m->loss_part, nb, m->P, m->grad, loss_out ? loss_out : m->loss_part + m->max_blocks, m->master, m->adam_m,
        m->adam_v, lr_t, b1, b2, eps, m->w16);
    MOQ_LAUNCH_CHECK("moq_mlp_train_step");
    return MOQ_OK;
}

int moq_mlp_set_engine(moq_mlp* m, int32_t engine)
{
    using namespace moq;
    if (!m || (engine != MOQ_MLP_CUDA_CORES && engine != MOQ_MLP_TENSOR_CORES)) return fail(MOQ_ERR_ARG, "moq_mlp_set_engine: bad argument");
    m->engine = engine;
    return MOQ_OK;
}

int moq_mlp_status(moq_mlp* m, void* stream)
{
    using namespace moq;
    if (!m) return fail(MOQ_ERR_ARG, "moq_mlp_status: NULL handle");
    cudaStream_t st = as_stream(stream);
    int32_t h = 0;
    MOQ_CUDA_TRY(cudaMemcpyAsync(&h, m->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MOQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) {
        MOQ_CUDA_TRY(cudaMemsetAsync(m->status, 0, sizeof(int32_t), st));
        return fail(MOQ_ERR_TIMEOUT, "moq_mlp: a tensor-core wait ran out of its budget");
    }
    return MOQ_OK;
}

int moq_mlp_make_rows(int32_t K, int32_t n_features, const float* lambda, const int64_t* cuts, int64_t M, const float* features,
                      const int64_t* offset, const int64_t* scale, float* X, float* T, void* stream)
{
    using namespace moq;
    if (K < 1 || K > kMaxOut || n_features < 0 || K + n_features > kMaxIn || M < 0 || !offset || !scale || (n_features > 0 && !features))
        return fail(MOQ_ERR_ARG, "moq_mlp_make_rows: bad shape or NULL constant");
    if (M == 0) return MOQ_OK;
    if (!lambda || !cuts || !X || !T) return fail(MOQ_ERR_ARG, "moq_mlp_make_rows: NULL device array");
    RowConsts c{};
    for (int i = 0; i < n_features; ++i) c.feat[i] = features[i];
    for (int k = 0; k < K; ++k) {
        c.offset[k] = (float)offset[k];
        c.inv_scale[k] = scale[k] > 0 ? 1.0f / (float)scale[k] : 1.0f;
    }
    const int din = K + n_features;
    k_mlp_rows<<<(unsigned)std::min<int64_t>(ceil_div(M * din, 256), 148 * 16), 256, 0, as_stream(stream)>>>(lambda, cuts, M, K, din, c, X, T);
    MOQ_LAUNCH_CHECK("moq_mlp_make_rows");
    return MOQ_OK;
}

int moq_lambda_propose(moq_mlp* m, const moq_archive* a, const float* features, int32_t n_features, const int64_t* offset,
                       const int64_t* scale, int32_t n_candidates, uint64_t seed, uint64_t round, float* lambda_out, int32_t R,
                       void* stream)
{
    using namespace moq;
    if (!m || !a || !lambda_out || !offset || !scale) return fail(MOQ_ERR_ARG, "moq_lambda_propose: NULL argument");
    const int K = m->dout;
    if (a->K != K || n_features != m->din - K || n_features < 0 || (n_features > 0 && !features))
        return fail(MOQ_ERR_ARG, "moq_lambda_propose: the MLP must map K + n_features inputs to the archive's K objectives");
    if (n_candidates < 1 || n_candidates > m->max_cand || R < 0 || R > n_candidates)
        return fail(MOQ_ERR_ARG, "moq_lambda_propose: need 1 <= R <= n_candidates <= max_candidates");
    if (R == 0) return MOQ_OK;
    cudaStream_t st = as_stream(stream);
    float hc[64];
    for (int i = 0; i < n_features; ++i) hc[i] = features[i];
    for (int k = 0; k < K; ++k) {
        hc[16 + k] = (float)offset[k];
        hc[24 + k] = scale[k] > 0 ? 1.0f / (float)scale[k] : 1.0f;
    }
    MOQ_CUDA_TRY(cudaMemcpyAsync(m->consts, hc, sizeof(hc), cudaMemcpyHostToDevice, st));
    int rc = moq_lambda_dirichlet(K, n_candidates, seed, round, m->cand, stream);
    if (rc != MOQ_OK) return rc;
    const int C = n_candidates;
    k_mlp_inputs<<<(unsigned)ceil_div((int64_t)C * m->din, 256), 256, 0, st>>>(m->cand, K, m->din, m->consts, C, m->cand_in);
    MOQ_LAUNCH_CHECK("moq_lambda_propose inputs");
    rc = moq_mlp_forward(m, m->cand_in, C, m->cand_pred, stream);
    if (rc != MOQ_OK) return rc;
    const int64_t *fc = nullptr, *cnt = nullptr;
    moq_archive_device_view(a, &fc, nullptr, nullptr, &cnt);
    uint32_t* key = reinterpret_cast<uint32_t*>(m->cand_score);
    k_gap_init<<<(unsigned)ceil_div(C, 256), 256, 0, st>>>(key, C);
    k_front_gap<<<dim3((unsigned)ceil_div(C, 256), kGapSplits), 256, 0, st>>>(m->cand_pred, C, K, fc, cnt, m->consts + 16, m->consts + 24, key);
    k_top_r<<<(unsigned)ceil_div(C, 64), 64, 0, st>>>(key, m->cand, C, K, R, lambda_out);
    MOQ_LAUNCH_CHECK("moq_lambda_propose select");
    return MOQ_OK;
}

}  // extern "C"
