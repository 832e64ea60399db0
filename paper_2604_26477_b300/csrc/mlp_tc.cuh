// The tensor-core engine of the surrogate MLP (mlp_tc.cu), called by the entry points in mlp.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace moq {

struct MlpTcArgs {
    const __nv_bfloat16* w;  // flat BF16 parameters W1, b1, W2, b2, W3, b3
    int32_t din, dout;
    int64_t oW1, ob1, oW2, ob2, oW3, ob3, P;
    const float* X;      // B x din
    const float* T;      // B x dout (training)
    int64_t B;
    float* Y;            // B x dout (forward) or NULL
    float* partial;      // training: one slot of P floats per 128-row tile
    float* loss_part;    // training: one float per tile
    int32_t* status;     // bit 0 latched when a tensor-core wait runs out
};

constexpr int kMlpTcRows = 128;  // rows per CTA (one TMEM lane per row)

// forward (train = false: Y) or forward + backward (train = true: gradient slots, loss parts)
cudaError_t launch_mlp_tc(const MlpTcArgs& a, bool train, cudaStream_t st);

}  // namespace moq
