// Error reporting and defaults of the C ABI.
#include <stdarg.h>
#include <stdio.h>

#include "moq_common.cuh"

namespace moq {

static thread_local char g_last_msg[512] = "";
static thread_local int g_last_code = MOQ_OK;

int fail(int code, const char* fmt, ...)
{
    g_last_code = code;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_msg, sizeof(g_last_msg), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t err, const char* what)
{
    if (err == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(MOQ_ERR_OOM, "%s: %s", what, cudaGetErrorString(err));
    }
    return fail(MOQ_ERR_CUDA, "%s: %s", what, cudaGetErrorString(err));
}

}  // namespace moq

extern "C" {

const char* moq_strerror(int code)
{
    switch (code) {
    case MOQ_OK: return "success";
    case MOQ_ERR_ARG: return "invalid argument";
    case MOQ_ERR_OOM: return "out of device memory";
    case MOQ_ERR_CUDA: return "CUDA error";
    case MOQ_ERR_TIMEOUT: return "device wait timed out";
    case MOQ_ERR_CAPACITY: return "capacity exceeded";
    case MOQ_ERR_OVERFLOW: return "result outside the exact integer range";
    case MOQ_ERR_UNSUPPORTED: return "not supported by the library";
    default: return "unknown status";
    }
}

const char* moq_last_error_message(void) { return moq::g_last_msg; }

int moq_last_status(void) { return moq::g_last_code; }

void moq_default_params(moq_sample_params* p)
{
    if (!p) return;
    p->variant = MOQ_DSB;
    p->steps = 1000;
    p->dt = 1.0f;
    p->a0 = 1.0f;
    p->alpha = 0.0f;
    p->init_amp = 0.1f;
    p->noise_sqrt_dt = 0;
    p->schedule = nullptr;
    p->x_init = nullptr;
    p->y_init = nullptr;
    p->x_out = nullptr;
    p->y_out = nullptr;
    p->replica_offset = 0;
    p->precision = MOQ_PREC_FP32;
}

}  // extern "C"
