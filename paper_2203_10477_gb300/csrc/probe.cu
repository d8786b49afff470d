// probe.cu -- arithmetic-pipe throughput probe (a measurement utility of the
// library, not a step of the method).
//
// The span kernels are bound by the FP64 pipe (canonical form: one add and
// two fused multiply-adds per update) or by the FP32 pipe (increment form:
// three adds and one fused multiply-add).  Their roofline is the pipe's rate
// divided by the instructions per update.  This kernel measures that rate on
// the device it runs on: every thread advances eight independent chains of
// fused multiply-adds, so the pipe, not the latency of one chain, sets the
// time.  It changes no device setting and allocates nothing; the caller
// times it with events on `stream`.

#include <cstdint>

#include "../../include/rswr.h"
#include "rswr_internal.h"

using namespace rswr;

namespace {

template <typename Real>
__device__ __forceinline__ Real fma_rn(Real x, Real y, Real z);
template <>
__device__ __forceinline__ double fma_rn<double>(double x, double y, double z) { return __fma_rn(x, y, z); }
template <>
__device__ __forceinline__ float fma_rn<float>(float x, float y, float z) { return __fmaf_rn(x, y, z); }

template <typename Real>
__global__ void fma_probe_kernel(Real a, Real b, int64_t iters, Real* sink)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    Real x0 = (Real)threadIdx.x * (Real)1e-3, x1 = x0 + (Real)1, x2 = x0 + (Real)2, x3 = x0 + (Real)3;
    Real x4 = x0 + (Real)4, x5 = x0 + (Real)5, x6 = x0 + (Real)6, x7 = x0 + (Real)7;
#pragma unroll 16
    for (int64_t i = 0; i < iters; ++i) {
        x0 = fma_rn(x0, a, b);
        x1 = fma_rn(x1, a, b);
        x2 = fma_rn(x2, a, b);
        x3 = fma_rn(x3, a, b);
        x4 = fma_rn(x4, a, b);
        x5 = fma_rn(x5, a, b);
        x6 = fma_rn(x6, a, b);
        x7 = fma_rn(x7, a, b);
    }
    sink[tid] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

// The same with packed pairs of FP32 values (fma.rn.f32x2, or add.rn.f32x2
// when ADD): 16 FP32 lanes per iteration in 8 instructions.
template <bool ADD>
__global__ void fma2_probe_kernel(float a, float b, int64_t iters, float* sink)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t x[8], ab, bb;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ab) : "f"(a), "f"(a));
    asm("mov.b64 %0, {%1, %2};" : "=l"(bb) : "f"(b), "f"(b));
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float lo = (float)threadIdx.x * 1e-3f + (float)c, hi = lo + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x[c]) : "f"(lo), "f"(hi));
    }
#pragma unroll 16
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if constexpr (ADD)
                asm("add.rn.f32x2 %0, %0, %1;" : "+l"(x[c]) : "l"(bb));
            else
                asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(ab), "l"(bb));
        }
    }
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        acc += lo + hi;
    }
    sink[tid] = acc;
}

}  // namespace

extern "C" rswr_status rswr_fma_probe(int32_t dtype, int64_t iters, int32_t blocks, int32_t threads, void* sink,
                                      void* stream)
{
    if (iters < 1 || blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0 || !sink) {
        set_error_message("rswr_fma_probe: need iters >= 1, blocks >= 1, 32 <= threads <= 1024 (a multiple "
                          "of 32) and a sink");
        return RSWR_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == RSWR_F64)
        fma_probe_kernel<double><<<blocks, threads, 0, s>>>(0.999999, 1e-7, iters, static_cast<double*>(sink));
    else if (dtype == RSWR_F32)
        fma_probe_kernel<float><<<blocks, threads, 0, s>>>(0.999999f, 1e-7f, iters, static_cast<float*>(sink));
    else if (dtype == 2)
        fma2_probe_kernel<false><<<blocks, threads, 0, s>>>(0.999999f, 1e-7f, iters, static_cast<float*>(sink));
    else if (dtype == 3)
        fma2_probe_kernel<true><<<blocks, threads, 0, s>>>(0.999999f, 1e-7f, iters, static_cast<float*>(sink));
    else {
        set_error_message("rswr_fma_probe: dtype must be RSWR_F32, RSWR_F64, 2 (packed FP32 pairs) or 3 (packed adds)");
        return RSWR_EINVAL;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error_message(cudaGetErrorString(e));
        return RSWR_ECUDA;
    }
    return RSWR_OK;
}
