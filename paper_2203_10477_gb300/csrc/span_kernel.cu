// span_kernel.cu -- the variant registry of the RSWR span kernel: every
// variant of RSWR_SPAN_VARIANTS compiled without user point sources (the
// kernels of runs without them), plus the launch entry points.

#include <vector>

#include "span_kernel.cuh"

namespace rswr {

namespace {

// Every variant is compiled twice: without user point sources (fn, here) and
// with them (fn_src, span_kernel_src.cu; launched when SpanParams::srcs is
// set), so that runs without sources carry none of their code.
struct Entry {
    VariantInfo info;
    const void* fn;
    const void* fn_src;
    size_t smem;
};

template <typename Real, int FORM, int P, int NT, int KH, int MINB>
Entry make_entry_PLAIN()
{
    using G = Geom<P, NT, KH>;
    Entry e;
    e.info = VariantInfo{sizeof(Real) == 8 ? kF64 : kF32, FORM, P, NT, KH, G::W, NT, 0};
    e.fn = reinterpret_cast<const void*>(&span_kernel<Real, FORM, P, NT, KH, MINB, false>);
    e.fn_src = nullptr;
    e.smem = sizeof(Real) * (4 * G::W + G::XCH);
    return e;
}

// warp-specialised: NT compute threads + one producer warp
template <typename Real, int FORM, int P, int NT, int KH, int MINB>
Entry make_entry_WS()
{
    using G = Geom<P, NT, KH>;
    Entry e;
    e.info = VariantInfo{sizeof(Real) == 8 ? kF64 : kF32, FORM, P, NT, KH, G::W, NT + 32, G::FREE ? KH : 0};
    e.fn = reinterpret_cast<const void*>(&span_kernel_ws<Real, FORM, P, NT, KH, MINB, false>);
    e.fn_src = nullptr;
    e.smem = sizeof(Real) * (4 * G::W + G::XCH);
    return e;
}

#define RSWR_MAKE_ENTRY(kind, Real, FORM, P, NT, KH, MINB) make_entry_##kind<Real, FORM, P, NT, KH, MINB>(),

const Entry* table(int* n)
{
    static const std::vector<Entry> entries = [] {
        std::vector<Entry> e{RSWR_SPAN_VARIANTS(RSWR_MAKE_ENTRY)};
        for (size_t v = 0; v < e.size(); ++v) e[v].fn_src = span_src_kernel((int)v);
        return e;
    }();
    *n = (int)entries.size();
    return entries.data();
}

}  // namespace

int span_variant_count()
{
    int n;
    table(&n);
    return n;
}

VariantInfo span_variant_info(int v)
{
    int n;
    const Entry* e = table(&n);
    return e[v].info;
}

size_t span_smem_bytes(int v)
{
    int n;
    return table(&n)[v].smem;
}

cudaError_t span_prepare(int v)
{
    int n;
    const Entry& e = table(&n)[v];
    cudaError_t st = cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e.smem);
    if (st != cudaSuccess) return st;
    return cudaFuncSetAttribute(e.fn_src, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e.smem);
}

// the smaller residency of the two compilations
cudaError_t span_occupancy(int v, int* blocks_per_sm)
{
    int n;
    const Entry& e = table(&n)[v];
    cudaError_t st = span_prepare(v);
    if (st != cudaSuccess) return st;
    int a = 0, b = 0;
    st = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, e.fn, e.info.threads, e.smem);
    if (st != cudaSuccess) return st;
    st = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, e.fn_src, e.info.threads, e.smem);
    *blocks_per_sm = a < b ? a : b;
    return st;
}

cudaError_t span_launch(int v, const void* params, int grid, cudaStream_t s)
{
    int n;
    const Entry& e = table(&n)[v];
    const bool src = e.info.dtype == kF64 ? static_cast<const SpanParams<double>*>(params)->srcs != nullptr
                                          : static_cast<const SpanParams<float>*>(params)->srcs != nullptr;
    void* args[] = {const_cast<void*>(params)};
    return cudaLaunchKernel(src ? e.fn_src : e.fn, dim3(grid), dim3(e.info.threads), args, e.smem, s);
}

}  // namespace rswr
