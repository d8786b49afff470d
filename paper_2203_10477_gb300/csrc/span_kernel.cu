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

// resident tiles: NT threads, one CTA per tile, every tile on the GPU at once
template <typename Real, int FORM, int P, int NT, int KH, int MINB>
Entry make_entry_RES()
{
    using G = Geom<P, NT, KH>;
    Entry e;
    e.info = VariantInfo{sizeof(Real) == 8 ? kF64 : kF32, FORM, P, NT, KH, G::W, NT, G::FREE ? KH : 0, 1};
    e.fn = reinterpret_cast<const void*>(&span_kernel_res<Real, FORM, P, NT, KH, MINB, false>);
    e.fn_src = nullptr;
    e.smem = sizeof(Real) * (2 * G::W + G::XCH);
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

// Resident variants: a launch of `grid` CTAs asks for enough dynamic shared
// memory that at most ceil(grid / SMs) of them fit on one SM, so the CTAs
// spread over all SMs (the block scheduler fills an SM up to its occupancy;
// with one CTA per tile in lockstep, a crowded SM would set every span's pace).
size_t resident_smem(const Entry& e, int grid)
{
    int dev = 0, sms = 1, per_sm = 0, per_block = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) ||
        cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) {
        cudaGetLastError();
        return e.smem;
    }
    const int cap = (grid + sms - 1) / sms;
    cudaFuncAttributes fa{}, fb{};
    if (cudaFuncGetAttributes(&fa, e.fn) != cudaSuccess || cudaFuncGetAttributes(&fb, e.fn_src) != cudaSuccess) {
        cudaGetLastError();
        return e.smem;
    }
    const size_t stat = fa.sharedSizeBytes > fb.sharedSizeBytes ? fa.sharedSizeBytes : fb.sharedSizeBytes;
    // per CTA on an SM: dynamic + static shared memory + 1 KiB the runtime reserves
    long long want = (long long)per_sm / (cap > 0 ? cap : 1) - (long long)stat - 1024;
    if (want + (long long)stat > per_block) want = per_block - (long long)stat;
    want = want / 1024 * 1024;
    // the occupancy calculator has the last word: step down until cap CTAs fit
    for (; want > (long long)e.smem; want -= 1024) {
        int a = 0, b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, e.fn, e.info.threads, (size_t)want) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, e.fn_src, e.info.threads, (size_t)want) != cudaSuccess) {
            cudaGetLastError();
            return e.smem;
        }
        if (a >= cap && b >= cap) return (size_t)want;
    }
    return e.smem;
}

cudaError_t span_prepare(int v)
{
    int n;
    const Entry& e = table(&n)[v];
    int lim = (int)e.smem;
    if (e.info.resident) {  // launches may ask for more (resident_smem)
        int dev = 0, per_block = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
            per_block > lim)
            lim = per_block - 1024;  // room for the static shared memory
        cudaGetLastError();
    }
    cudaError_t st = cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (st != cudaSuccess) return st;
    return cudaFuncSetAttribute(e.fn_src, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
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
    if (e.info.resident)  // every CTA waits on its neighbours: they must all be resident
        return cudaLaunchCooperativeKernel(src ? e.fn_src : e.fn, dim3(grid), dim3(e.info.threads), args,
                                           resident_smem(e, grid), s);
    return cudaLaunchKernel(src ? e.fn_src : e.fn, dim3(grid), dim3(e.info.threads), args, e.smem, s);
}

}  // namespace rswr
