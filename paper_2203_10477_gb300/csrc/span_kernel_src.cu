// span_kernel_src.cu -- the span kernel variants compiled with user point
// sources (a separate translation unit so that both compilations of every
// variant build in parallel).

#include "span_kernel.cuh"

namespace rswr {

namespace {

template <typename Real, int FORM, int P, int NT, int KH, int MINB>
const void* src_kernel_PLAIN()
{
    return reinterpret_cast<const void*>(&span_kernel<Real, FORM, P, NT, KH, MINB, true>);
}

template <typename Real, int FORM, int P, int NT, int KH, int MINB>
const void* src_kernel_WS()
{
    return reinterpret_cast<const void*>(&span_kernel_ws<Real, FORM, P, NT, KH, MINB, true>);
}

template <typename Real, int FORM, int P, int NT, int KH, int MINB>
const void* src_kernel_RES()
{
    return reinterpret_cast<const void*>(&span_kernel_res<Real, FORM, P, NT, KH, MINB, true>);
}

#define RSWR_SRC_KERNEL(kind, Real, FORM, P, NT, KH, MINB) src_kernel_##kind<Real, FORM, P, NT, KH, MINB>(),

}  // namespace

const void* span_src_kernel(int v)
{
    static const void* const fns[] = {RSWR_SPAN_VARIANTS(RSWR_SRC_KERNEL)};
    return (v >= 0 && v < (int)(sizeof(fns) / sizeof(fns[0]))) ? fns[v] : nullptr;
}

}  // namespace rswr
