// mono_kernel.cu -- the monolithic (undecomposed) leapfrog, one time step per
// launch over the whole grid: the paper's "true solution" (Sec. 2.1) and the
// comparator that RSWR's temporal blocking is measured against.  Plus two
// small helpers used by every run: the final-level probe kernel and the
// level-0 boundary setter.
//
// HBM-bound by design: each step reads u^n (with neighbours) and the second
// state component, and writes the new level -- 3 values per point per step in
// the canonical form, 4 in the increment form.  Each thread owns 4 consecutive
// points loaded as one 16-byte (float4) or two 16-byte (double2) vectors.

#include "rswr_internal.h"

namespace rswr {

namespace {

template <typename Real>
struct V4;
template <>
struct V4<float> {
    __device__ static void load(const float* p, float (&r)[4])
    {
        const float4 v = *reinterpret_cast<const float4*>(p);
        r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    }
    __device__ static void store(float* p, const float (&r)[4])
    {
        *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
    }
};
template <>
struct V4<double> {
    __device__ static void load(const double* p, double (&r)[4])
    {
        const double2 a = reinterpret_cast<const double2*>(p)[0];
        const double2 b = reinterpret_cast<const double2*>(p)[1];
        r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
    }
    __device__ static void store(double* p, const double (&r)[4])
    {
        reinterpret_cast<double2*>(p)[0] = make_double2(r[0], r[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(r[2], r[3]);
    }
};

template <typename Real>
__device__ __forceinline__ void probe_one(const ProbeDev<Real>& pr, const Real* u, int64_t n)
{
    Real val;
    if (pr.kind == 0) val = u[pr.gidx];
    else val = rsub(u[pr.gidx + 1], u[pr.gidx - 1]);
    val = rmul(val, pr.scale);
    if (n <= pr.nmax) pr.out[n * pr.stride] = val;
}

static_assert(kMonoBlockPoints == 256 * 4, "block CSR of the sources assumes 256 threads x 4 points");

template <typename Real, int FORM>
__global__ void __launch_bounds__(256) mono_step_kernel(const __grid_constant__ MonoParams<Real> p)
{
    // probes of level n are read before anything of level n+1 exists in `cur`
    if (blockIdx.x == 0)
        for (int q = threadIdx.x; q < p.nprobe; q += blockDim.x) probe_one(p.probes[q], p.cur, p.n);

    const int64_t j0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (j0 >= p.nx) return;
    const int64_t g = p.base + j0;
    Real u[4], w[4], out_u[4], out_w[4];
    V4<Real>::load(p.cur + g, u);
    const Real ul0 = p.cur[g - 1];
    const Real ur3 = p.cur[g + 4];
    V4<Real>::load(p.prev + g, w);
    const Real c2 = p.c2, k = p.k;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const Real ul = i == 0 ? ul0 : u[i - 1];
        const Real ur = i == 3 ? ur3 : u[i + 1];
        if constexpr (FORM == kCanonical) {
            out_u[i] = rfma(c2, radd(ul, ur), rfma(k, u[i], -w[i]));
        } else {
            const Real v = rfma(c2, rsub(rsub(ur, u[i]), rsub(u[i], ul)), w[i]);
            out_w[i] = v;
            out_u[i] = radd(u[i], v);
        }
    }
    // Dirichlet nodes and points past the end of the grid
    if (j0 == 0 || j0 + 3 >= p.nx - 1) {
        const Real fa_old = p.fA ? p.fA[p.n] : Real(0), fa_new = p.fA ? p.fA[p.n + 1] : Real(0);
        const Real fb_old = p.fB ? p.fB[p.n] : Real(0), fb_new = p.fB ? p.fB[p.n + 1] : Real(0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t j = j0 + i;
            if (j == 0) {
                out_u[i] = fa_new;
                if constexpr (FORM == kIncrement) out_w[i] = rsub(fa_new, fa_old);
            } else if (j == p.nx - 1) {
                out_u[i] = fb_new;
                if constexpr (FORM == kIncrement) out_w[i] = rsub(fb_new, fb_old);
            } else if (j > p.nx - 1) {
                out_u[i] = Real(0);
                if constexpr (FORM == kIncrement) out_w[i] = Real(0);
            }
        }
    }
    // user point sources of this block's points, in the caller's order per point
    if (p.blk_src) {
        const int q1 = p.blk_src[blockIdx.x + 1];
        for (int q = p.blk_src[blockIdx.x]; q < q1; ++q) {
            const SrcDev<Real> sd = p.srcs[q];
            const int64_t r = sd.j - j0;
            if (r < 0 || r >= 4) continue;
            const Real sv = sd.samples[p.n + 1];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (i != r) continue;
                if constexpr (FORM == kCanonical) {
                    out_u[i] = radd(out_u[i], sv);
                } else {
                    out_w[i] = radd(out_w[i], sv);
                    out_u[i] = radd(u[i], out_w[i]);
                }
            }
        }
    }
    if constexpr (FORM == kCanonical) {
        V4<Real>::store(p.prev + g, out_u);  // u^{n+1} replaces u^{n-1}
    } else {
        V4<Real>::store(p.prev + g, out_w);  // v in place
        V4<Real>::store(p.unew + g, out_u);
    }
}

template <typename Real>
__global__ void probe_final_kernel(const ProbeDev<Real>* probes, int nprobe, const Real* u, int64_t level)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nprobe) probe_one(probes[i], u, level);
}

// Level 0: boundary nodes take the Dirichlet samples at t = 0; the second
// component there is "at rest" (canonical u^{-1} = u^0, increment v^0 = 0).
template <typename Real>
__global__ void set_boundary_kernel(Real* q0, Real* q1, const ProblemDev<Real>* problems, int nprob, int form)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    const ProblemDev<Real> pr = problems[p];
    const Real a = pr.fA ? pr.fA[0] : Real(0);
    const Real b = pr.fB ? pr.fB[0] : Real(0);
    q0[pr.base] = a;
    q0[pr.base + pr.nx - 1] = b;
    q1[pr.base] = form == kCanonical ? a : Real(0);
    q1[pr.base + pr.nx - 1] = form == kCanonical ? b : Real(0);
}

}  // namespace

cudaError_t mono_launch(int dtype, const void* params, cudaStream_t s)
{
    void* args[] = {const_cast<void*>(params)};
    int64_t nx;
    int form;
    const void* fn;
    if (dtype == kF32) {
        const auto* p = static_cast<const MonoParams<float>*>(params);
        nx = p->nx;
        form = p->form;
        fn = form == kCanonical ? reinterpret_cast<const void*>(&mono_step_kernel<float, kCanonical>)
                                : reinterpret_cast<const void*>(&mono_step_kernel<float, kIncrement>);
    } else {
        const auto* p = static_cast<const MonoParams<double>*>(params);
        nx = p->nx;
        form = p->form;
        fn = form == kCanonical ? reinterpret_cast<const void*>(&mono_step_kernel<double, kCanonical>)
                                : reinterpret_cast<const void*>(&mono_step_kernel<double, kIncrement>);
    }
    const int64_t groups = (nx + 3) / 4;
    const int grid = (int)((groups + 255) / 256);
    return cudaLaunchKernel(fn, dim3(grid), dim3(256), args, 0, s);
}

cudaError_t probe_final_launch(int dtype, const void* probes, int nprobe, const void* q0, int64_t level,
                               cudaStream_t s)
{
    if (nprobe <= 0) return cudaSuccess;
    const int grid = (nprobe + 127) / 128;
    if (dtype == kF32)
        probe_final_kernel<float><<<grid, 128, 0, s>>>(static_cast<const ProbeDev<float>*>(probes), nprobe,
                                                        static_cast<const float*>(q0), level);
    else
        probe_final_kernel<double><<<grid, 128, 0, s>>>(static_cast<const ProbeDev<double>*>(probes), nprobe,
                                                         static_cast<const double*>(q0), level);
    return cudaGetLastError();
}

cudaError_t set_boundary_launch(int dtype, int form, void* q0, void* q1, const void* problems, int nprob,
                                cudaStream_t s)
{
    const int grid = (nprob + 127) / 128;
    if (dtype == kF32)
        set_boundary_kernel<float><<<grid, 128, 0, s>>>(static_cast<float*>(q0), static_cast<float*>(q1),
                                                         static_cast<const ProblemDev<float>*>(problems), nprob,
                                                         form);
    else
        set_boundary_kernel<double><<<grid, 128, 0, s>>>(static_cast<double*>(q0), static_cast<double*>(q1),
                                                          static_cast<const ProblemDev<double>*>(problems), nprob,
                                                          form);
    return cudaGetLastError();
}

}  // namespace rswr
