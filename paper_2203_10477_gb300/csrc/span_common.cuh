// span_common.cuh -- device functions shared by the span kernel and the
// adjoint kernel: register <-> shared-memory staging, the halo exchange, the
// leapfrog step in the library's fixed operation order, boundary / source
// patches and the per-level probes.
#pragma once

#include "rswr_internal.h"

namespace rswr {
namespace span {

constexpr unsigned kFull = 0xffffffffu;

template <typename Real, int P>
struct Vec;
template <int P>
struct Vec<float, P> {
    static constexpr int N = 4;
    using T = float4;
};
template <int P>
struct Vec<double, P> {
    static constexpr int N = 2;
    using T = double2;
};

template <typename Real, int P>
__device__ __forceinline__ void smem_to_regs(const Real* s, Real (&r)[P])
{
    using V = typename Vec<Real, P>::T;
    constexpr int N = Vec<Real, P>::N;
    static_assert(P % N == 0, "points per thread must fill whole vectors");
    const V* sv = reinterpret_cast<const V*>(s);
#pragma unroll
    for (int i = 0; i < P / N; ++i) {
        V v = sv[i];
        if constexpr (N == 4) {
            r[4 * i + 0] = v.x;
            r[4 * i + 1] = v.y;
            r[4 * i + 2] = v.z;
            r[4 * i + 3] = v.w;
        } else {
            r[2 * i + 0] = v.x;
            r[2 * i + 1] = v.y;
        }
    }
}

template <typename Real, int P>
__device__ __forceinline__ void regs_to_smem(Real* s, const Real (&r)[P])
{
    using V = typename Vec<Real, P>::T;
    constexpr int N = Vec<Real, P>::N;
    V* sv = reinterpret_cast<V*>(s);
#pragma unroll
    for (int i = 0; i < P / N; ++i) {
        V v;
        if constexpr (N == 4) {
            v.x = r[4 * i + 0];
            v.y = r[4 * i + 1];
            v.z = r[4 * i + 2];
            v.w = r[4 * i + 3];
        } else {
            v.x = r[2 * i + 0];
            v.y = r[2 * i + 1];
        }
        sv[i] = v;
    }
}

// Neighbour values of the thread's first and last point: warp shuffles inside
// a warp, one shared slot per warp edge across warps.  At the two window ends
// the ghost mirrors the interior neighbour (zero-flux prediction guess).
template <typename Real, int P, int NW>
__device__ __forceinline__ void exchange(const Real (&u)[P], Real& lft, Real& rgt, Real* xch, int buf, int warp,
                                         int lane)
{
    lft = __shfl_up_sync(kFull, u[P - 1], 1);
    rgt = __shfl_down_sync(kFull, u[0], 1);
    Real* slot = xch + buf * NW * 2;
    if (lane == 0) slot[warp * 2 + 0] = u[0];
    if (lane == 31) slot[warp * 2 + 1] = u[P - 1];
    __syncthreads();
    if (lane == 0) lft = (warp > 0) ? slot[(warp - 1) * 2 + 1] : u[1];
    if (lane == 31) rgt = (warp < NW - 1) ? slot[(warp + 1) * 2 + 0] : u[P - 2];
}

// One leapfrog step of the thread's P points in the library's fixed order:
//   canonical: u' = fma(c2, uL + uR, fma(k, u, -u_prev))
//   increment: v' = fma(c2, (uR - u) - (u - uL), v);  u' = u + v'
// ((uL - u) + (uR - u) equals (uR - u) - (u - uL) bit for bit.)
template <typename Real, int FORM, int P>
__device__ __forceinline__ void leap_step(Real (&u)[P], Real (&w)[P], Real lft, Real rgt, Real c2, Real k)
{
    if constexpr (FORM == kIncrement) {
        Real d_prev = rsub(u[0], lft);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const Real ur = (i < P - 1) ? u[i + 1] : rgt;
            const Real d = rsub(ur, u[i]);
            const Real v = rfma(c2, rsub(d, d_prev), w[i]);
            d_prev = d;
            w[i] = v;
            u[i] = radd(u[i], v);
        }
    } else {
        Real ul = lft;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const Real uc = u[i];
            const Real ur = (i < P - 1) ? u[i + 1] : rgt;
            u[i] = rfma(c2, radd(ul, ur), rfma(k, uc, -w[i]));
            w[i] = uc;
            ul = uc;
        }
    }
}

// Points of a thread that need more than the stencil: the Dirichlet nodes
// (local index r0 -> j = 0, r1 -> j = nx-1), the point source (rs) and points
// outside [0, nx) (local indices outside [rlo, rhi]).  -1 = not owned.
struct Special {
    int r0, r1, rs, rlo, rhi;
};

template <typename Real, int P>
__device__ __forceinline__ Real select_reg(const Real (&u)[P], int r)
{
    Real v = u[0];
#pragma unroll
    for (int i = 1; i < P; ++i)
        if (i == r) v = u[i];
    return v;
}

// Applied right after leap_step to the thread's special points (step n -> n+1):
//   source:    canonical u' += s;  increment v' += s, u' = u_old + v'
//   Dirichlet: u' = f(n+1);  increment v' = f(n+1) - f(n)  (canonical keeps u_prev = f(n))
//   outside:   u' = 0, second component 0
template <typename Real, int FORM, int P>
__device__ __forceinline__ void patch_special(Real (&u)[P], Real (&w)[P], const Special& sp, Real uold_s, Real sval,
                                              Real fa_old, Real fa_new, Real fb_old, Real fb_new)
{
#pragma unroll
    for (int i = 0; i < P; ++i) {
        if (i == sp.rs) {
            if constexpr (FORM == kIncrement) {
                w[i] = radd(w[i], sval);
                u[i] = radd(uold_s, w[i]);
            } else {
                u[i] = radd(u[i], sval);
            }
        }
        if (i == sp.r0) {
            u[i] = fa_new;
            if constexpr (FORM == kIncrement) w[i] = rsub(fa_new, fa_old);
        }
        if (i == sp.r1) {
            u[i] = fb_new;
            if constexpr (FORM == kIncrement) w[i] = rsub(fb_new, fb_old);
        }
        if (i < sp.rlo || i > sp.rhi) {
            u[i] = Real(0);
            w[i] = Real(0);
        }
    }
}

// Interface output waveforms and receiver samples of level n (recorded before
// the step that leaves level n).  Only the owner thread of a point writes.
template <typename Real, int P>
__device__ __forceinline__ void record_probes(const Real (&u)[P], Real lft, Real rgt, int64_t wabs, int tid,
                                              int pb, int pe, const ProbeDev<Real>* probes, int64_t n)
{
    for (int q = pb; q < pe; ++q) {
        const int64_t li = probes[q].gidx - wabs - (int64_t)tid * P;
        if (li < 0 || li >= P) continue;
        const int r = (int)li;
        Real um = lft, uc = u[0], up = rgt;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (i == r) {
                uc = u[i];
                um = (i > 0) ? u[i - 1] : lft;
                up = (i < P - 1) ? u[i + 1] : rgt;
            }
        }
        const ProbeDev<Real> pr = probes[q];
        Real val = (pr.kind == 0) ? uc : rsub(up, um);
        val = rmul(val, pr.scale);
        if (n <= pr.nmax) pr.out[n * pr.stride] = val;
    }
}

}  // namespace span
}  // namespace rswr
