// span_common.cuh -- device functions shared by the span kernel and the
// adjoint kernel: register <-> shared-memory staging, the halo exchange, the
// leapfrog step in the library's fixed operation order, boundary / source
// patches and the per-level probes.
#pragma once

#include <type_traits>

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
// BAR: the barrier the window's warps share (block_sync).
template <typename Real, int P, int NW, int BAR = 0>
__device__ __forceinline__ void exchange(const Real (&u)[P], Real& lft, Real& rgt, Real* xch, int buf, int warp,
                                         int lane)
{
    lft = __shfl_up_sync(kFull, u[P - 1], 1);
    rgt = __shfl_down_sync(kFull, u[0], 1);
    Real* slot = xch + buf * NW * 2;
    if (lane == 0) slot[warp * 2 + 0] = u[0];
    if (lane == 31) slot[warp * 2 + 1] = u[P - 1];
    block_sync<BAR>();
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

// Per-level samples (boundary waveforms, point sources) of a span held across a
// warp: lane l keeps the samples of steps base + l (c0) and base + 32 + l (c1);
// the caller reloads c1 32 steps before it is needed, so the step loop never
// waits on global memory for them.  Only these two values per stream live
// across steps.  Every call is made by all lanes of the warp with the same
// arguments.
template <typename Real>
struct WarpChunk {
    Real c0, c1;
    // the sample of step base + d, 0 <= d <= 32
    __device__ __forceinline__ Real get(int d) const
    {
        const Real v0 = __shfl_sync(kFull, c0, d & 31);
        const Real v1 = __shfl_sync(kFull, c1, d & 31);
        return d < 32 ? v0 : v1;
    }
};

// a[level * stride] for 0 <= level <= nmax, else 0
template <typename Real>
__device__ __forceinline__ Real level_sample(const Real* a, int64_t stride, int64_t level, int64_t nmax)
{
    return (a != nullptr && level >= 0 && level <= nmax) ? a[level * stride] : Real(0);
}

// Points of a thread that need more than the stencil (register index, -1 = not
// held): the Dirichlet nodes (r0: j = 0, r1: j = nx-1), the point source (rs)
// and the two points outside the grid next to the nodes (rm: j = -1, rp: j = nx).
// Every other point outside [0, nx) keeps the value 0 by itself: it starts at 0
// (state arrays and pads are zeroed) and so do its neighbours, and a 3-point
// update of zeros is an exact 0 in both forms.  Only rm and rp, whose update
// reads a node, are reset after each step, so outside points stay 0 and never
// reach a grid point.
struct Special {
    int r0, r1, rs, rm, rp;
};

// The special points among the P points from problem coordinate lo on.
template <int P>
__device__ __forceinline__ Special make_special(int64_t lo, int64_t nx, int64_t js)
{
    auto loc = [&](int64_t j) -> int { return (j >= lo && j < lo + P) ? (int)(j - lo) : -1; };
    return Special{loc(0), loc(nx - 1), js >= 0 ? loc(js) : -1, loc(-1), loc(nx)};
}

__device__ __forceinline__ bool any_special(const Special& sp)
{
    return sp.r0 >= 0 || sp.r1 >= 0 || sp.rs >= 0 || sp.rm >= 0 || sp.rp >= 0;
}

// f(I) on register I = r of a register array (I a compile-time constant), by a
// binary tree of branches over r: log2(P) compares instead of one per register.
template <int P, int LO = 0, int HI = P, typename F>
__device__ __forceinline__ void reg_apply(int r, F&& f)
{
    if constexpr (HI - LO == 1) {
        f(std::integral_constant<int, LO>{});
    } else {
        constexpr int MID = (LO + HI) / 2;
        if (r < MID) reg_apply<P, LO, MID>(r, f);
        else reg_apply<P, MID, HI>(r, f);
    }
}

// f(I) on register I = r through a switch (a jump table: one indirect branch
// instead of a tree of compares, which the compiler may turn into predicated
// code that every lane executes); registers 1 .. P-2 only, P <= 32.
template <int P, typename F>
__device__ __forceinline__ void reg_switch(int r, F&& f)
{
    static_assert(P <= 32, "reg_switch covers 32 registers");
#define RSWR_CASE(i)                                                     \
    case i:                                                              \
        if constexpr (i > 0 && i < P - 1) f(std::integral_constant<int, i>{}); \
        break;
    switch (r) {
        RSWR_CASE(1) RSWR_CASE(2) RSWR_CASE(3) RSWR_CASE(4) RSWR_CASE(5) RSWR_CASE(6) RSWR_CASE(7) RSWR_CASE(8)
        RSWR_CASE(9) RSWR_CASE(10) RSWR_CASE(11) RSWR_CASE(12) RSWR_CASE(13) RSWR_CASE(14) RSWR_CASE(15)
        RSWR_CASE(16) RSWR_CASE(17) RSWR_CASE(18) RSWR_CASE(19) RSWR_CASE(20) RSWR_CASE(21) RSWR_CASE(22)
        RSWR_CASE(23) RSWR_CASE(24) RSWR_CASE(25) RSWR_CASE(26) RSWR_CASE(27) RSWR_CASE(28) RSWR_CASE(29)
        RSWR_CASE(30)
        default:
            break;
    }
#undef RSWR_CASE
}

template <typename Real, int P>
__device__ __forceinline__ Real reg_get(const Real (&u)[P], int r)
{
    Real v = Real(0);
    reg_apply<P>(r, [&](auto I) { v = u[decltype(I)::value]; });
    return v;
}

// Applied right after leap_step to the thread's special points (step n -> n+1):
//   source:    canonical u' += s;  increment v' += s, u' = u_old + v'
//   Dirichlet: u' = f(n+1);  increment v' = f(n+1) - f(n)  (canonical keeps u_prev = f(n))
//   j = -1, j = nx: u' = 0, second component 0
template <typename Real, int FORM, int P>
__device__ __forceinline__ void patch_special(Real (&u)[P], Real (&w)[P], const Special& sp, Real uold_s, Real sval,
                                              Real fa_old, Real fa_new, Real fb_old, Real fb_new)
{
    if (sp.rs >= 0)
        reg_apply<P>(sp.rs, [&](auto I) {
            constexpr int i = decltype(I)::value;
            if constexpr (FORM == kIncrement) {
                w[i] = radd(w[i], sval);
                u[i] = radd(uold_s, w[i]);
            } else {
                u[i] = radd(u[i], sval);
            }
        });
    // a node and its outside neighbour: the same register tree; the neighbour
    // sits in the next lane over when the node is the thread's first / last point
    if (sp.r0 >= 0)
        reg_apply<P>(sp.r0, [&](auto I) {
            constexpr int i = decltype(I)::value;
            u[i] = fa_new;
            if constexpr (FORM == kIncrement) w[i] = rsub(fa_new, fa_old);
            if constexpr (i > 0) {
                u[i - 1] = Real(0);
                w[i - 1] = Real(0);
            }
        });
    else if (sp.rm == P - 1) {
        u[P - 1] = Real(0);
        w[P - 1] = Real(0);
    }
    if (sp.r1 >= 0)
        reg_apply<P>(sp.r1, [&](auto I) {
            constexpr int i = decltype(I)::value;
            u[i] = fb_new;
            if constexpr (FORM == kIncrement) w[i] = rsub(fb_new, fb_old);
            if constexpr (i < P - 1) {
                u[i + 1] = Real(0);
                w[i + 1] = Real(0);
            }
        });
    else if (sp.rp == 0) {
        u[0] = Real(0);
        w[0] = Real(0);
    }
}

// One point source at register r after a step: the sample s is added to the
// new value (canonical form) or to the new increment, which then re-forms the
// value from the level-n value uold (increment form).
template <typename Real, int FORM, int P>
__device__ __forceinline__ void add_source_at(Real (&u)[P], Real (&w)[P], int r, Real s, Real uold)
{
    reg_apply<P>(r, [&](auto I) {
        constexpr int i = decltype(I)::value;
        if constexpr (FORM == kIncrement) {
            w[i] = radd(w[i], s);
            u[i] = radd(uold, w[i]);
        } else {
            u[i] = radd(u[i], s);
        }
    });
}

// The same step as exchange() + leap_step(), reordered to hide the halo
// latency: the thread posts its edge values (shuffles + shared slots), updates
// its interior points 1..P-2, waits at the block barrier, then fetches the
// cross-warp halos and updates points 0 and P-1.  Every update is the same
// expression on the same operands as leap_step(), so the bits are identical.
template <typename Real, int FORM, int P, int NW, int BAR = 0>
__device__ __forceinline__ void split_step(Real (&u)[P], Real (&w)[P], Real c2, Real k, Real* xch, int buf,
                                           int warp, int lane)
{
    static_assert(P >= 3, "split step needs interior points");
    Real lft = __shfl_up_sync(kFull, u[P - 1], 1);
    Real rgt = __shfl_down_sync(kFull, u[0], 1);
    Real* slot = xch + buf * NW * 2;
    if (lane == 0) slot[warp * 2 + 0] = u[0];
    if (lane == 31) slot[warp * 2 + 1] = u[P - 1];
    const Real m_l = u[1];      // mirror ghosts at the window ends (zero-flux guess)
    const Real m_r = u[P - 2];
    if constexpr (FORM == kIncrement) {
        const Real d0 = rsub(u[1], u[0]);
        Real dprev = d0;
#pragma unroll
        for (int i = 1; i < P - 1; ++i) {
            const Real d = rsub(u[i + 1], u[i]);
            const Real v = rfma(c2, rsub(d, dprev), w[i]);
            dprev = d;
            w[i] = v;
            u[i] = radd(u[i], v);
        }
        block_sync<BAR>();
        if (lane == 0) lft = (warp > 0) ? slot[(warp - 1) * 2 + 1] : m_l;
        if (lane == 31) rgt = (warp < NW - 1) ? slot[(warp + 1) * 2 + 0] : m_r;
        {
            const Real v = rfma(c2, rsub(d0, rsub(u[0], lft)), w[0]);
            w[0] = v;
            u[0] = radd(u[0], v);
        }
        {
            const Real v = rfma(c2, rsub(rsub(rgt, u[P - 1]), dprev), w[P - 1]);
            w[P - 1] = v;
            u[P - 1] = radd(u[P - 1], v);
        }
    } else {
        const Real u0 = u[0], uP1 = u[P - 1];
        Real ul = u0;
#pragma unroll
        for (int i = 1; i < P - 1; ++i) {
            const Real uc = u[i];
            const Real un = rfma(c2, radd(ul, u[i + 1]), rfma(k, uc, -w[i]));
            w[i] = uc;
            u[i] = un;
            ul = uc;
        }
        block_sync<BAR>();
        if (lane == 0) lft = (warp > 0) ? slot[(warp - 1) * 2 + 1] : m_l;
        if (lane == 31) rgt = (warp < NW - 1) ? slot[(warp + 1) * 2 + 0] : m_r;
        u[0] = rfma(c2, radd(lft, m_l), rfma(k, u0, -w[0]));
        w[0] = u0;
        u[P - 1] = rfma(c2, radd(ul, rgt), rfma(k, uP1, -w[P - 1]));
        w[P - 1] = uP1;
    }
}

// Interface output waveforms and receiver samples of level n (recorded before
// the step that leaves level n).  Only the owner thread of a point writes: the
// thread whose first point sits at window index tb, registers [rlo, rhi).
template <typename Real, int P>
__device__ __forceinline__ void record_probes(const Real (&u)[P], Real lft, Real rgt, int64_t wabs, int tb, int rlo,
                                              int rhi, int pb, int pe, const ProbeDev<Real>* probes, int64_t n)
{
    for (int q = pb; q < pe; ++q) {
        const int64_t li = probes[q].gidx - wabs - (int64_t)tb;
        if (li < rlo || li >= rhi) continue;
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

// A tile's probes staged in shared memory once per tile; each thread keeps the
// indices of (at most two) probes whose point it owns.
constexpr int kTileProbes = 16;

template <typename Real, int P>
__device__ __forceinline__ void owned_probes(const ProbeDev<Real>* sp, int np, int64_t wabs, int tb, int rlo, int rhi,
                                             int& q0, int& q1)
{
    q0 = -1;
    q1 = -1;
    for (int q = 0; q < np; ++q) {
        const int64_t li = sp[q].gidx - wabs - (int64_t)tb;
        if (li >= rlo && li < rhi) {
            if (q0 < 0) q0 = q;
            else q1 = q;
        }
    }
}

// u[r-1], u[r], u[r+1] of a register index r known only at run time: a
// binary tree of branches on r (log2 P compares, then three moves) instead of
// P-way selects; only the owner thread of a probe takes it.
template <typename Real, int P, int LO, int HI>
__device__ __forceinline__ void pick3(const Real (&u)[P], Real lft, Real rgt, int r, Real& um, Real& uc, Real& up)
{
    if constexpr (HI - LO == 1) {
        uc = u[LO];
        um = LO > 0 ? u[LO > 0 ? LO - 1 : 0] : lft;
        up = LO < P - 1 ? u[LO < P - 1 ? LO + 1 : P - 1] : rgt;
    } else {
        constexpr int MID = (LO + HI) / 2;
        if (r < MID) pick3<Real, P, LO, MID>(u, lft, rgt, r, um, uc, up);
        else pick3<Real, P, MID, HI>(u, lft, rgt, r, um, uc, up);
    }
}

template <typename Real, int P>
__device__ __forceinline__ void record_owned(const Real (&u)[P], Real lft, Real rgt, const ProbeDev<Real>& pr,
                                             int64_t wabs, int tb, int64_t n)
{
    const int r = (int)(pr.gidx - wabs - (int64_t)tb);
    Real um, uc, up;
    pick3<Real, P, 0, P>(u, lft, rgt, r, um, uc, up);
    Real val = (pr.kind == 0) ? uc : rsub(up, um);
    val = rmul(val, pr.scale);
    if (n <= pr.nmax) pr.out[n * pr.stride] = val;
}

// A probe owned by this thread, prepared once per tile: `ptr` is the output
// of the current level and advances by `stride` every step; `count` levels of
// the span are recorded (the probe stops at its nmax).
template <typename Real>
struct OwnedProbe {
    Real* ptr;
    int64_t stride;
    Real scale;
    int r;       // register index of the probed point
    int kind;    // 0: u_j, 1: u_{j+1} - u_{j-1}
    int count;
};

template <typename Real>
__device__ __forceinline__ OwnedProbe<Real> own_probe(const ProbeDev<Real>& pr, int64_t wabs, int tb, int64_t n0,
                                                      int steps)
{
    OwnedProbe<Real> o;
    o.r = (int)(pr.gidx - wabs - (int64_t)tb);
    o.kind = pr.kind;
    o.scale = pr.scale;
    o.stride = pr.stride;
    const int64_t c = pr.nmax - n0 + 1;
    o.count = c < 0 ? 0 : (c > steps ? steps : (int)c);
    o.ptr = o.count > 0 ? pr.out + n0 * pr.stride : pr.out;
    return o;
}

// Records level n0 + s (called once per step, s = 0, 1, ...).
template <typename Real, int P>
__device__ __forceinline__ void record_step(OwnedProbe<Real>& o, const Real (&u)[P], Real lft, Real rgt, int s)
{
    if (s < o.count) {
        Real um, uc, up;
        pick3<Real, P, 0, P>(u, lft, rgt, o.r, um, uc, up);
        const Real val = (o.kind == 0) ? uc : rsub(up, um);
        *o.ptr = rmul(val, o.scale);
        o.ptr += o.stride;
    }
}

// Overlapping warp windows (KH > 0): warp w covers window points
// [w (32P - 2KH), w (32P - 2KH) + 32P) and owns all but KH points at each end.
// Every KH steps the halo points are refreshed from the neighbours' owned
// points through shared memory (double-buffered slots, one block barrier);
// in between, warps advance with shuffles only and the contamination from
// their window ends stays inside the halos.
template <typename Real, int P, int NW, int KH, int BAR = 0>
__device__ __forceinline__ void refresh_halos(Real (&u)[P], Real (&w)[P], Real* hx, int buf, int warp, int lane)
{
    static_assert(P >= 2 * KH, "a thread must hold a halo and the owned points next to it");
    using V = typename Vec<Real, P>::T;
    constexpr int N = Vec<Real, P>::N;
    static_assert(KH % N == 0, "halo width must fill whole vectors");
    // slots: [buffer][warp][side: 0 = first owned, 1 = last owned][component][KH], vector aligned
    Real* b = hx + buf * NW * 4 * KH;
    if (lane == 0 || lane == 31) {
        const int side = lane == 0 ? 0 : 1;
        V* su = reinterpret_cast<V*>(b + ((warp * 2 + side) * 2 + 0) * KH);
        V* sw = reinterpret_cast<V*>(b + ((warp * 2 + side) * 2 + 1) * KH);
#pragma unroll
        for (int k = 0; k < KH / N; ++k) {
            V vu, vw;
            const int o = (lane == 0) ? KH + k * N : P - 2 * KH + k * N;
            if constexpr (N == 4) {
                vu = lane == 0 ? V{u[KH + 4 * k], u[KH + 4 * k + 1], u[KH + 4 * k + 2], u[KH + 4 * k + 3]}
                               : V{u[P - 2 * KH + 4 * k], u[P - 2 * KH + 4 * k + 1], u[P - 2 * KH + 4 * k + 2],
                                   u[P - 2 * KH + 4 * k + 3]};
                vw = lane == 0 ? V{w[KH + 4 * k], w[KH + 4 * k + 1], w[KH + 4 * k + 2], w[KH + 4 * k + 3]}
                               : V{w[P - 2 * KH + 4 * k], w[P - 2 * KH + 4 * k + 1], w[P - 2 * KH + 4 * k + 2],
                                   w[P - 2 * KH + 4 * k + 3]};
            } else {
                vu = lane == 0 ? V{u[KH + 2 * k], u[KH + 2 * k + 1]} : V{u[P - 2 * KH + 2 * k], u[P - 2 * KH + 2 * k + 1]};
                vw = lane == 0 ? V{w[KH + 2 * k], w[KH + 2 * k + 1]} : V{w[P - 2 * KH + 2 * k], w[P - 2 * KH + 2 * k + 1]};
            }
            (void)o;
            su[k] = vu;
            sw[k] = vw;
        }
    }
    block_sync<BAR>();
    if ((lane == 0 && warp > 0) || (lane == 31 && warp < NW - 1)) {
        const int src = lane == 0 ? ((warp - 1) * 2 + 1) : ((warp + 1) * 2 + 0);
        const V* su = reinterpret_cast<const V*>(b + (src * 2 + 0) * KH);
        const V* sw = reinterpret_cast<const V*>(b + (src * 2 + 1) * KH);
#pragma unroll
        for (int k = 0; k < KH / N; ++k) {
            const V vu = su[k], vw = sw[k];
            if (lane == 0) {
                if constexpr (N == 4) {
                    u[4 * k] = vu.x; u[4 * k + 1] = vu.y; u[4 * k + 2] = vu.z; u[4 * k + 3] = vu.w;
                    w[4 * k] = vw.x; w[4 * k + 1] = vw.y; w[4 * k + 2] = vw.z; w[4 * k + 3] = vw.w;
                } else {
                    u[2 * k] = vu.x; u[2 * k + 1] = vu.y;
                    w[2 * k] = vw.x; w[2 * k + 1] = vw.y;
                }
            } else {
                if constexpr (N == 4) {
                    u[P - KH + 4 * k] = vu.x; u[P - KH + 4 * k + 1] = vu.y; u[P - KH + 4 * k + 2] = vu.z;
                    u[P - KH + 4 * k + 3] = vu.w;
                    w[P - KH + 4 * k] = vw.x; w[P - KH + 4 * k + 1] = vw.y; w[P - KH + 4 * k + 2] = vw.z;
                    w[P - KH + 4 * k + 3] = vw.w;
                } else {
                    u[P - KH + 2 * k] = vu.x; u[P - KH + 2 * k + 1] = vu.y;
                    w[P - KH + 2 * k] = vw.x; w[P - KH + 2 * k + 1] = vw.y;
                }
            }
        }
    }
}

// Neighbour values inside a warp window (shuffles; mirror ghost at its ends).
template <typename Real, int P>
__device__ __forceinline__ void warp_neighbours(const Real (&u)[P], Real& lft, Real& rgt, int lane)
{
    lft = __shfl_up_sync(kFull, u[P - 1], 1);
    rgt = __shfl_down_sync(kFull, u[0], 1);
    if (lane == 0) lft = u[1];
    if (lane == 31) rgt = u[P - 2];
}

// `steps` leapfrog steps of a warp window (neighbours by shuffles, mirror
// ghosts at the window's ends) in the order: the thread's two end points, the
// shuffles of their new values for the next step, then the interior points,
// so that the shuffle latency hides behind the interior updates.  Every update
// is the same expression on the same operands as leap_step(), so the bits are
// identical.  `rec(u, lft, rgt, s)` sees every level s = 0 .. steps-1 with its
// neighbours before it is advanced (probe recording; it must not shuffle).
struct NoRecord {
    template <typename U, typename Real>
    __device__ __forceinline__ void operator()(const U&, Real, Real, int) const {}
};

// Special points in the edges-first loop (Dirichlet nodes, a point source, the
// outside points next to the nodes; see patch_special): pre(u, s) runs before
// step s (samples, level-n values), edges(u, n0, v0, nl, vl) patches the new
// values of the thread's first and last register before they are shuffled,
// interior(u, w) the registers in between after their update.
struct NoPatch {
    template <typename U>
    __device__ __forceinline__ void pre(const U&, int) {}
    template <typename U, typename Real>
    __device__ __forceinline__ void edges(const U&, Real&, Real&, Real&, Real&) {}
    template <typename U>
    __device__ __forceinline__ void interior(U&, U&) {}
};

template <typename Real, int FORM, int P, typename Rec = NoRecord, typename Patch = NoPatch>
__device__ __forceinline__ void warp_steps_edges_first(Real (&u)[P], Real (&w)[P], Real c2, Real k, int steps,
                                                       int lane, Rec rec = Rec{}, Patch patch = Patch{})
{
    static_assert(P >= 3, "edges-first order needs interior points");
    Real lft, rgt;
    warp_neighbours<Real, P>(u, lft, rgt, lane);
    for (int s = 0; s < steps; ++s) {
        rec(u, lft, rgt, s);
        patch.pre(u, s);
        Real n0, nl, v0, vl;  // new first / last point and their second components
        Real d0 = Real(0);
        if constexpr (FORM == kIncrement) {
            d0 = rsub(u[1], u[0]);
            const Real dm = rsub(u[P - 1], u[P - 2]);
            v0 = rfma(c2, rsub(d0, rsub(u[0], lft)), w[0]);
            vl = rfma(c2, rsub(rsub(rgt, u[P - 1]), dm), w[P - 1]);
            n0 = radd(u[0], v0);
            nl = radd(u[P - 1], vl);
        } else {
            n0 = rfma(c2, radd(lft, u[1]), rfma(k, u[0], -w[0]));
            v0 = u[0];
            nl = rfma(c2, radd(u[P - 2], rgt), rfma(k, u[P - 1], -w[P - 1]));
            vl = u[P - 1];
        }
        patch.edges(u, n0, v0, nl, vl);
        Real nlft = __shfl_up_sync(kFull, nl, 1);
        Real nrgt = __shfl_down_sync(kFull, n0, 1);
        if constexpr (FORM == kIncrement) {
            Real dprev = d0;
#pragma unroll
            for (int i = 1; i < P - 1; ++i) {
                const Real d = rsub(u[i + 1], u[i]);
                const Real v = rfma(c2, rsub(d, dprev), w[i]);
                dprev = d;
                w[i] = v;
                u[i] = radd(u[i], v);
            }
        } else {
            Real ul = u[0];
#pragma unroll
            for (int i = 1; i < P - 1; ++i) {
                const Real uc = u[i];
                const Real un = rfma(c2, radd(ul, u[i + 1]), rfma(k, uc, -w[i]));
                w[i] = uc;
                u[i] = un;
                ul = uc;
            }
        }
        u[0] = n0;
        w[0] = v0;
        u[P - 1] = nl;
        w[P - 1] = vl;
        patch.interior(u, w);
        if (lane == 0) nlft = u[1];
        if (lane == 31) nrgt = u[P - 2];
        lft = nlft;
        rgt = nrgt;
    }
}

// The patch of the special points for warp_steps_edges_first, with the same
// effect as leap_step + patch_special: a register takes, in this order, the
// source (canonical u' += s; increment v' += s, u' = u_old + v'), the left node
// (u' = f_A(n+1); increment v' = f_A(n+1) - f_A(n)), the outside point next to
// it (0, 0), the right node, the outside point next to it.  Samples come from
// the warp's chunks (f_A / f_B at level n0 + d, the source at level n0 + d + 1).
// Whether a special point of the thread sits between its first and last
// register (the register trees of EdgePatch::interior are needed).
template <int P>
__device__ __forceinline__ bool interior_special(const Special& sp)
{
    auto in = [](int r) { return r > 0 && r < P - 1; };
    return in(sp.rs) || in(sp.r0) || in(sp.rm) || in(sp.r1) || in(sp.rp);
}

// INTERIOR = false: every special point of the warp sits on a thread's first
// or last register, so interior() has nothing to do and is compiled out (the
// register trees, which the compiler turns into predicated code that every lane
// executes each step, are what make the patched loop slow).
template <typename Real, int FORM, int P, typename Reload, bool INTERIOR = true>
struct EdgePatch {
    Special sp;
    WarpChunk<Real>* ca;
    WarpChunk<Real>* cb;
    WarpChunk<Real>* cs;
    bool wa, wb, wsrc;
    int* cbase;       // first step of the current chunk
    Reload* reload;   // reload(first): loads the chunk after the one starting at `first`
    Real fa_old, fa_new, fb_old, fb_new, sval, uold_s;
    int d;

    template <typename U>
    __device__ __forceinline__ void pre(const U& u, int s)
    {
        step_samples(s);
        capture(u);
    }
    __device__ __forceinline__ void step_samples(int s)
    {
        d = s - *cbase;
        if (d == 32) {
            *cbase += 32;
            ca->c0 = ca->c1;
            cb->c0 = cb->c1;
            cs->c0 = cs->c1;
            (*reload)(*cbase, false);
            d = 0;
        }
        fa_old = fa_new = fb_old = fb_new = sval = Real(0);
        if (wsrc) sval = cs->get(d);
        if (wa) {
            fa_old = ca->get(d);
            fa_new = ca->get(d + 1);
        }
        if (wb) {
            fb_old = cb->get(d);
            fb_new = cb->get(d + 1);
        }
    }
    __device__ __forceinline__ void at(int i, Real& x, Real& y)
    {
        if (sp.rs == i) {
            if constexpr (FORM == kIncrement) {
                y = radd(y, sval);
                x = radd(uold_s, y);
            } else {
                x = radd(x, sval);
            }
        }
        if (sp.r0 == i) {
            x = fa_new;
            if constexpr (FORM == kIncrement) y = rsub(fa_new, fa_old);
        }
        if (sp.rm == i) x = y = Real(0);
        if (sp.r1 == i) {
            x = fb_new;
            if constexpr (FORM == kIncrement) y = rsub(fb_new, fb_old);
        }
        if (sp.rp == i) x = y = Real(0);
    }
    template <typename U>
    __device__ __forceinline__ void capture(const U& u)
    {
        // the level-n value of the source point (increment form)
        if constexpr (FORM == kIncrement)
            if (sp.rs >= 0) uold_s = reg_get<Real, P>(u, sp.rs);
    }
    template <typename U>
    __device__ __forceinline__ void edges(const U& u, Real& n0, Real& v0, Real& nl, Real& vl)
    {
        at(0, n0, v0);
        at(P - 1, nl, vl);
    }
    template <typename U>
    __device__ __forceinline__ void interior(U& u, U& w)
    {
        if constexpr (!INTERIOR) return;
        // one jump-table branch per special point held between the end registers
        auto one = [&](int r) {
            if (r > 0 && r < P - 1)
                reg_switch<P>(r, [&](auto I) {
                    constexpr int i = decltype(I)::value;
                    at(i, u[i], w[i]);
                });
        };
        one(sp.rs);
        if (sp.r0 != sp.rs) one(sp.r0);
        one(sp.rm);
        if (sp.r1 != sp.rs) one(sp.r1);
        one(sp.rp);
    }
};

// Write the registers a thread owns, [own_lo, own_hi), back to the shared window.
template <typename Real, int P, int KH>
__device__ __forceinline__ void owned_to_smem(Real* s, const Real (&r)[P], int own_lo, int own_hi)
{
    if (KH == 0 || (own_lo == 0 && own_hi == P)) {
        regs_to_smem<Real, P>(s, r);
    } else {
#pragma unroll
        for (int i = 0; i < P; ++i)
            if (i >= own_lo && i < own_hi) s[i] = r[i];
    }
}

}  // namespace span
}  // namespace rswr
