// adjoint_kernel.cu -- one span of the discrete adjoint sweep with the forward
// levels recomputed in shared memory (the gradient workload of the library;
// the paper has no adjoint).
//
// For a receiver trace y^n = u^n_{j_r} and a cotangent wbar = dL/dy, the adjoint
// variables lambda^n = dL/du^n obey the leapfrog backward in time with zero
// Dirichlet data and the source wbar at j_r.  The library runs them forward in
// reversed time (level m = lambda^{T+1-m}).  Their pairing with the forward
// field gives
//     dL/dc2 = sum_n sum_j lambda^{n+1}_j ((u^n_{j-1} + u^n_{j+1}) - 2 u^n_j),
//     dL/da  = dL/dc2 * 2 c2 / a.
// The forward levels come from span-boundary states stored every span of the
// current segment (recomputed from sqrt-spaced checkpoints by the span kernel);
// inside one span this kernel recomputes them in registers and keeps the
// Laplacian of every level of the span in shared memory, then steps lambda and
// accumulates the products on the tile's core.
//
// Per tile: 1-D TMA loads of both state pairs -> u phase (len levels, Laplacians
// to shared memory) -> lambda phase (len steps: dL/dfA probe at j = 1, pairing,
// leapfrog step, source) -> TMA store of lambda's core -> one double per tile
// (block reduction in a fixed order; the host sums tiles and spans in a fixed
// order too, so the result is deterministic).
//
// The FP32 persistent sweep keeps the Laplacians in tensor memory instead
// (TMEM, tmem.cuh): a thread's P values of level s in columns [s P, s P + P) of
// its own lane.  Shared memory then holds only the staged windows, so twice as
// many CTAs fit on an SM; the values and the order of every operation are the
// same, so the results are bit-identical to the shared-memory store.

#include <algorithm>

#include "rswr_internal.h"
#include "span_common.cuh"
#include "tmem.cuh"

namespace rswr {

namespace {

using namespace span;

// Geometry and data of one adjoint tile.
template <typename Real>
struct AdjTile {
    const ProblemDev<Real>* pu;  // forward problem
    const ProblemDev<Real>* pl;  // adjoint problem
    TileDev td;
    int64_t gj0;                 // problem coordinate of the window start
    int64_t n0, m0;              // first forward / adjoint level of the span
    int len;                     // steps of the span
};

// One tile of the adjoint sweep on a staged window (stage[0..1]: the forward
// pair at level n0, stage[2..3]: the adjoint pair at level m0; each thread reads
// and writes only its own P points).  u phase: len forward levels recomputed in
// registers, the Laplacian of each level to `laps`; lambda phase: the probes
// (dL/dfA), the pairing with the Laplacians on the core, len adjoint steps.
// The adjoint pair is written back to stage[2..3].  Returns this thread's part of
// sum lambda^{n+1} lap(u^n).  BAR: the barrier of the window's threads; `buf`
// (the exchange-slot parity) continues across calls so that consecutive
// exchanges always alternate slots.  TM: the Laplacians go to tensor memory at
// tm (this warp's first lane, column 0) instead of `laps`.
template <typename Real, int FORM, int P, int NT, int SA, int BAR, bool TM = false>
__device__ __forceinline__ Real adj_tile(const AdjParams<Real>& prm, const AdjTile<Real>& at, Real* stage, Real* laps,
                                         Real* xch, int& buf, uint32_t tm = 0)
{
    static_assert(!TM || (sizeof(Real) == 4 && P % 8 == 0 && NT == 128),
                  "TMEM store: FP32 words, whole 8-column chunks, one warp per lane quadrant");
    constexpr int W = NT * P;
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const ProblemDev<Real>& pu = *at.pu;
    const ProblemDev<Real>& pl = *at.pl;
    const int64_t nx = pu.nx;
    const int64_t gj0 = at.gj0;
    const int64_t wabs = pu.base + gj0;
    const int64_t gj = gj0 + (int64_t)tid * P;
    const Real c2 = pu.c2, kk = pu.k;
    const bool edge = (gj0 <= 0) || (gj0 + W - 1 >= nx - 1);
    const bool has_src = pl.js >= 0 && pl.js >= gj0 && pl.js < gj0 + W;
    const int len = at.len;
    // layout of the Laplacian store within a level: FP32 point-major across the
    // threads (consecutive threads touch consecutive words: no bank conflicts);
    // FP64 thread-major (a thread's points in 16-byte pieces; the FP64 pipe,
    // not shared memory, bounds this kernel)
    constexpr bool kPointMajor = sizeof(Real) == 4;
    constexpr int lap_stride = kPointMajor ? NT : 1;
    const int lap_base = kPointMajor ? tid : tid * P;

    // ---- u phase: levels n0 .. n0+len-1, Laplacians of every level to shared memory
    {
        Real u[P], w[P];
        smem_to_regs<Real, P>(stage + 0 * W + tid * P, u);
        smem_to_regs<Real, P>(stage + 1 * W + tid * P, w);
        const Special sp = make_special<P>(gj, nx, -1);
        const bool special = edge && any_special(sp);
        // Dirichlet samples of the span through the warp (warp-uniform choices)
        WarpChunk<Real> ca{}, cb{};
        bool wa = false, wb = false;
        int cbase = 0;
        if (edge) {
            wa = __any_sync(kFull, sp.r0 >= 0) && pu.fA != nullptr;
            wb = __any_sync(kFull, sp.r1 >= 0) && pu.fB != nullptr;
            if (wa) {
                ca.c0 = level_sample(pu.fA, 1, at.n0 + lane, prm.T);
                ca.c1 = level_sample(pu.fA, 1, at.n0 + 32 + lane, prm.T);
            }
            if (wb) {
                cb.c0 = level_sample(pu.fB, 1, at.n0 + lane, prm.T);
                cb.c1 = level_sample(pu.fB, 1, at.n0 + 32 + lane, prm.T);
            }
        }
        // one level: its Laplacian to shared memory and (STEP) the step to the
        // next level; the last level of the span only stores its Laplacian
        auto level = [&](auto step_c, int s) {
            constexpr bool STEP = decltype(step_c)::value;
            Real lft, rgt;
            exchange<Real, P, NW, BAR>(u, lft, rgt, xch, buf, warp, lane);
            buf ^= 1;
            [[maybe_unused]] Real* lp = laps + s * W + lap_base;  // point i of this thread at lp[i * lap_stride]
            [[maybe_unused]] Real lv[P];  // TM: the level's Laplacians, stored after the pass
            auto put = [&](int i, Real x) {
                if constexpr (TM) lv[i] = x;
                else lp[i * lap_stride] = x;
            };
            // one pass: the Laplacian of this level (from the step's own neighbour
            // sum, (uL + uR) - 2u = fma(-2, u, uL + uR) exactly) and the step
            if constexpr (FORM == kCanonical) {
                Real ul = lft;
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    const Real uc = u[i];
                    const Real ur = i < P - 1 ? u[i + 1] : rgt;
                    const Real sum = radd(ul, ur);
                    put(i, rfma(Real(-2), uc, sum));
                    if constexpr (STEP) {
                        u[i] = rfma(c2, sum, rfma(kk, uc, -w[i]));
                        w[i] = uc;
                    }
                    ul = uc;
                }
            } else {
                Real d_prev = rsub(u[0], lft);
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    const Real ur = i < P - 1 ? u[i + 1] : rgt;
                    const Real d = rsub(ur, u[i]);
                    const Real lap = rsub(d, d_prev);
                    d_prev = d;
                    put(i, lap);
                    if constexpr (STEP) {
                        const Real v = rfma(c2, lap, w[i]);
                        w[i] = v;
                        u[i] = radd(u[i], v);
                    }
                }
            }
            if constexpr (TM) {
#pragma unroll
                for (int c = 0; c < P / 8; ++c) {
                    uint32_t b[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) b[q] = __float_as_uint(lv[8 * c + q]);
                    tmem_st8(tm + (uint32_t)(s * P + 8 * c), b);
                }
            }
            if constexpr (STEP) {
                // samples through the warp: wa / wb are warp-uniform, so every
                // lane takes part in the shuffles; only the patch is per thread
                if (s - cbase == 32) {
                    cbase += 32;
                    ca.c0 = ca.c1;
                    cb.c0 = cb.c1;
                    if (wa) ca.c1 = level_sample(pu.fA, 1, at.n0 + cbase + 32 + lane, prm.T);
                    if (wb) cb.c1 = level_sample(pu.fB, 1, at.n0 + cbase + 32 + lane, prm.T);
                }
                Real fa_old = Real(0), fa_new = Real(0), fb_old = Real(0), fb_new = Real(0);
                if (wa) {
                    fa_old = ca.get(s - cbase);
                    fa_new = ca.get(s - cbase + 1);
                }
                if (wb) {
                    fb_old = cb.get(s - cbase);
                    fb_new = cb.get(s - cbase + 1);
                }
                if (special)
                    patch_special<Real, FORM, P>(u, w, sp, Real(0), Real(0), fa_old, fa_new, fb_old, fb_new);
            }
        };
        for (int s = 0; s + 1 < len; ++s) level(std::true_type{}, s);
        if (len > 0) level(std::false_type{}, len - 1);
        if constexpr (TM) tmem_wait_st();  // the lambda phase loads what this thread stored
    }

    // ---- lambda phase: levels m0 .. m0+len-1 pair with u levels n0+len-1 .. n0
    Real racc = Real(0);
    Real l[P], lw[P];
    smem_to_regs<Real, P>(stage + 2 * W + tid * P, l);
    smem_to_regs<Real, P>(stage + 3 * W + tid * P, lw);
    const Special sp = make_special<P>(gj, nx, has_src ? pl.js : -1);
    const bool special = (edge || has_src) && any_special(sp);
    // the source samples (cotangent) of the span through the warp: level m0 + 1 + i
    WarpChunk<Real> cs{};
    bool wsrc = false;
    int sbase = 0;
    if (has_src) {
        wsrc = __any_sync(kFull, sp.rs >= 0);
        if (wsrc) {
            cs.c0 = level_sample(pl.src, pl.src_stride, at.m0 + 1 + lane, prm.T);
            cs.c1 = level_sample(pl.src, pl.src_stride, at.m0 + 33 + lane, prm.T);
        }
    }
    // core points that are interior grid points: [jlo, jhi)
    const int64_t core_lo = gj0 + prm.H, core_hi = core_lo + prm.core;
    const int64_t jlo = core_lo > 1 ? core_lo : 1;
    const int64_t jhi = core_hi < nx - 1 ? core_hi : nx - 1;
    // the same range in this thread's register indices
    const int ilo = (int)(jlo - gj <= 0 ? 0 : (jlo - gj >= P ? P : jlo - gj));
    const int ihi = (int)(jhi - gj <= 0 ? 0 : (jhi - gj >= P ? P : jhi - gj));
    for (int s = 0; s < len; ++s) {
        // TM: the pairing level's Laplacians are fetched while the neighbours
        // are exchanged
        uint32_t lb[TM ? P : 1];
        if constexpr (TM) {
#pragma unroll
            for (int c = 0; c < P / 8; ++c)
                tmem_ld8(tm + (uint32_t)((len - 1 - s) * P + 8 * c), *reinterpret_cast<uint32_t(*)[8]>(lb + 8 * c));
        }
        Real lft, rgt;
        exchange<Real, P, NW, BAR>(l, lft, rgt, xch, buf, warp, lane);
        buf ^= 1;
        const int64_t m = at.m0 + s;
        if (at.td.probe_end > at.td.probe_begin)
            record_probes<Real, P>(l, lft, rgt, wabs, tid * P, 0, P, at.td.probe_begin, at.td.probe_end, prm.probes,
                                   m);
        // each thread reads the Laplacians of its own points only
        if constexpr (TM) {
            __syncwarp();
#pragma unroll
            for (int c = 0; c < P / 8; ++c) tmem_wait_ld(*reinterpret_cast<uint32_t(*)[8]>(lb + 8 * c));
#pragma unroll
            for (int i = 0; i < P; ++i)
                if (i >= ilo && i < ihi) racc = rfma(l[i], __uint_as_float(lb[i]), racc);
        } else {
            const Real* lp = laps + (len - 1 - s) * W + lap_base;
#pragma unroll
            for (int i = 0; i < P; ++i)
                if (i >= ilo && i < ihi) racc = rfma(l[i], lp[i * lap_stride], racc);
        }
        Real sval = Real(0);  // src at level m + 1
        if (wsrc) {
            if (s - sbase == 32) {
                sbase += 32;
                cs.c0 = cs.c1;
                cs.c1 = level_sample(pl.src, pl.src_stride, at.m0 + sbase + 33 + lane, prm.T);
            }
            sval = cs.get(s - sbase);
        }
        if (special) {
            // the increment form adds the source to v before u' = u + v: keep u
            const Real uold = (FORM == kIncrement && sp.rs >= 0) ? reg_get<Real, P>(l, sp.rs) : Real(0);
            leap_step<Real, FORM, P>(l, lw, lft, rgt, c2, kk);
            patch_special<Real, FORM, P>(l, lw, sp, uold, sval, Real(0), Real(0), Real(0), Real(0));
        } else {
            leap_step<Real, FORM, P>(l, lw, lft, rgt, c2, kk);
        }
    }
    regs_to_smem<Real, P>(stage + 2 * W + tid * P, l);
    regs_to_smem<Real, P>(stage + 3 * W + tid * P, lw);
    return racc;
}

// Special-point patch of adj_tile_fw, applied after a step (the rules of
// patch_special; the special points of one thread are distinct registers, so
// the order in which they are patched does not matter).  The thread's end
// registers are patched with predicated selects; a special point between them
// takes one jump-table branch (reg_switch) instead of a tree of branches on
// its register index.
template <typename Real, int FORM, int P>
__device__ __forceinline__ void patch_fast(Real (&u)[P], Real (&w)[P], const Special& sp, Real uold_s, Real sval,
                                           Real fa_old, Real fa_new, Real fb_old, Real fb_new)
{
    auto at = [&](int i, Real& x, Real& y) {
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
    };
    at(0, u[0], w[0]);
    at(P - 1, u[P - 1], w[P - 1]);
    auto one = [&](int r) {
        if (r > 0 && r < P - 1)
            reg_switch<P>(r, [&](auto I) {
                constexpr int i = decltype(I)::value;
                at(i, u[i], w[i]);
            });
    };
    one(sp.rs);
    one(sp.r0);
    one(sp.rm);
    one(sp.r1);
    one(sp.rp);
}

// The patch when every special point of the thread sits on an end register in
// the usual way: the left node on register 0 with the outside point j = -1 on
// the previous thread's last register, the right node on register P-1 with
// j = nx on the next thread's register 0, and no source (the persistent
// sweep's tiles start on multiples of P, so the left side always looks like
// this, and the right side whenever nx is a multiple of P).  Selects only;
// fixed_ends() tells whether it applies to a thread.
struct EndPatch {
    bool a0, z0, bl, zl;  // register 0: left node / outside; register P-1: right node / outside
};

template <int P>
__device__ __forceinline__ bool fixed_ends(const Special& sp)
{
    return sp.rs < 0 && (sp.r0 == -1 || sp.r0 == 0) && (sp.rm == -1 || sp.rm == P - 1) &&
           (sp.r1 == -1 || sp.r1 == P - 1) && (sp.rp == -1 || sp.rp == 0);
}

template <typename Real, int FORM, int P>
__device__ __forceinline__ void patch_ends(Real (&u)[P], Real (&w)[P], const EndPatch& ep, Real fa_old, Real fa_new,
                                           Real fb_old, Real fb_new)
{
    if constexpr (FORM == kIncrement) {
        const Real da = rsub(fa_new, fa_old), db = rsub(fb_new, fb_old);
        u[0] = ep.a0 ? fa_new : (ep.z0 ? Real(0) : u[0]);
        w[0] = ep.a0 ? da : (ep.z0 ? Real(0) : w[0]);
        u[P - 1] = ep.bl ? fb_new : (ep.zl ? Real(0) : u[P - 1]);
        w[P - 1] = ep.bl ? db : (ep.zl ? Real(0) : w[P - 1]);
    } else {
        u[0] = ep.a0 ? fa_new : (ep.z0 ? Real(0) : u[0]);
        w[0] = ep.z0 ? Real(0) : w[0];
        u[P - 1] = ep.bl ? fb_new : (ep.zl ? Real(0) : u[P - 1]);
        w[P - 1] = ep.zl ? Real(0) : w[P - 1];
    }
}

// u[r] for a register index known at run time (one jump-table branch).
template <typename Real, int P>
__device__ __forceinline__ Real reg_get_sw(const Real (&u)[P], int r)
{
    Real v = u[0];
    if (r == P - 1) v = u[P - 1];
    else if (r > 0) reg_switch<P>(r, [&](auto I) { v = u[decltype(I)::value]; });
    return v;
}

// The probe sample of level n0 + s (record_step with a jump table).
template <typename Real, int P>
__device__ __forceinline__ void record_sw(OwnedProbe<Real>& o, const Real (&u)[P], Real lft, Real rgt, int s)
{
    if (s < o.count) {
        Real um = lft, uc = u[0], up = u[1];
        if (o.r == 1) {  // the boundary-gradient probe (j = 1 on a tile that starts on a multiple of P)
            um = u[0];
            uc = u[1];
            up = u[2];
        } else if (o.r == P - 1) {
            um = u[P - 2];
            uc = u[P - 1];
            up = rgt;
        } else if (o.r > 0) {
            reg_switch<P>(o.r, [&](auto I) {
                constexpr int i = decltype(I)::value;
                um = u[i - 1];
                uc = u[i];
                up = u[i + 1];
            });
        }
        const Real val = (o.kind == 0) ? uc : rsub(up, um);
        *o.ptr = rmul(val, o.scale);
        o.ptr += o.stride;
    }
}

// The same tile with free warp windows (FP32, Laplacians in TMEM).  Warp w
// works on the 32 P points of the tile window from w (32 P - 2 KH) on and owns
// the middle 32 P - 2 KH of them; its neighbours come from shuffles only, with
// mirror ghosts at the ends of its window, so no level waits for the other
// warps.  A level loses one valid point at each end of a warp window, and
// KH >= len keeps the owned points exact (the Waveform Time Span argument on
// the warp window).  The owned points of the four warps are the tile core
// [KH, W - KH), so the tile halo is KH.  The adjoint pair goes to `out`
// ([2][W]), not back to the stage: a neighbouring warp may still have to read
// its halo from the stage.  Every point update and every pairing is the same
// operation on the same operands as in adj_tile, so the bits are the same.
template <typename Real, int FORM, int P, int NT, int SA, int KH>
__device__ __forceinline__ Real adj_tile_fw(const AdjParams<Real>& prm, const AdjTile<Real>& at, const Real* stage,
                                            Real* out, uint32_t tm)
{
    constexpr int NW = NT / 32;
    constexpr int WO = 32 * P - 2 * KH;  // points a warp owns
    constexpr int W = NW * WO + 2 * KH;  // tile window
    static_assert(sizeof(Real) == 4 && P % 8 == 0 && NT == 128, "TMEM store: FP32, 8-column chunks, 4 warps");
    static_assert(KH % P == 0 && KH >= SA && WO > 0, "warp halo: whole threads, at least one span long");
    static_assert(SA <= 31, "the samples of a span are held across one warp");
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int tb = warp * WO + lane * P;  // the thread's first point in the tile window
    const bool own = lane >= KH / P && lane < 32 - KH / P;
    const ProblemDev<Real>& pu = *at.pu;
    const ProblemDev<Real>& pl = *at.pl;
    const int64_t nx = pu.nx;
    const int64_t gj0 = at.gj0;
    const int64_t wabs = pu.base + gj0;
    const int64_t gj = gj0 + tb;
    const Real c2 = pu.c2, kk = pu.k;
    const bool edge = (gj0 <= 0) || (gj0 + W - 1 >= nx - 1);
    const bool has_src = pl.js >= 0 && pl.js >= gj0 && pl.js < gj0 + W;
    const int len = at.len;

    // ---- u phase: levels n0 .. n0+len-1, their Laplacians to TMEM
    {
        Real u[P], w[P];
        smem_to_regs<Real, P>(stage + 0 * W + tb, u);
        smem_to_regs<Real, P>(stage + 1 * W + tb, w);
        const Special sp = make_special<P>(gj, nx, -1);
        // warp-uniform: every lane of a warp that holds a special point runs the
        // patch (its selects leave the other lanes' points alone), so that the
        // level loop is not split into a patched and a plain copy that the
        // warp would run one after the other
        const bool special = __any_sync(kFull, edge && any_special(sp));
        // end registers only, in every lane of the warp: the select patch
        const bool ends = special && __all_sync(kFull, fixed_ends<P>(sp));
        const EndPatch ep{sp.r0 == 0, sp.rp == 0, sp.r1 == P - 1, sp.rm == P - 1};
        // the Dirichlet samples of levels n0 .. n0+31 across the warp (len <= 31:
        // one shuffle per level), the previous level's carried in a register
        Real ca = Real(0), cb = Real(0), fa_old = Real(0), fb_old = Real(0);
        bool wa = false, wb = false;
        if (edge) {
            wa = __any_sync(kFull, sp.r0 >= 0) && pu.fA != nullptr;
            wb = __any_sync(kFull, sp.r1 >= 0) && pu.fB != nullptr;
            if (wa) {
                ca = level_sample(pu.fA, 1, at.n0 + lane, prm.T);
                fa_old = __shfl_sync(kFull, ca, 0);
            }
            if (wb) {
                cb = level_sample(pu.fB, 1, at.n0 + lane, prm.T);
                fb_old = __shfl_sync(kFull, cb, 0);
            }
        }
        auto level = [&](auto step_c, int s) {
            constexpr bool STEP = decltype(step_c)::value;
            Real lft, rgt;
            warp_neighbours<Real, P>(u, lft, rgt, lane);
            uint32_t b[P];
            if constexpr (FORM == kCanonical) {
                Real ul = lft;
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    const Real uc = u[i];
                    const Real ur = i < P - 1 ? u[i + 1] : rgt;
                    const Real sum = radd(ul, ur);
                    b[i] = __float_as_uint(rfma(Real(-2), uc, sum));
                    if constexpr (STEP) {
                        u[i] = rfma(c2, sum, rfma(kk, uc, -w[i]));
                        w[i] = uc;
                    }
                    ul = uc;
                }
            } else {
                Real d_prev = rsub(u[0], lft);
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    const Real ur = i < P - 1 ? u[i + 1] : rgt;
                    const Real d = rsub(ur, u[i]);
                    const Real lap = rsub(d, d_prev);
                    d_prev = d;
                    b[i] = __float_as_uint(lap);
                    if constexpr (STEP) {
                        const Real v = rfma(c2, lap, w[i]);
                        w[i] = v;
                        u[i] = radd(u[i], v);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < P / 8; ++c)
                tmem_st8(tm + (uint32_t)(s * P + 8 * c), *reinterpret_cast<const uint32_t(*)[8]>(b + 8 * c));
            if constexpr (STEP) {
                const Real fa_new = wa ? __shfl_sync(kFull, ca, s + 1) : Real(0);
                const Real fb_new = wb ? __shfl_sync(kFull, cb, s + 1) : Real(0);
                if (ends) patch_ends<Real, FORM, P>(u, w, ep, fa_old, fa_new, fb_old, fb_new);
                else if (special) patch_fast<Real, FORM, P>(u, w, sp, Real(0), Real(0), fa_old, fa_new, fb_old, fb_new);
                fa_old = fa_new;
                fb_old = fb_new;
            }
        };
        for (int s = 0; s + 1 < len; ++s) level(std::true_type{}, s);
        if (len > 0) level(std::false_type{}, len - 1);
        tmem_wait_st();  // the lambda phase loads what this thread stored
    }

    // ---- lambda phase: levels m0 .. m0+len-1 pair with u levels n0+len-1 .. n0
    Real racc = Real(0);
    Real l[P], lw[P];
    smem_to_regs<Real, P>(stage + 2 * W + tb, l);
    smem_to_regs<Real, P>(stage + 3 * W + tb, lw);
    const Special sp = make_special<P>(gj, nx, has_src ? pl.js : -1);
    const bool special = __any_sync(kFull, (edge || has_src) && any_special(sp));  // warp-uniform, as above
    const bool ends = special && __all_sync(kFull, fixed_ends<P>(sp));
    const EndPatch ep{sp.r0 == 0, sp.rp == 0, sp.r1 == P - 1, sp.rm == P - 1};
    // the source samples of levels m0+1 .. m0+32 across the warp
    Real cs = Real(0);
    bool wsrc = false;
    if (has_src) {
        wsrc = __any_sync(kFull, sp.rs >= 0);
        if (wsrc) cs = level_sample(pl.src, pl.src_stride, at.m0 + 1 + lane, prm.T);
    }
    // owned points that are interior grid points, in register indices
    int ilo = 0, ihi = 0;
    if (own) {
        ilo = (int)(1 - gj <= 0 ? 0 : (1 - gj >= P ? P : 1 - gj));
        ihi = (int)(nx - 1 - gj <= 0 ? 0 : (nx - 1 - gj >= P ? P : nx - 1 - gj));
    }
    const bool full_core = ilo == 0 && ihi == P;
    // probes (dL/dfA samples): read once per tile; the owner thread of a
    // probed point records it every level (more than two on one thread: the
    // general path)
    const int rhi = own ? P : 0;
    OwnedProbe<Real> o0{};  // count 0: records nothing
    int nown = 0;
    for (int q = at.td.probe_begin; q < at.td.probe_end; ++q) {
        const int64_t li = prm.probes[q].gidx - wabs - (int64_t)tb;
        if (li >= 0 && li < rhi) {
            if (nown == 0) o0 = own_probe(prm.probes[q], wabs, tb, at.m0, len);
            ++nown;
        }
    }
    nown = __reduce_max_sync(kFull, nown);  // warp-uniform: the owner records, the other lanes pass
    for (int s = 0; s < len; ++s) {
        uint32_t lb[P];
#pragma unroll
        for (int c = 0; c < P / 8; ++c)
            tmem_ld8(tm + (uint32_t)((len - 1 - s) * P + 8 * c), *reinterpret_cast<uint32_t(*)[8]>(lb + 8 * c));
        Real lft, rgt;
        warp_neighbours<Real, P>(l, lft, rgt, lane);
        if (nown > 1)
            record_probes<Real, P>(l, lft, rgt, wabs, tb, 0, rhi, at.td.probe_begin, at.td.probe_end, prm.probes,
                                   at.m0 + s);
        else if (nown > 0)
            record_sw<Real, P>(o0, l, lft, rgt, s);
        __syncwarp();
#pragma unroll
        for (int c = 0; c < P / 8; ++c) tmem_wait_ld(*reinterpret_cast<uint32_t(*)[8]>(lb + 8 * c));
        if (full_core) {
#pragma unroll
            for (int i = 0; i < P; ++i) racc = rfma(l[i], __uint_as_float(lb[i]), racc);
        } else {
#pragma unroll
            for (int i = 0; i < P; ++i)
                if (i >= ilo && i < ihi) racc = rfma(l[i], __uint_as_float(lb[i]), racc);
        }
        const Real sval = wsrc ? __shfl_sync(kFull, cs, s) : Real(0);
        Real uold = Real(0);  // the level-m value at the source (increment form)
        if (FORM == kIncrement && special && !ends) uold = reg_get_sw<Real, P>(l, sp.rs);
        leap_step<Real, FORM, P>(l, lw, lft, rgt, c2, kk);
        if (ends) patch_ends<Real, FORM, P>(l, lw, ep, Real(0), Real(0), Real(0), Real(0));
        else if (special) patch_fast<Real, FORM, P>(l, lw, sp, uold, sval, Real(0), Real(0), Real(0), Real(0));
    }
    if (own) {
        regs_to_smem<Real, P>(out + 0 * W + tb, l);
        regs_to_smem<Real, P>(out + 1 * W + tb, lw);
    }
    return racc;
}

// Sum of racc over the window's threads in a fixed order (warp shuffles, then
// the warps in order); the result is valid in thread 0.
template <int NT, int BAR>
__device__ __forceinline__ double block_sum(double acc, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    block_sync<BAR>();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < NT / 32; ++q) t += red[q];
    return t;
}

template <typename Real, int FORM, int P, int NT, int SA>
__global__ void __launch_bounds__(NT) adjoint_kernel(const __grid_constant__ AdjParams<Real> prm)
{
    constexpr int W = NT * P;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Real* stage = reinterpret_cast<Real*>(smem_raw);  // [4][W]: u q0, u q1, lambda q0, lambda q1
    Real* laps = stage + 4 * W;                       // [SA][W]
    Real* xch = laps + SA * W;                        // [2][NW][2]
    __shared__ __align__(8) uint64_t bar;
    __shared__ double red[NW];
    __shared__ __align__(16) ProblemDev<Real> s_pu, s_pl;

    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async_smem();
    }
    __syncthreads();
    uint32_t phase = 0;
    int buf = 0;

    for (int64_t tile = blockIdx.x; tile < prm.ntiles; tile += gridDim.x) {
        AdjTile<Real> at;
        at.td = prm.tiles[tile];
        at.pu = &s_pu;  // shared-memory copies, written by thread 0 below
        at.pl = &s_pl;
        at.gj0 = (int64_t)at.td.local * prm.core - prm.H;
        at.n0 = prm.n0;
        at.m0 = prm.m0;
        at.len = prm.len;
        if (tid == 0) {
            s_pu = prm.prob_u[at.td.problem];
            s_pl = prm.prob_l[at.td.problem];
            const int64_t wabs = s_pu.base + at.gj0;
            constexpr uint32_t bytes = W * sizeof(Real);
            bulk_wait_read_all();  // the previous tile's store has read the stage
            fence_proxy_async_global();
            mbar_arrive_expect_tx(&bar, 4 * bytes);
            bulk_load(stage + 0 * W, prm.u0 + wabs, bytes, &bar);
            bulk_load(stage + 1 * W, prm.u1 + wabs, bytes, &bar);
            bulk_load(stage + 2 * W, prm.l0 + wabs, bytes, &bar);
            bulk_load(stage + 3 * W, prm.l1 + wabs, bytes, &bar);
        }
        const bool ok = mbar_wait_bounded(&bar, phase, prm.wait_ns, &prm.err->code);
        if (ok) phase ^= 1u;
        else latch_error(prm.err, kDevTimeoutLoad, (int)tile, (int)prm.n0, 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                mbar_wait_bounded(&bar, phase, prm.wait_ns, nullptr);
                bulk_wait_all();
            }
            return;
        }
        const Real racc = adj_tile<Real, FORM, P, NT, SA, 0>(prm, at, stage, laps, xch, buf);
        fence_proxy_async_smem();
        const double t = block_sum<NT, 0>((double)racc, red);
        if (tid == 0) {
            prm.partial[tile] = t;
            const int64_t dst = at.pu->base + (int64_t)at.td.local * prm.core;
            const uint32_t bytes = (uint32_t)prm.core * sizeof(Real);
            bulk_store(prm.l0_out + dst, stage + 2 * W + prm.H, bytes);
            bulk_store(prm.l1_out + dst, stage + 3 * W + prm.H, bytes);
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait_all();
}

// ---- persistent, warp-specialised adjoint sweep --------------------------------
// All spans of the adjoint sweep in one launch when the forward state at every
// span start is kept.  Tickets run over (processing index kp, tile), span
// K = nspans - 1 - kp (last span first); ticket (kp, i) starts once tiles i-1,
// i, i+1 have published kp - 1 (their adjoint cores are its halo, and they no
// longer read the buffer it writes).  A producer warp takes the tickets, loads
// the four windows of a tile with TMA into one of two stages, stores the
// adjoint core and publishes; the compute threads run adj_tile with a named
// barrier among themselves (barrier 1) and write the tile's partial sum.

template <typename Real>
struct AdjStage {
    ProblemDev<Real> pu;  // copies of the tile's forward and adjoint problem records
    ProblemDev<Real> pl;
    TileDev td;
    long long ticket;     // -1: no more work
    int kp;               // processing index (span K = nspans - 1 - kp)
    int tile;
    int64_t gj0, n0, m0;
    int len;
    int pad_;
};

// outb: where the compute threads leave the adjoint pair of stage y ([2][W] at
// outb + 2 W y), or nullptr: back in the stage's adjoint windows.
template <typename Real, int W>
__device__ void adj_producer(const AdjParams<Real>& prm, Real* stage, uint64_t* full_bar, uint64_t* empty_bar,
                             AdjStage<Real>* info, const Real* outb)
{
    const unsigned long long total = (unsigned long long)prm.nspans * (unsigned long long)prm.ntiles;
    auto grab = [&]() -> long long {
        if (*(volatile int*)&prm.err->code != 0) return -1;
        const unsigned long long t = atomicAdd(prm.ticket, 1ull);
        return t < total ? (long long)t : -1;
    };
    // tile count of the problem of the last ticket looked at
    int cached_problem = -1;
    int64_t cached_nt = 0;
    // neighbour flags: three independent relaxed loads, then one acquire fence
    auto ready = [&](long long t) -> bool {
        const int kp = (int)(t / prm.ntiles);
        if (kp == 0) return true;
        const int tile = (int)(t % prm.ntiles);
        const int f0 = ld_relaxed(prm.done + tile);
        const int fl = tile > 0 ? ld_relaxed(prm.done + tile - 1) : kp;
        const int fr = tile + 1 < prm.ntiles ? ld_relaxed(prm.done + tile + 1) : kp;
        const TileDev td = prm.tiles[tile];
        if (td.problem != cached_problem) {
            cached_nt = prm.prob_l[td.problem].ntiles;
            cached_problem = td.problem;
        }
        const bool ok = f0 >= kp && (td.local == 0 || fl >= kp) && (td.local + 1 >= cached_nt || fr >= kp);
        if (ok) fence_acq_rel_gpu();
        return ok;
    };
    auto wait_ready = [&](long long t) -> bool {
        if (ready(t)) return true;
        const long long t0 = global_ns();
        unsigned ns = 32;
        for (;;) {
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
            if (ready(t)) return true;
            if (*(volatile int*)&prm.err->code != 0) return false;
            if (global_ns() - t0 > prm.wait_ns) {
                latch_error(prm.err, kDevTimeoutFlag, (int)(t % prm.ntiles), (int)(t / prm.ntiles), 1);
                return false;
            }
        }
    };
    uint32_t fpar = 0u, epar = 0u, armed = 0u;
    constexpr uint32_t bytes = W * sizeof(Real);
    auto arm = [&](int y, long long t) {
        AdjStage<Real>& si = info[y];
        si.ticket = t;
        if (t >= 0) {
            const int kp = (int)(t / prm.ntiles);
            const int tile = (int)(t % prm.ntiles);
            const int64_t K = (int64_t)prm.nspans - 1 - kp;
            const TileDev td = prm.tiles[tile];
            const int64_t gj0 = (int64_t)td.local * prm.core - prm.H;
            const int64_t wabs = prm.prob_u[td.problem].base + gj0;
            Real* st = stage + y * 4 * W;
            // the windows first (bytes expected, no arrival yet), then the stage record
            fence_proxy_async_global();
            mbar_expect_tx(&full_bar[y], 4 * bytes);
            bulk_load(st + 0 * W, prm.uck0 + K * prm.ck_stride + wabs, bytes, &full_bar[y]);
            bulk_load(st + 1 * W, prm.uck1 + K * prm.ck_stride + wabs, bytes, &full_bar[y]);
            bulk_load(st + 2 * W, prm.lq0[kp & 1] + wabs, bytes, &full_bar[y]);
            bulk_load(st + 3 * W, prm.lq1[kp & 1] + wabs, bytes, &full_bar[y]);
            const int64_t n0 = K * prm.SA;
            const int len = (int)((prm.T - n0 < prm.SA) ? (prm.T - n0) : prm.SA);
            si.kp = kp;
            si.tile = tile;
            si.gj0 = gj0;
            si.n0 = n0;
            si.len = len;
            si.m0 = prm.T - (n0 + len - 1);
            si.td = td;
            si.pu = prm.prob_u[td.problem];
            si.pl = prm.prob_l[td.problem];
        }
        mbar_arrive(&full_bar[y]);  // the one arrival of the phase, after the record
        fpar ^= 1u << y;
        armed |= 1u << y;
    };
    auto store_core = [&](int y) {
        const AdjStage<Real>& si = info[y];
        const int64_t dst = si.pu.base + (int64_t)si.td.local * prm.core;
        const uint32_t cbytes = (uint32_t)prm.core * sizeof(Real);
        const Real* src = outb ? outb + y * 2 * W : stage + y * 4 * W + 2 * W;
        const int out = (si.kp + 1) & 1;
        bulk_store(prm.lq0[out] + dst, src + prm.H, cbytes);
        bulk_store(prm.lq1[out] + dst, src + W + prm.H, cbytes);
        bulk_commit();
    };
    auto publish = [&](int y) {
        fence_proxy_async_global();
        __threadfence();
        st_release(prm.done + info[y].tile, info[y].kp + 1);
    };

    // As the span kernel's producer: stage y holds t (being computed), stage
    // y ^ 1 holds tn (armed, or waiting for its neighbours); the producer never
    // waits for a ticket's neighbours while it holds an unpublished older tile.
    int y = 0;
    long long t = grab();
    if (t >= 0 && !wait_ready(t)) t = -1;
    arm(0, t);
    long long tn = -1;
    bool tn_armed = true;
    if (t >= 0) {
        tn = grab();
        tn_armed = tn < 0 || ready(tn);
        if (tn_armed) arm(1, tn);
    }
    while (t >= 0) {
        const long long tnn = tn >= 0 ? grab() : -1;
        if (!mbar_wait_backoff(&empty_bar[y], (epar >> y) & 1u, prm.wait_ns, &prm.err->code)) {
            latch_error(prm.err, kDevTimeoutLoad, (int)(t % prm.ntiles), (int)(t / prm.ntiles), 1);
            if (!tn_armed) arm(y ^ 1, -1);
            break;
        }
        epar ^= 1u << y;
        store_core(y);
        bool published = false;
        if (!tn_armed) {
            bulk_wait_all();
            publish(y);
            published = true;
            if (!wait_ready(tn)) {
                arm(y ^ 1, -1);
                break;
            }
            arm(y ^ 1, tn);
            tn_armed = true;
        }
        if (tn < 0) {
            if (!published) {
                bulk_wait_all();
                publish(y);
            }
            break;
        }
        bulk_wait_read_all();
        // stage y's record (tile, kp) is still needed by publish: keep it until then
        const int pub_tile = info[y].tile, pub_kp = info[y].kp;
        const bool tnn_armed = tnn < 0 || ready(tnn);
        if (tnn_armed) arm(y, tnn);
        if (!published) {
            bulk_wait_all();
            fence_proxy_async_global();
            __threadfence();
            st_release(prm.done + pub_tile, pub_kp + 1);
        }
        t = tn;
        tn = tnn;
        tn_armed = tnn_armed;
        y ^= 1;
    }
    bulk_wait_all();
    for (int st = 0; st < 2; ++st)
        if ((armed >> st) & 1u) mbar_wait_bounded(&full_bar[st], ((fpar >> st) & 1u) ^ 1u, prm.wait_ns, nullptr);
}

// Columns of tensor memory a CTA of the TMEM variant allocates: SA levels of P
// words per lane, rounded up to a power of two (at least 32).
__host__ __device__ constexpr int tmem_cols(int n)
{
    int c = 32;
    while (c < n) c *= 2;
    return c;
}

// Points of the CTA window: NT P, or with free warp windows of halo KH the
// owned points of the warps plus the two halos.
template <int P, int NT, int KH>
__host__ __device__ constexpr int ws_window()
{
    return KH > 0 ? (NT / 32) * (32 * P - 2 * KH) + 2 * KH : NT * P;
}

template <typename Real, int FORM, int P, int NT, int SA, bool TM, int KH>
__global__ void __launch_bounds__(NT + 32) adjoint_kernel_ws(const __grid_constant__ AdjParams<Real> prm)
{
    constexpr int W = ws_window<P, NT, KH>();
    constexpr int NW = NT / 32;
    constexpr uint32_t NCOL = (uint32_t)tmem_cols(SA * P);
    static_assert(!TM || NCOL <= 512, "the Laplacian store exceeds the tensor memory of an SM");
    static_assert(KH == 0 || TM, "free warp windows keep the Laplacians in TMEM");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Real* stage = reinterpret_cast<Real*>(smem_raw);  // [2 stages][4][W]
    Real* laps = stage + 8 * W;                       // [SA][W] (not with TM); with KH: [2 stages][2][W] out
    Real* xch = laps + (TM ? 0 : SA * W);             // [2][NW][2] (not with KH)
    Real* outb = KH > 0 ? laps : nullptr;
    __shared__ __align__(8) uint64_t full_bar[2];
    __shared__ __align__(8) uint64_t empty_bar[2];
    __shared__ __align__(16) AdjStage<Real> s_info[2];
    __shared__ double red[NW];
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    if constexpr (TM) {
        // before the producer takes a ticket: a CTA that waited here would hold none
        if (warp == 0) {
            tmem_alloc(&s_tmem, NCOL);
            tmem_relinquish();
        }
        tmem_fence_before_sync();
    }
    if (tid == NT) {
        mbar_init(&full_bar[0], 1);
        mbar_init(&full_bar[1], 1);
        mbar_init(&empty_bar[0], NW);
        mbar_init(&empty_bar[1], NW);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async_smem();
    }
    __syncthreads();  // the last CTA-wide barrier: from here on only barrier 1 (compute threads)
    if (warp == NW) {
        if (lane == 0) adj_producer<Real, W>(prm, stage, full_bar, empty_bar, s_info, outb);
        return;
    }
    uint32_t tm = 0;
    if constexpr (TM) {
        tmem_fence_after_sync();
        tm = tmem_addr(s_tmem, 32u * (uint32_t)(warp & 3), 0u);
    }
    uint32_t fpar = 0u;
    int y = 0, buf = 0;
    for (;;) {
        const bool ok = mbar_wait_bounded(&full_bar[y], (fpar >> y) & 1u, prm.wait_ns, &prm.err->code);
        fpar ^= 1u << y;
        if (!ok) latch_error(prm.err, kDevTimeoutLoad, -1, -1, 1);
        if (block_sync_or<NT>(!ok)) break;  // one decision for all compute threads
        const AdjStage<Real>& si = s_info[y];
        if (si.ticket < 0) break;
        AdjTile<Real> at;
        at.td = si.td;
        at.pu = &si.pu;  // shared-memory copies: no global round trip per tile
        at.pl = &si.pl;
        at.gj0 = si.gj0;
        at.n0 = si.n0;
        at.m0 = si.m0;
        at.len = si.len;
        Real* st = stage + y * 4 * W;
        Real racc;
        if constexpr (KH > 0) racc = adj_tile_fw<Real, FORM, P, NT, SA, KH>(prm, at, st, outb + y * 2 * W, tm);
        else racc = adj_tile<Real, FORM, P, NT, SA, NT, TM>(prm, at, st, laps, xch, buf, tm);
        const double t = block_sum<NT, NT>((double)racc, red);
        if (tid == 0) prm.partial[(int64_t)(prm.nspans - 1 - si.kp) * prm.ntiles + si.tile] = t;
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_bar[y]);
        y ^= 1;
    }
    if constexpr (TM) {
        // every compute thread leaves the loop together (both exits are decided
        // for all of them), with no TMEM access in flight
        tmem_fence_before_sync();
        block_sync<NT>();
        if (warp == 0) {
            tmem_fence_after_sync();
            tmem_dealloc(s_tmem, NCOL);
        }
    }
}

template <typename Real>
__global__ void adj_init_kernel(Real* l0, Real* l1, const ProblemDev<Real>* prob_l, int nprob, const Real* wbar,
                                int64_t T, int form)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    const ProblemDev<Real> pr = prob_l[p];
    if (pr.js < 0) return;
    const Real w = wbar[(int64_t)p * (T + 1) + T];
    l0[pr.base + pr.js] = w;                          // lambda^T = wbar[T] e_{j_r}
    l1[pr.base + pr.js] = form == kCanonical ? Real(0) : w;  // lambda^{T+1} = 0 / increment
}

// dL/da per problem in a fixed order, in two stages.  Stage 1: block b of
// problem p sums the partials of spans [b nspans / B, (b + 1) nspans / B) (each
// thread a fixed strided set of tiles, then a fixed tree); stage 2: one thread
// per problem adds the B block sums in order and scales.
constexpr int kRedThreads = 256;

__global__ void adj_reduce_stage1(const double* partial, int64_t nspans, int64_t ntiles, const int64_t* tile0,
                                  const int64_t* tcount, int B, double* tmp)
{
    const int p = (int)(blockIdx.x / B), b = (int)(blockIdx.x % B);
    __shared__ double red[kRedThreads];
    const int64_t tc = tcount[p], t0 = tile0[p];
    const int64_t k0 = (int64_t)b * nspans / B, k1 = (int64_t)(b + 1) * nspans / B;
    double acc = 0.0;
    for (int64_t k = k0; k < k1; ++k) {
        const double* row = partial + k * ntiles + t0;
        for (int64_t t = threadIdx.x; t < tc; t += kRedThreads) acc += row[t];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) tmp[(int64_t)p * B + b] = red[0];
}

__global__ void adj_reduce_stage2(const double* tmp, int B, const double* scale, double* out, int nprob)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    double t = 0.0;
    for (int b = 0; b < B; ++b) t += tmp[(int64_t)p * B + b];
    out[p] = t * scale[p];
}

struct AEntry {
    VariantInfo info;
    int SA;
    const void* fn;
    size_t smem;
};

template <typename Real, int FORM, int P, int NT, int SA>
AEntry make_aentry()
{
    constexpr int W = NT * P;
    AEntry e;
    e.info = VariantInfo{sizeof(Real) == 8 ? kF64 : kF32, FORM, P, NT, 0, NT * P, NT, 0};
    e.SA = SA;
    e.fn = reinterpret_cast<const void*>(&adjoint_kernel<Real, FORM, P, NT, SA>);
    e.smem = sizeof(Real) * ((4 + SA) * W + 4 * (NT / 32));
    return e;
}

const AEntry* atable(int* n)
{
    static const AEntry entries[] = {
        make_aentry<double, kCanonical, 4, 256, 8>(),
        make_aentry<double, kIncrement, 4, 256, 8>(),
        make_aentry<float, kIncrement, 8, 128, 16>(),
        make_aentry<float, kCanonical, 8, 128, 16>(),
    };
    *n = (int)(sizeof(entries) / sizeof(entries[0]));
    return entries;
}

}  // namespace

int adj_variant_count()
{
    int n;
    atable(&n);
    return n;
}

VariantInfo adj_variant_info(int v)
{
    int n;
    return atable(&n)[v].info;
}

int adj_variant_span(int v)
{
    int n;
    return atable(&n)[v].SA;
}

cudaError_t adj_prepare(int v)
{
    int n;
    const AEntry& e = atable(&n)[v];
    return cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e.smem);
}

cudaError_t adj_occupancy(int v, int* blocks_per_sm)
{
    int n;
    const AEntry& e = atable(&n)[v];
    cudaError_t st = adj_prepare(v);
    if (st != cudaSuccess) return st;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, e.fn, e.info.NT, e.smem);
}

cudaError_t adj_launch(int v, const void* params, int grid, cudaStream_t s)
{
    int n;
    const AEntry& e = atable(&n)[v];
    void* args[] = {const_cast<void*>(params)};
    return cudaLaunchKernel(e.fn, dim3(grid), dim3(e.info.NT), args, e.smem, s);
}

// ---- persistent adjoint kernels (one per dtype / form) -----------------------

namespace {

struct WsEntry {
    int dtype, form, W, SA, threads;
    const void* fn;
    size_t smem;      // dynamic shared memory the kernel uses
    int tmem_cols;    // TMEM columns per CTA (0: Laplacians in shared memory)
    int halo;         // the tile halo the kernel needs (free warp windows), 0: any
};

template <typename Real, int FORM, int P, int NT, int SA, bool TM, int KH = 0>
WsEntry make_ws()
{
    constexpr int W = ws_window<P, NT, KH>();
    const size_t words = KH > 0 ? 12 * W : (8 + (TM ? 0 : SA)) * W + 4 * (NT / 32);
    return WsEntry{sizeof(Real) == 8 ? kF64 : kF32, FORM, W, SA, NT + 32,
                   reinterpret_cast<const void*>(&adjoint_kernel_ws<Real, FORM, P, NT, SA, TM, KH>),
                   sizeof(Real) * words, TM ? tmem_cols(SA * P) : 0, KH};
}

const WsEntry* ws_find(int dtype, int form)
{
    static const WsEntry entries[] = {
        make_ws<double, kCanonical, 4, 128, 8, false>(),
        make_ws<double, kIncrement, 4, 128, 8, false>(),
        make_ws<float, kIncrement, 8, 128, 16, true, 16>(),
        make_ws<float, kCanonical, 8, 128, 16, true, 16>(),
    };
    for (const WsEntry& e : entries)
        if (e.dtype == dtype && e.form == form) return &e;
    return nullptr;
}

// CTAs of the kernel that fit on one SM with `smem` bytes of dynamic shared
// memory, from its shared memory, registers and threads.  The runtime's
// occupancy calculator answers 1 for any kernel that allocates tensor memory
// (it cannot know how many columns a CTA takes), while the SM holds as many
// such CTAs as these three resources allow; 0 if an attribute is unavailable.
int resident_ctas(const void* fn, int threads, size_t smem)
{
    int dev = 0, per_sm = 0, regs_sm = 0, thr_sm = 0, blk_sm = 0;
    cudaFuncAttributes fa{};
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int warps = (threads + 31) / 32;
    // shared memory: dynamic + static + the 1 KiB the runtime reserves per CTA
    const long long per_cta = (long long)smem + (long long)fa.sharedSizeBytes + 1024;
    // registers: allocated per warp in units of 256
    const long long regs_warp = ((long long)fa.numRegs * 32 + 255) / 256 * 256;
    long long n = per_sm / per_cta;
    if (regs_warp > 0) n = std::min<long long>(n, regs_sm / (regs_warp * warps));
    n = std::min<long long>(n, thr_sm / (warps * 32));
    n = std::min<long long>(n, blk_sm);
    return (int)std::max<long long>(n, 0);
}

// Dynamic shared memory of a launch.  With a TMEM store the CTAs of one SM
// must not ask for more than its 512 columns together, so the launch asks for
// enough shared memory that no more than 512 / tmem_cols CTAs fit; 0 if that
// cannot be arranged.
size_t ws_launch_smem(const WsEntry& e)
{
    if (e.tmem_cols == 0) return e.smem;
    int dev = 0, per_sm = 0, per_block = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, e.fn) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int cap = 512 / e.tmem_cols;
    // cap CTAs of (dynamic + static + the 1 KiB the runtime reserves) fill the SM
    long long want = (long long)per_sm / cap - (long long)fa.sharedSizeBytes - 1024;
    if (want + (long long)fa.sharedSizeBytes > per_block) want = per_block - (long long)fa.sharedSizeBytes;
    want = want / 1024 * 1024;
    if (want < (long long)e.smem) return 0;
    if (cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int bps = resident_ctas(e.fn, e.threads, (size_t)want);
    return (bps >= 1 && bps <= cap) ? (size_t)want : 0;
}

}  // namespace

int adj_ws_span(int dtype, int form)
{
    const WsEntry* e = ws_find(dtype, form);
    return e ? e->SA : 0;
}

int adj_ws_window(int dtype, int form)
{
    const WsEntry* e = ws_find(dtype, form);
    return e ? e->W : 0;
}

int adj_ws_halo(int dtype, int form)
{
    const WsEntry* e = ws_find(dtype, form);
    return e ? e->halo : 0;
}

cudaError_t adj_ws_prepare(int dtype, int form)
{
    const WsEntry* e = ws_find(dtype, form);
    if (!e) return cudaErrorInvalidValue;
    const size_t smem = ws_launch_smem(*e);
    if (smem == 0) return cudaErrorInvalidConfiguration;
    return cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t adj_ws_occupancy(int dtype, int form, int* blocks_per_sm)
{
    const WsEntry* e = ws_find(dtype, form);
    if (!e) return cudaErrorInvalidValue;
    cudaError_t st = adj_ws_prepare(dtype, form);
    if (st != cudaSuccess) return st;
    if (e->tmem_cols > 0) {
        *blocks_per_sm = resident_ctas(e->fn, e->threads, ws_launch_smem(*e));
        return cudaSuccess;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, e->fn, e->threads, ws_launch_smem(*e));
}

cudaError_t adj_ws_launch(int dtype, int form, const void* params, int grid, cudaStream_t s)
{
    const WsEntry* e = ws_find(dtype, form);
    if (!e) return cudaErrorInvalidValue;
    const size_t smem = ws_launch_smem(*e);
    if (smem == 0) return cudaErrorInvalidConfiguration;
    void* args[] = {const_cast<void*>(params)};
    return cudaLaunchKernel(e->fn, dim3(grid), dim3(e->threads), args, smem, s);
}

cudaError_t adj_init_launch(int dtype, int form, void* l0, void* l1, const void* prob_l, int nprob, const void* wbar,
                            int64_t T, cudaStream_t s)
{
    const int grid = (nprob + 127) / 128;
    if (dtype == kF32)
        adj_init_kernel<float><<<grid, 128, 0, s>>>(static_cast<float*>(l0), static_cast<float*>(l1),
                                                     static_cast<const ProblemDev<float>*>(prob_l), nprob,
                                                     static_cast<const float*>(wbar), T, form);
    else
        adj_init_kernel<double><<<grid, 128, 0, s>>>(static_cast<double*>(l0), static_cast<double*>(l1),
                                                      static_cast<const ProblemDev<double>*>(prob_l), nprob,
                                                      static_cast<const double*>(wbar), T, form);
    return cudaGetLastError();
}

int adj_reduce_blocks(int64_t nspans, int nprob)
{
    // enough blocks to fill the GPU for one large problem, few for many problems
    int64_t b = std::min<int64_t>(nspans, 256);
    while (b > 1 && b * nprob > 4096) b /= 2;
    return (int)std::max<int64_t>(b, 1);
}

cudaError_t adj_reduce_launch(const double* partial, int64_t nspans, int64_t ntiles, const int64_t* tile0,
                              const int64_t* tcount, const double* scale, double* out, int nprob, double* tmp,
                              cudaStream_t s)
{
    const int B = adj_reduce_blocks(nspans, nprob);
    adj_reduce_stage1<<<(unsigned)B * (unsigned)nprob, kRedThreads, 0, s>>>(partial, nspans, ntiles, tile0, tcount,
                                                                            B, tmp);
    adj_reduce_stage2<<<(nprob + 127) / 128, 128, 0, s>>>(tmp, B, scale, out, nprob);
    return cudaGetLastError();
}

}  // namespace rswr
