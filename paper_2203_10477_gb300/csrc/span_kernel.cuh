// span_kernel.cuh -- the RSWR span kernel (predict / select / update of one
// time span over overlapping windows), sm_103a.  The kernel templates live
// here; span_kernel.cu registers the variants compiled without user point
// sources, span_kernel_src.cu the same variants compiled with them.
//
// Paper mapping (arXiv 2203.10477):
//   predict (Sec. 2.3): a CTA stages its window -- the owned core plus H >= S
//       halo points on each side -- into shared memory with 1-D TMA bulk
//       copies and advances it S leapfrog steps in registers.  Each window end
//       that is not a physical boundary is an input boundary whose flux is
//       guessed (mirror ghost, zero flux).
//   select  (Sec. 2.4, Waveform Time Span Theorem): the guessed edges corrupt
//       one more point per step (discrete domain of dependence), so after
//       S <= H steps the core is exact; select is the index range of the
//       write-back, no data pass.
//   update  (Sec. 2.5, combination) + redo (Sec. 2.6): the core of both final
//       levels is written back with a TMA bulk store; the next span's windows
//       read it.  Interface output waveforms (Sec. 2.2) are recorded per step
//       by the probe table.
//   N > 2 (Sec. 3): all windows of all problems run in one launch; in
//       persistent mode the global span loop is replaced by per-tile
//       neighbour flags, so spans overlap across the domain.
//
// The CTA windows refine the user's subdomains: every core lies in one
// subdomain's window span and the result on a core does not depend on how the
// domain is cut (the same theorems), so the combined state equals the
// monolithic leapfrog bit for bit.
//
// Data path per CTA:  TMA load (stage x^1, next tile) || registers: S steps of
// 3-point leapfrog; halos by warp shuffles + one shared-memory slot per warp
// edge per step || TMA store of the core (stage x).

#pragma once

#include <cstdio>
#include <type_traits>

#include "rswr_internal.h"
#include "span_common.cuh"

namespace rswr {

namespace {

using namespace span;

// ---- ticket bookkeeping (thread 0 only) ----------------------------------

template <typename Real>
__device__ __forceinline__ long long grab_ticket(const SpanParams<Real>& prm, int it)
{
    if (prm.span >= 0) {
        const long long t = (long long)blockIdx.x + (long long)it * gridDim.x;
        return t < prm.ntiles ? (long long)prm.span * prm.ntiles + t : -1;
    }
    if (*(volatile int*)&prm.err->code != 0) return -1;  // another CTA gave up: stop taking work
    const unsigned long long total = (unsigned long long)prm.nspans * (unsigned long long)prm.ntiles;
    const unsigned long long t = atomicAdd(prm.ticket, 1ull);
    return t < total ? (long long)t : -1;
}

// Persistent mode: a ticket (span k, tile i) may start once tile i and its
// neighbours in the same problem have completed span k-1 (their cores are the
// halos of window i, and they no longer read the buffer span k writes).
template <typename Real>
__device__ __forceinline__ bool deps_ready(const SpanParams<Real>& prm, long long t)
{
    if (prm.span >= 0) return true;
    const int k = (int)(t / prm.ntiles);
    if (k == 0) return true;
    const int tile = (int)(t % prm.ntiles);
    const TileDev td = prm.tiles[tile];
    const int64_t nt = prm.problems[td.problem].ntiles;
    if (ld_acquire(prm.done + tile) < k) return false;
    if (td.local > 0 && ld_acquire(prm.done + tile - 1) < k) return false;
    if (td.local + 1 < nt && ld_acquire(prm.done + tile + 1) < k) return false;
    return true;
}

template <typename Real>
__device__ bool wait_deps(const SpanParams<Real>& prm, long long t)
{
    if (deps_ready(prm, t)) return true;
    const long long t0 = global_ns();
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
        if (deps_ready(prm, t)) return true;
        if (*(volatile int*)&prm.err->code != 0) return false;
        if (global_ns() - t0 > prm.wait_ns) {
            latch_error(prm.err, kDevTimeoutFlag, (int)(t % prm.ntiles), (int)(t / prm.ntiles), 0);
            return false;
        }
    }
}

// Steps of the launch's span that starts at level n0: S, or what is left of
// the run.  The run's length is T, or *steps_dev when the span is chosen on
// the device (then a span past it takes no steps: its tiles pass through).
template <typename Real>
__device__ __forceinline__ int span_steps(const SpanParams<Real>& prm, int64_t n0)
{
    const int64_t T = prm.steps_dev ? (int64_t)*prm.steps_dev : prm.T;
    const int64_t r = T - n0;
    return (int)(r < 0 ? 0 : (r < prm.S ? r : prm.S));
}

// State arrays read (span k) and written (span k + 1) by a span; comp 0 / 1
// selects the first / second component.
template <typename Real>
__device__ __forceinline__ Real* span_state(const SpanParams<Real>& prm, int comp, int level_span)
{
    Real* const* q = comp ? prm.q1 : prm.q0;
    return prm.ck_stride ? q[0] + (int64_t)level_span * prm.ck_stride : q[level_span & 1];
}

template <typename Real, int W>
__device__ __forceinline__ void issue_load(const SpanParams<Real>& prm, long long t, Real* stage_y, uint64_t* bar)
{
    const int k = (int)(t / prm.ntiles);
    const int tile = (int)(t % prm.ntiles);
    const TileDev td = prm.tiles[tile];
    const int64_t off = prm.problems[td.problem].base + (int64_t)td.local * prm.core - prm.H;
    constexpr uint32_t bytes = W * sizeof(Real);
    fence_proxy_async_global();
    mbar_arrive_expect_tx(bar, 2 * bytes);
    bulk_load(stage_y, span_state(prm, 0, k) + off, bytes, bar);
    bulk_load(stage_y + W, span_state(prm, 1, k) + off, bytes, bar);
}

// The same copies for the warp-specialised producer: the bytes are expected
// without an arrival (the producer arrives once the stage's record is written).
template <typename Real, int W>
__device__ __forceinline__ void issue_load_tx(const SpanParams<Real>& prm, long long t, Real* stage_y, uint64_t* bar)
{
    const int k = (int)(t / prm.ntiles);
    const int tile = (int)(t % prm.ntiles);
    const TileDev td = prm.tiles[tile];
    const int64_t off = prm.problems[td.problem].base + (int64_t)td.local * prm.core - prm.H;
    constexpr uint32_t bytes = W * sizeof(Real);
    fence_proxy_async_global();
    mbar_expect_tx(bar, 2 * bytes);
    bulk_load(stage_y, span_state(prm, 0, k) + off, bytes, bar);
    bulk_load(stage_y + W, span_state(prm, 1, k) + off, bytes, bar);
}

// Caller guarantees that the bulk store of ticket t has completed.
template <typename Real>
__device__ __forceinline__ void publish(const SpanParams<Real>& prm, long long t)
{
    const int k = (int)(t / prm.ntiles);
    const int tile = (int)(t % prm.ntiles);
    if (prm.span >= 0) return;
    if (tile == prm.inject_tile && k == prm.inject_span) return;  // host-requested missing flag (tests)
    fence_proxy_async_global();
    __threadfence();
    st_release(prm.done + tile, k + 1);
}

}  // namespace

// Window geometry of a variant: KH = 0 -> warps tile the window back to back;
// KH > 0 -> warp windows overlap by 2 KH points (see refresh_halos).
// FREE: the warp halo is at least the span (P < 2 KH: a thread cannot hold a
// halo and the owned points next to it, so halos are never refreshed and the
// span is limited to KH steps).
template <int P, int NT, int KH>
struct Geom {
    static constexpr int NW = NT / 32;
    static constexpr bool FREE = KH > 0 && P < 2 * KH;
    static constexpr int CW = KH == 0 ? 32 * P : 32 * P - 2 * KH;  // window offset between warps
    static constexpr int W = KH == 0 ? NT * P : NW * CW + 2 * KH;   // points per CTA window
    static constexpr int XCH = ((4 * NW + 15) / 16) * 16 + (FREE ? 0 : 8 * NW * KH);  // exchange slots (values)
};

// The predict phase of one tile (Sec. 2.3): `steps` leapfrog steps of the
// thread's P points u, w (window index tb of its first point), with the
// tile's probes recorded at every level and the special points (Dirichlet
// nodes, sources, points outside the grid) patched after every step.  Point
// sources apply at every copy of their point in the window, halo included,
// so the core equals the monolithic solve with the sources (Sec. 2.4).
// BAR is the barrier the window's warps share (block_sync); every branch
// below that contains one depends on per-tile values only, so all threads of
// the window take it together.  The step loop is instantiated six times
// (probes yes/no x {plain, special points, special points + user sources}) so
// that a plain interior tile runs the bare stencil with no per-step tests.
template <typename Real, int FORM, int P, int NW, int KH, int BAR, bool USRC, bool EDGE_FAST = false>
__device__ __forceinline__ void predict_tile(const SpanParams<Real>& prm, const ProblemDev<Real>& pr,
                                             const TileDev& td, Real (&u)[P], Real (&w)[P], int64_t gj0, int64_t n0,
                                             int steps, int tb, int own_lo, int own_hi,
                                             const ProbeDev<Real>* tprobes, int np, Real* xch, Real* hx, int warp,
                                             int lane, bool edge)
{
    constexpr int CW = KH == 0 ? 32 * P : 32 * P - 2 * KH;
    constexpr int W = KH == 0 ? NW * 32 * P : NW * CW + 2 * KH;
    const int64_t nx = pr.nx;
    const int64_t wabs = pr.base + gj0;
    const int64_t gj = gj0 + tb;
    const bool has_src = pr.js >= 0 && pr.js >= gj0 && pr.js < gj0 + W;
    const bool has_usrc = USRC && td.src_end > td.src_begin;  // never together with has_src (host)
    const bool slow = edge || has_src;
    const bool has_probe = np > 0;
    const bool few_probes = np <= kTileProbes;
    const Real c2 = pr.c2, kk = pr.k;

    const bool many_probes = has_probe && !few_probes;

    // special points of this thread (edge / source tiles only)
    auto special_points = [&](int64_t sj) { return make_special<P>(gj, nx, sj); };

    int buf = 0;
    // steps [s_begin, s_end) of the span; PR: record probes, SP: patch special
    // points.  What only PR or SP needs is set up inside its instantiation.
    auto run = [&](auto probe_c, auto special_c, auto user_c, int s_begin, int s_end) {
        constexpr bool PR = decltype(probe_c)::value;
        constexpr bool US = decltype(user_c)::value;  // the tile has user point sources
        constexpr bool SP = decltype(special_c)::value || US;
        // probes this thread owns: two in registers, any further ones read from shared memory
        OwnedProbe<Real> op0{}, op1{};
        int nown = 0;
        uint32_t more = 0u;
        if constexpr (PR) {
            if (few_probes) {
                for (int q = 0; q < np; ++q) {
                    const int64_t li = tprobes[q].gidx - wabs - (int64_t)tb;
                    if (li >= own_lo && li < own_hi) {
                        if (nown == 0) op0 = own_probe<Real>(tprobes[q], wabs, tb, n0 + s_begin, s_end - s_begin);
                        else if (nown == 1) op1 = own_probe<Real>(tprobes[q], wabs, tb, n0 + s_begin, s_end - s_begin);
                        else more |= 1u << q;
                        ++nown;
                    }
                }
            }
        }
        Special sp{-1, -1, -1, -1, -1};
        // boundary and source samples of the span, through the warp (warp-uniform choices):
        // fA / fB at level n0 + s_begin + i, the source at level n0 + s_begin + i + 1
        WarpChunk<Real> ca{}, cb{}, cs{};
        bool wa = false, wb = false, wsrc = false;
        int cbase = 0;
        // the chunked source: the problem's own (adjoint runs) or the one user
        // source among the warp's points (its samples in s_usrc[warp]); with
        // more, `multi` reads the tile's list at every step (level-n values of
        // held source points in uo_m)
        __shared__ const Real* s_usrc[NW];
        int64_t sj = has_src ? pr.js : -1;
        bool multi = false;
        Real uo_m[P];
        auto reload = [&](int first, bool both) {  // chunk(s) of steps first + lane (+ 32)
            const int64_t lv = n0 + s_begin + first + lane;
            if (wa) {
                if (both) ca.c0 = level_sample(pr.fA, 1, lv, prm.T);
                ca.c1 = level_sample(pr.fA, 1, lv + 32, prm.T);
            }
            if (wb) {
                if (both) cb.c0 = level_sample(pr.fB, 1, lv, prm.T);
                cb.c1 = level_sample(pr.fB, 1, lv + 32, prm.T);
            }
            if (wsrc) {
                const Real* sptr = US ? s_usrc[warp] : pr.src;
                const int64_t sstride = US ? 1 : pr.src_stride;
                if (both) cs.c0 = level_sample(sptr, sstride, lv + 1, prm.T);
                cs.c1 = level_sample(sptr, sstride, lv + 33, prm.T);
            }
        };
        if constexpr (SP) {
            if constexpr (US) {
                const int64_t wlo = gj - (int64_t)lane * P;  // the warp's first point (warp-uniform)
                int cnt = 0;
                for (int q = td.src_begin; q < td.src_end; ++q) {
                    const SrcDev<Real> sd = prm.srcs[q];
                    if (sd.j >= wlo && sd.j < wlo + 32 * P) {
                        if (cnt == 0) {
                            sj = sd.j;
                            if (lane == 0) s_usrc[warp] = sd.samples;
                        }
                        ++cnt;
                    }
                }
                __syncwarp();
                multi = cnt > 1;
                if (multi) sj = -1;
            }
            sp = special_points(sj);
            wa = __any_sync(kFull, sp.r0 >= 0) && pr.fA != nullptr;
            wb = __any_sync(kFull, sp.r1 >= 0) && pr.fB != nullptr;
            wsrc = __any_sync(kFull, sp.rs >= 0);
            reload(0, true);
        }
        // the probe recording of the edges-first loops: each level recorded by its
        // owner before it is advanced
        auto recf = [&](const Real(&uu)[P], Real l, Real r, int s) {
            if (nown > 0) record_step<Real, P>(op0, uu, l, r, s);
            if (nown > 1) record_step<Real, P>(op1, uu, l, r, s);
            for (uint32_t m = more; m != 0u; m &= m - 1u)
                record_owned<Real, P>(uu, l, r, tprobes[__ffs(m) - 1], wabs, tb, n0 + s_begin + s);
        };
        if constexpr (EDGE_FAST && KH > 0 && SP && !US) {
            // (resident tiles, where an edge or source tile paces every span)
            // free / refreshed warp windows of an edge or source tile: the warp's
            // choice (uniform across its lanes); a warp without special points
            // runs the bare (or recording) loop, one with them the edges-first
            // loop with the points patched
            if (!many_probes) {
                const bool wsp = __any_sync(kFull, any_special(sp));
                const bool wpr = PR && __any_sync(kFull, nown > 0);
                if (!wsp) {
                    if (wpr) warp_steps_edges_first<Real, FORM, P>(u, w, c2, kk, s_end - s_begin, lane, recf);
                    else warp_steps_edges_first<Real, FORM, P>(u, w, c2, kk, s_end - s_begin, lane);
                    return;
                }
                auto steps_with = [&](auto ep) {
                    if (wpr)
                        warp_steps_edges_first<Real, FORM, P>(u, w, c2, kk, s_end - s_begin, lane, recf, ep);
                    else
                        warp_steps_edges_first<Real, FORM, P>(u, w, c2, kk, s_end - s_begin, lane, NoRecord{}, ep);
                };
                if (__any_sync(kFull, interior_special<P>(sp)))
                    steps_with(EdgePatch<Real, FORM, P, decltype(reload), true>{sp, &ca, &cb, &cs, wa, wb, wsrc,
                                                                                 &cbase, &reload});
                else
                    steps_with(EdgePatch<Real, FORM, P, decltype(reload), false>{sp, &ca, &cb, &cs, wa, wb, wsrc,
                                                                                  &cbase, &reload});
                return;
            }
        }
        if constexpr (KH > 0 && !SP) {
            if constexpr (!PR) {
                // plain interior tile of a warp window: the bare stencil, edges first
                warp_steps_edges_first<Real, FORM, P>(u, w, c2, kk, s_end - s_begin, lane);
                return;
            } else {
                // interior tile with probes: edges first as well, each level
                // recorded by its owner before it is advanced; a warp that owns
                // none of the tile's probes runs the bare stencil (warp-uniform)
                if (!many_probes && !__any_sync(kFull, nown > 0)) {
                    warp_steps_edges_first<Real, FORM, P>(u, w, c2, kk, s_end - s_begin, lane);
                    return;
                }
                if (!many_probes) {
                    warp_steps_edges_first<Real, FORM, P>(u, w, c2, kk, s_end - s_begin, lane, recf);
                    return;
                }
            }
        }
        for (int s = s_begin; s < s_end; ++s) {
            Real lft, rgt;
            if constexpr (KH > 0) {
                warp_neighbours<Real, P>(u, lft, rgt, lane);
            } else {
                exchange<Real, P, NW, BAR>(u, lft, rgt, xch, buf, warp, lane);
                buf ^= 1;
            }
            const int64_t n = n0 + s;
            if constexpr (PR) {
                if (nown > 0) record_step<Real, P>(op0, u, lft, rgt, s - s_begin);
                if (nown > 1) record_step<Real, P>(op1, u, lft, rgt, s - s_begin);
                for (uint32_t m = more; m != 0u; m &= m - 1u)
                    record_owned<Real, P>(u, lft, rgt, tprobes[__ffs(m) - 1], wabs, tb, n);
                if (many_probes)
                    record_probes<Real, P>(u, lft, rgt, wabs, tb, own_lo, own_hi, td.probe_begin, td.probe_end,
                                           prm.probes, n);
            }
            if constexpr (SP) {
                const int d = s - s_begin - cbase;
                if (d == 32) {
                    // move to the next chunk; load the one after it
                    cbase += 32;
                    ca.c0 = ca.c1;
                    cb.c0 = cb.c1;
                    cs.c0 = cs.c1;
                    reload(cbase, false);
                }
                const int dd = s - s_begin - cbase;
                Real uold_s = Real(0), sval = Real(0);
                Real fa_old = Real(0), fa_new = Real(0), fb_old = Real(0), fb_new = Real(0);
                if (wsrc) sval = cs.get(dd);  // src at level n + 1
                if (wa) {
                    fa_old = ca.get(dd);
                    fa_new = ca.get(dd + 1);
                }
                if (wb) {
                    fb_old = cb.get(dd);
                    fb_new = cb.get(dd + 1);
                }
                if constexpr (FORM == kIncrement) {
                    if (sp.rs >= 0) uold_s = reg_get<Real, P>(u, sp.rs);
                    if (US && multi)
                        for (int q = td.src_begin; q < td.src_end; ++q) {
                            const int64_t li = prm.srcs[q].j - gj;
                            if (li >= 0 && li < P) uo_m[li] = reg_get<Real, P>(u, (int)li);
                        }
                }
                leap_step<Real, FORM, P>(u, w, lft, rgt, c2, kk);
                patch_special<Real, FORM, P>(u, w, sp, uold_s, sval, fa_old, fa_new, fb_old, fb_new);
                if (US && multi)
                    for (int q = td.src_begin; q < td.src_end; ++q) {
                        const SrcDev<Real> sd = prm.srcs[q];
                        const int64_t li = sd.j - gj;
                        if (li < 0 || li >= P) continue;
                        const Real sv = level_sample(sd.samples, 1, n + 1, prm.T);
                        add_source_at<Real, FORM, P>(u, w, (int)li, sv,
                                                     FORM == kIncrement ? uo_m[li] : Real(0));
                    }
            } else {
                leap_step<Real, FORM, P>(u, w, lft, rgt, c2, kk);
            }
        }
    };
    // The instantiation is chosen from per-tile values only: every lane of a
    // warp (and, with exchange(), every thread of the window) must execute the
    // same shuffle and barrier instructions.  On a slow tile every thread runs
    // the patching loop; for a thread without special points the patch is a no-op.
    // Tiles with user point sources take instantiations of their own (in the
    // kernels compiled with USRC only).
    using Yes = std::true_type;
    using No = std::false_type;
    auto run_steps = [&](int s_begin, int s_end) {
        if (has_probe) {
            if (has_usrc) run(Yes{}, Yes{}, Yes{}, s_begin, s_end);
            else if (slow) run(Yes{}, Yes{}, No{}, s_begin, s_end);
            else run(Yes{}, No{}, No{}, s_begin, s_end);
        } else {
            if (has_usrc) run(No{}, Yes{}, Yes{}, s_begin, s_end);
            else if (slow) run(No{}, Yes{}, No{}, s_begin, s_end);
            else run(No{}, No{}, No{}, s_begin, s_end);
        }
    };

    if constexpr (KH > 0) {
        if constexpr (P >= 2 * KH) {
            // warp halos refreshed every KH steps
            for (int s0 = 0; s0 < steps; s0 += KH) {
                if (s0 > 0) {
                    refresh_halos<Real, P, NW, KH, BAR>(u, w, hx, buf, warp, lane);
                    buf ^= 1;
                }
                run_steps(s0, (s0 + KH < steps) ? s0 + KH : steps);
            }
        } else {
            // free warp windows: the warp halo covers the whole span (steps <= KH,
            // checked by the caller), so warps never exchange data inside a span
            run_steps(0, steps);
        }
    } else {
        if (!slow && !has_usrc && !has_probe) {
            // interior tile: halo latency hidden behind the interior updates
            for (int s = 0; s < steps; ++s) {
                split_step<Real, FORM, P, NW, BAR>(u, w, c2, kk, xch, buf, warp, lane);
                buf ^= 1;
            }
        } else {
            run_steps(0, steps);
        }
    }
}

// Registers [own_lo, own_hi) of a thread that it owns: warp w owns its window
// minus KH halo points at each end that has a neighbouring warp (the outer
// halos of the first and last warp have no neighbour and belong to them).
// When KH > P the halo spans several threads, some of which own nothing.
template <int P, int NW, int KH>
__device__ __forceinline__ void owned_range(int warp, int lane, int& own_lo, int& own_hi)
{
    const int lo_w = (KH > 0 && warp > 0) ? KH : 0;
    const int hi_w = (KH > 0 && warp < NW - 1) ? 32 * P - KH : 32 * P;
    const int a = lo_w - lane * P, b = hi_w - lane * P;
    own_lo = a < 0 ? 0 : (a > P ? P : a);
    own_hi = b < 0 ? 0 : (b > P ? P : b);
}

template <typename Real, int FORM, int P, int NT, int KH, int MINB, bool USRC>
__global__ void __launch_bounds__(NT, MINB) span_kernel(const __grid_constant__ SpanParams<Real> prm)
{
    using G = Geom<P, NT, KH>;
    constexpr int W = G::W;
    constexpr int NW = G::NW;
    static_assert(W % 4 == 0, "windows must span whole 16-byte units");
    static_assert(KH == 0 || P >= 2 * KH, "this kernel refreshes warp halos");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Real* stage = reinterpret_cast<Real*>(smem_raw);  // [2 stages][2 components][W]
    Real* xch = stage + 4 * W;                        // [2 buffers][NW][2]  (+ halo slots when KH > 0)
    Real* hx = xch + ((4 * NW + 15) / 16) * 16;  // vector-aligned halo slots
    __shared__ __align__(8) uint64_t full_bar[2];
    __shared__ long long s_ticket[2];
    __shared__ int s_abort;
    __shared__ ProbeDev<Real> s_probes[kTileProbes];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    // thread-0 pipeline state
    long long pending = -1;         // ticket stored one iteration ago, not yet published
    uint32_t issued = 0u;           // bit s: stage s has a load that has not been waited for
    bool deferred = false;
    int it = 0;

    if (tid == 0) {
        mbar_init(&full_bar[0], 1);
        mbar_init(&full_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async_smem();
        s_abort = 0;
        const long long t0 = grab_ticket(prm, it++);
        s_ticket[0] = t0;
        if (t0 >= 0) {
            if (wait_deps(prm, t0)) {
                issue_load<Real, W>(prm, t0, stage, &full_bar[0]);
                issued = 1u;
            } else {
                s_abort = 1;
            }
        }
    }
    __syncthreads();

    uint32_t phase = 0u;  // bit s: parity of the next phase of stage s
    int x = 0;
    bool aborted = s_abort != 0;
    while (!aborted) {
        const long long t = s_ticket[x];
        if (t < 0) break;

        // thread 0: take the next ticket and prefetch its window into the other stage
        if (tid == 0) {
            const long long tn = grab_ticket(prm, it++);
            deferred = false;
            if (tn >= 0) {
                if (deps_ready(prm, tn)) {
                    bulk_wait_read_all();  // the store issued from stage x^1 has read its data
                    issue_load<Real, W>(prm, tn, stage + (x ^ 1) * 2 * W, &full_bar[x ^ 1]);
                    issued |= 1u << (x ^ 1);
                } else {
                    deferred = true;
                }
            }
            s_ticket[x ^ 1] = tn;
        }

        // all: wait for the current stage
        const bool ok = mbar_wait_bounded(&full_bar[x], (phase >> x) & 1u, prm.wait_ns, &prm.err->code);
        if (ok) {
            phase ^= 1u << x;
            issued &= ~(1u << x);
        } else {
            latch_error(prm.err, kDevTimeoutLoad, (int)(t % prm.ntiles), (int)(t / prm.ntiles), 0);
        }
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }

        // ---- tile geometry
        const int k = (int)(t / prm.ntiles);
        const int tile = (int)(t % prm.ntiles);
        const TileDev td = prm.tiles[tile];
        const ProblemDev<Real>& pr = prm.problems[td.problem];
        const int64_t gj0 = (int64_t)td.local * prm.core - prm.H;  // problem coordinate of window start
        const int64_t n0 = (int64_t)k * prm.S;
        const int steps = span_steps(prm, n0);
        const bool edge = (gj0 <= 0) || (gj0 + W - 1 >= pr.nx - 1);
        const int tb = warp * G::CW + lane * P;  // window index of the thread's first point
        int own_lo, own_hi;
        owned_range<P, NW, KH>(warp, lane, own_lo, own_hi);

        Real* su = stage + x * 2 * W;
        Real* sw = su + W;
        Real u[P], w[P];
        smem_to_regs<Real, P>(su + tb, u);
        smem_to_regs<Real, P>(sw + tb, w);

        // probes of this tile: staged in shared memory
        const int np = td.probe_end - td.probe_begin;
        if (np > 0 && np <= kTileProbes) {
            if (tid < np) s_probes[tid] = prm.probes[td.probe_begin + tid];
            __syncthreads();
        }

        predict_tile<Real, FORM, P, NW, KH, 0, USRC>(prm, pr, td, u, w, gj0, n0, steps, tb, own_lo, own_hi, s_probes,
                                                  np, xch, hx, warp, lane, edge);

        // ---- select + update: write the window back, store only the core
        __syncthreads();  // every thread has read its window (KH > 0: windows overlap)
        owned_to_smem<Real, P, KH>(su + tb, u, own_lo, own_hi);
        owned_to_smem<Real, P, KH>(sw + tb, w, own_lo, own_hi);
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            const int64_t dst = pr.base + (int64_t)td.local * prm.core;
            const uint32_t bytes = (uint32_t)prm.core * sizeof(Real);
            bulk_store(span_state(prm, 0, k + 1) + dst, su + prm.H, bytes);
            bulk_store(span_state(prm, 1, k + 1) + dst, sw + prm.H, bytes);
            bulk_commit();
            if (pending >= 0) {
                // the store of the previous tile is complete once at most one group is pending
                asm volatile("cp.async.bulk.wait_group 1;" ::: "memory");
                publish(prm, pending);
            }
            pending = t;
            if (deferred) {
                bulk_wait_all();
                publish(prm, pending);
                pending = -1;
                const long long tn = s_ticket[x ^ 1];
                if (wait_deps(prm, tn)) {
                    issue_load<Real, W>(prm, tn, stage + (x ^ 1) * 2 * W, &full_bar[x ^ 1]);
                    issued |= 1u << (x ^ 1);
                } else {
                    s_abort = 1;
                }
            }
        }
        if (__syncthreads_or(tid == 0 && s_abort != 0)) {
            aborted = true;
            break;
        }
        x ^= 1;
    }

    if (tid == 0) {
        bulk_wait_all();
        if (!aborted && pending >= 0) publish(prm, pending);
        for (int st = 0; st < 2; ++st) {
            // let an issued load land before the CTA's shared memory is released
            if ((issued >> st) & 1u) mbar_wait_bounded(&full_bar[st], (phase >> st) & 1u, prm.wait_ns, nullptr);
        }
    }
}

// ---- warp-specialised span kernel --------------------------------------------
// NT compute threads (NT/32 warps) and one producer warp.  Lane 0 of the
// producer warp takes the tickets, waits for the neighbour flags, fills the
// stages with TMA loads, stores the finished cores and publishes the flags;
// the compute warps only wait for a full stage, run the span and hand the
// stage back.
//
// Stage y (two of them) cycles through: producer arms full_bar[y] (a TMA load
// with its transaction bytes, or a plain arrival with ticket -1 = stop) ->
// compute warps wait full_bar[y], copy their windows to registers and arrive on
// read_bar[y] -> step -> wait read_bar[y] (every warp has read the stage; in
// practice long complete), write their owned points back, fence the async
// proxy and arrive on empty_bar[y] (one arrival per warp) -> producer waits
// empty_bar[y], bulk-stores the core, waits for the store to complete and
// publishes the tile; only then is stage y armed again.  The stage's ticket,
// tile geometry, a copy of its problem record and its probe table sit beside
// the stage and are written only while the stage belongs to the producer.
//
// With free warp windows (no data exchange between warps inside a span) the
// compute warps share no barrier at all: each warp decides on its own to stop.
// Variants that exchange halos between warps (KH = 0, or refreshed warp halos)
// take one decision for all compute threads at a named barrier (barrier 1,
// which the producer never joins) so that their per-step barriers stay uniform.

template <typename Real>
struct StageInfo {
    ProblemDev<Real> pr;  // copy of the tile's problem record
    TileDev td;
    long long ticket;     // -1: no more work
    int64_t gj0;          // problem coordinate of the window start
    int64_t n0;           // first level of the span
    int k;                // span
    int tile;
    int np;               // probes of the tile (staged when np <= kTileProbes)
    int steps;            // steps of this span
    int edge;             // the window touches a physical boundary
    int pad_;
};

template <typename Real, int W>
__device__ void producer_loop(const SpanParams<Real>& prm, Real* stage, uint64_t* full_bar, uint64_t* empty_bar,
                              StageInfo<Real>* info, ProbeDev<Real> (*sprobes)[kTileProbes])
{
    int it = 0;
    uint32_t fpar = 0u;   // bit y: parity of the next phase of full_bar[y] the producer arms
    uint32_t epar = 0u;   // bit y: parity of the next phase of empty_bar[y]
    uint32_t armed = 0u;  // bit y: full_bar[y] has been armed at least once

    // tile count of the problem of the last ticket looked at (consecutive
    // tiles mostly belong to the same problem)
    int cached_problem = -1;
    int64_t cached_nt = 0;
    auto problem_tiles = [&](int q) -> int64_t {
        if (q != cached_problem) {
            cached_nt = prm.problems[q].ntiles;
            cached_problem = q;
        }
        return cached_nt;
    };

    // neighbour flags of ticket t: three independent relaxed loads, then one
    // acquire fence (instead of three acquire loads in a row)
    auto ready = [&](long long t) -> bool {
        if (prm.span >= 0) return true;
        const int k = (int)(t / prm.ntiles);
        if (k == 0) return true;
        const int tile = (int)(t % prm.ntiles);
        const int f0 = ld_relaxed(prm.done + tile);
        const int fl = tile > 0 ? ld_relaxed(prm.done + tile - 1) : k;
        const int fr = tile + 1 < prm.ntiles ? ld_relaxed(prm.done + tile + 1) : k;
        const TileDev td = prm.tiles[tile];
        const int64_t nt = problem_tiles(td.problem);
        const bool ok = f0 >= k && (td.local == 0 || fl >= k) && (td.local + 1 >= nt || fr >= k);
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
                latch_error(prm.err, kDevTimeoutFlag, (int)(t % prm.ntiles), (int)(t / prm.ntiles), 0);
                return false;
            }
        }
    };

    auto arm = [&](int y, long long t) {
        StageInfo<Real>& si = info[y];
        si.ticket = t;
        if (t >= 0) {
            const int tile = (int)(t % prm.ntiles);
            const int k = (int)(t / prm.ntiles);
            const TileDev td = prm.tiles[tile];
            const ProblemDev<Real>& pr = prm.problems[td.problem];
            const int np = td.probe_end - td.probe_begin;
            const int64_t gj0 = (int64_t)td.local * prm.core - prm.H;
            const int64_t n0 = (int64_t)k * prm.S;
            // the window first: the copy is in flight while the stage's record is written
            issue_load_tx<Real, W>(prm, t, stage + y * 2 * W, &full_bar[y]);
            si.pr = pr;
            si.td = td;
            si.gj0 = gj0;
            si.n0 = n0;
            si.k = k;
            si.tile = tile;
            si.np = np;
            si.steps = span_steps(prm, n0);
            si.edge = (gj0 <= 0) || (gj0 + W - 1 >= pr.nx - 1);
            if (np > 0 && np <= kTileProbes)
                for (int q = 0; q < np; ++q) sprobes[y][q] = prm.probes[td.probe_begin + q];
        }
        // the stage's record is complete before the phase can be observed
        // (complete_tx needs this arrival too)
        mbar_arrive(&full_bar[y]);
        fpar ^= 1u << y;
        armed |= 1u << y;
    };
    auto store_core = [&](int y) {
        const StageInfo<Real>& si = info[y];
        const int64_t dst = si.pr.base + (int64_t)si.td.local * prm.core;
        const uint32_t bytes = (uint32_t)prm.core * sizeof(Real);
        Real* su = stage + y * 2 * W;
        bulk_store(span_state(prm, 0, si.k + 1) + dst, su + prm.H, bytes);
        bulk_store(span_state(prm, 1, si.k + 1) + dst, su + W + prm.H, bytes);
        bulk_commit();
    };

    // Stage y holds ticket t (being computed), stage y ^ 1 ticket tn (armed,
    // or waiting for its neighbours).  The producer never waits for the
    // neighbours of a ticket while it holds an unpublished older tile.
    int y = 0;
    long long t = grab_ticket(prm, it++);
    if (t >= 0 && !wait_ready(t)) t = -1;
    arm(0, t);
    long long tn = -1;
    bool tn_armed = true;
    if (t >= 0) {
        tn = grab_ticket(prm, it++);
        tn_armed = tn < 0 || ready(tn);
        if (tn_armed) arm(1, tn);
    }
    while (t >= 0) {
        // the ticket after tn, fetched now so that the atomic's latency overlaps the compute of t
        const long long tnn = tn >= 0 ? grab_ticket(prm, it++) : -1;
        if (!mbar_wait_backoff(&empty_bar[y], (epar >> y) & 1u, prm.wait_ns, &prm.err->code)) {
            latch_error(prm.err, kDevTimeoutLoad, (int)(t % prm.ntiles), (int)(t / prm.ntiles), 0);
            if (!tn_armed) arm(y ^ 1, -1);
            break;
        }
        epar ^= 1u << y;
        store_core(y);  // select + update of tile t
        bool published = false;
        if (!tn_armed) {
            // tn may need the tile just computed: publish it, then wait for tn's neighbours
            bulk_wait_all();
            publish(prm, t);
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
                publish(prm, t);
            }
            break;
        }
        // refill stage y with tnn as soon as the store has read it
        bulk_wait_read_all();
        const bool tnn_armed = tnn < 0 || ready(tnn);
        if (tnn_armed) arm(y, tnn);
        if (!published) {
            bulk_wait_all();
            publish(prm, t);
        }
        t = tn;
        tn = tnn;
        tn_armed = tnn_armed;
        y ^= 1;
    }
    bulk_wait_all();
    // let every armed phase complete (a load in flight) before shared memory is released
    for (int st = 0; st < 2; ++st)
        if ((armed >> st) & 1u)
            mbar_wait_bounded(&full_bar[st], ((fpar >> st) & 1u) ^ 1u, prm.wait_ns, nullptr);
}

template <typename Real, int FORM, int P, int NT, int KH, int MINB, bool USRC>
__global__ void __launch_bounds__(NT + 32, MINB) span_kernel_ws(const __grid_constant__ SpanParams<Real> prm)
{
    using G = Geom<P, NT, KH>;
    constexpr int W = G::W;
    constexpr int NW = G::NW;
    constexpr bool kFree = G::FREE;
    static_assert(W % 4 == 0, "windows must span whole 16-byte units");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Real* stage = reinterpret_cast<Real*>(smem_raw);  // [2 stages][2 components][W]
    Real* xch = stage + 4 * W;
    Real* hx = xch + ((4 * NW + 15) / 16) * 16;
    __shared__ __align__(8) uint64_t full_bar[2];
    __shared__ __align__(8) uint64_t empty_bar[2];
    __shared__ __align__(8) uint64_t read_bar[2];
    __shared__ __align__(16) StageInfo<Real> s_info[2];
    __shared__ ProbeDev<Real> s_probes[2][kTileProbes];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    if (tid == NT) {
        mbar_init(&full_bar[0], 1);
        mbar_init(&full_bar[1], 1);
        mbar_init(&empty_bar[0], NW);
        mbar_init(&empty_bar[1], NW);
        mbar_init(&read_bar[0], NW);
        mbar_init(&read_bar[1], NW);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async_smem();
    }
    __syncthreads();  // the last CTA-wide barrier: from here on only barrier 1 (compute threads)

    if (warp == NW) {
        if (lane == 0) producer_loop<Real, W>(prm, stage, full_bar, empty_bar, s_info, s_probes);
        return;
    }

    const int tb = warp * G::CW + lane * P;  // window index of the thread's first point
    int own_lo, own_hi;
    owned_range<P, NW, KH>(warp, lane, own_lo, own_hi);
    uint32_t fpar = 0u, rpar = 0u;
    int y = 0;
    for (;;) {
        const bool ok = mbar_wait_bounded(&full_bar[y], (fpar >> y) & 1u, prm.wait_ns, &prm.err->code);
        fpar ^= 1u << y;
        Real* su = stage + y * 2 * W;
        Real* sw = su + W;
        Real u[P], w[P];
        smem_to_regs<Real, P>(su + tb, u);
        smem_to_regs<Real, P>(sw + tb, w);
        if (!ok) latch_error(prm.err, kDevTimeoutLoad, -1, -1, 0);
        if constexpr (kFree) {
            // this warp's decision; its window is in registers
            if (__any_sync(kFull, !ok)) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(&read_bar[y]);
        } else {
            // one decision for all compute threads; after this barrier stage y is only written
            if (block_sync_or<NT>(!ok)) break;
        }
        const StageInfo<Real>& si = s_info[y];
        if (si.ticket < 0) break;

        const int steps = si.steps;
        if (kFree && steps > KH) {
            // the host never schedules a span longer than a free variant's warp halo
            if (tid == 0) latch_error(prm.err, kDevBadTicket, si.tile, si.k, 0);
        } else {
            predict_tile<Real, FORM, P, NW, KH, NT, USRC>(prm, si.pr, si.td, u, w, si.gj0, si.n0, steps, tb, own_lo,
                                                       own_hi, s_probes[y], si.np, xch, hx, warp, lane,
                                                       si.edge != 0);
        }
        if constexpr (kFree) {
            // every warp has read its window from stage y before anyone overwrites it
            const bool rd = mbar_wait_bounded(&read_bar[y], (rpar >> y) & 1u, prm.wait_ns, &prm.err->code);
            if (!rd) latch_error(prm.err, kDevTimeoutLoad, si.tile, si.k, 0);
        }
        rpar ^= 1u << y;
        owned_to_smem<Real, P, KH>(su + tb, u, own_lo, own_hi);
        owned_to_smem<Real, P, KH>(sw + tb, w, own_lo, own_hi);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_bar[y]);
        y ^= 1;
    }
}

// ---- resident tiles: one CTA keeps its tile for the whole run ----------------
// On a grid whose tiles all fit on the GPU at once (a cooperative launch of
// one CTA per tile) a span is about one wave of tiles, and reloading every
// window through global memory each span puts a load, the S steps, a store
// and a flag round trip on the critical path of every span.  Here each CTA
// keeps its window in shared memory and registers for all spans; after a span
// only the H core points next to each window end (both components) go
// through global memory: written to a double-buffered exchange slot, a
// release flag per tile, a bounded acquire wait for the two neighbours, and
// their strips become this window's halos.  The points outside the grid stay
// 0 (as in the reloading kernels, whose halo loads read the zero pads).  The
// select is the same index range, so the result is the same bit for bit.
template <typename Real>
__device__ bool wait_neighbours(const SpanParams<Real>& prm, int tile, bool left, bool right, int target, int k)
{
    auto ready = [&]() {
        return (!left || ld_acquire(prm.done + tile - 1) >= target) &&
               (!right || ld_acquire(prm.done + tile + 1) >= target);
    };
    if (ready()) return true;
    const long long t0 = global_ns();
    unsigned ns = 32;
    for (;;) {
        __nanosleep(ns);
        if (ns < 64) ns <<= 1;
        if (ready()) return true;
        if (*(volatile int*)&prm.err->code != 0) return false;
        if (global_ns() - t0 > prm.wait_ns) {
            latch_error(prm.err, kDevTimeoutFlag, tile, k, 0);
            return false;
        }
    }
}

template <typename Real, int FORM, int P, int NT, int KH, int MINB, bool USRC>
__global__ void __launch_bounds__(NT, MINB) span_kernel_res(const __grid_constant__ SpanParams<Real> prm)
{
    using G = Geom<P, NT, KH>;
    constexpr int W = G::W;
    constexpr int NW = G::NW;
    static_assert(W % 4 == 0, "windows must span whole 16-byte units");
    static_assert(KH == 0 || G::FREE || P >= 2 * KH, "this kernel refreshes warp halos");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Real* su = reinterpret_cast<Real*>(smem_raw);  // [2 components][W]: one stage
    Real* sw = su + W;
    Real* xch = su + 2 * W;
    Real* hx = xch + ((4 * NW + 15) / 16) * 16;
    __shared__ __align__(8) uint64_t full_bar;
    __shared__ ProbeDev<Real> s_probes[kTileProbes];
    __shared__ int s_ok;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const int tile = blockIdx.x;
    const TileDev td = prm.tiles[tile];
    const ProblemDev<Real>& pr = prm.problems[td.problem];
    const int H = prm.H;
    const int64_t gj0 = (int64_t)td.local * prm.core - H;
    const bool edge = (gj0 <= 0) || (gj0 + W - 1 >= pr.nx - 1);
    const bool left = td.local > 0;
    const bool right = td.local + 1 < pr.ntiles;
    const int tb = warp * G::CW + lane * P;
    int own_lo, own_hi;
    owned_range<P, NW, KH>(warp, lane, own_lo, own_hi);
    const int np = td.probe_end - td.probe_begin;
    if (np > 0 && np <= kTileProbes && tid < np) s_probes[tid] = prm.probes[td.probe_begin + tid];

    // the window at level 0
    if (tid == 0) {
        mbar_init(&full_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async_smem();
        issue_load<Real, W>(prm, (long long)tile, su, &full_bar);
    }
    __syncthreads();
    {
        const bool ok = mbar_wait_bounded(&full_bar, 0u, prm.wait_ns, &prm.err->code);
        if (!ok) latch_error(prm.err, kDevTimeoutLoad, tile, 0, 0);
        if (__syncthreads_or(!ok)) return;
    }

    for (int k = 0; k < prm.nspans; ++k) {
        const int64_t n0 = (int64_t)k * prm.S;
        const int steps = span_steps(prm, n0);
        Real u[P], w[P];
        smem_to_regs<Real, P>(su + tb, u);
        smem_to_regs<Real, P>(sw + tb, w);
        predict_tile<Real, FORM, P, NW, KH, 0, USRC, true>(prm, pr, td, u, w, gj0, n0, steps, tb, own_lo, own_hi,
                                                        s_probes, np, xch, hx, warp, lane, edge);
        __syncthreads();  // every window is read (KH > 0: they overlap) before owned points are written back
        owned_to_smem<Real, P, KH>(su + tb, u, own_lo, own_hi);
        owned_to_smem<Real, P, KH>(sw + tb, w, own_lo, own_hi);
        __syncthreads();
        if (k + 1 == prm.nspans) break;
        if (prm.ck_stride) {
            // every span state kept (the adjoint's checkpoint sweep): the core
            // of level n0 + steps into state k + 1 (the last one after the loop)
            const int64_t dst = pr.base + (int64_t)td.local * prm.core;
            Real* d0 = span_state(prm, 0, k + 1) + dst;
            Real* d1 = span_state(prm, 1, k + 1) + dst;
            for (int i = tid; i < prm.core; i += NT) {
                d0[i] = su[H + i];
                d1[i] = sw[H + i];
            }
        }

        // strips out: the first and last H core points, both components
        const int par = k & 1;
        Real* xb = prm.xbuf;
        for (int i = tid; i < 4 * H; i += NT) {
            const int side = i / (2 * H), comp = (i / H) & 1, j = i % H;
            const Real* src = (comp ? sw : su) + (side ? W - 2 * H : H) + j;
            xb[((((int64_t)tile * 2 + par) * 2 + side) * 2 + comp) * H + j] = *src;
        }
        // the CTA barrier orders every thread's strip stores before thread 0's
        // gpu-scope release of the flag, and a release is cumulative: a
        // neighbour that acquires the flag sees the strips
        __syncthreads();
        if (tid == 0) {
            // (test hook: the injected tile stops publishing from that span on, so
            // its neighbours' bounded waits expire)
            if (!(tile == prm.inject_tile && k >= prm.inject_span)) st_release(prm.done + tile, k + 1);
            s_ok = wait_neighbours(prm, tile, left, right, k + 1, k) ? 1 : 0;
        }
        __syncthreads();
        if (!s_ok) return;
        // halos in: the left neighbour's last core points, the right neighbour's first ones (L2 reads)
        for (int i = tid; i < 4 * H; i += NT) {
            const int side = i / (2 * H), comp = (i / H) & 1, j = i % H;
            if (side == 0 && left)
                (comp ? sw : su)[j] = __ldcg(xb + ((((int64_t)(tile - 1) * 2 + par) * 2 + 1) * 2 + comp) * H + j);
            if (side == 1 && right)
                (comp ? sw : su)[W - H + j] = __ldcg(xb + ((((int64_t)(tile + 1) * 2 + par) * 2 + 0) * 2 + comp) * H + j);
        }
        __syncthreads();
    }
    // the final level: the core into the state array of the last span
    const int64_t dst = pr.base + (int64_t)td.local * prm.core;
    Real* d0 = span_state(prm, 0, prm.nspans) + dst;
    Real* d1 = span_state(prm, 1, prm.nspans) + dst;
    for (int i = tid; i < prm.core; i += NT) {
        d0[i] = su[H + i];
        d1[i] = sw[H + i];
    }
}

}  // namespace rswr

// The registered variants, in variant-index order: WS = warp-specialised
// (NT compute threads + one producer warp), PLAIN = single-role CTA, RES =
// resident tiles (one CTA per tile for the whole run; small grids only).
// Arguments: kind, Real, form, P (points per thread), NT (compute threads),
// KH (warp halo; 0: warps exchange neighbours every step), MINB (CTAs per SM
// the register allocation must allow).  The first variant of each dtype/form
// that accepts a plan's span is its default (the fastest measured on the c2
// workload); the autotuner times them all.
//   FP32 increment: free warp windows (spans <= 32), then spans <= 16, then
//     refreshed warp halos (any span);  FP32 canonical;  FP64 canonical;
//   FP64 increment.
#define RSWR_SPAN_VARIANTS(X)                          \
    X(WS, float, kIncrement, 24, 128, 32, 4)           \
    X(WS, float, kIncrement, 28, 128, 32, 4)           \
    X(WS, float, kIncrement, 16, 128, 32, 5)           \
    X(WS, float, kIncrement, 24, 128, 16, 4)           \
    X(WS, float, kIncrement, 16, 128, 16, 5)           \
    X(WS, float, kIncrement, 16, 128, 8, 5)            \
    X(PLAIN, float, kIncrement, 16, 128, 8, 4)         \
    X(PLAIN, float, kIncrement, 16, 128, 0, 4)         \
    X(WS, float, kCanonical, 24, 128, 32, 4)           \
    X(PLAIN, float, kCanonical, 16, 128, 0, 4)         \
    X(WS, double, kCanonical, 8, 128, 0, 4)            \
    X(WS, double, kCanonical, 8, 256, 0, 2)            \
    X(PLAIN, double, kCanonical, 8, 128, 0, 4)         \
    X(PLAIN, double, kCanonical, 8, 256, 0, 2)         \
    X(PLAIN, double, kIncrement, 8, 256, 0, 2)         \
    X(RES, float, kIncrement, 28, 128, 32, 4)          \
    X(RES, float, kIncrement, 16, 128, 32, 5)          \
    X(RES, double, kCanonical, 8, 256, 0, 2)

namespace rswr {
// span_kernel_src.cu: variant v compiled with user point sources
const void* span_src_kernel(int v);
}  // namespace rswr
