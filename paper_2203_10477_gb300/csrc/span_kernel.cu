// span_kernel.cu -- the RSWR span kernel (predict / select / update of one
// time span over overlapping windows), sm_103a.
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

#include <cstdio>

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
    bulk_load(stage_y, prm.q0[k & 1] + off, bytes, bar);
    bulk_load(stage_y + W, prm.q1[k & 1] + off, bytes, bar);
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
template <int P, int NT, int KH>
struct Geom {
    static constexpr int NW = NT / 32;
    static constexpr int CW = KH == 0 ? 32 * P : 32 * P - 2 * KH;  // window offset between warps
    static constexpr int W = KH == 0 ? NT * P : NW * CW + 2 * KH;   // points per CTA window
    static constexpr int XCH = ((4 * NW + 15) / 16) * 16 + 8 * NW * KH;  // exchange slots (values)
};

template <typename Real, int FORM, int P, int NT, int KH, int PK, int MINB>
__global__ void __launch_bounds__(NT, MINB) span_kernel(const __grid_constant__ SpanParams<Real> prm)
{
    using G = Geom<P, NT, KH>;
    constexpr int W = G::W;
    constexpr int NW = G::NW;
    static_assert(W % 4 == 0, "windows must span whole 16-byte units");
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
        const int64_t nx = pr.nx;
        const int64_t gj0 = (int64_t)td.local * prm.core - prm.H;  // problem coordinate of window start
        const int64_t wabs = pr.base + gj0;
        const int64_t n0 = (int64_t)k * prm.S;
        const int steps = (int)((prm.T - n0 < prm.S) ? (prm.T - n0) : prm.S);
        const bool edge = (gj0 <= 0) || (gj0 + W - 1 >= nx - 1);
        const bool has_src = pr.js >= 0 && pr.js >= gj0 && pr.js < gj0 + W;
        const bool slow = edge || has_src;
        const bool has_probe = td.probe_end > td.probe_begin;
        const Real c2 = pr.c2, kk = pr.k;
        const int tb = warp * G::CW + lane * P;  // window index of the thread's first point
        const int64_t gj = gj0 + tb;
        // registers this thread owns (the others are a warp halo, KH > 0); the
        // outer halos of the first and last warp have no neighbour and belong to them
        const int own_lo = (KH > 0 && lane == 0 && warp > 0) ? KH : 0;
        const int own_hi = (KH > 0 && lane == 31 && warp < NW - 1) ? P - KH : P;

        Real* su = stage + x * 2 * W;
        Real* sw = su + W;
        Real u[P], w[P];
        smem_to_regs<Real, P>(su + tb, u);
        smem_to_regs<Real, P>(sw + tb, w);

        // probes of this tile: staged in shared memory, owners found once
        const int np = td.probe_end - td.probe_begin;
        const bool few_probes = np <= kTileProbes;
        int pq0 = -1, pq1 = -1;
        if (has_probe && few_probes) {
            if (tid < np) s_probes[tid] = prm.probes[td.probe_begin + tid];
            __syncthreads();
            owned_probes<Real, P>(s_probes, np, wabs, tb, own_lo, own_hi, pq0, pq1);
        }

        // ---- predict: S leapfrog steps of the window
        // special points of this thread (edge / source tiles only)
        Special sp{-1, -1, -1, 0, P - 1};
        bool special = false;
        if (slow) {
            const int64_t lo = gj;
            auto loc = [&](int64_t j) -> int { return (j >= lo && j < lo + P) ? (int)(j - lo) : -1; };
            sp.r0 = loc(0);
            sp.r1 = loc(nx - 1);
            sp.rs = has_src ? loc(pr.js) : -1;
            sp.rlo = (int)(lo >= 0 ? 0 : (-lo > P ? P : -lo));
            sp.rhi = (int)(nx - 1 - lo >= P - 1 ? P - 1 : (nx - 1 - lo < -1 ? -1 : nx - 1 - lo));
            special = sp.r0 >= 0 || sp.r1 >= 0 || sp.rs >= 0 || sp.rlo > 0 || sp.rhi < P - 1;
        }

        // ---- predict: S leapfrog steps of the window
        int buf = 0;
        bool done_packed = false;
        if constexpr (PK && KH > 0 && FORM == kIncrement && sizeof(Real) == 4) {
            if (!slow && !has_probe) {
                packed_increment_steps<P, NW, KH>(u, w, c2, steps, hx, buf, warp, lane);
                done_packed = true;
            }
        }
        if (done_packed) {
        } else if constexpr (KH > 0) {
            for (int s0 = 0; s0 < steps; s0 += KH) {
                if (s0 > 0) {
                    refresh_halos<Real, P, NW, KH>(u, w, hx, buf, warp, lane);
                    buf ^= 1;
                }
                const int s1 = (s0 + KH < steps) ? s0 + KH : steps;
                for (int s = s0; s < s1; ++s) {
                    Real lft, rgt;
                    warp_neighbours<Real, P>(u, lft, rgt, lane);
                    const int64_t n = n0 + s;
                    if (has_probe) {
                        if (few_probes) {
                            if (pq0 >= 0) record_owned<Real, P>(u, lft, rgt, s_probes[pq0], wabs, tb, n);
                            if (pq1 >= 0) record_owned<Real, P>(u, lft, rgt, s_probes[pq1], wabs, tb, n);
                        } else {
                            record_probes<Real, P>(u, lft, rgt, wabs, tb, own_lo, own_hi, td.probe_begin,
                                                   td.probe_end, prm.probes, n);
                        }
                    }
                    if (special) {
                        Real uold_s = Real(0), sval = Real(0);
                        if (sp.rs >= 0) {
                            sval = pr.src[(n + 1) * pr.src_stride];
                            if constexpr (FORM == kIncrement) uold_s = select_reg<Real, P>(u, sp.rs);
                        }
                        const Real fa_old = pr.fA ? pr.fA[n] : Real(0);
                        const Real fa_new = pr.fA ? pr.fA[n + 1] : Real(0);
                        const Real fb_old = pr.fB ? pr.fB[n] : Real(0);
                        const Real fb_new = pr.fB ? pr.fB[n + 1] : Real(0);
                        leap_step<Real, FORM, P>(u, w, lft, rgt, c2, kk);
                        patch_special<Real, FORM, P>(u, w, sp, uold_s, sval, fa_old, fa_new, fb_old, fb_new);
                    } else {
                        leap_step<Real, FORM, P>(u, w, lft, rgt, c2, kk);
                    }
                }
            }
        } else if (!slow && !has_probe) {
            // interior tile: halo latency hidden behind the interior updates
            for (int s = 0; s < steps; ++s) {
                split_step<Real, FORM, P, NW>(u, w, c2, kk, xch, buf, warp, lane);
                buf ^= 1;
            }
        } else
        for (int s = 0; s < steps; ++s) {
            Real lft, rgt;
            exchange<Real, P, NW>(u, lft, rgt, xch, buf, warp, lane);
            buf ^= 1;
            const int64_t n = n0 + s;
            if (has_probe) {
                if (few_probes) {
                    if (pq0 >= 0) record_owned<Real, P>(u, lft, rgt, s_probes[pq0], wabs, tb, n);
                    if (pq1 >= 0) record_owned<Real, P>(u, lft, rgt, s_probes[pq1], wabs, tb, n);
                } else {
                    record_probes<Real, P>(u, lft, rgt, wabs, tb, 0, P, td.probe_begin, td.probe_end, prm.probes, n);
                }
            }
            if (special) {
                Real uold_s = Real(0), sval = Real(0);
                if (sp.rs >= 0) {
                    sval = pr.src[(n + 1) * pr.src_stride];
                    if constexpr (FORM == kIncrement) uold_s = select_reg<Real, P>(u, sp.rs);
                }
                const Real fa_old = pr.fA ? pr.fA[n] : Real(0);
                const Real fa_new = pr.fA ? pr.fA[n + 1] : Real(0);
                const Real fb_old = pr.fB ? pr.fB[n] : Real(0);
                const Real fb_new = pr.fB ? pr.fB[n + 1] : Real(0);
                leap_step<Real, FORM, P>(u, w, lft, rgt, c2, kk);
                patch_special<Real, FORM, P>(u, w, sp, uold_s, sval, fa_old, fa_new, fb_old, fb_new);
            } else {
                leap_step<Real, FORM, P>(u, w, lft, rgt, c2, kk);
            }
        }

        // ---- select + update: write the window back, store only the core
        __syncthreads();  // every thread has read its window (KH > 0: windows overlap)
        owned_to_smem<Real, P, KH>(su + tb, u, own_lo, own_hi);
        owned_to_smem<Real, P, KH>(sw + tb, w, own_lo, own_hi);
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            const int64_t dst = pr.base + (int64_t)td.local * prm.core;
            const uint32_t bytes = (uint32_t)prm.core * sizeof(Real);
            const int b = (k + 1) & 1;
            bulk_store(prm.q0[b] + dst, su + prm.H, bytes);
            bulk_store(prm.q1[b] + dst, sw + prm.H, bytes);
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

// ---- variant registry ------------------------------------------------------

namespace {

struct Entry {
    VariantInfo info;
    const void* fn;
    size_t smem;
};

// PK: packed FP32 pairs on interior tiles; MINB: CTAs per SM the register
// allocation must allow.
template <typename Real, int FORM, int P, int NT, int KH, int PK = 0, int MINB = 2>
Entry make_entry()
{
    using G = Geom<P, NT, KH>;
    Entry e;
    e.info = VariantInfo{sizeof(Real) == 8 ? kF64 : kF32, FORM, P, NT, KH, G::W};
    e.fn = reinterpret_cast<const void*>(&span_kernel<Real, FORM, P, NT, KH, PK, MINB>);
    e.smem = sizeof(Real) * (4 * G::W + G::XCH);
    return e;
}

// The first entry of each dtype/form is its default (the fastest measured on
// the c2 workload); the autotuner times them all.
const Entry* table(int* n)
{
    static const Entry entries[] = {
        make_entry<float, kIncrement, 16, 128, 8, 0, 4>(),
        make_entry<float, kIncrement, 16, 128, 8, 0, 6>(),
        make_entry<float, kIncrement, 16, 128, 8, 1, 4>(),
        make_entry<float, kIncrement, 16, 128, 4, 0, 4>(),
        make_entry<float, kIncrement, 16, 128, 0, 0, 4>(),
        make_entry<float, kIncrement, 16, 256, 0, 0, 2>(),
        make_entry<float, kIncrement, 8, 256, 0, 0, 3>(),
        make_entry<float, kCanonical, 16, 128, 0, 0, 4>(),
        make_entry<double, kCanonical, 8, 256, 0, 0, 2>(),
        make_entry<double, kCanonical, 8, 128, 0, 0, 4>(),
        make_entry<double, kCanonical, 16, 256, 0, 0, 1>(),
        make_entry<double, kCanonical, 8, 256, 4, 0, 2>(),
        make_entry<double, kIncrement, 8, 256, 0, 0, 2>(),
    };
    *n = (int)(sizeof(entries) / sizeof(entries[0]));
    return entries;
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
    return cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e.smem);
}

cudaError_t span_occupancy(int v, int* blocks_per_sm)
{
    int n;
    const Entry& e = table(&n)[v];
    cudaError_t st = span_prepare(v);
    if (st != cudaSuccess) return st;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, e.fn, e.info.NT, e.smem);
}

cudaError_t span_launch(int v, const void* params, int grid, cudaStream_t s)
{
    int n;
    const Entry& e = table(&n)[v];
    void* args[] = {const_cast<void*>(params)};
    return cudaLaunchKernel(e.fn, dim3(grid), dim3(e.info.NT), args, e.smem, s);
}

}  // namespace rswr
