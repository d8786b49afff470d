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

#include "rswr_internal.h"
#include "span_common.cuh"

namespace rswr {

namespace {

using namespace span;

template <typename Real, int P>
__device__ __forceinline__ Special special_points(int64_t gj, int64_t nx, int64_t js)
{
    Special sp{-1, -1, -1, 0, P - 1};
    auto loc = [&](int64_t j) -> int { return (j >= gj && j < gj + P) ? (int)(j - gj) : -1; };
    sp.r0 = loc(0);
    sp.r1 = loc(nx - 1);
    sp.rs = js >= 0 ? loc(js) : -1;
    sp.rlo = (int)(gj >= 0 ? 0 : (-gj > P ? P : -gj));
    sp.rhi = (int)(nx - 1 - gj >= P - 1 ? P - 1 : (nx - 1 - gj < -1 ? -1 : nx - 1 - gj));
    return sp;
}

__device__ __forceinline__ bool is_special(const Special& sp, int P)
{
    return sp.r0 >= 0 || sp.r1 >= 0 || sp.rs >= 0 || sp.rlo > 0 || sp.rhi < P - 1;
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

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async_smem();
    }
    __syncthreads();
    uint32_t phase = 0;

    for (int64_t tile = blockIdx.x; tile < prm.ntiles; tile += gridDim.x) {
        const TileDev td = prm.tiles[tile];
        const ProblemDev<Real>& pu = prm.prob_u[td.problem];
        const ProblemDev<Real>& pl = prm.prob_l[td.problem];
        const int64_t nx = pu.nx;
        const int64_t gj0 = (int64_t)td.local * prm.core - prm.H;
        const int64_t wabs = pu.base + gj0;
        if (tid == 0) {
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

        const int64_t gj = gj0 + (int64_t)tid * P;
        const Real c2 = pu.c2, kk = pu.k;
        const bool edge = (gj0 <= 0) || (gj0 + W - 1 >= nx - 1);
        const bool has_src = pl.js >= 0 && pl.js >= gj0 && pl.js < gj0 + W;
        const int len = prm.len;

        // ---- u phase: levels n0 .. n0+len-1, Laplacians of every level to shared memory
        {
            Real u[P], w[P];
            smem_to_regs<Real, P>(stage + 0 * W + tid * P, u);
            smem_to_regs<Real, P>(stage + 1 * W + tid * P, w);
            const Special sp = special_points<Real, P>(gj, nx, -1);
            const bool special = edge && is_special(sp, P);
            int buf = 0;
            for (int s = 0; s < len; ++s) {
                Real lft, rgt;
                exchange<Real, P, NW>(u, lft, rgt, xch, buf, warp, lane);
                buf ^= 1;
                Real* lp = laps + s * W + tid * P;
                const bool step = s + 1 < len;
                // one pass: the Laplacian of this level (from the step's own neighbour
                // sum, (uL + uR) - 2u = fma(-2, u, uL + uR) exactly) and the step
                if constexpr (FORM == kCanonical) {
                    Real ul = lft;
#pragma unroll
                    for (int i = 0; i < P; ++i) {
                        const Real uc = u[i];
                        const Real ur = i < P - 1 ? u[i + 1] : rgt;
                        const Real sum = radd(ul, ur);
                        lp[i] = rfma(Real(-2), uc, sum);
                        if (step) {
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
                        lp[i] = lap;
                        if (step) {
                            const Real v = rfma(c2, lap, w[i]);
                            w[i] = v;
                            u[i] = radd(u[i], v);
                        }
                    }
                }
                if (step && special) {
                    const int64_t n = prm.n0 + s;
                    const Real fa_old = pu.fA ? pu.fA[n] : Real(0), fa_new = pu.fA ? pu.fA[n + 1] : Real(0);
                    const Real fb_old = pu.fB ? pu.fB[n] : Real(0), fb_new = pu.fB ? pu.fB[n + 1] : Real(0);
                    patch_special<Real, FORM, P>(u, w, sp, Real(0), Real(0), fa_old, fa_new, fb_old, fb_new);
                }
            }
        }
        __syncthreads();

        // ---- lambda phase: levels m0 .. m0+len-1 pair with u levels n0+len-1 .. n0
        Real racc = Real(0);
        {
            Real l[P], lw[P];
            smem_to_regs<Real, P>(stage + 2 * W + tid * P, l);
            smem_to_regs<Real, P>(stage + 3 * W + tid * P, lw);
            const Special sp = special_points<Real, P>(gj, nx, has_src ? pl.js : -1);
            const bool special = (edge || has_src) && is_special(sp, P);
            // core points that are interior grid points: [lo, hi) in local thread indices
            const int64_t core_lo = gj0 + prm.H, core_hi = core_lo + prm.core;
            const int64_t jlo = core_lo > 1 ? core_lo : 1;
            const int64_t jhi = core_hi < nx - 1 ? core_hi : nx - 1;
            int buf = 0;
            for (int s = 0; s < len; ++s) {
                Real lft, rgt;
                exchange<Real, P, NW>(l, lft, rgt, xch, buf, warp, lane);
                buf ^= 1;
                const int64_t m = prm.m0 + s;
                if (td.probe_end > td.probe_begin)
                    record_probes<Real, P>(l, lft, rgt, wabs, tid * P, 0, P, td.probe_begin, td.probe_end, prm.probes, m);
                const Real* lp = laps + (len - 1 - s) * W + tid * P;
#pragma unroll
                for (int i = 0; i < P; ++i) {
                    const int64_t j = gj + i;
                    if (j >= jlo && j < jhi) racc = rfma(l[i], lp[i], racc);
                }
                if (special) {
                    const Real sval = sp.rs >= 0 ? pl.src[(m + 1) * pl.src_stride] : Real(0);
                    // the increment form adds the source to v before u' = u + v: keep u
                    const Real uold = (FORM == kIncrement && sp.rs >= 0) ? select_reg<Real, P>(l, sp.rs) : Real(0);
                    leap_step<Real, FORM, P>(l, lw, lft, rgt, c2, kk);
                    patch_special<Real, FORM, P>(l, lw, sp, uold, sval, Real(0), Real(0), Real(0), Real(0));
                } else {
                    leap_step<Real, FORM, P>(l, lw, lft, rgt, c2, kk);
                }
            }
            __syncthreads();
            regs_to_smem<Real, P>(stage + 2 * W + tid * P, l);
            regs_to_smem<Real, P>(stage + 3 * W + tid * P, lw);
        }
        fence_proxy_async_smem();
        double acc = (double)racc;
        // block reduction of acc in a fixed order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) red[warp] = acc;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int q = 0; q < NW; ++q) t += red[q];
            prm.partial[tile] = t;
            const int64_t dst = pu.base + (int64_t)td.local * prm.core;
            const uint32_t bytes = (uint32_t)prm.core * sizeof(Real);
            bulk_store(prm.l0_out + dst, stage + 2 * W + prm.H, bytes);
            bulk_store(prm.l1_out + dst, stage + 3 * W + prm.H, bytes);
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait_all();
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

// One block per problem; fixed-order sum over (span, tile).
__global__ void adj_reduce_kernel(const double* partial, int64_t nspans, int64_t ntiles, const int64_t* tile0,
                                  const int64_t* tcount, const double* scale, double* out)
{
    const int p = blockIdx.x;
    __shared__ double red[256];
    double acc = 0.0;
    const int64_t n = nspans * tcount[p];
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int64_t k = i / tcount[p], t = i % tcount[p];
        acc += partial[k * ntiles + tile0[p] + t];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[p] = red[0] * scale[p];
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

cudaError_t adj_reduce_launch(const double* partial, int64_t nspans, int64_t ntiles, const int64_t* tile0,
                              const int64_t* tcount, const double* scale, double* out, int nprob, cudaStream_t s)
{
    adj_reduce_kernel<<<nprob, 256, 0, s>>>(partial, nspans, ntiles, tile0, tcount, scale, out);
    return cudaGetLastError();
}

}  // namespace rswr
