// paper_kernel.cu -- RSWR exactly as the paper states it (arXiv 2203.10477,
// Sec. 2.3-2.6, Sec. 3), on the GPU: adaptive spans chosen from the data.
//
// One span:
//   rswr_iface_kernel  (one CTA per interface i | i+1, Sec. 2.3-2.4): predicts
//       subdomains i and i+1 on the part of their windows that can reach the
//       overlap within the predictive span tau (zero input-flux guess at
//       their input boundaries), records the predicted output flux waveforms
//       both neighbours need for the update (Sec. 2.5), compares the two
//       predictions on the overlap and takes, as the pair's maximum span,
//       the largest number of leading steps over which they agree exactly at
//       some overlap point; the global span is the minimum over pairs (Sec. 3,
//       atomicMin).
//   paper_select_kernel: caps the span by the Waveform Time Span Theorem
//       (Sec. 2.4), records it, and copies the span's boundary samples for the
//       span kernel.
//   rswr_resolve_kernel (tiles of each subdomain's part of the combined
//       solution, Sec. 2.5): solves the subdomain again over the span with
//       its input flux set to the neighbour's predicted output flux
//       (Neumann ghost u_{L-1} = u_{L+1} - 2 dx g, u_{R+1} = u_{R-1} + 2 dx g)
//       and writes the points of Omega_i not covered by a window further left.
//   paper_advance_kernel: the next span starts span levels later, with the
//       predictive span ceil((1 + beta) * span) (Sec. 2.6).
// The run's progress lives on the device (PaperState), so the host queues the
// kernels of many spans and reads the state back once per batch.  Simple
// kernels: one window in shared memory per CTA, a block barrier per step.
// The bulk of every span runs on the span kernel.

#include "rswr_internal.h"

namespace rswr {

namespace {

template <typename Real>
__device__ __forceinline__ void upd(int form, Real c2, Real k, Real uL, Real uC, Real uR, Real w, Real& un, Real& wn)
{
    if (form == kCanonical) {
        un = rfma(c2, radd(uL, uR), rfma(k, uC, -w));
        wn = uC;
    } else {
        const Real v = rfma(c2, radd(rsub(uL, uC), rsub(uR, uC)), w);
        un = radd(uC, v);
        wn = v;
    }
}

template <typename Real>
__device__ __forceinline__ Real dir_w(int form, Real f_old, Real f_new)
{
    return form == kCanonical ? f_old : rsub(f_new, f_old);
}

__device__ __forceinline__ int64_t win_l(int64_t i, int64_t nx, int64_t N, int64_t el)
{
    const int64_t b0 = i * nx / N;
    return b0 - el < 0 ? 0 : b0 - el;
}

__device__ __forceinline__ int64_t win_r(int64_t i, int64_t nx, int64_t N, int64_t er)
{
    const int64_t b1 = (i + 1) * nx / N;
    return b1 - 1 + er > nx - 1 ? nx - 1 : b1 - 1 + er;
}

// One step of a window [lo, hi] of subdomain `sub` held in shared memory.
// Edge rules: Dirichlet at the grid ends; at the subdomain's input boundaries
// either the zero-flux guess (g == nullptr) or the Neumann ghost from g[s];
// a cut that is not a subdomain boundary gets the mirror (its points are
// outside the part of the window that is kept).
template <typename Real>
__device__ void window_step(int form, Real c2, Real k, Real two_dx, int64_t nx, int64_t lo, int64_t hi, int64_t Lsub,
                            int64_t Rsub, const Real* gL, const Real* gR, int s, const Real* fA, const Real* fB,
                            int64_t n, const Real* u, const Real* w, Real* un, Real* wn)
{
    for (int64_t j = lo + threadIdx.x; j <= hi; j += blockDim.x) {
        const int64_t o = j - lo;
        if (j == 0) {
            const Real a0 = fA ? fA[n] : Real(0), a1 = fA ? fA[n + 1] : Real(0);
            un[o] = a1;
            wn[o] = dir_w<Real>(form, a0, a1);
            continue;
        }
        if (j == nx - 1) {
            const Real b0 = fB ? fB[n] : Real(0), b1 = fB ? fB[n + 1] : Real(0);
            un[o] = b1;
            wn[o] = dir_w<Real>(form, b0, b1);
            continue;
        }
        Real uL, uR;
        if (j == lo) {
            if (j == Lsub && gL) uL = rsub(u[o + 1], rmul(two_dx, gL[s]));
            else uL = u[o + 1];
        } else {
            uL = u[o - 1];
        }
        if (j == hi) {
            if (j == Rsub && gR) uR = radd(u[o - 1], rmul(two_dx, gR[s]));
            else uR = u[o - 1];
        } else {
            uR = u[o + 1];
        }
        upd<Real>(form, c2, k, uL, u[o], uR, w[o], un[o], wn[o]);
    }
}

template <typename Real>
__global__ void rswr_iface_kernel(const __grid_constant__ PaperParams<Real> p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t i = blockIdx.x;  // interface between subdomains i and i+1
    const int64_t nx = p.nx, N = p.N;
    const int64_t Li = win_l(i, nx, N, p.el), Ri = win_r(i, nx, N, p.er);
    const int64_t Ln = win_l(i + 1, nx, N, p.el), Rn = win_r(i + 1, nx, N, p.er);
    if (p.st && p.st->done) return;  // (every thread reads the same word)
    const int steps = p.st ? p.st->steps : p.steps;
    const int64_t n0 = p.st ? p.st->n0 : p.n0;
    const int64_t a0 = Ln - steps > Li ? Ln - steps : Li;  // prediction of i: [a0, Ri]
    const int64_t b1 = Ri + steps < Rn ? Ri + steps : Rn;  // prediction of i+1: [Ln, b1]
    const int64_t na = Ri - a0 + 1, nb = b1 - Ln + 1, nov = Ri - Ln + 1;
    Real* s = reinterpret_cast<Real*>(smem_raw);
    Real* ua = s;
    Real* wa = ua + na;
    Real* ua2 = wa + na;
    Real* wa2 = ua2 + na;
    Real* ub = wa2 + na;
    Real* wb = ub + nb;
    Real* ub2 = wb + nb;
    Real* wb2 = ub2 + nb;
    int* agree = reinterpret_cast<int*>(wb2 + nb);  // [nov]: leading steps of exact agreement, -1 = stopped
    for (int64_t o = threadIdx.x; o < na; o += blockDim.x) {
        ua[o] = p.u[a0 + o];
        wa[o] = p.w[a0 + o];
    }
    for (int64_t o = threadIdx.x; o < nb; o += blockDim.x) {
        ub[o] = p.u[Ln + o];
        wb[o] = p.w[Ln + o];
    }
    for (int64_t o = threadIdx.x; o < nov; o += blockDim.x) agree[o] = 0;
    __syncthreads();
    for (int st = 0; st < steps; ++st) {
        const int64_t n = n0 + st;
        // output flux waveforms at level n: subdomain i at Ln (for i+1), i+1 at Ri (for i)
        if (threadIdx.x == 0) {
            p.gL[(i + 1) * p.tau_stride + st] = rdiv(rsub(ua[Ln + 1 - a0], ua[Ln - 1 - a0]), p.two_dx);
            p.gR[i * p.tau_stride + st] = rdiv(rsub(ub[Ri + 1 - Ln], ub[Ri - 1 - Ln]), p.two_dx);
        }
        window_step<Real>(p.form, p.c2, p.k, p.two_dx, nx, a0, Ri, Li, Ri, nullptr, nullptr, st, p.fA, p.fB, n, ua, wa,
                          ua2, wa2);
        window_step<Real>(p.form, p.c2, p.k, p.two_dx, nx, Ln, b1, Ln, Rn, nullptr, nullptr, st, p.fA, p.fB, n, ub, wb,
                          ub2, wb2);
        __syncthreads();
        for (int64_t o = threadIdx.x; o < nov; o += blockDim.x) {
            if (agree[o] >= 0) {
                if (ua2[Ln + o - a0] == ub2[o]) agree[o] = st + 1;
                else agree[o] = -(agree[o] + 1);  // stop, remembering the count
            }
        }
        Real* t;
        t = ua; ua = ua2; ua2 = t;
        t = wa; wa = wa2; wa2 = t;
        t = ub; ub = ub2; ub2 = t;
        t = wb; wb = wb2; wb2 = t;
        __syncthreads();
    }
    // the pair's maximum span: largest agreement over the overlap
    __shared__ int best;
    if (threadIdx.x == 0) best = 0;
    __syncthreads();
    for (int64_t o = threadIdx.x; o < nov; o += blockDim.x) {
        const int a = agree[o] >= 0 ? agree[o] : -agree[o] - 1;
        atomicMax(&best, a);
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicMin(p.span_min, best);
}

template <typename Real>
__global__ void rswr_resolve_kernel(const __grid_constant__ PaperParams<Real> p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t t = blockIdx.x;
    const int64_t i = p.tile_sub[t], c0 = p.tile_lo[t], c1 = p.tile_hi[t];  // owned [c0, c1) of subdomain i
    const int64_t nx = p.nx, N = p.N;
    const int64_t Li = win_l(i, nx, N, p.el), Ri = win_r(i, nx, N, p.er);
    const int span = p.st ? p.st->span : p.steps;
    const int64_t n0 = p.st ? p.st->n0 : p.n0;
    if (span <= 0) return;  // the run is complete (every thread reads the same word)
    const int64_t lo = c0 - span > Li ? c0 - span : Li;
    const int64_t hi = c1 - 1 + span < Ri ? c1 - 1 + span : Ri;
    const int64_t nw = hi - lo + 1;
    Real* s = reinterpret_cast<Real*>(smem_raw);
    Real* u = s;
    Real* w = u + nw;
    Real* u2 = w + nw;
    Real* w2 = u2 + nw;
    for (int64_t o = threadIdx.x; o < nw; o += blockDim.x) {
        u[o] = p.u[lo + o];
        w[o] = p.w[lo + o];
    }
    __syncthreads();
    const Real* gL = (i > 0 && Li > 0) ? p.gL + i * p.tau_stride : nullptr;
    const Real* gR = (i + 1 < N && Ri < nx - 1) ? p.gR + i * p.tau_stride : nullptr;
    for (int st = 0; st < span; ++st) {
        window_step<Real>(p.form, p.c2, p.k, p.two_dx, nx, lo, hi, Li, Ri, gL, gR, st, p.fA, p.fB, n0 + st, u, w,
                          u2, w2);
        __syncthreads();
        Real* tt;
        tt = u; u = u2; u2 = tt;
        tt = w; w = w2; w2 = tt;
    }
    for (int64_t j = c0 + threadIdx.x; j < c1; j += blockDim.x) {
        p.uo[j] = u[j - lo];
        p.wo[j] = w[j - lo];
    }
}

// The re-solved zones into the combined state: points [tile_lo, tile_hi) of
// every zone tile, from the scratch pair (plain arrays) to the state pair.
template <typename Real>
__global__ void paper_scatter_kernel(const Real* su, const Real* sw, Real* du, Real* dw, const int64_t* lo,
                                     const int64_t* hi, const PaperState* st)
{
    if (st && st->span <= 0) return;  // the run is complete: nothing was re-solved
    const int64_t t = blockIdx.x;
    for (int64_t j = lo[t] + threadIdx.x; j < hi[t]; j += blockDim.x) {
        du[j] = su[j];
        dw[j] = sw[j];
    }
}

// The select step's end (Sec. 2.4, Sec. 3): the global span is the minimum
// over the pairs (the word the interface CTAs lowered), at most the
// predictive steps and the Theorem's cap, at least 1; recorded as span number
// `count`.  Then the span kernel's boundary samples: levels n0 .. n0+nsamp-1
// of fA and fB (0 past level T) into fAs, fBs.
template <typename Real>
__global__ void paper_select_kernel(PaperState* st, const int* word, int cap, const Real* fA, const Real* fB,
                                    Real* fAs, Real* fBs, int nsamp, int64_t T, int64_t* spans, int64_t spans_cap)
{
    __shared__ int s_span;
    __shared__ int64_t s_n0;
    if (threadIdx.x == 0) {
        int span = 0;
        if (!st->done) {
            span = *word < st->steps ? *word : st->steps;
            if (span > cap) span = cap;
            if (span < 1) span = 1;
            if (spans && st->count < spans_cap) spans[st->count] = span;
        }
        st->span = span;
        s_span = span;
        s_n0 = st->n0;
    }
    __syncthreads();
    if (s_span <= 0) return;
    for (int i = threadIdx.x; i < nsamp; i += blockDim.x) {
        const int64_t lv = s_n0 + i;
        fAs[i] = (fA && lv <= T) ? fA[lv] : Real(0);
        fBs[i] = (fB && lv <= T) ? fB[lv] : Real(0);
    }
}

// The next span (Sec. 2.6): n0 advances by the span, the predictive span
// becomes ceil((1 + beta) span) (beta in thousandths, exact integer
// arithmetic) capped at tau_max, the predictive steps min(tau, T - n0).
__global__ void paper_advance_kernel(PaperState* st, int64_t T, int64_t beta_m, int64_t tau_max)
{
    if (st->done || st->span <= 0) return;
    const int64_t span = st->span;
    st->n0 += span;
    st->count += 1;
    int64_t tau = (span * (1000 + beta_m) + 999) / 1000;
    if (tau > tau_max) tau = tau_max;
    st->tau = (int32_t)tau;
    const int64_t rem = T - st->n0;
    st->steps = (int32_t)(tau < rem ? tau : rem);
    st->done = st->n0 >= T ? 1 : 0;
}

}  // namespace

cudaError_t paper_select_launch(int dtype, PaperState* st, const int* word, int cap, const void* fA, const void* fB,
                                void* fAs, void* fBs, int nsamp, int64_t T, int64_t* spans, int64_t spans_cap,
                                cudaStream_t s)
{
    if (dtype == kF64)
        paper_select_kernel<double><<<1, 256, 0, s>>>(st, word, cap, static_cast<const double*>(fA),
                                                      static_cast<const double*>(fB), static_cast<double*>(fAs),
                                                      static_cast<double*>(fBs), nsamp, T, spans, spans_cap);
    else
        paper_select_kernel<float><<<1, 256, 0, s>>>(st, word, cap, static_cast<const float*>(fA),
                                                     static_cast<const float*>(fB), static_cast<float*>(fAs),
                                                     static_cast<float*>(fBs), nsamp, T, spans, spans_cap);
    return cudaGetLastError();
}

cudaError_t paper_advance_launch(PaperState* st, int64_t T, int64_t beta_m, int64_t tau_max, cudaStream_t s)
{
    paper_advance_kernel<<<1, 1, 0, s>>>(st, T, beta_m, tau_max);
    return cudaGetLastError();
}

cudaError_t paper_scatter_launch(int dtype, const void* su, const void* sw, void* du, void* dw, const int64_t* lo,
                                 const int64_t* hi, int ntiles, const PaperState* st, cudaStream_t s)
{
    if (ntiles <= 0) return cudaSuccess;
    if (dtype == kF64)
        paper_scatter_kernel<double><<<ntiles, 128, 0, s>>>(static_cast<const double*>(su),
                                                            static_cast<const double*>(sw), static_cast<double*>(du),
                                                            static_cast<double*>(dw), lo, hi, st);
    else
        paper_scatter_kernel<float><<<ntiles, 128, 0, s>>>(static_cast<const float*>(su), static_cast<const float*>(sw),
                                                           static_cast<float*>(du), static_cast<float*>(dw), lo, hi, st);
    return cudaGetLastError();
}

cudaError_t paper_iface_launch(int dtype, const void* params, int n_iface, size_t smem, cudaStream_t s)
{
    if (n_iface <= 0) return cudaSuccess;
    void* args[] = {const_cast<void*>(params)};
    const void* fn = dtype == kF64 ? reinterpret_cast<const void*>(&rswr_iface_kernel<double>)
                                   : reinterpret_cast<const void*>(&rswr_iface_kernel<float>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // (measured: 256 threads per interface 51 us per span on the c2 grid, 32 threads 62 us)
    return cudaLaunchKernel(fn, dim3(n_iface), dim3(256), args, smem, s);
}

cudaError_t paper_resolve_launch(int dtype, const void* params, int ntiles, size_t smem, cudaStream_t s)
{
    void* args[] = {const_cast<void*>(params)};
    const void* fn = dtype == kF64 ? reinterpret_cast<const void*>(&rswr_resolve_kernel<double>)
                                   : reinterpret_cast<const void*>(&rswr_resolve_kernel<float>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // zone tiles are a few span lengths wide: two warps per tile (measured on
    // the c2 grid: 34 us per span against 41 us with 256 threads)
    return cudaLaunchKernel(fn, dim3(ntiles), dim3(64), args, smem, s);
}

}  // namespace rswr
