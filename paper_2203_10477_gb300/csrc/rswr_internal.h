// rswr_internal.h -- data structures shared by the RSWR kernels and the host
// runtime of librswr (not part of the public C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "rswr_device.cuh"

namespace rswr {

enum Form : int { kCanonical = 0, kIncrement = 1 };
enum DType : int { kF32 = 0, kF64 = 1 };

// One independent 1-D problem inside a plan or a batch.  Grid point j of the
// problem lives at index base + j of every state array; the arrays are padded
// with at least H zero points on both sides of every problem.
template <typename Real>
struct ProblemDev {
    int64_t base;
    int64_t nx;
    int64_t tile0;       // global index of the problem's first tile
    int64_t ntiles;
    const Real* fA;      // Dirichlet samples, level n at fA[n]; NULL means 0
    const Real* fB;
    const Real* src;     // point source: added to point js at level n: src[n * src_stride]
    int64_t src_stride;
    int64_t js;          // -1: no source
    Real c2;
    Real k;              // 2 - 2 c2
};

struct TileDev {
    int32_t problem;
    int32_t local;        // tile index within its problem (core starts at local * core)
    int32_t probe_begin;  // probes whose point lies in this tile's core
    int32_t probe_end;
    int32_t src_begin;    // user point sources whose point lies in this tile's window
    int32_t src_end;      // (halo included), in the caller's order
};

// A user point source (the pulse sources of the paper's Sec. 4 experiments):
// when level n+1 of point j is formed, samples[n+1] is added to it (canonical
// form) or to its increment v^{n+1}, which then re-forms u^{n+1} (increment
// form).  Sources at one point apply in the caller's order.
template <typename Real>
struct SrcDev {
    int64_t j;            // problem coordinate of the point (0 < j < nx-1)
    const Real* samples;  // level-n sample at samples[n], n = 0..T
};

// A per-level sample of the state: kind 0 records u_j * scale, kind 1 records
// (u_{j+1} - u_{j-1}) * scale.  Level n goes to out[n * stride] for n <= nmax.
template <typename Real>
struct ProbeDev {
    int64_t gidx;  // absolute index of point j in the state arrays
    Real* out;
    int64_t stride;
    int64_t nmax;
    Real scale;
    int32_t kind;
};

template <typename Real>
struct SpanParams {
    const ProblemDev<Real>* problems;
    const TileDev* tiles;
    const ProbeDev<Real>* probes;
    const SrcDev<Real>* srcs;  // user sources, grouped by tile (TileDev::src_begin/src_end)
    Real* q0[2];  // ping-pong state: [buffer] first component (u^n)
    Real* q1[2];  // second component (u^{n-1} canonical, v^n increment)
    int64_t ntiles;
    int64_t T;           // total steps of the run
    int32_t H;           // halo width of a CTA window (>= S)
    int32_t core;        // owned points per tile (window W = core + 2H)
    int32_t S;           // steps per span
    int32_t nspans;
    int32_t span;        // >= 0: launch covers that span only; -1: persistent over all spans
    int32_t inject_tile; // test hook: this tile never publishes span inject_span (-1: off)
    int32_t inject_span;
    int32_t pad_;
    unsigned long long* ticket;  // persistent mode: global ticket counter (zeroed per launch)
    int* done;                   // persistent mode: spans completed per tile (zeroed per launch)
    DevError* err;
    long long wait_ns;           // bound of every device-side wait
    int64_t ck_stride;           // 0: span k reads q[k & 1] and writes q[(k + 1) & 1];
                                 // > 0: span k reads q[0] + k * ck_stride and writes
                                 // q[0] + (k + 1) * ck_stride (every span state kept)
    Real* xbuf;                  // resident variants: halo strips, [tile][span parity][side][component][H]
    const int32_t* steps_dev;    // non-null: the run's length is *steps_dev (<= T), read on the device
                                 // (the paper-literal path chooses its span there); later spans of the
                                 // launch then take no steps and pass their tiles through
};

template <typename Real>
struct MonoParams {
    const Real* cur;   // u^n (canonical) / u^n (increment)
    Real* prev;        // canonical: u^{n-1} in, u^{n+1} out (in place); increment: v^n in/out
    Real* unew;        // increment: u^{n+1} out; canonical: unused
    const ProbeDev<Real>* probes;
    int32_t nprobe;
    int32_t form;
    int64_t base;
    int64_t nx;
    int64_t n;         // level of `cur`
    const Real* fA;
    const Real* fB;
    const SrcDev<Real>* srcs;   // user sources sorted by point (stable: same-point order kept)
    const int32_t* blk_src;     // [grid + 1]: the sources of step-kernel block b are [blk_src[b], blk_src[b+1])
    Real c2;
    Real k;
};

// One span of the adjoint sweep over the tiles of an adjoint tiling.  The
// forward state (u) at level n0 is recomputed for `len` levels inside the
// kernel; the adjoint state (lambda, run in reversed time) advances from level
// m0 = T - (n0 + len - 1) by `len` steps.
template <typename Real>
struct AdjParams {
    const ProblemDev<Real>* prob_u;  // forward problem: Dirichlet data, no source
    const ProblemDev<Real>* prob_l;  // adjoint problem: zero Dirichlet data, source at j_r
    const TileDev* tiles;            // adjoint tiling (probe ranges: dL/dfA samples)
    const ProbeDev<Real>* probes;
    const Real* u0;                  // forward state pair at level n0
    const Real* u1;
    const Real* l0;                  // adjoint state pair at level m0
    const Real* l1;
    Real* l0_out;                    // adjoint state pair at level m0 + len
    Real* l1_out;
    double* partial;                 // [ntiles]: sum over the span of lambda^{n+1}_j lap(u^n)_j on the core
    int64_t ntiles;
    int64_t n0;
    int64_t m0;
    int32_t len;
    int32_t H;
    int32_t core;
    int32_t pad_;
    DevError* err;
    long long wait_ns;
    // persistent sweep over all spans (every span-start state of the forward
    // problem kept): span K starts from uck0/uck1 + K * ck_stride; lambda
    // ping-pongs between lq0/lq1[0] and [1]; the spans run last first
    const Real* uck0;
    const Real* uck1;
    int64_t ck_stride;
    Real* lq0[2];
    Real* lq1[2];
    int64_t T;
    int32_t SA;
    int32_t nspans;
    unsigned long long* ticket;
    int* done;
};

// The paper-literal run's progress, kept on the device so that the host can
// queue many spans without reading each span back (paper_kernel.cu).
struct PaperState {
    int64_t n0;     // first level of the current span
    int32_t tau;    // predictive span (Sec. 2.6)
    int32_t steps;  // predictive steps of the current span: min(tau, T - n0)
    int32_t span;   // the span selected for the current span (0: the run is complete)
    int32_t count;  // spans taken so far
    int32_t done;   // 1 once n0 has reached T
    int32_t pad_;
};

// The paper-literal span (paper_kernel.cu): plain (unpadded) state arrays.
template <typename Real>
struct PaperParams {
    const Real* u;   // state pair at level n0
    const Real* w;
    Real* uo;        // combined state pair at level n0 + span
    Real* wo;
    const Real* fA;
    const Real* fB;
    Real* gL;        // [N][tau_stride]: predicted flux for the left input boundary of subdomain i
    Real* gR;        // [N][tau_stride]: ... for its right input boundary
    int* span_min;   // global span (atomicMin over interfaces)
    const int64_t* tile_sub;  // re-solve tiles: subdomain and owned range [lo, hi)
    const int64_t* tile_lo;
    const int64_t* tile_hi;
    int64_t nx, N, el, er, n0, tau_stride;
    int32_t steps;   // predictive steps (iface kernel) or selected span (re-solve kernel)
    int32_t form;
    Real c2, k, two_dx;
    const PaperState* st;  // non-null: n0, steps and the span come from here (n0 / steps above unused)
};

struct VariantInfo {
    int dtype;
    int form;
    int P;   // points per thread
    int NT;  // threads per CTA
    int KH;  // warp halo (0: warps exchange neighbours every step)
    int W;   // points per CTA window
    int threads;   // threads per CTA at launch (NT, or NT + a producer warp)
    int max_span;  // longest span the variant runs (0: any that fits the window)
    int resident;  // 1: one CTA per tile for the whole run (cooperative launch, grid = tiles)
};

// span_kernel.cu
int span_variant_count();
VariantInfo span_variant_info(int v);
size_t span_smem_bytes(int v);
cudaError_t span_prepare(int v);  // sets the dynamic shared-memory attribute
cudaError_t span_occupancy(int v, int* blocks_per_sm);
cudaError_t span_launch(int v, const void* params, int grid, cudaStream_t s);

// adjoint_kernel.cu
int adj_variant_count();
VariantInfo adj_variant_info(int v);
int adj_variant_span(int v);  // largest span the variant's shared-memory store holds
cudaError_t adj_prepare(int v);
cudaError_t adj_occupancy(int v, int* blocks_per_sm);
cudaError_t adj_launch(int v, const void* params, int grid, cudaStream_t s);
// persistent sweep over all spans (AdjParams' persistent fields), warp-specialised
cudaError_t adj_ws_prepare(int dtype, int form);
cudaError_t adj_ws_occupancy(int dtype, int form, int* blocks_per_sm);
cudaError_t adj_ws_launch(int dtype, int form, const void* params, int grid, cudaStream_t s);
int adj_ws_span(int dtype, int form);    // span the persistent kernel's Laplacian store holds (0: none)
int adj_ws_window(int dtype, int form);  // points per CTA window of the persistent kernel
int adj_ws_halo(int dtype, int form);    // tile halo the persistent kernel needs (0: any halo >= the span)
// lambda at level 1 of the reversed-time sweep: wbar[T] at j_r (interior receivers only)
cudaError_t adj_init_launch(int dtype, int form, void* l0, void* l1, const void* prob_l, int nprob,
                            const void* wbar, int64_t T, cudaStream_t s);
// dL/da[p] = 2 c2_p / a_p * sum of the partials of problem p's tiles over all
// spans, in a fixed order; tmp holds adj_reduce_blocks(nspans, nprob) * nprob doubles
int adj_reduce_blocks(int64_t nspans, int nprob);
cudaError_t adj_reduce_launch(const double* partial, int64_t nspans, int64_t ntiles, const int64_t* tile0,
                              const int64_t* tcount, const double* scale, double* out, int nprob, double* tmp,
                              cudaStream_t s);

// paper_kernel.cu
cudaError_t paper_scatter_launch(int dtype, const void* su, const void* sw, void* du, void* dw, const int64_t* lo,
                                 const int64_t* hi, int ntiles, const PaperState* st, cudaStream_t s);
cudaError_t paper_iface_launch(int dtype, const void* params, int n_iface, size_t smem, cudaStream_t s);
cudaError_t paper_select_launch(int dtype, PaperState* st, const int* word, int cap, const void* fA, const void* fB,
                                void* fAs, void* fBs, int nsamp, int64_t T, int64_t* spans, int64_t spans_cap,
                                cudaStream_t s);
cudaError_t paper_advance_launch(PaperState* st, int64_t T, int64_t beta_m, int64_t tau_max, cudaStream_t s);
cudaError_t paper_resolve_launch(int dtype, const void* params, int ntiles, size_t smem, cudaStream_t s);

// rswr_api.cu: sets the message returned by rswr_last_error_message()
void set_error_message(const char* m);

// mono_kernel.cu
constexpr int kMonoBlockPoints = 1024;  // grid points per block of the monolithic step kernel
cudaError_t mono_launch(int dtype, const void* params, cudaStream_t s);
cudaError_t probe_final_launch(int dtype, const void* probes, int nprobe, const void* q0, int64_t level,
                               cudaStream_t s);
cudaError_t set_boundary_launch(int dtype, int form, void* q0, void* q1, const void* problems, int nprob,
                                cudaStream_t s);

}  // namespace rswr
