// rswr_api.cu -- host runtime of librswr: plans, batches, the padded state
// layout, the probe tables, and the run / adjoint entry points of include/rswr.h.
//
// A plan is a batch of one problem.  Both are an Engine: a list of problems,
// each tiled into CTA windows of W = core + 2H points, stored back to back in
// four padded state arrays (two ping-pong pairs).  Device memory is allocated
// once at creation and reused by every run.

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/rswr.h"
#include "rswr_internal.h"

using namespace rswr;

namespace {

thread_local std::string g_msg;

rswr_status fail(rswr_status st, const std::string& m)
{
    g_msg = m;
    return st;
}

#define RSWR_CUDA(call)                                                                            \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(RSWR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));           \
    } while (0)

constexpr int kSpanCap = 256;     // largest span a CTA window supports
constexpr int64_t kAlign = 32;    // every problem region starts on a 32-element boundary

struct ProbHost {
    int64_t nx;
    double xa, xb, a, dt;
    int32_t n_sub, ov;
    double c, c2, k, inv2dx;
    float c2f, kf, inv2dxf;
    int64_t base = 0, tile0 = 0, ntiles = 0, off = 0;
};

// Coefficients of paper Eq. (2.1) on the uniform grid (see include/rswr.h).
void coefficients(ProbHost& p)
{
    const double dx = (p.xb - p.xa) / (double)(p.nx - 1);
    p.c = p.a * p.dt / dx;
    p.c2 = p.c * p.c;
    p.k = 2.0 - 2.0 * p.c2;
    p.inv2dx = 1.0 / (2.0 * dx);
    p.c2f = (float)p.c2;
    p.kf = 2.0f - 2.0f * p.c2f;
    p.inv2dxf = (float)p.inv2dx;
}

rswr_status validate(const rswr_problem& q)
{
    if (q.nx < 3) return fail(RSWR_EINVAL, "nx must be >= 3");
    if (!(q.a > 0.0) || !(q.dt > 0.0) || !(q.xb > q.xa)) return fail(RSWR_EINVAL, "need a > 0, dt > 0, xb > xa");
    if (q.n_sub < 1) return fail(RSWR_EINVAL, "n_sub must be >= 1");
    if (q.overlap < 2) return fail(RSWR_EOVERLAP, "overlap must be >= 2");
    if (q.nx / q.n_sub < q.overlap) return fail(RSWR_EOVERLAP, "every core must hold at least `overlap` points");
    ProbHost p{};
    p.nx = q.nx; p.xa = q.xa; p.xb = q.xb; p.a = q.a; p.dt = q.dt;
    coefficients(p);
    if (!(p.c <= 1.0)) return fail(RSWR_ECFL, "Courant number a*dt/dx = " + std::to_string(p.c) + " > 1");
    return RSWR_OK;
}

struct Engine {
    int dtype = kF64;
    int form = kCanonical;
    int device = 0;
    int num_sms = 1;
    int variant = 0;
    int mode = RSWR_MODE_PERSISTENT;
    double wait_s = 5.0;
    int64_t ck_spacing = 0;  // adjoint checkpoint spacing in spans (0: automatic)
    int S = 1, H = 4, W = 0, core = 0, P = 0, NT = 0;
    int inject_tile = -1, inject_span = -1;
    bool is_plan = true;
    bool part = false;  // a part [lo, hi) of a larger grid (rswr_plan_create_part)

    std::vector<ProbHost> probs;
    int64_t ntiles = 0, state_len = 0, packed_len = 0;
    std::vector<TileDev> h_tiles;
    std::vector<int64_t> h_offsets;

    void* q0[2] = {nullptr, nullptr};
    void* q1[2] = {nullptr, nullptr};
    size_t state_cap = 0;  // elements allocated per state array
    void* d_problems = nullptr;
    void* d_tiles = nullptr;
    size_t tiles_cap = 0;
    void* d_probes = nullptr;
    size_t probes_cap = 0;
    int64_t* d_offsets = nullptr;
    unsigned long long* d_ticket = nullptr;
    int* d_done = nullptr;
    size_t done_cap = 0;
    void* d_xbuf = nullptr;  // resident variants: halo strips of every tile
    size_t xbuf_cap = 0;     // bytes
    DevError* d_err = nullptr;
    void* d_host_stage = nullptr;  // rswr_run_host staging
    size_t host_stage_cap = 0;
    void* d_scratch[2] = {nullptr, nullptr};  // adjoint scratch outputs
    size_t scratch_cap = 0;
    cudaEvent_t ev_start = nullptr;  // caller-owned timing events (rswr_*_set_kernel_events)
    cudaEvent_t ev_stop = nullptr;
    // adjoint workspace (rswr_adjoint with dL/da): states, tables, partial sums
    void* adj_mem = nullptr;
    size_t adj_mem_cap = 0;
    PaperState* h_pstate = nullptr;  // pinned: the paper-literal run's progress, read back once per batch
    // Span states of a forward run kept in adj_mem for the next rswr_adjoint
    // (rswr_run_keep): valid while `kept` holds and the key matches.
    struct KeptKey {
        const void* fA;
        const void* fB;
        int64_t T;
        int SA, vf, va, core_f, core_a;
        int64_t C;
        bool ws;
        size_t arr, need;
        bool operator==(const KeptKey& o) const
        {
            return fA == o.fA && fB == o.fB && T == o.T && SA == o.SA && vf == o.vf && va == o.va &&
                   core_f == o.core_f && core_a == o.core_a && C == o.C && ws == o.ws && arr == o.arr &&
                   need == o.need;
        }
    };
    bool kept = false;
    KeptKey kept_key{};
    // CUDA graph of the last run's device work, replayed while the arguments repeat
    bool use_graph = true;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<int64_t> graph_key;
    // user point sources (rswr_plan_set_sources / rswr_batch_set_sources):
    // problem, point and the sample row of each, in the caller's order
    struct UserSrc {
        int64_t p, j, row;
    };
    std::vector<UserSrc> usrc;
    const void* usrc_samples = nullptr;  // device, row r at usrc_samples + r * usrc_pitch elements
    int64_t usrc_pitch = 0;
    void* d_srcs = nullptr;  // the device source tables of the last run
    size_t srcs_cap = 0;     // bytes
    bool srcs_live = false;  // the last span run's tiles hold sources (selects the kernels compiled for them)

    size_t esize() const { return dtype == kF64 ? 8 : 4; }
};

void free_engine(Engine* e)
{
    if (!e) return;
    cudaDeviceSynchronize();
    for (int b = 0; b < 2; ++b) {
        cudaFree(e->q0[b]);
        cudaFree(e->q1[b]);
        cudaFree(e->d_scratch[b]);
    }
    cudaFree(e->d_problems);
    cudaFree(e->d_tiles);
    cudaFree(e->d_probes);
    cudaFree(e->d_srcs);
    cudaFree(e->d_offsets);
    cudaFree(e->d_ticket);
    cudaFree(e->d_done);
    cudaFree(e->d_xbuf);
    if (e->h_pstate) cudaFreeHost(e->h_pstate);
    cudaFree(e->d_err);
    cudaFree(e->d_host_stage);
    cudaFree(e->adj_mem);
    if (e->graph_exec) cudaGraphExecDestroy(e->graph_exec);
    if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
    delete e;
}

bool variant_takes_span(const VariantInfo& vi, int S) { return vi.max_span == 0 || S <= vi.max_span; }

int default_variant(int dtype, int form, int S)
{
    // first registered variant of the dtype/form that runs spans of S steps
    // (resident variants fit small grids only: chosen by the autotuner or the caller)
    for (int v = 0; v < span_variant_count(); ++v) {
        const VariantInfo vi = span_variant_info(v);
        if (vi.dtype == dtype && vi.form == form && !vi.resident && variant_takes_span(vi, S)) return v;
    }
    return -1;
}

// Lays out tiles and padded problem regions for the current variant and S;
// (re)allocates the state arrays when they grow.
rswr_status layout(Engine* e)
{
    const VariantInfo vi = span_variant_info(e->variant);
    e->P = vi.P;
    e->NT = vi.NT;
    e->W = vi.W;
    e->H = (e->S + 3) / 4 * 4;
    e->core = e->W - 2 * e->H;
    if (!variant_takes_span(vi, e->S)) return fail(RSWR_EINVAL, "span longer than the warp halo of this variant");
    if (e->core < e->H || e->core < 4) return fail(RSWR_EINVAL, "span too long for the CTA window of this variant");
    const int64_t pad = e->H + 8;
    int64_t at = 0, tile = 0, off = 0;
    e->h_tiles.clear();
    e->h_offsets.assign(e->probs.size() + 1, 0);
    for (size_t p = 0; p < e->probs.size(); ++p) {
        ProbHost& ph = e->probs[p];
        ph.ntiles = (ph.nx + e->core - 1) / e->core;
        ph.base = at + pad;
        ph.tile0 = tile;
        ph.off = off;
        for (int64_t t = 0; t < ph.ntiles; ++t) e->h_tiles.push_back(TileDev{(int32_t)p, (int32_t)t, 0, 0, 0, 0});
        int64_t len = pad + ph.ntiles * e->core + pad;
        len = (len + kAlign - 1) / kAlign * kAlign;
        at += len;
        tile += ph.ntiles;
        off += ph.nx;
        e->h_offsets[p + 1] = off;
    }
    e->ntiles = tile;
    e->state_len = at;
    // alignment contract of the 1-D bulk copies: windows and cores start on
    // 16-byte boundaries and span whole 16-byte units
    if (e->H % 4 || e->core % 4 || e->W % 4) return fail(RSWR_EINVAL, "internal: misaligned tiling");
    for (const ProbHost& ph : e->probs)
        if (ph.base % 4 || ph.base - e->H < 0) return fail(RSWR_EINVAL, "internal: misaligned problem base");
    e->packed_len = off;
    if (e->ntiles > (int64_t)1 << 31) return fail(RSWR_EINVAL, "too many tiles");

    const size_t es = e->esize();
    if ((size_t)e->state_len > e->state_cap) {
        for (int b = 0; b < 2; ++b) {
            cudaFree(e->q0[b]);
            cudaFree(e->q1[b]);
            e->q0[b] = e->q1[b] = nullptr;
        }
        for (int b = 0; b < 2; ++b) {
            if (cudaMalloc(&e->q0[b], es * e->state_len) != cudaSuccess ||
                cudaMalloc(&e->q1[b], es * e->state_len) != cudaSuccess) {
                cudaGetLastError();
                e->state_cap = 0;
                return fail(RSWR_ENOMEM, "state arrays: cudaMalloc failed");
            }
        }
        e->state_cap = e->state_len;
    }
    for (int b = 0; b < 2; ++b) {
        RSWR_CUDA(cudaMemset(e->q0[b], 0, es * e->state_len));
        RSWR_CUDA(cudaMemset(e->q1[b], 0, es * e->state_len));
    }
    if (e->h_tiles.size() > e->tiles_cap) {
        cudaFree(e->d_tiles);
        e->d_tiles = nullptr;
        if (cudaMalloc(&e->d_tiles, sizeof(TileDev) * e->h_tiles.size()) != cudaSuccess)
            return fail(RSWR_ENOMEM, "tile table");
        e->tiles_cap = e->h_tiles.size();
    }
    RSWR_CUDA(cudaMemcpy(e->d_tiles, e->h_tiles.data(), sizeof(TileDev) * e->h_tiles.size(), cudaMemcpyHostToDevice));
    if ((size_t)e->ntiles > e->done_cap) {
        cudaFree(e->d_done);
        e->d_done = nullptr;
        if (cudaMalloc(&e->d_done, sizeof(int) * e->ntiles) != cudaSuccess) return fail(RSWR_ENOMEM, "flags");
        e->done_cap = e->ntiles;
    }
    RSWR_CUDA(cudaMemcpy(e->d_offsets, e->h_offsets.data(), sizeof(int64_t) * e->h_offsets.size(),
                         cudaMemcpyHostToDevice));
    if (vi.resident) {
        const size_t xb = es * 8 * (size_t)e->H * (size_t)e->ntiles;
        if (xb > e->xbuf_cap) {
            cudaFree(e->d_xbuf);
            e->d_xbuf = nullptr;
            e->xbuf_cap = 0;
            if (cudaMalloc(&e->d_xbuf, xb) != cudaSuccess) return fail(RSWR_ENOMEM, "halo exchange slots");
            e->xbuf_cap = xb;
        }
    }
    return RSWR_OK;
}

rswr_status make_engine(Engine** out, int nprob, const rswr_problem* pr, int32_t dtype, int32_t form, bool is_plan)
{
    *out = nullptr;
    if (nprob < 1 || !pr) return fail(RSWR_EINVAL, "need at least one problem");
    if (dtype != RSWR_F32 && dtype != RSWR_F64) return fail(RSWR_EINVAL, "dtype must be RSWR_F32 or RSWR_F64");
    int f;
    if (form == RSWR_FORM_DEFAULT) f = dtype == RSWR_F64 ? kCanonical : kIncrement;
    else if (form == RSWR_FORM_CANONICAL) f = kCanonical;
    else if (form == RSWR_FORM_INCREMENT) f = kIncrement;
    else return fail(RSWR_EINVAL, "bad form");
    for (int p = 0; p < nprob; ++p) {
        rswr_status st = validate(pr[p]);
        if (st != RSWR_OK) return st;
    }
    Engine* e = new (std::nothrow) Engine();
    if (!e) return fail(RSWR_ENOMEM, "host allocation");
    e->dtype = dtype == RSWR_F64 ? kF64 : kF32;
    e->form = f;
    e->is_plan = is_plan;
    int S = 1 << 30;
    for (int p = 0; p < nprob; ++p) {
        ProbHost ph{};
        ph.nx = pr[p].nx; ph.xa = pr[p].xa; ph.xb = pr[p].xb; ph.a = pr[p].a; ph.dt = pr[p].dt;
        ph.n_sub = pr[p].n_sub; ph.ov = pr[p].overlap;
        coefficients(ph);
        e->probs.push_back(ph);
        S = std::min(S, pr[p].overlap / 2);
    }
    e->S = std::min(S, kSpanCap);
    e->variant = default_variant(e->dtype, e->form, e->S);
    if (e->variant < 0) {
        delete e;
        return fail(RSWR_ENOTSUP, "no kernel variant for this dtype/form");
    }
    cudaError_t ce = cudaGetDevice(&e->device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, e->device);
    if (ce == cudaSuccess) ce = cudaMalloc(&e->d_problems, (e->dtype == kF64 ? sizeof(ProblemDev<double>)
                                                                               : sizeof(ProblemDev<float>)) * nprob);
    if (ce == cudaSuccess) ce = cudaMalloc(&e->d_offsets, sizeof(int64_t) * (nprob + 1));
    if (ce == cudaSuccess) ce = cudaMalloc(&e->d_ticket, sizeof(unsigned long long));
    if (ce == cudaSuccess) ce = cudaMalloc(&e->d_err, sizeof(DevError));
    if (ce == cudaSuccess) ce = cudaMemset(e->d_err, 0, sizeof(DevError));
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) {
        free_engine(e);
        return fail(RSWR_ECUDA, std::string("engine setup: ") + cudaGetErrorString(ce));
    }
    for (int v = 0; v < span_variant_count(); ++v) {
        ce = span_prepare(v);
        if (ce != cudaSuccess) {
            free_engine(e);
            return fail(RSWR_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(ce));
        }
    }
    rswr_status st = layout(e);
    if (st != RSWR_OK) {
        free_engine(e);
        return st;
    }
    *out = e;
    return RSWR_OK;
}

// ---- pack / unpack between caller-packed arrays and the padded layout ----

template <typename Real>
__global__ void unpack_kernel(Real* state, const Real* packed, const int64_t* offsets, int nprob,
                              const ProblemDev<Real>* problems, int64_t total)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nprob - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (offsets[mid] <= i) lo = mid; else hi = mid - 1;
        }
        state[problems[lo].base + (i - offsets[lo])] = packed[i];
    }
}

template <typename Real>
__global__ void pack_kernel(Real* packed, const Real* state, const int64_t* offsets, int nprob,
                            const ProblemDev<Real>* problems, int64_t total)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nprob - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (offsets[mid] <= i) lo = mid; else hi = mid - 1;
        }
        packed[i] = state[problems[lo].base + (i - offsets[lo])];
    }
}

int grid_for(int64_t n, int sms) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8)); }

template <typename Real>
rswr_status unpack(Engine* e, void* state, const void* packed, cudaStream_t s)
{
    if (e->probs.size() == 1) {
        RSWR_CUDA(cudaMemcpyAsync(static_cast<Real*>(state) + e->probs[0].base, packed, sizeof(Real) * e->probs[0].nx,
                                  cudaMemcpyDeviceToDevice, s));
        return RSWR_OK;
    }
    unpack_kernel<Real><<<grid_for(e->packed_len, e->num_sms), 256, 0, s>>>(
        static_cast<Real*>(state), static_cast<const Real*>(packed), e->d_offsets, (int)e->probs.size(),
        static_cast<const ProblemDev<Real>*>(e->d_problems), e->packed_len);
    RSWR_CUDA(cudaGetLastError());
    return RSWR_OK;
}

template <typename Real>
rswr_status pack(Engine* e, void* packed, const void* state, cudaStream_t s)
{
    if (e->probs.size() == 1) {
        RSWR_CUDA(cudaMemcpyAsync(packed, static_cast<const Real*>(state) + e->probs[0].base,
                                  sizeof(Real) * e->probs[0].nx, cudaMemcpyDeviceToDevice, s));
        return RSWR_OK;
    }
    pack_kernel<Real><<<grid_for(e->packed_len, e->num_sms), 256, 0, s>>>(
        static_cast<Real*>(packed), static_cast<const Real*>(state), e->d_offsets, (int)e->probs.size(),
        static_cast<const ProblemDev<Real>*>(e->d_problems), e->packed_len);
    RSWR_CUDA(cudaGetLastError());
    return RSWR_OK;
}

// ---- one run ----------------------------------------------------------

struct ProbeReq {
    int64_t p;      // problem
    int64_t j;      // grid point
    int kind;       // 0 value, 1 flux
    double scale;   // 0 -> use inv2dx (flux) / 1 (value)
    void* out;
    int64_t stride;
    int64_t nmax;
    bool scale_is_c2 = false;
};

struct RunReq {
    const void* fA = nullptr;   // packed nprob x (T+1) or single
    const void* fB = nullptr;
    int64_t T = 0;
    const void* q0 = nullptr;
    const void* q1 = nullptr;
    void* out0 = nullptr;
    void* out1 = nullptr;
    std::vector<ProbeReq> probes;
    // point sources (adjoint runs): per problem js (-1 none), src base pointer and stride
    std::vector<int64_t> js;
    const void* src = nullptr;      // packed: problem p's source starts at src + p*src_pitch
    int64_t src_pitch = 0;
    int64_t src_stride = 1;
    bool mono = false;
    bool user_src = false;  // apply the engine's user point sources
    bool from_state = false;  // continue from the engine's state q[0] as it is (no level-0 set-up)
    const int32_t* steps_dev = nullptr;  // the run's length on the device (<= T; SpanParams::steps_dev)
};

template <typename Real>
rswr_status upload_problems(Engine* e, const RunReq& r, cudaStream_t s)
{
    std::vector<ProblemDev<Real>> h(e->probs.size());
    for (size_t p = 0; p < e->probs.size(); ++p) {
        const ProbHost& ph = e->probs[p];
        ProblemDev<Real>& d = h[p];
        d.base = ph.base;
        d.nx = ph.nx;
        d.tile0 = ph.tile0;
        d.ntiles = ph.ntiles;
        d.fA = r.fA ? static_cast<const Real*>(r.fA) + p * (r.T + 1) : nullptr;
        d.fB = r.fB ? static_cast<const Real*>(r.fB) + p * (r.T + 1) : nullptr;
        d.js = (!r.js.empty() && r.src) ? r.js[p] : -1;
        d.src = (d.js >= 0) ? static_cast<const Real*>(r.src) + p * r.src_pitch : nullptr;
        d.src_stride = r.src_stride;
        if (sizeof(Real) == 8) {
            d.c2 = (Real)ph.c2;
            d.k = (Real)ph.k;
        } else {
            d.c2 = (Real)ph.c2f;
            d.k = (Real)ph.kf;
        }
    }
    RSWR_CUDA(cudaMemcpyAsync(e->d_problems, h.data(), sizeof(ProblemDev<Real>) * h.size(), cudaMemcpyHostToDevice, s));
    return RSWR_OK;
}

template <typename Real>
rswr_status upload_probes(Engine* e, const RunReq& r, int* nprobe, bool* tiles_dirty, cudaStream_t s)
{
    std::vector<ProbeDev<Real>> h;
    h.reserve(r.probes.size());
    for (const ProbeReq& q : r.probes) {
        const ProbHost& ph = e->probs[q.p];
        ProbeDev<Real> d{};
        d.gidx = ph.base + q.j;
        d.out = static_cast<Real*>(q.out);
        d.stride = q.stride;
        d.nmax = q.nmax;
        d.kind = q.kind;
        double sc = q.scale;
        if (q.scale_is_c2) d.scale = sizeof(Real) == 8 ? (Real)ph.c2 : (Real)ph.c2f;
        else if (q.kind == 1) d.scale = sizeof(Real) == 8 ? (Real)ph.inv2dx : (Real)ph.inv2dxf;
        else d.scale = (Real)sc;
        h.push_back(d);
    }
    std::sort(h.begin(), h.end(), [](const ProbeDev<Real>& a, const ProbeDev<Real>& b) { return a.gidx < b.gidx; });
    *nprobe = (int)h.size();
    // per-tile ranges over the sorted probes: a probe belongs to the tile whose core holds its point
    bool changed = false;
    size_t q = 0;
    for (size_t t = 0; t < e->h_tiles.size(); ++t) {
        TileDev& td = e->h_tiles[t];
        const int64_t lo = e->probs[td.problem].base + (int64_t)td.local * e->core;
        const int64_t hi = lo + e->core;
        while (q < h.size() && h[q].gidx < lo) ++q;
        size_t q2 = q;
        while (q2 < h.size() && h[q2].gidx < hi) ++q2;
        if (td.probe_begin != (int32_t)q || td.probe_end != (int32_t)q2) changed = true;
        td.probe_begin = (int32_t)q;
        td.probe_end = (int32_t)q2;
    }
    *tiles_dirty |= changed;
    if (!h.empty()) {
        if (h.size() > e->probes_cap) {
            RSWR_CUDA(cudaStreamSynchronize(s));
            cudaFree(e->d_probes);
            e->d_probes = nullptr;
            if (cudaMalloc(&e->d_probes, sizeof(ProbeDev<Real>) * h.size()) != cudaSuccess)
                return fail(RSWR_ENOMEM, "probe table");
            e->probes_cap = h.size();
        }
        RSWR_CUDA(cudaMemcpyAsync(e->d_probes, h.data(), sizeof(ProbeDev<Real>) * h.size(), cudaMemcpyHostToDevice, s));
    }
    return RSWR_OK;
}

int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Device tables of the user point sources of a run (one allocation):
//   span runs: SrcDev entries grouped by tile -- every source whose point lies
//     in the tile's window [t core - H, t core - H + W), in the caller's
//     order -- with the ranges in TileDev::src_begin/src_end;
//   monolithic runs: SrcDev entries sorted by point (stable), then the int32
//     CSR of the step kernel's blocks (kMonoBlockPoints points each).
// Sources at the Dirichlet nodes never apply (the boundary data wins).
template <typename Real>
rswr_status upload_sources(Engine* e, const RunReq& r, bool* tiles_dirty, int64_t* mono_blk_off, cudaStream_t s)
{
    *mono_blk_off = -1;
    e->srcs_live = false;
    std::vector<std::pair<int64_t, SrcDev<Real>>> ent;  // (sort key, entry)
    const bool use = r.user_src && !e->usrc.empty();
    if (use) {
        if (e->usrc_pitch < r.T + 1) return fail(RSWR_EINVAL, "source samples hold fewer than T+1 levels");
        for (const Engine::UserSrc& q : e->usrc) {
            const ProbHost& ph = e->probs[q.p];
            if (q.j <= 0 || q.j >= ph.nx - 1) continue;
            const SrcDev<Real> d{q.j, static_cast<const Real*>(e->usrc_samples) + q.row * e->usrc_pitch};
            if (r.mono) {
                ent.push_back({q.j, d});
                continue;
            }
            const int64_t t_lo = std::max<int64_t>(0, floor_div(q.j + e->H - e->W, e->core) + 1);
            const int64_t t_hi = std::min<int64_t>(ph.ntiles - 1, floor_div(q.j + e->H, e->core));
            for (int64_t t = t_lo; t <= t_hi; ++t) ent.push_back({ph.tile0 + t, d});
        }
        std::stable_sort(ent.begin(), ent.end(),
                         [](const std::pair<int64_t, SrcDev<Real>>& a, const std::pair<int64_t, SrcDev<Real>>& b) {
                             return a.first < b.first;
                         });
    }
    // tile ranges (empty for monolithic runs and runs without sources)
    size_t q = 0;
    for (size_t t = 0; t < e->h_tiles.size(); ++t) {
        TileDev& td = e->h_tiles[t];
        size_t q2 = q;
        if (!r.mono)
            while (q2 < ent.size() && ent[q2].first == (int64_t)t) ++q2;
        if (td.src_begin != (int32_t)q || td.src_end != (int32_t)q2) *tiles_dirty = true;
        td.src_begin = (int32_t)q;
        td.src_end = (int32_t)q2;
        q = q2;
    }
    if (ent.empty()) return RSWR_OK;
    std::vector<SrcDev<Real>> tab;
    tab.reserve(ent.size());
    for (const auto& x : ent) tab.push_back(x.second);
    std::vector<int32_t> blk;
    if (r.mono) {
        const int64_t nblk = (e->probs[0].nx + kMonoBlockPoints - 1) / kMonoBlockPoints;
        blk.resize(nblk + 1);
        size_t i = 0;
        for (int64_t b = 0; b <= nblk; ++b) {
            while (i < ent.size() && ent[i].first < b * kMonoBlockPoints) ++i;
            blk[b] = (int32_t)i;
        }
    }
    const size_t tab_bytes = sizeof(SrcDev<Real>) * tab.size();
    const size_t need = tab_bytes + sizeof(int32_t) * blk.size();
    if (need > e->srcs_cap) {
        RSWR_CUDA(cudaStreamSynchronize(s));
        cudaFree(e->d_srcs);
        e->d_srcs = nullptr;
        e->srcs_cap = 0;
        if (cudaMalloc(&e->d_srcs, need) != cudaSuccess) return fail(RSWR_ENOMEM, "source table");
        e->srcs_cap = need;
    }
    std::vector<unsigned char> host(need);
    std::memcpy(host.data(), tab.data(), tab_bytes);
    if (!blk.empty()) std::memcpy(host.data() + tab_bytes, blk.data(), sizeof(int32_t) * blk.size());
    RSWR_CUDA(cudaMemcpyAsync(e->d_srcs, host.data(), need, cudaMemcpyHostToDevice, s));
    if (r.mono) *mono_blk_off = (int64_t)tab_bytes;
    else e->srcs_live = true;
    return RSWR_OK;
}

template <typename Real>
SpanParams<Real> span_params(Engine* e, int64_t T, int nspans)
{
    SpanParams<Real> prm{};
    prm.problems = static_cast<const ProblemDev<Real>*>(e->d_problems);
    prm.tiles = static_cast<const TileDev*>(e->d_tiles);
    prm.probes = static_cast<const ProbeDev<Real>*>(e->d_probes);
    prm.srcs = e->srcs_live ? static_cast<const SrcDev<Real>*>(e->d_srcs) : nullptr;
    for (int b = 0; b < 2; ++b) {
        prm.q0[b] = static_cast<Real*>(e->q0[b]);
        prm.q1[b] = static_cast<Real*>(e->q1[b]);
    }
    prm.ntiles = e->ntiles;
    prm.T = T;
    prm.H = e->H;
    prm.core = e->core;
    prm.S = e->S;
    prm.nspans = nspans;
    prm.span = -1;
    prm.inject_tile = e->inject_tile;
    prm.inject_span = e->inject_span;
    prm.ticket = e->d_ticket;
    prm.done = e->d_done;
    prm.xbuf = static_cast<Real*>(e->d_xbuf);
    prm.err = e->d_err;
    prm.wait_ns = (long long)(e->wait_s * 1e9);
    return prm;
}

template <typename Real>
rswr_status prepare_tables(Engine* e, const RunReq& r, int* nprobe, int64_t* mono_blk_off, cudaStream_t s)
{
    rswr_status st = upload_problems<Real>(e, r, s);
    if (st != RSWR_OK) return st;
    bool dirty = false;
    if ((st = upload_probes<Real>(e, r, nprobe, &dirty, s)) != RSWR_OK) return st;
    if ((st = upload_sources<Real>(e, r, &dirty, mono_blk_off, s)) != RSWR_OK) return st;
    if (dirty)
        RSWR_CUDA(cudaMemcpyAsync(e->d_tiles, e->h_tiles.data(), sizeof(TileDev) * e->h_tiles.size(),
                                  cudaMemcpyHostToDevice, s));
    return RSWR_OK;
}

// The device work of one run (capturable in a CUDA graph: no host sync, no
// host-to-device copies).
template <typename Real>
rswr_status device_work(Engine* e, const RunReq& r, int nprobe, int64_t mono_blk_off, cudaStream_t s)
{
    const size_t es = sizeof(Real);
    rswr_status st = RSWR_OK;
    if (!r.from_state) RSWR_CUDA(cudaMemsetAsync(e->d_err, 0, sizeof(DevError), s));

    // level-0 state into buffer 0
    if (r.from_state) {
        // the state is already in buffer 0 (a continued run)
    } else if (!r.q0) {
        RSWR_CUDA(cudaMemsetAsync(e->q0[0], 0, es * e->state_len, s));
        RSWR_CUDA(cudaMemsetAsync(e->q1[0], 0, es * e->state_len, s));
    } else {
        if ((st = unpack<Real>(e, e->q0[0], r.q0, s)) != RSWR_OK) return st;
        if (r.q1) {
            if ((st = unpack<Real>(e, e->q1[0], r.q1, s)) != RSWR_OK) return st;
        } else if (e->form == kCanonical) {
            if ((st = unpack<Real>(e, e->q1[0], r.q0, s)) != RSWR_OK) return st;
        } else {
            RSWR_CUDA(cudaMemsetAsync(e->q1[0], 0, es * e->state_len, s));
        }
    }
    if (!r.from_state)
        RSWR_CUDA(set_boundary_launch(e->dtype, e->form, e->q0[0], e->q1[0], e->d_problems, (int)e->probs.size(), s));

    const void* fin0;
    const void* fin1;
    if (e->ev_start) RSWR_CUDA(cudaEventRecordWithFlags(e->ev_start, s, cudaEventRecordExternal));
    if (!r.mono) {
        const int nspans = (int)((r.T + e->S - 1) / e->S);
        SpanParams<Real> prm = span_params<Real>(e, r.T, nspans);
        prm.steps_dev = r.steps_dev;
        int bps = 0;
        RSWR_CUDA(span_occupancy(e->variant, &bps));
        if (bps < 1) return fail(RSWR_ENOTSUP, "span kernel does not fit on an SM");
        if (nspans > 0) {
            if (span_variant_info(e->variant).resident) {
                // one CTA per tile for the whole run: every tile must be resident at once
                if ((int64_t)bps * e->num_sms < e->ntiles)
                    return fail(RSWR_ENOTSUP, "resident variant: " + std::to_string(e->ntiles) +
                                                  " tiles do not fit on the GPU at once");
                RSWR_CUDA(cudaMemsetAsync(e->d_done, 0, sizeof(int) * e->ntiles, s));
                RSWR_CUDA(span_launch(e->variant, &prm, (int)e->ntiles, s));
            } else if (e->mode == RSWR_MODE_PERSISTENT) {
                RSWR_CUDA(cudaMemsetAsync(e->d_ticket, 0, sizeof(unsigned long long), s));
                RSWR_CUDA(cudaMemsetAsync(e->d_done, 0, sizeof(int) * e->ntiles, s));
                const int grid = (int)std::min<int64_t>((int64_t)bps * e->num_sms, (int64_t)nspans * e->ntiles);
                RSWR_CUDA(span_launch(e->variant, &prm, grid, s));
            } else {
                const int grid = (int)std::min<int64_t>((int64_t)bps * e->num_sms, e->ntiles);
                for (int k = 0; k < nspans; ++k) {
                    prm.span = k;
                    RSWR_CUDA(span_launch(e->variant, &prm, grid, s));
                }
            }
        }
        fin0 = e->q0[nspans & 1];
        fin1 = e->q1[nspans & 1];
    } else {
        // monolithic: canonical alternates u^n between q0[0] and q1[0]; increment keeps v in q1[0]
        MonoParams<Real> mp{};
        mp.probes = static_cast<const ProbeDev<Real>*>(e->d_probes);
        mp.nprobe = nprobe;
        mp.form = e->form;
        const ProbHost& ph = e->probs[0];
        mp.base = ph.base;
        mp.nx = ph.nx;
        mp.fA = static_cast<const Real*>(r.fA);
        mp.fB = static_cast<const Real*>(r.fB);
        if (mono_blk_off >= 0) {
            mp.srcs = static_cast<const SrcDev<Real>*>(e->d_srcs);
            mp.blk_src = reinterpret_cast<const int32_t*>(static_cast<const char*>(e->d_srcs) + mono_blk_off);
        }
        mp.c2 = sizeof(Real) == 8 ? (Real)ph.c2 : (Real)ph.c2f;
        mp.k = sizeof(Real) == 8 ? (Real)ph.k : (Real)ph.kf;
        Real* a = static_cast<Real*>(e->q0[0]);
        Real* b = static_cast<Real*>(e->q1[0]);
        Real* ua = static_cast<Real*>(e->q0[0]);
        Real* ub = static_cast<Real*>(e->q0[1]);
        for (int64_t n = 0; n < r.T; ++n) {
            mp.n = n;
            if (e->form == kCanonical) {
                mp.cur = a;
                mp.prev = b;
                mp.unew = nullptr;
                RSWR_CUDA(mono_launch(e->dtype, &mp, s));
                std::swap(a, b);
            } else {
                mp.cur = ua;
                mp.prev = b;
                mp.unew = ub;
                RSWR_CUDA(mono_launch(e->dtype, &mp, s));
                std::swap(ua, ub);
            }
        }
        if (e->form == kCanonical) {
            fin0 = a;
            fin1 = b;
        } else {
            fin0 = ua;
            fin1 = b;
        }
    }
    if (e->ev_stop) RSWR_CUDA(cudaEventRecordWithFlags(e->ev_stop, s, cudaEventRecordExternal));
    RSWR_CUDA(probe_final_launch(e->dtype, e->d_probes, nprobe, fin0, r.T, s));
    if (r.out0 && (st = pack<Real>(e, r.out0, fin0, s)) != RSWR_OK) return st;
    if (r.out1 && (st = pack<Real>(e, r.out1, fin1, s)) != RSWR_OK) return st;
    return RSWR_OK;
}

// Everything that determines the device work of a run.
std::vector<int64_t> run_key(const Engine* e, const RunReq& r)
{
    auto P = [](const void* p) { return (int64_t)(intptr_t)p; };
    std::vector<int64_t> k{r.mono, P(r.fA), P(r.fB), r.T, P(r.q0), P(r.q1), P(r.out0), P(r.out1), P(r.src),
                           r.src_pitch, r.src_stride, e->variant, e->mode, e->S, e->H, P(e->ev_start),
                           P(e->ev_stop), e->inject_tile, e->inject_span, (int64_t)(e->wait_s * 1e3),
                           (int64_t)r.probes.size(), r.user_src ? (int64_t)e->usrc.size() : -1, P(e->d_srcs),
                           e->srcs_live};
    for (const ProbeReq& q : r.probes) {
        k.insert(k.end(), {q.p, q.j, q.kind, P(q.out), q.stride, q.nmax, q.scale_is_c2});
        int64_t sb;
        std::memcpy(&sb, &q.scale, sizeof(sb));
        k.push_back(sb);
    }
    k.insert(k.end(), r.js.begin(), r.js.end());
    return k;
}

template <typename Real>
rswr_status run_graph(Engine* e, const RunReq& r, int nprobe, int64_t mono_blk_off, cudaStream_t s)
{
    std::vector<int64_t> key = run_key(e, r);
    key.push_back(mono_blk_off);
    if (!e->graph_exec || key != e->graph_key) {
        if (e->graph_exec) {
            cudaGraphExecDestroy(e->graph_exec);
            e->graph_exec = nullptr;
        }
        e->graph_key.clear();
        RSWR_CUDA(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal));
        rswr_status st = device_work<Real>(e, r, nprobe, mono_blk_off, e->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(e->cap_stream, &g);
        if (st != RSWR_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (ce != cudaSuccess) return fail(RSWR_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&e->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            e->graph_exec = nullptr;
            return fail(RSWR_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        }
        e->graph_key = key;
    }
    RSWR_CUDA(cudaGraphLaunch(e->graph_exec, s));
    return RSWR_OK;
}

template <typename Real>
rswr_status run_impl(Engine* e, const RunReq& r, cudaStream_t s)
{
    int nprobe = 0;
    int64_t mono_blk_off = -1;
    rswr_status st = prepare_tables<Real>(e, r, &nprobe, &mono_blk_off, s);
    if (st != RSWR_OK) return st;
    // resident variants launch cooperatively: directly, not from a captured graph
    if (e->use_graph && !span_variant_info(e->variant).resident) return run_graph<Real>(e, r, nprobe, mono_blk_off, s);
    return device_work<Real>(e, r, nprobe, mono_blk_off, s);
}

rswr_status run_engine(Engine* e, const RunReq& r, cudaStream_t s)
{
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != e->device) RSWR_CUDA(cudaSetDevice(e->device));
    rswr_status st = e->dtype == kF64 ? run_impl<double>(e, r, s) : run_impl<float>(e, r, s);
    if (cur != e->device && cur >= 0) cudaSetDevice(cur);
    return st;
}

rswr_status check_engine(Engine* e, cudaStream_t s, int32_t* code, int32_t* tile, int32_t* span)
{
    RSWR_CUDA(cudaStreamSynchronize(s));
    DevError h{};
    RSWR_CUDA(cudaMemcpy(&h, e->d_err, sizeof(h), cudaMemcpyDeviceToHost));
    if (code) *code = h.code;
    if (tile) *tile = h.tile;
    if (span) *span = h.span;
    if (h.code == kDevTimeoutLoad || h.code == kDevTimeoutFlag)
        return fail(RSWR_ETIMEOUT, "device wait expired (code " + std::to_string(h.code) + ", tile " +
                                       std::to_string(h.tile) + ", span " + std::to_string(h.span) + ")");
    if (h.code != 0) return fail(RSWR_ECUDA, "device error code " + std::to_string(h.code));
    return RSWR_OK;
}

rswr_status fill_info(const Engine* e, rswr_plan_info* info)
{
    if (!e || !info) return fail(RSWR_EINVAL, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    const ProbHost& p = e->probs[0];
    info->nx = p.nx;
    info->dtype = e->dtype == kF64 ? RSWR_F64 : RSWR_F32;
    info->form = e->form == kCanonical ? RSWR_FORM_CANONICAL : RSWR_FORM_INCREMENT;
    info->n_sub = p.n_sub;
    info->overlap = p.ov;
    info->c = p.c;
    info->c2 = p.c2;
    info->k = p.k;
    info->inv2dx = p.inv2dx;
    info->c2f = p.c2f;
    info->kf = p.kf;
    info->inv2dxf = p.inv2dxf;
    info->span_steps = e->S;
    info->halo = e->H;
    info->core = e->core;
    info->window = e->W;
    info->points_per_thread = e->P;
    info->threads_per_cta = e->NT;
    info->variant = e->variant;
    info->mode = e->mode;
    info->ntiles = e->ntiles;
    info->state_len = e->state_len;
    info->workspace_bytes = (int64_t)(4 * e->state_cap * e->esize());
    return RSWR_OK;
}

rswr_status set_variant(Engine* e, int32_t v)
{
    if (v < 0 || v >= span_variant_count()) return fail(RSWR_EINVAL, "variant out of range");
    const VariantInfo vi = span_variant_info(v);
    if (vi.dtype != e->dtype || vi.form != e->form) return fail(RSWR_EINVAL, "variant has another dtype or form");
    const int old = e->variant;
    e->variant = v;
    rswr_status st = layout(e);
    if (st != RSWR_OK) {
        e->variant = old;
        layout(e);
    }
    return st;
}

// interface output-waveform probes of one problem (see rswr_run)
void add_trace_probes(const ProbHost& ph, int64_t p, void* traces, int64_t T, size_t es, std::vector<ProbeReq>& out)
{
    const int64_t N = ph.n_sub, el = (ph.ov + 1) / 2, er = ph.ov / 2;
    for (int64_t i = 0; i + 1 < N; ++i) {
        const int64_t b1 = (i + 1) * ph.nx / N;
        const int64_t Lnext = std::max<int64_t>(b1 - el, 0);
        const int64_t Rthis = std::min<int64_t>(b1 - 1 + er, ph.nx - 1);
        char* base = static_cast<char*>(traces);
        out.push_back(ProbeReq{p, Lnext, 1, 0.0, base + es * ((2 * i + 0) * (T + 1)), 1, T});
        out.push_back(ProbeReq{p, Rthis, 1, 0.0, base + es * ((2 * i + 1) * (T + 1)), 1, T});
    }
}

rswr_status plan_run(Engine* e, const void* fA, const void* fB, int64_t T, const void* q0, const void* q1, void* out0,
                     void* out1, void* traces, int64_t j_r, void* recv, void* stream, bool mono)
{
    if (!e) return fail(RSWR_EINVAL, "NULL plan");
    if (T < 0 || T > ((int64_t)1 << 40)) return fail(RSWR_EINVAL, "T out of range");
    if (!out0 || !out1) return fail(RSWR_EINVAL, "out0 and out1 are required");
    const ProbHost& ph = e->probs[0];
    if (recv && (j_r < 0 || j_r >= ph.nx)) return fail(RSWR_EINVAL, "receiver index outside the grid");
    if (e->inject_tile >= 0 && mono) return fail(RSWR_EINVAL, "fault injection applies to RSWR runs only");
    RunReq r;
    r.fA = fA;
    r.fB = fB;
    r.T = T;
    r.q0 = q0;
    r.q1 = q1;
    r.out0 = out0;
    r.out1 = out1;
    r.mono = mono;
    r.user_src = true;
    if (traces) add_trace_probes(ph, 0, traces, T, e->esize(), r.probes);
    if (recv) r.probes.push_back(ProbeReq{0, j_r, 0, 1.0, recv, 1, T});
    return run_engine(e, r, static_cast<cudaStream_t>(stream));
}

rswr_status set_sources(Engine* e, int64_t nsrc, const int32_t* problem, const int64_t* j, const void* samples,
                        int64_t pitch)
{
    if (nsrc < 0 || nsrc > ((int64_t)1 << 24)) return fail(RSWR_EINVAL, "source count out of range");
    std::vector<Engine::UserSrc> v;
    if (nsrc > 0) {
        if (!j || !samples) return fail(RSWR_EINVAL, "points and samples are required");
        if (pitch < 1) return fail(RSWR_EINVAL, "sample pitch must be >= 1");
        if (reinterpret_cast<uintptr_t>(samples) % e->esize()) return fail(RSWR_EINVAL, "misaligned samples");
        v.reserve(nsrc);
        for (int64_t q = 0; q < nsrc; ++q) {
            const int64_t p = problem ? problem[q] : 0;
            if (p < 0 || p >= (int64_t)e->probs.size()) return fail(RSWR_EINVAL, "source problem out of range");
            if (j[q] < 0 || j[q] >= e->probs[p].nx) return fail(RSWR_EINVAL, "source point outside the grid");
            v.push_back(Engine::UserSrc{p, j[q], q});
        }
    }
    e->usrc = std::move(v);
    e->usrc_samples = nsrc > 0 ? samples : nullptr;
    e->usrc_pitch = nsrc > 0 ? pitch : 0;
    return RSWR_OK;
}

// dL/dfA of a receiver-trace functional: the adjoint variables run forward in
// reversed time (level m = lambda^{T+1-m}) from rest, with zero Dirichlet data
// and the source wbar[T-n] entering at step n -> n+1 at j_r; the probe at
// j = 1 with scale c2 yields grad[T - m] = c2 lambda^{T+1-m}_1.
rswr_status adjoint_g(Engine* e, int64_t T, const int64_t* j_r, const void* wbar, void* grad, cudaStream_t s)
{
    const size_t es = e->esize();
    const int np = (int)e->probs.size();
    if (e->scratch_cap < (size_t)e->packed_len) {
        for (int b = 0; b < 2; ++b) {
            cudaFree(e->d_scratch[b]);
            e->d_scratch[b] = nullptr;
            if (cudaMalloc(&e->d_scratch[b], es * e->packed_len) != cudaSuccess) return fail(RSWR_ENOMEM, "scratch");
        }
        e->scratch_cap = e->packed_len;
    }
    RunReq r;
    r.T = T + 1;
    r.out0 = e->d_scratch[0];
    r.out1 = e->d_scratch[1];
    r.js.assign(np, -1);
    r.src = static_cast<const char*>(wbar) + es * (T + 1);
    r.src_pitch = T + 1;
    r.src_stride = -1;
    RSWR_CUDA(cudaMemsetAsync(grad, 0, es * (T + 1) * np, s));
    bool any = false;
    for (int p = 0; p < np; ++p) {
        const int64_t j = j_r[p];
        char* g = static_cast<char*>(grad) + es * (T + 1) * p;
        if (j == 0) {
            // the receiver is the Dirichlet node itself: dL/dfA = wbar
            RSWR_CUDA(cudaMemcpyAsync(g, static_cast<const char*>(wbar) + es * (T + 1) * p, es * (T + 1),
                                      cudaMemcpyDeviceToDevice, s));
            continue;
        }
        if (j >= e->probs[p].nx - 1) continue;  // right Dirichlet node: no dependence on fA
        r.js[p] = j;
        ProbeReq q{p, 1, 0, 0.0, g + es * T, -1, T};
        q.scale_is_c2 = true;
        r.probes.push_back(q);
        any = true;
    }
    if (!any) return RSWR_OK;
    return run_engine(e, r, s);
}

}  // namespace

namespace {

// Gradients of <wbar, receiver trace> w.r.t. fA and a with the forward levels
// recomputed from checkpoints (see adjoint_kernel.cu for the kernel side).
//   spans of SA steps (SA <= the adjoint variant's shared-memory store and <= S);
//   checkpoints every C = ceil(sqrt(#spans)) spans during one forward sweep;
//   per segment of C spans, last first: the span kernel recomputes the state at
//   the start of every span of the segment, then the adjoint kernel runs the
//   segment's spans last first (reversed-time adjoint levels ascending).
// Forward-only use of the sweep below (rswr_run_keep): keep every span state,
// record the receiver trace, write the final state pair.
struct KeepReq {
    int64_t j_rec;  // receiver grid index, or -1
    void* recv;     // T+1 samples, or NULL
    void* out0;
    void* out1;
};

template <typename Real>
rswr_status adjoint_full(Engine* e, int64_t T, const int64_t* j_r, const void* fA, const void* fB, const void* wbar,
                         void* grad, double* grad_a, cudaStream_t s, const KeepReq* keep = nullptr)
{
    const int np = (int)e->probs.size();
    const size_t es = sizeof(Real);
    int va = -1;
    for (int v = 0; v < adj_variant_count(); ++v) {
        const VariantInfo vi = adj_variant_info(v);
        if (vi.dtype == e->dtype && vi.form == e->form) {
            va = v;
            break;
        }
    }
    if (va < 0) return fail(RSWR_ENOTSUP, "no adjoint kernel for this dtype/form");
    const VariantInfo ai = adj_variant_info(va);
    const int SA = std::min(e->S, adj_variant_span(va));
    // halo of both tilings: at least the span (rounded to 16 bytes of FP32);
    // the persistent FP32 sweep's free warp windows ask for their own below
    int H = (SA + 3) / 4 * 4;
    // the sweeps launch span by span or with tickets: a resident plan variant
    // gives way to the default one of its dtype and form (but runs the
    // checkpoint sweep itself when every span state is kept; below)
    const VariantInfo vplan = span_variant_info(e->variant);
    const int v_default = default_variant(e->dtype, e->form, SA);
    int vf = vplan.resident ? v_default : e->variant;
    if (vf < 0) return fail(RSWR_ENOTSUP, "no span kernel variant for the adjoint sweep");
    VariantInfo fi = span_variant_info(vf);
    int core_f = fi.W - 2 * H;
    int64_t pad = H + 8;
    const int64_t nspans = (T + SA - 1) / SA;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };

    // layout shared by the forward tiling (core_f) and the adjoint tiling (core_a)
    std::vector<int64_t> base(np), t0f(np), tcf(np), t0a(np), tca(np);
    int64_t ntf = 0, nta = 0, slen = 0;
    size_t arr = 0;
    int core_a = 0;
    auto make_layout = [&](int ca) {
        core_a = ca;
        int64_t at = 0;
        ntf = nta = 0;
        for (int p = 0; p < np; ++p) {
            const int64_t nx = e->probs[p].nx;
            tcf[p] = (nx + core_f - 1) / core_f;
            tca[p] = (nx + core_a - 1) / core_a;
            t0f[p] = ntf;
            t0a[p] = nta;
            ntf += tcf[p];
            nta += tca[p];
            base[p] = at + pad;
            int64_t len = pad + std::max(tcf[p] * core_f, tca[p] * core_a) + pad;
            at += (len + kAlign - 1) / kAlign * kAlign;
        }
        slen = at;
        arr = up(es * slen);
    };
    // Checkpoint spacing: every span boundary when all of them fit in half of the
    // free device memory (no recompute sweep), else sqrt(#spans) of them.
    auto spacing = [&]() -> int64_t {
        if (e->ck_spacing > 0) return std::min<int64_t>(e->ck_spacing, std::max<int64_t>(nspans, 1));
        int64_t c = std::max<int64_t>(1, (int64_t)std::ceil(std::sqrt((double)std::max<int64_t>(nspans, 1))));
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            const size_t avail = free_b + e->adj_mem_cap;
            if ((size_t)(nspans + 6) * 2 * arr < avail / 2) c = 1;
        } else {
            cudaGetLastError();
        }
        return c;
    };
    // With every span state kept the whole adjoint sweep is one persistent launch
    // (its own window); otherwise one launch of the per-span kernel per span.
    const int w_ws = adj_ws_window(e->dtype, e->form);
    const int h_ws = adj_ws_halo(e->dtype, e->form);  // 0: any halo >= the span
    bool use_ws = w_ws > 0 && adj_ws_span(e->dtype, e->form) >= SA &&
                  (h_ws > 0 ? h_ws >= H && fi.W - 2 * h_ws >= h_ws && w_ws - 2 * h_ws >= h_ws : w_ws - 2 * H >= H);
    if (core_f < H || ai.W - 2 * H < H) return fail(RSWR_EINVAL, "adjoint tiling: window too small");
    const int H_span = H;
    auto set_halo = [&](int h) {
        H = h;
        core_f = fi.W - 2 * H;
        pad = H + 8;
    };
    int64_t C;
    if (use_ws) {
        if (h_ws > 0) set_halo(h_ws);
        make_layout(w_ws - 2 * H);
        C = spacing();
        if (C != 1) {
            use_ws = false;
            set_halo(H_span);
        }
    }
    if (!use_ws) {
        make_layout(ai.W - 2 * H);
        C = spacing();
    }
    // A resident plan variant runs the checkpoint sweep when every span state
    // is kept (one launch, the tile windows on chip, each span's core written
    // out) and the sweep's tiles all fit on the GPU at once: on small grids the
    // ticketed sweep is paced by one tile's chain per span.
    bool res_sweep = false;
    if (vplan.resident && use_ws && C == 1 && variant_takes_span(vplan, SA) && vplan.W - 2 * H >= H) {
        const int core_r = vplan.W - 2 * H;
        int64_t ntr = 0;
        for (int p = 0; p < np; ++p) ntr += (e->probs[p].nx + core_r - 1) / core_r;
        int bps_r = 0;
        RSWR_CUDA(span_occupancy(e->variant, &bps_r));
        if ((int64_t)bps_r * e->num_sms >= ntr) {
            vf = e->variant;
            fi = vplan;
            core_f = core_r;
            make_layout(w_ws - 2 * H);
            C = spacing();
            res_sweep = C == 1;
            if (!res_sweep) {
                vf = v_default;
                fi = span_variant_info(vf);
                core_f = fi.W - 2 * H;
                make_layout(w_ws - 2 * H);
                C = spacing();
                if (C != 1) {
                    use_ws = false;
                    set_halo(H_span);
                    make_layout(ai.W - 2 * H);
                    C = spacing();
                }
            }
        }
    }
    if (keep && C != 1) return fail(RSWR_ENOMEM, "the span states of this run do not fit in device memory");
    const int64_t nck = std::max<int64_t>(1, (nspans + C - 1) / C);
    const int64_t nstates = nck + C + 4;  // checkpoints | segment | forward work pair | adjoint pair

    // one device block: states, partial sums, tables
    const size_t b_states = 2 * arr * nstates;
    const size_t b_partial = up(sizeof(double) * std::max<int64_t>(nspans, 1) * nta);
    const size_t b_tiles = up(sizeof(TileDev) * (ntf + nta));
    const size_t b_prob = up(sizeof(ProblemDev<Real>) * 2 * np);
    const size_t b_probes = up(sizeof(ProbeDev<Real>) * (np + 1));  // adjoint probes | forward receiver
    const size_t b_red = up(sizeof(int64_t) * 2 * np + sizeof(double) * np);
    const size_t b_done = up(sizeof(int) * std::max<int64_t>(ntf, nta));
    const size_t b_rtmp = up(sizeof(double) * (size_t)adj_reduce_blocks(std::max<int64_t>(nspans, 1), np) * np);
    const size_t need = b_states + b_partial + b_tiles + b_prob + b_probes + b_red + b_done + b_rtmp;
    // the span states of an earlier sweep with the same inputs and layout are
    // still in the workspace: the forward sweep can be skipped
    const Engine::KeptKey key{fA, fB, T, SA, vf, va, core_f, core_a, C, use_ws, arr, need};
    const bool reuse = !keep && e->kept && e->kept_key == key && need <= e->adj_mem_cap;
    if (!reuse) e->kept = false;
    if (need > e->adj_mem_cap) {
        RSWR_CUDA(cudaStreamSynchronize(s));
        cudaFree(e->adj_mem);
        e->adj_mem = nullptr;
        e->adj_mem_cap = 0;
        if (cudaMalloc(&e->adj_mem, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(RSWR_ENOMEM, "adjoint workspace (" + std::to_string(need) + " bytes)");
        }
        e->adj_mem_cap = need;
    }
    char* mem = static_cast<char*>(e->adj_mem);
    auto state0 = [&](int64_t i) { return reinterpret_cast<Real*>(mem + (2 * i) * arr); };
    auto state1 = [&](int64_t i) { return reinterpret_cast<Real*>(mem + (2 * i + 1) * arr); };
    char* q = mem + b_states;
    double* partial = reinterpret_cast<double*>(q);
    q += b_partial;
    TileDev* d_tiles_f = reinterpret_cast<TileDev*>(q);
    TileDev* d_tiles_a = d_tiles_f + ntf;
    q += b_tiles;
    ProblemDev<Real>* d_pu = reinterpret_cast<ProblemDev<Real>*>(q);
    ProblemDev<Real>* d_pl = d_pu + np;
    q += b_prob;
    ProbeDev<Real>* d_probes = reinterpret_cast<ProbeDev<Real>*>(q);
    q += b_probes;
    int64_t* d_t0 = reinterpret_cast<int64_t*>(q);
    int64_t* d_tc = d_t0 + np;
    double* d_scale = reinterpret_cast<double*>(d_tc + np);
    q += b_red;
    int* d_done = reinterpret_cast<int*>(q);
    q += b_done;
    double* d_rtmp = reinterpret_cast<double*>(q);
    const int64_t CK0 = 0, SG0 = nck, WK0 = nck + C, LM0 = nck + C + 2;

    // host tables
    std::vector<TileDev> ht;
    ht.reserve(ntf + nta);
    for (int p = 0; p < np; ++p)
        for (int64_t t = 0; t < tcf[p]; ++t) ht.push_back(TileDev{p, (int32_t)t, 0, 0, 0, 0});
    std::vector<ProbeDev<Real>> hp;
    std::vector<ProblemDev<Real>> hpr(2 * np);
    std::vector<double> hscale(np);
    for (int p = 0; p < np; ++p) {
        const ProbHost& ph = e->probs[p];
        const bool interior = j_r[p] > 0 && j_r[p] < ph.nx - 1;
        for (int64_t t = 0; t < tca[p]; ++t) {
            TileDev td{p, (int32_t)t, (int32_t)hp.size(), (int32_t)hp.size(), 0, 0};
            if (t == 0 && interior) td.probe_end += 1;  // grid point 1 lies in the first core
            ht.push_back(td);
            if (t == 0 && interior) {
                ProbeDev<Real> pr{};
                pr.gidx = base[p] + 1;
                pr.out = static_cast<Real*>(grad) + (int64_t)p * (T + 1) + T;
                pr.stride = -1;
                pr.nmax = T;
                pr.scale = sizeof(Real) == 8 ? (Real)ph.c2 : (Real)ph.c2f;
                pr.kind = 0;
                hp.push_back(pr);
            }
        }
        const Real c2 = sizeof(Real) == 8 ? (Real)ph.c2 : (Real)ph.c2f;
        const Real k = sizeof(Real) == 8 ? (Real)ph.k : (Real)ph.kf;
        ProblemDev<Real>& u = hpr[p];
        u = ProblemDev<Real>{};
        u.base = base[p];
        u.nx = ph.nx;
        u.tile0 = t0f[p];
        u.ntiles = tcf[p];
        u.fA = fA ? static_cast<const Real*>(fA) + (int64_t)p * (T + 1) : nullptr;
        u.fB = fB ? static_cast<const Real*>(fB) + (int64_t)p * (T + 1) : nullptr;
        u.js = -1;
        u.c2 = c2;
        u.k = k;
        ProblemDev<Real>& l = hpr[np + p];
        l = u;
        l.tile0 = t0a[p];
        l.ntiles = tca[p];
        l.fA = nullptr;
        l.fB = nullptr;
        l.js = interior ? j_r[p] : -1;
        l.src = wbar ? static_cast<const Real*>(wbar) + (int64_t)p * (T + 1) + T + 1 : nullptr;
        l.src_stride = -1;
        hscale[p] = 2.0 * ph.c2 / ph.a;
    }
    // the forward tiles carry no probes, except the receiver of a kept forward run
    int fwd_probe = -1;
    if (keep && keep->recv && np == 1) {
        fwd_probe = (int)hp.size();
        ProbeDev<Real> pr{};
        pr.gidx = base[0] + keep->j_rec;
        pr.out = static_cast<Real*>(keep->recv);
        pr.stride = 1;
        pr.nmax = T;
        pr.scale = (Real)1;
        pr.kind = 0;
        hp.push_back(pr);
        TileDev& td = ht[t0f[0] + keep->j_rec / core_f];
        td.probe_begin = fwd_probe;
        td.probe_end = fwd_probe + 1;
    }
    RSWR_CUDA(cudaMemcpyAsync(d_tiles_f, ht.data(), sizeof(TileDev) * ht.size(), cudaMemcpyHostToDevice, s));
    RSWR_CUDA(cudaMemcpyAsync(d_pu, hpr.data(), sizeof(ProblemDev<Real>) * hpr.size(), cudaMemcpyHostToDevice, s));
    if (!hp.empty())
        RSWR_CUDA(cudaMemcpyAsync(d_probes, hp.data(), sizeof(ProbeDev<Real>) * hp.size(), cudaMemcpyHostToDevice, s));
    std::vector<int64_t> hred(2 * np);
    for (int p = 0; p < np; ++p) {
        hred[p] = t0a[p];
        hred[np + p] = tca[p];
    }
    RSWR_CUDA(cudaMemcpyAsync(d_t0, hred.data(), sizeof(int64_t) * 2 * np, cudaMemcpyHostToDevice, s));
    RSWR_CUDA(cudaMemcpyAsync(d_scale, hscale.data(), sizeof(double) * np, cudaMemcpyHostToDevice, s));
    RSWR_CUDA(cudaMemsetAsync(e->d_err, 0, sizeof(DevError), s));

    if (!keep) {
        // dL/dfA: zero, or wbar itself for a receiver on the left Dirichlet node
        RSWR_CUDA(cudaMemsetAsync(grad, 0, es * (T + 1) * np, s));
        for (int p = 0; p < np; ++p)
            if (j_r[p] == 0)
                RSWR_CUDA(cudaMemcpyAsync(static_cast<char*>(grad) + es * (T + 1) * p,
                                          static_cast<const char*>(wbar) + es * (T + 1) * p, es * (T + 1),
                                          cudaMemcpyDeviceToDevice, s));
        RSWR_CUDA(cudaMemsetAsync(partial, 0, b_partial, s));
    }

    int bps_f = 0, bps_a = 0;
    RSWR_CUDA(span_occupancy(vf, &bps_f));
    RSWR_CUDA(adj_occupancy(va, &bps_a));
    const int grid_f = (int)std::min<int64_t>((int64_t)std::max(bps_f, 1) * e->num_sms, ntf);
    const int grid_a = (int)std::min<int64_t>((int64_t)std::max(bps_a, 1) * e->num_sms, nta);

    SpanParams<Real> fp{};
    fp.problems = d_pu;
    fp.tiles = d_tiles_f;
    fp.probes = fwd_probe >= 0 ? d_probes : nullptr;
    fp.ntiles = ntf;
    fp.T = T;
    fp.H = H;
    fp.core = core_f;
    fp.S = SA;
    fp.nspans = (int32_t)nspans;
    fp.inject_tile = -1;
    fp.inject_span = -1;
    fp.err = e->d_err;
    fp.wait_ns = (long long)(e->wait_s * 1e9);
    auto forward_span = [&](int64_t k, Real* s0, Real* s1, Real* d0, Real* d1) -> rswr_status {
        fp.span = (int32_t)k;
        fp.q0[k & 1] = s0;
        fp.q1[k & 1] = s1;
        fp.q0[(k + 1) & 1] = d0;
        fp.q1[(k + 1) & 1] = d1;
        RSWR_CUDA(span_launch(vf, &fp, grid_f, s));
        return RSWR_OK;
    };

    // forward sweep with checkpoints (skipped when an earlier sweep's states are kept)
    const int64_t last_ck_span = (nck - 1) * C;
    if (!reuse) {
    RSWR_CUDA(cudaMemsetAsync(state0(CK0), 0, 2 * arr, s));
    RSWR_CUDA(set_boundary_launch(e->dtype, e->form, state0(CK0), state1(CK0), d_pu, np, s));
    if (res_sweep && (keep ? nspans : last_ck_span) > 0) {
        // resident tiles: one cooperative launch over every span of the sweep
        // (a kept forward run: all of them, the final state into state nspans)
        SpanParams<Real> cp = fp;
        cp.span = -1;
        cp.nspans = (int32_t)(keep ? nspans : last_ck_span);
        cp.ck_stride = (int64_t)(2 * arr / es);
        cp.q0[0] = state0(CK0);
        cp.q1[0] = state1(CK0);
        cp.q0[1] = cp.q1[1] = nullptr;
        cp.done = d_done;
        const size_t xb = es * 8 * (size_t)H * (size_t)ntf;
        if (xb > e->xbuf_cap) {
            RSWR_CUDA(cudaStreamSynchronize(s));
            cudaFree(e->d_xbuf);
            e->d_xbuf = nullptr;
            e->xbuf_cap = 0;
            if (cudaMalloc(&e->d_xbuf, xb) != cudaSuccess) {
                cudaGetLastError();
                return fail(RSWR_ENOMEM, "halo exchange slots");
            }
            e->xbuf_cap = xb;
        }
        cp.xbuf = static_cast<Real*>(e->d_xbuf);
        RSWR_CUDA(cudaMemsetAsync(d_done, 0, sizeof(int) * ntf, s));
        RSWR_CUDA(span_launch(vf, &cp, (int)ntf, s));
    } else if (C == 1 && last_ck_span > 0) {
        // every span state is kept: the whole sweep is one persistent launch in
        // which span k reads state k and writes state k + 1 (neighbour flags as in
        // rswr_run; the states are distinct arrays, so only read-after-write waits)
        SpanParams<Real> cp = fp;
        cp.span = -1;
        cp.nspans = (int32_t)last_ck_span;
        cp.ck_stride = (int64_t)(2 * arr / es);
        cp.q0[0] = state0(CK0);
        cp.q1[0] = state1(CK0);
        cp.q0[1] = cp.q1[1] = nullptr;
        cp.ticket = static_cast<unsigned long long*>(e->d_ticket);
        cp.done = d_done;
        RSWR_CUDA(cudaMemsetAsync(e->d_ticket, 0, sizeof(unsigned long long), s));
        RSWR_CUDA(cudaMemsetAsync(d_done, 0, sizeof(int) * ntf, s));
        const int grid = (int)std::min<int64_t>((int64_t)std::max(bps_f, 1) * e->num_sms, last_ck_span * ntf);
        RSWR_CUDA(span_launch(vf, &cp, grid, s));
    } else {
        for (int64_t k = 0; k < last_ck_span; ++k) {
            const int64_t si = (k % C == 0) ? CK0 + k / C : WK0 + (k & 1);
            const int64_t di = ((k + 1) % C == 0) ? CK0 + (k + 1) / C : WK0 + ((k + 1) & 1);
            rswr_status st = forward_span(k, state0(si), state1(si), state0(di), state1(di));
            if (st != RSWR_OK) return st;
        }
    }
    }
    // only a kept forward run (rswr_run_keep) leaves states for a later call: an
    // ordinary adjoint call must not, since its caller may change fA in place
    if (keep) {
        e->kept = true;
        e->kept_key = key;
    }

    if (keep) {
        // a kept forward run: the last span into the work pair, the receiver's
        // last level, the final state pair
        Real* f0 = state0(CK0);
        Real* f1 = state1(CK0);
        if (res_sweep && nspans > 0) {
            // the resident sweep ran every span: the final state is state nspans
            // (the segment slot, unused when every span state is kept)
            f0 = state0(CK0 + nspans);
            f1 = state1(CK0 + nspans);
        } else if (nspans > 0) {
            const int64_t k = nspans - 1;  // C == 1: state k is checkpoint k
            rswr_status st = forward_span(k, state0(CK0 + k), state1(CK0 + k), state0(WK0), state1(WK0));
            if (st != RSWR_OK) return st;
            f0 = state0(WK0);
            f1 = state1(WK0);
        }
        if (fwd_probe >= 0) RSWR_CUDA(probe_final_launch(e->dtype, d_probes + fwd_probe, 1, f0, T, s));
        const int64_t nx = e->probs[0].nx;
        RSWR_CUDA(cudaMemcpyAsync(keep->out0, f0 + base[0], es * nx, cudaMemcpyDeviceToDevice, s));
        RSWR_CUDA(cudaMemcpyAsync(keep->out1, f1 + base[0], es * nx, cudaMemcpyDeviceToDevice, s));
        return RSWR_OK;
    }

    // adjoint sweep
    RSWR_CUDA(cudaMemsetAsync(state0(LM0), 0, 4 * arr, s));  // both adjoint pairs
    RSWR_CUDA(adj_init_launch(e->dtype, e->form, state0(LM0), state1(LM0), d_pl, np, wbar, T, s));
    AdjParams<Real> ap{};
    ap.prob_u = d_pu;
    ap.prob_l = d_pl;
    ap.tiles = d_tiles_a;
    ap.probes = d_probes;
    ap.ntiles = nta;
    ap.H = H;
    ap.core = core_a;
    ap.err = e->d_err;
    ap.wait_ns = (long long)(e->wait_s * 1e9);
    ap.T = T;
    int cur = 0;
    if (use_ws) {
        // all spans, last first, in one launch; the forward state at the start of
        // span K is checkpoint K (C == 1)
        AdjParams<Real> wp = ap;
        wp.partial = partial;
        wp.uck0 = state0(CK0);
        wp.uck1 = state1(CK0);
        wp.ck_stride = (int64_t)(2 * arr / es);
        wp.lq0[0] = state0(LM0);
        wp.lq1[0] = state1(LM0);
        wp.lq0[1] = state0(LM0 + 1);
        wp.lq1[1] = state1(LM0 + 1);
        wp.T = T;
        wp.SA = SA;
        wp.nspans = (int32_t)nspans;
        wp.ticket = static_cast<unsigned long long*>(e->d_ticket);
        wp.done = d_done;
        int bps_w = 0;
        RSWR_CUDA(adj_ws_occupancy(e->dtype, e->form, &bps_w));
        if (bps_w < 1) return fail(RSWR_ENOTSUP, "adjoint kernel does not fit on an SM");
        RSWR_CUDA(cudaMemsetAsync(e->d_ticket, 0, sizeof(unsigned long long), s));
        RSWR_CUDA(cudaMemsetAsync(d_done, 0, sizeof(int) * nta, s));
        const int grid = (int)std::min<int64_t>((int64_t)bps_w * e->num_sms, nspans * nta);
        if (nspans > 0) RSWR_CUDA(adj_ws_launch(e->dtype, e->form, &wp, grid, s));
    }
    for (int64_t g = use_ws ? -1 : nck - 1; g >= 0; --g) {
        const int64_t k_lo = g * C, k_hi = std::min<int64_t>((g + 1) * C, nspans);
        auto seg = [&](int64_t i) { return i == 0 ? CK0 + g : SG0 + i; };
        for (int64_t k = k_lo; k + 1 < k_hi; ++k) {
            const int64_t si = seg(k - k_lo), di = seg(k - k_lo + 1);
            rswr_status st = forward_span(k, state0(si), state1(si), state0(di), state1(di));
            if (st != RSWR_OK) return st;
        }
        for (int64_t K = k_hi - 1; K >= k_lo; --K) {
            const int64_t ui = seg(K - k_lo);
            ap.u0 = state0(ui);
            ap.u1 = state1(ui);
            ap.l0 = state0(LM0 + cur);
            ap.l1 = state1(LM0 + cur);
            ap.l0_out = state0(LM0 + (cur ^ 1));
            ap.l1_out = state1(LM0 + (cur ^ 1));
            ap.n0 = K * SA;
            ap.len = (int32_t)std::min<int64_t>(SA, T - K * SA);
            ap.m0 = T - (ap.n0 + ap.len - 1);
            ap.partial = partial + K * nta;
            RSWR_CUDA(adj_launch(va, &ap, grid_a, s));
            cur ^= 1;
        }
    }
    if (grad_a) {
        if (nspans > 0)
            RSWR_CUDA(adj_reduce_launch(partial, nspans, nta, d_t0, d_tc, d_scale, grad_a, np, d_rtmp, s));
        else
            RSWR_CUDA(cudaMemsetAsync(grad_a, 0, sizeof(double) * np, s));
    }
    return RSWR_OK;
}

rswr_status adjoint_dispatch(Engine* e, int64_t T, const int64_t* j_r, const void* fA, const void* fB,
                             const void* wbar, void* grad, double* grad_a, cudaStream_t s)
{
    for (int v = 0; v < adj_variant_count(); ++v) {
        cudaError_t ce = adj_prepare(v);
        if (ce != cudaSuccess) return fail(RSWR_ECUDA, std::string("adjoint attributes: ") + cudaGetErrorString(ce));
    }
    return e->dtype == kF64 ? adjoint_full<double>(e, T, j_r, fA, fB, wbar, grad, grad_a, s)
                            : adjoint_full<float>(e, T, j_r, fA, fB, wbar, grad, grad_a, s);
}

}  // namespace

namespace {

// ---- autotuner -----------------------------------------------------------
// Times every kernel variant of the engine's dtype/form, both scheduling modes
// and spans S and S/2 on `probe_steps` steps of a zero-data run of the
// engine's own problems, keeps the fastest, and remembers it per
// (dtype, form, log2 points, problems, S) in a process-wide table that can be
// persisted to the file named by RSWR_AUTOTUNE_CACHE.

struct TuneChoice {
    int variant, mode, S;
};

std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune;
bool g_tune_loaded = false;

std::string tune_key(const Engine* e, int S_max)
{
    int64_t n = e->packed_len;
    int lg = 0;
    while ((int64_t(1) << (lg + 1)) <= n) ++lg;
    return std::to_string(e->dtype) + ":" + std::to_string(e->form) + ":" + std::to_string(lg) + ":" +
           std::to_string(e->probs.size() > 1 ? 1 : 0) + ":" + std::to_string(S_max);
}

void tune_load()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = std::getenv("RSWR_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char key[128];
    int v, m, S;
    while (std::fscanf(f, "%127s %d %d %d", key, &v, &m, &S) == 4) g_tune[key] = TuneChoice{v, m, S};
    std::fclose(f);
}

void tune_save()
{
    const char* path = std::getenv("RSWR_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "w");
    if (!f) return;
    for (const auto& kv : g_tune) std::fprintf(f, "%s %d %d %d\n", kv.first.c_str(), kv.second.variant, kv.second.mode, kv.second.S);
    std::fclose(f);
}

rswr_status apply_choice(Engine* e, const TuneChoice& c)
{
    const int oldS = e->S, oldV = e->variant;
    e->S = c.S;
    e->variant = c.variant;
    rswr_status st = layout(e);
    if (st != RSWR_OK) {
        e->S = oldS;
        e->variant = oldV;
        layout(e);
        return st;
    }
    e->mode = c.mode;
    return RSWR_OK;
}

int span_limit(const Engine* e)
{
    int S = 1 << 30;
    for (const ProbHost& p : e->probs) S = std::min(S, p.ov / 2);
    return std::min(S, kSpanCap);
}

rswr_status autotune_engine(Engine* e, int64_t probe_steps, int32_t* variant, cudaStream_t s, bool use_cache)
{
    if (probe_steps < 1) return fail(RSWR_EINVAL, "probe_steps must be >= 1");
    const int S_max = span_limit(e);
    const std::string key = tune_key(e, S_max);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_load();
        auto it = g_tune.find(key);
        if (use_cache && it != g_tune.end()) {
            rswr_status st = apply_choice(e, it->second);
            if (st == RSWR_OK) {
                if (variant) *variant = e->variant;
                return RSWR_OK;
            }
        }
    }
    const size_t es = e->esize();
    if (e->scratch_cap < (size_t)e->packed_len) {
        for (int b = 0; b < 2; ++b) {
            cudaFree(e->d_scratch[b]);
            e->d_scratch[b] = nullptr;
            if (cudaMalloc(&e->d_scratch[b], es * e->packed_len) != cudaSuccess) return fail(RSWR_ENOMEM, "scratch");
        }
        e->scratch_cap = e->packed_len;
    }
    cudaEvent_t a, b;
    RSWR_CUDA(cudaEventCreate(&a));
    RSWR_CUDA(cudaEventCreate(&b));
    const cudaEvent_t keep0 = e->ev_start, keep1 = e->ev_stop;
    e->ev_start = e->ev_stop = nullptr;
    const TuneChoice keep{e->variant, e->mode, e->S};
    TuneChoice best = keep;
    float best_ms = 1e30f;
    RunReq r;
    r.T = probe_steps;
    r.out0 = e->d_scratch[0];
    r.out1 = e->d_scratch[1];
    std::vector<int> spans{S_max};
    if (S_max / 2 >= 4) spans.push_back(S_max / 2);
    for (int v = 0; v < span_variant_count(); ++v) {
        const VariantInfo vi = span_variant_info(v);
        if (vi.dtype != e->dtype || vi.form != e->form) continue;
        for (int S : spans) {
            for (int mode = 0; mode < (vi.resident ? 1 : 2); ++mode) {
                if (apply_choice(e, TuneChoice{v, mode, S}) != RSWR_OK) continue;
                if (run_engine(e, r, s) != RSWR_OK) continue;  // warm-up (and graph capture)
                RSWR_CUDA(cudaEventRecord(a, s));
                rswr_status st = run_engine(e, r, s);
                RSWR_CUDA(cudaEventRecord(b, s));
                RSWR_CUDA(cudaEventSynchronize(b));
                float ms = 0.f;
                RSWR_CUDA(cudaEventElapsedTime(&ms, a, b));
                if (st == RSWR_OK && ms < best_ms) {
                    best_ms = ms;
                    best = TuneChoice{v, mode, S};
                }
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    e->ev_start = keep0;
    e->ev_stop = keep1;
    rswr_status st = apply_choice(e, best);
    if (st != RSWR_OK) return st;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[key] = best;
        tune_save();
    }
    if (variant) *variant = e->variant;
    return RSWR_OK;
}

}  // namespace

namespace {

// ---- the paper-literal span loop (see paper_kernel.cu) --------------------
// Per span: predict + select on every interface (rswr_iface_kernel, the span
// read back to the host), then the update.  The update re-solves every
// subdomain window over the span with the neighbours' predicted output fluxes
// as Neumann data (Sec. 2.5).  A point farther than the span from both input
// boundaries of its window depends only on the true state, through the same
// operations as the monolithic leapfrog, so there the re-solve gives the
// monolithic bits: the whole grid is advanced by the span kernel (the plan's
// fast path, from the state it keeps), and only the kept points within the
// span of an input boundary ("zones") are re-solved with the paper's rule
// (rswr_resolve_kernel, from the span-start state into scratch, scattered into
// the result).  Same bits as re-solving every window.
template <typename Real>
rswr_status run_paper(Engine* e, const Real* fA, const Real* fB, int64_t T, const Real* q0, const Real* q1, Real* out0,
                      Real* out1, int64_t* spans, int64_t spans_cap, int64_t* nspans, double beta, cudaStream_t s)
{
    const ProbHost& ph = e->probs[0];
    const int64_t nx = ph.nx, N = ph.n_sub, ov = ph.ov, el = (ov + 1) / 2, er = ov / 2;
    const size_t es = sizeof(Real);
    e->kept = false;  // the workspace below overwrites kept span states
    int64_t cap = (int64_t)std::ceil((double)(ov - 1) / (2.0 * ph.c)) - 1;
    if (cap < 1) cap = 1;
    int64_t tau = ov;
    // beta in thousandths: ceil((1 + beta) span) in exact integer arithmetic
    const int64_t beta_m = (int64_t)std::llround(beta * 1000.0);
    const int64_t tau_max = (std::max(tau, cap) * (1000 + beta_m) + 999) / 1000 + 1;
    auto wl = [&](int64_t i) { return std::max<int64_t>(i * nx / N - el, 0); };
    auto wr = [&](int64_t i) { return std::min<int64_t>((i + 1) * nx / N - 1 + er, nx - 1); };
    // zone tiles: the kept points of subdomain i (from its left neighbour's
    // window end on) within tau_max >= any span of an input boundary, in chunks
    constexpr int64_t CH = 1024;
    std::vector<int64_t> tsub, tlo, thi;
    for (int64_t i = 0; i < N; ++i) {
        const int64_t L = wl(i), R = wr(i);
        const int64_t from = (i == 0) ? L : wr(i - 1) + 1;
        std::vector<std::pair<int64_t, int64_t>> z;  // [lo, hi)
        if (i > 0 && L > 0 && L + tau_max - 1 >= from) z.push_back({from, std::min(R, L + tau_max - 1) + 1});
        if (i + 1 < N && R < nx - 1) z.push_back({std::max(from, R - tau_max + 1), R + 1});
        if (z.size() == 2 && z[1].first <= z[0].second) z = {{z[0].first, z[1].second}};
        for (auto& r : z)
            for (int64_t c = r.first; c < r.second; c += CH) {
                tsub.push_back(i);
                tlo.push_back(c);
                thi.push_back(std::min(c + CH, r.second));
            }
    }
    const int64_t nt = (int64_t)tsub.size();
    // workspace: the zones' scratch pair, flux waveforms, tiles, span word
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t b_state = up(es * nx);
    const size_t b_g = up(es * N * tau_max);
    const size_t b_t = up(sizeof(int64_t) * std::max<int64_t>(nt, 1));
    // the span kernel runs nsub spans of S steps per paper span (the last ones
    // may take fewer or none: the span is chosen on the device), reading the
    // span's boundary samples from a copy of nsamp levels
    const int64_t nsub = (cap + e->S - 1) / e->S;
    const int nsamp = (int)(nsub * e->S + 1);
    const size_t b_samp = up(es * (size_t)nsamp);
    const int64_t rec_cap = spans ? std::min<int64_t>(spans_cap, std::max<int64_t>(T, 1)) : 0;
    const size_t b_rec = up(sizeof(int64_t) * (size_t)std::max<int64_t>(rec_cap, 1));
    const size_t need = 2 * b_state + 2 * b_g + 3 * b_t + 256 + 2 * b_samp + b_rec + up(sizeof(PaperState));
    if (need > e->adj_mem_cap) {
        RSWR_CUDA(cudaStreamSynchronize(s));
        cudaFree(e->adj_mem);
        e->adj_mem = nullptr;
        e->adj_mem_cap = 0;
        if (cudaMalloc(&e->adj_mem, need) != cudaSuccess) return fail(RSWR_ENOMEM, "paper-literal workspace");
        e->adj_mem_cap = need;
    }
    char* m = static_cast<char*>(e->adj_mem);
    Real* Y0 = reinterpret_cast<Real*>(m);
    Real* Y1 = reinterpret_cast<Real*>(m + b_state);
    Real* gL = reinterpret_cast<Real*>(m + 2 * b_state);
    Real* gR = reinterpret_cast<Real*>(m + 2 * b_state + b_g);
    int64_t* d_sub = reinterpret_cast<int64_t*>(m + 2 * b_state + 2 * b_g);
    int64_t* d_lo = reinterpret_cast<int64_t*>(m + 2 * b_state + 2 * b_g + b_t);
    int64_t* d_hi = reinterpret_cast<int64_t*>(m + 2 * b_state + 2 * b_g + 2 * b_t);
    int* d_span = reinterpret_cast<int*>(m + 2 * b_state + 2 * b_g + 3 * b_t);
    char* m2 = m + 2 * b_state + 2 * b_g + 3 * b_t + 256;
    Real* d_fAs = reinterpret_cast<Real*>(m2);
    Real* d_fBs = reinterpret_cast<Real*>(m2 + b_samp);
    int64_t* d_rec = reinterpret_cast<int64_t*>(m2 + 2 * b_samp);
    PaperState* d_st = reinterpret_cast<PaperState*>(m2 + 2 * b_samp + b_rec);
    if (nt > 0) {
        RSWR_CUDA(cudaMemcpyAsync(d_sub, tsub.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice, s));
        RSWR_CUDA(cudaMemcpyAsync(d_lo, tlo.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice, s));
        RSWR_CUDA(cudaMemcpyAsync(d_hi, thi.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice, s));
    }

    // level 0 (paper Sec. 2.1, or the given state) in the plan's own state
    // arrays; the runs below continue from there (no graph capture: the span
    // kernel's arguments change every span)
    const bool keep_graph = e->use_graph;
    e->use_graph = false;
    struct Restore {
        Engine* e;
        bool g;
        ~Restore() { e->use_graph = g; }
    } restore{e, keep_graph};
    {
        RunReq r;
        r.fA = fA;
        r.fB = fB;
        r.T = 0;
        r.q0 = q0;
        r.q1 = q1;
        rswr_status st = run_impl<Real>(e, r, s);
        if (st != RSWR_OK) return st;
    }

    PaperParams<Real> pp{};
    pp.fA = fA;
    pp.fB = fB;
    pp.gL = gL;
    pp.gR = gR;
    pp.span_min = d_span;
    pp.tile_sub = d_sub;
    pp.tile_lo = d_lo;
    pp.tile_hi = d_hi;
    pp.nx = nx;
    pp.N = N;
    pp.el = el;
    pp.er = er;
    pp.tau_stride = tau_max;
    pp.form = e->form;
    pp.c2 = sizeof(Real) == 8 ? (Real)ph.c2 : (Real)ph.c2f;
    pp.k = sizeof(Real) == 8 ? (Real)ph.k : (Real)ph.kf;
    const double dx = (ph.xb - ph.xa) / (double)(nx - 1);
    pp.two_dx = (Real)(2.0 * dx);
    if (!e->h_pstate && cudaMallocHost(&e->h_pstate, sizeof(PaperState)) != cudaSuccess) {
        cudaGetLastError();
        e->h_pstate = nullptr;
        return fail(RSWR_ENOMEM, "pinned host state");
    }
    // the run's progress on the device: the span is chosen there, so the host
    // queues spans without reading each one back
    {
        PaperState h0{};
        h0.n0 = 0;
        h0.tau = (int32_t)tau;
        h0.steps = (int32_t)std::min<int64_t>(tau, T);
        h0.done = T <= 0 ? 1 : 0;
        *e->h_pstate = h0;
        RSWR_CUDA(cudaMemcpyAsync(d_st, e->h_pstate, sizeof(PaperState), cudaMemcpyHostToDevice, s));
    }
    pp.st = d_st;
    pp.steps = (int32_t)tau_max;  // (sizes only: the kernels take steps and span from d_st)
    const size_t smem_i = es * (8 * (size_t)(ov + tau_max + 2)) + sizeof(int) * (size_t)(ov + 2);
    const size_t smem_r = es * 4 * (size_t)(CH + 2 * cap + 2);
    int64_t n0 = 0, m_count = 0;
    while (n0 < T) {
        // as many spans as the run needs at least (each advances at most cap
        // levels), so the batch never runs past T; then one read-back
        const int64_t batch = std::max<int64_t>(1, (T - n0 + cap - 1) / cap);
        for (int64_t b = 0; b < batch; ++b) {
            // the state at level n0 (nsub spans of the span kernel per paper
            // span: after an odd number the state is in buffer 1, swapped below)
            pp.u = static_cast<Real*>(e->q0[0]) + ph.base;
            pp.w = static_cast<Real*>(e->q1[0]) + ph.base;
            // predict + select (Sec. 2.3, 2.4, Sec. 3): every pair lowers the span
            // word (bytes 0x7f: a value above any span) with atomicMin
            RSWR_CUDA(cudaMemsetAsync(d_span, 0x7f, sizeof(int), s));
            RSWR_CUDA(paper_iface_launch(e->dtype, &pp, (int)(N - 1), smem_i, s));
            RSWR_CUDA(paper_select_launch(e->dtype, d_st, d_span, (int)cap, fA, fB, d_fAs, d_fBs, nsamp, T,
                                          rec_cap > 0 ? d_rec : nullptr, rec_cap, s));
            // update (Sec. 2.5): the zones next to input boundaries from the span-start state
            pp.uo = Y0;
            pp.wo = Y1;
            if (nt > 0) RSWR_CUDA(paper_resolve_launch(e->dtype, &pp, (int)nt, smem_r, s));
            // ... and every other point through the span kernel
            RunReq r;
            r.fA = fA ? d_fAs : nullptr;
            r.fB = fB ? d_fBs : nullptr;
            r.T = nsub * e->S;
            r.steps_dev = &d_st->span;
            r.from_state = true;
            rswr_status st = run_impl<Real>(e, r, s);
            if (st != RSWR_OK) return st;
            if (nsub & 1) {  // the result is in buffer 1: make it the current state
                std::swap(e->q0[0], e->q0[1]);
                std::swap(e->q1[0], e->q1[1]);
            }
            RSWR_CUDA(paper_scatter_launch(e->dtype, Y0, Y1, static_cast<Real*>(e->q0[0]) + ph.base,
                                           static_cast<Real*>(e->q1[0]) + ph.base, d_lo, d_hi, (int)nt, d_st, s));
            RSWR_CUDA(paper_advance_launch(d_st, T, beta_m, tau_max, s));
        }
        RSWR_CUDA(cudaMemcpyAsync(e->h_pstate, d_st, sizeof(PaperState), cudaMemcpyDeviceToHost, s));
        RSWR_CUDA(cudaStreamSynchronize(s));
        const int64_t before = n0;
        n0 = e->h_pstate->n0;
        m_count = e->h_pstate->count;
        if (n0 <= before) {
            rswr_status st = check_engine(e, s, nullptr, nullptr, nullptr);
            if (st != RSWR_OK) return st;
            return fail(RSWR_ECUDA, "paper-literal run made no progress");
        }
    }
    if (spans && m_count > 0)
        RSWR_CUDA(cudaMemcpyAsync(spans, d_rec, sizeof(int64_t) * (size_t)std::min<int64_t>(m_count, rec_cap),
                                  cudaMemcpyDeviceToHost, s));
    if (nspans) *nspans = m_count;
    RSWR_CUDA(cudaMemcpyAsync(out0, static_cast<Real*>(e->q0[0]) + ph.base, es * nx, cudaMemcpyDeviceToDevice, s));
    RSWR_CUDA(cudaMemcpyAsync(out1, static_cast<Real*>(e->q1[0]) + ph.base, es * nx, cudaMemcpyDeviceToDevice, s));
    return check_engine(e, s, nullptr, nullptr, nullptr);
}

}  // namespace

void rswr::set_error_message(const char* m) { g_msg = m; }

// ===========================================================================
// C ABI
// ===========================================================================

struct rswr_plan_s {
    Engine* e;
};
struct rswr_batch_s {
    Engine* e;
};

extern "C" {

const char* rswr_status_string(rswr_status s)
{
    switch (s) {
        case RSWR_OK: return "RSWR_OK";
        case RSWR_EINVAL: return "RSWR_EINVAL";
        case RSWR_ECFL: return "RSWR_ECFL";
        case RSWR_EOVERLAP: return "RSWR_EOVERLAP";
        case RSWR_ENOMEM: return "RSWR_ENOMEM";
        case RSWR_ECUDA: return "RSWR_ECUDA";
        case RSWR_ETIMEOUT: return "RSWR_ETIMEOUT";
        case RSWR_ENOTSUP: return "RSWR_ENOTSUP";
    }
    return "unknown status";
}

const char* rswr_last_error_message(void) { return g_msg.c_str(); }

int32_t rswr_version(void) { return 100; }

rswr_status rswr_plan_create(rswr_plan_t* plan, double xa, double xb, double a, int64_t nx, double dt, int32_t n_sub,
                             int32_t overlap, int32_t dtype, int32_t form, uint32_t flags)
{
    if (!plan) return fail(RSWR_EINVAL, "plan is NULL");
    *plan = nullptr;
    (void)flags;
    rswr_problem q{nx, xa, xb, a, dt, n_sub, overlap};
    Engine* e = nullptr;
    rswr_status st = make_engine(&e, 1, &q, dtype, form, true);
    if (st != RSWR_OK) return st;
    *plan = new (std::nothrow) rswr_plan_s{e};
    if (!*plan) {
        free_engine(e);
        return fail(RSWR_ENOMEM, "host allocation");
    }
    return RSWR_OK;
}

rswr_status rswr_plan_create_part(rswr_plan_t* plan, double xa, double xb, double a, int64_t nx, double dt,
                                  int64_t lo, int64_t hi, int32_t n_sub, int32_t overlap, int32_t dtype, int32_t form,
                                  uint32_t flags)
{
    if (!plan) return fail(RSWR_EINVAL, "plan is NULL");
    *plan = nullptr;
    (void)flags;
    if (lo < 0 || hi > nx || hi - lo < 3) return fail(RSWR_EINVAL, "need 0 <= lo, hi <= nx and hi - lo >= 3");
    // the whole grid fixes the coefficients (and the Courant-number check)
    const rswr_problem g{nx, xa, xb, a, dt, 1, 2};
    rswr_status st = validate(g);
    if (st != RSWR_OK) return st;
    ProbHost whole{};
    whole.nx = nx; whole.xa = xa; whole.xb = xb; whole.a = a; whole.dt = dt;
    coefficients(whole);
    // the part: hi - lo points of the same spacing, its own decomposition
    const double dx = (xb - xa) / (double)(nx - 1);
    const rswr_problem q{hi - lo, xa + (double)lo * dx, xa + (double)(hi - 1) * dx, a, dt, n_sub, overlap};
    Engine* e = nullptr;
    st = make_engine(&e, 1, &q, dtype, form, true);
    if (st != RSWR_OK) return st;
    ProbHost& ph = e->probs[0];
    ph.c = whole.c; ph.c2 = whole.c2; ph.k = whole.k; ph.inv2dx = whole.inv2dx;
    ph.c2f = whole.c2f; ph.kf = whole.kf; ph.inv2dxf = whole.inv2dxf;
    e->part = true;
    *plan = new (std::nothrow) rswr_plan_s{e};
    if (!*plan) {
        free_engine(e);
        return fail(RSWR_ENOMEM, "host allocation");
    }
    return RSWR_OK;
}

void rswr_plan_destroy(rswr_plan_t plan)
{
    if (!plan) return;
    free_engine(plan->e);
    delete plan;
}

rswr_status rswr_plan_get_info(rswr_plan_t plan, rswr_plan_info* info)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    return fill_info(plan->e, info);
}

rswr_status rswr_plan_set_span(rswr_plan_t plan, int32_t S)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    Engine* e = plan->e;
    if (S < 1 || S > e->probs[0].ov / 2 || S > kSpanCap)
        return fail(RSWR_EOVERLAP, "span must satisfy 1 <= S <= floor(overlap/2)");
    const int old = e->S, oldv = e->variant;
    e->S = S;
    // a variant whose warp halo is shorter than S gives way to the default one for S
    if (!variant_takes_span(span_variant_info(e->variant), S)) e->variant = default_variant(e->dtype, e->form, S);
    rswr_status st = e->variant >= 0 ? layout(e) : fail(RSWR_ENOTSUP, "no kernel variant runs this span");
    if (st != RSWR_OK) {
        e->S = old;
        e->variant = oldv;
        layout(e);
    }
    return st;
}

rswr_status rswr_plan_set_variant(rswr_plan_t plan, int32_t variant)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    return set_variant(plan->e, variant);
}

rswr_status rswr_plan_set_mode(rswr_plan_t plan, int32_t mode)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    if (mode != RSWR_MODE_PERSISTENT && mode != RSWR_MODE_PER_SPAN) return fail(RSWR_EINVAL, "bad mode");
    plan->e->mode = mode;
    return RSWR_OK;
}

rswr_status rswr_plan_set_wait_limit(rswr_plan_t plan, double seconds)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    if (!(seconds > 0.0) || seconds > 3600.0) return fail(RSWR_EINVAL, "wait limit out of range");
    plan->e->wait_s = seconds;
    return RSWR_OK;
}

rswr_status rswr_plan_set_checkpoint_spacing(rswr_plan_t plan, int64_t spans)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    if (spans < 0) return fail(RSWR_EINVAL, "checkpoint spacing must be >= 0");
    plan->e->ck_spacing = spans;
    return RSWR_OK;
}

rswr_status rswr_plan_set_sources(rswr_plan_t plan, int64_t nsrc, const int64_t* j, const void* samples,
                                  int64_t pitch)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    return set_sources(plan->e, nsrc, nullptr, j, samples, pitch);
}

rswr_status rswr_plan_inject_missing_flag(rswr_plan_t plan, int32_t tile, int32_t span)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    if (tile >= plan->e->ntiles) return fail(RSWR_EINVAL, "tile out of range");
    plan->e->inject_tile = tile < 0 ? -1 : tile;
    plan->e->inject_span = span;
    return RSWR_OK;
}

rswr_status rswr_plan_set_kernel_events(rswr_plan_t plan, void* start, void* stop)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    if ((start == nullptr) != (stop == nullptr)) return fail(RSWR_EINVAL, "give both events or neither");
    plan->e->ev_start = static_cast<cudaEvent_t>(start);
    plan->e->ev_stop = static_cast<cudaEvent_t>(stop);
    return RSWR_OK;
}

rswr_status rswr_plan_check(rswr_plan_t plan, void* stream, int32_t* code, int32_t* tile, int32_t* span)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    return check_engine(plan->e, static_cast<cudaStream_t>(stream), code, tile, span);
}

rswr_status rswr_run(rswr_plan_t plan, const void* fA, const void* fB, int64_t T, const void* q0, const void* q1,
                     void* out0, void* out1, void* traces, int64_t j_r, void* recv, void* stream)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    return plan_run(plan->e, fA, fB, T, q0, q1, out0, out1, traces, j_r, recv, stream, false);
}

rswr_status rswr_mono(rswr_plan_t plan, const void* fA, const void* fB, int64_t T, const void* q0, const void* q1,
                      void* out0, void* out1, void* traces, int64_t j_r, void* recv, void* stream)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    return plan_run(plan->e, fA, fB, T, q0, q1, out0, out1, traces, j_r, recv, stream, true);
}

rswr_status rswr_run_host(rswr_plan_t plan, const void* fA, const void* fB, int64_t T, const void* q0,
                          const void* q1, void* out0, void* out1, void* traces, int64_t j_r, void* recv, void* stream)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    Engine* e = plan->e;
    if (T < 0) return fail(RSWR_EINVAL, "T < 0");
    if (!out0 || !out1) return fail(RSWR_EINVAL, "out0 and out1 are required");
    const size_t es = e->esize();
    const int64_t nx = e->probs[0].nx;
    const int64_t ntr = traces ? (int64_t)(e->probs[0].n_sub - 1) * 2 * (T + 1) : 0;
    // staging layout: fA | fB | q0 | q1 | out0 | out1 | traces | recv
    const size_t need = es * (2 * (T + 1) + 4 * nx + ntr + (T + 1)) + 8 * 64;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (need > e->host_stage_cap) {
        RSWR_CUDA(cudaStreamSynchronize(s));
        cudaFree(e->d_host_stage);
        e->d_host_stage = nullptr;
        if (cudaMalloc(&e->d_host_stage, need) != cudaSuccess) return fail(RSWR_ENOMEM, "host staging");
        e->host_stage_cap = need;
    }
    char* at = static_cast<char*>(e->d_host_stage);
    auto take = [&](size_t bytes) {
        char* p = at;
        at += (bytes + 255) / 256 * 256;
        return p;
    };
    char* dfA = fA ? take(es * (T + 1)) : nullptr;
    char* dfB = fB ? take(es * (T + 1)) : nullptr;
    char* dq0 = q0 ? take(es * nx) : nullptr;
    char* dq1 = q1 ? take(es * nx) : nullptr;
    char* do0 = take(es * nx);
    char* do1 = take(es * nx);
    char* dtr = traces ? take(es * ntr) : nullptr;
    char* drc = recv ? take(es * (T + 1)) : nullptr;
    if ((size_t)(at - static_cast<char*>(e->d_host_stage)) > e->host_stage_cap) return fail(RSWR_ENOMEM, "staging");
    if (fA) RSWR_CUDA(cudaMemcpyAsync(dfA, fA, es * (T + 1), cudaMemcpyHostToDevice, s));
    if (fB) RSWR_CUDA(cudaMemcpyAsync(dfB, fB, es * (T + 1), cudaMemcpyHostToDevice, s));
    if (q0) RSWR_CUDA(cudaMemcpyAsync(dq0, q0, es * nx, cudaMemcpyHostToDevice, s));
    if (q1) RSWR_CUDA(cudaMemcpyAsync(dq1, q1, es * nx, cudaMemcpyHostToDevice, s));
    rswr_status st = plan_run(e, dfA, dfB, T, dq0, dq1, do0, do1, dtr, j_r, drc, stream, false);
    if (st != RSWR_OK) return st;
    RSWR_CUDA(cudaMemcpyAsync(out0, do0, es * nx, cudaMemcpyDeviceToHost, s));
    RSWR_CUDA(cudaMemcpyAsync(out1, do1, es * nx, cudaMemcpyDeviceToHost, s));
    if (traces) RSWR_CUDA(cudaMemcpyAsync(traces, dtr, es * ntr, cudaMemcpyDeviceToHost, s));
    if (recv) RSWR_CUDA(cudaMemcpyAsync(recv, drc, es * (T + 1), cudaMemcpyDeviceToHost, s));
    return check_engine(e, s, nullptr, nullptr, nullptr);
}

rswr_status rswr_run_keep(rswr_plan_t plan, const void* fA, const void* fB, int64_t T, int64_t j_r, void* recv,
                          void* out0, void* out1, void* stream)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    Engine* e = plan->e;
    if (T < 0 || T > ((int64_t)1 << 40)) return fail(RSWR_EINVAL, "T out of range");
    if (!out0 || !out1) return fail(RSWR_EINVAL, "out0 and out1 are required");
    if (recv && (j_r < 0 || j_r >= e->probs[0].nx)) return fail(RSWR_EINVAL, "receiver index outside the grid");
    if (!e->usrc.empty()) return fail(RSWR_ENOTSUP, "a kept run has no user point sources");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int v = 0; v < adj_variant_count(); ++v) {
        cudaError_t ce = adj_prepare(v);
        if (ce != cudaSuccess) return fail(RSWR_ECUDA, std::string("adjoint attributes: ") + cudaGetErrorString(ce));
    }
    const KeepReq k{recv ? j_r : -1, recv, out0, out1};
    const int64_t none = -1;
    rswr_status st = e->dtype == kF64 ? adjoint_full<double>(e, T, &none, fA, fB, nullptr, nullptr, nullptr, s, &k)
                                      : adjoint_full<float>(e, T, &none, fA, fB, nullptr, nullptr, nullptr, s, &k);
    if (st == RSWR_ENOMEM) {
        // the span states do not fit: a plain run, nothing kept
        e->kept = false;
        return plan_run(e, fA, fB, T, nullptr, nullptr, out0, out1, nullptr, recv ? j_r : -1, recv, stream, false);
    }
    return st;
}

rswr_status rswr_adjoint(rswr_plan_t plan, const void* fA, const void* fB, int64_t T, int64_t j_r, const void* wbar,
                         void* grad_fA, double* grad_a, void* stream)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    Engine* e = plan->e;
    if (T < 0) return fail(RSWR_EINVAL, "T < 0");
    if (!wbar || !grad_fA) return fail(RSWR_EINVAL, "wbar and grad_fA are required");
    if (j_r < 0 || j_r >= e->probs[0].nx) return fail(RSWR_EINVAL, "receiver index outside the grid");
    if (!e->usrc.empty()) return fail(RSWR_ENOTSUP, "the adjoint runs without user point sources");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grad_a) return adjoint_dispatch(e, T, &j_r, fA, fB, wbar, grad_fA, grad_a, s);
    return adjoint_g(e, T, &j_r, wbar, grad_fA, s);
}

rswr_status rswr_batch_create(rswr_batch_t* batch, int32_t nprob, const rswr_problem* problems, int32_t dtype,
                              int32_t form, uint32_t flags)
{
    if (!batch) return fail(RSWR_EINVAL, "batch is NULL");
    *batch = nullptr;
    (void)flags;
    Engine* e = nullptr;
    rswr_status st = make_engine(&e, nprob, problems, dtype, form, false);
    if (st != RSWR_OK) return st;
    *batch = new (std::nothrow) rswr_batch_s{e};
    if (!*batch) {
        free_engine(e);
        return fail(RSWR_ENOMEM, "host allocation");
    }
    return RSWR_OK;
}

void rswr_batch_destroy(rswr_batch_t batch)
{
    if (!batch) return;
    free_engine(batch->e);
    delete batch;
}

rswr_status rswr_batch_offsets(rswr_batch_t batch, int64_t* offsets)
{
    if (!batch || !offsets) return fail(RSWR_EINVAL, "NULL argument");
    std::copy(batch->e->h_offsets.begin(), batch->e->h_offsets.end(), offsets);
    return RSWR_OK;
}

rswr_status rswr_batch_get_info(rswr_batch_t batch, rswr_plan_info* info)
{
    if (!batch) return fail(RSWR_EINVAL, "NULL batch");
    return fill_info(batch->e, info);
}

rswr_status rswr_batch_set_mode(rswr_batch_t batch, int32_t mode)
{
    if (!batch) return fail(RSWR_EINVAL, "NULL batch");
    if (mode != RSWR_MODE_PERSISTENT && mode != RSWR_MODE_PER_SPAN) return fail(RSWR_EINVAL, "bad mode");
    batch->e->mode = mode;
    return RSWR_OK;
}

rswr_status rswr_batch_set_variant(rswr_batch_t batch, int32_t variant)
{
    if (!batch) return fail(RSWR_EINVAL, "NULL batch");
    return set_variant(batch->e, variant);
}

rswr_status rswr_batch_set_wait_limit(rswr_batch_t batch, double seconds)
{
    if (!batch) return fail(RSWR_EINVAL, "NULL batch");
    if (!(seconds > 0.0) || seconds > 3600.0) return fail(RSWR_EINVAL, "wait limit out of range");
    batch->e->wait_s = seconds;
    return RSWR_OK;
}

rswr_status rswr_batch_set_checkpoint_spacing(rswr_batch_t batch, int64_t spans)
{
    if (!batch) return fail(RSWR_EINVAL, "NULL batch");
    if (spans < 0) return fail(RSWR_EINVAL, "checkpoint spacing must be >= 0");
    batch->e->ck_spacing = spans;
    return RSWR_OK;
}

rswr_status rswr_batch_set_kernel_events(rswr_batch_t batch, void* start, void* stop)
{
    if (!batch) return fail(RSWR_EINVAL, "NULL batch");
    if ((start == nullptr) != (stop == nullptr)) return fail(RSWR_EINVAL, "give both events or neither");
    batch->e->ev_start = static_cast<cudaEvent_t>(start);
    batch->e->ev_stop = static_cast<cudaEvent_t>(stop);
    return RSWR_OK;
}

rswr_status rswr_batch_check(rswr_batch_t batch, void* stream, int32_t* code, int32_t* tile, int32_t* span)
{
    if (!batch) return fail(RSWR_EINVAL, "NULL batch");
    return check_engine(batch->e, static_cast<cudaStream_t>(stream), code, tile, span);
}

rswr_status rswr_batch_set_sources(rswr_batch_t batch, int64_t nsrc, const int32_t* problem, const int64_t* j,
                                   const void* samples, int64_t pitch)
{
    if (!batch) return fail(RSWR_EINVAL, "NULL batch");
    if (nsrc > 0 && !problem) return fail(RSWR_EINVAL, "problem indices are required");
    return set_sources(batch->e, nsrc, problem, j, samples, pitch);
}

rswr_status rswr_batch_run(rswr_batch_t batch, const void* fA, const void* fB, int64_t T, const void* q0,
                           const void* q1, void* out0, void* out1, const int64_t* j_r, void* recv, void* stream)
{
    if (!batch) return fail(RSWR_EINVAL, "NULL batch");
    Engine* e = batch->e;
    if (T < 0) return fail(RSWR_EINVAL, "T < 0");
    if (!out0 || !out1) return fail(RSWR_EINVAL, "out0 and out1 are required");
    RunReq r;
    r.fA = fA;
    r.fB = fB;
    r.T = T;
    r.q0 = q0;
    r.q1 = q1;
    r.out0 = out0;
    r.out1 = out1;
    r.user_src = true;
    if (recv && j_r) {
        for (size_t p = 0; p < e->probs.size(); ++p) {
            if (j_r[p] < 0) continue;
            if (j_r[p] >= e->probs[p].nx) return fail(RSWR_EINVAL, "receiver index outside the grid");
            r.probes.push_back(ProbeReq{(int64_t)p, j_r[p], 0, 1.0,
                                        static_cast<char*>(recv) + e->esize() * (T + 1) * p, 1, T});
        }
    }
    return run_engine(e, r, static_cast<cudaStream_t>(stream));
}

rswr_status rswr_batch_adjoint(rswr_batch_t batch, const void* fA, const void* fB, int64_t T, const int64_t* j_r,
                               const void* wbar, void* grad_fA, double* grad_a, void* stream)
{
    if (!batch) return fail(RSWR_EINVAL, "NULL batch");
    Engine* e = batch->e;
    if (T < 0 || !j_r || !wbar || !grad_fA) return fail(RSWR_EINVAL, "bad argument");
    for (size_t p = 0; p < e->probs.size(); ++p)
        if (j_r[p] < 0 || j_r[p] >= e->probs[p].nx) return fail(RSWR_EINVAL, "receiver index outside the grid");
    if (!e->usrc.empty()) return fail(RSWR_ENOTSUP, "the adjoint runs without user point sources");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (grad_a) return adjoint_dispatch(e, T, j_r, fA, fB, wbar, grad_fA, grad_a, s);
    return adjoint_g(e, T, j_r, wbar, grad_fA, s);
}

rswr_status rswr_plan_autotune(rswr_plan_t plan, int64_t probe_steps, int32_t* variant, void* stream)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    return autotune_engine(plan->e, probe_steps, variant, static_cast<cudaStream_t>(stream), true);
}

rswr_status rswr_batch_autotune(rswr_batch_t batch, int64_t probe_steps, int32_t* variant, void* stream)
{
    if (!batch) return fail(RSWR_EINVAL, "NULL batch");
    return autotune_engine(batch->e, probe_steps, variant, static_cast<cudaStream_t>(stream), true);
}

rswr_status rswr_plan_set_graph(rswr_plan_t plan, int32_t enable)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    plan->e->use_graph = enable != 0;
    return RSWR_OK;
}

rswr_status rswr_batch_set_graph(rswr_batch_t batch, int32_t enable)
{
    if (!batch) return fail(RSWR_EINVAL, "NULL batch");
    batch->e->use_graph = enable != 0;
    return RSWR_OK;
}

rswr_status rswr_run_paper(rswr_plan_t plan, const void* fA, const void* fB, int64_t T, const void* q0,
                           const void* q1, void* out0, void* out1, int64_t* spans, int64_t spans_cap,
                           int64_t* nspans, void* stream)
{
    if (!plan) return fail(RSWR_EINVAL, "NULL plan");
    Engine* e = plan->e;
    if (T < 0) return fail(RSWR_EINVAL, "T < 0");
    if (!out0 || !out1) return fail(RSWR_EINVAL, "out0 and out1 are required");
    const ProbHost& ph = e->probs[0];
    if (ph.ov + 64 > 2048) return fail(RSWR_EINVAL, "paper-literal path supports overlaps up to 1984 points");
    if (!e->usrc.empty()) return fail(RSWR_ENOTSUP, "the paper-literal path runs without user point sources");
    if (e->part) return fail(RSWR_ENOTSUP, "the paper-literal path runs on whole grids only");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (e->dtype == kF64)
        return run_paper<double>(e, static_cast<const double*>(fA), static_cast<const double*>(fB), T,
                                 static_cast<const double*>(q0), static_cast<const double*>(q1),
                                 static_cast<double*>(out0), static_cast<double*>(out1), spans, spans_cap, nspans,
                                 0.1, s);
    return run_paper<float>(e, static_cast<const float*>(fA), static_cast<const float*>(fB), T,
                            static_cast<const float*>(q0), static_cast<const float*>(q1), static_cast<float*>(out0),
                            static_cast<float*>(out1), spans, spans_cap, nspans, 0.1, s);
}

int32_t rswr_variant_count(void) { return span_variant_count(); }

rswr_status rswr_variant_get(int32_t v, int32_t* dtype, int32_t* form, int32_t* points_per_thread,
                             int32_t* threads_per_cta)
{
    if (v < 0 || v >= span_variant_count()) return fail(RSWR_EINVAL, "variant out of range");
    const VariantInfo vi = span_variant_info(v);
    if (dtype) *dtype = vi.dtype == kF64 ? RSWR_F64 : RSWR_F32;
    if (form) *form = vi.form == kCanonical ? RSWR_FORM_CANONICAL : RSWR_FORM_INCREMENT;
    if (points_per_thread) *points_per_thread = vi.P;
    if (threads_per_cta) *threads_per_cta = vi.NT;
    return RSWR_OK;
}

rswr_status rswr_variant_get_kind(int32_t v, int32_t* kind)
{
    if (v < 0 || v >= span_variant_count()) return fail(RSWR_EINVAL, "variant out of range");
    if (!kind) return fail(RSWR_EINVAL, "kind is NULL");
    const VariantInfo vi = span_variant_info(v);
    *kind = vi.resident ? RSWR_VARIANT_RESIDENT : (vi.threads > vi.NT ? RSWR_VARIANT_WARP_SPECIALISED
                                                                     : RSWR_VARIANT_SINGLE_ROLE);
    return RSWR_OK;
}

rswr_status rswr_variant_get_tiling(int32_t v, int32_t* warp_halo, int32_t* window, int32_t* max_span,
                                    int32_t* threads_launched)
{
    if (v < 0 || v >= span_variant_count()) return fail(RSWR_EINVAL, "variant out of range");
    const VariantInfo vi = span_variant_info(v);
    if (warp_halo) *warp_halo = vi.KH;
    if (window) *window = vi.W;
    if (max_span) *max_span = vi.max_span;
    if (threads_launched) *threads_launched = vi.threads;
    return RSWR_OK;
}

}  // extern "C"
