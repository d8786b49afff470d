// noalloc.cu -- rswr_run_noalloc: an RSWR run that never allocates memory.
//
// Who needs it: callers that are not allowed to call cudaMalloc (or any other
// allocating routine) on the path where they solve.  Two common cases: code
// that runs inside a framework whose caching allocator has already reserved
// the device memory the process may use, so a direct cudaMalloc either fails
// or steals memory the framework counts on; and latency-critical loops, where
// cudaMalloc / cudaFree synchronise the device and stall every stream.  The
// plan API allocates its workspace once at rswr_plan_create; this entry point
// instead works in a fixed scratch area compiled into the library.
//
// The scratch area is a file-scope __device__ array of kScratchBytes.  Every
// GPU that loads this part of the library holds it until the process exits.
// Host code must not pass the array's name to a kernel (on the host that name
// is only a stand-in, not a device address), so the first call on each device
// asks the runtime for the array's device address with cudaGetSymbolAddress,
// with that device current, and remembers it.  That first call should be made
// before any stream capture begins.
//
// Every call uses the same scratch area, which keeps whatever the previous
// call left there: each call clears the parts that must start at zero.  Two
// calls whose work overlaps on the GPU (for example on two streams without an
// ordering between them) race on the scratch area and give wrong results.
//
// Each call waits for its own work at the end and reads the device error
// record back (a bounded wait inside a kernel that ran out of time is
// reported as RSWR_ETIMEOUT).  The remembered device address belongs to the
// device's current context: after cudaDeviceReset the library has to be
// loaded again before this entry point is used on that device.

#include <cstring>
#include <mutex>
#include <string>

#include "../../include/rswr.h"
#include "rswr_internal.h"

using namespace rswr;

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// failures are reported through rswr_last_error_message()
rswr_status nfail(rswr_status st, const std::string& m)
{
    set_error_message(m.c_str());
    return st;
}

// Device address of the scratch array on the current device (set-up once per device).
rswr_status scratch_address(void** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nfail(RSWR_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return nfail(RSWR_ENOTSUP, "device index beyond the supported range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return nfail(RSWR_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RSWR_OK;
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// the scratch layout gives the problem record and the error record one
// 256-byte slot each
static_assert(sizeof(ProblemDev<double>) <= 256 && sizeof(ProblemDev<float>) <= 256,
              "problem record larger than its scratch slot");
static_assert(sizeof(DevError) <= 256, "error record larger than its scratch slot");

// Writes the one-problem table and the tile table into the scratch area and
// clears the device error record.
template <typename Real>
__global__ void noalloc_tables_kernel(ProblemDev<Real>* prob, TileDev* tiles, DevError* err, int64_t base,
                                      int64_t nx, int64_t ntiles, const Real* fA, const Real* fB, Real c2, Real k)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        ProblemDev<Real> p{};
        p.base = base;
        p.nx = nx;
        p.tile0 = 0;
        p.ntiles = ntiles;
        p.fA = fA;
        p.fB = fB;
        p.src = nullptr;
        p.src_stride = 0;
        p.js = -1;
        p.c2 = c2;
        p.k = k;
        *prob = p;
        err->code = 0;
        err->tile = 0;
        err->span = 0;
        err->where = 0;
    }
    if (i < ntiles) tiles[i] = TileDev{0, (int32_t)i, 0, 0, 0, 0};
}

template <typename Real>
rswr_status run_noalloc(const rswr_problem& q, int form, const void* fA, const void* fB, int64_t T, const void* q0,
                        const void* q1, void* out0, void* out1, cudaStream_t s)
{
    // stencil coefficients (same definitions as the plan API)
    const double dx = (q.xb - q.xa) / (double)(q.nx - 1);
    const double c = q.a * q.dt / dx;
    const double c2d = c * c;
    const double kd = 2.0 - 2.0 * c2d;
    const float c2f = (float)c2d;
    const float kf = 2.0f - 2.0f * c2f;
    if (!(c <= 1.0)) return nfail(RSWR_ECFL, "Courant number a*dt/dx > 1");

    // kernel variant and tiling: the default variant of this dtype/form for the
    // span S = floor(overlap / 2), one launch per span
    const int dtype = sizeof(Real) == 8 ? kF64 : kF32;
    const int S = q.overlap / 2 < 256 ? q.overlap / 2 : 256;
    int v = -1;
    for (int i = 0; i < span_variant_count(); ++i) {
        const VariantInfo vi = span_variant_info(i);
        if (vi.dtype == dtype && vi.form == form && !vi.resident && (vi.max_span == 0 || S <= vi.max_span)) {
            v = i;
            break;
        }
    }
    if (v < 0) return nfail(RSWR_ENOTSUP, "no kernel variant for this dtype/form");
    const VariantInfo vi = span_variant_info(v);
    const int W = vi.W;
    const int H = (S + 3) / 4 * 4;
    const int core = W - 2 * H;
    if (core < H || core < 4) return nfail(RSWR_EINVAL, "overlap too large for the CTA window");
    const int64_t ntiles = (q.nx + core - 1) / core;
    const int64_t pad = H + 8;
    const int64_t len = (int64_t)round_up((size_t)(pad + ntiles * core + pad), 32);

    // scratch layout: problem | tiles | error record | 4 state arrays
    const size_t off_tiles = 256;
    const size_t off_err = round_up(off_tiles + sizeof(TileDev) * (size_t)ntiles, 256);
    const size_t off_state = off_err + 256;
    const size_t arr = round_up(sizeof(Real) * (size_t)len, 256);
    const size_t need = off_state + 4 * arr;
    if (need > kScratchBytes)
        return nfail(RSWR_EINVAL, "problem needs " + std::to_string(need) + " bytes of scratch; the no-allocation "
                                  "entry point has " + std::to_string(kScratchBytes) + " (use rswr_plan_create)");

    void* base_ptr = nullptr;
    rswr_status st = scratch_address(&base_ptr);
    if (st != RSWR_OK) return st;
    unsigned char* sb = static_cast<unsigned char*>(base_ptr);
    auto* prob = reinterpret_cast<ProblemDev<Real>*>(sb);
    auto* tiles = reinterpret_cast<TileDev*>(sb + off_tiles);
    auto* err = reinterpret_cast<DevError*>(sb + off_err);
    Real* st0[2] = {reinterpret_cast<Real*>(sb + off_state), reinterpret_cast<Real*>(sb + off_state + arr)};
    Real* st1[2] = {reinterpret_cast<Real*>(sb + off_state + 2 * arr), reinterpret_cast<Real*>(sb + off_state + 3 * arr)};

#define NA_CUDA(call)                                                                                     \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return nfail(RSWR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

    // the scratch area keeps the previous call's contents: clear every state array
    NA_CUDA(cudaMemsetAsync(sb + off_state, 0, 4 * arr, s));
    const Real c2 = sizeof(Real) == 8 ? (Real)c2d : (Real)c2f;
    const Real kk = sizeof(Real) == 8 ? (Real)kd : (Real)kf;
    const int64_t nthreads = ntiles > 1 ? ntiles : 1;
    noalloc_tables_kernel<Real><<<(unsigned)((nthreads + 255) / 256), 256, 0, s>>>(
        prob, tiles, err, pad, q.nx, ntiles, static_cast<const Real*>(fA), static_cast<const Real*>(fB), c2, kk);
    NA_CUDA(cudaGetLastError());
    if (q0) {
        NA_CUDA(cudaMemcpyAsync(st0[0] + pad, q0, sizeof(Real) * q.nx, cudaMemcpyDeviceToDevice, s));
        if (q1)
            NA_CUDA(cudaMemcpyAsync(st1[0] + pad, q1, sizeof(Real) * q.nx, cudaMemcpyDeviceToDevice, s));
        else if (form == kCanonical)
            NA_CUDA(cudaMemcpyAsync(st1[0] + pad, q0, sizeof(Real) * q.nx, cudaMemcpyDeviceToDevice, s));
    }
    NA_CUDA(set_boundary_launch(dtype, form, st0[0], st1[0], prob, 1, s));

    const int nspans = (int)((T + S - 1) / S);
    SpanParams<Real> prm{};
    prm.problems = prob;
    prm.tiles = tiles;
    prm.probes = nullptr;
    for (int b = 0; b < 2; ++b) {
        prm.q0[b] = st0[b];
        prm.q1[b] = st1[b];
    }
    prm.ntiles = ntiles;
    prm.T = T;
    prm.H = H;
    prm.core = core;
    prm.S = S;
    prm.nspans = nspans;
    prm.inject_tile = -1;
    prm.inject_span = -1;
    prm.ticket = nullptr;
    prm.done = nullptr;
    prm.err = err;
    prm.wait_ns = 5000000000LL;
    int bps = 0;
    NA_CUDA(span_occupancy(v, &bps));
    int sms = 1, dev = 0;
    NA_CUDA(cudaGetDevice(&dev));
    NA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t g = (int64_t)(bps > 0 ? bps : 1) * sms;
    const int grid = (int)(g < ntiles ? g : ntiles);
    for (int kspan = 0; kspan < nspans; ++kspan) {
        prm.span = kspan;
        NA_CUDA(span_launch(v, &prm, grid, s));
    }
    const int fin = nspans & 1;
    NA_CUDA(cudaMemcpyAsync(out0, st0[fin] + pad, sizeof(Real) * q.nx, cudaMemcpyDeviceToDevice, s));
    NA_CUDA(cudaMemcpyAsync(out1, st1[fin] + pad, sizeof(Real) * q.nx, cudaMemcpyDeviceToDevice, s));
    // the device error record of this call: wait for the run, then read it
    DevError h{};
    NA_CUDA(cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
#undef NA_CUDA
    if (h.code == kDevTimeoutLoad || h.code == kDevTimeoutFlag)
        return nfail(RSWR_ETIMEOUT, "device wait expired (code " + std::to_string(h.code) + ", tile " +
                                        std::to_string(h.tile) + ", span " + std::to_string(h.span) + ")");
    if (h.code != 0) return nfail(RSWR_ECUDA, "device error code " + std::to_string(h.code));
    return RSWR_OK;
}

}  // namespace

extern "C" rswr_status rswr_run_noalloc(double xa, double xb, double a, int64_t nx, double dt, int32_t n_sub,
                                        int32_t overlap, int32_t dtype, const void* fA, const void* fB, int64_t T,
                                        const void* q0, const void* q1, void* out0, void* out1, void* stream)
{
    if (!out0 || !out1) return nfail(RSWR_EINVAL, "out0 and out1 are required");
    if (T < 0) return nfail(RSWR_EINVAL, "T < 0");
    if (nx < 3 || n_sub < 1 || !(a > 0.0) || !(dt > 0.0) || !(xb > xa))
        return nfail(RSWR_EINVAL, "need nx >= 3, n_sub >= 1, a > 0, dt > 0, xb > xa");
    if (overlap < 2 || nx / n_sub < overlap) return nfail(RSWR_EOVERLAP, "overlap < 2 or a core shorter than it");
    if (dtype != RSWR_F32 && dtype != RSWR_F64) return nfail(RSWR_EINVAL, "dtype must be RSWR_F32 or RSWR_F64");
    const rswr_problem q{nx, xa, xb, a, dt, n_sub, overlap};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the scratch address and the launch size come from the current device,
    // so the stream must belong to it
    if (s) {
        int cur = -1, sdev = -1;
        if (cudaGetDevice(&cur) != cudaSuccess || cudaStreamGetDevice(s, &sdev) != cudaSuccess)
            return nfail(RSWR_ECUDA, "cannot query the device of the stream");
        if (cur != sdev) return nfail(RSWR_EINVAL, "the stream belongs to another device than the current one");
    }
    if (dtype == RSWR_F64) return run_noalloc<double>(q, kCanonical, fA, fB, T, q0, q1, out0, out1, s);
    return run_noalloc<float>(q, kIncrement, fA, fB, T, q0, q1, out0, out1, s);
}
