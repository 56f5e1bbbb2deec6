// pp_noalloc.cu -- pp_fields_noalloc: the field of Eq. B for callers that
// cannot allocate device memory.
//
// Sources are staged hi/lo (two floats per coordinate, about 48 significant
// bits), so close pairs keep their separations and the field meets the 1e-5
// relative-L2 tolerance also on inputs whose closest pairs sit 1e3 times closer
// than the bunch size (single FP32 staging loses ~3e-5 there).
//
// Some callers cannot call cudaMalloc at all: code that runs inside a
// memory pool or arena owned by a host framework that forbids foreign
// allocations, code that must never trigger the allocator's implicit device
// synchronisation in a latency-critical loop, or a plug-in that may only use
// the buffers it is handed.  This entry point serves them.  It takes device
// inputs and outputs from the caller and keeps every intermediate (SoA copy of
// the positions, staged hi/lo float4 sources, j-split partial sums, tickets,
// moment partials, error word) in one file-scope __device__ array of fixed size.
//
// The array exists on every GPU that loads this library, for the lifetime of
// the process (kScratchBytes, 4.09 MB).  All calls on a device share it
// and it keeps the last call's contents; the entry point clears the parts that
// must start at zero (tickets, error word) on every call.  Calls whose work
// overlaps on the GPU (several host threads, or several streams) race on the
// array and must be serialised by the caller.
//
// The host-side name of a __device__ array is only a stand-in for it, not a
// device address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it together with
// the identity of the device's current context; make that first call before any
// stream capture.  If the context was destroyed and recreated since (for
// example after cudaDeviceReset), the next call sees another context identity
// and looks the address up again instead of writing through a stale one.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda.h>

#include "../../include/pp.h"
#include "pp_internal.h"

using namespace ppk;

namespace {

constexpr int kNoAllocMaxN = PP_FIELDS_NOALLOC_MAX_N;    // largest N accepted
constexpr int kNoAllocMaxSplit = 8;                      // j-chunks per i-block
constexpr int kT = 128, kR = 2, kTile = 128, kStages = 4;
constexpr int kBI = kT * kR;
constexpr int kMaxPad = (kNoAllocMaxN + kPad - 1) / kPad * kPad;
constexpr int kMaxNib = (kNoAllocMaxN + kBI - 1) / kBI;

// Byte offsets of the parts of the scratch array (each 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffSoa = 0;                                              // 3 x double[max_pad]
constexpr size_t kOffStage = align256(kOffSoa + 3 * sizeof(double) * kMaxPad);  // float4[2 max_pad]
constexpr size_t kOffPartial = align256(kOffStage + 2 * sizeof(float4) * kMaxPad);
constexpr size_t kOffTickets =
    align256(kOffPartial + sizeof(double) * kNoAllocMaxSplit * 3 * (size_t)kMaxNib * kBI);
constexpr size_t kOffMomPart = align256(kOffTickets + sizeof(unsigned) * kMaxNib);
constexpr size_t kOffMomOut = align256(kOffMomPart + sizeof(double) * kMomBlocks * kMomSlots);
constexpr size_t kOffErr = align256(kOffMomOut + sizeof(double) * kMomSlots);
constexpr size_t kScratchBytes = align256(kOffErr + 2 * sizeof(int));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
unsigned char *g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};   // context identity of each address

// Errors are reported through pp_last_error(), like every other call.
pp_status na_fail(pp_status s, const char *m)
{
    set_last_error(m);
    return s;
}

pp_status na_cuda(cudaError_t e, const char *where)
{
    char msg[256];
    std::snprintf(msg, sizeof(msg), "%s: %s", where, cudaGetErrorString(e));
    set_last_error(msg);
    return PP_ERR_CUDA;
}

#define NA_CUDA(call)                                      \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return na_cuda(e_, #call);  \
    } while (0)

// Identity of the calling thread's current CUDA context (unique for the life of
// the process; a context recreated after a device reset gets a new one), or 0
// where the driver does not report one.
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static const std::pair<GetCurrent, GetId> fns = [] {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult q1{}, q2{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault,
                                             &q1) != cudaSuccess || q1 != cudaDriverEntryPointSuccess)
            a = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess || q2 != cudaDriverEntryPointSuccess)
            b = nullptr;
        return std::make_pair(reinterpret_cast<GetCurrent>(a), reinterpret_cast<GetId>(b));
    }();
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!fns.first || !fns.second || fns.first(&ctx) != CUDA_SUCCESS || !ctx ||
        fns.second(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array on the current device: looked up once
// per device (with that device current), and again if the device's context
// has been recreated since.
pp_status scratch_address(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return na_fail(PP_ERR_ARG, "device ordinal out of range");
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> g(g_setup_lock);
    if (!g_scratch_addr[dev] || ctx == 0 || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return na_cuda(e, "cudaGetSymbolAddress(scratch)");
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return PP_OK;
}

}  // namespace

extern "C" pp_status pp_fields_noalloc(int64_t N, double w, double softening, const double *pos,
                                       double *E_out, void *stream_handle)
{
    if (N < 1 || N > kNoAllocMaxN)
        return na_fail(PP_ERR_ARG, "pp_fields_noalloc: N must be in [1, PP_FIELDS_NOALLOC_MAX_N = 16384]");
    if (!pos || !E_out) return na_fail(PP_ERR_ARG, "pp_fields_noalloc: null pointer");
    if (!(std::isfinite(w) && w > 0)) return na_fail(PP_ERR_ARG, "w must be finite and > 0");
    if (!(std::isfinite(softening) && softening >= 0))
        return na_fail(PP_ERR_ARG, "softening must be finite and >= 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream_handle);
    int dev = 0;
    NA_CUDA(cudaGetDevice(&dev));
    unsigned char *base = nullptr;
    if (pp_status s = scratch_address(dev, &base)) return s;

    const int n = (int)N;
    const int npad = (n + kPad - 1) / kPad * kPad;
    double *sx = reinterpret_cast<double *>(base + kOffSoa);
    double *sy = sx + kMaxPad, *sz = sy + kMaxPad;
    float4 *stage = reinterpret_cast<float4 *>(base + kOffStage);
    double *partial = reinterpret_cast<double *>(base + kOffPartial);
    unsigned *tickets = reinterpret_cast<unsigned *>(base + kOffTickets);
    double *mom_part = reinterpret_cast<double *>(base + kOffMomPart);
    double *mom_out = reinterpret_cast<double *>(base + kOffMomOut);
    int *err = reinterpret_cast<int *>(base + kOffErr);

    const int nib = (n + kBI - 1) / kBI;
    NA_CUDA(cudaMemsetAsync(tickets, 0, sizeof(unsigned) * nib, st));
    NA_CUDA(cudaMemsetAsync(err, 0, 2 * sizeof(int), st));
    NA_CUDA(launch_aos_to_soa(pos, n, sx, sy, sz, err + 1, st));

    // staging frame: centroid and the power of two nearest the RMS radius
    double m[kMomSlots];
    NA_CUDA(launch_moments(0, n, sx, sy, sz, sx, sy, sz, 0, 0, 0, mom_part, mom_out, st));
    NA_CUDA(cudaMemcpyAsync(m, mom_out, sizeof(m), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    const double cx = m[0] / n, cy = m[1] / n, cz = m[2] / n;
    NA_CUDA(launch_moments(1, n, sx, sy, sz, sx, sy, sz, cx, cy, cz, mom_part, mom_out, st));
    NA_CUDA(cudaMemcpyAsync(m, mom_out, sizeof(m), cudaMemcpyDeviceToHost, st));
    int flags[2] = {0, 0};
    NA_CUDA(cudaMemcpyAsync(flags, err, sizeof(flags), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    if (flags[1]) return na_fail(PP_ERR_ARG, "non-finite position");
    const double rms = std::sqrt(m[0] / n);
    double l0 = 1.0;
    if (std::isfinite(rms) && rms > 0.0) {
        int e = (int)std::lround(std::log2(rms));
        e = e < -200 ? -200 : (e > 200 ? 200 : e);
        l0 = std::ldexp(1.0, e);
    }
    // hi parts at stage[0, npad), lo parts at stage[npad, 2 npad)
    NA_CUDA(launch_stage(sx, sy, sz, n, npad, stage, STAGE_F32X2, cx, cy, cz, 1.0 / l0, st));

    const int tiles = npad / kTile;
    const int nsplit_req = tiles < kNoAllocMaxSplit ? tiles : kNoAllocMaxSplit;
    const int chunk_tiles = (tiles + nsplit_req - 1) / nsplit_req;
    ForceArgs a{};
    a.src = stage;
    a.n = n;
    a.npad = npad;
    a.nib = nib;
    a.jchunk = chunk_tiles * kTile;
    a.nsplit = (tiles + chunk_tiles - 1) / chunk_tiles;
    a.mode = MODE_FIELDS;
    const double epsl = softening / l0;
    a.eps2d = epsl * epsl;
    a.eps2f = (float)a.eps2d;
    a.partial = partial;
    a.tickets = tickets;
    a.nipad = nib * kBI;
    a.out = E_out;
    a.escale = -kCoulomb * kE * w / (l0 * l0);
    a.cx = cx;
    a.cy = cy;
    a.cz = cz;
    a.inv_l0 = 1.0 / l0;
    a.err = err;
    a.timeout_ns = 1000000000ull;
    void *args[] = {&a};
    const void *fn = reinterpret_cast<const void *>(
        &force_f32_kernel<kT, kR, kTile, kStages, ACC_FP64FOLD, 4, true>);
    NA_CUDA(cudaLaunchKernel(fn, dim3(nib * a.nsplit), dim3(kT), args,
                             (size_t)kStages * kTile * sizeof(float4) * 2, st));
    NA_CUDA(cudaMemcpyAsync(flags, err, sizeof(flags), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    if (flags[0]) return na_fail(PP_ERR_TIMEOUT, "a device-side wait ran out of time");
    return PP_OK;
}
