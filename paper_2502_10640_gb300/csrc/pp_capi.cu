// pp_capi.cu -- the C ABI declared in include/pp.h: context lifetime, device
// memory, launch planning (variant and j-split choice), CUDA-graph step
// blocks, error words and status codes.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "../../include/pp.h"
#include "pp_internal.h"

using namespace ppk;

namespace {

thread_local std::string g_last_error;

pp_status fail(pp_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

pp_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(PP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PP_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
    } while (0)

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

void ppk::set_last_error(const char *msg) { g_last_error = msg; }

struct pp_ctx {
    int64_t n = 0;
    int npad = 0;
    double w = 1, dt = 0, eps = 0;
    int device = 0;
    int sms = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;

    // FP64 state, SoA: r[3], v[3], a[3], each npad long, in one allocation.
    double *state = nullptr;
    double *r[3] = {}, *v[3] = {}, *a[3] = {};
    void *stage[2] = {};           // float4 (or double4 for FP64 pair math) [npad]
    size_t stage_bytes = 0;        // per buffer: 32 bytes per entry fits every layout
    double *aos = nullptr;         // [n][3] scratch for host transfers / outputs
    double *phi = nullptr;         // [n]
    double *wts = nullptr;         // per-particle weights [npad] (null: all equal to w)
    float *wrel = nullptr;         // w_i / w as staged [npad]
    double *partial = nullptr;     // split partials
    size_t partial_bytes = 0;
    unsigned *tickets = nullptr;
    int tickets_cap = 0;
    double *mom_partials = nullptr;
    double *mom_out = nullptr;
    int *err = nullptr;            // [0]: wait ran out, [1]: non-finite input
    unsigned *res_flags = nullptr; // grid-barrier counter of the resident kernel
    void *ord_ws = nullptr;        // spatial-order workspace (tile-box guard variants)
    size_t ord_bytes = 0;
    double *mom_host = nullptr;    // pinned
    int *err_host = nullptr;       // pinned copy of err[0..1], read after each synchronisation

    int parity = 0;
    bool loaded = false;
    int64_t step = 0;
    double cx = 0, cy = 0, cz = 0, l0 = 1;

    int acc = PP_ACC_FP64FOLD;
    int positions = PP_POS_SINGLE;   // in force: SINGLE, SPLIT or GUARDED
    bool positions_auto = true;      // PP_POS_AUTO (the default): decide at every load
    double auto_rel_single = NAN;    // last AUTO measurements against hi/lo staging
    double auto_rel_guarded = NAN;
    int split_override = 0;
    int variant_override = -1;
    int graph_block = 16;
    uint64_t timeout_ns = 1000000000ull;
    int skip_copy = 0;
    int resident = PP_RESIDENT_AUTO;  // small-N stepping in one cooperative launch
    bool res_plan_valid = false;      // cached resident plan and the settings it was made for
    int64_t res_plan_key[6] = {};
    alignas(8) unsigned char res_plan[64] = {};

    // cached step graphs for (graph_block, start parity)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_steps = 0;
};

namespace {

void drop_graphs(pp_ctx *c)
{
    for (auto &g : c->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    c->graph_steps = 0;
}

bool f64_pairs(const pp_ctx *c) { return c->acc == PP_ACC_FP64_FULL; }

const Variant *variant_by_name(const char *want)
{
    int count = 0;
    const Variant *vs = variants(&count);
    for (int i = 0; i < count; ++i)
        if (std::strcmp(vs[i].name, want) == 0) return &vs[i];
    std::fprintf(stderr, "pp: no kernel variant named %s\n", want);
    std::abort();   // a missing table entry is a build error, not a runtime condition
}

// From this N on, guarded staging sorts the sources in space each pass and
// tests tile boxes instead of every pair.  Measured on GB300 (ms per step, the
// fastest box form against the fastest per-pair form, uniform balls and
// Gaussians alike): 3.61 against 3.75 at N = 98304, 6.21 against 6.50 at
// 131072, 23.6 against 24.9 at 262144, 366 against 397 at 2^20; below 98304
// the per-pair test wins (1.67 against 1.75 at 65536, 0.45 against 0.58 at
// 32768), its small tiles filling the GPU better.  512-source box tiles (hi
// and lo in a two-stage ring) from kBoxGuardWideN on, 256 below; the pair loop
// unrolled twice (2-4 % faster than once).
constexpr int64_t kBoxGuardMinN = 98304;
constexpr int64_t kBoxGuardWideN = 196608;

// The variant that runs this context's force passes: the override if it fits
// the accumulation and positions modes, else the default for N.
const Variant *force_variant(const pp_ctx *c)
{
    if (f64_pairs(c)) return variant_by_name("f64.full.t128r2k128");
    int count = 0;
    const Variant *vs = variants(&count);
    const int want_kind = c->wts ? KIND_FORCE32W : KIND_FORCE32;
    if (c->variant_override >= 0 && c->variant_override < count) {
        const Variant &v = vs[c->variant_override];
        if (v.kind == want_kind && v.acc == c->acc && v.positions == c->positions) return &v;
    }
    const bool big = c->n >= 32768, mid = c->n >= 8192;
    if (c->positions == PP_POS_GUARDED) {   // hi/lo staged, hi parts streamed
        if (c->wts)
            return variant_by_name(c->n >= kBoxGuardMinN ? "f32x2wbguard.sfold64.t128r4k512s2m4"
                                   : big ? "f32x2wguard.sfold64.t128r4k512m4"
                                   : mid ? "f32x2wguard.fold64.t128r2k128"
                                         : "f32x2wguard.fold64.t64r1k128");
        if (c->acc == PP_ACC_KAHAN)
            return variant_by_name(c->n >= kBoxGuardWideN ? "f32x2bguard.kahan.st128r4k512s2m4u2"
                                   : big ? "f32x2guard.kahan.st128r4k512m4u1"
                                   : mid ? "f32x2guard.kahan.t128r2k128"
                                         : "f32x2guard.kahan.t64r1k128");
        if (c->n >= kBoxGuardMinN)   // spatially sorted sources, one test per tile
            return variant_by_name(c->n >= kBoxGuardWideN ? "f32x2bguard.sfold64.t128r4k512s2m4u2"
                                                          : "f32x2bguard.sfold64.t128r4k256m4u2");
        return variant_by_name(c->n >= 49152 ? "f32x2guard.fold64.t128r2k128"
                                             : "f32x2guard.fold64.t64r1k128");
    }
    if (c->wts && c->positions == PP_POS_SPLIT) {  // weights on hi/lo staged sources
        if (c->n >= 32768) return variant_by_name("f32x2wsplit.sfold64.t128r2k512m4");
        if (c->n >= 8192) return variant_by_name("f32x2wsplit.sfold64.t128r4k256m4");
        return variant_by_name("f32x2wsplit.fold64.t64r1k128");
    }
    if (c->wts) {  // per-particle weights: packed kernels that read the weight lanes
        if (c->n >= 32768) return variant_by_name("f32x2w.sfold64.t128r4k512m4");
        if (c->n >= 8192) return variant_by_name("f32x2w.fold64.t128r2k128");
        return variant_by_name("f32x2w.fold64.t64r1k128");
    }
    if (c->positions == PP_POS_SPLIT && c->acc == PP_ACC_KAHAN) {
        if (c->n >= 32768) return variant_by_name("f32x2split.kahan.st128r2k512m4");
        if (c->n >= 8192) return variant_by_name("f32x2split.kahan.st128r4k256m4");
        return variant_by_name("f32x2split.kahan.t64r1k128");
    }
    if (c->positions == PP_POS_SPLIT) {
        if (c->n >= 32768) return variant_by_name("f32x2split.sfold64.t128r2k512m4");
        if (c->n >= 8192) return variant_by_name("f32x2split.sfold64.t128r4k256m4");
        return variant_by_name("f32x2split.fold64.t64r1k128");
    }
    if (c->acc == PP_ACC_KAHAN) {  // packed pair math, compensated FP32 fold
        if (c->n >= 32768) return variant_by_name("f32x2.kahan.st128r4k1024s2m4u2");
        if (c->n >= 8192) return variant_by_name("f32x2.kahan.t128r2k128");
        return variant_by_name("f32x2.kahan.t64r1k128");
    }
    // packed f32x2 pair math; defaults from GB300 measurements (ms per step at
    // N = 8192 / 32768 / 98304 / 262144: 0.039 / 0.410 / 3.36 / 22.5 for the
    // chosen forms against 0.047 / 0.458 / 3.49 / 23.1 for the next best);
    // pp_autotune refines them per device and N
    if (c->n >= 196608) return variant_by_name("f32x2.sfold64.t128r4k1024s2m4u2");
    if (c->n >= 49152) return variant_by_name("f32x2.sfold64.t128r2k512m6");
    if (c->n >= 12288) return variant_by_name("f32x2.fold64.t128r2k128");
    return variant_by_name("f32x2.fold64.t64r1k128");
}

// Staging layout the force kernels of this context read.
int stage_kind(const pp_ctx *c) { return force_variant(c)->stage; }

// Pick the variant for a kind of pass.
const Variant *pick_variant(const pp_ctx *c, int kind)
{
    if (kind == KIND_PHI32)
        return variant_by_name(c->n >= 32768 ? "phi32.fold64.t256r2k256" : "phi32.fold64.t128r1k128");
    return force_variant(c);
}

// Can at least one cluster of this variant be resident on the device?
bool cluster_fits(const Variant &v)
{
    if (v.cluster > 8 &&
        cudaFuncSetAttribute(v.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(v.cluster);
    cfg.blockDim = dim3(v.T);
    cfg.dynamicSmemBytes = v.smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)v.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, v.fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n >= 1;
}

// Resident CTAs per SM of a variant (queried once per variant and process).
int resident_ctas(const Variant &v)
{
    static std::mutex lock;
    static std::map<std::pair<int, int>, int> cache;   // (device, variant) -> CTAs per SM
    int count = 0, dev = 0;
    const Variant *vs = variants(&count);
    const int idx = (int)(&v - vs);
    if (idx < 0 || idx >= count || cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> g(lock);
    auto it = cache.find({dev, idx});
    if (it != cache.end()) return it->second;
    int occ = 0;
    // the attribute is per device and must be set before the occupancy query
    cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v.fn, v.T, v.smem) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    cache[{dev, idx}] = occ;
    return occ;
}

struct Plan {
    const Variant *v;
    int nib, nsplit, jchunk, grid, nipad;
};

// Choose S, the number of j-chunks per i-block, to fill the GPU: minimise
// (waves of CTAs) x (tiles per CTA + fixed per-CTA overhead).
Plan make_plan(pp_ctx *c, int kind)
{
    Plan pl{};
    pl.v = pick_variant(c, kind);
    const int BI = pl.v->T * pl.v->R;
    pl.nib = (int)((c->n + BI - 1) / BI);
    pl.nipad = pl.nib * BI;
    const int tiles = c->npad / pl.v->tile;
    const int occ = resident_ctas(*pl.v);
    const int64_t slots = (int64_t)c->sms * occ;
    int best_s = 1;
    double best_cost = 1e300;
    const int smax = std::min(tiles, 512);
    for (int s = 1; s <= smax; ++s) {
        const int chunk_tiles = (tiles + s - 1) / s;
        const int s_eff = (tiles + chunk_tiles - 1) / chunk_tiles;
        if (s_eff != s) continue;
        const int64_t ctas = (int64_t)pl.nib * s;
        const int64_t waves = (ctas + slots - 1) / slots;
        // per-CTA set-up (targets, barriers, first copy) and the split
        // epilogue cost about a quarter of a tile
        const double cost = (double)waves * (chunk_tiles + 0.25);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best_s = s;
        }
    }
    if (c->split_override > 0) best_s = std::min(c->split_override, tiles);
    if (pl.v->cluster > 0) {
        // one cluster per target block, one source chunk per CTA of the cluster
        const int cl = pl.v->cluster;
        pl.jchunk = ((tiles + cl - 1) / cl) * pl.v->tile;
        pl.nsplit = cl;
        pl.grid = pl.nib * cl;
        return pl;
    }
    const int chunk_tiles = (tiles + best_s - 1) / best_s;
    pl.jchunk = chunk_tiles * pl.v->tile;
    pl.nsplit = (tiles + chunk_tiles - 1) / chunk_tiles;
    pl.grid = pl.nib * pl.nsplit;
    return pl;
}

pp_status ensure_workspace(pp_ctx *c, const Plan &pl)
{
    if (pl.v->order) {
        const size_t need = order_workspace_bytes(c->npad, pl.v->tile);
        if (need > c->ord_bytes) {
            if (c->ord_ws) cudaFree(c->ord_ws);
            c->ord_ws = nullptr;
            c->ord_bytes = 0;
            if (cudaMalloc(&c->ord_ws, need) != cudaSuccess) {
                cudaGetLastError();
                return fail(PP_ERR_NOMEM, "cannot allocate the spatial-order workspace");
            }
            c->ord_bytes = need;
            drop_graphs(c);
        }
    }
    const int ncomp = (pl.v->kind == KIND_PHI32) ? 1 : 3;
    const size_t need = (pl.nsplit > 1 && pl.v->cluster == 0)
                            ? (size_t)pl.nsplit * ncomp * pl.nipad * sizeof(double)
                            : 0;
    if (need > c->partial_bytes) {
        if (c->partial) cudaFree(c->partial);
        c->partial = nullptr;
        c->partial_bytes = 0;
        if (cudaMalloc(&c->partial, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(PP_ERR_NOMEM, "cannot allocate the j-split workspace");
        }
        c->partial_bytes = need;
        drop_graphs(c);
    }
    if (pl.nib > c->tickets_cap) {
        if (c->tickets) cudaFree(c->tickets);
        c->tickets = nullptr;
        if (cudaMalloc(&c->tickets, pl.nib * sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            return fail(PP_ERR_NOMEM, "cannot allocate the ticket array");
        }
        PP_CUDA(cudaMemsetAsync(c->tickets, 0, pl.nib * sizeof(unsigned), c->stream));
        c->tickets_cap = pl.nib;
        drop_graphs(c);
    }
    return PP_OK;
}

ForceArgs base_args(const pp_ctx *c, const Plan &pl, int mode, const void *src, void *dst,
                    double *out)
{
    ForceArgs a{};
    a.src = src;
    a.n = (int)c->n;
    a.npad = c->npad;
    a.nib = pl.nib;
    a.nsplit = pl.nsplit;
    a.jchunk = pl.jchunk;
    a.mode = mode;
    const double epsl = c->eps / c->l0;
    a.eps2d = epsl * epsl;
    a.eps2f = (float)a.eps2d;
    a.partial = c->partial;
    a.tickets = c->tickets;
    a.nipad = pl.nipad;
    for (int k = 0; k < 3; ++k) {
        a.r[k] = c->r[k];
        a.v[k] = c->v[k];
        a.a[k] = c->a[k];
    }
    a.dst = dst;
    a.out = out;
    a.wrel = c->wrel;
    // a_i = k e^2 w / (m_e L0^2) * sum_j d'/|d'|^3   (Eq. F with Eq. E, staged units)
    a.cscale = kCoulomb * kE * kE * c->w / (kMe * c->l0 * c->l0);
    // E_i = (m_e / q_e) a_i, q_e = -e
    a.escale = -kCoulomb * kE * c->w / (c->l0 * c->l0);
    a.dt = c->dt;
    a.half_dt = c->dt / 2.0;
    a.half_dt2 = c->dt * c->dt / 2.0;
    a.cx = c->cx;
    a.cy = c->cy;
    a.cz = c->cz;
    a.inv_l0 = 1.0 / c->l0;
    a.err = c->err;
    a.timeout_ns = c->timeout_ns;
    a.skip_copy = 0;
    return a;
}

// Read and clear the device error word; maps it to a status.
pp_status check_device_errors(pp_ctx *c, bool reset_state_on_timeout)
{
    int *h = c->err_host;
    PP_CUDA(cudaMemcpyAsync(h, c->err, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PP_CUDA(cudaStreamSynchronize(c->stream));
    if (h[0]) {
        PP_CUDA(cudaMemsetAsync(c->err, 0, 2 * sizeof(int), c->stream));
        if (c->tickets) PP_CUDA(cudaMemsetAsync(c->tickets, 0, c->tickets_cap * sizeof(unsigned), c->stream));
        PP_CUDA(cudaStreamSynchronize(c->stream));
        if (reset_state_on_timeout) c->loaded = false;
        return fail(PP_ERR_TIMEOUT, "a device-side wait ran out of time; the particle state is "
                                    "unspecified until particles are loaded or a state is set");
    }
    return PP_OK;
}

// Launch the plan's force kernel; a variant that works on spatially sorted
// sources first sorts a.src into the context's order workspace (sized by
// ensure_workspace) and passes the sorted copy, permutation and tile boxes.
cudaError_t launch_force(pp_ctx *c, const Plan &pl, ForceArgs a)
{
    if (pl.v->order) {
        const OrderWork w = order_carve(c->ord_ws, c->npad, pl.v->tile);
        const cudaError_t e =
            launch_spatial_order(a.src, (int)c->n, c->npad, pl.v->tile, w, c->stream);
        if (e != cudaSuccess) return e;
        a.src = w.sorted;
        a.perm = w.perm;
        a.boxes = w.boxes;
    }
    return launch_variant(*pl.v, a, pl.grid, c->stream);
}

// One force pass over staged sources src.
pp_status force_pass(pp_ctx *c, int mode, const void *src, void *dst, double *out)
{
    const int kind = (mode == MODE_PHI) ? KIND_PHI32 : (f64_pairs(c) ? KIND_FORCE64 : KIND_FORCE32);
    const Plan pl = make_plan(c, kind);
    pp_status st = ensure_workspace(c, pl);
    if (st != PP_OK) return st;
    ForceArgs a = base_args(c, pl, mode, src, dst, out);
    a.skip_copy = c->skip_copy;
    c->skip_copy = 0;
    PP_CUDA(launch_force(c, pl, a));
    return PP_OK;
}

pp_status stage_current(pp_ctx *c, void *dst, int kind)
{
    PP_CUDA(launch_stage(c->r[0], c->r[1], c->r[2], (int)c->n, c->npad, dst, kind, c->cx, c->cy,
                         c->cz, 1.0 / c->l0, c->stream, c->wrel));
    return PP_OK;
}

// The step epilogue writes staged entries i < n only, so the padding tail of
// both ping-pong buffers must hold far-away weight-0 sources of the current
// staging type before any step runs.
pp_status pad_both(pp_ctx *c)
{
    for (int b = 0; b < 2; ++b)
        PP_CUDA(launch_fill_padding(c->stage[b], (int)c->n, c->npad, stage_kind(c), c->stream));
    return PP_OK;
}

// Stage the pending positions drift(r_n, v_n, a_n) into stage[parity].
pp_status restage_pending(pp_ctx *c, bool sync = true)
{
    if (pp_status st = pad_both(c)) return st;
    PP_CUDA(launch_stage_drift(c->r, c->v, c->a, (int)c->n, c->npad, c->stage[c->parity],
                               stage_kind(c), c->dt, c->dt * c->dt / 2.0, c->cx, c->cy, c->cz,
                               1.0 / c->l0, c->stream, c->wrel));
    if (sync) PP_CUDA(cudaStreamSynchronize(c->stream));
    return PP_OK;
}

bool valid_mem(int kind) { return kind >= PP_MEM_HOST && kind <= PP_MEM_HOST_MAPPED; }

// Size of the CUDA allocation holding p, from the driver's pointer attributes
// (false where the driver does not report a range for this kind of memory).
bool allocation_range(const void *p, uintptr_t *start, size_t *size)
{
    using GetAttr = CUresult (*)(void *, CUpointer_attribute, CUdeviceptr);
    static GetAttr fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<GetAttr>(f);
    }();
    if (!fn) return false;
    CUdeviceptr st = 0;
    size_t sz = 0;
    if (fn(&st, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, (CUdeviceptr)(uintptr_t)p) != CUDA_SUCCESS ||
        fn(&sz, CU_POINTER_ATTRIBUTE_RANGE_SIZE, (CUdeviceptr)(uintptr_t)p) != CUDA_SUCCESS ||
        sz == 0)
        return false;
    *start = (uintptr_t)st;
    *size = sz;
    return true;
}

// True if the byte at q is mapped page-locked host memory whose device-side
// address is q - base + dbase.
bool mapped_byte(uintptr_t q, uintptr_t base, uintptr_t dbase)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, reinterpret_cast<const void *>(q)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost && at.devicePointer &&
           (uintptr_t)at.devicePointer == dbase + (q - base);
}

// Device-side address of a caller's PP_MEM_HOST_MAPPED buffer of `bytes`
// bytes.  The buffer must be page-locked host memory that CUDA maps into the
// device address space, and all of it must lie in one such allocation.  This
// is checked on the host, before any kernel touches the buffer: its first and
// last bytes must be mapped with contiguous device addresses, and the whole
// range must lie inside the allocation range the driver reports; where the
// driver reports none, every 4 KB page of the range is checked instead.
pp_status mapped_view(const void *p, size_t bytes, const void **dptr)
{
    if (!p || bytes == 0) return fail(PP_ERR_ARG, "PP_MEM_HOST_MAPPED buffer is empty");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return fail(PP_ERR_ARG, "PP_MEM_HOST_MAPPED buffer is not CUDA page-locked host memory");
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer)
        return fail(PP_ERR_ARG, "PP_MEM_HOST_MAPPED buffer is not mapped page-locked host memory");
    const uintptr_t lo = (uintptr_t)p, hi = lo + bytes, dlo = (uintptr_t)at.devicePointer;
    if (hi < lo || !mapped_byte(hi - 1, lo, dlo))
        return fail(PP_ERR_ARG, "PP_MEM_HOST_MAPPED buffer extends past its allocation");
    uintptr_t start = 0;
    size_t size = 0;
    if (allocation_range(p, &start, &size)) {
        if (lo < start || hi > start + size)
            return fail(PP_ERR_ARG, "PP_MEM_HOST_MAPPED buffer extends past its allocation");
    } else {
        for (uintptr_t q = (lo & ~(uintptr_t)4095) + 4096; q < hi; q += 4096)
            if (!mapped_byte(q, lo, dlo))
                return fail(PP_ERR_ARG, "PP_MEM_HOST_MAPPED buffer extends past its allocation");
    }
    *dptr = at.devicePointer;
    return PP_OK;
}

// Copy [n][3] from the caller into SoA dst; check finiteness.  Host memory
// goes through the copy engine into library scratch; device memory and mapped
// host memory are read by the conversion kernel itself.
pp_status import_aos(pp_ctx *c, const double *src, int kind, double *const dst[3])
{
    const size_t bytes = (size_t)c->n * 3 * sizeof(double);
    const double *dsrc = src;
    if (kind == PP_MEM_HOST) {
        PP_CUDA(cudaMemcpyAsync(c->aos, src, bytes, cudaMemcpyHostToDevice, c->stream));
        dsrc = c->aos;
    } else if (kind == PP_MEM_HOST_MAPPED) {
        const void *d = nullptr;
        if (pp_status st = mapped_view(src, bytes, &d)) return st;
        dsrc = static_cast<const double *>(d);
    }
    PP_CUDA(launch_aos_to_soa(dsrc, (int)c->n, dst[0], dst[1], dst[2], c->err + 1, c->stream));
    return PP_OK;
}

pp_status export_aos(pp_ctx *c, double *const src[3], double *out, int kind)
{
    const size_t bytes = (size_t)c->n * 3 * sizeof(double);
    double *target = out;
    if (kind == PP_MEM_HOST) {
        target = c->aos;
    } else if (kind == PP_MEM_HOST_MAPPED) {
        const void *d = nullptr;
        if (pp_status st = mapped_view(out, bytes, &d)) return st;
        target = static_cast<double *>(const_cast<void *>(d));
    }
    PP_CUDA(launch_soa_to_aos(src[0], src[1], src[2], (int)c->n, target, c->stream));
    if (kind == PP_MEM_HOST)
        PP_CUDA(cudaMemcpyAsync(out, c->aos, bytes, cudaMemcpyDeviceToHost, c->stream));
    return PP_OK;
}

pp_status take_bad_input_flag(pp_ctx *c, bool *bad)
{
    int *h = c->err_host + 1;
    PP_CUDA(cudaMemcpyAsync(h, c->err + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PP_CUDA(cudaStreamSynchronize(c->stream));
    const bool set = *h != 0;
    if (set) PP_CUDA(cudaMemsetAsync(c->err + 1, 0, sizeof(int), c->stream));
    *bad = set;
    return PP_OK;
}

pp_status moments(pp_ctx *c, int pass, const double *x, double out[kMomSlots])
{
    PP_CUDA(launch_moments(pass, (int)c->n, pass == 2 ? x : c->r[0], c->r[1], c->r[2], c->v[0],
                           c->v[1], c->v[2], c->cx, c->cy, c->cz, c->mom_partials, c->mom_out,
                           c->stream, c->wts));
    PP_CUDA(cudaMemcpyAsync(c->mom_host, c->mom_out, kMomSlots * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream));
    PP_CUDA(cudaStreamSynchronize(c->stream));
    std::memcpy(out, c->mom_host, kMomSlots * sizeof(double));
    return PP_OK;
}

// Choose the staging frame: centre = centroid, L0 = power of two nearest the
// RMS radius (so scaling by 1/L0 is exact).
pp_status choose_frame(pp_ctx *c)
{
    double m[kMomSlots];
    c->cx = c->cy = c->cz = 0.0;
    pp_status st = moments(c, 0, nullptr, m);
    if (st != PP_OK) return st;
    const double n = (double)c->n;
    const double cx = m[0] / n, cy = m[1] / n, cz = m[2] / n;
    c->cx = cx;
    c->cy = cy;
    c->cz = cz;
    st = moments(c, 1, nullptr, m);
    if (st != PP_OK) return st;
    const double rms = std::sqrt(m[0] / n);
    double l0 = 1.0;
    if (std::isfinite(rms) && rms > 0.0) {
        int e = (int)std::lround(std::log2(rms));
        e = std::max(-200, std::min(200, e));
        l0 = std::ldexp(1.0, e);
    }
    c->l0 = l0;
    return PP_OK;
}

bool graph_capturable(const pp_ctx *c) { return c->graph_block > 0 && c->stream != nullptr; }

pp_status build_graphs(pp_ctx *c)
{
    drop_graphs(c);
    const int kind = f64_pairs(c) ? KIND_FORCE64 : KIND_FORCE32;
    const Plan pl = make_plan(c, kind);
    pp_status st = ensure_workspace(c, pl);
    if (st != PP_OK) return st;
    for (int p0 = 0; p0 < 2; ++p0) {
        cudaGraph_t g = nullptr;
        PP_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        int par = p0;
        cudaError_t le = cudaSuccess;
        for (int k = 0; k < c->graph_block && le == cudaSuccess; ++k) {
            ForceArgs a = base_args(c, pl, MODE_STEP, c->stage[par], c->stage[par ^ 1], nullptr);
            le = launch_force(c, pl, a);
            par ^= 1;
        }
        cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
        if (le != cudaSuccess) return cuda_fail(le, "launch during graph capture");
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
        cudaError_t ie = cudaGraphInstantiate(&c->graph[p0], g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
    }
    c->graph_steps = c->graph_block;
    return PP_OK;
}

pp_status check_ctx(const pp_ctx *c)
{
    if (!c) return fail(PP_ERR_ARG, "null context");
    return PP_OK;
}


// ---- resident small-N stepping ------------------------------------------------
// Largest N whose staged sources fit one CTA's shared memory alongside the
// partial sums (npad = 12288: 192 KB + 12 KB); hi/lo staging needs twice the
// bytes per source.
constexpr int64_t kResidentMaxN = 12288;
constexpr int64_t kResidentMaxNSplit = 6144;
// Largest N for PP_RESIDENT_AUTO.  Measured on GB300 the resident kernel is
// faster than the per-launch kernels at every N up to the fit limit (2.9x at
// N = 64, 1.8x at 4096, 1.3x at 12288), so the two limits coincide.
constexpr int64_t kResidentAutoMaxN = kResidentMaxN;
// CTA size: 512 threads from this N on (more warps to hide latency once the
// pair work dominates), 256 below (fewer partial sums per target).
constexpr int64_t kResidentWideN = 3072;
// Steps per cooperative launch (bounds a launch to tens of milliseconds).
constexpr int64_t kResidentMaxSteps = 4096;
// Largest grid of the resident kernel (one CTA per SM).
constexpr int kResidentMaxGrid = 256;

struct ResidentPlan {
    bool ok = false;
    int form = 0, grid = 0, threads = 0, bt = 0, q = 0, chunk = 0, nsrc = 0;
};

// Can pp_step use the resident kernel, and how is the work split?
ResidentPlan compute_resident_plan(const pp_ctx *c, bool automatic)
{
    ResidentPlan rp;
    if (c->positions == PP_POS_GUARDED) return rp;   // per-launch kernels only
    const bool split = c->positions == PP_POS_SPLIT;
    const int64_t limit = split ? kResidentMaxNSplit
                                : (automatic ? kResidentAutoMaxN : kResidentMaxN);
    if (c->n > limit || c->acc == PP_ACC_FP64_FULL ||
        stage_kind(c) != (split ? STAGE_F32IX2 : STAGE_F32I))
        return rp;
    // hi/lo staging runs resident with the FP64 fold and equal weights only (weights
    // with the compensated fold are excluded by the library's modes)
    if (split && (c->acc == PP_ACC_KAHAN || c->wrel)) return rp;
    const int form = split ? RES_SPLIT
                           : c->acc == PP_ACC_KAHAN ? RES_KAHAN : c->wrel ? RES_WEIGHTED : RES_PLAIN;
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device) != cudaSuccess) {
        cudaGetLastError();
        return rp;
    }
    if (!coop) return rp;
    static DeviceOnce configured;
    if (configured.run(0, [] {
            return resident_configure((int)round_up(kResidentMaxN, kPad),
                                      (int)round_up(kResidentMaxNSplit, kPad));
        }) != cudaSuccess) {
        cudaGetLastError();
        return rp;
    }
    const int threads = c->n >= kResidentWideN ? 512 : 256;
    int occ = 0;
    if (resident_occupancy(c->npad, threads, form, &occ) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        return rp;
    }
    rp.threads = threads;
    rp.form = form;
    // one CTA per SM at most, and at least 8 targets per CTA; an even number of
    // targets per CTA keeps every CTA's staged block a whole number of source pairs
    const int64_t g0 = std::min<int64_t>((int64_t)c->sms, std::max<int64_t>(1, (c->n + 7) / 8));
    rp.bt = (int)round_up((c->n + g0 - 1) / g0, 2);
    if (3 * rp.bt > threads) return rp;   // one thread per (component, target) item
    rp.grid = (int)((c->n + rp.bt - 1) / rp.bt);
    if (rp.grid > c->sms * occ || rp.grid > kResidentMaxGrid) return rp;
    rp.nsrc = (int)round_up(c->n, 2);
    const int qmax = threads / rp.bt;
    // at least 32 sources per thread: fewer partial sums to add at tiny N
    rp.chunk = (int)round_up(std::max((rp.nsrc + qmax - 1) / qmax, std::min(rp.nsrc, 32)), 2);
    rp.q = (rp.nsrc + rp.chunk - 1) / rp.chunk;
    rp.ok = true;
    return rp;
}

// The plan depends only on settings that change between calls, so it is kept
// with the key it was made for (no device queries on every pp_step).
ResidentPlan resident_plan(pp_ctx *c, bool automatic)
{
    const int64_t key[6] = {c->acc, c->positions, c->wts != nullptr, c->variant_override,
                            automatic, c->device};
    if (c->res_plan_valid && std::equal(key, key + 6, c->res_plan_key)) {
        ResidentPlan rp;
        std::memcpy(&rp, c->res_plan, sizeof(rp));
        return rp;
    }
    const ResidentPlan rp = compute_resident_plan(c, automatic);
    static_assert(sizeof(ResidentPlan) <= sizeof(c->res_plan), "plan cache too small");
    std::memcpy(c->res_plan, &rp, sizeof(rp));
    std::copy(key, key + 6, c->res_plan_key);
    c->res_plan_valid = true;
    return rp;
}

pp_status step_resident(pp_ctx *c, const ResidentPlan &rp, int64_t nsteps)
{
    Plan pl{};
    pl.nib = 1;
    pl.nsplit = 1;
    ForceArgs a = base_args(c, pl, MODE_STEP, nullptr, nullptr, nullptr);
    a.skip_copy = c->skip_copy;
    c->skip_copy = 0;
    ResidentArgs ra{};
    ra.stage[0] = c->stage[0];
    ra.stage[1] = c->stage[1];
    ra.bt = rp.bt;
    ra.q = rp.q;
    ra.chunk = rp.chunk;
    ra.nsrc = rp.nsrc;
    ra.flags = c->res_flags;
    for (int64_t left = nsteps; left > 0;) {
        const int k = (int)std::min(left, kResidentMaxSteps);
        ra.parity0 = c->parity;
        ra.nsteps = k;
        PP_CUDA(cudaMemsetAsync(ra.flags, 0, sizeof(unsigned), c->stream));
        PP_CUDA(launch_resident(a, ra, rp.grid, rp.threads, rp.form, c->stream));
        a.skip_copy = 0;
        c->parity ^= (k & 1);
        left -= k;
    }
    return PP_OK;
}

// Fields of the current positions with positions mode `mode` into out (device).
pp_status fields_with(pp_ctx *c, int mode, double *out)
{
    c->positions = mode;
    void *scratch = c->stage[c->parity ^ 1];
    pp_status st = stage_current(c, scratch, stage_kind(c));
    if (st == PP_OK) st = force_pass(c, MODE_FIELDS, scratch, nullptr, out);
    return st;
}

// Relative L2 difference |a - b| / |b| of two device [n][3] arrays.
pp_status rel_diff(pp_ctx *c, const double *a, const double *b, double *parts, double *rel)
{
    double h[2 * kDiffBlocks];
    PP_CUDA(launch_diff_norms(a, b, (int)(3 * c->n), parts, c->stream));
    PP_CUDA(cudaMemcpyAsync(h, parts, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    PP_CUDA(cudaStreamSynchronize(c->stream));
    double d2 = 0.0, b2 = 0.0;
    for (int k = 0; k < kDiffBlocks; ++k) {
        d2 += h[2 * k];
        b2 += h[2 * k + 1];
    }
    *rel = b2 > 0 ? std::sqrt(d2 / b2) : 0.0;
    return PP_OK;
}

// PP_POS_AUTO: the fastest staging whose fields at the current positions agree with
// those of hi/lo staging (about 1e-7 of the FP64 result) within 5e-6 in relative L2,
// half the 1e-5 field tolerance.  Preference order: single staging (fastest; runs on
// the resident small-N kernel); hi/lo staging where the resident kernel can run it
// (small N, where steps are latency-bound and resident stepping wins); guarded
// staging (the single-staging loop with close-pair tiles summed on hi/lo parts);
// hi/lo staging.
pp_status decide_positions(pp_ctx *c)
{
    if (f64_pairs(c)) return PP_OK;   // FP64 sources: nothing to choose
    const size_t bytes = (size_t)c->n * 3 * sizeof(double);
    double *e_split = nullptr, *parts = nullptr;
    if (cudaMalloc(&e_split, bytes) != cudaSuccess ||
        cudaMalloc(&parts, 2 * kDiffBlocks * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(e_split);
        return fail(PP_ERR_NOMEM, "cannot allocate the positions-mode check");
    }
    constexpr double kAutoTol = 5e-6;
    c->auto_rel_single = c->auto_rel_guarded = NAN;
    int chosen = PP_POS_SPLIT;
    pp_status st = fields_with(c, PP_POS_SPLIT, e_split);
    if (st == PP_OK) st = fields_with(c, PP_POS_SINGLE, c->aos);
    if (st == PP_OK) st = rel_diff(c, c->aos, e_split, parts, &c->auto_rel_single);
    if (st == PP_OK && !(c->auto_rel_single <= kAutoTol)) {
        c->positions = PP_POS_SPLIT;
        const bool resident_split =
            c->resident != PP_RESIDENT_OFF && compute_resident_plan(c, true).ok;
        if (!resident_split) {
            st = fields_with(c, PP_POS_GUARDED, c->aos);
            if (st == PP_OK) st = rel_diff(c, c->aos, e_split, parts, &c->auto_rel_guarded);
            if (st == PP_OK && c->auto_rel_guarded <= kAutoTol) chosen = PP_POS_GUARDED;
        }
    } else if (st == PP_OK) {
        chosen = PP_POS_SINGLE;
    }
    cudaFree(e_split);
    cudaFree(parts);
    if (st == PP_OK) st = check_device_errors(c, true);
    c->positions = st == PP_OK ? chosen : PP_POS_SINGLE;
    drop_graphs(c);
    return st;
}

}  // namespace

extern "C" {

const char *pp_version(void) { return "pp-gb300 0.1 (sm_103a)"; }

const char *pp_last_error(const pp_ctx *) { return g_last_error.c_str(); }

double pp_pairs_per_step(int64_t N) { return (double)N * (double)N; }

const char *pp_variant_name(int index)
{
    int count = 0;
    const Variant *vs = variants(&count);
    return (index >= 0 && index < count) ? vs[index].name : nullptr;
}

pp_status pp_staging_check(const pp_ctx *c, double *single_rel, double *guarded_rel)
{
    if (!c) return fail(PP_ERR_ARG, "null context");
    if (single_rel) *single_rel = c->auto_rel_single;
    if (guarded_rel) *guarded_rel = c->auto_rel_guarded;
    return PP_OK;
}

pp_status pp_get_n(const pp_ctx *c, int64_t *n)
{
    if (!c || !n) return fail(PP_ERR_ARG, "null argument");
    *n = c->n;
    return PP_OK;
}

pp_status pp_destroy(pp_ctx *c)
{
    if (!c) return PP_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    cudaFree(c->state);
    cudaFree(c->stage[0]);
    cudaFree(c->stage[1]);
    cudaFree(c->aos);
    cudaFree(c->phi);
    cudaFree(c->wts);
    cudaFree(c->wrel);
    cudaFree(c->partial);
    cudaFree(c->tickets);
    cudaFree(c->mom_partials);
    cudaFree(c->mom_out);
    cudaFree(c->err);
    cudaFree(c->res_flags);
    cudaFree(c->ord_ws);
    if (c->mom_host) cudaFreeHost(c->mom_host);
    if (c->err_host) cudaFreeHost(c->err_host);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
    return PP_OK;
}

pp_status pp_create(int64_t N, double w, double dt, double softening, pp_ctx **out)
{
    if (!out) return fail(PP_ERR_ARG, "out is null");
    *out = nullptr;
    if (N < 1 || N > (int64_t(1) << 28)) return fail(PP_ERR_ARG, "N must be in [1, 2^28]");
    if (!(std::isfinite(w) && w > 0)) return fail(PP_ERR_ARG, "w must be finite and > 0");
    if (!(std::isfinite(dt) && dt > 0)) return fail(PP_ERR_ARG, "dt must be finite and > 0");
    if (!(std::isfinite(softening) && softening >= 0))
        return fail(PP_ERR_ARG, "softening must be finite and >= 0");
    pp_ctx *c = new pp_ctx();
    c->n = N;
    c->npad = (int)round_up(N, kPad);
    c->w = w;
    c->dt = dt;
    c->eps = softening;
    auto bail = [&](pp_status s, const std::string &m) {
        pp_destroy(c);
        return fail(s, m);
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) return bail(PP_ERR_CUDA, "no CUDA device");
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess)
        return bail(PP_ERR_CUDA, "cudaGetDeviceProperties failed");
    c->sms = prop.multiProcessorCount;
    if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(PP_ERR_CUDA, "cudaStreamCreate failed");
    c->stream = c->own_stream;
    if (const char *env = std::getenv("PP_TIMEOUT_NS")) {   // default bound of device waits
        const long long t = std::atoll(env);
        if (t >= 1000 && t <= 60000000000ll) c->timeout_ns = (uint64_t)t;
    }
    const size_t np = (size_t)c->npad;
    c->stage_bytes = np * sizeof(double4);  // room for either staging type
    bool okm = cudaMalloc(&c->state, 9 * np * sizeof(double)) == cudaSuccess &&
               cudaMalloc(&c->stage[0], c->stage_bytes) == cudaSuccess &&
               cudaMalloc(&c->stage[1], c->stage_bytes) == cudaSuccess &&
               cudaMalloc(&c->aos, (size_t)N * 3 * sizeof(double)) == cudaSuccess &&
               cudaMalloc(&c->phi, np * sizeof(double)) == cudaSuccess &&
               cudaMalloc(&c->mom_partials, kMomBlocks * kMomSlots * sizeof(double)) == cudaSuccess &&
               cudaMalloc(&c->mom_out, kMomSlots * sizeof(double)) == cudaSuccess &&
               cudaMalloc(&c->err, 4 * sizeof(int)) == cudaSuccess &&
               cudaMalloc(&c->res_flags, kResidentMaxGrid * sizeof(unsigned)) == cudaSuccess &&
               cudaMallocHost(&c->mom_host, kMomSlots * sizeof(double)) == cudaSuccess &&
               cudaMallocHost(&c->err_host, 4 * sizeof(int)) == cudaSuccess;
    if (!okm) {
        cudaGetLastError();
        return bail(PP_ERR_NOMEM, "device allocation failed");
    }
    for (int k = 0; k < 3; ++k) {
        c->r[k] = c->state + (0 + k) * np;
        c->v[k] = c->state + (3 + k) * np;
        c->a[k] = c->state + (6 + k) * np;
    }
    if (cudaMemsetAsync(c->state, 0, 9 * np * sizeof(double), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->err, 0, 4 * sizeof(int), c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return bail(PP_ERR_CUDA, "initial memset failed");
    *out = c;
    return PP_OK;
}

pp_status pp_set_option(pp_ctx *c, int key, int64_t value)
{
    if (pp_status s = check_ctx(c)) return s;
    switch (key) {
    case PP_OPT_ACC:
    case PP_OPT_POSITIONS: {
        if (key == PP_OPT_ACC && (value < PP_ACC_FP64FOLD || value > PP_ACC_FP64_FULL))
            return fail(PP_ERR_ARG, "bad acc mode");
        if (key == PP_OPT_POSITIONS && value != PP_POS_SINGLE && value != PP_POS_SPLIT &&
            value != PP_POS_AUTO && value != PP_POS_GUARDED)
            return fail(PP_ERR_ARG, "bad positions mode");
        const int new_acc = key == PP_OPT_ACC ? (int)value : c->acc;
        const bool new_auto = key == PP_OPT_POSITIONS ? value == PP_POS_AUTO : c->positions_auto;
        const int new_pos = key == PP_OPT_POSITIONS ? (value == PP_POS_AUTO ? c->positions : (int)value)
                                                    : c->positions;
        if (c->wts && new_acc == PP_ACC_KAHAN)
            return fail(PP_ERR_ARG, "per-particle weights need PP_ACC_FP64FOLD or PP_ACC_FP64_FULL");
        c->positions_auto = new_auto;
        const int old_kind = stage_kind(c);
        c->acc = new_acc;
        c->positions = new_pos;
        drop_graphs(c);
        if (c->loaded && old_kind != stage_kind(c)) {
            // the pending r_{n+1} is staged in the old layout: restage it
            PP_CUDA(cudaSetDevice(c->device));
            return restage_pending(c);
        }
        return PP_OK;
    }
    case PP_OPT_STREAM:
        drop_graphs(c);
        c->stream = value ? reinterpret_cast<cudaStream_t>(value) : c->own_stream;
        return PP_OK;
    case PP_OPT_SPLIT:
        if (value < 0 || value > 4096) return fail(PP_ERR_ARG, "split must be in [0, 4096]");
        c->split_override = (int)value;
        drop_graphs(c);
        return PP_OK;
    case PP_OPT_GRAPH_BLOCK:
        if (value < 0 || value > 4096) return fail(PP_ERR_ARG, "graph block must be in [0, 4096]");
        c->graph_block = (int)value;
        drop_graphs(c);
        return PP_OK;
    case PP_OPT_TIMEOUT_NS:
        if (value < 1000 || value > 60000000000ll) return fail(PP_ERR_ARG, "timeout out of range");
        c->timeout_ns = (uint64_t)value;
        drop_graphs(c);
        return PP_OK;
    case PP_OPT_VARIANT: {
        int count = 0;
        variants(&count);
        if (value < -1 || value >= count) return fail(PP_ERR_ARG, "no such variant");
        const int old_kind = stage_kind(c);
        c->variant_override = (int)value;
        drop_graphs(c);
        if (c->loaded && old_kind != stage_kind(c)) {
            PP_CUDA(cudaSetDevice(c->device));
            return restage_pending(c);
        }
        return PP_OK;
    }
    case PP_OPT_TEST_SKIP_COPY:
        c->skip_copy = value ? 1 : 0;
        return PP_OK;
    case PP_OPT_RESIDENT:
        if (value < PP_RESIDENT_OFF || value > PP_RESIDENT_ON)
            return fail(PP_ERR_ARG, "bad resident mode");
        c->resident = (int)value;
        return PP_OK;
    default:
        return fail(PP_ERR_ARG, "unknown option key");
    }
}

pp_status pp_get_option(const pp_ctx *c, int key, int64_t *value)
{
    if (!c || !value) return fail(PP_ERR_ARG, "null argument");
    switch (key) {
    case PP_OPT_ACC: *value = c->acc; return PP_OK;
    case PP_OPT_POSITIONS: *value = c->positions; return PP_OK;
    case PP_OPT_POSITIONS_AUTO: *value = c->positions_auto ? 1 : 0; return PP_OK;
    case PP_OPT_STREAM: *value = (int64_t)reinterpret_cast<intptr_t>(c->stream); return PP_OK;
    case PP_OPT_SPLIT: *value = c->split_override; return PP_OK;
    case PP_OPT_GRAPH_BLOCK: *value = c->graph_block; return PP_OK;
    case PP_OPT_TIMEOUT_NS: *value = (int64_t)c->timeout_ns; return PP_OK;
    case PP_OPT_RESIDENT: *value = c->resident; return PP_OK;
    case PP_OPT_RESIDENT_ACTIVE:
        *value = (c->resident != PP_RESIDENT_OFF &&
                  compute_resident_plan(c, c->resident == PP_RESIDENT_AUTO).ok) ? 1 : 0;
        return PP_OK;
    case PP_OPT_VARIANT: {
        int count = 0;
        const Variant *vs = variants(&count);
        *value = (int64_t)(force_variant(c) - vs);
        return PP_OK;
    }
    case PP_OPT_LAUNCHES_PER_PASS: {
        const Variant *v = force_variant(c);
        *value = 1 + (v->order ? order_launches(c->npad) : 0);
        return PP_OK;
    }
    default: return fail(PP_ERR_ARG, "unknown option key");
    }
}

pp_status pp_load_particles(pp_ctx *c, const double *pos, const double *vel, int on_device)
{
    NvtxRange nvtx_("pp_load_particles");
    if (pp_status s = check_ctx(c)) return s;
    if (!pos) return fail(PP_ERR_ARG, "pos is null");
    if (!valid_mem(on_device)) return fail(PP_ERR_ARG, "bad memory kind");
    PP_CUDA(cudaSetDevice(c->device));
    drop_graphs(c);
    c->loaded = false;
    pp_status st = import_aos(c, pos, on_device, c->r);
    if (st != PP_OK) return st;
    if (vel) {
        st = import_aos(c, vel, on_device, c->v);
        if (st != PP_OK) return st;
    } else {
        for (int k = 0; k < 3; ++k)
            PP_CUDA(cudaMemsetAsync(c->v[k], 0, c->npad * sizeof(double), c->stream));
    }
    bool bad = false;
    st = take_bad_input_flag(c, &bad);
    if (st != PP_OK) return st;
    if (bad) return fail(PP_ERR_ARG, "non-finite position or velocity");
    st = choose_frame(c);
    if (st != PP_OK) return st;
    if (c->positions_auto) {
        st = pad_both(c);
        if (st == PP_OK) st = decide_positions(c);
        if (st != PP_OK) return st;
    }
    // a_0 = F(r_0) (needed by the first Eq. G); the epilogue stages r_1.
    c->parity = 0;
    st = pad_both(c);
    if (st != PP_OK) return st;
    st = stage_current(c, c->stage[1], stage_kind(c));
    if (st != PP_OK) return st;
    st = force_pass(c, MODE_INIT, c->stage[1], c->stage[0], nullptr);
    if (st != PP_OK) return st;
    st = check_device_errors(c, true);
    if (st != PP_OK) return st;
    c->loaded = true;
    c->step = 0;
    return PP_OK;
}

pp_status pp_set_weights(pp_ctx *c, const double *w, int on_device)
{
    if (pp_status s = check_ctx(c)) return s;
    PP_CUDA(cudaSetDevice(c->device));
    if (!valid_mem(on_device)) return fail(PP_ERR_ARG, "bad memory kind");
    if (c->acc == PP_ACC_KAHAN)
        return fail(PP_ERR_ARG, "per-particle weights need PP_ACC_FP64FOLD or PP_ACC_FP64_FULL");
    if (!w) {
        cudaFree(c->wts);
        cudaFree(c->wrel);
        c->wts = nullptr;
        c->wrel = nullptr;
    } else {
        if (!c->wts) {
            if (cudaMalloc(&c->wts, (size_t)c->npad * sizeof(double)) != cudaSuccess ||
                cudaMalloc(&c->wrel, (size_t)c->npad * sizeof(float)) != cudaSuccess) {
                cudaGetLastError();
                cudaFree(c->wts);
                cudaFree(c->wrel);
                c->wts = nullptr;
                c->wrel = nullptr;
                return fail(PP_ERR_NOMEM, "cannot allocate the weight arrays");
            }
        }
        const size_t bytes = (size_t)c->n * sizeof(double);
        PP_CUDA(cudaMemcpyAsync(c->wts, w, bytes, on_device == PP_MEM_DEVICE
                                                      ? cudaMemcpyDeviceToDevice
                                                      : cudaMemcpyHostToDevice, c->stream));
        int bad = 0;
        PP_CUDA(cudaMemsetAsync(c->err + 1, 0, sizeof(int), c->stream));
        PP_CUDA(launch_weights(c->wts, (int)c->n, c->w, c->wrel, c->err + 1, c->stream));
        PP_CUDA(cudaMemcpyAsync(&bad, c->err + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        PP_CUDA(cudaStreamSynchronize(c->stream));
        if (bad) {
            PP_CUDA(cudaMemsetAsync(c->err + 1, 0, sizeof(int), c->stream));
            cudaFree(c->wts);
            cudaFree(c->wrel);
            c->wts = nullptr;
            c->wrel = nullptr;
            return fail(PP_ERR_ARG, "weights must be finite and > 0");
        }
    }
    drop_graphs(c);
    if (!c->loaded) return PP_OK;
    // the acceleration belongs to the weights: recompute a(r) and restage r_{n+1}
    // (PP_POS_AUTO first decides the staging again for the weighted sum)
    pp_status st = PP_OK;
    if (c->positions_auto) {
        st = pad_both(c);
        if (st == PP_OK) st = decide_positions(c);
        if (st != PP_OK) return st;
    }
    st = pad_both(c);
    if (st == PP_OK) st = stage_current(c, c->stage[c->parity ^ 1], stage_kind(c));
    if (st == PP_OK)
        st = force_pass(c, MODE_INIT, c->stage[c->parity ^ 1], c->stage[c->parity], nullptr);
    if (st == PP_OK) st = check_device_errors(c, true);
    return st;
}

pp_status pp_set_state(pp_ctx *c, const double *pos, const double *vel, const double *acc,
                       int64_t step, const double *frame, int on_device)
{
    NvtxRange nvtx_("pp_set_state");
    if (pp_status s = check_ctx(c)) return s;
    if (!pos || !vel || !acc) return fail(PP_ERR_ARG, "pos, vel and acc are required");
    if (!valid_mem(on_device)) return fail(PP_ERR_ARG, "bad memory kind");
    if (frame) {
        if (!(std::isfinite(frame[0]) && std::isfinite(frame[1]) && std::isfinite(frame[2]) &&
              std::isfinite(frame[3]) && frame[3] > 0))
            return fail(PP_ERR_ARG, "invalid staging frame");
        int e = 0;
        if (std::frexp(frame[3], &e) != 0.5) return fail(PP_ERR_ARG, "frame scale must be a power of two");
        if (frame[4] != (double)PP_POS_SINGLE && frame[4] != (double)PP_POS_SPLIT &&
            frame[4] != (double)PP_POS_GUARDED)
            return fail(PP_ERR_ARG, "frame staging must be PP_POS_SINGLE, _SPLIT or _GUARDED");
    }
    PP_CUDA(cudaSetDevice(c->device));
    drop_graphs(c);
    c->loaded = false;
    bool bad = false;
    // PP_POS_AUTO resumes with the staging the saved run used (bitwise resume); an
    // explicit positions mode of this context is kept as it is
    if (frame && c->positions_auto && !f64_pairs(c)) c->positions = (int)frame[4];
    if (frame && on_device != PP_MEM_HOST) {
        // device or mapped host buffers: one pass converts the state, checks it and
        // stages r_{n+1} = Eq. G(r_n, v_n, a_n); one synchronisation
        const size_t bytes = (size_t)c->n * 3 * sizeof(double);
        const double *src[3] = {pos, vel, acc};
        if (on_device == PP_MEM_HOST_MAPPED) {
            for (auto &q : src) {
                const void *d = nullptr;
                if (pp_status st = mapped_view(q, bytes, &d)) return st;
                q = static_cast<const double *>(d);
            }
        }
        c->cx = frame[0];
        c->cy = frame[1];
        c->cz = frame[2];
        c->l0 = frame[3];
        c->parity = 0;
        PP_CUDA(launch_fill_padding(c->stage[1], (int)c->n, c->npad, stage_kind(c), c->stream));
        PP_CUDA(launch_import_state(src[0], src[1], src[2], (int)c->n, c->npad, c->r, c->v, c->a,
                                    c->stage[0], stage_kind(c), c->dt, c->dt * c->dt / 2.0, c->cx,
                                    c->cy, c->cz, 1.0 / c->l0, c->wrel, c->err + 1, c->stream));
        pp_status st = take_bad_input_flag(c, &bad);
        if (st != PP_OK) return st;
        if (bad) return fail(PP_ERR_ARG, "non-finite state");
        c->loaded = true;
        c->step = step;
        return PP_OK;
    }
    pp_status st = import_aos(c, pos, on_device, c->r);
    if (st == PP_OK) st = import_aos(c, vel, on_device, c->v);
    if (st == PP_OK) st = import_aos(c, acc, on_device, c->a);
    if (st != PP_OK) return st;
    if (frame) {
        // the frame is given: stage r_{n+1} = Eq. G(r_n, v_n, a_n) exactly as the
        // step epilogue would, and check the input with the same synchronisation
        c->cx = frame[0];
        c->cy = frame[1];
        c->cz = frame[2];
        c->l0 = frame[3];
        c->parity = 0;
        st = restage_pending(c, false);
        if (st == PP_OK) st = take_bad_input_flag(c, &bad);
        if (st != PP_OK) return st;
        if (bad) return fail(PP_ERR_ARG, "non-finite state");
    } else {
        st = take_bad_input_flag(c, &bad);
        if (st != PP_OK) return st;
        if (bad) return fail(PP_ERR_ARG, "non-finite state");
        st = choose_frame(c);
        if (st != PP_OK) return st;
        c->parity = 0;
        if (c->positions_auto) {   // a fresh frame: decide the staging for these positions
            st = pad_both(c);
            if (st == PP_OK) st = decide_positions(c);
            if (st != PP_OK) return st;
        }
        st = restage_pending(c);
        if (st != PP_OK) return st;
    }
    c->loaded = true;
    c->step = step;
    return PP_OK;
}

pp_status pp_check_mapped(const void *p, int64_t bytes)
{
    if (bytes <= 0) return fail(PP_ERR_ARG, "bytes must be > 0");
    const void *d = nullptr;
    return mapped_view(p, (size_t)bytes, &d);
}

pp_status pp_get_state(pp_ctx *c, double *pos, double *vel, double *acc, int64_t *step,
                       double *frame, int on_device)
{
    NvtxRange nvtx_("pp_get_state");
    if (pp_status s = check_ctx(c)) return s;
    if (!valid_mem(on_device)) return fail(PP_ERR_ARG, "bad memory kind");
    if (!c->loaded) return fail(PP_ERR_STATE, "no particles loaded");
    PP_CUDA(cudaSetDevice(c->device));
    pp_status st;
    if (on_device != PP_MEM_HOST) {
        // device or mapped host buffers: one pass writes all requested arrays
        const size_t bytes = (size_t)c->n * 3 * sizeof(double);
        double *dst[3] = {pos, vel, acc};
        if (on_device == PP_MEM_HOST_MAPPED) {
            for (auto &q : dst) {
                if (!q) continue;
                const void *d = nullptr;
                if ((st = mapped_view(q, bytes, &d)) != PP_OK) return st;
                q = static_cast<double *>(const_cast<void *>(d));
            }
        }
        if (dst[0] || dst[1] || dst[2])
            PP_CUDA(launch_export_state(c->r, c->v, c->a, (int)c->n, dst[0], dst[1], dst[2],
                                        c->stream));
    } else {
        if (pos && (st = export_aos(c, c->r, pos, on_device)) != PP_OK) return st;
        if (vel && (st = export_aos(c, c->v, vel, on_device)) != PP_OK) return st;
        if (acc && (st = export_aos(c, c->a, acc, on_device)) != PP_OK) return st;
    }
    if (step) *step = c->step;
    if (frame) {
        frame[0] = c->cx;
        frame[1] = c->cy;
        frame[2] = c->cz;
        frame[3] = c->l0;
        frame[4] = (double)c->positions;
    }
    PP_CUDA(cudaStreamSynchronize(c->stream));
    return PP_OK;
}

pp_status pp_get_particles(pp_ctx *c, double *pos, double *vel, int on_device)
{
    return pp_get_state(c, pos, vel, nullptr, nullptr, nullptr, on_device);
}

pp_status pp_compute_fields(pp_ctx *c, double *E_out, int on_device)
{
    NvtxRange nvtx_("pp_compute_fields");
    if (pp_status s = check_ctx(c)) return s;
    if (!E_out) return fail(PP_ERR_ARG, "E_out is null");
    if (!valid_mem(on_device)) return fail(PP_ERR_ARG, "bad memory kind");
    if (!c->loaded) return fail(PP_ERR_STATE, "no particles loaded");
    PP_CUDA(cudaSetDevice(c->device));
    double *target = E_out;
    if (on_device == PP_MEM_HOST) {
        target = c->aos;
    } else if (on_device == PP_MEM_HOST_MAPPED) {
        const void *d = nullptr;
        if (pp_status st = mapped_view(E_out, (size_t)c->n * 3 * sizeof(double), &d)) return st;
        target = static_cast<double *>(const_cast<void *>(d));
    }
    // stage the current r_n into the idle buffer; the pending r_{n+1} stays put
    void *scratch = c->stage[c->parity ^ 1];
    pp_status st = stage_current(c, scratch, stage_kind(c));
    if (st != PP_OK) return st;
    st = force_pass(c, MODE_FIELDS, scratch, nullptr, target);
    if (st != PP_OK) return st;
    if (on_device == PP_MEM_HOST)
        PP_CUDA(cudaMemcpyAsync(E_out, c->aos, (size_t)c->n * 3 * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
    return check_device_errors(c, false);
}

pp_status pp_step(pp_ctx *c, int64_t nsteps)
{
    NvtxRange nvtx_("pp_step");
    if (pp_status s = check_ctx(c)) return s;
    if (nsteps < 0) return fail(PP_ERR_ARG, "nsteps must be >= 0");
    if (!c->loaded) return fail(PP_ERR_STATE, "no particles loaded");
    PP_CUDA(cudaSetDevice(c->device));
    int64_t left = nsteps;
    if (c->resident != PP_RESIDENT_OFF && nsteps > 0) {
        const ResidentPlan rp = resident_plan(c, c->resident == PP_RESIDENT_AUTO);
        if (rp.ok) {
            pp_status st = step_resident(c, rp, nsteps);
            if (st == PP_OK) st = check_device_errors(c, true);
            if (st != PP_OK) return st;
            c->step += nsteps;
            return PP_OK;
        }
    }
    if (graph_capturable(c) && !c->skip_copy && left >= c->graph_block) {
        if (c->graph_steps != c->graph_block || !c->graph[0]) {
            pp_status st = build_graphs(c);
            if (st != PP_OK) return st;
        }
        while (left >= c->graph_steps) {
            PP_CUDA(cudaGraphLaunch(c->graph[c->parity], c->stream));
            c->parity ^= (c->graph_steps & 1);
            left -= c->graph_steps;
        }
    }
    for (; left > 0; --left) {
        pp_status st = force_pass(c, MODE_STEP, c->stage[c->parity], c->stage[c->parity ^ 1], nullptr);
        if (st != PP_OK) return st;
        c->parity ^= 1;
    }
    pp_status st = check_device_errors(c, true);
    if (st != PP_OK) return st;
    c->step += nsteps;
    return PP_OK;
}

pp_status pp_autotune(pp_ctx *c, pp_tune_result *out)
{
    NvtxRange nvtx_("pp_autotune");
    if (pp_status s = check_ctx(c)) return s;
    if (!c->loaded) return fail(PP_ERR_STATE, "no particles loaded");
    PP_CUDA(cudaSetDevice(c->device));
    int count = 0;
    const Variant *vs = variants(&count);
    const int saved_variant = c->variant_override, saved_split = c->split_override;
    const int old_kind = stage_kind(c);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PP_CUDA(cudaEventCreate(&e0));
    PP_CUDA(cudaEventCreate(&e1));
    void *scratch = c->stage[c->parity ^ 1];
    int best_v = -1, best_s = 0, tried = 0;
    double best_ms = 1e300;
    pp_status st = PP_OK;
    // where steps run on the resident small-N kernel, only variants with its staging
    // layout are candidates, so that the choice does not take the steps off it
    const bool keep_resident = c->resident != PP_RESIDENT_OFF &&
                               compute_resident_plan(c, c->resident == PP_RESIDENT_AUTO).ok;
    for (int v = 0; v < count && st == PP_OK; ++v) {
        if (vs[v].kind != (c->wts ? KIND_FORCE32W : KIND_FORCE32) || vs[v].acc != c->acc ||
            vs[v].positions != c->positions)
            continue;
        if (keep_resident &&
            vs[v].stage != (c->positions == PP_POS_SPLIT ? STAGE_F32IX2 : STAGE_F32I))
            continue;
        if (vs[v].cluster > 0 && !cluster_fits(vs[v])) continue;   // cannot launch here
        c->variant_override = v;
        c->split_override = 0;
        const Plan base = make_plan(c, vs[v].kind);
        const int tiles = c->npad / vs[v].tile;
        int cand[4] = {base.nsplit, std::max(1, base.nsplit / 2), std::min(tiles, 2 * base.nsplit),
                       std::max(1, base.nsplit / 4)};
        st = stage_current(c, scratch, vs[v].stage);
        const int ncand = vs[v].cluster > 0 ? 1 : 4;   // a cluster fixes the split
        for (int k = 0; k < ncand && st == PP_OK; ++k) {
            bool dup = false;
            for (int q = 0; q < k; ++q) dup |= cand[q] == cand[k];
            if (dup) continue;
            c->split_override = cand[k];
            // one untimed pass, one pass to size the measurement, then the timed passes
            st = force_pass(c, MODE_FIELDS, scratch, nullptr, c->aos);
            if (st != PP_OK) break;
            PP_CUDA(cudaEventRecord(e0, c->stream));
            st = force_pass(c, MODE_FIELDS, scratch, nullptr, c->aos);
            PP_CUDA(cudaEventRecord(e1, c->stream));
            PP_CUDA(cudaEventSynchronize(e1));
            float first = 0.f;
            PP_CUDA(cudaEventElapsedTime(&first, e0, e1));
            // about 20 ms of timed passes per candidate (3 to 50 passes)
            const int reps = std::max(3, std::min(50, (int)(20.0 / std::max(first, 1e-3f))));
            PP_CUDA(cudaEventRecord(e0, c->stream));
            for (int r = 0; r < reps && st == PP_OK; ++r)
                st = force_pass(c, MODE_FIELDS, scratch, nullptr, c->aos);
            PP_CUDA(cudaEventRecord(e1, c->stream));
            PP_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            PP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            const double per = ms / reps;
            ++tried;
            if (per < best_ms) {
                best_ms = per;
                best_v = v;
                best_s = cand[k];
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == PP_OK) st = check_device_errors(c, false);
    if (st != PP_OK || best_v < 0) {
        c->variant_override = saved_variant;
        c->split_override = saved_split;
        return st != PP_OK ? st : fail(PP_ERR_STATE, "no variant fits the context's modes");
    }
    c->variant_override = best_v;
    c->split_override = best_s;
    drop_graphs(c);
    if (old_kind != stage_kind(c)) {
        st = restage_pending(c);
        if (st != PP_OK) return st;
    }
    if (out) {
        out->variant = best_v;
        out->split = best_s;
        out->ms_per_pass = best_ms;
        out->candidates = tried;
    }
    return PP_OK;
}

pp_status pp_diagnostics(pp_ctx *c, pp_diag *d, int with_pe)
{
    NvtxRange nvtx_("pp_diagnostics");
    if (pp_status s = check_ctx(c)) return s;
    if (!d) return fail(PP_ERR_ARG, "out is null");
    if (!c->loaded) return fail(PP_ERR_STATE, "no particles loaded");
    PP_CUDA(cudaSetDevice(c->device));
    const double n = (double)c->n;
    double m0[kMomSlots], m1[kMomSlots];
    const double scx = c->cx, scy = c->cy, scz = c->cz;
    c->cx = c->cy = c->cz = 0.0;
    pp_status st = moments(c, 0, nullptr, m0);
    if (st != PP_OK) return st;
    const double cx = m0[0] / n, cy = m0[1] / n, cz = m0[2] / n;
    c->cx = cx;
    c->cy = cy;
    c->cz = cz;
    st = moments(c, 1, nullptr, m1);
    c->cx = scx;
    c->cy = scy;
    c->cz = scz;
    if (st != PP_OK) return st;
    // with per-particle weights the moment sums already carry w_i
    const double mw = c->wts ? kMe : kMe * c->w;
    d->t = (double)c->step * c->dt;
    d->step = c->step;
    d->rms_radius = std::sqrt(m1[0] / n);
    d->ke = 0.5 * mw * m1[1];
    d->px = mw * m1[2];
    d->py = mw * m1[3];
    d->pz = mw * m1[4];
    const double x2 = m1[5] / n, vx2 = m1[6] / n, xvx = m1[7] / n;
    const double e2 = x2 * vx2 - xvx * xvx;
    d->emit_x = std::sqrt(e2 > 0 ? e2 : 0.0);
    d->x_rms = std::sqrt(x2);
    d->x_max = m1[10];
    d->vx_rms = std::sqrt(vx2);
    d->vx_max = m1[11];
    d->cx = cx;
    d->cy = cy;
    d->cz = cz;
    d->pe = NAN;
    if (with_pe) {
        // phi'_i = sum_{j != i} 1/sqrt(|d'|^2 + eps'^2); PE = 1/2 k e^2 w^2 / L0 * sum_i phi'_i
        // the potential pass always uses FP32 sources, staged into the idle buffer
        void *scratch = c->stage[c->parity ^ 1];
        st = stage_current(c, scratch, STAGE_F32);
        if (st == PP_OK) st = force_pass(c, MODE_PHI, scratch, nullptr, c->phi);
        if (st != PP_OK) return st;
        st = check_device_errors(c, false);
        if (st != PP_OK) return st;
        double mp[kMomSlots];
        st = moments(c, 2, c->phi, mp);
        if (st != PP_OK) return st;
        // sum_i w_i phi'_i (weights) or sum_i phi'_i (equal weights, times w)
        d->pe = 0.5 * kCoulomb * kE * kE * c->w / c->l0 * mp[0] * (c->wts ? 1.0 : c->w);
    }
    return PP_OK;
}

}  // extern "C"
