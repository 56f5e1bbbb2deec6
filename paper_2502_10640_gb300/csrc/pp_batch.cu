// pp_batch.cu -- batch context: many independent bunches stepped together by
// one persistent kernel launch per time step, admitted against a device-memory
// budget, with CUDA-graph step blocks.  C ABI in include/pp.h (pp_batch_*).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pp.h"
#include "pp_batch.cuh"
#include "pp_internal.h"

using namespace ppk;

namespace {

constexpr int kMaxBunches = 4096;

pp_status bfail(pp_status s, const std::string &m)
{
    set_last_error(m.c_str());
    return s;
}

pp_status bcuda(cudaError_t e, const char *where)
{
    return bfail(PP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define B_CUDA(call)                                       \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return bcuda(e_, #call);    \
    } while (0)

// Tiling of one bunch: a function of its N and of its staging only.
struct Layout {
    int npad, nib, nipad, nsplit, jchunk;
};

Layout layout_for(int64_t n, int staging)
{
    Layout L{};
    const int bi = batch_block(staging);
    L.npad = (int)((n + kPad - 1) / kPad * kPad);
    L.nib = (int)((n + bi - 1) / bi);
    L.nipad = L.nib * bi;
    L.jchunk = kBatchJChunk;
    L.nsplit = (L.npad + L.jchunk - 1) / L.jchunk;
    return L;
}

// Device memory of one bunch, laid out to hold either staging (so the footprint
// is a function of N only): state, two staging buffers of 32 bytes per source
// (hi/lo), partial sums and tickets for the larger of the two tilings, and an
// [N][3] transfer buffer.
struct Footprint {
    size_t state_bytes, stage_bytes, partial_bytes, ticket_bytes, aos_bytes, total;
};

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

Footprint footprint_for(int64_t n)
{
    const Layout a = layout_for(n, POS_SINGLE), b = layout_for(n, POS_SPLIT);
    Footprint F{};
    F.state_bytes = (size_t)9 * a.npad * sizeof(double);
    F.stage_bytes = (size_t)2 * a.npad * sizeof(float4);
    const size_t nipad = (size_t)std::max(a.nipad, b.nipad);
    F.partial_bytes = a.nsplit > 1 ? (size_t)a.nsplit * 3 * nipad * sizeof(double) : 0;
    F.ticket_bytes = (size_t)std::max(a.nib, b.nib) * sizeof(unsigned);
    F.aos_bytes = (size_t)3 * n * sizeof(double);
    F.total = al256(F.state_bytes) + 2 * al256(F.stage_bytes) + al256(F.partial_bytes) +
              al256(F.ticket_bytes) + al256(F.aos_bytes);
    return F;
}

struct Slot {
    bool active = false;
    int64_t n = 0;
    double w = 1, dt = 0, eps = 0;
    int staging = POS_SINGLE;      // POS_SINGLE, POS_SPLIT or POS_GUARDED (set at pp_batch_add)
    Layout L{};
    Footprint F{};
    unsigned char *mem = nullptr;  // one allocation holding everything below
    double *r[3] = {}, *v[3] = {}, *a[3] = {};
    void *stage[2] = {};
    double *partial = nullptr;
    unsigned *tickets = nullptr;
    double *aos = nullptr;         // [n][3] transfer scratch
    int parity = 0;
    int64_t step = 0;
    double cx = 0, cy = 0, cz = 0, l0 = 1;
};

// Compiled shapes of the batch kernel (see pp_batch.cuh: all give bitwise the
// same results).  The first is the default.
struct Shape {
    const char *name;
    const void *fn;
    int threads;
};

template <int T, int MINB, int UNROLL>
Shape make_shape(const char *name)
{
    return Shape{name,
                 reinterpret_cast<const void *>(
                     &batch_f32x2_kernel<T, kBatchTile, kBatchStages, MINB, UNROLL>),
                 T};
}

const Shape kShapes[] = {
    make_shape<128, 4, 2>("t128m4u2"),
    make_shape<128, 4, 1>("t128m4u1"),
    make_shape<128, 3, 2>("t128m3u2"),
    make_shape<256, 2, 1>("t256m2u1"),
    make_shape<256, 2, 2>("t256m2u2"),
};
constexpr int kNumShapes = (int)(sizeof(kShapes) / sizeof(kShapes[0]));

size_t batch_smem()
{
    return (size_t)kBatchStages * kBatchTile * sizeof(float4) +
           (size_t)3 * kBatchBIMax * sizeof(double);
}

}  // namespace

struct pp_batch {
    int device = 0;
    int sms = 0;
    int shape = 0;                    // index into kShapes
    int grid = 0;                     // persistent CTAs of that shape
    int positions = PP_POS_AUTO;      // staging of bunches added from now on
    cudaStream_t own_stream = nullptr, stream = nullptr;
    int64_t budget = 0, used = 0;
    std::vector<Slot> slots;
    BunchDesc *d_descs = nullptr;     // [kMaxBunches]
    BatchHeader *d_hdr = nullptr;
    BunchDesc *d_init_desc = nullptr; // one bunch, for its own passes at pp_batch_add
    BatchHeader *d_init_hdr = nullptr;
    unsigned *d_queue = nullptr;
    int *d_err = nullptr;             // [0] wait ran out, [1] non-finite input
    double *mom_partials = nullptr, *mom_out = nullptr, *mom_host = nullptr;
    int *err_host = nullptr;          // pinned copy of the error word
    bool dirty = true;
    int graph_block = 16;
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    uint64_t timeout_ns = 1000000000ull;
    int skip_copy = 0;                // test hook for the next launch (PP_OPT_TEST_SKIP_COPY)
    std::vector<int> order;           // active slots in table order
};

namespace {

void drop_graph(pp_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_steps = 0;
}

// Make shape k the batch's kernel: shared-memory attribute and persistent grid
// (one CTA per resident slot on every SM).
pp_status select_shape(pp_batch *b, int k)
{
    const Shape &sh = kShapes[k];
    B_CUDA(cudaFuncSetAttribute(sh.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)batch_smem()));
    int occ = 0;
    B_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, sh.fn, sh.threads, batch_smem()));
    if (occ < 1) return bfail(PP_ERR_CUDA, "batch kernel does not fit on an SM");
    b->shape = k;
    b->grid = b->sms * occ;
    drop_graph(b);
    return PP_OK;
}

BunchDesc make_desc(const Slot &s, int mode, int parity0, int item_base, double *out = nullptr)
{
    BunchDesc d{};
    d.stage[0] = s.stage[0];
    d.stage[1] = s.stage[1];
    for (int c = 0; c < 3; ++c) {
        d.r[c] = s.r[c];
        d.v[c] = s.v[c];
        d.a[c] = s.a[c];
    }
    d.partial = s.partial;
    d.tickets = s.tickets;
    d.out = out;
    d.n = (int)s.n;
    d.npad = s.L.npad;
    d.nib = s.L.nib;
    d.nsplit = s.L.nsplit;
    d.jchunk = s.L.jchunk;
    d.nipad = s.L.nipad;
    d.item_base = item_base;
    d.parity0 = parity0;
    d.mode = mode;
    d.staging = s.staging;
    const double epsl = s.eps / s.l0;
    d.eps2f = (float)(epsl * epsl);
    // a = k e^2 w / (m_e L0^2) * sum (Eq. F with Eq. E); E = (m_e / q_e) a, q_e = -e
    d.cscale = kCoulomb * kE * kE * s.w / (kMe * s.l0 * s.l0);
    d.escale = -kCoulomb * kE * s.w / (s.l0 * s.l0);
    d.dt = s.dt;
    d.half_dt = s.dt / 2.0;
    d.half_dt2 = s.dt * s.dt / 2.0;
    d.cx = s.cx;
    d.cy = s.cy;
    d.cz = s.cz;
    d.inv_l0 = 1.0 / s.l0;
    return d;
}

int stage_kind_of(const Slot &s) { return s.staging == POS_SINGLE ? STAGE_F32I : STAGE_F32IX2; }

pp_status launch_batch(pp_batch *b, const BunchDesc *descs, const BatchHeader *hdr, int step_k)
{
    B_CUDA(cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned), b->stream));
    const Shape &sh = kShapes[b->shape];
    int *err = b->d_err;
    unsigned *queue = b->d_queue;
    unsigned long long tmo = b->timeout_ns;
    int skip = b->skip_copy;
    b->skip_copy = 0;
    void *args[] = {(void *)&descs, (void *)&hdr, (void *)&queue, (void *)&step_k, (void *)&err,
                    (void *)&tmo, (void *)&skip};
    B_CUDA(cudaLaunchKernel(sh.fn, dim3(b->grid), dim3(sh.threads), args, batch_smem(), b->stream));
    return PP_OK;
}

pp_status read_errors(pp_batch *b, int *flags)
{
    B_CUDA(cudaMemcpyAsync(b->err_host, b->d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                           b->stream));
    B_CUDA(cudaStreamSynchronize(b->stream));
    flags[0] = b->err_host[0];
    flags[1] = b->err_host[1];
    if (flags[0] || flags[1]) B_CUDA(cudaMemsetAsync(b->d_err, 0, 2 * sizeof(int), b->stream));
    return PP_OK;
}

// Device table of the active bunches in `mode` (MODE_STEP for stepping; MODE_FIELDS
// writes each bunch's field into its transfer buffer).  Table order: largest source
// chunk first (ties by slot), so that the queue hands out the full-size items of the
// big bunches first and the short items of small bunches fill the tail of the step
// (longest-processing-time-first).  The order changes only which CTA takes an
// item, never an item's arithmetic.
pp_status write_table(pp_batch *b, int mode)
{
    std::vector<BunchDesc> h;
    b->order.clear();
    for (int i = 0; i < (int)b->slots.size(); ++i)
        if (b->slots[i].active) b->order.push_back(i);
    std::stable_sort(b->order.begin(), b->order.end(), [b](int x, int y) {
        const Layout &lx = b->slots[x].L, &ly = b->slots[y].L;
        return std::min(lx.npad, lx.jchunk) > std::min(ly.npad, ly.jchunk);
    });
    int items = 0;
    for (int i : b->order) {
        const Slot &s = b->slots[i];
        h.push_back(make_desc(s, mode, s.parity, items, mode == MODE_FIELDS ? s.aos : nullptr));
        items += s.L.nib * s.L.nsplit;
    }
    BatchHeader hdr{(int)h.size(), items};
    if (!h.empty())
        B_CUDA(cudaMemcpyAsync(b->d_descs, h.data(), h.size() * sizeof(BunchDesc),
                               cudaMemcpyHostToDevice, b->stream));
    B_CUDA(cudaMemcpyAsync(b->d_hdr, &hdr, sizeof(hdr), cudaMemcpyHostToDevice, b->stream));
    B_CUDA(cudaStreamSynchronize(b->stream));
    b->dirty = mode != MODE_STEP;
    return PP_OK;
}

pp_status upload_table(pp_batch *b) { return write_table(b, MODE_STEP); }

pp_status slot_moments(pp_batch *b, Slot &s, int pass, double cx, double cy, double cz,
                       double out[kMomSlots])
{
    B_CUDA(launch_moments(pass, (int)s.n, s.r[0], s.r[1], s.r[2], s.v[0], s.v[1], s.v[2], cx, cy,
                          cz, b->mom_partials, b->mom_out, b->stream));
    B_CUDA(cudaMemcpyAsync(b->mom_host, b->mom_out, kMomSlots * sizeof(double),
                           cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(cudaStreamSynchronize(b->stream));
    std::memcpy(out, b->mom_host, kMomSlots * sizeof(double));
    return PP_OK;
}

// One pass of the batch kernel over a single bunch (its own tiling), from
// positions staged into stage[1]: MODE_INIT (a_0, stages r_1 into stage[0]) or
// MODE_FIELDS (E into `out`).
pp_status slot_pass(pp_batch *b, Slot &s, int mode, double *out)
{
    BunchDesc d = make_desc(s, mode, 1, 0, out);
    BatchHeader h{1, s.L.nib * s.L.nsplit};
    B_CUDA(cudaMemcpyAsync(b->d_init_desc, &d, sizeof(d), cudaMemcpyHostToDevice, b->stream));
    B_CUDA(cudaMemcpyAsync(b->d_init_hdr, &h, sizeof(h), cudaMemcpyHostToDevice, b->stream));
    return launch_batch(b, b->d_init_desc, b->d_init_hdr, 0);
}

// Field of one bunch at its current positions with staging `staging` (the batch
// kernel, the bunch's own tiling for that staging), from sources staged into
// stage[1], into out.
pp_status slot_fields(pp_batch *b, Slot &s, int staging, double *out)
{
    s.staging = staging;
    s.L = layout_for(s.n, staging);
    B_CUDA(launch_stage(s.r[0], s.r[1], s.r[2], (int)s.n, s.L.npad, s.stage[1], stage_kind_of(s),
                        s.cx, s.cy, s.cz, 1.0 / s.l0, b->stream));
    return slot_pass(b, s, MODE_FIELDS, out);
}

// |a - b| / |b| (relative L2) of two device [n][3] arrays; synchronises.
pp_status slot_rel_diff(pp_batch *b, const Slot &s, const double *a, const double *ref,
                        double *rel)
{
    B_CUDA(launch_diff_norms(a, ref, (int)(3 * s.n), b->mom_partials, b->stream));
    double h[2 * kDiffBlocks];
    B_CUDA(cudaMemcpyAsync(h, b->mom_partials, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
    int flags[2] = {0, 0};
    if (pp_status st = read_errors(b, flags)) return st;
    if (flags[0]) return bfail(PP_ERR_TIMEOUT, "a device-side wait ran out of time");
    double d2 = 0.0, b2 = 0.0;
    for (int k = 0; k < kDiffBlocks; ++k) {
        d2 += h[2 * k];
        b2 += h[2 * k + 1];
    }
    *rel = b2 > 0 ? std::sqrt(d2 / b2) : 0.0;
    return PP_OK;
}

// PP_POS_AUTO for one bunch: the first of single and guarded staging whose field
// differs from the hi/lo-staged one by at most 5e-6 in relative L2 (half the 1e-5
// field tolerance), else hi/lo staging.  The decision reads nothing but the bunch's
// own positions, so it is the same alone and in any mix.
pp_status decide_slot_staging(pp_batch *b, Slot &s, int *staging)
{
    // the hi/lo field goes to stage[0] (32 bytes per source: room for [N][3]
    // doubles), a candidate's to the transfer buffer; sources in stage[1]
    double *e_split = static_cast<double *>(s.stage[0]);
    double *e_cand = s.aos;
    double rel = 0.0;
    if (pp_status st = slot_fields(b, s, POS_SPLIT, e_split)) return st;
    for (int cand : {POS_SINGLE, POS_GUARDED}) {
        if (pp_status st = slot_fields(b, s, cand, e_cand)) return st;
        if (pp_status st = slot_rel_diff(b, s, e_cand, e_split, &rel)) return st;
        if (rel <= 5e-6) {
            *staging = cand;
            return PP_OK;
        }
    }
    *staging = POS_SPLIT;
    return PP_OK;
}

// Potential energy of one bunch: phi'_i = sum_{j != i} 1/|r'_ij| by the FP32 pair
// kernel on freshly staged positions (scratch allocated for the call), then
// PE = 1/2 k e^2 w^2 / L0 * sum_i phi'_i.
pp_status slot_potential(pp_batch *b, Slot &s, double *pe)
{
    int count = 0;
    const Variant *vs = variants(&count);
    const Variant *v = nullptr;
    for (int i = 0; i < count; ++i)
        if (std::strcmp(vs[i].name, "phi32.fold64.t256r2k256") == 0) v = &vs[i];
    if (!v) return bfail(PP_ERR_STATE, "potential kernel missing");
    const int n = (int)s.n, npad = s.L.npad, BI = v->T * v->R;
    const int nib = (n + BI - 1) / BI, tiles = npad / v->tile;
    int S = std::min(tiles, std::max(1, (4 * b->sms + nib - 1) / nib));
    const int chunk_tiles = (tiles + S - 1) / S;
    S = (tiles + chunk_tiles - 1) / chunk_tiles;
    float4 *stage = nullptr;
    double *phi = nullptr, *partial = nullptr;
    unsigned *tickets = nullptr;
    auto cleanup = [&]() {
        cudaFree(stage);
        cudaFree(phi);
        cudaFree(partial);
        cudaFree(tickets);
    };
    if (cudaMalloc(&stage, (size_t)npad * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&phi, (size_t)npad * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&partial, (size_t)S * nib * BI * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&tickets, (size_t)nib * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return bfail(PP_ERR_NOMEM, "cannot allocate the potential-energy scratch");
    }
    ForceArgs a{};
    a.src = stage;
    a.n = n;
    a.npad = npad;
    a.nib = nib;
    a.nsplit = S;
    a.jchunk = chunk_tiles * v->tile;
    a.mode = MODE_PHI;
    const double epsl = s.eps / s.l0;
    a.eps2d = epsl * epsl;
    a.eps2f = (float)a.eps2d;
    a.partial = partial;
    a.tickets = tickets;
    a.nipad = nib * BI;
    a.out = phi;
    a.err = b->d_err;
    a.timeout_ns = b->timeout_ns;
    double m[kMomSlots];
    int flags[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(tickets, 0, (size_t)nib * sizeof(unsigned), b->stream);
    if (e == cudaSuccess)
        e = launch_stage(s.r[0], s.r[1], s.r[2], n, npad, stage, STAGE_F32, s.cx, s.cy, s.cz,
                         1.0 / s.l0, b->stream);
    if (e == cudaSuccess) e = launch_variant(*v, a, nib * S, b->stream);
    if (e == cudaSuccess)
        e = launch_moments(2, n, phi, nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, 0,
                           b->mom_partials, b->mom_out, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(m, b->mom_out, sizeof(m), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cleanup();
    if (e != cudaSuccess) return bcuda(e, "potential-energy pass");
    if (pp_status st = read_errors(b, flags)) return st;
    if (flags[0]) return bfail(PP_ERR_TIMEOUT, "a device-side wait ran out of time");
    *pe = 0.5 * kCoulomb * kE * kE * s.w * s.w / s.l0 * m[0];
    return PP_OK;
}

pp_status check_slot(const pp_batch *b, int slot)
{
    if (!b) return bfail(PP_ERR_ARG, "null batch");
    if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].active)
        return bfail(PP_ERR_ARG, "no such slot");
    return PP_OK;
}

void free_slot(pp_batch *b, Slot &s)
{
    if (s.mem) cudaFree(s.mem);
    b->used -= (int64_t)s.F.total;
    s = Slot{};
}

}  // namespace

extern "C" {

pp_status pp_batch_footprint(int64_t N, int64_t *bytes)
{
    if (!bytes || N < 1 || N > (int64_t(1) << 28)) return bfail(PP_ERR_ARG, "bad N or null bytes");
    *bytes = (int64_t)footprint_for(N).total;
    return PP_OK;
}

pp_status pp_batch_destroy(pp_batch *b)
{
    if (!b) return PP_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (auto &s : b->slots)
        if (s.active) free_slot(b, s);
    cudaFree(b->d_descs);
    cudaFree(b->d_hdr);
    cudaFree(b->d_init_desc);
    cudaFree(b->d_init_hdr);
    cudaFree(b->d_queue);
    cudaFree(b->d_err);
    cudaFree(b->mom_partials);
    cudaFree(b->mom_out);
    if (b->mom_host) cudaFreeHost(b->mom_host);
    if (b->err_host) cudaFreeHost(b->err_host);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
    delete b;
    return PP_OK;
}

pp_status pp_batch_create(int64_t budget_bytes, pp_batch **out)
{
    if (!out) return bfail(PP_ERR_ARG, "out is null");
    *out = nullptr;
    if (budget_bytes <= 0) return bfail(PP_ERR_ARG, "budget must be > 0");
    pp_batch *b = new pp_batch();
    b->budget = budget_bytes;
    auto bail = [&](pp_status s, const char *m) {
        pp_batch_destroy(b);
        return bfail(s, m);
    };
    if (cudaGetDevice(&b->device) != cudaSuccess) return bail(PP_ERR_CUDA, "no CUDA device");
    if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
        return bail(PP_ERR_CUDA, "cannot query SM count");
    if (select_shape(b, 0) != PP_OK) {
        cudaGetLastError();
        return bail(PP_ERR_CUDA, "cannot configure the batch kernel");
    }
    if (cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(PP_ERR_CUDA, "cudaStreamCreate failed");
    b->stream = b->own_stream;
    if (const char *env = std::getenv("PP_TIMEOUT_NS")) {
        const long long t = std::atoll(env);
        if (t >= 1000 && t <= 60000000000ll) b->timeout_ns = (uint64_t)t;
    }
    const bool ok = cudaMalloc(&b->d_descs, kMaxBunches * sizeof(BunchDesc)) == cudaSuccess &&
                    cudaMalloc(&b->d_hdr, sizeof(BatchHeader)) == cudaSuccess &&
                    cudaMalloc(&b->d_init_desc, sizeof(BunchDesc)) == cudaSuccess &&
                    cudaMalloc(&b->d_init_hdr, sizeof(BatchHeader)) == cudaSuccess &&
                    cudaMalloc(&b->d_queue, sizeof(unsigned)) == cudaSuccess &&
                    cudaMalloc(&b->d_err, 2 * sizeof(int)) == cudaSuccess &&
                    cudaMalloc(&b->mom_partials, kMomBlocks * kMomSlots * sizeof(double)) == cudaSuccess &&
                    cudaMalloc(&b->mom_out, kMomSlots * sizeof(double)) == cudaSuccess &&
                    cudaMallocHost(&b->mom_host, kMomSlots * sizeof(double)) == cudaSuccess &&
                    cudaMallocHost(&b->err_host, 2 * sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return bail(PP_ERR_NOMEM, "device allocation failed");
    }
    BatchHeader empty{0, 0};
    if (cudaMemcpy(b->d_hdr, &empty, sizeof(empty), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_err, 0, 2 * sizeof(int)) != cudaSuccess)
        return bail(PP_ERR_CUDA, "initialisation failed");
    *out = b;
    return PP_OK;
}

pp_status pp_batch_set_option(pp_batch *b, int key, int64_t value)
{
    if (!b) return bfail(PP_ERR_ARG, "null batch");
    switch (key) {
    case PP_OPT_STREAM:
        drop_graph(b);
        b->stream = value ? reinterpret_cast<cudaStream_t>(value) : b->own_stream;
        return PP_OK;
    case PP_OPT_GRAPH_BLOCK:
        if (value < 0 || value > 4096) return bfail(PP_ERR_ARG, "graph block must be in [0, 4096]");
        drop_graph(b);
        b->graph_block = (int)value;
        return PP_OK;
    case PP_OPT_TEST_SKIP_COPY:
        b->skip_copy = value ? 1 : 0;
        return PP_OK;
    case PP_OPT_TIMEOUT_NS:
        if (value < 1000 || value > 60000000000ll) return bfail(PP_ERR_ARG, "timeout out of range");
        drop_graph(b);
        b->timeout_ns = (uint64_t)value;
        return PP_OK;
    case PP_OPT_POSITIONS:
        if (value != PP_POS_SINGLE && value != PP_POS_SPLIT && value != PP_POS_AUTO &&
            value != PP_POS_GUARDED)
            return bfail(PP_ERR_ARG, "bad positions mode");
        b->positions = (int)value;
        return PP_OK;
    case PP_OPT_VARIANT:
        if (value < -1 || value >= kNumShapes) return bfail(PP_ERR_ARG, "no such batch shape");
        B_CUDA(cudaSetDevice(b->device));
        return select_shape(b, value < 0 ? 0 : (int)value);
    default:
        return bfail(PP_ERR_ARG, "option not supported by batch contexts");
    }
}

pp_status pp_batch_get_option(pp_batch *b, int slot, int key, int64_t *value)
{
    if (!b || !value) return bfail(PP_ERR_ARG, "null argument");
    if (slot >= 0) {
        if (pp_status st = check_slot(b, slot)) return st;
        if (key != PP_OPT_POSITIONS) return bfail(PP_ERR_ARG, "option not kept per bunch");
        *value = b->slots[slot].staging;
        return PP_OK;
    }
    if (slot != -1) return bfail(PP_ERR_ARG, "slot must be -1 (the batch) or a bunch's slot");
    switch (key) {
    case PP_OPT_POSITIONS: *value = b->positions; return PP_OK;
    case PP_OPT_VARIANT: *value = b->shape; return PP_OK;
    case PP_OPT_GRAPH_BLOCK: *value = b->graph_block; return PP_OK;
    case PP_OPT_TIMEOUT_NS: *value = (int64_t)b->timeout_ns; return PP_OK;
    case PP_OPT_STREAM: *value = (int64_t)reinterpret_cast<intptr_t>(b->stream); return PP_OK;
    default: return bfail(PP_ERR_ARG, "unknown option key");
    }
}

const char *pp_batch_shape_name(int index)
{
    return (index >= 0 && index < kNumShapes) ? kShapes[index].name : nullptr;
}

pp_status pp_batch_autotune(pp_batch *b, pp_tune_result *out)
{
    NvtxRange nvtx_("pp_batch_autotune");
    if (!b) return bfail(PP_ERR_ARG, "null batch");
    B_CUDA(cudaSetDevice(b->device));
    int nactive = 0;
    for (auto &s : b->slots) nactive += s.active;
    if (nactive == 0) return bfail(PP_ERR_STATE, "no bunches to tune on");
    // MODE_FIELDS passes over every active bunch (fields into the transfer buffers):
    // the bunches' states are untouched
    if (pp_status st = write_table(b, MODE_FIELDS)) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    B_CUDA(cudaEventCreate(&e0));
    B_CUDA(cudaEventCreate(&e1));
    const int saved = b->shape;
    int best = -1;
    double best_ms = 1e300;
    pp_status st = PP_OK;
    for (int k = 0; k < kNumShapes && st == PP_OK; ++k) {
        st = select_shape(b, k);
        if (st != PP_OK) break;
        st = launch_batch(b, b->d_descs, b->d_hdr, 0);   // untimed first pass
        if (st != PP_OK) break;
        constexpr int kReps = 3;
        cudaEventRecord(e0, b->stream);
        for (int r = 0; r < kReps && st == PP_OK; ++r) st = launch_batch(b, b->d_descs, b->d_hdr, 0);
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = bcuda(cudaGetLastError(), "autotune timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / kReps < best_ms) {
            best_ms = ms / kReps;
            best = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int flags[2] = {0, 0};
    if (st == PP_OK) st = read_errors(b, flags);
    if (st == PP_OK && flags[0]) st = bfail(PP_ERR_TIMEOUT, "a device-side wait ran out of time");
    b->dirty = true;   // the step table is rewritten before the next step
    if (st != PP_OK || best < 0) {
        select_shape(b, saved);
        return st != PP_OK ? st : bfail(PP_ERR_STATE, "no shape could be timed");
    }
    if (pp_status s2 = select_shape(b, best)) return s2;
    if (out) {
        out->variant = best;
        out->split = 0;
        out->ms_per_pass = best_ms;
        out->candidates = kNumShapes;
    }
    return PP_OK;
}

pp_status pp_batch_add(pp_batch *b, int64_t N, double w, double dt, double softening,
                       const double *pos, const double *vel, int on_device, int *slot_out)
{
    NvtxRange nvtx_("pp_batch_add");
    if (!b || !pos || !slot_out) return bfail(PP_ERR_ARG, "null argument");
    if (on_device < PP_MEM_HOST || on_device > PP_MEM_HOST_MAPPED)
        return bfail(PP_ERR_ARG, "bad memory kind");
    if (N < 1 || N > (int64_t(1) << 28)) return bfail(PP_ERR_ARG, "N must be in [1, 2^28]");
    if (!(std::isfinite(w) && w > 0) || !(std::isfinite(dt) && dt > 0) ||
        !(std::isfinite(softening) && softening >= 0))
        return bfail(PP_ERR_ARG, "w, dt must be finite and > 0; softening finite and >= 0");
    B_CUDA(cudaSetDevice(b->device));
    const Footprint F = footprint_for(N);
    if (b->used + (int64_t)F.total > b->budget)
        return bfail(PP_ERR_NOMEM, "the bunch does not fit in the remaining memory budget");
    int idx = -1;
    for (int i = 0; i < (int)b->slots.size(); ++i)
        if (!b->slots[i].active) {
            idx = i;
            break;
        }
    int nactive = 0;
    for (auto &s : b->slots) nactive += s.active;
    if (nactive >= kMaxBunches) return bfail(PP_ERR_NOMEM, "too many bunches");
    if (idx < 0) {
        idx = (int)b->slots.size();
        b->slots.emplace_back();
    }
    Slot &s = b->slots[idx];
    s = Slot{};
    s.n = N;
    s.w = w;
    s.dt = dt;
    s.eps = softening;
    s.F = F;
    s.staging = b->positions == PP_POS_AUTO ? POS_SINGLE : b->positions;
    s.L = layout_for(N, s.staging);
    if (cudaMalloc(&s.mem, F.total) != cudaSuccess) {
        cudaGetLastError();
        s = Slot{};
        return bfail(PP_ERR_NOMEM, "device allocation failed");
    }
    b->used += (int64_t)F.total;
    unsigned char *p = s.mem;
    double *state = reinterpret_cast<double *>(p);
    p += al256(F.state_bytes);
    for (int c = 0; c < 3; ++c) {
        s.r[c] = state + (size_t)(0 + c) * s.L.npad;
        s.v[c] = state + (size_t)(3 + c) * s.L.npad;
        s.a[c] = state + (size_t)(6 + c) * s.L.npad;
    }
    s.stage[0] = p;
    p += al256(F.stage_bytes);
    s.stage[1] = p;
    p += al256(F.stage_bytes);
    s.partial = reinterpret_cast<double *>(p);
    p += al256(F.partial_bytes);
    s.tickets = reinterpret_cast<unsigned *>(p);
    p += al256(F.ticket_bytes);
    s.aos = reinterpret_cast<double *>(p);
    s.active = true;
    auto undo = [&](pp_status st, const std::string &m) {
        free_slot(b, s);
        return bfail(st, m);
    };
    const size_t bytes = (size_t)N * 3 * sizeof(double);
    if (cudaMemsetAsync(state, 0, F.state_bytes, b->stream) != cudaSuccess ||
        cudaMemsetAsync(s.tickets, 0, F.ticket_bytes, b->stream) != cudaSuccess)
        return undo(PP_ERR_CUDA, "memset failed");
    const double *src = pos;
    if (on_device != PP_MEM_DEVICE) {
        if (cudaMemcpyAsync(s.aos, pos, bytes, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
            return undo(PP_ERR_CUDA, "copy of positions failed");
        src = s.aos;
    }
    if (launch_aos_to_soa(src, (int)N, s.r[0], s.r[1], s.r[2], b->d_err + 1, b->stream) != cudaSuccess)
        return undo(PP_ERR_CUDA, "layout conversion failed");
    if (vel) {
        const double *vs = vel;
        if (on_device != PP_MEM_DEVICE) {
            if (cudaMemcpyAsync(s.aos, vel, bytes, cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
                return undo(PP_ERR_CUDA, "copy of velocities failed");
            vs = s.aos;
        }
        if (launch_aos_to_soa(vs, (int)N, s.v[0], s.v[1], s.v[2], b->d_err + 1, b->stream) != cudaSuccess)
            return undo(PP_ERR_CUDA, "layout conversion failed");
    }
    int flags[2] = {0, 0};
    if (read_errors(b, flags) != PP_OK) return undo(PP_ERR_CUDA, "error word read failed");
    if (flags[1]) return undo(PP_ERR_ARG, "non-finite position or velocity");
    // staging frame of this bunch: its centroid and power-of-two RMS radius
    double m[kMomSlots];
    if (slot_moments(b, s, 0, 0, 0, 0, m) != PP_OK) return undo(PP_ERR_CUDA, "moments failed");
    s.cx = m[0] / N;
    s.cy = m[1] / N;
    s.cz = m[2] / N;
    if (slot_moments(b, s, 1, s.cx, s.cy, s.cz, m) != PP_OK) return undo(PP_ERR_CUDA, "moments failed");
    const double rms = std::sqrt(m[0] / N);
    s.l0 = 1.0;
    if (std::isfinite(rms) && rms > 0) s.l0 = std::ldexp(1.0, std::max(-200, std::min(200, (int)std::lround(std::log2(rms)))));
    if (b->positions == PP_POS_AUTO) {
        int staging = POS_SPLIT;
        if (pp_status st = decide_slot_staging(b, s, &staging)) {
            const std::string msg = pp_last_error(nullptr);
            return undo(st, msg);
        }
        s.staging = staging;
        s.L = layout_for(N, s.staging);
    }
    // a_0 = F(r_0) with the batch kernel itself (the bunch's own tiling), staging r_1
    if (launch_fill_padding(s.stage[0], (int)N, s.L.npad, stage_kind_of(s), b->stream) != cudaSuccess ||
        launch_stage(s.r[0], s.r[1], s.r[2], (int)N, s.L.npad, s.stage[1], stage_kind_of(s), s.cx,
                     s.cy, s.cz, 1.0 / s.l0, b->stream) != cudaSuccess)
        return undo(PP_ERR_CUDA, "staging failed");
    if (slot_pass(b, s, MODE_INIT, nullptr) != PP_OK)
        return undo(PP_ERR_CUDA, "initial force pass failed to launch");
    if (read_errors(b, flags) != PP_OK) return undo(PP_ERR_CUDA, "error word read failed");
    if (flags[0]) return undo(PP_ERR_TIMEOUT, "a device-side wait ran out of time");
    s.parity = 0;
    s.step = 0;
    b->dirty = true;
    *slot_out = idx;
    return PP_OK;
}

pp_status pp_batch_remove(pp_batch *b, int slot)
{
    if (pp_status st = check_slot(b, slot)) return st;
    B_CUDA(cudaSetDevice(b->device));
    B_CUDA(cudaStreamSynchronize(b->stream));
    free_slot(b, b->slots[slot]);
    b->dirty = true;
    return PP_OK;
}

pp_status pp_batch_step(pp_batch *b, int64_t nsteps)
{
    NvtxRange nvtx_("pp_batch_step");
    if (!b) return bfail(PP_ERR_ARG, "null batch");
    if (nsteps < 0) return bfail(PP_ERR_ARG, "nsteps must be >= 0");
    B_CUDA(cudaSetDevice(b->device));
    if (b->dirty) {
        if (pp_status st = upload_table(b)) return st;
    }
    if (b->order.empty() || nsteps == 0) return PP_OK;
    int64_t left = nsteps;
    const int gb = b->graph_block;
    if (gb > 0 && (gb % 2) == 0 && left >= gb && b->stream != nullptr && !b->skip_copy) {
        if (!b->graph || b->graph_steps != gb) {
            drop_graph(b);
            cudaGraph_t g = nullptr;
            B_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            pp_status st = PP_OK;
            for (int k = 0; k < gb && st == PP_OK; ++k) st = launch_batch(b, b->d_descs, b->d_hdr, k);
            cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
            if (st != PP_OK) return st;
            if (ce != cudaSuccess) return bcuda(ce, "cudaStreamEndCapture");
            cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (ie != cudaSuccess) return bcuda(ie, "cudaGraphInstantiate");
            b->graph_steps = gb;
        }
        while (left >= gb) {      // even blocks leave every bunch's parity unchanged
            B_CUDA(cudaGraphLaunch(b->graph, b->stream));
            left -= gb;
        }
    }
    for (int64_t k = 0; k < left; ++k) {
        if (pp_status st = launch_batch(b, b->d_descs, b->d_hdr, (int)k)) return st;
    }
    int flags[2] = {0, 0};
    if (pp_status st = read_errors(b, flags)) return st;
    if (flags[0]) {
        // results of this call are void; restart the bunches from their last state is not
        // possible, so the caller must re-add them
        for (int i : b->order) b->slots[i].step = -1;
        return bfail(PP_ERR_TIMEOUT, "a device-side wait ran out of time; bunch states are "
                                     "unspecified and must be re-added");
    }
    for (int i : b->order) {
        Slot &s = b->slots[i];
        s.step += nsteps;
        s.parity ^= (int)(left & 1);
    }
    if (left & 1) b->dirty = true;   // parity0 in the table changed
    return PP_OK;
}

pp_status pp_batch_get_state(pp_batch *b, int slot, double *pos, double *vel, double *acc,
                             int64_t *step, int on_device)
{
    if (pp_status st = check_slot(b, slot)) return st;
    if (on_device < PP_MEM_HOST || on_device > PP_MEM_HOST_MAPPED)
        return bfail(PP_ERR_ARG, "bad memory kind");
    B_CUDA(cudaSetDevice(b->device));
    Slot &s = b->slots[slot];
    if (s.step < 0) return bfail(PP_ERR_STATE, "bunch state is unspecified after a timeout");
    double *const *arrs[3] = {s.r, s.v, s.a};
    double *outs[3] = {pos, vel, acc};
    const size_t bytes = (size_t)s.n * 3 * sizeof(double);
    for (int k = 0; k < 3; ++k) {
        if (!outs[k]) continue;
        double *target = on_device == PP_MEM_DEVICE ? outs[k] : s.aos;
        B_CUDA(launch_soa_to_aos(arrs[k][0], arrs[k][1], arrs[k][2], (int)s.n, target, b->stream));
        if (on_device != PP_MEM_DEVICE)
            B_CUDA(cudaMemcpyAsync(outs[k], s.aos, bytes, cudaMemcpyDeviceToHost, b->stream));
    }
    if (step) *step = s.step;
    B_CUDA(cudaStreamSynchronize(b->stream));
    return PP_OK;
}

pp_status pp_batch_diagnostics(pp_batch *b, int slot, pp_diag *d, int with_pe)
{
    if (pp_status st = check_slot(b, slot)) return st;
    if (!d) return bfail(PP_ERR_ARG, "out is null");
    B_CUDA(cudaSetDevice(b->device));
    Slot &s = b->slots[slot];
    if (s.step < 0) return bfail(PP_ERR_STATE, "bunch state is unspecified after a timeout");
    double m0[kMomSlots], m1[kMomSlots];
    if (pp_status st = slot_moments(b, s, 0, 0, 0, 0, m0)) return st;
    const double n = (double)s.n;
    const double cx = m0[0] / n, cy = m0[1] / n, cz = m0[2] / n;
    if (pp_status st = slot_moments(b, s, 1, cx, cy, cz, m1)) return st;
    const double mw = kMe * s.w;
    d->t = (double)s.step * s.dt;
    d->step = s.step;
    d->rms_radius = std::sqrt(m1[0] / n);
    d->ke = 0.5 * mw * m1[1];
    d->pe = NAN;
    if (with_pe) {
        if (pp_status st = slot_potential(b, s, &d->pe)) return st;
    }
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
    return PP_OK;
}

pp_status pp_batch_info(pp_batch *b, int64_t *active, int64_t *bytes_used, int64_t *budget)
{
    if (!b) return bfail(PP_ERR_ARG, "null batch");
    int64_t n = 0;
    for (auto &s : b->slots) n += s.active;
    if (active) *active = n;
    if (bytes_used) *bytes_used = b->used;
    if (budget) *budget = b->budget;
    return PP_OK;
}

}  // extern "C"
