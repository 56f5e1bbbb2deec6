// pp_batch.cuh -- many independent bunches of uneven size in one persistent
// launch per time step (the same physics as the single-bunch kernels: Eq. B/E
// force sum, Eq. G/H push).
//
// Work items are (bunch b, block of targets, j-chunk of sources).  The tiling
// of a bunch depends only on its own N and its own staging (single, hi/lo or
// guarded, chosen from its own positions), so a bunch's results are bitwise the
// same alone or in any mix.  CTAs pull items from a global queue (one atomic per
// item); which CTA computes an item does not change its arithmetic, and the S
// partial sums of a target block are added by the last arriving CTA in an
// order fixed by S.
//
// Compiled shapes differ in threads per CTA (and so targets per thread, the
// block of targets being fixed), in the register budget per thread and in the
// unrolling of the pair loop only; the source tile (and so every FP32 partial
// sum), the j-chunk and the order of every addition are the same in all of
// them, so every shape gives bitwise the same results and the autotuner may
// pick any of them for any mix.
#pragma once

#include "pp_force.cuh"

namespace ppk {

// Sources per tile with single staging; hi/lo items use half-size tiles so that
// a stage holds the hi and the lo tile in the same shared-memory bytes.
constexpr int kBatchTile = 1024, kBatchStages = 2;
constexpr int kBatchJChunk = 8192;   // sources per work item (a multiple of the tile)

// Targets per block of a bunch: a function of its staging only (the same in
// every compiled shape, so that the partial-sum layout never changes).
__host__ __device__ constexpr int batch_block(int staging) { return staging == POS_SPLIT ? 256 : 512; }
constexpr int kBatchBIMax = 512;

// One bunch as the batch kernel sees it (device memory, rewritten by the host
// between step blocks).
struct BunchDesc {
    void *stage[2];          // STAGE_F32I (single) or STAGE_F32IX2 (hi/lo, guarded); npad entries
    double *r[3], *v[3], *a[3];
    double *partial;         // [nsplit][3][nipad]
    unsigned *tickets;       // [nib], zero between launches
    double *out;             // MODE_FIELDS: E [n][3]
    int n, npad, nib, nsplit, jchunk, nipad;
    int item_base;           // index of the bunch's first work item
    int parity0;             // staging parity at step_k = 0 of the launch sequence
    int mode;                // MODE_STEP, MODE_INIT or MODE_FIELDS
    int staging;             // POS_SINGLE, POS_SPLIT or POS_GUARDED
    float eps2f;
    double cscale, escale, dt, half_dt, half_dt2, cx, cy, cz, inv_l0;
};

struct BatchHeader {
    int nbunch;
    int nitems;
};

// Full kernel arguments of one bunch for the current step.
__device__ __forceinline__ ForceArgs item_args(const BunchDesc &d, int par, int *err,
                                               unsigned long long timeout_ns, int skip)
{
    ForceArgs p{};
    p.src = d.stage[par];
    p.dst = d.stage[par ^ 1];
    p.n = d.n;
    p.npad = d.npad;
    p.nib = d.nib;
    p.nsplit = d.nsplit;
    p.jchunk = d.jchunk;
    p.mode = d.mode;
    p.eps2f = d.eps2f;
    p.partial = d.partial;
    p.tickets = d.tickets;
    p.nipad = d.nipad;
    for (int c = 0; c < 3; ++c) {
        p.r[c] = d.r[c];
        p.v[c] = d.v[c];
        p.a[c] = d.a[c];
    }
    p.out = d.out;
    p.cscale = d.cscale;
    p.escale = d.escale;
    p.dt = d.dt;
    p.half_dt = d.half_dt;
    p.half_dt2 = d.half_dt2;
    p.cx = d.cx;
    p.cy = d.cy;
    p.cz = d.cz;
    p.inv_l0 = d.inv_l0;
    p.err = err;
    p.timeout_ns = timeout_ns;
    p.skip_copy = skip;
    return p;
}

// Shared state of one persistent CTA.
struct BatchCta {
    float4 *ring;            // kBatchStages x kBatchTile float4
    double *sacc;            // [3][kBatchBIMax] FP64 accumulators
    uint64_t *full, *empty;  // ring barriers
    int *s_abort, *s_flag;
};

// One work item of one bunch.  R targets per thread, TILE sources per tile
// (with hi/lo staging, hi and lo tiles of TILE sources each share one stage of
// the ring; guarded staging streams the hi parts, see tile_guarded).  g counts
// the tiles this CTA has streamed through the ring (it sets each tile's ring
// slot and barrier phase).  Returns false if a bounded wait ran out (the ring
// is drained; the CTA must exit).
template <int T, int R, int TILE, int STAGES, int UNROLL, int POS>
__device__ __forceinline__ bool batch_item(const BunchDesc *__restrict__ descs, int bunch,
                                           int local, int step_k, const BatchCta &cta, int &g,
                                           int *err, unsigned long long timeout_ns, int skip)
{
    constexpr bool SPLIT = POS == POS_SPLIT, GUARD = POS == POS_GUARDED;
    constexpr int BI = T * R;
    static_assert(BI == batch_block(POS), "block of targets fixed by the staging");
    static_assert(TILE % 2 == 0 && (SPLIT ? 2 * TILE : TILE) <= kBatchTile, "tile fits a stage");
    const int tid = threadIdx.x;
    const BunchDesc &d = descs[bunch];
    const int ib = local % d.nib;
    const int split = local / d.nib;
    const int par = (d.parity0 + step_k) & 1;

    // Arguments of the tile loop only: the epilogue's arguments are read from
    // the descriptor again after the loop, so they hold no registers during it.
    ForceArgs p{};
    p.src = d.stage[par];
    p.n = d.n;
    p.npad = d.npad;
    p.jchunk = d.jchunk;
    p.eps2f = d.eps2f;
    p.err = err;
    p.timeout_ns = timeout_ns;
    p.skip_copy = skip;

    const int i0 = ib * BI;
    const int j0 = split * p.jchunk;
    const int j1 = min(j0 + p.jchunk, p.npad);
    const int ntiles = (j1 - j0) / TILE;

    // with SPLIT the ring's bytes hold STAGES hi tiles followed by STAGES lo tiles
    Ring<float4, TILE, STAGES, SPLIT> rg{cta.ring, SPLIT ? cta.ring + STAGES * TILE : nullptr,
                                         cta.full, cta.empty};
    double *sacc = cta.sacc;
    const float *srcf = static_cast<const float *>(p.src);
    f2_t X[R], Y[R], Z[R], XL[R], YL[R], ZL[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = i0 + r * T + tid;
        float x = -1e18f, y = -1e18f, z = -1e18f;   // targets past n: far from everything
        float xl = 0.f, yl = 0.f, zl = 0.f;
        if (i < p.n) {
            const float *q = srcf + 8 * (size_t)(i >> 1) + (i & 1);
            x = q[0];
            y = q[2];
            z = q[4];
            if (SPLIT) {
                const float *ql = q + 4 * (size_t)p.npad;
                xl = ql[0];
                yl = ql[2];
                zl = ql[4];
            }
        }
        X[r] = f2_pack(x, x);
        Y[r] = f2_pack(y, y);
        Z[r] = f2_pack(z, z);
        XL[r] = f2_pack(xl, xl);
        YL[r] = f2_pack(yl, yl);
        ZL[r] = f2_pack(zl, zl);
        sacc[r * T + tid] = sacc[kBatchBIMax + r * T + tid] = sacc[2 * kBatchBIMax + r * T + tid] = 0.0;
    }
    const f2_t EPS2 = f2_pack(p.eps2f, p.eps2f);
    float thr[R];
    if (GUARD) guard_thresholds<T, R>(X, Y, Z, i0, p.n, thr);
    const float *glo = srcf + 4 * (size_t)p.npad;
    int issued = 0, seen = 0;
    const bool ok = run_tiles<float4, T, TILE, STAGES, SPLIT>(
        p, rg, j0, ntiles, issued, seen,
        [&](const float4 *tile, const float4 *tlo, int jfirst) {
            float3 fg[R];
            if (GUARD) {
                tile_guarded<T, R, BI, TILE, false, UNROLL>(tile, jfirst, i0, p.n, glo, X, Y, Z,
                                                           thr, EPS2, p.eps2f, fg);
            } else {
                f2_t AX[R], AY[R], AZ[R];
                float MS[R];
                tile_packed<R, TILE, false, SPLIT, UNROLL>(tile, tlo, X, Y, Z, XL, YL, ZL, EPS2,
                                                           AX, AY, AZ, MS);
#pragma unroll
                for (int r = 0; r < R; ++r)
                    fg[r] = tile_partial<TILE, false, SPLIT>(AX[r], AY[r], AZ[r], tile, tlo, X[r],
                                                             Y[r], Z[r], XL[r], YL[r], ZL[r],
                                                             p.eps2f);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float3 f = fg[r];
                sacc[r * T + tid] += (double)f.x;
                sacc[kBatchBIMax + r * T + tid] += (double)f.y;
                sacc[2 * kBatchBIMax + r * T + tid] += (double)f.z;
            }
        },
        g);
    if (!ok) {
        *cta.s_abort = 1;
        atomicOr(err, 1);
    }
    __syncthreads();
    if (*cta.s_abort) {
        ring_drain(p, rg, issued, seen, ntiles, g);
        return false;
    }
    g += ntiles;
    const ForceArgs pe = item_args(descs[bunch], par, err, timeout_ns, skip);
    double ax64[R], ay64[R], az64[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        ax64[r] = sacc[r * T + tid];
        ay64[r] = sacc[kBatchBIMax + r * T + tid];
        az64[r] = sacc[2 * kBatchBIMax + r * T + tid];
    }
    bool finish = true;
    if (pe.nsplit > 1) {
        finish = split_publish<T, R>(pe, ib, split, ax64, ay64, az64, 3, cta.s_flag);
        if (finish) split_gather<T, R>(pe, ib, ax64, ay64, az64, 3);
    }
    if (finish) {
#pragma unroll
        for (int r = 0; r < R; ++r)
            finish_particle<(SPLIT || GUARD) ? STAGE_F32IX2 : STAGE_F32I>(
                pe, i0 + r * T + tid, ax64[r], ay64[r], az64[r]);
    }
    return true;
}

// The persistent batch kernel.  T threads per CTA: single-staging and guarded
// items give each thread 512 / T targets, hi/lo items 256 / T targets and
// half-size tiles.
// MINB: CTAs per SM the register budget is sized for.  UNROLL: unrolling of the
// packed pair loop.
template <int T, int TILE, int STAGES, int MINB, int UNROLL>
__global__ void __launch_bounds__(T, MINB)
    batch_f32x2_kernel(const BunchDesc *__restrict__ descs, const BatchHeader *__restrict__ hdr,
                       unsigned *queue, int step_k, int *err, unsigned long long timeout_ns,
                       int skip_copy)
{
    constexpr int RS = batch_block(POS_SINGLE) / T, RH = batch_block(POS_SPLIT) / T;
    static_assert(RS >= 1 && RH >= 1, "at most 256 threads per CTA");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar_full[STAGES], bar_empty[STAGES];
    __shared__ int s_abort, s_flag, s_item;

    const int tid = threadIdx.x;
    BatchCta cta{reinterpret_cast<float4 *>(smem_raw),
                 reinterpret_cast<double *>(smem_raw + (size_t)STAGES * TILE * sizeof(float4)),
                 bar_full, bar_empty, &s_abort, &s_flag};
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_empty[s], T / 32);
        }
        s_abort = 0;
        fence_barrier_init();
    }
    const int nbunch = hdr->nbunch;
    const int nitems = hdr->nitems;
    int g = 0;  // tiles streamed through the ring so far by this CTA
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= nitems) break;
        int lo = 0, hi = nbunch - 1;  // last bunch whose first item is <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (descs[mid].item_base <= item) lo = mid;
            else hi = mid - 1;
        }
        const int local = item - descs[lo].item_base;
        const int skip = (skip_copy && item == 0) ? 2 : 0;   // test hook: item 0 loses a tile
        const int staging = descs[lo].staging;
        const bool ok =
            staging == POS_SPLIT
                ? batch_item<T, RH, TILE / 2, STAGES, UNROLL, POS_SPLIT>(descs, lo, local, step_k,
                                                                         cta, g, err, timeout_ns, skip)
            : staging == POS_GUARDED
                ? batch_item<T, RS, TILE, STAGES, UNROLL, POS_GUARDED>(descs, lo, local, step_k,
                                                                       cta, g, err, timeout_ns, skip)
                : batch_item<T, RS, TILE, STAGES, UNROLL, POS_SINGLE>(descs, lo, local, step_k,
                                                                      cta, g, err, timeout_ns, skip);
        if (!ok) return;
        __syncthreads();  // s_item and the shared accumulators are reused next
    }
}

}  // namespace ppk
