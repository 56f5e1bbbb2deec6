// pp_batch.cuh -- many independent bunches of uneven size in one persistent
// launch per time step (the same physics as the single-bunch kernels: Eq. B/E
// force sum, Eq. G/H push).
//
// Work items are (bunch b, block of BI targets, j-chunk of JCHUNK sources).
// The tiling of a bunch depends only on its own N (BI and JCHUNK are fixed),
// so a bunch's results are bitwise the same alone or in any mix.  CTAs pull
// items from a global queue (one atomic per item); which CTA computes an item
// does not change its arithmetic, and the S partial sums of a target block are
// added by the last arriving CTA in an order fixed by S.
#pragma once

#include "pp_force.cuh"

namespace ppk {

// 1024-source tiles in a two-stage ring and the pair loop unrolled twice:
// measured fastest for this kernel on the 64-bunch mix (unrolling once, which
// suits the single-bunch kernel, is 13 % slower here).
constexpr int kBatchT = 128, kBatchR = 4, kBatchTile = 1024, kBatchStages = 2, kBatchMinB = 4;
constexpr int kBatchUnroll = 2;
constexpr int kBatchBI = kBatchT * kBatchR;
constexpr int kBatchJChunk = 8192;   // sources per work item (a multiple of the tile)

// One bunch as the batch kernel sees it (device memory, rewritten by the host
// between step blocks).
struct BunchDesc {
    void *stage[2];          // interleaved FP32 staging (STAGE_F32I), npad entries each
    double *r[3], *v[3], *a[3];
    double *partial;         // [nsplit][3][nipad]
    unsigned *tickets;       // [nib], zero between launches
    int n, npad, nib, nsplit, jchunk, nipad;
    int item_base;           // index of the bunch's first work item
    int parity0;             // staging parity at step_k = 0 of the launch sequence
    int mode;                // MODE_STEP or MODE_INIT
    float eps2f;
    double cscale, dt, half_dt, half_dt2, cx, cy, cz, inv_l0;
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
    p.cscale = d.cscale;
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

template <int T, int R, int TILE, int STAGES, int MINB>
__global__ void __launch_bounds__(T, MINB)
    batch_f32x2_kernel(const BunchDesc *__restrict__ descs, const BatchHeader *__restrict__ hdr,
                       unsigned *queue, int step_k, int *err, unsigned long long timeout_ns,
                       int skip_copy)
{
    constexpr int BI = T * R;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar_full[STAGES], bar_empty[STAGES];
    __shared__ int s_abort, s_flag, s_item;

    const int tid = threadIdx.x;
    Ring<float4, TILE, STAGES> rg{reinterpret_cast<float4 *>(smem_raw), nullptr, bar_full,
                                  bar_empty};
    double *sacc = reinterpret_cast<double *>(smem_raw + (size_t)STAGES * TILE * sizeof(float4));
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
        const BunchDesc &d = descs[lo];
        const int local = item - d.item_base;
        const int ib = local % d.nib;
        const int split = local / d.nib;
        const int par = (d.parity0 + step_k) & 1;

        // Arguments of the tile loop only: the epilogue's arguments are read from
        // the descriptor again after the loop, so they hold no registers during it.
        const int skip = (skip_copy && item == 0) ? 2 : 0;   // test hook: item 0 loses a tile
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

        const float *srcf = static_cast<const float *>(p.src);
        f2_t X[R], Y[R], Z[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i0 + r * T + tid;
            float x = -1e18f, y = -1e18f, z = -1e18f;
            if (i < p.n) {
                const float *q = srcf + 8 * (size_t)(i >> 1) + (i & 1);
                x = q[0];
                y = q[2];
                z = q[4];
            }
            X[r] = f2_pack(x, x);
            Y[r] = f2_pack(y, y);
            Z[r] = f2_pack(z, z);
            sacc[r * T + tid] = sacc[BI + r * T + tid] = sacc[2 * BI + r * T + tid] = 0.0;
        }
        const f2_t EPS2 = f2_pack(p.eps2f, p.eps2f);
        int issued = 0, seen = 0;
        const bool ok = run_tiles<float4, T, TILE, STAGES, false>(
            p, rg, j0, ntiles, issued, seen,
            [&](const float4 *tile, const float4 *, int) {
                f2_t AX[R], AY[R], AZ[R];
                tile_packed<R, TILE, false, false, kBatchUnroll>(tile, nullptr, X, Y, Z, X, Y, Z, EPS2, AX,
                                                      AY, AZ);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float3 f = tile_partial<TILE, false, false>(
                        AX[r], AY[r], AZ[r], tile, nullptr, X[r], Y[r], Z[r], X[r], Y[r], Z[r],
                        p.eps2f);
                    const float fx = f.x, fy = f.y, fz = f.z;
                    sacc[r * T + tid] += (double)fx;
                    sacc[BI + r * T + tid] += (double)fy;
                    sacc[2 * BI + r * T + tid] += (double)fz;
                }
            },
            g);
        if (!ok) {
            s_abort = 1;
            atomicOr(err, 1);
        }
        __syncthreads();
        if (s_abort) {
            ring_drain(p, rg, issued, seen, ntiles, g);
            return;
        }
        g += ntiles;
        const ForceArgs pe = item_args(descs[lo], par, err, timeout_ns, skip);
        double ax64[R], ay64[R], az64[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            ax64[r] = sacc[r * T + tid];
            ay64[r] = sacc[BI + r * T + tid];
            az64[r] = sacc[2 * BI + r * T + tid];
        }
        bool finish = true;
        if (pe.nsplit > 1) {
            finish = split_publish<T, R>(pe, ib, split, ax64, ay64, az64, 3, &s_flag);
            if (finish) split_gather<T, R>(pe, ib, ax64, ay64, az64, 3);
        }
        if (finish) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                finish_particle<STAGE_F32I>(pe, i0 + r * T + tid, ax64[r], ay64[r], az64[r]);
        }
        __syncthreads();  // s_item and the shared accumulators are reused next
    }
}

}  // namespace ppk
