// pp_force.cuh -- the O(N^2) direct Coulomb sum (arXiv 2502.10640, Eq. B/E)
// with the Velocity-Verlet push (Eq. G/H) fused into its epilogue.
//
// Work decomposition.  A CTA owns BI = T*R target particles i (R per thread,
// strided by T so loads coalesce) and one j-chunk of the staged source array.
// With S > 1 chunks per i-block, each CTA writes FP64 partial sums, and the
// CTA that finishes an i-block last (an atomic ticket decides who) adds the S
// partials in an order fixed by S alone and runs the epilogue.  The ticket
// picks only *who* sums, never the order, so results are bitwise reproducible.
//
// Data movement.  Staged sources are float4 (x', y', z', q') in units of a
// power-of-two length L0 about a fixed centre.  One thread streams TILE-sized
// j-tiles through a STAGES-deep shared-memory ring with 1D bulk copies (TMA)
// tracked by mbarriers; every warp releases a stage through an "empty"
// mbarrier, after which the producer refills it.  All waits are bounded.
//
// Pair math (per pair, FP32): d = r_i - r_j; s = d.d + eps'^2;
// inv = rsqrt(s) on the SFU; acc += inv^3 * d.  Equal weights factor out of
// the sum (Sec. 2.1), so no per-pair weight multiply is needed.
// Per TILE the FP32 partials are folded into FP64 (or into a compensated FP32
// hi/lo pair); a non-finite tile partial (a pair with s == 0: the self pair
// when eps = 0, or coincident particles) is recomputed for that particle with
// the zero-distance pairs skipped, which is the reading of Eq. B used here.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pp_device.cuh"

namespace ppk {

enum Mode : int {
    MODE_STEP = 0,    // a_{n+1} from staged r_{n+1}; epilogue: Eq. G recompute, Eq. H, stage r_{n+2}
    MODE_FIELDS = 1,  // E = escale * sum, written [N][3]; state untouched
    MODE_INIT = 2,    // a_0 from staged r_0; epilogue: store a_0, stage r_1 (Eq. G)
    MODE_PHI = 3      // phi'_i = sum_{j != i} 1/sqrt(s); written [N]
};

enum Acc : int { ACC_FP64FOLD = 0, ACC_KAHAN = 1, ACC_FP64FULL = 2 };

// Positions modes a force kernel implements (the values of the public pp_positions).
enum PosKind : int { POS_SINGLE = 0, POS_SPLIT = 1, POS_GUARDED = 3 };

struct ForceArgs {
    const void *src;        // staged sources: float4[npad] (or double4[npad] for FP64 pair math)
    int n;                  // real particles
    int npad;               // staged length (multiple of the tile)
    int nib;                // i-blocks
    int nsplit;             // j-chunks per i-block (S)
    int jchunk;             // sources per chunk (multiple of the tile)
    int mode;
    float eps2f;            // (eps / L0)^2
    double eps2d;
    double *partial;        // [S][3][nipad] FP64 partial sums (S > 1)
    unsigned *tickets;      // [nib] arrival counters, zero between launches
    int nipad;              // nib * BI
    double *r[3];           // state, SoA, [n] each
    double *v[3];
    double *a[3];
    void *dst;              // staging written by the epilogue (float4 or double4)
    double *out;            // fields [n][3] (MODE_FIELDS) or phi [n] (MODE_PHI)
    const float *wrel;      // per-particle weight / reference weight, or null (all 1)
    double cscale;          // a = cscale * sum
    double escale;          // E = escale * sum
    double dt, half_dt, half_dt2;
    double cx, cy, cz, inv_l0;
    int *err;               // device error word (bit 0: a wait ran out)
    unsigned long long timeout_ns;
    int skip_copy;          // test hook: 1 = CTA 0 withholds its last tile copy, 2 = this CTA does
    // Spatially ordered passes (tile-box guard): src is the staged array in
    // sorted order; target k of the kernel is particle perm[k] for every
    // epilogue read and write; boxes[2t], boxes[2t+1] are the lower and upper
    // corners of the hi parts of sorted tile t (null: particle order).
    const int *perm;
    const float4 *boxes;
};

// ---- FP64 push arithmetic, written so that no multiply-add is fused: the
// drift of Eq. G is evaluated as (r + v dt) + a (dt^2/2) and the kick of
// Eq. H as v + (a_old + a_new) (dt/2), each operation rounded once.
__device__ __forceinline__ double drift(double r, double v, double a, double dt, double half_dt2)
{
    return __dadd_rn(__dadd_rn(r, __dmul_rn(v, dt)), __dmul_rn(a, half_dt2));
}

__device__ __forceinline__ double kick(double v, double a_old, double a_new, double half_dt)
{
    return __dadd_rn(v, __dmul_rn(__dadd_rn(a_old, a_new), half_dt));
}

// Staged source layouts.
//  STAGE_F32:   float4 (x', y', z', 1) per particle, npad entries.
//  STAGE_F32X2: float4 hi[npad] followed by float4 lo[npad], with
//               hi = fl32(p') and lo = fl32(p' - hi): about 48 significant bits.
//  STAGE_F64:   double4 (x', y', z', 1) per particle (FP64 pair math).
//  STAGE_F32I:  sources interleaved by pairs for packed f32x2 arithmetic: the
//               32 bytes of pair k = (2k, 2k+1) hold x_2k x_2k+1 y_2k y_2k+1
//               z_2k z_2k+1 w_2k w_2k+1 (same 16 bytes per source as STAGE_F32).
//  STAGE_F32IX2: the hi parts in the interleaved layout, followed (at float
//               offset 4 npad) by the lo parts in the same layout.
// p' = (r - centre) / L0 with L0 a power of two, so the scaling is exact.
// The weight slot carries w_j / W (W the context's reference weight; 1 for
// equal weights); kernels that assume equal weights do not read it.
// Padding entries (n <= i < npad) sit at 1e18 with weight 0.
enum StageKind : int { STAGE_F32 = 0, STAGE_F32X2 = 1, STAGE_F64 = 2, STAGE_F32I = 3,
                       STAGE_F32IX2 = 4 };

__device__ __forceinline__ void store_interleaved(void *dst, int i, float x, float y, float z,
                                                  float w)
{
    float *f = static_cast<float *>(dst) + 8 * (size_t)(i >> 1) + (i & 1);
    f[0] = x;
    f[2] = y;
    f[4] = z;
    f[6] = w;
}

__device__ __forceinline__ double staged_coord(double x, double c, double inv_l0)
{
    return __dmul_rn(__dsub_rn(x, c), inv_l0);
}

template <int KIND>
__device__ __forceinline__ void store_staged(void *dst, int npad, int i, double x, double y,
                                             double z, double cx, double cy, double cz,
                                             double inv_l0, float qw = 1.0f)
{
    const double px = staged_coord(x, cx, inv_l0);
    const double py = staged_coord(y, cy, inv_l0);
    const double pz = staged_coord(z, cz, inv_l0);
    if (KIND == STAGE_F64) {
        static_cast<double4 *>(dst)[i] = make_double4(px, py, pz, (double)qw);
    } else if (KIND == STAGE_F32I || KIND == STAGE_F32IX2) {
        const float hx = __double2float_rn(px), hy = __double2float_rn(py),
                    hz = __double2float_rn(pz);
        store_interleaved(dst, i, hx, hy, hz, qw);
        if (KIND == STAGE_F32IX2)
            store_interleaved(static_cast<float *>(dst) + 4 * (size_t)npad, i,
                              __double2float_rn(px - (double)hx), __double2float_rn(py - (double)hy),
                              __double2float_rn(pz - (double)hz), 0.0f);
    } else {
        const float hx = __double2float_rn(px), hy = __double2float_rn(py),
                    hz = __double2float_rn(pz);
        static_cast<float4 *>(dst)[i] = make_float4(hx, hy, hz, qw);
        if (KIND == STAGE_F32X2)
            static_cast<float4 *>(dst)[(size_t)npad + i] =
                make_float4(__double2float_rn(px - (double)hx), __double2float_rn(py - (double)hy),
                            __double2float_rn(pz - (double)hz), 0.0f);
    }
}

template <int KIND>
__device__ __forceinline__ void store_padding(void *dst, int npad, int i)
{
    if (KIND == STAGE_F64) {
        static_cast<double4 *>(dst)[i] = make_double4(1e18, 1e18, 1e18, 0.0);
    } else if (KIND == STAGE_F32I || KIND == STAGE_F32IX2) {
        store_interleaved(dst, i, 1e18f, 1e18f, 1e18f, 0.f);
        if (KIND == STAGE_F32IX2)
            store_interleaved(static_cast<float *>(dst) + 4 * (size_t)npad, i, 0.f, 0.f, 0.f, 0.f);
    } else {
        static_cast<float4 *>(dst)[i] = make_float4(1e18f, 1e18f, 1e18f, 0.f);
        if (KIND == STAGE_F32X2)
            static_cast<float4 *>(dst)[(size_t)npad + i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Epilogue for particle i given its full FP64 sum (staged units).
template <int KIND>
__device__ __forceinline__ void finish_particle(const ForceArgs &p, int i, double sx, double sy,
                                                double sz)
{
    if (i >= p.n) return;
    if (p.perm) i = p.perm[i];
    if (p.mode == MODE_FIELDS) {
        p.out[3 * (size_t)i + 0] = p.escale * sx;
        p.out[3 * (size_t)i + 1] = p.escale * sy;
        p.out[3 * (size_t)i + 2] = p.escale * sz;
        return;
    }
    if (p.mode == MODE_PHI) {
        p.out[i] = sx;
        return;
    }
    const double an[3] = {p.cscale * sx, p.cscale * sy, p.cscale * sz};
    double rn[3];
    if (p.mode == MODE_STEP) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double r0 = p.r[c][i], v0 = p.v[c][i], a0 = p.a[c][i];
            const double r1 = drift(r0, v0, a0, p.dt, p.half_dt2);   // Eq. G (as staged)
            const double v1 = kick(v0, a0, an[c], p.half_dt);         // Eq. H
            p.r[c][i] = r1;
            p.v[c][i] = v1;
            p.a[c][i] = an[c];
            rn[c] = drift(r1, v1, an[c], p.dt, p.half_dt2);           // next Eq. G, staged only
        }
    } else {  // MODE_INIT
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            p.a[c][i] = an[c];
            rn[c] = drift(p.r[c][i], p.v[c][i], an[c], p.dt, p.half_dt2);
        }
    }
    store_staged<KIND>(p.dst, p.npad, i, rn[0], rn[1], rn[2], p.cx, p.cy, p.cz, p.inv_l0,
                       p.wrel ? p.wrel[i] : 1.0f);
}

// Shared-memory ring + barriers of one CTA.  With TWO, every stage holds a
// second tile (the lo parts of split staging, read from src + npad).
template <class E, int TILE, int STAGES, bool TWO = false>
struct Ring {
    E *buf;
    E *buf2;
    uint64_t *full;
    uint64_t *empty;
};

// Test hook (PP_OPT_TEST_SKIP_COPY): is the copy of local tile t withheld?
__device__ __forceinline__ bool copy_withheld(const ForceArgs &p, int t, int ntiles)
{
    return t == ntiles - 1 && (p.skip_copy == 2 || (p.skip_copy == 1 && blockIdx.x == 0));
}

// Warp-uniform bounded wait: lane 0 waits (bounded), the verdict is shared
// with the warp, then every lane observes the completed phase itself (which
// gives each thread acquire ordering on the bulk-copied data).  All lanes
// return the same value, so no lane can leave the warp behind at a later
// warp-synchronous point.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait_bounded(bar, parity, limit_ns) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return false;
    const int mine = mbar_wait_bounded(bar, parity, limit_ns) ? 1 : 0;
    return __all_sync(0xffffffffu, mine) != 0;
}

// Stream the CTA's j-tiles through the ring and call body(tile, tile_lo,
// j_first) for each.  Lane 0 of warp 0 issues the bulk copies.  A stage is
// refilled only after every warp has released it; the producer never blocks
// for that while other tiles are ready to consume: after each tile it issues
// whatever refills are already possible (non-blocking probe of the "empty"
// barriers) and waits only when the very tile it needs next is not issued
// yet.  Returns false if a wait ran out; the value is uniform within each
// warp.  On false the caller must run ring_drain before the CTA exits.
//
// g0 is the number of tiles this CTA already streamed through the same ring
// (persistent kernels run several work items back to back); ring slot and
// barrier phase of local tile t follow from g = g0 + t.  Every earlier tile
// must have been released by all warps before the call (a CTA-wide barrier).
template <class E, int T, int TILE, int STAGES, bool TWO, class Body>
__device__ __forceinline__ bool run_tiles(const ForceArgs &p,
                                          const Ring<E, TILE, STAGES, TWO> &rg, int j0,
                                          int ntiles, int &issued, int &seen, Body &&body,
                                          int g0 = 0)
{
    const int tid = threadIdx.x;
    const E *src = static_cast<const E *>(p.src);
    constexpr uint32_t kBytes = TILE * sizeof(E);
    auto issue = [&](int t) {
        const int s = (g0 + t) % STAGES;
        mbar_arrive_expect_tx(&rg.full[s], TWO ? 2 * kBytes : kBytes);
        const bool withhold = copy_withheld(p, t, ntiles);
        if (!withhold) {
            const size_t off = (size_t)j0 + (size_t)t * TILE;
            bulk_g2s(rg.buf + s * TILE, src + off, kBytes, &rg.full[s]);
            if (TWO) bulk_g2s(rg.buf2 + s * TILE, src + (size_t)p.npad + off, kBytes, &rg.full[s]);
        }
    };
    // tile t may be issued once global tile g0 + t - STAGES has been released
    auto released = [&](int t, bool block) {
        const int u = g0 + t - STAGES;
        if (u < 0) return true;
        uint64_t *bar = &rg.empty[u % STAGES];
        const uint32_t par = (u / STAGES) & 1;
        return block ? mbar_wait_bounded(bar, par, p.timeout_ns) : mbar_test_wait(bar, par);
    };
    int next = 0;  // next local tile to issue (meaningful on thread 0 only)
    int ok0 = 1;
    if (tid == 0) {
        for (; next < STAGES && next < ntiles; ++next) {
            if (!released(next, true)) {
                ok0 = 0;
                break;
            }
            issue(next);
        }
        issued = next;
    }
    if (tid < 32 && !__shfl_sync(0xffffffffu, ok0, 0)) return false;
    for (int t = 0; t < ntiles; ++t) {
        const int g = g0 + t;
        const int s = g % STAGES;
        const uint32_t ph = (g / STAGES) & 1;
        if (tid < 32) {  // warp 0: make sure tile t has been issued
            int ok = 1;
            if (tid == 0) {
                while (ok && next <= t) {
                    ok = released(next, true);
                    if (ok) {
                        issue(next);
                        issued = ++next;
                    }
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) return false;
        }
        if (!warp_wait(&rg.full[s], ph, p.timeout_ns)) return false;
        if (tid == 0) seen = t + 1;
        body(rg.buf + s * TILE, TWO ? rg.buf2 + s * TILE : nullptr, j0 + t * TILE);
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&rg.empty[s]);
        if (tid == 0) {  // refill every stage that is already free, without waiting
            while (next < ntiles && released(next, false)) {
                issue(next);
                issued = ++next;
            }
        }
    }
    return true;
}

// After a failed wait: thread 0 waits (bounded) for copies it issued that
// have not been observed complete, so no bulk copy still targets shared
// memory when the CTA exits.
template <class E, int TILE, int STAGES, bool TWO>
__device__ __forceinline__ void ring_drain(const ForceArgs &p,
                                           const Ring<E, TILE, STAGES, TWO> &rg, int issued,
                                           int seen, int ntiles, int g0 = 0)
{
    if (threadIdx.x != 0) return;
    for (int t = seen; t < issued; ++t) {
        const bool withheld = copy_withheld(p, t, ntiles);
        if (withheld) continue;
        const int g = g0 + t;
        mbar_wait_bounded(&rg.full[g % STAGES], (g / STAGES) & 1, p.timeout_ns);
    }
}

// ---- pair loops ----------------------------------------------------------

// Separation component.  Single staging: d = p_i - p_j.  Split staging:
// d = (hi_i - hi_j) + (lo_i - lo_j); for a close pair the hi difference is
// exact (Sterbenz), so d keeps about 48 significant bits of the positions.
template <bool SPLIT>
__device__ __forceinline__ float sep(float hi_i, float lo_i, float hi_j, float lo_j)
{
    if (SPLIT) return (hi_i - hi_j) + (lo_i - lo_j);
    return hi_i - hi_j;
}

// Fast loop: TILE sources against R targets, no checks.
template <int R, int TILE, bool SPLIT>
__device__ __forceinline__ void tile_fast(const float4 *__restrict__ tile,
                                          const float4 *__restrict__ tlo, const float (&xi)[R],
                                          const float (&yi)[R], const float (&zi)[R],
                                          const float (&xl)[R], const float (&yl)[R],
                                          const float (&zl)[R], float eps2, float (&fx)[R],
                                          float (&fy)[R], float (&fz)[R])
{
#pragma unroll 4
    for (int j = 0; j < TILE; ++j) {
        const float4 q = tile[j];
        float4 l = make_float4(0.f, 0.f, 0.f, 0.f);
        if (SPLIT) l = tlo[j];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float dx = sep<SPLIT>(xi[r], xl[r], q.x, l.x);
            const float dy = sep<SPLIT>(yi[r], yl[r], q.y, l.y);
            const float dz = sep<SPLIT>(zi[r], zl[r], q.z, l.z);
            const float s = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
            const float inv = rsqrt_sfu(s);
            const float inv3 = inv * inv * inv;
            fx[r] = fmaf(inv3, dx, fx[r]);
            fy[r] = fmaf(inv3, dy, fy[r]);
            fz[r] = fmaf(inv3, dz, fz[r]);
        }
    }
}

// Safe loop for one target: pairs with s == 0 add nothing.  Same operations
// in the same order as tile_fast for every other pair.
template <int TILE, bool SPLIT>
__device__ __noinline__ float3 tile_safe1(const float4 *__restrict__ tile,
                                          const float4 *__restrict__ tlo, float x, float y,
                                          float z, float xl, float yl, float zl, float eps2)
{
    float ax = 0.f, ay = 0.f, az = 0.f;
    for (int j = 0; j < TILE; ++j) {
        const float4 q = tile[j];
        float4 l = make_float4(0.f, 0.f, 0.f, 0.f);
        if (SPLIT) l = tlo[j];
        const float dx = sep<SPLIT>(x, xl, q.x, l.x);
        const float dy = sep<SPLIT>(y, yl, q.y, l.y);
        const float dz = sep<SPLIT>(z, zl, q.z, l.z);
        const float s = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
        if (s > 0.f) {
            const float inv = rsqrt_sfu(s);
            const float inv3 = inv * inv * inv;
            ax = fmaf(inv3, dx, ax);
            ay = fmaf(inv3, dy, ay);
            az = fmaf(inv3, dz, az);
        }
    }
    return make_float3(ax, ay, az);
}

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Split-path epilogue shared by all kernels: write partials, take a ticket,
// and let the last CTA of the i-block sum the S partials (split_gather).
// Returns true on the CTA that must finish the i-block.
template <int T, int R>
__device__ __forceinline__ bool split_publish(const ForceArgs &p, int ib, int split,
                                              const double (&sx)[R], const double (&sy)[R],
                                              const double (&sz)[R], int ncomp, int *s_flag)
{
    const int tid = threadIdx.x;
    const size_t stride = (size_t)p.nipad;
    double *base = p.partial + (size_t)split * ncomp * stride;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = ib * T * R + r * T + tid;
        base[i] = sx[r];
        if (ncomp == 3) {
            base[stride + i] = sy[r];
            base[2 * stride + i] = sz[r];
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned prev = atomicAdd(&p.tickets[ib], 1u);
        *s_flag = (prev == (unsigned)(p.nsplit - 1));
    }
    __syncthreads();
    if (!*s_flag) return false;
    __threadfence();
    return true;
}

// The finishing CTA adds the S partials of each of its targets.  For each
// target the loads of U consecutive chunks (all three components) are issued
// together so their L2 latencies overlap; lane u accumulates chunks u, u+U,
// u+2U, ... and the U lanes are combined by a fixed tree.  The summation order
// is a fixed function of S, so results stay bitwise reproducible.
template <int T, int R>
__device__ __forceinline__ void split_gather(const ForceArgs &p, int ib, double (&sx)[R],
                                             double (&sy)[R], double (&sz)[R], int ncomp)
{
    constexpr int U = 4;
    const int tid = threadIdx.x;
    const size_t stride = (size_t)p.nipad;
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const int i = ib * T * R + r * T + tid;
        double acc[3][U];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int u = 0; u < U; ++u) acc[c][u] = 0.0;
        for (int s0 = 0; s0 < p.nsplit; s0 += U) {
            double v[3][U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int s = s0 + u;
                const double *base = p.partial + (size_t)s * ncomp * stride + i;
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    v[c][u] = (s < p.nsplit && c < ncomp) ? ld_cg(base + c * stride) : 0.0;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int u = 0; u < U; ++u) acc[c][u] += v[c][u];
        }
        double t[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) t[c] = (acc[c][0] + acc[c][1]) + (acc[c][2] + acc[c][3]);
        // R is small and unrolled elsewhere; select the output slot explicitly
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (q == r) {
                sx[q] = t[0];
                sy[q] = t[1];
                sz[q] = t[2];
            }
    }
    if (tid == 0) p.tickets[ib] = 0u;
}

// ---- FP32 pair math, FP64 or compensated fold ------------------------------
// SPLIT selects the hi/lo staging (about 48-bit separations at +6 FP32
// operations per pair); otherwise sources and targets are single floats.
template <int T, int R, int TILE, int STAGES, int ACC, int MINB, bool SPLIT>
__global__ void __launch_bounds__(T, MINB) force_f32_kernel(const ForceArgs p)
{
    constexpr int BI = T * R;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar_full[STAGES], bar_empty[STAGES];
    __shared__ int s_abort, s_flag;

    const int tid = threadIdx.x;
    const int ib = blockIdx.x % p.nib;
    const int split = blockIdx.x / p.nib;
    const int i0 = ib * BI;
    const int j0 = split * p.jchunk;
    const int j1 = min(j0 + p.jchunk, p.npad);
    const int ntiles = (j1 - j0) / TILE;

    float4 *ring = reinterpret_cast<float4 *>(smem_raw);
    Ring<float4, TILE, STAGES, SPLIT> rg{ring, SPLIT ? ring + STAGES * TILE : nullptr, bar_full,
                                         bar_empty};
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_empty[s], T / 32);
        }
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();

    const float4 *src = static_cast<const float4 *>(p.src);
    float xi[R], yi[R], zi[R], xl[R], yl[R], zl[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = i0 + r * T + tid;
        // targets past n sit far away from every source and from the padding
        const float4 q = (i < p.n) ? src[i] : make_float4(-1e18f, -1e18f, -1e18f, 0.f);
        xi[r] = q.x;
        yi[r] = q.y;
        zi[r] = q.z;
        const float4 l = (SPLIT && i < p.n) ? src[(size_t)p.npad + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        xl[r] = l.x;
        yl[r] = l.y;
        zl[r] = l.z;
    }

    double dx64[R], dy64[R], dz64[R];  // FP64 fold (ACC_FP64FOLD)
    float hx[R], hy[R], hz[R], lx[R], ly[R], lz[R];  // compensated fold (ACC_KAHAN)
#pragma unroll
    for (int r = 0; r < R; ++r) {
        dx64[r] = dy64[r] = dz64[r] = 0.0;
        hx[r] = hy[r] = hz[r] = lx[r] = ly[r] = lz[r] = 0.f;
    }
    const float eps2 = p.eps2f;

    int issued = 0, seen = 0;
    const bool ok = run_tiles<float4, T, TILE, STAGES, SPLIT>(
        p, rg, j0, ntiles, issued, seen, [&](const float4 *tile, const float4 *tlo, int) {
            float fx[R], fy[R], fz[R];
#pragma unroll
            for (int r = 0; r < R; ++r) fx[r] = fy[r] = fz[r] = 0.f;
            tile_fast<R, TILE, SPLIT>(tile, tlo, xi, yi, zi, xl, yl, zl, eps2, fx, fy, fz);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!isfinite(fx[r] + fy[r] + fz[r])) {
                    const float3 f = tile_safe1<TILE, SPLIT>(tile, tlo, xi[r], yi[r], zi[r], xl[r],
                                                             yl[r], zl[r], eps2);
                    fx[r] = f.x;
                    fy[r] = f.y;
                    fz[r] = f.z;
                }
                if (ACC == ACC_KAHAN) {
                    float s, e;
                    two_sum(hx[r], fx[r], s, e); hx[r] = s; lx[r] = __fadd_rn(lx[r], e);
                    two_sum(hy[r], fy[r], s, e); hy[r] = s; ly[r] = __fadd_rn(ly[r], e);
                    two_sum(hz[r], fz[r], s, e); hz[r] = s; lz[r] = __fadd_rn(lz[r], e);
                } else {
                    dx64[r] += (double)fx[r];
                    dy64[r] += (double)fy[r];
                    dz64[r] += (double)fz[r];
                }
            }
        });
    if (!ok) {
        s_abort = 1;
        atomicOr(p.err, 1);
    }
    __syncthreads();
    if (s_abort) {
        ring_drain(p, rg, issued, seen, ntiles);
        return;
    }
    if (ACC == ACC_KAHAN) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            dx64[r] = (double)hx[r] + (double)lx[r];
            dy64[r] = (double)hy[r] + (double)ly[r];
            dz64[r] = (double)hz[r] + (double)lz[r];
        }
    }
    if (p.nsplit > 1) {
        if (!split_publish<T, R>(p, ib, split, dx64, dy64, dz64, 3, &s_flag)) return;
        split_gather<T, R>(p, ib, dx64, dy64, dz64, 3);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        finish_particle<SPLIT ? STAGE_F32X2 : STAGE_F32>(p, i0 + r * T + tid, dx64[r], dy64[r],
                                                         dz64[r]);
}

// ---- potential: phi'_i = sum_{j != i, s > 0} 1/sqrt(s), FP32 pairs, FP64 fold ----
template <int T, int R, int TILE, int STAGES>
__global__ void __launch_bounds__(T) phi_f32_kernel(const ForceArgs p)
{
    constexpr int BI = T * R;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar_full[STAGES], bar_empty[STAGES];
    __shared__ int s_abort, s_flag;

    const int tid = threadIdx.x;
    const int ib = blockIdx.x % p.nib;
    const int split = blockIdx.x / p.nib;
    const int i0 = ib * BI;
    const int j0 = split * p.jchunk;
    const int j1 = min(j0 + p.jchunk, p.npad);
    const int ntiles = (j1 - j0) / TILE;

    Ring<float4, TILE, STAGES> rg{reinterpret_cast<float4 *>(smem_raw), nullptr, bar_full, bar_empty};
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_empty[s], T / 32);
        }
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();

    const float4 *src = static_cast<const float4 *>(p.src);
    float xi[R], yi[R], zi[R];
    int gi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = i0 + r * T + tid;
        gi[r] = i;
        const float4 q = (i < p.n) ? src[i] : make_float4(-1e18f, -1e18f, -1e18f, 0.f);
        xi[r] = q.x;
        yi[r] = q.y;
        zi[r] = q.z;
    }
    double acc[R], dummy[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = dummy[r] = 0.0;
    const float eps2 = p.eps2f;
    int issued = 0, seen = 0;
    const bool ok = run_tiles<float4, T, TILE, STAGES, false>(
        p, rg, j0, ntiles, issued, seen, [&](const float4 *tile, const float4 *, int jfirst) {
            float f[R];
#pragma unroll
            for (int r = 0; r < R; ++r) f[r] = 0.f;
            for (int j = 0; j < TILE; ++j) {
                const float4 q = tile[j];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float dx = xi[r] - q.x;
                    const float dy = yi[r] - q.y;
                    const float dz = zi[r] - q.z;
                    const float s = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
                    // padding sources carry q.w = 0
                    const float term = (s > 0.f && jfirst + j != gi[r]) ? q.w * rsqrt_sfu(s) : 0.f;
                    f[r] += term;
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] += (double)f[r];
        });
    if (!ok) {
        s_abort = 1;
        atomicOr(p.err, 1);
    }
    __syncthreads();
    if (s_abort) {
        ring_drain(p, rg, issued, seen, ntiles);
        return;
    }
    if (p.nsplit > 1) {
        if (!split_publish<T, R>(p, ib, split, acc, dummy, dummy, 1, &s_flag)) return;
        split_gather<T, R>(p, ib, acc, dummy, dummy, 1);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) finish_particle<STAGE_F32>(p, i0 + r * T + tid, acc[r], 0.0, 0.0);
}

// ---- FP64 pair math and accumulation (comparison path) ---------------------
template <int T, int R, int TILE, int STAGES>
__global__ void __launch_bounds__(T) force_f64_kernel(const ForceArgs p)
{
    constexpr int BI = T * R;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar_full[STAGES], bar_empty[STAGES];
    __shared__ int s_abort, s_flag;

    const int tid = threadIdx.x;
    const int ib = blockIdx.x % p.nib;
    const int split = blockIdx.x / p.nib;
    const int i0 = ib * BI;
    const int j0 = split * p.jchunk;
    const int j1 = min(j0 + p.jchunk, p.npad);
    const int ntiles = (j1 - j0) / TILE;

    Ring<double4, TILE, STAGES> rg{reinterpret_cast<double4 *>(smem_raw), nullptr, bar_full,
                                   bar_empty};
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_empty[s], T / 32);
        }
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();

    const double4 *src = static_cast<const double4 *>(p.src);
    double xi[R], yi[R], zi[R], ax[R], ay[R], az[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = i0 + r * T + tid;
        const double4 q = (i < p.n) ? src[i] : make_double4(-1e18, -1e18, -1e18, 0.0);
        xi[r] = q.x;
        yi[r] = q.y;
        zi[r] = q.z;
        ax[r] = ay[r] = az[r] = 0.0;
    }
    const double eps2 = p.eps2d;
    int issued = 0, seen = 0;
    const bool ok = run_tiles<double4, T, TILE, STAGES, false>(
        p, rg, j0, ntiles, issued, seen, [&](const double4 *tile, const double4 *, int) {
            for (int j = 0; j < TILE; ++j) {
                const double4 q = tile[j];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const double dx = xi[r] - q.x;
                    const double dy = yi[r] - q.y;
                    const double dz = zi[r] - q.z;
                    const double s = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));
                    if (s > 0.0) {
                        const double inv = rsqrt(s);
                        const double inv3 = q.w * inv * inv * inv;  // source weight ratio
                        ax[r] = fma(inv3, dx, ax[r]);
                        ay[r] = fma(inv3, dy, ay[r]);
                        az[r] = fma(inv3, dz, az[r]);
                    }
                }
            }
        });
    if (!ok) {
        s_abort = 1;
        atomicOr(p.err, 1);
    }
    __syncthreads();
    if (s_abort) {
        ring_drain(p, rg, issued, seen, ntiles);
        return;
    }
    if (p.nsplit > 1) {
        if (!split_publish<T, R>(p, ib, split, ax, ay, az, 3, &s_flag)) return;
        split_gather<T, R>(p, ib, ax, ay, az, 3);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        finish_particle<STAGE_F64>(p, i0 + r * T + tid, ax[r], ay[r], az[r]);
}


// ---- packed FP32x2 pair math (sm_100+ f32x2 instructions), FP64 fold --------
// Sources are read two at a time from the interleaved layout, so one f32x2
// instruction evaluates the same target against sources 2k and 2k+1; each
// target keeps even-source and odd-source partial sums in the two lanes of its
// accumulators and adds them at every fold.  Per pair: 5.5 f32x2 instructions
// (11 FP32 lane operations, as in the scalar loop) and one SFU rsqrt, so the
// FP32 work needs half the issue slots.
typedef unsigned long long f2_t;   // two floats in one 64-bit register pair

__device__ __forceinline__ f2_t f2_pack(float lo, float hi)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void f2_unpack(f2_t v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b)
{
    f2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b)
{
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b)
{
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c)
{
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Maximum of three floats in one instruction (sm_100+).
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Guarded staging (PP_POS_GUARDED): sources and targets carry hi/lo staged
// positions, the pair loop runs on the hi parts only (single-staging cost) and
// keeps, per target, the largest reciprocal softened separation rsqrt(s) of the
// tile (one three-input maximum per two pairs over the SFU's results, on the
// ALU pipe, while the FMA pipe bounds the loop).  A tile holding a source with
// s < (|p_i| / 2^8)^2, i.e. rsqrt(s) > 2^8 / |p_i|, is summed
// again for that target with hi/lo separations: the single-staging error of a
// pair term is about 3 u |p| / s^(3/2) (u = 2^-24), so every pair left to the
// hi parts has s^(1/2) >= 2^16 u |p_i| and a relative error below about 5e-5,
// while the few pairs close enough to spoil the sum get the ~48-bit
// separations of split staging.  The tile that holds the CTA's own targets
// (where the self pair, d = 0 and s = eps^2, would always pass the test) is
// summed with hi/lo separations from the start, its lo parts read from L2.
// Returns target i's threshold on rsqrt(s): 2^8 / |p_i| (+inf at p_i = 0).
__device__ __forceinline__ float guard_threshold(float x, float y, float z)
{
    const float p2 = fmaf(z, z, fmaf(y, y, x * x));
    return 256.0f * rsqrt_sfu(p2);
}

// Scalar loop over an interleaved tile for one target: pairs with s == 0 add
// nothing (the fallback when a packed tile sum is not finite).
template <int TILE, bool WEIGHTED = false, bool SPLITPOS = false>
__device__ __noinline__ float3 tile_safe1_interleaved(const float *__restrict__ tile,
                                                      const float *__restrict__ tlo, float x,
                                                      float y, float z, float xl, float yl,
                                                      float zl, float eps2)
{
    float ax = 0.f, ay = 0.f, az = 0.f;
    for (int j = 0; j < TILE; ++j) {
        const float *q = tile + 8 * (j >> 1) + (j & 1);
        float dx = x - q[0];
        float dy = y - q[2];
        float dz = z - q[4];
        if (SPLITPOS) {
            const float *ql = tlo + 8 * (j >> 1) + (j & 1);
            dx = dx + (xl - ql[0]);
            dy = dy + (yl - ql[2]);
            dz = dz + (zl - ql[4]);
        }
        const float s = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
        if (s > 0.f) {
            const float inv = rsqrt_sfu(s);
            const float inv3 = WEIGHTED ? inv * inv * inv * q[6] : inv * inv * inv;
            ax = fmaf(inv3, dx, ax);
            ay = fmaf(inv3, dy, ay);
            az = fmaf(inv3, dz, az);
        }
    }
    return make_float3(ax, ay, az);
}


// One tile of the packed pair loop: TILE interleaved sources, two per f32x2
// operation, against R targets.  AX/AY/AZ receive each target's partial sums
// over the even (low lane) and odd (high lane) sources of the tile.
// With GUARD, MS[r] receives the largest rsqrt(s) of target r over the tile.
template <int R, int TILE, bool WEIGHTED, bool SPLITPOS, int UNROLL, bool GUARD = false>
__device__ __forceinline__ void tile_packed(const float4 *__restrict__ tile,
                                            const float4 *__restrict__ tlo, const f2_t (&X)[R],
                                            const f2_t (&Y)[R], const f2_t (&Z)[R],
                                            const f2_t (&XL)[R], const f2_t (&YL)[R],
                                            const f2_t (&ZL)[R], f2_t EPS2, f2_t (&AX)[R],
                                            f2_t (&AY)[R], f2_t (&AZ)[R], float (&MS)[R])
{
#pragma unroll
    for (int r = 0; r < R; ++r) {
        AX[r] = AY[r] = AZ[r] = 0ull;
        if (GUARD) MS[r] = 0.f;
    }
#pragma unroll UNROLL
    for (int k = 0; k < TILE / 2; ++k) {
        const float4 a = tile[2 * k];       // x0 x1 y0 y1
        const float4 b = tile[2 * k + 1];   // z0 z1 w0 w1
        const f2_t XJ = f2_pack(a.x, a.y), YJ = f2_pack(a.z, a.w), ZJ = f2_pack(b.x, b.y);
        const f2_t WJ = f2_pack(b.z, b.w);
        f2_t XJL = 0ull, YJL = 0ull, ZJL = 0ull;
        if (SPLITPOS) {
            const float4 al = tlo[2 * k];
            const float4 bl = tlo[2 * k + 1];
            XJL = f2_pack(al.x, al.y);
            YJL = f2_pack(al.z, al.w);
            ZJL = f2_pack(bl.x, bl.y);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            f2_t DX = f2_sub(X[r], XJ);
            f2_t DY = f2_sub(Y[r], YJ);
            f2_t DZ = f2_sub(Z[r], ZJ);
            if (SPLITPOS) {
                DX = f2_add(DX, f2_sub(XL[r], XJL));
                DY = f2_add(DY, f2_sub(YL[r], YJL));
                DZ = f2_add(DZ, f2_sub(ZL[r], ZJL));
            }
            const f2_t S = f2_fma(DZ, DZ, f2_fma(DY, DY, f2_fma(DX, DX, EPS2)));
            float s0, s1;
            f2_unpack(S, s0, s1);
            const float q0 = rsqrt_sfu(s0), q1 = rsqrt_sfu(s1);
            if (GUARD) MS[r] = fmax3(MS[r], q0, q1);
            const f2_t INV = f2_pack(q0, q1);
            const f2_t INV3 = WEIGHTED ? f2_mul(f2_mul(f2_mul(INV, INV), INV), WJ)
                                       : f2_mul(f2_mul(INV, INV), INV);
            AX[r] = f2_fma(INV3, DX, AX[r]);
            AY[r] = f2_fma(INV3, DY, AY[r]);
            AZ[r] = f2_fma(INV3, DZ, AZ[r]);
        }
    }
}

// Guarded tile partial of one target (PP_POS_GUARDED): the two lanes added; if
// the tile holds a close pair (ms > thr, ms the largest rsqrt(s) of the tile)
// or the sum is not finite (a pair with s == 0), the tile is summed again for
// this target with hi/lo separations by the scalar loop (which also skips
// zero-distance pairs).  tile: hi parts in
// shared memory; glo: the same sources' lo parts in global memory; the
// target's lo parts are read from global memory only on this rare path.
template <int TILE, bool WEIGHTED>
__device__ __forceinline__ float3 tile_partial_guarded(f2_t AX, f2_t AY, f2_t AZ, float ms,
                                                       float thr, const float4 *tile,
                                                       const float *glo, f2_t X, f2_t Y, f2_t Z,
                                                       const float *tgt_lo, float eps2)
{
    float x0, x1, y0, y1, z0, z1;
    f2_unpack(AX, x0, x1);
    f2_unpack(AY, y0, y1);
    f2_unpack(AZ, z0, z1);
    float3 f = make_float3(x0 + x1, y0 + y1, z0 + z1);
    if (ms > thr || !isfinite(f.x + f.y + f.z)) {
        float xs, ys, zs, dummy;
        f2_unpack(X, xs, dummy);
        f2_unpack(Y, ys, dummy);
        f2_unpack(Z, zs, dummy);
        f = tile_safe1_interleaved<TILE, WEIGHTED, true>(reinterpret_cast<const float *>(tile), glo,
                                                         xs, ys, zs, __ldcg(tgt_lo),
                                                         __ldcg(tgt_lo + 2), __ldcg(tgt_lo + 4),
                                                         eps2);
    }
    return f;
}

// Tile partial of one target: the two lanes added; a non-finite result (a pair
// with s == 0) is recomputed by the scalar loop that skips zero-distance pairs.
template <int TILE, bool WEIGHTED, bool SPLITPOS>
__device__ __forceinline__ float3 tile_partial(f2_t AX, f2_t AY, f2_t AZ, const float4 *tile,
                                               const float4 *tlo, f2_t X, f2_t Y, f2_t Z, f2_t XL,
                                               f2_t YL, f2_t ZL, float eps2)
{
    float x0, x1, y0, y1, z0, z1;
    f2_unpack(AX, x0, x1);
    f2_unpack(AY, y0, y1);
    f2_unpack(AZ, z0, z1);
    float3 f = make_float3(x0 + x1, y0 + y1, z0 + z1);
    if (!isfinite(f.x + f.y + f.z)) {
        float xs, ys, zs, xl, yl, zl, dummy;
        f2_unpack(X, xs, dummy);
        f2_unpack(Y, ys, dummy);
        f2_unpack(Z, zs, dummy);
        f2_unpack(XL, xl, dummy);
        f2_unpack(YL, yl, dummy);
        f2_unpack(ZL, zl, dummy);
        f = tile_safe1_interleaved<TILE, WEIGHTED, SPLITPOS>(
            reinterpret_cast<const float *>(tile), reinterpret_cast<const float *>(tlo), xs, ys,
            zs, xl, yl, zl, eps2);
    }
    return f;
}

// One tile of guarded staging (PP_POS_GUARDED) for the R targets i0 + r T + tid
// of a block of BI targets: the tile overlapping the block (the self pairs'
// tile) is summed with hi/lo separations, the lo parts of its sources and
// targets read from L2; any other tile on the hi parts, with the close-pair
// check of tile_partial_guarded.  tile: hi parts in shared memory; glo: the lo
// parts of the staged array (4 npad floats after its start); f: per-target
// FP32 tile partials.
template <int T, int R, int BI, int TILE, bool WEIGHTED, int UNROLL>
__device__ __forceinline__ void tile_guarded(const float4 *__restrict__ tile, int jfirst, int i0,
                                             int n, const float *__restrict__ glo,
                                             const f2_t (&X)[R], const f2_t (&Y)[R],
                                             const f2_t (&Z)[R], const float (&thr)[R], f2_t EPS2,
                                             float eps2, float3 (&f)[R])
{
    const int tid = threadIdx.x;
    f2_t AX[R], AY[R], AZ[R];
    float MS[R];
    const bool diag = jfirst < i0 + BI && i0 < jfirst + TILE;
    if (diag) {
        f2_t XL[R], YL[R], ZL[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i0 + r * T + tid;
            float xl = 0.f, yl = 0.f, zl = 0.f;
            if (i < n) {
                const float *ql = glo + 8 * (size_t)(i >> 1) + (i & 1);
                xl = ql[0];
                yl = ql[2];
                zl = ql[4];
            }
            XL[r] = f2_pack(xl, xl);
            YL[r] = f2_pack(yl, yl);
            ZL[r] = f2_pack(zl, zl);
        }
        const float4 *dlo = reinterpret_cast<const float4 *>(glo + 4 * (size_t)jfirst);
        tile_packed<R, TILE, WEIGHTED, true, UNROLL>(tile, dlo, X, Y, Z, XL, YL, ZL, EPS2, AX, AY,
                                                     AZ, MS);
    } else {
        tile_packed<R, TILE, WEIGHTED, false, UNROLL, true>(tile, nullptr, X, Y, Z, X, Y, Z, EPS2,
                                                            AX, AY, AZ, MS);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = i0 + r * T + tid;
        f[r] = tile_partial_guarded<TILE, WEIGHTED>(
            AX[r], AY[r], AZ[r], diag ? 0.f : MS[r], thr[r], tile, glo + 4 * (size_t)jfirst,
            X[r], Y[r], Z[r], glo + 8 * (size_t)(i >> 1) + (i & 1), eps2);
    }
}

// Box-guarded tile (GUARD == 2, spatially sorted sources): the tile's sources
// lie in the box [blo, bhi] (hi parts), so no pair of target r in it can have
// rsqrt(s) above rsqrt(dbox^2 + eps^2), dbox the target's distance to the box.
// A warp where that bound passes some target's threshold (2^8 / |p_i|), or
// whose CTA owns the tile's targets (the self pairs), sums the tile with hi/lo
// separations for all its targets (packed; the ring carries the lo parts of
// the tile, the targets' lo parts are read from L2); every other warp takes
// the hi parts only, with no test per pair.  The tile partial keeps the
// non-finite check of tile_partial_guarded (pairs with s == 0).
template <int T, int R, int BI, int TILE, bool WEIGHTED, int UNROLL>
__device__ __forceinline__ void tile_boxed(const float4 *__restrict__ tile,
                                           const float4 *__restrict__ tlo, int jfirst, int i0,
                                           int n, const float *__restrict__ glo,
                                           const float4 *__restrict__ box, const f2_t (&X)[R],
                                           const f2_t (&Y)[R], const f2_t (&Z)[R],
                                           const float (&thr)[R], f2_t EPS2, float eps2,
                                           float3 (&f)[R])
{
    const int tid = threadIdx.x;
    const float4 blo = box[0], bhi = box[1];
    bool close = jfirst < i0 + BI && i0 < jfirst + TILE;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float x, y, z, dummy;
        f2_unpack(X[r], x, dummy);
        f2_unpack(Y[r], y, dummy);
        f2_unpack(Z[r], z, dummy);
        const float dx = fmax3(blo.x - x, x - bhi.x, 0.f);
        const float dy = fmax3(blo.y - y, y - bhi.y, 0.f);
        const float dz = fmax3(blo.z - z, z - bhi.z, 0.f);
        const float sb = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
        close |= rsqrt_sfu(sb) > thr[r];
    }
    close = __any_sync(0xffffffffu, close);
    f2_t AX[R], AY[R], AZ[R];
    float MS[R];
    if (close) {
        f2_t XL[R], YL[R], ZL[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i0 + r * T + tid;
            float xl = 0.f, yl = 0.f, zl = 0.f;
            if (i < n) {
                const float *ql = glo + 8 * (size_t)(i >> 1) + (i & 1);
                xl = ql[0];
                yl = ql[2];
                zl = ql[4];
            }
            XL[r] = f2_pack(xl, xl);
            YL[r] = f2_pack(yl, yl);
            ZL[r] = f2_pack(zl, zl);
        }
        tile_packed<R, TILE, WEIGHTED, true, UNROLL>(tile, tlo, X, Y, Z, XL, YL, ZL, EPS2, AX, AY,
                                                     AZ, MS);
    } else {
        tile_packed<R, TILE, WEIGHTED, false, UNROLL>(tile, nullptr, X, Y, Z, X, Y, Z, EPS2, AX,
                                                      AY, AZ, MS);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = i0 + r * T + tid;
        f[r] = tile_partial_guarded<TILE, WEIGHTED>(AX[r], AY[r], AZ[r], 0.f, thr[r], tile,
                                                    glo + 4 * (size_t)jfirst, X[r], Y[r], Z[r],
                                                    glo + 8 * (size_t)(i >> 1) + (i & 1), eps2);
    }
}

// GUARD: per-target close-pair thresholds on rsqrt(s) (+inf for targets past n,
// which sit far from everything).
template <int T, int R>
__device__ __forceinline__ void guard_thresholds(const f2_t (&X)[R], const f2_t (&Y)[R],
                                                 const f2_t (&Z)[R], int i0, int n,
                                                 float (&thr)[R])
{
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float x, y, z, dummy;
        f2_unpack(X[r], x, dummy);
        f2_unpack(Y[r], y, dummy);
        f2_unpack(Z[r], z, dummy);
        thr[r] = i0 + r * T + (int)threadIdx.x < n ? guard_threshold(x, y, z) : INFINITY;
    }
}

// SMEM_ACC keeps the FP64 fold accumulators in shared memory (BI x 3 doubles
// per CTA) instead of registers, trading a shared load/store per fold for
// fewer registers and so more resident warps.
// WEIGHTED multiplies each pair term by the source's weight ratio w_j / W
// (taken from the staged weight lanes): one more f32x2 multiply per two pairs.
// SPLITPOS reads hi/lo staged sources (STAGE_F32IX2) and forms each
// separation as (hi_i - hi_j) + (lo_i - lo_j): three f32x2 operations per
// component instead of one.
// KAHAN folds each tile partial into a compensated FP32 pair (TwoSum: hi
// takes the rounded sum, lo collects the exact rounding errors) instead of an
// FP64 accumulator: six FP32 additions per component and tile on the FP32
// pipe in place of a conversion and an add on the FP64 pipe, which runs at a
// small fraction of the FP32 rate on this GPU.  With SMEM_ACC the pairs live
// in shared memory ([hi x,y,z][lo x,y,z] x BI floats, the same bytes as the
// FP64 accumulators).  The pair is converted to FP64 (hi + lo) once, after
// the last tile.
// GUARD (PP_POS_GUARDED) reads hi/lo staged sources (STAGE_F32IX2) but streams and
// sums the hi parts only, recomputing with hi/lo separations the (target, tile)
// partials that hold a close pair (see guard_threshold): GUARD == 1 finds
// them by the largest rsqrt(s) of each tile, GUARD == 2 (spatially sorted
// sources, p.perm and p.boxes set) by each tile's bounding box (tile_boxed).
template <int T, int R, int TILE, int STAGES, int MINB, bool SMEM_ACC = false,
          bool WEIGHTED = false, bool SPLITPOS = false, int UNROLL = 2, bool KAHAN = false,
          int GUARD = 0>
__global__ void __launch_bounds__(T, MINB) force_f32x2_kernel(const ForceArgs p)
{
    static_assert(!(GUARD != 0 && SPLITPOS), "guarded staging sums the hi parts only");
    // the ring carries the lo parts too with hi/lo staging and with the box guard
    constexpr bool TWO = SPLITPOS || GUARD == 2;
    constexpr int BI = T * R;
    static_assert(TILE % 2 == 0, "sources are consumed in pairs");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar_full[STAGES], bar_empty[STAGES];
    __shared__ int s_abort, s_flag;

    const int tid = threadIdx.x;
    const int ib = blockIdx.x % p.nib;
    const int split = blockIdx.x / p.nib;
    const int i0 = ib * BI;
    const int j0 = split * p.jchunk;
    const int j1 = min(j0 + p.jchunk, p.npad);
    const int ntiles = (j1 - j0) / TILE;

    float4 *ring = reinterpret_cast<float4 *>(smem_raw);
    Ring<float4, TILE, STAGES, TWO> rg{ring, TWO ? ring + STAGES * TILE : nullptr,
                                            bar_full, bar_empty};
    // FP64 accumulators in shared memory follow the tile ring(s): [3][BI]
    double *sacc = reinterpret_cast<double *>(
        smem_raw + (size_t)STAGES * TILE * sizeof(float4) * (TWO ? 2 : 1));
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_empty[s], T / 32);
        }
        s_abort = 0;
        fence_barrier_init();
    }
    float *skah = reinterpret_cast<float *>(sacc);  // KAHAN && SMEM_ACC: [6][BI]
    if (SMEM_ACC) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (KAHAN) {
#pragma unroll
                for (int c = 0; c < 6; ++c) skah[c * BI + r * T + tid] = 0.f;
            } else {
                sacc[r * T + tid] = sacc[BI + r * T + tid] = sacc[2 * BI + r * T + tid] = 0.0;
            }
        }
    }
    __syncthreads();

    const float *srcf = static_cast<const float *>(p.src);
    f2_t X[R], Y[R], Z[R], XL[R], YL[R], ZL[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = i0 + r * T + tid;
        float x = -1e18f, y = -1e18f, z = -1e18f;  // targets past n: far from everything
        float xl = 0.f, yl = 0.f, zl = 0.f;
        if (i < p.n) {
            const float *q = srcf + 8 * (size_t)(i >> 1) + (i & 1);
            x = q[0];
            y = q[2];
            z = q[4];
            if (SPLITPOS) {
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
    }
    double ax64[R], ay64[R], az64[R];
#pragma unroll
    for (int r = 0; r < R; ++r) ax64[r] = ay64[r] = az64[r] = 0.0;
    float kh[KAHAN && !SMEM_ACC ? 6 * R : 1];  // register compensated pairs
#pragma unroll
    for (int c = 0; c < (KAHAN && !SMEM_ACC ? 6 * R : 1); ++c) kh[c] = 0.f;
    const f2_t EPS2 = f2_pack(p.eps2f, p.eps2f);
    // GUARD: close-pair threshold per target; the lo parts live 4 npad floats
    // after the hi parts
    float thr[R];
    if (GUARD != 0) guard_thresholds<T, R>(X, Y, Z, i0, p.n, thr);
    const float *glo = srcf + 4 * (size_t)p.npad;

    int issued = 0, seen = 0;
    const bool ok = run_tiles<float4, T, TILE, STAGES, TWO>(
        p, rg, j0, ntiles, issued, seen, [&](const float4 *tile, const float4 *tlo, int jfirst) {
            float3 fg[R];
            if (GUARD == 1) {
                tile_guarded<T, R, BI, TILE, WEIGHTED, UNROLL>(tile, jfirst, i0, p.n, glo, X, Y, Z,
                                                              thr, EPS2, p.eps2f, fg);
            } else if (GUARD == 2) {
                tile_boxed<T, R, BI, TILE, WEIGHTED, UNROLL>(tile, tlo, jfirst, i0, p.n, glo,
                                                            p.boxes + 2 * (jfirst / TILE), X, Y,
                                                            Z, thr, EPS2, p.eps2f, fg);
            } else {
                f2_t AX[R], AY[R], AZ[R];
                float MS[R];
                tile_packed<R, TILE, WEIGHTED, SPLITPOS, UNROLL>(tile, tlo, X, Y, Z, XL, YL, ZL,
                                                                 EPS2, AX, AY, AZ, MS);
#pragma unroll
                for (int r = 0; r < R; ++r)
                    fg[r] = tile_partial<TILE, WEIGHTED, SPLITPOS>(AX[r], AY[r], AZ[r], tile, tlo,
                                                                   X[r], Y[r], Z[r], XL[r], YL[r],
                                                                   ZL[r], p.eps2f);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float3 f = fg[r];
                const float fx = f.x, fy = f.y, fz = f.z;
                if (KAHAN) {
                    const float fc[3] = {fx, fy, fz};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float hs, e;
                        if (SMEM_ACC) {
                            float &hi = skah[c * BI + r * T + tid];
                            float &lo = skah[(3 + c) * BI + r * T + tid];
                            two_sum(hi, fc[c], hs, e);
                            hi = hs;
                            lo = __fadd_rn(lo, e);
                        } else {
                            two_sum(kh[6 * r + c], fc[c], hs, e);
                            kh[6 * r + c] = hs;
                            kh[6 * r + 3 + c] = __fadd_rn(kh[6 * r + 3 + c], e);
                        }
                    }
                } else if (SMEM_ACC) {
                    sacc[r * T + tid] += (double)fx;
                    sacc[BI + r * T + tid] += (double)fy;
                    sacc[2 * BI + r * T + tid] += (double)fz;
                } else {
                    ax64[r] += (double)fx;
                    ay64[r] += (double)fy;
                    az64[r] += (double)fz;
                }
            }
        });
    if (!ok) {
        s_abort = 1;
        atomicOr(p.err, 1);
    }
    __syncthreads();
    if (s_abort) {
        ring_drain(p, rg, issued, seen, ntiles);
        return;
    }
    if (KAHAN) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            double v[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                v[c] = SMEM_ACC ? (double)skah[c * BI + r * T + tid] +
                                      (double)skah[(3 + c) * BI + r * T + tid]
                                : (double)kh[6 * r + c] + (double)kh[6 * r + 3 + c];
            ax64[r] = v[0];
            ay64[r] = v[1];
            az64[r] = v[2];
        }
    } else if (SMEM_ACC) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            ax64[r] = sacc[r * T + tid];
            ay64[r] = sacc[BI + r * T + tid];
            az64[r] = sacc[2 * BI + r * T + tid];
        }
    }
    if (p.nsplit > 1) {
        if (!split_publish<T, R>(p, ib, split, ax64, ay64, az64, 3, &s_flag)) return;
        split_gather<T, R>(p, ib, ax64, ay64, az64, 3);
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        finish_particle<(SPLITPOS || GUARD != 0) ? STAGE_F32IX2 : STAGE_F32I>(p, i0 + r * T + tid,
                                                                         ax64[r], ay64[r], az64[r]);
}


// ---- j-split reduced through distributed shared memory -----------------------
// A thread-block cluster of CL CTAs owns one block of BI targets; CTA rank q of
// the cluster sums the q-th of CL source chunks into its shared-memory FP64
// accumulators.  After a cluster barrier, rank 0 adds the CL partial sums from
// its peers' shared memory in the fixed order q = 0..CL-1 (ld.shared::cluster)
// and runs the epilogue; a second barrier keeps the peers' shared memory alive
// until rank 0 has read it.  No global partials, fences or tickets: the
// reduction costs two cluster barriers and CL distributed-shared-memory reads
// per value, which shortens the per-step latency chain at small N.
template <int T, int R, int TILE, int STAGES, int MINB, int CL>
__global__ void __launch_bounds__(T, MINB) force_f32x2_cluster_kernel(const ForceArgs p)
{
    constexpr int BI = T * R;
    static_assert(TILE % 2 == 0, "sources are consumed in pairs");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t bar_full[STAGES], bar_empty[STAGES];
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int rank = (int)cluster_ctarank();        // == blockIdx.x % CL
    const int ib = blockIdx.x / CL;
    const int i0 = ib * BI;
    const int j0 = rank * p.jchunk;
    const int j1 = min(j0 + p.jchunk, p.npad);
    const int ntiles = j1 > j0 ? (j1 - j0) / TILE : 0;

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
#pragma unroll
    for (int r = 0; r < R; ++r)
        sacc[r * T + tid] = sacc[BI + r * T + tid] = sacc[2 * BI + r * T + tid] = 0.0;
    __syncthreads();

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
    }
    const f2_t EPS2 = f2_pack(p.eps2f, p.eps2f);
    int issued = 0, seen = 0;
    const bool ok = run_tiles<float4, T, TILE, STAGES, false>(
        p, rg, j0, ntiles, issued, seen, [&](const float4 *tile, const float4 *, int) {
            f2_t AX[R], AY[R], AZ[R];
            float MS[R];
            tile_packed<R, TILE, false, false, 2>(tile, nullptr, X, Y, Z, X, Y, Z, EPS2, AX, AY,
                                                  AZ, MS);
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
        });
    if (!ok) {
        s_abort = 1;
        atomicOr(p.err, 1);
    }
    __syncthreads();
    if (s_abort) ring_drain(p, rg, issued, seen, ntiles);
    cluster_sync();  // every CTA's partials (and abort flag) are visible to rank 0
    if (rank == 0) {
        int any_abort = 0;
        for (int q = 0; q < CL; ++q) any_abort |= ld_peer_s32(peer_smem(&s_abort, (uint32_t)q));
        if (!any_abort) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                double t[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const uint32_t a0 = peer_smem(&sacc[c * BI + r * T + tid], 0);
                    double acc = 0.0;
                    for (int q = 0; q < CL; ++q) {
                        // the same offset in CTA q: shared windows of a cluster are laid out
                        // by rank, so map each peer explicitly
                        acc += ld_peer_f64(q == 0 ? a0 : peer_smem(&sacc[c * BI + r * T + tid],
                                                                   (uint32_t)q));
                    }
                    t[c] = acc;
                }
                finish_particle<STAGE_F32I>(p, i0 + r * T + tid, t[0], t[1], t[2]);
            }
        }
    }
    cluster_sync();  // keep every CTA's shared memory alive until rank 0 has read it
}

}  // namespace ppk
