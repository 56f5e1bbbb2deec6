// pp_resident.cu -- small-N time stepping with every step of a pp_step call in
// one cooperative launch: the Eq. B/E force sum and the Eq. G/H push of step
// n+1 follow those of step n inside the same kernel, instead of one launch (and
// one j-split round trip through global memory) per step.
//
// At small N a step of the per-launch kernels is bound by latency, not by the
// FP32 pipe: CTA start-up, the first bulk copy, the partial-sum publication
// and gather, and the launch itself cost more than the 11 FP32 lane
// operations per pair.  Here each CTA keeps the whole staged source array in
// shared memory, owns BT targets (BT even), and splits the sources of each
// target over Q threads; the push runs one (component, target) item per
// thread, which keeps that item's FP64 r, v, a in registers for the whole
// launch.  The decomposition depends only on N and the SM count, so results
// are bitwise reproducible on a given device.
//
// Steps are separated by a grid-wide barrier: after its push a CTA arrives on
// one counter (release reduction); at the next step thread 0 waits (acquire
// loads, bounded) until every CTA has arrived and then issues the copy of the
// whole staged source array into shared memory as kResChunks 1D bulk copies
// (TMA) on one mbarrier, which every thread waits on (bounded).  (Tried and
// dropped: a flag per CTA with each block or group of blocks copied as soon as
// its producer published it; the polling of ~150 flags per CTA cost more than
// the overlap gained, 15.7 against 10.7 us per step at N = 4096.)
//
// FP64 runs at a small fraction of the FP32 rate on this GPU, so the sums stay
// in compensated FP32 (TwoSum) until each (component, target) item's final
// value: a thread's partial over its sources is an FP32 (hi, lo) pair, the Q
// pairs of an item are added with TwoSum in a fixed order, and only the result
// and the Eq. G/H push are FP64.
#include "pp_internal.h"

namespace ppk {

namespace {

constexpr int kResFold = 512;   // sources per FP32 partial before the compensated fold
constexpr int kResChunks = 8;   // bulk copies per step
// Floor on s = |d|^2 + eps^2 (staged units): the self pair (d = 0 exactly)
// then contributes rsqrt(s)^3 * 0 = 0 without a per-pair test, and for every
// separation the FP32 staging resolves (|d| > 1e-8 L0) the floor changes s by
// less than one FP32 rounding.  rsqrt(1e-24)^3 = 1e36 stays finite.
constexpr float kSelfFloor = 1e-24f;

// Arrive on the grid-barrier counter (release: this CTA's earlier writes, made
// visible to thread 0 by the CTA barrier before the call, are published).
__device__ __forceinline__ void grid_arrive(unsigned *bar)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
}

// Wait (bounded) until the counter reaches target; acquire ordering on success.
__device__ __forceinline__ bool grid_wait(const unsigned *bar, unsigned target, uint64_t limit_ns)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
    if (v >= target) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
        if (v >= target) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// Order this thread's generic-proxy view of memory (the acquired barrier and the
// data it publishes) before its following async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async;" ::: "memory");
}

// hi + lo += x, compensated (TwoSum on hi, errors collected in lo).
__device__ __forceinline__ void comp_add(float &hi, float &lo, float x)
{
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo = __fadd_rn(lo, e);
}

// One component of the MODE_STEP epilogue (finish_particle, component-wise),
// on state held in registers: a_{n+1} from the sum, Eq. G as staged, Eq. H,
// and the staged coordinate of the next Eq. G (with SPLIT its hi and lo
// parts).  Component 0 also writes the weight slot (w_i / W with per-particle
// weights, else 1).
template <bool W, bool SPLIT>
__device__ __forceinline__ void push_component(const ForceArgs &p, int i, int c, double cc,
                                               double sum, double &r, double &v, double &a,
                                               void *dst)
{
    const double an = p.cscale * sum;
    const double r1 = drift(r, v, a, p.dt, p.half_dt2);   // Eq. G (as staged)
    const double v1 = kick(v, a, an, p.half_dt);          // Eq. H
    r = r1;
    v = v1;
    a = an;
    const double rn = drift(r1, v1, an, p.dt, p.half_dt2);   // next Eq. G, staged only
    float *f = static_cast<float *>(dst) + 8 * (size_t)(i >> 1) + (i & 1);
    const double pc = staged_coord(rn, cc, p.inv_l0);
    const float hi = __double2float_rn(pc);
    f[2 * c] = hi;
    if (c == 0) f[6] = W ? p.wrel[i] : 1.0f;
    if (SPLIT) {   // lo parts in the same layout, 4 npad floats further on
        float *fl = f + 4 * (size_t)p.npad;
        fl[2 * c] = __double2float_rn(pc - (double)hi);
        if (c == 0) fl[6] = 0.0f;
    }
}

// W: per-particle weights, each pair term multiplied by the source's staged
// weight ratio w_j / W (one more f32x2 multiply per two pairs).
// SPLIT: hi/lo staged positions (STAGE_F32IX2): shared memory holds both
// parts, and each separation is (hi_i - hi_j) + (lo_i - lo_j).
template <int NT, bool W, bool SPLIT>
__global__ void __launch_bounds__(NT, 1)
    force_resident_kernel(const ForceArgs p, const ResidentArgs ra)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *sj4 = reinterpret_cast<float4 *>(smem_raw);   // staged sources, interleaved pairs
    const float *sj = reinterpret_cast<const float *>(smem_raw);
    constexpr int NPARTS = SPLIT ? 2 : 1;                  // hi (and lo) copies, npad each
    // per-thread partial sums: [hi x, y, z][lo x, y, z] x NT floats
    float *part = reinterpret_cast<float *>(smem_raw + (size_t)NPARTS * p.npad * sizeof(float4));
    __shared__ uint64_t s_bar;   // completion of one step's source copies
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int tl = tid % ra.bt, qi = tid / ra.bt;
    const int i = blockIdx.x * ra.bt + tl;
    const bool work = qi < ra.q && i < p.n;
    const int j0 = min(qi * ra.chunk, ra.nsrc), j1 = min(j0 + ra.chunk, ra.nsrc);
    const float eps2 = fmaxf(p.eps2f, kSelfFloor);
    const f2_t EPS2 = f2_pack(eps2, eps2);
    const int nblk = gridDim.x;

    // Each (component, target) item of the CTA belongs to one thread for the
    // whole launch (3 BT <= threads): that thread alone reads and writes the
    // item's r, v, a, so it keeps them in registers and stores them once at
    // the end.
    const int oc = tid / ra.bt, oti = tid - oc * ra.bt;
    const int oi = blockIdx.x * ra.bt + oti;
    const bool owner = tid < 3 * ra.bt && oi < p.n;
    double *const rc = oc == 0 ? p.r[0] : oc == 1 ? p.r[1] : p.r[2];
    double *const vc = oc == 0 ? p.v[0] : oc == 1 ? p.v[1] : p.v[2];
    double *const ac = oc == 0 ? p.a[0] : oc == 1 ? p.a[1] : p.a[2];
    const double occ = oc == 0 ? p.cx : oc == 1 ? p.cy : p.cz;
    double r_o = 0.0, v_o = 0.0, a_o = 0.0;
    if (owner) {
        r_o = rc[oi];
        v_o = vc[oi];
        a_o = ac[oi];
    }
    if (tid == 0) {
        mbar_init(&s_bar, 1);
        s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();

    for (int s = 0; s < ra.nsteps; ++s) {
        const int par = (ra.parity0 + s) & 1;
        const float4 *src = static_cast<const float4 *>(par ? ra.stage[1] : ra.stage[0]);
        // Copy phase: once every CTA has pushed step s - 1 (at s = 0 the sources
        // were staged before the launch), thread 0 copies the staged array into
        // shared memory in kResChunks bulk copies.  If the barrier wait runs out,
        // the copies are issued all the same (of stale data; the step is void), so
        // that the phase completes before the CTA gives up.
        if (tid == 0) {
            if (s > 0 && !grid_wait(ra.flags, nblk * (unsigned)s, p.timeout_ns)) {
                s_abort = 1;
                atomicOr(p.err, 1);
            }
            fence_proxy_async();
            mbar_arrive_expect_tx(&s_bar, 16u * (uint32_t)ra.nsrc * NPARTS);
            const int per = (ra.nsrc / 2 + kResChunks - 1) / kResChunks * 2;   // even
            for (int c0 = 0; c0 < ra.nsrc; c0 += per) {
                const uint32_t bytes = 16u * (uint32_t)min(per, ra.nsrc - c0);
                bulk_g2s(sj4 + c0, src + c0, bytes, &s_bar);
                if (SPLIT) bulk_g2s(sj4 + p.npad + c0, src + p.npad + c0, bytes, &s_bar);
            }
        }
        if (!mbar_wait_bounded(&s_bar, (uint32_t)(s & 1), p.timeout_ns)) {
            s_abort = 1;
            atomicOr(p.err, 1);
            mbar_wait_bounded(&s_bar, (uint32_t)(s & 1), p.timeout_ns);   // copies in flight
        }
        __syncthreads();
        if (s_abort) return;   // the state is left unspecified (the call reports the timeout)

        float hx = 0.f, hy = 0.f, hz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
        if (work) {
            const float *q = sj + 8 * (i >> 1) + (i & 1);
            const f2_t X = f2_pack(q[0], q[0]), Y = f2_pack(q[2], q[2]), Z = f2_pack(q[4], q[4]);
            const float *ql = q + 4 * (size_t)p.npad;
            const f2_t XL = SPLIT ? f2_pack(ql[0], ql[0]) : 0ull;
            const f2_t YL = SPLIT ? f2_pack(ql[2], ql[2]) : 0ull;
            const f2_t ZL = SPLIT ? f2_pack(ql[4], ql[4]) : 0ull;
            for (int t0 = j0; t0 < j1; t0 += kResFold) {
                const int t1 = min(t0 + kResFold, j1);
                f2_t AX = 0ull, AY = 0ull, AZ = 0ull;
#pragma unroll 4
                for (int j = t0; j < t1; j += 2) {
                    const float4 a = sj4[j];       // x_j x_j+1 y_j y_j+1
                    const float4 b = sj4[j + 1];   // z_j z_j+1 w_j w_j+1
                    f2_t DX = f2_sub(X, f2_pack(a.x, a.y));
                    f2_t DY = f2_sub(Y, f2_pack(a.z, a.w));
                    f2_t DZ = f2_sub(Z, f2_pack(b.x, b.y));
                    if (SPLIT) {
                        const float4 al = sj4[p.npad + j], bl = sj4[p.npad + j + 1];
                        DX = f2_add(DX, f2_sub(XL, f2_pack(al.x, al.y)));
                        DY = f2_add(DY, f2_sub(YL, f2_pack(al.z, al.w)));
                        DZ = f2_add(DZ, f2_sub(ZL, f2_pack(bl.x, bl.y)));
                    }
                    const f2_t S = f2_fma(DZ, DZ, f2_fma(DY, DY, f2_fma(DX, DX, EPS2)));
                    float s0, s1;
                    f2_unpack(S, s0, s1);
                    const f2_t INV = f2_pack(rsqrt_sfu(s0), rsqrt_sfu(s1));
                    const f2_t INV3 = W ? f2_mul(f2_mul(f2_mul(INV, INV), INV), f2_pack(b.z, b.w))
                                        : f2_mul(f2_mul(INV, INV), INV);
                    AX = f2_fma(INV3, DX, AX);
                    AY = f2_fma(INV3, DY, AY);
                    AZ = f2_fma(INV3, DZ, AZ);
                }
                float x0, x1, y0, y1, z0, z1;
                f2_unpack(AX, x0, x1);
                f2_unpack(AY, y0, y1);
                f2_unpack(AZ, z0, z1);
                comp_add(hx, lx, x0 + x1);
                comp_add(hy, ly, y0 + y1);
                comp_add(hz, lz, z0 + z1);
            }
        }
        part[tid] = hx;
        part[NT + tid] = hy;
        part[2 * NT + tid] = hz;
        part[3 * NT + tid] = lx;
        part[4 * NT + tid] = ly;
        part[5 * NT + tid] = lz;
        __syncthreads();
        // Epilogue, one (component, target) item per thread: the Q partials of
        // the item added with TwoSum in a fixed order, then FP64 for the push.
        if (owner) {
            float h = 0.f, l = 0.f;
            for (int k = 0; k < ra.q; ++k) {
                const int t = k * ra.bt + oti;
                comp_add(h, l, part[oc * NT + t]);
                l = __fadd_rn(l, part[(3 + oc) * NT + t]);
            }
            const double sum = (double)h + (double)l;
            push_component<W, SPLIT>(p, oi, oc, occ, sum, r_o, v_o, a_o,
                                     par ? ra.stage[0] : ra.stage[1]);
        }
        __syncthreads();   // every owner's staged writes of step s are done
        // arrive for step s (test hook: CTA 0 withholds its first arrival, so every
        // CTA's wait runs out)
        if (tid == 0 && !(p.skip_copy && blockIdx.x == 0 && s == 0)) grid_arrive(ra.flags);
    }
    if (p.skip_copy && tid == 0) {
        // test hook with a single step: wait for the last arrivals too
        if (!grid_wait(ra.flags, nblk * (unsigned)ra.nsteps, p.timeout_ns)) atomicOr(p.err, 1);
    }
    if (owner) {
        rc[oi] = r_o;
        vc[oi] = v_o;
        ac[oi] = a_o;
    }
}

template <int NT>
const void *resident_fn_nt(int form)
{
    switch (form) {
    case RES_WEIGHTED: return reinterpret_cast<const void *>(&force_resident_kernel<NT, true, false>);
    case RES_SPLIT: return reinterpret_cast<const void *>(&force_resident_kernel<NT, false, true>);
    case RES_KAHAN:   // the resident kernel folds compensated in every form
        return reinterpret_cast<const void *>(&force_resident_kernel<NT, false, false>);
    default: return reinterpret_cast<const void *>(&force_resident_kernel<NT, false, false>);
    }
}

const void *resident_fn(int threads, int form)
{
    return threads == 512 ? resident_fn_nt<512>(form) : resident_fn_nt<256>(form);
}

}  // namespace

size_t resident_smem(int npad, int threads, int form)
{
    return (size_t)(form == RES_SPLIT ? 2 : 1) * npad * sizeof(float4) +
           6 * (size_t)threads * sizeof(float);
}

cudaError_t resident_configure(int npad_single, int npad_split)
{
    for (int threads : {256, 512})
        for (int form : {RES_PLAIN, RES_WEIGHTED, RES_SPLIT, RES_KAHAN}) {
            const int npad = form == RES_SPLIT ? npad_split : npad_single;
            cudaError_t e = cudaFuncSetAttribute(resident_fn(threads, form),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)resident_smem(npad, threads, form));
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

cudaError_t resident_occupancy(int npad, int threads, int form, int *blocks_per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, resident_fn(threads, form),
                                                         threads,
                                                         resident_smem(npad, threads, form));
}

cudaError_t launch_resident(const ForceArgs &a, const ResidentArgs &ra, int grid, int threads,
                            int form, cudaStream_t stream)
{
    ForceArgs ca = a;
    ResidentArgs cr = ra;
    void *args[] = {&ca, &cr};
    return cudaLaunchCooperativeKernel(resident_fn(threads, form), dim3(grid), dim3(threads), args,
                                       resident_smem(a.npad, threads, form), stream);
}

}  // namespace ppk
