// pp_resident.cu -- small-N time stepping with every step of a pp_step call in
// one cooperative launch: the Eq. B/E force sum and the Eq. G/H push of step
// n+1 follow those of step n inside the same kernel, separated by a grid-wide
// barrier, instead of one launch (and one j-split round trip through global
// memory) per step.
//
// At small N a step of the per-launch kernels is bound by latency, not by the
// FP32 pipe: CTA start-up, the first bulk copy, the partial-sum publication
// and gather, and the launch itself cost more than the 11 FP32 lane
// operations per pair.  Here each CTA keeps the whole staged source array in
// shared memory (loaded once per step from L2), owns BT targets, and splits
// the sources of each target over Q threads; the Q FP64 partials of a target
// are added in a fixed order, and the push runs one (component, target) item
// per thread, which keeps that item's FP64 r, v, a in registers for the whole
// launch.  The decomposition depends only on N and the SM count, so
// results are bitwise reproducible on a given device.
#include "pp_internal.h"

namespace ppk {

namespace {

constexpr int kResFold = 512;   // sources per FP32 partial before the FP64 fold
// Floor on s = |d|^2 + eps^2 (staged units): the self pair (d = 0 exactly)
// then contributes rsqrt(s)^3 * 0 = 0 without a per-pair test, and for every
// separation the FP32 staging resolves (|d| > 1e-8 L0) the floor changes s by
// less than one FP32 rounding.  rsqrt(1e-24)^3 = 1e36 stays finite.
constexpr float kSelfFloor = 1e-24f;

// Grid-wide barrier of a cooperative launch.  Every CTA arrives once per
// barrier; `target` is the arrival count that completes this one.  Thread 0
// waits at most limit_ns; the verdict is shared with the CTA.
__device__ bool grid_sync_bounded(unsigned *bar, unsigned target, uint64_t limit_ns, bool arrive,
                                  int *s_flag)
{
    __syncthreads();   // the CTA's step writes happen before thread 0's release
    if (threadIdx.x == 0) {
        int ok = 1;
        if (arrive) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        const uint64_t t0 = globaltimer_ns();
        for (;;) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
            if (v >= target) break;
            if (globaltimer_ns() - t0 > limit_ns) {
                ok = 0;
                break;
            }
        }
        *s_flag = ok;
    }
    __syncthreads();   // ... and before every thread's reads of the next step
    return *s_flag != 0;
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
// KAHAN (PP_ACC_KAHAN): a thread folds its FP32 tile partials into a
// compensated FP32 pair (TwoSum) instead of FP64; the threads' pairs are
// then added in FP64 in the fixed order, like the FP64-fold form.
template <int NT, bool W, bool SPLIT, bool KAHAN = false>
__global__ void __launch_bounds__(NT, 1)
    force_resident_kernel(const ForceArgs p, const ResidentArgs ra)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *sj4 = reinterpret_cast<float4 *>(smem_raw);   // staged sources, interleaved pairs
    const float *sj = reinterpret_cast<const float *>(smem_raw);
    constexpr int NPARTS = SPLIT ? 2 : 1;                  // hi (and lo) copies, npad each
    double *part =
        reinterpret_cast<double *>(smem_raw + (size_t)NPARTS * p.npad * sizeof(float4));
    __shared__ int s_flag;

    const int tid = threadIdx.x;
    const int tl = tid % ra.bt, qi = tid / ra.bt;
    const int i = blockIdx.x * ra.bt + tl;
    const bool work = qi < ra.q && i < p.n;
    const int j0 = min(qi * ra.chunk, ra.nsrc), j1 = min(j0 + ra.chunk, ra.nsrc);
    const float eps2 = fmaxf(p.eps2f, kSelfFloor);
    const f2_t EPS2 = f2_pack(eps2, eps2);

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

    for (int s = 0; s < ra.nsteps; ++s) {
        const int par = (ra.parity0 + s) & 1;
        // other CTAs wrote these entries during the previous step: read through L2
        const float4 *src = static_cast<const float4 *>(par ? ra.stage[1] : ra.stage[0]);
        for (int k = tid; k < ra.nsrc; k += NT) sj4[k] = __ldcg(src + k);
        if (SPLIT)
            for (int k = tid; k < ra.nsrc; k += NT) sj4[p.npad + k] = __ldcg(src + p.npad + k);
        __syncthreads();

        double sx = 0.0, sy = 0.0, sz = 0.0;
        float kh[3] = {0.f, 0.f, 0.f}, kl[3] = {0.f, 0.f, 0.f};   // KAHAN: hi, lo per component
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
                if (KAHAN) {
                    const float f[3] = {x0 + x1, y0 + y1, z0 + z1};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        float hs, e;
                        two_sum(kh[c], f[c], hs, e);
                        kh[c] = hs;
                        kl[c] = __fadd_rn(kl[c], e);
                    }
                } else {
                    sx += (double)(x0 + x1);
                    sy += (double)(y0 + y1);
                    sz += (double)(z0 + z1);
                }
            }
            if (KAHAN) {
                sx = (double)kh[0] + (double)kl[0];
                sy = (double)kh[1] + (double)kl[1];
                sz = (double)kh[2] + (double)kl[2];
            }
        }
        part[tid] = sx;
        part[NT + tid] = sy;
        part[2 * NT + tid] = sz;
        __syncthreads();
        // Epilogue, one (component, target) item per thread: the FP64 pipe runs
        // at a small fraction of the FP32 rate here, so the sums and the push are
        // spread over as many warps (and SM sub-partitions) as there are items.
        if (owner) {
            double sum = 0.0;
            for (int k = 0; k < ra.q; ++k) sum += part[oc * NT + k * ra.bt + oti];   // fixed order
            push_component<W, SPLIT>(p, oi, oc, occ, sum, r_o, v_o, a_o,
                                     par ? ra.stage[0] : ra.stage[1]);
        }
        if (s + 1 < ra.nsteps || p.skip_copy) {
            // test hook: CTA 0 withholds its first arrival, so every CTA's wait runs
            // out (the barrier is then taken after a last step too)
            const bool arrive = !(p.skip_copy && blockIdx.x == 0 && s == 0);
            if (!grid_sync_bounded(ra.bar, gridDim.x * (unsigned)(s + 1), p.timeout_ns, arrive,
                                   &s_flag)) {
                if (tid == 0) atomicOr(p.err, 1);
                return;   // the state is left unspecified (the call reports the timeout)
            }
        }
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
    case RES_KAHAN:
        return reinterpret_cast<const void *>(&force_resident_kernel<NT, false, false, true>);
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
           3 * (size_t)threads * sizeof(double);
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
