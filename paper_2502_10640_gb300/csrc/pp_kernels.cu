// pp_kernels.cu -- the table of compiled force-kernel variants and their launcher.
#include <cfloat>
#include <cmath>

#include "pp_internal.h"

namespace ppk {

namespace {

template <int T, int R, int TILE, int STAGES, int ACC, int MINB, bool SPLIT = false>
Variant make_f32(const char *name)
{
    return Variant{name, KIND_FORCE32, ACC, SPLIT ? STAGE_F32X2 : STAGE_F32, T, R, TILE, STAGES,
                   reinterpret_cast<const void *>(
                       &force_f32_kernel<T, R, TILE, STAGES, ACC, MINB, SPLIT>),
                   (size_t)STAGES * TILE * sizeof(float4) * (SPLIT ? 2 : 1), 0,
                   SPLIT ? POS_SPLIT : POS_SINGLE};
}

template <int T, int R, int TILE, int STAGES, int MINB, bool SMEM_ACC = false,
          bool WEIGHTED = false, bool SPLITPOS = false, int UNROLL = 2, bool KAHAN = false,
          int GUARD = 0>
Variant make_f32x2(const char *name)
{
    return Variant{name, WEIGHTED ? KIND_FORCE32W : KIND_FORCE32, KAHAN ? ACC_KAHAN : ACC_FP64FOLD,
                   (SPLITPOS || GUARD != 0) ? STAGE_F32IX2 : STAGE_F32I, T, R, TILE, STAGES,
                   reinterpret_cast<const void *>(
                       &force_f32x2_kernel<T, R, TILE, STAGES, MINB, SMEM_ACC, WEIGHTED, SPLITPOS,
                                           UNROLL, KAHAN, GUARD>),
                   (size_t)STAGES * TILE * sizeof(float4) * (SPLITPOS || GUARD == 2 ? 2 : 1) +
                       (SMEM_ACC ? (size_t)3 * T * R * sizeof(double) : 0),
                   0, GUARD != 0 ? POS_GUARDED : SPLITPOS ? POS_SPLIT : POS_SINGLE,
                   GUARD == 2 ? 1 : 0};
}

// Guarded staging: hi/lo staged, hi parts streamed, close-pair tiles recomputed.
template <int T, int R, int TILE, int STAGES, int MINB, bool SMEM_ACC = false,
          bool WEIGHTED = false, int UNROLL = 2, bool KAHAN = false>
Variant make_guard(const char *name)
{
    return make_f32x2<T, R, TILE, STAGES, MINB, SMEM_ACC, WEIGHTED, false, UNROLL, KAHAN, 1>(
        name);
}

// Guarded staging on spatially sorted sources: close tiles found by their
// bounding boxes (no test per pair); the ring carries hi and lo tiles.
template <int T, int R, int TILE, int STAGES, int MINB, bool SMEM_ACC = false,
          bool WEIGHTED = false, int UNROLL = 2, bool KAHAN = false>
Variant make_box_guard(const char *name)
{
    return make_f32x2<T, R, TILE, STAGES, MINB, SMEM_ACC, WEIGHTED, false, UNROLL, KAHAN, 2>(
        name);
}

template <int T, int R, int TILE, int STAGES, int MINB, int CL>
Variant make_cluster(const char *name)
{
    return Variant{name, KIND_FORCE32, ACC_FP64FOLD, STAGE_F32I, T, R, TILE, STAGES,
                   reinterpret_cast<const void *>(
                       &force_f32x2_cluster_kernel<T, R, TILE, STAGES, MINB, CL>),
                   (size_t)STAGES * TILE * sizeof(float4) + (size_t)3 * T * R * sizeof(double), CL,
                   POS_SINGLE};
}

template <int T, int R, int TILE, int STAGES>
Variant make_phi(const char *name)
{
    return Variant{name, KIND_PHI32, ACC_FP64FOLD, STAGE_F32, T, R, TILE, STAGES,
                   reinterpret_cast<const void *>(&phi_f32_kernel<T, R, TILE, STAGES>),
                   (size_t)STAGES * TILE * sizeof(float4), 0, POS_SINGLE};
}

template <int T, int R, int TILE, int STAGES>
Variant make_f64(const char *name)
{
    return Variant{name, KIND_FORCE64, ACC_FP64FULL, STAGE_F64, T, R, TILE, STAGES,
                   reinterpret_cast<const void *>(&force_f64_kernel<T, R, TILE, STAGES>),
                   (size_t)STAGES * TILE * sizeof(double4), 0, POS_SINGLE};
}

const Variant kVariants[] = {
    // scalar FP32 pair math (one source per instruction)
    make_f32<256, 4, 256, 4, ACC_FP64FOLD, 2>("f32.fold64.t256r4k256"),
    make_f32<128, 2, 128, 4, ACC_FP64FOLD, 4>("f32.fold64.t128r2k128"),
    make_f32<128, 1, 128, 4, ACC_FP64FOLD, 4>("f32.fold64.t128r1k128"),
    make_f32<256, 4, 256, 4, ACC_KAHAN, 2>("f32.kahan.t256r4k256"),
    make_f32<128, 2, 128, 4, ACC_KAHAN, 4>("f32.kahan.t128r2k128"),
    make_f32<256, 4, 256, 4, ACC_FP64FOLD, 2, true>("f32split.fold64.t256r4k256"),
    make_f32<128, 2, 128, 4, ACC_FP64FOLD, 4, true>("f32split.fold64.t128r2k128"),
    // packed f32x2 pair math (two sources per instruction)
    make_f32x2<256, 4, 256, 4, 2>("f32x2.fold64.t256r4k256"),
    make_f32x2<128, 2, 128, 4, 4>("f32x2.fold64.t128r2k128"),
    make_f32x2<256, 4, 512, 3, 2>("f32x2.fold64.t256r4k512"),
    make_f32x2<128, 4, 512, 3, 4, true>("f32x2.sfold64.t128r4k512m4"),
    make_f32x2<128, 4, 256, 4, 4, true>("f32x2.sfold64.t128r4k256m4"),
    make_f32x2<128, 4, 512, 3, 5, true>("f32x2.sfold64.t128r4k512m5"),
    make_f32x2<128, 2, 512, 3, 6, true>("f32x2.sfold64.t128r2k512m6"),
    make_f32x2<128, 4, 512, 3, 4, true, false, false, 1>("f32x2.sfold64.t128r4k512m4u1"),
    make_f32x2<128, 4, 1024, 2, 4, true, false, false, 1>("f32x2.sfold64.t128r4k1024s2m4u1"),
    make_f32x2<128, 4, 1024, 2, 4, true, false, false, 2>("f32x2.sfold64.t128r4k1024s2m4u2"),
    make_f32x2<64, 1, 128, 4, 8>("f32x2.fold64.t64r1k128"),
    make_f32x2<64, 2, 128, 4, 8>("f32x2.fold64.t64r2k128"),
    // packed pair math, tile partials folded into compensated FP32 pairs
    make_f32x2<128, 4, 512, 3, 4, true, false, false, 1, true>("f32x2.kahan.st128r4k512m4u1"),
    make_f32x2<128, 4, 512, 3, 4, true, false, false, 2, true>("f32x2.kahan.st128r4k512m4"),
    make_f32x2<128, 4, 1024, 2, 4, true, false, false, 2, true>("f32x2.kahan.st128r4k1024s2m4u2"),
    make_f32x2<128, 2, 128, 4, 4, false, false, false, 2, true>("f32x2.kahan.t128r2k128"),
    make_f32x2<64, 1, 128, 4, 8, false, false, false, 2, true>("f32x2.kahan.t64r1k128"),
    // j-split reduced through distributed shared memory of a thread-block cluster
    make_cluster<64, 1, 128, 4, 8, 8>("f32x2cl8.dsmem.t64r1k128"),
    make_cluster<64, 1, 128, 4, 8, 16>("f32x2cl16.dsmem.t64r1k128"),
    make_cluster<128, 1, 128, 4, 8, 16>("f32x2cl16.dsmem.t128r1k128"),
    make_cluster<128, 2, 128, 4, 4, 8>("f32x2cl8.dsmem.t128r2k128"),
    // packed pair math on hi/lo split positions
    make_f32x2<128, 2, 512, 3, 4, true, false, true>("f32x2split.sfold64.t128r2k512m4"),
    make_f32x2<128, 4, 256, 3, 4, true, false, true>("f32x2split.sfold64.t128r4k256m4"),
    make_f32x2<64, 1, 128, 4, 8, false, false, true>("f32x2split.fold64.t64r1k128"),
    // hi/lo split positions with the compensated FP32 fold
    make_f32x2<128, 2, 512, 3, 4, true, false, true, 2, true>("f32x2split.kahan.st128r2k512m4"),
    make_f32x2<128, 4, 256, 3, 4, true, false, true, 2, true>("f32x2split.kahan.st128r4k256m4"),
    make_f32x2<64, 1, 128, 4, 8, false, false, true, 2, true>("f32x2split.kahan.t64r1k128"),
    // hi/lo split positions with per-particle weights (FP64 fold)
    make_f32x2<128, 2, 512, 3, 4, true, true, true>("f32x2wsplit.sfold64.t128r2k512m4"),
    make_f32x2<128, 4, 256, 3, 4, true, true, true>("f32x2wsplit.sfold64.t128r4k256m4"),
    make_f32x2<64, 1, 128, 4, 8, false, true, true>("f32x2wsplit.fold64.t64r1k128"),
    // guarded staging: single-precision pair loop, close-pair tiles summed with hi/lo
    make_guard<128, 4, 1024, 2, 4, true, false, 1>("f32x2guard.sfold64.t128r4k1024s2m4u1"),
    make_guard<128, 4, 512, 3, 4, true, false, 1>("f32x2guard.sfold64.t128r4k512m4u1"),
    make_guard<128, 2, 128, 4, 4>("f32x2guard.fold64.t128r2k128"),
    make_guard<64, 1, 128, 4, 8>("f32x2guard.fold64.t64r1k128"),
    make_guard<128, 4, 512, 3, 4, true, false, 1, true>("f32x2guard.kahan.st128r4k512m4u1"),
    make_guard<128, 2, 128, 4, 4, false, false, 2, true>("f32x2guard.kahan.t128r2k128"),
    make_guard<64, 1, 128, 4, 8, false, false, 2, true>("f32x2guard.kahan.t64r1k128"),
    // guarded staging on spatially sorted sources (tile boxes instead of a test per pair)
    make_box_guard<128, 4, 512, 2, 4, true, false, 1>("f32x2bguard.sfold64.t128r4k512s2m4u1"),
    make_box_guard<128, 4, 512, 2, 4, true, false, 2>("f32x2bguard.sfold64.t128r4k512s2m4u2"),
    make_box_guard<128, 4, 256, 4, 4, true, false, 1>("f32x2bguard.sfold64.t128r4k256m4u1"),
    make_box_guard<128, 4, 256, 4, 4, true, false, 2>("f32x2bguard.sfold64.t128r4k256m4u2"),
    make_box_guard<128, 4, 512, 2, 4, true, false, 1, true>("f32x2bguard.kahan.st128r4k512s2m4u1"),
    make_box_guard<128, 4, 512, 2, 4, true, false, 2, true>("f32x2bguard.kahan.st128r4k512s2m4u2"),
    make_box_guard<128, 4, 512, 2, 4, true, true>("f32x2wbguard.sfold64.t128r4k512s2m4"),
    make_guard<128, 4, 512, 3, 4, true, true>("f32x2wguard.sfold64.t128r4k512m4"),
    make_guard<128, 2, 128, 4, 4, false, true>("f32x2wguard.fold64.t128r2k128"),
    make_guard<64, 1, 128, 4, 8, false, true>("f32x2wguard.fold64.t64r1k128"),
    // per-particle weights (sources scaled by w_j / W)
    make_f32x2<128, 4, 512, 3, 4, true, true>("f32x2w.sfold64.t128r4k512m4"),
    make_f32x2<128, 2, 128, 4, 4, false, true>("f32x2w.fold64.t128r2k128"),
    make_f32x2<64, 1, 128, 4, 8, false, true>("f32x2w.fold64.t64r1k128"),
    // potential (diagnostics) and all-FP64 comparison path
    make_phi<256, 2, 256, 4>("phi32.fold64.t256r2k256"),
    make_phi<128, 1, 128, 4>("phi32.fold64.t128r1k128"),
    make_f64<128, 2, 128, 3>("f64.full.t128r2k128"),
};

}  // namespace

const Variant *variants(int *count)
{
    *count = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
    return kVariants;
}

cudaError_t launch_variant(const Variant &v, const ForceArgs &a, int grid, cudaStream_t stream)
{
    static DeviceOnce smem_attr, cluster_attr;
    const int idx = (int)(&v - kVariants);
    cudaError_t e = smem_attr.run(idx, [&] {
        return cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    });
    if (e != cudaSuccess) return e;
    ForceArgs copy = a;
    void *args[] = {&copy};
    if (v.cluster <= 0) return cudaLaunchKernel(v.fn, dim3(grid), dim3(v.T), args, v.smem, stream);
    if (v.cluster > 8) {
        e = cluster_attr.run(idx, [&] {
            return cudaFuncSetAttribute(v.fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        });
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(v.T);
    cfg.dynamicSmemBytes = v.smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)v.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, v.fn, args);
}

}  // namespace ppk
