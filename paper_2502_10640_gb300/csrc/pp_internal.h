// pp_internal.h -- host-side interface between the C ABI layer and the
// kernel translation unit.  Not installed; not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <mutex>
#include <set>
#include <utility>

#include <nvtx3/nvToolsExt.h>

#include "pp_force.cuh"

namespace ppk {

// NVTX range for the duration of a scope (visible under Nsight tools; a no-op
// otherwise).  Marks the host-side phases: load, step blocks, fields,
// diagnostics, autotuning, batch steps.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// CODATA 2018 (SI).  The paper prints no constants.
constexpr double kE = 1.602176634e-19;      // elementary charge, C (exact)
constexpr double kMe = 9.1093837015e-31;    // electron mass, kg
constexpr double kEps0 = 8.8541878128e-12;  // vacuum permittivity, F/m
constexpr double kPi = 3.14159265358979323846;
constexpr double kCoulomb = 1.0 / (4.0 * kPi * kEps0);  // 1/(4 pi eps0), Eq. A

// Staged arrays are padded to a multiple of this many entries.
constexpr int kPad = 1024;

enum Kind : int { KIND_FORCE32 = 0, KIND_PHI32 = 1, KIND_FORCE64 = 2, KIND_FORCE32W = 3 };

struct Variant {
    const char *name;
    int kind;
    int acc;      // Acc
    int stage;    // StageKind of the sources it reads
    int T, R, tile, stages;
    const void *fn;
    size_t smem;  // dynamic shared memory bytes
    int cluster;  // CTAs per thread-block cluster (0: no cluster; the j-split is then S
                  // global-partial chunks chosen by the planner, else exactly `cluster`)
    int positions;  // PosKind
    int order = 0;  // 1: the pass sorts the staged sources in space first (tile-box guard)
};

// One-time set-up per (device, key), e.g. a kernel's shared-memory attribute:
// CUDA function attributes are per device, so the set-up runs once on every
// device that uses the kernel.  Thread-safe; a failed set-up is retried.
class DeviceOnce {
public:
    template <class F>
    cudaError_t run(int key, F &&setup)
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return cudaGetLastError();
        {
            std::lock_guard<std::mutex> g(mu_);
            if (done_.count({dev, key})) return cudaSuccess;
        }
        const cudaError_t e = setup();
        if (e == cudaSuccess) {
            std::lock_guard<std::mutex> g(mu_);
            done_.insert({dev, key});
        }
        return e;
    }

private:
    std::mutex mu_;
    std::set<std::pair<int, int>> done_;
};

// Record the message pp_last_error() returns on this thread.
void set_last_error(const char *msg);

// Table of compiled force-kernel variants.
const Variant *variants(int *count);

// Launch one variant with the given arguments on `stream`.
cudaError_t launch_variant(const Variant &v, const ForceArgs &a, int grid, cudaStream_t stream);

// Resident small-N stepping: all steps of one pp_step call in one cooperative
// launch (pp_resident.cu).  The staged source array lives in each CTA's
// shared memory.
struct ResidentArgs {
    void *stage[2];   // ping-pong staging (STAGE_F32I or STAGE_F32IX2), npad entries each
    int parity0;      // buffer holding the staged r_{n+1} at the first step
    int nsteps;
    int bt;           // targets per CTA (grid = ceil(n / bt))
    int q;            // threads (source chunks) per target, bt * q <= threads per CTA
    int chunk;        // sources per chunk, even
    int nsrc;         // sources summed: n rounded up to even (the odd tail is padding)
    unsigned *flags;  // [0]: grid-barrier arrival counter, zero at launch
};
// threads per CTA: 256 or 512 (the compiled instantiations).  Forms: plain
// (single staging, equal weights), per-particle weights, hi/lo staging
// (STAGE_F32IX2, both parts in shared memory); the compensated-fold form runs
// the plain kernel (the resident kernel folds compensated in every form).
// bt (targets per CTA) is even.
enum ResidentForm : int { RES_PLAIN = 0, RES_WEIGHTED = 1, RES_SPLIT = 2, RES_KAHAN = 3 };
size_t resident_smem(int npad, int threads, int form);
cudaError_t resident_configure(int npad_single, int npad_split);
cudaError_t resident_occupancy(int npad, int threads, int form, int *blocks_per_sm);
cudaError_t launch_resident(const ForceArgs &a, const ResidentArgs &ra, int grid, int threads,
                            int form, cudaStream_t stream);

// Deterministic O(N) kernels.
// AoS [n][3] -> three SoA arrays; sets *bad to 1 if any input is not finite.
cudaError_t launch_aos_to_soa(const double *in, int n, double *x, double *y, double *z, int *bad,
                              cudaStream_t s);
cudaError_t launch_soa_to_aos(const double *x, const double *y, const double *z, int n,
                              double *out, cudaStream_t s);
// Stage FP64 positions into float4 (or double4) sources; entries n..npad-1
// become padding (far away, weight 0).
// wrel: per-particle weight ratios written into the weight slot (null: 1).
cudaError_t launch_stage(const double *x, const double *y, const double *z, int n, int npad,
                         void *dst, int stage_kind, double cx, double cy, double cz, double inv_l0,
                         cudaStream_t s, const float *wrel = nullptr);

// Weight ratios wrel[i] = (float)(w[i] / w_ref); sets *bad if a weight is not finite or <= 0.
cudaError_t launch_weights(const double *w, int n, double w_ref, float *wrel, int *bad,
                           cudaStream_t s);

// Write the padding entries n..npad-1 of a staging buffer (far away, weight 0).
cudaError_t launch_fill_padding(void *dst, int n, int npad, int stage_kind, cudaStream_t s);

// Stage the next positions of Eq. G, drift(r, v, a), exactly as the step
// epilogue stages them (used after a state is restored).
cudaError_t launch_stage_drift(double *const r[3], double *const v[3], double *const a[3], int n,
                               int npad, void *dst, int stage_kind, double dt, double half_dt2,
                               double cx, double cy, double cz, double inv_l0, cudaStream_t s,
                               const float *wrel = nullptr);

// Whole-state import (pp_set_state): [n][3] r, v, a (device-accessible) ->
// SoA state + *bad flag + drift(r, v, a) staged into dst with its padding.
cudaError_t launch_import_state(const double *pos, const double *vel, const double *acc, int n,
                                int npad, double *const r[3], double *const v[3],
                                double *const a[3], void *dst, int kind, double dt,
                                double half_dt2, double cx, double cy, double cz, double inv_l0,
                                const float *wrel, int *bad, cudaStream_t s);
// Whole-state export (pp_get_state): SoA r, v, a -> [n][3] device-accessible
// arrays; null outputs are skipped.
cudaError_t launch_export_state(double *const r[3], double *const v[3], double *const a[3], int n,
                                double *pos, double *vel, double *acc, cudaStream_t s);

// Moments over n particles in a fixed reduction order.
//  pass 0: sums of x, y, z                                     -> out[0..2]
//  pass 1: sum |r-c|^2, sum w|v|^2, sum w vx, w vy, w vz, sum x^2,
//          sum vx^2, sum x vx (out[0..7]); max x, max vx (out[10], out[11])
//  pass 2: sum of w times the values in x (one array)          -> out[0]
// wts: per-particle weights, or null for weight 1.
constexpr int kMomSlots = 12;
constexpr int kMomBlocks = 240;
cudaError_t launch_moments(int pass, int n, const double *x, const double *y, const double *z,
                           const double *vx, const double *vy, const double *vz, double cx,
                           double cy, double cz, double *block_partials, double *out,
                           cudaStream_t s, const double *wts = nullptr);

// Sums of |a - b|^2 and |b|^2 over n3 doubles: partials[2k], partials[2k+1] for
// k < kDiffBlocks (a fixed reduction order; the host adds the blocks in order).
constexpr int kDiffBlocks = 120;
// Spatial order of staged sources (tile-box guard, pp_order.cu): one device
// workspace per context, carved into the sort keys (a power of two >= npad),
// the sorted hi/lo copy of the staged array (STAGE_F32IX2), the tile boxes,
// the permutation (sorted index -> particle index) and the bounding box.
struct OrderWork {
    unsigned long long *keys;
    int nkeys;
    float *sorted;
    float4 *boxes;
    int *perm;
    float *bbox_part;
    float *bbox;
};
int order_nkeys(int npad);
int order_launches(int npad);   // kernel launches of launch_spatial_order
size_t order_workspace_bytes(int npad, int tile);
OrderWork order_carve(void *base, int npad, int tile);
// Sorts the n staged sources of stage (STAGE_F32IX2, npad entries) along a
// Morton curve of their hi positions (ties impossible: the index is part of the
// key) and writes the sorted copy, permutation and boxes of tiles of `tile`.
cudaError_t launch_spatial_order(const void *stage, int n, int npad, int tile, const OrderWork &w,
                                 cudaStream_t s);

cudaError_t launch_diff_norms(const double *a, const double *b, int n3, double *partials,
                              cudaStream_t s);

}  // namespace ppk
