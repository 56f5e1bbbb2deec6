// pp_state.cu -- the O(N) helper kernels around the force passes: layout
// conversion between [n][3] arrays and the SoA state, staging of positions
// (Eq. G drifts included), weights, padding and deterministic moment
// reductions for the diagnostics (Eq. I).
#include <cfloat>
#include <cmath>

#include "pp_internal.h"

namespace ppk {

// ---- O(N) kernels ----------------------------------------------------------

namespace {

// The [n][3] side is walked as a flat array of 3n doubles, so that a warp reads
// (or writes) 32 consecutive doubles: this side may be host memory mapped into
// the device address space, where every access crosses the CPU-GPU link.
__global__ void aos_to_soa_kernel(const double *__restrict__ in, int n, double *x, double *y,
                                  double *z, int *bad)
{
    const size_t total = 3 * (size_t)n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const double a = in[t];
        if (!isfinite(a)) atomicOr(bad, 1);
        const size_t i = t / 3;
        const int c = (int)(t - 3 * i);
        (c == 0 ? x : c == 1 ? y : z)[i] = a;
    }
}

__global__ void soa_to_aos_kernel(const double *__restrict__ x, const double *__restrict__ y,
                                  const double *__restrict__ z, int n, double *out)
{
    const size_t total = 3 * (size_t)n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t i = t / 3;
        const int c = (int)(t - 3 * i);
        out[t] = (c == 0 ? x : c == 1 ? y : z)[i];
    }
}

// Whole-state import for pp_set_state: r, v, a as [n][3] (device memory or
// mapped host memory) -> SoA state, finiteness flag, and the pending Eq. G
// positions drift(r, v, a) staged into dst (padding entries n..npad-1
// included), in one pass.  One thread per particle.
template <int KIND>
__global__ void import_state_kernel(const double *__restrict__ pos, const double *__restrict__ vel,
                                    const double *__restrict__ acc, int n, int npad, double *rx,
                                    double *ry, double *rz, double *vx, double *vy, double *vz,
                                    double *ax, double *ay, double *az, void *dst, double dt,
                                    double half_dt2, double cx, double cy, double cz,
                                    double inv_l0, const float *__restrict__ wrel, int *bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x) {
        if (i >= n) {
            store_padding<KIND>(dst, npad, i);
            continue;
        }
        const size_t b = 3 * (size_t)i;
        const double r0 = pos[b], r1 = pos[b + 1], r2 = pos[b + 2];
        const double v0 = vel[b], v1 = vel[b + 1], v2 = vel[b + 2];
        const double a0 = acc[b], a1 = acc[b + 1], a2 = acc[b + 2];
        if (!(isfinite(r0) && isfinite(r1) && isfinite(r2) && isfinite(v0) && isfinite(v1) &&
              isfinite(v2) && isfinite(a0) && isfinite(a1) && isfinite(a2)))
            atomicOr(bad, 1);
        rx[i] = r0; ry[i] = r1; rz[i] = r2;
        vx[i] = v0; vy[i] = v1; vz[i] = v2;
        ax[i] = a0; ay[i] = a1; az[i] = a2;
        store_staged<KIND>(dst, npad, i, drift(r0, v0, a0, dt, half_dt2),
                           drift(r1, v1, a1, dt, half_dt2), drift(r2, v2, a2, dt, half_dt2), cx,
                           cy, cz, inv_l0, wrel ? wrel[i] : 1.0f);
    }
}

// Whole-state export for pp_get_state: up to three SoA triples -> [n][3]
// arrays (device memory or mapped host memory; a null output is skipped), in
// one pass walked as flat arrays so that a warp writes 32 consecutive doubles.
__global__ void export_state_kernel(const double *__restrict__ rx, const double *__restrict__ ry,
                                    const double *__restrict__ rz, const double *__restrict__ vx,
                                    const double *__restrict__ vy, const double *__restrict__ vz,
                                    const double *__restrict__ ax, const double *__restrict__ ay,
                                    const double *__restrict__ az, int n, double *pos,
                                    double *vel, double *acc)
{
    const size_t per = 3 * (size_t)n, total = 3 * per;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int arr = (int)(t / per);
        const size_t f = t - arr * per;
        double *out = arr == 0 ? pos : arr == 1 ? vel : acc;
        if (!out) continue;
        const size_t i = f / 3;
        const int c = (int)(f - 3 * i);
        const double *src = arr == 0 ? (c == 0 ? rx : c == 1 ? ry : rz)
                          : arr == 1 ? (c == 0 ? vx : c == 1 ? vy : vz)
                                     : (c == 0 ? ax : c == 1 ? ay : az);
        out[f] = src[i];
    }
}

template <int KIND>
__global__ void stage_kernel(const double *__restrict__ x, const double *__restrict__ y,
                             const double *__restrict__ z, int n, int npad, void *dst, double cx,
                             double cy, double cz, double inv_l0, const float *__restrict__ wrel)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x) {
        if (i < n)
            store_staged<KIND>(dst, npad, i, x[i], y[i], z[i], cx, cy, cz, inv_l0,
                               wrel ? wrel[i] : 1.0f);
        else store_padding<KIND>(dst, npad, i);
    }
}

template <int KIND>
__global__ void stage_drift_kernel(const double *__restrict__ rx, const double *__restrict__ ry,
                                   const double *__restrict__ rz, const double *__restrict__ vx,
                                   const double *__restrict__ vy, const double *__restrict__ vz,
                                   const double *__restrict__ ax, const double *__restrict__ ay,
                                   const double *__restrict__ az, int n, int npad, void *dst,
                                   double dt, double half_dt2, double cx, double cy, double cz,
                                   double inv_l0, const float *__restrict__ wrel)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x) {
        if (i < n) {
            store_staged<KIND>(dst, npad, i, drift(rx[i], vx[i], ax[i], dt, half_dt2),
                               drift(ry[i], vy[i], ay[i], dt, half_dt2),
                               drift(rz[i], vz[i], az[i], dt, half_dt2), cx, cy, cz, inv_l0,
                               wrel ? wrel[i] : 1.0f);
        } else {
            store_padding<KIND>(dst, npad, i);
        }
    }
}

__global__ void weights_kernel(const double *__restrict__ w, int n, double inv_ref, float *wrel,
                               int *bad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double x = w[i];
        if (!(isfinite(x) && x > 0.0)) atomicOr(bad, 1);
        wrel[i] = __double2float_rn(x * inv_ref);
    }
}

template <int KIND>
__global__ void fill_padding_kernel(void *dst, int n, int npad)
{
    for (int i = n + blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += gridDim.x * blockDim.x)
        store_padding<KIND>(dst, npad, i);
}

constexpr int kMomThreads = 256;

// Fixed-shape tree over the block: identical summation order on every run.
__device__ void block_sum(double *sh, int k, double v)
{
    sh[k * kMomThreads + threadIdx.x] = v;
}

__global__ void __launch_bounds__(kMomThreads)
    moments_kernel(int pass, int n, const double *__restrict__ x, const double *__restrict__ y,
                   const double *__restrict__ z, const double *__restrict__ vx,
                   const double *__restrict__ vy, const double *__restrict__ vz, double cx,
                   double cy, double cz, double *partials, const double *__restrict__ wts)
{
    __shared__ double sh[kMomSlots * kMomThreads];
    double acc[kMomSlots];
    for (int k = 0; k < kMomSlots; ++k) acc[k] = 0.0;
    acc[10] = -INFINITY;
    acc[11] = -INFINITY;
    const int chunk = (n + gridDim.x - 1) / gridDim.x;
    const int lo = blockIdx.x * chunk;
    const int hi = min(n, lo + chunk);
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        if (pass == 0) {
            acc[0] += x[i];
            acc[1] += y[i];
            acc[2] += z[i];
        } else if (pass == 1) {
            const double dx = x[i] - cx, dy = y[i] - cy, dz = z[i] - cz;
            const double wi = wts ? wts[i] : 1.0;
            acc[0] += dx * dx + dy * dy + dz * dz;
            acc[1] += wi * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]);
            acc[2] += wi * vx[i];
            acc[3] += wi * vy[i];
            acc[4] += wi * vz[i];
            acc[5] += x[i] * x[i];
            acc[6] += vx[i] * vx[i];
            acc[7] += x[i] * vx[i];
            acc[10] = fmax(acc[10], x[i]);
            acc[11] = fmax(acc[11], vx[i]);
        } else {
            acc[0] += wts ? wts[i] * x[i] : x[i];
        }
    }
    for (int k = 0; k < kMomSlots; ++k) block_sum(sh, k, acc[k]);
    __syncthreads();
    for (int stride = kMomThreads / 2; stride > 0; stride >>= 1) {
        if (threadIdx.x < stride) {
            for (int k = 0; k < kMomSlots; ++k) {
                double *s = sh + k * kMomThreads;
                s[threadIdx.x] = (k >= 10) ? fmax(s[threadIdx.x], s[threadIdx.x + stride])
                                           : s[threadIdx.x] + s[threadIdx.x + stride];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < kMomSlots)
        partials[blockIdx.x * kMomSlots + threadIdx.x] = sh[threadIdx.x * kMomThreads];
}

__global__ void moments_finish_kernel(const double *__restrict__ partials, int nblocks,
                                      double *out)
{
    const int k = threadIdx.x;
    if (k >= kMomSlots) return;
    double acc = (k >= 10) ? -INFINITY : 0.0;
    for (int b = 0; b < nblocks; ++b) {
        const double v = partials[b * kMomSlots + k];
        acc = (k >= 10) ? fmax(acc, v) : acc + v;
    }
    out[k] = acc;
}

int grid_for(int n, int threads)
{
    int g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    return g;
}

}  // namespace

cudaError_t launch_aos_to_soa(const double *in, int n, double *x, double *y, double *z, int *bad,
                              cudaStream_t s)
{
    aos_to_soa_kernel<<<grid_for(3 * n, 256), 256, 0, s>>>(in, n, x, y, z, bad);
    return cudaGetLastError();
}

cudaError_t launch_soa_to_aos(const double *x, const double *y, const double *z, int n,
                              double *out, cudaStream_t s)
{
    soa_to_aos_kernel<<<grid_for(3 * n, 256), 256, 0, s>>>(x, y, z, n, out);
    return cudaGetLastError();
}

cudaError_t launch_stage(const double *x, const double *y, const double *z, int n, int npad,
                         void *dst, int kind, double cx, double cy, double cz, double inv_l0,
                         cudaStream_t s, const float *wrel)
{
    const int g = grid_for(npad, 256);
    if (kind == STAGE_F32IX2)
        stage_kernel<STAGE_F32IX2><<<g, 256, 0, s>>>(x, y, z, n, npad, dst, cx, cy, cz, inv_l0, wrel);
    else if (kind == STAGE_F32I)
        stage_kernel<STAGE_F32I><<<g, 256, 0, s>>>(x, y, z, n, npad, dst, cx, cy, cz, inv_l0, wrel);
    else if (kind == STAGE_F32)
        stage_kernel<STAGE_F32><<<g, 256, 0, s>>>(x, y, z, n, npad, dst, cx, cy, cz, inv_l0, wrel);
    else if (kind == STAGE_F32X2)
        stage_kernel<STAGE_F32X2><<<g, 256, 0, s>>>(x, y, z, n, npad, dst, cx, cy, cz, inv_l0, wrel);
    else
        stage_kernel<STAGE_F64><<<g, 256, 0, s>>>(x, y, z, n, npad, dst, cx, cy, cz, inv_l0, wrel);
    return cudaGetLastError();
}

cudaError_t launch_weights(const double *w, int n, double w_ref, float *wrel, int *bad,
                           cudaStream_t s)
{
    weights_kernel<<<grid_for(n, 256), 256, 0, s>>>(w, n, 1.0 / w_ref, wrel, bad);
    return cudaGetLastError();
}

cudaError_t launch_fill_padding(void *dst, int n, int npad, int kind, cudaStream_t s)
{
    if (npad <= n) return cudaSuccess;
    const int g = grid_for(npad - n, 256);
    if (kind == STAGE_F32IX2) fill_padding_kernel<STAGE_F32IX2><<<g, 256, 0, s>>>(dst, n, npad);
    else if (kind == STAGE_F32I) fill_padding_kernel<STAGE_F32I><<<g, 256, 0, s>>>(dst, n, npad);
    else if (kind == STAGE_F32) fill_padding_kernel<STAGE_F32><<<g, 256, 0, s>>>(dst, n, npad);
    else if (kind == STAGE_F32X2) fill_padding_kernel<STAGE_F32X2><<<g, 256, 0, s>>>(dst, n, npad);
    else fill_padding_kernel<STAGE_F64><<<g, 256, 0, s>>>(dst, n, npad);
    return cudaGetLastError();
}

cudaError_t launch_stage_drift(double *const r[3], double *const v[3], double *const a[3], int n,
                               int npad, void *dst, int kind, double dt, double half_dt2,
                               double cx, double cy, double cz, double inv_l0, cudaStream_t s,
                               const float *wrel)
{
    const int g = grid_for(npad, 256);
#define PP_SD_ARGS r[0], r[1], r[2], v[0], v[1], v[2], a[0], a[1], a[2], n, npad, dst, dt, half_dt2, \
                   cx, cy, cz, inv_l0, wrel
    if (kind == STAGE_F32IX2) stage_drift_kernel<STAGE_F32IX2><<<g, 256, 0, s>>>(PP_SD_ARGS);
    else if (kind == STAGE_F32I) stage_drift_kernel<STAGE_F32I><<<g, 256, 0, s>>>(PP_SD_ARGS);
    else if (kind == STAGE_F32) stage_drift_kernel<STAGE_F32><<<g, 256, 0, s>>>(PP_SD_ARGS);
    else if (kind == STAGE_F32X2) stage_drift_kernel<STAGE_F32X2><<<g, 256, 0, s>>>(PP_SD_ARGS);
    else stage_drift_kernel<STAGE_F64><<<g, 256, 0, s>>>(PP_SD_ARGS);
#undef PP_SD_ARGS
    return cudaGetLastError();
}

cudaError_t launch_import_state(const double *pos, const double *vel, const double *acc, int n,
                                int npad, double *const r[3], double *const v[3],
                                double *const a[3], void *dst, int kind, double dt,
                                double half_dt2, double cx, double cy, double cz, double inv_l0,
                                const float *wrel, int *bad, cudaStream_t s)
{
    const int g = grid_for(npad, 256);
#define PP_IS_ARGS pos, vel, acc, n, npad, r[0], r[1], r[2], v[0], v[1], v[2], a[0], a[1], a[2], \
                   dst, dt, half_dt2, cx, cy, cz, inv_l0, wrel, bad
    if (kind == STAGE_F32IX2) import_state_kernel<STAGE_F32IX2><<<g, 256, 0, s>>>(PP_IS_ARGS);
    else if (kind == STAGE_F32I) import_state_kernel<STAGE_F32I><<<g, 256, 0, s>>>(PP_IS_ARGS);
    else if (kind == STAGE_F32) import_state_kernel<STAGE_F32><<<g, 256, 0, s>>>(PP_IS_ARGS);
    else if (kind == STAGE_F32X2) import_state_kernel<STAGE_F32X2><<<g, 256, 0, s>>>(PP_IS_ARGS);
    else import_state_kernel<STAGE_F64><<<g, 256, 0, s>>>(PP_IS_ARGS);
#undef PP_IS_ARGS
    return cudaGetLastError();
}

cudaError_t launch_export_state(double *const r[3], double *const v[3], double *const a[3], int n,
                                double *pos, double *vel, double *acc, cudaStream_t s)
{
    export_state_kernel<<<grid_for(3 * n, 256), 256, 0, s>>>(r[0], r[1], r[2], v[0], v[1], v[2],
                                                            a[0], a[1], a[2], n, pos, vel, acc);
    return cudaGetLastError();
}

cudaError_t launch_moments(int pass, int n, const double *x, const double *y, const double *z,
                           const double *vx, const double *vy, const double *vz, double cx,
                           double cy, double cz, double *block_partials, double *out,
                           cudaStream_t s, const double *wts)
{
    moments_kernel<<<kMomBlocks, kMomThreads, 0, s>>>(pass, n, x, y, z, vx, vy, vz, cx, cy, cz,
                                                      block_partials, wts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    moments_finish_kernel<<<1, 32, 0, s>>>(block_partials, kMomBlocks, out);
    return cudaGetLastError();
}


// Deterministic sums of |a - b|^2 and |b|^2 over n3 doubles (one pass per block,
// fixed tree; the host adds the kDiffBlocks block results in order).
constexpr int kDiffThreads = 256;

__global__ void __launch_bounds__(kDiffThreads)
    diff_norms_kernel(const double *__restrict__ a, const double *__restrict__ b, int n3,
                      double *partials)
{
    __shared__ double sd[kDiffThreads], sb[kDiffThreads];
    const int chunk = (n3 + gridDim.x - 1) / gridDim.x;
    const int lo = blockIdx.x * chunk, hi = min(n3, lo + chunk);
    double d2 = 0.0, b2 = 0.0;
    for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) {
        const double d = a[k] - b[k];
        d2 += d * d;
        b2 += b[k] * b[k];
    }
    sd[threadIdx.x] = d2;
    sb[threadIdx.x] = b2;
    __syncthreads();
    for (int s = kDiffThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sd[threadIdx.x] += sd[threadIdx.x + s];
            sb[threadIdx.x] += sb[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = sd[0];
        partials[2 * blockIdx.x + 1] = sb[0];
    }
}

cudaError_t launch_diff_norms(const double *a, const double *b, int n3, double *partials,
                              cudaStream_t s)
{
    diff_norms_kernel<<<kDiffBlocks, kDiffThreads, 0, s>>>(a, b, n3, partials);
    return cudaGetLastError();
}

}  // namespace ppk
