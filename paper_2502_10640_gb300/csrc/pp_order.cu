// pp_order.cu -- spatial order of the staged sources for the tile-box guard.
//
// Guarded staging (PP_POS_GUARDED) sums a (target, tile) partial with hi/lo
// separations when the tile may hold a source closer to the target than
// |p_i| / 2^8.  In particle order a tile's sources are spread over the whole
// bunch, so the test has to run per pair.  Sorted along a Morton curve, the
// sources of a tile fill a small box, and one test per target and tile against
// that box decides for all of its pairs.  Per force pass:
//
//   1. the bounding box of the staged hi positions (two small reductions);
//   2. a 64-bit key per source: its 30-bit Morton code (10 bits per axis over
//      the bounding box) above its index, so that keys are unique and the
//      order is a function of the positions alone (bitwise-reproducible
//      results, also across a checkpoint and resume);
//   3. a bitonic sort of the keys (shared-memory stages up to 2048 keys per
//      block, global compare-exchange steps above);
//   4. the sorted copy of the staged array (hi and lo parts, interleaved
//      layout) and the permutation sorted index -> particle index;
//   5. the box of each tile of the sorted copy (hi parts, real sources only).
//
// The whole order costs 60 launches and about 0.5 ms at N = 2^20 (measured on
// GB300), 0.13 % of a step of the O(N^2) pass it serves.
#include <cfloat>

#include "pp_internal.h"

namespace ppk {

namespace {

constexpr int kBboxBlocks = 256;
constexpr int kBboxThreads = 256;
constexpr int kSortLocal = 2048;   // keys sorted per block in shared memory

__device__ __forceinline__ void load_hi(const float *stage, int k, float &x, float &y, float &z)
{
    const float *f = stage + 8 * (size_t)(k >> 1) + (k & 1);
    x = f[0];
    y = f[2];
    z = f[4];
}

// Block-wide min/max of three values; thread 0 holds the result.
__device__ __forceinline__ void block_minmax(float (&mn)[3], float (&mx)[3])
{
    __shared__ float sm[32][6];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sm[w][c] = mn[c];
            sm[w][3 + c] = mx[c];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                mn[c] = fminf(mn[c], sm[q][c]);
                mx[c] = fmaxf(mx[c], sm[q][3 + c]);
            }
    }
}

__global__ void __launch_bounds__(kBboxThreads) bbox_partial_kernel(const float *stage, int n,
                                                                    float *part)
{
    float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        float v[3];
        load_hi(stage, k, v[0], v[1], v[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            mn[c] = fminf(mn[c], v[c]);
            mx[c] = fmaxf(mx[c], v[c]);
        }
    }
    block_minmax(mn, mx);
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            part[6 * blockIdx.x + c] = mn[c];
            part[6 * blockIdx.x + 3 + c] = mx[c];
        }
}

__global__ void __launch_bounds__(kBboxThreads) bbox_final_kernel(const float *part, int nparts,
                                                                  float *bbox)
{
    float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int q = threadIdx.x; q < nparts; q += blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            mn[c] = fminf(mn[c], part[6 * q + c]);
            mx[c] = fmaxf(mx[c], part[6 * q + 3 + c]);
        }
    block_minmax(mn, mx);
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            bbox[c] = mn[c];
            bbox[3 + c] = mx[c];
        }
}

// 10 low bits of v spread to every third bit.
__device__ __forceinline__ uint32_t spread3(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t cell10(float v, float lo, float scale)
{
    const float q = floorf((v - lo) * scale);
    return (uint32_t)fminf(fmaxf(q, 0.f), 1023.f);
}

// keys[k]: Morton code of source k above k (k < n); k alone with the top 32
// bits set for the padding entries n <= k < nkeys, which so stay in place at
// the end.
__global__ void morton_keys_kernel(const float *stage, int n, int nkeys, const float *bbox,
                                   unsigned long long *keys)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkeys) return;
    if (k >= n) {
        keys[k] = 0xffffffff00000000ull | (unsigned)k;
        return;
    }
    float v[3];
    load_hi(stage, k, v[0], v[1], v[2]);
    uint32_t code = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float lo = bbox[c], ext = bbox[3 + c] - lo;
        const float scale = ext > 0.f ? 1024.f / ext : 0.f;
        code |= spread3(cell10(v[c], lo, scale)) << (2 - c);
    }
    keys[k] = ((unsigned long long)code << 32) | (unsigned)k;
}

__device__ __forceinline__ void cmp_swap(unsigned long long &a, unsigned long long &b, bool up)
{
    if ((a > b) == up) {
        const unsigned long long t = a;
        a = b;
        b = t;
    }
}

// Bitonic stages inside blocks of L = 2 * blockDim.x keys held in shared
// memory.  kfix == 0: the full sort of each block (k = 2 .. L); kfix > L: the
// steps j = L/2 .. 1 of the merge of size kfix.  Direction: ascending where
// (global index & k) == 0.
__global__ void __launch_bounds__(kSortLocal / 2) bitonic_local_kernel(unsigned long long *keys,
                                                                     int kfix)
{
    __shared__ unsigned long long sk[kSortLocal];
    const int L = 2 * (int)blockDim.x;
    const size_t base = (size_t)blockIdx.x * L;
    const int t = threadIdx.x;
    sk[t] = keys[base + t];
    sk[t + blockDim.x] = keys[base + t + blockDim.x];
    __syncthreads();
    const int k0 = kfix ? kfix : 2, k1 = kfix ? kfix : L;
    for (int k = k0; k <= k1; k <<= 1) {
        for (int j = (kfix ? L : k) >> 1; j > 0; j >>= 1) {
            const int i = 2 * j * (t / j) + (t % j);
            const bool up = ((base + i) & (size_t)k) == 0;
            cmp_swap(sk[i], sk[i + j], up);
            __syncthreads();
        }
    }
    keys[base + t] = sk[t];
    keys[base + t + blockDim.x] = sk[t + blockDim.x];
}

// One global compare-exchange step (k, j) of the bitonic sort, j >= L.
__global__ void bitonic_global_kernel(unsigned long long *keys, int npairs, int k, int j)
{
    const int pidx = blockIdx.x * blockDim.x + threadIdx.x;
    if (pidx >= npairs) return;
    const int i = 2 * j * (pidx / j) + (pidx % j);
    const bool up = (i & k) == 0;
    unsigned long long a = keys[i], b = keys[i + j];
    if ((a > b) == up) {
        keys[i] = b;
        keys[i + j] = a;
    }
}

// Sorted copy (hi and lo parts, interleaved layout) and the permutation.
__global__ void order_gather_kernel(const float *stage, int npad,
                                    const unsigned long long *keys, int *perm, float *sorted)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npad) return;
    const int src = (int)(keys[k] & 0xffffffffull);
    perm[k] = src;
    const float *f = stage + 8 * (size_t)(src >> 1) + (src & 1);
    float *g = sorted + 8 * (size_t)(k >> 1) + (k & 1);
    const float *fl = f + 4 * (size_t)npad;
    float *gl = g + 4 * (size_t)npad;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        g[2 * c] = f[2 * c];
        gl[2 * c] = fl[2 * c];
    }
}

// boxes[2t], boxes[2t + 1]: lower and upper corners of the hi parts of the real
// sources (k < n) of sorted tile t; an empty box (+inf, -inf) for a tile of
// padding only.  One warp per tile.
__global__ void tile_boxes_kernel(const float *sorted, int n, int tile, int ntiles,
                                  float4 *boxes)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= ntiles) return;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    const int k1 = min((w + 1) * tile, n);
    for (int k = w * tile + lane; k < k1; k += 32) {
        float v[3];
        load_hi(sorted, k, v[0], v[1], v[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            mn[c] = fminf(mn[c], v[c]);
            mx[c] = fmaxf(mx[c], v[c]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        }
    if (lane == 0) {
        boxes[2 * w] = make_float4(mn[0], mn[1], mn[2], 0.f);
        boxes[2 * w + 1] = make_float4(mx[0], mx[1], mx[2], 0.f);
    }
}

}  // namespace

int order_nkeys(int npad)
{
    int m = 2;
    while (m < npad) m <<= 1;
    return m;
}

int order_launches(int npad)
{
    const int nkeys = order_nkeys(npad);
    const int L = nkeys < kSortLocal ? nkeys : kSortLocal;
    int count = 3 + 1 + 2;   // bounding box (2), keys, local sort; gather, boxes
    for (int k = 2 * L; k <= nkeys; k <<= 1) {
        for (int j = k >> 1; j >= L; j >>= 1) ++count;
        ++count;
    }
    return count;
}

size_t order_workspace_bytes(int npad, int tile)
{
    const size_t nkeys = (size_t)order_nkeys(npad);
    const size_t ntiles = (size_t)npad / tile;
    return nkeys * sizeof(unsigned long long) + (size_t)npad * 2 * sizeof(float4) +
           ntiles * 2 * sizeof(float4) + (size_t)npad * sizeof(int) +
           (size_t)(6 * kBboxBlocks + 8) * sizeof(float);
}

OrderWork order_carve(void *base, int npad, int tile)
{
    OrderWork w{};
    char *p = static_cast<char *>(base);
    w.nkeys = order_nkeys(npad);
    w.keys = reinterpret_cast<unsigned long long *>(p);
    p += (size_t)w.nkeys * sizeof(unsigned long long);
    w.sorted = reinterpret_cast<float *>(p);
    p += (size_t)npad * 2 * sizeof(float4);
    w.boxes = reinterpret_cast<float4 *>(p);
    p += (size_t)(npad / tile) * 2 * sizeof(float4);
    w.perm = reinterpret_cast<int *>(p);
    p += (size_t)npad * sizeof(int);
    w.bbox_part = reinterpret_cast<float *>(p);
    w.bbox = w.bbox_part + 6 * kBboxBlocks;
    return w;
}

cudaError_t launch_spatial_order(const void *stage, int n, int npad, int tile, const OrderWork &w,
                                 cudaStream_t s)
{
    if (n < 1 || npad < n || tile < 1 || npad % tile != 0 || w.nkeys < npad ||
        (w.nkeys & (w.nkeys - 1)) != 0)
        return cudaErrorInvalidValue;
    const float *st = static_cast<const float *>(stage);
    bbox_partial_kernel<<<kBboxBlocks, kBboxThreads, 0, s>>>(st, n, w.bbox_part);
    bbox_final_kernel<<<1, kBboxThreads, 0, s>>>(w.bbox_part, kBboxBlocks, w.bbox);
    morton_keys_kernel<<<(w.nkeys + 255) / 256, 256, 0, s>>>(st, n, w.nkeys, w.bbox, w.keys);
    const int L = w.nkeys < kSortLocal ? w.nkeys : kSortLocal;
    bitonic_local_kernel<<<w.nkeys / L, L / 2, 0, s>>>(w.keys, 0);
    for (int k = 2 * L; k <= w.nkeys; k <<= 1) {
        for (int j = k >> 1; j >= L; j >>= 1)
            bitonic_global_kernel<<<(w.nkeys / 2 + 255) / 256, 256, 0, s>>>(w.keys, w.nkeys / 2,
                                                                            k, j);
        bitonic_local_kernel<<<w.nkeys / L, L / 2, 0, s>>>(w.keys, k);
    }
    order_gather_kernel<<<(npad + 255) / 256, 256, 0, s>>>(st, npad, w.keys, w.perm, w.sorted);
    const int ntiles = npad / tile;
    tile_boxes_kernel<<<(ntiles * 32 + 255) / 256, 256, 0, s>>>(w.sorted, n, tile, ntiles,
                                                                w.boxes);
    return cudaGetLastError();
}

}  // namespace ppk
