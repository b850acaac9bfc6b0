// Stages a6-a7: exact-size CSR assembly of M (exclusive scan of the kept
// counts, rows copied from the staging buffer sorted by column) and y = M x.
#include "mcmi_internal.cuh"
#include "kernels.h"

namespace mcmi {

namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ long long warp_incl_scan(long long v)
{
    const int l = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        const long long nb = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (l >= o) v += nb;
    }
    return v;
}

// exclusive scan of the block's tile; returns the tile total to thread 0 via *total
__device__ __forceinline__ long long block_excl_scan(long long v, long long *red, long long *total)
{
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const long long incl = warp_incl_scan(v);
    if (l == 31) red[w] = incl;
    __syncthreads();
    if (w == 0) {
        const long long x = l < (int)(blockDim.x >> 5) ? red[l] : 0;
        const long long xi = warp_incl_scan(x);
        if (l < (int)(blockDim.x >> 5)) red[l] = xi - x;
        if (l == 31) *total = xi;
    }
    __syncthreads();
    return red[w] + incl - v;
}
}  // namespace

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int32_t *__restrict__ counts, int64_t n,
                                                             int64_t *__restrict__ out, int64_t *__restrict__ tile_sum)
{
    __shared__ long long red[32];
    __shared__ long long total;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    long long v[kScanItems], sum = 0;
#pragma unroll
    for (int u = 0; u < kScanItems; ++u) {
        v[u] = base + u < n ? (long long)counts[base + u] : 0;
        sum += v[u];
    }
    long long run = block_excl_scan(sum, red, &total);
#pragma unroll
    for (int u = 0; u < kScanItems; ++u) {
        if (base + u < n) out[base + u] = run;
        run += v[u];
    }
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_top(int64_t *__restrict__ tile_sum, int64_t ntiles,
                                                   int64_t *__restrict__ out_total)
{
    __shared__ long long red[32];
    __shared__ long long total;
    long long carry = 0;
    for (int64_t b = 0; b < ntiles; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const long long v = i < ntiles ? tile_sum[i] : 0;
        const long long ex = block_excl_scan(v, red, &total);
        if (i < ntiles) tile_sum[i] = carry + ex;
        __syncthreads();
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *out_total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(int64_t *__restrict__ out, int64_t n,
                                                           const int64_t *__restrict__ tile_sum)
{
    const long long add = tile_sum[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int u = threadIdx.x; u < kScanTile; u += blockDim.x)
        if (base + u < n) out[base + u] += add;
}

size_t scan_tmp_elems(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

cudaError_t scan_counts(const int32_t *counts, int64_t n, int64_t *out, int64_t *tile_tmp, cudaStream_t s)
{
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles > 0) k_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, s>>>(counts, n, out, tile_tmp);
    k_scan_top<<<1, 1024, 0, s>>>(tile_tmp, ntiles, out + n);
    if (ntiles > 0) k_scan_add<<<(unsigned)ntiles, kScanThreads, 0, s>>>(out, n, tile_tmp);
    return cudaGetLastError();
}

// One warp per row: entries of the staging buffer placed at their rank by
// column (columns are unique inside a row).
__global__ void k_assemble(int64_t rows, const int64_t *__restrict__ row_ptr, const int64_t *__restrict__ st_off,
                           const int32_t *__restrict__ st_cnt, const uint32_t *__restrict__ st_col,
                           const float *__restrict__ st_val, int32_t *__restrict__ out_col,
                           float *__restrict__ out_val)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < rows; r += nwarps) {
        const int cnt = st_cnt[r];
        const int64_t off = st_off[r], dst = row_ptr[r];
        if (cnt <= 32) {
            const uint32_t c = lane < cnt ? st_col[off + lane] : 0xFFFFFFFFu;
            const float v = lane < cnt ? st_val[off + lane] : 0.0f;
            int rank = 0;
            for (int j = 0; j < cnt; ++j) {
                const uint32_t cj = __shfl_sync(0xFFFFFFFFu, c, j);
                rank += cj < c;
            }
            if (lane < cnt) {
                out_col[dst + rank] = (int32_t)c;
                out_val[dst + rank] = v;
            }
        } else {
            for (int e = lane; e < cnt; e += 32) {
                const uint32_t c = st_col[off + e];
                int rank = 0;
                for (int j = 0; j < cnt; ++j) rank += st_col[off + j] < c;
                out_col[dst + rank] = (int32_t)c;
                out_val[dst + rank] = st_val[off + e];
            }
        }
    }
}

cudaError_t launch_assemble(int64_t rows, const int64_t *row_ptr, const int64_t *st_off, const int32_t *st_cnt,
                            const uint32_t *st_col, const float *st_val, int32_t *out_col, float *out_val,
                            cudaStream_t s)
{
    const int bs = 256;
    int64_t g = (rows * 32 + bs - 1) / bs;
    if (g > 148 * 16) g = 148 * 16;
    if (g < 1) g = 1;
    k_assemble<<<(unsigned)g, bs, 0, s>>>(rows, row_ptr, st_off, st_cnt, st_col, st_val, out_col, out_val);
    return cudaGetLastError();
}

// y = M x, eight lanes per row.
__global__ void k_spmv(int64_t rows, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                       const float *__restrict__ val, const float *__restrict__ x, float *__restrict__ y)
{
    const int sub = threadIdx.x & 7;
    const int64_t grp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) >> 3;
    // the loop bound is uniform across the warp (4 row groups per warp) so
    // that every lane reaches the shuffles
    for (int64_t r0 = grp & ~(int64_t)3; r0 < rows; r0 += ngrp) {
        const int64_t r = r0 + (grp & 3);
        float acc = 0.0f;
        if (r < rows)
            for (int64_t k = rp[r] + sub; k < rp[r + 1]; k += 8)
                acc = fmaf(__ldg(val + k), __ldg(x + __ldg(col + k)), acc);
        acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 4);
        acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 2);
        acc += __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
        if (sub == 0 && r < rows) y[r] = acc;
    }
}

cudaError_t launch_spmv(int64_t rows, const int64_t *rp, const int32_t *col, const float *val, const float *x,
                        float *y, cudaStream_t s)
{
    const int bs = 256;
    int64_t g = (rows * 8 + bs - 1) / bs;
    if (g > 148 * 16) g = 148 * 16;
    if (g < 1) g = 1;
    k_spmv<<<(unsigned)g, bs, 0, s>>>(rows, rp, col, val, x, y);
    return cudaGetLastError();
}

}  // namespace mcmi
