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

// Rows are copied from the staging buffer sorted by column (columns are
// distinct inside a row).  Entries travel as one 64-bit key, column in the
// high word and the value's bits in the low word, sorted by a bitonic network
// in the form whose comparators all put the smaller key at the lower index:
// merging blocks of k starts with the mirror step (i, i ^ (k - 1)) and goes on
// with the half-cleaners (i, i + j), j = k/4, ..., 1.  Padding a row to a
// power of two with +inf keys therefore never moves an entry, and a comparator
// whose upper index lies past the row's end can simply be skipped.
constexpr int kAsmWarps = 4;            // warps per block of k_assemble
constexpr int kAsmWarpMax = 1024;       // rows up to this length: one warp, shared memory
constexpr int kAsmLongThreads = 256;    // threads per block of k_assemble_long
constexpr int kAsmTile = 4096;          // shared-memory tile of k_assemble_long
constexpr unsigned long long kKeyInf = ~0ull;

__device__ __forceinline__ unsigned long long pack_entry(uint32_t c, float v)
{
    return ((unsigned long long)c << 32) | __float_as_uint(v);
}

__device__ __forceinline__ void cmp_swap(unsigned long long *a, int i, int l)
{
    const unsigned long long x = a[i], y = a[l];
    if (x > y) {
        a[i] = y;
        a[l] = x;
    }
}

// pair q of a step whose comparators span distance h: lower index
__device__ __forceinline__ int64_t pair_lo(int64_t q, int64_t h) { return ((q & ~(h - 1)) << 1) | (q & (h - 1)); }

// sorts a[0, P) (P a power of two) in shared memory with NT cooperating
// threads t = 0..NT-1 (one warp, or the whole block)
template <int NT, bool WARP>
__device__ __forceinline__ void bitonic_shared(unsigned long long *a, int P, int t)
{
    for (int k = 2; k <= P; k <<= 1) {
        for (int q = t; q < (P >> 1); q += NT) {
            const int i = (int)pair_lo(q, k >> 1);
            cmp_swap(a, i, i ^ (k - 1));
        }
        if (WARP) __syncwarp(); else __syncthreads();
        for (int j = k >> 2; j > 0; j >>= 1) {
            for (int q = t; q < (P >> 1); q += NT) {
                const int i = (int)pair_lo(q, j);
                cmp_swap(a, i, i + j);
            }
            if (WARP) __syncwarp(); else __syncthreads();
        }
    }
}

// bitonic_shared for one warp and a compile-time P: each lane first loads
// the pairs of all its comparators of a step (they are disjoint), then
// compares and stores, so the loads of a step are in flight together
// instead of each waiting for the stores before it
template <int P>
__device__ __forceinline__ void bitonic_warp_batched(unsigned long long *a, int t)
{
    constexpr int C = P / 64;             // comparators per lane and step
    constexpr int CB = C < 8 ? C : 8;     // taken in batches of at most 8 (registers)
#pragma unroll 1
    for (int k = 2; k <= P; k <<= 1) {
#pragma unroll 1
        for (int j = k >> 1; j > 0; j >>= 1) {
            const bool mirror = j == (k >> 1);   // first step of a merge: (i, i ^ (k - 1))
#pragma unroll
            for (int c0 = 0; c0 < C; c0 += CB) {
                int lo[CB];
                unsigned long long x[CB], y[CB];
#pragma unroll
                for (int c = 0; c < CB; ++c) {
                    lo[c] = (int)pair_lo(t + 32 * (c0 + c), j);
                    x[c] = a[lo[c]];
                    y[c] = a[mirror ? (lo[c] ^ (k - 1)) : (lo[c] + j)];
                }
#pragma unroll
                for (int c = 0; c < CB; ++c)
                    if (x[c] > y[c]) {
                        a[lo[c]] = y[c];
                        a[mirror ? (lo[c] ^ (k - 1)) : (lo[c] + j)] = x[c];
                    }
            }
            __syncwarp();
        }
    }
}

// rows of at most wmax entries (32, or kAsmWarpMax with kAsmWarpMax keys of
// dynamic shared memory per warp), one warp per row; longer rows are left to
// k_assemble_long
__global__ void __launch_bounds__(32 * kAsmWarps) k_assemble(
    int64_t rows, const int64_t *__restrict__ row_ptr, const int64_t *__restrict__ st_off,
    const int32_t *__restrict__ st_cnt, const uint32_t *__restrict__ st_col, const float *__restrict__ st_val,
    int32_t *__restrict__ out_col, float *__restrict__ out_val, int wmax)
{
    extern __shared__ unsigned long long sk[];
    const int lane = threadIdx.x & 31;
    unsigned long long *key = sk + (threadIdx.x >> 5) * kAsmWarpMax;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < rows; r += nwarps) {
        const int cnt = st_cnt[r];
        const int64_t off = st_off[r], dst = row_ptr[r];
        if (cnt <= 32) {
            // rank by shuffles
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
        } else if (cnt <= wmax) {
            int P = 64;
            while (P < cnt) P <<= 1;
            for (int i = lane; i < P; i += 32) key[i] = i < cnt ? pack_entry(st_col[off + i], st_val[off + i]) : kKeyInf;
            __syncwarp();
            switch (P) {
            case 64: bitonic_warp_batched<64>(key, lane); break;
            case 128: bitonic_warp_batched<128>(key, lane); break;
            case 256: bitonic_warp_batched<256>(key, lane); break;
            case 512: bitonic_warp_batched<512>(key, lane); break;
            default: bitonic_warp_batched<1024>(key, lane); break;
            }
            for (int i = lane; i < cnt; i += 32) {
                const unsigned long long x = key[i];
                out_col[dst + i] = (int32_t)(x >> 32);
                out_val[dst + i] = __uint_as_float((uint32_t)x);
            }
            __syncwarp();
        }
    }
}

// one global comparator of the long-row sort on the output arrays
__device__ __forceinline__ void cmp_swap_global(int32_t *col, float *val, int64_t i, int64_t l)
{
    const int32_t x = col[i], y = col[l];
    if (x > y) {
        col[i] = y;
        col[l] = x;
        const float t = val[i];
        val[i] = val[l];
        val[l] = t;
    }
}

// rows longer than wmax, one block per row: tiles of kAsmTile entries
// are sorted in shared memory and written out; merges of larger blocks run
// their steps of distance >= kAsmTile on the output arrays in global memory
// and the shorter half-cleaners tile by tile in shared memory
__global__ void __launch_bounds__(kAsmLongThreads) k_assemble_long(
    int64_t rows, const int64_t *__restrict__ row_ptr, const int64_t *__restrict__ st_off,
    const int32_t *__restrict__ st_cnt, const uint32_t *__restrict__ st_col, const float *__restrict__ st_val,
    int32_t *out_col, float *out_val, int wmax)
{
    __shared__ unsigned long long tile[kAsmTile];
    __shared__ int64_t list[kAsmLongThreads];
    __shared__ int nlist;
    const int t = threadIdx.x;
    for (int64_t base = (int64_t)blockIdx.x * kAsmLongThreads; base < rows;
         base += (int64_t)gridDim.x * kAsmLongThreads) {
        if (t == 0) nlist = 0;
        __syncthreads();
        if (base + t < rows && st_cnt[base + t] > wmax) list[atomicAdd(&nlist, 1)] = base + t;
        __syncthreads();
        const int nl = nlist;
        for (int li = 0; li < nl; ++li) {
            const int64_t r = list[li];
            const int64_t cnt = st_cnt[r], off = st_off[r];
            int32_t *oc = out_col + row_ptr[r];
            float *ov = out_val + row_ptr[r];
            int64_t P = 1;
            while (P < cnt) P <<= 1;
            const int tp = P < kAsmTile ? (int)P : kAsmTile;
            // tiles sorted in shared memory
            for (int64_t c0 = 0; c0 < cnt; c0 += kAsmTile) {
                for (int i = t; i < tp; i += kAsmLongThreads)
                    tile[i] = c0 + i < cnt ? pack_entry(st_col[off + c0 + i], st_val[off + c0 + i]) : kKeyInf;
                __syncthreads();
                bitonic_shared<kAsmLongThreads, false>(tile, tp, t);
                for (int i = t; i < kAsmTile && c0 + i < cnt; i += kAsmLongThreads) {
                    const unsigned long long x = tile[i];
                    oc[c0 + i] = (int32_t)(x >> 32);
                    ov[c0 + i] = __uint_as_float((uint32_t)x);
                }
                __syncthreads();
            }
            // merges of blocks larger than a tile
            for (int64_t k = 2 * (int64_t)kAsmTile; k <= P; k <<= 1) {
                for (int64_t q = t; q < (P >> 1); q += kAsmLongThreads) {
                    const int64_t i = pair_lo(q, k >> 1), l = i ^ (k - 1);
                    if (l < cnt) cmp_swap_global(oc, ov, i, l);
                }
                __syncthreads();
                for (int64_t j = k >> 2; j >= kAsmTile; j >>= 1) {
                    for (int64_t q = t; q < (P >> 1); q += kAsmLongThreads) {
                        const int64_t i = pair_lo(q, j), l = i + j;
                        if (l < cnt) cmp_swap_global(oc, ov, i, l);
                    }
                    __syncthreads();
                }
                for (int64_t c0 = 0; c0 < cnt; c0 += kAsmTile) {
                    for (int i = t; i < kAsmTile; i += kAsmLongThreads)
                        tile[i] = c0 + i < cnt ? pack_entry((uint32_t)oc[c0 + i], ov[c0 + i]) : kKeyInf;
                    __syncthreads();
                    for (int j = kAsmTile >> 1; j > 0; j >>= 1) {
                        for (int q = t; q < (kAsmTile >> 1); q += kAsmLongThreads) {
                            const int i = (int)pair_lo(q, j);
                            cmp_swap(tile, i, i + j);
                        }
                        __syncthreads();
                    }
                    for (int i = t; i < kAsmTile && c0 + i < cnt; i += kAsmLongThreads) {
                        const unsigned long long x = tile[i];
                        oc[c0 + i] = (int32_t)(x >> 32);
                        ov[c0 + i] = __uint_as_float((uint32_t)x);
                    }
                    __syncthreads();
                }
            }
        }
        __syncthreads();   // list and nlist are rewritten in the next iteration
    }
}

static int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

cudaError_t launch_assemble(int64_t rows, const int64_t *row_ptr, const int64_t *st_off, const int32_t *st_cnt,
                            const uint32_t *st_col, const float *st_val, int32_t *out_col, float *out_val,
                            int64_t max_cnt, cudaStream_t s)
{
    if (rows <= 0) return cudaGetLastError();
    const int sms = sm_count();
    const int bs = 32 * kAsmWarps;
    // rows known to fit a warp's shuffles need no shared memory (more blocks per SM)
    const bool small = max_cnt > 0 && max_cnt <= 32;
    const int wmax = small ? 32 : kAsmWarpMax;
    const size_t smem = small ? 0 : (size_t)kAsmWarps * kAsmWarpMax * sizeof(unsigned long long);
    int64_t g = (rows * 32 + bs - 1) / bs;
    if (g > (int64_t)sms * 32) g = (int64_t)sms * 32;
    k_assemble<<<(unsigned)g, bs, smem, s>>>(rows, row_ptr, st_off, st_cnt, st_col, st_val, out_col, out_val, wmax);
    if (small) return cudaGetLastError();
    int64_t gl = (rows + kAsmLongThreads - 1) / kAsmLongThreads;
    if (gl > (int64_t)sms * 6) gl = (int64_t)sms * 6;
    k_assemble_long<<<(unsigned)gl, kAsmLongThreads, 0, s>>>(rows, row_ptr, st_off, st_cnt, st_col, st_val, out_col,
                                                             out_val, wmax);
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
