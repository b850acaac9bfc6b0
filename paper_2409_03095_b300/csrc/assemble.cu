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

// Stable LSD radix sort of n <= kAsmWarpMax 32-bit keys in a[] by their bits
// [lo, lo + bits), 8 bits per pass, by one warp (b[]: scratch of n keys,
// cnt[]: 256 counters).  Each pass counts the digits, scans the counts, and
// scatters the keys 32 at a time in their input order: lanes holding the
// same digit find each other with __match_any_sync and take consecutive
// places, so every pass is stable.  Returns the buffer holding the result.
__device__ __forceinline__ uint32_t *radix_warp(uint32_t *a, uint32_t *b, uint32_t *cnt, int n, int lo, int bits,
                                                int lane)
{
    const uint32_t lt = (1u << lane) - 1u;
    for (int sh = lo; sh < lo + bits; sh += 8) {
        for (int d = lane; d < 256; d += 32) cnt[d] = 0u;
        __syncwarp();
        for (int i = lane; i < n; i += 32) atomicAdd(&cnt[(a[i] >> sh) & 255u], 1u);
        __syncwarp();
        // exclusive scan: lane l holds counters 8l .. 8l + 7
        uint32_t c8[8], tot = 0u;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            c8[u] = cnt[8 * lane + u];
            tot += c8[u];
        }
        uint32_t incl = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t nb = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += nb;
        }
        uint32_t run = incl - tot;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            cnt[8 * lane + u] = run;
            run += c8[u];
        }
        __syncwarp();
        for (int base = 0; base < n; base += 32) {
            const int i = base + lane;
            const bool v = i < n;
            const uint32_t k = v ? a[i] : 0u;
            const uint32_t d = (k >> sh) & 255u;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, v ? d : 256u + (uint32_t)lane);
            const uint32_t pos = cnt[d] + (uint32_t)__popc(peers & lt);
            __syncwarp();
            if (v && 31 - __clz(peers) == lane) cnt[d] += (uint32_t)__popc(peers);   // the group's last lane
            __syncwarp();
            if (v) b[pos] = k;
        }
        __syncwarp();
        uint32_t *t = a;
        a = b;
        b = t;
    }
    return a;
}

// rows of at most wmax entries (32, or kAsmWarpMax with kAsmWarpMax keys of
// dynamic shared memory per warp), one warp per row; longer rows are left to
// k_assemble_long.  A row whose columns span less than 2^22 is sorted by a
// radix sort of 32-bit keys (column - row minimum) << 10 | staging index;
// wider rows take the bitonic network on (column, value) keys.
__global__ void __launch_bounds__(32 * kAsmWarps) k_assemble(
    int64_t rows, const int64_t *__restrict__ row_ptr, const int64_t *__restrict__ st_off,
    const int32_t *__restrict__ st_cnt, const uint32_t *__restrict__ st_col, const float *__restrict__ st_val,
    int32_t *__restrict__ out_col, float *__restrict__ out_val, int wmax)
{
    extern __shared__ unsigned long long sk[];
    const int lane = threadIdx.x & 31;
    unsigned long long *key = sk + (threadIdx.x >> 5) * kAsmWarpMax;
    uint32_t *rcnt = reinterpret_cast<uint32_t *>(sk + kAsmWarps * kAsmWarpMax) + (threadIdx.x >> 5) * 256;
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
            // the row's column range decides the sort
            uint32_t cmin = 0xFFFFFFFFu, cmax = 0u;
            for (int i = lane; i < cnt; i += 32) {
                const uint32_t c = st_col[off + i];
                cmin = min(cmin, c);
                cmax = max(cmax, c);
            }
            for (int o = 16; o > 0; o >>= 1) {
                cmin = min(cmin, __shfl_xor_sync(0xFFFFFFFFu, cmin, o));
                cmax = max(cmax, __shfl_xor_sync(0xFFFFFFFFu, cmax, o));
            }
            const uint32_t range = cmax - cmin;
            if (range < (1u << 22)) {
                uint32_t *ka = reinterpret_cast<uint32_t *>(key), *kb = ka + kAsmWarpMax;
                for (int i = lane; i < cnt; i += 32) ka[i] = ((st_col[off + i] - cmin) << 10) | (uint32_t)i;
                __syncwarp();
                const int bits = range ? 32 - __clz(range) : 1;
                const uint32_t *sorted = radix_warp(ka, kb, rcnt, cnt, 10, bits, lane);
                for (int i = lane; i < cnt; i += 32) {
                    const uint32_t k = sorted[i];
                    out_col[dst + i] = (int32_t)(cmin + (k >> 10));
                    out_val[dst + i] = st_val[off + (k & 1023u)];
                }
                __syncwarp();
                continue;
            }
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

// Stable LSD radix sort of n <= kAsmTile 32-bit keys by their bits
// [lo, lo + bits), 8 bits per pass, by the whole block (kAsmLongThreads
// threads): warp w owns a contiguous segment of the keys, counts its digits
// in its own 256 counters, and after a block-wide scan over (digit, warp)
// scatters its segment 32 keys at a time in input order (lanes with the same
// digit take consecutive places, found with __match_any_sync), so every
// pass is stable.  Returns the buffer holding the result.
__device__ __forceinline__ uint32_t *radix_block(uint32_t *a, uint32_t *b, uint32_t *cnt, uint32_t *dsum, int n,
                                                 int lo, int bits)
{
    constexpr int NW = kAsmLongThreads / 32;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int seg = (((n + NW - 1) / NW) + 31) & ~31;
    const int s0 = w * seg, s1 = min(n, s0 + seg);
    uint32_t *my = cnt + 256 * w;
    for (int sh = lo; sh < lo + bits; sh += 8) {
        for (int d = lane; d < 256; d += 32) my[d] = 0u;
        __syncwarp();
        for (int i = s0 + lane; i < s1; i += 32) atomicAdd(&my[(a[i] >> sh) & 255u], 1u);
        __syncthreads();
        // digit totals, their exclusive scan, then each warp's cursor per digit
        if (t < 256) {
            uint32_t tot = 0u;
            for (int v = 0; v < NW; ++v) tot += cnt[256 * v + t];
            dsum[t] = tot;
        }
        __syncthreads();
        if (t < 32) {
            uint32_t c8[8], tot = 0u;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                c8[u] = dsum[8 * t + u];
                tot += c8[u];
            }
            uint32_t incl = tot;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t nb = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (t >= o) incl += nb;
            }
            uint32_t run = incl - tot;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                dsum[8 * t + u] = run;
                run += c8[u];
            }
        }
        __syncthreads();
        if (t < 256) {
            uint32_t run = dsum[t];
            for (int v = 0; v < NW; ++v) {
                const uint32_t c = cnt[256 * v + t];
                cnt[256 * v + t] = run;
                run += c;
            }
        }
        __syncthreads();
        for (int base = s0; base < s1; base += 32) {
            const int i = base + lane;
            const bool v = i < s1;
            const uint32_t k = v ? a[i] : 0u;
            const uint32_t d = (k >> sh) & 255u;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, v ? d : 256u + (uint32_t)lane);
            const uint32_t pos = my[d] + (uint32_t)__popc(peers & lt);
            __syncwarp();
            if (v && 31 - __clz(peers) == lane) my[d] += (uint32_t)__popc(peers);   // the group's last lane
            __syncwarp();
            if (v) b[pos] = k;
        }
        __syncthreads();
        uint32_t *tmp = a;
        a = b;
        b = tmp;
    }
    return a;
}

// rows longer than wmax, one block per row.  A row of at most kAsmTile
// entries whose columns span less than 2^20 is sorted by a block radix sort
// of 32-bit keys (column - row minimum) << 12 | staging index.  Other rows:
// tiles of kAsmTile entries are sorted in shared memory and written out;
// merges of larger blocks run their steps of distance >= kAsmTile on the
// output arrays in global memory and the shorter half-cleaners tile by tile
// in shared memory
__global__ void __launch_bounds__(kAsmLongThreads) k_assemble_long(
    int64_t rows, const int64_t *__restrict__ row_ptr, const int64_t *__restrict__ st_off,
    const int32_t *__restrict__ st_cnt, const uint32_t *__restrict__ st_col, const float *__restrict__ st_val,
    int32_t *out_col, float *out_val, int wmax)
{
    __shared__ unsigned long long tile[kAsmTile];
    __shared__ uint32_t rcnt[256 * (kAsmLongThreads / 32)], rsum[256];
    __shared__ uint32_t rmin[kAsmLongThreads / 32], rmax[kAsmLongThreads / 32];
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
            if (cnt <= kAsmTile) {
                uint32_t lo = 0xFFFFFFFFu, hi = 0u;
                for (int64_t i = t; i < cnt; i += kAsmLongThreads) {
                    const uint32_t c = st_col[off + i];
                    lo = min(lo, c);
                    hi = max(hi, c);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    lo = min(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
                    hi = max(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
                }
                if ((t & 31) == 0) {
                    rmin[t >> 5] = lo;
                    rmax[t >> 5] = hi;
                }
                __syncthreads();
                uint32_t cmin = rmin[0], cmax = rmax[0];
                for (int v = 1; v < kAsmLongThreads / 32; ++v) {
                    cmin = min(cmin, rmin[v]);
                    cmax = max(cmax, rmax[v]);
                }
                const uint32_t range = cmax - cmin;
                if (range < (1u << 20)) {   // block-uniform
                    uint32_t *ka = reinterpret_cast<uint32_t *>(tile), *kb = ka + kAsmTile;
                    for (int i = t; i < (int)cnt; i += kAsmLongThreads)
                        ka[i] = ((st_col[off + i] - cmin) << 12) | (uint32_t)i;
                    __syncthreads();
                    const int bits = range ? 32 - __clz(range) : 1;
                    const uint32_t *sorted = radix_block(ka, kb, rcnt, rsum, (int)cnt, 12, bits);
                    for (int i = t; i < (int)cnt; i += kAsmLongThreads) {
                        const uint32_t k = sorted[i];
                        oc[i] = (int32_t)(cmin + (k >> 12));
                        ov[i] = st_val[off + (k & 4095u)];
                    }
                    __syncthreads();
                    continue;
                }
            }
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
    // per warp: kAsmWarpMax 64-bit keys (or two buffers of 32-bit radix keys) and 256 radix counters
    const size_t smem = small ? 0 : (size_t)kAsmWarps * (kAsmWarpMax * sizeof(unsigned long long) + 256 * sizeof(uint32_t));
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

// y = M x, LANES lanes per row (8 for short rows, a warp for long ones).
template <int LANES>
__global__ void k_spmv(int64_t rows, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                       const float *__restrict__ val, const float *__restrict__ x, float *__restrict__ y)
{
    constexpr int G = 32 / LANES;   // rows per warp
    const int sub = threadIdx.x & (LANES - 1);
    const int64_t grp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LANES;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / LANES;
    // the loop bound is uniform across the warp (G row groups per warp) so
    // that every lane reaches the shuffles
    for (int64_t r0 = grp - (grp % G); r0 < rows; r0 += ngrp) {
        const int64_t r = r0 + (grp % G);
        float acc = 0.0f;
        if (r < rows)
            for (int64_t k = rp[r] + sub; k < rp[r + 1]; k += LANES)
                acc = fmaf(__ldg(val + k), __ldg(x + __ldg(col + k)), acc);
#pragma unroll
        for (int o = LANES / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (sub == 0 && r < rows) y[r] = acc;
    }
}

cudaError_t launch_spmv(int64_t rows, int64_t nnz, const int64_t *rp, const int32_t *col, const float *val,
                        const float *x, float *y, cudaStream_t s)
{
    const int bs = 256;
    // rows of more than 64 entries on average take a warp each
    const bool wide = rows > 0 && nnz > 64 * rows;
    const int lanes = wide ? 32 : 8;
    int64_t g = (rows * lanes + bs - 1) / bs;
    if (g > 148 * 16) g = 148 * 16;
    if (g < 1) g = 1;
    if (wide) k_spmv<32><<<(unsigned)g, bs, 0, s>>>(rows, rp, col, val, x, y);
    else k_spmv<8><<<(unsigned)g, bs, 0, s>>>(rows, rp, col, val, x, y);
    return cudaGetLastError();
}

}  // namespace mcmi
