// Stages a3-a5 of the hot path in one kernel: the random walks of Eq. 2,
// the row accumulator (on-chip hash + global overflow table), the phase-4
// column scaling (fused: each visit adds W / d_col) and the Sec. IV-B
// filter, writing each row's kept entries to a staging buffer.
//
// One block per row at a time (rows taken from a device queue), threads as
// chains: a thread that finishes a chain takes the next chain index of the
// row, so live chains stay packed into the block's warps.
#include "mcmi_internal.cuh"
#include "kernels.h"

namespace mcmi {

namespace {

constexpr int kProbeOnChip = 32;   // on-chip probe window before overflowing
constexpr uint32_t kDead = 0x80000000u;

__device__ __forceinline__ uint32_t hash_home(uint32_t key, int log2)
{
    return (key * 0x9E3779B1u) >> (32 - log2);
}

// Compensated (Kahan) FP32 add of v into a packed {sum, compensation} word.
__device__ __forceinline__ void kahan_add(unsigned long long *p, float v)
{
    unsigned long long old = *(volatile unsigned long long *)p, assumed;
    do {
        assumed = old;
        const float sum = __uint_as_float((uint32_t)assumed);
        const float c = __uint_as_float((uint32_t)(assumed >> 32));
        const float y = __fsub_rn(v, c);
        const float t = __fadd_rn(sum, y);
        const float cn = __fsub_rn(__fsub_rn(t, sum), y);
        const unsigned long long nv =
            (unsigned long long)__float_as_uint(t) | ((unsigned long long)__float_as_uint(cn) << 32);
        old = atomicCAS(p, assumed, nv);
    } while (old != assumed);
}

template <int PREC>
__device__ __forceinline__ void acc_add(unsigned long long *p, double v)
{
    if (PREC == 64)
        atomicAdd(reinterpret_cast<double *>(p), v);
    else
        kahan_add(p, (float)v);
}

template <int PREC>
__device__ __forceinline__ double acc_value(unsigned long long raw, int N)
{
    if (PREC == 64) return __ddiv_rn(__longlong_as_double((long long)raw), (double)N);
    const float sum = __uint_as_float((uint32_t)raw);
    const float c = __uint_as_float((uint32_t)(raw >> 32));
    return (double)__fdiv_rn(__fsub_rn(sum, c), (float)N);
}

template <int PREC>
__device__ __forceinline__ void acc_merge(unsigned long long *dst, unsigned long long src)
{
    if (PREC == 64) {
        atomicAdd(reinterpret_cast<double *>(dst), __longlong_as_double((long long)src));
    } else {
        const float sum = __uint_as_float((uint32_t)src);
        const float c = __uint_as_float((uint32_t)(src >> 32));
        kahan_add(dst, __fsub_rn(sum, c));
    }
}

__device__ __forceinline__ float block_max(float v, float *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    v = l < (int)(blockDim.x >> 5) ? red[l] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}

__device__ __forceinline__ unsigned long long block_sum(unsigned long long v, unsigned long long *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    v = l < (int)(blockDim.x >> 5) ? red[l] : 0ull;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Ranking key of the filter: magnitude first, then the smaller column.
__device__ __forceinline__ unsigned long long rank_key(double v, uint32_t col)
{
    return ((unsigned long long)__float_as_uint(fabsf((float)v)) << 32) | (unsigned long long)(~col);
}

}  // namespace

template <int PREC, int TABLE, bool DUMP>
__global__ void __launch_bounds__(256) k_walk(WalkArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = 1 << a.log2H;
    unsigned long long *s_vals = reinterpret_cast<unsigned long long *>(smem);
    uint32_t *s_keys = reinterpret_cast<uint32_t *>(s_vals + H);
    uint32_t *s_cnt = s_keys + H;   // DUMP only

    __shared__ long long s_row, s_pos;
    __shared__ int s_next_chain;
    __shared__ uint32_t s_nspill, s_fill, s_wpos;
    __shared__ long long s_off;
    __shared__ float s_redf[32];
    __shared__ unsigned long long s_redu[32];
    __shared__ uint32_t s_hist[256];
    __shared__ unsigned long long s_prefix;
    __shared__ uint32_t s_kk;

    const int tid = threadIdx.x, B = blockDim.x;
    const uint32_t fill_cap = (uint32_t)(H - (H >> 2));      // on-chip table kept <= 75% full
    const int G = 1 << a.log2G;
    uint32_t *gk = a.g_keys + ((size_t)blockIdx.x << a.log2G);
    unsigned long long *gv = a.g_vals + ((size_t)blockIdx.x << a.log2G);
    uint32_t *gc = a.g_cnt + ((size_t)blockIdx.x << a.log2G);
    uint32_t *gl = a.g_list + ((size_t)blockIdx.x << a.log2G);
    const long long total = a.row_list ? a.n_list : a.row_end - a.row_begin;

    for (int h = tid; h < H; h += B) {
        s_keys[h] = kEmpty;
        s_vals[h] = 0ull;
        if (DUMP) s_cnt[h] = 0u;
    }
    if (tid == 0) { s_nspill = 0; s_fill = 0; }

    // Adds value v at column col of the current row.
    auto accumulate = [&](uint32_t col, double v) {
        uint32_t h = hash_home(col, a.log2H);
#pragma unroll 1
        for (int p = 0; p < kProbeOnChip; ++p) {
            const uint32_t k = ((volatile uint32_t *)s_keys)[h];
            bool hit = k == col;
            if (!hit && k == kEmpty) {
                if (*(volatile uint32_t *)&s_fill >= fill_cap) break;
                const uint32_t old = atomicCAS(&s_keys[h], kEmpty, col);
                if (old == kEmpty) atomicAdd(&s_fill, 1u);
                hit = old == kEmpty || old == col;
            }
            if (hit) {
                acc_add<PREC>(&s_vals[h], v);
                if (DUMP) atomicAdd(&s_cnt[h], 1u);
                return;
            }
            h = (h + 1) & (uint32_t)(H - 1);
        }
        // global overflow table (never more than half full by its sizing)
        uint32_t g = hash_home(col, a.log2G);
#pragma unroll 1
        for (int p = 0; p < G; ++p) {
            const uint32_t k = ((volatile uint32_t *)gk)[g];
            bool hit = k == col;
            if (!hit && k == kEmpty) {
                const uint32_t old = atomicCAS(&gk[g], kEmpty, col);
                if (old == kEmpty) {
                    const uint32_t slot = atomicAdd(&s_nspill, 1u);
                    gl[slot] = g;
                }
                hit = old == kEmpty || old == col;
            }
            if (hit) {
                acc_add<PREC>(&gv[g], v);
                if (DUMP) atomicAdd(&gc[g], 1u);
                return;
            }
            g = (g + 1) & (uint32_t)(G - 1);
        }
        report(a.st, s_row, MCMI_ERR_CAPACITY);
    };

    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const long long pos = (long long)atomicAdd(&a.st->work, 1ull);
            s_pos = pos < total ? pos : -1;
            s_row = pos < total ? (a.row_list ? a.row_list[pos] : a.row_begin + pos) : -1;
            s_next_chain = B;
            if (s_row >= 0) {
                // t = 0 visits of all N chains: weight 1 at the row itself.
                const uint32_t r = (uint32_t)s_row;
                const uint32_t h = hash_home(r, a.log2H);
                s_keys[h] = r;
                s_fill = 1;
                if (PREC == 64) {
                    const double invd = a.rowd[r].y;
                    s_vals[h] = (unsigned long long)__double_as_longlong(__dmul_rn((double)a.N, invd));
                } else {
                    const float invd = __uint_as_float(__ldg(&a.slots[4 * (size_t)r].z));
                    s_vals[h] = (unsigned long long)__float_as_uint(__fmul_rn((float)a.N, invd));
                }
                if (DUMP) s_cnt[h] = (uint32_t)a.N;
            }
        }
        __syncthreads();
        const long long row = s_row, pos = s_pos;
        if (row < 0) break;
        const long long idx = (a.row_list && !a.out_by_row) ? pos : row - a.row_begin;
        const uint32_t rlo = (uint32_t)row, rhi = (uint32_t)((unsigned long long)row >> 32);

        // ---- walks (Eq. 2) ----
        unsigned long long my_steps = 0;
        for (int k = tid; k < a.N; k = atomicAdd(&s_next_chain, 1)) {
            uint32_t st = (uint32_t)row;
            float w = 1.0f;            // FP32 weight (the FP64 path keeps it as the stop shadow)
            double w64 = 1.0;
            uint4 r4 = make_uint4(0, 0, 0, 0);
            int t = 0;
#pragma unroll 1
            for (;;) {
                const uint4 *sp = a.slots + 4 * (size_t)st;
                const uint4 h0 = __ldg(sp);
                const uint4 h1 = __ldg(sp + 1);
                const uint4 h2 = __ldg(sp + 2);
                const uint4 h3 = __ldg(sp + 3);
                double2 rd = make_double2(0.0, 0.0);
                if (PREC == 64) rd = __ldg(a.rowd + st);
                if (t > 0) {
                    if (PREC == 64)
                        accumulate(st, __dmul_rn(w64, rd.y));
                    else
                        accumulate(st, (double)__fmul_rn(w, __uint_as_float(h0.z)));
                }
                const uint32_t Q = h0.x;
                if (t == a.L || !(fabsf(w) >= a.delta_f) || Q == 0u) break;
                if ((t & 3) == 0) r4 = philox4x32_10(make_uint4((uint32_t)(t >> 2), (uint32_t)k, rlo, rhi), a.key0, a.key1);
                const int ph = t & 3;
                const uint32_t r = ph == 0 ? r4.x : ph == 1 ? r4.y : ph == 2 ? r4.z : r4.w;
                const uint32_t deg = h0.w & ~kOolFlag;
                uint32_t cs;
                if (TABLE == MCMI_TABLE_CUMULATIVE) {
                    const uint32_t x = __umulhi(r, Q);
                    if (!(h0.w & kOolFlag)) {
                        const uint32_t m = (h1.x <= x) + (h1.z <= x) + (h2.x <= x) + (h2.z <= x) +
                                           (h3.x <= x) + (h3.z <= x);
                        cs = m == 0 ? h1.y : m == 1 ? h1.w : m == 2 ? h2.y : m == 3 ? h2.w : m == 4 ? h3.y : h3.w;
                    } else {
                        const uint32_t *T = a.ool_a + h1.x;
                        uint32_t lo = 0, hi = deg - 1;
#pragma unroll 1
                        while (lo < hi) {
                            const uint32_t mid = (lo + hi) >> 1;
                            if (x < __ldg(T + mid)) hi = mid; else lo = mid + 1;
                        }
                        cs = __ldg(a.ool_b + h1.x + lo);
                    }
                } else {
                    const unsigned long long pr = (unsigned long long)r * deg;
                    const uint32_t b = (uint32_t)(pr >> 32);
                    const uint32_t y = __umulhi((uint32_t)pr, Q);
                    uint32_t prob, own, al;
                    if (!(h0.w & kOolFlag)) {
                        prob = b == 0 ? h1.x : b == 1 ? h1.w : b == 2 ? h2.z : h3.y;
                        own = b == 0 ? h1.y : b == 1 ? h2.x : b == 2 ? h2.w : h3.z;
                        al = b == 0 ? h1.z : b == 1 ? h2.y : b == 2 ? h3.x : h3.w;
                    } else {
                        const uint4 bk = __ldg(a.ool_bkt + h1.x + b);
                        prob = bk.x; own = bk.y; al = bk.z;
                    }
                    cs = y < prob ? own : al;
                }
                const float f = __uint_as_float(h0.y);
                const bool neg = (cs & kNegBit) != 0u;
                w = __fmul_rn(w, neg ? -f : f);
                if (PREC == 64) w64 = __dmul_rn(w64, neg ? -rd.x : rd.x);
                st = cs & ~kNegBit;
                ++t;
            }
            my_steps += (unsigned long long)t;
        }
        __syncthreads();

        // ---- row statistics ----
        const unsigned long long row_steps = block_sum(my_steps, s_redu);
        if (tid == 0) {
            atomicAdd(&a.st->steps, row_steps);
            if (a.row_steps) a.row_steps[idx] = row_steps;
            if (s_nspill) atomicAdd(&a.st->spilled, (unsigned long long)s_nspill);
            s_wpos = 0;
        }
        const uint32_t nsp = s_nspill;
        // overflow entries whose key also sits on chip are merged into it
        for (uint32_t e = tid; e < nsp; e += B) {
            const uint32_t g = gl[e];
            const uint32_t key = gk[g];
            uint32_t h = hash_home(key, a.log2H);
            for (int p = 0; p < kProbeOnChip; ++p) {
                const uint32_t k = s_keys[h];
                if (k == kEmpty) break;
                if (k == key) {
                    acc_merge<PREC>(&s_vals[h], gv[g]);
                    if (DUMP) atomicAdd(&s_cnt[h], gc[g]);
                    gl[e] = g | kDead;
                    break;
                }
                h = (h + 1) & (uint32_t)(H - 1);
            }
        }
        __syncthreads();

        if (DUMP) {
            // every accumulator entry, unfiltered
            for (int h = tid; h < H; h += B) {
                const uint32_t k = s_keys[h];
                if (k == kEmpty) continue;
                const uint32_t p = atomicAdd(&s_wpos, 1u);
                if (p < (uint32_t)a.d_cap) {
                    a.d_col[idx * a.d_cap + p] = (int32_t)k;
                    a.d_val[idx * a.d_cap + p] = acc_value<PREC>(s_vals[h], a.N);
                    a.d_vis[idx * a.d_cap + p] = s_cnt[h];
                }
            }
            for (uint32_t e = tid; e < nsp; e += B) {
                const uint32_t g = gl[e];
                if (g & kDead) continue;
                const uint32_t p = atomicAdd(&s_wpos, 1u);
                if (p < (uint32_t)a.d_cap) {
                    a.d_col[idx * a.d_cap + p] = (int32_t)gk[g];
                    a.d_val[idx * a.d_cap + p] = acc_value<PREC>(gv[g], a.N);
                    a.d_vis[idx * a.d_cap + p] = gc[g];
                }
            }
            __syncthreads();
            if (tid == 0) {
                const uint32_t c = s_wpos;
                a.d_count[idx] = c <= (uint32_t)a.d_cap ? (int32_t)c : -1;
                if (c > (uint32_t)a.d_cap) report(a.st, row, MCMI_ERR_CAPACITY);
            }
        } else {
            // ---- Sec. IV-B filter: diagonal kept; tau rule; top-k ----
            float lmax = 0.0f;
            for (int h = tid; h < H; h += B)
                if (s_keys[h] != kEmpty) lmax = fmaxf(lmax, fabsf((float)acc_value<PREC>(s_vals[h], a.N)));
            for (uint32_t e = tid; e < nsp; e += B)
                if (!(gl[e] & kDead)) lmax = fmaxf(lmax, fabsf((float)acc_value<PREC>(gv[gl[e]], a.N)));
            // the row maximum in the accumulator's precision, then the FP64 threshold
            double rowmax = (double)block_max(lmax, s_redf);
            if (PREC == 64) {
                // exact FP64 maximum for the FP64 path
                unsigned long long lm = 0;
                for (int h = tid; h < H; h += B)
                    if (s_keys[h] != kEmpty) {
                        const double v = fabs(acc_value<PREC>(s_vals[h], a.N));
                        lm = max(lm, (unsigned long long)__double_as_longlong(v));
                    }
                for (uint32_t e = tid; e < nsp; e += B)
                    if (!(gl[e] & kDead)) {
                        const double v = fabs(acc_value<PREC>(gv[gl[e]], a.N));
                        lm = max(lm, (unsigned long long)__double_as_longlong(v));
                    }
                for (int o = 16; o > 0; o >>= 1) lm = max(lm, __shfl_xor_sync(0xFFFFFFFFu, lm, o));
                __syncthreads();
                if ((tid & 31) == 0) s_redu[tid >> 5] = lm;
                __syncthreads();
                lm = 0;
                for (int w = 0; w < (B >> 5); ++w) lm = max(lm, s_redu[w]);
                rowmax = __longlong_as_double((long long)lm);
            }
            const double thr = a.tau > 0.0 ? __dmul_rn(a.tau, rowmax) : 0.0;
            const uint32_t rowc = (uint32_t)row;
            auto is_cand = [&](uint32_t k, double v) -> bool {
                return k != rowc && (a.tau <= 0.0 || fabs(v) >= thr);
            };
            unsigned long long nc_l = 0;
            for (int h = tid; h < H; h += B) {
                const uint32_t k = s_keys[h];
                if (k != kEmpty && is_cand(k, acc_value<PREC>(s_vals[h], a.N))) ++nc_l;
            }
            for (uint32_t e = tid; e < nsp; e += B) {
                const uint32_t g = gl[e];
                if (!(g & kDead) && is_cand(gk[g], acc_value<PREC>(gv[g], a.N))) ++nc_l;
            }
            const unsigned long long nc = block_sum(nc_l, s_redu);
            const bool select = a.top_k > 0 && nc > (unsigned long long)a.top_k;
            unsigned long long kstar = 0;
            if (select) {
                // radix select of the top_k-th largest ranking key, 8 bits per pass
                if (tid == 0) { s_prefix = 0; s_kk = (uint32_t)a.top_k; }
                unsigned long long mask = 0;
                for (int shift = 56; shift >= 0; shift -= 8) {
                    for (int b = tid; b < 256; b += B) s_hist[b] = 0;
                    __syncthreads();
                    const unsigned long long pre = s_prefix;
                    for (int h = tid; h < H; h += B) {
                        const uint32_t k = s_keys[h];
                        if (k == kEmpty) continue;
                        const double v = acc_value<PREC>(s_vals[h], a.N);
                        if (!is_cand(k, v)) continue;
                        const unsigned long long rk = rank_key(v, k);
                        if ((rk & mask) == pre) atomicAdd(&s_hist[(rk >> shift) & 255u], 1u);
                    }
                    for (uint32_t e = tid; e < nsp; e += B) {
                        const uint32_t g = gl[e];
                        if (g & kDead) continue;
                        const double v = acc_value<PREC>(gv[g], a.N);
                        if (!is_cand(gk[g], v)) continue;
                        const unsigned long long rk = rank_key(v, gk[g]);
                        if ((rk & mask) == pre) atomicAdd(&s_hist[(rk >> shift) & 255u], 1u);
                    }
                    __syncthreads();
                    if (tid < 32) {
                        // warp scan from the top bin down: lane l owns bins 255-8l .. 248-8l
                        uint32_t c8[8], tot = 0;
#pragma unroll
                        for (int u = 0; u < 8; ++u) { c8[u] = s_hist[255 - 8 * tid - u]; tot += c8[u]; }
                        uint32_t incl = tot;
                        for (int o = 1; o < 32; o <<= 1) {
                            const uint32_t nb = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                            if (tid >= o) incl += nb;
                        }
                        const uint32_t kk = s_kk;
                        const uint32_t excl = incl - tot;
                        const bool mine = excl < kk && incl >= kk;
                        if (mine) {
                            uint32_t cum = excl;
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                if (cum + c8[u] >= kk) {
                                    s_prefix = pre | ((unsigned long long)(255 - 8 * tid - u) << shift);
                                    s_kk = kk - cum;
                                    break;
                                }
                                cum += c8[u];
                            }
                        }
                    }
                    mask |= 255ull << shift;
                    __syncthreads();
                }
                kstar = s_prefix;
            }
            const unsigned long long nk = 1ull + (select ? (unsigned long long)a.top_k : nc);
            if (tid == 0) {
                const unsigned long long off = atomicAdd(&a.st->cursor, nk);
                if (off + nk > a.st_cap) {
                    const unsigned long long dnum = atomicAdd(&a.st->deferred, 1ull);
                    a.deferred_list[dnum] = row;
                    a.row_cnt[idx] = -1;
                    s_off = -1;
                } else {
                    a.row_off[idx] = (int64_t)off;
                    a.row_cnt[idx] = (int32_t)nk;
                    s_off = (long long)off;
                }
            }
            __syncthreads();
            const long long off = s_off;
            if (off >= 0) {
                auto emit = [&](uint32_t k, double v) {
                    bool keep = k == rowc;
                    if (!keep && is_cand(k, v)) keep = !select || rank_key(v, k) >= kstar;
                    if (keep) {
                        const uint32_t p = atomicAdd(&s_wpos, 1u);
                        a.st_col[off + p] = k;
                        a.st_val[off + p] = (float)v;
                    }
                };
                for (int h = tid; h < H; h += B) {
                    const uint32_t k = s_keys[h];
                    if (k != kEmpty) emit(k, acc_value<PREC>(s_vals[h], a.N));
                }
                for (uint32_t e = tid; e < nsp; e += B) {
                    const uint32_t g = gl[e];
                    if (!(g & kDead)) emit(gk[g], acc_value<PREC>(gv[g], a.N));
                }
            }
        }
        __syncthreads();
        // ---- reset the accumulator for the next row ----
        for (int h = tid; h < H; h += B) {
            s_keys[h] = kEmpty;
            s_vals[h] = 0ull;
            if (DUMP) s_cnt[h] = 0u;
        }
        for (uint32_t e = tid; e < nsp; e += B) {
            const uint32_t g = gl[e] & ~kDead;
            gk[g] = kEmpty;
            gv[g] = 0ull;
            gc[g] = 0u;
        }
        if (tid == 0) { s_nspill = 0; s_fill = 0; }
    }
}

template <int PREC, int TABLE, bool DUMP>
static cudaError_t launch_walk_t(const WalkArgs &a, int grid, int threads, size_t smem, cudaStream_t s)
{
    auto fn = k_walk<PREC, TABLE, DUMP>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

size_t walk_smem_bytes(int log2H, bool dump)
{
    return ((size_t)1 << log2H) * (dump ? 16 : 12);
}

cudaError_t walk_occupancy(int precision, int table, bool dump, int threads, int log2H, int *blocks_per_sm)
{
    const size_t smem = walk_smem_bytes(log2H, dump);
    const void *fn = nullptr;
#define MCMI_PICK(P, T, D) if (precision == P && table == T && dump == D) fn = (const void *)k_walk<P, T, D>;
    MCMI_PICK(32, 0, false) MCMI_PICK(32, 1, false) MCMI_PICK(64, 0, false) MCMI_PICK(64, 1, false)
    MCMI_PICK(32, 0, true) MCMI_PICK(32, 1, true) MCMI_PICK(64, 0, true) MCMI_PICK(64, 1, true)
#undef MCMI_PICK
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, threads, smem);
}

cudaError_t launch_walk(const WalkArgs &a, int precision, int table, bool dump, int grid, int threads,
                        cudaStream_t s)
{
    const size_t smem = walk_smem_bytes(a.log2H, dump);
    if (precision == 64) {
        if (table == MCMI_TABLE_ALIAS)
            return dump ? launch_walk_t<64, 1, true>(a, grid, threads, smem, s)
                        : launch_walk_t<64, 1, false>(a, grid, threads, smem, s);
        return dump ? launch_walk_t<64, 0, true>(a, grid, threads, smem, s)
                    : launch_walk_t<64, 0, false>(a, grid, threads, smem, s);
    }
    if (table == MCMI_TABLE_ALIAS)
        return dump ? launch_walk_t<32, 1, true>(a, grid, threads, smem, s)
                    : launch_walk_t<32, 1, false>(a, grid, threads, smem, s);
    return dump ? launch_walk_t<32, 0, true>(a, grid, threads, smem, s)
                : launch_walk_t<32, 0, false>(a, grid, threads, smem, s);
}

}  // namespace mcmi
