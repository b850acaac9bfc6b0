// Stage a1 + a2 of the hot path: CSR validation, the Eq. 1 split with
// Jacobi scaling (FP64), and the per-row integer sampling tables.
#include "mcmi_internal.cuh"
#include "kernels.h"

namespace mcmi {

// One thread per row: row_ptr bounds, strictly increasing in-range columns,
// finite values.
__global__ void k_validate(int64_t n, int64_t nnz, const int64_t *__restrict__ rp,
                           const int32_t *__restrict__ col, const double *__restrict__ val,
                           DevState *st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = rp[i], b = rp[i + 1];
        if (i == 0 && a != 0) report(st, 0, MCMI_ERR_BAD_CSR);
        if (i == n - 1 && b != nnz) report(st, i, MCMI_ERR_BAD_CSR);
        if (a < 0 || b < a || b > nnz) {
            report(st, i, MCMI_ERR_BAD_CSR);
            continue;
        }
        int64_t prev = -1;
        bool diag = false;
        for (int64_t k = a; k < b; ++k) {
            const int64_t c = col[k];
            if (c < 0 || c >= n || c <= prev) report(st, i, MCMI_ERR_BAD_CSR);
            if (!isfinite(val[k])) report(st, i, MCMI_ERR_BAD_CSR);
            diag |= (c == i);
            prev = c;
        }
        if (diag) atomicAdd(&st->ndiag, 1ull);
    }
}

// Rows ordered by the length of their CSR row, longest first, in 16 classes
// (class 15 - min(floor(log2(len)), 15)), so that the threads of a warp of
// the one-thread-per-row kernels below get rows of similar length: on
// power-law rows a warp otherwise waits for its longest row.  The order
// inside a class is arbitrary; the kernels' results do not depend on it.
constexpr int kLenClasses = 16;

__device__ __forceinline__ int len_class(int64_t len)
{
    const int b = len > 0 ? 63 - __clzll((unsigned long long)len) : 0;
    return kLenClasses - 1 - (b < kLenClasses - 1 ? b : kLenClasses - 1);
}

// counts[0 .. 16): rows per class
__global__ void k_len_count(int64_t n, const int64_t *__restrict__ rp, unsigned long long *__restrict__ counts)
{
    __shared__ unsigned int h[kLenClasses];
    if (threadIdx.x < kLenClasses) h[threadIdx.x] = 0u;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[len_class(rp[i + 1] - rp[i])], 1u);
    __syncthreads();
    if (threadIdx.x < kLenClasses && h[threadIdx.x]) atomicAdd(&counts[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

// order[...]: the rows, class by class (counts from k_len_count; cursor[16]
// zero at launch).  Each block reserves its range of every class with one
// atomic, then places its rows inside it.
__global__ void k_len_scatter(int64_t n, const int64_t *__restrict__ rp, const unsigned long long *__restrict__ counts,
                              unsigned long long *__restrict__ cursor, int32_t *__restrict__ order)
{
    __shared__ unsigned int h[kLenClasses];
    __shared__ unsigned long long base[kLenClasses];
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < n; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        if (threadIdx.x < kLenClasses) h[threadIdx.x] = 0u;
        __syncthreads();
        const int c = i < n ? len_class(rp[i + 1] - rp[i]) : 0;
        const unsigned int pos = i < n ? atomicAdd(&h[c], 1u) : 0u;
        __syncthreads();
        if (threadIdx.x < kLenClasses) {
            unsigned long long start = 0;
            for (int k = 0; k < (int)threadIdx.x; ++k) start += counts[k];
            base[threadIdx.x] = start + (h[threadIdx.x] ? atomicAdd(&cursor[threadIdx.x], (unsigned long long)h[threadIdx.x]) : 0ull);
        }
        __syncthreads();
        if (i < n) order[base[c] + pos] = (int32_t)i;
        __syncthreads();
    }
}

// ||B||_inf for the Eq. 1 augmentation.
__global__ void k_rownorm(int64_t n, const int64_t *__restrict__ rp, const double *__restrict__ val,
                          DevState *st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double r = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) r = __dadd_rn(r, fabs(val[k]));
        atomicMax(&st->bnorm_bits, (unsigned long long)__double_as_longlong(r));
    }
}

// Eq. 1 + Jacobi scaling: d_i = b_ii + alpha ||B|| sgn(b_ii), c_ij = -b_ij/d_i,
// s_i = sum_j |c_ij| in CSR order (explicitly rounded operations, no FMA).
__global__ void k_split(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                        const double *__restrict__ val, double alpha, double *__restrict__ d,
                        double *__restrict__ s, DevState *st, const int32_t *__restrict__ order)
{
    const double bnorm = __longlong_as_double((long long)st->bnorm_bits);
    // this thread's extremes over its rows, combined per warp before the
    // device-wide atomics (s_i >= 0: the bit patterns order like the values)
    unsigned long long smax = 0, smin = ~0ull, dmax = 0, omax = 0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = order ? (int64_t)order[q] : q;
        const int64_t a = rp[i], b = rp[i + 1];
        double bii = 0.0;
        unsigned long long ndeg = 0;   // off-diagonals and their largest |j - i|
        for (int64_t k = a; k < b; ++k) {
            if (col[k] == i) {
                bii = val[k];
            } else {
                ++ndeg;
                const long long o = (long long)col[k] - (long long)i;
                const unsigned long long ao = (unsigned long long)(o < 0 ? -o : o);
                omax = ao > omax ? ao : omax;
            }
        }
        dmax = ndeg > dmax ? ndeg : dmax;
        double di = bii;
        if (alpha > 0.0) di = __dadd_rn(bii, __dmul_rn(__dmul_rn(alpha, bnorm), bii < 0.0 ? -1.0 : 1.0));
        if (di == 0.0) {
            report(st, i, MCMI_ERR_ZERO_DIAG);
            d[i] = 0.0;
            s[i] = 0.0;
            continue;
        }
        double si = 0.0;
        for (int64_t k = a; k < b; ++k) {
            if (col[k] == i) continue;
            si = __dadd_rn(si, fabs(__ddiv_rn(-val[k], di)));
        }
        d[i] = di;
        s[i] = si;
        if (!(si < 1.0)) report(st, i, MCMI_ERR_NOT_CONTRACTIVE);
        const unsigned long long sb = (unsigned long long)__double_as_longlong(si);
        smax = sb > smax ? sb : smax;
        if (si > 0.0) smin = sb < smin ? sb : smin;
    }
    // every lane reaches this point (the row loop has no early exit)
    for (int o = 16; o > 0; o >>= 1) {
        smax = max(smax, __shfl_xor_sync(0xFFFFFFFFu, smax, o));
        smin = min(smin, __shfl_xor_sync(0xFFFFFFFFu, smin, o));
        dmax = max(dmax, __shfl_xor_sync(0xFFFFFFFFu, dmax, o));
        omax = max(omax, __shfl_xor_sync(0xFFFFFFFFu, omax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&st->smax_bits, smax);
        if (smin != ~0ull) atomicMin(&st->smin_bits, smin);
        atomicMax(&st->max_deg, dmax);
        atomicMax(&st->max_off, omax);
    }
}

// Integer weight of one entry: max(1, floor(|c|/s scale)); 0 if c == 0.
// scale = 2^31, or 2^20 for the compact table.
__device__ __forceinline__ uint32_t entry_weight(double b, double di, double si, bool *neg,
                                                double scale = 2147483648.0)
{
    const double c = __ddiv_rn(-b, di);
    *neg = c < 0.0;
    if (c == 0.0 || !(si > 0.0)) return 0u;
    const double x = floor(__dmul_rn(__ddiv_rn(fabs(c), si), scale));
    const uint32_t q = (uint32_t)x;
    return q < 1u ? 1u : q;
}

// One thread per row: the 64-byte slot (header + inline table) or the
// out-of-line table at [row_ptr[i], row_ptr[i] + deg); for the compact
// table the 32-byte record and the FP32 1/d_i.
//   cumulative: T_m = q_0 + ... + q_m; a draw x = floor(r Q / 2^32) picks
//               the smallest m with x < T_m.
//   alias:      Walker/Vose over weights q_j * deg with bucket capacity Q;
//               LIFO work lists filled in CSR order.
__global__ void k_tables(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                         const double *__restrict__ val, const double *__restrict__ d,
                         const double *__restrict__ s, int table, uint4 *__restrict__ slots,
                         uint32_t *__restrict__ ool_a, uint32_t *__restrict__ ool_b,
                         uint32_t *__restrict__ ool_c, uint4 *__restrict__ ool_bkt,
                         unsigned long long *__restrict__ wscratch,
                         uint32_t *__restrict__ small_stk, uint32_t *__restrict__ large_stk,
                         double2 *__restrict__ rowd, float *__restrict__ invd32, const int32_t *__restrict__ order)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = order ? (int64_t)order[q] : q;
        const int64_t a = rp[i], b = rp[i + 1];
        const double di = d[i], si = s[i];
        if (table == MCMI_TABLE_COMPACT) {
            // 32-byte record (layout in mcmi_internal.cuh); the host checked
            // that every row has at most six off-diagonals within the offset range
            uint32_t T[kCompactMaxDeg], h[kCompactMaxDeg];
#pragma unroll
            for (int u = 0; u < kCompactMaxDeg; ++u) { T[u] = 0u; h[u] = 0u; }
            uint32_t Q = 0, m = 0;
            for (int64_t k = a; k < b; ++k) {
                if (col[k] == i) continue;
                bool ng;
                Q += entry_weight(val[k], di, si, &ng, 1048576.0);
                const uint32_t hv = ((uint32_t)(col[k] - (int32_t)i) << 1 | (ng ? 1u : 0u)) & 0xFFFFu;
#pragma unroll
                for (int u = 0; u < kCompactMaxDeg; ++u)
                    if (u == (int)m) { T[u] = Q; h[u] = hv; }
                ++m;
            }
            // thresholds past the last transition hold Q: never below a draw
#pragma unroll
            for (int u = 0; u < kCompactMaxDeg; ++u)
                if (u >= (int)m) T[u] = Q;
            const unsigned long long A = (unsigned long long)Q | ((unsigned long long)T[0] << 21) |
                                         ((unsigned long long)T[1] << 42);
            const unsigned long long Bt = (unsigned long long)T[2] | ((unsigned long long)T[3] << 21) |
                                          ((unsigned long long)T[4] << 42);
            uint4 *o = slots + 2 * i;
            o[0] = make_uint4(__float_as_uint(__double2float_rn(si)), (uint32_t)A, (uint32_t)(A >> 32), (uint32_t)Bt);
            o[1] = make_uint4((uint32_t)(Bt >> 32), h[0] | h[1] << 16, h[2] | h[3] << 16, h[4] | h[5] << 16);
            invd32[i] = __double2float_rn(__ddiv_rn(1.0, di));
            if (rowd) rowd[i] = make_double2(si, __ddiv_rn(1.0, di));
            continue;
        }
        uint32_t w[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) w[k] = 0u;
        // pass 1: the degree; for alias rows also each weight and sign, kept
        // in wscratch (q | neg << 32) so that the FP64 divisions run once
        uint32_t deg = 0;
        for (int64_t k = a; k < b; ++k) deg += col[k] != i;
        const bool cum_row = table == MCMI_TABLE_CUMULATIVE || (table == MCMI_TABLE_HYBRID && deg <= (uint32_t)kInlineCum);
        unsigned long long Q = 0;
        if (!cum_row) {
            uint32_t m = 0;
            for (int64_t k = a; k < b; ++k) {
                if (col[k] == i) continue;
                bool ng;
                const uint32_t q = entry_weight(val[k], di, si, &ng);
                Q += q;
                wscratch[(uint32_t)a + m++] = (unsigned long long)q | (ng ? (1ull << 32) : 0ull);
            }
        }
        w[0] = (uint32_t)Q;
        w[1] = __float_as_uint(__double2float_rn(si));
        w[2] = __float_as_uint(__double2float_rn(__ddiv_rn(1.0, di)));
        if (invd32) invd32[i] = __uint_as_float(w[2]);
        if (rowd) rowd[i] = make_double2(si, __ddiv_rn(1.0, di));
        const uint32_t begin = (uint32_t)a;
        // the hybrid table takes the cumulative layout for rows of at most
        // kInlineCum transitions (always inline) and the alias layout otherwise
        if (cum_row) {
            const bool inl = deg <= (uint32_t)kInlineCum;
            w[3] = deg | (inl ? 0u : kOolFlag) | (table == MCMI_TABLE_HYBRID ? kCumFlag : 0u);
            if (inl) {
#pragma unroll
                for (int m = 0; m < kInlineCum; ++m) { w[4 + 2 * m] = 0xFFFFFFFFu; w[5 + 2 * m] = 0u; }
            } else {
                w[4] = begin;
            }
            uint32_t T = 0, m = 0;
            for (int64_t k = a; k < b; ++k) {
                if (col[k] == i) continue;
                bool ng;
                T += entry_weight(val[k], di, si, &ng);
                const uint32_t cs = (uint32_t)col[k] | (ng ? kNegBit : 0u);
                if (inl) {
                    // unrolled store into the register array (m < 6)
#pragma unroll
                    for (int u = 0; u < kInlineCum; ++u)
                        if (u == (int)m) { w[4 + 2 * u] = T; w[5 + 2 * u] = cs; }
                } else {
                    ool_a[begin + m] = T;
                    ool_b[begin + m] = cs;
                }
                ++m;
            }
            w[0] = T;   // Q
        } else {
            const bool inl = deg <= (uint32_t)kInlineAlias;
            w[3] = deg | (inl ? 0u : kOolFlag);
            if (!inl) w[4] = begin;
            // weights q_j * deg and the two LIFO lists (scratch at [begin, begin+deg))
            uint32_t ns = 0, nl = 0, m = 0;
            for (int64_t k = a; k < b; ++k) {
                if (col[k] == i) continue;
                const unsigned long long qn = wscratch[begin + m];
                const bool ng = (qn >> 32) != 0ull;
                const unsigned long long wj = (qn & 0xFFFFFFFFull) * deg;
                wscratch[begin + m] = wj;
                ool_b[begin + m] = (uint32_t)col[k] | (ng ? kNegBit : 0u);  // own col|sign (CSR order)
                if (wj < Q) small_stk[begin + ns++] = m; else large_stk[begin + nl++] = m;
                ++m;
            }
            while (ns > 0 && nl > 0) {
                const uint32_t sm = small_stk[begin + --ns];
                const uint32_t lg = large_stk[begin + --nl];
                const unsigned long long ws = wscratch[begin + sm];
                ool_a[begin + sm] = (uint32_t)ws;
                ool_c[begin + sm] = lg;                       // alias as a row-local index for now
                const unsigned long long wl = wscratch[begin + lg] - (Q - ws);
                wscratch[begin + lg] = wl;
                if (wl < Q) small_stk[begin + ns++] = lg; else large_stk[begin + nl++] = lg;
            }
            while (nl > 0) { const uint32_t lg = large_stk[begin + --nl]; ool_a[begin + lg] = (uint32_t)Q; ool_c[begin + lg] = lg; }
            while (ns > 0) { const uint32_t sm = small_stk[begin + --ns]; ool_a[begin + sm] = (uint32_t)Q; ool_c[begin + sm] = sm; }
            // alias index -> alias col|sign; inline copy for short rows
            for (uint32_t bkt = 0; bkt < deg; ++bkt) {
                const uint32_t al = ool_b[begin + ool_c[begin + bkt]];
                if (inl) {
#pragma unroll
                    for (int u = 0; u < kInlineAlias; ++u)
                        if (u == (int)bkt) {
                            w[4 + 3 * u] = ool_a[begin + bkt];
                            w[5 + 3 * u] = ool_b[begin + bkt];
                            w[6 + 3 * u] = al;
                        }
                } else {
                    wscratch[begin + bkt] = al;   // stash: ool_c is still read as an index below
                }
            }
            if (!inl)
                for (uint32_t bkt = 0; bkt < deg; ++bkt) {
                    ool_c[begin + bkt] = (uint32_t)wscratch[begin + bkt];
                    ool_bkt[begin + bkt] = make_uint4(ool_a[begin + bkt], ool_b[begin + bkt], ool_c[begin + bkt], 0u);
                }
        }
        uint4 *o = slots + 4 * i;
        o[0] = make_uint4(w[0], w[1], w[2], w[3]);
        o[1] = make_uint4(w[4], w[5], w[6], w[7]);
        o[2] = make_uint4(w[8], w[9], w[10], w[11]);
        o[3] = make_uint4(w[12], w[13], w[14], w[15]);
    }
}

void launch_validate(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *col, const double *val,
                     DevState *st, cudaStream_t s)
{
    const int bs = 256;
    const int64_t g = (n + bs - 1) / bs;
    k_validate<<<(unsigned)(g < 148 * 32 ? g : 148 * 32), bs, 0, s>>>(n, nnz, rp, col, val, st);
}

void launch_rownorm(int64_t n, const int64_t *rp, const double *val, DevState *st, cudaStream_t s)
{
    const int bs = 256;
    const int64_t g = (n + bs - 1) / bs;
    k_rownorm<<<(unsigned)(g < 148 * 32 ? g : 148 * 32), bs, 0, s>>>(n, rp, val, st);
}

cudaError_t launch_len_order(int64_t n, const int64_t *rp, unsigned long long *counts32, int32_t *order,
                             cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counts32, 0, 2 * kLenClasses * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int bs = 256;
    const int64_t g = (n + bs - 1) / bs;
    const unsigned grid = (unsigned)(g < 148 * 8 ? (g < 1 ? 1 : g) : 148 * 8);
    k_len_count<<<grid, bs, 0, s>>>(n, rp, counts32);
    k_len_scatter<<<grid, bs, 0, s>>>(n, rp, counts32, counts32 + kLenClasses, order);
    return cudaGetLastError();
}

void launch_split(int64_t n, const int64_t *rp, const int32_t *col, const double *val, double alpha,
                  double *d, double *sv, DevState *st, cudaStream_t s, const int32_t *order)
{
    const int bs = 256;
    const int64_t g = (n + bs - 1) / bs;
    k_split<<<(unsigned)(g < 148 * 32 ? g : 148 * 32), bs, 0, s>>>(n, rp, col, val, alpha, d, sv, st, order);
}

void launch_tables(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const double *d,
                   const double *sv, int table, uint4 *slots, uint32_t *a, uint32_t *b, uint32_t *c,
                   uint4 *bkt, unsigned long long *wscr, uint32_t *sstk, uint32_t *lstk, double2 *rowd,
                   float *invd32, cudaStream_t s, const int32_t *order)
{
    const int bs = 128;
    const int64_t g = (n + bs - 1) / bs;
    k_tables<<<(unsigned)(g < 148 * 64 ? g : 148 * 64), bs, 0, s>>>(n, rp, col, val, d, sv, table, slots, a,
                                                                     b, c, bkt, wscr, sstk, lstk, rowd, invd32, order);
}

}  // namespace mcmi
