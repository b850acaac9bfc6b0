// Learned proposal (an extension of the method; not in the paper): an
// 8-32-32-1 BF16 MLP g_ij > 0 of per-edge features reweights the transition
// weights |c_ij|; the walk multiplies by c_ij / p_ij with the table's own
// probability p_ij = q_ij / Q_i, so the Eq. 2 estimator stays unbiased.
//
// Kernels: the network's inference fused into the table build, per-row
// second moments of the walks (the training signal), forward/backward
// passes of the training loss and an Adam update.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "mcmi.h"

namespace mcmi {

namespace {

constexpr int kIn = 8, kHid = 32;
constexpr int kW1 = 0, kB1 = 256, kW2 = 288, kB2 = 1312, kW3 = 1344, kB3 = 1376;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Parameters of one block in shared memory: weights rounded to BF16 once,
// biases FP32.
__device__ __forceinline__ void load_params(const float *__restrict__ th, float *sp)
{
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
        const bool bias = (i >= kB1 && i < kW2) || (i >= kB2 && i < kW3) || i == kB3;
        sp[i] = bias ? th[i] : bf16r(th[i]);
    }
    __syncthreads();
}

// Forward pass of the BF16 network (inputs, weights and hidden activations
// BF16; exact products, FP32 sums in index order); g = squareplus(z) clamped
// to [1/16, 16].  Optionally keeps the activations for the backward pass.
__device__ __forceinline__ float mlp_forward(const float *sp, const float *feat, float *x, float *h1, float *h2,
                                             float *zout, bool round_hidden)
{
    for (int k = 0; k < kIn; ++k) x[k] = round_hidden ? bf16r(feat[k]) : feat[k];
    for (int o = 0; o < kHid; ++o) {
        float acc = sp[kB1 + o];
        for (int k = 0; k < kIn; ++k) acc = __fadd_rn(acc, __fmul_rn(sp[kW1 + o * kIn + k], x[k]));
        acc = acc > 0.0f ? acc : 0.0f;
        h1[o] = round_hidden ? bf16r(acc) : acc;
    }
    for (int o = 0; o < kHid; ++o) {
        float acc = sp[kB2 + o];
        for (int k = 0; k < kHid; ++k) acc = __fadd_rn(acc, __fmul_rn(sp[kW2 + o * kHid + k], h1[k]));
        acc = acc > 0.0f ? acc : 0.0f;
        h2[o] = round_hidden ? bf16r(acc) : acc;
    }
    float z = sp[kB3];
    for (int k = 0; k < kHid; ++k) z = __fadd_rn(z, __fmul_rn(sp[kW3 + k], h2[k]));
    if (zout) *zout = z;
    float g = __fmul_rn(0.5f, __fadd_rn(z, __fsqrt_rn(__fadd_rn(__fmul_rn(z, z), 4.0f))));
    return fminf(fmaxf(g, 0.0625f), 16.0f);
}

// Edge features: p_ij = |c|/s_i, s_i, s_j, 1/deg_i, 1/deg_j,
// |d_i|/(|d_i|+|d_j|), |c|/max_k|c_ik|, sign(c); FP64 then FP32.
__device__ __forceinline__ void edge_features(double c, double si, double sj, int degi, int degj, double di,
                                              double dj, double maxabs, float *f)
{
    f[0] = __double2float_rn(__ddiv_rn(fabs(c), si));
    f[1] = __double2float_rn(si);
    f[2] = __double2float_rn(sj);
    f[3] = __double2float_rn(__ddiv_rn(1.0, (double)degi));
    f[4] = degj > 0 ? __double2float_rn(__ddiv_rn(1.0, (double)degj)) : 0.0f;
    f[5] = __double2float_rn(__ddiv_rn(fabs(di), __dadd_rn(fabs(di), fabs(dj))));
    f[6] = __double2float_rn(__ddiv_rn(fabs(c), maxabs));
    f[7] = c < 0.0 ? -1.0f : 1.0f;
}

__global__ void k_degree(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col, int *deg)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int m = 0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) m += col[k] != i;
        deg[i] = m;
    }
}

// Learned tables, one thread per row: g from the network, weights
// w_ij = |c_ij| g_ij, q_ij = max(1, floor(w_ij / sum_k w_ik 2^31)) (0 for
// c == 0), Walker/Vose alias buckets over q (as for the |c| proposal) with
// the factor f = fl32(c Q / q) of both entries of each bucket.
__global__ void __launch_bounds__(128) k_tables_learned(
    int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col, const double *__restrict__ val,
    const double *__restrict__ d, const double *__restrict__ s, const int *__restrict__ deg,
    const float *__restrict__ th, uint4 *__restrict__ slots, uint32_t *__restrict__ ool_a,
    uint32_t *__restrict__ ool_b, uint32_t *__restrict__ ool_c, uint4 *__restrict__ lbkt,
    unsigned long long *__restrict__ wscratch, uint32_t *__restrict__ small_stk, uint32_t *__restrict__ large_stk)
{
    __shared__ float sp[kMlpParams];
    load_params(th, sp);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = rp[i], b = rp[i + 1];
        const double di = d[i], si = s[i];
        const uint32_t begin = (uint32_t)a;
        double maxabs = 0.0;
        for (int64_t k = a; k < b; ++k)
            if (col[k] != i) maxabs = fmax(maxabs, fabs(__ddiv_rn(-val[k], di)));
        // pass 1: w_ij (stored as FP64 bits in the scratch) and their sum
        double wsum = 0.0;
        uint32_t m = 0;
        float x[kIn], h1[kHid], h2[kHid], feat[kIn];
        for (int64_t k = a; k < b; ++k) {
            if (col[k] == i) continue;
            const int64_t j = col[k];
            const double c = __ddiv_rn(-val[k], di);
            double w = 0.0;
            if (c != 0.0) {
                edge_features(c, si, s[j], deg[i], deg[j], di, d[j], maxabs, feat);
                const float g = mlp_forward(sp, feat, x, h1, h2, nullptr, true);
                w = __dmul_rn(fabs(c), (double)g);
            }
            wscratch[begin + m] = (unsigned long long)__double_as_longlong(w);
            wsum = __dadd_rn(wsum, w);
            ++m;
        }
        const uint32_t dg = m;
        // pass 2: integer weights and their total
        unsigned long long Q = 0;
        for (uint32_t t = 0; t < dg; ++t) {
            const double w = __longlong_as_double((long long)wscratch[begin + t]);
            uint32_t q = 0;
            if (w > 0.0) {
                q = (uint32_t)floor(__dmul_rn(__ddiv_rn(w, wsum), 2147483648.0));
                if (q < 1u) q = 1u;
            }
            ool_a[begin + t] = q;
            Q += q;
        }
        // pass 3: own col|sign, factor f = c Q / q, Vose over q * deg
        uint32_t ns = 0, nl = 0;
        m = 0;
        for (int64_t k = a; k < b; ++k) {
            if (col[k] == i) continue;
            const double c = __ddiv_rn(-val[k], di);
            const uint32_t q = ool_a[begin + m];
            const float f = q > 0 ? __double2float_rn(__ddiv_rn(__dmul_rn(c, (double)Q), (double)q)) : 0.0f;
            ool_b[begin + m] = (uint32_t)col[k] | (c < 0.0 ? kNegBit : 0u);
            ool_c[begin + m] = __float_as_uint(f);   // factor of entry m (CSR order), read below
            const unsigned long long wj = (unsigned long long)q * dg;
            wscratch[begin + m] = wj;
            if (wj < Q) small_stk[begin + ns++] = m; else large_stk[begin + nl++] = m;
            ++m;
        }
        // Vose (LIFO lists filled in CSR order); each entry's probability and
        // alias index are parked in words 0 and 1 of its own 32-byte bucket
        uint32_t *tmp = reinterpret_cast<uint32_t *>(lbkt + 2 * (size_t)begin);
        while (ns > 0 && nl > 0) {
            const uint32_t sm = small_stk[begin + --ns];
            const uint32_t lg = large_stk[begin + --nl];
            const unsigned long long ws = wscratch[begin + sm];
            tmp[8 * sm] = (uint32_t)ws;
            tmp[8 * sm + 1] = lg;
            const unsigned long long wl = wscratch[begin + lg] - (Q - ws);
            wscratch[begin + lg] = wl;
            if (wl < Q) small_stk[begin + ns++] = lg; else large_stk[begin + nl++] = lg;
        }
        while (nl > 0) { const uint32_t lg = large_stk[begin + --nl]; tmp[8 * lg] = (uint32_t)Q; tmp[8 * lg + 1] = lg; }
        while (ns > 0) { const uint32_t sm = small_stk[begin + --ns]; tmp[8 * sm] = (uint32_t)Q; tmp[8 * sm + 1] = sm; }
        // buckets {prob, own col|sign, alias col|sign, f_own, f_alias, 0, 0, 0}
        for (uint32_t t = 0; t < dg; ++t) {
            const uint32_t prob = tmp[8 * t], al = tmp[8 * t + 1];
            lbkt[2 * ((size_t)begin + t)] = make_uint4(prob, ool_b[begin + t], ool_b[begin + al], ool_c[begin + t]);
            lbkt[2 * ((size_t)begin + t) + 1] = make_uint4(ool_c[begin + al], 0u, 0u, 0u);
        }
        // layout-neutral copies for the table export: prob, own, alias col|sign
        for (uint32_t t = 0; t < dg; ++t) {
            const uint4 bk = lbkt[2 * ((size_t)begin + t)];
            ool_a[begin + t] = bk.x;
            ool_c[begin + t] = bk.z;
        }
        uint4 *o = slots + 4 * i;
        o[0] = make_uint4((uint32_t)Q, __float_as_uint(__double2float_rn(si)),
                          __float_as_uint(__double2float_rn(__ddiv_rn(1.0, di))), dg | kOolFlag);
        o[1] = make_uint4(begin, 0u, 0u, 0u);
        o[2] = make_uint4(0u, 0u, 0u, 0u);
        o[3] = make_uint4(0u, 0u, 0u, 0u);
    }
}

}  // namespace

namespace {

// Second moment of the chains of every row: m_i = (1/N) sum_chains sum_t W_t^2
// (t = 0 included), one thread per (row, chain); the same paths as the build.
template <int TABLE>
__global__ void k_row_moments(WalkArgs a, int64_t n, float *__restrict__ m)
{
    const int64_t items = n * (int64_t)a.N;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < items;
         it += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = it / a.N;
        const uint32_t k = (uint32_t)(it - row * a.N);
        uint32_t st = (uint32_t)row;
        float w = 1.0f, sum = 1.0f;
        uint4 r4 = make_uint4(0, 0, 0, 0);
        for (int t = 0;; ++t) {
            uint32_t s[16];
            constexpr int kWords = TABLE == MCMI_TABLE_COMPACT ? 2 : 4;   // uint4 per record
            const uint4 *sp = a.slots + kWords * (size_t)st;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint4 v = u < kWords ? __ldg(sp + u) : make_uint4(0u, 0u, 0u, 0u);
                s[4 * u] = v.x; s[4 * u + 1] = v.y; s[4 * u + 2] = v.z; s[4 * u + 3] = v.w;
            }
            if (t == a.L || !(fabsf(w) >= a.delta_f) || record_q<TABLE>(s) == 0u) break;
            if ((t & 3) == 0)
                r4 = philox4x32_10(make_uint4((uint32_t)(t >> 2), k, (uint32_t)row, (uint32_t)((uint64_t)row >> 32)),
                                   a.key0, a.key1);
            const int ph = t & 3;
            const uint32_t r = ph == 0 ? r4.x : ph == 1 ? r4.y : ph == 2 ? r4.z : r4.w;
            float f;
            const uint32_t cs = pick_transition<TABLE>(s, r, a, &f, st);
            w = __fmul_rn(w, f);
            sum = __fadd_rn(sum, __fmul_rn(w, w));
            st = cs & ~kNegBit;
        }
        atomicAdd(&m[row], __fdiv_rn(sum, (float)a.N));
    }
}

// Training edges of one matrix (CSR order; diagonal slots are dummies with
// p = 0): features, p = |c_ij| / s_i, the target row's moment and the row.
__global__ void k_train_edges(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                              const double *__restrict__ val, const double *__restrict__ d,
                              const double *__restrict__ s, const int *__restrict__ deg,
                              const float *__restrict__ mrow, int64_t row_base, int64_t edge_base,
                              float *__restrict__ feat, float *__restrict__ p, float *__restrict__ mt,
                              int32_t *__restrict__ rid)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double di = d[i], si = s[i];
        double maxabs = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (col[k] != i) maxabs = fmax(maxabs, fabs(__ddiv_rn(-val[k], di)));
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            const int64_t e = edge_base + k;
            float *f = feat + 8 * e;
            rid[e] = (int32_t)(row_base + i);
            const double c = col[k] == i ? 0.0 : __ddiv_rn(-val[k], di);
            if (c == 0.0 || !(si > 0.0)) {
                for (int u = 0; u < 8; ++u) f[u] = 0.0f;
                p[e] = 0.0f;
                mt[e] = 1.0f;
                continue;
            }
            const int64_t j = col[k];
            edge_features(c, si, s[j], deg[i], deg[j], di, d[j], maxabs, f);
            p[e] = f[0];
            mt[e] = mrow[j];
        }
    }
}

// C_i = sum_j p_ij sqrt(m_j) (squared in the loss)
__global__ void k_train_c(int64_t E, const float *__restrict__ p, const float *__restrict__ mt,
                          const int32_t *__restrict__ rid, float *__restrict__ Cs)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
        if (p[e] > 0.0f) atomicAdd(&Cs[rid[e]], p[e] * sqrtf(mt[e]));
}

// Forward: A_i = sum_j p g, B_i = sum_j p m / g.
__global__ void __launch_bounds__(128) k_train_fwd(int64_t E, const float *__restrict__ feat, const float *__restrict__ p,
                                                   const float *__restrict__ mt, const int32_t *__restrict__ rid,
                                                   const float *__restrict__ th, float *__restrict__ A,
                                                   float *__restrict__ Bs, int round_bf16)
{
    __shared__ float sp[kMlpParams];
    if (round_bf16) {
        load_params(th, sp);
    } else {
        for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sp[i] = th[i];
        __syncthreads();
    }
    float x[kIn], h1[kHid], h2[kHid];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        if (!(p[e] > 0.0f)) continue;
        float fe[kIn];
        for (int u = 0; u < kIn; ++u) fe[u] = round_bf16 ? feat[8 * e + u] : feat[8 * e + u];
        const float g = mlp_forward(sp, fe, x, h1, h2, nullptr, round_bf16 != 0);
        atomicAdd(&A[rid[e]], p[e] * g);
        atomicAdd(&Bs[rid[e]], p[e] * mt[e] / g);
    }
}

__global__ void k_train_loss(int64_t R, const float *__restrict__ A, const float *__restrict__ Bs,
                             const float *__restrict__ Cs, float *__restrict__ out /* [0] sum, [1] rows */)
{
    float acc = 0.0f, cnt = 0.0f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < R; i += (int64_t)gridDim.x * blockDim.x)
        if (Cs[i] > 0.0f) {
            acc += A[i] * Bs[i] / (Cs[i] * Cs[i]);
            cnt += 1.0f;
        }
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], acc);
        atomicAdd(&out[1], cnt);
    }
}

__device__ __forceinline__ float warp_sum(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Backward: dL/dg_ij = (p B_i - A_i p m / g^2) / (C_i^2 R), through the
// clamped squareplus and the network (BF16 roundings taken as identity).
// One edge per lane; parameter gradients summed across the warp with
// shuffles into a per-warp shared copy, then into the global gradient.
__global__ void __launch_bounds__(128) k_train_bwd(int64_t E, const float *__restrict__ feat, const float *__restrict__ p,
                                                   const float *__restrict__ mt, const int32_t *__restrict__ rid,
                                                   const float *__restrict__ th, const float *__restrict__ A,
                                                   const float *__restrict__ Bs, const float *__restrict__ Cs,
                                                   const float *__restrict__ rows_valid, float *__restrict__ grad,
                                                   int round_bf16)
{
    __shared__ float sp[kMlpParams];
    __shared__ float gw[4][kMlpParams];
    if (round_bf16) {
        load_params(th, sp);
    } else {
        for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sp[i] = th[i];
        __syncthreads();
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = lane; i < kMlpParams; i += 32) gw[warp][i] = 0.0f;
    __syncwarp();
    const float invR = 1.0f / fmaxf(rows_valid[0], 1.0f);
    float x[kIn], h1[kHid], h2[kHid];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform loop bound so that every lane reaches the shuffles
    for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x + warp * 32; e0 < E; e0 += stride) {
        const int64_t e = e0 + lane;
        float dz = 0.0f;
        bool live = e < E && p[e] > 0.0f;
        if (live) {
            float z;
            const float g = mlp_forward(sp, feat + 8 * e, x, h1, h2, &z, round_bf16 != 0);
            const int64_t i = rid[e];
            const float Ci2 = Cs[i] * Cs[i];
            const float dg = (p[e] * Bs[i] - A[i] * p[e] * mt[e] / (g * g)) / Ci2 * invR;
            const float r = sqrtf(z * z + 4.0f);
            const float graw = 0.5f * (z + r);
            const bool clamped = graw < 0.0625f || graw > 16.0f;
            dz = clamped ? 0.0f : dg * 0.5f * (1.0f + z / r);
        } else {
            for (int u = 0; u < kIn; ++u) x[u] = 0.0f;
            for (int u = 0; u < kHid; ++u) { h1[u] = 0.0f; h2[u] = 0.0f; }
        }
        // layer 3
        for (int k = 0; k < kHid; ++k) {
            const float v = warp_sum(dz * h2[k]);
            if (lane == 0) gw[warp][kW3 + k] += v;
        }
        {
            const float v = warp_sum(dz);
            if (lane == 0) gw[warp][kB3] += v;
        }
        // layer 2
        float d2[kHid];
        for (int o = 0; o < kHid; ++o) d2[o] = h2[o] > 0.0f ? dz * sp[kW3 + o] : 0.0f;
        for (int o = 0; o < kHid; ++o) {
            const float vb = warp_sum(d2[o]);
            if (lane == 0) gw[warp][kB2 + o] += vb;
            for (int k = 0; k < kHid; ++k) {
                const float v = warp_sum(d2[o] * h1[k]);
                if (lane == 0) gw[warp][kW2 + o * kHid + k] += v;
            }
        }
        // layer 1
        for (int k = 0; k < kHid; ++k) {
            float dh = 0.0f;
            for (int o = 0; o < kHid; ++o) dh += sp[kW2 + o * kHid + k] * d2[o];
            const float d1 = h1[k] > 0.0f ? dh : 0.0f;
            const float vb = warp_sum(d1);
            if (lane == 0) gw[warp][kB1 + k] += vb;
            for (int u = 0; u < kIn; ++u) {
                const float v = warp_sum(d1 * x[u]);
                if (lane == 0) gw[warp][kW1 + k * kIn + u] += v;
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
        const float v = gw[0][i] + gw[1][i] + gw[2][i] + gw[3][i];
        if (v != 0.0f) atomicAdd(&grad[i], v);
    }
}

__global__ void k_adam(float *__restrict__ th, const float *__restrict__ grad, float *__restrict__ m1,
                       float *__restrict__ m2, float lr, float b1, float b2, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float g = grad[i];
    m1[i] = b1 * m1[i] + (1.0f - b1) * g;
    m2[i] = b2 * m2[i] + (1.0f - b2) * g * g;
    th[i] -= lr * (m1[i] / c1) / (sqrtf(m2[i] / c2) + 1e-8f);
}

int grid_of(int64_t work, int bs, int cap)
{
    const int64_t g = (work + bs - 1) / bs;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t launch_row_moments(const WalkArgs &a, int table, int64_t n, float *m, cudaStream_t s)
{
    const int g = grid_of(n * (int64_t)a.N, 256, 148 * 16);
    if (table == MCMI_TABLE_COMPACT)
        k_row_moments<MCMI_TABLE_COMPACT><<<g, 256, 0, s>>>(a, n, m);
    else if (table != MCMI_TABLE_CUMULATIVE)   // alias and hybrid tables
        k_row_moments<MCMI_TABLE_ALIAS><<<g, 256, 0, s>>>(a, n, m);
    else
        k_row_moments<MCMI_TABLE_CUMULATIVE><<<g, 256, 0, s>>>(a, n, m);
    return cudaGetLastError();
}

cudaError_t launch_train_edges(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const double *d,
                               const double *sv, const int *deg, const float *mrow, int64_t row_base,
                               int64_t edge_base, float *feat, float *p, float *mt, int32_t *rid, cudaStream_t s)
{
    k_train_edges<<<grid_of(n, 128, 148 * 16), 128, 0, s>>>(n, rp, col, val, d, sv, deg, mrow, row_base, edge_base,
                                                           feat, p, mt, rid);
    return cudaGetLastError();
}

// loss and (optionally) gradient of the training objective on E edges / R rows
cudaError_t train_pass(int64_t E, int64_t R, const float *feat, const float *p, const float *mt, const int32_t *rid,
                       const float *th, float *A, float *Bs, float *Cs, float *lossbuf, float *grad, bool need_c,
                       int round_bf16, cudaStream_t s)
{
    cudaMemsetAsync(A, 0, R * 4, s);
    cudaMemsetAsync(Bs, 0, R * 4, s);
    cudaMemsetAsync(lossbuf, 0, 8, s);
    if (need_c) {
        cudaMemsetAsync(Cs, 0, R * 4, s);
        k_train_c<<<grid_of(E, 256, 148 * 16), 256, 0, s>>>(E, p, mt, rid, Cs);
    }
    k_train_fwd<<<grid_of(E, 128, 148 * 8), 128, 0, s>>>(E, feat, p, mt, rid, th, A, Bs, round_bf16);
    k_train_loss<<<grid_of(R, 256, 148 * 4), 256, 0, s>>>(R, A, Bs, Cs, lossbuf);
    if (grad) {
        cudaMemsetAsync(grad, 0, kMlpParams * 4, s);
        k_train_bwd<<<grid_of(E, 128, 148 * 4), 128, 0, s>>>(E, feat, p, mt, rid, th, A, Bs, Cs, lossbuf + 1, grad,
                                                           round_bf16);
    }
    return cudaGetLastError();
}

cudaError_t launch_adam(float *th, const float *grad, float *m1, float *m2, float lr, int step, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f;
    k_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(th, grad, m1, m2, lr, b1, b2, 1.0f - powf(b1, (float)step),
                                                    1.0f - powf(b2, (float)step));
    return cudaGetLastError();
}

cudaError_t launch_degree(int64_t n, const int64_t *rp, const int32_t *col, int *deg, cudaStream_t s)
{
    int64_t g = (n + 255) / 256;
    k_degree<<<(unsigned)(g > 148 * 16 ? 148 * 16 : (g < 1 ? 1 : g)), 256, 0, s>>>(n, rp, col, deg);
    return cudaGetLastError();
}

cudaError_t launch_tables_learned(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                                  const double *d, const double *sv, const int *deg, const float *th, uint4 *slots,
                                  uint32_t *a, uint32_t *b, uint32_t *c, uint4 *lbkt, unsigned long long *wscr,
                                  uint32_t *sstk, uint32_t *lstk, cudaStream_t s)
{
    int64_t g = (n + 127) / 128;
    k_tables_learned<<<(unsigned)(g > 148 * 8 ? 148 * 8 : (g < 1 ? 1 : g)), 128, 0, s>>>(
        n, rp, col, val, d, sv, deg, th, slots, a, b, c, lbkt, wscr, sstk, lstk);
    return cudaGetLastError();
}

}  // namespace mcmi
