// Matrix reduction (Algorithm 1, step 2; Sec. III, "Matrix Reduction"):
// before the split, drop a set share of the off-diagonal entries of B that
// are smallest in magnitude.  Either the floor(fraction * nnz_off) smallest
// |b_ij| (ties: the earlier entry in CSR order goes first), or every |b_ij|
// below lo + fraction (hi - lo) of the off-diagonal value range.  The
// selection is exact: |b_ij| is compared by the bits of the non-negative
// FP64 value, whose integer order is the order of the values.
//
// One thread per row for the row-level passes; the k-th smallest key is
// found by an 8-bit radix select whose histograms are summed in shared
// memory per block.
#include "kernels.h"

namespace mcmi {

namespace {

__device__ __forceinline__ unsigned long long abs_bits(double v)
{
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}

// out[0] += off-diagonal entries, out[1] = min |b| bits, out[2] = max |b| bits
__global__ void k_offstats(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const double *__restrict__ val, unsigned long long *out)
{
    unsigned long long cnt = 0, mn = ~0ull, mx = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (col[k] != (int32_t)i) {
                const unsigned long long b = abs_bits(val[k]);
                ++cnt;
                mn = b < mn ? b : mn;
                mx = b > mx ? b : mx;
            }
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
        mn = min(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (cnt) atomicAdd(&out[0], cnt);
        atomicMin(&out[1], mn);
        atomicMax(&out[2], mx);
    }
}

// 256-bin histogram of the digit (bits >> shift) & 255 of the off-diagonal
// keys whose bits under `mask` equal `prefix`
__global__ void k_abs_hist(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const double *__restrict__ val, unsigned long long prefix, unsigned long long mask,
                           int shift, unsigned int *hist)
{
    __shared__ unsigned int h[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (col[k] != (int32_t)i) {
                const unsigned long long b = abs_bits(val[k]);
                if ((b & mask) == prefix) atomicAdd(&h[(b >> shift) & 255u], 1u);
            }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

// Drop rule of one stored entry of row i.  range mode: |b| < thr.  entries
// mode: key < T, or key == T among the first `need` such entries in CSR order
// (eq_rank: the entry's rank among the off-diagonal entries equal to T).
struct DropRule {
    int mode;
    double thr;
    unsigned long long T;
    long long need;
};

__device__ __forceinline__ bool dropped(const DropRule &r, double v, long long eq_rank)
{
    if (r.mode == MCMI_REDUCE_RANGE) return fabs(v) < r.thr;
    const unsigned long long b = abs_bits(v);
    return b < r.T || (b == r.T && eq_rank < r.need);
}

// per row: off-diagonal entries whose key equals T
__global__ void k_eq_count(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const double *__restrict__ val, unsigned long long T, int32_t *eqc)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = 0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) c += (col[k] != (int32_t)i && abs_bits(val[k]) == T);
        eqc[i] = c;
    }
}

// per row: entries kept (pass 1) or written to the reduced CSR (pass 2)
template <bool WRITE>
__global__ void k_keep(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                       const double *__restrict__ val, DropRule rule, const int64_t *__restrict__ eq_off,
                       int32_t *kc, const int64_t *__restrict__ out_rp, int32_t *out_col, double *out_val)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        long long eq = eq_off ? eq_off[i] : 0;
        int64_t o = WRITE ? out_rp[i] : 0;
        int32_t kept = 0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            const double v = val[k];
            bool drop = false;
            if (col[k] != (int32_t)i) {
                drop = dropped(rule, v, eq);
                if (rule.mode == MCMI_REDUCE_ENTRIES && abs_bits(v) == rule.T) ++eq;
            }
            if (drop) continue;
            if (WRITE) {
                out_col[o] = col[k];
                out_val[o] = v;
                ++o;
            }
            ++kept;
        }
        if (!WRITE) kc[i] = kept;
    }
}

int grid_for(int64_t n)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

cudaError_t launch_offstats(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                            unsigned long long *out, cudaStream_t s)
{
    if (n > 0) k_offstats<<<grid_for(n), 256, 0, s>>>(n, rp, col, val, out);
    return cudaGetLastError();
}

cudaError_t launch_abs_hist(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                            unsigned long long prefix, unsigned long long mask, int shift, unsigned int *hist,
                            cudaStream_t s)
{
    if (n > 0) k_abs_hist<<<grid_for(n), 256, 0, s>>>(n, rp, col, val, prefix, mask, shift, hist);
    return cudaGetLastError();
}

cudaError_t launch_eq_count(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                            unsigned long long T, int32_t *eqc, cudaStream_t s)
{
    if (n > 0) k_eq_count<<<grid_for(n), 256, 0, s>>>(n, rp, col, val, T, eqc);
    return cudaGetLastError();
}

cudaError_t launch_keep(int64_t n, const int64_t *rp, const int32_t *col, const double *val, int mode, double thr,
                        unsigned long long T, long long need, const int64_t *eq_off, int32_t *kc,
                        const int64_t *out_rp, int32_t *out_col, double *out_val, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const DropRule rule{mode, thr, T, need};
    if (out_rp)
        k_keep<true><<<grid_for(n), 256, 0, s>>>(n, rp, col, val, rule, eq_off, kc, out_rp, out_col, out_val);
    else
        k_keep<false><<<grid_for(n), 256, 0, s>>>(n, rp, col, val, rule, eq_off, kc, nullptr, nullptr, nullptr);
    return cudaGetLastError();
}

}  // namespace mcmi
