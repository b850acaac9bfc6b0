// Batched builds: gather many CSR matrices into one block-diagonal CSR (so
// that one persistent walk launch drains the rows of all of them from one
// device queue) and split the resulting M back into one CSR per matrix.
#include "kernels.h"

namespace mcmi {

namespace {

__device__ __forceinline__ int find_block(const int64_t *base, int count, int64_t g)
{
    int lo = 0, hi = count - 1;   // last b with base[b] <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// per matrix of a batch: the largest off-diagonal count of a row (out[2b])
// and the largest |j - i| of an off-diagonal entry (out[2b + 1]); blockIdx.y
// + y0 is the matrix
__global__ void k_fit_stats(const BatchIn *in, int y0, unsigned long long *out)
{
    const int b = y0 + (int)blockIdx.y;
    const BatchIn m = in[b];
    unsigned long long dmax = 0, omax = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m.n; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long deg = 0;
        for (int64_t k = m.rp[i]; k < m.rp[i + 1]; ++k) {
            const long long o = (long long)m.col[k] - (long long)i;
            if (o == 0) continue;
            ++deg;
            const unsigned long long ao = (unsigned long long)(o < 0 ? -o : o);
            omax = ao > omax ? ao : omax;
        }
        dmax = deg > dmax ? deg : dmax;
    }
    for (int o = 16; o > 0; o >>= 1) {
        dmax = max(dmax, __shfl_xor_sync(0xFFFFFFFFu, dmax, o));
        omax = max(omax, __shfl_xor_sync(0xFFFFFFFFu, omax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[2 * b], dmax);
        atomicMax(&out[2 * b + 1], omax);
    }
}

__global__ void k_concat_rows(const BatchIn *in, int count, const int64_t *row_base, int64_t total_rows,
                              int64_t total_nnz, int64_t *rp)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total_rows;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int b = find_block(row_base, count, g);
        rp[g] = in[b].nnz_base + in[b].rp[g - row_base[b]];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rp[total_rows] = total_nnz;
}

__global__ void k_concat_entries(const BatchIn *in, int count, const int64_t *nnz_base, int64_t total_nnz,
                                 int32_t *col, double *val)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total_nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int b = find_block(nnz_base, count, e);
        const int64_t k = e - nnz_base[b];
        col[e] = in[b].col[k] + (int32_t)in[b].row_base;
        val[e] = in[b].val[k];
    }
}

__global__ void k_split_rows(const BatchOut *out, int count, const int64_t *row_base, int64_t total_rows,
                             const int64_t *rpM)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g <= total_rows;
         g += (int64_t)gridDim.x * blockDim.x) {
        if (g == total_rows) {
            // closing entry of the last matrix
            const BatchOut &o = out[count - 1];
            o.rp[o.n] = rpM[g] - o.nnz_base;
            continue;
        }
        const int b = find_block(row_base, count, g);
        const BatchOut &o = out[b];
        const int64_t i = g - row_base[b];
        o.rp[i] = rpM[g] - o.nnz_base;
        if (i == 0 && b > 0) {
            // closing entry of the previous matrix
            const BatchOut &p = out[b - 1];
            p.rp[p.n] = rpM[g] - p.nnz_base;
        }
    }
}

__global__ void k_split_entries(const BatchOut *out, int count, const int64_t *nnzM_base, int64_t total_nnz,
                                const int32_t *colM, const float *valM)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total_nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int b = find_block(nnzM_base, count, e);
        const BatchOut &o = out[b];
        const int64_t k = e - o.nnz_base;
        o.col[k] = colM[e] - (int32_t)o.row_base;
        o.val[k] = valM[e];
    }
}

int grid_for(int64_t work)
{
    int64_t g = (work + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 148 * 16 ? 148 * 16 : g));
}

}  // namespace

cudaError_t launch_fit_stats(const BatchIn *in, int count, unsigned long long *out, cudaStream_t s)
{
    cudaMemsetAsync(out, 0, sizeof(unsigned long long) * 2 * (size_t)count, s);
    for (int y0 = 0; y0 < count; y0 += 65535) {
        const int ny = count - y0 < 65535 ? count - y0 : 65535;
        k_fit_stats<<<dim3(4, (unsigned)ny), 256, 0, s>>>(in, y0, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_concat(const BatchIn *in, int count, const int64_t *row_base, const int64_t *nnz_base,
                          int64_t total_rows, int64_t total_nnz, int64_t *rp, int32_t *col, double *val,
                          cudaStream_t s)
{
    k_concat_rows<<<grid_for(total_rows), 256, 0, s>>>(in, count, row_base, total_rows, total_nnz, rp);
    if (total_nnz > 0)
        k_concat_entries<<<grid_for(total_nnz), 256, 0, s>>>(in, count, nnz_base, total_nnz, col, val);
    return cudaGetLastError();
}

cudaError_t launch_split(const BatchOut *out, int count, const int64_t *row_base, const int64_t *nnzM_base,
                         int64_t total_rows, int64_t total_nnz, const int64_t *rpM, const int32_t *colM,
                         const float *valM, cudaStream_t s)
{
    k_split_rows<<<grid_for(total_rows + 1), 256, 0, s>>>(out, count, row_base, total_rows, rpM);
    if (total_nnz > 0)
        k_split_entries<<<grid_for(total_nnz), 256, 0, s>>>(out, count, nnzM_base, total_nnz, colM, valM);
    return cudaGetLastError();
}

}  // namespace mcmi
