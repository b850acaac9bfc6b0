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
