// Recovery of B^-1 from Bhat^-1 (Eq. 3; Algorithm 1, step 5), a dense
// diagnostic for small n: S = Bhat - B is diagonal, and for i = n-1, ..., 0
// with s_i != 0,
//     X <- X + g x_col(i) x_row(i),   g = s_i / (1 - s_i X_ii),
// a rank-one update of the dense n x n row-major X by its own column i and
// row i.  Each step copies column i and row i (and g) out of X first, then
// updates X; products and sums are single IEEE FP64 operations, in the order
// (g x_col) x_row.  Also: the dense copy of a preconditioner M.
#include "kernels.h"

namespace mcmi {

namespace {

// s_i = d_i - b_ii: the diagonal of S = Bhat - B, from the split's d
__global__ void k_aug_diag(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const double *__restrict__ val, const double *__restrict__ d, double *s)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double bii = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (col[k] == (int32_t)i) bii = val[k];
        s[i] = __dsub_rn(d[i], bii);
    }
}

// column i and row i of X, and g (gs[0]); flag[0] = 1 if the denominator is 0
__global__ void k_sm_gather(int64_t n, const double *__restrict__ X, int64_t i, const double *__restrict__ s,
                            double *c, double *r, double *gs, int *flag)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n; a += (int64_t)gridDim.x * blockDim.x) {
        c[a] = X[a * n + i];
        r[a] = X[i * n + a];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double den = __dsub_rn(1.0, __dmul_rn(s[i], X[i * n + i]));
        if (den == 0.0) {
            flag[0] = 1;
            gs[0] = 0.0;
        } else {
            gs[0] = __ddiv_rn(s[i], den);
        }
    }
}

__global__ void k_sm_update(int64_t n, double *X, const double *__restrict__ c, const double *__restrict__ r,
                            const double *__restrict__ gs, const int *__restrict__ flag)
{
    if (flag[0]) return;
    const double g = gs[0];
    const int64_t total = n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = e / n, b = e - a * n;
        X[e] = __dadd_rn(X[e], __dmul_rn(__dmul_rn(g, c[a]), r[b]));
    }
}

// dense copy of a CSR with FP32 values (rows x ncols, row-major, zero-filled by the caller)
__global__ void k_csr_dense(int64_t rows, int64_t ncols, const int64_t *__restrict__ rp,
                            const int32_t *__restrict__ col, const float *__restrict__ val, double *X)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) X[i * ncols + col[k]] = (double)val[k];
}

int grid_of(int64_t work, int cap_per_sm)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (work + 255) / 256;
    const int64_t cap = (int64_t)sms * cap_per_sm;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

}  // namespace

cudaError_t launch_aug_diag(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const double *d,
                            double *s, cudaStream_t st)
{
    if (n > 0) k_aug_diag<<<grid_of(n, 8), 256, 0, st>>>(n, rp, col, val, d, s);
    return cudaGetLastError();
}

cudaError_t launch_sm_step(int64_t n, double *X, int64_t i, const double *s, double *c, double *r, double *gs,
                           int *flag, cudaStream_t st)
{
    k_sm_gather<<<grid_of(n, 4), 256, 0, st>>>(n, X, i, s, c, r, gs, flag);
    k_sm_update<<<grid_of(n * n, 8), 256, 0, st>>>(n, X, c, r, gs, flag);
    return cudaGetLastError();
}

cudaError_t launch_csr_dense(int64_t rows, int64_t ncols, const int64_t *rp, const int32_t *col, const float *val,
                             double *X, cudaStream_t st)
{
    if (rows > 0) k_csr_dense<<<grid_of(rows, 8), 256, 0, st>>>(rows, ncols, rp, col, val, X);
    return cudaGetLastError();
}

}  // namespace mcmi
