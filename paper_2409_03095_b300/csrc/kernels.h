// Host-side launchers of libmcmi's kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mcmi_internal.cuh"

namespace mcmi {

void launch_validate(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *col, const double *val,
                     DevState *st, cudaStream_t s);
void launch_rownorm(int64_t n, const int64_t *rp, const double *val, DevState *st, cudaStream_t s);
// rows ordered by CSR row length, longest first (counts32: 32 words of scratch)
cudaError_t launch_len_order(int64_t n, const int64_t *rp, unsigned long long *counts32, int32_t *order,
                             cudaStream_t s);
// order: rows in the order the threads take them (nullptr: 0 .. n-1)
void launch_split(int64_t n, const int64_t *rp, const int32_t *col, const double *val, double alpha,
                  double *d, double *sv, DevState *st, cudaStream_t s, const int32_t *order = nullptr);
void launch_tables(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const double *d,
                   const double *sv, int table, uint4 *slots, uint32_t *a, uint32_t *b, uint32_t *c,
                   uint4 *bkt, unsigned long long *wscr, uint32_t *sstk, uint32_t *lstk, double2 *rowd,
                   float *invd32, cudaStream_t s, const int32_t *order = nullptr);

size_t walk_smem_bytes(int precision, int log2H, bool dump);
// 32-bit cells per block of the walk-time magnitude sketch (a.cells)
size_t walk_sketch_cells();
// depth: loads per thread in flight after the walks (4 or 8)
cudaError_t walk_occupancy(int precision, int table, int acc, bool dump, int cpt, int depth, int threads, int log2H,
                           int *blocks_per_sm);
cudaError_t launch_walk(const WalkArgs &a, int precision, int table, int acc, bool dump, int cpt, int depth,
                        int grid, int threads, cudaStream_t s);

// exclusive scan of int32 counts into int64 offsets (out has n+1 entries)
cudaError_t scan_counts(const int32_t *counts, int64_t n, int64_t *out, int64_t *block_tmp, cudaStream_t s);
size_t scan_tmp_elems(int64_t n);

// max_cnt: an upper bound of the entries of any row, or 0 if unknown
cudaError_t launch_assemble(int64_t rows, const int64_t *row_ptr, const int64_t *st_off, const int32_t *st_cnt,
                            const uint32_t *st_col, const float *st_val, int32_t *out_col, float *out_val,
                            int64_t max_cnt, cudaStream_t s);
// message returned by mcmi_last_error() on this host thread
void set_error_message(const char *msg);

// learned proposal
cudaError_t launch_degree(int64_t n, const int64_t *rp, const int32_t *col, int *deg, cudaStream_t s);
cudaError_t launch_tables_learned(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                                  const double *d, const double *sv, const int *deg, const float *th, uint4 *slots,
                                  uint32_t *a, uint32_t *b, uint32_t *c, uint4 *lbkt, unsigned long long *wscr,
                                  uint32_t *sstk, uint32_t *lstk, cudaStream_t s);
cudaError_t launch_row_moments(const WalkArgs &a, int table, int64_t n, float *m, cudaStream_t s);
cudaError_t launch_train_edges(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const double *d,
                               const double *sv, const int *deg, const float *mrow, int64_t row_base,
                               int64_t edge_base, float *feat, float *p, float *mt, int32_t *rid, cudaStream_t s);
cudaError_t train_pass(int64_t E, int64_t R, const float *feat, const float *p, const float *mt, const int32_t *rid,
                       const float *th, float *A, float *Bs, float *Cs, float *lossbuf, float *grad, bool need_c,
                       int round_bf16, cudaStream_t s);
cudaError_t launch_adam(float *th, const float *grad, float *m1, float *m2, float lr, int step, cudaStream_t s);

// batched builds: one matrix of the batch, in and out
struct BatchIn {
    const int64_t *rp;
    const int32_t *col;
    const double *val;
    int64_t n, nnz, row_base, nnz_base;
};
struct BatchOut {
    int64_t *rp;
    int32_t *col;
    float *val;
    int64_t n, row_base, nnz_base;   // nnz_base: first entry of this matrix in the batched M
};
// per matrix b: out[2b] = largest off-diagonal count of a row, out[2b + 1] =
// largest |j - i| (device, 2 count words)
cudaError_t launch_fit_stats(const BatchIn *in, int count, unsigned long long *out, cudaStream_t s);
cudaError_t launch_concat(const BatchIn *in, int count, const int64_t *row_base, const int64_t *nnz_base,
                          int64_t total_rows, int64_t total_nnz, int64_t *rp, int32_t *col, double *val,
                          cudaStream_t s);
cudaError_t launch_split(const BatchOut *out, int count, const int64_t *row_base, const int64_t *nnzM_base,
                         int64_t total_rows, int64_t total_nnz, const int64_t *rpM, const int32_t *colM,
                         const float *valM, cudaStream_t s);

cudaError_t launch_spmv(int64_t rows, int64_t nnz, const int64_t *rp, const int32_t *col, const float *val,
                        const float *x, float *y, cudaStream_t s);

// recovery of B^-1 (Eq. 3) and dense copies
cudaError_t launch_aug_diag(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const double *d,
                            double *s, cudaStream_t st);
cudaError_t launch_sm_step(int64_t n, double *X, int64_t i, const double *s, double *c, double *r, double *gs,
                           int *flag, cudaStream_t st);
cudaError_t launch_csr_dense(int64_t rows, int64_t ncols, const int64_t *rp, const int32_t *col, const float *val,
                             double *X, cudaStream_t st);

// matrix reduction
cudaError_t launch_offstats(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                            unsigned long long *out, cudaStream_t s);
cudaError_t launch_abs_hist(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                            unsigned long long prefix, unsigned long long mask, int shift, unsigned int *hist,
                            cudaStream_t s);
cudaError_t launch_eq_count(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                            unsigned long long T, int32_t *eqc, cudaStream_t s);
cudaError_t launch_keep(int64_t n, const int64_t *rp, const int32_t *col, const double *val, int mode, double thr,
                        unsigned long long T, long long need, const int64_t *eq_off, int32_t *kc,
                        const int64_t *out_rp, int32_t *out_col, double *out_val, cudaStream_t s);

}  // namespace mcmi
