/*
 * mcmi.h -- C ABI of the B300 (sm_103a) Markov Chain Monte Carlo Matrix
 * Inversion ((MC)^2MI) sparse-approximate-inverse preconditioner.
 *
 * Method (Lebedev & Alexandrov, "On Advanced Monte Carlo Methods for Linear
 * Algebra on Advanced Accelerator Architectures"): split B = Bhat - C
 * (Eq. 1), scale by D = diag(Bhat) so that C = I - D^-1 Bhat has
 * ||C||_inf < 1 (Sec. III-A, Sec. IV-A phases 1-2), estimate the rows of
 * (I - C)^-1 by random walks over the Neumann series (Eq. 2, phase 3),
 * scale column j by 1/d_j (phase 4), and keep per row the entries largest in
 * magnitude (Sec. IV-B).  The recovery of B^-1 from Bhat^-1 (Eq. 3,
 * phase 5) is not part of the build: the paper notes it costs O(n^3) and is
 * usually skipped (Sec. IV); mcmi_recover_dense provides it for small dense
 * matrices, as a diagnostic.
 *
 * Conventions for every entry point:
 *  - Pointers named "device" must point to device memory of the current CUDA
 *    device; "host" pointers to host memory.  Input arrays are owned by the
 *    caller and only read during the call.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *    ordered on it.  Entry points that must learn a size on the host
 *    (mcmi_build*, mcmi_walk_dump) synchronise `stream` before returning,
 *    because the size of M is only known once the walks have run;
 *    mcmi_apply and mcmi_debug_tables do not.
 *  - Return value: MCMI_OK or an error code.  On error no output handle is
 *    produced (*M_out == NULL) and mcmi_last_error() describes the cause.
 *  - Matrices: CSR, int64 row_ptr[n+1] (row_ptr[0] == 0, non-decreasing,
 *    row_ptr[n] == nnz), int32 col[nnz] strictly increasing inside a row and
 *    in [0, n), float64 val[nnz] finite.  nnz must be below 2^32.
 *  - Determinism: a walk is a function of (seed, row, chain, step) only, so
 *    the same inputs and seed give the same paths and visit counts on any
 *    launch configuration, row subset or table layout of the same table
 *    type.  With the default accumulator (MCMI_ACC_FIXED64) each row sum is
 *    the exact sum of the walk weights in 64-bit fixed point, independent
 *    of the order of the additions, so M is bit-reproducible across runs,
 *    launch shapes, row shardings and batched builds.  The opt-in
 *    MCMI_ACC_KAHAN32 accumulator adds FP32 values with a compensation word
 *    in an order that depends on thread timing: its results can differ in
 *    the last bits between runs.
 */
#ifndef MCMI_H
#define MCMI_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MCMI_OK = 0,
    MCMI_ERR_ARG = 1,             /* null pointer, bad size or unsupported parameter */
    MCMI_ERR_BAD_CSR = 2,         /* malformed CSR: row_ptr, column order/range, non-finite value */
    MCMI_ERR_ZERO_DIAG = 3,       /* d_i = bhat_ii == 0 for some row (Eq. 1 needs d_i != 0) */
    MCMI_ERR_NOT_CONTRACTIVE = 4, /* some s_i = ||c_i||_1 >= 1: raise alpha (Eq. 1) */
    MCMI_ERR_OOM = 5,             /* device allocation failed */
    MCMI_ERR_CUDA = 6,            /* a CUDA runtime call failed */
    MCMI_ERR_TIMEOUT = 7,         /* a bounded device-side wait gave up */
    MCMI_ERR_CAPACITY = 8         /* an internal device capacity was exceeded */
} mcmi_status;

/* Sampling table of the transition probabilities p_ij = |c_ij| / s_i.    */
enum {
    MCMI_TABLE_AUTO = -1,       /* compact when every row fits it (and the accumulator is
                                 * FIXED64, no learned proposal); else cumulative for at most
                                 * six off-diagonals per row on average, hybrid otherwise */
    MCMI_TABLE_CUMULATIVE = 0,  /* integer cumulative thresholds (weights at the scale 2^31) */
    MCMI_TABLE_ALIAS = 1,       /* integer Walker/Vose alias buckets */
    MCMI_TABLE_HYBRID = 2,      /* per row: cumulative for at most 6 transitions (inline), alias otherwise */
    MCMI_TABLE_COMPACT = 3      /* cumulative thresholds at the scale 2^20 in one 32-byte record per
                                 * row (half the gather bytes of the 64-byte records); every row must
                                 * have at most 6 off-diagonals, each with |j - i| <= 16383, and the
                                 * accumulator must be FIXED64 (else MCMI_ERR_ARG) */
};

/* Row accumulator of the walk kernel.                                    */
enum {
    MCMI_ACC_FIXED64 = 0,  /* exact 64-bit fixed-point sum of the weights (deterministic) */
    MCMI_ACC_KAHAN32 = 1   /* FP32 sums of W/d_j with a compensation word (precision 32 only) */
};

typedef struct {
    int64_t n;              /* rows (= columns) */
    int64_t nnz;            /* stored entries */
    const int64_t *row_ptr; /* device, n+1 */
    const int32_t *col;     /* device, nnz */
    const double *val;      /* device, nnz */
} mcmi_csr;

/* Parameters of one preconditioner build.  Fill with mcmi_params_default.  */
typedef struct {
    double eps;          /* accuracy epsilon; used only to derive chains when chains == 0 */
    double delta;        /* weight cutoff: a chain stops once |W| < delta (tested on the FP32 weight) */
    double filter_tau;   /* keep |M_ij| >= tau * max_j |M_ij|; 0 disables */
    double alpha;        /* Eq. 1 augmentation bhat_ii = b_ii + alpha ||B||_inf sgn(b_ii); 0 = none */
    uint64_t seed;       /* Philox key */
    int32_t chains;      /* chains N per row (0: from eps and max_i s_i) */
    int32_t max_len;     /* maximum transitions L per chain (>= 0) */
    int32_t top_k;       /* keep at most top_k off-diagonals per row; 0 disables */
    int32_t precision;   /* 32: FP32 walk weights; 64: FP64 walk weights (row sums per `accumulator`) */
    int32_t table;       /* MCMI_TABLE_* */
    int32_t threads;     /* threads per block of the walk kernel (0 = auto; 64, 128 or 256) */
    int32_t hash_log2;   /* log2 of the on-chip accumulator slots per block (0 = auto) */
    int32_t accumulator; /* MCMI_ACC_*: row sums exact in 64-bit fixed point (default) or FP32 Kahan */
    int64_t row_begin;   /* build rows [row_begin, row_end) only; both 0 = all rows */
    int64_t row_end;
    int32_t chains_per_thread; /* chains each walk thread advances in turn: 1 or 2 (0 = auto) */
    int32_t load_depth;  /* global loads each walk thread keeps in flight in the loops after the
                          * walks: 4 (FP32: 64 registers, eight 128-thread blocks per SM) or 8
                          * (72 registers, seven blocks; fewer L2 round trips through the overflow
                          * log); 0 = auto: 8 for FP32 walks on matrices of more than six
                          * off-diagonals per row on average, else 4 */
    const struct mcmi_proposal_s *proposal; /* learned proposal (mcmi_proposal_*), NULL = p_ij = |c_ij|/s_i */
} mcmi_params;

/* Counters of the last build (all optional outputs).                      */
typedef struct {
    uint64_t steps;         /* transitions taken, summed over rows and chains */
    int64_t rows;           /* rows built */
    int64_t nnz;            /* entries of M */
    double max_s;           /* max_i ||c_i||_1 */
    int32_t chains;         /* N used */
    int32_t max_len_bound;  /* no chain can take more transitions than this */
    int32_t table;          /* table type used */
    int32_t hash_log2;      /* accumulator slots used (log2) */
    int64_t spilled;        /* distinct columns reduced from the overflow log (visits that did not fit on
                             * chip); with tau or top-k, FP32 fixed-point builds first drop the log's
                             * columns whose magnitude bound is below the threshold, and those are not
                             * counted */
    int64_t deferred_rows;  /* rows re-run because the first output buffer was full */
    float ms_prepare;       /* split + tables (CUDA events on the build stream) */
    float ms_walk;          /* walk stage incl. overflow-log set-up and deferred rows */
    float ms_assemble;      /* CSR assembly */
    float ms_walk_kernel;   /* the first walk kernel launch alone */
    int32_t launches;       /* kernels this build launched */
    int32_t threads;        /* walk threads per block used */
    int32_t chains_per_thread; /* chains each walk thread advanced */
    int32_t load_depth;     /* load depth used */
} mcmi_stats;

typedef struct mcmi_matrix_s *mcmi_matrix;

/* Defaults: eps 0.01, delta 1e-3, tau 0, alpha 0, seed 1, chains 128,
 * max_len 256, top_k 0, precision 32, table AUTO, accumulator FIXED64,
 * all rows.                                                              */
void mcmi_params_default(mcmi_params *p);

/* Build M ~ Bhat^-1 restricted to the sparsity the filter keeps (Eq. 2 walks,
 * phase 4 column scaling, Sec. IV-B filter).  Uses mcmi_params_default for
 * every parameter not in the argument list.  Synchronises `stream`.
 * B: device CSR (see conventions).  M_out: receives a library-owned handle
 * (free with mcmi_free).                                                  */
mcmi_status mcmi_build(const mcmi_csr *B, double eps, double delta, int32_t chains,
                       double filter_tau, uint64_t seed, void *stream, mcmi_matrix *M_out);

/* As mcmi_build with every parameter given; `stats` may be NULL.           */
mcmi_status mcmi_build_ex(const mcmi_csr *B, const mcmi_params *p, void *stream,
                          mcmi_matrix *M_out, mcmi_stats *stats);

/* Result of mcmi_autotune.                                                */
typedef struct {
    int32_t threads;            /* walk threads per block chosen */
    int32_t chains_per_thread;  /* chains each thread advances */
    int32_t hash_log2;          /* on-chip accumulator slots (log2) */
    int32_t table;              /* sampling table type */
    int32_t trials;             /* configurations timed */
    float best_ms;              /* walk time of the sample rows, configuration chosen */
    float default_ms;           /* same with the default plan (p as given, 0 fields = auto) */
    int32_t load_depth;         /* load depth chosen (4 or 8) */
    int64_t sample_rows;        /* rows in the timed sample */
} mcmi_tune_result;

/* Autotuner: times the walk kernel (CUDA events; each configuration twice,
 * the faster launch counts) on a sample of about 1/32 of the rows (8192 to
 * 65536 rows, in 32 windows spread evenly over the build's row range; a
 * batch's block-diagonal matrix mixes very different matrices): first the
 * default plan (p as given, its 0 fields auto), then every launch shape
 * (threads per block 64/128/256, 1 or 2 chains per thread) and on-chip
 * accumulator size (2^9 .. 2^13 slots) for each table type (all four when
 * p->table is MCMI_TABLE_AUTO; compact only where the rows fit it and the
 * accumulator is FIXED64), then the best of those at the other load
 * depth.  The best trial replaces the default plan only when it is at least
 * 2% faster.  Writes the choice into p->threads, p->chains_per_thread,
 * p->hash_log2, p->table and p->load_depth.  p: in/out (host); res: optional
 * (host).  Synchronises `stream`; allocates stream-ordered scratch.  Errors
 * as mcmi_build_ex.                                                       */
mcmi_status mcmi_autotune(const mcmi_csr *B, mcmi_params *p, void *stream, mcmi_tune_result *res);

/* Batched build of `count` independent matrices (each n >= 1) with the same
 * parameters: the matrices are gathered into one block-diagonal CSR so that
 * one persistent walk launch drains the rows of all of them from a single
 * device queue; the walk and the row-offset scan run as one CUDA graph,
 * whose executable form is kept per host thread and device and updated in
 * place for the next batched build when the topology matches.  A
 * row's random numbers are keyed by its index inside its own matrix, so
 * Ms[b] equals what mcmi_build_ex gives for Bs[b] alone with the same
 * parameters and table type.  If p->threads, p->chains_per_thread and
 * p->hash_log2 are all 0, the autotuner of mcmi_autotune picks them and the
 * load depth on the batch, for the table type the parameters give (AUTO:
 * its automatic choice, never another type, so that the batch walks the
 * same paths whatever the trials' timings).  With p->table AUTO (FIXED64 accumulator, no
 * learned proposal), a batch in which the compact table fits some matrices
 * but not others is built as two batches, one per group (each autotuned as
 * above when the shape is 0); stats then sum the two, and report the table
 * and launch shape of the group with more rows.  Bs: host array of device
 * CSRs; Ms: host array of `count` handles, set on success (NULL on error);
 * stats: optional aggregate.  Row ranges are not allowed.  Synchronises
 * `stream`.                                                              */
mcmi_status mcmi_build_batched(const mcmi_csr *Bs, int32_t count, const mcmi_params *p, void *stream,
                               mcmi_matrix *Ms, mcmi_stats *stats);

/* ---------------------------------------------------------------------
 * Learned proposal (an extension, not in the paper).  An 8-32-32-1 MLP
 * evaluated as a BF16 network (inputs, weights and hidden activations
 * rounded to bfloat16, exact products, FP32 sums in index order, FP32
 * biases) maps edge features -- p_ij = |c_ij|/s_i, s_i, s_j, 1/deg_i,
 * 1/deg_j, |d_i|/(|d_i|+|d_j|), |c_ij|/max_k|c_ik|, sign(c_ij) -- to
 * g_ij = squareplus(z) clamped to [1/16, 16].  The table samples
 * q_ij proportional to |c_ij| g_ij and the walk multiplies the weight by
 * c_ij Q_i / q_ij, so the Eq. 2 estimator stays unbiased.  Set
 * mcmi_params.proposal to use it (precision 32; alias tables).
 * Parameters (MCMI_MLP_PARAMS floats): W1[32][8], b1[32], W2[32][32],
 * b2[32], w3[32], b3.
 * --------------------------------------------------------------------- */
#define MCMI_MLP_PARAMS 1377
typedef struct mcmi_proposal_s *mcmi_proposal;

/* params: host float[MCMI_MLP_PARAMS], or NULL for the default start
 * (Glorot-uniform weights from a fixed sequence, zero biases).  Allocates
 * the device copy with cudaMalloc on the current device.                */
mcmi_status mcmi_proposal_create(const float *params, mcmi_proposal *out);
/* Current parameters to host float[MCMI_MLP_PARAMS] (synchronous).        */
mcmi_status mcmi_proposal_get(mcmi_proposal P, float *params);
void mcmi_proposal_free(mcmi_proposal P);

/* Training signal: m_i = (1/N) sum over row i's N chains of sum_t W_t^2
 * (t = 0 included; the walks of p, same paths as mcmi_build_ex).
 * m: device float[n].  Synchronises `stream`.                            */
mcmi_status mcmi_row_moments(const mcmi_csr *B, const mcmi_params *p, float *m, void *stream);

/* Training loss of the proposal on one matrix, given row moments m_rows
 * (device float[n]): the mean over rows with edges of
 * (sum_j p_ij g_ij)(sum_j p_ij m_j / g_ij) / (sum_j p_ij sqrt(m_j))^2,
 * >= 1, = 1 when g is proportional to sqrt(m) in every row (the
 * second-moment-optimal one-step proposal).  *loss (host); grad (host
 * float[MCMI_MLP_PARAMS] or NULL) receives d loss / d params (BF16
 * roundings taken as identity).  round_bf16 = 0 runs the network in FP32.
 * p supplies alpha for the split.  Synchronises `stream`.               */
mcmi_status mcmi_proposal_loss_grad(const mcmi_csr *B, const float *m_rows, const mcmi_params *p, mcmi_proposal P,
                                    int round_bf16, float *loss, float *grad, void *stream);

typedef struct {
    int32_t steps;      /* Adam steps over the whole training set */
    float lr;           /* Adam learning rate */
    int32_t chains;     /* chains per row for the row moments */
    int32_t max_len;    /* walk length limit for the row moments */
    double delta;       /* weight cutoff for the row moments */
    double alpha;       /* Eq. 1 augmentation of the training matrices */
    uint64_t seed;      /* Philox key of the walks */
    int32_t round_bf16; /* 1: train the BF16 network used at inference */
    int32_t reserved;
} mcmi_train_params;

/* Train P in place on `count` matrices (device CSRs): row moments from the
 * |c|-proposal walks, then tp->steps Adam steps on the loss above, with
 * the project's forward/backward kernels.  loss_history: host
 * float[tp->steps] or NULL.  Synchronises `stream`.                      */
mcmi_status mcmi_proposal_train(const mcmi_csr *Bs, int32_t count, const mcmi_train_params *tp, mcmi_proposal P,
                                float *loss_history, void *stream);

/* Device CSR of M (library-owned, valid until mcmi_free): rows
 * [row_begin, row_end) of the build, columns global, entries sorted by
 * column, FP32 values.  Any output pointer may be NULL.  Does not sync.    */
mcmi_status mcmi_matrix_csr(mcmi_matrix M, int64_t *rows, int64_t *row_begin, int64_t *nnz,
                            const int64_t **row_ptr, const int32_t **col, const float **val);

/* Copy M into caller-owned device buffers: row_ptr int64[rows+1], col
 * int32[nnz], val float[nnz] (sizes from mcmi_matrix_csr).  Asynchronous
 * on `stream`.                                                           */
mcmi_status mcmi_matrix_copy(mcmi_matrix M, int64_t *row_ptr, int32_t *col, float *val, void *stream);

/* y = M x (Sec. III-A: M is applied directly as a preconditioner).
 * x: device float[n] (global columns); y: device float[rows of M].
 * Asynchronous on `stream`.                                               */
mcmi_status mcmi_apply(mcmi_matrix M, const float *x, float *y, void *stream);

/* Krylov judge of the preconditioner (the paper tests its preconditioners
 * with GMRES and BiCGstab, Sec. VI; the GPU path keeps FP64 for this
 * residual): solve B x = b with right preconditioning B M y = b, x = M y.
 * method: MCMI_SOLVE_BICGSTAB or MCMI_SOLVE_GMRES (restarted every
 * `restart` inner iterations; 0 = 30).  B: device CSR (FP64); M: handle
 * from mcmi_build* or NULL (no preconditioner; rows outside a row-range M
 * act as identity); b: device double[n]; x: device double[n], output
 * (starts from 0).  Stops when the recurrence's residual norm reaches
 * rtol ||b|| or after maxit iterations (BiCGstab: full iterations; GMRES:
 * inner iterations).  *iters (host) = iterations done; *relres (host) =
 * the true FP64 residual ||b - B x|| / ||b|| recomputed at exit.
 * Synchronises `stream`; allocates its work vectors stream-ordered.      */
enum { MCMI_SOLVE_BICGSTAB = 0, MCMI_SOLVE_GMRES = 1 };
mcmi_status mcmi_solve(const mcmi_csr *B, mcmi_matrix M, const double *b, double *x, int method, double rtol,
                       int32_t maxit, int32_t restart, int32_t *iters, double *relres, void *stream);

/* Release a handle (stream-ordered on the stream it was built on).  NULL ok. */
void mcmi_free(mcmi_matrix M);

/* ---------------------------------------------------------------------
 * Recovery of B^-1 from Bhat^-1 (Eq. 3; Algorithm 1, step 5), a dense
 * O(n^3) diagnostic of the gap between Bhat^-1 and B^-1 for small n.
 * S = Bhat - B is diagonal: s_i = d_i - b_ii, d_i the Eq. 1 diagonal for
 * `alpha`.  For i = n-1, ..., 0 with s_i != 0,
 *     X <- X + g X e_i e_i^T X,  g = s_i / (1 - s_i X_ii)
 * (each step reads column i, row i and X_ii before updating; FP64, the
 * product taken as (g x_col) x_row).  B: device CSR; X: device dense
 * double[n * n], row-major, holding Bhat^-1 or an approximation of it on
 * entry and the recovered matrix on return.  n <= 16384.  Synchronises
 * `stream`.  Errors: MCMI_ERR_ARG (bad pointers or n, alpha < 0, a zero
 * denominator), MCMI_ERR_BAD_CSR, MCMI_ERR_ZERO_DIAG, MCMI_ERR_CUDA.     */
mcmi_status mcmi_recover_dense(const mcmi_csr *B, double alpha, double *X, void *stream);

/* Dense copy of M: X device double[rows * n_cols], row-major (rows, n_cols
 * from mcmi_matrix_csr; M's rows start at row_begin).  Asynchronous.      */
mcmi_status mcmi_matrix_dense(mcmi_matrix M, double *X, void *stream);

/* ---------------------------------------------------------------------
 * Matrix reduction (Algorithm 1, step 2; Sec. III, "Matrix Reduction"):
 * before the split, drop a set share of the off-diagonal entries of B that
 * are smallest in magnitude (diagonal entries are always kept; the others
 * keep their order).  mode:
 *   MCMI_REDUCE_ENTRIES: the floor(fraction * nnz_off) smallest |b_ij|,
 *     ties broken by position in CSR order (the earlier entry goes first);
 *   MCMI_REDUCE_RANGE: every |b_ij| < lo + fraction (hi - lo), lo and hi
 *     the smallest and largest off-diagonal |b_ij|, in FP64 in that order
 *     (the "% of the value range of the entries removed" of Sec. V).
 * B: device CSR (read only; columns need not be sorted); fraction in
 * [0, 1].  *R receives a library-owned device CSR (FP64 values) of the same
 * size n, viewed with mcmi_reduced_csr and released with
 * mcmi_reduced_free; *dropped (host, optional) the number of entries
 * removed.  Synchronises `stream`.  Errors: MCMI_ERR_ARG (bad pointers,
 * fraction or mode), MCMI_ERR_OOM, MCMI_ERR_CUDA; on error *R = NULL.     */
#define MCMI_REDUCE_ENTRIES 0
#define MCMI_REDUCE_RANGE 1
typedef struct mcmi_reduced_s *mcmi_reduced;
mcmi_status mcmi_reduce(const mcmi_csr *B, double fraction, int32_t mode, void *stream, mcmi_reduced *R,
                        int64_t *dropped);

/* View of a reduced matrix (device pointers owned by R, valid until
 * mcmi_reduced_free): pass *view to the builds as their B.               */
mcmi_status mcmi_reduced_csr(mcmi_reduced R, mcmi_csr *view);

/* Copy a reduced matrix into caller-owned device buffers: row_ptr
 * int64[n+1], col int32[nnz], val double[nnz] (sizes from
 * mcmi_reduced_csr).  Asynchronous on `stream`.                          */
mcmi_status mcmi_reduced_copy(mcmi_reduced R, int64_t *row_ptr, int32_t *col, double *val, void *stream);

/* Release a reduced matrix (stream-ordered on its stream).  NULL ok.      */
void mcmi_reduced_free(mcmi_reduced R);

/* Description of the last error on the calling host thread.               */
const char *mcmi_last_error(void);

/* ---------------------------------------------------------------------
 * Parity entry points (the same kernels, exposing intermediate results).
 * --------------------------------------------------------------------- */

/* Unfiltered Eq. 2 estimate of listed rows: for rows[p] (device int64,
 * nrows of them) writes out_count[p] entries at p*cap .. into out_col
 * (int32), out_val (float64: (1/N) sum_visits W / d_col, i.e. the row of
 * D-scaled estimate before filtering) and out_visits (uint32 visit counts),
 * unsorted, and out_steps[p] = transitions of the row's N chains.
 * All outputs device.  A row with more than cap entries sets out_count[p]
 * to -1 and the call returns MCMI_ERR_CAPACITY.  Synchronises `stream`.   */
mcmi_status mcmi_walk_dump(const mcmi_csr *B, const mcmi_params *p, const int64_t *rows,
                           int64_t nrows, int64_t cap, int32_t *out_count, uint64_t *out_steps,
                           int32_t *out_col, double *out_val, uint32_t *out_visits, void *stream);

/* The split and the sampling tables as built for the walk kernel.
 * out_d, out_s: device float64[n] (d_i, s_i = ||c_i||_1).
 * out_slot: device uint32[16 n]: the 64-byte row record of each row:
 *   [0] Q (sum of the row's integer weights; 0 = no transition),
 *   [1] fl32(s_i) bits, [2] fl32(1/d_i) bits, [3] deg | 0x80000000 if the
 *   row's table is out of line, [4..15] inline table or [4] = first index of
 *   the out-of-line table.
 *   Cumulative inline: up to 6 pairs (T_m, col_m | neg_m << 31), unused
 *   pairs (0xFFFFFFFF, 0).  Alias inline: up to 4 triples (prob_b,
 *   col_b | neg_b << 31, alias col | neg << 31).
 * out_a, out_b, out_c: device uint32[nnz] out-of-line tables (cumulative: a
 *   = T_m, b = col|neg; alias: a = prob, b = own col|neg, c = alias col|neg),
 *   row i's table starting at slot[4].  Asynchronous on `stream`.         */
mcmi_status mcmi_debug_tables(const mcmi_csr *B, const mcmi_params *p, double *out_d,
                              double *out_s, uint32_t *out_slot, uint32_t *out_a,
                              uint32_t *out_b, uint32_t *out_c, void *stream);

/* Gather roofline probe (measurement; the walk's access pattern without its
 * arithmetic).  Fills a device buffer of footprint_bytes with random
 * records of record_bytes (64: the 64-byte records, two 256-bit loads each;
 * 32: the compact table's records, one 256-bit load), then every thread of
 * blocks_per_sm x SMs blocks of threads_per_block threads follows two chains
 * of `steps` dependent random record reads (the next index taken from the
 * record read).  *records_per_s (host) receives the rate, timed with CUDA
 * events on `stream`.  Allocates and frees its buffer stream-ordered;
 * synchronises `stream`.  Errors: MCMI_ERR_ARG (footprint < 4096,
 * record_bytes not 32 or 64, bad launch shape), MCMI_ERR_OOM, MCMI_ERR_CUDA.
 * The paper names random memory access as the method's limiter (Sec. I,
 * Sec. IV-B).                                                            */
mcmi_status mcmi_gather_roofline(uint64_t footprint_bytes, int record_bytes, int threads_per_block,
                                 int blocks_per_sm, int steps, double *records_per_s, void *stream);

/* Gather roofline probe for the hybrid table's access pattern (measurement).
 * Like mcmi_gather_roofline with 64-byte records over
 * record_footprint_bytes, except that after a share bucket_share (0..1) of
 * the record reads, chosen by a hash of the record read, the chain reads one
 * 16-byte bucket (one 128-bit load, dependent on the record) of a second
 * buffer of bucket_footprint_bytes and takes the next record index from it:
 * the walk's steps out of rows whose alias table is stored out of line.
 * *records_per_s (host) receives the record reads per second (each with its
 * bucket read where taken), the faster of two schedules: the bucket read
 * within the step, or in the chain's next read slot while the lanes of the
 * other chains go on (the walk's schedule on alias tables).  Allocates and frees both buffers
 * stream-ordered; synchronises `stream`.  Errors: MCMI_ERR_ARG (a footprint
 * < 4096, bucket_share outside [0, 1], bad launch shape), MCMI_ERR_OOM,
 * MCMI_ERR_CUDA.  (Sec. I, Sec. IV-B: random memory access limits the
 * method.)                                                               */
mcmi_status mcmi_gather_roofline_mix(uint64_t record_footprint_bytes, uint64_t bucket_footprint_bytes,
                                     double bucket_share, int threads_per_block, int blocks_per_sm, int steps,
                                     double *records_per_s, void *stream);

/* ---------------------------------------------------------------------
 * Allocation-free entry point.  The paper has no counterpart: this is a
 * service for callers that must not allocate device memory at the point of
 * the call (a caller on a latency budget, where an allocation may block on
 * the driver; a program that hands out all of its device memory up front
 * from its own arena; a fixed-size device heap).
 *
 * mcmi_exclusive_scan_noalloc: offsets[i] = counts[0] + ... + counts[i-1]
 * for i = 0..n, so offsets[n] is the total -- the step that turns per-row
 * entry counts into CSR row pointers.  counts: device int32[n]; offsets:
 * device int64[n+1]; both owned by the caller.  Asynchronous on `stream`.
 * It calls no allocator: its scratch is a fixed device array of 16385
 * int64 words (128 KB) that every GPU loading this library keeps until the
 * process exits, so n may be at most 33,554,432; larger n returns
 * MCMI_ERR_ARG with a message naming the limit.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  The
 * address is kept for the life of the process: cudaDeviceReset, or
 * anything else that destroys the device's primary context, leaves it
 * stale, so after a reset this entry point must not be called again in the
 * same process.  All calls share the one array and it keeps the last
 * call's partial sums: calls that may overlap on the GPU (other streams,
 * other host threads) race and must be ordered by the caller.
 * --------------------------------------------------------------------- */
mcmi_status mcmi_exclusive_scan_noalloc(const int32_t *counts, int64_t n, int64_t *offsets, void *stream);

/* Library version string. */
const char *mcmi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MCMI_H */
