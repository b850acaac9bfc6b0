// C ABI of libmcmi: argument checks, device memory, stage ordering on the
// caller's stream, and the sizes the host must learn (max_i s_i, nnz of M).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "mcmi.h"
#include "mcmi_internal.cuh"

using namespace mcmi;

struct mcmi_matrix_s {
    int64_t rows = 0, row_begin = 0, n_cols = 0, nnz = 0;
    int64_t *rp = nullptr;
    int32_t *col = nullptr;
    float *val = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
};

// A reduced input matrix (FP64 CSR, device, library-owned).
struct mcmi_reduced_s {
    int64_t n = 0, nnz = 0;
    int64_t *rp = nullptr;
    int32_t *col = nullptr;
    double *val = nullptr;
    cudaStream_t stream = nullptr;
};

namespace {

thread_local std::string g_err;

mcmi_status fail(mcmi_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

mcmi_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? MCMI_ERR_OOM : MCMI_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// One memory pool per device with a high release threshold, so that repeated
// builds reuse device memory instead of returning it to the driver.
std::mutex g_pool_mu;
cudaMemPool_t g_pools[128] = {};

cudaError_t device_pool(int dev, cudaMemPool_t *out)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p;
        cudaError_t e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
        g_pools[dev] = p;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

// Stream-ordered device allocations released together when the owner ends.
struct Scratch {
    cudaStream_t s;
    cudaMemPool_t pool = nullptr;
    std::vector<void *> ptrs;
    cudaError_t err = cudaSuccess;
    explicit Scratch(cudaStream_t st) : s(st)
    {
        int dev = 0;
        err = cudaGetDevice(&dev);
        if (err == cudaSuccess) err = device_pool(dev, &pool);
    }
    template <class T>
    T *get(size_t count)
    {
        if (err != cudaSuccess) return nullptr;
        void *p = nullptr;
        const size_t bytes = count > 0 ? count * sizeof(T) : 16;
        err = cudaMallocFromPoolAsync(&p, bytes, pool, s);
        if (err != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    void release(void *p)
    {
        for (auto &q : ptrs)
            if (q == p) {
                cudaFreeAsync(q, s);
                q = nullptr;
            }
    }
    // hand ownership of p to the caller
    void keep(void *p)
    {
        for (auto &q : ptrs)
            if (q == p) q = nullptr;
    }
    ~Scratch()
    {
        for (void *p : ptrs)
            if (p) cudaFreeAsync(p, s);
    }
};

const char *status_name(int c)
{
    switch (c) {
    case MCMI_ERR_ARG: return "invalid argument";
    case MCMI_ERR_BAD_CSR: return "malformed CSR (row_ptr, column order/range, or non-finite value)";
    case MCMI_ERR_ZERO_DIAG: return "zero diagonal after the split (d_i == 0)";
    case MCMI_ERR_NOT_CONTRACTIVE: return "||c_i||_1 >= 1: the Neumann series need not converge (raise alpha)";
    case MCMI_ERR_CAPACITY: return "internal capacity exceeded";
    case MCMI_ERR_TIMEOUT: return "device wait timed out";
    default: return "error";
    }
}

// smallest float >= delta: |w| < delta (in FP64) <=> |w| < delta_f for float w
float delta_float(double delta)
{
    float f = (float)delta;
    if ((double)f < delta) f = nextafterf(f, INFINITY);
    return f;
}

// No chain outlives the FP32 product of fl32(max_i s_i): rounding is monotone.
int32_t walk_len_bound(double smax, double delta, int32_t L)
{
    const float f = (float)smax;
    if (!(delta > 0.0) || f >= 1.0f) return L;
    const float df = delta_float(delta);
    float w = 1.0f;
    int32_t t = 0;
    while (t < L && w >= df) {
        w = w * f;
        ++t;
    }
    return t;
}

int ceil_log2(uint64_t v)
{
    int l = 0;
    while ((1ull << l) < v) ++l;
    return l;
}

struct Prepared {
    int64_t n = 0, nnz = 0;
    double *d = nullptr, *s = nullptr;
    uint4 *slots = nullptr;
    uint32_t *a = nullptr, *b = nullptr, *c = nullptr;
    uint4 *bkt = nullptr;
    uint4 *lbkt = nullptr;       // learned proposal: 32-byte buckets
    float *invd32 = nullptr;     // fl32(1/d_i): compact table, and FP32 builds of the |c| proposal
    bool learned = false;
    double2 *rowd = nullptr;
    double smax = 0.0, smin = 0.0;
    int table = MCMI_TABLE_CUMULATIVE;
    int32_t N = 0, Lb = 0;
    DevState *st = nullptr;
};

mcmi_status check_csr(const mcmi_csr *B)
{
    if (!B) return fail(MCMI_ERR_ARG, "B is NULL");
    if (B->n < 0 || B->nnz < 0) return fail(MCMI_ERR_ARG, "negative size");
    if (B->n >= (1ll << 31) - 1) return fail(MCMI_ERR_ARG, "n must be below 2^31-1");
    if (B->nnz >= (1ll << 32)) return fail(MCMI_ERR_ARG, "nnz must be below 2^32");
    if (B->n > 0 && (!B->row_ptr || (B->nnz > 0 && (!B->col || !B->val))))
        return fail(MCMI_ERR_ARG, "NULL CSR array");
    return MCMI_OK;
}

mcmi_status check_params(const mcmi_params *p)
{
    if (!p) return fail(MCMI_ERR_ARG, "params is NULL");
    if (!(p->delta >= 0.0) || !(p->filter_tau >= 0.0) || !(p->alpha >= 0.0))
        return fail(MCMI_ERR_ARG, "delta, filter_tau and alpha must be >= 0");
    if (p->chains < 0 || p->max_len < 0 || p->top_k < 0) return fail(MCMI_ERR_ARG, "negative count");
    if (p->chains == 0 && !(p->eps > 0.0)) return fail(MCMI_ERR_ARG, "chains == 0 needs eps > 0");
    if (p->precision != 32 && p->precision != 64) return fail(MCMI_ERR_ARG, "precision must be 32 or 64");
    if (p->table < -1 || p->table > 3) return fail(MCMI_ERR_ARG, "unknown table type");
    if (p->table == MCMI_TABLE_COMPACT && p->accumulator != MCMI_ACC_FIXED64)
        return fail(MCMI_ERR_ARG, "the compact table needs the FIXED64 accumulator");
    if (p->table == MCMI_TABLE_COMPACT && p->proposal)
        return fail(MCMI_ERR_ARG, "a learned proposal uses its own alias table");
    if (p->chains_per_thread < 0 || p->chains_per_thread > 2)
        return fail(MCMI_ERR_ARG, "chains_per_thread must be 0, 1 or 2");
    if (p->threads != 0 && p->threads != 64 && p->threads != 128 && p->threads != 256)
        return fail(MCMI_ERR_ARG, "threads must be 0, 64, 128 or 256");
    if (p->load_depth != 0 && p->load_depth != 4 && p->load_depth != 8)
        return fail(MCMI_ERR_ARG, "load_depth must be 0, 4 or 8");
    if (p->threads == 256 && p->chains_per_thread == 2)
        return fail(MCMI_ERR_ARG, "256 threads per block need chains_per_thread 1");
    if (p->hash_log2 != 0 && (p->hash_log2 < 6 || p->hash_log2 > 13)) return fail(MCMI_ERR_ARG, "hash_log2 out of [6, 13]");
    if (p->accumulator != MCMI_ACC_FIXED64 && p->accumulator != MCMI_ACC_KAHAN32)
        return fail(MCMI_ERR_ARG, "unknown accumulator");
    if (p->accumulator == MCMI_ACC_KAHAN32 && p->precision != 32)
        return fail(MCMI_ERR_ARG, "the Kahan FP32 accumulator needs precision 32");
    if (p->proposal && p->precision != 32) return fail(MCMI_ERR_ARG, "a learned proposal needs precision 32");
    if (p->proposal && !p->proposal->d_params) return fail(MCMI_ERR_ARG, "proposal has no parameters");
    return MCMI_OK;
}

mcmi_status read_state(DevState *st, DevState *h, cudaStream_t s)
{
    cudaError_t e = cudaMemcpyAsync(h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "device state read");
    if (h->err != ~0ull) {
        const int code = (int)(h->err & 0xFF);
        const long long row = (long long)(h->err >> 8);
        return fail((mcmi_status)code, "%s (row %lld)", status_name(code), row);
    }
    return MCMI_OK;
}

// Stages a1 + a2: validation, split (FP64), integer tables.
mcmi_status prepare(const mcmi_csr *B, const mcmi_params *p, cudaStream_t s, Scratch &S, Prepared &P,
                    bool keep_debug)
{
    P.n = B->n;
    P.nnz = B->nnz;
    const int64_t n = B->n, nnz = B->nnz;
    P.st = S.get<DevState>(1);
    P.d = S.get<double>(n);
    P.s = S.get<double>(n);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation");
    cudaMemsetAsync(P.st, 0, sizeof(DevState), s);
    cudaMemsetAsync(&P.st->err, 0xFF, sizeof(unsigned long long), s);
    cudaMemsetAsync(&P.st->smin_bits, 0xFF, sizeof(unsigned long long), s);
    launch_validate(n, nnz, B->row_ptr, B->col, B->val, P.st, s);
    DevState h;
    mcmi_status r = read_state(P.st, &h, s);
    if (r != MCMI_OK) return r;
    if (p->alpha > 0.0) launch_rownorm(n, B->row_ptr, B->val, P.st, s);
    // the split and the tables take one row per thread, in an order that
    // gives each warp rows of similar length (from 2^16 rows on: below, the
    // two ordering launches cost more than the balance gains)
    int32_t *order = nullptr;
    unsigned long long *ocnt = nullptr;
    if (n >= (1 << 16)) {
        order = S.get<int32_t>(n);
        ocnt = S.get<unsigned long long>(32);
        if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation");
        cudaError_t oe = launch_len_order(n, B->row_ptr, ocnt, order, s);
        if (oe != cudaSuccess) return cuda_fail(oe, "row order");
    }
    launch_split(n, B->row_ptr, B->col, B->val, p->alpha, P.d, P.s, P.st, s, order);
    r = read_state(P.st, &h, s);
    if (r != MCMI_OK) return r;
    double smax;
    memcpy(&smax, &h.smax_bits, sizeof(double));
    P.smax = smax;
    if (h.smin_bits != ~0ull) memcpy(&P.smin, &h.smin_bits, sizeof(double));
    int table = p->table;
    // the compact table needs every row within its 32-byte record
    const bool compact_fits = h.max_deg <= (unsigned long long)kCompactMaxDeg &&
                              h.max_off <= (unsigned long long)kCompactMaxOff;
    if (table == MCMI_TABLE_COMPACT && !compact_fits)
        return fail(MCMI_ERR_ARG, "compact table: a row has %llu off-diagonals or |j - i| = %llu (at most %d and %d)",
                    (unsigned long long)h.max_deg, (unsigned long long)h.max_off, kCompactMaxDeg, kCompactMaxOff);
    // automatic choice: the compact table (one 32-byte load per step) where
    // every row fits it; else short rows on average favour the inline
    // cumulative table (one 64-byte load per step); otherwise the hybrid
    // table keeps rows of at most 6 transitions inline and gives longer rows
    // alias buckets
    if (table == MCMI_TABLE_AUTO) {
        if (compact_fits && p->accumulator == MCMI_ACC_FIXED64 && !p->proposal)
            table = MCMI_TABLE_COMPACT;
        else
            table = (nnz - (int64_t)h.ndiag) <= 6 * n ? MCMI_TABLE_CUMULATIVE : MCMI_TABLE_HYBRID;
    }
    if (p->proposal) table = MCMI_TABLE_ALIAS;   // learned proposals use 32-byte alias buckets
    P.table = table;
    P.learned = p->proposal != nullptr;
    if (p->chains > 0) {
        P.N = p->chains;
    } else {
        const double v = 0.6745 / (p->eps * (1.0 - smax));
        const double N = std::ceil(v * v);
        P.N = N > (double)(1 << 24) ? (1 << 24) : (int32_t)N;
    }
    // learned weights are not bounded by max_i s_i: no shorter bound than L
    P.Lb = P.learned ? p->max_len : walk_len_bound(smax, p->delta, p->max_len);
    const bool alias_kind = table == MCMI_TABLE_ALIAS || table == MCMI_TABLE_HYBRID;
    P.slots = S.get<uint4>((size_t)n * (table == MCMI_TABLE_COMPACT ? 2 : 4));
    // fl32(1/d_i) per row: the compact table's only copy; beside the other
    // tables' records (the finish after the walks then gathers from 4 bytes
    // per row, which stay in L2, instead of the 64-byte records)
    if (table == MCMI_TABLE_COMPACT || (p->precision == 32 && !P.learned)) P.invd32 = S.get<float>(n);
    P.a = S.get<uint32_t>(nnz);
    P.b = S.get<uint32_t>(nnz);
    unsigned long long *wscr = nullptr;
    uint32_t *sstk = nullptr, *lstk = nullptr;
    if (alias_kind || keep_debug) P.c = S.get<uint32_t>(nnz);
    if (alias_kind) {
        P.bkt = S.get<uint4>(nnz);
        wscr = S.get<unsigned long long>(nnz);
        sstk = S.get<uint32_t>(nnz);
        lstk = S.get<uint32_t>(nnz);
    }
    if (p->precision == 64) P.rowd = S.get<double2>(n);
    int *deg = nullptr;
    if (P.learned) {
        P.lbkt = S.get<uint4>((size_t)nnz * 2);
        deg = S.get<int>(n);
    }
    if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation");
    if (keep_debug) {
        cudaMemsetAsync(P.a, 0, nnz * 4, s);
        cudaMemsetAsync(P.b, 0, nnz * 4, s);
        cudaMemsetAsync(P.c, 0, nnz * 4, s);
    }
    if (P.learned) {
        // the network's inference fused into the table build
        launch_degree(n, B->row_ptr, B->col, deg, s);
        launch_tables_learned(n, B->row_ptr, B->col, B->val, P.d, P.s, deg, p->proposal->d_params, P.slots, P.a,
                              P.b, P.c, P.lbkt, wscr, sstk, lstk, s);
        S.release(deg);
    } else {
        launch_tables(n, B->row_ptr, B->col, B->val, P.d, P.s, table, P.slots, P.a, P.b, P.c, P.bkt, wscr, sstk,
                      lstk, P.rowd, P.invd32, s, order);
    }
    if (ocnt) S.release(ocnt);
    if (order) S.release(order);
    if (wscr) S.release(wscr);
    if (sstk) S.release(sstk);
    if (lstk) S.release(lstk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "table kernels");
    return MCMI_OK;
}

struct WalkPlan {
    int threads = 128, cpt = 2, depth = 4, log2H = 11, grid = 1;
};

mcmi_status plan_walk(const mcmi_params *p, const Prepared &P, int64_t rows, bool dump, WalkPlan &W)
{
    // default: 128 threads with one chain each (8 blocks = 8 rows in flight
    // per SM with a 2^11-slot table); the autotuner may pick 2 chains per
    // thread or other block sizes
    W.cpt = p->chains_per_thread ? p->chains_per_thread : 1;
    W.threads = p->threads ? p->threads : 128;
    // load depth 8 for FP32 walks on matrices of more than six off-diagonals
    // per row on average: their walks spread over many more columns than the
    // on-chip table holds, and the loops over the overflow log dominate; 4
    // (eight blocks per SM) otherwise.  FP64 walks spill at depth 8.
    W.depth = p->load_depth ? p->load_depth : ((p->precision == 32 && (P.nnz - P.n) > 6 * P.n) ? 8 : 4);
    // distinct columns a row can reach: at most N (Lb + 1) visits, at most n columns
    const uint64_t reach = (uint64_t)P.N * (uint64_t)(P.Lb + 2);
    const uint64_t distinct = reach < (uint64_t)P.n ? reach : (uint64_t)P.n;
    if (p->hash_log2) {
        W.log2H = p->hash_log2;
    } else {
        // on-chip table at most ~75% full for the reachable columns, capped at
        // 2^11 slots (24 KB) so that eight blocks share an SM; rows that reach
        // more columns log the excess visits and reduce them after the walks
        int l = ceil_log2((distinct * 4) / 3 + 1);
        W.log2H = l < 8 ? 8 : (l > 11 ? 11 : l);
    }
    int bps = 0;
    cudaError_t e = walk_occupancy(p->precision, P.table, p->accumulator, dump, W.cpt, W.depth, W.threads, W.log2H,
                                   &bps);
    if (e != cudaSuccess) return cuda_fail(e, "walk occupancy");
    if (bps < 1) return fail(MCMI_ERR_ARG, "walk kernel does not fit (threads %d, hash 2^%d)", W.threads, W.log2H);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t grid = (int64_t)sms * bps;
    if (grid > rows) grid = rows;
    W.grid = (int)(grid < 1 ? 1 : grid);
    return MCMI_OK;
}

void fill_walk_args(WalkArgs &a, const mcmi_params *p, const Prepared &P, const WalkPlan &W)
{
    memset(&a, 0, sizeof(a));
    a.slots = P.slots;
    a.invd32 = P.invd32;
    a.ool_a = P.a;
    a.ool_b = P.b;
    a.ool_bkt = P.bkt;
    a.lbkt = P.lbkt;
    a.w_limit = 1024.0f;
    a.rowd = P.rowd;
    a.N = P.N;
    a.L = p->max_len;
    a.delta_f = delta_float(p->delta);
    a.key0 = (uint32_t)p->seed;
    a.key1 = (uint32_t)(p->seed >> 32);
    a.log2H = W.log2H;
    a.tau = p->filter_tau;
    // Fixed-point scale 2^F: at most the F for which N (L_bound + 1) weights
    // of magnitude <= 1 stay below 2^62.  A small F keeps most weights below
    // 2^32, so the high-word atomic is rare.
    //  - FP32 walks with the |c| proposal: every accumulated weight is at
    //    least w_min = fl32(delta_f fl32(min_i s_i)) (the first weight below the
    //    cutoff, |W| >= delta_f times |f| >= fl32(s_min), rounded to nearest),
    //    so F = 23 - floor(log2 w_min) makes every FP32 weight an exact
    //    integer multiple of 2^-F: the sums are exact.
    //  - FP64 walks: F keeps the rounding of every weight below 2^-25 relative.
    //  - A learned proposal's weights may exceed 1: 10 more bits of head-room,
    //    and the kernel reports MCMI_ERR_CAPACITY if |W| ever passes 1024.
    //    Its factors |f_ij| = sum_k |c_ik| g_ik / g_ij are at least s_i / 256
    //    (g is clamped to [1/16, 16]), so its smallest weight is taken 2^8
    //    below delta min s, which keeps the same 2^-25 relative rounding
    //    (up to the Fmax cap).
    const double visits = (double)P.N * (double)(P.Lb + 1) + 1.0;
    const int Fmax = 62 - (int)std::ceil(std::log2(visits)) - (P.learned ? 10 : 0);
    int F = Fmax;
    const double wmin = p->delta * (double)(float)P.smin / (P.learned ? 256.0 : 1.0);
    if (p->precision == 32 && !P.learned && a.delta_f > 0.0f && P.smin > 0.0) {
        const float wmin32 = a.delta_f * (float)P.smin;   // IEEE single product, no contraction
        int e = 0;
        std::frexp(wmin32, &e);                             // wmin32 = m 2^e, m in [0.5, 1)
        const int Fexact = 23 - (e - 1);
        F = Fexact < 31 ? 31 : Fexact;
        if (F > Fmax) F = Fmax;
    } else if (wmin > 0.0) {
        const int Fneed = 25 + (int)std::ceil(-std::log2(wmin));
        F = Fneed < 31 ? 31 : Fneed;
        if (F > Fmax) F = Fmax;
    }
    a.fix_shift = F < 8 ? 8 : (F > 62 ? 62 : F);
    a.fix_inv = std::ldexp(1.0, -a.fix_shift);
    a.fin_scale = (float)(a.fix_inv / (double)P.N);
    a.top_k = p->top_k;
    a.st = P.st;
    a.count_steps = 1;
    // sketch kernels: the code of |1/d_j| rides in the spare top bits of the
    // log's column words when at least 9 are free (columns below 2^23) and the
    // table's value words can hold the cells; otherwise the walks add to the
    // global cells
    int nb = 0;
    while (nb < 31 && ((int64_t)1 << nb) < P.n) ++nb;   // bits of the largest column index
    const int cb = 32 - nb;
    a.sk_code_bits = (cb >= 9 && 2 * ((size_t)1 << W.log2H) >= walk_sketch_cells()) ? (cb < 12 ? cb : 12) : 0;
}

// Per-block overflow log (visits in arrival order, then bucketed: two
// regions) and entry list.  A row makes at most N Lb visits after t = 0, so
// the log never fills; the list takes the on-chip entries and the log's
// distinct columns.  When the regions of all blocks would pass a quarter of
// the free device memory, fewer blocks are launched.
mcmi_status alloc_overflow(Scratch &S, WalkPlan &W, const Prepared &P, bool dump, WalkArgs &a)
{
    const uint64_t logc = (uint64_t)P.N * (uint64_t)(P.Lb + 1);
    const uint64_t entc = logc + ((uint64_t)1 << W.log2H);
    if (entc > 0xFFFFFFF0ull) return fail(MCMI_ERR_ARG, "N (L + 1) = %llu visits per row is too large", (unsigned long long)logc);
    a.log_cap = (uint32_t)logc;
    a.ent_cap = (uint32_t)entc;
    const size_t per_block = (size_t)logc * 2 * 16 + (size_t)entc * (dump ? 16 : 12);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && (size_t)W.grid * per_block > fr / 4) {
        const size_t g = (fr / 4) / per_block;
        W.grid = g < 1 ? 1 : (int)g;
    }
    const size_t G = (size_t)W.grid;
    a.log_key = S.get<uint2>(G * 2 * logc);
    a.log_val = S.get<unsigned long long>(G * 2 * logc);
    a.ent_col = S.get<uint32_t>(G * entc);
    a.ent_val = S.get<unsigned long long>(G * entc);
    a.ent_cnt = dump ? S.get<uint32_t>(G * entc) : nullptr;
    a.cells = dump ? nullptr : S.get<uint32_t>(G * walk_sketch_cells());
    if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation (overflow log)");
    if (a.cells) {
        const cudaError_t e = cudaMemsetAsync(a.cells, 0, G * walk_sketch_cells() * sizeof(uint32_t), S.s);
        if (e != cudaSuccess) return cuda_fail(e, "sketch cells");
    }
    return MCMI_OK;
}

void reset_queue(DevState *st, cudaStream_t s)
{
    cudaMemsetAsync(&st->work, 0, sizeof(unsigned long long), s);
}

// One timed walk launch over the rows of a device list with plan W
// (autotuner trial).
mcmi_status time_walk(const mcmi_params *p, const Prepared &P, WalkPlan W, const int64_t *list, int64_t rows,
                      cudaStream_t s, float *ms)
{
    Scratch S(s);
    WalkArgs a;
    fill_walk_args(a, p, P, W);
    a.row_list = list;
    a.n_list = rows;
    a.out_by_row = 0;
    mcmi_status r = alloc_overflow(S, W, P, false, a);
    if (r != MCMI_OK) return r;
    const uint64_t per_row = p->top_k > 0 ? (uint64_t)(p->top_k + 1) : 512;
    a.st_cap = (uint64_t)rows * per_row + 1024;
    a.st_col = S.get<uint32_t>(a.st_cap);
    a.st_val = S.get<float>(a.st_cap);
    a.row_off = S.get<int64_t>(rows);
    a.row_cnt = S.get<int32_t>(rows);
    a.deferred_list = S.get<int64_t>(rows);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation (autotune)");
    cudaMemsetAsync(&P.st->cursor, 0, 8, s);
    cudaMemsetAsync(&P.st->deferred, 0, 8, s);
    reset_queue(P.st, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    cudaError_t e = launch_walk(a, p->precision, P.table, p->accumulator, false, W.cpt, W.depth, W.grid, W.threads, s);
    cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "walk kernel (autotune)");
    DevState h;
    return read_state(P.st, &h, s);
}

}  // namespace

// keep_table: only the table the parameters give (AUTO: its automatic
// choice) is tried, so that the tuned build walks the same paths as an
// untuned one and its output does not depend on the trials' timings.
static mcmi_status autotune_impl(const mcmi_csr *B, mcmi_params *p, void *stream, mcmi_tune_result *res,
                                 bool keep_table)
{
    mcmi_status r = check_csr(B);
    if (r == MCMI_OK) r = check_params(p);
    if (r != MCMI_OK) return r;
    if (B->n == 0) return fail(MCMI_ERR_ARG, "empty matrix");
    const int64_t n = B->n;
    const int64_t rb0 = (p->row_begin == 0 && p->row_end == 0) ? 0 : p->row_begin;
    const int64_t re0 = (p->row_begin == 0 && p->row_end == 0) ? n : p->row_end;
    if (rb0 < 0 || re0 <= rb0 || re0 > n) return fail(MCMI_ERR_ARG, "bad row range");
    cudaStream_t s = (cudaStream_t)stream;
    // sample: about 1/32 of the rows, 8192 .. 65536 (several rows per
    // resident block, so that the last rows' tail does not decide a trial),
    // in 32 equal windows spread evenly over the row range (a batch's
    // block-diagonal matrix mixes very different matrices)
    const int64_t range = re0 - rb0;
    int64_t ns = range / 32;
    ns = ns < 8192 ? 8192 : (ns > 65536 ? 65536 : ns);
    if (ns > range) ns = range;
    std::vector<int64_t> hrows((size_t)ns);
    {
        const int64_t nwin = ns < 32 ? 1 : 32, wlen = ns / nwin;
        int64_t k = 0;
        for (int64_t w = 0; w < nwin; ++w) {
            const int64_t len = w == nwin - 1 ? ns - k : wlen;
            const int64_t start = rb0 + (nwin == 1 ? 0 : (range - len) * w / (nwin - 1));
            for (int64_t j = 0; j < len; ++j) hrows[(size_t)k++] = start + j;
        }
    }
    Scratch SL(s);
    int64_t *sample = SL.get<int64_t>((size_t)ns);
    if (SL.err != cudaSuccess) return cuda_fail(SL.err, "allocation (autotune sample)");
    cudaError_t ce = cudaMemcpyAsync(sample, hrows.data(), (size_t)ns * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_fail(ce, "autotune sample copy");
    int trials = 0;
    // one configuration: the faster of two launches on the sample
    auto trial = [&](const mcmi_params &q, const Prepared &P, WalkPlan &W, float *ms, bool *fits) -> mcmi_status {
        *fits = plan_walk(&q, P, ns, false, W) == MCMI_OK;
        if (!*fits) return MCMI_OK;
        float t0 = 0.0f, t1 = 0.0f;
        mcmi_status rr = time_walk(&q, P, W, sample, ns, s, &t0);
        if (rr == MCMI_OK) rr = time_walk(&q, P, W, sample, ns, s, &t1);
        *ms = t0 < t1 ? t0 : t1;
        ++trials;
        return rr;
    };
    // the default plan first: a trial replaces it only when at least 2% faster
    mcmi_params bestp = *p;
    float dflt = -1.0f;
    {
        Scratch S(s);
        if (S.err != cudaSuccess) return cuda_fail(S.err, "memory pool");
        Prepared P;
        r = prepare(B, p, s, S, P, false);
        if (r != MCMI_OK) return r;
        WalkPlan W;
        bool fits = false;
        r = trial(*p, P, W, &dflt, &fits);
        if (r != MCMI_OK) return r;
        if (!fits) return fail(MCMI_ERR_ARG, "walk kernel does not fit with the given parameters");
        bestp.threads = W.threads;
        bestp.chains_per_thread = W.cpt;
        bestp.hash_log2 = W.log2H;
        bestp.load_depth = W.depth;
        bestp.table = P.table;
    }
    float best = dflt;
    const float bar = 0.98f * dflt;
    struct Shape { int threads, cpt; } shapes[] = {{128, 1}, {256, 1}, {128, 2}, {64, 2}};
    const int hashes[] = {9, 10, 11, 12, 13};
    int tables[4] = {MCMI_TABLE_CUMULATIVE, MCMI_TABLE_ALIAS, MCMI_TABLE_HYBRID, MCMI_TABLE_COMPACT};
    const bool compact_ok = p->accumulator == MCMI_ACC_FIXED64 && !p->proposal;
    const int ntab = (p->table == MCMI_TABLE_AUTO && !keep_table) ? (compact_ok ? 4 : 3) : 1;
    if (p->table != MCMI_TABLE_AUTO) tables[0] = p->table;
    else if (keep_table) tables[0] = bestp.table;   // the automatic choice, resolved by the default trial
    mcmi_params cand = bestp;
    float cand_ms = 1e30f;
    for (int ti = 0; ti < ntab; ++ti) {
        mcmi_params q = *p;
        q.table = tables[ti];
        Scratch S(s);
        if (S.err != cudaSuccess) return cuda_fail(S.err, "memory pool");
        Prepared P;
        r = prepare(B, &q, s, S, P, false);
        if (r != MCMI_OK && q.table == MCMI_TABLE_COMPACT && p->table == MCMI_TABLE_AUTO) continue;   // rows do not fit
        if (r != MCMI_OK) return r;
        for (const Shape &sh : shapes)
            for (int hl : hashes) {
                q.threads = sh.threads;
                q.chains_per_thread = sh.cpt;
                q.hash_log2 = hl;
                WalkPlan W;
                float ms = 0.0f;
                bool fits = false;
                r = trial(q, P, W, &ms, &fits);
                if (r != MCMI_OK) return r;
                if (fits && ms < cand_ms) {
                    cand_ms = ms;
                    cand = q;
                    cand.load_depth = W.depth;
                }
            }
    }
    // the best shape at the other load depth
    {
        mcmi_params q = cand;
        Scratch S(s);
        if (S.err != cudaSuccess) return cuda_fail(S.err, "memory pool");
        Prepared P;
        r = prepare(B, &q, s, S, P, false);
        if (r != MCMI_OK) return r;
        q.load_depth = cand.load_depth == 8 ? 4 : 8;
        WalkPlan W;
        float ms = 0.0f;
        bool fits = false;
        r = trial(q, P, W, &ms, &fits);
        if (r != MCMI_OK) return r;
        if (fits && ms < cand_ms) {
            cand_ms = ms;
            cand = q;
        }
    }
    if (cand_ms < bar) {
        best = cand_ms;
        bestp = cand;
    }
    p->threads = bestp.threads;
    p->chains_per_thread = bestp.chains_per_thread;
    p->hash_log2 = bestp.hash_log2;
    p->table = bestp.table;
    p->load_depth = bestp.load_depth;
    if (res) {
        res->threads = bestp.threads;
        res->chains_per_thread = bestp.chains_per_thread;
        res->hash_log2 = bestp.hash_log2;
        res->table = bestp.table;
        res->load_depth = bestp.load_depth;
        res->trials = trials;
        res->best_ms = best;
        res->default_ms = dflt;
        res->sample_rows = ns;
    }
    return MCMI_OK;
}

extern "C" mcmi_status mcmi_autotune(const mcmi_csr *B, mcmi_params *p, void *stream, mcmi_tune_result *res)
{
    return autotune_impl(B, p, stream, res, false);
}

void mcmi::set_error_message(const char *msg) { g_err = msg; }

extern "C" {

const char *mcmi_last_error(void) { return g_err.c_str(); }

const char *mcmi_version(void) { return "mcmi-b300 0.1 (sm_103a)"; }

void mcmi_params_default(mcmi_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->eps = 0.01;
    p->delta = 1e-3;
    p->filter_tau = 0.0;
    p->alpha = 0.0;
    p->seed = 1;
    p->chains = 128;
    p->max_len = 256;
    p->top_k = 0;
    p->precision = 32;
    p->table = MCMI_TABLE_AUTO;
}

mcmi_status mcmi_build_ex(const mcmi_csr *B, const mcmi_params *p, void *stream, mcmi_matrix *M_out,
                          mcmi_stats *stats)
{
    if (!M_out) return fail(MCMI_ERR_ARG, "M_out is NULL");
    *M_out = nullptr;
    mcmi_status r = check_csr(B);
    if (r == MCMI_OK) r = check_params(p);
    if (r != MCMI_OK) return r;
    const int64_t n = B->n;
    const int64_t rb = (p->row_begin == 0 && p->row_end == 0) ? 0 : p->row_begin;
    const int64_t re = (p->row_begin == 0 && p->row_end == 0) ? n : p->row_end;
    if (rb < 0 || re < rb || re > n) return fail(MCMI_ERR_ARG, "row range [%lld, %lld) outside [0, %lld)",
                                                 (long long)rb, (long long)re, (long long)n);
    const int64_t rows = re - rb;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch S(s);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "memory pool");
    mcmi_matrix M = new mcmi_matrix_s();
    M->rows = rows;
    M->row_begin = rb;
    M->n_cols = n;
    M->stream = s;
    cudaGetDevice(&M->device);
    auto give_up = [&](mcmi_status st) {
        if (M->rp) cudaFreeAsync(M->rp, s);
        if (M->col) cudaFreeAsync(M->col, s);
        if (M->val) cudaFreeAsync(M->val, s);
        delete M;
        return st;
    };
    if (stats) memset(stats, 0, sizeof(*stats));
    if (n == 0 || rows == 0) {
        M->rp = S.get<int64_t>(rows + 1);
        if (S.err != cudaSuccess) return give_up(cuda_fail(S.err, "allocation"));
        S.keep(M->rp);
        cudaMemsetAsync(M->rp, 0, (rows + 1) * sizeof(int64_t), s);
        cudaStreamSynchronize(s);
        *M_out = M;
        return MCMI_OK;
    }
    cudaEvent_t ev[6];
    for (auto &e : ev) cudaEventCreate(&e);
    struct EvGuard { cudaEvent_t *e; ~EvGuard() { for (int i = 0; i < 6; ++i) cudaEventDestroy(e[i]); } } evg{ev};
    int launches = 3 + (p->alpha > 0.0 ? 1 : 0);   // validate, split, tables (+ row norms)
    cudaEventRecord(ev[0], s);

    Prepared P;
    r = prepare(B, p, s, S, P, false);
    if (r != MCMI_OK) return give_up(r);
    cudaEventRecord(ev[1], s);

    WalkPlan W;
    r = plan_walk(p, P, rows, false, W);
    if (r != MCMI_OK) return give_up(r);
    WalkArgs a;
    fill_walk_args(a, p, P, W);
    a.row_begin = rb;
    a.row_end = re;
    r = alloc_overflow(S, W, P, false, a);
    if (r != MCMI_OK) return give_up(r);
    const uint64_t reach = (uint64_t)P.N * (uint64_t)(P.Lb + 2);
    const uint64_t distinct = reach < (uint64_t)n ? reach : (uint64_t)n;
    // staging entries: exact for top-k; for the tau rule an estimate of up to
    // 512 kept entries per row (rows that do not fit are re-run), bounded by
    // a quarter of the free device memory
    uint64_t per_row = p->top_k > 0 ? (uint64_t)(p->top_k + 1) : 512;
    if (per_row > distinct + 1) per_row = distinct + 1;
    uint64_t cap = (uint64_t)rows * per_row + 1024;
    if (p->top_k == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && cap * 8 > fr / 4) cap = fr / 32 + 1024;
    }
    a.st_col = S.get<uint32_t>(cap);
    a.st_val = S.get<float>(cap);
    a.st_cap = cap;
    a.row_off = S.get<int64_t>(rows);
    a.row_cnt = S.get<int32_t>(rows);
    a.deferred_list = S.get<int64_t>(rows);
    if (S.err != cudaSuccess) return give_up(cuda_fail(S.err, "allocation (staging)"));
    reset_queue(P.st, s);
    cudaEventRecord(ev[4], s);
    cudaError_t e = launch_walk(a, p->precision, P.table, p->accumulator, false, W.cpt, W.depth, W.grid, W.threads, s);
    if (e != cudaSuccess) return give_up(cuda_fail(e, "walk kernel launch"));
    cudaEventRecord(ev[5], s);
    ++launches;
    DevState h;
    r = read_state(P.st, &h, s);
    if (r != MCMI_OK) return give_up(r);
    int64_t deferred = (int64_t)h.deferred;
    if (deferred > 0) {
        // rows that found the staging buffer full run again (same seed, so the
        // same walks) into a buffer large enough for any row
        const uint64_t need = h.cursor + (uint64_t)deferred * (distinct + 1);
        uint32_t *col2 = S.get<uint32_t>(need);
        float *val2 = S.get<float>(need);
        int64_t *list2 = S.get<int64_t>(deferred);
        if (S.err != cudaSuccess) return give_up(cuda_fail(S.err, "allocation (staging regrowth)"));
        cudaMemcpyAsync(col2, a.st_col, cap * 4, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(val2, a.st_val, cap * 4, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(list2, a.deferred_list, deferred * 8, cudaMemcpyDeviceToDevice, s);
        S.release(a.st_col);
        S.release(a.st_val);
        a.st_col = col2;
        a.st_val = val2;
        a.st_cap = need;
        a.row_list = list2;
        a.n_list = deferred;
        a.out_by_row = 1;
        a.count_steps = 0;   // their transitions were counted in the first launch
        cudaMemsetAsync(&P.st->deferred, 0, 8, s);
        reset_queue(P.st, s);
        WalkPlan W2 = W;
        W2.grid = (int)(deferred < W.grid ? deferred : W.grid);
        e = launch_walk(a, p->precision, P.table, p->accumulator, false, W2.cpt, W2.depth, W2.grid, W2.threads, s);
        if (e != cudaSuccess) return give_up(cuda_fail(e, "walk kernel launch (deferred rows)"));
        ++launches;
        r = read_state(P.st, &h, s);
        if (r != MCMI_OK) return give_up(r);
        if (h.deferred) return give_up(fail(MCMI_ERR_CAPACITY, "staging buffer still full"));
    }
    cudaEventRecord(ev[2], s);

    M->rp = S.get<int64_t>(rows + 1);
    int64_t *tmp = S.get<int64_t>(scan_tmp_elems(rows));
    if (S.err != cudaSuccess) return give_up(cuda_fail(S.err, "allocation (row_ptr)"));
    S.keep(M->rp);
    e = scan_counts(a.row_cnt, rows, M->rp, tmp, s);
    if (e != cudaSuccess) return give_up(cuda_fail(e, "scan"));
    int64_t nnzM = 0;
    e = cudaMemcpyAsync(&nnzM, M->rp + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return give_up(cuda_fail(e, "nnz read"));
    M->nnz = nnzM;
    M->col = S.get<int32_t>(nnzM);
    M->val = S.get<float>(nnzM);
    if (S.err != cudaSuccess) return give_up(cuda_fail(S.err, "allocation (M)"));
    S.keep(M->col);
    S.keep(M->val);
    e = launch_assemble(rows, M->rp, a.row_off, a.row_cnt, a.st_col, a.st_val, M->col, M->val,
                        p->top_k > 0 ? (int64_t)p->top_k + 1 : 0, s);
    if (e != cudaSuccess) return give_up(cuda_fail(e, "assembly"));
    launches += 4;   // three scan kernels + assembly
    cudaEventRecord(ev[3], s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return give_up(cuda_fail(e, "build"));
    if (stats) {
        stats->steps = h.steps;
        stats->rows = rows;
        stats->nnz = nnzM;
        stats->max_s = P.smax;
        stats->chains = P.N;
        stats->max_len_bound = P.Lb;
        stats->table = P.table;
        stats->hash_log2 = W.log2H;
        stats->spilled = (int64_t)h.spilled;
        stats->deferred_rows = deferred;
        cudaEventElapsedTime(&stats->ms_prepare, ev[0], ev[1]);
        cudaEventElapsedTime(&stats->ms_walk, ev[1], ev[2]);
        cudaEventElapsedTime(&stats->ms_assemble, ev[2], ev[3]);
        cudaEventElapsedTime(&stats->ms_walk_kernel, ev[4], ev[5]);
        stats->launches = launches;
        stats->threads = W.threads;
        stats->chains_per_thread = W.cpt;
        stats->load_depth = W.depth;
    }
    *M_out = M;
    return MCMI_OK;
}

mcmi_status mcmi_build(const mcmi_csr *B, double eps, double delta, int32_t chains, double filter_tau,
                       uint64_t seed, void *stream, mcmi_matrix *M_out)
{
    mcmi_params p;
    mcmi_params_default(&p);
    p.eps = eps;
    p.delta = delta;
    p.chains = chains;
    p.filter_tau = filter_tau;
    p.seed = seed;
    return mcmi_build_ex(B, &p, stream, M_out, nullptr);
}

static mcmi_status batched_impl(const mcmi_csr *Bs, int32_t count, const mcmi_params *p_in, void *stream,
                                mcmi_matrix *Ms, mcmi_stats *stats)
{
    if (!Bs || !Ms || count < 1) return fail(MCMI_ERR_ARG, "batched build needs count >= 1 matrices and outputs");
    for (int32_t b = 0; b < count; ++b) Ms[b] = nullptr;
    mcmi_status r = check_params(p_in);
    if (r != MCMI_OK) return r;
    if (p_in->row_begin || p_in->row_end) return fail(MCMI_ERR_ARG, "row ranges do not apply to batched builds");
    std::vector<BatchIn> in(count);
    std::vector<int64_t> row_base(count + 1), nnz_base(count + 1);
    int64_t tn = 0, tz = 0;
    for (int32_t b = 0; b < count; ++b) {
        r = check_csr(&Bs[b]);
        if (r != MCMI_OK) return fail(r, "matrix %d: %s", b, g_err.c_str());
        if (Bs[b].n < 1) return fail(MCMI_ERR_ARG, "matrix %d is empty", b);
        in[b] = BatchIn{Bs[b].row_ptr, Bs[b].col, Bs[b].val, Bs[b].n, Bs[b].nnz, tn, tz};
        row_base[b] = tn;
        nnz_base[b] = tz;
        tn += Bs[b].n;
        tz += Bs[b].nnz;
    }
    row_base[count] = tn;
    nnz_base[count] = tz;
    if (tn >= (1ll << 31) - 1 || tz >= (1ll << 32)) return fail(MCMI_ERR_ARG, "batch too large (rows < 2^31, nnz < 2^32)");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch S(s);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "memory pool");
    cudaEvent_t ev[6];
    for (auto &e : ev) cudaEventCreate(&e);
    struct EvGuard { cudaEvent_t *e; ~EvGuard() { for (int i = 0; i < 6; ++i) cudaEventDestroy(e[i]); } } evg{ev};
    cudaEventRecord(ev[0], s);

    // block-diagonal concatenation (global column = local column + row base)
    BatchIn *d_in = S.get<BatchIn>(count);
    int64_t *d_row_base = S.get<int64_t>(count + 1), *d_nnz_base = S.get<int64_t>(count + 1);
    int64_t *rp_all = S.get<int64_t>(tn + 1);
    int32_t *col_all = S.get<int32_t>(tz);
    double *val_all = S.get<double>(tz);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation (batch)");
    cudaMemcpyAsync(d_in, in.data(), sizeof(BatchIn) * count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_row_base, row_base.data(), 8 * (count + 1), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_nnz_base, nnz_base.data(), 8 * (count + 1), cudaMemcpyHostToDevice, s);
    cudaError_t e = launch_concat(d_in, count, d_row_base, d_nnz_base, tn, tz, rp_all, col_all, val_all, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch concatenation");
    mcmi_csr Ball{tn, tz, rp_all, col_all, val_all};
    int launches = 2;

    // launch shape: the autotuner, unless the caller fixed it
    mcmi_params q = *p_in;
    mcmi_tune_result tune{};
    if (q.threads == 0 && q.chains_per_thread == 0 && q.hash_log2 == 0) {
        // launch shape, accumulator size and load depth only: the table stays
        // the one the parameters give, so the batch's paths do not depend on
        // the autotuner's timings
        r = autotune_impl(&Ball, &q, stream, &tune, true);
        if (r != MCMI_OK) return r;
    }
    Prepared P;
    r = prepare(&Ball, &q, s, S, P, false);
    if (r != MCMI_OK) return r;
    launches += 3 + (q.alpha > 0.0 ? 1 : 0);
    cudaEventRecord(ev[1], s);
    WalkPlan W;
    r = plan_walk(&q, P, tn, false, W);
    if (r != MCMI_OK) return r;
    WalkArgs a;
    fill_walk_args(a, &q, P, W);
    a.row_begin = 0;
    a.row_end = tn;
    a.batch_row_base = d_row_base;
    a.batch_count = count;
    r = alloc_overflow(S, W, P, false, a);
    if (r != MCMI_OK) return r;
    const uint64_t reach = (uint64_t)P.N * (uint64_t)(P.Lb + 2);
    const uint64_t distinct = reach < (uint64_t)tn ? reach : (uint64_t)tn;
    uint64_t per_row = q.top_k > 0 ? (uint64_t)(q.top_k + 1) : 512;
    if (per_row > distinct + 1) per_row = distinct + 1;
    uint64_t cap = (uint64_t)tn * per_row + 1024;
    if (q.top_k == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && cap * 8 > fr / 4) cap = fr / 32 + 1024;
    }
    a.st_col = S.get<uint32_t>(cap);
    a.st_val = S.get<float>(cap);
    a.st_cap = cap;
    a.row_off = S.get<int64_t>(tn);
    a.row_cnt = S.get<int32_t>(tn);
    a.deferred_list = S.get<int64_t>(tn);
    int64_t *rpM = S.get<int64_t>(tn + 1);
    int64_t *tmp = S.get<int64_t>(scan_tmp_elems(tn));
    if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation (batch staging)");

    // walk + scan as one CUDA graph on a private stream ordered after `s`.
    // The executable graph of the previous batched build on this host
    // thread and device is updated in place (cudaGraphExecUpdate) when the
    // new capture has the same topology, so repeated builds pay the capture
    // but not the instantiation.
    struct GraphCache {
        cudaGraphExec_t exec = nullptr;
        int device = -1;
        ~GraphCache() { if (exec) cudaGraphExecDestroy(exec); }
    };
    static thread_local GraphCache gcache;
    int cur_dev = 0;
    cudaGetDevice(&cur_dev);
    if (gcache.exec && gcache.device != cur_dev) {
        cudaGraphExecDestroy(gcache.exec);
        gcache.exec = nullptr;
    }
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[2], 0);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(&P.st->work, 0, 8, cs);
        cudaMemsetAsync(&P.st->cursor, 0, 8, cs);
        cudaMemsetAsync(&P.st->deferred, 0, 8, cs);
        cudaEventRecord(ev[4], cs);
        cudaError_t e1 = launch_walk(a, q.precision, P.table, q.accumulator, false, W.cpt, W.depth, W.grid, W.threads, cs);
        cudaEventRecord(ev[5], cs);
        cudaError_t e2 = scan_counts(a.row_cnt, tn, rpM, tmp, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
    }
    if (e == cudaSuccess && gcache.exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(gcache.exec, graph, &info) == cudaSuccess) {
            gexec = gcache.exec;
        } else {
            cudaGetLastError();   // an update that does not apply is not an error of this build
            cudaGraphExecDestroy(gcache.exec);
            gcache.exec = nullptr;
        }
    }
    if (e == cudaSuccess && !gexec) {
        e = cudaGraphInstantiate(&gexec, graph, 0);
        if (e == cudaSuccess) {
            gcache.exec = gexec;
            gcache.device = cur_dev;
        }
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(gexec, cs);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[3], 0);
    if (graph) cudaGraphDestroy(graph);
    if (cs) {
        cudaStreamSynchronize(cs);
        cudaStreamDestroy(cs);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batched walk graph");
    launches += 4;
    DevState h;
    r = read_state(P.st, &h, s);
    if (r != MCMI_OK) return r;
    const int64_t deferred = (int64_t)h.deferred;
    if (deferred > 0) {
        // rows whose output did not fit: run again (same walks) into a larger buffer
        const uint64_t need = h.cursor + (uint64_t)deferred * (distinct + 1);
        uint32_t *col2 = S.get<uint32_t>(need);
        float *val2 = S.get<float>(need);
        int64_t *list2 = S.get<int64_t>(deferred);
        if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation (staging regrowth)");
        cudaMemcpyAsync(col2, a.st_col, cap * 4, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(val2, a.st_val, cap * 4, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(list2, a.deferred_list, deferred * 8, cudaMemcpyDeviceToDevice, s);
        a.st_col = col2;
        a.st_val = val2;
        a.st_cap = need;
        a.row_list = list2;
        a.n_list = deferred;
        a.out_by_row = 1;
        a.count_steps = 0;
        cudaMemsetAsync(&P.st->deferred, 0, 8, s);
        reset_queue(P.st, s);
        const int g2 = (int)(deferred < W.grid ? deferred : W.grid);
        e = launch_walk(a, q.precision, P.table, q.accumulator, false, W.cpt, W.depth, g2, W.threads, s);
        if (e == cudaSuccess) e = scan_counts(a.row_cnt, tn, rpM, tmp, s);
        if (e != cudaSuccess) return cuda_fail(e, "walk kernel launch (deferred rows)");
        launches += 4;
        r = read_state(P.st, &h, s);
        if (r != MCMI_OK) return r;
        if (h.deferred) return fail(MCMI_ERR_CAPACITY, "staging buffer still full");
    }
    // batched M, then one CSR per matrix
    std::vector<int64_t> nnzM_base(count + 1);
    for (int32_t b = 0; b <= count; ++b)
        cudaMemcpyAsync(&nnzM_base[b], rpM + row_base[b], 8, cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "nnz read");
    const int64_t nnzM = nnzM_base[count];
    int32_t *colM = S.get<int32_t>(nnzM);
    float *valM = S.get<float>(nnzM);
    BatchOut *d_out = S.get<BatchOut>(count);
    int64_t *d_nnzM_base = S.get<int64_t>(count + 1);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation (batched M)");
    e = launch_assemble(tn, rpM, a.row_off, a.row_cnt, a.st_col, a.st_val, colM, valM,
                        q.top_k > 0 ? (int64_t)q.top_k + 1 : 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "assembly");
    std::vector<BatchOut> out(count);
    std::vector<mcmi_matrix> made;
    auto undo = [&](mcmi_status st) {
        for (auto m : made) mcmi_free(m);
        for (int32_t b = 0; b < count; ++b) Ms[b] = nullptr;
        return st;
    };
    for (int32_t b = 0; b < count; ++b) {
        mcmi_matrix M = new mcmi_matrix_s();
        M->rows = Bs[b].n;
        M->row_begin = 0;
        M->n_cols = Bs[b].n;
        M->nnz = nnzM_base[b + 1] - nnzM_base[b];
        M->stream = s;
        cudaGetDevice(&M->device);
        M->rp = S.get<int64_t>(M->rows + 1);
        M->col = S.get<int32_t>(M->nnz);
        M->val = S.get<float>(M->nnz);
        made.push_back(M);
        if (S.err != cudaSuccess) return undo(cuda_fail(S.err, "allocation (outputs)"));
        S.keep(M->rp);
        S.keep(M->col);
        S.keep(M->val);
        out[b] = BatchOut{M->rp, M->col, M->val, M->rows, row_base[b], nnzM_base[b]};
    }
    cudaMemcpyAsync(d_out, out.data(), sizeof(BatchOut) * count, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_nnzM_base, nnzM_base.data(), 8 * (count + 1), cudaMemcpyHostToDevice, s);
    e = launch_split(d_out, count, d_row_base, d_nnzM_base, tn, nnzM, rpM, colM, valM, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return undo(cuda_fail(e, "batch split"));
    launches += 3;
    for (int32_t b = 0; b < count; ++b) Ms[b] = made[b];
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->steps = h.steps;
        stats->rows = tn;
        stats->nnz = nnzM;
        stats->max_s = P.smax;
        stats->chains = P.N;
        stats->max_len_bound = P.Lb;
        stats->table = P.table;
        stats->hash_log2 = W.log2H;
        stats->spilled = (int64_t)h.spilled;
        stats->deferred_rows = deferred;
        cudaEventElapsedTime(&stats->ms_prepare, ev[0], ev[1]);
        // the walk, timed by the event nodes inside the graph (else the whole graph)
        if (cudaEventElapsedTime(&stats->ms_walk_kernel, ev[4], ev[5]) != cudaSuccess) {
            cudaGetLastError();
            cudaEventElapsedTime(&stats->ms_walk_kernel, ev[2], ev[3]);
        }
        cudaEventElapsedTime(&stats->ms_walk, ev[2], ev[3]);
        stats->launches = launches;
        stats->threads = W.threads;
        stats->chains_per_thread = W.cpt;
        stats->load_depth = W.depth;
    }
    return MCMI_OK;
}

// A batch whose matrices differ in table type (AUTO choosing the compact
// table for some and not for others) is built as two batches, one per group,
// so that the stencil-like matrices keep their 32-byte records; the outputs
// keep the callers' order.
mcmi_status mcmi_build_batched(const mcmi_csr *Bs, int32_t count, const mcmi_params *p_in, void *stream,
                               mcmi_matrix *Ms, mcmi_stats *stats)
{
    if (!Bs || !Ms || count < 1 || !p_in) return batched_impl(Bs, count, p_in, stream, Ms, stats);
    const bool may_split = count > 1 && p_in->table == MCMI_TABLE_AUTO && p_in->accumulator == MCMI_ACC_FIXED64 &&
                           !p_in->proposal && !p_in->row_begin && !p_in->row_end;
    if (!may_split) return batched_impl(Bs, count, p_in, stream, Ms, stats);
    for (int32_t b = 0; b < count; ++b) {
        Ms[b] = nullptr;
        mcmi_status r = check_csr(&Bs[b]);
        if (r != MCMI_OK || Bs[b].n < 1) return batched_impl(Bs, count, p_in, stream, Ms, stats);   // reports it
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<unsigned long long> fit(2 * (size_t)count);
    {
        Scratch S(s);
        std::vector<BatchIn> in(count);
        for (int32_t b = 0; b < count; ++b) in[b] = BatchIn{Bs[b].row_ptr, Bs[b].col, Bs[b].val, Bs[b].n, Bs[b].nnz, 0, 0};
        BatchIn *d_in = S.get<BatchIn>(count);
        unsigned long long *d_fit = S.get<unsigned long long>(2 * (size_t)count);
        if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation (batch table check)");
        cudaError_t e = cudaMemcpyAsync(d_in, in.data(), sizeof(BatchIn) * count, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = launch_fit_stats(d_in, count, d_fit, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(fit.data(), d_fit, sizeof(unsigned long long) * 2 * count, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "batch table check");
    }
    std::vector<int32_t> grp[2];
    for (int32_t b = 0; b < count; ++b) {
        const bool fits = fit[2 * b] <= (unsigned long long)kCompactMaxDeg && fit[2 * b + 1] <= (unsigned long long)kCompactMaxOff;
        grp[fits ? 0 : 1].push_back(b);
    }
    if (grp[0].empty() || grp[1].empty()) return batched_impl(Bs, count, p_in, stream, Ms, stats);
    mcmi_stats st[2];
    int64_t rows[2] = {0, 0};
    for (int g = 0; g < 2; ++g) {
        std::vector<mcmi_csr> sub;
        for (int32_t b : grp[g]) {
            sub.push_back(Bs[b]);
            rows[g] += Bs[b].n;
        }
        std::vector<mcmi_matrix> out(sub.size(), nullptr);
        memset(&st[g], 0, sizeof(mcmi_stats));
        mcmi_status r = batched_impl(sub.data(), (int32_t)sub.size(), p_in, stream, out.data(), &st[g]);
        if (r != MCMI_OK) {
            for (int32_t b = 0; b < count; ++b) {
                if (Ms[b]) mcmi_free(Ms[b]);
                Ms[b] = nullptr;
            }
            return r;
        }
        for (size_t k = 0; k < out.size(); ++k) Ms[grp[g][k]] = out[k];
    }
    if (stats) {
        const mcmi_stats &big = rows[0] >= rows[1] ? st[0] : st[1];
        *stats = big;   // table, launch shape and chains of the group with more rows
        stats->steps = st[0].steps + st[1].steps;
        stats->rows = st[0].rows + st[1].rows;
        stats->nnz = st[0].nnz + st[1].nnz;
        stats->max_s = st[0].max_s > st[1].max_s ? st[0].max_s : st[1].max_s;
        stats->max_len_bound = st[0].max_len_bound > st[1].max_len_bound ? st[0].max_len_bound : st[1].max_len_bound;
        stats->spilled = st[0].spilled + st[1].spilled;
        stats->deferred_rows = st[0].deferred_rows + st[1].deferred_rows;
        stats->ms_prepare = st[0].ms_prepare + st[1].ms_prepare;
        stats->ms_walk = st[0].ms_walk + st[1].ms_walk;
        stats->ms_assemble = st[0].ms_assemble + st[1].ms_assemble;
        stats->ms_walk_kernel = st[0].ms_walk_kernel + st[1].ms_walk_kernel;
        stats->launches = st[0].launches + st[1].launches + 1;
    }
    return MCMI_OK;
}

mcmi_status mcmi_matrix_csr(mcmi_matrix M, int64_t *rows, int64_t *row_begin, int64_t *nnz,
                            const int64_t **row_ptr, const int32_t **col, const float **val)
{
    if (!M) return fail(MCMI_ERR_ARG, "M is NULL");
    if (rows) *rows = M->rows;
    if (row_begin) *row_begin = M->row_begin;
    if (nnz) *nnz = M->nnz;
    if (row_ptr) *row_ptr = M->rp;
    if (col) *col = M->col;
    if (val) *val = M->val;
    return MCMI_OK;
}

mcmi_status mcmi_matrix_copy(mcmi_matrix M, int64_t *row_ptr, int32_t *col, float *val, void *stream)
{
    if (!M) return fail(MCMI_ERR_ARG, "M is NULL");
    if (!row_ptr || (M->nnz > 0 && (!col || !val))) return fail(MCMI_ERR_ARG, "NULL output");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(row_ptr, M->rp, (M->rows + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && M->nnz > 0)
        e = cudaMemcpyAsync(col, M->col, M->nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && M->nnz > 0)
        e = cudaMemcpyAsync(val, M->val, M->nnz * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "matrix copy");
    return MCMI_OK;
}

mcmi_status mcmi_apply(mcmi_matrix M, const float *x, float *y, void *stream)
{
    if (!M) return fail(MCMI_ERR_ARG, "M is NULL");
    if (M->rows > 0 && (!x || !y)) return fail(MCMI_ERR_ARG, "NULL vector");
    if (M->rows == 0) return MCMI_OK;
    cudaError_t e = launch_spmv(M->rows, M->nnz, M->rp, M->col, M->val, x, y, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "apply");
    return MCMI_OK;
}

void mcmi_free(mcmi_matrix M)
{
    if (!M) return;
    if (M->rp) cudaFreeAsync(M->rp, M->stream);
    if (M->col) cudaFreeAsync(M->col, M->stream);
    if (M->val) cudaFreeAsync(M->val, M->stream);
    delete M;
}

mcmi_status mcmi_walk_dump(const mcmi_csr *B, const mcmi_params *p, const int64_t *rows, int64_t nrows,
                           int64_t cap, int32_t *out_count, uint64_t *out_steps, int32_t *out_col,
                           double *out_val, uint32_t *out_visits, void *stream)
{
    mcmi_status r = check_csr(B);
    if (r == MCMI_OK) r = check_params(p);
    if (r != MCMI_OK) return r;
    if (nrows < 0 || cap < 1) return fail(MCMI_ERR_ARG, "nrows < 0 or cap < 1");
    if (nrows == 0) return MCMI_OK;
    if (!rows || !out_count || !out_steps || !out_col || !out_val || !out_visits)
        return fail(MCMI_ERR_ARG, "NULL output");
    if (B->n == 0) return fail(MCMI_ERR_ARG, "rows listed for an empty matrix");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch S(s);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "memory pool");
    Prepared P;
    r = prepare(B, p, s, S, P, false);
    if (r != MCMI_OK) return r;
    WalkPlan W;
    r = plan_walk(p, P, nrows, true, W);
    if (r != MCMI_OK) return r;
    WalkArgs a;
    fill_walk_args(a, p, P, W);
    a.row_list = rows;
    a.n_list = nrows;
    a.row_begin = 0;
    a.row_end = B->n;
    a.out_by_row = 0;
    r = alloc_overflow(S, W, P, true, a);
    if (r != MCMI_OK) return r;
    a.d_count = out_count;
    a.d_col = out_col;
    a.d_val = out_val;
    a.d_vis = out_visits;
    a.d_cap = cap;
    a.row_steps = out_steps;
    reset_queue(P.st, s);
    cudaError_t e = launch_walk(a, p->precision, P.table, p->accumulator, true, W.cpt, W.depth, W.grid, W.threads, s);
    if (e != cudaSuccess) return cuda_fail(e, "walk kernel launch");
    DevState h;
    return read_state(P.st, &h, s);
}

mcmi_status mcmi_debug_tables(const mcmi_csr *B, const mcmi_params *p, double *out_d, double *out_s,
                              uint32_t *out_slot, uint32_t *out_a, uint32_t *out_b, uint32_t *out_c,
                              void *stream)
{
    mcmi_status r = check_csr(B);
    if (r == MCMI_OK) r = check_params(p);
    if (r != MCMI_OK) return r;
    if (B->n == 0) return MCMI_OK;
    if (!out_d || !out_s || !out_slot || !out_a || !out_b || !out_c) return fail(MCMI_ERR_ARG, "NULL output");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch S(s);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "memory pool");
    Prepared P;
    r = prepare(B, p, s, S, P, true);
    if (r != MCMI_OK) return r;
    const int64_t n = B->n, nnz = B->nnz;
    cudaMemcpyAsync(out_d, P.d, n * 8, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(out_s, P.s, n * 8, cudaMemcpyDeviceToDevice, s);
    // 64-byte records, or the compact table's 32-byte records packed at the start
    cudaMemcpyAsync(out_slot, P.slots, n * (P.table == MCMI_TABLE_COMPACT ? 32 : 64), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(out_a, P.a, nnz * 4, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(out_b, P.b, nnz * 4, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(out_c, P.c, nnz * 4, cudaMemcpyDeviceToDevice, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "table export");
    return MCMI_OK;
}

// ---------------------------------------------------------------- learned proposal

mcmi_status mcmi_proposal_create(const float *params, mcmi_proposal *out)
{
    if (!out) return fail(MCMI_ERR_ARG, "out is NULL");
    *out = nullptr;
    mcmi_proposal P = new mcmi_proposal_s();
    if (params) {
        memcpy(P->h_params, params, sizeof(P->h_params));
    } else {
        // Glorot-uniform weights from a fixed split-mix sequence, zero biases:
        // g starts near 1 (the |c| proposal)
        uint64_t x = 0x9E3779B97F4A7C15ull;
        auto next = [&]() {
            x += 0x9E3779B97F4A7C15ull;
            uint64_t z = x;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            return (double)((z ^ (z >> 31)) >> 11) * 0x1.0p-53;
        };
        memset(P->h_params, 0, sizeof(P->h_params));
        const int lay[3][3] = {{0, 8, 32}, {288, 32, 32}, {1344, 32, 1}};   // offset, fan-in, fan-out
        for (auto &L : lay) {
            const double a = std::sqrt(6.0 / (L[1] + L[2]));
            for (int i = 0; i < L[1] * L[2]; ++i) P->h_params[L[0] + i] = (float)((2.0 * next() - 1.0) * a);
        }
    }
    cudaGetDevice(&P->device);
    cudaError_t e = cudaMalloc(&P->d_params, kMlpParams * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(P->d_params, P->h_params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (P->d_params) cudaFree(P->d_params);
        delete P;
        return cuda_fail(e, "proposal parameters");
    }
    *out = P;
    return MCMI_OK;
}

mcmi_status mcmi_proposal_get(mcmi_proposal P, float *params)
{
    if (!P || !params) return fail(MCMI_ERR_ARG, "NULL argument");
    cudaError_t e = cudaMemcpy(P->h_params, P->d_params, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "proposal parameters");
    memcpy(params, P->h_params, sizeof(P->h_params));
    return MCMI_OK;
}

void mcmi_proposal_free(mcmi_proposal P)
{
    if (!P) return;
    if (P->d_params) cudaFree(P->d_params);
    delete P;
}

mcmi_status mcmi_row_moments(const mcmi_csr *B, const mcmi_params *p, float *m, void *stream)
{
    mcmi_status r = check_csr(B);
    if (r == MCMI_OK) r = check_params(p);
    if (r != MCMI_OK) return r;
    if (!m) return fail(MCMI_ERR_ARG, "m is NULL");
    if (B->n == 0) return MCMI_OK;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch S(s);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "memory pool");
    Prepared P;
    r = prepare(B, p, s, S, P, false);
    if (r != MCMI_OK) return r;
    WalkPlan W;
    WalkArgs a;
    fill_walk_args(a, p, P, W);
    cudaMemsetAsync(m, 0, B->n * sizeof(float), s);
    cudaError_t e = launch_row_moments(a, P.table, B->n, m, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "row moments");
    return MCMI_OK;
}

namespace {

// training edges of one matrix appended at edge_base / row_base
mcmi_status train_edges_of(const mcmi_csr *B, const mcmi_params *p, const float *m_rows, int64_t row_base,
                           int64_t edge_base, float *feat, float *pe, float *mt, int32_t *rid, cudaStream_t s)
{
    Scratch S(s);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "memory pool");
    DevState *st = S.get<DevState>(1);
    double *d = S.get<double>(B->n), *sv = S.get<double>(B->n);
    int *deg = S.get<int>(B->n);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation");
    cudaMemsetAsync(st, 0, sizeof(DevState), s);
    cudaMemsetAsync(&st->err, 0xFF, 8, s);
    launch_validate(B->n, B->nnz, B->row_ptr, B->col, B->val, st, s);
    if (p->alpha > 0.0) launch_rownorm(B->n, B->row_ptr, B->val, st, s);
    launch_split(B->n, B->row_ptr, B->col, B->val, p->alpha, d, sv, st, s);
    DevState h;
    mcmi_status r = read_state(st, &h, s);
    if (r != MCMI_OK) return r;
    launch_degree(B->n, B->row_ptr, B->col, deg, s);
    cudaError_t e = launch_train_edges(B->n, B->row_ptr, B->col, B->val, d, sv, deg, m_rows, row_base, edge_base, feat,
                                       pe, mt, rid, s);
    if (e != cudaSuccess) return cuda_fail(e, "training edges");
    return MCMI_OK;
}

}  // namespace

mcmi_status mcmi_proposal_loss_grad(const mcmi_csr *B, const float *m_rows, const mcmi_params *p, mcmi_proposal P,
                                    int round_bf16, float *loss, float *grad, void *stream)
{
    mcmi_status r = check_csr(B);
    if (r == MCMI_OK) r = check_params(p);
    if (r != MCMI_OK) return r;
    if (!P || !m_rows || !loss || B->n == 0) return fail(MCMI_ERR_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch S(s);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "memory pool");
    const int64_t E = B->nnz, R = B->n;
    float *feat = S.get<float>(E * 8), *pe = S.get<float>(E), *mt = S.get<float>(E);
    int32_t *rid = S.get<int32_t>(E);
    float *A = S.get<float>(R), *Bs = S.get<float>(R), *Cs = S.get<float>(R), *lb = S.get<float>(2);
    float *g = grad ? S.get<float>(kMlpParams) : nullptr;
    if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation");
    r = train_edges_of(B, p, m_rows, 0, 0, feat, pe, mt, rid, s);
    if (r != MCMI_OK) return r;
    cudaError_t e = train_pass(E, R, feat, pe, mt, rid, P->d_params, A, Bs, Cs, lb, g, true, round_bf16, s);
    float h[2] = {0.0f, 0.0f};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, lb, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, g, kMlpParams * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "training pass");
    *loss = h[1] > 0.0f ? h[0] / h[1] : 0.0f;
    return MCMI_OK;
}

mcmi_status mcmi_proposal_train(const mcmi_csr *Bs, int32_t count, const mcmi_train_params *tp, mcmi_proposal P,
                                float *loss_history, void *stream)
{
    if (!Bs || count < 1 || !tp || !P || tp->steps < 0 || !(tp->lr > 0.0f) || tp->chains < 1)
        return fail(MCMI_ERR_ARG, "bad training argument");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch S(s);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "memory pool");
    int64_t E = 0, R = 0;
    for (int32_t b = 0; b < count; ++b) {
        mcmi_status r = check_csr(&Bs[b]);
        if (r != MCMI_OK) return r;
        E += Bs[b].nnz;
        R += Bs[b].n;
    }
    float *feat = S.get<float>(E * 8), *pe = S.get<float>(E), *mt = S.get<float>(E);
    int32_t *rid = S.get<int32_t>(E);
    float *A = S.get<float>(R), *Bv = S.get<float>(R), *Cs = S.get<float>(R), *lb = S.get<float>(2);
    float *g = S.get<float>(kMlpParams), *m1 = S.get<float>(kMlpParams), *m2 = S.get<float>(kMlpParams);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation (training set)");
    // training signal: second moments of the |c|-proposal walks of every row
    mcmi_params wp;
    mcmi_params_default(&wp);
    wp.chains = tp->chains;
    wp.max_len = tp->max_len;
    wp.delta = tp->delta;
    wp.alpha = tp->alpha;
    wp.seed = tp->seed;
    int64_t eb = 0, rb = 0;
    for (int32_t b = 0; b < count; ++b) {
        Scratch T(s);
        float *mrow = T.get<float>(Bs[b].n);
        if (T.err != cudaSuccess) return cuda_fail(T.err, "allocation");
        mcmi_status r = mcmi_row_moments(&Bs[b], &wp, mrow, stream);
        if (r == MCMI_OK) r = train_edges_of(&Bs[b], &wp, mrow, rb, eb, feat, pe, mt, rid, s);
        if (r != MCMI_OK) return fail(r, "training matrix %d: %s", b, g_err.c_str());
        eb += Bs[b].nnz;
        rb += Bs[b].n;
    }
    cudaMemsetAsync(m1, 0, kMlpParams * 4, s);
    cudaMemsetAsync(m2, 0, kMlpParams * 4, s);
    const int rnd = tp->round_bf16;
    for (int32_t it = 0; it < tp->steps; ++it) {
        cudaError_t e = train_pass(E, R, feat, pe, mt, rid, P->d_params, A, Bv, Cs, lb, g, it == 0, rnd, s);
        if (e == cudaSuccess) e = launch_adam(P->d_params, g, m1, m2, tp->lr, it + 1, s);
        if (e != cudaSuccess) return cuda_fail(e, "training step");
        if (loss_history) {
            float h[2];
            e = cudaMemcpyAsync(h, lb, 8, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "training loss");
            loss_history[it] = h[1] > 0.0f ? h[0] / h[1] : 0.0f;
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(P->h_params, P->d_params, kMlpParams * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "training");
    return MCMI_OK;
}

mcmi_status mcmi_recover_dense(const mcmi_csr *B, double alpha, double *X, void *stream)
{
    mcmi_status r = check_csr(B);
    if (r != MCMI_OK) return r;
    if (!X && B->n > 0) return fail(MCMI_ERR_ARG, "X is NULL");
    if (!(alpha >= 0.0)) return fail(MCMI_ERR_ARG, "alpha must be >= 0");
    if (B->n > 16384) return fail(MCMI_ERR_ARG, "the dense recovery is a diagnostic for n <= 16384");
    const int64_t n = B->n;
    if (n == 0) return MCMI_OK;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch S(s);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "memory pool");
    DevState *st = S.get<DevState>(1);
    double *d = S.get<double>(n), *sv = S.get<double>(n), *sd = S.get<double>(n);
    double *c = S.get<double>(n), *rr = S.get<double>(n), *gs = S.get<double>(1);
    int *flag = S.get<int>(1);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation (recovery)");
    cudaMemsetAsync(st, 0, sizeof(DevState), s);
    cudaMemsetAsync(&st->err, 0xFF, sizeof(unsigned long long), s);
    cudaMemsetAsync(&st->smin_bits, 0xFF, sizeof(unsigned long long), s);
    cudaMemsetAsync(flag, 0, sizeof(int), s);
    launch_validate(n, B->nnz, B->row_ptr, B->col, B->val, st, s);
    DevState h;
    r = read_state(st, &h, s);
    if (r != MCMI_OK) return r;
    if (alpha > 0.0) launch_rownorm(n, B->row_ptr, B->val, st, s);
    launch_split(n, B->row_ptr, B->col, B->val, alpha, d, sv, st, s);
    cudaError_t e = cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "device state read");
    // the recovery needs Bhat, not a contractive split: only other errors count
    if (h.err != ~0ull && (int)(h.err & 0xFF) != MCMI_ERR_NOT_CONTRACTIVE) return read_state(st, &h, s);
    e = launch_aug_diag(n, B->row_ptr, B->col, B->val, d, sd, s);
    std::vector<double> sh((size_t)n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sh.data(), sd, n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "recovery set-up");
    for (int64_t i = n - 1; i >= 0 && e == cudaSuccess; --i)
        if (sh[(size_t)i] != 0.0) e = launch_sm_step(n, X, i, sd, c, rr, gs, flag, s);
    int hf = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "recovery");
    if (hf) return fail(MCMI_ERR_ARG, "zero denominator 1 - s_i X_ii in the recovery (Eq. 3)");
    return MCMI_OK;
}

mcmi_status mcmi_matrix_dense(mcmi_matrix M, double *X, void *stream)
{
    if (!M || (!X && M->rows > 0)) return fail(MCMI_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(X, 0, (size_t)M->rows * (size_t)M->n_cols * sizeof(double), s);
    if (e == cudaSuccess) e = launch_csr_dense(M->rows, M->n_cols, M->rp, M->col, M->val, X, s);
    if (e != cudaSuccess) return cuda_fail(e, "dense copy of M");
    return MCMI_OK;
}

mcmi_status mcmi_reduce(const mcmi_csr *B, double fraction, int32_t mode, void *stream, mcmi_reduced *R_out,
                        int64_t *dropped)
{
    if (!R_out) return fail(MCMI_ERR_ARG, "R is NULL");
    *R_out = nullptr;
    mcmi_status r = check_csr(B);
    if (r != MCMI_OK) return r;
    if (!(fraction >= 0.0 && fraction <= 1.0)) return fail(MCMI_ERR_ARG, "fraction must be in [0, 1]");
    if (mode != MCMI_REDUCE_ENTRIES && mode != MCMI_REDUCE_RANGE) return fail(MCMI_ERR_ARG, "unknown reduction mode");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch S(s);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "memory pool");
    const int64_t n = B->n;
    unsigned long long *stats = S.get<unsigned long long>(3);
    unsigned int *hist = S.get<unsigned int>(256);
    int32_t *kc = S.get<int32_t>(n);
    int64_t *rp2 = S.get<int64_t>(n + 1);
    int64_t *tmp = S.get<int64_t>(scan_tmp_elems(n));
    if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation (reduction)");
    // off-diagonal count and |b| range
    unsigned long long hs[3] = {0ull, ~0ull, 0ull};
    cudaMemcpyAsync(stats, hs, sizeof(hs), cudaMemcpyHostToDevice, s);
    cudaError_t e = launch_offstats(n, B->row_ptr, B->col, B->val, stats, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "reduction statistics");
    const int64_t noff = (int64_t)hs[0];
    const int rmode = mode;
    double thr = 0.0;
    unsigned long long T = 0ull;
    long long need = 0;
    int64_t *eq_off = nullptr;
    if (mode == MCMI_REDUCE_RANGE) {
        double lo = 0.0, hi = 0.0;
        const unsigned long long lob = hs[1], hib = hs[2];
        memcpy(&lo, &lob, 8);
        memcpy(&hi, &hib, 8);
        thr = noff > 0 ? lo + fraction * (hi - lo) : 0.0;   // FP64, this order (no contraction)
    } else {
        const int64_t kdrop = (int64_t)std::floor(fraction * (double)noff);
        if (kdrop > 0) {   // (kdrop == 0: T = 0 and need = 0 drop nothing)
            // radix select of the kdrop-th smallest key (8 bits per pass, from the top)
            unsigned long long prefix = 0ull, mask = 0ull;
            long long rank = kdrop;   // 1-based rank inside the current prefix group
            unsigned int h[256];
            for (int shift = 56; shift >= 0; shift -= 8) {
                cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned int), s);
                e = launch_abs_hist(n, B->row_ptr, B->col, B->val, prefix, mask, shift, hist, s);
                if (e == cudaSuccess) e = cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) return cuda_fail(e, "reduction select");
                long long cum = 0;
                int digit = 255;
                for (int d = 0; d < 256; ++d) {
                    if (cum + (long long)h[d] >= rank) {
                        digit = d;
                        break;
                    }
                    cum += h[d];
                }
                rank -= cum;
                prefix |= (unsigned long long)digit << shift;
                mask |= 255ull << shift;
            }
            T = prefix;     // key of the kdrop-th smallest entry
            need = rank;    // entries equal to T that are dropped (the first ones in CSR order)
            int32_t *eqc = S.get<int32_t>(n);
            eq_off = S.get<int64_t>(n + 1);
            if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation (reduction ranks)");
            e = launch_eq_count(n, B->row_ptr, B->col, B->val, T, eqc, s);
            if (e == cudaSuccess) e = scan_counts(eqc, n, eq_off, tmp, s);
            if (e != cudaSuccess) return cuda_fail(e, "reduction ranks");
        }
    }
    e = launch_keep(n, B->row_ptr, B->col, B->val, rmode, thr, T, need, eq_off, kc, nullptr, nullptr, nullptr, s);
    if (e == cudaSuccess) e = scan_counts(kc, n, rp2, tmp, s);
    int64_t nnz2 = 0;
    if (e == cudaSuccess && n > 0) e = cudaMemcpyAsync(&nnz2, rp2 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "reduction counts");
    int32_t *col2 = S.get<int32_t>(nnz2);
    double *val2 = S.get<double>(nnz2);
    if (S.err != cudaSuccess) return cuda_fail(S.err, "allocation (reduced matrix)");
    e = launch_keep(n, B->row_ptr, B->col, B->val, rmode, thr, T, need, eq_off, nullptr, rp2, col2, val2, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "reduction compaction");
    mcmi_reduced R = new mcmi_reduced_s();
    R->n = n;
    R->nnz = nnz2;
    R->rp = rp2;
    R->col = col2;
    R->val = val2;
    R->stream = s;
    S.keep(rp2);
    S.keep(col2);
    S.keep(val2);
    if (n == 0) cudaMemsetAsync(rp2, 0, sizeof(int64_t), s);
    if (dropped) *dropped = B->nnz - nnz2;
    *R_out = R;
    return MCMI_OK;
}

mcmi_status mcmi_reduced_csr(mcmi_reduced R, mcmi_csr *view)
{
    if (!R || !view) return fail(MCMI_ERR_ARG, "NULL argument");
    view->n = R->n;
    view->nnz = R->nnz;
    view->row_ptr = R->rp;
    view->col = R->col;
    view->val = R->val;
    return MCMI_OK;
}

mcmi_status mcmi_reduced_copy(mcmi_reduced R, int64_t *row_ptr, int32_t *col, double *val, void *stream)
{
    if (!R || !row_ptr || ((!col || !val) && R->nnz > 0)) return fail(MCMI_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(row_ptr, R->rp, (R->n + 1) * sizeof(int64_t), cudaMemcpyDefault, s);
    if (e == cudaSuccess && R->nnz > 0) e = cudaMemcpyAsync(col, R->col, R->nnz * sizeof(int32_t), cudaMemcpyDefault, s);
    if (e == cudaSuccess && R->nnz > 0) e = cudaMemcpyAsync(val, R->val, R->nnz * sizeof(double), cudaMemcpyDefault, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy of the reduced matrix");
    return MCMI_OK;
}

void mcmi_reduced_free(mcmi_reduced R)
{
    if (!R) return;
    if (R->rp) cudaFreeAsync(R->rp, R->stream);
    if (R->col) cudaFreeAsync(R->col, R->stream);
    if (R->val) cudaFreeAsync(R->val, R->stream);
    delete R;
}

}  // extern "C"
