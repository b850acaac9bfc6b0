// Internal definitions shared by the kernels of libmcmi (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mcmi.h"

namespace mcmi {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;      // empty accumulator key
constexpr uint32_t kOolFlag = 0x80000000u;    // slot word 3: table stored out of line
constexpr uint32_t kNegBit = 0x80000000u;     // record: sign of c_ij
constexpr int kInlineCum = 6;                 // cumulative pairs that fit a 64-byte slot
constexpr int kInlineAlias = 4;               // alias triples that fit a 64-byte slot
constexpr int kWalkThreadsMax = 128;          // walk kernel: threads per block (two chains each)
constexpr int kWalkMinBlocks = 6;             // resident blocks per SM the register budget targets

// Device-side counters and the first error of a launch sequence.
struct DevState {
    unsigned long long err;        // min over (row << 8 | code); ~0 = no error
    unsigned long long smax_bits;  // bits of max_i s_i (s_i >= 0, so integer order = float order)
    unsigned long long smin_bits;  // bits of min over s_i > 0 (~0 if none)
    unsigned long long bnorm_bits; // bits of ||B||_inf
    unsigned long long steps;      // transitions taken
    unsigned long long spilled;    // entries placed in the global overflow table
    unsigned long long cursor;     // staging entries claimed
    unsigned long long deferred;   // rows that found the staging buffer full
    unsigned long long work;       // next row-queue position
    unsigned long long ndiag;      // rows that have a stored diagonal
};

__device__ __forceinline__ void report(DevState *st, long long row, int code)
{
    atomicMin(&st->err, ((unsigned long long)row << 8) | (unsigned long long)code);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit products on counter words 0 and 2, word permutation, key
// xor; key bumped by the Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Arguments of the walk kernel.
struct WalkArgs {
    const uint4 *slots;           // 4 x uint4 per row
    const uint32_t *ool_a, *ool_b;    // cumulative out-of-line: thresholds, col|sign
    const uint4 *ool_bkt;             // alias out-of-line buckets {prob, own, alias, 0}
    const double2 *rowd;          // FP64 path: {s_i, 1/d_i}
    int64_t row_begin, row_end;   // rows when row_list == nullptr
    const int64_t *row_list;      // explicit rows (global indices)
    int64_t n_list;
    int out_by_row;               // list mode: outputs indexed by row - row_begin
    int count_steps;              // add the rows' transitions to the device counter
    const int64_t *batch_row_base; // block-diagonal batch: first row of each matrix (nullptr: one matrix)
    int batch_count;
    int32_t N, L;
    float delta_f;                // smallest float >= delta
    int fix_shift;                // fixed-point accumulator scale: weight w is added as round(w 2^F)
    double fix_inv;               // 2^-F
    uint32_t key0, key1;
    int log2H;                    // on-chip slots per block
    // global overflow accumulator, one region per block
    uint32_t *g_keys;
    unsigned long long *g_vals;
    uint32_t *g_cnt;
    uint32_t *g_list;
    int log2G;
    // filter
    double tau;
    int32_t top_k;
    // production output: staging + per-row offsets
    uint32_t *st_col;
    float *st_val;
    unsigned long long st_cap;
    int64_t *row_off;
    int32_t *row_cnt;
    int64_t *deferred_list;
    uint64_t *row_steps;          // optional per-row transitions
    // parity dump
    int32_t *d_count;
    int32_t *d_col;
    double *d_val;
    uint32_t *d_vis;
    int64_t d_cap;
    DevState *st;
};

}  // namespace mcmi
