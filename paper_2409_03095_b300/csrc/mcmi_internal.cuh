// Internal definitions shared by the kernels of libmcmi (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mcmi.h"

// Learned proposal: the network's parameters on the device (and a host copy).
struct mcmi_proposal_s {
    float *d_params = nullptr;
    float h_params[1377];
    int device = 0;
};

namespace mcmi {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;      // empty accumulator key
constexpr uint32_t kOolFlag = 0x80000000u;    // slot word 3: table stored out of line
constexpr uint32_t kCumFlag = 0x40000000u;    // slot word 3: hybrid table, this row is cumulative (inline)
constexpr uint32_t kNegBit = 0x80000000u;     // record: sign of c_ij
constexpr int kInlineCum = 6;                 // cumulative pairs that fit a 64-byte slot
constexpr int kInlineAlias = 4;               // alias triples that fit a 64-byte slot
constexpr int kMlpParams = 1377;              // learned proposal: 8-32-32-1 network parameters
// Compact table: one 32-byte record per row (at most six transitions, each
// column within kCompactMaxOff of the row), weights at the scale 2^20.
//   word 0:    fl32(s_i)
//   words 1-2: Q | T_1 << 21 | T_2 << 42 (a 64-bit word of 21-bit fields)
//   words 3-4: T_3 | T_4 << 21 | T_5 << 42 (unused thresholds hold Q)
//   words 5-7: six 16-bit fields (col - i) << 1 | sign(c_ij), two per word
constexpr int kCompactMaxDeg = 6;
constexpr int kCompactMaxOff = 16383;
constexpr uint32_t kField21 = 0x1FFFFFu;

// Device-side counters and the first error of a launch sequence.
struct DevState {
    unsigned long long err;        // min over (row << 8 | code); ~0 = no error
    unsigned long long smax_bits;  // bits of max_i s_i (s_i >= 0, so integer order = float order)
    unsigned long long smin_bits;  // bits of min over s_i > 0 (~0 if none)
    unsigned long long bnorm_bits; // bits of ||B||_inf
    unsigned long long steps;      // transitions taken
    unsigned long long spilled;    // distinct columns reduced from the overflow log
    unsigned long long cursor;     // staging entries claimed
    unsigned long long deferred;   // rows that found the staging buffer full
    unsigned long long work;       // next row-queue position
    unsigned long long ndiag;      // rows that have a stored diagonal
    unsigned long long max_deg;    // largest off-diagonal count of a row
    unsigned long long max_off;    // largest |j - i| of an off-diagonal entry
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
    const uint4 *slots;           // 4 x uint4 per row (compact table: 2 x uint4)
    const float *invd32;          // compact table: fl32(1/d_i) per row
    const uint32_t *ool_a, *ool_b;    // cumulative out-of-line: thresholds, col|sign
    const uint4 *ool_bkt;             // alias out-of-line buckets {prob, own, alias, 0}
    const uint4 *lbkt;                // learned proposal: 32-byte alias buckets with weight factors
    float w_limit;                    // learned proposal: largest |W| the fixed-point sums can take
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
    float fin_scale;              // 2^-F / N in FP32 (finished values of FP32 builds)
    uint32_t key0, key1;
    int log2H;                    // on-chip slots per block
    // visits that find the on-chip table full go to a per-block log (column,
    // addend); after the walks the log is reduced on chip, in hash-range
    // passes, into a per-block list of the row's distinct entries
    uint2 *log_key;               // {column, FP32 bits of its 1/d_j}; sketch kernels: {column, FP32 bits of W}
    unsigned long long *log_val;
    uint32_t log_cap;             // log entries per block (>= the visits of one row)
    uint32_t *ent_col;
    unsigned long long *ent_val;  // finished values M_ij (FP64 bits, or FP32 bits in the low word)
    uint32_t *ent_cnt;            // parity dump: visit counts
    uint32_t *cells;              // walk-time magnitude sketch: walk_sketch_cells() words per block, zero
                                  // at launch (each block clears its cells after a row that used them)
    int sk_code_bits;             // sketch kernels: 9..12 = the top bits of a log entry's column word hold
                                  // a rounded-up code of |1/d_j| and the sketch is built after the walks
                                  // in shared memory (cells unused); 0 = walk-time sketch in cells
    uint32_t ent_cap;             // entries per block (>= log_cap + on-chip slots)
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

// Total weight Q of a row's record (0: no transition, the chain stops).
template <int TABLE>
__device__ __forceinline__ uint32_t record_q(const uint32_t (&s)[16])
{
    return TABLE == MCMI_TABLE_COMPACT ? (s[1] & kField21) : s[0];
}

// One transition out of the row whose 64-byte record is s[16], driven by the
// 32-bit random word r.  Returns col | neg << 31 of the picked entry and the
// FP32 weight factor in *f: sign(c) fl32(s_i) for the |c| proposal, the
// stored fl32(c Q / q) for a learned one.
//   cumulative: x = floor(r Q / 2^32), the smallest m with x < T_m (inline
//               pairs, or a binary search out of line);
//   alias:      bucket b = floor(r deg / 2^32), the low 32 bits of r deg
//               scaled to [0, Q) against the bucket's threshold;
//   hybrid:     the alias kernels; rows flagged kCumFlag (at most 6
//               transitions) hold an inline cumulative record;
//   compact:    the cumulative rule on the 32-byte record (row: its index,
//               for the column offsets).
template <int TABLE>
__device__ __forceinline__ uint32_t pick_transition(const uint32_t (&s)[16], uint32_t r, const WalkArgs &a,
                                                    float *f, uint32_t row = 0u)
{
    if (TABLE == MCMI_TABLE_COMPACT) {
        const unsigned long long A = (unsigned long long)s[1] | ((unsigned long long)s[2] << 32);
        const unsigned long long Bt = (unsigned long long)s[3] | ((unsigned long long)s[4] << 32);
        const uint32_t Qc = (uint32_t)A & kField21;
        const uint32_t x = __umulhi(r, Qc);
        const uint32_t m = (((uint32_t)(A >> 21) & kField21) <= x) + ((uint32_t)(A >> 42) <= x) +
                           (((uint32_t)Bt & kField21) <= x) + (((uint32_t)(Bt >> 21) & kField21) <= x) +
                           ((uint32_t)(Bt >> 42) <= x);
        const uint32_t pair = m < 2u ? s[5] : (m < 4u ? s[6] : s[7]);
        const uint32_t h = (m & 1u) ? (pair >> 16) : (pair & 0xFFFFu);
        const int off = (int)(int16_t)(uint16_t)h >> 1;
        const uint32_t cs = (uint32_t)((int)row + off) | ((h & 1u) ? kNegBit : 0u);
        const float fs = __uint_as_float(s[0]);
        *f = (h & 1u) ? -fs : fs;
        return cs;
    }
    const uint32_t Q = s[0];
    const uint32_t deg = s[3] & ~(kOolFlag | kCumFlag);
    uint32_t cs;
    if (TABLE == MCMI_TABLE_CUMULATIVE || (s[3] & kCumFlag)) {
        const uint32_t x = __umulhi(r, Q);
        if (!(s[3] & kOolFlag)) {
            const uint32_t m = (s[4] <= x) + (s[6] <= x) + (s[8] <= x) + (s[10] <= x) + (s[12] <= x) + (s[14] <= x);
            cs = m == 0 ? s[5] : m == 1 ? s[7] : m == 2 ? s[9] : m == 3 ? s[11] : m == 4 ? s[13] : s[15];
        } else {
            const uint32_t *T = a.ool_a + s[4];
            uint32_t lo = 0, hi = deg - 1;
#pragma unroll 1
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (x < __ldg(T + mid)) hi = mid; else lo = mid + 1;
            }
            cs = __ldg(a.ool_b + s[4] + lo);
        }
    } else {
        const unsigned long long pr = (unsigned long long)r * deg;
        const uint32_t b = (uint32_t)(pr >> 32);
        const uint32_t y = __umulhi((uint32_t)pr, Q);
        uint32_t prob, own, al;
        if (!(s[3] & kOolFlag)) {
            prob = b == 0 ? s[4] : b == 1 ? s[7] : b == 2 ? s[10] : s[13];
            own = b == 0 ? s[5] : b == 1 ? s[8] : b == 2 ? s[11] : s[14];
            al = b == 0 ? s[6] : b == 1 ? s[9] : b == 2 ? s[12] : s[15];
        } else if (a.lbkt) {
            // learned bucket: {prob, own, alias, f_own, f_alias, 0, 0, 0}
            uint32_t v[8];
            asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7])
                         : "l"(a.lbkt + 2 * ((size_t)s[4] + b)));
            const bool own_pick = y < v[0];
            *f = __uint_as_float(own_pick ? v[3] : v[4]);
            return own_pick ? v[1] : v[2];
        } else {
            const uint4 bk = __ldg(a.ool_bkt + s[4] + b);
            prob = bk.x; own = bk.y; al = bk.z;
        }
        cs = y < prob ? own : al;
    }
    const float fs = __uint_as_float(s[1]);
    *f = (cs & kNegBit) ? -fs : fs;
    return cs;
}

}  // namespace mcmi
