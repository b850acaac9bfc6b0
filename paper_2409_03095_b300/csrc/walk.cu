// Stages a3-a5 of the hot path in one kernel: the random walks of Eq. 2,
// the row accumulator (on-chip hash + overflow log), the phase-4 column
// scaling by 1/d_j and the Sec. IV-B filter, writing each row's kept entries
// to a staging buffer.
//
// One block per row at a time (rows taken from a device queue), threads as
// chains: a thread that finishes a chain takes the next chain index of the
// row, so live chains stay packed into the block's warps.
//
// Accumulators (per visited column of the row being built):
//  ACC_FIXED64 (default): the exact sum of the walk weights as a 64-bit
//    fixed-point integer (scale 2^F chosen on the host so that N (L+1)
//    weights of magnitude < 1 cannot overflow), added with two native 32-bit
//    integer atomics (low word with return, carry into the high word).  The
//    sum is independent of the order of the additions, so it is
//    deterministic; 1/d_j is applied once per entry at the end.
//  ACC_KAHAN32: FP32 sums of W/d_j with a compensation word; the rounding
//    error of each addition is computed exactly from the returned previous
//    sum (Knuth's TwoSum) and added to the compensation.
//
// Rows that reach more columns than the on-chip table holds (random sparse
// matrices: nearly every visit after the first steps is a new column) append
// the visits that find the table full to a per-block log in global memory:
// one store, off the chain's dependent path.  After the walks, log entries of
// columns on chip are added there; if any remain, the on-chip entries are
// moved to a per-block entry list and the rest of the log is reduced on chip
// in passes over disjoint hash ranges of the column index (a pass whose
// columns do not fit is retried on half its range), each pass appending its
// finished entries to the list.
#include <type_traits>

#include "mcmi_internal.cuh"
#include "kernels.h"


namespace mcmi {

namespace {

constexpr int kProbeOnChip = 32;   // on-chip probe window before overflowing
constexpr uint32_t kPartMul = 0x85EBCA77u;   // odd: col -> col * kPartMul permutes the 32-bit keys
constexpr uint32_t kSketchMul = 0xC2B2AE35u;  // odd: cell of a column in the log's magnitude sketch
// Magnitude sketch of the overflow log (the FP32 fixed-point production
// kernel at load depth 8): every logged visit adds its magnitude
// |W| |1/d_j| to one cell (hash of the column), in units of
// |1/d_i| 2^-kCellUnitLog2 of the row i; a visit of 2^31 / (log capacity)
// units or more sets the cell's top bit instead (the cell is then always
// kept), so that the sums of a row's visits stay below 2^31.  Either after
// the walks, from a code of |1/d_j| in the log entries' column words, into
// 2^kCellsCodeLog2 cells in the emptied table; or (columns too wide for the
// code) during the walks into kCells cells of a per-block array in global
// memory, updated by L2 atomics, so that the shared memory left to the L1
// cache is unchanged.
// A presence map of kPresBits bits (hash of the column) holds a superset of
// the columns on chip; once the table is at its cap, a visit whose bit is
// clear goes straight to the log without probing the table.
constexpr int kCellsLog2 = 10;
constexpr int kCells = 1 << kCellsLog2;
// cells of the sketch built after the walks (in the emptied table's value
// words, 2H of them at most): clearing shared cells costs little, so it
// takes more than the global cells' 1024
constexpr int kCellsCodeLog2 = 12;
constexpr int kCellUnitLog2 = 14;
constexpr uint32_t kCellFlag = 0x80000000u;
constexpr int kPresLog2 = 14;                 // 16384 bits in 512 words
constexpr uint32_t kPresMul = 0xCC9E2D51u;    // odd: bit of a column in the presence map

__device__ __forceinline__ uint32_t hash_home(uint32_t key, int log2)
{
    return (key * 0x9E3779B1u) >> (32 - log2);
}

// Log entries of the sketch kernels with cb code bits (9..12): the column
// in the low 32 - cb bits; in the top cb bits, bits 30 .. 31 - cb of the
// FP32 pattern of |1/d_j| rounded up, at most 2^cb - 2, so that the decoded
// value is >= |1/d_j| (infinite or NaN at the top codes) and a packed word
// never equals the empty key 0xFFFFFFFF.
__device__ __forceinline__ uint32_t sketch_pack(uint32_t col, float invd, int cb)
{
    const uint32_t sh = 31u - (uint32_t)cb;
    const uint32_t b = __float_as_uint(invd) & 0x7FFFFFFFu;
    const uint32_t code = min((b >> sh) + ((b & ((1u << sh) - 1u)) != 0u), (1u << cb) - 2u);
    return col | (code << (sh + 1u));
}

__device__ __forceinline__ float sketch_decode(uint32_t word, int cb)
{
    return __uint_as_float((word >> (32 - cb)) << (31 - cb));
}

// w * 2^F (scale = 2^F as a float) rounded to the nearest integer, ties to
// even, by one float-to-integer conversion: the product is exact, and for
// FP32 walks with the |c| proposal F makes it an integer (every weight is a
// multiple of 2^-F), so the result is exact too.  (A learned proposal's F
// leaves head-room instead; its products may round.)
__device__ __forceinline__ long long fix_f32s(float w, float scale)
{
    return __float2ll_rn(__fmul_rn(w, scale));
}

// w * 2^F rounded to the nearest integer for an FP64 w (|w| < 1), with
// integer instructions (FP64 arithmetic issues at a small fraction of the
// FP32 rate).
__device__ __forceinline__ long long fix_f64(double w, int F)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(w);
    const int e = (int)((b >> 52) & 0x7FFull);
    if (e == 0) return 0;
    const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
    const int s = e - 1075 + F;
    long long v;
    if (s >= 0) v = m << s;
    else if (s > -63) v = (m + (1ll << (-s - 1))) >> (-s);
    else v = 0;
    return (b >> 63) ? -v : v;
}

// Exact 64-bit add into a shared word from two native 32-bit atomics.
__device__ __forceinline__ void fix_add_shared(uint32_t *lo_w, uint32_t *hi_w, long long v)
{
    const uint32_t lo = (uint32_t)v, hi = (uint32_t)((unsigned long long)v >> 32);
    const uint32_t old = atomicAdd(lo_w, lo);
    const uint32_t carry = (uint32_t)(old + lo < old);
    if (hi + carry) atomicAdd(hi_w, hi + carry);
}

__device__ __forceinline__ void fix_add_shared(unsigned long long *p, long long v)
{
    uint32_t *w = reinterpret_cast<uint32_t *>(p);
    fix_add_shared(w, w + 1, v);
}

// Compensated FP32 add of v into the {sum, comp} pair.
__device__ __forceinline__ void comp_add(float *sum, float *comp, float v)
{
    const float a = atomicAdd(sum, v);
    const float s = __fadd_rn(a, v);
    const float bp = __fsub_rn(s, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(v, bp));
    if (err != 0.0f) atomicAdd(comp, err);
}

__device__ __forceinline__ void comp_add(unsigned long long *p, float v)
{
    float *w = reinterpret_cast<float *>(p);
    comp_add(w, w + 1, v);
}

__device__ __forceinline__ float block_max(float v, float *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    v = l < (int)(blockDim.x >> 5) ? red[l] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    return v;
}

__device__ __forceinline__ unsigned long long block_sum(unsigned long long v, unsigned long long *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    v = l < (int)(blockDim.x >> 5) ? red[l] : 0ull;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Warp 0 picks, from a 256-bin histogram scanned from the top bin down, the
// bin holding the kk-th largest key; writes the digit and the rank inside it.
__device__ __forceinline__ void pick_bin(const uint32_t *hist, uint32_t kk, uint32_t *digit, uint32_t *rank)
{
    const int l = threadIdx.x;
    uint32_t c8[8], tot = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        c8[u] = hist[255 - 8 * l - u];
        tot += c8[u];
    }
    uint32_t incl = tot;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t nb = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (l >= o) incl += nb;
    }
    const uint32_t excl = incl - tot;
    if (excl < kk && incl >= kk) {
        uint32_t cum = excl;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (cum + c8[u] >= kk) {
                *digit = 255 - 8 * l - u;
                *rank = kk - cum;
                break;
            }
            cum += c8[u];
        }
    }
}

// 64-byte row record as two 256-bit loads (one 32-B sector each).
__device__ __forceinline__ void load_slot(const uint4 *sp, uint32_t (&w)[16])
{
    asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                 : "l"(sp));
    asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]), "=r"(w[13]), "=r"(w[14]), "=r"(w[15])
                 : "l"(sp + 2));
}

// 32-byte compact record as one 256-bit load (one sector); w[8..15] unused.
__device__ __forceinline__ void load_rec32(const uint4 *sp, uint32_t (&w)[16])
{
    asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]), "=r"(w[7])
                 : "l"(sp));
}

}  // namespace

// Register cap and load depth.  The loops after the walks take their global
// loads in batches of DEPTH (UF) and DEPTH/2 (UL) per thread.  DEPTH 4 keeps
// an FP32 walk with one chain per thread at 64 registers, so eight 128-thread
// blocks (1024 chains) share an SM; DEPTH 8 needs 72 (seven blocks) but
// halves the L2 round trips of those loops, which pays for rows that send
// most of their visits through the overflow log, and its FP32 variant also
// filters the log through a magnitude sketch before reducing it.  FP64 walks
// take 72 registers at either depth rather than spill.
template <int PREC, int TABLE, int ACC, bool DUMP, int CPT, int DEPTH>
__global__ void __maxnreg__(CPT == 2 ? 80 : ((PREC == 64 || DEPTH == 8) ? 72 : 64)) k_walk(WalkArgs a)
{
    constexpr bool FIX = ACC == MCMI_ACC_FIXED64;
    constexpr bool CMP = TABLE == MCMI_TABLE_COMPACT;   // 32-byte records, 1/d_j from invd32
    // 8-byte log entries, the log's magnitude sketch and the presence map, in
    // the FP32 fixed-point production kernel for log-heavy rows (load depth 8;
    // on the stencil-like rows of the depth-4 kernel they cost 12%)
    constexpr bool SKETCH = FIX && PREC == 32 && !DUMP && DEPTH == 8;
    // finished values and the filter work in the build's precision: FP32
    // builds use no FP64 instruction per entry (FP64 issues at a small
    // fraction of the FP32 rate)
    using VT = typename std::conditional<PREC == 64, double, float>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = 1 << a.log2H;
    // per slot: a 64-bit value (fixed-point sum, or FP32 {sum, comp}; after
    // the walks the finished value of M_ij) as a low and a high 32-bit word in
    // two arrays, so that the low words of neighbouring slots fall in
    // neighbouring banks; the key; and an auxiliary word (visit counts in the
    // parity build, candidate list for FP64 values)
    uint32_t *s_lo = reinterpret_cast<uint32_t *>(smem);
    uint32_t *s_hi = s_lo + H;
    uint32_t *s_keys = s_hi + H;
    uint32_t *s_aux = s_keys + H;
    auto vword = [&](uint32_t h) -> unsigned long long {
        return (unsigned long long)s_lo[h] | ((unsigned long long)s_hi[h] << 32);
    };
    auto set_vword = [&](uint32_t h, unsigned long long v) {
        s_lo[h] = (uint32_t)v;
        s_hi[h] = (uint32_t)(v >> 32);
    };
    auto val_add = [&](uint32_t h, unsigned long long add) {
        if (FIX) fix_add_shared(&s_lo[h], &s_hi[h], (long long)add);
        else comp_add(reinterpret_cast<float *>(&s_lo[h]), reinterpret_cast<float *>(&s_hi[h]),
                      __uint_as_float((uint32_t)add));
    };
    // FP32 values leave the high words free for the candidate list
    auto list_at = [&](uint32_t p) -> uint32_t & {
        return PREC == 64 ? s_aux[p] : s_hi[p];
    };

    __shared__ long long s_row, s_pos, s_key_row;
    __shared__ int s_next_chain;
    __shared__ uint32_t s_fill, s_wpos, s_ncand, s_nlog, s_nent, s_nred, s_nsub, s_nmrg;
    __shared__ long long s_off;
    __shared__ double s_diag;
    __shared__ unsigned long long s_pass_lo, s_pass_hi;
    __shared__ float s_redf[32];
    __shared__ unsigned long long s_redu[32];
    // s_hist (256 words) and s_bstart (257) are used after the walks only;
    // during the walks the first 512 words hold the presence map
    __shared__ uint32_t s_hb[256 + 257];
    uint32_t *const s_hist = s_hb;
    uint32_t *const s_bstart = s_hb + 256;
    uint32_t *const s_pres = s_hb;
    __shared__ uint32_t s_digit, s_rank;
    __shared__ float s_cscale;   // the log's sketch: units per |W| |1/d_j| for the current row

    const int tid = threadIdx.x, B = blockDim.x;
    // on-chip table kept <= 87.5% full during the walks with the compact table
    // (banded rows: a 64^3 7-point stencil row visits up to ~1600 columns, all
    // of which then stay in a 2^11-slot table), <= 75% with the others (rows
    // that overflow anyway gain more from shorter probes)
    const uint32_t fill_cap = (uint32_t)(H - (H >> (CMP ? 3 : 2)));
    // log: the visits in arrival order, then the same entries bucketed by hash range
    uint2 *lc = a.log_key + (size_t)blockIdx.x * 2 * a.log_cap;
    unsigned long long *lv = a.log_val + (size_t)blockIdx.x * 2 * a.log_cap;
    uint2 *lc2 = lc + a.log_cap;
    unsigned long long *lv2 = lv + a.log_cap;
    uint32_t *ec = a.ent_col + (size_t)blockIdx.x * a.ent_cap;
    unsigned long long *ev = a.ent_val + (size_t)blockIdx.x * a.ent_cap;
    uint32_t *ecn = DUMP ? a.ent_cnt + (size_t)blockIdx.x * a.ent_cap : nullptr;
    const long long total = a.row_list ? a.n_list : a.row_end - a.row_begin;
    const int F = a.fix_shift;
    const float scaleF = __uint_as_float((uint32_t)(F + 127) << 23);   // 2^F (F <= 62)
    const bool use_tau = a.tau > 0.0;
    uint32_t *const g_cells = SKETCH ? a.cells + (size_t)blockIdx.x * kCells : nullptr;   // zero between rows
    // the log's sketch: largest units one entry adds (a row logs at most log_cap visits)
    const float cell_cap = (float)(kCellFlag / (a.log_cap > 0u ? a.log_cap : 1u) - 1u);
    // the column of a log entry's word (sketch kernels may keep a code in its top bits)
    const uint32_t colmask = (SKETCH && a.sk_code_bits) ? (0xFFFFFFFFu >> a.sk_code_bits) : 0xFFFFFFFFu;
    // cells of the sketch: built after the walks (code form), or the walk-time global cells
    const int cell_log2 = (SKETCH && a.sk_code_bits) ? min(kCellsCodeLog2, a.log2H + 1) : kCellsLog2;

    for (int h = tid; h < H; h += B) {
        s_keys[h] = kEmpty;
        s_lo[h] = 0u;
        s_hi[h] = 0u;
        if (DUMP) s_aux[h] = 0u;
    }
    if (SKETCH) {
        for (int c = tid; c < (1 << (kPresLog2 - 5)); c += B) s_pres[c] = 0u;
    }
    if (tid == 0) { s_fill = 0; s_nlog = 0; s_nent = 0; s_nred = 0; s_nmrg = 0; }

    // Slot of col in the on-chip table, inserting it if absent; -1 when it
    // is not added.  Linear probing over 4-slot buckets, one 16-byte read per
    // bucket; a key always takes the first empty slot in probe order, so a
    // search that meets an empty slot before the key knows the key is absent.
    // -1: the column is absent and cannot be inserted (table at its fill cap,
    // or no free slot within the probe window), or the table is at its cap
    // and the column was not in the buckets searched.
    // In the sketch kernels (walk == true in the walk loop): a column
    // sets its presence bit, then takes a fill ticket (never given back),
    // then claims its slot, and only a ticket below the cap may insert.  So
    // once a visit has read a fill at the cap, a column whose bit it then
    // finds clear can never be inserted: the visit returns -2 and goes to
    // the main log, whose columns are never on chip.  A visit that read the
    // table and still found no slot returns -1 and goes to the merge log,
    // whose columns are looked up on chip after the walks.
    bool seen_cap = false;   // this thread has read the fill at the cap during the current row's walks
    auto onchip_slot = [&](uint32_t col, bool walk) -> int {
        uint32_t bkt = hash_home(col, a.log2H - 2);
        const uint32_t nb = (uint32_t)(H >> 2);
        // the cap is read once, alongside the first bucket: lanes probing at
        // the same time may each still insert, so the table can pass the cap
        // by up to a block's threads (a small table may fill up; a probe then
        // gives up after its bucket limit and the visit is logged)
        const bool pres = SKETCH && walk;
        bool capped = pres && seen_cap;   // the fill only grows: once seen at the cap, it stays there
        if (!capped) {
            uint32_t fill_now;
            if (pres) {   // acquire: the presence bits set before the tickets read here are seen below
                asm volatile("ld.acquire.cta.shared.u32 %0, [%1];"
                             : "=r"(fill_now) : "r"((uint32_t)__cvta_generic_to_shared(&s_fill)) : "memory");
            } else {
                fill_now = *(volatile uint32_t *)&s_fill;
            }
            capped = fill_now >= fill_cap;
            if (pres && capped) seen_cap = true;
        }
        const uint32_t pb = (col * kPresMul) >> (32 - kPresLog2);
        if (pres && capped && !((*(volatile uint32_t *)&s_pres[pb >> 5] >> (pb & 31)) & 1u)) return -2;
        bool marked = false;
#pragma unroll 1
        for (int p = 0; p < kProbeOnChip / 4; ++p) {
            uint4 kv;
            asm volatile("ld.volatile.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(kv.x), "=r"(kv.y), "=r"(kv.z), "=r"(kv.w)
                         : "r"((uint32_t)__cvta_generic_to_shared(s_keys + 4 * bkt)));
            const int slot = kv.x == col ? 0 : kv.y == col ? 1 : kv.z == col ? 2 : kv.w == col ? 3 : -1;
            if (slot >= 0) return (int)(4 * bkt) + slot;
            const int e = kv.x == kEmpty ? 0 : kv.y == kEmpty ? 1 : kv.z == kEmpty ? 2 : kv.w == kEmpty ? 3 : -1;
            if (e >= 0) {
                if (capped) return -1;
                if (pres && !marked) {
                    atomicOr(&s_pres[pb >> 5], 1u << (pb & 31));
                    marked = true;
                    __threadfence_block();   // the bit before the ticket
                    if (atomicAdd(&s_fill, 1u) >= fill_cap) return -1;
                }
                const uint32_t old = atomicCAS(&s_keys[4 * bkt + e], kEmpty, col);
                if (!pres && old == kEmpty) atomicAdd(&s_fill, 1u);
                if (old == kEmpty || old == col) return (int)(4 * bkt) + e;
                --p;   // another key took the slot: read the bucket again
                continue;
            }
            // a full bucket without the key: once the table is at its cap, the
            // search stops here (the visit is logged; the merge after the walks
            // finds the key if it sits further on)
            if (capped) return -1;
            bkt = (bkt + 1) & (nb - 1);
        }
        return -1;
    };
    // Adds one visit to the on-chip table (the addend: the fixed-point weight,
    // or the FP32 bits of W / d_j for the Kahan accumulator); false when it
    // was not added.  The atomics come after the probe loop, where the lanes
    // of a warp have re-converged, so that one instruction serves them all.
    auto onchip_add = [&](uint32_t col, unsigned long long add) -> bool {
        const int h = onchip_slot(col, false);
        if (h < 0) return false;
        val_add((uint32_t)h, add);
        if (DUMP) atomicAdd(&s_aux[h], 1u);
        return true;
    };
    // Slot of col on chip, or -1; no insertion (used once no insertions run):
    // the bucket probe of onchip_add, ended by the first bucket with a free slot.
    auto onchip_find = [&](uint32_t col) -> int {
        uint32_t bkt = hash_home(col, a.log2H - 2);
        const uint32_t nb = (uint32_t)(H >> 2);
        for (int p = 0; p < kProbeOnChip / 4; ++p) {
            const uint4 kv = *reinterpret_cast<const uint4 *>(s_keys + 4 * bkt);
            if (kv.x == col) return (int)(4 * bkt);
            if (kv.y == col) return (int)(4 * bkt + 1);
            if (kv.z == col) return (int)(4 * bkt + 2);
            if (kv.w == col) return (int)(4 * bkt + 3);
            if (kv.x == kEmpty || kv.y == kEmpty || kv.z == kEmpty || kv.w == kEmpty) return -1;
            bkt = (bkt + 1) & (nb - 1);
        }
        return -1;
    };
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const long long pos = (long long)atomicAdd(&a.st->work, 1ull);
            s_pos = pos < total ? pos : -1;
            s_row = pos < total ? (a.row_list ? a.row_list[pos] : a.row_begin + pos) : -1;
            // random-number key of the row: its index inside its own matrix
            // when several matrices are built as one block-diagonal batch
            s_key_row = s_row;
            if (s_row >= 0 && a.batch_row_base) {
                int lo = 0, hi = a.batch_count - 1;   // last matrix whose first row <= s_row
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.batch_row_base[mid] <= s_row) lo = mid; else hi = mid - 1;
                }
                s_key_row = s_row - a.batch_row_base[lo];
            }
            s_next_chain = CPT * B;   // chains tid, tid + B, ... start at once
            if (s_row >= 0) {
                // t = 0 visits of all N chains: weight 1 at the row itself
                const uint32_t r = (uint32_t)s_row;
                const uint32_t h = 4 * hash_home(r, a.log2H - 2);   // first slot of its bucket
                s_keys[h] = r;
                s_fill = 1;
                if (SKETCH) {
                    const uint32_t pb = (r * kPresMul) >> (32 - kPresLog2);
                    s_pres[pb >> 5] |= 1u << (pb & 31);
                    // sketch units of this row: |1/d_i| 2^-kCellUnitLog2
                    const float invd_r = CMP ? __ldg(a.invd32 + r) : __uint_as_float(__ldg(&a.slots[4 * (size_t)r].z));
                    s_cscale = __fdiv_rn((float)(1u << kCellUnitLog2), fabsf(invd_r));
                }
                if (FIX) {
                    set_vword(h, (unsigned long long)((long long)a.N << F));
                } else {
                    const float invd = __uint_as_float(__ldg(&a.slots[4 * (size_t)r].z));
                    const float s0 = __fmul_rn((float)a.N, invd);
                    const float c0 = __fmaf_rn((float)a.N, invd, -s0);   // exact residual of the product
                    // the pair holds sum + comp == value; the compensation is
                    // stored as an addend, the TwoSum errors are added to it
                    set_vword(h, (unsigned long long)__float_as_uint(s0) |
                                     ((unsigned long long)__float_as_uint(c0) << 32));
                }
                if (DUMP) s_aux[h] = (uint32_t)a.N;
            }
        }
        __syncthreads();
        const long long row = s_row, pos = s_pos;
        if (row < 0) break;
        const long long idx = (a.row_list && !a.out_by_row) ? pos : row - a.row_begin;
        const uint32_t rlo = (uint32_t)s_key_row, rhi = (uint32_t)((unsigned long long)s_key_row >> 32);

        // ---- walks (Eq. 2): each thread advances CPT chains in turn, so that
        // CPT dependent gathers are in flight per thread; a chain that stops
        // is replaced by the row's next chain index ----
        unsigned long long my_steps = 0;
        seen_cap = false;
        uint32_t st[CPT];
        float w[CPT];            // FP32 weight (the FP64 path keeps it as the stop shadow)
        double w64[CPT];
        uint4 r4[CPT];
        int t[CPT], k[CPT];
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
            k[j] = tid + j * B;
            st[j] = (uint32_t)row;
            w[j] = 1.0f;
            w64[j] = 1.0;
            t[j] = 0;
            r4[j] = make_uint4(0, 0, 0, 0);
        }
        // All lanes of a warp run every iteration (the loop test is a warp
        // vote), so that the shared atomics of a step are issued by the whole
        // warp at once; lanes without a live chain only take part in the votes.
        // Every chain takes its step t = 0 in an iteration whose number is a
        // multiple of 4 (a lane whose chain stopped waits up to 3 iterations,
        // t < 0, before the next one starts), so that t = it (mod 4) for every
        // live chain and the Philox blocks of a warp are drawn together.
        const uint32_t lane = (uint32_t)tid & 31u;
        uint32_t it = 0;
#pragma unroll 1
        while (__any_sync(0xFFFFFFFFu, k[0] < a.N || (CPT > 1 && k[CPT - 1] < a.N))) {
            uint32_t s[CPT][16];
            double2 rd[CPT];
#pragma unroll
            for (int j = 0; j < CPT; ++j)
                if (k[j] < a.N && t[j] >= 0) {
                    if (CMP) load_rec32(a.slots + 2 * (size_t)st[j], s[j]);
                    else load_slot(a.slots + 4 * (size_t)st[j], s[j]);
                    if (PREC == 64) rd[j] = __ldg(a.rowd + st[j]);
                }
            // the block of step t (Eq. 2's draws, four per counter), computed
            // while the gathers are in flight; a chain that stops in this
            // iteration, or has not started, draws a block it does not use
            const uint32_t ph = it & 3u;
            if (ph == 0u) {
#pragma unroll
                for (int j = 0; j < CPT; ++j)
                    r4[j] = philox4x32_10(make_uint4((uint32_t)(t[j] >> 2), (uint32_t)k[j], rlo, rhi), a.key0, a.key1);
            }
#pragma unroll
            for (int j = 0; j < CPT; ++j) {
                const bool live = k[j] < a.N && t[j] >= 0;
                const bool acc = live && t[j] > 0;   // the visit of st[j] (t = 0 is counted at the row start)
                unsigned long long add = 0ull;
                int h = -1;
                if (acc) {
                    // a learned proposal's weights are not bounded by 1: the host
                    // leaves head-room in the fixed-point scale up to w_limit
                    if (FIX && a.lbkt && !(fabsf(w[j]) <= a.w_limit)) report(a.st, s_row, MCMI_ERR_CAPACITY);
                    if (FIX) add = (unsigned long long)(PREC == 64 ? fix_f64(w64[j], F) : fix_f32s(w[j], scaleF));
                    else add = (unsigned long long)__float_as_uint(__fmul_rn(w[j], __uint_as_float(s[j][2])));
                    h = onchip_slot(st[j], true);
                }
                __syncwarp();
                if (acc && h >= 0) {
                    val_add((uint32_t)h, add);
                    if (DUMP) atomicAdd(&s_aux[h], 1u);
                }
                // visits that do not fit on chip go to the log with the FP32 bits
                // of 1/d_col from the record just read; one atomic per warp
                // (sketch kernels: the main log for h == -2, the merge log in
                // the second region for h == -1)
                const bool to_log = acc && h < 0;
                const uint32_t lall = __ballot_sync(0xFFFFFFFFu, to_log);
                if (lall) {
                    const uint32_t lmg = SKETCH ? __ballot_sync(0xFFFFFFFFu, to_log && h == -1) : 0u;
                    const uint32_t lm = lall & ~lmg;
                    const uint32_t lt = (1u << lane) - 1u;
                    uint32_t base = 0, mbase = 0;
                    if (lm) {
                        const int first = __ffs(lm) - 1;
                        if ((int)lane == first) base = atomicAdd(&s_nlog, (uint32_t)__popc(lm));
                        base = __shfl_sync(0xFFFFFFFFu, base, first);
                    }
                    if (SKETCH && lmg) {
                        const int first = __ffs(lmg) - 1;
                        if ((int)lane == first) mbase = atomicAdd(&s_nmrg, (uint32_t)__popc(lmg));
                        mbase = __shfl_sync(0xFFFFFFFFu, mbase, first);
                    }
                    if (to_log) {
                        const bool mrg = SKETCH && h == -1;
                        const uint32_t pos = mrg ? mbase + (uint32_t)__popc(lmg & lt) : base + (uint32_t)__popc(lm & lt);
                        if (pos < a.log_cap) {
                            if (SKETCH) {
                                // one 8-byte entry {column, FP32 bits of W}: the
                                // addend fix_f32s(W) is recomputed when read; the
                                // column word carries the code of |1/d_j| for the
                                // sketch built after the walks, or the visit adds
                                // its magnitude to the global cells now
                                const float invd_j = CMP ? __ldg(a.invd32 + st[j]) : __uint_as_float(s[j][2]);
                                if (a.sk_code_bits) {
                                    (mrg ? lc2 : lc)[pos] =
                                        make_uint2(sketch_pack(st[j], invd_j, a.sk_code_bits), __float_as_uint(w[j]));
                                } else {
                                    (mrg ? lc2 : lc)[pos] = make_uint2(st[j], __float_as_uint(w[j]));
                                    const float q = __fmul_ru(__fmul_ru(fabsf(w[j]), fabsf(invd_j)), s_cscale);
                                    uint32_t *cell = &g_cells[(st[j] * kSketchMul) >> (32 - kCellsLog2)];
                                    if (q < cell_cap) atomicAdd(cell, (uint32_t)ceilf(q));
                                    else atomicOr(cell, kCellFlag);   // large, infinite or NaN
                                }
                            } else {
                                lc[pos] = make_uint2(st[j], CMP ? 0u : s[j][2]);   // compact: 1/d_j looked up later
                                lv[pos] = add;
                            }
                        } else {
                            report(a.st, s_row, MCMI_ERR_CAPACITY);   // cannot happen: a row makes at most N Lb visits
                        }
                    }
                }
                if (!live) {
                    t[j] += t[j] < 0;   // waiting for an iteration that is a multiple of 4
                    continue;
                }
                const uint32_t Q = record_q<TABLE>(s[j]);
                if (t[j] == a.L || !(fabsf(w[j]) >= a.delta_f) || Q == 0u) {
                    my_steps += (unsigned long long)t[j];
                    k[j] = atomicAdd(&s_next_chain, 1);
                    st[j] = (uint32_t)row;
                    w[j] = 1.0f;
                    w64[j] = 1.0;
                    t[j] = -(int)(3u - ph);   // its step 0 comes in the next iteration that is a multiple of 4
                    continue;
                }
                const uint32_t r = ph == 0u ? r4[j].x : ph == 1u ? r4[j].y : ph == 2u ? r4[j].z : r4[j].w;
                float fl;
                const uint32_t cs = pick_transition<TABLE>(s[j], r, a, &fl, st[j]);
                const bool neg = (cs & kNegBit) != 0u;
                w[j] = __fmul_rn(w[j], fl);
                if (PREC == 64) w64[j] = __dmul_rn(w64[j], neg ? -rd[j].x : rd[j].x);
                st[j] = cs & ~kNegBit;
                ++t[j];
            }
            ++it;
        }
        __syncthreads();

        // ---- row statistics ----
        if (!SKETCH) {   // the sketch kernels still need the presence map (cleared after the merge)
            for (int b = tid; b < 256; b += B) s_hist[b] = 0;
        }
        const unsigned long long row_steps = block_sum(my_steps, s_redu);
        if (tid == 0) {
            if (a.count_steps) atomicAdd(&a.st->steps, row_steps);
            if (a.row_steps) a.row_steps[idx] = row_steps;
            s_wpos = 0;
            s_ncand = 0;
        }
        uint32_t nlog = min(s_nlog, a.log_cap);
        const uint32_t nmrg = min(s_nmrg, a.log_cap);   // 0 in the kernels without the sketch
        const bool touched = nlog != 0u || nmrg != 0u;   // the row's sketch cells were used

        // finished values M_ij = (1/N) X_ij / d_j of the raw accumulator
        // words; invd = 1/d_j (FP32: the 4-byte-per-row array, which stays in
        // L2, else the record's copy; or FP64), unused by the Kahan
        // accumulator, whose sums are already scaled
        auto load_invd = [&](uint32_t col) -> VT {
            if (!FIX) return (VT)0;
            if (PREC == 64) return (VT)__ldg(&a.rowd[col].y);
            if (CMP || a.invd32) return (VT)__ldg(a.invd32 + col);
            return (VT)__uint_as_float(__ldg(&a.slots[4 * (size_t)col].z));
        };
        auto finish = [&](unsigned long long raw, VT invd) -> VT {
            if (PREC == 64) {
                const double X = __dmul_rn(__ll2double_rn((long long)raw), a.fix_inv);   // exact scaling
                return (VT)__dmul_rn(__ddiv_rn(X, (double)a.N), (double)invd);
            } else if (FIX) {
                // fl32(|X| 2^F), then (2^-F / N) and 1/d_j: three FP32 roundings
                const long long x = (long long)raw;
                // correctly rounded (ties to even), so the result scales exactly
                // with powers of two of |X| and does not depend on F
                const float m = __ull2float_rn((unsigned long long)(x < 0 ? -x : x));
                const float v = __fmul_rn(__fmul_rn(m, a.fin_scale), (float)invd);
                return (VT)(x < 0 ? -v : v);
            } else {
                const float sum = __uint_as_float((uint32_t)raw), c = __uint_as_float((uint32_t)(raw >> 32));
                return (VT)__fdiv_rn(__fadd_rn(sum, c), (float)a.N);
            }
        };
        // a finished value as stored: FP64 bits, or FP32 bits in the low word
        auto enc = [&](VT v) -> unsigned long long {
            if (PREC == 64) return (unsigned long long)__double_as_longlong((double)v);
            return (unsigned long long)__float_as_uint((float)v);
        };
        auto dec = [&](unsigned long long b) -> VT {
            if (PREC == 64) return (VT)__longlong_as_double((long long)b);
            return (VT)__uint_as_float((uint32_t)b);
        };
        auto sval = [&](uint32_t h) -> VT { return dec(vword(h)); };
        auto clear_table = [&]() {
            for (int h = tid; h < H; h += B) {
                s_keys[h] = kEmpty;
                s_lo[h] = 0u;
                s_hi[h] = 0u;
                if (DUMP || PREC == 64) s_aux[h] = 0u;
            }
        };
        // The loops below take their global loads in batches (UF, UL per
        // thread) issued before any of them is used: one L2 round trip per
        // batch instead of one per element.
        constexpr int UF = DEPTH, UL = DEPTH / 2;
        VT lmax = (VT)0;   // largest |M_ij| this thread has finished
        // Entries of the log below lowthr can never be kept: lowthr is tau
        // times a lower bound of the row maximum, rounded down, or with top-k
        // a lower bound of the k-th largest off-diagonal magnitude, whichever
        // is larger, so the entry list keeps only possible candidates (0: keep
        // everything).
        VT lowthr = (VT)0;
        // sketch kernels with tau: tau |M_ii| (rounded down) also bounds the
        // threshold from below, before any other entry is finished: the
        // diagonal is exact after the walks (inserted first, in the first slot
        // of its home bucket, where every visit of it finds it), so on-chip
        // entries below it need not go to the entry list
        VT lowpre = (VT)0;
        uint32_t nred = 0;   // distinct log columns this thread reduced (statistics)
        // Finishes the on-chip entries, in place, or appended to the entry
        // list with the table cleared (from_log: entries reduced from the log).
        auto finish_table = [&](bool to_list, bool from_log) {
            for (int h0 = tid; h0 < H; h0 += UF * B) {
                uint32_t key[UF];
                VT invd[UF];
#pragma unroll
                for (int u = 0; u < UF; ++u) key[u] = h0 + u * B < H ? s_keys[h0 + u * B] : kEmpty;
#pragma unroll
                for (int u = 0; u < UF; ++u) invd[u] = key[u] != kEmpty ? load_invd(key[u]) : (VT)0;
#pragma unroll
                for (int u = 0; u < UF; ++u) {
                    if (key[u] == kEmpty) continue;
                    const int h = h0 + u * B;
                    const VT v = finish(vword(h), invd[u]);
                    const VT av = v < (VT)0 ? -v : v;
                    lmax = av > lmax ? av : lmax;
                    if (key[u] == (uint32_t)row) s_diag = (double)v;
                    if (to_list) {
                        nred += from_log;
                        if (!(av < (from_log ? lowthr : lowpre))) {
                            const uint32_t p = atomicAdd(&s_nent, 1u);
                            ec[p] = key[u];
                            ev[p] = enc(v);
                            if (DUMP) ecn[p] = s_aux[h];
                        }
                        s_keys[h] = kEmpty;
                        s_lo[h] = 0u;
                        s_hi[h] = 0u;
                        if (DUMP || PREC == 64) s_aux[h] = 0u;
                    } else {
                        set_vword(h, enc(v));
                    }
                }
            }
        };

        // ---- the overflow log ----
        // the addend of log entry e: stored, or recomputed from the FP32
        // weight of an 8-byte entry (the same conversion as during the walk)
        auto log_add = [&](uint2 key, const unsigned long long *vals, uint32_t e) -> unsigned long long {
            if (SKETCH) return (unsigned long long)fix_f32s(__uint_as_float(key.y), scaleF);
            return vals[e];
        };
        // 1/d_j of a log entry's column: carried in the entry, or looked up
        auto log_invd = [&](uint2 key) -> VT {
            if (SKETCH || PREC == 64 || CMP) return load_invd(key.x & colmask);
            return (VT)__uint_as_float(key.y);
        };
        uint32_t nrem = 0;
        if (SKETCH && touched) {   // block-uniform
            // the merge log's columns are looked up on chip and added there;
            // those not found join the main log, whose columns are not on chip
            for (uint32_t e0 = tid; e0 < nmrg; e0 += UF * B) {
                uint2 key[UF];
#pragma unroll
                for (int u = 0; u < UF; ++u) key[u] = e0 + u * B < nmrg ? lc2[e0 + u * B] : make_uint2(kEmpty, 0u);
#pragma unroll
                for (int u = 0; u < UF; ++u) {
                    if (key[u].x == kEmpty) continue;
                    const int h = onchip_find(key[u].x & colmask);
                    if (h >= 0) {
                        val_add((uint32_t)h, log_add(key[u], lv, 0u));
                    } else {
                        const uint32_t p = atomicAdd(&s_nlog, 1u);   // < log_cap: the two logs hold one row's visits
                        if (p < a.log_cap) lc[p] = key[u];
                    }
                }
            }
            __syncthreads();
            nlog = min(s_nlog, a.log_cap);
            nrem = nlog;
            // the presence map's words become the histogram again
            for (int b = tid; b < 256; b += B) s_hist[b] = 0;
            __syncthreads();
        } else if (nlog) {   // block-uniform
            // entries whose column is on chip are added there; the others are
            // counted per hash-range bucket (top 8 bits of col * kPartMul)
            for (uint32_t e0 = tid; e0 < nlog; e0 += UL * B) {
                uint32_t key[UL];
#pragma unroll
                for (int u = 0; u < UL; ++u) key[u] = e0 + u * B < nlog ? lc[e0 + u * B].x : kEmpty;
#pragma unroll
                for (int u = 0; u < UL; ++u) {
                    if (key[u] == kEmpty) continue;
                    const uint32_t e = e0 + u * B;
                    const int h = onchip_find(key[u]);
                    if (h >= 0) {
                        const unsigned long long add = lv[e];
                        val_add((uint32_t)h, add);
                        if (DUMP) atomicAdd(&s_aux[h], 1u);
                        lc[e].x = kEmpty;
                    } else {
                        ++nrem;
                        atomicAdd(&s_hist[(key[u] * kPartMul) >> 24], 1u);
                    }
                }
            }
            nrem = (uint32_t)block_sum(nrem, s_redu);
        }
        if (nrem) {   // block-uniform
            if (SKETCH && use_tau && PREC == 32) {
                if (tid == 0) {
                    const uint32_t rr = (uint32_t)row;
                    const uint32_t h0 = 4u * hash_home(rr, a.log2H - 2);
                    const float vd = fabsf((float)finish(vword(h0), load_invd(rr)));
                    s_redf[0] = __fmul_rd(__double2float_rd(a.tau), vd);
                }
                __syncthreads();
                lowpre = (VT)s_redf[0];
                __syncthreads();
            }
            finish_table(true, false);
            if (!DUMP && use_tau) {
                // the on-chip entries (the diagonal among them) bound the row maximum from below
                VT rm;
                if (PREC == 64) {
                    unsigned long long lm = (unsigned long long)__double_as_longlong((double)lmax);
                    for (int o = 16; o > 0; o >>= 1) lm = max(lm, __shfl_xor_sync(0xFFFFFFFFu, lm, o));
                    __syncthreads();
                    if ((tid & 31) == 0) s_redu[tid >> 5] = lm;
                    __syncthreads();
                    lm = 0;
                    for (int w = 0; w < (B >> 5); ++w) lm = max(lm, s_redu[w]);
                    rm = (VT)__longlong_as_double((long long)lm);
                    lowthr = (VT)__dmul_rd(a.tau, (double)rm);
                } else {
                    rm = (VT)block_max((float)lmax, s_redf);
                    lowthr = (VT)__fmul_rd(__double2float_rd(a.tau), (float)rm);
                }
            }
            if (!DUMP && PREC == 32 && a.top_k > 0 && a.top_k < B) {
                // top-k bound: the (k+1)-th largest of the threads' maxima over
                // the on-chip entries.  At least k + 1 distinct entries reach
                // it, at most one of them the diagonal, so the row's k-th
                // largest off-diagonal |M_ij| does too: an entry below it is
                // not selected (or fails tau, if fewer than k pass).
                __syncthreads();
                s_bstart[tid] = __float_as_uint((float)lmax);   // |v| >= 0: bit order is value order
                __syncthreads();
                const uint32_t mine = s_bstart[tid];
                int rank = 0;
                for (int u = 0; u < B; ++u) {
                    const uint32_t o = s_bstart[u];
                    rank += (o > mine) || (o == mine && u < tid);
                }
                if (rank == a.top_k) s_digit = mine;
                __syncthreads();
                const float kb = __uint_as_float(s_digit);
                if (kb > (float)lowthr) lowthr = (VT)kb;
                __syncthreads();
            }
            // Magnitude sketch of the log (SKETCH kernels): cell c holds at
            // least s_cscale times the sum of |W| |1/d_j| over the main log's
            // entries (cells built below) or over all logged visits (walk-time
            // global cells) of the columns that hash to it, or has its top bit
            // set.  A column
            // that is not on chip finishes at |M_ij| <= (cell / (s_cscale N))
            // (1 + 2^-21) (the conversion and the finish's two products round
            // to nearest), so a column whose cell stays below
            // Tc = lowthr s_cscale N (1 - 2^-20), rounded down, is under lowthr
            // and can never be kept: its entries are neither bucketed nor
            // reduced.  (lowthr = 0: every cell is kept.)
            uint32_t Tc = 0u;
            if (SKETCH && lowthr > (VT)0) {
                const float tf = __fmul_rd(__fmul_rd(__fmul_rd((float)lowthr, s_cscale), (float)a.N), 1.0f - 0x1p-20f);
                Tc = !(tf >= 0.0f) ? 0u : (tf >= 2147483648.0f ? kCellFlag : (uint32_t)tf);
            }
            // the cells, staged in the emptied table's value words: copied
            // from the walk-time cells (one coalesced copy instead of a gather
            // per log entry), or built here from the main log's codes of
            // |1/d_j| (the same units, by the same rounded-up products, of a
            // value >= |1/d_j|; only the main log's columns, which the merge
            // has left off chip)
            const bool staged = SKETCH && 2 * H >= (1 << cell_log2);   // block-uniform
            if (staged) {
                if (a.sk_code_bits) {
                    if (Tc != 0u) {   // block-uniform (Tc = 0: every cell is hot)
                        __syncthreads();   // the table is empty
                        for (uint32_t e0 = tid; e0 < nlog; e0 += UF * B) {
                            uint2 key[UF];
#pragma unroll
                            for (int u = 0; u < UF; ++u) key[u] = e0 + u * B < nlog ? lc[e0 + u * B] : make_uint2(kEmpty, 0u);
#pragma unroll
                            for (int u = 0; u < UF; ++u) {
                                if (key[u].x == kEmpty) continue;
                                const float q = __fmul_ru(__fmul_ru(fabsf(__uint_as_float(key[u].y)),
                                                                    sketch_decode(key[u].x, a.sk_code_bits)), s_cscale);
                                uint32_t *cell = &s_lo[((key[u].x & colmask) * kSketchMul) >> (32 - cell_log2)];
                                if (q < cell_cap) atomicAdd(cell, (uint32_t)ceilf(q));
                                else atomicOr(cell, kCellFlag);   // large, infinite or NaN
                            }
                        }
                    }
                } else {
                    for (int c = tid; c < kCells / 4; c += B)
                        reinterpret_cast<uint4 *>(s_lo)[c] = __ldcg(reinterpret_cast<const uint4 *>(g_cells) + c);
                }
                __syncthreads();
            }
            auto hot = [&](uint32_t col) -> bool {
                const uint32_t ci = (col * kSketchMul) >> (32 - cell_log2);
                const uint32_t c = staged ? s_lo[ci] : (a.sk_code_bits ? kCellFlag : __ldcg(&g_cells[ci]));
                return (c & kCellFlag) || c >= Tc;
            };
            // SKETCH: one pass keeps the entries of hot cells, appended in
            // arrival order to lc2 and counted per hash-range bucket; they are
            // then bucketed into lc (free once this pass is over)
            if (SKETCH) {
                if (tid == 0) s_nsub = 0u;
                __syncthreads();
                for (uint32_t e0 = tid; e0 < nlog; e0 += UF * B) {
                    uint2 key[UF];
#pragma unroll
                    for (int u = 0; u < UF; ++u) key[u] = e0 + u * B < nlog ? lc[e0 + u * B] : make_uint2(kEmpty, 0u);
#pragma unroll
                    for (int u = 0; u < UF; ++u)
                        if (key[u].x != kEmpty && hot(key[u].x & colmask)) {
                            atomicAdd(&s_hist[((key[u].x & colmask) * kPartMul) >> 24], 1u);
                            lc2[atomicAdd(&s_nsub, 1u)] = key[u];
                        }
                }
                __syncthreads();
                if (staged) {   // the value words back to zero
                    for (int c = tid; c < (1 << cell_log2) / 4; c += B) reinterpret_cast<uint4 *>(s_lo)[c] = make_uint4(0, 0, 0, 0);
                    __syncthreads();
                }
            }
            // SKETCH: when the kept entries fit the emptied table's pass size,
            // one pass adds them all on chip and finishes them (a few L2
            // round trips, instead of one warp per hash bucket); if a probe
            // window overflows, the table is cleared and the bucketed
            // reduction below runs instead
            const uint32_t per_pass = (uint32_t)(H - (H >> 2)) - (uint32_t)((H - (H >> 2)) >> 2);
            bool reduced = false;
            if (SKETCH && s_nsub <= per_pass) {   // block-uniform
                if (tid == 0) s_fill = 0;
                __syncthreads();
                const uint32_t nh = s_nsub;
                bool ok = true;
                for (uint32_t e0 = tid; e0 < nh; e0 += UF * B) {
                    uint2 key[UF];
#pragma unroll
                    for (int u = 0; u < UF; ++u) key[u] = e0 + u * B < nh ? lc2[e0 + u * B] : make_uint2(kEmpty, 0u);
#pragma unroll
                    for (int u = 0; u < UF; ++u)
                        if (key[u].x != kEmpty && !onchip_add(key[u].x & colmask, log_add(key[u], lv2, 0u))) ok = false;
                }
                if (__syncthreads_or(!ok)) {
                    clear_table();
                } else {
                    finish_table(true, true);
                    reduced = true;
                }
                __syncthreads();
                if (tid == 0) s_fill = 0;
                __syncthreads();
            }
            if (!reduced) {   // block-uniform
                // bucket starts: exclusive scan of the 256 counts (warp 0, 8 per lane)
                if (tid < 32) {
                    uint32_t c8[8], tot = 0;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        c8[u] = s_hist[8 * tid + u];
                        tot += c8[u];
                    }
                    uint32_t incl = tot;
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t nb = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                        if (tid >= o) incl += nb;
                    }
                    uint32_t run = incl - tot;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        s_bstart[8 * tid + u] = run;
                        s_hist[8 * tid + u] = run;   // scatter cursor
                        run += c8[u];
                    }
                    if (tid == 31) s_bstart[256] = run;
                }
                __syncthreads();
                // bucketed copy: SKETCH kernels scatter their compact list of hot
                // entries from lc2 into lc, the others the whole log from lc into lc2
                const uint2 *src = SKETCH ? lc2 : lc;
                uint2 *const lb = SKETCH ? lc : lc2;
                const uint32_t nsrc = SKETCH ? s_nsub : nlog;
                for (uint32_t e0 = tid; e0 < nsrc; e0 += UL * B) {
                    uint2 key[UL];
                    unsigned long long val[UL];
#pragma unroll
                    for (int u = 0; u < UL; ++u) key[u] = e0 + u * B < nsrc ? src[e0 + u * B] : make_uint2(kEmpty, 0u);
                    if (!SKETCH) {
#pragma unroll
                        for (int u = 0; u < UL; ++u) val[u] = key[u].x != kEmpty ? lv[e0 + u * B] : 0ull;
                    }
#pragma unroll
                    for (int u = 0; u < UL; ++u) {
                        if (key[u].x == kEmpty) continue;
                        const uint32_t p = atomicAdd(&s_hist[((key[u].x & colmask) * kPartMul) >> 24], 1u);
                        lb[p] = key[u];
                        if (!SKETCH) lv2[p] = val[u];
                    }
                }
                if (tid == 0) s_fill = 0;
                __syncthreads();
                // Buckets of at most 32 entries: one warp each.  Lanes holding the
                // same column find each other with __match_any_sync; the group's
                // lowest lane sums it in a per-warp scratch row of 64-bit words
                // (over the empty table's low words, which needs 2B <= H slots) and
                // appends the finished entry.
                // (the sketch kernels reach here only when their kept entries did not
                // fit one pass: hash-range passes through the table handle them faster
                // than one warp per bucket)
                const bool by_warp = !SKETCH && 2 * B <= H;
                if (by_warp) {
                    unsigned long long *scratch = reinterpret_cast<unsigned long long *>(s_lo) + (tid & ~31);
                    constexpr int UB = 2;   // buckets per iteration: their loads are in flight together
                    const int nw = B >> 5;
                    for (int bk0 = tid >> 5; bk0 < 256; bk0 += UB * nw) {
                        uint2 key[UB];
                        unsigned long long val[UB];
                        uint32_t cnt[UB];
#pragma unroll
                        for (int u = 0; u < UB; ++u) {
                            const int bk = bk0 + u * nw;
                            const uint32_t s0 = bk < 256 ? s_bstart[bk] : 0u;
                            cnt[u] = bk < 256 ? s_bstart[bk + 1] - s0 : 0u;
                            const bool act = cnt[u] <= 32u && lane < cnt[u];
                            key[u] = act ? lb[s0 + lane] : make_uint2(kEmpty, 0u);
                            val[u] = act ? log_add(key[u], lv2, s0 + lane) : 0ull;
                        }
#pragma unroll
                        for (int u = 0; u < UB; ++u) {
                            if (cnt[u] == 0u || cnt[u] > 32u) continue;   // warp-uniform
                            const bool act = lane < cnt[u];
                            const uint32_t grp = __match_any_sync(0xFFFFFFFFu, key[u].x);
                            const uint32_t leader = (uint32_t)__ffs(grp) - 1u;
                            // a column seen once is its own sum; groups of several
                            // lanes add up in the warp's scratch row
                            const bool single = (grp & (grp - 1u)) == 0u;
                            if (!__all_sync(0xFFFFFFFFu, single || !act)) {
                                scratch[lane] = 0ull;
                                __syncwarp();
                                if (act && !single) {
                                    if (FIX) fix_add_shared(&scratch[leader], (long long)val[u]);
                                    else comp_add(&scratch[leader], __uint_as_float((uint32_t)val[u]));
                                }
                                __syncwarp();
                            }
                            const bool lead = act && lane == leader;
                            VT v = (VT)0;
                            bool keep = false;
                            if (lead) {
                                const VT invd = log_invd(key[u]);
                                v = finish(single ? val[u] : scratch[lane], invd);
                                const VT av = v < (VT)0 ? -v : v;
                                lmax = av > lmax ? av : lmax;
                                keep = !(av < lowthr);
                                ++nred;
                            }
                            const uint32_t lm = __ballot_sync(0xFFFFFFFFu, keep);
                            const int first = __ffs(lm) - 1;
                            uint32_t base = 0;
                            if (lm && (int)lane == first) base = atomicAdd(&s_nent, (uint32_t)__popc(lm));
                            if (lm) base = __shfl_sync(0xFFFFFFFFu, base, first);
                            if (keep) {
                                const uint32_t p = base + (uint32_t)__popc(lm & ((1u << lane) - 1u));
                                ec[p] = key[u].x;
                                ev[p] = enc(v);
                                if (DUMP) ecn[p] = (uint32_t)__popc(grp);
                            }
                            __syncwarp();
                        }
                    }
                    scratch[lane] = 0ull;
                }
                // larger buckets stay pending: s_hist[b] = entries of pending bucket b, else 0
                for (int bk = tid; bk < 256; bk += B) {
                    const uint32_t cnt = s_bstart[bk + 1] - s_bstart[bk];
                    s_hist[bk] = (cnt > 32u || !by_warp) ? cnt : 0u;
                }
                // Pending buckets: passes over hash ranges [lo, hi) holding at most
                // per_pass of their entries (so at most per_pass distinct columns)
                // through the on-chip table; a pass that still does not fit is
                // retried on the lower half of its range.
                unsigned long long lo = 0, retry_hi = 0;
                for (;;) {
                    __syncthreads();
                    if (tid == 0) {
                        unsigned long long l = lo, h = retry_hi;
                        if (!h) {
                            uint32_t b0 = (uint32_t)(l >> 24);
                            while (b0 < 256u && s_hist[b0] == 0u) ++b0;
                            if (b0 > (uint32_t)(l >> 24)) l = (unsigned long long)b0 << 24;
                            if (b0 < 256u) {
                                uint32_t b1 = b0 + 1, c = s_hist[b0];
                                while (b1 < 256u && c + s_hist[b1] <= per_pass) c += s_hist[b1++];
                                h = (unsigned long long)b1 << 24;
                            } else {
                                l = h = 1ull << 32;
                            }
                        }
                        s_pass_lo = l;
                        s_pass_hi = h;
                    }
                    __syncthreads();
                    lo = s_pass_lo;
                    const unsigned long long hi = s_pass_hi;
                    if (lo >= (1ull << 32)) break;
                    const uint32_t e0 = s_bstart[lo >> 24], e1 = s_bstart[((hi - 1) >> 24) + 1];
                    bool ok = true;
                    for (uint32_t eb = e0 + tid; eb < e1 && ok; eb += UL * B) {
                        uint32_t key[UL];
                        unsigned long long val[UL];
#pragma unroll
                        for (int u = 0; u < UL; ++u) {
                            const uint2 kk = eb + u * B < e1 ? lb[eb + u * B] : make_uint2(kEmpty, 0u);
                            key[u] = kk.x == kEmpty ? kEmpty : (kk.x & colmask);
                            val[u] = kk.x != kEmpty ? log_add(kk, lv2, eb + u * B) : 0ull;
                        }
#pragma unroll
                        for (int u = 0; u < UL; ++u) {
                            if (key[u] == kEmpty) continue;
                            const unsigned long long hv = key[u] * kPartMul;
                            if (hv < lo || hv >= hi || s_hist[hv >> 24] == 0u) continue;
                            if (!onchip_add(key[u], val[u])) ok = false;
                        }
                    }
                    if (__syncthreads_or(!ok)) {
                        clear_table();
                        if (hi - lo > 1) {
                            retry_hi = lo + ((hi - lo) >> 1);
                        } else {   // one hash value is one column, which always fits: not reached
                            report(a.st, row, MCMI_ERR_CAPACITY);
                            retry_hi = 0;
                            lo = hi;
                        }
                    } else {
                        finish_table(true, true);
                        retry_hi = 0;
                        lo = hi;
                    }
                    __syncthreads();
                    if (tid == 0) s_fill = 0;
                }
            }   // !reduced
            __syncthreads();
            if (nred) atomicAdd(&s_nred, nred);
            __syncthreads();
            if (tid == 0) atomicAdd(&a.st->spilled, (unsigned long long)s_nred);
        } else {
            finish_table(false, false);
        }
        __syncthreads();
        const uint32_t nent = s_nent;

        if (DUMP) {
            auto dump = [&](uint32_t col, VT v, uint32_t vis) {
                const uint32_t p = atomicAdd(&s_wpos, 1u);
                if (p < (uint32_t)a.d_cap) {
                    a.d_col[idx * a.d_cap + p] = (int32_t)col;
                    a.d_val[idx * a.d_cap + p] = (double)v;
                    a.d_vis[idx * a.d_cap + p] = vis;
                }
            };
            for (int h = tid; h < H; h += B)
                if (s_keys[h] != kEmpty) dump(s_keys[h], sval(h), s_aux[h]);
            for (uint32_t e = tid; e < nent; e += B) dump(ec[e], dec(ev[e]), ecn[e]);
            __syncthreads();
            if (tid == 0) {
                const uint32_t c = s_wpos;
                a.d_count[idx] = c <= (uint32_t)a.d_cap ? (int32_t)c : -1;
                if (c > (uint32_t)a.d_cap) report(a.st, row, MCMI_ERR_CAPACITY);
            }
        } else {
            // ---- Sec. IV-B filter: diagonal kept; tau rule; top-k ----
            VT rowmax;
            if (PREC == 64) {
                // |M_ij| >= 0: the order of the FP64 bit patterns is the order of the values
                unsigned long long lm = (unsigned long long)__double_as_longlong((double)lmax);
                for (int o = 16; o > 0; o >>= 1) lm = max(lm, __shfl_xor_sync(0xFFFFFFFFu, lm, o));
                __syncthreads();
                if ((tid & 31) == 0) s_redu[tid >> 5] = lm;
                __syncthreads();
                lm = 0;
                for (int w = 0; w < (B >> 5); ++w) lm = max(lm, s_redu[w]);
                rowmax = (VT)__longlong_as_double((long long)lm);
            } else {
                rowmax = (VT)block_max((float)lmax, s_redf);
            }
            // threshold tau * rowmax in FP64; an FP32 build compares against the
            // smallest float >= it, which keeps exactly the same entries
            const double thr64 = use_tau ? __dmul_rn(a.tau, (double)rowmax) : 0.0;
            const VT thr = PREC == 64 ? (VT)thr64 : (VT)__double2float_ru(thr64);
            const uint32_t rowc = (uint32_t)row;
            // top-k (FP32): only entries reaching kb, the (k+1)-th largest of
            // the threads' maxima, can be selected (k + 1 distinct entries
            // reach it, at most one the diagonal); the rest are not candidates
            float kb = 0.0f;
            if (PREC == 32 && a.top_k > 0 && a.top_k < B) {
                __syncthreads();
                s_bstart[tid] = __float_as_uint((float)lmax);
                __syncthreads();
                const uint32_t mine = s_bstart[tid];
                int rank = 0;
                for (int u = 0; u < B; ++u) {
                    const uint32_t o = s_bstart[u];
                    rank += (o > mine) || (o == mine && u < tid);
                }
                if (rank == a.top_k) s_digit = mine;
                __syncthreads();
                kb = __uint_as_float(s_digit);
                __syncthreads();
            }
            auto is_cand = [&](uint32_t k, VT v) -> bool {
                return k != rowc && (!use_tau || fabs(v) >= thr) && (PREC != 32 || fabsf((float)v) >= kb);
            };
            // candidates: on-chip slot h as h, entry-list element e as H + e
            const uint32_t list_cap = (uint32_t)H;
            for (int h = tid; h < H; h += B) {
                const uint32_t k = s_keys[h];
                if (k != kEmpty && is_cand(k, sval(h))) {
                    const uint32_t p = atomicAdd(&s_ncand, 1u);
                    if (p < list_cap) list_at(p) = (uint32_t)h;
                }
            }
            for (uint32_t e0 = tid; e0 < nent; e0 += UL * B) {
                uint32_t key[UL];
                unsigned long long raw[UL];
#pragma unroll
                for (int u = 0; u < UL; ++u) {
                    key[u] = e0 + u * B < nent ? ec[e0 + u * B] : kEmpty;
                    raw[u] = e0 + u * B < nent ? ev[e0 + u * B] : 0ull;
                }
#pragma unroll
                for (int u = 0; u < UL; ++u) {
                    if (key[u] != kEmpty && is_cand(key[u], dec(raw[u]))) {
                        const uint32_t p = atomicAdd(&s_ncand, 1u);
                        if (p < list_cap) list_at(p) = (uint32_t)H + e0 + u * B;
                    }
                }
            }
            __syncthreads();
            const uint32_t nc = s_ncand;
            const bool compact = nc <= list_cap;
            const bool select = a.top_k > 0 && nc > (uint32_t)a.top_k;
            // visit every candidate: fn(magnitude bits, column, value)
            auto for_cands = [&](auto fn) {
                if (compact) {
                    for (uint32_t i = tid; i < nc; i += B) {
                        const uint32_t c = list_at(i);
                        const uint32_t col = c < (uint32_t)H ? s_keys[c] : ec[c - H];
                        const VT v = c < (uint32_t)H ? sval(c) : dec(ev[c - H]);
                        fn(__float_as_uint(fabsf((float)v)), col, v);
                    }
                } else {
                    for (int h = tid; h < H; h += B) {
                        const uint32_t k = s_keys[h];
                        if (k == kEmpty) continue;
                        const VT v = sval(h);
                        if (is_cand(k, v)) fn(__float_as_uint(fabsf((float)v)), k, v);
                    }
                    for (uint32_t e = tid; e < nent; e += B) {
                        const VT v = dec(ev[e]);
                        if (is_cand(ec[e], v)) fn(__float_as_uint(fabsf((float)v)), ec[e], v);
                    }
                }
            };
            uint32_t vstar = 0, cstar_inv = 0;
            if (select && compact && nc <= 64u) {
                // few candidates: warp 0 ranks the keys (magnitude bits << 32 |
                // ~col; larger is preferred) by shuffles, two per lane; the
                // top_k-th key gives the magnitude and tie bounds of the rule
                if (tid < 32) {
                    auto key_of = [&](uint32_t i) -> unsigned long long {
                        const uint32_t c = list_at(i);
                        const uint32_t col = c < (uint32_t)H ? s_keys[c] : ec[c - H];
                        const VT v = c < (uint32_t)H ? sval(c) : dec(ev[c - H]);
                        return ((unsigned long long)__float_as_uint(fabsf((float)v)) << 32) | (~col);
                    };
                    const uint32_t l = (uint32_t)tid;
                    const unsigned long long K0 = l < nc ? key_of(l) : 0ull;           // 0: no entry
                    const unsigned long long K1 = l + 32u < nc ? key_of(l + 32u) : 0ull;
                    int r0 = 0, r1 = 0;
                    for (int j = 0; j < 32; ++j) {
                        const unsigned long long x0 = __shfl_sync(0xFFFFFFFFu, K0, j);
                        const unsigned long long x1 = __shfl_sync(0xFFFFFFFFu, K1, j);
                        r0 += (x0 > K0) + (x1 > K0);
                        r1 += (x0 > K1) + (x1 > K1);
                    }
                    if (l < nc && r0 == a.top_k - 1) s_pass_lo = K0;
                    if (l + 32u < nc && r1 == a.top_k - 1) s_pass_lo = K1;
                }
                __syncthreads();
                vstar = (uint32_t)(s_pass_lo >> 32);
                cstar_inv = (uint32_t)s_pass_lo;
            } else if (select) {
                // magnitude bits of compact candidate i
                auto cand_mag = [&](uint32_t i) -> uint32_t {
                    const uint32_t c = list_at(i);
                    const VT v = c < (uint32_t)H ? sval(c) : dec(ev[c - H]);
                    return __float_as_uint(fabsf((float)v));
                };
                // After the first pass the candidates of the chosen bin (usually
                // few) are listed in s_bstart, and later passes visit only them.
                bool narrow = false;
                uint32_t nsub = 0;
                auto for_bin = [&](auto fn) {   // fn(magnitude bits, column) over the bin's candidates
                    if (narrow) {
                        for (uint32_t t = tid; t < nsub; t += B) {
                            const uint32_t i = s_bstart[t];
                            const uint32_t c = list_at(i);
                            fn(cand_mag(i), c < (uint32_t)H ? s_keys[c] : ec[c - H]);
                        }
                    } else {
                        for_cands([&](uint32_t mag, uint32_t col, VT) { fn(mag, col); });
                    }
                };
                // radix select of the top_k-th largest magnitude (FP32 bits), 8 bits per pass
                uint32_t pre = 0, mask = 0, kk = (uint32_t)a.top_k;
                for (int shift = 24; shift >= 0; shift -= 8) {
                    for (int b = tid; b < 256; b += B) s_hist[b] = 0;
                    __syncthreads();
                    for_bin([&](uint32_t mag, uint32_t) {
                        if ((mag & mask) == pre) atomicAdd(&s_hist[(mag >> shift) & 255u], 1u);
                    });
                    __syncthreads();
                    if (tid < 32) pick_bin(s_hist, kk, &s_digit, &s_rank);
                    __syncthreads();
                    pre |= s_digit << shift;
                    kk = s_rank;
                    mask |= 255u << shift;
                    if (shift == 24 && compact && s_hist[s_digit] <= 256u) {
                        if (tid == 0) s_nsub = 0;
                        __syncthreads();
                        for (uint32_t i = tid; i < nc; i += B)
                            if ((cand_mag(i) & mask) == pre) s_bstart[atomicAdd(&s_nsub, 1u)] = i;
                        __syncthreads();
                        nsub = s_nsub;
                        narrow = true;
                    }
                    __syncthreads();
                }
                vstar = pre;               // magnitude bits of the top_k-th largest
                const uint32_t keep_ties = kk;
                unsigned long long eq_l = 0;
                for_bin([&](uint32_t mag, uint32_t) { eq_l += (mag == vstar); });
                const unsigned long long neq = block_sum(eq_l, s_redu);
                if (neq > keep_ties) {
                    // equal magnitudes: keep the keep_ties smallest columns (radix select on ~col)
                    uint32_t cpre = 0, cmask = 0, ck = keep_ties;
                    for (int shift = 24; shift >= 0; shift -= 8) {
                        for (int b = tid; b < 256; b += B) s_hist[b] = 0;
                        __syncthreads();
                        for_bin([&](uint32_t mag, uint32_t col) {
                            const uint32_t inv = ~col;
                            if (mag == vstar && (inv & cmask) == cpre) atomicAdd(&s_hist[(inv >> shift) & 255u], 1u);
                        });
                        __syncthreads();
                        if (tid < 32) pick_bin(s_hist, ck, &s_digit, &s_rank);
                        __syncthreads();
                        cpre |= s_digit << shift;
                        ck = s_rank;
                        cmask |= 255u << shift;
                        __syncthreads();
                    }
                    cstar_inv = cpre;
                }
            }
            const unsigned long long nk = 1ull + (select ? (unsigned long long)a.top_k : nc);
            if (tid == 0) {
                const unsigned long long off = atomicAdd(&a.st->cursor, nk);
                if (off + nk > a.st_cap) {
                    const unsigned long long dnum = atomicAdd(&a.st->deferred, 1ull);
                    a.deferred_list[dnum] = row;
                    a.row_cnt[idx] = -1;
                    s_off = -1;
                } else {
                    a.row_off[idx] = (int64_t)off;
                    a.row_cnt[idx] = (int32_t)nk;
                    s_off = (long long)off;
                }
            }
            __syncthreads();
            const long long off = s_off;
            if (off >= 0) {
                auto put = [&](uint32_t k, VT v) {
                    const uint32_t p = atomicAdd(&s_wpos, 1u);
                    a.st_col[off + p] = k;
                    a.st_val[off + p] = (float)v;
                };
                // the diagonal (always present: inserted before the walks)
                if (tid == 0) put(rowc, (VT)s_diag);
                for_cands([&](uint32_t mag, uint32_t col, VT v) {
                    const bool keep = !select || mag > vstar || (mag == vstar && (~col) >= cstar_inv);
                    if (keep) put(col, v);
                });
            }
        }
        __syncthreads();
        // ---- reset the accumulator for the next row ----
        clear_table();
        if (SKETCH) {
            if (touched && !a.sk_code_bits) {   // block-uniform: only a row that logged visits touched its cells
                for (int c = tid; c < kCells / 4; c += B) reinterpret_cast<uint4 *>(g_cells)[c] = make_uint4(0, 0, 0, 0);
            }
            for (int c = tid; c < (1 << (kPresLog2 - 5)); c += B) s_pres[c] = 0u;
        }
        if (tid == 0) { s_fill = 0; s_nlog = 0; s_nent = 0; s_nred = 0; s_nmrg = 0; }
    }
}

// per slot: 8-B value word, 4-B key, and 4 B of counts / candidate list where needed
size_t walk_smem_bytes(int precision, int log2H, bool dump)
{
    return ((size_t)1 << log2H) * ((dump || precision == 64) ? 16 : 12);
}

size_t walk_sketch_cells() { return (size_t)kCells; }

namespace {
using WalkFn = void (*)(WalkArgs);

template <bool D, int C, int U>
WalkFn pick_walk(int precision, int table, int acc)
{
    // table: MCMI_TABLE_* (hybrid runs the alias kernels); the compact table
    // only with the fixed-point accumulator (the parameter check enforces it)
    if (precision == 64) {
        if (table == MCMI_TABLE_COMPACT) return k_walk<64, MCMI_TABLE_COMPACT, MCMI_ACC_FIXED64, D, C, U>;
        return table ? k_walk<64, 1, MCMI_ACC_FIXED64, D, C, U> : k_walk<64, 0, MCMI_ACC_FIXED64, D, C, U>;
    }
    if (acc == MCMI_ACC_KAHAN32)
        return table ? k_walk<32, 1, MCMI_ACC_KAHAN32, D, C, U> : k_walk<32, 0, MCMI_ACC_KAHAN32, D, C, U>;
    if (table == MCMI_TABLE_COMPACT) return k_walk<32, MCMI_TABLE_COMPACT, MCMI_ACC_FIXED64, D, C, U>;
    return table ? k_walk<32, 1, MCMI_ACC_FIXED64, D, C, U> : k_walk<32, 0, MCMI_ACC_FIXED64, D, C, U>;
}

template <int U>
WalkFn walk_kernel_d(int precision, int table, int acc, bool dump, int cpt)
{
    if (cpt == 1) return dump ? pick_walk<true, 1, U>(precision, table, acc) : pick_walk<false, 1, U>(precision, table, acc);
    return dump ? pick_walk<true, 2, U>(precision, table, acc) : pick_walk<false, 2, U>(precision, table, acc);
}

WalkFn walk_kernel(int precision, int table, int acc, bool dump, int cpt, int depth)
{
    return depth == 8 ? walk_kernel_d<8>(precision, table, acc, dump, cpt)
                      : walk_kernel_d<4>(precision, table, acc, dump, cpt);
}
}  // namespace

cudaError_t walk_occupancy(int precision, int table, int acc, bool dump, int cpt, int depth, int threads, int log2H,
                           int *blocks_per_sm)
{
    const size_t smem = walk_smem_bytes(precision, log2H, dump);
    const WalkFn fn = walk_kernel(precision, table, acc, dump, cpt, depth);
    cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void *)fn, threads, smem);
}

cudaError_t launch_walk(const WalkArgs &a, int precision, int table, int acc, bool dump, int cpt, int depth,
                        int grid, int threads, cudaStream_t s)
{
    const size_t smem = walk_smem_bytes(precision, a.log2H, dump);
    const WalkFn fn = walk_kernel(precision, table, acc, dump, cpt, depth);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    if (cap == cudaStreamCaptureStatusNone) {   // during graph capture it was set by walk_occupancy
        cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    fn<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mcmi
