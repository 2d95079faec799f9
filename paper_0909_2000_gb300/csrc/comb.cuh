// comb.cuh -- the seaweed strip-comb kernel for alignment plots (sm_103a).
//
// Method (Krusche & Tiskin, "Computing alignment plots efficiently"):
//   * Theorem 3.1: for each x-window (a "strip" of w rows), comb the strip
//     against all of y, column by column.  One seaweed starts at the top of
//     every column and one leaves at the bottom.  The LCS of the strip and
//     the y-window ending at column J is w - d(J).  Here d(J) counts the
//     seaweeds that started inside the window and have already left at the
//     bottom inside it.
//   * Section 2 cell rule: the seaweeds entering a cell from the left (h)
//     and from the top (v) swap directions in a match cell, or when they
//     have crossed before; otherwise they cross.  With seaweeds keyed by
//     start column (larger = newer), "crossed before" means h is newer than
//     v.  So the bottom output is h if (match or h >= v), else v.
//   * Section 3: keys need only O(log w) bits (Proposition 3.4).  A seaweed
//     older than the window is irrelevant, and all such seaweeds can share
//     one key.  The vector step is the paper's anti-diagonal
//     compare/exchange with a match mask and a masked blend.
//
// GB300 mapping:
//   * SWAR: one 32-bit register holds the same comb row of NS strips that
//     are next to each other (4 x 8-bit lanes, 3 x 10-bit lanes or 2 x
//     16-bit lanes).  Strip i+b, row k reads x[i+b+k], so a row register is
//     an NS-character window of x.  The match mask of each aligned x word is
//     computed once per column, and the other rows' masks are lane shifts of
//     those masks, done as multiplies on the FMA pipe (the cells keep the
//     ALU pipe busy).
//   * Keys are start columns, not distances, so columns need no increment.
//     Every Rr columns all keys drop by Rr, saturating at 0 (0 = "older
//     than any window").  The new seaweed's key cycles in [w, KMAX].
//   * Each CTA warp owns one tile: a group of strips times a chunk of plot
//     columns.  A chunk starting at column c0 starts a fresh comb at c0 and
//     runs w - 1 warm-up columns.  That is exact for every window starting
//     at or after c0: seaweeds from before c0 are all older than those
//     windows.
//   * d(J) is kept with a ring of "left validly" flags indexed by start
//     column.  This is an O(1)-per-column stand-in for the paper's min-heap
//     B, with the same numbers.
//   * When a strip's rows are split over G lanes, the wavefront is skewed
//     by one column per lane, and v passes down with a warp shuffle.
//   * Results are staged in shared memory and written to HBM as
//     row-contiguous, sector-aligned stores (16 bytes per thread where the
//     rows allow).
//   * Tiles whose characters all share the top bit take a shorter mismatch
//     test (one logic instruction fewer per x word).
//
// Score mode ({2,1,0}, Section 2): the comb runs on the '$'-interleaved
// strings x' = $x0$x1..., y' = $y0$y1...  Rows and columns alternate '$'
// and a character; '$' matches only '$', so no byte value is reserved.
// Keys are start *pairs* floor(s/2) (the (w,2)-restricted matrix of
// Definition 3.2 and Proposition 3.4).  Only windows at even offsets
// exist, and the value is T = 2w - d.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ap {

constexpr int kWarpsPerBlock = 4;
#ifndef AP_MIN_BLOCKS
#define AP_MIN_BLOCKS 1   // minimum resident blocks per SM asked of the compiler
#endif
constexpr int kOB = 32;   // plot columns staged per flush (one per lane; a power of two)

struct CombParams {
    const uint8_t *x;
    const uint8_t *y;
    int64_t m, n;
    int32_t w;          // window length (key window, in units)
    int32_t renorm;     // steps between key renormalisations
    int64_t rows, cols; // plot shape
    int64_t chunk;      // plot columns per tile
    int64_t nsg;        // strip groups (warps along the plot rows)
    int64_t ntiles;     // nsg * column chunks
    int64_t tile0;      // first tile of this launch (for split launches)
    void *out;
    int64_t ld;         // elements between plot rows
    int32_t out_bytes;  // 1 or 2
    int32_t vec_ok;     // output pointer/ld allow aligned vector stores
    int32_t ring;       // ring slots (power of two > w)
    // Runtime constants for the FMA-pipe forms of shifts and adds: one = 1,
    // shmul[r] = 2^(32 - 8r) for byte shifts r = 1..3.  Passed at run time so
    // the compiler keeps them as integer multiply-adds (FMA pipe) instead of
    // turning them into ALU shifts; the ALU pipe is the comb's bottleneck.
    uint32_t one;
    uint32_t shmul[4];
    // Row shifts of 10-bit lanes (three per register, bits 30-31 unused):
    // rows r = 1, 2 past an aligned word are (a >> 10r) | (b << (30 - 10r)),
    // the high word of a * shmul[r] plus b * shlo[r] (for byte lanes
    // shlo = shmul).  spread_hi = 2^23 and spread_lo = 0x3FF turn the
    // compare bits of 10-bit lanes into full-lane masks on the FMA pipe.
    uint32_t shlo[4];
    uint32_t spread_hi, spread_lo;
    int64_t step;       // x offset between consecutive plot rows (vertical step h)
    int32_t warp_words; // shared-memory words per warp of a plain launch
    uint32_t scale;     // plot values are scale x the comb's values (gcd of the scores)
    int32_t mu;         // the blow-up's '$' count per character (variants built with MU = -1)
    int32_t tab;        // G > 1 tables: the row split's rounding mode (tabg_split_mode), 0 for none
    uint32_t *dbg;      // debug builds: violation bits of the bounds checks (device), else null
};

// Bounds checks of debug builds (compiled with AP_DEBUG_BOUNDS): a failed
// check sets its bit in *p.dbg and the access it guards is skipped, so a
// wrong index is reported (ap_debug_bounds) instead of touching memory
// outside its buffer.  In other builds every check is the constant true.
enum : uint32_t {
    kDbgPlotStore = 1u,    // a plot store outside rows x cols
    kDbgYRead = 2u,        // a y read outside [0, n)
    kDbgXRead = 4u,        // an x read outside [0, m)
    kDbgRing = 8u,         // an exit-ring slot outside the ring
    kDbgTable = 16u,       // a match-table read outside the tables
};
#ifdef AP_DEBUG_BOUNDS
__device__ __forceinline__ bool ap_check(uint32_t *flag, bool ok, uint32_t code)
{
    if (!ok && flag) atomicOr(flag, code);
    return ok;
}
#define AP_CHECK(p, cond, code) ap_check((p).dbg, (cond), (code))
#else
#define AP_CHECK(p, cond, code) true
#endif

// ---------------------------------------------------------------------------
// SWAR lane formats
// ---------------------------------------------------------------------------

struct U8Lanes {
    static constexpr int NS = 4;        // strips per register
    static constexpr int BITS = 8;
    static constexpr bool FULL = false; // keys use 7 bits; bit 7 is the compare bit
    static constexpr int RPW = 4;       // rows per aligned x word
    static constexpr int KMAX = 127;
    static constexpr uint32_t ONES = 0x01010101u;
    static constexpr uint32_t MSB = 0x80808080u;
    static constexpr uint32_t LOW = 0x7F7F7F7Fu;
    static constexpr uint32_t SIGNREP = 0xBA98u;   // each byte := its sign bit
    static constexpr uint32_t MASK = 0xFFu;
};

// 8-bit lanes with full 8-bit keys (windows up to 254): compares and
// subtractions handle the top bit separately.
struct U8FLanes {
    static constexpr int NS = 4;
    static constexpr int BITS = 8;
    static constexpr bool FULL = true;
    static constexpr int RPW = 4;
    static constexpr int KMAX = 255;
    static constexpr uint32_t ONES = 0x01010101u;
    static constexpr uint32_t MSB = 0x80808080u;
    static constexpr uint32_t LOW = 0x7F7F7F7Fu;
    static constexpr uint32_t SIGNREP = 0xBA98u;
    static constexpr uint32_t MASK = 0xFFu;
};

// 10-bit lanes (windows 257..480): three strips per register in bits 0-29,
// 9-bit keys with bit 9 of each lane as the compare bit.  No byte permute
// spreads a 10-bit lane, so masks are spread by two multiplies (FMA pipe).
struct U10Lanes {
    static constexpr int NS = 3;
    static constexpr int BITS = 10;
    static constexpr bool FULL = false;
    static constexpr int RPW = 3;
    static constexpr int KMAX = 511;
    static constexpr uint32_t ONES = 0x00100401u;
    static constexpr uint32_t MSB = 0x20080200u;
    static constexpr uint32_t LOW = 0x1FF7FDFFu;
    static constexpr uint32_t SIGNREP = 0u;         // not used
    static constexpr uint32_t MASK = 0x3FFu;
};

struct U16Lanes {
    static constexpr int NS = 2;
    static constexpr int BITS = 16;
    static constexpr bool FULL = false;
    static constexpr int RPW = 2;
    static constexpr int KMAX = 32767;
    static constexpr uint32_t ONES = 0x00010001u;
    static constexpr uint32_t MSB = 0x80008000u;
    static constexpr uint32_t LOW = 0x7FFF7FFFu;
    static constexpr uint32_t SIGNREP = 0xBB99u;   // each half := its sign bit
    static constexpr uint32_t MASK = 0xFFFFu;
};

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
    return r;
}

__device__ __forceinline__ uint32_t mul_hi(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
    return r;
}

// Per-half unsigned maximum and minimum of two 16-bit lane pairs (one
// instruction each on sm_90 and later).
__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b)
{
    uint32_t r;
    asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

// Full-width unsigned a >= b in every lane, as the lane's top bit (other bits
// are junk): compare the low bits with the top bit forced on a and off b (no
// borrow between lanes), then let the top bits decide where they differ.
template <class L>
__device__ __forceinline__ uint32_t ge_lanes(uint32_t a, uint32_t b, uint32_t neg1)
{
    const uint32_t t = mad_lo(b & L::LOW, neg1, a | L::MSB);   // MSB: a_low >= b_low
    return (a & ~b) | (~(a ^ b) & t);
}

// Lane-wise (a - b) modulo the lane width, with no borrow between lanes.
template <class L>
__device__ __forceinline__ uint32_t sub_lanes(uint32_t a, uint32_t b)
{
    const uint32_t lo = (a | L::MSB) - (b & L::LOW);
    return lo ^ ((a ^ ~b) & L::MSB);
}

// Full-lane mask from each lane's compare bit (the other bits are junk):
// one byte permute for 8- and 16-bit lanes; for 10-bit lanes the compare
// bits are isolated and multiplied out, (t & MSB) / 2^9 * 0x3FF, as a high
// and a low multiply with run-time factors (FMA pipe).
template <class L>
__device__ __forceinline__ uint32_t spread(uint32_t t, uint32_t sph, uint32_t spl)
{
    if (L::BITS == 10) return mad_lo(mul_hi(t & L::MSB, sph), spl, 0u);
    return prmt(t, 0u, L::SIGNREP);
}

// Row register for rows r = 1..RPW-1 past an aligned word: the lanes start r
// characters further into the x stream, i.e. the 64-bit pair (b:a) shifted
// right by 8r bits = (a >> 8r) | (b << (32 - 8r)).  Both halves are integer
// multiplies by s = 2^(32 - 8r) (high and low word), so the shift runs on the
// FMA pipe and leaves the ALU pipe to the cells.
// (For 10-bit lanes the low-word factor is 2^(30 - 10r), a separate s_lo.)
__device__ __forceinline__ uint32_t row_shift(uint32_t a, uint32_t b, uint32_t s, uint32_t s_lo)
{
    return mad_lo(b, s_lo, mul_hi(a, s));
}

// Mismatch flags of one aligned word: lane MSB set iff x != y (any byte
// values).  ((e & LOW) + LOW) has its MSB set iff the low bits of e are
// nonzero, and never carries across lanes.  OR-ing e adds the top bit.  The
// add is a multiply-add by one (FMA pipe).
template <class L>
__device__ __forceinline__ uint32_t mismatch_word(uint32_t xw, uint32_t yb, uint32_t one)
{
    return mad_lo((xw ^ yb) & L::LOW, one, L::LOW) | (xw ^ yb);
}

// Full-lane mismatch mask of one aligned word: 0xFF.. in lanes where x != y.
// When x ^ y can never have the lane's top bit, (x ^ y) + LOW alone flags
// the mismatches (one logic instruction fewer):
// * 10- and 16-bit lanes: the characters are bytes;
// * ST (same top bit): every character the tile compares is below 128, or
//   every one is at least 128 (checked per tile by tile_same_top).
template <class L, bool ST = false>
__device__ __forceinline__ uint32_t mismatch_mask(uint32_t xw, uint32_t yb, uint32_t one,
                                                  uint32_t sph, uint32_t spl)
{
    if (ST || L::BITS != 8) return spread<L>(mad_lo(xw ^ yb, one, L::LOW), sph, spl);
    return spread<L>(mismatch_word<L>(xw, yb, one), sph, spl);
}

// One comb cell on NS strips at once.
//   h: seaweed entering from the left (stays in the row register),
//   v: seaweed entering from the top (travels down the column),
//   mm: full-lane mask, all ones where the cell is a mismatch (a padding row
//   is all ones: it never matches).
// Bottom output = h where (match or h >= v), else v; right output = other.
// The match is folded into the left key, hc = h | 0x80 in mismatch lanes and
// 0xFF in match lanes, so one subtraction hc - v (a multiply-add on the FMA
// pipe) gives the swap decision in each lane's top bit: always in a match
// lane, and h >= v otherwise (keys are at most 0x7F.., no borrow between
// lanes).  hc does not depend on v, so the dependency chain from one cell to
// the next is three instructions: subtract, sign-spread, select.
//
// With full 8-bit keys (U8FLanes) the top bit belongs to the key, so the
// match is folded in as hm = 0xFF in match lanes (>= any key) and the swap
// decision is the full-width compare hm >= v.
#ifndef AP_GEN_MM
// 1: 16-bit lanes form both outputs with 16x2 min/max (see cell).  Measured
// against the logic cells: {2,1,0} on 40k DNA, w = 200, 177.7 -> 127.6 ms;
// {3,1,0}, 30k, w = 100, 125.5 -> 96.8 ms; LCS on 40k protein, w = 300,
// 98.0 -> 92.5 ms; LCS step 5, 60k DNA, w = 300, 51.2 -> 49.1 ms.
#define AP_GEN_MM 1
#endif

#ifndef AP_GEN_HNF8
// 1: full 8-bit keys in the general path form the right output as
// (h + v) - bottom on the FMA pipe (exact, as in the table path): 40k
// protein, w = 200, 47.1 -> 45.5 ms; 60k DNA with step 5, w = 200, 22.5 ->
// 22.1 ms.
#define AP_GEN_HNF8 1
#endif

template <class L>
__device__ __forceinline__ void cell(uint32_t &h, uint32_t &v, uint32_t mm, uint32_t neg1,
                                     uint32_t sph, uint32_t spl, uint32_t one = 1u)
{
    if constexpr (AP_GEN_MM != 0 && L::BITS == 16) {
        // 16-bit lanes: the key's top bit is free, so hc = h + 0x8000 in match
        // lanes exceeds every key: bottom = max(hc, v) without that bit,
        // right = min(hc, v); elsewhere the larger key goes down.
        const uint32_t hc = h | (~mm & L::MSB);
        const uint32_t b = max_u16x2(hc, v);
        h = min_u16x2(hc, v);
        v = b & L::LOW;
        return;
    }
    uint32_t M;
    if (L::FULL) {
        const uint32_t hm = h | ~mm;
        M = prmt(ge_lanes<L>(hm, v, neg1), 0u, L::SIGNREP);
    } else {
        const uint32_t hc = h | ~mm | L::MSB;   // (10-bit lanes: bits 30-31 are junk, never read)
        const uint32_t t = mad_lo(v, neg1, hc);  // hc - v
        M = spread<L>(t, sph, spl);
    }
    const uint32_t vn = (h & M) | (v & ~M);
    if (L::FULL && AP_GEN_HNF8 != 0) h = mad_lo(vn, neg1, mad_lo(h, one, v));
    else h = h ^ v ^ vn;
    v = vn;
}

// Mismatch cell (no match possible): swap iff h >= v.
template <class L>
__device__ __forceinline__ void cell_mismatch(uint32_t &h, uint32_t &v, uint32_t neg1,
                                              uint32_t sph, uint32_t spl)
{
    if constexpr (AP_GEN_MM != 0 && L::BITS == 16) {
        const uint32_t b = max_u16x2(h, v);
        h = min_u16x2(h, v);
        v = b;
        return;
    }
    const uint32_t M = L::FULL ? prmt(ge_lanes<L>(h, v, neg1), 0u, L::SIGNREP)
                               : spread<L>(h - v + L::MSB, sph, spl);
    const uint32_t vn = (h & M) | (v & ~M);
    h = h ^ v ^ vn;
    v = vn;
}

// Keys drop by rr, saturating at 0.  rr_bias = (half - rr) per lane for
// keys below half; rrv = rr per lane for full-width keys.
template <class L>
__device__ __forceinline__ uint32_t renorm_key(uint32_t k, uint32_t rr_bias, uint32_t rrv,
                                               uint32_t one, uint32_t neg1, uint32_t sph,
                                               uint32_t spl)
{
    if (L::FULL) {
        const uint32_t M = prmt(ge_lanes<L>(k, rrv, neg1), 0u, L::SIGNREP);
        return sub_lanes<L>(k, rrv) & M;
    }
    uint32_t t = mad_lo(k, one, rr_bias);     // lane: k + (half - rr), MSB iff k >= rr
    uint32_t M = spread<L>(t, sph, spl);
    return t & M & L::LOW;
}

// ---------------------------------------------------------------------------
// Output staging flush
// ---------------------------------------------------------------------------
//
// stage[jj * (NGRP + 1) + grp] holds, for staged plot column jj, the NS values
// of group grp's strips (one per lane).  The warp writes `cnt` columns
// starting at plot column jbase for its SPW strip rows.
//
// One-thread strip groups with 8-bit lanes write full blocks of kOB = 32
// columns into 16-byte aligned rows with 16-byte stores:
// * byte plots (LCS kernels): two threads pack 16 columns each of one row;
//   measured against 4-byte stores on 100k DNA plots, w = 16: 21.9 -> 19.2
//   ms, w = 32: 38.5 -> 34.8 ms, w = 100: 89.2 -> 87.6 ms;
// * 16-bit plots (score kernels, WIDE): four threads pack 8 columns each;
//   the 20k protein score plot went 6.20 -> 6.05 ms.
// (One routine for both widths and all group sizes cost registers and was
// slower.)  Other blocks use 4-byte (8-bit) or 8-byte (16-bit) stores, 8
// threads per row and 4 rows per pass, or a scalar path; each store
// instruction writes whole 32-byte sectors.
template <class L>
__device__ __forceinline__ uint32_t lane_of(uint32_t w, int b)
{
    return (w >> (L::BITS * b)) & L::MASK;
}

template <class L, int NGRP, bool WIDE = false>
__device__ __forceinline__ void flush_stage(const CombParams &p, const uint32_t *stage,
                                            int64_t iw, int64_t jbase, int cnt, int lane)
{
    constexpr int NS = L::NS;
    constexpr int SPW = NGRP * NS;
    // Output words are scaled lane by lane in one multiply: every lane's
    // product fits its lane (the output width was checked against scale x
    // the largest value), so no carry crosses a lane.
    const uint32_t sc = p.scale;
    if (WIDE && L::BITS == 8 && NGRP == 32 && p.out_bytes == 2 && cnt == kOB &&
        ((((uintptr_t)p.out) | (uintptr_t)(2 * p.ld)) & 15u) == 0) {
        // byte values widened to 16 bits: four threads per row (8 columns
        // each), 8 rows per pass
        const int part = lane & 3, rp = lane >> 2;
#pragma unroll 1
        for (int it = 0; it < SPW / 8; ++it) {
            const int rw = it * 8 + rp;
            const int64_t i = iw + rw;
            const int grp = rw / NS;
            const uint32_t b = (uint32_t)(rw % NS);
            const uint32_t *sp = stage + (8 * part) * (NGRP + 1) + grp;
            uint32_t wv[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) wv[c] = sp[c * (NGRP + 1)];
            const uint32_t sel = b | ((b + 4u) << 4);
            uint32_t o4[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) o4[k] = prmt(prmt(wv[2 * k], wv[2 * k + 1], sel), 0u, 0x4140u) * sc;
            if (i < p.rows && AP_CHECK(p, jbase + 8 * part + 8 <= p.cols, kDbgPlotStore))
                *(uint4 *)((uint16_t *)p.out + i * p.ld + jbase + 8 * part) =
                    make_uint4(o4[0], o4[1], o4[2], o4[3]);
        }
        return;
    }
    if (!WIDE && L::BITS == 8 && NGRP == 32 && p.out_bytes == 1 && cnt == kOB &&
        ((((uintptr_t)p.out) | (uintptr_t)p.ld) & 15u) == 0) {
        // two threads per row (16 columns each), 16 rows per pass
        const int half = lane & 1, rp = lane >> 1;
#pragma unroll 1
        for (int it = 0; it < SPW / 16; ++it) {
            const int rw = it * 16 + rp;
            const int64_t i = iw + rw;
            const int grp = rw / NS;
            const uint32_t b = (uint32_t)(rw % NS);
            const uint32_t *sp = stage + (16 * half) * (NGRP + 1) + grp;
            uint32_t wv[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) wv[c] = sp[c * (NGRP + 1)];
            const uint32_t sel = b | ((b + 4u) << 4);
            uint32_t o4[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                o4[k] = prmt(prmt(wv[4 * k], wv[4 * k + 1], sel), prmt(wv[4 * k + 2], wv[4 * k + 3], sel),
                             0x5410u) * sc;
            if (i < p.rows && AP_CHECK(p, jbase + 16 * half + 16 <= p.cols, kDbgPlotStore))
                *(uint4 *)((uint8_t *)p.out + i * p.ld + jbase + 16 * half) =
                    make_uint4(o4[0], o4[1], o4[2], o4[3]);
        }
        return;
    }
    if (p.vec_ok) {
        const int cb = lane & 7;
        const int j4 = 4 * cb;
#pragma unroll 1
        for (int it = 0; it < SPW / 4; ++it) {
            const int rw = it * 4 + (lane >> 3);
            const int64_t i = iw + rw;
            if (i >= p.rows || j4 >= cnt) continue;
            if (!AP_CHECK(p, jbase + (j4 + 4 <= cnt ? j4 + 4 : cnt) <= p.cols, kDbgPlotStore)) continue;
            const int grp = rw / NS, b = rw % NS;
            const uint32_t *sp = stage + j4 * (NGRP + 1) + grp;
            const uint32_t w0 = sp[0], w1 = sp[NGRP + 1], w2 = sp[2 * (NGRP + 1)], w3 = sp[3 * (NGRP + 1)];
            const int64_t off = i * p.ld + jbase + j4;
            if (L::BITS == 10) {                // lanes are not byte-aligned: shift out
                const uint32_t v0 = lane_of<L>(w0, b) * sc, v1 = lane_of<L>(w1, b) * sc;
                const uint32_t v2 = lane_of<L>(w2, b) * sc, v3 = lane_of<L>(w3, b) * sc;
                if (p.out_bytes == 1) {
                    uint8_t *o = (uint8_t *)p.out + off;
                    const uint32_t word = v0 | (v1 << 8) | (v2 << 16) | (v3 << 24);
                    if (j4 + 4 <= cnt) {
                        *(uint32_t *)o = word;
                    } else {
                        for (int t = 0; t < cnt - j4; ++t) o[t] = (uint8_t)(word >> (8 * t));
                    }
                } else {
                    uint16_t *o = (uint16_t *)p.out + off;
                    if (j4 + 4 <= cnt) {
                        *(uint2 *)o = make_uint2(v0 | (v1 << 16), v2 | (v3 << 16));
                    } else {
                        const uint32_t v4[4] = {v0, v1, v2, v3};
                        for (int t = 0; t < cnt - j4; ++t) o[t] = (uint16_t)v4[t];
                    }
                }
                continue;
            }
            // byte index of lane b's low byte inside a staged word
            const uint32_t bb = (uint32_t)(b * (L::BITS / 8));
            if (p.out_bytes == 1) {
                const uint32_t sel = bb | ((bb + 4u) << 4);
                const uint32_t lo = prmt(w0, w1, sel), hi = prmt(w2, w3, sel);
                const uint32_t word = prmt(lo, hi, 0x5410u) * sc;
                uint8_t *o = (uint8_t *)p.out + off;
                if (j4 + 4 <= cnt) {
                    *(uint32_t *)o = word;
                } else {
                    for (int t = 0; t < cnt - j4; ++t) o[t] = (uint8_t)(word >> (8 * t));
                }
            } else {
                uint32_t lo, hi;
                if (L::BITS == 8) {
                    const uint32_t sel = bb | ((bb + 4u) << 4);
                    lo = prmt(prmt(w0, w1, sel), 0u, 0x4140u) * sc;
                    hi = prmt(prmt(w2, w3, sel), 0u, 0x4140u) * sc;
                } else {
                    const uint32_t sel = bb | ((bb + 1u) << 4) | ((bb + 4u) << 8) | ((bb + 5u) << 12);
                    lo = prmt(w0, w1, sel) * sc;
                    hi = prmt(w2, w3, sel) * sc;
                }
                uint16_t *o = (uint16_t *)p.out + off;
                if (j4 + 4 <= cnt) {
                    *(uint2 *)o = make_uint2(lo, hi);
                } else {
                    const uint32_t v4[4] = {lo & 0xFFFFu, lo >> 16, hi & 0xFFFFu, hi >> 16};
                    for (int t = 0; t < cnt - j4; ++t) o[t] = (uint16_t)v4[t];
                }
            }
        }
    } else {
#pragma unroll 1
        for (int rw = 0; rw < SPW; ++rw) {
            const int64_t i = iw + rw;
            if (i >= p.rows) break;
            if (lane < cnt && AP_CHECK(p, jbase + lane < p.cols, kDbgPlotStore)) {
                const uint32_t v = lane_of<L>(stage[lane * (NGRP + 1) + rw / NS], rw % NS) * sc;
                const int64_t off = i * p.ld + jbase + lane;
                if (p.out_bytes == 1) ((uint8_t *)p.out)[off] = (uint8_t)v;
                else ((uint16_t *)p.out)[off] = (uint16_t)v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------
//
// L      lane format (U8Lanes, U8FLanes, U10Lanes or U16Lanes)
// R      physical comb rows held by each thread
// G      threads per strip group (the strip's rows are split over them)
// NU, MU blow-up of the score scheme {NU, MU, 0}: every character becomes
//        MU '$' followed by NU - MU copies of itself (Section 2 for {2,1,0});
//        NU = 1 is LCS; MU = -1 takes the '$' count from p.mu at run time
//        (one kernel for every MU of a NU)
// PADU   trailing units (rows for LCS, row groups of NU otherwise) of each
//        thread that may be padding (never match)
// XR     vertical step: plot row r is the x-window at r * step, so the NS
//        strips of a register are not neighbours; each thread then keeps one
//        x word per unit (gathered once per tile) and computes each unit's
//        match mask directly instead of lane-shifting shared masks
// ST     every character this tile compares shares the top bit: the short
//        mismatch test is exact (chosen per tile by comb_tile_dispatch)
//
// Each step combs two physical columns, interleaved row by row, so a thread
// always has two independent dependency chains:
//   LCS:   columns 2u and 2u+1 (unit u = two plot columns, keys per column);
//   score: the '$' column and the character column of y' pair u (keys per pair).
// Threads of a strip group are skewed by one step: thread g works on unit
// u = s - g and takes its top seaweeds from thread g-1 by warp shuffle.
template <class L, int R, int G, int NU, int MU, int PADU, bool XR, bool ST = false>
__device__ __forceinline__ void comb_tile(const CombParams &p, int64_t sg, int64_t ch,
                                          uint32_t *ring)
{
    constexpr bool SCORE = NU > 1;
    constexpr int NS = L::NS;
    constexpr int NGRP = 32 / G;
    constexpr int SPW = NGRP * NS;                    // strips per warp
    constexpr int RP = R / NU;                        // x characters (units) per thread
    constexpr int NQ = XR ? RP : RP / L::RPW + 1;     // x words (aligned, or one per unit)
    static_assert(NU >= 1 && MU >= -1 && MU < NU && (NU > 1 || MU == 0), "bad blow-up");
    static_assert(XR ? (R % NU == 0) : (R % (NU * L::RPW) == 0),
                  "R must fill whole units (vertical step) or whole x words");
    static_assert(PADU <= RP, "padding window larger than the lane");

    const int lane = threadIdx.x & 31;
    const int g = (G == 1) ? 0 : (lane % G);
    const int grp = lane / G;
    uint32_t *stage = ring + p.ring * NGRP;

    const int64_t iw = sg * SPW;                  // first strip of the warp
    const int64_t ig = iw + (int64_t)grp * NS;    // first strip of the group
    const int64_t c0 = ch * p.chunk;
    const int64_t c1 = (c0 + p.chunk < p.cols) ? c0 + p.chunk : p.cols;
    const int wk = p.w;                            // window, in key units

    // x rows (LCS) or pairs (score) held by this thread: [ub, ub + nreal).
    const int ub = (g * wk) / G;
    const int nreal = ((g + 1) * wk) / G - ub;

    // x words: the aligned words of this thread's stream x[ig + ub ...], or
    // (vertical step) unit q's character of each of the NS strips.
    uint32_t xw[NQ];
    if (!XR) {
        const int64_t base = ig + ub;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            uint32_t wv = 0;
#pragma unroll
            for (int t = 0; t < L::RPW; ++t) {
                const int64_t idx = base + q * L::RPW + t;
                const uint32_t c = (idx < p.m && AP_CHECK(p, idx >= 0, kDbgXRead)) ? (uint32_t)__ldg(p.x + idx) : 0u;
                wv |= c << (L::BITS * t);
            }
            xw[q] = wv;
        }
    } else {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            uint32_t wv = 0;
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                const int64_t idx = (ig + b) * p.step + ub + q;
                const uint32_t c = (idx < p.m && AP_CHECK(p, idx >= 0, kDbgXRead)) ? (uint32_t)__ldg(p.x + idx) : 0u;
                wv |= c << (L::BITS * b);
            }
            xw[q] = wv;
        }
    }
    // Padding masks for the last PADU units of the thread (all ones: the
    // row never matches).
    uint32_t padm[PADU > 0 ? PADU : 1];
#pragma unroll
    for (int t = 0; t < PADU; ++t)
        padm[t] = ((RP - PADU + t) >= nreal) ? 0xFFFFFFFFu : 0u;

    for (int e = lane; e < p.ring * NGRP; e += 32) ring[e] = 0u;
    __syncwarp();

    uint32_t h[R];
#pragma unroll
    for (int k = 0; k < R; ++k) h[k] = 0u;

    // Columns (LCS) or pairs (score) combed by this tile (chunks are capped at
    // 2^30 columns, so tile-local indices fit in 32 bits).
    const int ncomb = (int)(c1 - c0) + wk - 1;
    const int nunits = SCORE ? ncomb : (ncomb + 1) / 2;
    const int steps = nunits + G - 1;
    const uint32_t wvec = (uint32_t)(NU * wk) * L::ONES;
    const uint32_t inval_bias = (uint32_t)((1u << (L::BITS - 1)) - (uint32_t)wk) * L::ONES;
    const int kdrop = SCORE ? p.renorm : 2 * p.renorm;
    const uint32_t rr_bias = (uint32_t)((1u << (L::BITS - 1)) - (uint32_t)kdrop) * L::ONES;
    const uint32_t rrv = (uint32_t)kdrop * L::ONES;
    const uint32_t wkv = (uint32_t)wk * L::ONES;
    const int ring_mask = p.ring - 1;
    const uint32_t ring_maskv = (uint32_t)ring_mask * L::ONES;
    const int plot_cols = (int)(c1 - c0);
    const uint8_t *ytile = p.y + c0;                  // y of this tile
    const int ylast = (int)(p.n - 1 - c0);            // last valid index into ytile

    const uint32_t one = p.one;
    const uint32_t neg1 = 0u - p.one;
    const uint32_t sh1 = p.shmul[1], sh2 = p.shmul[2], sh3 = p.shmul[3];
    const uint32_t sl1 = p.shlo[1], sl2 = p.shlo[2], sl3 = p.shlo[3];
    const uint32_t sph = p.spread_hi, spl = p.spread_lo;
    // multipliers of the shift for rows r = 1..RPW-1 past an aligned word
    // (16-bit lanes: r = 1 is a 2-byte shift)
    auto shm = [&](int r) -> uint32_t {
        return (L::BITS == 16) ? sh2 : (r == 1 ? sh1 : (r == 2 ? sh2 : sh3));
    };
    auto shl = [&](int r) -> uint32_t {
        return (L::BITS == 16) ? sl2 : (r == 1 ? sl1 : (r == 2 ? sl2 : sl3));
    };

    int kc = wk;        // key of the first seaweed starting in this thread's unit
    int since = 0;      // steps since the last renormalisation
    uint32_t d = 0;     // per strip: seaweeds counted in the current window
    uint32_t vdown[NU > 1 ? NU : 2];
#pragma unroll
    for (int c = 0; c < (NU > 1 ? NU : 2); ++c) vdown[c] = 0u;

    // Exit counting (Theorem 3.1's queue B as a ring of "left validly" flags,
    // one byte per strip, indexed by start column (LCS) or pair (score)).
    //
    // 8-bit keys: keys never exceed ring - 1 (the plan derives the key range
    // from the ring size), so every age is below the ring size.  An exit too
    // old for the window (age >= w) then maps to the slot of a start older
    // than the window, which is already zero and is next read only after a
    // later start re-uses it.  Storing its zero flag there is harmless, so
    // the update needs no branch: each strip stores its 0/1 flag.  The four
    // slots come from one byte-wise subtraction.
    uint8_t *ring8 = (uint8_t *)(ring + grp);
    auto count_exit = [&](uint32_t ex, uint32_t knew, int col) {
        const uint32_t age = knew - ex;                       // per lane, >= 0
        const uint32_t inval = (L::FULL ? ge_lanes<L>(age, wkv, neg1)
                                        : age + inval_bias) & L::MSB;   // age >= w
        const uint32_t valid = (inval ^ L::MSB) >> (L::BITS - 1);
        d += valid;
        if (L::BITS == 8) {
            const uint32_t colb = (uint32_t)(col & ring_mask) * L::ONES;
            // (col - age) mod ring per lane (the ring has 256 slots with full keys)
            const uint32_t slots = L::FULL ? sub_lanes<L>(colb, age)
                                           : (colb + L::MSB - age) & ring_maskv;
            // every byte of slots is already a slot number (< ring), and
            // every byte of valid is 0 or 1: one byte permute extracts each
            // (LCS; the score kernels keep shifts, which cost them fewer
            // registers)
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                const uint32_t slot = SCORE ? (slots >> (8 * b)) & (uint32_t)ring_mask
                                            : prmt(slots, 0u, 0x4440u | (uint32_t)b);
                if (!AP_CHECK(p, slot < (uint32_t)p.ring, kDbgRing)) continue;
                uint8_t *e = ring8 + slot * (uint32_t)(NGRP * 4) + b;
                const uint8_t f = SCORE ? (uint8_t)((valid >> (8 * b)) & 1u)
                                        : (uint8_t)prmt(valid, 0u, 0x4440u | (uint32_t)b);
                if (SCORE) *e = (uint8_t)(*e + f);
                else *e = f;
            }
        } else {
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                if ((valid >> (L::BITS * b)) & 1u) {
                    const int a = (int)((age >> (L::BITS * b)) & L::MASK);
                    uint32_t *e = ring + ((col - a) & ring_mask) * NGRP + grp;
                    *e += 1u << (L::BITS * b);
                }
            }
        }
    };
    auto expire = [&](int col) {            // start `col - w` leaves the window
        // (8-bit keys: for col < w the slot belongs to a future start and is 0)
        if (L::BITS == 8 || col >= wk) {
            uint32_t *e = ring + ((col - wk) & ring_mask) * NGRP + grp;
            d -= *e;
            *e = 0u;
        }
    };
    auto stage_out = [&](int col) {
        if (col >= wk - 1 && col < ncomb) {
            // col >= w - 1 here, so the two forms agree; each is the one that
            // measured faster for its kernel family (register allocation)
            const int jj = SCORE ? (col - (wk - 1)) % kOB
                                 : (int)((uint32_t)(col - (wk - 1)) & (kOB - 1));
            stage[jj * (NGRP + 1) + grp] = wvec - d;
        }
    };
    auto maybe_flush = [&](int col) {       // uniform across the warp
        if (col >= wk - 1 && col < ncomb) {
            const int jo = col - (wk - 1);
            const int jm = SCORE ? jo % kOB : (jo & (kOB - 1));   // jo >= 0
            if (jm == kOB - 1 || jo == plot_cols - 1) {
                __syncwarp();
                const int cnt = jm + 1;
                flush_stage<L, NGRP, (NU > 1)>(p, stage, iw, c0 + jo - (cnt - 1), cnt, lane);
                __syncwarp();
            }
        }
    };
    // One thread per strip group: every column it reads lies inside y (the
    // last column a tile combs, plus the odd padding column of a two-column
    // step, is at most n - 1).  Skewed threads clamp.
    auto ychar = [&](int yi) -> uint32_t {
        if (G > 1) yi = yi < 0 ? 0 : (yi > ylast ? ylast : yi);
        if (!AP_CHECK(p, yi >= 0 && yi <= ylast, kDbgYRead)) return 0u;
        return (uint32_t)__ldg(ytile + yi);
    };

    for (int s = 0; s < steps; ++s) {
        const int u = s - g;              // this thread's unit
        if (u > 0) {
            kc += SCORE ? 1 : 2;
            if (++since == p.renorm) {     // Proposition 3.4: old keys collapse to 0
#pragma unroll
                for (int k = 0; k < R; ++k) h[k] = renorm_key<L>(h[k], rr_bias, rrv, one, neg1, sph, spl);
                kc = wk;
                since = 0;
            }
        }
        const uint32_t knew0 = (uint32_t)kc * L::ONES;
        const uint32_t knew1 = SCORE ? knew0 : knew0 + L::ONES;

        if (!SCORE) {
            uint32_t va, vb;              // top seaweeds of the two columns
            if (G > 1) {
                const uint32_t in0 = __shfl_up_sync(0xffffffffu, vdown[0], 1);
                const uint32_t in1 = __shfl_up_sync(0xffffffffu, vdown[1], 1);
                va = (g == 0) ? knew0 : in0;
                vb = (g == 0) ? knew1 : in1;
            } else {
                va = knew0;
                vb = knew1;
            }
            const uint32_t yb0 = ychar(2 * u) * L::ONES;
            const uint32_t yb1 = ychar(2 * u + 1) * L::ONES;
            uint32_t mm0[XR ? 1 : NQ], mm1[XR ? 1 : NQ];
            if (!XR) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    mm0[q] = mismatch_mask<L, ST>(xw[q], yb0, one, sph, spl);
                    mm1[q] = mismatch_mask<L, ST>(xw[q], yb1, one, sph, spl);
                }
            }
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const int q = k / L::RPW, r = k % L::RPW;
                uint32_t m0, m1;
                if (XR) {
                    m0 = mismatch_mask<L, ST>(xw[k], yb0, one, sph, spl);
                    m1 = mismatch_mask<L, ST>(xw[k], yb1, one, sph, spl);
                } else {
                    m0 = (r == 0) ? mm0[q] : row_shift(mm0[q], mm0[q + 1], shm(r), shl(r));
                    m1 = (r == 0) ? mm1[q] : row_shift(mm1[q], mm1[q + 1], shm(r), shl(r));
                }
                const int pi = k - (R - PADU);
                if (pi >= 0) {
                    m0 |= padm[pi < 0 ? 0 : pi];
                    m1 |= padm[pi < 0 ? 0 : pi];
                }
                cell<L>(h[k], va, m0, neg1, sph, spl, one);
                cell<L>(h[k], vb, m1, neg1, sph, spl, one);
            }
            vdown[0] = va;
            vdown[1] = vb;
        } else {
            // One unit of y': MU '$' columns, then NU - MU columns of y[u].  Rows
            // come in units of NU: MU '$' rows, then NU - MU rows of the x
            // character.  '$' meets '$': match (unless padding); '$' meets a
            // character: mismatch; character meets character: compare.
            uint32_t v[NU];
#pragma unroll
            for (int c = 0; c < NU; ++c) {
                if (G > 1) {
                    const uint32_t in = __shfl_up_sync(0xffffffffu, vdown[c], 1);
                    v[c] = (g == 0) ? knew0 : in;
                } else {
                    v[c] = knew0;
                }
            }
            const uint32_t yb = ychar(u) * L::ONES;
            uint32_t mm[XR ? 1 : NQ];
            if (!XR) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) mm[q] = mismatch_mask<L, ST>(xw[q], yb, one, sph, spl);
            }
#pragma unroll
            for (int q = 0; q < RP; ++q) {
                const int pi = q - (RP - PADU);
                const uint32_t pad = (pi >= 0) ? padm[pi < 0 ? 0 : pi] : 0u;
                const int qq = q / L::RPW, r = q % L::RPW;
                uint32_t mq = XR ? mismatch_mask<L, ST>(xw[q], yb, one, sph, spl)
                                 : ((r == 0) ? mm[qq] : row_shift(mm[qq], mm[qq + 1], shm(r), shl(r)));
                if (pi >= 0) mq |= pad;
#pragma unroll
                for (int rho = 0; rho < NU; ++rho) {
                    const int k = NU * q + rho;
#pragma unroll
                    for (int c = 0; c < NU; ++c) {
                        if constexpr (MU < 0) {
                            // '$' rows and columns known at run time only
                            // (uniform over the launch): select the cell's mask
                            const bool rd = rho < p.mu, cd = c < p.mu;
                            const uint32_t m = (rd && cd) ? pad : ((rd != cd) ? 0xFFFFFFFFu : mq);
                            cell<L>(h[k], v[c], m, neg1, sph, spl, one);
                            continue;
                        }
                        const bool row_dollar = rho < MU, col_dollar = c < MU;
                        if (row_dollar && col_dollar) {
                            if (pi >= 0) {
                                cell<L>(h[k], v[c], pad, neg1, sph, spl, one);
                            } else {
                                const uint32_t tmp = h[k];
                                h[k] = v[c];
                                v[c] = tmp;
                            }
                        } else if (row_dollar != col_dollar) {
                            cell_mismatch<L>(h[k], v[c], neg1, sph, spl);
                        } else {
                            cell<L>(h[k], v[c], mq, neg1, sph, spl, one);
                        }
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < NU; ++c) vdown[c] = v[c];
        }

        // ---- bottom threads: count exits (Theorem 3.1) and stage the plot ----
        const int ubot = s - (G - 1);       // the bottom threads' unit (warp-uniform)
        const bool bottom = (g == G - 1) && u >= 0 && u < nunits;
        if (!SCORE) {
            const int col0 = 2 * ubot, col1 = 2 * ubot + 1;
            if (bottom) {
                expire(col0);
                count_exit(vdown[0], knew0, col0);
                stage_out(col0);
            }
            if (ubot >= 0) maybe_flush(col0);
            if (bottom && col1 < ncomb) {
                expire(col1);
                count_exit(vdown[1], knew1, col1);
                stage_out(col1);
            }
            if (ubot >= 0) maybe_flush(col1);
        } else {
            if (bottom) {
                expire(ubot);
#pragma unroll
                for (int c = 0; c < NU; ++c) count_exit(vdown[c], knew0, ubot);
                stage_out(ubot);
            }
            if (ubot >= 0) maybe_flush(ubot);
        }
    }
}

// Shared-memory words one warp needs for a tile: the exit ring plus the
// output stage (variants with match tables add tab_words(R)).
template <int G>
__host__ __device__ constexpr int comb_warp_words(int ring)
{
    return ring * (32 / G) + kOB * (32 / G + 1);
}

// True if every character the tile compares has the same top bit (all
// below 128, or all at least 128): the x positions from its first strip's
// window to its last strip's (with a vertical step, the gaps between them
// too) and the y positions of its columns and warm-up.  Warp-uniform; it
// reads about (chunk + w) / 32 bytes per lane, once per tile.
template <class L, int G>
__device__ __forceinline__ bool tile_same_top(const CombParams &p, int64_t sg, int64_t ch)
{
    constexpr int SPW = (32 / G) * L::NS;
    const int lane = threadIdx.x & 31;
    const int64_t iw = sg * SPW;
    const int64_t c0 = ch * p.chunk;
    const int64_t c1 = (c0 + p.chunk < p.cols) ? c0 + p.chunk : p.cols;
    const int64_t xe = (iw + SPW - 1) * p.step + p.w;      // past the last strip's window
    const int64_t x1 = (xe < p.m) ? xe : p.m;
    const int64_t y1 = (c1 + p.w - 1 < p.n) ? c1 + p.w - 1 : p.n;
    uint32_t o = 0u, a = 0xFFu;
    for (int64_t i = iw * p.step + lane; i < x1; i += 32) {
        const uint32_t c = __ldg(p.x + i);
        o |= c;
        a &= c;
    }
    for (int64_t j = c0 + lane; j < y1; j += 32) {
        const uint32_t c = __ldg(p.y + j);
        o |= c;
        a &= c;
    }
    o = __reduce_or_sync(0xffffffffu, o);
    a = __reduce_and_sync(0xffffffffu, a);
    return (o & 0x80u) == 0u || (a & 0x80u) != 0u;
}

// ---------------------------------------------------------------------------
// Match tables for small alphabets (LCS, 7-bit keys, one thread per strip
// group)
// ---------------------------------------------------------------------------
//
// A row register of thread `grp` at row k holds the strips iw + 4 grp + b
// (b = 0..3), whose row-k characters are x[iw + 4 grp + k + b]: the four
// characters at warp position p = 4 grp + k.  The match word of that row
// against a y character c is a function of p and c alone, so a warp whose x
// characters (all SPW + R + 3 of them) take at most kTabSyms distinct values
// keeps, in shared memory, one word per (symbol, position):
//     T[s][p] byte b = 0xFF if x[iw + p + b] == sym[s], else 0x80
// (slot kTabSyms: every byte 0x80, for y characters absent from the warp's
// x).  That is the "h | ~mismatch | MSB" operand of the cell: the column's
// row masks become one 16-byte shared load per four rows, with no compare,
// spread or row shift per column.  A y character's slot comes from a
// 256-entry byte map.  Warps with more distinct characters take the general
// path.
constexpr int kTabSyms = 4;

__host__ __device__ constexpr int tab_positions(int R) { return 4 * 31 + R; }

// Shared words of the tables: (kTabSyms + 1) tables, the y map (256 bytes),
// the presence bit set (8 words) and the symbols (8 bytes).
__host__ __device__ constexpr int tab_words(int R)
{
    return ((kTabSyms + 1) * tab_positions(R) + 64 + 8 + 2 + 3) / 4 * 4;   // keeps 16-byte alignment
}

// Which compiled variants carry the table path.
__host__ __device__ constexpr bool has_tables(int key_bits, int groups, int nu, bool xrows)
{
    return key_bits == 7 && groups == 1 && nu == 1 && !xrows;
}

#ifndef AP_TAB_CPS
#define AP_TAB_CPS 2   // plot columns per step of the table path (2 to 4)
#endif
#ifndef AP_TAB_SEL
// 1: the one-thread tables hold byte-permute selectors (match: take 0xFF from
// a constant; mismatch: spread the compare's sign bit) instead of OR masks,
// so that h | 0x80 becomes a multiply-add and the cell has one logic
// instruction fewer (see cell_sel).  Measured on the 100k DNA plot, w = 100,
// comb alone: 59.3 ms, against 62.2 ms for OR masks.
#define AP_TAB_SEL 1
#endif
#ifndef AP_TAB_HNF
// Columns of each step whose right output is formed on the FMA pipe.  With OR
// masks one of the two was best (62.2 ms against 65.3 ms for none and 65.9 ms
// for both); with selectors, whose h + 0x80.. already runs on the FMA pipe,
// none (59.3 ms against 65.5 ms for one and 71.2 ms for both).  Finer mixes
// lost as well: the FMA right output on every third, fourth or sixth cell
// 62.0, 61.8 and 60.8 ms; every third cell on the ALU pipe alone (t by one
// three-input add) and the others wholly on the FMA pipe 62.6 ms.  The fewest
// issued instructions win, not the balance of the two pipes.
#define AP_TAB_HNF 0
#endif

// Builds the warp's tables; false (warp-uniform) if the x characters of the
// warp take more than kTabSyms values.
template <int R, bool SEL = false>
__device__ __forceinline__ bool build_tables(const CombParams &p, int64_t iw, uint32_t *tab,
                                             int lane)
{
    constexpr int P = tab_positions(R);
    uint32_t *tb = tab;
    uint8_t *ymap = (uint8_t *)(tab + (kTabSyms + 1) * P);
    uint32_t *bits = tab + (kTabSyms + 1) * P + 64;
    uint8_t *sym = (uint8_t *)(bits + 8);
    if (lane < 8) bits[lane] = 0u;
    __syncwarp();
    // every x character a row of the warp reads: positions 0 .. P + 2
    for (int q = lane; q < P + 3; q += 32) {
        const int64_t idx = iw + q;
        if (idx < p.m) {
            const uint32_t c = __ldg(p.x + idx);
            atomicOr(&bits[c >> 5], 1u << (c & 31u));
        }
    }
    __syncwarp();
    const uint32_t wbits = (lane < 8) ? bits[lane] : 0u;
    const int cnt = __popc(wbits);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 7);
    if (total > kTabSyms) return false;
    // slot of every byte value: its rank among the present characters, or
    // kTabSyms if absent; lane l maps the bytes 8l .. 8l + 7 (word l / 4)
    const int before = __shfl_sync(0xffffffffu, incl - cnt, lane >> 2);
    const uint32_t wl = __shfl_sync(0xffffffffu, wbits, lane >> 2);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const uint32_t c = (uint32_t)(lane * 8 + t);
        const uint32_t bit = c & 31u;
        const bool present = (wl >> bit) & 1u;
        const int rank = before + __popc(wl & ((1u << bit) - 1u));
        ymap[c] = (uint8_t)(present ? rank : kTabSyms);
        if (present) sym[rank] = (uint8_t)c;
    }
    __syncwarp();
    for (int q = lane; q < P; q += 32) {
        uint32_t ch[4];
        bool in[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t idx = iw + q + b;
            in[b] = idx < p.m;
            ch[b] = in[b] ? (uint32_t)__ldg(p.x + idx) : 0u;
        }
        for (int s = 0; s < total; ++s) {
            const uint32_t c = sym[s];
            uint32_t wv = 0u;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const bool hit = in[b] && ch[b] == c;
                if (SEL) wv |= (hit ? 4u + b : 8u + b) << (4 * b);     // selector nibble of lane b
                else wv |= (hit ? 0xFFu : 0x80u) << (8 * b);
            }
            tb[s * P + q] = wv;
        }
        tb[kTabSyms * P + q] = SEL ? 0xBA98u : 0x80808080u;
    }
    __syncwarp();
    return true;
}

// One comb cell with the match folded in by a table word X (0xFF in match
// lanes, 0x80 in mismatch lanes; padding rows are masked to 0x80 by pk):
// hc = h | (X & pk), then as in cell<U8Lanes>.  FMA_HN forms the right
// output as (h + v) - bottom with two multiply-adds (lane sums stay below
// 256, so no carry or borrow crosses a lane) instead of one logic
// instruction (a compile-time constant after unrolling).
__device__ __forceinline__ void cell_tab(uint32_t &h, uint32_t &v, uint32_t X, uint32_t pk,
                                         uint32_t one, uint32_t neg1, bool FMA_HN)
{
    const uint32_t hc = h | (X & pk);
    const uint32_t t = mad_lo(v, neg1, hc);                 // hc - v
    const uint32_t M = prmt(t, 0u, U8Lanes::SIGNREP);
    const uint32_t vn = (h & M) | (v & ~M);
    if (FMA_HN) h = mad_lo(vn, neg1, mad_lo(h, one, v));
    else h = h ^ v ^ vn;
    v = vn;
}

// One comb cell with the match folded into the byte permute (selector tables,
// AP_TAB_SEL): t = (h + 0x80..) - v on the FMA pipe gives h >= v in each
// lane's top bit (keys are 7 bits: no carry or borrow crosses a lane); the
// selector S takes 0xFF from `ones` in match lanes and spreads t's sign bit
// in mismatch lanes, so M is the swap mask of cell_tab.
__device__ __forceinline__ void cell_sel(uint32_t &h, uint32_t &v, uint32_t S, uint32_t one,
                                         uint32_t neg1, uint32_t c80, bool FMA_HN)
{
    const uint32_t t = mad_lo(v, neg1, mad_lo(h, one, c80));
    const uint32_t M = prmt(t, 0xFFFFFFFFu, S);
    const uint32_t vn = (h & M) | (v & ~M);
    if (FMA_HN) h = mad_lo(vn, neg1, mad_lo(h, one, v));
    else h = h ^ v ^ vn;
    v = vn;
}

// 16-byte shared-memory load at a 32-bit shared address.
__device__ __forceinline__ uint4 lds128(uint32_t saddr)
{
    uint4 r;
    asm("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "r"(saddr));
    return r;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// The LCS comb of one tile through the tables (one thread per strip group,
// 7-bit keys in 8-bit lanes).  The same method, window count and output as
// comb_tile; CPS plot columns per step (CPS independent dependency chains per
// thread), each column's row words read from the table of its y character.
template <int R, int PADU, int CPS, int HNF, bool SEL = false>
__device__ __forceinline__ void comb_tile_tab(const CombParams &p, int64_t sg, int64_t ch,
                                              uint32_t *ring, const uint32_t *tab)
{
    using L = U8Lanes;
    constexpr int NS = 4;
    constexpr int NGRP = 32;
    constexpr int SPW = NGRP * NS;
    constexpr int P = tab_positions(R);
    static_assert(R % 4 == 0, "rows in whole x words");
    static_assert(CPS >= 2 && CPS <= 4, "two to four columns per step");
    static_assert(PADU <= R, "padding window larger than the lane");

    const int lane = threadIdx.x & 31;
    const int grp = lane;
    uint32_t *stage = ring + p.ring * NGRP;
    const uint8_t *ymap = (const uint8_t *)(tab + (kTabSyms + 1) * P);

    const int64_t iw = sg * SPW;
    const int64_t c0 = ch * p.chunk;
    const int64_t c1 = (c0 + p.chunk < p.cols) ? c0 + p.chunk : p.cols;
    const int wk = p.w;

    // padding rows never match: OR masks are ANDed with the no-match word,
    // selectors replaced by the all-mismatch selector (pk = 0 in those rows)
    uint32_t pk[PADU > 0 ? PADU : 1];
#pragma unroll
    for (int t = 0; t < PADU; ++t)
        pk[t] = ((R - PADU + t) >= wk) ? (SEL ? 0u : 0x80808080u) : 0xFFFFFFFFu;
    const uint32_t c80 = 0x80808080u;

    for (int e = lane; e < p.ring * NGRP; e += 32) ring[e] = 0u;
    __syncwarp();

    uint32_t h[R];
#pragma unroll
    for (int k = 0; k < R; ++k) h[k] = 0u;

    const int ncomb = (int)(c1 - c0) + wk - 1;
    const int steps = (ncomb + CPS - 1) / CPS;
    const uint32_t wvec = (uint32_t)wk * L::ONES;
    const uint32_t inval_bias = (uint32_t)(128u - (uint32_t)wk) * L::ONES;
    // renormalise every rsteps steps, by CPS * rsteps key units (p.renorm is
    // given for two-column steps)
    const int rsteps = (p.renorm * 2) / CPS;
    const int kdrop = CPS * rsteps;
    const uint32_t rr_bias = (uint32_t)(128u - (uint32_t)kdrop) * L::ONES;
    const int ring_mask = p.ring - 1;
    const uint32_t ring_maskv = (uint32_t)ring_mask * L::ONES;
    const int plot_cols = (int)(c1 - c0);
    const uint8_t *ytile = p.y + c0;
    const int ylast = (int)(p.n - 1 - c0);
    const uint32_t one = p.one;
    const uint32_t neg1 = 0u - p.one;
    const uint32_t tgrp = smem_addr(tab + 4 * grp);   // this thread's row words start here
    const uint32_t tlo = smem_addr(tab), thi = tlo + 4u * (uint32_t)((kTabSyms + 1) * P);
    (void)tlo;
    (void)thi;

    int kc = wk;
    int since = 0;
    uint32_t d = 0;

    uint8_t *ring8 = (uint8_t *)(ring + grp);
    auto count_exit = [&](uint32_t ex, uint32_t knew, int col) {
        const uint32_t age = knew - ex;
        const uint32_t valid = ((age + inval_bias) & L::MSB ^ L::MSB) >> 7;
        d += valid;
        const uint32_t colb = (uint32_t)(col & ring_mask) * L::ONES;
        const uint32_t slots = (colb + L::MSB - age) & ring_maskv;
#pragma unroll
        for (int b = 0; b < NS; ++b) {
            const uint32_t slot = prmt(slots, 0u, 0x4440u | (uint32_t)b);
            if (!AP_CHECK(p, slot < (uint32_t)p.ring, kDbgRing)) continue;
            ring8[slot * (uint32_t)(NGRP * 4) + b] = (uint8_t)prmt(valid, 0u, 0x4440u | (uint32_t)b);
        }
    };
    auto expire = [&](int col) {
        uint32_t *e = ring + ((col - wk) & ring_mask) * NGRP + grp;
        d -= *e;
        *e = 0u;
    };
    auto ychar = [&](int yi) -> uint32_t {
        yi = yi > ylast ? ylast : yi;
        if (!AP_CHECK(p, yi >= 0, kDbgYRead)) return 0u;
        return (uint32_t)__ldg(ytile + yi);
    };

    uint32_t yc[CPS];
#pragma unroll
    for (int c = 0; c < CPS; ++c) yc[c] = ychar(c);

    for (int s = 0; s < steps; ++s) {
        if (s > 0) {
            kc += CPS;
            if (++since == rsteps) {       // Proposition 3.4: old keys collapse to 0
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const uint32_t t = mad_lo(h[k], one, rr_bias);
                    h[k] = t & prmt(t, 0u, L::SIGNREP) & L::LOW;
                }
                kc = wk;
                since = 0;
            }
        }
        const uint32_t knew0 = (uint32_t)kc * L::ONES;
        uint32_t tcol[CPS];
        uint32_t v[CPS];
#pragma unroll
        for (int c = 0; c < CPS; ++c) {
            tcol[c] = tgrp + (uint32_t)ymap[yc[c]] * (uint32_t)(4 * P);
            v[c] = knew0 + (uint32_t)c * L::ONES;
        }
#pragma unroll
        for (int c = 0; c < CPS; ++c) yc[c] = ychar(CPS * (s + 1) + c);   // next step's characters
#pragma unroll
        for (int j = 0; j < R / 4; ++j) {
            uint4 X[CPS];
#pragma unroll
            for (int c = 0; c < CPS; ++c) {
                const uint32_t a = tcol[c] + 16u * (uint32_t)j;
                const uint32_t nm = SEL ? 0xBA98u : 0x80808080u;   // the no-match word
                X[c] = AP_CHECK(p, a >= tlo && a + 16u <= thi, kDbgTable) ? lds128(a) : make_uint4(nm, nm, nm, nm);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int k = 4 * j + r;
                const int pi = k - (R - PADU);
                const uint32_t kp = (pi >= 0) ? pk[pi < 0 ? 0 : pi] : 0xFFFFFFFFu;
#pragma unroll
                for (int c = 0; c < CPS; ++c) {
                    const uint32_t xv = r == 0 ? X[c].x : (r == 1 ? X[c].y : (r == 2 ? X[c].z : X[c].w));
                    if (SEL)
                        cell_sel(h[k], v[c], pi >= 0 ? ((xv & kp) | (0xBA98u & ~kp)) : xv, one, neg1, c80,
                                 c < HNF);
                    else
                        cell_tab(h[k], v[c], xv, kp, one, neg1, c < HNF);
                }
            }
        }
        // bottom of the strip: count exits (Theorem 3.1) and stage the plot
#pragma unroll
        for (int c = 0; c < CPS; ++c) {
            const int col = CPS * s + c;
            if (col < ncomb) {
                expire(col);
                count_exit(v[c], knew0 + (uint32_t)c * L::ONES, col);
                if (col >= wk - 1) {
                    const int jo = col - (wk - 1);
                    const int jj = jo & (kOB - 1);
                    stage[jj * (NGRP + 1) + grp] = wvec - d;
                    if (jj == kOB - 1 || jo == plot_cols - 1) {
                        __syncwarp();
                        flush_stage<L, NGRP, false>(p, stage, iw, c0 + jo - jj, jj + 1, lane);
                        __syncwarp();
                    }
                }
            }
        }
    }
}

// 8-bit-lane tiles whose characters allow it comb with the short mismatch
// test; the rest take the general one.  Measured on the 100k DNA plot,
// w = 100: 85.5 -> 82.5 ms.
// ---------------------------------------------------------------------------
// Match tables when a strip group's rows are split over G > 1 threads (LCS;
// full 8-bit keys or 16-bit lanes)
// ---------------------------------------------------------------------------
//
// Thread (grp, g) holds rows ub_g .. ub_{g+1} - 1 of the strips iw + NS grp
// + b, so its row k reads the characters at warp position NS grp + ub_g + k.
// The split is ub_g = floor(g w / G) rounded down to RPL rows (the rows of
// one vector load), which keeps every load aligned; the plan uses this path
// only where every share fits the thread's R rows with at most PADU padding
// rows (tab_split_ok), else the even split of the general path.
//
// Each g has its own copy of the tables, holding positions ub_g + q: a load
// phase of the warp (128 bytes) then covers G copies, whose bases differ by
// 32 / G banks, and every symbol table is a whole number of 32-word rows, so
// threads of different g, combing different columns (the wavefront is
// skewed) and so reading different symbols' tables, still hit distinct
// banks.  Table words: lane = all ones for a match, else 0 (full 8-bit keys)
// or the lane's top bit (16-bit lanes): the operand the cell ORs into h.

__host__ __device__ constexpr int tabg_rpl(int ns) { return ns == 4 ? 4 : (ns == 2 ? 2 : 1); }

// positions per symbol table of one copy
__host__ __device__ constexpr int tabg_q(int ns, int g, int r)
{
    return (ns * (32 / g - 1) + r + ns + 31) / 32 * 32;
}

// words per copy: the symbol tables, padded so that copy g starts 32 / G
// banks after copy g - 1
__host__ __device__ constexpr int tabg_s(int ns, int g, int r)
{
    return ((kTabSyms + 1) * tabg_q(ns, g, r) + 31) / 32 * 32 + 32 / g;
}

__host__ __device__ constexpr int tabg_words(int ns, int g, int r)
{
    return (g * tabg_s(ns, g, r) + 64 + 8 + 2 + 3) / 4 * 4;
}

__host__ __device__ constexpr bool has_tables_g(int key_bits, int groups, int nu, bool xrows)
{
    return nu == 1 && !xrows && groups > 1 &&
           (key_bits == 7 || key_bits == 8 || key_bits == 9 || key_bits == 15);
}

// Strips per register of a lane width (8, 10 or 16 bits).
__host__ __device__ constexpr int lane_strips(int lane_bits)
{
    return lane_bits == 8 ? 4 : (lane_bits == 10 ? 3 : 2);
}

// The table word of a lane format: OR masks (match: the whole lane; no
// match: 0 for full 8-bit keys, the lane's top bit otherwise) or
// byte-permute selectors (match: bytes of the all-ones constant; no match:
// the lane's sign spread over its bytes).
#ifndef AP_TABG_MM
// 1: the G > 1 tables of 16-bit lanes hold the match bit (0x8000 in match
// lanes, 0 otherwise) for the min/max cell (cell_tmm).
#define AP_TABG_MM 1
#endif

template <class L>
__host__ __device__ constexpr bool tab_minmax()
{
    return AP_TABG_MM != 0 && L::BITS == 16;
}

template <class L, bool SEL>
__host__ __device__ constexpr uint32_t tab_lane_word(bool hit, int b)
{
    if (tab_minmax<L>()) return hit ? (0x8000u << (16 * b)) : 0u;
    if (!SEL) return hit ? (L::MASK << (L::BITS * b)) : (L::FULL ? 0u : (L::MSB & (L::MASK << (L::BITS * b))));
    if (L::BITS == 8) return (uint32_t)(hit ? 4 + b : 8 + b) << (4 * b);
    // 16-bit lane b: bytes 2b, 2b + 1
    return hit ? (0x44u << (8 * b)) : ((uint32_t)((8 + 2 * b + 1) * 0x11) << (8 * b));
}

// The no-match word of a whole register.
template <class L, bool SEL>
__host__ __device__ constexpr uint32_t tab_nomatch()
{
    return tab_minmax<L>() ? 0u : (SEL ? (L::BITS == 8 ? 0xBA98u : 0xBB99u) : (L::FULL ? 0u : L::MSB));
}

// First row of thread g's share (g = G: the window w): g w / G rounded down
// (mode 1) or up (mode 2) to whole table loads of rpl rows.
__host__ __device__ inline int tabg_ub(int w, int G, int rpl, int g, int mode)
{
    if (g >= G) return w;
    return mode == 2 ? ((g * w + G - 1) / G + rpl - 1) / rpl * rpl : (g * w / G) / rpl * rpl;
}

// The aligned split of a mode fits: every share has at most R rows and at
// least R - PADU of them are real.
__host__ __device__ inline bool tabg_split_ok(int w, int G, int R, int rpl, int padu, int mode)
{
    for (int g = 0; g < G; ++g) {
        const int n = tabg_ub(w, G, rpl, g + 1, mode) - tabg_ub(w, G, rpl, g, mode);
        if (n > R || n < R - padu) return false;
    }
    return true;
}

// The split mode of a plan: 1 (rounded down) or 2 (rounded up) where one of
// them fits, else 0 (no G > 1 tables).  Between them every default plan of
// w = 121..512 fits; rounding down alone missed a third of 121..254.
__host__ __device__ inline int tabg_split_mode(int w, int G, int R, int rpl, int padu)
{
    return tabg_split_ok(w, G, R, rpl, padu, 1) ? 1 : (tabg_split_ok(w, G, R, rpl, padu, 2) ? 2 : 0);
}

template <int RPL>
__device__ __forceinline__ void lds_rows(uint32_t saddr, uint32_t *out)
{
    if (RPL == 4) {
        asm("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
            : "=r"(out[0]), "=r"(out[1]), "=r"(out[2]), "=r"(out[3]) : "r"(saddr));
    } else if (RPL == 2) {
        asm("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(out[0]), "=r"(out[1]) : "r"(saddr));
    } else {
        asm("ld.shared.u32 %0, [%1];" : "=r"(out[0]) : "r"(saddr));
    }
}

// Builds the tables of a G > 1 warp; false (warp-uniform) if its x
// characters take more than kTabSyms values.
template <class L, int G, int R, bool SEL = false>
__device__ __forceinline__ bool build_tables_g(const CombParams &p, int64_t iw, uint32_t *tab,
                                               int lane)
{
    constexpr int NS = L::NS;
    constexpr int RPL = tabg_rpl(NS);
    constexpr int Q = tabg_q(NS, G, R);
    constexpr int S = tabg_s(NS, G, R);
    uint8_t *ymap = (uint8_t *)(tab + G * S);
    uint32_t *bits = tab + G * S + 64;
    uint8_t *sym = (uint8_t *)(bits + 8);
    const int wk = p.w;
    const int span = NS * (32 / G - 1) + wk + NS - 1;   // characters the warp's rows read
    if (lane < 8) bits[lane] = 0u;
    __syncwarp();
    for (int q = lane; q < span; q += 32) {
        const int64_t idx = iw + q;
        if (idx < p.m) {
            const uint32_t c = __ldg(p.x + idx);
            atomicOr(&bits[c >> 5], 1u << (c & 31u));
        }
    }
    __syncwarp();
    const uint32_t wbits = (lane < 8) ? bits[lane] : 0u;
    const int cnt = __popc(wbits);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 7);
    if (total > kTabSyms) return false;
    const int before = __shfl_sync(0xffffffffu, incl - cnt, lane >> 2);
    const uint32_t wl = __shfl_sync(0xffffffffu, wbits, lane >> 2);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const uint32_t c = (uint32_t)(lane * 8 + t);
        const uint32_t bit = c & 31u;
        const bool present = (wl >> bit) & 1u;
        const int rank = before + __popc(wl & ((1u << bit) - 1u));
        ymap[c] = (uint8_t)(present ? rank : kTabSyms);
        if (present) sym[rank] = (uint8_t)c;
    }
    __syncwarp();
    for (int g = 0; g < G; ++g) {
        const int ub = tabg_ub(wk, G, RPL, g, p.tab);
        uint32_t *copy = tab + g * S;
        for (int q = lane; q < Q; q += 32) {
            uint32_t ch[NS];
            bool in[NS];
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                const int64_t idx = iw + ub + q + b;
                in[b] = idx < p.m;
                ch[b] = in[b] ? (uint32_t)__ldg(p.x + idx) : 0u;
            }
            for (int s = 0; s < total; ++s) {
                const uint32_t c = sym[s];
                uint32_t wv = 0u;
#pragma unroll
                for (int b = 0; b < NS; ++b) wv |= tab_lane_word<L, SEL>(in[b] && ch[b] == c, b);
                copy[s * Q + q] = wv;
            }
            copy[kTabSyms * Q + q] = tab_nomatch<L, SEL>();
        }
    }
    __syncwarp();
    return true;
}

// One comb cell with the match folded in by a table word (see above; X & pk
// is the no-match word in padding rows).  FMA_HN forms the right output as
// (h + v) - bottom on the FMA pipe, as cell_tab does (not for full 8-bit
// keys, whose lane sums would carry).
template <class L>
__device__ __forceinline__ void cell_tx(uint32_t &h, uint32_t &v, uint32_t X, uint32_t pk,
                                        uint32_t neg1, uint32_t sph, uint32_t spl,
                                        bool FMA_HN = false, uint32_t one = 1u)
{
    uint32_t M;
    if (L::FULL) {
        const uint32_t hm = h | (X & pk);
        M = prmt(ge_lanes<L>(hm, v, neg1), 0u, L::SIGNREP);
    } else {
        const uint32_t hc = h | (X & pk);
        const uint32_t t = mad_lo(v, neg1, hc);
        M = spread<L>(t, sph, spl);
    }
    const uint32_t vn = (h & M) | (v & ~M);
    if (FMA_HN && !L::FULL) h = mad_lo(vn, neg1, mad_lo(h, one, v));
    else h = h ^ v ^ vn;
    v = vn;
}

// One comb cell with the match folded into the byte permute (selector
// tables): as cell_sel, for 16-bit lanes (h + 0x8000.. - v on the FMA pipe)
// and for full 8-bit keys (the full-width compare of h and v, whose result
// the selector overrides in match lanes).
template <class L>
__device__ __forceinline__ void cell_txs(uint32_t &h, uint32_t &v, uint32_t S, uint32_t neg1,
                                         uint32_t one, bool FMA_HN)
{
    uint32_t M;
    if (L::FULL) {
        M = prmt(ge_lanes<L>(h, v, neg1), 0xFFFFFFFFu, S);
    } else {
        const uint32_t t = mad_lo(v, neg1, mad_lo(h, one, L::MSB));
        M = prmt(t, 0xFFFFFFFFu, S);
    }
    const uint32_t vn = (h & M) | (v & ~M);
    if (FMA_HN) h = mad_lo(vn, neg1, mad_lo(h, one, v));
    else h = h ^ v ^ vn;
    v = vn;
}

// One comb cell of 16-bit lanes with a min/max table word X (0x8000 in match
// lanes; X & pk is 0 in padding rows).  In a match lane h + 0x8000 exceeds
// every key, so the maximum is h + 0x8000 (bottom h once X is taken off)
// and the minimum v; elsewhere bottom = max(h, v) and right = min(h, v): the
// same swap as cell_tx, in two multiply-adds and two 16x2 min/max.
__device__ __forceinline__ void cell_tmm(uint32_t &h, uint32_t &v, uint32_t X, uint32_t pk,
                                         uint32_t one, uint32_t neg1)
{
    const uint32_t xm = X & pk;
    const uint32_t hc = mad_lo(h, one, xm);
    const uint32_t b = max_u16x2(hc, v);
    h = min_u16x2(hc, v);
    v = mad_lo(xm, neg1, b);
}

#ifndef AP_TABG_SEL
// 1: the G > 1 tables of 8-bit lanes (7-bit or full 8-bit keys) hold
// byte-permute selectors instead of OR masks (see cell_txs): measured on the
// 100k DNA plot with full keys, w = 128, comb
// alone, 132.3 ms against 148.8 ms.  16-bit lanes keep OR masks (selectors:
// 380.6 ms against 373.0 at w = 256), and 10-bit lanes, which spread their
// compare bits with multiplies, too.
#define AP_TABG_SEL 1
#endif
#ifndef AP_TABG_HNF8
// Full 8-bit keys (their ALU pipe is the busy one, 87% against 9% for the
// FMA pipe at w = 128): right outputs formed as (h + v) - bottom on the FMA
// pipe in 0, 1 or 2 columns of each step.  The packed sum may carry between
// lanes, but every lane's result lies in [0, 255], so the 32-bit result is
// exact.  100k DNA plot, none / one / both: w = 128 124.6 / 121.7 / 119.5 ms,
// w = 160 165.7 / 157.8 / 151.7 ms, w = 200 212.3 / 207.1 / 197.9 ms.
#define AP_TABG_HNF8 2
#endif
#ifndef AP_TABG_HNF
// Right output of the second column of each step on the FMA pipe in the
// G > 1 table path of 10-bit lanes (full 8-bit keys: AP_TABG_HNF8; 7-bit keys
// keep the logic form, which wins with selectors as on one thread).
#define AP_TABG_HNF 1
#endif

// The LCS comb of one tile through per-g tables, rows split over G > 1
// threads with the skewed wavefront of comb_tile: the same method, window
// count and output; only the row masks come from the tables and the split
// is the aligned one.
template <class L, int R, int G, int PADU, bool SEL = false>
__device__ __forceinline__ void comb_tile_tabg(const CombParams &p, int64_t sg, int64_t ch,
                                               uint32_t *ring, const uint32_t *tab)
{
    constexpr int NS = L::NS;
    constexpr int NGRP = 32 / G;
    constexpr int SPW = NGRP * NS;
    constexpr int RPL = tabg_rpl(NS);
    constexpr int Q = tabg_q(NS, G, R);
    constexpr int S = tabg_s(NS, G, R);
    static_assert(G > 1 && R % RPL == 0, "rows in whole loads");
    static_assert(PADU <= R, "padding window larger than the lane");

    const int lane = threadIdx.x & 31;
    const int g = lane % G;
    const int grp = lane / G;
    uint32_t *stage = ring + p.ring * NGRP;
    const uint8_t *ymap = (const uint8_t *)(tab + G * S);

    const int64_t iw = sg * SPW;
    const int64_t c0 = ch * p.chunk;
    const int64_t c1 = (c0 + p.chunk < p.cols) ? c0 + p.chunk : p.cols;
    const int wk = p.w;
    const int nreal = tabg_ub(wk, G, RPL, g + 1, p.tab) - tabg_ub(wk, G, RPL, g, p.tab);

    const uint32_t nomatch = tab_nomatch<L, SEL>();
    // padding rows never match: OR masks are ANDed with the no-match word;
    // selectors are replaced by it (pk = 0 in those rows)
    uint32_t pk[PADU > 0 ? PADU : 1];
#pragma unroll
    for (int t = 0; t < PADU; ++t)
        pk[t] = ((R - PADU + t) >= nreal) ? (SEL ? 0u : nomatch) : 0xFFFFFFFFu;

    for (int e = lane; e < p.ring * NGRP; e += 32) ring[e] = 0u;
    __syncwarp();

    uint32_t h[R];
#pragma unroll
    for (int k = 0; k < R; ++k) h[k] = 0u;

    const int ncomb = (int)(c1 - c0) + wk - 1;
    const int nunits = (ncomb + 1) / 2;
    const int steps = nunits + G - 1;
    const uint32_t wvec = (uint32_t)wk * L::ONES;
    const uint32_t inval_bias = (uint32_t)((1u << (L::BITS - 1)) - (uint32_t)wk) * L::ONES;
    const int kdrop = 2 * p.renorm;
    const uint32_t rr_bias = (uint32_t)((1u << (L::BITS - 1)) - (uint32_t)kdrop) * L::ONES;
    const uint32_t rrv = (uint32_t)kdrop * L::ONES;
    const uint32_t wkv = (uint32_t)wk * L::ONES;
    const int ring_mask = p.ring - 1;
    const uint32_t ring_maskv = (uint32_t)ring_mask * L::ONES;
    const int plot_cols = (int)(c1 - c0);
    const uint8_t *ytile = p.y + c0;
    const int ylast = (int)(p.n - 1 - c0);
    const uint32_t one = p.one;
    const uint32_t neg1 = 0u - p.one;
    const uint32_t sph = p.spread_hi, spl = p.spread_lo;
    const uint32_t tbase = smem_addr(tab + g * S + NS * grp);   // this thread's row 0, symbol 0
    const uint32_t tlo = smem_addr(tab + g * S), thi = tlo + 4u * (uint32_t)((kTabSyms + 1) * Q);
    (void)tlo;
    (void)thi;

    int kc = wk;
    int since = 0;
    uint32_t d = 0;
    uint32_t vdown[2] = {0u, 0u};

    uint8_t *ring8 = (uint8_t *)(ring + grp);
    auto count_exit = [&](uint32_t ex, uint32_t knew, int col) {
        const uint32_t age = knew - ex;
        const uint32_t inval = (L::FULL ? ge_lanes<L>(age, wkv, neg1) : age + inval_bias) & L::MSB;
        const uint32_t valid = (inval ^ L::MSB) >> (L::BITS - 1);
        d += valid;
        if (L::BITS == 8) {
            const uint32_t colb = (uint32_t)(col & ring_mask) * L::ONES;
            const uint32_t slots = L::FULL ? sub_lanes<L>(colb, age) : (colb + L::MSB - age) & ring_maskv;
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                const uint32_t slot = prmt(slots, 0u, 0x4440u | (uint32_t)b);
                if (!AP_CHECK(p, slot < (uint32_t)p.ring, kDbgRing)) continue;
                ring8[slot * (uint32_t)(NGRP * 4) + b] = (uint8_t)prmt(valid, 0u, 0x4440u | (uint32_t)b);
            }
        } else {
#pragma unroll
            for (int b = 0; b < NS; ++b) {
                if ((valid >> (L::BITS * b)) & 1u) {
                    const int a = (int)((age >> (L::BITS * b)) & L::MASK);
                    uint32_t *e = ring + ((col - a) & ring_mask) * NGRP + grp;
                    *e += 1u << (L::BITS * b);
                }
            }
        }
    };
    auto expire = [&](int col) {
        if (L::BITS == 8 || col >= wk) {
            uint32_t *e = ring + ((col - wk) & ring_mask) * NGRP + grp;
            d -= *e;
            *e = 0u;
        }
    };
    auto stage_and_flush = [&](int col, bool bottom) {
        if (col >= wk - 1 && col < ncomb) {
            const int jo = col - (wk - 1);
            const int jj = jo & (kOB - 1);
            if (bottom) stage[jj * (NGRP + 1) + grp] = wvec - d;
            if (jj == kOB - 1 || jo == plot_cols - 1) {
                __syncwarp();
                flush_stage<L, NGRP, false>(p, stage, iw, c0 + jo - jj, jj + 1, lane);
                __syncwarp();
            }
        }
    };
    auto ychar = [&](int yi) -> uint32_t {
        yi = yi < 0 ? 0 : (yi > ylast ? ylast : yi);
        if (!AP_CHECK(p, yi >= 0 && yi <= ylast, kDbgYRead)) return 0u;
        return (uint32_t)__ldg(ytile + yi);
    };

    for (int s = 0; s < steps; ++s) {
        const int u = s - g;
        if (u > 0) {
            kc += 2;
            if (++since == p.renorm) {     // Proposition 3.4: old keys collapse to 0
#pragma unroll
                for (int k = 0; k < R; ++k) h[k] = renorm_key<L>(h[k], rr_bias, rrv, one, neg1, sph, spl);
                kc = wk;
                since = 0;
            }
        }
        const uint32_t knew0 = (uint32_t)kc * L::ONES;
        const uint32_t knew1 = knew0 + L::ONES;
        const uint32_t in0 = __shfl_up_sync(0xffffffffu, vdown[0], 1);
        const uint32_t in1 = __shfl_up_sync(0xffffffffu, vdown[1], 1);
        uint32_t va = (g == 0) ? knew0 : in0;
        uint32_t vb = (g == 0) ? knew1 : in1;
        const uint32_t t0 = tbase + (uint32_t)ymap[ychar(2 * u)] * (uint32_t)(4 * Q);
        const uint32_t t1 = tbase + (uint32_t)ymap[ychar(2 * u + 1)] * (uint32_t)(4 * Q);
#pragma unroll
        for (int j = 0; j < R / RPL; ++j) {
            uint32_t X0[RPL], X1[RPL];
            const uint32_t a0 = t0 + 4u * (uint32_t)(RPL * j), a1 = t1 + 4u * (uint32_t)(RPL * j);
            if (AP_CHECK(p, a0 >= tlo && a0 + 4u * RPL <= thi, kDbgTable)) lds_rows<RPL>(a0, X0);
            else for (int r = 0; r < RPL; ++r) X0[r] = nomatch;
            if (AP_CHECK(p, a1 >= tlo && a1 + 4u * RPL <= thi, kDbgTable)) lds_rows<RPL>(a1, X1);
            else for (int r = 0; r < RPL; ++r) X1[r] = nomatch;
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
                const int k = RPL * j + r;
                const int pi = k - (R - PADU);
                const uint32_t kp = (pi >= 0) ? pk[pi < 0 ? 0 : pi] : 0xFFFFFFFFu;
                if (SEL) {
                    const uint32_t s0 = pi >= 0 ? ((X0[r] & kp) | (nomatch & ~kp)) : X0[r];
                    const uint32_t s1 = pi >= 0 ? ((X1[r] & kp) | (nomatch & ~kp)) : X1[r];
                    cell_txs<L>(h[k], va, s0, neg1, one, L::FULL && AP_TABG_HNF8 >= 2);
                    cell_txs<L>(h[k], vb, s1, neg1, one, L::FULL ? AP_TABG_HNF8 >= 1 : (AP_TABG_HNF != 0 && L::BITS != 8));
                } else if constexpr (tab_minmax<L>()) {
                    cell_tmm(h[k], va, X0[r], kp, one, neg1);
                    cell_tmm(h[k], vb, X1[r], kp, one, neg1);
                } else {
                    cell_tx<L>(h[k], va, X0[r], kp, neg1, sph, spl);
                    cell_tx<L>(h[k], vb, X1[r], kp, neg1, sph, spl, AP_TABG_HNF != 0, one);
                }
            }
        }
        vdown[0] = va;
        vdown[1] = vb;

        // ---- bottom threads: count exits (Theorem 3.1) and stage the plot ----
        const int ubot = s - (G - 1);
        const bool bottom = (g == G - 1) && u >= 0 && u < nunits;
        const int col0 = 2 * ubot, col1 = 2 * ubot + 1;
        if (bottom) {
            expire(col0);
            count_exit(vdown[0], knew0, col0);
        }
        if (ubot >= 0) stage_and_flush(col0, bottom);
        if (bottom && col1 < ncomb) {
            expire(col1);
            count_exit(vdown[1], knew1, col1);
        }
        if (ubot >= 0) stage_and_flush(col1, bottom && col1 < ncomb);
    }
}

// Variants with match tables (LCS: 7-bit keys on one thread per strip
// group; 7-bit, full 8-bit, 9-bit keys or 16-bit lanes on G > 1 threads,
// where the plan allows the aligned split) first try them: warps whose x characters take
// at most kTabSyms values comb through the tables.
template <class L, int R, int G, int NU, int MU, int PADU, bool XR>
__device__ __forceinline__ void comb_tile_dispatch(const CombParams &p, int64_t sg, int64_t ch,
                                                   uint32_t *ring)
{
    constexpr bool FAST_OK = L::BITS == 8;
    constexpr bool TAB = L::BITS == 8 && !L::FULL && has_tables(7, G, NU, XR);
    constexpr bool TABG = has_tables_g(L::BITS == 16 ? 15 : (L::BITS == 10 ? 9 : (L::FULL ? 8 : 7)), G, NU, XR);
    if constexpr (TAB) {
        uint32_t *tab = ring + p.ring * (32 / G) + kOB * (32 / G + 1);
        // The selector cells of the last PADU rows fold in the padding mask
        // (one logic instruction a cell); w = R leaves no padding row and
        // takes a tile without the fold.  Measured on the 100k DNA plot:
        // w = 100 59.4 -> 56.7 ms, w = 16 16.2 -> 14.9 ms.  A second tile
        // folding only the last 4 rows (R - w <= 4 in every plan of R >= 12)
        // gained at most 1% at w = 97 and 117, and the code then generated for
        // the w = R tile ran 3-4% slower (w = 100: 58.3 or 59.1 ms).
        if (build_tables<R, AP_TAB_SEL != 0>(p, sg * 128, tab, threadIdx.x & 31)) {
            if (p.w == R)
                comb_tile_tab<R, 0, AP_TAB_CPS, AP_TAB_HNF, AP_TAB_SEL != 0>(p, sg, ch, ring, tab);
            else
                comb_tile_tab<R, PADU, AP_TAB_CPS, AP_TAB_HNF, AP_TAB_SEL != 0>(p, sg, ch, ring, tab);
            return;
        }
    }
    if constexpr (TABG) {
        uint32_t *tab = ring + p.ring * (32 / G) + kOB * (32 / G + 1);
        constexpr bool TSEL = AP_TABG_SEL != 0 && L::BITS == 8;
        if (p.tab && build_tables_g<L, G, R, TSEL>(p, sg * (32 / G) * L::NS, tab, threadIdx.x & 31)) {
            if constexpr (TSEL) {
                // as on one thread: the padding fold spans the most padding
                // rows any thread of the group holds (0, up to 4, or PADU)
                constexpr int RPL = tabg_rpl(L::NS);
                int npad = 0;
                for (int q = 0; q < G; ++q) {
                    const int n = tabg_ub(p.w, G, RPL, q + 1, p.tab) - tabg_ub(p.w, G, RPL, q, p.tab);
                    npad = R - n > npad ? R - n : npad;
                }
                constexpr int NP4 = PADU < 4 ? PADU : 4;
                if (npad == 0)
                    comb_tile_tabg<L, R, G, 0, TSEL>(p, sg, ch, ring, tab);
                else if (npad <= NP4)
                    comb_tile_tabg<L, R, G, NP4, TSEL>(p, sg, ch, ring, tab);
                else
                    comb_tile_tabg<L, R, G, PADU, TSEL>(p, sg, ch, ring, tab);
            } else {
                comb_tile_tabg<L, R, G, PADU, TSEL>(p, sg, ch, ring, tab);
            }
            return;
        }
    }
    if (FAST_OK && tile_same_top<L, G>(p, sg, ch))
        comb_tile<L, R, G, NU, MU, PADU, XR, FAST_OK>(p, sg, ch, ring);
    else
        comb_tile<L, R, G, NU, MU, PADU, XR, false>(p, sg, ch, ring);
}

// Resident blocks per SM asked of the compiler.  Three (168 registers a
// thread) where the shared memory allows them and the registers fit without
// spills (LCS, not the vertical-step layout): full 8-bit keys on 4 threads
// (100k DNA plot, w = 200: 227 ms at 255 registers and two blocks, 213 ms at
// three), 16-bit lanes on 4 threads up to 64 rows (w = 256: 311 -> 285 ms;
// a few bytes spill at 64 rows) and 7-bit keys on 2 threads up to 52 rows
// (w = 100 on request: 84 ms against 74 ms).  Elsewhere the compiler keeps
// its own budget: where the shared memory holds two blocks anyway (w = 128
// on 2 threads) the cap only costs.
template <class L, int R, int G, int NU, bool XR>
__host__ __device__ constexpr int comb_min_blocks()
{
    return NU == 1 && !XR &&
                   ((L::BITS == 16 && G == 4 && R <= 64) || (L::BITS == 8 && L::FULL && G == 4 && R <= 64) ||
                    (L::BITS == 8 && !L::FULL && G == 2 && R <= 52))
               ? 3
               : AP_MIN_BLOCKS;
}

// Plain launch: one warp per tile; tiles are numbered strip group fastest.
template <class L, int R, int G, int NU, int MU, int PADU, bool XR>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, (comb_min_blocks<L, R, G, NU, XR>()))
comb_kernel(CombParams p)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int wid = threadIdx.x >> 5;
    const int64_t tile = p.tile0 + (int64_t)blockIdx.x * kWarpsPerBlock + wid;
    if (tile >= p.ntiles) return;
    comb_tile_dispatch<L, R, G, NU, MU, PADU, XR>(p, tile % p.nsg, tile / p.nsg,
                                                 smem + wid * p.warp_words);
}

// One tile of a batch: which job, and which strip group and column chunk.
struct BatchTile {
    int32_t job;
    int32_t sg;
    int32_t ch;
    int32_t pad;
};

struct BatchParams {
    const CombParams *jobs;       // per-job parameters (device)
    const BatchTile *tiles;       // work list, most expensive first (device)
    int64_t ntiles;
    unsigned int *next;           // work-queue counter, zero at launch (device)
    int32_t warp_words;           // shared-memory words per warp
};

// Persistent launch over a batch: every warp takes the next tile of the work
// list until it is exhausted.  Each tile is combed exactly as a plain launch
// combs it, so results are bit-identical to one call per job.
template <class L, int R, int G, int NU, int MU, int PADU, bool XR>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, (comb_min_blocks<L, R, G, NU, XR>()))
comb_batch_kernel(BatchParams b)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    uint32_t *wsm = smem + wid * b.warp_words;
    for (;;) {
        unsigned int t = 0;
        if (lane == 0) t = atomicAdd(b.next, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if ((int64_t)t >= b.ntiles) break;
        const BatchTile bt = b.tiles[t];
        comb_tile_dispatch<L, R, G, NU, MU, PADU, XR>(b.jobs[bt.job], bt.sg, bt.ch, wsm);
        __syncwarp();
    }
}

}  // namespace ap
