// dot_mul.cuh -- device building blocks of the column-sum multiply
// (Alg. 2 re-shaped for warps); see dot_mul.cu for the method.
#pragma once

#include "dot_internal.cuh"

#define MUL_WARPS 4
// Resident blocks per SM the compiler must allow (caps registers per thread).
// Both blocks' sums stay live through the row loop (colsum_pair): R = 8 fits
// 4 blocks of 4 warps (128 registers), R = 4 fits 6 (80 registers; the
// smallest products need the occupancy more), and R = 16 and the R = 12
// square fit 3 (168 registers, without spills; left free the compiler takes
// up to ~200 and only 2 blocks fit).  The R = 12 general product already
// fits 3 when left free and measured 7% slower with the cap.
__host__ __device__ constexpr int dot_mul_min_blocks(int R, bool sqr = false)
{
    return R <= 4 ? 6 : (R <= 8 ? 4 : (R == 12 && !sqr ? 1 : 3));
}

// Column sums of one block of R columns, kept as three 32-bit words each:
// S_k = s2[k] X^2 + s1[k] X + s0[k]  (S_k < m 2^64 needs 64 + log2 m bits).
// One partial product a * w_k is formed independently (Alg. 2 Phase 2: its low
// and high halves) and added into column k with one carry chain of three words
// (Phases 3-4 for that column).  Per product: 2 multiplies on the FMA pipe and
// 3 adds on the integer ALU pipe, which run side by side.
template <int R>
__device__ __forceinline__ void mac_cols(uint32_t (&s0)[R], uint32_t (&s1)[R], uint32_t (&s2)[R], uint32_t a,
                                         const uint32_t (&w)[R])
{
#pragma unroll
    for (int k = 0; k < R; ++k)
        asm("{\n\t.reg .u32 lo, hi;\n\t"
            "mul.lo.u32 lo, %3, %4;\n\t"
            "mul.hi.u32 hi, %3, %4;\n\t"
            "add.cc.u32 %0, %0, lo;\n\t"
            "addc.cc.u32 %1, %1, hi;\n\t"
            "addc.u32 %2, %2, 0;\n\t}"
            : "+r"(s0[k]), "+r"(s1[k]), "+r"(s2[k])
            : "r"(a), "r"(w[k]));
}

// Positional value of the block, W = sum_k S_k X^k, as R + 2 words.  The sum
// is below m X^(R+1) (1 + 1/X), so R + 2 words always hold it.
template <int R>
__device__ __forceinline__ void cols_to_positional(const uint32_t (&s0)[R], const uint32_t (&s1)[R],
                                                   const uint32_t (&s2)[R], uint32_t (&W)[R + 2])
{
    uint64_t c = 0;
#pragma unroll
    for (int j = 0; j < R + 2; ++j) {
        uint64_t t = c;
        if (j < R) t += s0[j];
        if (j >= 1 && j - 1 < R) t += s1[j - 1];
        if (j >= 2) t += s2[j - 2];
        W[j] = (uint32_t)t;
        c = t >> 32;
    }
}

// R words from shared memory: 16-byte loads when R % 4 == 0 (the caller's
// address is then 16-byte aligned), one word at a time otherwise.
template <int R>
__device__ __forceinline__ void lds_vec(const uint32_t *p, uint32_t *v)
{
    if constexpr (R % 4 == 0) {
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            const uint4 t = reinterpret_cast<const uint4 *>(p)[q];
            v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = p[k];
    }
}

// Positional sums W = sum_{k<R} S_{c0+k} X^k of both column blocks of lane t,
// the low one [tR, tR + R) and the high one [m' + tR, m' + tR + R), with
// S_c = sum_{i+j=c} A_i B_j.  As = A[0..m'), Bs = B[-R .. m'+R) (zeros outside
// [0, m)), both in shared memory.  For row i a block needs B[c0 + k - i],
// k < R: a window of R values that slides down by one per row, so each row
// reads A_i (a broadcast) and one new B value; rows are unrolled R at a time
// so the slide is register renaming.  Both blocks run in ONE loop of T + 1
// row groups (T = m'/R lanes per op).  The low block needs row groups 0 .. t and the high block t .. T-1, so
// every lane runs the same T + 1 groups; summing the two blocks one after the
// other would instead keep the warp busy for 2T groups with, on average, half
// its lanes idle (lane t's low block is short where its high block is long).
// At the switch the running sums are copied aside and the window restarts for
// the high block; the high block's sums are the final sums minus the copy.
template <int R>
__device__ __forceinline__ void colsum_pair(const uint32_t *As, const uint32_t *Bs, int t, int T, int mp,
                                            uint32_t (&Wl)[R + 2], uint32_t (&Wh)[R + 2])
{
    uint32_t s0[R], s1[R], s2[R], l0[R], l1[R], l2[R];
#pragma unroll
    for (int k = 0; k < R; ++k) s0[k] = s1[k] = s2[k] = l0[k] = l1[k] = l2[k] = 0;
    uint32_t w[R];
    lds_vec<R>(Bs + R + t * R, w);   // w[k] = B[tR + k]: the low block at row 0
    int cb = t * R;                  // first column of the current block
    int i0 = 0;                      // first row of the current group
    for (int g = 0; g <= T; ++g) {
        if (g == t + 1) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                l0[k] = s0[k];
                l1[k] = s1[k];
                l2[k] = s2[k];
            }
            cb = mp + t * R;
            i0 = t * R;
            lds_vec<R>(Bs + R + mp, w);   // w[k] = B[cb + k - i0] = B[m' + k] (zero padding)
        }
#pragma unroll
        for (int ii = 0; ii < R; ++ii) {
            mac_cols<R>(s0, s1, s2, As[i0 + ii], w);
#pragma unroll
            for (int k = R - 1; k > 0; --k) w[k] = w[k - 1];
            w[0] = Bs[R + cb - (i0 + ii) - 1];
        }
        i0 += R;
    }
    // high sums = final - low (three-word subtraction per column; never negative)
#pragma unroll
    for (int k = 0; k < R; ++k)
        asm("sub.cc.u32 %0, %0, %3;\n\tsubc.cc.u32 %1, %1, %4;\n\tsubc.u32 %2, %2, %5;"
            : "+r"(s0[k]), "+r"(s1[k]), "+r"(s2[k])
            : "r"(l0[k]), "r"(l1[k]), "r"(l2[k]));
    cols_to_positional<R>(l0, l1, l2, Wl);
    cols_to_positional<R>(s0, s1, s2, Wh);
}

// One column: (s2:s1:s0) += a * w
__device__ __forceinline__ void mac1(uint32_t &s0, uint32_t &s1, uint32_t &s2, uint32_t a, uint32_t w)
{
    asm("{\n\t.reg .u32 lo, hi;\n\t"
        "mul.lo.u32 lo, %3, %4;\n\t"
        "mul.hi.u32 hi, %3, %4;\n\t"
        "add.cc.u32 %0, %0, lo;\n\t"
        "addc.cc.u32 %1, %1, hi;\n\t"
        "addc.u32 %2, %2, 0;\n\t}"
        : "+r"(s0), "+r"(s1), "+r"(s2)
        : "r"(a), "r"(w));
}

// The same block for a square, A = B (As and Bs hold the same operand):
// S_c = 2 sum_{i<j, i+j=c} A_i A_j + [c even] A_{c/2}^2, so only rows with
// 2i < c are summed (about half of them), doubled, and the diagonal square
// added.  Rows with 2i < c0 feed every column of the block and use the
// sliding window (sqr_colsum_pair); the few rows with c0 <= 2i < c0 + R feed
// only the columns c > 2i and are summed one column at a time here, from row
// i0 (the first row the window did not take) on.
template <int R>
__device__ __forceinline__ void sqr_block_tail(const uint32_t *As, const uint32_t *Bs, int c0, int mp, int i0,
                                               uint32_t (&s0)[R], uint32_t (&s1)[R], uint32_t (&s2)[R],
                                               uint32_t (&W)[R + 2])
{
    const int i_top = min((c0 + R - 1) >> 1, mp - 1);   // last row with 2i < c0 + R
    for (int i = i0; i <= i_top; ++i) {
        const uint32_t ai = As[i];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int j = c0 + k - i;   // j > i >= 0; A is zero past m
            mac1(s0[k], s1[k], s2[k], ai, j > i ? Bs[R + j] : 0u);
        }
    }
    // double the off-diagonal sums, add the squares A_{c/2}^2 of even columns
#pragma unroll
    for (int k = 0; k < R; ++k) {
        s2[k] = (s2[k] << 1) | (s1[k] >> 31);
        s1[k] = (s1[k] << 1) | (s0[k] >> 31);
        s0[k] <<= 1;
        const int c = c0 + k;
        const uint32_t d = (c & 1) ? 0u : As[c >> 1];
        mac1(s0[k], s1[k], s2[k], d, d);
    }
    cols_to_positional<R>(s0, s1, s2, W);
}

// Both blocks of lane t for a square, as colsum_pair: the low block takes the
// row groups that lie wholly below the diagonal of [tR, tR + R) (rows from 0),
// the high block those of [m' + tR, ...) (rows from tR); the two counts add up
// to about T/2 for every lane, so one loop covers both with (at most) one
// group of imbalance.  Each block's near-diagonal rows follow the loop.
template <int R>
__device__ __forceinline__ void sqr_colsum_pair(const uint32_t *As, const uint32_t *Bs, int t, int mp,
                                                uint32_t (&Wl)[R + 2], uint32_t (&Wh)[R + 2])
{
    const int cl = t * R, ch = mp + t * R;
    // full groups: rows i < c0 / 2 for every column of the block
    const int n_lo = (((cl - 1) >> 1) + 1) / R;        // from row 0
    const int n_hi = (((ch - 1) >> 1) + 1 - cl) / R;   // from row tR
    uint32_t s0[R], s1[R], s2[R], l0[R], l1[R], l2[R];
#pragma unroll
    for (int k = 0; k < R; ++k) s0[k] = s1[k] = s2[k] = l0[k] = l1[k] = l2[k] = 0;
    uint32_t w[R];
    lds_vec<R>(Bs + R + cl, w);   // w[k] = A[tR + k]: the low block at row 0
    int cb = cl, i0 = 0;
    for (int g = 0;; ++g) {
        if (g == n_lo) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                l0[k] = s0[k];
                l1[k] = s1[k];
                l2[k] = s2[k];
            }
            cb = ch;
            i0 = cl;
            lds_vec<R>(Bs + R + mp, w);   // w[k] = A[ch + k - tR] = A[m' + k] (zero padding)
        }
        if (g == n_lo + n_hi) break;
#pragma unroll
        for (int ii = 0; ii < R; ++ii) {
            mac_cols<R>(s0, s1, s2, As[i0 + ii], w);
#pragma unroll
            for (int k = R - 1; k > 0; --k) w[k] = w[k - 1];
            w[0] = Bs[R + cb - (i0 + ii) - 1];
        }
        i0 += R;
    }
#pragma unroll
    for (int k = 0; k < R; ++k)
        asm("sub.cc.u32 %0, %0, %3;\n\tsubc.cc.u32 %1, %1, %4;\n\tsubc.u32 %2, %2, %5;"
            : "+r"(s0[k]), "+r"(s1[k]), "+r"(s2[k])
            : "r"(l0[k]), "r"(l1[k]), "r"(l2[k]));
    sqr_block_tail<R>(As, Bs, cl, mp, n_lo * R, l0, l1, l2, Wl);
    sqr_block_tail<R>(As, Bs, ch, mp, cl + n_hi * R, s0, s1, s2, Wh);
}

// Copy limbs [t R, t R + R) of an m-limb row into shared memory (zeros past m).
// 16-byte copies need R % 4 == 0 (block starts t R on 16-byte boundaries).
template <int R>
__device__ __forceinline__ void stage_row(const uint32_t *row, uint32_t *dst, int t, int m, bool vec)
{
    const int l0 = t * R;
    if (R % 4 == 0 && vec && l0 + R <= m) {
#pragma unroll
        for (int q = 0; q < R / 4; ++q)
            reinterpret_cast<uint4 *>(dst + l0)[q] = ld_stream4(row + l0 + 4 * q);
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) dst[l0 + k] = (l0 + k < m) ? ld_stream1(row + l0 + k) : 0u;
    }
}

template <int R>
__device__ __forceinline__ void store_block(uint32_t *row, int pos, int len, const uint32_t (&v)[R], bool vec)
{
    if (R % 4 == 0 && vec && pos + R <= len) {
#pragma unroll
        for (int q = 0; q < R / 4; ++q)
            st_stream4(row + pos + 4 * q, make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k)
            if (pos + k < len) st_stream1(row + pos + k, v[k]);
    }
}

// One op on a run of T lanes (lane t of the run, grp-th run of the warp), of
// which the first tn = mp / R hold column blocks.  Every lane of the warp must
// call this (it uses warp collectives); lanes with on == false or t >= tn take
// part without touching memory.  The low half of the product is resolved and
// stored before the high blocks are summed, so only its carry-out and the two
// overflow words of the top low block are kept across.
template <int R, bool SQR = false>
__device__ __forceinline__ void mul_group(const uint32_t *As, const uint32_t *Bs, int t, int T,
                                          int tn, int grp, bool on, int m, int mp, uint32_t *prow,
                                          bool vec_out, uint32_t smask, uint32_t tmask)
{
    const int lane = (int)lane_id();
    on = on && t < tn;
    const int last = min(grp * T + max(tn, 1) - 1, 31);
    uint32_t W[R + 2], WH[R + 2];
    uint32_t wl, wh, mid;
    // both blocks in one pass (the lanes t < tn of a run take the same row groups)
    if (on) {
        if (SQR) sqr_colsum_pair<R>(As, Bs, t, mp, W, WH);
        else colsum_pair<R>(As, Bs, t, tn, mp, W, WH);
    } else {
#pragma unroll
        for (int k = 0; k < R + 2; ++k) W[k] = WH[k] = 0;
    }
    {   // low blocks [tR, tR + R): positions 0 .. m' - 1
        // the two overflow words of each block belong to the next block
        const uint32_t ul = __shfl_up_sync(DOT_FULL, W[R], 1), uh = __shfl_up_sync(DOT_FULL, W[R + 1], 1);
        wl = __shfl_sync(DOT_FULL, W[R], last);   // top low block -> first high block
        wh = __shfl_sync(DOT_FULL, W[R + 1], last);
        uint32_t l[R], h[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            l[k] = W[k];
            h[k] = 0;
        }
        h[0] = t ? ul : 0u;
        h[1] = t ? uh : 0u;
        Segment<false, R> sg;
        sg.phase12(l, h);
        WarpCarry wc;
        wc.resolve(on ? sg.g() : 0u, on ? sg.p() : 0u, 0u, smask, tmask);
        mid = wc.carry_out(last);   // carry from the low half into the high half
        sg.apply(wc.carry_in(lane));
        if (on) store_block<R>(prow, t * R, 2 * m, sg.r, vec_out);
    }
    {   // high blocks [m' + tR, m' + tR + R)
#pragma unroll
        for (int k = 0; k < R + 2; ++k) W[k] = WH[k];
        const uint32_t ul = __shfl_up_sync(DOT_FULL, W[R], 1), uh = __shfl_up_sync(DOT_FULL, W[R + 1], 1);
        uint32_t l[R], h[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            l[k] = W[k];
            h[k] = 0;
        }
        h[0] = t ? ul : wl;
        h[1] = t ? uh : wh;
        Segment<false, R> sg;
        sg.phase12(l, h);
        WarpCarry wc;
        wc.resolve(on ? sg.g() : 0u, on ? sg.p() : 0u, t == 0 ? mid : 0u, smask, tmask);
        sg.apply(wc.carry_in(lane));
        if (on) store_block<R>(prow, mp + t * R, 2 * m, sg.r, vec_out);
    }
}

