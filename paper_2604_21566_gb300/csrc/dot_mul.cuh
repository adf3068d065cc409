// dot_mul.cuh -- device building blocks of the column-sum multiply
// (Alg. 2 re-shaped for warps); see dot_mul.cu for the method.
#pragma once

#include "dot_internal.cuh"

#define MUL_WARPS 4
// Resident blocks per SM the compiler must allow (caps registers per thread):
// 6 blocks of 4 warps fit R <= 8 in 80 registers without spills; R = 16
// needs its ~170 registers.
__host__ __device__ constexpr int dot_mul_min_blocks(int R) { return R <= 8 ? 6 : 1; }

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

template <int R>
__device__ __forceinline__ void lds_vec(const uint32_t *p, uint32_t *v)
{
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
        const uint4 t = reinterpret_cast<const uint4 *>(p)[q];
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
    }
}

// Positional sum W = sum_{k<R} S_{c0+k} X^k of the block of columns [c0, c0+R),
// S_c = sum_{i+j=c} A_i B_j.  As = A[0..m'), Bs = B[-R .. m'+R) (zeros outside
// [0, m)), both in shared memory.  For row i the block needs B[c0 + k - i],
// k < R: a window of R values that slides down by one per row, so each row
// reads A_i (a broadcast) and one new B value; rows are unrolled R at a time
// so the slide is register renaming.
template <int R>
__device__ __forceinline__ void colsum_block(const uint32_t *As, const uint32_t *Bs, int c0, int mp,
                                             uint32_t (&W)[R + 2])
{
    uint32_t s0[R], s1[R], s2[R];
#pragma unroll
    for (int k = 0; k < R; ++k) s0[k] = s1[k] = s2[k] = 0;
    const int i_lo = max(0, c0 - mp + 1);
    const int i_hi = min(c0 + R - 1, mp - 1);
    int i0 = (i_lo / R) * R;
    if (i0 <= i_hi) {
        uint32_t w[R];
        lds_vec<R>(Bs + R + (c0 - i0), w);   // w[k] = B[c0 + k - i0]
        for (; i0 <= i_hi; i0 += R) {
#pragma unroll
            for (int ii = 0; ii < R; ++ii) {
                mac_cols<R>(s0, s1, s2, As[i0 + ii], w);
#pragma unroll
                for (int k = R - 1; k > 0; --k) w[k] = w[k - 1];
                w[0] = Bs[R + c0 - (i0 + ii) - 1];
            }
        }
    }
    cols_to_positional<R>(s0, s1, s2, W);
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
// sliding window; the few rows with c0 <= 2i < c0 + R feed only the columns
// c > 2i and are summed one column at a time.
template <int R>
__device__ __forceinline__ void sqr_colsum_block(const uint32_t *As, const uint32_t *Bs, int c0, int mp,
                                                 uint32_t (&W)[R + 2])
{
    uint32_t s0[R], s1[R], s2[R];
#pragma unroll
    for (int k = 0; k < R; ++k) s0[k] = s1[k] = s2[k] = 0;
    const int i_lo = max(0, c0 - mp + 1);
    const int i_full = min((c0 - 1) >> 1, mp - 1);   // last row with 2i < c0 (-1: none)
    int i0 = (i_lo / R) * R;
    if (i0 + R - 1 <= i_full) {
        uint32_t w[R];
        lds_vec<R>(Bs + R + (c0 - i0), w);   // w[k] = A[c0 + k - i0]
        for (; i0 + R - 1 <= i_full; i0 += R) {
#pragma unroll
            for (int ii = 0; ii < R; ++ii) {
                mac_cols<R>(s0, s1, s2, As[i0 + ii], w);
#pragma unroll
                for (int k = R - 1; k > 0; --k) w[k] = w[k - 1];
                w[0] = Bs[R + c0 - (i0 + ii) - 1];
            }
        }
    }
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

// Copy limbs [t R, t R + R) of an m-limb row into shared memory (zeros past m).
template <int R>
__device__ __forceinline__ void stage_row(const uint32_t *row, uint32_t *dst, int t, int m, bool vec)
{
    const int l0 = t * R;
    if (vec && l0 + R <= m) {
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
    if (vec && pos + R <= len) {
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
    uint32_t W[R + 2];
    uint32_t wl, wh, mid;
    {   // low blocks [tR, tR + R): positions 0 .. m' - 1
        if (on) {
            if (SQR) sqr_colsum_block<R>(As, Bs, t * R, mp, W);
            else colsum_block<R>(As, Bs, t * R, mp, W);
        } else {
#pragma unroll
            for (int k = 0; k < R + 2; ++k) W[k] = 0;
        }
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
        if (on) {
            if (SQR) sqr_colsum_block<R>(As, Bs, mp + t * R, mp, W);
            else colsum_block<R>(As, Bs, mp + t * R, mp, W);
        } else {
#pragma unroll
            for (int k = 0; k < R + 2; ++k) W[k] = 0;
        }
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

