// dot_mul.cuh -- device building blocks of the column-sum multiply
// (Alg. 2 re-shaped for warps); see dot_mul.cu for the method.
#pragma once

#include "dot_internal.cuh"

#define MUL_WARPS 4

#define DOT_S_(x) #x
#define DOT_S(x) DOT_S_(x)
#define MLO(d, a, w) "mad.lo.cc.u32 %" DOT_S(d) ", %" DOT_S(a) ", %" DOT_S(w) ", %" DOT_S(d) ";\n\t"
#define MCLO(d, a, w) "madc.lo.cc.u32 %" DOT_S(d) ", %" DOT_S(a) ", %" DOT_S(w) ", %" DOT_S(d) ";\n\t"
#define MCHI(d, a, w) "madc.hi.cc.u32 %" DOT_S(d) ", %" DOT_S(a) ", %" DOT_S(w) ", %" DOT_S(d) ";\n\t"

// W[0..R+2) += a * (w_0 + w_1 X + ... + w_{R-1} X^{R-1})
template <int R>
__device__ __forceinline__ void mac_row(uint32_t (&W)[R + 2], uint32_t a, const uint32_t (&w)[R]);

template <>
__device__ __forceinline__ void mac_row<4>(uint32_t (&W)[6], uint32_t a, const uint32_t (&w)[4])
{
    // even products: words (0,1), (2,3); then carry into 4, 5
    asm(MLO(0, 6, 7) MCHI(1, 6, 7) MCLO(2, 6, 8) MCHI(3, 6, 8)
        "addc.cc.u32 %4, %4, 0;\n\t"
        "addc.u32 %5, %5, 0;"
        : "+r"(W[0]), "+r"(W[1]), "+r"(W[2]), "+r"(W[3]), "+r"(W[4]), "+r"(W[5])
        : "r"(a), "r"(w[0]), "r"(w[2]));
    // odd products: words (1,2), (3,4); then carry into 5
    asm(MLO(0, 5, 6) MCHI(1, 5, 6) MCLO(2, 5, 7) MCHI(3, 5, 7)
        "addc.u32 %4, %4, 0;"
        : "+r"(W[1]), "+r"(W[2]), "+r"(W[3]), "+r"(W[4]), "+r"(W[5])
        : "r"(a), "r"(w[1]), "r"(w[3]));
}

template <>
__device__ __forceinline__ void mac_row<8>(uint32_t (&W)[10], uint32_t a, const uint32_t (&w)[8])
{
    asm(MLO(0, 10, 11) MCHI(1, 10, 11) MCLO(2, 10, 12) MCHI(3, 10, 12)
        MCLO(4, 10, 13) MCHI(5, 10, 13) MCLO(6, 10, 14) MCHI(7, 10, 14)
        "addc.cc.u32 %8, %8, 0;\n\t"
        "addc.u32 %9, %9, 0;"
        : "+r"(W[0]), "+r"(W[1]), "+r"(W[2]), "+r"(W[3]), "+r"(W[4]), "+r"(W[5]), "+r"(W[6]),
          "+r"(W[7]), "+r"(W[8]), "+r"(W[9])
        : "r"(a), "r"(w[0]), "r"(w[2]), "r"(w[4]), "r"(w[6]));
    asm(MLO(0, 9, 10) MCHI(1, 9, 10) MCLO(2, 9, 11) MCHI(3, 9, 11)
        MCLO(4, 9, 12) MCHI(5, 9, 12) MCLO(6, 9, 13) MCHI(7, 9, 13)
        "addc.u32 %8, %8, 0;"
        : "+r"(W[1]), "+r"(W[2]), "+r"(W[3]), "+r"(W[4]), "+r"(W[5]), "+r"(W[6]), "+r"(W[7]),
          "+r"(W[8]), "+r"(W[9])
        : "r"(a), "r"(w[1]), "r"(w[3]), "r"(w[5]), "r"(w[7]));
}

template <>
__device__ __forceinline__ void mac_row<16>(uint32_t (&W)[18], uint32_t a, const uint32_t (&w)[16])
{
    asm(MLO(0, 18, 19) MCHI(1, 18, 19) MCLO(2, 18, 20) MCHI(3, 18, 20)
        MCLO(4, 18, 21) MCHI(5, 18, 21) MCLO(6, 18, 22) MCHI(7, 18, 22)
        MCLO(8, 18, 23) MCHI(9, 18, 23) MCLO(10, 18, 24) MCHI(11, 18, 24)
        MCLO(12, 18, 25) MCHI(13, 18, 25) MCLO(14, 18, 26) MCHI(15, 18, 26)
        "addc.cc.u32 %16, %16, 0;\n\t"
        "addc.u32 %17, %17, 0;"
        : "+r"(W[0]), "+r"(W[1]), "+r"(W[2]), "+r"(W[3]), "+r"(W[4]), "+r"(W[5]), "+r"(W[6]),
          "+r"(W[7]), "+r"(W[8]), "+r"(W[9]), "+r"(W[10]), "+r"(W[11]), "+r"(W[12]),
          "+r"(W[13]), "+r"(W[14]), "+r"(W[15]), "+r"(W[16]), "+r"(W[17])
        : "r"(a), "r"(w[0]), "r"(w[2]), "r"(w[4]), "r"(w[6]), "r"(w[8]), "r"(w[10]), "r"(w[12]),
          "r"(w[14]));
    asm(MLO(0, 17, 18) MCHI(1, 17, 18) MCLO(2, 17, 19) MCHI(3, 17, 19)
        MCLO(4, 17, 20) MCHI(5, 17, 20) MCLO(6, 17, 21) MCHI(7, 17, 21)
        MCLO(8, 17, 22) MCHI(9, 17, 22) MCLO(10, 17, 23) MCHI(11, 17, 23)
        MCLO(12, 17, 24) MCHI(13, 17, 24) MCLO(14, 17, 25) MCHI(15, 17, 25)
        "addc.u32 %16, %16, 0;"
        : "+r"(W[1]), "+r"(W[2]), "+r"(W[3]), "+r"(W[4]), "+r"(W[5]), "+r"(W[6]), "+r"(W[7]),
          "+r"(W[8]), "+r"(W[9]), "+r"(W[10]), "+r"(W[11]), "+r"(W[12]), "+r"(W[13]),
          "+r"(W[14]), "+r"(W[15]), "+r"(W[16]), "+r"(W[17])
        : "r"(a), "r"(w[1]), "r"(w[3]), "r"(w[5]), "r"(w[7]), "r"(w[9]), "r"(w[11]), "r"(w[13]),
          "r"(w[15]));
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
// [0, m)), both in shared memory.  Rows i are taken R at a time; the needed
// B values form a window that slides down by R per group.
template <int R>
__device__ __forceinline__ void colsum_block(const uint32_t *As, const uint32_t *Bs, int c0, int mp,
                                             uint32_t (&W)[R + 2])
{
#pragma unroll
    for (int k = 0; k < R + 2; ++k) W[k] = 0;
    const int i_lo = max(0, c0 - mp + 1);
    const int i_hi = min(c0 + R - 1, mp - 1);
    int i0 = (i_lo / R) * R;
    if (i0 > i_hi) return;
    uint32_t bw[2 * R];
    // window bw[q] = B[c0 - i0 - R + q]
    lds_vec<2 * R>(Bs + R + (c0 - i0 - R), bw);
    for (;;) {
        uint32_t av[R];
        lds_vec<R>(As + i0, av);
#pragma unroll
        for (int ii = 0; ii < R; ++ii) {
            uint32_t w[R];
#pragma unroll
            for (int k = 0; k < R; ++k) w[k] = bw[R + k - ii];
            mac_row<R>(W, av[ii], w);
        }
        i0 += R;
        if (i0 > i_hi) break;
#pragma unroll
        for (int q = 0; q < R; ++q) bw[R + q] = bw[q];
        lds_vec<R>(Bs + R + (c0 - i0 - R), bw);
    }
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
// part without touching memory.
template <int R>
__device__ __forceinline__ void mul_group(const uint32_t *As, const uint32_t *Bs, int t, int T,
                                          int tn, int grp, bool on, int m, int mp, uint32_t *prow,
                                          bool vec_out, uint32_t smask, uint32_t tmask)
{
    const int lane = (int)lane_id();
    on = on && t < tn;
    uint32_t W0[R + 2], W1[R + 2];
    if (on) {
        colsum_block<R>(As, Bs, t * R, mp, W0);
        colsum_block<R>(As, Bs, mp + t * R, mp, W1);
    } else {
#pragma unroll
        for (int k = 0; k < R + 2; ++k) W0[k] = W1[k] = 0;
    }
    // overflow words of each block move to the next block in position order
    const int last = min(grp * T + max(tn, 1) - 1, 31);
    const uint32_t u0l = __shfl_up_sync(DOT_FULL, W0[R], 1), u0h = __shfl_up_sync(DOT_FULL, W0[R + 1], 1);
    const uint32_t u1l = __shfl_up_sync(DOT_FULL, W1[R], 1), u1h = __shfl_up_sync(DOT_FULL, W1[R + 1], 1);
    const uint32_t wl = __shfl_sync(DOT_FULL, W0[R], last), wh = __shfl_sync(DOT_FULL, W0[R + 1], last);
    uint32_t h0[R], h1[R], l0[R], l1[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        h0[k] = h1[k] = 0;
        l0[k] = W0[k];
        l1[k] = W1[k];
    }
    h0[0] = t ? u0l : 0u;
    h0[1] = t ? u0h : 0u;
    h1[0] = t ? u1l : wl;
    h1[1] = t ? u1h : wh;
    Segment<false, R> s0, s1;
    s0.phase12(l0, h0);
    s1.phase12(l1, h1);
    WarpCarry c0, c1;
    c0.resolve(on ? s0.g() : 0u, on ? s0.p() : 0u, 0u, smask, tmask);
    const uint32_t mid = c0.carry_out(last);   // carry from the low half into the high half
    c1.resolve(on ? s1.g() : 0u, on ? s1.p() : 0u, t == 0 ? mid : 0u, smask, tmask);
    s0.apply(c0.carry_in(lane));
    s1.apply(c1.carry_in(lane));
    if (on) {
        store_block<R>(prow, t * R, 2 * m, s0.r, vec_out);
        store_block<R>(prow, mp + t * R, 2 * m, s1.r, vec_out);
    }
}

