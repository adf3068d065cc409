// dot_mul.cu -- batched and ragged multi-limb multiplication.
//
// DoT multiplication (Alg. 2, Theorem 2, Sec. 3.2) computes every partial
// product A_i * B_j independently, sums them by output column c = i + j
// ("vertical and crosswise"), and resolves the column overflows in a separate
// carry pass.  On the GPU:
//  * Column sums (Alg. 2 Phases 1-4).  Thread t of an op's group owns two
//    blocks of R consecutive columns, [tR, tR+R) and [m' + tR, m' + tR + R)
//    (m' = m rounded up to R), so every thread does the same m' R products:
//    column c has c+1 pairs and column m'+c has m'-1-c.  For each i it adds
//    the R products A_i * B_{c-i} of its block into a positional accumulator
//    W = sum_k S_{c0+k} X^k of R+2 words.  The products of even k occupy
//    disjoint word pairs (k, k+1), and so do those of odd k, so each half is
//    one unbroken mad.lo.cc / madc.hi.cc carry chain: 2 IMAD-class
//    instructions per product plus 3 per row.  Phase 1's gather is index
//    arithmetic on operands staged in shared memory; nothing is materialised.
//  * Carry resolution (Alg. 2 Phase 5), made parallel.  A block's two top
//    words overlap the next block's two bottom words, so the product is
//    L + H: L the blocks' low R words side by side, H their overflow words
//    shifted to the next block.  That is one multi-limb addition, resolved
//    with the add kernel's generate/propagate lookahead across the group's
//    lanes (low blocks first, then high blocks).
#include "dot_internal.cuh"
#include "dot_plan.h"

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

// One op on a run of T lanes (lane t of the run, grp-th run of the warp).
// Every lane of the warp must call this (it uses warp collectives); lanes with
// on == false take part without touching memory.
template <int R>
__device__ __forceinline__ void mul_group(const uint32_t *As, const uint32_t *Bs, int t, int T,
                                          int grp, bool on, int m, int mp, uint32_t *prow,
                                          bool vec_out, uint32_t smask, uint32_t tmask)
{
    const int lane = (int)lane_id();
    uint32_t W0[R + 2], W1[R + 2];
    if (on) {
        colsum_block<R>(As, Bs, t * R, mp, W0);
        colsum_block<R>(As, Bs, mp + t * R, mp, W1);
    } else {
#pragma unroll
        for (int k = 0; k < R + 2; ++k) W0[k] = W1[k] = 0;
    }
    // overflow words of each block move to the next block in position order
    const int last = min(grp * T + T - 1, 31);
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

// Batched product: runs of T = m'/R lanes, 32/T ops per warp.
template <int R>
__global__ void __launch_bounds__(MUL_WARPS * 32)
mul_batched_kernel(const uint32_t *a, const uint32_t *b, uint32_t *p, int m, int mp, int T,
                   size_t batch, int vec_in, int vec_out)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
    const int opw = 32 / T;
    const int grp = lane / T, t = lane - grp * T;
    const bool lane_on = grp < opw;
    const int region = 2 * mp + 2 * R;
    uint32_t *As = smem + (size_t)(warp * opw + (lane_on ? grp : 0)) * region;
    uint32_t *Bs = As + mp;
    const uint32_t smask = run_start_mask(T), tmask = run_top_mask(T);
    // the B pads never change
    if (lane_on) {
        for (int k = t; k < R; k += T) {
            Bs[k] = 0;
            Bs[R + mp + k] = 0;
        }
    }
    const size_t wglobal = (size_t)blockIdx.x * MUL_WARPS + warp;
    const size_t nw = (size_t)gridDim.x * MUL_WARPS;
    for (size_t op0 = wglobal * opw; op0 < batch; op0 += nw * opw) {
        const size_t op = op0 + grp;
        const bool on = lane_on && op < batch;
        if (on) {
            stage_row<R>(a + op * (size_t)m, As, t, m, vec_in);
            stage_row<R>(b + op * (size_t)m, Bs + R, t, m, vec_in);
        }
        __syncwarp();
        mul_group<R>(As, Bs, t, T, grp, on, m, mp, p + op * 2 * (size_t)m, vec_out, smask, tmask);
        __syncwarp();
    }
}

// Ragged product: one op per warp, T = ceil(m_k / R) lanes; ops of m_k > 32 R
// are left to a kernel with larger R (size classes), m_k > DOT_MUL_MAX_LIMBS
// records DOT_EUNSUPPORTED.
template <int R>
__global__ void __launch_bounds__(MUL_WARPS * 32)
mul_ragged_kernel(const uint32_t *a, const uint32_t *b, uint32_t *p, const uint64_t *off,
                  const uint64_t *poff, size_t batch, int m_min, int m_max, uint32_t *status)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
    constexpr int MPMAX = 32 * R;
    uint32_t *As = smem + (size_t)warp * (2 * MPMAX + 2 * R);
    const size_t wglobal = (size_t)blockIdx.x * MUL_WARPS + warp;
    const size_t nw = (size_t)gridDim.x * MUL_WARPS;
    for (size_t op = wglobal; op < batch; op += nw) {
        const uint64_t lo = off[op], hi = off[op + 1];
        if (hi < lo) {
            if (lane == 0 && m_min == 0) record_status(status, DOT_EINVAL);
            continue;
        }
        const uint64_t m64 = hi - lo;
        if (m64 > DOT_MUL_MAX_LIMBS) {
            if (lane == 0 && m_min == 0) record_status(status, DOT_EUNSUPPORTED);
            continue;
        }
        const int m = (int)m64;
        if (m < m_min || m > m_max || m == 0) continue;
        const int T = (m + R - 1) / R;
        const int mp = T * R;
        uint32_t *Bs = As + mp;
        const int t = lane;
        const bool on = lane < T;
        const bool vec_in = ((lo & 3) == 0) && ((m & 3) == 0) && aligned16(a) && aligned16(b);
        const bool vec_out = ((poff[op] & 3) == 0) && ((m & 1) == 0) && aligned16(p);
        if (on) {
            stage_row<R>(a + lo, As, t, m, vec_in);
            stage_row<R>(b + lo, Bs + R, t, m, vec_in);
        }
        for (int k = lane; k < R; k += 32) {
            Bs[k] = 0;
            Bs[R + mp + k] = 0;
        }
        __syncwarp();
        mul_group<R>(As, Bs, t, T, 0, on, m, mp, p + poff[op], vec_out, run_start_mask(T), run_top_mask(T));
        __syncwarp();
    }
}

// ------------------------------------------------------------- launchers
template <int R>
static dot_status_t launch_mul_batched(dot_ctx_t ctx, const dot_plan_t &pl, const uint32_t *a,
                                       const uint32_t *b, uint32_t *p, size_t m, size_t batch,
                                       cudaStream_t st)
{
    const int T = pl.lanes_per_op, mp = (int)pl.m_pad;
    const int opw = 32 / T;
    const size_t smem = (size_t)MUL_WARPS * opw * (2 * mp + 2 * R) * 4;
    const void *fn = (const void *)mul_batched_kernel<R>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DOT_ECUDA;
    const bool vec_in = (m % 4 == 0) && aligned16(a) && aligned16(b);
    const bool vec_out = (m % 2 == 0) && aligned16(p);
    const size_t need = dot_ceil_div(batch, (size_t)opw * MUL_WARPS);
    const size_t cap = (size_t)ctx->num_sms * dot_blocks_per_sm(fn, MUL_WARPS * 32, smem);
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    mul_batched_kernel<R><<<grid, MUL_WARPS * 32, smem, st>>>(a, b, p, (int)m, mp, T, batch, vec_in, vec_out);
    return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
}

template <int R>
static dot_status_t launch_mul_ragged(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *p,
                                      const uint64_t *off, const uint64_t *poff, size_t batch,
                                      int m_min, int m_max, cudaStream_t st)
{
    const size_t smem = (size_t)MUL_WARPS * (2 * 32 * R + 2 * R) * 4;
    const void *fn = (const void *)mul_ragged_kernel<R>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DOT_ECUDA;
    const size_t need = dot_ceil_div(batch, (size_t)MUL_WARPS);
    const size_t cap = (size_t)ctx->num_sms * dot_blocks_per_sm(fn, MUL_WARPS * 32, smem);
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    mul_ragged_kernel<R><<<grid, MUL_WARPS * 32, smem, st>>>(a, b, p, off, poff, batch, m_min, m_max,
                                                            ctx->d_status);
    return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
}

extern "C" {

DOT_API dot_status_t dot_mul(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *p, size_t m,
                             size_t batch, dot_stream_t stream)
{
    dot_status_t rc = dot_check_ctx(ctx);
    if (rc != DOT_OK) return rc;
    if (batch == 0 || m == 0) return DOT_OK;
    if (m > DOT_MUL_MAX_LIMBS) return DOT_EUNSUPPORTED;
    if (!a || !b || !p) return DOT_EINVAL;
    if (batch > SIZE_MAX / 8 / m) return DOT_EINVAL;
    const size_t in = m * batch * 4, out = 2 * in;
    if (any_overlap(p, out, a, in) || any_overlap(p, out, b, in)) return DOT_EINVAL;
    dot_plan_t pl;
    rc = dot_make_plan(DOT_OP_MUL, m, batch, true, &pl);
    if (rc != DOT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    switch (pl.seg_limbs) {
    case 4: return launch_mul_batched<4>(ctx, pl, a, b, p, m, batch, st);
    case 8: return launch_mul_batched<8>(ctx, pl, a, b, p, m, batch, st);
    default: return launch_mul_batched<16>(ctx, pl, a, b, p, m, batch, st);
    }
}

DOT_API dot_status_t dot_mul_ragged(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *p,
                                    const uint64_t *off, const uint64_t *poff, size_t batch,
                                    dot_stream_t stream)
{
    dot_status_t rc = dot_check_ctx(ctx);
    if (rc != DOT_OK) return rc;
    if (batch == 0) return DOT_OK;
    if (!a || !b || !p || !off || !poff) return DOT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // size classes: R = 8 handles m <= 256, R = 16 handles 256 < m <= 512
    rc = launch_mul_ragged<8>(ctx, a, b, p, off, poff, batch, 0, 256, st);
    if (rc != DOT_OK) return rc;
    return launch_mul_ragged<16>(ctx, a, b, p, off, poff, batch, 257, DOT_MUL_MAX_LIMBS, st);
}

}  // extern "C"
