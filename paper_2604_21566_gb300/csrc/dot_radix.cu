// dot_radix.cu -- batched products in an unsaturated radix.
//
// Sec. 2.1 contrasts the saturated limb representation (radix 2^32 or 2^64)
// with an unsaturated one that keeps headroom in every limb to simplify
// carry handling; the paper's 5x5 multiply runs on 52-bit digits because its
// IFMA multiplier takes 52-bit operands (Sec. 3.3).  Here the multiplier is
// the 32 x 32 -> 64-bit integer multiply, and the digits are 27 bits wide, so
// that one column sum of up to 2^10 digit products (each below 2^54) fits a
// 64-bit word: each partial product is ONE mad.wide.u32 into its column, with
// no carry chain (the saturated form needs two multiplies and a three-word
// add chain per product, csrc/dot_mul.cuh).  The price is more products:
// (32/27)^2 = 1.40x as many for the same number of bits.
//
// Structure as dot_mul (Alg. 2 on warps): lane t of an op's run owns the low
// column block [tR, tR + R) and the high block [n' + tR, ...), both summed in
// one row loop over operands staged in shared memory; each block's column
// sums become R + 2 digits (its positional value in radix 2^27); the blocks'
// two overflow digits overlap the next block, and that multi-digit addition
// is resolved with the warp lookahead, in radix 2^27: a digit sum r of two
// digits generates when r >= 2^27 and propagates when r == 2^27 - 1.
#include "dot_internal.cuh"
#include "dot_plan.h"
#include "dot_mul.cuh"

#define UNSAT_MASK ((1u << DOT_UNSAT_BITS) - 1u)

// One digit product into a 64-bit column sum.
__device__ __forceinline__ void mad27(uint64_t &s, uint32_t a, uint32_t w)
{
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(s) : "r"(a), "r"(w));
}

// Positional value sum_k S_k 2^(27 k) of a block as R + 2 digits: each S_k is
// below 2^63 (n <= 512 digits), the carry below 2^37, so two digits beyond the
// block hold the rest.
template <int R>
__device__ __forceinline__ void digits27(const uint64_t (&S)[R], uint32_t (&W)[R + 2])
{
    uint64_t c = 0;
#pragma unroll
    for (int j = 0; j < R + 2; ++j) {
        const uint64_t t = c + (j < R ? S[j] : 0ull);
        W[j] = (uint32_t)t & UNSAT_MASK;
        c = t >> DOT_UNSAT_BITS;
    }
}

// Column sums of lane t's two blocks, as colsum_pair in dot_mul.cuh (same row
// loop, window sliding down by one per row), with 64-bit sums.
template <int R>
__device__ __forceinline__ void colsum27_pair(const uint32_t *As, const uint32_t *Bs, int t, int T, int mp,
                                              uint32_t (&Wl)[R + 2], uint32_t (&Wh)[R + 2])
{
    uint64_t s[R], l[R];
#pragma unroll
    for (int k = 0; k < R; ++k) s[k] = l[k] = 0;
    uint32_t w[R];
    lds_vec<R>(Bs + R + t * R, w);   // w[k] = B[tR + k]: the low block at row 0
    int cb = t * R, i0 = 0;
    for (int g = 0; g <= T; ++g) {
        if (g == t + 1) {
#pragma unroll
            for (int k = 0; k < R; ++k) l[k] = s[k];
            cb = mp + t * R;
            i0 = t * R;
            lds_vec<R>(Bs + R + mp, w);   // B[m' + k]: zero padding
        }
#pragma unroll
        for (int ii = 0; ii < R; ++ii) {
            const uint32_t a = As[i0 + ii];
#pragma unroll
            for (int k = 0; k < R; ++k) mad27(s[k], a, w[k]);
#pragma unroll
            for (int k = R - 1; k > 0; --k) w[k] = w[k - 1];
            w[0] = Bs[R + cb - (i0 + ii) - 1];
        }
        i0 += R;
    }
#pragma unroll
    for (int k = 0; k < R; ++k) s[k] -= l[k];
    digits27<R>(l, Wl);
    digits27<R>(s, Wh);
}

// A segment of SEG digit sums r_i = x_i + y_i (each below 2^28): generate and
// propagate bits in radix 2^27, and the resolved digits.
template <int SEG>
struct Segment27 {
    uint32_t r[SEG];
    uint32_t gm, pm;

    __device__ __forceinline__ void phase12(const uint32_t (&x)[SEG], const uint32_t (&y)[SEG])
    {
        gm = pm = 0;
#pragma unroll
        for (int i = 0; i < SEG; ++i) {
            r[i] = x[i] + y[i];
            gm |= (r[i] >> DOT_UNSAT_BITS) << i;
            pm |= (uint32_t)(r[i] == UNSAT_MASK) << i;
        }
    }
    __device__ __forceinline__ uint32_t g() const { return (((gm << 1) + pm) >> SEG) & 1u; }
    __device__ __forceinline__ uint32_t p() const { return pm == (SEG == 32 ? DOT_FULL : ((1u << SEG) - 1u)); }
    __device__ __forceinline__ void apply(uint32_t cin)
    {
        const uint32_t cm = (((gm << 1) | cin) + pm) ^ pm;
#pragma unroll
        for (int i = 0; i < SEG; ++i) r[i] = (r[i] + ((cm >> i) & 1u)) & UNSAT_MASK;
    }
};

// One op on a run of T lanes, as mul_group: the low half of the product is
// resolved and stored first, then the high half with the low half's carry.
template <int R>
__device__ __forceinline__ void mul27_group(const uint32_t *As, const uint32_t *Bs, int t, int T, int grp,
                                            bool on, int n, int mp, uint32_t *prow, bool vec_out, uint32_t smask,
                                            uint32_t tmask)
{
    const int lane = (int)lane_id();
    const int last = min(grp * T + T - 1, 31);
    uint32_t W[R + 2], WH[R + 2];
    uint32_t wl, wh, mid;
    if (on) {
        colsum27_pair<R>(As, Bs, t, T, mp, W, WH);
    } else {
#pragma unroll
        for (int k = 0; k < R + 2; ++k) W[k] = WH[k] = 0;
    }
    {   // low blocks: digit positions 0 .. m' - 1
        const uint32_t ul = __shfl_up_sync(DOT_FULL, W[R], 1), uh = __shfl_up_sync(DOT_FULL, W[R + 1], 1);
        wl = __shfl_sync(DOT_FULL, W[R], last);
        wh = __shfl_sync(DOT_FULL, W[R + 1], last);
        uint32_t l[R], h[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            l[k] = W[k];
            h[k] = 0;
        }
        h[0] = t ? ul : 0u;
        h[1] = t ? uh : 0u;
        Segment27<R> sg;
        sg.phase12(l, h);
        WarpCarry wc;
        wc.resolve(on ? sg.g() : 0u, on ? sg.p() : 0u, 0u, smask, tmask);
        mid = wc.carry_out(last);
        sg.apply(wc.carry_in(lane));
        if (on) store_block<R>(prow, t * R, 2 * n, sg.r, vec_out);
    }
    {   // high blocks
        const uint32_t ul = __shfl_up_sync(DOT_FULL, WH[R], 1), uh = __shfl_up_sync(DOT_FULL, WH[R + 1], 1);
        uint32_t l[R], h[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            l[k] = WH[k];
            h[k] = 0;
        }
        h[0] = t ? ul : wl;
        h[1] = t ? uh : wh;
        Segment27<R> sg;
        sg.phase12(l, h);
        WarpCarry wc;
        wc.resolve(on ? sg.g() : 0u, on ? sg.p() : 0u, t == 0 ? mid : 0u, smask, tmask);
        sg.apply(wc.carry_in(lane));
        if (on) store_block<R>(prow, mp + t * R, 2 * n, sg.r, vec_out);
    }
}

template <int R>
__global__ void __launch_bounds__(MUL_WARPS * 32, R <= 8 ? 4 : 2)
mul_unsat_kernel(const uint32_t *a, const uint32_t *b, uint32_t *p, int n, int mp, int T, size_t batch,
                 int vec_in, int vec_out, uint32_t *status)
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
        uint32_t bad = 0;
        if (on) {
            stage_row<R>(a + op * (size_t)n, As, t, n, vec_in);
            stage_row<R>(b + op * (size_t)n, Bs + R, t, n, vec_in);
#pragma unroll
            for (int k = 0; k < R; ++k) bad |= As[t * R + k] | Bs[R + t * R + k];
        }
        // a digit of 2^27 or more is outside the representation: recorded,
        // and that op's product is unspecified
        if (__ballot_sync(DOT_FULL, (bad >> DOT_UNSAT_BITS) != 0) && lane == 0) record_status(status, DOT_EINVAL);
        __syncwarp();
        mul27_group<R>(As, Bs, t, T, grp, on, n, mp, p + op * 2 * (size_t)n, vec_out != 0, smask, tmask);
        __syncwarp();
    }
}

template <int R>
static dot_status_t launch_unsat(dot_ctx_t ctx, const dot_plan_t &pl, const uint32_t *a, const uint32_t *b,
                                 uint32_t *p, size_t n, size_t batch, cudaStream_t st)
{
    const int T = pl.lanes_per_op, mp = (int)pl.m_pad;
    const int opw = 32 / T;
    const size_t smem = (size_t)MUL_WARPS * opw * (2 * mp + 2 * R) * 4;
    const void *fn = (const void *)mul_unsat_kernel<R>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DOT_ECUDA;
    const bool vec_in = (n % 4 == 0) && aligned16(a) && aligned16(b);
    const bool vec_out = (n % 2 == 0) && aligned16(p);
    const size_t need = dot_ceil_div(batch, (size_t)opw * MUL_WARPS);
    const size_t cap = (size_t)ctx->num_sms * dot_blocks_per_sm(fn, MUL_WARPS * 32, smem);
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    mul_unsat_kernel<R><<<grid, MUL_WARPS * 32, smem, st>>>(a, b, p, (int)n, mp, T, batch, vec_in, vec_out,
                                                           ctx->d_status);
    return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
}

extern "C" DOT_API dot_status_t dot_mul_unsat(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *p,
                                              size_t n, size_t batch, dot_stream_t stream)
{
    DeviceScope scope;
    dot_status_t rc = dot_check_ctx(ctx, scope);
    if (rc != DOT_OK) return rc;
    if (batch == 0 || n == 0) return DOT_OK;
    if (n > DOT_UNSAT_MAX_DIGITS) return DOT_EUNSUPPORTED;
    if (!a || !b || !p) return DOT_EINVAL;
    if (batch > SIZE_MAX / 8 / n) return DOT_EINVAL;
    const size_t in = n * batch * 4, out = 2 * in;
    if (any_overlap(p, out, a, in) || any_overlap(p, out, b, in)) return DOT_EINVAL;
    // the column-block shape of the saturated multiply fits the same digit
    // counts (always the column-sum plan, whatever the size)
    dot_plan_t pl;
    rc = dot_make_plan(DOT_OP_MUL, n, batch, true, &pl, dot_mul_cols(n));
    if (rc != DOT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    switch (pl.seg_limbs) {
    case 4: return launch_unsat<4>(ctx, pl, a, b, p, n, batch, st);
    case 8: return launch_unsat<8>(ctx, pl, a, b, p, n, batch, st);
    case 12: return launch_unsat<12>(ctx, pl, a, b, p, n, batch, st);
    default: return launch_unsat<16>(ctx, pl, a, b, p, n, batch, st);
    }
}
