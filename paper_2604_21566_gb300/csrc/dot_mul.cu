// dot_mul.cu -- batched and ragged multi-limb multiplication.
//
// DoT multiplication (Alg. 2, Theorem 2, Sec. 3.2) computes every partial
// product A_i * B_j independently, sums them by output column c = i + j
// ("vertical and crosswise"), and resolves the column overflows in a separate
// carry pass.  On the GPU:
//  * Column sums (Alg. 2 Phases 1-4).  Thread t of an op's group owns two
//    blocks of R consecutive columns, [tR, tR+R) and [m' + tR, m' + tR + R)
//    (m' = m rounded up to R), so every thread does the same m' R products:
//    column c has c+1 pairs and column m'+c has m'-1-c.  Both blocks run in
//    one loop over row groups (low block first), so no lane of a warp idles
//    while another finishes a longer block.  For each i it forms
//    the R products A_i * B_{c-i} of its block independently (low and high
//    halves: 2 multiplies on the FMA pipe) and adds each into its column's
//    three-word sum (3 adds on the ALU pipe, in parallel with the next
//    multiplies).  At the end of the block the R column sums become one
//    positional value W = sum_k S_{c0+k} X^k of R+2 words.  Phase 1's gather
//    is index arithmetic on operands staged in shared memory; nothing is
//    materialised.
//  * Carry resolution (Alg. 2 Phase 5), made parallel.  A block's two top
//    words overlap the next block's two bottom words, so the product is
//    L + H: L the blocks' low R words side by side, H their overflow words
//    shifted to the next block.  That is one multi-limb addition, resolved
//    with the add kernel's generate/propagate lookahead across the group's
//    lanes (low blocks first, then high blocks).
#include "dot_internal.cuh"
#include "dot_plan.h"

#include "dot_mul.cuh"

// smallest operand (limbs) squared with the symmetric column sums
#define DOT_SQR_MIN_LIMBS 128

// Batched product: runs of T = m'/R lanes, 32/T ops per warp.  SQR: the
// square of a (b is a), with half the partial products.
template <int R, bool SQR>
__global__ void __launch_bounds__(MUL_WARPS * 32, dot_mul_min_blocks(R, SQR))
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
        mul_group<R, SQR>(As, Bs, t, T, T, grp, on, m, mp, p + op * 2 * (size_t)m, vec_out, smask, tmask);
        __syncwarp();
    }
}

// Ragged product: one op per warp, T = ceil(m_k / R) lanes; ops of m_k > 32 R
// are left to a kernel with larger R (size classes), m_k > DOT_MUL_MAX_LIMBS
// records DOT_EUNSUPPORTED.
template <int R>
__global__ void __launch_bounds__(MUL_WARPS * 32, dot_mul_min_blocks(R))
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
        mul_group<R>(As, Bs, t, T, T, 0, on, m, mp, p + poff[op], vec_out, run_start_mask(T), run_top_mask(T));
        __syncwarp();
    }
}

// ------------------------------------------------ one product per thread
// Operands of at most 16 limbs: each thread multiplies one pair held in
// registers (no shared memory, no warp collectives, so a launch of a few
// thousand products is one memory round trip).  Column c = i + j of the
// product collects x_i y_j in two three-word sums, over even and odd i (two
// independent add chains), and one carry pass turns the columns into the
// 2m limbs in order (Alg. 2 Phases 2-5 within one thread).  M >= m at compile
// time; limbs past m read as 0.
__device__ __forceinline__ void add3w(uint32_t &s0, uint32_t &s1, uint32_t &s2, uint32_t t0, uint32_t t1, uint32_t t2)
{
    asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, %5;"
        : "+r"(s0), "+r"(s1), "+r"(s2) : "r"(t0), "r"(t1), "r"(t2));
}

template <int M>
__global__ void __launch_bounds__(256)
mul_thread_kernel(const uint32_t *a, const uint32_t *b, uint32_t *p, int m, size_t batch, int vec_in, int vec_out)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t op = (size_t)blockIdx.x * blockDim.x + threadIdx.x; op < batch; op += stride) {
        uint32_t x[M], y[M];
        const uint32_t *ar = a + op * (size_t)m, *br = b + op * (size_t)m;
        if (vec_in) {   // m % 4 == 0 and 16-byte aligned rows
#pragma unroll
            for (int q = 0; q < M / 4; ++q) {
                uint4 u = make_uint4(0u, 0u, 0u, 0u), v = u;
                if (4 * q < m) {
                    u = ld_stream4(ar + 4 * q);
                    v = ld_stream4(br + 4 * q);
                }
                x[4 * q] = u.x; x[4 * q + 1] = u.y; x[4 * q + 2] = u.z; x[4 * q + 3] = u.w;
                y[4 * q] = v.x; y[4 * q + 1] = v.y; y[4 * q + 2] = v.z; y[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < M; ++i) {
                x[i] = i < m ? ld_stream1(ar + i) : 0u;
                y[i] = i < m ? ld_stream1(br + i) : 0u;
            }
        }
        uint32_t o[2 * M];
        uint32_t c0 = 0, c1 = 0, c2 = 0;   // carry into the column, three words
#pragma unroll
        for (int c = 0; c < 2 * M - 1; ++c) {
            uint32_t e0 = 0, e1 = 0, e2 = 0, d0 = 0, d1 = 0, d2 = 0;
#pragma unroll
            for (int i = (c - M + 1 > 0 ? c - M + 1 : 0); i <= (c < M - 1 ? c : M - 1); ++i) {
                if (i & 1) mac1(d0, d1, d2, x[i], y[c - i]);
                else mac1(e0, e1, e2, x[i], y[c - i]);
            }
            add3w(c0, c1, c2, e0, e1, e2);
            add3w(c0, c1, c2, d0, d1, d2);
            o[c] = c0;
            c0 = c1;
            c1 = c2;
            c2 = 0;
        }
        o[2 * M - 1] = c0;
        uint32_t *pr = p + op * 2 * (size_t)m;
        if (vec_out) {   // 2m % 4 == 0 and 16-byte aligned rows
#pragma unroll
            for (int q = 0; q < M / 2; ++q)
                if (4 * q < 2 * m) st_stream4(pr + 4 * q, make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]));
        } else {
#pragma unroll
            for (int c = 0; c < 2 * M; ++c)
                if (c < 2 * m) st_stream1(pr + c, o[c]);
        }
    }
}

// Products of 17..32 limbs, one per thread, for batches that give every SM
// many threads: the operands stay in registers, each column is summed in four
// interleaved chains (rows i mod 4, so that consecutive products do not wait
// on one carry chain), and the result leaves four limbs at a time as the
// columns complete instead of being held whole.  Blocks of 64 threads spread
// a batch of 2^16 over the SMs within one block of the mean (256-thread
// blocks left some SMs twice the work of others).
#define MUL_THREAD_WIDE_THREADS 64
template <int M>
__global__ void __launch_bounds__(MUL_THREAD_WIDE_THREADS)
mul_thread_wide_kernel(const uint32_t *a, const uint32_t *b, uint32_t *p, int m, size_t batch, int vec_in,
                       int vec_out)
{
    static_assert(M % 4 == 0, "columns leave in groups of four");
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t op = (size_t)blockIdx.x * blockDim.x + threadIdx.x; op < batch; op += stride) {
        uint32_t x[M], y[M];
        const uint32_t *ar = a + op * (size_t)m, *br = b + op * (size_t)m;
        if (vec_in) {   // m % 4 == 0 and 16-byte aligned rows
#pragma unroll
            for (int q = 0; q < M / 4; ++q) {
                uint4 u = make_uint4(0u, 0u, 0u, 0u), v = u;
                if (4 * q < m) {
                    u = ld_stream4(ar + 4 * q);
                    v = ld_stream4(br + 4 * q);
                }
                x[4 * q] = u.x; x[4 * q + 1] = u.y; x[4 * q + 2] = u.z; x[4 * q + 3] = u.w;
                y[4 * q] = v.x; y[4 * q + 1] = v.y; y[4 * q + 2] = v.z; y[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int i = 0; i < M; ++i) {
                x[i] = i < m ? ld_stream1(ar + i) : 0u;
                y[i] = i < m ? ld_stream1(br + i) : 0u;
            }
        }
        uint32_t *pr = p + op * 2 * (size_t)m;
        uint32_t ob[4];
        uint32_t c0 = 0, c1 = 0, c2 = 0;   // carry into the column, three words
#pragma unroll
        for (int c = 0; c < 2 * M; ++c) {
            if (c < 2 * M - 1) {
                uint32_t e[4][3];
#pragma unroll
                for (int q = 0; q < 4; ++q) e[q][0] = e[q][1] = e[q][2] = 0u;
#pragma unroll
                for (int i = (c - M + 1 > 0 ? c - M + 1 : 0); i <= (c < M - 1 ? c : M - 1); ++i)
                    mac1(e[i & 3][0], e[i & 3][1], e[i & 3][2], x[i], y[c - i]);
#pragma unroll
                for (int q = 0; q < 4; ++q) add3w(c0, c1, c2, e[q][0], e[q][1], e[q][2]);
                ob[c & 3] = c0;
                c0 = c1;
                c1 = c2;
                c2 = 0;
            } else {
                ob[c & 3] = c0;
            }
            if ((c & 3) == 3) {   // limbs c - 3 .. c are final
                const int c4 = c - 3;
                if (vec_out) {    // 2m % 4 == 0: a group is wholly inside the row or past it
                    if (c4 < 2 * m) st_stream4(pr + c4, make_uint4(ob[0], ob[1], ob[2], ob[3]));
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (c4 + k < 2 * m) st_stream1(pr + c4 + k, ob[k]);
                }
            }
        }
    }
}

template <int M>
static dot_status_t launch_mul_thread(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *p, size_t m,
                                      size_t batch, cudaStream_t st)
{
    const void *fn;
    if constexpr (M > DOT_MUL_THREAD_MAX) fn = (const void *)mul_thread_wide_kernel<M>;
    else fn = (const void *)mul_thread_kernel<M>;
    const bool vec_in = (m % 4 == 0) && aligned16(a) && aligned16(b);
    const bool vec_out = (m % 2 == 0) && aligned16(p);
    const int bs = M > DOT_MUL_THREAD_MAX ? MUL_THREAD_WIDE_THREADS : 256;
    const size_t need = dot_ceil_div(batch, (size_t)bs);
    const size_t cap = (size_t)ctx->num_sms * dot_blocks_per_sm(fn, bs, 0);
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    if constexpr (M > DOT_MUL_THREAD_MAX)
        mul_thread_wide_kernel<M><<<grid, MUL_THREAD_WIDE_THREADS, 0, st>>>(a, b, p, (int)m, batch, vec_in, vec_out);
    else
        mul_thread_kernel<M><<<grid, 256, 0, st>>>(a, b, p, (int)m, batch, vec_in, vec_out);
    return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
}

static dot_status_t launch_mul_thread_any(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *p,
                                          size_t m, size_t batch, cudaStream_t st)
{
    if (m <= 2) return launch_mul_thread<2>(ctx, a, b, p, m, batch, st);
    if (m <= 4) return launch_mul_thread<4>(ctx, a, b, p, m, batch, st);
    if (m <= 8) return launch_mul_thread<8>(ctx, a, b, p, m, batch, st);
    if (m <= 12) return launch_mul_thread<12>(ctx, a, b, p, m, batch, st);
    if (m <= 16) return launch_mul_thread<16>(ctx, a, b, p, m, batch, st);
    if (m <= 24) return launch_mul_thread<24>(ctx, a, b, p, m, batch, st);
    return launch_mul_thread<32>(ctx, a, b, p, m, batch, st);
}

// ------------------------------------------------------------- launchers
template <int R, bool SQR = false>
static dot_status_t launch_mul_batched(dot_ctx_t ctx, const dot_plan_t &pl, const uint32_t *a,
                                       const uint32_t *b, uint32_t *p, size_t m, size_t batch,
                                       cudaStream_t st)
{
    const int T = pl.lanes_per_op, mp = (int)pl.m_pad;
    const int opw = 32 / T;
    const size_t smem = (size_t)MUL_WARPS * opw * (2 * mp + 2 * R) * 4;
    const void *fn = (const void *)mul_batched_kernel<R, SQR>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DOT_ECUDA;
    const bool vec_in = (m % 4 == 0) && aligned16(a) && aligned16(b);
    const bool vec_out = (m % 2 == 0) && aligned16(p);
    const size_t need = dot_ceil_div(batch, (size_t)opw * MUL_WARPS);
    const size_t cap = (size_t)ctx->num_sms * dot_blocks_per_sm(fn, MUL_WARPS * 32, smem);
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    mul_batched_kernel<R, SQR><<<grid, MUL_WARPS * 32, smem, st>>>(a, b, p, (int)m, mp, T, batch, vec_in, vec_out);
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
    DeviceScope scope;
    dot_status_t rc = dot_check_ctx(ctx, scope);
    if (rc != DOT_OK) return rc;
    if (batch == 0 || m == 0) return DOT_OK;
    if (m > DOT_MUL_MAX_LIMBS) return DOT_EUNSUPPORTED;
    if (!a || !b || !p) return DOT_EINVAL;
    if (batch > SIZE_MAX / 8 / m) return DOT_EINVAL;
    const size_t in = m * batch * 4, out = 2 * in;
    if (any_overlap(p, out, a, in) || any_overlap(p, out, b, in)) return DOT_EINVAL;
    dot_plan_t pl;
    rc = dot_make_plan(DOT_OP_MUL, m, batch, true, &pl, ctx->tune[DOT_OP_MUL][dot_tune_bucket(m)]);
    if (rc != DOT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (pl.kernel == DOT_K_MUL_THREAD) return launch_mul_thread_any(ctx, a, b, p, m, batch, st);
    switch (pl.seg_limbs) {
    case 4: return launch_mul_batched<4>(ctx, pl, a, b, p, m, batch, st);
    case 8: return launch_mul_batched<8>(ctx, pl, a, b, p, m, batch, st);
    case 12: return launch_mul_batched<12>(ctx, pl, a, b, p, m, batch, st);
    default: return launch_mul_batched<16>(ctx, pl, a, b, p, m, batch, st);
    }
}

DOT_API dot_status_t dot_sqr(dot_ctx_t ctx, const uint32_t *a, uint32_t *p, size_t m, size_t batch,
                             dot_stream_t stream)
{
    DeviceScope scope;
    dot_status_t rc = dot_check_ctx(ctx, scope);
    if (rc != DOT_OK) return rc;
    if (batch == 0 || m == 0) return DOT_OK;
    if (m > DOT_MUL_MAX_LIMBS) return DOT_EUNSUPPORTED;
    if (!a || !p) return DOT_EINVAL;
    if (batch > SIZE_MAX / 8 / m) return DOT_EINVAL;
    const size_t in = m * batch * 4, out = 2 * in;
    if (any_overlap(p, out, a, in)) return DOT_EINVAL;
    dot_plan_t pl;
    const int knob = ctx->tune[DOT_OP_MUL][dot_tune_bucket(m)];
    rc = dot_make_plan(DOT_OP_MUL, m, batch, true, &pl, knob ? knob : dot_mul_cols(m, true));
    if (rc != DOT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (pl.kernel == DOT_K_MUL_THREAD) return launch_mul_thread_any(ctx, a, a, p, m, batch, st);
    // Below 128 limbs the rows near the diagonal, summed one column at a time,
    // cost about what the halving saves (measured against the general
    // product: 0.95x at m = 64, 1.21x at m = 128, 1.46x at m = 256), so small
    // squares take the general product.
    const bool sym = m >= DOT_SQR_MIN_LIMBS;
    switch (pl.seg_limbs) {
    case 4: return sym ? launch_mul_batched<4, true>(ctx, pl, a, a, p, m, batch, st)
                       : launch_mul_batched<4, false>(ctx, pl, a, a, p, m, batch, st);
    case 8: return sym ? launch_mul_batched<8, true>(ctx, pl, a, a, p, m, batch, st)
                       : launch_mul_batched<8, false>(ctx, pl, a, a, p, m, batch, st);
    case 12: return sym ? launch_mul_batched<12, true>(ctx, pl, a, a, p, m, batch, st)
                        : launch_mul_batched<12, false>(ctx, pl, a, a, p, m, batch, st);
    default: return sym ? launch_mul_batched<16, true>(ctx, pl, a, a, p, m, batch, st)
                        : launch_mul_batched<16, false>(ctx, pl, a, a, p, m, batch, st);
    }
}

DOT_API dot_status_t dot_mul_ragged(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *p,
                                    const uint64_t *off, const uint64_t *poff, size_t batch,
                                    dot_stream_t stream)
{
    DeviceScope scope;
    dot_status_t rc = dot_check_ctx(ctx, scope);
    if (rc != DOT_OK) return rc;
    if (batch == 0) return DOT_OK;
    if (!a || !b || !p || !off || !poff) return DOT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // size classes: R = 8 handles m <= 256, R = 12 256 < m <= 384 and R = 16
    // 384 < m <= 512, so that an op's ceil(m / R) lanes fill most of its warp
    rc = launch_mul_ragged<8>(ctx, a, b, p, off, poff, batch, 0, 256, st);
    if (rc != DOT_OK) return rc;
    rc = launch_mul_ragged<12>(ctx, a, b, p, off, poff, batch, 257, 384, st);
    if (rc != DOT_OK) return rc;
    return launch_mul_ragged<16>(ctx, a, b, p, off, poff, batch, 385, DOT_MUL_MAX_LIMBS, st);
}

}  // extern "C"
