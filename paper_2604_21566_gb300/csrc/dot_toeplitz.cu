// dot_toeplitz.cu -- one fixed operand times a batch of operands on the
// tensor cores (tcgen05.mma), and the same product on the INT32 path.
//
// Theorem 2 (Sec. 3.2) writes A*B as column sums S_c = sum_{i+j=c} A_i B_j.
// With 8-bit digits (bytes) instead of 32-bit limbs the column sums of a
// fixed A against many B_j form one matrix product:
//     C[j][c] = sum_t beta_{j,t} alpha_{c-t},   T[t][c] = alpha_{c-t},
// i.e. C = Bbytes x T with T an upper-banded Toeplitz matrix (K = 4m digits,
// 8m output columns).  Digits are 0..255, exact in fp16, and every C entry is
// at most K * 255^2 = 16,646,400 < 2^24 for K <= 256, so fp32 accumulation is
// exact.  The fp32 column sums are then regrouped four at a time into
// 32-bit-limb positions, L_l = sum_q C[4l + q] 2^(8q) < 2^49, and normalised
// by one carry pass per row (Alg. 2 Phase 5) in the epilogue.
//
// Kernel layout (one CTA of 512 threads per SM, persistent over tiles of 128
// operands; K = 256 digits, 512 output columns):
//   * T is block-Toeplitz in 128 x 128 blocks: block (k-block kb, column
//     block cb) depends only on d = cb - kb, and only d = 0, 1, 2 are nonzero.
//     The three distinct blocks (96 KB of fp16) are built once per CTA in
//     shared memory in the canonical no-swizzle K-major layout (row groups
//     of a k chunk contiguous).
//   * Each tile's digits are converted to fp16 into one of two 64 KB shared
//     tiles; the next tile is staged while the current tile's products run.
//   * One thread issues 6 block pairs x 8 k-steps of tcgen05.mma (M = 128,
//     N = 128, K = 16) into four 128-column fp32 accumulators in tensor memory
//     (all 512 columns), then commits to an mbarrier.
//   * Four warps per tensor-memory lane quadrant read the accumulators back
//     (tcgen05.ld), each a quarter of a row's columns, regroup them into limb
//     positions and resolve the carries with generate/propagate masks.
#include <cuda_fp16.h>
#include <string.h>

#include "dot_internal.cuh"
#include "dot_plan.h"
#include "dot_mul.cuh"

#define TZ_THREADS 512          // four warps per tensor-memory lane quadrant
#define TZ_M 128                 // operands per tile (MMA M)
#define TZ_K 256                 // digits per operand (bytes of 64 limbs)
#define TZ_NB 128                // columns per accumulator block (MMA N)
#define TZ_TBLOCK (128 * 128 * 2)            // bytes of one 128 x 128 fp16 block
#define TZ_ATILE (TZ_M * TZ_K * 2)           // bytes of one fp16 operand tile
#define TZ_SMEM (3 * TZ_TBLOCK + 2 * TZ_ATILE + 64 + TZ_K + 16 * TZ_M)
#define TZ_MAX_LIMBS 64

// ------------------------------------------------------------ tcgen05 glue
// Shared-memory matrix descriptor, canonical K-major layout without swizzle:
// core matrices of 8 rows x 16 bytes; lbo = byte distance between core
// matrices adjacent in K, sbo = between core matrices adjacent in M/N.
__device__ __forceinline__ uint64_t tz_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version bits 46..48 = 0b001; no swizzle
    return d;
}

// Byte offset of element (row, k) of a K-major tile of `rows` rows: core
// matrix (row group i, k chunk j) at (j * rows / 8 + i) * 128, so the row
// groups of one k chunk are contiguous (sbo = 128 B, lbo = rows * 16 B) and an
// MMA's k-slice is two contiguous blocks -- no shared-memory bank conflicts.
__device__ __forceinline__ uint32_t tz_off(int row, int k, int rows)
{
    return (uint32_t)((((k >> 3) * (rows >> 3) + (row >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

// instruction descriptor: D fp32, A and B fp16, both K-major, M = 128, N = 128
__device__ __forceinline__ uint32_t tz_idesc()
{
    return (1u << 4) | ((uint32_t)(TZ_NB >> 3) << 17) | ((uint32_t)(TZ_M >> 4) << 24);
}

__device__ __forceinline__ void tz_mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(dtmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void tz_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tz_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                   "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                   "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tz_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tz_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// two digit values (0..255) as a pair of fp16: 0x6400 | v encodes 1024 + v
__device__ __forceinline__ uint32_t tz_pack2(uint32_t v0, uint32_t v1)
{
    const uint32_t biased = 0x64006400u | v0 | (v1 << 16);
    __half2 h = *reinterpret_cast<const __half2 *>(&biased);
    h = __hsub2(h, __halves2half2(__ushort_as_half(0x6400), __ushort_as_half(0x6400)));
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Two digits (bytes sel of x) as a pair of fp16 values without conversion
// instructions: 0x6400 | v is the fp16 encoding of 1024 + v (v < 1024), and
// one packed half subtraction of 1024 leaves v exactly.
__device__ __forceinline__ uint32_t tz_digits2(uint32_t x, uint32_t sel)
{
    const uint32_t biased = __byte_perm(x, 0x64u, sel);   // bytes [d0, 0x64, d1, 0x64]
    __half2 h = *reinterpret_cast<const __half2 *>(&biased);
    h = __hsub2(h, __halves2half2(__ushort_as_half(0x6400), __ushort_as_half(0x6400)));
    return *reinterpret_cast<const uint32_t *>(&h);
}

// four digits of limb x -> two fp16 pairs
__device__ __forceinline__ uint32_t tz_lo_pair(uint32_t x) { return tz_digits2(x, 0x4140); }
__device__ __forceinline__ uint32_t tz_hi_pair(uint32_t x) { return tz_digits2(x, 0x4342); }

// an exact fp32 integer below 2^24 as uint32, with ALU operations only:
// mantissa with its hidden bit, shifted right by (150 - biased exponent)
__device__ __forceinline__ uint32_t tz_f2u(uint32_t bits)
{
    const uint32_t mant = (bits & 0x7FFFFFu) | 0x800000u;
    return __funnelshift_rc(mant, 0u, 150u - (bits >> 23));
}

// --------------------------------------------------------------- kernel
// Stage one tile's digits as fp16 into a K-major operand tile.  Four threads
// share each operand row (tid & 127), a quarter row (16 limbs, 64 digits)
// each; every load is issued before any is used.
__device__ __forceinline__ void tz_stage(unsigned char *sA, const uint32_t *b, int m, size_t batch, size_t tile,
                                         int tid)
{
    const int row = tid & (TZ_M - 1), qr = tid >> 7;
    const size_t op = tile * TZ_M + row;
    const uint32_t *src = b + op * (size_t)m + 16 * qr;
    uint32_t x[16];
    if (op < batch && m == TZ_MAX_LIMBS && aligned16(src)) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(src) + q);
            x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int l = 0; l < 16; ++l) x[l] = (op < batch && 16 * qr + l < m) ? __ldcs(src + l) : 0u;
    }
#pragma unroll
    for (int l2 = 0; l2 < 8; ++l2) {   // two limbs = 8 digits per store
        const uint32_t x0 = x[2 * l2], x1 = x[2 * l2 + 1];
        const uint4 v = make_uint4(tz_lo_pair(x0), tz_hi_pair(x0), tz_lo_pair(x1), tz_hi_pair(x1));
        *reinterpret_cast<uint4 *>(sA + tz_off(row, 64 * qr + 8 * l2, TZ_M)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// fixed: m limbs (m <= 64), b: [batch][m], p: [batch][2m].
// Per CTA: the Toeplitz blocks once, then for each of its tiles: issue the
// tile's products (operand buffer it & 1), stage the next tile into the other
// buffer while they run, wait, and drain the accumulators.
__global__ void __launch_bounds__(TZ_THREADS, 1)
toeplitz_mma_kernel(const uint32_t *fixed, const uint32_t *b, uint32_t *p, int m, size_t batch,
                    uint32_t *status, uint64_t wait_ns)
{
    extern __shared__ __align__(128) unsigned char tz_smem[];
    unsigned char *sT = tz_smem;                       // 3 Toeplitz blocks, d = 0, 1, 2
    unsigned char *sA0 = tz_smem + 3 * TZ_TBLOCK;      // operand tiles (double buffer)
    uint64_t *bar = (uint64_t *)(sA0 + 2 * TZ_ATILE);
    uint32_t *tmem_slot = (uint32_t *)(bar + 1);
    unsigned char *alpha = (unsigned char *)(bar + 8);
    uint32_t *xch = (uint32_t *)(alpha + TZ_K);        // [quarter][row]: top high word, then (g, p)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    // digits of the fixed operand (zero beyond its m limbs)
    for (int k = tid; k < TZ_K; k += TZ_THREADS)
        alpha[k] = (k < 4 * m) ? (unsigned char)(fixed[k >> 2] >> (8 * (k & 3))) : 0;
    __syncthreads();
    // Toeplitz block d, element (n, k) = alpha[128 d + n - k] when 0 <= . < 256
    for (int idx = tid; idx < 3 * 128 * 16; idx += TZ_THREADS) {
        const int d = idx / (128 * 16), rem = idx - d * 128 * 16, n = rem & 127, kc = rem >> 7;
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            uint32_t v[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int k = kc * 8 + 2 * h + e;
                const int s = 128 * d + n - k;
                v[e] = (s >= 0 && s < TZ_K) ? alpha[s] : 0u;
            }
            w[h] = tz_pack2(v[0], v[1]);
        }
        *reinterpret_cast<uint4 *>(sT + d * TZ_TBLOCK + tz_off(n, kc * 8, 128)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const size_t ntiles = (batch + TZ_M - 1) / TZ_M;
    if (blockIdx.x < ntiles) tz_stage(sA0, b, m, batch, blockIdx.x, tid);
    tz_fence_before();
    __syncthreads();
    tz_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = tz_idesc();
    const int quad = warp & 3, qc = warp >> 2;   // TMEM lane quadrant, column quarter
    const int row = 32 * quad + lane;
    uint32_t phase = 0;
    bool failed = false;

    int it = 0;
    for (size_t tile = blockIdx.x; tile < ntiles && !failed; tile += gridDim.x, ++it) {
        unsigned char *sA = sA0 + (it & 1) * TZ_ATILE;
        // ---- one thread issues the block products of this tile
        if (tid == 0) {
#pragma unroll 1
            for (int cb = 0; cb < 4; ++cb) {
                uint32_t acc = 0;
#pragma unroll 1
                for (int kb = 0; kb < 2; ++kb) {
                    const int d = cb - kb;
                    if (d < 0 || d > 2) continue;
#pragma unroll
                    for (int s = 0; s < 8; ++s) {
                        const uint64_t ad = tz_desc(smem_u32(sA) + (uint32_t)(16 * kb + 2 * s) * (TZ_M * 16), TZ_M * 16, 128);
                        const uint64_t bd = tz_desc(smem_u32(sT + d * TZ_TBLOCK) + (uint32_t)(2 * s) * (128 * 16), 128 * 16, 128);
                        tz_mma(tmem + (uint32_t)(cb * TZ_NB), ad, bd, idesc, acc);
                        acc = 1;
                    }
                }
            }
            tz_commit(bar);
        }
        // ---- stage the next tile into the other buffer while the products run
        const size_t next = tile + gridDim.x;
        if (next < ntiles) tz_stage(sA0 + ((it + 1) & 1) * TZ_ATILE, b, m, batch, next, tid);
        // ---- the products are done (or the bounded wait ran out: then record
        // it, give them one more period to drain, and stop after this tile)
        const int late = !mbar_wait_bounded(bar, phase, wait_ns);
        failed = __syncthreads_or(late) != 0;
        if (failed) {
            if (tid == 0) record_status(status, DOT_ETIMEOUT);
            mbar_wait_bounded(bar, phase, wait_ns);
        }
        phase ^= 1u;
        tz_fence_after();
        // ---- epilogue: limbs [32 qc, 32 qc + 32) of operand row `row`.
        // Each limb position collects L_l = sum_q C[4l + q] 2^(8q) < 2^49; with
        // lo_l = L_l mod 2^32 and hi_l = L_l >> 32 the product is the two-term
        // sum  sum_l lo_l X^l + sum_l hi_l X^(l+1), whose 1-bit carries are
        // resolved by the Phase 4 mask identity inside each quarter and by the
        // quarters' published (generate, propagate) pairs across quarters.
        {
            uint32_t r[32];
            uint32_t G = 0, Pm = 0;
            uint32_t hi_prev = 0, lo_first = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                uint32_t v[32];
                tz_ld32(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(128 * qc + 32 * c), v);
#pragma unroll
                for (int l = 0; l < 8; ++l) {
                    const int li = 8 * c + l;
                    // exact fp32 integers -> uint32: half on the XU, half on the ALU
                    const uint32_t f0 = __float2uint_rz(__uint_as_float(v[4 * l]));
                    const uint32_t f1 = tz_f2u(v[4 * l + 1]);
                    const uint32_t f2 = __float2uint_rz(__uint_as_float(v[4 * l + 2]));
                    const uint32_t f3 = tz_f2u(v[4 * l + 3]);
                    uint64_t L = (uint64_t)f1 * 256u + f0;
                    L += (uint64_t)f2 * 65536u;
                    L += (uint64_t)f3 * 16777216u;
                    const uint32_t lo = (uint32_t)L;
                    if (li == 0) {
                        lo_first = lo;   // its high-word partner comes from the previous quarter
                        r[0] = lo;
                    } else {
                        r[li] = lo + hi_prev;
                        G |= (uint32_t)(r[li] < lo) << li;
                        Pm |= (uint32_t)(r[li] == DOT_FULL) << li;
                    }
                    hi_prev = (uint32_t)(L >> 32);
                }
            }
            xch[qc * TZ_M + row] = hi_prev;   // top high word of this quarter
            __syncthreads();
            const uint32_t h_in = qc ? xch[(qc - 1) * TZ_M + row] : 0u;
            r[0] = lo_first + h_in;
            G |= (uint32_t)(r[0] < lo_first);
            Pm |= (uint32_t)(r[0] == DOT_FULL);
            // quarter aggregate: carry out with carry-in 0, and "all limbs propagate"
            const uint32_t g_q = (uint32_t)((((uint64_t)G << 1) + Pm) >> 32) & 1u;
            const uint32_t p_q = Pm == DOT_FULL;
            __syncthreads();
            xch[qc * TZ_M + row] = g_q | (p_q << 1);
            __syncthreads();
            uint32_t cin = 0;
            for (int q = 0; q < qc; ++q) {
                const uint32_t gp = xch[q * TZ_M + row];
                cin = (gp & 1u) | ((gp >> 1) & cin);
            }
            const uint32_t C = (((G << 1) | cin) + Pm) ^ Pm;   // carries into each limb
            const size_t op = tile * TZ_M + row;
            if (op < batch && !failed) {
                uint32_t *prow = p + op * (size_t)(2 * m);
                const int l0 = 32 * qc;
                const bool vec = ((((uintptr_t)(prow + l0)) & 15) == 0) && (l0 + 32 <= 2 * m);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    uint32_t o[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) o[e] = r[4 * q + e] + ((C >> (4 * q + e)) & 1u);
                    if (vec) {
                        st_stream4(prow + l0 + 4 * q, make_uint4(o[0], o[1], o[2], o[3]));
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (l0 + 4 * q + e < 2 * m) st_stream1(prow + l0 + 4 * q + e, o[e]);
                    }
                }
            }
        }
        tz_fence_before();
        __syncthreads();
        tz_fence_after();
    }
    tz_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512) : "memory");
}

// ------------------------------------------------------------ INT32 path
// The batched column-sum multiply with the fixed operand broadcast (row
// stride 0), one op per run of lanes as in dot_mul.
template <int R>
__global__ void __launch_bounds__(MUL_WARPS * 32, dot_mul_min_blocks(R))
mul_shared_int_kernel(const uint32_t *fixed, const uint32_t *b, uint32_t *p, int m, int mp, int T,
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
    if (lane_on) {
        for (int k = t; k < R; k += T) {
            Bs[k] = 0;
            Bs[R + mp + k] = 0;
        }
        stage_row<R>(fixed, As, t, m, vec_in != 0);   // the fixed operand, staged once
    }
    const size_t wglobal = (size_t)blockIdx.x * MUL_WARPS + warp;
    const size_t nw = (size_t)gridDim.x * MUL_WARPS;
    for (size_t op0 = wglobal * opw; op0 < batch; op0 += nw * opw) {
        const size_t op = op0 + grp;
        const bool on = lane_on && op < batch;
        if (on) stage_row<R>(b + op * (size_t)m, Bs + R, t, m, vec_in != 0);
        __syncwarp();
        mul_group<R>(As, Bs, t, T, T, grp, on, m, mp, p + op * 2 * (size_t)m, vec_out != 0, smask, tmask);
        __syncwarp();
    }
}

template <int R>
static dot_status_t launch_shared_int(dot_ctx_t ctx, const dot_plan_t &pl, const uint32_t *fixed,
                                      const uint32_t *b, uint32_t *p, size_t m, size_t batch, cudaStream_t st)
{
    const int T = pl.lanes_per_op, mp = (int)pl.m_pad;
    const int opw = 32 / T;
    const size_t smem = (size_t)MUL_WARPS * opw * (2 * mp + 2 * R) * 4;
    const void *fn = (const void *)mul_shared_int_kernel<R>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return DOT_ECUDA;
    const bool vec_in = (m % 4 == 0) && aligned16(fixed) && aligned16(b);
    const bool vec_out = (m % 2 == 0) && aligned16(p);
    const size_t need = dot_ceil_div(batch, (size_t)opw * MUL_WARPS);
    const size_t cap = (size_t)ctx->num_sms * dot_blocks_per_sm(fn, MUL_WARPS * 32, smem);
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    mul_shared_int_kernel<R><<<grid, MUL_WARPS * 32, smem, st>>>(fixed, b, p, (int)m, mp, T, batch, vec_in, vec_out);
    return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
}

extern "C" {

DOT_API dot_status_t dot_mul_shared(dot_ctx_t ctx, const uint32_t *fixed, const uint32_t *b, uint32_t *p,
                                    size_t m, size_t batch, int use_tensor_cores, dot_stream_t stream)
{
    dot_status_t rc = dot_check_ctx(ctx);
    if (rc != DOT_OK) return rc;
    if (batch == 0 || m == 0) return DOT_OK;
    if (!fixed || !b || !p) return DOT_EINVAL;
    if (m > DOT_MUL_MAX_LIMBS || (use_tensor_cores && m > TZ_MAX_LIMBS)) return DOT_EUNSUPPORTED;
    if (batch > SIZE_MAX / 8 / m) return DOT_EINVAL;
    const size_t in = m * batch * 4, out = 2 * in;
    if (any_overlap(p, out, b, in) || any_overlap(p, out, fixed, m * 4)) return DOT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (use_tensor_cores) {
        if (cudaFuncSetAttribute((const void *)toeplitz_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TZ_SMEM) != cudaSuccess)
            return DOT_ECUDA;
        const size_t ntiles = (batch + TZ_M - 1) / TZ_M;
        const unsigned grid = (unsigned)(ntiles < (size_t)ctx->num_sms ? ntiles : (size_t)ctx->num_sms);
        toeplitz_mma_kernel<<<grid, TZ_THREADS, TZ_SMEM, st>>>(fixed, b, p, (int)m, batch, ctx->d_status,
                                                              ctx->wait_limit_ns);
        return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
    }
    dot_plan_t pl;
    rc = dot_make_plan(DOT_OP_MUL, m, batch, true, &pl, ctx->tune[DOT_OP_MUL][dot_tune_bucket(m)]);
    if (rc != DOT_OK) return rc;
    switch (pl.seg_limbs) {
    case 4: return launch_shared_int<4>(ctx, pl, fixed, b, p, m, batch, st);
    case 8: return launch_shared_int<8>(ctx, pl, fixed, b, p, m, batch, st);
    default: return launch_shared_int<16>(ctx, pl, fixed, b, p, m, batch, st);
    }
}

}  // extern "C"
