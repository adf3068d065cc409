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
// Kernel layout (one CTA of 17 warps per SM, persistent over tiles of 128
// operands; K = 256 digits, 512 output columns):
//   * T is block-Toeplitz in 128 x 128 blocks: block (k-block kb, column
//     block cb) depends only on d = cb - kb, and only d = 0, 1, 2 are nonzero.
//     The three distinct blocks (96 KB of fp16) are built once per CTA in
//     shared memory in the canonical no-swizzle K-major layout (row groups
//     of a k chunk contiguous).
//   * Each tile's digits are converted to fp16 into a 64 KB shared tile.
//   * One issuer thread issues 6 block pairs x 8 k-steps of tcgen05.mma
//     (M = 128, N = 128, K = 16) into four 128-column fp32 accumulators in
//     tensor memory (all 512 columns), in two halves, each committed to an
//     mbarrier.
//   * Sixteen worker warps (four per tensor-memory lane quadrant) drain each
//     half (tcgen05.ld), regroup columns into limb positions, resolve the
//     carries with generate/propagate masks, and stage the next tile, while
//     the tensor core fills the other half.
#include <cuda_fp16.h>
#include <string.h>

#include "dot_internal.cuh"
#include "dot_plan.h"
#include "dot_mul.cuh"

#define TZ_WORKERS 512          // 16 worker warps: staging and epilogue
#define TZ_THREADS (TZ_WORKERS + 32)   // + one issuer warp
#define TZ_M 128                 // operands per tile (MMA M)
#define TZ_K 256                 // digits per operand (bytes of 64 limbs)
#define TZ_NB 128                // columns per accumulator block (MMA N)
#define TZ_TBLOCK (128 * 128 * 2)            // bytes of one 128 x 128 fp16 block
#define TZ_ATILE (TZ_M * TZ_K * 2)           // bytes of one fp16 operand tile
#define TZ_OUT_STRIDE 68                   // words per staged output row (64 limbs + pad)
#define TZ_OUT (TZ_M * TZ_OUT_STRIDE * 4)  // bytes of one staged half tile of product limbs
#define TZ_SMEM (3 * TZ_TBLOCK + TZ_ATILE + TZ_OUT + 128 + TZ_K + 40 * TZ_M)
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
// Staging split in two: the next tile's limbs are loaded into registers early
// (their latency hides behind the current tile's drain) and converted into the
// fp16 tile once the tensor core is done with it.
__device__ __forceinline__ void tz_load(uint32_t (&x)[16], const uint32_t *b, int m, size_t batch, size_t tile, int w)
{
    const int row = w & (TZ_M - 1), qr = w >> 7;
    const size_t op = tile * TZ_M + row;
    const uint32_t *src = b + op * (size_t)m + 16 * qr;
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
}

__device__ __forceinline__ void tz_convert(unsigned char *sA, const uint32_t (&x)[16], int w)
{
    const int row = w & (TZ_M - 1), qr = w >> 7;
#pragma unroll
    for (int l2 = 0; l2 < 8; ++l2) {
        const uint32_t x0 = x[2 * l2], x1 = x[2 * l2 + 1];
        const uint4 v = make_uint4(tz_lo_pair(x0), tz_hi_pair(x0), tz_lo_pair(x1), tz_hi_pair(x1));
        *reinterpret_cast<uint4 *>(sA + tz_off(row, 64 * qr + 8 * l2, TZ_M)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tz_workers_sync() { asm volatile("bar.sync 1, %0;" :: "n"(TZ_WORKERS) : "memory"); }

// worker barrier that also returns whether any worker passed v != 0
__device__ __forceinline__ int tz_workers_sync_or(int v)
{
    int r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\t"
                 "bar.red.or.pred q, 1, %2, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
                 : "=r"(r) : "r"(v), "n"(TZ_WORKERS) : "memory");
    return r;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}

// The products of one accumulator half: column blocks cb0, cb0 + 1, each the
// sum over k-blocks kb of (operand k-block kb) x (Toeplitz block cb - kb).
__device__ __forceinline__ void tz_issue_half(uint32_t tmem, const unsigned char *sA, const unsigned char *sT,
                                              int cb0, uint32_t idesc)
{
#pragma unroll 1
    for (int cb = cb0; cb < cb0 + 2; ++cb) {
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
}

// Epilogue of accumulator half h for operand row `row`, limbs [64 h + 16 seg,
// + 16).  Each limb position collects L_l = sum_q C[4l + q] 2^(8q) < 2^49;
// with lo_l = L_l mod 2^32 and hi_l = L_l >> 32 the product is the two-term
// sum  sum_l lo_l X^l + sum_l hi_l X^(l+1), whose 1-bit carries are resolved
// by the Phase 4 mask identity inside each segment and by the segments'
// published (generate, propagate) pairs across segments.  carry_h / hi_h hold,
// per row, the carry and the top high word passed from half 0 to half 1.
__device__ __forceinline__ int tz_epilogue(uint32_t tmem, int h, int quad, int seg, int lane, uint32_t *xch,
                                           uint32_t *carry_h, uint32_t *hi_h, uint32_t *out, uint32_t *p, int m,
                                           size_t batch, size_t tile, int late)
{
    const int row = 32 * quad + lane;
    uint32_t r[16];
    uint32_t G = 0, Pm = 0, hi_prev = 0, lo_first = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        uint32_t v[32];
        tz_ld32(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(256 * h + 64 * seg + 32 * c), v);
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
                lo_first = lo;   // its high-word partner comes from the previous segment
                r[0] = lo;
            } else {
                r[li] = lo + hi_prev;
                G |= (uint32_t)(r[li] < lo) << li;
                Pm |= (uint32_t)(r[li] == DOT_FULL) << li;
            }
            hi_prev = (uint32_t)(L >> 32);
        }
    }
    xch[seg * TZ_M + row] = hi_prev;   // top high word of this segment
    if (h == 0 && seg == 3) hi_h[row] = hi_prev;
    // every worker learns whether any of them found its products late
    const int any_late = tz_workers_sync_or(late);
    const uint32_t h_in = seg ? xch[(seg - 1) * TZ_M + row] : (h ? hi_h[row] : 0u);
    r[0] = lo_first + h_in;
    G |= (uint32_t)(r[0] < lo_first);
    Pm |= (uint32_t)(r[0] == DOT_FULL);
    // segment aggregate: carry out with carry-in 0, and "all 16 limbs propagate"
    const uint32_t g_s = ((G << 1) + Pm) >> 16 & 1u;
    const uint32_t p_s = Pm == 0xFFFFu;
    tz_workers_sync();
    xch[seg * TZ_M + row] = g_s | (p_s << 1);
    tz_workers_sync();
    uint32_t cin = h ? carry_h[row] : 0u;
    for (int q = 0; q < seg; ++q) {
        const uint32_t gp = xch[q * TZ_M + row];
        cin = (gp & 1u) | ((gp >> 1) & cin);
    }
    const uint32_t C = (((G << 1) | cin) + Pm) ^ Pm;   // carries into each limb
    if (h == 0 && seg == 3) carry_h[row] = ((G >> 15) | ((Pm >> 15) & (C >> 15))) & 1u;
    // stage this segment's 16 result limbs, then write whole row segments out
    uint32_t *orow = out + row * TZ_OUT_STRIDE + 16 * seg;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t o[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) o[e] = r[4 * q + e] + ((C >> (4 * q + e)) & 1u);
        *reinterpret_cast<uint4 *>(orow + 4 * q) = make_uint4(o[0], o[1], o[2], o[3]);
    }
    tz_workers_sync();
    if (!any_late) {
        const int w = 32 * (4 * seg + quad) + lane;   // worker index
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int g = w + TZ_WORKERS * k, orw = g >> 4, c = g & 15;   // 16 chunks of 4 limbs per row
            const size_t op = tile * TZ_M + orw;
            const int l0 = 64 * h + 4 * c;
            if (op < batch && l0 < 2 * m) {
                const uint4 v = *reinterpret_cast<const uint4 *>(out + orw * TZ_OUT_STRIDE + 4 * c);
                uint32_t *dst = p + op * (size_t)(2 * m) + l0;
                if ((((uintptr_t)dst) & 15) == 0 && l0 + 4 <= 2 * m) {
                    st_stream4(dst, v);
                } else {
                    const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (l0 + e < 2 * m) st_stream1(dst + e, vv[e]);
                }
            }
        }
    }
    return any_late;
}

// fixed: m limbs (m <= 64), b: [batch][m], p: [batch][2m].
// Warp specialised: warp 16 allocates tensor memory and issues every product
// (one lane); warps 0..15 stage operand tiles as fp16 digits and drain the
// accumulators.  The 512 accumulator columns are two halves (column blocks
// 0-1 and 2-3) so that the tensor core fills one half while the workers drain
// the other:
//   issuer : for each tile t: wait staged(t); wait free0(t-1); issue half 0
//            -> full0(t); wait free1(t-1); issue half 1 -> full1(t)
//   workers: stage(0) -> staged(0); for each tile t: load tile t+1's limbs
//            into registers; wait full0(t); drain half 0 -> free0(t); wait
//            full1(t) (the fp16 tile is then free); convert t+1 ->
//            staged(t+1); drain half 1 -> free1(t)
// Drained limbs go through a staged output tile in shared memory so that
// every row segment is written to global memory by consecutive lanes.
// Every wait is bounded; a wait that runs out records DOT_ETIMEOUT, the CTA
// stops after its current tile, and the issuer waits (bounded) for its own
// products in flight before tensor memory is freed.
__global__ void __launch_bounds__(TZ_THREADS, 1)
toeplitz_mma_kernel(const uint32_t *fixed, const uint32_t *b, uint32_t *p, int m, size_t batch,
                    uint32_t *status, uint64_t wait_ns)
{
    extern __shared__ __align__(128) unsigned char tz_smem[];
    unsigned char *sT = tz_smem;                       // 3 Toeplitz blocks, d = 0, 1, 2
    unsigned char *sA = tz_smem + 3 * TZ_TBLOCK;       // fp16 operand tile
    uint32_t *out = (uint32_t *)(sA + TZ_ATILE);       // staged half tile of product limbs
    uint64_t *bars = (uint64_t *)((unsigned char *)out + TZ_OUT);
    uint64_t *bar_staged = bars, *bar_full = bars + 1, *bar_free = bars + 3;
    uint32_t *tmem_slot = (uint32_t *)(bars + 8);
    unsigned char *alpha = (unsigned char *)bars + 128;
    uint32_t *xch = (uint32_t *)(alpha + TZ_K);        // [half][segment][row]: top high word, then (g, p)
    uint32_t *carry_h = xch + 8 * TZ_M;                // [row]: carry from half 0 into half 1
    uint32_t *hi_h = carry_h + TZ_M;                   // [row]: top high word of half 0
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer = warp == TZ_WORKERS / 32;
    const size_t ntiles = (batch + TZ_M - 1) / TZ_M;

    if (issuer) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        if (lane == 0) {
            mbar_init(bar_staged, TZ_WORKERS);
            mbar_init(bar_full + 0, 1);
            mbar_init(bar_full + 1, 1);
            mbar_init(bar_free + 0, TZ_WORKERS);
            mbar_init(bar_free + 1, TZ_WORKERS);
            mbar_init_fence();
        }
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
        for (int hh = 0; hh < 4; ++hh) {
            uint32_t v[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int k = kc * 8 + 2 * hh + e;
                const int s = 128 * d + n - k;
                v[e] = (s >= 0 && s < TZ_K) ? alpha[s] : 0u;
            }
            w[hh] = tz_pack2(v[0], v[1]);
        }
        *reinterpret_cast<uint4 *>(sT + d * TZ_TBLOCK + tz_off(n, kc * 8, 128)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tz_fence_before();
    __syncthreads();
    tz_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (issuer) {
        if (lane == 0) {
            const uint32_t idesc = tz_idesc();
            int halves = 0;   // issued, for the final drain
            int it = 0;
            for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
                const uint32_t ph = (uint32_t)(it & 1), pph = (uint32_t)((it - 1) & 1);
                if (!mbar_wait_bounded(bar_staged, ph, wait_ns)) break;
                if (it > 0 && !mbar_wait_bounded(bar_free + 0, pph, wait_ns)) break;
                tz_fence_after();
                tz_issue_half(tmem, sA, sT, 0, idesc);
                tz_commit(bar_full + 0);
                ++halves;
                if (it > 0 && !mbar_wait_bounded(bar_free + 1, pph, wait_ns)) break;
                tz_fence_after();
                tz_issue_half(tmem, sA, sT, 2, idesc);
                tz_commit(bar_full + 1);
                ++halves;
            }
            // drain our own last products (a parity wait on a completed phase
            // returns at once)
            if (halves > 0) mbar_wait_bounded(bar_full + ((halves - 1) & 1), (uint32_t)(((halves - 1) >> 1) & 1), wait_ns);
        }
        __syncwarp();
    } else {
        const int quad = warp & 3, seg = warp >> 2;   // TMEM lane quadrant, 16-limb segment
        int late = 0;
        uint32_t x[16];
        if (blockIdx.x < ntiles) {
            tz_load(x, b, m, batch, blockIdx.x, tid);
            tz_convert(sA, x, tid);
            mbar_arrive(bar_staged);
        }
        int it = 0;
        for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const uint32_t ph = (uint32_t)(it & 1);
            const size_t next = tile + gridDim.x;
            if (next < ntiles) tz_load(x, b, m, batch, next, tid);
            late |= !mbar_wait_bounded(bar_full + 0, ph, wait_ns);
            tz_fence_after();
            int any_late = tz_epilogue(tmem, 0, quad, seg, lane, xch, carry_h, hi_h, out, p, m, batch, tile, late);
            tz_fence_before();
            mbar_arrive(bar_free + 0);
            late = !mbar_wait_bounded(bar_full + 1, ph, wait_ns);
            // every product of this tile is done: the fp16 tile is free
            if (next < ntiles) {
                tz_convert(sA, x, tid);
                mbar_arrive(bar_staged);
            }
            tz_fence_after();
            any_late |= tz_epilogue(tmem, 1, quad, seg, lane, xch + 4 * TZ_M, carry_h, hi_h, out, p, m, batch, tile,
                                    late);
            tz_fence_before();
            mbar_arrive(bar_free + 1);
            late = 0;
            if (any_late) {   // the same for every worker (barrier vote)
                if (tid == 0) record_status(status, DOT_ETIMEOUT);
                break;
            }
        }
    }
    tz_fence_before();
    __syncthreads();
    tz_fence_after();
    if (issuer)
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
