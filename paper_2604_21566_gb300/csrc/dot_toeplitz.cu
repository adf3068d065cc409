// dot_toeplitz.cu -- one fixed operand times a batch of operands on the
// tensor cores (tcgen05.mma), and the same product on the INT32 path.
//
// Theorem 2 (Sec. 3.2) writes A*B as column sums S_c = sum_{i+j=c} A_i B_j.
// With 8-bit digits (bytes) instead of 32-bit limbs the column sums of a
// fixed A against many B_j form one matrix product:
//     C[j][c] = sum_t beta_{j,t} alpha_{c-t},   T[t][c] = alpha_{c-t},
// i.e. C = Bdigits x T with T an upper-banded Toeplitz matrix (K = 4m digits,
// 8m output columns), regrouped four columns at a time into 32-bit limb
// positions and normalised by one carry pass per row (Alg. 2 Phase 5).
//
// Digit encoding.  The fixed operand is rewritten in balanced digits
//     a_i = d_i + [d_{i-1} >= 128] - 256 [d_i >= 128]  in [-128, 128]
// (4m + 1 of them; the same value), and every batch digit enters shifted,
// s_t = beta_t - 128 in [-128, 127].  Then every product is at most 2^14 in
// magnitude and every raw sum R_c = sum_t s_t a_{c-t} lies in [-2^22, 2^22],
// so an fp32 accumulator started at M = 1.5 * 2^23 stays in [2^23, 2^24],
// where fp32 holds every integer exactly, and its bit pattern minus the bits
// of M is R_c itself -- no float-to-integer conversion.  The true
// column sum is C_c = R_c + 128 W_c with W_c the sum of the a_u over the
// window u = c - t, t in [0, 4m): a per-column constant.  With v_c the bits
// of R_c + M, the product is
//     P = sum_l (sum_q v_{4l+q} 2^(8q)) 2^(32 l) + K  (mod 2^(64 m)),
// K = sum_l (128 sum_q W_{4l+q} 2^(8q) - bits(M) * 0x01010101) 2^(32 l), one
// constant per fixed operand, normalised once into 2m 32-bit limbs; every
// term is then nonnegative and the per-row carry pass is unsigned.
//
// Kernel layout (one CTA of 17 warps per SM, persistent over tiles of 128
// operands; K = 256 digits, 512 output columns):
//   * T is block-Toeplitz in 128 x 128 blocks: block (k-block kb, column
//     block cb) depends only on d = cb - kb, and only d = 0, 1, 2 are nonzero.
//     The three distinct blocks (96 KB of fp16) are built once per CTA in
//     shared memory, stacked along N (rows 128 d + n), K-major with the
//     128-byte swizzle.
//   * Each tile's digits are converted to fp16 into two 32 KB k-block
//     buffers that swap roles every tile, so that the next tile's first
//     k-block is staged while the tensor core still works on the current
//     tile's other k-block.
//   * One issuer thread issues, per 256-column accumulator half, a rank-one
//     bias product (3072 x 4096 = M, which also resets the half) and the
//     k-block products (tcgen05.mma, M = 128, K = 16) into four 128-column
//     fp32 accumulator blocks filling all 512 tensor-memory columns; each
//     half is committed to an mbarrier.
//     Where two column blocks take adjacent Toeplitz blocks from the same
//     k-block, one N = 256 product covers both: the operands are read from
//     shared memory once for twice the work, which matters because N = 128
//     products from shared memory nearly saturate its bandwidth.
//   * Sixteen worker warps (four per tensor-memory lane quadrant) drain each
//     half (tcgen05.ld) and release it, build limb values with 64-bit
//     multiply-adds, carry them serially inside 16-limb segments, exchange
//     one word per segment to resolve carries across segments, and stage the
//     half tile in shared memory, while the tensor core fills the other half
//     and the next tile's limbs are in flight.
//   * One store thread writes each staged half tile out with two tensor
//     stores (TMA), off the workers' path; before its first store its warp
//     computes the constant K while the first tile's products run.
#include <cuda.h>
#include <cuda_fp16.h>
#include <string.h>

#include "dot_internal.cuh"
#include "dot_plan.h"
#include "dot_mul.cuh"

#define TZ_WORKERS 512          // 16 worker warps: staging and epilogue
#define TZ_THREADS (TZ_WORKERS + 64)   // + one issuer warp + one store warp
#define TZ_M 128                 // operands per tile (MMA M)
#define TZ_K 256                 // digits per operand (bytes of 64 limbs)
#define TZ_NB 128                // columns per accumulator block (MMA N)
#define TZ_MAX_LIMBS 64
#define TZ_DIGITS (TZ_K + 8)     // balanced digits of the fixed operand (4m + 1 used)
#define TZ_TBLOCK (128 * 128 * 2)            // bytes of one 128 x 128 fp16 block
#define TZ_ATILE (TZ_M * TZ_K * 2)           // bytes of the two fp16 k-block buffers
#define TZ_KBUF (TZ_ATILE / 2)               // one 128-row x 128-digit k-block buffer
#define TZ_BIAS_A (128 * 16 * 2)             // bias operands, 128 x 16 and 256 x 16 fp16
#define TZ_BIAS_B (256 * 16 * 2)
#define TZ_BOX (TZ_M * 128)                // one staged box: 128 rows x 32 limbs, 128-byte swizzle
#define TZ_OUT (2 * TZ_BOX)                // bytes of one staged half tile of product limbs
#define TZ_RDIG 512                        // fp16 reversed-digit copy length
#define TZ_RCOPY (TZ_RDIG * 2 + 16)        // bytes between the 8 shifted copies (padded)
// shared-memory carve-up, from a 1024-byte aligned base
#define TZ_OFF_A (3 * TZ_TBLOCK)
#define TZ_OFF_OUT (TZ_OFF_A + TZ_ATILE)
#define TZ_OFF_BIAS (TZ_OFF_OUT + TZ_OUT)                 // bias operands A, B
#define TZ_OFF_KN (TZ_OFF_BIAS + TZ_BIAS_A + TZ_BIAS_B)   // uint32 [128]: K as normalised limbs
#define TZ_OFF_XCH (TZ_OFF_KN + 128 * 4)                  // uint2 [2 halves][4 segments][128 rows]
#define TZ_OFF_CARRY (TZ_OFF_XCH + 2 * 4 * TZ_M * 8)      // int32 [128]: carry word half 0 -> half 1
#define TZ_OFF_DIG (TZ_OFF_CARRY + TZ_M * 4)              // int32 [TZ_DIGITS]: balanced digits
#define TZ_OFF_PRE (TZ_OFF_DIG + TZ_DIGITS * 4)           // int32 [TZ_DIGITS + 8]: their prefix sums
#define TZ_OFF_BARS (TZ_OFF_PRE + (TZ_DIGITS + 8) * 4)    // 10 mbarriers, tensor-memory address, flag
#define TZ_SMEM (1024 + TZ_OFF_BARS + 128)                // + alignment slack
// fp32 bits of the accumulator start value M = 1.5 * 2^23 = 3072 * 4096
#define TZ_MAGIC_BITS 0x4B400000u
#define TZ_TROWS 384             // stacked Toeplitz rows (3 blocks)
static_assert(TZ_DIGITS <= TZ_THREADS, "one balanced digit per thread");
// Toeplitz chunk (d, n, k chunk) holds digits a[s0], a[s0-1], .., a[s0-7],
// s0 = 128 d + n - 8 kc in [-120, 383]; with r[i] = a[383 - i] that run is
// r[383 - s0 .. + 7], which the shifted copy (383 - s0) % 8 holds 16-byte aligned
#define TZ_RTOP 383

// ------------------------------------------------------------ tcgen05 glue
// Shared-memory matrix descriptor, K-major with the 128-byte swizzle: a tile
// is stored as atom columns of 64 k (128 bytes per row); inside a column, row r
// sits at (r / 8) * 1024 + (r % 8) * 128 bytes (sbo = 1024 B between 8-row
// groups) and its 16-byte chunk c at position c ^ (r % 8).  A K = 16 slice
// starts 32 bytes further along the row per step; lbo is unused.
__device__ __forceinline__ uint64_t tz_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;              // lbo (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;    // sbo
    d |= (uint64_t)1 << 46;              // descriptor version bits 46..48 = 0b001
    d |= (uint64_t)2 << 61;              // layout: 128-byte swizzle
    return d;
}

// Descriptor of a bias operand (rows x 16 fp16) without swizzle: core
// matrices of 8 rows x 16 bytes, the row groups of one 8-k chunk contiguous
// (sbo = 128 B), the two k chunks rows * 16 bytes apart (lbo).
__device__ __forceinline__ uint64_t tz_desc_plain(uint32_t saddr, int rows)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(((uint32_t)rows * 16u) >> 4) << 16;
    d |= (uint64_t)(128 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Byte offset of element (row, k) of a K-major tile of `rows` rows in the
// swizzled layout above (tile base 1024-byte aligned).  Eight consecutive rows
// writing the same 16-byte chunk hit eight distinct bank groups.
__device__ __forceinline__ uint32_t tz_off(int row, int k, int rows)
{
    const int c = (k >> 3) & 7;
    return (uint32_t)((k >> 6) * rows * 128 + ((row >> 3) << 10) + ((row & 7) << 7) + ((c ^ (row & 7)) << 4) +
                      ((k & 7) << 1));
}

// instruction descriptor: D fp32, A and B fp16, both K-major, M = 128, N = n
__device__ __forceinline__ uint32_t tz_idesc(int n)
{
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TZ_M >> 4) << 24);
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

// 32 consecutive columns of this warp's 32 lanes; the registers are valid only
// after tz_ld_wait
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
}

// Wait for this thread's tensor-memory loads; the registers pass through the
// statement so that no use of them is scheduled before it.
__device__ __forceinline__ void tz_ld_wait(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]),
                   "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]),
                   "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :: "memory");
}

__device__ __forceinline__ void tz_pin(uint32_t (&r)[32])
{
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]),
                   "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]),
                   "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :: "memory");
}

__device__ __forceinline__ void tz_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tz_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// the tensor stores of this thread have read their shared-memory source
__device__ __forceinline__ void tz_bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// one 2-D tensor store (box of 32 limbs x 128 rows at limb x, row y) from a
// 128-byte-swizzled staging box, in this thread's bulk group
__device__ __forceinline__ void tz_tma_store(const CUtensorMap *map, const void *src, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];"
                 :: "l"(map), "r"(smem_u32(src)), "r"(x), "r"(y) : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Staged limbs of a half tile: two boxes (limbs 0-31, 32-63) of 128 rows x
// 128 bytes, 16-byte chunk c of row r at position c ^ (r % 8) -- the layout
// the tensor store expects for the 128-byte swizzle, and conflict-free for
// 32 rows writing the same chunk.  `chunk` counts 4-limb chunks, 0..15.
__device__ __forceinline__ uint32_t *tz_stage(uint32_t *out, int row, int chunk)
{
    const int c = chunk & 7;
    return out + (chunk >> 3) * (TZ_BOX / 4) + row * 32 + ((c ^ (row & 7)) << 2);
}
__device__ __forceinline__ void tz_bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Two digit values as a pair of fp16 without conversion instructions:
// 0x6400 | u is the fp16 encoding of 1024 + u (0 <= u < 1024), so one packed
// half subtraction of 1024 + bias leaves u - bias exactly.
__device__ __forceinline__ uint32_t tz_half2_minus(uint32_t biased, uint16_t sub_bits)
{
    __half2 h = *reinterpret_cast<const __half2 *>(&biased);
    h = __hsub2(h, __halves2half2(__ushort_as_half(sub_bits), __ushort_as_half(sub_bits)));
    return *reinterpret_cast<const uint32_t *>(&h);
}

// balanced digits v0, v1 in [-128, 128] -> fp16 pair
__device__ __forceinline__ uint32_t tz_pack_signed2(int v0, int v1)
{
    return tz_half2_minus(0x64006400u | (uint32_t)(v0 + 128) | ((uint32_t)(v1 + 128) << 16), 0x6480);
}

// bytes sel of limb x, each shifted by -128, as an fp16 pair
__device__ __forceinline__ uint32_t tz_shifted2(uint32_t x, uint32_t sel)
{
    return tz_half2_minus(__byte_perm(x, 0x64u, sel), 0x6480);   // bytes [d0, 0x64, d1, 0x64]
}

// --------------------------------------------------------------- kernel
// Staging split in two: the next tile's limbs are loaded into registers early
// (their latency hides behind the current tile's drain) and converted into the
// fp16 k-block buffers once the tensor core is done with them.  Worker w holds
// row w % 128's limbs 8q .. 8q + 7 of each k-block (q = w / 128), so that all
// workers convert each k-block together: x[0..8) for k-block 0, x[8..16) for 1.
__device__ __forceinline__ void tz_load(uint32_t (&x)[16], const uint32_t *b, int m, size_t batch, size_t tile, int w)
{
    const int row = w & (TZ_M - 1), q = w >> 7;
    const size_t op = tile * TZ_M + row;
    const uint32_t *src = b + op * (size_t)m + 8 * q;
    if (op < batch && m == TZ_MAX_LIMBS && aligned16(src)) {
#pragma unroll
        for (int kb = 0; kb < 2; ++kb)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint4 v = __ldcs(reinterpret_cast<const uint4 *>(src + 32 * kb) + h);
                x[8 * kb + 4 * h] = v.x; x[8 * kb + 4 * h + 1] = v.y;
                x[8 * kb + 4 * h + 2] = v.z; x[8 * kb + 4 * h + 3] = v.w;
            }
    } else {
#pragma unroll
        for (int l = 0; l < 16; ++l) {
            const int limb = 32 * (l >> 3) + 8 * q + (l & 7);
            x[l] = (op < batch && limb < m) ? __ldcs(b + op * (size_t)m + limb) : 0u;
        }
    }
}

// Digits beyond the operand's 4m enter as 0 (not -128), so that every batch
// row has exactly the digit window that the limb constants assume.  Worker w
// converts row w % 128's limbs 8q .. 8q + 7 of k-block kb (q = w / 128):
// digits 32q .. 32q + 31 of the k-block, into its buffer kbuf.
__device__ __forceinline__ void tz_convert(unsigned char *kbuf, const uint32_t (&x)[16], int kb, int w, int m)
{
    const int row = w & (TZ_M - 1), q = w >> 7;
    const int limb0 = 32 * kb + 8 * q;   // first limb of the operand held here
    const bool full = limb0 + 8 <= m;
#pragma unroll
    for (int l2 = 0; l2 < 4; ++l2) {
        const uint32_t x0 = x[8 * kb + 2 * l2], x1 = x[8 * kb + 2 * l2 + 1];
        uint4 v = make_uint4(tz_shifted2(x0, 0x4140), tz_shifted2(x0, 0x4342), tz_shifted2(x1, 0x4140),
                             tz_shifted2(x1, 0x4342));
        if (!full) {
            if (limb0 + 2 * l2 >= m) v.x = v.y = 0u;
            if (limb0 + 2 * l2 + 1 >= m) v.z = v.w = 0u;
        }
        *reinterpret_cast<uint4 *>(kbuf + tz_off(row, 32 * q + 8 * l2, TZ_M)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// k-block kb of tile number it (counted per CTA) lives in buffer kb ^ (it & 1)
__device__ __forceinline__ unsigned char *tz_kbuf(unsigned char *sA, int kb, int it)
{
    return sA + TZ_KBUF * (kb ^ (it & 1));
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

// One arrival per warp once all its lanes got here (worker barriers count
// warps: hundreds of single-thread arrivals on one barrier word serialise).
__device__ __forceinline__ void tz_warp_arrive(uint64_t *bar)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

// k-steps of one product: a k-block buffer (descriptor adesc of its base)
// against stacked Toeplitz rows from 128 d0 (descriptor bdesc of that row),
// n = 128 or 256 of them, into accumulator columns col; the first step
// overwrites the accumulator when acc0 == 0.  Unrolled with constant
// descriptor offsets (the start-address field holds address / 16): the
// issuing warp shares its scheduler with busy worker warps, so each product
// must cost it only a few independent instructions.
__device__ __forceinline__ void tz_issue_kblock(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                                uint32_t acc0)
{
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        // k = 16 s inside the k-block: atom column s / 4, 32 bytes per step inside it
        const uint64_t ad = adesc + (uint64_t)(((s >> 2) * TZ_M * 128 + (s & 3) * 32) >> 4);
        const uint64_t bd = bdesc + (uint64_t)(((s >> 2) * TZ_TROWS * 128 + (s & 3) * 32) >> 4);
        tz_mma(dtmem, ad, bd, idesc, s > 0 ? 1u : acc0);
    }
}

// Epilogue of accumulator half h for operand row `row`, limbs [64 h + 16 seg,
// + 16); mid(late) runs between the arithmetic and the exchange.  Limb position l collects sum_q v_{4l+q} 2^(8q) + K_l (unsigned,
// below 2^56); a serial carry inside the segment gives 16 limbs and a carry
// word.  Each segment publishes (carry word, first limb, "limbs 1..15 all
// ones"), from which every segment derives its incoming carry word: adding a
// word w to a segment whose first limb is o_0 moves a carry out of it only if
// o_0 + w >= 2^32 and the rest are all ones.  carry_h holds, per row, the
// carry word from half 0 into half 1; the carry out of the top limb is
// dropped (the product is taken mod 2^(64 m), which it fits).
template <typename Mid>
__device__ __forceinline__ int tz_epilogue(Mid mid, uint32_t tmem, int h, int quad, int seg, int lane, uint64_t *bar_free,
                                           const uint32_t *Kn, uint2 *xch, uint32_t *carry_h, uint32_t *out,
                                           uint32_t *p, int m, size_t batch, size_t tile, int late,
                                           const CUtensorMap *pmap, uint64_t *bar_staged_out, uint64_t *bar_out_free,
                                           int use, uint32_t *out_flags, int &late_out, uint32_t *status,
                                           uint64_t wait_ns)
{
    const int row = 32 * quad + lane;
    const int w = 32 * (4 * seg + quad) + lane;   // worker index
    const uint32_t taddr = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(256 * h + 64 * seg);
    const uint4 *kq = reinterpret_cast<const uint4 *>(Kn + 64 * h + 16 * seg);
    uint32_t o[16];
    uint32_t hi = 0;
    // two passes of 32 columns (8 limbs) keep register pressure down
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        uint32_t v[32];
        tz_ld32(taddr + 32 * pass, v);
        tz_ld_wait(v);
        if (pass == 1) {
            // all of this thread's columns are in registers: the tensor core may refill them
            tz_fence_before();
            tz_warp_arrive(bar_free);
        }
        // the limb values first (independent of each other), then the carry
        // chain, which costs two dependent adds per limb
        uint64_t L[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int l = 8 * pass + j;
            const uint4 k4 = kq[l >> 2];
            const uint32_t k = (l & 3) == 0 ? k4.x : (l & 3) == 1 ? k4.y : (l & 3) == 2 ? k4.z : k4.w;
            L[j] = (uint64_t)k + v[4 * j] + (uint64_t)v[4 * j + 1] * 256u + (uint64_t)v[4 * j + 2] * 65536u +
                   (uint64_t)v[4 * j + 3] * 16777216u;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint64_t acc = L[j] + hi;
            o[8 * pass + j] = (uint32_t)acc;
            hi = (uint32_t)(acc >> 32);
        }
    }
    uint32_t all1 = o[1];
#pragma unroll
    for (int l = 2; l < 16; ++l) all1 &= o[l];
    if (seg < 3) xch[seg * TZ_M + row] = make_uint2((hi << 1) | (uint32_t)(all1 == DOT_FULL), o[0]);
    // work that should not wait for the rest of the epilogue (it may change late)
    mid(late);
    // every worker learns whether any of them found its products late
    const int any_late = tz_workers_sync_or(late);
    uint32_t c = h ? carry_h[row] : 0u;
    for (int q = 0; q < seg; ++q) {
        const uint2 e = xch[q * TZ_M + row];
        const uint64_t s0 = (uint64_t)e.y + c;
        c = (e.x >> 1) + (uint32_t)((s0 >> 32) != 0 && (e.x & 1u));
    }
    // add the incoming carry word; a carry out of the first limb ripples
    // through the rest only while they are all ones
    const uint64_t s0 = (uint64_t)o[0] + c;
    o[0] = (uint32_t)s0;
    uint32_t rip = (uint32_t)(s0 >> 32);   // 0 or 1
    if (rip != 0) {
#pragma unroll
        for (int l = 1; l < 16; ++l) {
            const uint32_t x = o[l];
            o[l] = x + rip;
            rip = x == DOT_FULL ? rip : 0u;
        }
    }
    if (h == 0 && seg == 3) carry_h[row] = hi + rip;
    // stage this segment's 16 result limbs once the store thread has read the
    // previous half tile out of the staging buffer (a wait that runs out is
    // recorded, the half tile is not stored, and the next vote stops the CTA)
    late_out = use > 0 && !mbar_wait_bounded(bar_out_free, (uint32_t)((use - 1) & 1), wait_ns);
    if (late_out) {
        record_status(status, DOT_ETIMEOUT);
        atomicOr(out_flags, 1u);   // skip this half tile's stores
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4 *>(tz_stage(out, row, 4 * seg + q)) =
            make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    if (w == 0 && any_late) atomicOr(out_flags, 3u);   // skip, and stop after this tile
    if (pmap) {
        // the store thread writes the half tile out
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tz_warp_arrive(bar_staged_out);
        return any_late;
    }
    const int skip = tz_workers_sync_or(late_out) | any_late;
    if (!skip) {
        const int l0 = 64 * h;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int g = w + TZ_WORKERS * k, orw = g >> 4, cc = g & 15;   // 16 chunks of 4 limbs per row
            const size_t op = tile * TZ_M + orw;
            const int lc = l0 + 4 * cc;
            if (op < batch && lc < 2 * m) {
                const uint4 vv = *reinterpret_cast<const uint4 *>(tz_stage(out, orw, cc));
                uint32_t *dst = p + op * (size_t)(2 * m) + lc;
                const uint32_t e4[4] = {vv.x, vv.y, vv.z, vv.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (lc + e < 2 * m) st_stream1(dst + e, e4[e]);
            }
        }
    }
    // the staging buffer is free again once every worker has read its chunks
    tz_warp_arrive(bar_staged_out);
    return any_late;
}

// The store thread: per staged half tile, two tensor stores (limbs 64 h + 0..31,
// + 32..63 of the tile's 128 rows; rows past the batch and limbs past 2m are
// clipped), then the staging buffer is handed back once the stores have read
// it.  Without a tensor map the workers store, and this thread only passes the
// buffer on.  It mirrors the workers' tile loop and stops where they stop.
__device__ __forceinline__ void tz_store_loop(const CUtensorMap *pmap, const uint32_t *out, uint64_t *bar_staged_out,
                                              uint64_t *bar_out_free, volatile uint32_t *out_flags, int m,
                                              size_t ntiles, uint64_t wait_ns)
{
    if (pmap) asm volatile("prefetch.tensormap [%0];" :: "l"(pmap) : "memory");
    int use = 0;
    uint32_t stop = 0;
    for (size_t tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x) {
        for (int h = 0; h < 2; ++h, ++use) {
            if (!mbar_wait_bounded(bar_staged_out, (uint32_t)(use & 1), wait_ns)) {
                stop = 1;
                break;
            }
            const uint32_t f = *out_flags;
            *out_flags = 0u;
            stop |= f & 2u;
            if (pmap) {
                const int l0 = 64 * h;
                if (!(f & 1u)) {
                    if (l0 < 2 * m) tz_tma_store(pmap, out, l0, (int)(tile * TZ_M));
                    if (l0 + 32 < 2 * m) tz_tma_store(pmap, out + TZ_BOX / 4, l0 + 32, (int)(tile * TZ_M));
                }
                tz_bulk_wait_read();
            }
            mbar_arrive(bar_out_free);
        }
    }
    if (pmap) tz_bulk_wait_all();
}

// The constant K (one warp): prefix sums of the balanced digits, the per-limb
// constants c_l = 128 sum_q W_{4l+q} 2^(8q) - bits(M) * 0x01010101 (W_c = sum
// of a_u over u in [max(0, c - 4m + 1), min(c, 4m)]), and K = sum_{l < 2m}
// c_l 2^(32 l) as 128 limbs mod 2^(64 m): lane j takes limbs 4j..4j+3 through
// a signed serial carry, then the lanes pass carry words up until they no
// longer change.
__device__ __forceinline__ void tz_make_k(const int32_t *dig, int32_t *pre, uint32_t *Kn, int m, int lane)
{
    const int nd = 4 * m;
    // prefix sums pre[u] = a_0 + ... + a_{u-1}, 9 digits per lane
    int loc[9], sum = 0;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const int u = 9 * lane + j;
        loc[j] = u < TZ_DIGITS ? dig[u] : 0;
        sum += loc[j];
    }
    int incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    int run = incl - sum;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const int u = 9 * lane + j;
        if (u <= TZ_DIGITS) pre[u] = run;
        run += loc[j];
    }
    __syncwarp();
    uint32_t t[4];
    int64_t acc = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int l = 4 * lane + j;
        int64_t k = 0;
        if (l < 2 * m) {
            k = -(int64_t)TZ_MAGIC_BITS * 0x01010101;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = 4 * l + q;
                const int lo = c - nd + 1 > 0 ? c - nd + 1 : 0, hi = c < nd ? c : nd;
                const int64_t W = lo <= hi ? (int64_t)(pre[hi + 1] - pre[lo]) : 0;
                k += W * 128 * ((int64_t)1 << (8 * q));
            }
        }
        acc = k + (acc >> 32);
        t[j] = (uint32_t)acc;
    }
    const int64_t cw = acc >> 32;   // this lane's carry word with carry-in 0
    const bool ones = (t[1] & t[2] & t[3]) == DOT_FULL, zeros = (t[1] | t[2] | t[3]) == 0u;
    int64_t ci = __shfl_up_sync(0xffffffffu, cw, 1);
    if (lane == 0) ci = 0;
    for (int round = 0; round < 32; ++round) {
        const int64_t s0 = (int64_t)t[0] + ci;
        const int64_t co = cw + (int64_t)(s0 >= ((int64_t)1 << 32) && ones) - (int64_t)(s0 < 0 && zeros);
        int64_t nci = __shfl_up_sync(0xffffffffu, co, 1);
        if (lane == 0) nci = 0;
        if (__all_sync(0xffffffffu, nci == ci)) break;
        ci = nci;
    }
    // apply the carry-in word: a carry or borrow out of limb 0 ripples
    // while the next limbs are all ones / all zero
    const int64_t s0 = (int64_t)t[0] + ci;
    t[0] = (uint32_t)s0;
    int32_t rip = (int32_t)(s0 >> 32);
#pragma unroll
    for (int j = 1; j < 4; ++j) {
        const uint32_t x = t[j];
        t[j] = x + (uint32_t)rip;
        rip = (rip > 0 && x == DOT_FULL) || (rip < 0 && x == 0u) ? rip : 0;
    }
    reinterpret_cast<uint4 *>(Kn)[lane] = make_uint4(t[0], t[1], t[2], t[3]);
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
//            into registers; wait full0(t); drain half 0 (free0(t) as soon as
//            it is in registers); wait full1(t) (the fp16 tile is then free);
//            convert t+1 -> staged(t+1); drain half 1 (free1(t))
// Every wait is bounded; a wait that runs out records DOT_ETIMEOUT, the CTA
// stops after its current tile, and the issuer waits (bounded) for its own
// products in flight before tensor memory is freed.
__global__ void __launch_bounds__(TZ_THREADS, 1)
toeplitz_mma_kernel(const uint32_t *fixed, const uint32_t *b, uint32_t *p, int m, size_t batch,
                    const __grid_constant__ CUtensorMap pmap_param, int use_map, uint32_t *status, uint64_t wait_ns)
{
    extern __shared__ __align__(128) unsigned char tz_smem[];
    // swizzled tiles need a 1024-byte aligned base
    unsigned char *base = tz_smem + ((1024u - (smem_u32(tz_smem) & 1023u)) & 1023u);
    unsigned char *sT = base;                          // Toeplitz blocks d = 0, 1, 2
    unsigned char *sA = base + TZ_OFF_A;               // two fp16 k-block buffers
    unsigned char *sBias = base + TZ_OFF_BIAS;         // bias operands (A then B)
    uint32_t *out = (uint32_t *)(base + TZ_OFF_OUT);   // staged half tile of product limbs
    uint32_t *Kn = (uint32_t *)(base + TZ_OFF_KN);
    uint2 *xch = (uint2 *)(base + TZ_OFF_XCH);
    uint32_t *carry_h = (uint32_t *)(base + TZ_OFF_CARRY);
    int32_t *dig = (int32_t *)(base + TZ_OFF_DIG);
    int32_t *pre = (int32_t *)(base + TZ_OFF_PRE);
    uint64_t *bars = (uint64_t *)(base + TZ_OFF_BARS);
    uint64_t *bar_staged = bars, *bar_full = bars + 2, *bar_free = bars + 4;   // staged: per k-block
    uint64_t *bar_staged_out = bars + 6, *bar_out_free = bars + 7, *bar_kb1done = bars + 8;
    uint64_t *bar_kn = bars + 9;   // the constant K is ready
    uint32_t *tmem_slot = (uint32_t *)(bars + 10);
    uint32_t *out_flags = tmem_slot + 1;   // bit 0: skip the stores, bit 1: stop after the tile
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer = warp == TZ_WORKERS / 32, storer = warp == TZ_WORKERS / 32 + 1;
    const size_t ntiles = (batch + TZ_M - 1) / TZ_M;
    const CUtensorMap *pmap = use_map ? &pmap_param : nullptr;
    const int nd = 4 * m;   // digits of each operand

    // the fixed operand's digits first (their latency gates the set-up), then
    // the first tile's limbs, in flight during the set-up
    uint32_t dk_word = 0, dp_word = 0;
    const int kdig = tid;   // TZ_DIGITS <= TZ_THREADS: one digit per thread
    if (kdig < TZ_DIGITS) {
        if (kdig < nd) dk_word = fixed[kdig >> 2];
        if (kdig >= 1 && kdig - 1 < nd) dp_word = fixed[(kdig - 1) >> 2];
    }
    uint32_t x[16];
    if (tid < TZ_WORKERS && blockIdx.x < ntiles) tz_load(x, b, m, batch, blockIdx.x, tid);
    if (issuer) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        if (lane == 0) {
            mbar_init(bar_staged + 0, TZ_WORKERS / 32);   // arrivals per warp
            mbar_init(bar_staged + 1, TZ_WORKERS / 32);
            mbar_init(bar_kb1done, 1);
            mbar_init(bar_full + 0, 1);
            mbar_init(bar_full + 1, 1);
            mbar_init(bar_free + 0, TZ_WORKERS / 32);
            mbar_init(bar_free + 1, TZ_WORKERS / 32);
            mbar_init(bar_staged_out, TZ_WORKERS / 32);
            mbar_init(bar_out_free, 1);
            mbar_init(bar_kn, 1);
            *out_flags = 0u;
            mbar_init_fence();
        }
    }
    // bias operands: column k = 0 of A holds 3072, of B 4096 (fp16), the rest
    // 0; rows' k-chunk 0 fills the first rows * 16 bytes of each
    for (int i = tid; i < (TZ_BIAS_A + TZ_BIAS_B) / 16; i += TZ_THREADS) {
        const bool in_b = i >= TZ_BIAS_A / 16;
        const int chunk = in_b ? i - TZ_BIAS_A / 16 : i;
        const uint32_t first = chunk < (in_b ? 256 : 128) ? (in_b ? 0x6C00u : 0x6A00u) : 0u;
        *reinterpret_cast<uint4 *>(sBias + 16 * i) = make_uint4(first, 0u, 0u, 0u);
    }
    // balanced digits a_k = d_k + [d_{k-1} >= 128] - 256 [d_k >= 128], k <= 4m
    if (kdig < TZ_DIGITS) {
        const uint32_t dk = (dk_word >> (8 * (kdig & 3))) & 0xFFu;
        const uint32_t dp = kdig >= 1 ? (dp_word >> (8 * ((kdig - 1) & 3))) & 0xFFu : 0u;
        dig[kdig] = (int32_t)dk + (int32_t)(dp >= 128u) - 256 * (int32_t)(dk >= 128u);
    }
    __syncthreads();
    // 8 shifted copies of the reversed digits as fp16: copy o, entry i = r[i + o]
    unsigned char *rcopy = sA;   // the operand tile is free until the first conversion
    for (int i = tid; i < 8 * TZ_RDIG / 2; i += TZ_THREADS) {
        const int o = i / (TZ_RDIG / 2), e = 2 * (i - o * (TZ_RDIG / 2));
        int v[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int u = TZ_RTOP - (e + j + o);
            v[j] = (u >= 0 && u <= nd) ? dig[u] : 0;
        }
        *reinterpret_cast<uint32_t *>(rcopy + o * TZ_RCOPY + 2 * e) = tz_pack_signed2(v[0], v[1]);
    }
    __syncthreads();
    if (!storer) {
        // Toeplitz block d, element (n, k) = a[128 d + n - k] when 0 <= . <= 4m:
        // each 8-k chunk is one aligned 16-byte run of a shifted copy
        for (int idx = tid; idx < 3 * 128 * 16; idx += TZ_WORKERS + 32) {
            const int d = idx / (128 * 16), rem = idx - d * 128 * 16, n = rem & 127, kc = rem >> 7;
            const int i0 = TZ_RTOP - (128 * d + n - 8 * kc), o = i0 & 7;
            const uint4 chunk = *reinterpret_cast<const uint4 *>(rcopy + o * TZ_RCOPY + 2 * (i0 - o));
            *reinterpret_cast<uint4 *>(sT + tz_off(128 * d + n, kc * 8, TZ_TROWS)) = chunk;
        }
    }
    __syncthreads();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tz_fence_before();
    __syncthreads();
    tz_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (issuer) {
        if (lane == 0) {
            int halves = 0;   // issued, for the final drain
            int it = 0;
            const uint32_t i128 = tz_idesc(128), i256 = tz_idesc(256);
            const uint64_t dT = tz_desc(smem_u32(sT));
            const uint64_t dbuf[2] = {tz_desc(smem_u32(sA)), tz_desc(smem_u32(sA + TZ_KBUF))};
            const uint64_t drow = (uint64_t)((128 * 128) >> 4);   // 128 stacked rows
            const uint64_t dbias_a = tz_desc_plain(smem_u32(sBias), 128);
            const uint64_t dbias_b = tz_desc_plain(smem_u32(sBias + TZ_BIAS_A), 256);
            for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
                const uint32_t ph = (uint32_t)(it & 1), pph = (uint32_t)((it - 1) & 1);
                // k-block kb of this tile sits in buffer kb ^ (it & 1)
                const uint64_t dkb0 = dbuf[it & 1], dkb1 = dbuf[(it & 1) ^ 1];
                // half 0: bias -> columns 0-255 (N = 256, resets them);
                //         kb 0 x blocks d = 0, 1 -> columns 0-255; kb 1 x d = 0 -> 128-255
                if (!mbar_wait_bounded(bar_staged + 0, ph, wait_ns)) break;
                if (it > 0 && !mbar_wait_bounded(bar_free + 0, pph, wait_ns)) break;
                tz_fence_after();
                tz_mma(tmem, dbias_a, dbias_b, i256, 0u);
                tz_issue_kblock(tmem, dkb0, dT, i256, 1u);
                if (!mbar_wait_bounded(bar_staged + 1, ph, wait_ns)) break;
                tz_fence_after();
                tz_issue_kblock(tmem + 128, dkb1, dT, i128, 1u);
                tz_commit(bar_full + 0);
                ++halves;
                // half 1: bias -> columns 256-511 (resets them); kb 1 x d = 1, 2 ->
                //         256-511, after which kb 1's buffer is free; kb 0 x d = 2 -> 256-383
                if (it > 0 && !mbar_wait_bounded(bar_free + 1, pph, wait_ns)) break;
                tz_fence_after();
                tz_mma(tmem + 256, dbias_a, dbias_b, i256, 0u);
                tz_issue_kblock(tmem + 256, dkb1, dT + drow, i256, 1u);
                tz_commit(bar_kb1done);
                tz_issue_kblock(tmem + 256, dkb0, dT + 2 * drow, i128, 1u);
                tz_commit(bar_full + 1);
                ++halves;
            }
            // drain our own last products (a parity wait on a completed phase
            // returns at once)
            if (halves > 0) mbar_wait_bounded(bar_full + ((halves - 1) & 1), (uint32_t)(((halves - 1) >> 1) & 1), wait_ns);
        }
        __syncwarp();
    } else if (storer) {
        tz_make_k(dig, pre, Kn, m, lane);
        tz_warp_arrive(bar_kn);
        if (lane == 0) tz_store_loop(pmap, out, bar_staged_out, bar_out_free, out_flags, m, ntiles, wait_ns);
        __syncwarp();
    } else {
        const int quad = warp & 3, seg = warp >> 2;   // TMEM lane quadrant, 16-limb segment
        int late = 0;
        if (blockIdx.x < ntiles) {
            for (int kb = 0; kb < 2; ++kb) {
                tz_convert(tz_kbuf(sA, kb, 0), x, kb, tid, m);
                tz_warp_arrive(bar_staged + kb);
            }
        }
        int it = 0;
        for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
            const uint32_t ph = (uint32_t)(it & 1);
            const size_t next = tile + gridDim.x;
            if (next < ntiles) tz_load(x, b, m, batch, next, tid);
            late |= !mbar_wait_bounded(bar_full + 0, ph, wait_ns);
            if (it == 0) late |= !mbar_wait_bounded(bar_kn, 0u, wait_ns);
            tz_fence_after();
            int late_out = 0;
            // stage the next tile: its k-block 0 goes into this tile's k-block 1
            // buffer as soon as the products reading that are done (in the middle
            // of the half-0 epilogue), its k-block 1 into this tile's k-block 0
            // buffer once the whole tile is done
            auto stage_kb0 = [&](int &lt) {
                if (next < ntiles) {
                    lt |= !mbar_wait_bounded(bar_kb1done, ph, wait_ns);
                    tz_convert(tz_kbuf(sA, 0, it + 1), x, 0, tid, m);
                    tz_warp_arrive(bar_staged + 0);
                }
            };
            int any_late = tz_epilogue(stage_kb0, tmem, 0, quad, seg, lane, bar_free + 0, Kn, xch, carry_h, out, p, m,
                                       batch, tile, late, pmap, bar_staged_out, bar_out_free, 2 * it, out_flags,
                                       late_out, status, wait_ns);
            late = late_out;
            late |= !mbar_wait_bounded(bar_full + 1, ph, wait_ns);
            if (next < ntiles) {
                tz_convert(tz_kbuf(sA, 1, it + 1), x, 1, tid, m);
                tz_warp_arrive(bar_staged + 1);
            }
            tz_fence_after();
            any_late |= tz_epilogue([](int &) {}, tmem, 1, quad, seg, lane, bar_free + 1, Kn, xch + 4 * TZ_M, carry_h, out, p, m,
                                    batch, tile, late, pmap, bar_staged_out, bar_out_free, 2 * it + 1, out_flags,
                                    late_out, status, wait_ns);
            late = late_out;   // carried into the next tile's first vote
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

// cuTensorMapEncodeTiled, looked up once through the runtime (no driver
// library link); null if the driver does not offer it
typedef CUresult (*tz_encode_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static tz_encode_fn tz_encoder()
{
    static const tz_encode_fn fn = []() -> tz_encode_fn {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return (tz_encode_fn)f;
    }();
    return fn;
}

// Tensor map of the product rows p: [batch][2m] uint32, boxes of 32 limbs x
// 128 rows with the 128-byte swizzle.  False where the tensor store cannot
// serve (odd m: rows not 16-byte multiples; p unaligned; coordinates past
// int32), and the kernel then writes rows with plain stores.
static bool tz_make_map(CUtensorMap *map, uint32_t *p, size_t m, size_t batch)
{
    memset(map, 0, sizeof *map);
    const tz_encode_fn enc = tz_encoder();
    if (!enc || m % 2 != 0 || !aligned16(p) || batch > (size_t)INT32_MAX) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * m), (cuuint64_t)batch};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * m * 4)};
    const cuuint32_t box[2] = {32, TZ_M};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, p, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

extern "C" {

DOT_API dot_status_t dot_mul_shared(dot_ctx_t ctx, const uint32_t *fixed, const uint32_t *b, uint32_t *p,
                                    size_t m, size_t batch, int use_tensor_cores, dot_stream_t stream)
{
    DeviceScope scope;
    dot_status_t rc = dot_check_ctx(ctx, scope);
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
        CUtensorMap map;
        const int use_map = tz_make_map(&map, p, m, batch) ? 1 : 0;
        toeplitz_mma_kernel<<<grid, TZ_THREADS, TZ_SMEM, st>>>(fixed, b, p, (int)m, batch, map, use_map,
                                                              ctx->d_status, ctx->wait_limit_ns);
        return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
    }
    dot_plan_t pl;
    rc = dot_make_plan(DOT_OP_MUL, m, batch, true, &pl, ctx->tune[DOT_OP_MUL][dot_tune_bucket(m)]);
    if (rc != DOT_OK) return rc;
    switch (pl.seg_limbs) {
    case 4: return launch_shared_int<4>(ctx, pl, fixed, b, p, m, batch, st);
    case 8: return launch_shared_int<8>(ctx, pl, fixed, b, p, m, batch, st);
    case 12: return launch_shared_int<12>(ctx, pl, fixed, b, p, m, batch, st);
    default: return launch_shared_int<16>(ctx, pl, fixed, b, p, m, batch, st);
    }
}

}  // extern "C"
