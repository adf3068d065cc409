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
// magnitude, and a sum over at most 256 batch digits lies in [-2^22, 2^22],
// so an fp32 accumulator started at M = 1.5 * 2^23 stays in [2^23, 2^24],
// where fp32 holds every integer exactly and its bit pattern is bits(M) plus
// the sum -- no float-to-integer conversion.  Operands above 64 limbs have
// more than 256 batch digits: their K dimension is split into slices of two
// 128-digit k-blocks, each slice accumulated in a region of its own, and the
// slices' bit patterns are added as integers before the carry pass.  The true
// column sum is C_c = R_c + 128 W_c with W_c the sum of the a_u over the
// window u = c - t, t in [0, 4m): a per-column constant.  With v_c the sum of
// the slices' bits for column c, the product is
//     P = sum_l (sum_q v_{4l+q} 2^(8q)) 2^(32 l) + K  (mod 2^(64 m)),
// K = sum_l (128 sum_q W_{4l+q} 2^(8q) - S bits(M) 0x01010101) 2^(32 l) for S
// slices: one constant per fixed operand, normalised once into 2m limbs, so
// every term is nonnegative and the per-row carry pass is unsigned.
//
// Operands of the Toeplitz product.  Reversing the order of the N rows of
// the B operand of one product turns its Toeplitz block into a Hankel block:
// row n' holds a_{C - n' - k} for k = 0..127, a window that starts one digit
// later in a reversed digit array for each next row.  So every block of every
// diagonal is read from ONE small array: eight interleaved copies of the
// reversed digits, shifted by 0..7, laid out so that the 16-byte chunk that
// starts at any index i sits at (i / 8) * 128 + (i % 8) * 16 bytes.  A
// K-major operand without swizzle then has its 8-row core matrices at 128-byte
// steps both along N and along K (the two descriptor strides alias, which is
// fine for an operand that is only read), and the diagonal d = cb - kb only
// moves the start address.  The product's columns come out reversed inside
// each 128-column block, which the epilogue undoes when it reads them.
//
// Kernel layout (one CTA of 18 warps per SM, persistent over tiles of 128
// operands; output in blocks of 128 columns = 32 limbs):
//   * Block pipeline: block i of the CTA's sequence (tile-major) accumulates
//     in tensor-memory unit i mod 2 (S regions of 128 columns each), and is
//     drained, regrouped and stored by worker group i mod 4 (four warps, one
//     per tensor-memory lane quadrant, so that each thread owns one operand
//     row of the block).  The carry word of each row passes from block to
//     block through shared memory, and only its addition waits for the
//     previous block.
//   * One issuer thread issues, per block and region, a rank-one bias product
//     (3072 x 4096 = M, which also resets the region) and the products of
//     every k-block that meets the block (tcgen05.mma, M = 128, N = 128,
//     K = 16), then commits the block to its group's mbarrier.
//   * Batch digits are converted to fp16 by the worker groups.  Up to 64
//     limbs they are written to tensor memory (tcgen05.st) and the products
//     read their A operand from there, so that shared memory feeds only the
//     B operand; the k-block slots of two tiles alternate, and a group
//     converts its share of the next tile after draining its block.  Up to
//     128 limbs they go to one shared-memory slot per k-block, refilled with
//     the next tile's k-block as soon as the last block that reads it has
//     its products -- by the group of that block, before it drains it.
//   * Each group stages its block's 32 limbs per row (128-byte swizzle) and
//     one of its threads writes the block with a tensor store (TMA): one
//     16 KB box, where per-thread row stores (rows 8m bytes apart) would
//     split every warp store into 32 partial lines.
//   * The constant K is formed while the first products run: a prefix scan
//     of the fixed operand's balanced digits and the per-limb constants by
//     the worker warps, the normalisation into limbs by warp 17.
#include <cuda.h>
#include <cuda_fp16.h>
#include <string.h>

#include "dot_internal.cuh"
#include "dot_plan.h"
#include "dot_mul.cuh"

#define TZ_WORKERS 512                 // 16 worker warps: four groups of four
#define TZ_THREADS (TZ_WORKERS + 64)   // + the issuer warp + the constant warp
#define TZ_M 128                       // operands per tile (MMA M)
#define TZ_MAX_LIMBS 128
#define TZ_KBUF (TZ_M * 128 * 2)       // one k-block slot: 128 rows x 128 digits, fp16
#define TZ_BIAS_BYTES (128 * 16 * 2)   // one bias operand, 128 x 16 fp16
#define TZ_DIGITS (4 * TZ_MAX_LIMBS + 1)
#define TZ_BOX (TZ_M * 128)            // one staged block: 128 rows x 32 limbs, 128-byte swizzle
#define TZ_DIG_WORDS 576               // >= TZ_DIGITS + 40, a multiple of 16 words
// fp32 bits of the accumulator start value M = 1.5 * 2^23 = 3072 * 4096
#define TZ_MAGIC_BITS 0x4B400000u
static_assert(TZ_DIG_WORDS >= TZ_DIGITS + 40 && TZ_DIG_WORDS % 16 == 0, "digit arrays");
static_assert(TZ_DIGITS <= TZ_THREADS, "one balanced digit per thread");

// Storage for S K slices.  One slice (up to 64 limbs, at most 2 k-blocks):
// the batch digits live in tensor memory, four k-block slots of 64 columns
// (two tiles, alternating) after two accumulator units of 128 columns, and
// each group has two staging boxes in shared memory, so that it stages its
// next block while the tensor store of the previous one still reads.  Two
// slices (up to 128 limbs, 4 k-blocks): two accumulator units of 256
// columns, four k-block slots in shared memory (slot kb holds k-block kb of
// one tile after another) and one box per group.  Shared memory is carved
// from a 1024-byte aligned base.
template <int S>
struct TzLayout {
    static constexpr int KBMAX = 2 * S;                   // k-blocks, and the most diagonals per column block
    static constexpr bool ATM = S == 1;                   // batch digits in tensor memory
    static constexpr bool ALT = S == 1;                   // slots alternate between tiles
    static constexpr int NU = 2;                          // accumulator units
    static constexpr int ACOL = 128 * S * NU;             // tensor-memory column of the digit slots
    static constexpr int ASLOTS = 4;                      // k-block slots
    static constexpr int SMEM_SLOTS = ATM ? 0 : ASLOTS;   // of them in shared memory
    static constexpr int BOXES = ATM ? 2 : 1;             // staging boxes per group
    static constexpr int HLEN = 128 * KBMAX + 256;        // entries of the reversed digit array
    static constexpr int OFF_OUT = SMEM_SLOTS * TZ_KBUF;
    static constexpr int OFF_H = OFF_OUT + 4 * BOXES * TZ_BOX;       // interleaved reversed digits
    static constexpr int OFF_BIAS = OFF_H + HLEN * 16;               // bias operands A, B
    static constexpr int OFF_KN = OFF_BIAS + 2 * TZ_BIAS_BYTES;      // uint32 [2 * TZ_MAX_LIMBS]: K
    static constexpr int OFF_CW = OFF_KN + 2 * TZ_MAX_LIMBS * 4;     // uint32 [4][128]: carry words
    static constexpr int OFF_DIG = OFF_CW + 4 * TZ_M * 4;            // int32 [TZ_DIG_WORDS]: balanced digits
    static constexpr int OFF_PRE = OFF_DIG + 4 * TZ_DIG_WORDS;       // int32 [TZ_DIG_WORDS]: prefix sums
    static constexpr int OFF_BARS = OFF_PRE + 4 * TZ_DIG_WORDS;      // mbarriers, tensor-memory address, flags
    static constexpr int SMEM = 1024 + OFF_BARS + 256;
    static_assert(OFF_H % 128 == 0 && OFF_BIAS % 128 == 0 && OFF_KN % 16 == 0 && OFF_CW % 16 == 0,
                  "operand and vector alignment");
    static_assert(OFF_BARS % 16 == 0, "mbarriers are 8-byte aligned");
    static_assert(OFF_OUT % 1024 == 0 && TZ_BOX % 1024 == 0, "swizzled staging boxes");
    static_assert(SMEM <= 227 * 1024, "shared memory");
    static_assert(ACOL + (ATM ? 64 * ASLOTS : 0) <= 512, "tensor memory");
};

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

// a * b + c (64-bit c and result)
__device__ __forceinline__ uint64_t tz_madw(uint32_t a, uint32_t b, uint64_t c)
{
    uint64_t d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// the same with the A operand read from tensor memory at atmem
__device__ __forceinline__ void tz_mma_ta(uint32_t dtmem, uint32_t atmem, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
                 :: "r"(dtmem), "r"(atmem), "l"(bd), "r"(idesc), "r"(acc) : "memory");
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

// 16 consecutive columns of this warp's 32 lanes (valid after a wait)
__device__ __forceinline__ void tz_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

// wait for this thread's tensor-memory loads, pinning two 16-column results
__device__ __forceinline__ void tz_ld_wait16x2(uint32_t (&a)[16], uint32_t (&b)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]),
                   "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]),
                   "+r"(a[14]), "+r"(a[15]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]),
                   "+r"(b[5]), "+r"(b[6]), "+r"(b[7]), "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]),
                   "+r"(b[12]), "+r"(b[13]), "+r"(b[14]), "+r"(b[15])
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

// all but the N most recent tensor stores of this thread have read their
// shared-memory source
template <int N>
__device__ __forceinline__ void tz_bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;" :: "n"(N) : "memory"); }

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
// Descriptor of the interleaved reversed-digit array as a K-major operand
// without swizzle: 8-row core matrices 128 bytes apart both along N (stride
// offset) and along K (leading offset).
__device__ __forceinline__ uint64_t tz_desc_hankel(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;   // next 8-k chunk
    d |= (uint64_t)(128 >> 4) << 32;   // next 8 rows
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(bar)) : "memory");
}

// One arrival per warp once all its lanes got here (barrier counts are in
// warps: hundreds of single-thread arrivals on one barrier word serialise).
__device__ __forceinline__ void tz_warp_arrive(uint64_t *bar)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

// Barrier 2 + g among the four warps of worker group g, which also returns
// whether any of them passed v != 0.
__device__ __forceinline__ int tz_group_sync_or(int g, int v)
{
    int r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\t"
                 "bar.red.or.pred q, %2, 128, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
                 : "=r"(r) : "r"(v), "r"(2 + g) : "memory");
    return r;
}

// Conversion unit (k-block kb, half h) of a tile, 16 limbs per thread of a
// worker group.  Into tensor memory (TM): limbs 16 h .. 16 h + 15 of the
// k-block for all 128 rows, thread j taking row j (its tensor-memory lane).
// Into a shared-memory slot: rows 64 h .. 64 h + 63, thread j taking limbs
// 16 (j % 2) .. + 15 of row 64 h + j / 2.  Rows past the batch read as zero.
template <bool TM>
__device__ __forceinline__ void tz_unit_load(uint32_t (&x)[16], const uint32_t *b, int m, size_t batch, size_t tile,
                                             int kb, int h, int j)
{
    const int row = TM ? j : 64 * h + (j >> 1);
    const size_t op = tile * TZ_M + row;
    const int l0 = 32 * kb + 16 * (TM ? h : j & 1);
    const uint32_t *src = b + op * (size_t)m + l0;
    // volatile: the loads issue here, not next to their first use, so that
    // their latency overlaps the work in between
    if (op < batch && l0 + 16 <= m && aligned16(src)) {
#pragma unroll
        for (int h = 0; h < 4; ++h)
            asm volatile("ld.global.cs.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(x[4 * h]), "=r"(x[4 * h + 1]), "=r"(x[4 * h + 2]), "=r"(x[4 * h + 3])
                         : "l"(src + 4 * h));
    } else {
#pragma unroll
        for (int l = 0; l < 16; ++l) {
            x[l] = 0u;
            if (op < batch && l0 + l < m) asm volatile("ld.global.cs.u32 %0, [%1];" : "=r"(x[l]) : "l"(src + l));
        }
    }
}

// The unit's digits, shifted by -128, as fp16 pairs into tensor memory: the
// A operand of the tensor-core product read from tensor memory holds row r
// in lane r, k elements 2c and 2c + 1 in column c (low and high half).  taddr
// addresses the warp's lane quadrant at the unit's first column.  Digits
// beyond the operand's 4m enter as 0 (not -128).
__device__ __forceinline__ void tz_unit_tmem(uint32_t taddr, const uint32_t (&x)[16], int l0, int m)
{
    uint32_t w[32];
    if (l0 + 16 <= m) {
#pragma unroll
        for (int l = 0; l < 16; ++l) {
            w[2 * l] = tz_shifted2(x[l], 0x4140);
            w[2 * l + 1] = tz_shifted2(x[l], 0x4342);
        }
    } else {
#pragma unroll
        for (int l = 0; l < 16; ++l) {
            const bool in = l0 + l < m;
            w[2 * l] = in ? tz_shifted2(x[l], 0x4140) : 0u;
            w[2 * l + 1] = in ? tz_shifted2(x[l], 0x4342) : 0u;
        }
    }
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
                 "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                 "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
                 :: "r"(taddr), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]),
                    "r"(w[7]), "r"(w[8]), "r"(w[9]), "r"(w[10]), "r"(w[11]), "r"(w[12]), "r"(w[13]), "r"(w[14]),
                    "r"(w[15]), "r"(w[16]), "r"(w[17]), "r"(w[18]), "r"(w[19]), "r"(w[20]), "r"(w[21]),
                    "r"(w[22]), "r"(w[23]), "r"(w[24]), "r"(w[25]), "r"(w[26]), "r"(w[27]), "r"(w[28]),
                    "r"(w[29]), "r"(w[30]), "r"(w[31])
                 : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// The unit's digits, shifted by -128, as fp16 into a k-block slot (128-byte
// swizzled, K-major).  Digits beyond the operand's 4m enter as 0 (not -128),
// so that every batch row has exactly the digit window the constant K assumes.
__device__ __forceinline__ void tz_unit_convert(unsigned char *slot, const uint32_t (&x)[16], int kb, int rh, int j,
                                                int m)
{
    const int row = 64 * rh + (j >> 1);
    const int lk0 = 16 * (j & 1);
    const int limb0 = 32 * kb + lk0;
#pragma unroll
    for (int l2 = 0; l2 < 8; ++l2) {
        const uint32_t x0 = x[2 * l2], x1 = x[2 * l2 + 1];
        uint4 v = make_uint4(tz_shifted2(x0, 0x4140), tz_shifted2(x0, 0x4342), tz_shifted2(x1, 0x4140),
                             tz_shifted2(x1, 0x4342));
        if (limb0 + 2 * l2 >= m) v.x = v.y = 0u;
        if (limb0 + 2 * l2 + 1 >= m) v.z = v.w = 0u;
        *reinterpret_cast<uint4 *>(slot + tz_off(row, 4 * (lk0 + 2 * l2), TZ_M)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The constant K = sum_{l < 2m} c_l 2^(32 l) mod 2^(64 m), with per-limb
// constants c_l = 128 sum_q W_{4l+q} 2^(8q) - S bits(M) 0x01010101 and W_c the
// sum of the balanced digits a_u over u in [max(0, c - 4m + 1), min(c, 4m)]
// (pre[u + 1] = a_0 + .. + a_u).  c_l of one limb:
__device__ __forceinline__ int64_t tz_limb_const(const int32_t *pre, int l, int nd, int S)
{
    int64_t k = -(int64_t)S * (int64_t)TZ_MAGIC_BITS * 0x01010101;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = 4 * l + q;
        const int lo = c - nd + 1 > 0 ? c - nd + 1 : 0, hi = c < nd ? c : nd;
        const int64_t W = lo <= hi ? (int64_t)(pre[hi + 1] - pre[lo]) : 0;
        k += W * 128 * ((int64_t)1 << (8 * q));
    }
    return k;
}

// K as 2m limbs from the c_l (one warp): each lane takes ceil(2m / 32)
// consecutive limbs through a signed serial carry, then the lanes pass carry
// words up until they no longer change.  Limbs from 2m on are written 0 by
// the caller.
__device__ __forceinline__ void tz_norm_k(const int64_t *ck, uint32_t *Kn, int m, int lane)
{
    // lane j takes limbs lpl j .. lpl j + lpl - 1, lpl = ceil(2m / 32) <= 8
    const int lpl = (2 * m + 31) >> 5;
    int64_t kl[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int l = lpl * lane + j;
        kl[j] = j < lpl && l < 2 * m ? ck[l] : 0;
    }
    uint32_t t[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    int64_t acc = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j < lpl) {   // past lpl the lane's carry word stays in acc
            acc = kl[j] + (acc >> 32);
            t[j] = (uint32_t)acc;
        }
    }
    const int64_t cw = acc >> 32;   // this lane's carry word with carry-in 0
    uint32_t all = DOT_FULL, any = 0u;
#pragma unroll
    for (int j = 1; j < 8; ++j) {
        if (j < lpl) {
            all &= t[j];
            any |= t[j];
        }
    }
    const bool ones = all == DOT_FULL, zeros = any == 0u;
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
    // apply the carry-in word: a carry or borrow out of limb 0 ripples while
    // the next limbs are all ones / all zero
    const int64_t s0 = (int64_t)t[0] + ci;
    t[0] = (uint32_t)s0;
    int32_t rip = (int32_t)(s0 >> 32);
#pragma unroll
    for (int j = 1; j < 8; ++j) {
        const uint32_t x = t[j];
        t[j] = x + (uint32_t)rip;
        rip = (rip > 0 && x == DOT_FULL) || (rip < 0 && x == 0u) ? rip : 0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int l = lpl * lane + j;
        if (j < lpl && l < 2 * m) Kn[l] = t[j];
    }
}

// named barriers of the 16 worker warps and warp 17 (544 threads) while they
// form K: 6 = prefix sums written, 7 = limb constants written
__device__ __forceinline__ void tz_kbar_sync(int id) { asm volatile("bar.sync %0, 544;" :: "r"(id) : "memory"); }
__device__ __forceinline__ void tz_kbar_arrive(int id) { asm volatile("bar.arrive %0, 544;" :: "r"(id) : "memory"); }

// fixed: m limbs (m <= 64 for S = 1, m <= 128 for S = 2), b: [batch][m],
// p: [batch][2m].  Warp 16 allocates tensor memory and issues every product
// (one lane); warp 17 normalises the constant K; warps 0..15 are four worker
// groups.  The CTA's blocks are numbered i = 0, 1, .. over its tiles (CB
// blocks per tile, CB = ceil(8m / 128)); block i accumulates in tensor-memory
// unit i mod NU (NU = 2 units of S regions) and is finished by group
// i mod 4.  Hand-offs (mbarriers; arrival counts in warps):
//   full[g]   block i's products done (tcgen05.commit), g = i mod 4   issuer -> group
//   free[u]   block i drained into registers (4), u = i mod NU  group -> issuer
//   carry[s]  block i's carry words in cw[s] (4), s = i mod 4    group -> next group
//   staged[k] a k-block slot holds the next tile's digits (8)    groups -> issuer
//   kn        the constant K is ready (1)                        warp 17 -> groups
// k-block slots: one slice alternates two tiles' slots (tensor memory), and
// a group converts its block's share of the next tile's digits after
// draining the block; two slices refill slot kb once the tile's last block
// that reads it has its products, and that block's group converts before it
// drains.  Either way from limbs loaded at the end of the group's previous
// block.
// Each barrier's consecutive phases are waited by one and the same party (a
// group waits full[g] for its blocks i, i + 4, ..; the issuer waits every
// free, staged phase), so a parity wait can never mistake a phase two back
// for the one it wants; and no producer can run two phases ahead of its
// consumer: every re-arm waits (through the others) for the consumer of the
// previous phase.
// Every wait is bounded; a wait that runs out records DOT_ETIMEOUT and sets a
// stop flag that every role checks between blocks (groups agree on it through
// their barrier), and the issuer waits (bounded) for its own last products
// before tensor memory is freed.
// 96 registers a thread at most: the 18 warps spread over the SM's four
// 16K-register partitions, five of them on two partitions
template <int S>
__global__ void __launch_bounds__(TZ_THREADS, 1)
toeplitz_mma_kernel(const uint32_t *fixed, const uint32_t *b, uint32_t *p, int m, size_t batch,
                    const __grid_constant__ CUtensorMap pmap_param, int use_map, uint32_t *status, uint64_t wait_ns)
{
    using Lay = TzLayout<S>;
    constexpr int NU = Lay::NU;
    extern __shared__ __align__(128) unsigned char tz_smem[];
    // swizzled tiles need a 1024-byte aligned base
    unsigned char *base = tz_smem + ((1024u - (smem_u32(tz_smem) & 1023u)) & 1023u);
    unsigned char *sA = base;
    unsigned char *sH = base + Lay::OFF_H;
    unsigned char *sBias = base + Lay::OFF_BIAS;
    uint32_t *Kn = (uint32_t *)(base + Lay::OFF_KN);
    uint32_t *cw = (uint32_t *)(base + Lay::OFF_CW);
    int32_t *dig = (int32_t *)(base + Lay::OFF_DIG);
    int32_t *pre = (int32_t *)(base + Lay::OFF_PRE);
    uint64_t *bars = (uint64_t *)(base + Lay::OFF_BARS);
    uint64_t *bar_full = bars, *bar_free = bars + 4, *bar_carry = bars + 8, *bar_staged = bars + 12;
    uint64_t *bar_kn = bars + 20;
    uint32_t *tmem_slot = (uint32_t *)(bars + 21);
    volatile uint32_t *stopf = tmem_slot + 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer = warp == TZ_WORKERS / 32, kwarp = warp == TZ_WORKERS / 32 + 1;
    const size_t ntiles = (batch + TZ_M - 1) / TZ_M;
    const CUtensorMap *pmap = use_map ? &pmap_param : nullptr;
    const int nd = 4 * m;                       // digits of each operand
    const int KB = (nd + 127) >> 7;             // k-blocks, and the most diagonals meeting a column block
    const int CB = (8 * m + 127) >> 7;          // column blocks of 128 (32 limbs)
    // k-block slot of tile number ts and its staging barrier (phase = use of
    // the slot): alternating between tiles, or slot kb
    constexpr bool alt = Lay::ALT;
    auto sidx = [&](int ts, int kb) { return alt ? KB * (ts & 1) + kb : kb; };
    auto slot = [&](int ts, int kb) -> unsigned char * { return sA + TZ_KBUF * sidx(ts, kb); };
    auto spar = [&](int ts) { return (uint32_t)(alt ? (ts >> 1) & 1 : ts & 1); };

    // the fixed operand's digits first (their latency gates the set-up), then
    // the first tile's limbs, in flight during the set-up
    uint32_t dk_word = 0, dp_word = 0;
    if (tid <= nd) {
        if (tid < nd) dk_word = fixed[tid >> 2];
        if (tid >= 1) dp_word = fixed[(tid - 1) >> 2];
    }
    // worker group g = warp / 4 (warps 0..15), its warp's lane quadrant and
    // the row j a thread owns
    const int g = warp >> 2, quad = warp & 3, j = tid & 127;
    // the first tile's units un = g and g + 4 of a worker group
    uint32_t xa[16], xb[16];
    if (tid < TZ_WORKERS && blockIdx.x < ntiles) {
        if (g < 2 * KB) tz_unit_load<Lay::ATM>(xa, b, m, batch, blockIdx.x, g >> 1, g & 1, j);
        if (g + 4 < 2 * KB) tz_unit_load<Lay::ATM>(xb, b, m, batch, blockIdx.x, (g + 4) >> 1, g & 1, j);
    }
    if (issuer) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(tmem_slot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        if (lane == 0) {
            for (int i = 0; i < 4; ++i) {
                mbar_init(bar_full + i, 1);
                mbar_init(bar_free + i, 4);
                mbar_init(bar_carry + i, 4);
            }
            for (int i = 0; i < 8; ++i) mbar_init(bar_staged + i, 8);
            mbar_init(bar_kn, 1);
            *stopf = 0u;
            mbar_init_fence();
        }
    }
    // bias operands: column k = 0 of A holds 3072, of B 4096 (fp16), the rest 0
    for (int i = tid; i < 2 * TZ_BIAS_BYTES / 16; i += TZ_THREADS) {
        const bool in_b = i >= TZ_BIAS_BYTES / 16;
        const int chunk = in_b ? i - TZ_BIAS_BYTES / 16 : i;
        const uint32_t first = chunk < 128 ? (in_b ? 0x6C00u : 0x6A00u) : 0u;
        *reinterpret_cast<uint4 *>(sBias + 16 * i) = make_uint4(first, 0u, 0u, 0u);
    }
    // balanced digits a_k = d_k + [d_{k-1} >= 128] - 256 [d_k >= 128], k <= 4m
    if (tid <= nd) {
        const uint32_t dk = tid < nd ? (dk_word >> (8 * (tid & 3))) & 0xFFu : 0u;
        const uint32_t dp = tid >= 1 ? (dp_word >> (8 * ((tid - 1) & 3))) & 0xFFu : 0u;
        dig[tid] = (int32_t)dk + (int32_t)(dp >= 128u) - 256 * (int32_t)(dk >= 128u);
    }
    tz_fence_before();
    __syncthreads();
    tz_fence_after();
    const uint32_t tmem = *tmem_slot;
    // unit un (k-block un / 2, half un % 2) of tile number tsn from the limbs
    // in x, by the four warps of a worker group
    auto convert = [&](int tsn, int un, const uint32_t (&x)[16]) {
        const int kb = un >> 1, h = un & 1;
        if (Lay::ATM)
            tz_unit_tmem(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(Lay::ACOL + 64 * sidx(tsn, kb) + 32 * h),
                         x, 32 * kb + 16 * h, m);
        else
            tz_unit_convert(slot(tsn, kb), x, kb, h, j, m);
        tz_fence_before();
        tz_warp_arrive(bar_staged + sidx(tsn, kb));
    };
    // K is formed by the worker warps and warp 17 (scan index ks, 544 threads):
    // a scan of the balanced digits inside each warp, warp totals into Kn
    // (free until K itself is written)
    const bool kthr = tid < TZ_WORKERS || kwarp;
    const int ks = kwarp ? TZ_WORKERS + lane : tid;
    int incl = 0;
    if (kthr) {
        incl = ks <= nd ? dig[ks] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) Kn[ks >> 5] = (uint32_t)incl;
    }
    // the reversed digits Rv(i) = a_{J - i}, J = 128 KB + 127, as eight
    // interleaved copies: the chunk of Rv(i .. i + 7) at (i / 8) * 128 + (i % 8) * 16
    {
        const int J = 128 * KB + 127, L = 128 * KB + 256;
        for (int i = tid; i < L; i += TZ_THREADS) {
            int v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int u = J - (i + e);
                v[e] = (u >= 0 && u <= nd) ? dig[u] : 0;
            }
            *reinterpret_cast<uint4 *>(sH + (i >> 3) * 128 + (i & 7) * 16) =
                make_uint4(tz_pack_signed2(v[0], v[1]), tz_pack_signed2(v[2], v[3]), tz_pack_signed2(v[4], v[5]),
                           tz_pack_signed2(v[6], v[7]));
        }
    }
    // the first tile's digits: unit un by group un mod 4
    if (tid < TZ_WORKERS && blockIdx.x < ntiles) {
        if (g < 2 * KB) convert(0, g, xa);
        if (g + 4 < 2 * KB) convert(0, g + 4, xb);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tz_fence_before();
    __syncthreads();
    tz_fence_after();
    if (kthr) {
        // prefix sums pre[u + 1] = a_0 + .. + a_u, then the limb constants c_l
        // (over the digit array, which nothing reads any more) and the zero
        // limbs of K past 2m
        int off = 0;
        for (int w = 0; w < (ks >> 5); ++w) off += (int)Kn[w];
        if (ks <= nd) pre[ks + 1] = incl + off;
        if (ks == 0) pre[0] = 0;
        tz_kbar_sync(6);
        int64_t *ck = reinterpret_cast<int64_t *>(dig);
        if (ks < 2 * m) ck[ks] = tz_limb_const(pre, ks, nd, S);
        else if (ks < 2 * TZ_MAX_LIMBS) Kn[ks] = 0u;
        if (kwarp) tz_kbar_sync(7);
        else tz_kbar_arrive(7);
    }

    if (issuer) {
        if (lane == 0) {
            const uint32_t i128 = tz_idesc(128);
            const uint64_t dH = tz_desc_hankel(smem_u32(sH));
            const uint64_t dba = tz_desc_plain(smem_u32(sBias), 128);
            const uint64_t dbb = tz_desc_plain(smem_u32(sBias + TZ_BIAS_BYTES), 128);
            int i = 0, last = -1;
            bool ok = true;
            for (int ts = 0; ok; ++ts) {
                const size_t tile = blockIdx.x + (size_t)ts * gridDim.x;
                if (tile >= ntiles) break;
                for (int cb = 0; cb < CB && ok; ++cb, ++i) {
                    const int u = i % NU, use = i / NU;
                    if (*stopf || (use > 0 && !mbar_wait_bounded(bar_free + u, (uint32_t)((use - 1) & 1), wait_ns))) {
                        ok = false;
                        break;
                    }
                    tz_fence_after();
#pragma unroll
                    for (int s = 0; s < S; ++s) tz_mma(tmem + 128 * (u * S + s), dba, dbb, i128, 0u);
                    const int kb_lo = cb - KB > 0 ? cb - KB : 0, kb_hi = cb < KB - 1 ? cb : KB - 1;
                    for (int kb = kb_lo; kb <= kb_hi; ++kb) {
                        if (kb == cb) {   // first block of the tile that reads this k-block
                            if (!mbar_wait_bounded(bar_staged + sidx(ts, kb), spar(ts), wait_ns)) {
                                ok = false;
                                break;
                            }
                            tz_fence_after();
                        }
                        const int d = cb - kb;
                        const uint32_t dcol = tmem + 128 * (u * S + (S == 2 ? kb >> 1 : 0));
                        const uint64_t bd0 = dH + (uint64_t)((2048 * (KB - d)) >> 4);
                        if (Lay::ATM) {
                            // k = 16 st: columns 8 st .. 8 st + 7 of the k-block's digits
                            const uint32_t acol = tmem + Lay::ACOL + 64 * sidx(ts, kb);
#pragma unroll
                            for (int st = 0; st < 8; ++st)
                                tz_mma_ta(dcol, acol + 8 * st, bd0 + (uint64_t)((st * 256) >> 4), i128, 1u);
                        } else {
                            const uint64_t ad0 = tz_desc(smem_u32(slot(ts, kb)));
#pragma unroll
                            for (int st = 0; st < 8; ++st) {
                                // k = 16 st: atom column st / 4 of A, 32 bytes per step inside it;
                                // two 8-k chunks of the reversed-digit array (256 bytes) per step
                                const uint64_t ad = ad0 + (uint64_t)(((st >> 2) * TZ_M * 128 + (st & 3) * 32) >> 4);
                                const uint64_t bd = bd0 + (uint64_t)((st * 256) >> 4);
                                tz_mma(dcol, ad, bd, i128, 1u);
                            }
                        }
                    }
                    if (!ok) break;
                    tz_commit(bar_full + (i & 3));
                    last = i;
                }
            }
            if (!ok) {
                record_status(status, DOT_ETIMEOUT);
                *stopf = 1u;
            }
            // our own products are done before tensor memory is freed (a
            // parity wait on a completed phase returns at once)
            if (last >= 0) mbar_wait_bounded(bar_full + (last & 3), (uint32_t)((last >> 2) & 1), wait_ns);
        }
        __syncwarp();
    } else if (kwarp) {
        tz_norm_k(reinterpret_cast<const int64_t *>(dig), Kn, m, lane);
        tz_warp_arrive(bar_kn);
    } else {
        int late = 0;
        // Conversion duty of block i: the units of the next tile whose slot
        // the block's products free -- alternating slots: the next tile's units
        // spread over the tile's blocks; slot kb: k-block kb once the last block
        // that reads it (kb + KB, or the tile's last) has its products.
        auto duty = [&](int i, int un) {
            const int ts = i / CB, cb = i - ts * CB;
            if (blockIdx.x + (size_t)(ts + 1) * gridDim.x >= ntiles) return false;
            if (alt) return un % CB == cb;
            const int kb = un >> 1, cl = kb + KB < CB - 1 ? kb + KB : CB - 1;
            return cl == cb;
        };
        auto next_duty = [&](int i, int un) {   // block i's first duty unit from un on (2 KB: none)
            while (un < 2 * KB && !duty(i, un)) ++un;
            return un;
        };
        // limbs of block i's first two duty units into xa, xb
        int xu0, xu1;
        auto prefetch = [&](int i) {
            xu0 = next_duty(i, 0);
            xu1 = xu0 < 2 * KB ? next_duty(i, xu0 + 1) : 2 * KB;
            const size_t tn = blockIdx.x + gridDim.x * (size_t)(i / CB + 1);
            if (xu0 < 2 * KB) tz_unit_load<Lay::ATM>(xa, b, m, batch, tn, xu0 >> 1, xu0 & 1, j);
            if (xu1 < 2 * KB) tz_unit_load<Lay::ATM>(xb, b, m, batch, tn, xu1 >> 1, xu1 & 1, j);
        };
        prefetch(g);
        late |= !mbar_wait_bounded(bar_kn, 0u, wait_ns);
        for (int i = g;; i += 4) {
            const int ts = i / CB, cb = i - ts * CB;
            const size_t tile = blockIdx.x + (size_t)ts * gridDim.x;
            if (tile >= ntiles) break;
            const int u = i % NU;
            uint32_t *out = (uint32_t *)(base + Lay::OFF_OUT +
                                         (g * Lay::BOXES + (Lay::BOXES == 2 ? (i >> 2) & 1 : 0)) * TZ_BOX);
            // the staging box is free once the group's store that last used it
            // has read it; the group agrees on stopping here (a named barrier
            // must never be left short of its participants)
            if (j == 0 && pmap) tz_bulk_wait_read<Lay::BOXES - 1>();
            if (tz_group_sync_or(g, (int)*stopf)) break;
            late |= !mbar_wait_bounded(bar_full + g, (uint32_t)((i >> 2) & 1), wait_ns);
            tz_fence_after();
            // conversion duty: the block's products are done, so the slots it
            // frees may take the next tile's digits.  Slot kb is needed again
            // soon: convert before draining; alternating slots are not needed
            // before the next tile: drain first, so that the unit is free sooner.
            if (!alt && xu0 < 2 * KB) {
                convert(ts + 1, xu0, xa);
                if (xu1 < 2 * KB) {
                    convert(ts + 1, xu1, xb);
                    for (int un = next_duty(i, xu1 + 1); un < 2 * KB; un = next_duty(i, un + 1)) {
                        tz_unit_load<Lay::ATM>(xa, b, m, batch, tile + gridDim.x, un >> 1, un & 1, j);
                        convert(ts + 1, un, xa);
                    }
                }
            }
            // drain the block, 32 columns (8 limbs) per pass; tensor-memory column
            // 127 - c of a region holds the block's column c.  One slice: the
            // next pass's columns load while this pass is summed.
            uint32_t hi = 0, all1 = DOT_FULL, o0 = 0;
            const uint32_t trow = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(128 * u * S);
            auto limbs = [&](const uint32_t (&v)[32], int pass) {
                const uint4 k0 = *reinterpret_cast<const uint4 *>(Kn + 32 * cb + 8 * pass);
                const uint4 k1 = *reinterpret_cast<const uint4 *>(Kn + 32 * cb + 8 * pass + 4);
                const uint32_t kk[8] = {k0.x, k0.y, k0.z, k0.w, k1.x, k1.y, k1.z, k1.w};
                // limb 8 pass + jj: columns 4 jj + q of the pass sit in register
                // 31 - 4 jj - q; each limb's sum is formed off the serial carry
                uint32_t o[8];
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const uint64_t L = (uint64_t)kk[jj] + v[31 - 4 * jj] + (uint64_t)v[30 - 4 * jj] * 256u +
                                       (uint64_t)v[29 - 4 * jj] * 65536u + (uint64_t)v[28 - 4 * jj] * 16777216u;
                    const uint64_t acc = L + hi;
                    o[jj] = (uint32_t)acc;
                    hi = (uint32_t)(acc >> 32);
                }
#pragma unroll
                for (int jj = 0; jj < 8; ++jj)
                    if (pass > 0 || jj > 0) all1 &= o[jj];
                if (pass == 0) o0 = o[0];
                *reinterpret_cast<uint4 *>(tz_stage(out, j, 2 * pass)) = make_uint4(o[0], o[1], o[2], o[3]);
                *reinterpret_cast<uint4 *>(tz_stage(out, j, 2 * pass + 1)) = make_uint4(o[4], o[5], o[6], o[7]);
            };
            if (S == 1) {
                uint32_t va[32], vb[32];
                tz_ld32(trow + 96, va);
                tz_ld_wait(va);
                tz_ld32(trow + 64, vb);
                limbs(va, 0);
                tz_ld_wait(vb);
                tz_ld32(trow + 32, va);
                limbs(vb, 1);
                tz_ld_wait(va);
                tz_ld32(trow, vb);
                limbs(va, 2);
                tz_ld_wait(vb);
                // every column of the block is in registers: the unit may be refilled
                tz_fence_before();
                tz_warp_arrive(bar_free + u);
                limbs(vb, 3);
            } else {
                // two slices: each pass sums 16-column halves of both regions
#pragma unroll
                for (int pass = 0; pass < 4; ++pass) {
                    uint32_t v[32];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        // columns 16 h .. 16 h + 15 of the pass sit at tensor-memory
                        // columns 127 - 32 pass - 16 h - 15 .. 127 - 32 pass - 16 h
                        uint32_t a0[16], a1[16];
                        const uint32_t taddr = trow + (uint32_t)(112 - 32 * pass - 16 * h);
                        tz_ld16(taddr, a0);
                        tz_ld16(taddr + 128, a1);
                        tz_ld_wait16x2(a0, a1);
                        // register r of the 16 holds pass column 16 h + 15 - r, which
                        // the 32-column order keeps in register 31 - (16 h + 15 - r)
#pragma unroll
                        for (int r = 0; r < 16; ++r) v[16 - 16 * h + r] = a0[r] + a1[r];
                    }
                    limbs(v, pass);
                }
                tz_fence_before();
                tz_warp_arrive(bar_free + u);
            }
            if (alt && xu0 < 2 * KB) {
                convert(ts + 1, xu0, xa);
                if (xu1 < 2 * KB) {
                    convert(ts + 1, xu1, xb);
                    for (int un = next_duty(i, xu1 + 1); un < 2 * KB; un = next_duty(i, un + 1)) {
                        tz_unit_load<Lay::ATM>(xa, b, m, batch, tile + gridDim.x, un >> 1, un & 1, j);
                        convert(ts + 1, un, xa);
                    }
                }
            }
            // the carry word from the previous block (every block waits, so that
            // the carry barriers stay in step; a tile's first block ignores it)
            uint32_t cin = 0;
            if (i > 0) {
                const int pi = i - 1;
                late |= !mbar_wait_bounded(bar_carry + (pi & 3), (uint32_t)((pi >> 2) & 1), wait_ns);
                if (cb != 0) cin = cw[(pi & 3) * TZ_M + j];
            }
            const uint64_t s0 = (uint64_t)o0 + cin;
            const uint32_t rip = (uint32_t)(s0 >> 32);
            tz_stage(out, j, 0)[0] = (uint32_t)s0;
            if (rip) {   // rare: the carry runs through limbs that are all ones
                for (int l = 1; l < 32; ++l) {
                    uint32_t *q = tz_stage(out, j, l >> 2) + (l & 3);
                    const uint32_t xv = *q;
                    *q = xv + 1u;
                    if (xv != DOT_FULL) break;
                }
            }
            cw[(i & 3) * TZ_M + j] = hi + (rip & (all1 == DOT_FULL ? 1u : 0u));
            tz_warp_arrive(bar_carry + (i & 3));
            // store the block: one tensor store of 32 limbs x 128 rows, or plain
            // stores of each thread's own row
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const int any_late = tz_group_sync_or(g, late);
            if (!any_late) {
                if (pmap) {
                    if (j == 0) tz_tma_store(pmap, out, 32 * cb, (int)(tile * TZ_M));
                } else {
                    const size_t op = tile * TZ_M + j;
                    if (op < batch) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const uint4 vv = *reinterpret_cast<const uint4 *>(tz_stage(out, j, c));
                            const uint32_t e4[4] = {vv.x, vv.y, vv.z, vv.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int l = 32 * cb + 4 * c + e;
                                if (l < 2 * m) st_stream1(p + op * (size_t)(2 * m) + l, e4[e]);
                            }
                        }
                    }
                }
            } else {
                if (j == 0) record_status(status, DOT_ETIMEOUT);
                *stopf = 1u;
                break;
            }
            // limbs of the group's next block's duty units
            prefetch(i + 4);
        }
        if (j == 0 && pmap) tz_bulk_wait_all();
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
        // up to 64 limbs one K slice (256 digits), up to 128 limbs two
        const bool split = m > 64;
        const void *fn = split ? (const void *)toeplitz_mma_kernel<2> : (const void *)toeplitz_mma_kernel<1>;
        const int smem = split ? TzLayout<2>::SMEM : TzLayout<1>::SMEM;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
            return DOT_ECUDA;
        const size_t ntiles = (batch + TZ_M - 1) / TZ_M;
        const unsigned grid = (unsigned)(ntiles < (size_t)ctx->num_sms ? ntiles : (size_t)ctx->num_sms);
        CUtensorMap map;
        const int use_map = tz_make_map(&map, p, m, batch) ? 1 : 0;
        if (split)
            toeplitz_mma_kernel<2><<<grid, TZ_THREADS, smem, st>>>(fixed, b, p, (int)m, batch, map, use_map,
                                                                     ctx->d_status, ctx->wait_limit_ns);
        else
            toeplitz_mma_kernel<1><<<grid, TZ_THREADS, smem, st>>>(fixed, b, p, (int)m, batch, map, use_map,
                                                                     ctx->d_status, ctx->wait_limit_ns);
        return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
    }
    // the column-sum plan (the fixed row is broadcast with stride 0)
    dot_plan_t pl;
    const int knob = ctx->tune[DOT_OP_MUL][dot_tune_bucket(m)];
    rc = dot_make_plan(DOT_OP_MUL, m, batch, true, &pl, knob ? knob : dot_mul_cols(m));
    if (rc != DOT_OK) return rc;
    switch (pl.seg_limbs) {
    case 4: return launch_shared_int<4>(ctx, pl, fixed, b, p, m, batch, st);
    case 8: return launch_shared_int<8>(ctx, pl, fixed, b, p, m, batch, st);
    case 12: return launch_shared_int<12>(ctx, pl, fixed, b, p, m, batch, st);
    default: return launch_shared_int<16>(ctx, pl, fixed, b, p, m, batch, st);
    }
}

}  // extern "C"
