/*
 * dot.h -- C ABI of libdot, a GB300 (sm_103a) library for exact multi-limb
 * unsigned integer add, subtract and multiply, after "Leveraging SIMD for
 * Accelerating Large-number Arithmetic" (DigitsOnTurbo, DoT).
 *
 * Number format (Sec. 2.1, Table 2).  An operand of m limbs is the integer
 *     A = sum_{i<m} A_i X^i,  X = 2^32,  0 <= A_i < X,
 * stored little-endian as uint32_t[m] (A_0 first).  A batch of equal-size
 * operands is row-major uint32_t[batch][m]; a ragged batch is packed
 * back-to-back with an offsets array (CSR style).
 *
 * Memory.  Unless a function says "host", every pointer is a device pointer
 * (cudaMalloc, torch tensors, ...) owned by the caller; the library never
 * frees it.  A dot_ctx_t owns all scratch (look-back tile states, counters,
 * the sticky status word, staging buffers, captured graphs).  Calls are
 * asynchronous on `stream` (a cudaStream_t passed as void*, NULL = legacy
 * default stream).  Calls that share a ctx must be ordered on one stream:
 * two in flight at once on different streams race on the ctx scratch.
 *
 * Aliasing.  For add/sub the result may alias an operand exactly (in-place,
 * s == a or s == b) but must not overlap it partially.  A product must not
 * overlap its operands.  Detectable violations give DOT_EINVAL.
 *
 * Errors.  Argument errors are returned synchronously before any launch and
 * nothing is written.  Launch failures give DOT_ECUDA.  Device-side errors
 * (a bounded wait that ran out) are recorded in the ctx and returned, and
 * cleared, by dot_ctx_check.  The library never exits, aborts or traps.
 *
 * There is no CPU fallback: every entry point runs its work on the GPU.
 */
#ifndef DOT_H
#define DOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DOT_API __attribute__((visibility("default")))
#else
#define DOT_API
#endif

#define DOT_ABI_VERSION 1

typedef enum dot_status {
    DOT_OK = 0,
    DOT_EINVAL = 1,        /* bad argument: null pointer, overlap, size overflow */
    DOT_ECUDA = 2,         /* a CUDA runtime call or kernel launch failed        */
    DOT_ENOMEM = 3,        /* scratch allocation failed                          */
    DOT_ETIMEOUT = 4,      /* a bounded device-side wait ran out (see check)     */
    DOT_EUNSUPPORTED = 5   /* size or mode outside what the kernels implement   */
} dot_status_t;

/* operation codes of mixed ragged descriptors */
enum { DOT_OP_ADD = 0, DOT_OP_SUB = 1, DOT_OP_MUL = 2 };

/* Largest operand (limbs) of the column-sum multiply kernels. */
#define DOT_MUL_MAX_LIMBS 512
/* Largest operand (limbs) of dot_mul_karatsuba (2^25 bits). */
#define DOT_KARA_MAX_LIMBS (1u << 20)
/* Digit width and largest operand (digits) of dot_mul_unsat. */
#define DOT_UNSAT_BITS 27
#define DOT_UNSAT_MAX_DIGITS 512

typedef struct dot_ctx *dot_ctx_t;
typedef void *dot_stream_t;   /* cudaStream_t */

/* ---------------------------------------------------------------- ctx --- */

/* Create a context on CUDA device `device`; allocates its scratch there.
 * *out is set only on DOT_OK.  Errors: DOT_EINVAL (out NULL), DOT_ECUDA,
 * DOT_ENOMEM. */
DOT_API dot_status_t dot_ctx_create(dot_ctx_t *out, int device);

/* Free a context and its scratch (synchronises its device).  NULL is a no-op. */
DOT_API void dot_ctx_destroy(dot_ctx_t ctx);

/* Synchronise `stream`, then return and clear the ctx's sticky device status
 * (DOT_OK, or DOT_ETIMEOUT if a bounded look-back wait ran out since the last
 * check), or DOT_ECUDA if the stream reports an error. */
DOT_API dot_status_t dot_ctx_check(dot_ctx_t ctx, dot_stream_t stream);

/* Upper bound, in nanoseconds, on any single device-side wait of this ctx
 * (default 2e9 = 2 s).  After it a waiting thread block records DOT_ETIMEOUT,
 * treats the missing carry as 0 and finishes, so every launch terminates. */
DOT_API dot_status_t dot_ctx_set_wait_limit(dot_ctx_t ctx, uint64_t nanoseconds);

/* Static description of a status code; never NULL. */
DOT_API const char *dot_status_str(dot_status_t status);

/* DOT_ABI_VERSION of the loaded library. */
DOT_API int dot_abi_version(void);

/* ------------------------------------------------------- add / subtract --- */

/* Batched addition, Alg. 1 (DoT-Add-Words) and Theorem 1 (Sec. 3.1):
 * for each row k < batch,  s[k] + carry_out[k] * X^m = a[k] + b[k].
 * a, b, s: uint32_t[batch][m]; carry_out: uint32_t[batch], each 0 or 1.
 * Operands longer than one thread block's tile are chained across blocks by
 * decoupled look-back.  m == 0 gives carry 0; batch == 0 is a no-op. */
DOT_API dot_status_t dot_add(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b,
                             uint32_t *s, uint32_t *carry_out, size_t m, size_t batch,
                             dot_stream_t stream);

/* Batched subtraction, the borrow mirror of Alg. 1 (Sec. 3.1, "Subtraction"):
 * d[k] - borrow_out[k] * X^m = a[k] - b[k], borrow_out[k] = 1 iff a[k] < b[k]
 * (the difference then wraps modulo X^m).  Layout as dot_add. */
DOT_API dot_status_t dot_sub(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b,
                             uint32_t *d, uint32_t *borrow_out, size_t m, size_t batch,
                             dot_stream_t stream);

/* Ragged addition / subtraction: op k has m_k = off[k+1] - off[k] limbs at
 * a + off[k], b + off[k], written to s + off[k]; carry/borrow to [k].
 * off: device uint64_t[batch + 1], non-decreasing (checked on the device:
 * a decreasing entry records DOT_EINVAL in the ctx and the op is skipped). */
DOT_API dot_status_t dot_add_ragged(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b,
                                    uint32_t *s, uint32_t *carry_out, const uint64_t *off,
                                    size_t batch, dot_stream_t stream);
DOT_API dot_status_t dot_sub_ragged(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b,
                                    uint32_t *d, uint32_t *borrow_out, const uint64_t *off,
                                    size_t batch, dot_stream_t stream);

/* mpn-style variants of the same addition and subtraction -- the library
 * primitives DoT replaces when integrated into a big-number library (Sec. 3.3,
 * "Implementation"; the textbook MPN-ADD-M of the appendix takes a carry-in
 * and operands of different lengths).  All are batched over rows k < batch,
 * one warp per op; results and carries as dot_add / dot_sub.  s (d) may be a
 * exactly; other overlaps of outputs with inputs give DOT_EINVAL. */

/* With a carry-in: s[k] + carry_out[k] X^m = a[k] + b[k] + [carry_in[k] != 0].
 * carry_in: device uint32_t[batch] (required).  m == 0 gives carry_out =
 * carry_in. */
DOT_API dot_status_t dot_add_nc(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b,
                                const uint32_t *carry_in, uint32_t *s, uint32_t *carry_out,
                                size_t m, size_t batch, dot_stream_t stream);
/* With a borrow-in: d[k] - borrow_out[k] X^m = a[k] - b[k] - [borrow_in[k] != 0]. */
DOT_API dot_status_t dot_sub_nc(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b,
                                const uint32_t *borrow_in, uint32_t *d, uint32_t *borrow_out,
                                size_t m, size_t batch, dot_stream_t stream);

/* One-limb operand: s[k] + carry_out[k] X^m = a[k] + b[k], where b is
 * uint32_t[batch] (one limb per op) and a, s are uint32_t[batch][m], m >= 1
 * (m == 0 with batch > 0: DOT_EINVAL). */
DOT_API dot_status_t dot_add_1(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *s,
                               uint32_t *carry_out, size_t m, size_t batch, dot_stream_t stream);
DOT_API dot_status_t dot_sub_1(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *d,
                               uint32_t *borrow_out, size_t m, size_t batch, dot_stream_t stream);

/* Unequal lengths: a is uint32_t[batch][ma], b is uint32_t[batch][mb] with
 * mb <= ma (else DOT_EINVAL), taken as zero-padded to ma limbs (the padding
 * of Theorem 2's proof); s: uint32_t[batch][ma] with
 * s[k] + carry_out[k] X^ma = a[k] + b[k] (d[k] - borrow_out[k] X^ma =
 * a[k] - b[k]).  ma == 0 gives carry 0. */
DOT_API dot_status_t dot_add_unequal(dot_ctx_t ctx, const uint32_t *a, size_t ma, const uint32_t *b,
                                     size_t mb, uint32_t *s, uint32_t *carry_out, size_t batch,
                                     dot_stream_t stream);
DOT_API dot_status_t dot_sub_unequal(dot_ctx_t ctx, const uint32_t *a, size_t ma, const uint32_t *b,
                                     size_t mb, uint32_t *d, uint32_t *borrow_out, size_t batch,
                                     dot_stream_t stream);

/* --------------------------------------------------------------- multiply --- */

/* Batched product, Alg. 2 (DoT-Mul-Words) and Theorem 2 (Sec. 3.2):
 * p[k] = a[k] * b[k] as exactly 2m limbs.  a, b: uint32_t[batch][m];
 * p: uint32_t[batch][2m], must not overlap a or b.  Column sums of
 * independent 32x32->64 partial products, then one exact carry-resolution
 * pass.  1 <= m <= DOT_MUL_MAX_LIMBS, else DOT_EUNSUPPORTED (m == 0: no-op). */
DOT_API dot_status_t dot_mul(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b,
                             uint32_t *p, size_t m, size_t batch, dot_stream_t stream);

/* Batched square, p[k] = a[k]^2 as 2m limbs: Theorem 2 (Sec. 3.2) with
 * A = B, where each column sum is twice the sum over the pairs i < j plus
 * the diagonal square A_{c/2}^2 -- half the partial products of dot_mul.
 * a: uint32_t[batch][m]; p: uint32_t[batch][2m], no overlap with a.
 * 1 <= m <= DOT_MUL_MAX_LIMBS, else DOT_EUNSUPPORTED (m == 0: no-op). */
DOT_API dot_status_t dot_sqr(dot_ctx_t ctx, const uint32_t *a, uint32_t *p, size_t m, size_t batch,
                             dot_stream_t stream);

/* Batched product of any size, p[k] = a[k] * b[k] as 2m limbs: the
 * appendix's MPN-KARATSUBA (Karatsuba, or Toom-Cook 2-way), a recursion that
 * ends in the column-sum base case (Sec. 2): above 384 limbs each level
 * splits at h = ceil(m / 2), forms |A_H - A_L| and |B_H - B_L| with their
 * signs, runs the three half-size products as one batched product over
 * 3 x batch operations, and combines P1 b^2 + (P1 + P0 - P2) b + P0 on the
 * add path; at or below 384 limbs it is dot_mul (whose 385..512-limb shape
 * is slower than one more level over 193..256-limb products).  Layout as
 * dot_mul; 1 <= m <= DOT_KARA_MAX_LIMBS (else DOT_EINVAL), m == 0 no-op.
 * Uses a workspace owned by ctx (about 14 m batch bytes per level, grown on
 * demand with a device synchronisation; DOT_ENOMEM if it cannot grow):
 * calls on one ctx must not overlap on the GPU. */
DOT_API dot_status_t dot_mul_karatsuba(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b,
                                       uint32_t *p, size_t m, size_t batch, dot_stream_t stream);

/* Batched product in an UNSATURATED radix (Sec. 2.1: limbs that keep
 * headroom to simplify carry handling; the paper's 5x5 multiply uses 52-bit
 * digits, Sec. 3.3).  An operand of n digits is A = sum_{i<n} A_i 2^(27 i),
 * each digit a uint32_t below 2^27 (DOT_UNSAT_BITS); p[k] = a[k] * b[k] as
 * exactly 2n such digits.  a, b: uint32_t[batch][n]; p: uint32_t[batch][2n],
 * no overlap with the inputs.  Every partial product is one 32 x 32 -> 64-bit
 * multiply-add into a 64-bit column sum (no carry chain: up to 2^10 digit
 * products fit), then the carry pass of Alg. 2 Phase 5 in radix 2^27.
 * 1 <= n <= DOT_UNSAT_MAX_DIGITS, else DOT_EUNSUPPORTED (n == 0: no-op).  An
 * input digit of 2^27 or more records DOT_EINVAL in the ctx (read by
 * dot_ctx_check) and leaves that product unspecified. */
DOT_API dot_status_t dot_mul_unsat(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *p,
                                   size_t n, size_t batch, dot_stream_t stream);

/* Ragged product: op k has m_k = off[k+1] - off[k] limbs (<= DOT_MUL_MAX_LIMBS,
 * larger ops record DOT_EUNSUPPORTED in the ctx and are skipped); its 2 m_k
 * product limbs go to p + poff[k].  off, poff: device uint64_t[batch + 1]. */
DOT_API dot_status_t dot_mul_ragged(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b,
                                    uint32_t *p, const uint64_t *off, const uint64_t *poff,
                                    size_t batch, dot_stream_t stream);

/* One fixed operand times a batch: p[k] = fixed * b[k] as 2m limbs.
 * fixed: uint32_t[m]; b: uint32_t[batch][m]; p: uint32_t[batch][2m] (no
 * overlap with the inputs).  The column sums of Theorem 2 (Sec. 3.2) over
 * 8-bit digits of a fixed operand form one matrix product with a Toeplitz
 * matrix; use_tensor_cores != 0 runs it on the tensor cores (tcgen05.mma,
 * fp16 digits -- the batch's shifted by -128, the fixed operand's balanced
 * to [-128, 128] -- with fp32 accumulation, exact because every partial sum
 * over at most 256 batch digits stays an integer within 2^22 of the
 * accumulator's start 1.5 * 2^23; operands of 65 to 128 limbs split K into two
 * such slices whose sums are added as integers before the carry pass) and
 * normalises the carries in the epilogue; it needs 1 <= m <= 128 (4096
 * bits), else DOT_EUNSUPPORTED.  use_tensor_cores == 0 runs the INT32
 * column-sum path of dot_mul (m <= DOT_MUL_MAX_LIMBS). */
DOT_API dot_status_t dot_mul_shared(dot_ctx_t ctx, const uint32_t *fixed, const uint32_t *b,
                                    uint32_t *p, size_t m, size_t batch, int use_tensor_cores,
                                    dot_stream_t stream);

/* ------------------------------------------------------------ mixed batch --- */

/* One operation of a mixed ragged batch (32 bytes).  Operand a occupies
 * a[a_off .. a_off + m), operand b occupies b[b_off .. b_off + m); the result
 * (m limbs for add/sub, 2m for mul) goes to r[r_off ..]; the carry/borrow of
 * descriptor i goes to carry[i] (0 for a product). */
typedef struct dot_desc {
    uint32_t op;      /* DOT_OP_ADD, DOT_OP_SUB or DOT_OP_MUL */
    uint32_t m;       /* limbs of each operand */
    uint64_t a_off;
    uint64_t b_off;
    uint64_t r_off;
} dot_desc_t;

/* Mixed ragged batch of add/sub/mul operations (device descriptors).
 * The library sorts the ops into size buckets on the device and runs them in
 * one persistent kernel replayed from a captured CUDA graph, with tile shapes
 * from its tuning table.  Mul ops need m <= DOT_MUL_MAX_LIMBS; larger ones and
 * unknown op codes record DOT_EUNSUPPORTED / DOT_EINVAL and are skipped. */
DOT_API dot_status_t dot_mixed_ragged(dot_ctx_t ctx, const dot_desc_t *desc, size_t nops,
                                      const uint32_t *a, const uint32_t *b, uint32_t *r,
                                      uint32_t *carry, dot_stream_t stream);

/* ---------------------------------------------------- host-buffer variants --- */

/* Same results as dot_add / dot_sub / dot_mul, but a, b and the outputs are
 * HOST pointers (pinned memory gives asynchronous copies; pageable memory
 * works but is staged by the driver).  The library copies the operands into
 * two ctx-owned device staging buffers chunk by chunk, computes, and copies
 * the results back: copies in and copies out run on two ctx streams and the
 * kernels on `stream`, so both copy directions stay busy at once.  Returns
 * after enqueueing; the host outputs are valid once `stream` has been
 * synchronised (dot_ctx_check does that). */
DOT_API dot_status_t dot_add_host(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b,
                                  uint32_t *s, uint32_t *carry_out, size_t m, size_t batch,
                                  dot_stream_t stream);
DOT_API dot_status_t dot_sub_host(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b,
                                  uint32_t *d, uint32_t *borrow_out, size_t m, size_t batch,
                                  dot_stream_t stream);
DOT_API dot_status_t dot_mul_host(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b,
                                  uint32_t *p, size_t m, size_t batch, dot_stream_t stream);

/* ------------------------------------------------------------ autotuning --- */

/* Tile and limbs-per-thread shapes, chosen per context and per size class
 * (op, bit length of m).  The paper fixes its SIMD width at compile time;
 * this table and the autotuner are this library's own.  A knob value is:
 *   DOT_OP_MUL: R, the output columns each thread accumulates (4, 8, 12 or
 *               16; needs m <= 32 R);
 *   DOT_OP_ADD / DOT_OP_SUB: segments per thread of the tiled look-back
 *               kernel (1, 2 or 4, i.e. 1024- to 4096-limb tiles; used only
 *               for operands longer than 512 limbs).
 * 0 restores the built-in choice.  Errors: DOT_EINVAL for an unknown op, m 0
 * or a value the kernels do not implement for m. */
DOT_API dot_status_t dot_tune_set(dot_ctx_t ctx, int op, size_t m, int value);
DOT_API dot_status_t dot_tune_get(dot_ctx_t ctx, int op, size_t m, int *value);

/* Time every valid knob for (op, m) on `batch` synthetic operand pairs
 * (device memory allocated and freed inside the call; synchronous, on the
 * ctx's private stream), keep the fastest in the table and return it in
 * *best (and its mean time per call in *best_ms, which may be NULL).
 * *best is 0 when the size has nothing to tune (add/sub of <= 512 limbs). */
DOT_API dot_status_t dot_autotune(dot_ctx_t ctx, int op, size_t m, size_t batch, int *best,
                                  float *best_ms);

/* ------------------------------------------------- allocation-free add --- */

/* dot_add without any device allocation, for callers that must not call
 * cudaMalloc: code that runs inside another allocator's callbacks, in a
 * latency-critical or signal-handling path that may not block on the driver's
 * memory manager, or in a process whose device memory is all owned by a pool
 * it cannot share.  (The paper has no counterpart: it is a packaging choice of
 * this library.)  Same result and layout as dot_add: s[k] + carry_out[k] X^m
 * = a[k] + b[k]; a, b, s, carry_out and stream belong to CUDA device `device`.
 *
 * No dot_ctx_t is used (creating one allocates).  The scratch of the tiled
 * look-back kernel is a fixed device array inside the library, which every GPU
 * that loads libdot holds until the process exits: 4 + 16384 64-bit words
 * (128 KiB), i.e. at most 16384 tiles per call, where one op of m limbs spans
 * ceil(m / tile) tiles of 1024 to 4096 limbs (256 to 1024 limbs when m % 4 != 0
 * or a row is not 16-byte aligned); larger calls return DOT_EUNSUPPORTED
 * before any launch.  Ops of at most 512 limbs (128 for the unaligned case)
 * run without tiles and have no limit on batch.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, which may load the library's kernels onto the
 * device); make that first call before any stream capture.  Every call
 * shares the one array: a call clears the part it uses on `stream` before
 * its kernel runs, and calls whose kernels overlap on the GPU (different
 * streams, or different host threads on one device) race and may give wrong
 * results.  There is no context to record a device-side wait timeout in:
 * such a timeout (a wait of over 2 s, which a healthy GPU never reaches) is
 * not reported.  Argument errors are returned as by dot_add. */
DOT_API dot_status_t dot_add_noalloc(int device, const uint32_t *a, const uint32_t *b,
                                     uint32_t *s, uint32_t *carry_out, size_t m, size_t batch,
                                     dot_stream_t stream);

/* ------------------------------------------------------- introspection --- */

/* The launch plan the library uses for one batched call (host logic only,
 * needs no GPU).  op is DOT_OP_ADD / SUB / MUL. */
typedef struct dot_plan {
    int kernel;          /* 1 warp-segmented add/sub, 2 tiled add/sub with
                            look-back, 3 column-sum multiply, 4 one product
                            per thread (m <= 16, or m <= 32 in batches of
                            at least 16384), 0 nothing to do */
    int seg_limbs;       /* limbs per thread segment (vector width)          */
    int lanes_per_op;    /* threads that cooperate on one op (<= 32), or the
                            threads of one tile for kernel 2                  */
    int chunks;          /* segments per thread                              */
    uint64_t tile_limbs; /* limbs per tile (kernel 2)                        */
    uint64_t tiles;      /* tiles per op (kernel 2)                          */
    uint64_t m_pad;      /* padded operand length (kernel 3)                 */
} dot_plan_t;

DOT_API dot_status_t dot_plan_batched(int op, size_t m, size_t batch, int vector_ok,
                                      dot_plan_t *out);

/* ----------------------------------------------------------- debug hook --- */

/* Test hook for the bounded waits: while set, the next dot_add / dot_sub on
 * this ctx that uses look-back never publishes the carry state of tile
 * `tile` of op 0, so its successor's wait runs out (DOT_ETIMEOUT at the next
 * dot_ctx_check; results of that op are then unspecified).  -1 clears it. */
DOT_API dot_status_t dot_debug_skip_publish(dot_ctx_t ctx, int64_t tile);

#ifdef __cplusplus
}
#endif

#endif /* DOT_H */
