/*
 * dot_probe.h -- C ABI of libdotprobe, the microbenchmarks that measure the
 * peaks libdot's kernels are reported against on the GPU they run on.
 *
 * These are measurement kernels, not part of the arithmetic: they compute
 * nothing a caller uses.  Each one runs a fixed instruction pattern in
 * independent chains with no memory traffic in its loop, so that its rate is
 * the ceiling of that pattern on the SM's pipes:
 *
 *   DOTP_MUL_PAIR     mul.lo.u32 + mul.hi.u32 of the same operands -- the two
 *                     multiplies of one 32 x 32 -> 64-bit limb product in the
 *                     column-sum multiply (Alg. 2 Phase 2, Sec. 3.2); unit: one
 *                     pair (= one limb product = two 32-bit multiplies);
 *   DOTP_COLSUM_R8    the column-sum multiply's whole inner step: per limb
 *                     product the two multiplies above and the three-word
 *                     add-with-carry into its column (Phases 2-4), on 8
 *                     columns per thread with a sliding window of the second
 *                     operand held in registers; unit: one limb product;
 *   DOTP_MADWIDE_R8   the same step with one mad.wide.u32 into a 64-bit
 *                     column sum (the unsaturated-radix form of Sec. 2.1 /
 *                     Sec. 3.3: digits below 2^27 need no carry chain);
 *                     unit: one digit product;
 *   DOTP_MUL_LO       mul.lo.u32 alone; unit: one 32-bit multiply;
 *   DOTP_EMPTY        an empty kernel (the launch floor); unit: one launch.
 *
 * and one tensor-pipe pattern per product shape of the fixed-operand
 * multiply (Sec. 3.2's column sums as a Toeplitz matrix product): one thread
 * per CTA issues `iters` x 4 tcgen05.mma of M = 128, N, K = 16 (fp16 digits,
 * fp32 accumulation) back to back into one accumulator, one CTA per SM (it
 * holds all of tensor memory; `threads` >= 32 only fills shared memory);
 * unit: one flop (2 M N K per instruction):
 *
 *   DOTP_MMA_N128_TMEM  N = 128, A read from tensor memory (the product of
 *                       the one-slice kernel, up to 64 limbs);
 *   DOTP_MMA_N128_SMEM  N = 128, A read from shared memory (two slices);
 *   DOTP_MMA_N256_TMEM  N = 256, A from tensor memory: the widest single-CTA
 *                       form.
 *
 * Memory: the probe allocates its own small output buffer for the duration of
 * the call.  Every call is synchronous.  Errors: a nonzero return is the
 * cudaError_t of the failing CUDA call; 1000 means a bad argument, 1001 that a
 * tensor-pipe probe's wait for its products ran out (no timing).
 */
#ifndef DOT_PROBE_H
#define DOT_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DOTP_API __attribute__((visibility("default")))
#else
#define DOTP_API
#endif

enum {
    DOTP_MUL_PAIR = 0,
    DOTP_COLSUM_R8 = 1,
    DOTP_MADWIDE_R8 = 2,
    DOTP_MUL_LO = 3,
    DOTP_EMPTY = 4,
    DOTP_MMA_N128_TMEM = 5,
    DOTP_MMA_N128_SMEM = 6,
    DOTP_MMA_N256_TMEM = 7
};

/* Run probe `kind` on the current device: `blocks` thread blocks of `threads`
 * threads (a multiple of 32, at most 1024), each thread `iters` loop steps;
 * one untimed launch, then `reps` launches timed with CUDA events.  *ms is the
 * mean time of one launch and *units the units (see above) one launch
 * performs. */
DOTP_API int dotp_run(int kind, int blocks, int threads, int iters, int reps, float *ms,
                      double *units);

/* SM count and the largest resident blocks per SM of probe `kind` at
 * `threads` threads per block, on the current device. */
DOTP_API int dotp_occupancy(int kind, int threads, int *sms, int *blocks_per_sm);

#ifdef __cplusplus
}
#endif

#endif /* DOT_PROBE_H */
