// dot_plan.h -- host-side choice of kernel and shape for one batched call.
// Pure integer logic (no CUDA calls), shared by the launchers and the
// exported dot_plan_batched().
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "dot.h"

enum {
    DOT_K_NONE = 0,
    DOT_K_ADDSUB_WARP = 1,   // whole ops inside one warp (runs of lanes)
    DOT_K_ADDSUB_TILE = 2,   // tiles of 256 threads chained by look-back
    DOT_K_MUL_COLSUM = 3,    // column-block sums + carry resolution
    DOT_K_MUL_THREAD = 4     // one product per thread, operands in registers
};
// largest operand (limbs) of the one-product-per-thread multiply
#define DOT_MUL_THREAD_MAX 16
// up to 32 limbs one product per thread too, when the batch gives every SM
// many threads (smaller batches spread an op over several lanes instead)
#define DOT_MUL_THREAD_WIDE_MAX 32
#define DOT_MUL_THREAD_WIDE_MIN_BATCH 16384

#define DOT_TILE_THREADS 256
#define DOT_WARP_MAX_CHUNKS 4

static inline size_t dot_ceil_div(size_t a, size_t b) { return (a + b - 1) / b; }

// Columns per thread block of the multiply for operand length m.
static inline int dot_mul_cols(size_t m, bool sqr = false)
{
    // Above 16 limbs: the R in {8, 12, 16} that leaves the fewest lane-steps
    // idle.  A warp holds floor(32 / T) ops of T = ceil(m / R) lanes; each lane
    // sums m' + R rows of R columns (m' = T R) for m^2 useful products per op.
    // (R = 4 scores as well at 32-64 limbs but measured slower: it reuses
    // each window value for only 4 products.)  A square sums its up to 1.5 R
    // near-diagonal rows per block one column at a time, which costs R = 16
    // too much: it takes 16 only above 384 limbs, where nothing else fits.
    if (m <= 16) return 4;
    int best = 8;
    double best_eff = -1.0;
    const int rs[3] = {8, 12, 16};
    for (int R : rs) {
        if (m > (size_t)32 * R || (sqr && R == 16 && m <= 384)) continue;
        const size_t T = (m + R - 1) / R, mp = T * R;
        const double eff = (double)(32 / T) * (double)m * (double)m / (32.0 * (double)(mp + R) * R);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = R;
        }
    }
    return best;
}

// Size bucket of the tuning table: the bit length of m (m in [2^(b-1), 2^b)).
#define DOT_TUNE_BUCKETS 65
static inline int dot_tune_bucket(size_t m)
{
    int b = 0;
    while (m) {
        ++b;
        m >>= 1;
    }
    return b;
}

// Whether `knob` is a shape the kernels implement for (op, m):
//   mul    -- R, the columns per block: 4, 8, 12 or 16 with m <= 32 R;
//   add/sub -- segments per thread of the tiled look-back kernel: 1, 2 or 4.
static inline bool dot_knob_valid(int op, size_t m, int knob)
{
    if (op == DOT_OP_MUL) return (knob == 4 || knob == 8 || knob == 12 || knob == 16) && m <= (size_t)32 * knob;
    return knob == 1 || knob == 2 || knob == 4;
}

// knob: a tuned shape (see dot_knob_valid), or 0 for the built-in choice.
static inline dot_status_t dot_make_plan(int op, size_t m, size_t batch, bool vec, dot_plan_t *pl, int knob = 0)
{
    pl->kernel = DOT_K_NONE;
    pl->seg_limbs = 1;
    pl->lanes_per_op = 0;
    pl->chunks = 0;
    pl->tile_limbs = 0;
    pl->tiles = 0;
    pl->m_pad = m;
    if (op != DOT_OP_ADD && op != DOT_OP_SUB && op != DOT_OP_MUL) return DOT_EINVAL;
    if (batch == 0) return DOT_OK;
    if (op == DOT_OP_MUL) {
        if (m == 0) return DOT_OK;
        if (m > DOT_MUL_MAX_LIMBS) return DOT_EUNSUPPORTED;
        const bool by_thread = m <= DOT_MUL_THREAD_MAX ||
                               (m <= DOT_MUL_THREAD_WIDE_MAX && batch >= DOT_MUL_THREAD_WIDE_MIN_BATCH);
        if (by_thread && !(knob && dot_knob_valid(op, m, knob))) {
            // small operands: one product per thread (a tuned column shape
            // selects the column-sum kernel instead)
            pl->kernel = DOT_K_MUL_THREAD;
            pl->seg_limbs = (int)m;
            pl->lanes_per_op = 1;
            pl->chunks = 1;
            return DOT_OK;
        }
        const int R = (knob && dot_knob_valid(op, m, knob)) ? knob : dot_mul_cols(m);
        pl->kernel = DOT_K_MUL_COLSUM;
        pl->seg_limbs = R;
        pl->m_pad = dot_ceil_div(m, (size_t)R) * R;
        pl->lanes_per_op = (int)(pl->m_pad / R);
        pl->chunks = 2;
        return DOT_OK;
    }
    if (m == 0) {
        // carries are 0; the warp kernel writes them
        pl->kernel = DOT_K_ADDSUB_WARP;
        pl->lanes_per_op = 1;
        pl->chunks = 1;
        return DOT_OK;
    }
    const int seg = vec ? 4 : 1;
    const size_t q = dot_ceil_div(m, (size_t)seg);   // segments per op
    pl->seg_limbs = seg;
    if (q <= 32u * DOT_WARP_MAX_CHUNKS) {
        pl->kernel = DOT_K_ADDSUB_WARP;
        if (q <= 32) {
            pl->lanes_per_op = (int)q;
            pl->chunks = 1;
        } else {
            pl->lanes_per_op = 32;
            pl->chunks = (int)dot_ceil_div(q, 32);
        }
        return DOT_OK;
    }
    pl->kernel = DOT_K_ADDSUB_TILE;
    pl->lanes_per_op = DOT_TILE_THREADS;
    // segments per thread: 4 for long operands, fewer for short ones
    const size_t per4 = (size_t)DOT_TILE_THREADS * seg * 4;
    pl->chunks = (knob && dot_knob_valid(op, m, knob)) ? knob : (m >= per4 ? 4 : (m >= per4 / 2 ? 2 : 1));
    pl->tile_limbs = (uint64_t)DOT_TILE_THREADS * seg * pl->chunks;
    pl->tiles = dot_ceil_div(m, (size_t)pl->tile_limbs);
    return DOT_OK;
}
