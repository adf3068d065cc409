// dot_warp_op.cuh -- one whole add/sub per warp: the routine behind the
// ragged kernels, the mixed batch and the mpn-style variants (Alg. 1 with
// w = 32 lanes); see dot_addsub.cu for the method.
#pragma once

#include "dot_internal.cuh"

// One op of m limbs processed by one warp.  The warp walks it in groups of
// 4 x 32 limbs (loads first), resolving each 32-limb chunk with the ballot
// lookahead and passing the chunk carry-out on: Alg. 1's chunk loop with
// w = 32 lanes.  All 32 lanes must call it.  Operand limbs come from la(i) and
// lb(i) (i < m; a shorter operand returns 0 past its end: a carry then
// propagates through limbs equal to 2^32 - 1, a borrow through zeros), result
// limbs go to st(i, v), and cin in {0, 1} enters below limb 0.  Returns the
// carry (borrow) out of limb m - 1 to every lane; cin when m == 0.
template <bool SUB, typename LA, typename LB, typename ST>
__device__ __forceinline__ uint32_t addsub_warp_run(LA la, LB lb, ST st, size_t m, uint32_t cin0)
{
    constexpr int K = 4;
    const int lane = (int)lane_id();
    uint32_t cin = cin0, fin = 0;
    for (size_t c0 = 0; c0 < m; c0 += 32 * K) {
        uint32_t x[K][1], y[K][1];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const size_t li = c0 + (size_t)k * 32 + lane;
            x[k][0] = li < m ? la(li) : 0u;
            y[k][0] = li < m ? lb(li) : 0u;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const size_t li = c0 + (size_t)k * 32 + lane;
            Segment<SUB, 1> sg;
            sg.phase12(x[k], y[k]);
            const bool on = li < m;
            WarpCarry wc;
            wc.resolve(on ? sg.g() : 0u, on ? sg.p() : 0u, lane == 0 ? cin : 0u, 1u, 0x80000000u);
            const uint32_t c = wc.carry_in(lane);
            sg.apply(c);
            if (on) {
                st(li, sg.r[0]);
                if (li == m - 1) fin = sg.cout(c);
            }
            cin = wc.carry_out(31);
        }
    }
    return m ? __shfl_sync(DOT_FULL, fin, (int)((m - 1) & 31)) : cin0;
}

// The same on rows in memory: a (m limbs), b (mb <= m limbs, zero beyond), s;
// the carry (borrow) out goes to *cout.
template <bool SUB>
__device__ __forceinline__ void addsub_warp_op(const uint32_t *a, const uint32_t *b, uint32_t *s,
                                               size_t m, uint32_t *cout, size_t mb, uint32_t cin0)
{
    const uint32_t c = addsub_warp_run<SUB>([=](size_t i) { return ld_stream1(a + i); },
                                            [=](size_t i) { return i < mb ? ld_stream1(b + i) : 0u; },
                                            [=](size_t i, uint32_t v) { st_stream1(s + i, v); }, m, cin0);
    if (lane_id() == 0) *cout = c;
}
