// dot_warp_op.cuh -- one whole add/sub per warp: the routine behind the
// ragged kernels, the mixed batch and the mpn-style variants (Alg. 1 with
// w = 32 lanes); see dot_addsub.cu for the method.
#pragma once

#include "dot_internal.cuh"

// One op of m limbs processed by one warp.  The warp walks it in groups of
// 4 x 32 limbs (loads first), resolving each 32-limb chunk with the ballot
// lookahead and passing the chunk carry-out on: Alg. 1's chunk loop with
// w = 32 lanes.  All 32 lanes must call it.  General form (mpn-style
// variants): b has mb <= m limbs and is zero beyond them -- past mb a carry
// propagates through limbs equal to 2^32 - 1 (a borrow through zeros) -- and
// cin in {0, 1} enters below limb 0; for m == 0 the carry-out is cin.
template <bool SUB>
__device__ __forceinline__ void addsub_warp_op(const uint32_t *a, const uint32_t *b, uint32_t *s,
                                               size_t m, uint32_t *cout, size_t mb, uint32_t cin0)
{
    constexpr int K = 4;
    const int lane = (int)lane_id();
    uint32_t cin = cin0;
    for (size_t c0 = 0; c0 < m; c0 += 32 * K) {
        uint32_t x[K][1], y[K][1];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const size_t li = c0 + (size_t)k * 32 + lane;
            x[k][0] = li < m ? ld_stream1(a + li) : 0u;
            y[k][0] = li < mb ? ld_stream1(b + li) : 0u;
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
                st_stream1(s + li, sg.r[0]);
                if (li == m - 1) *cout = sg.cout(c);
            }
            cin = wc.carry_out(31);
        }
    }
    if (m == 0 && lane == 0) *cout = cin0;
}
