// dot_addsub.cuh -- device building blocks of the carry-decoupled add/sub
// (Alg. 1 re-shaped for warps); see dot_addsub.cu for the method.
#pragma once

#include "dot_internal.cuh"

// --------------------------------------------------------------- loading
template <int SEG>
__device__ __forceinline__ void load_seg(const uint32_t *p, uint32_t (&v)[SEG])
{
    if constexpr (SEG == 4) {
        const uint4 q = ld_stream4(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
        for (int i = 0; i < SEG; ++i) v[i] = ld_stream1(p + i);
    }
}

template <int SEG>
__device__ __forceinline__ void store_seg(uint32_t *p, const uint32_t (&v)[SEG])
{
    if constexpr (SEG == 4) {
        st_stream4(p, make_uint4(v[0], v[1], v[2], v[3]));
    } else {
#pragma unroll
        for (int i = 0; i < SEG; ++i) st_stream1(p + i, v[i]);
    }
}

// One op of m limbs processed by one warp.  The warp walks it in groups of
// 4 x 32 limbs (loads first), resolving each 32-limb chunk with the ballot
// lookahead and passing the chunk carry-out on: Alg. 1's chunk loop with
// w = 32 lanes.  All 32 lanes must call it.
template <bool SUB>
__device__ __forceinline__ void addsub_warp_op(const uint32_t *a, const uint32_t *b, uint32_t *s,
                                               size_t m, uint32_t *cout)
{
    constexpr int K = 4;
    const int lane = (int)lane_id();
    uint32_t cin = 0;
    for (size_t c0 = 0; c0 < m; c0 += 32 * K) {
        uint32_t x[K][1], y[K][1];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const size_t li = c0 + (size_t)k * 32 + lane;
            if (li < m) {
                x[k][0] = ld_stream1(a + li);
                y[k][0] = ld_stream1(b + li);
            } else {
                x[k][0] = y[k][0] = 0;
            }
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
    if (m == 0 && lane == 0) *cout = 0;
}
