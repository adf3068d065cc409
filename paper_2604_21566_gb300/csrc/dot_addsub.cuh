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
