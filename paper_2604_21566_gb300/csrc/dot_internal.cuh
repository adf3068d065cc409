// dot_internal.cuh -- shared device primitives and the context layout of libdot.
//
// Carry handling follows DoT's addition (Alg. 1, Sec. 3.1): Phase 1 adds the
// limbs independently, Phase 2 derives per-limb generate bits (r < a, the
// carry lemma of the appendix) and propagate bits (r == 2^32-1), and
// Phases 3-4 resolve the carries with the Kogge-Stone mask trick
//     carries = ((G << 1 | c_in) + P) ^ P,
// an integer add on bitmasks whose carry chain runs exactly through the
// propagating positions.  The same identity is used at three levels: limbs
// inside a thread's segment, segments across the 32 lanes of a warp (masks
// from __ballot_sync), and tiles across thread blocks (decoupled look-back).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "dot.h"

#define DOT_FULL 0xffffffffu

// ------------------------------------------------------------------ context
struct dot_ctx {
    int device;
    int num_sms;
    // sticky device status (DOT_OK or an error code), cleared by dot_ctx_check
    uint32_t *d_status;
    // look-back scratch: [0] tile ticket, [1] blocks done, [2..3] 64-bit epoch
    unsigned long long *d_counters;
    // per-tile look-back states, (epoch << 2) | code
    unsigned long long *d_tile_state;
    size_t tile_state_cap;
    uint64_t wait_limit_ns;
    int64_t debug_skip_tile;
    // staging for the host-buffer entry points
    void *d_stage;
    size_t stage_bytes;
    cudaStream_t side[2];   // [0] copies in, [1] copies out
    // per staging buffer: [0,1] inputs copied in, [2,3] kernel done, [4,5]
    // results copied out; [6] call start, [7] copies out finished
    cudaEvent_t ev[8];
    // mixed-batch scratch and captured graph (dot_mixed.cu), created on first use
    void *mixed;
    // tuned shape per (op, bit length of m); 0 = built-in choice (dot_tune.cu)
    unsigned char tune[3][65];
    // general workspace (Karatsuba levels), grown on demand by dot_work
    void *d_work;
    size_t work_bytes;
};

// A device workspace of at least `bytes` (256-byte aligned) owned by the ctx;
// growing it synchronises the device.  Calls that use it on one ctx must not
// overlap on the GPU.
dot_status_t dot_work(dot_ctx_t ctx, size_t bytes, void **out);

void dot_mixed_release(dot_ctx_t ctx);

// look-back tile state codes (low two bits of a state word)
enum { LB_EMPTY = 0, LB_PROP = 1, LB_INCL0 = 2, LB_INCL1 = 3 };

struct LookbackArgs {
    unsigned long long *state;      // one word per tile (ticket order)
    unsigned long long *counters;   // ticket, done, epoch
    uint32_t *status;
    uint64_t wait_limit_ns;
    long long skip_tile;            // debug hook: tile of op 0 that never publishes, or -1
};

// -------------------------------------------------------------- small utils
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void record_status(uint32_t *status, uint32_t code)
{
    if (status) atomicCAS(status, (uint32_t)DOT_OK, code);
}

// ------------------------------------------- mbarrier + bulk async copies
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(bar)), "r"(count) : "memory");
}

// make barrier initialisation visible to the async (copy / tensor) proxy
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One bulk copy global -> shared (16-byte aligned, size a multiple of 16),
// completing `bytes` of transaction count on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return done != 0;
}

// Wait for phase `parity` of `bar`, at most limit_ns; false if it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// streaming loads/stores: each byte is touched once
__device__ __forceinline__ uint4 ld_stream4(const uint32_t *p)
{
    return __ldcs(reinterpret_cast<const uint4 *>(p));
}
__device__ __forceinline__ uint32_t ld_stream1(const uint32_t *p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream4(uint32_t *p, uint4 v)
{
    __stcs(reinterpret_cast<uint4 *>(p), v);
}
__device__ __forceinline__ void st_stream1(uint32_t *p, uint32_t v) { __stcs(p, v); }

// --------------------------------------------------------- segment phases
// One thread's segment of SEG consecutive limbs.  Phase 1 forms r_i = a_i +- b_i
// (mod 2^32) independently; Phase 2 records the generate bit g_i and the
// propagate bit p_i of each limb in the masks gm, pm:
//   add: g_i = [r_i < a_i],  p_i = [r_i == 2^32-1]
//   sub: g_i = [a_i < b_i],  p_i = [a_i == b_i]   (borrows instead of carries)
template <bool SUB, int SEG>
struct Segment {
    uint32_t r[SEG];
    uint32_t gm, pm;

    __device__ __forceinline__ void phase12(const uint32_t (&x)[SEG], const uint32_t (&y)[SEG])
    {
        gm = 0;
        pm = 0;
#pragma unroll
        for (int i = 0; i < SEG; ++i) {
            if (!SUB) {
                r[i] = x[i] + y[i];
                gm |= (uint32_t)(r[i] < x[i]) << i;
                pm |= (uint32_t)(r[i] == DOT_FULL) << i;
            } else {
                r[i] = x[i] - y[i];
                gm |= (uint32_t)(x[i] < y[i]) << i;
                pm |= (uint32_t)(x[i] == y[i]) << i;
            }
        }
    }
    // segment generate: carry out of the segment with carry-in 0
    __device__ __forceinline__ uint32_t g() const { return (((gm << 1) + pm) >> SEG) & 1u; }
    // segment propagate: every limb propagates
    __device__ __forceinline__ uint32_t p() const
    {
        return pm == (SEG == 32 ? DOT_FULL : ((1u << SEG) - 1u));
    }
    // Phases 3-4: add the resolved carry into each limb.  cin is the carry
    // into limb 0; the mask trick gives the carry into every limb at once.
    __device__ __forceinline__ void apply(uint32_t cin)
    {
        const uint32_t cm = (((gm << 1) | cin) + pm) ^ pm;
#pragma unroll
        for (int i = 0; i < SEG; ++i) {
            const uint32_t c = (cm >> i) & 1u;
            r[i] = SUB ? r[i] - c : r[i] + c;
        }
    }
    // carry out of the segment for carry-in cin
    __device__ __forceinline__ uint32_t cout(uint32_t cin) const
    {
        return ((((gm << 1) | cin) + pm) >> SEG) & 1u;
    }
};

// ---------------------------------------------------- warp carry-lookahead
// Lanes are grouped in runs of `lpo` consecutive lanes (runs start at the
// bits of start_mask; top_mask marks each run's last lane).  Lane l supplies
// its segment's (g, p); lanes of a run form one carry chain, with carry-in
// `run_cin` taken from the run's first lane.  Returns the mask of carries
// INTO each lane's segment (bit l).  No carry crosses from one run into the
// next: the generate bit of a run's top lane and its propagate bit are
// masked, and a run's carry-out is computed by run_carry_out().
struct WarpCarry {
    uint32_t G, P, C;

    __device__ __forceinline__ void resolve(uint32_t g, uint32_t p, uint32_t run_cin,
                                            uint32_t start_mask, uint32_t top_mask)
    {
        G = __ballot_sync(DOT_FULL, g);
        P = __ballot_sync(DOT_FULL, p);
        const uint32_t CI = __ballot_sync(DOT_FULL, run_cin) & start_mask;
        const uint32_t X = ((G << 1) & ~start_mask) | CI;
        const uint32_t Pm = P & ~top_mask;
        C = (X + Pm) ^ Pm;
    }
    __device__ __forceinline__ uint32_t carry_in(int lane) const { return (C >> lane) & 1u; }
    // carry out of the segment held by lane L
    __device__ __forceinline__ uint32_t carry_out(int L) const
    {
        return ((G >> L) | ((P >> L) & (C >> L))) & 1u;
    }
};

// run masks for runs of lpo lanes (lpo <= 32): start bits at 0, lpo, 2 lpo, ...
__host__ __device__ inline uint32_t run_start_mask(int lpo)
{
    uint32_t m = 0;
    for (int k = 0; k + lpo <= 32; k += lpo) m |= 1u << k;
    return m;
}
__host__ __device__ inline uint32_t run_top_mask(int lpo)
{
    uint32_t m = 0;
    for (int k = 0; k + lpo <= 32; k += lpo) m |= 1u << (k + lpo - 1);
    return m;
}

// composition of carry states: segment (g_hi, p_hi) above (g_lo, p_lo)
__device__ __forceinline__ void gp_compose(uint32_t &g, uint32_t &p, uint32_t g_hi, uint32_t p_hi)
{
    g = g_hi | (p_hi & g);
    p = p_hi & p;
}

// ------------------------------------------------------------ host helpers
// Makes a CUDA device current for the lifetime of the object and puts the
// caller's device back when it goes out of scope, so that no entry point
// leaves the calling thread on another device.  Kernels launched meanwhile
// keep running on the device they were launched on.
class DeviceScope {
  public:
    DeviceScope() = default;
    DeviceScope(const DeviceScope &) = delete;
    DeviceScope &operator=(const DeviceScope &) = delete;
    ~DeviceScope()
    {
        if (prev_ >= 0) cudaSetDevice(prev_);
    }
    dot_status_t enter(int device)
    {
        int cur = -1;
        if (cudaGetDevice(&cur) != cudaSuccess) return DOT_ECUDA;
        if (cur == device) return DOT_OK;
        if (cudaSetDevice(device) != cudaSuccess) return DOT_ECUDA;
        if (prev_ < 0) prev_ = cur;
        return DOT_OK;
    }

  private:
    int prev_ = -1;   // device to restore, or -1 when nothing was switched
};

dot_status_t dot_lookback_prepare(dot_ctx_t ctx, size_t tiles, LookbackArgs *out);
// validates ctx and makes its device current for the lifetime of `scope`
dot_status_t dot_check_ctx(dot_ctx_t ctx, DeviceScope &scope);
int dot_blocks_per_sm(const void *kernel, int threads, size_t smem);

// ranges [p, p + n) overlap partially (not identical, not disjoint)
static inline bool partial_overlap(const void *x, size_t xn, const void *y, size_t yn)
{
    const uintptr_t a = (uintptr_t)x, b = (uintptr_t)y;
    if (!xn || !yn) return false;
    if (a == b) return false;
    return a < b + yn && b < a + xn;
}
static inline bool any_overlap(const void *x, size_t xn, const void *y, size_t yn)
{
    const uintptr_t a = (uintptr_t)x, b = (uintptr_t)y;
    if (!xn || !yn) return false;
    return a < b + yn && b < a + xn;
}
__host__ __device__ inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }
