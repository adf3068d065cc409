// dot_probe.cu -- microbenchmarks behind the integer-pipe rooflines of the
// column-sum multiply (see include/dot_probe.h).  Each kernel repeats one
// instruction pattern in independent chains with no memory access in its
// loop; every value feeds a later step or the final store, so nothing can be
// hoisted or removed, and no chain can be rewritten into fewer multiplies
// (each step multiplies two different, freshly computed values).
#include <cuda_runtime.h>
#include <stdint.h>

#include "dot_probe.h"
#include "dot_mul.cuh"   // mac_cols: the multiply's own product step

#define PROBE_CHAINS 8
#define PROBE_R 8

// mul.lo + mul.hi of the same operands, the pair one limb product costs
__global__ void probe_mul_pair(uint32_t seed, int iters, uint32_t *out)
{
    uint32_t x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = seed ^ (threadIdx.x * 0x9E3779B9u + k * 0x85EBCA6Bu + blockIdx.x);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) {
            uint32_t lo, hi;
            asm("mul.lo.u32 %0, %2, %3;\n\tmul.hi.u32 %1, %2, %3;"
                : "=r"(lo), "=r"(hi) : "r"(x[k]), "r"(x[(k + 1) % PROBE_CHAINS]));
            x[k] = lo ^ hi;
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) r ^= x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// mul.lo alone
__global__ void probe_mul_lo(uint32_t seed, int iters, uint32_t *out)
{
    uint32_t x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = seed ^ (threadIdx.x * 0x9E3779B9u + k * 0x85EBCA6Bu + blockIdx.x);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k)
            asm("mul.lo.u32 %0, %0, %1;" : "+r"(x[k]) : "r"(x[(k + 1) % PROBE_CHAINS]));
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) r ^= x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// The column-sum step of the multiply: R columns of three-word sums, a
// window of the second operand sliding down by one per row (as in
// colsum_pair, but the new window value and the row's first operand come
// from registers instead of shared memory).
__global__ void probe_colsum(uint32_t seed, int iters, uint32_t *out)
{
    uint32_t s0[PROBE_R], s1[PROBE_R], s2[PROBE_R], w[PROBE_R];
#pragma unroll
    for (int k = 0; k < PROBE_R; ++k) {
        s0[k] = s1[k] = s2[k] = 0;
        w[k] = seed ^ (threadIdx.x * 0x9E3779B9u + k * 0x85EBCA6Bu + blockIdx.x);
    }
    uint32_t a = seed + threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int ii = 0; ii < PROBE_R; ++ii) {
            mac_cols<PROBE_R>(s0, s1, s2, a, w);
            a = w[PROBE_R - 1];
#pragma unroll
            for (int k = PROBE_R - 1; k > 0; --k) w[k] = w[k - 1];
            w[0] = s0[ii];
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < PROBE_R; ++k) r ^= s0[k] ^ s1[k] ^ s2[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// The same step with one 32 x 32 -> 64-bit multiply-add into a 64-bit column
// sum per product (digits small enough that the sum needs no carry chain).
__global__ void probe_madwide(uint32_t seed, int iters, uint32_t *out)
{
    uint64_t s[PROBE_R];
    uint32_t w[PROBE_R];
#pragma unroll
    for (int k = 0; k < PROBE_R; ++k) {
        s[k] = 0;
        w[k] = seed ^ (threadIdx.x * 0x9E3779B9u + k * 0x85EBCA6Bu + blockIdx.x);
    }
    uint32_t a = seed + threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int ii = 0; ii < PROBE_R; ++ii) {
#pragma unroll
            for (int k = 0; k < PROBE_R; ++k)
                asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(s[k]) : "r"(a), "r"(w[k]));
            a = w[PROBE_R - 1];
#pragma unroll
            for (int k = PROBE_R - 1; k > 0; --k) w[k] = w[k - 1];
            w[0] = (uint32_t)s[ii];
        }
    }
    uint64_t r = 0;
#pragma unroll
    for (int k = 0; k < PROBE_R; ++k) r ^= s[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (uint32_t)(r ^ (r >> 32));
}

__global__ void probe_empty() {}

// ------------------------------------------------------------ tensor pipe
// One thread per CTA issues iters x 4 tcgen05.mma of M = 128, N, K = 16 (fp16
// in, fp32 accumulate) into one tensor-memory accumulator, A from shared or
// tensor memory, B from shared memory (128-byte swizzled, K-major, ones and
// zeros), then commits and waits (bounded) for them.  One CTA per SM (it
// takes all 512 tensor-memory columns).  out[block] = 1 if the wait ran out.
#define PROBE_MMA_SMEM (16384 + 32768 + 1024 + 64)

__device__ __forceinline__ uint32_t probe_su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t probe_desc_sw128(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

template <int N, bool ATM>
__global__ void __launch_bounds__(1024, 1) probe_mma(int iters, uint32_t *out)
{
    extern __shared__ __align__(1024) unsigned char probe_sm[];
    unsigned char *base = probe_sm + ((1024u - (probe_su32(probe_sm) & 1023u)) & 1023u);
    unsigned char *sA = base, *sB = base + 16384;   // A: 128 x 64 fp16, B: 256 x 64 fp16
    uint64_t *bar = (uint64_t *)(base + 49152);
    uint32_t *slot = (uint32_t *)(bar + 1);
    for (int i = threadIdx.x; i < 49152 / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(base)[i] = make_uint4(0x3C003C00u, 0u, 0u, 0u);
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" :: "r"(probe_su32(slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(probe_su32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    if (threadIdx.x == 0) {
        // D fp32, A and B fp16, K-major, M = 128, N
        const uint32_t idesc = (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        const uint64_t ad = probe_desc_sw128(probe_su32(sA)), bd = probe_desc_sw128(probe_su32(sB));
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int st = 0; st < 4; ++st) {
                const uint64_t b = bd + (uint64_t)((st * 32) >> 4);
                if (ATM)
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
                                 :: "r"(tmem), "r"(tmem + 256 + 8 * st), "l"(b), "r"(idesc), "r"(1) : "memory");
                else
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                                 :: "r"(tmem), "l"(ad + (uint64_t)((st * 32) >> 4)), "l"(b), "r"(idesc), "r"(1)
                                 : "memory");
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :: "r"(probe_su32(bar)) : "memory");
        uint32_t done = 0;
        for (long k = 0; k < (1L << 28) && !done; ++k)
            asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(done) : "r"(probe_su32(bar)) : "memory");
        out[blockIdx.x] = done ? 0u : 1u;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(tmem) : "memory");
}

static bool probe_is_mma(int kind) { return kind >= DOTP_MMA_N128_TMEM && kind <= DOTP_MMA_N256_TMEM; }
static int probe_mma_n(int kind) { return kind == DOTP_MMA_N256_TMEM ? 256 : 128; }

static const void *probe_fn(int kind)
{
    switch (kind) {
    case DOTP_MUL_PAIR: return (const void *)probe_mul_pair;
    case DOTP_COLSUM_R8: return (const void *)probe_colsum;
    case DOTP_MADWIDE_R8: return (const void *)probe_madwide;
    case DOTP_MUL_LO: return (const void *)probe_mul_lo;
    case DOTP_EMPTY: return (const void *)probe_empty;
    case DOTP_MMA_N128_TMEM: return (const void *)probe_mma<128, true>;
    case DOTP_MMA_N128_SMEM: return (const void *)probe_mma<128, false>;
    case DOTP_MMA_N256_TMEM: return (const void *)probe_mma<256, true>;
    }
    return nullptr;
}

static cudaError_t probe_launch(int kind, int blocks, int threads, int iters, uint32_t *out, cudaStream_t st)
{
    const uint32_t seed = 0x2545F491u;
    switch (kind) {
    case DOTP_MUL_PAIR: probe_mul_pair<<<blocks, threads, 0, st>>>(seed, iters, out); break;
    case DOTP_COLSUM_R8: probe_colsum<<<blocks, threads, 0, st>>>(seed, iters, out); break;
    case DOTP_MADWIDE_R8: probe_madwide<<<blocks, threads, 0, st>>>(seed, iters, out); break;
    case DOTP_MUL_LO: probe_mul_lo<<<blocks, threads, 0, st>>>(seed, iters, out); break;
    case DOTP_MMA_N128_TMEM: probe_mma<128, true><<<blocks, threads, PROBE_MMA_SMEM, st>>>(iters, out); break;
    case DOTP_MMA_N128_SMEM: probe_mma<128, false><<<blocks, threads, PROBE_MMA_SMEM, st>>>(iters, out); break;
    case DOTP_MMA_N256_TMEM: probe_mma<256, true><<<blocks, threads, PROBE_MMA_SMEM, st>>>(iters, out); break;
    default: probe_empty<<<blocks, threads, 0, st>>>(); break;
    }
    return cudaGetLastError();
}

extern "C" {

DOTP_API int dotp_occupancy(int kind, int threads, int *sms, int *blocks_per_sm)
{
    const void *fn = probe_fn(kind);
    if (!fn || !sms || !blocks_per_sm || threads < 32 || threads > 1024 || threads % 32) return 1000;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && probe_is_mma(kind)) *blocks_per_sm = 1;   // all of tensor memory per CTA
    else if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, threads, 0);
    return (int)e;
}

DOTP_API int dotp_run(int kind, int blocks, int threads, int iters, int reps, float *ms, double *units)
{
    if (!probe_fn(kind) || !ms || !units || blocks < 1 || threads < 32 || threads > 1024 || threads % 32 ||
        iters < 1 || reps < 1)
        return 1000;
    const double per_thread = kind == DOTP_MUL_PAIR || kind == DOTP_MUL_LO ? (double)iters * PROBE_CHAINS
                            : kind == DOTP_EMPTY ? 0.0
                                                 : (double)iters * PROBE_R * PROBE_R;
    *units = kind == DOTP_EMPTY ? 1.0
           : probe_is_mma(kind) ? 2.0 * 128 * probe_mma_n(kind) * 16 * 4 * (double)iters * blocks
                                : per_thread * blocks * threads;
    if (probe_is_mma(kind) &&
        cudaFuncSetAttribute(probe_fn(kind), cudaFuncAttributeMaxDynamicSharedMemorySize, PROBE_MMA_SMEM) !=
            cudaSuccess)
        return (int)cudaGetLastError();
    uint32_t *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void **)&out, (size_t)blocks * threads * 4);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = probe_launch(kind, blocks, threads, iters, out, st);   // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = probe_launch(kind, blocks, threads, iters, out, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    *ms = t / (float)reps;
    if (st) cudaStreamSynchronize(st);
    if (e == cudaSuccess && probe_is_mma(kind)) {   // a wait that ran out voids the timing
        uint32_t flags[1024];
        for (int b0 = 0; b0 < blocks && e == cudaSuccess; b0 += 1024) {
            const int nb = blocks - b0 < 1024 ? blocks - b0 : 1024;
            e = cudaMemcpy(flags, out + b0, (size_t)nb * 4, cudaMemcpyDeviceToHost);
            for (int k = 0; k < nb && e == cudaSuccess; ++k)
                if (flags[k]) {
                    if (st) cudaStreamDestroy(st);
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    cudaFree(out);
                    return 1001;
                }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    return (int)e;
}

}  // extern "C"
