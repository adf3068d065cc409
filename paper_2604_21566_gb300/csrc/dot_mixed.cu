// dot_mixed.cu -- mixed ragged batches of add / sub / mul descriptors.
//
// The paper runs one operation at a time on one core.  Here a batch of many
// operations of uneven sizes goes through one pass on the device:
//   1. classify: each descriptor gets a size bucket (by op and limb count);
//      per-block histograms, one atomic per bucket per block for its slot;
//   2. plan: one warp turns the bucket counts into offsets and work-item
//      ranges (and clears the counts for the next call);
//   3. scatter: op indices are written bucket by bucket;
//   4. add/sub: the additions and subtractions (Alg. 1), one warp per op
//      above 128 limbs and four ops per warp below, 32 warps per SM so that
//      enough of them have loads in flight (as one item each behind the
//      products, claimed one at a time, they ran at a seventh of the memory
//      bandwidth);
//   5. run: two persistent kernels for the products, one for the
//      257..512-limb buckets and one for the rest (so that the smaller
//      shapes are not held to the registers, and the occupancy, of the
//      largest); each warp takes work items from its kernel's counter,
//      heaviest buckets first (longest-processing-time order), and runs the
//      multiply (column-block sums, Alg. 2) for the item's ops.  Small
//      multiplies share a warp: a bucket fixes the run width T, and each op
//      of the item takes a run of T lanes.  A bucket also fixes the columns
//      per lane R, chosen so that an op's ceil(m / R) lanes fill most of its
//      run: above 256 limbs one bucket per 32 limbs, R = ceil(m / 32) = 9..16,
//      so that 29 to 32 of the 32 lanes work; 129..256 limbs take R = 6, 7
//      or 8.  A warp's time for one op goes as (ceil(m / R) + 1) R^2, so a
//      wider R than the op needs costs as much as idle lanes: with R = 16
//      and 12 for 257..512 limbs and R = 8 for 129..256, the 200k-op batch
//      of the benchmark took 7% longer.
// The six launches are captured once into a CUDA graph per context (the
// add/sub kernel and the smaller products on one branch, the largest
// products on another); later calls only update the graph's kernel-node
// parameters and replay it.
#include <stdlib.h>
#include <string.h>

#include "dot_internal.cuh"
#include "dot_plan.h"
#include "dot_addsub.cuh"
#include "dot_warp_op.cuh"
#include "dot_mul.cuh"

// bucket ids, in processing order (heaviest first): BK_R<R> runs one
// multiply per warp with R columns per lane; BK_M8B / BK_M8A / BK_M4 run 2 /
// 4 / 8 multiplies per warp; BK_ASL / BK_ASS are the add/sub ops
enum {
    BK_R16 = 0, BK_R15, BK_R14, BK_R13, BK_R12, BK_R11, BK_R10, BK_R9,   // 257..512 limbs
    BK_R8, BK_R7, BK_R6,                                                  // 129..256 limbs
    BK_M8B, BK_M8A, BK_M4, BK_ASL, BK_ASS, NBK
};
static_assert(NBK <= 16, "a slot keeps the bucket id in its top 4 bits");
#define MIX_WARPS 4
__host__ __device__ constexpr int cmax(int x, int y) { return x > y ? x : y; }
#define MIX_MAX_OPS (1ull << 28)

struct MixedMeta {
    uint32_t count[NBK];   // filled by classify, cleared by plan
    uint32_t n[NBK];       // ops per bucket
    uint32_t base[NBK];    // first slot of each bucket in `order`
    uint32_t item_base[NBK + 1];
    uint32_t pad;
    unsigned long long next_item[2];   // work counters of the two product kernels
    unsigned long long done[2];
};

struct MixedScratch {
    uint32_t *slot;
    uint32_t *order;
    MixedMeta *meta;
    size_t cap;
    cudaGraphExec_t exec;
    cudaGraph_t graph;
    cudaGraphNode_t node[6];
    int persist_blocks, narrow_blocks;
    int as_blocks;
    cudaEvent_t fork, join;
};

__host__ __device__ inline int bucket_ops_per_item(int bk)
{
    switch (bk) {
    case BK_M8B: return 2;
    case BK_M8A: return 4;
    case BK_M4: return 8;
    default: return 1;
    }
}

// bucket of one descriptor; -1: nothing to run (m == 0), -2: bad op, -3: mul too long
__device__ __forceinline__ int bucket_of(uint32_t op, uint32_t m)
{
    if (op > DOT_OP_MUL) return -2;
    if (m == 0) return -1;
    if (op != DOT_OP_MUL) return m > 128 ? BK_ASL : BK_ASS;
    if (m > DOT_MUL_MAX_LIMBS) return -3;
    if (m > 256) return BK_R16 + (16 - (int)((m + 31) / 32));   // R = ceil(m / 32): ceil(m / R) <= 32
    if (m > 224) return BK_R8;
    if (m > 192) return BK_R7;
    if (m > 128) return BK_R6;
    if (m > 64) return BK_M8B;
    if (m > 16) return BK_M8A;
    return BK_M4;
}

__global__ void __launch_bounds__(256)
mixed_classify(const dot_desc_t *desc, size_t nops, uint32_t *slot, MixedMeta *meta, uint32_t *carry,
               uint32_t *status)
{
    __shared__ uint32_t s_cnt[NBK], s_base[NBK];
    if (threadIdx.x < NBK) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    int bk = -1;
    uint32_t rank = 0;
    if (i < nops) {
        const uint32_t op = desc[i].op, m = desc[i].m;
        bk = bucket_of(op, m);
        if (bk < 0) {
            carry[i] = 0;
            if (bk == -2) record_status(status, DOT_EINVAL);
            if (bk == -3) record_status(status, DOT_EUNSUPPORTED);
        } else {
            rank = atomicAdd(&s_cnt[bk], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x < NBK)
        s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(&meta->count[threadIdx.x], s_cnt[threadIdx.x]) : 0u;
    __syncthreads();
    if (i < nops) slot[i] = bk >= 0 ? (((uint32_t)bk << 28) | (s_base[bk] + rank)) : 0xffffffffu;
}

__global__ void mixed_plan(MixedMeta *meta)
{
    if (threadIdx.x == 0) {
        uint32_t base = 0, items = 0;
        for (int b = 0; b < NBK; ++b) {
            const uint32_t c = meta->count[b];
            meta->n[b] = c;
            meta->base[b] = base;
            meta->item_base[b] = items;
            base += c;
            items += (c + bucket_ops_per_item(b) - 1) / bucket_ops_per_item(b);
            meta->count[b] = 0;
        }
        meta->item_base[NBK] = items;
    }
}

__global__ void __launch_bounds__(256)
mixed_scatter(const uint32_t *slot, size_t nops, const MixedMeta *meta, uint32_t *order)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nops) return;
    const uint32_t s = slot[i];
    if (s == 0xffffffffu) return;
    order[meta->base[s >> 28] + (s & 0x0fffffffu)] = (uint32_t)i;
}

// staging words one warp needs for shape (R, T): 32 / T ops, each with its A
// row, its B row and the B pads
__host__ __device__ constexpr int mix_region_words(int R, int T) { return (32 / T) * (2 * T * R + 2 * R); }

// the ops of one multiply work item: run grp of the warp takes op k0 + grp;
// RW: the staging words the caller gives each warp
template <int R, int T, int RW>
__device__ __forceinline__ void mixed_mul_item(const dot_desc_t *desc, const uint32_t *order, uint32_t base,
                                               uint32_t n, uint32_t k0, const uint32_t *a, const uint32_t *b,
                                               uint32_t *r, uint32_t *carry, uint32_t *wsmem)
{
    constexpr int REGION = 2 * T * R + 2 * R;
    static_assert(mix_region_words(R, T) <= RW, "staging region");
    const int lane = (int)lane_id();
    const int grp = lane / T, t = lane - grp * T;
    const uint32_t idx = k0 + grp;
    const bool valid = idx < n;
    uint32_t op = 0, m = 0;
    uint64_t ao = 0, bo = 0, ro = 0;
    if (valid) {
        op = order[base + idx];
        const dot_desc_t d = desc[op];
        m = d.m;
        ao = d.a_off;
        bo = d.b_off;
        ro = d.r_off;
    }
    const int tn = (int)((m + R - 1) / R);
    const int mp = tn * R;
    uint32_t *As = wsmem + grp * REGION;
    uint32_t *Bs = As + mp;
    if (valid) {
        const bool va = ((ao & 3) == 0) && aligned16(a);
        const bool vb = ((bo & 3) == 0) && aligned16(b);
        if (t < tn) {
            stage_row<R>(a + ao, As, t, (int)m, va);
            stage_row<R>(b + bo, Bs + R, t, (int)m, vb);
        }
        for (int k = t; k < R; k += T) {
            Bs[k] = 0;
            Bs[R + mp + k] = 0;
        }
    }
    __syncwarp();
    const bool vec_out = ((ro & 3) == 0) && aligned16(r);
    mul_group<R>(As, Bs, t, T, tn, grp, valid, (int)m, mp, r + ro, vec_out, run_start_mask(T),
                 run_top_mask(T));
    if (valid && t == 0) carry[op] = 0;
    __syncwarp();
}

#define MIX_AS_THREADS 256
#define MIX_AS_BLOCKS_PER_SM 8

// Four limbs of one lane for an add (sub false) or a subtract (sub true),
// the op chosen at run time: the short-op path packs adds and subtracts into
// one warp.  Same phases as Segment<SUB, 4> (dot_internal.cuh).
struct SegAS {
    uint32_t r[4];
    uint32_t gm, pm;
    __device__ __forceinline__ void phase12(const uint32_t (&x)[4], const uint32_t (&y)[4], bool sub)
    {
        gm = 0;
        pm = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            r[i] = sub ? x[i] - y[i] : x[i] + y[i];
            gm |= (uint32_t)(sub ? x[i] < y[i] : r[i] < x[i]) << i;
            pm |= (uint32_t)(sub ? x[i] == y[i] : r[i] == DOT_FULL) << i;
        }
    }
    __device__ __forceinline__ uint32_t g() const { return (((gm << 1) + pm) >> 4) & 1u; }
    __device__ __forceinline__ uint32_t p() const { return pm == 0xfu; }
    // carry (borrow) into limb j of the four, 0 <= j <= 4, for carry-in cin
    // (bit j of the carry mask that apply() uses)
    __device__ __forceinline__ uint32_t carry_at(uint32_t cin, int j) const
    {
        return (((((gm << 1) | cin) + pm) ^ pm) >> j) & 1u;
    }
    __device__ __forceinline__ void apply(uint32_t cin, bool sub)
    {
        const uint32_t cm = (((gm << 1) | cin) + pm) ^ pm;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t c = (cm >> i) & 1u;
            r[i] = sub ? r[i] - c : r[i] + c;
        }
    }
};

// Add/sub ops of at most 128 limbs, four per warp: run g = lane / 8 takes
// op 4 i + g of the short bucket, and lane t = lane % 8 of the run holds limbs
// 32 k + 4 t .. 32 k + 4 t + 3 of its chunk k < 4, so one chunk of 32 limbs is
// one run of the warp's ballot lookahead and all of an op's loads are in
// flight at once (one op per warp left most lanes idle: these ops average
// about 36 limbs).  Limbs past m read as 0 and are not stored; the carry
// (borrow) out of limb m - 1 is read off the lane that holds it.
__device__ __forceinline__ void mixed_addsub_short(const dot_desc_t *desc, const uint32_t *order, uint32_t base,
                                                   uint32_t n, size_t item, const uint32_t *a, const uint32_t *b,
                                                   uint32_t *r, uint32_t *carry)
{
    const int lane = (int)lane_id();
    const int grp = lane >> 3, t = lane & 7;
    const size_t idx = item * 4 + (size_t)grp;
    const bool valid = idx < n;
    uint32_t op = 0;
    dot_desc_t d{};
    if (valid) {
        op = order[base + idx];
        d = desc[op];
    }
    const uint32_t m = valid ? d.m : 0u;
    const bool sub = d.op == DOT_OP_SUB;
    const uint32_t *ar = a + d.a_off, *br = b + d.b_off;
    uint32_t x[4][4], y[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t li = 32u * k + 4u * t + i;
            x[k][i] = li < m ? ld_stream1(ar + li) : 0u;
            y[k][i] = li < m ? ld_stream1(br + li) : 0u;
        }
    uint32_t cin = 0, fin = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t l0 = 32u * k + 4u * t;
        const bool on = l0 < m;
        SegAS sg;
        sg.phase12(x[k], y[k], sub);
        WarpCarry wc;
        wc.resolve(on ? sg.g() : 0u, on ? sg.p() : 0u, t == 0 ? cin : 0u, 0x01010101u, 0x80808080u);
        const uint32_t c = wc.carry_in(lane);
        if (on && m - 1 < l0 + 4) fin = sg.carry_at(c, (int)(m - l0));   // limb m - 1 is one of these four
        sg.apply(c, sub);
        uint32_t *rr = r + d.r_off;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (l0 + i < m) st_stream1(rr + l0 + i, sg.r[i]);
        cin = wc.carry_out((lane & ~7) | 7);   // out of the run's chunk: into its next chunk
    }
    const int src = (grp << 3) | (int)(((m - 1) & 31u) >> 2);
    fin = __shfl_sync(DOT_FULL, fin, src);
    if (valid && t == 0) carry[op] = fin;
}

// The add/sub ops: the long bucket first, warp k taking ops k, k + W, ...
// (the next op's index and descriptor load while the current op runs, so that
// only the op's own data loads sit on its critical path), then the short
// bucket four ops per warp.
__global__ void __launch_bounds__(MIX_AS_THREADS, 4)
mixed_addsub(const dot_desc_t *desc, const uint32_t *order, const MixedMeta *meta, const uint32_t *a,
             const uint32_t *b, uint32_t *r, uint32_t *carry)
{
    const uint32_t n = meta->n[BK_ASL], base = meta->base[BK_ASL];
    const size_t wg = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nw = ((size_t)gridDim.x * blockDim.x) >> 5;
    size_t k = wg;
    uint32_t op = 0;
    dot_desc_t d{};
    if (k < n) {
        op = order[base + k];
        d = desc[op];
    }
    for (; k < n; k += nw) {
        const uint32_t cur = op;
        const dot_desc_t dc = d;
        if (k + nw < n) {   // prefetch the next op's index and descriptor
            op = order[base + k + nw];
            d = desc[op];
        }
        if (dc.op == DOT_OP_SUB)
            addsub_warp_op<true>(a + dc.a_off, b + dc.b_off, r + dc.r_off, dc.m, carry + cur, dc.m, 0u);
        else
            addsub_warp_op<false>(a + dc.a_off, b + dc.b_off, r + dc.r_off, dc.m, carry + cur, dc.m, 0u);
    }
    const uint32_t ns = meta->n[BK_ASS], bs = meta->base[BK_ASS];
    const size_t items = ((size_t)ns + 3) / 4;
    for (size_t it = wg; it < items; it += nw) mixed_addsub_short(desc, order, bs, ns, it, a, b, r, carry);
}

// The products in two persistent kernels, each over a range of buckets
// [LO, HI) with a work counter of its own: the 257..512-limb buckets (R = 9
// to 16, the most registers) and the rest (R <= 8), so that the smaller
// shapes run at the occupancy their registers allow instead of the largest
// shape's.
// Register caps: 3 blocks per SM for the 257..512-limb kernel (each shape
// alone needs at most 164 registers, but the eight inlined together took 242
// uncapped, which left 2 blocks per SM) and 4 for the other.
template <int LO, int HI, int K>
__global__ void __launch_bounds__(MIX_WARPS * 32, LO == BK_R16 ? 3 : 4)
mixed_run(const dot_desc_t *desc, const uint32_t *order, MixedMeta *meta, const uint32_t *a,
          const uint32_t *b, uint32_t *r, uint32_t *carry)
{
    // per-warp staging words: the largest shape of the kernel's buckets
    constexpr int RW = LO == BK_R16 ? mix_region_words(16, 32)
                                    : cmax(cmax(mix_region_words(8, 32), mix_region_words(8, 16)),
                                           cmax(mix_region_words(8, 8), mix_region_words(4, 4)));
    __shared__ __align__(16) uint32_t smem[MIX_WARPS * RW];
    const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
    uint32_t *wsmem = smem + warp * RW;
    const uint32_t first = meta->item_base[LO], total = meta->item_base[HI];
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = first + atomicAdd(&meta->next_item[K], 1ull);
        item = __shfl_sync(DOT_FULL, item, 0);
        if (item >= total) break;
        int bk = LO;
#pragma unroll
        for (int q = LO + 1; q < HI; ++q)
            if (item >= meta->item_base[q]) bk = q;
        const uint32_t n = meta->n[bk], base = meta->base[bk];
        const uint32_t k0 = (uint32_t)(item - meta->item_base[bk]) * bucket_ops_per_item(bk);
        if constexpr (LO == BK_R16) {
            switch (bk) {
            case BK_R16: mixed_mul_item<16, 32, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            case BK_R15: mixed_mul_item<15, 32, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            case BK_R14: mixed_mul_item<14, 32, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            case BK_R13: mixed_mul_item<13, 32, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            case BK_R12: mixed_mul_item<12, 32, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            case BK_R11: mixed_mul_item<11, 32, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            case BK_R10: mixed_mul_item<10, 32, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            default: mixed_mul_item<9, 32, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            }
        } else {
            switch (bk) {
            case BK_R8: mixed_mul_item<8, 32, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            case BK_R7: mixed_mul_item<7, 32, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            case BK_R6: mixed_mul_item<6, 32, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            case BK_M8B: mixed_mul_item<8, 16, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            case BK_M8A: mixed_mul_item<8, 8, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            default: mixed_mul_item<4, 4, RW>(desc, order, base, n, k0, a, b, r, carry, wsmem); break;
            }
        }
    }
    // the last warp out clears the work counter for the next call
    if (lane == 0) {
        __threadfence();
        const unsigned long long prev = atomicAdd(&meta->done[K], 1ull);
        if (prev == (unsigned long long)gridDim.x * MIX_WARPS - 1) {
            meta->next_item[K] = 0;
            meta->done[K] = 0;
            __threadfence();
        }
    }
}
#define MIX_RUN_WIDE mixed_run<BK_R16, BK_R8, 0>
#define MIX_RUN_NARROW mixed_run<BK_R8, BK_ASL, 1>

// ------------------------------------------------------------------ host
static MixedScratch *g_scratch_of(dot_ctx_t ctx);

struct MixedArgs {
    const dot_desc_t *desc;
    size_t nops;
    uint32_t *slot, *order, *carry, *status, *r;
    MixedMeta *meta;
    const uint32_t *a, *b;
};

// p3 serves both the add/sub and the run kernel (the same parameter list)
static void fill_params(const MixedArgs &A, void **p0, void **p1, void **p2, void **p3)
{
    // pointers to the argument values of the four kernels (must outlive the call)
    p0[0] = (void *)&A.desc; p0[1] = (void *)&A.nops; p0[2] = (void *)&A.slot; p0[3] = (void *)&A.meta;
    p0[4] = (void *)&A.carry; p0[5] = (void *)&A.status;
    p1[0] = (void *)&A.meta;
    p2[0] = (void *)&A.slot; p2[1] = (void *)&A.nops; p2[2] = (void *)&A.meta; p2[3] = (void *)&A.order;
    p3[0] = (void *)&A.desc; p3[1] = (void *)&A.order; p3[2] = (void *)&A.meta; p3[3] = (void *)&A.a;
    p3[4] = (void *)&A.b; p3[5] = (void *)&A.r; p3[6] = (void *)&A.carry;
}

static dot_status_t mixed_prepare(dot_ctx_t ctx, MixedScratch *S, size_t nops)
{
    if (S->meta == nullptr) {
        if (cudaMalloc((void **)&S->meta, sizeof(MixedMeta)) != cudaSuccess) return DOT_ENOMEM;
        if (cudaMemset(S->meta, 0, sizeof(MixedMeta)) != cudaSuccess) return DOT_ECUDA;
        // the product kernel takes every SM at its full occupancy (with two
        // blocks per SM instead of three, to leave the add/sub branch room,
        // the products ran 1.4x slower); the add/sub blocks fill in as the
        // product blocks finish
        S->persist_blocks = ctx->num_sms * dot_blocks_per_sm((const void *)MIX_RUN_WIDE, MIX_WARPS * 32, 0);
        S->narrow_blocks = ctx->num_sms * dot_blocks_per_sm((const void *)MIX_RUN_NARROW, MIX_WARPS * 32, 0);
        S->as_blocks = ctx->num_sms * MIX_AS_BLOCKS_PER_SM;
        if (cudaEventCreateWithFlags(&S->fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&S->join, cudaEventDisableTiming) != cudaSuccess)
            return DOT_ECUDA;
    }
    if (nops > S->cap) {
        size_t cap = S->cap ? S->cap : 4096;
        while (cap < nops) cap *= 2;
        if (cudaDeviceSynchronize() != cudaSuccess) return DOT_ECUDA;
        cudaFree(S->slot);
        cudaFree(S->order);
        S->slot = S->order = nullptr;
        S->cap = 0;
        if (cudaMalloc((void **)&S->slot, cap * 4) != cudaSuccess ||
            cudaMalloc((void **)&S->order, cap * 4) != cudaSuccess)
            return DOT_ENOMEM;
        S->cap = cap;
    }
    return DOT_OK;
}

static dot_status_t mixed_capture(dot_ctx_t ctx, MixedScratch *S, const MixedArgs &A)
{
    // record the six launches once on a private stream, then keep the graph
    cudaStream_t cs = ctx->side[0];
    if (cudaStreamSynchronize(cs) != cudaSuccess) return DOT_ECUDA;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return DOT_ECUDA;
    const unsigned g1 = (unsigned)((A.nops + 255) / 256);
    mixed_classify<<<g1, 256, 0, cs>>>(A.desc, A.nops, A.slot, A.meta, A.carry, A.status);
    mixed_plan<<<1, 32, 0, cs>>>(A.meta);
    mixed_scatter<<<g1, 256, 0, cs>>>(A.slot, A.nops, A.meta, A.order);
    // the add/sub ops (memory-bound) and the products (ALU-bound) are two
    // parallel branches of the graph, so that their kernels share the SMs
    cudaStream_t cs2 = ctx->side[1];
    if (cudaEventRecord(S->fork, cs) != cudaSuccess || cudaStreamWaitEvent(cs2, S->fork, 0) != cudaSuccess)
        return DOT_ECUDA;
    mixed_addsub<<<S->as_blocks, MIX_AS_THREADS, 0, cs2>>>(A.desc, A.order, A.meta, A.a, A.b, A.r, A.carry);
    MIX_RUN_NARROW<<<S->narrow_blocks, MIX_WARPS * 32, 0, cs2>>>(A.desc, A.order, A.meta, A.a, A.b, A.r, A.carry);
    MIX_RUN_WIDE<<<S->persist_blocks, MIX_WARPS * 32, 0, cs>>>(A.desc, A.order, A.meta, A.a, A.b, A.r, A.carry);
    if (cudaEventRecord(S->join, cs2) != cudaSuccess || cudaStreamWaitEvent(cs, S->join, 0) != cudaSuccess)
        return DOT_ECUDA;
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess || !g) return DOT_ECUDA;
    size_t nn = 0;
    cudaGraphNode_t nodes[8];
    if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess || nn != 6) {
        cudaGraphDestroy(g);
        return DOT_ECUDA;
    }
    cudaGraphGetNodes(g, nodes, &nn);
    const void *fns[6] = {(const void *)mixed_classify, (const void *)mixed_plan, (const void *)mixed_scatter,
                          (const void *)mixed_addsub, (const void *)MIX_RUN_WIDE, (const void *)MIX_RUN_NARROW};
    for (size_t i = 0; i < nn; ++i) {
        cudaKernelNodeParams kp;
        if (cudaGraphKernelNodeGetParams(nodes[i], &kp) != cudaSuccess) {
            cudaGraphDestroy(g);
            return DOT_ECUDA;
        }
        for (int k = 0; k < 6; ++k)
            if (kp.func == fns[k]) S->node[k] = nodes[i];
    }
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return DOT_ECUDA;
    }
    S->graph = g;
    S->exec = ex;
    return DOT_OK;
}

static MixedScratch *g_scratch_of(dot_ctx_t ctx)
{
    if (!ctx->mixed) ctx->mixed = calloc(1, sizeof(MixedScratch));
    return (MixedScratch *)ctx->mixed;
}

void dot_mixed_release(dot_ctx_t ctx)
{
    MixedScratch *S = (MixedScratch *)ctx->mixed;
    if (!S) return;
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    if (S->fork) cudaEventDestroy(S->fork);
    if (S->join) cudaEventDestroy(S->join);
    cudaFree(S->slot);
    cudaFree(S->order);
    cudaFree(S->meta);
    free(S);
    ctx->mixed = nullptr;
}

extern "C" {

DOT_API dot_status_t dot_mixed_ragged(dot_ctx_t ctx, const dot_desc_t *desc, size_t nops,
                                      const uint32_t *a, const uint32_t *b, uint32_t *r,
                                      uint32_t *carry, dot_stream_t stream)
{
    DeviceScope scope;
    dot_status_t rc = dot_check_ctx(ctx, scope);
    if (rc != DOT_OK) return rc;
    if (nops == 0) return DOT_OK;
    if (!desc || !a || !b || !r || !carry || nops >= MIX_MAX_OPS) return DOT_EINVAL;
    MixedScratch *S = g_scratch_of(ctx);
    if (!S) return DOT_ENOMEM;
    rc = mixed_prepare(ctx, S, nops);
    if (rc != DOT_OK) return rc;
    MixedArgs A{desc, nops, S->slot, S->order, carry, ctx->d_status, r, S->meta, a, b};
    if (!S->exec) {
        rc = mixed_capture(ctx, S, A);
        if (rc != DOT_OK) return rc;
    }
    void *p0[6], *p1[1], *p2[4], *p3[7];
    fill_params(A, p0, p1, p2, p3);
    const unsigned g1 = (unsigned)((nops + 255) / 256);
    const void *fns[6] = {(const void *)mixed_classify, (const void *)mixed_plan, (const void *)mixed_scatter,
                          (const void *)mixed_addsub, (const void *)MIX_RUN_WIDE, (const void *)MIX_RUN_NARROW};
    void **params[6] = {p0, p1, p2, p3, p3, p3};
    const dim3 grids[6] = {dim3(g1), dim3(1), dim3(g1), dim3((unsigned)S->as_blocks),
                           dim3((unsigned)S->persist_blocks), dim3((unsigned)S->narrow_blocks)};
    const dim3 blocks[6] = {dim3(256), dim3(32), dim3(256), dim3(MIX_AS_THREADS), dim3(MIX_WARPS * 32),
                            dim3(MIX_WARPS * 32)};
    for (int k = 0; k < 6; ++k) {
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof kp);
        kp.func = (void *)fns[k];
        kp.gridDim = grids[k];
        kp.blockDim = blocks[k];
        kp.sharedMemBytes = 0;
        kp.kernelParams = params[k];
        kp.extra = nullptr;
        if (cudaGraphExecKernelNodeSetParams(S->exec, S->node[k], &kp) != cudaSuccess) return DOT_ECUDA;
    }
    return cudaGraphLaunch(S->exec, (cudaStream_t)stream) == cudaSuccess ? DOT_OK : DOT_ECUDA;
}

}  // extern "C"
