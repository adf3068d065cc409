// dot_addsub.cu -- batched and ragged multi-limb addition / subtraction.
//
// DoT addition (Alg. 1, Theorem 1, Sec. 3.1) re-shaped for a GPU:
//  * Phase 1 (independent limb adds) and Phase 2 (generate / propagate bits)
//    run on each thread's segment of 1 or 4 limbs, loaded with 128-bit
//    coalesced loads.
//  * Alg. 1's sequential chain of c_out between SIMD chunks is replaced by a
//    carry-lookahead: segment (g, p) bits are gathered with __ballot_sync
//    and resolved with the same mask identity Phase 4 uses,
//    carries = ((G << 1 | c_in) + P) ^ P.
//  * Operands longer than one thread block's tile are chained across blocks
//    by decoupled look-back over per-tile states in global memory.
//  * Phases 3-4 (adding the carries back) happen in registers before the
//    streaming store.
// Subtraction is the same with borrows (Sec. 3.1, "Subtraction").
#include <atomic>
#include <mutex>

#include "dot_internal.cuh"
#include "dot_plan.h"
#include "dot_addsub.cuh"
#include "dot_warp_op.cuh"

#define WARP_KERNEL_THREADS 256

// ======================================================= warp kernel (1)
// Each op lies inside one warp: runs of `lpo` lanes per op (several ops per
// warp when the op has at most 16 segments), or all 32 lanes and up to NCH
// chunks of 32 segments chained through the warp's carry-out.  U independent
// op groups are loaded before any is resolved, to keep enough bytes in flight.
template <bool SUB, int SEG, int NCH, int U>
__global__ void __launch_bounds__(WARP_KERNEL_THREADS)
addsub_warp_kernel(const uint32_t *a, const uint32_t *b, uint32_t *s, uint32_t *cout,
                   size_t m, size_t batch, int lpo, int nch)
{
    const int lane = (int)lane_id();
    const int opw = 32 / lpo;
    const int grp = lane / lpo;
    const int rel = lane - grp * lpo;
    const bool lane_on = grp < opw;
    const uint32_t smask = run_start_mask(lpo), tmask = run_top_mask(lpo);
    const size_t Q = (m + SEG - 1) / SEG;
    const int last_chunk = (int)((Q - 1) / (size_t)lpo);
    const int last_rel = (int)((Q - 1) % (size_t)lpo);
    const size_t warp_global = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const size_t per_iter = (size_t)opw * U;

    for (size_t base = warp_global * per_iter; base < batch; base += nwarps * per_iter) {
        uint32_t x[U][NCH][SEG], y[U][NCH][SEG];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t op = base + (size_t)u * opw + grp;
#pragma unroll
            for (int j = 0; j < NCH; ++j) {
                const size_t q = (size_t)j * lpo + rel;
                if (lane_on && op < batch && j < nch && q < Q) {
                    load_seg<SEG>(a + op * m + q * SEG, x[u][j]);
                    load_seg<SEG>(b + op * m + q * SEG, y[u][j]);
                } else {
#pragma unroll
                    for (int i = 0; i < SEG; ++i) x[u][j][i] = y[u][j][i] = 0;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const size_t op = base + (size_t)u * opw + grp;
            const bool op_on = lane_on && op < batch;
            uint32_t cin = 0;
#pragma unroll
            for (int j = 0; j < NCH; ++j) {
                if (j >= nch) break;
                const size_t q = (size_t)j * lpo + rel;
                const bool on = op_on && q < Q;
                Segment<SUB, SEG> sg;
                sg.phase12(x[u][j], y[u][j]);
                WarpCarry wc;
                wc.resolve(on ? sg.g() : 0u, on ? sg.p() : 0u, rel == 0 ? cin : 0u, smask, tmask);
                const uint32_t c = wc.carry_in(lane);
                sg.apply(c);
                if (on) store_seg<SEG>(s + op * m + q * SEG, sg.r);
                if (j == last_chunk) {
                    if (on && rel == last_rel) cout[op] = sg.cout(c);
                } else {
                    cin = wc.carry_out(31);   // lpo == 32 whenever there are several chunks
                }
            }
        }
    }
}

// ================================================= tiled kernel (2) + look-back
// A tile is DOT_TILE_THREADS threads x NCH chunks x SEG limbs of one op.  Tiles
// are taken in ticket order (atomic counter), so every tile's predecessor in
// its op has already been taken by a running block: the look-back wait always
// ends.  Each tile publishes its carry state (epoch-tagged): INCLUSIVE as soon
// as its own aggregate decides the carry-out (generate or kill), PROPAGATE
// otherwise, then INCLUSIVE once its carry-in is known.
// A tile state is one self-contained word (epoch and carry code): its reader
// needs nothing else the writer stored, so relaxed gpu-scope accesses are
// enough.  A release store would hold each publication until every earlier
// store of the block (the previous tile's sums) had drained to L2.
__device__ __forceinline__ unsigned long long ld_state(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_state(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

__device__ uint32_t lookback_carry(const LookbackArgs &lb, const unsigned long long *st_op,
                                   long long t, unsigned long long epoch, int lane)
{
    long long j_hi = t - 1;
    uint64_t t0 = 0;
    bool timing = false;
    for (;;) {
        const long long j = j_hi - lane;
        uint32_t code = LB_INCL0;   // before the op's first tile: carry 0
        if (j >= 0) {
            const unsigned long long w = ld_state(st_op + j);
            code = ((w >> 2) == epoch) ? (uint32_t)(w & 3ull) : (uint32_t)LB_EMPTY;
        }
        const uint32_t incl = __ballot_sync(DOT_FULL, code >= LB_INCL0);
        const uint32_t empty = __ballot_sync(DOT_FULL, code == LB_EMPTY);
        const uint32_t nearer = incl ? ((incl & (0u - incl)) - 1u) : DOT_FULL;
        if ((empty & nearer) == 0) {
            if (incl) {
                const int L = __ffs(incl) - 1;
                return __shfl_sync(DOT_FULL, code, L) & 1u;
            }
            j_hi -= 32;   // 32 propagating predecessors: keep walking back
            continue;
        }
        // a nearer predecessor has not published yet: wait (bounded); the
        // first polls are tight (a predecessor of the same round publishes
        // within a few hundred cycles), later ones back off
        uint64_t now = 0;
        if (lane == 0) now = globaltimer_ns();
        now = __shfl_sync(DOT_FULL, now, 0);
        if (!timing) {
            t0 = now;
            timing = true;
        } else if (now - t0 > lb.wait_limit_ns) {
            if (lane == 0) record_status(lb.status, DOT_ETIMEOUT);
            return 0;
        }
        if (now - t0 > 2000) __nanosleep(64);
    }
}

template <bool SUB, int SEG, int NCH>
__global__ void __launch_bounds__(DOT_TILE_THREADS)
addsub_tile_kernel(const uint32_t *a, const uint32_t *b, uint32_t *s, uint32_t *cout,
                   size_t m, size_t batch, unsigned long long tiles_per_op, LookbackArgs lb)
{
    constexpr int WARPS = DOT_TILE_THREADS / 32;
    constexpr unsigned long long TILE = (unsigned long long)DOT_TILE_THREADS * SEG * NCH;
    constexpr int WARP_LIMBS = 32 * SEG * NCH;
    __shared__ unsigned long long s_ticket;
    __shared__ uint32_t s_wagg[WARPS];
    __shared__ uint32_t s_cin;
    const int lane = (int)lane_id();
    const int warp = (int)(threadIdx.x >> 5);
    const unsigned long long epoch = lb.counters[2];
    const unsigned long long total = (unsigned long long)batch * tiles_per_op;

    for (;;) {
        if (threadIdx.x == 0) s_ticket = atomicAdd(&lb.counters[0], 1ull);
        __syncthreads();
        const unsigned long long ticket = s_ticket;
        if (ticket >= total) break;
        const unsigned long long op = ticket / tiles_per_op;
        const unsigned long long t = ticket - op * tiles_per_op;
        const size_t wbase = (size_t)(t * TILE) + (size_t)warp * WARP_LIMBS;
        const uint32_t *ar = a + op * m;
        const uint32_t *br = b + op * m;
        uint32_t *sr = s + op * m;

        uint32_t x[NCH][SEG], y[NCH][SEG];
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            const size_t li = wbase + ((size_t)j * 32 + lane) * SEG;
            if (li < m) {
                load_seg<SEG>(ar + li, x[j]);
                load_seg<SEG>(br + li, y[j]);
            } else {
#pragma unroll
                for (int i = 0; i < SEG; ++i) x[j][i] = y[j][i] = 0;
            }
        }
        Segment<SUB, SEG> sg[NCH];
        uint32_t G[NCH], P[NCH];
        uint32_t wg = 0, wp = 1;   // warp aggregate, composed chunk by chunk
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            sg[j].phase12(x[j], y[j]);
            const size_t li = wbase + ((size_t)j * 32 + lane) * SEG;
            const bool on = li < m;
            WarpCarry wc;
            wc.resolve(on ? sg[j].g() : 0u, on ? sg[j].p() : 0u, 0u, 1u, 0x80000000u);
            G[j] = wc.G;
            P[j] = wc.P;
            gp_compose(wg, wp, wc.carry_out(31), (uint32_t)(wc.P == DOT_FULL));
        }
        if (lane == 0) s_wagg[warp] = wg | (wp << 1);
        __syncthreads();

        if (warp == 0) {
            uint32_t tg = 0, tp = 1;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) gp_compose(tg, tp, s_wagg[w] & 1u, s_wagg[w] >> 1);
            unsigned long long *st_op = lb.state + (ticket - t);
            const bool skip = lb.skip_tile >= 0 && op == 0 && (long long)t == lb.skip_tile;
            uint32_t cin_tile = 0;
            if (t == 0) {
                if (lane == 0 && !skip)
                    st_state(st_op, (epoch << 2) | (tg ? LB_INCL1 : LB_INCL0));
            } else {
                if (lane == 0 && !skip)
                    st_state(st_op + t, (epoch << 2) | (tp ? LB_PROP : (tg ? LB_INCL1 : LB_INCL0)));
                cin_tile = lookback_carry(lb, st_op, (long long)t, epoch, lane);
                if (tp && lane == 0 && !skip)
                    st_state(st_op + t, (epoch << 2) | (cin_tile ? LB_INCL1 : LB_INCL0));
            }
            if (lane == 0) s_cin = cin_tile;
        }
        __syncthreads();

        // carry into this warp: the tile carry-in passed through the warps below
        uint32_t c = s_cin;
        for (int w = 0; w < warp; ++w) {
            uint32_t g = s_wagg[w] & 1u, p = s_wagg[w] >> 1;
            c = g | (p & c);
        }
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            const size_t li = wbase + ((size_t)j * 32 + lane) * SEG;
            const uint32_t Pm = P[j] & 0x7fffffffu;
            const uint32_t C = (((G[j] << 1) | c) + Pm) ^ Pm;
            const uint32_t ci = (C >> lane) & 1u;
            sg[j].apply(ci);
            if (li < m) {
                store_seg<SEG>(sr + li, sg[j].r);
                if (li + SEG >= m && t == tiles_per_op - 1) cout[op] = sg[j].cout(ci);
            }
            c = ((G[j] >> 31) | ((P[j] >> 31) & (C >> 31))) & 1u;
        }
        __syncthreads();
    }
    // the last block out resets the ticket counter and advances the epoch
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long prev = atomicAdd(&lb.counters[1], 1ull);
        if (prev == gridDim.x - 1) {
            lb.counters[0] = 0;
            lb.counters[1] = 0;
            __threadfence();
            lb.counters[2] = epoch + 1;
        }
    }
}

// ============================ tiled kernel (2b): bulk-copy prefetch + look-back
// Same tiles and look-back as above, for 16-byte aligned rows with m % 4 == 0.
// A persistent grid (one block per resident slot) takes tiles in ticket order
// from the atomic counter; each block holds one ticket in reserve, so the
// atomic's latency is paid while the previous copies are in flight rather
// than before the next copy can start.  Each block streams its tiles through
// two shared-memory stages (cp.async.bulk, completion counted on an mbarrier)
// and works one tile AHEAD: as soon as tile k + 1 has arrived it forms and
// publishes that tile's aggregate, and only then resolves tile k's carry-in and
// stores tile k.  A tile's predecessor therefore has almost always published
// already, and the look-back wait leaves the critical path; publishing only
// after the previous tile was stored made every block wait on its
// predecessor's progress, and the delays travelled along each op's tiles.
// The waits always end: a tile's predecessor has a lower ticket, taken
// earlier by a block that is running, and a block's tickets increase, so the
// lowest unfinished ticket never waits on a higher one.  Tickets also spread
// the tiles by arrival: a block whose copies come back early takes more of
// them (a static round-robin schedule ended with the slowest block).
template <bool SUB, int NCH>
struct TileRegs {
    Segment<SUB, 4> sg[NCH];
    uint32_t G[NCH], P[NCH];
};

template <bool SUB, int NCH>
__device__ __forceinline__ void tile_bulk_aggregate(const uint32_t *stage, unsigned long long ticket,
                                                    unsigned long long tiles_per_op, size_t m, int st,
                                                    TileRegs<SUB, NCH> &tr, uint32_t *wagg, int lane, int warp)
{
    constexpr unsigned long long TILE = (unsigned long long)DOT_TILE_THREADS * 4 * NCH;
    constexpr int WARP_LIMBS = 32 * 4 * NCH;
    const unsigned long long t = ticket % tiles_per_op;
    const size_t wbase = (size_t)(t * TILE) + (size_t)warp * WARP_LIMBS;
    const uint32_t *xa = stage + (2 * st) * TILE + warp * WARP_LIMBS;
    const uint32_t *xb = stage + (2 * st + 1) * TILE + warp * WARP_LIMBS;
    uint32_t wg = 0, wp = 1;
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
        const size_t li = wbase + ((size_t)j * 32 + lane) * 4;
        const bool on = li < m;
        uint32_t x[4] = {0u, 0u, 0u, 0u}, y[4] = {0u, 0u, 0u, 0u};
        if (on) {
            const uint4 qa = reinterpret_cast<const uint4 *>(xa)[j * 32 + lane];
            const uint4 qb = reinterpret_cast<const uint4 *>(xb)[j * 32 + lane];
            x[0] = qa.x; x[1] = qa.y; x[2] = qa.z; x[3] = qa.w;
            y[0] = qb.x; y[1] = qb.y; y[2] = qb.z; y[3] = qb.w;
        }
        tr.sg[j].phase12(x, y);
        WarpCarry wc;
        wc.resolve(on ? tr.sg[j].g() : 0u, on ? tr.sg[j].p() : 0u, 0u, 1u, 0x80000000u);
        tr.G[j] = wc.G;
        tr.P[j] = wc.P;
        gp_compose(wg, wp, wc.carry_out(31), (uint32_t)(wc.P == DOT_FULL));
    }
    if (lane == 0) wagg[warp] = wg | (wp << 1);
}

template <bool SUB, int NCH>
__device__ __forceinline__ void tile_bulk_apply(TileRegs<SUB, NCH> &tr, uint32_t *s, uint32_t *cout,
                                                unsigned long long ticket, unsigned long long tiles_per_op,
                                                size_t m, uint32_t c, int lane, int warp)
{
    constexpr unsigned long long TILE = (unsigned long long)DOT_TILE_THREADS * 4 * NCH;
    constexpr int WARP_LIMBS = 32 * 4 * NCH;
    const unsigned long long op = ticket / tiles_per_op;
    const unsigned long long t = ticket - op * tiles_per_op;
    const size_t wbase = (size_t)(t * TILE) + (size_t)warp * WARP_LIMBS;
    uint32_t *sr = s + op * m;
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
        const size_t li = wbase + ((size_t)j * 32 + lane) * 4;
        const uint32_t Pm = tr.P[j] & 0x7fffffffu;
        const uint32_t C = (((tr.G[j] << 1) | c) + Pm) ^ Pm;
        const uint32_t ci = (C >> lane) & 1u;
        tr.sg[j].apply(ci);
        if (li < m) {
            store_seg<4>(sr + li, tr.sg[j].r);
            if (li + 4 >= m && t == tiles_per_op - 1) cout[op] = tr.sg[j].cout(ci);
        }
        c = ((tr.G[j] >> 31) | ((tr.P[j] >> 31) & (C >> 31))) & 1u;
    }
}

template <bool SUB, int NCH>
__global__ void __launch_bounds__(DOT_TILE_THREADS, 3)
addsub_tile_bulk_kernel(const uint32_t *a, const uint32_t *b, uint32_t *s, uint32_t *cout,
                        size_t m, size_t batch, unsigned long long tiles_per_op, LookbackArgs lb)
{
    constexpr int WARPS = DOT_TILE_THREADS / 32;
    constexpr unsigned long long TILE = (unsigned long long)DOT_TILE_THREADS * 4 * NCH;
    extern __shared__ __align__(128) uint32_t stage[];   // [2][2][TILE]: stage, operand
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ unsigned long long s_ticket[2];
    // per-warp aggregates of tile k in slot k % 4 and its carry-in in s_cin[k % 2]:
    // with two CTA barriers per tile, a slot is rewritten only after every warp
    // has passed a barrier that follows its last read
    __shared__ uint32_t s_wagg[4][WARPS];
    __shared__ uint32_t s_cin[2];
    const int lane = (int)lane_id();
    const int warp = (int)(threadIdx.x >> 5);
    const unsigned long long epoch = lb.counters[2];
    const unsigned long long total = (unsigned long long)batch * tiles_per_op;

    unsigned long long reserve = 0;   // thread 0: the ticket this block takes next
    auto issue = [&](int st, int k) {   // thread 0: start the copies of this block's k-th tile
        const unsigned long long tk = reserve;
        if (tk < total) reserve = atomicAdd(&lb.counters[0], 1ull);
        s_ticket[st] = tk;
        if (tk < total) {
            const unsigned long long op = tk / tiles_per_op, t = tk - op * tiles_per_op;
            const size_t first = (size_t)(t * TILE);
            const size_t lim = (m - first < TILE) ? m - first : (size_t)TILE;
            const uint32_t bytes = (uint32_t)(lim * 4);
            mbar_arrive_expect_tx(&s_bar[st], 2 * bytes);
            bulk_g2s(stage + (2 * st) * TILE, a + op * m + first, bytes, &s_bar[st]);
            bulk_g2s(stage + (2 * st + 1) * TILE, b + op * m + first, bytes, &s_bar[st]);
        }
    };
    // warp 0: compose the block aggregate of tile k and publish it (INCLUSIVE
    // when it decides the carry-out, PROPAGATE otherwise)
    auto publish = [&](int k, unsigned long long ticket) {
        uint32_t tg = 0, tp = 1;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) gp_compose(tg, tp, s_wagg[k & 3][w] & 1u, s_wagg[k & 3][w] >> 1);
        const unsigned long long op = ticket / tiles_per_op, t = ticket - op * tiles_per_op;
        const bool skip = lb.skip_tile >= 0 && op == 0 && (long long)t == lb.skip_tile;
        if (lane == 0 && !skip)
            st_state(lb.state + ticket, (epoch << 2) | ((tp && t > 0) ? LB_PROP : (tg ? LB_INCL1 : LB_INCL0)));
    };
    // all threads: wait for tile k (stage st, ticket read by every thread
    // before the call), form its aggregates, publish, and reuse the stage for
    // tile k + 2
    auto take = [&](int st, int k, unsigned long long ticket, TileRegs<SUB, NCH> &tr) {
        if (!mbar_wait_bounded(&s_bar[st], (uint32_t)((k >> 1) & 1), lb.wait_limit_ns) && lane == 0)
            record_status(lb.status, DOT_ETIMEOUT);
        tile_bulk_aggregate<SUB, NCH>(stage, ticket, tiles_per_op, m, st, tr, s_wagg[k & 3], lane, warp);
        __syncthreads();   // stage st fully read, s_ticket[st] read by all; aggregates visible
        if (warp == 0) publish(k, ticket);
        if (threadIdx.x == 0) issue(st, k + 2);
    };
    // warp 0: carry into tile k (the look-back; a PROPAGATE tile then
    // publishes INCLUSIVE); all threads: add it in and store the tile
    auto finish = [&](int k, unsigned long long ticket, TileRegs<SUB, NCH> &tr) {
        const uint32_t *wagg = s_wagg[k & 3];
        if (warp == 0) {
            const unsigned long long op = ticket / tiles_per_op, t = ticket - op * tiles_per_op;
            uint32_t cin_tile = 0;
            if (t > 0) {
                const unsigned long long *st_op = lb.state + (ticket - t);
                uint32_t tg = 0, tp = 1;
#pragma unroll
                for (int w = 0; w < WARPS; ++w) gp_compose(tg, tp, wagg[w] & 1u, wagg[w] >> 1);
                cin_tile = lookback_carry(lb, st_op, (long long)t, epoch, lane);
                const bool skip = lb.skip_tile >= 0 && op == 0 && (long long)t == lb.skip_tile;
                if (tp && lane == 0 && !skip)
                    st_state(lb.state + ticket, (epoch << 2) | (cin_tile ? LB_INCL1 : LB_INCL0));
            }
            if (lane == 0) s_cin[k & 1] = cin_tile;
        }
        __syncthreads();
        uint32_t c = s_cin[k & 1];
        for (int w = 0; w < warp; ++w) {
            const uint32_t g = wagg[w] & 1u, p = wagg[w] >> 1;
            c = g | (p & c);
        }
        tile_bulk_apply<SUB, NCH>(tr, s, cout, ticket, tiles_per_op, m, c, lane, warp);
    };

    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_init_fence();
        reserve = atomicAdd(&lb.counters[0], 1ull);
        issue(0, 0);
        issue(1, 1);
    }
    __syncthreads();

    // Tiles alternate between two register sets (the loop is unrolled by two
    // so that neither is copied): tile k in A (k even) or B (k odd).  Tickets
    // are read from s_ticket before take() re-issues that stage.
    TileRegs<SUB, NCH> A, B;
    unsigned long long tA = s_ticket[0];
    if (tA < total) take(0, 0, tA, A);
    for (int k = 0; tA < total; k += 2) {
        const unsigned long long tB = s_ticket[1];   // tile k + 1
        if (tB < total) take(1, k + 1, tB, B);
        finish(k, tA, A);
        if (tB >= total) break;
        tA = s_ticket[0];                            // tile k + 2
        if (tA < total) take(0, k + 2, tA, A);
        finish(k + 1, tB, B);
    }
    // the last block out resets the ticket counter and advances the epoch
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned long long prev = atomicAdd(&lb.counters[1], 1ull);
        if (prev == gridDim.x - 1) {
            lb.counters[0] = 0;
            lb.counters[1] = 0;
            __threadfence();
            lb.counters[2] = epoch + 1;
        }
    }
}

// ===================================================== ragged kernel (one warp per op)
template <bool SUB>
__global__ void __launch_bounds__(WARP_KERNEL_THREADS)
addsub_ragged_kernel(const uint32_t *a, const uint32_t *b, uint32_t *s, uint32_t *cout,
                     const uint64_t *off, size_t batch, uint32_t *status)
{
    const size_t warp_global = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    for (size_t op = warp_global; op < batch; op += nwarps) {
        const uint64_t lo = off[op], hi = off[op + 1];
        if (hi < lo) {
            if (lane_id() == 0) {
                record_status(status, DOT_EINVAL);
                cout[op] = 0;
            }
            continue;
        }
        addsub_warp_op<SUB>(a + lo, b + lo, s + lo, (size_t)(hi - lo), cout + op, (size_t)(hi - lo), 0u);
    }
}

// ============================ general add/sub: carry-in, unequal lengths
// Op i: a_i (ma limbs) +/- b_i (mb <= ma limbs, zero-extended) + cin_i, the
// ma-limb result and its carry/borrow out; cin may be null (no carry-in), a
// nonzero cin_i counts as 1.  One warp per op (the mpn-style variants).
template <bool SUB>
__global__ void __launch_bounds__(WARP_KERNEL_THREADS)
addsub_general_kernel(const uint32_t *a, const uint32_t *b, const uint32_t *cin, uint32_t *s, uint32_t *cout,
                      size_t ma, size_t mb, size_t batch)
{
    const size_t warp_global = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    for (size_t op = warp_global; op < batch; op += nwarps) {
        const uint32_t c = cin ? (uint32_t)(cin[op] != 0u) : 0u;
        addsub_warp_op<SUB>(a + op * ma, b + op * mb, s + op * ma, ma, cout + op, mb, c);
    }
}

// =========================================================== host launchers
template <bool SUB, int SEG>
static cudaError_t launch_warp(dot_ctx_t ctx, const dot_plan_t &pl, const uint32_t *a,
                               const uint32_t *b, uint32_t *s, uint32_t *cout, size_t m,
                               size_t batch, cudaStream_t st)
{
    const int lpo = pl.lanes_per_op, nch = pl.chunks;
    const int opw = 32 / lpo;
    // Four op groups per warp keep bytes in flight on large batches; a batch
    // that would then occupy fewer than 8 warps per SM takes one group per
    // warp instead, so that every SM works on it (a call that small is one
    // memory round trip, bound by latency).
    const bool spread = nch == 1 && dot_ceil_div(batch, (size_t)opw * 4) < (size_t)ctx->num_sms * 8;
    const int U = (nch == 1 && !spread) ? 4 : 1;
    const size_t warp_iters = dot_ceil_div(batch, (size_t)opw * U);
    const size_t blocks_needed = dot_ceil_div(warp_iters, WARP_KERNEL_THREADS / 32);
    const void *fn;
    if (nch == 1) fn = spread ? (const void *)addsub_warp_kernel<SUB, SEG, 1, 1> : (const void *)addsub_warp_kernel<SUB, SEG, 1, 4>;
    else if (nch == 2) fn = (const void *)addsub_warp_kernel<SUB, SEG, 2, 1>;
    else fn = (const void *)addsub_warp_kernel<SUB, SEG, 4, 1>;
    const size_t cap = (size_t)ctx->num_sms * dot_blocks_per_sm(fn, WARP_KERNEL_THREADS, 0);
    const unsigned grid = (unsigned)(blocks_needed < cap ? blocks_needed : cap);
    if (nch == 1 && spread)
        addsub_warp_kernel<SUB, SEG, 1, 1><<<grid, WARP_KERNEL_THREADS, 0, st>>>(a, b, s, cout, m, batch, lpo, nch);
    else if (nch == 1)
        addsub_warp_kernel<SUB, SEG, 1, 4><<<grid, WARP_KERNEL_THREADS, 0, st>>>(a, b, s, cout, m, batch, lpo, nch);
    else if (nch == 2)
        addsub_warp_kernel<SUB, SEG, 2, 1><<<grid, WARP_KERNEL_THREADS, 0, st>>>(a, b, s, cout, m, batch, lpo, nch);
    else
        addsub_warp_kernel<SUB, SEG, 4, 1><<<grid, WARP_KERNEL_THREADS, 0, st>>>(a, b, s, cout, m, batch, lpo, nch);
    return cudaGetLastError();
}

template <bool SUB, int SEG>
static dot_status_t launch_tile(dot_ctx_t ctx, const dot_plan_t &pl, const uint32_t *a,
                                const uint32_t *b, uint32_t *s, uint32_t *cout, size_t m,
                                size_t batch, cudaStream_t st)
{
    LookbackArgs lb;
    const size_t tiles = (size_t)pl.tiles * batch;
    dot_status_t rc = dot_lookback_prepare(ctx, tiles, &lb);
    if (rc != DOT_OK) return rc;
    ctx->debug_skip_tile = -1;   // the hook fires once
    const unsigned long long tpo = pl.tiles;
    if constexpr (SEG == 4) {
        // 16-byte aligned rows: the kernel with bulk-copy prefetch
        const size_t smem = (size_t)2 * 2 * DOT_TILE_THREADS * 4 * pl.chunks * 4;
        const void *fb = pl.chunks == 1 ? (const void *)addsub_tile_bulk_kernel<SUB, 1>
                       : pl.chunks == 2 ? (const void *)addsub_tile_bulk_kernel<SUB, 2>
                                        : (const void *)addsub_tile_bulk_kernel<SUB, 4>;
        if (cudaFuncSetAttribute(fb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return DOT_ECUDA;
        // one block per resident slot (tickets balance the tiles among them)
        const size_t cap = (size_t)ctx->num_sms * dot_blocks_per_sm(fb, DOT_TILE_THREADS, smem);
        const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
        void *args[] = {(void *)&a, (void *)&b, (void *)&s, (void *)&cout, (void *)&m, (void *)&batch,
                        (void *)&tpo, (void *)&lb};
        const cudaError_t e = cudaLaunchKernel(fb, dim3(grid), dim3(DOT_TILE_THREADS), args, smem, st);
        return e == cudaSuccess ? DOT_OK : DOT_ECUDA;
    }
    const void *fn;
    if (pl.chunks == 1) fn = (const void *)addsub_tile_kernel<SUB, SEG, 1>;
    else if (pl.chunks == 2) fn = (const void *)addsub_tile_kernel<SUB, SEG, 2>;
    else fn = (const void *)addsub_tile_kernel<SUB, SEG, 4>;
    const size_t cap = (size_t)ctx->num_sms * dot_blocks_per_sm(fn, DOT_TILE_THREADS, 0);
    const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
    if (pl.chunks == 1)
        addsub_tile_kernel<SUB, SEG, 1><<<grid, DOT_TILE_THREADS, 0, st>>>(a, b, s, cout, m, batch, tpo, lb);
    else if (pl.chunks == 2)
        addsub_tile_kernel<SUB, SEG, 2><<<grid, DOT_TILE_THREADS, 0, st>>>(a, b, s, cout, m, batch, tpo, lb);
    else
        addsub_tile_kernel<SUB, SEG, 4><<<grid, DOT_TILE_THREADS, 0, st>>>(a, b, s, cout, m, batch, tpo, lb);
    return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
}

template <bool SUB>
static dot_status_t addsub_batched(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *s,
                                   uint32_t *cout, size_t m, size_t batch, cudaStream_t st)
{
    DeviceScope scope;
    dot_status_t rc = dot_check_ctx(ctx, scope);
    if (rc != DOT_OK) return rc;
    if (batch == 0) return DOT_OK;
    if (!cout) return DOT_EINVAL;
    if (m && (!a || !b || !s)) return DOT_EINVAL;
    if (m > SIZE_MAX / 4 / batch) return DOT_EINVAL;
    const size_t bytes = m * batch * 4;
    if (partial_overlap(s, bytes, a, bytes) || partial_overlap(s, bytes, b, bytes)) return DOT_EINVAL;
    if (any_overlap(cout, batch * 4, s, bytes) || any_overlap(cout, batch * 4, a, bytes) ||
        any_overlap(cout, batch * 4, b, bytes))
        return DOT_EINVAL;
    if (m == 0) return cudaMemsetAsync(cout, 0, batch * 4, st) == cudaSuccess ? DOT_OK : DOT_ECUDA;
    const bool vec = (m % 4 == 0) && aligned16(a) && aligned16(b) && aligned16(s);
    dot_plan_t pl;
    const int op = SUB ? DOT_OP_SUB : DOT_OP_ADD;
    rc = dot_make_plan(op, m, batch, vec, &pl, ctx->tune[op][dot_tune_bucket(m)]);
    if (rc != DOT_OK) return rc;
    if (pl.kernel == DOT_K_ADDSUB_WARP) {
        cudaError_t e = vec ? launch_warp<SUB, 4>(ctx, pl, a, b, s, cout, m, batch, st)
                            : launch_warp<SUB, 1>(ctx, pl, a, b, s, cout, m, batch, st);
        return e == cudaSuccess ? DOT_OK : DOT_ECUDA;
    }
    return vec ? launch_tile<SUB, 4>(ctx, pl, a, b, s, cout, m, batch, st)
               : launch_tile<SUB, 1>(ctx, pl, a, b, s, cout, m, batch, st);
}

template <bool SUB>
static dot_status_t addsub_ragged(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *s,
                                  uint32_t *cout, const uint64_t *off, size_t batch, cudaStream_t st)
{
    DeviceScope scope;
    dot_status_t rc = dot_check_ctx(ctx, scope);
    if (rc != DOT_OK) return rc;
    if (batch == 0) return DOT_OK;
    if (!a || !b || !s || !cout || !off) return DOT_EINVAL;
    const void *fn = (const void *)addsub_ragged_kernel<SUB>;
    const size_t cap = (size_t)ctx->num_sms * dot_blocks_per_sm(fn, WARP_KERNEL_THREADS, 0);
    const size_t need = dot_ceil_div(batch, WARP_KERNEL_THREADS / 32);
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    addsub_ragged_kernel<SUB><<<grid, WARP_KERNEL_THREADS, 0, st>>>(a, b, s, cout, off, batch, ctx->d_status);
    return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
}

template <bool SUB>
static dot_status_t addsub_general(dot_ctx_t ctx, const uint32_t *a, size_t ma, const uint32_t *b, size_t mb,
                                   const uint32_t *cin, uint32_t *s, uint32_t *cout, size_t batch, cudaStream_t st)
{
    DeviceScope scope;
    dot_status_t rc = dot_check_ctx(ctx, scope);
    if (rc != DOT_OK) return rc;
    if (batch == 0) return DOT_OK;
    if (mb > ma || !cout) return DOT_EINVAL;
    if ((ma && (!a || !s)) || (mb && !b)) return DOT_EINVAL;
    if (ma > SIZE_MAX / 4 / batch) return DOT_EINVAL;
    const size_t abytes = ma * batch * 4, bbytes = mb * batch * 4, cbytes = batch * 4;
    // s may be a exactly; s may be b exactly only when the rows have the same stride
    if (partial_overlap(s, abytes, a, abytes) || (mb != ma ? any_overlap(s, abytes, b, bbytes)
                                                           : partial_overlap(s, abytes, b, bbytes)))
        return DOT_EINVAL;
    if (any_overlap(cout, cbytes, s, abytes) || any_overlap(cout, cbytes, a, abytes) ||
        any_overlap(cout, cbytes, b, bbytes))
        return DOT_EINVAL;
    const void *fn = (const void *)addsub_general_kernel<SUB>;
    const size_t cap = (size_t)ctx->num_sms * dot_blocks_per_sm(fn, WARP_KERNEL_THREADS, 0);
    const size_t need = dot_ceil_div(batch, WARP_KERNEL_THREADS / 32);
    const unsigned grid = (unsigned)(need < cap ? need : cap);
    addsub_general_kernel<SUB><<<grid, WARP_KERNEL_THREADS, 0, st>>>(a, b, cin, s, cout, ma, mb, batch);
    return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
}

extern "C" {

DOT_API dot_status_t dot_add(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *s,
                             uint32_t *carry_out, size_t m, size_t batch, dot_stream_t stream)
{
    return addsub_batched<false>(ctx, a, b, s, carry_out, m, batch, (cudaStream_t)stream);
}

DOT_API dot_status_t dot_sub(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *d,
                             uint32_t *borrow_out, size_t m, size_t batch, dot_stream_t stream)
{
    return addsub_batched<true>(ctx, a, b, d, borrow_out, m, batch, (cudaStream_t)stream);
}

DOT_API dot_status_t dot_add_ragged(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *s,
                                    uint32_t *carry_out, const uint64_t *off, size_t batch,
                                    dot_stream_t stream)
{
    return addsub_ragged<false>(ctx, a, b, s, carry_out, off, batch, (cudaStream_t)stream);
}

DOT_API dot_status_t dot_sub_ragged(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *d,
                                    uint32_t *borrow_out, const uint64_t *off, size_t batch,
                                    dot_stream_t stream)
{
    return addsub_ragged<true>(ctx, a, b, d, borrow_out, off, batch, (cudaStream_t)stream);
}

DOT_API dot_status_t dot_add_nc(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, const uint32_t *carry_in,
                                uint32_t *s, uint32_t *carry_out, size_t m, size_t batch, dot_stream_t stream)
{
    if (!carry_in && batch) return DOT_EINVAL;
    return addsub_general<false>(ctx, a, m, b, m, carry_in, s, carry_out, batch, (cudaStream_t)stream);
}

DOT_API dot_status_t dot_sub_nc(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, const uint32_t *borrow_in,
                                uint32_t *d, uint32_t *borrow_out, size_t m, size_t batch, dot_stream_t stream)
{
    if (!borrow_in && batch) return DOT_EINVAL;
    return addsub_general<true>(ctx, a, m, b, m, borrow_in, d, borrow_out, batch, (cudaStream_t)stream);
}

DOT_API dot_status_t dot_add_1(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *s,
                               uint32_t *carry_out, size_t m, size_t batch, dot_stream_t stream)
{
    if (m == 0 && batch) return DOT_EINVAL;
    return addsub_general<false>(ctx, a, m, b, 1, nullptr, s, carry_out, batch, (cudaStream_t)stream);
}

DOT_API dot_status_t dot_sub_1(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *d,
                               uint32_t *borrow_out, size_t m, size_t batch, dot_stream_t stream)
{
    if (m == 0 && batch) return DOT_EINVAL;
    return addsub_general<true>(ctx, a, m, b, 1, nullptr, d, borrow_out, batch, (cudaStream_t)stream);
}

DOT_API dot_status_t dot_add_unequal(dot_ctx_t ctx, const uint32_t *a, size_t ma, const uint32_t *b, size_t mb,
                                     uint32_t *s, uint32_t *carry_out, size_t batch, dot_stream_t stream)
{
    return addsub_general<false>(ctx, a, ma, b, mb, nullptr, s, carry_out, batch, (cudaStream_t)stream);
}

DOT_API dot_status_t dot_sub_unequal(dot_ctx_t ctx, const uint32_t *a, size_t ma, const uint32_t *b, size_t mb,
                                     uint32_t *d, uint32_t *borrow_out, size_t batch, dot_stream_t stream)
{
    return addsub_general<true>(ctx, a, ma, b, mb, nullptr, d, borrow_out, batch, (cudaStream_t)stream);
}

}  // extern "C"

// ====================================================== allocation-free add
// dot_add_noalloc: the same addition as dot_add, for callers that cannot call
// cudaMalloc at all -- code running where the allocator is off limits (inside
// another allocator's callback, a signal or real-time path that may not block
// on the driver's memory manager, or a host that has handed all device memory
// to a pool it does not share).  It needs no dot_ctx_t (creating one
// allocates).  The look-back scratch of the tiled kernel lives instead in the
// fixed device array below, which every GPU that loads this library holds
// until the process exits.
#define DOT_NOALLOC_HDR 4          // [0] tile ticket, [1] blocks done, [2] epoch, [3] status word
#define DOT_NOALLOC_MAX_TILES 16384
#define DOT_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned long long
    g_noalloc_scratch[DOT_NOALLOC_HDR + DOT_NOALLOC_MAX_TILES];

// Device address of g_noalloc_scratch and the SM count, looked up once per
// device and published for every host thread: a reader that sees the address
// (acquire) also sees the SM count written before it (release); the lookup
// itself runs under a lock, so concurrent first calls look it up once.
static std::atomic<unsigned long long *> g_noalloc_addr[DOT_NOALLOC_MAX_DEVICES];
static int g_noalloc_sms[DOT_NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_lock;

// The caller has made `device` current.
static dot_status_t noalloc_setup(int device, unsigned long long **addr, int *sms)
{
    unsigned long long *p = g_noalloc_addr[device].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> guard(g_noalloc_lock);
        p = g_noalloc_addr[device].load(std::memory_order_relaxed);
        if (!p) {
            void *sym = nullptr;
            int n = 0;
            if (cudaGetSymbolAddress(&sym, g_noalloc_scratch) != cudaSuccess || !sym) return DOT_ECUDA;
            if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n < 1)
                return DOT_ECUDA;
            g_noalloc_sms[device] = n;
            p = (unsigned long long *)sym;
            g_noalloc_addr[device].store(p, std::memory_order_release);
        }
    }
    *addr = p;
    *sms = g_noalloc_sms[device];
    return DOT_OK;
}

template <bool SUB, int SEG>
static dot_status_t noalloc_launch(int sms, unsigned long long *scratch, const dot_plan_t &pl,
                                   const uint32_t *a, const uint32_t *b, uint32_t *s, uint32_t *cout,
                                   size_t m, size_t batch, cudaStream_t st)
{
    if (pl.kernel == DOT_K_ADDSUB_WARP) {
        const int lpo = pl.lanes_per_op, nch = pl.chunks, opw = 32 / lpo;
        const int U = (nch == 1) ? 4 : 1;
        const size_t need = dot_ceil_div(dot_ceil_div(batch, (size_t)opw * U), WARP_KERNEL_THREADS / 32);
        const void *fn = nch == 1 ? (const void *)addsub_warp_kernel<SUB, SEG, 1, 4>
                       : nch == 2 ? (const void *)addsub_warp_kernel<SUB, SEG, 2, 1>
                                  : (const void *)addsub_warp_kernel<SUB, SEG, 4, 1>;
        const size_t cap = (size_t)sms * dot_blocks_per_sm(fn, WARP_KERNEL_THREADS, 0);
        const unsigned grid = (unsigned)(need < cap ? need : cap);
        if (nch == 1)
            addsub_warp_kernel<SUB, SEG, 1, 4><<<grid, WARP_KERNEL_THREADS, 0, st>>>(a, b, s, cout, m, batch, lpo, nch);
        else if (nch == 2)
            addsub_warp_kernel<SUB, SEG, 2, 1><<<grid, WARP_KERNEL_THREADS, 0, st>>>(a, b, s, cout, m, batch, lpo, nch);
        else
            addsub_warp_kernel<SUB, SEG, 4, 1><<<grid, WARP_KERNEL_THREADS, 0, st>>>(a, b, s, cout, m, batch, lpo, nch);
        return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
    }
    const size_t tiles = (size_t)pl.tiles * batch;
    // the counters, epoch, status and this call's tile states must start at zero
    if (cudaMemsetAsync(scratch, 0, (DOT_NOALLOC_HDR + tiles) * sizeof(unsigned long long), st) != cudaSuccess)
        return DOT_ECUDA;
    LookbackArgs lb;
    lb.counters = scratch;
    lb.status = (uint32_t *)(scratch + 3);
    lb.state = scratch + DOT_NOALLOC_HDR;
    lb.wait_limit_ns = 2000000000ull;
    lb.skip_tile = -1;
    const void *fn = pl.chunks == 1 ? (const void *)addsub_tile_kernel<SUB, SEG, 1>
                   : pl.chunks == 2 ? (const void *)addsub_tile_kernel<SUB, SEG, 2>
                                    : (const void *)addsub_tile_kernel<SUB, SEG, 4>;
    const size_t cap = (size_t)sms * dot_blocks_per_sm(fn, DOT_TILE_THREADS, 0);
    const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
    const unsigned long long tpo = pl.tiles;
    if (pl.chunks == 1)
        addsub_tile_kernel<SUB, SEG, 1><<<grid, DOT_TILE_THREADS, 0, st>>>(a, b, s, cout, m, batch, tpo, lb);
    else if (pl.chunks == 2)
        addsub_tile_kernel<SUB, SEG, 2><<<grid, DOT_TILE_THREADS, 0, st>>>(a, b, s, cout, m, batch, tpo, lb);
    else
        addsub_tile_kernel<SUB, SEG, 4><<<grid, DOT_TILE_THREADS, 0, st>>>(a, b, s, cout, m, batch, tpo, lb);
    return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
}

extern "C" DOT_API dot_status_t dot_add_noalloc(int device, const uint32_t *a, const uint32_t *b, uint32_t *s,
                                                uint32_t *carry_out, size_t m, size_t batch, dot_stream_t stream)
{
    if (device < 0 || device >= DOT_NOALLOC_MAX_DEVICES) return DOT_EINVAL;
    if (batch == 0) return DOT_OK;
    if (!carry_out || (m && (!a || !b || !s))) return DOT_EINVAL;
    if (m > SIZE_MAX / 4 / batch) return DOT_EINVAL;
    const size_t bytes = m * batch * 4;
    if (partial_overlap(s, bytes, a, bytes) || partial_overlap(s, bytes, b, bytes)) return DOT_EINVAL;
    if (any_overlap(carry_out, batch * 4, s, bytes) || any_overlap(carry_out, batch * 4, a, bytes) ||
        any_overlap(carry_out, batch * 4, b, bytes))
        return DOT_EINVAL;
    const bool vec = (m % 4 == 0) && aligned16(a) && aligned16(b) && aligned16(s);
    dot_plan_t pl;
    dot_status_t rc = dot_make_plan(DOT_OP_ADD, m, batch, vec, &pl);
    if (rc != DOT_OK) return rc;
    if (pl.kernel == DOT_K_ADDSUB_TILE && (pl.tiles > DOT_NOALLOC_MAX_TILES ||
                                           batch > DOT_NOALLOC_MAX_TILES / pl.tiles))
        return DOT_EUNSUPPORTED;   // more tiles than the fixed scratch array holds
    // the caller's device is put back on every return path
    DeviceScope scope;
    if (scope.enter(device) != DOT_OK) return DOT_ECUDA;
    unsigned long long *scratch = nullptr;
    int sms = 0;
    rc = noalloc_setup(device, &scratch, &sms);
    if (rc != DOT_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (m == 0) return cudaMemsetAsync(carry_out, 0, batch * 4, st) == cudaSuccess ? DOT_OK : DOT_ECUDA;
    return vec ? noalloc_launch<false, 4>(sms, scratch, pl, a, b, s, carry_out, m, batch, st)
               : noalloc_launch<false, 1>(sms, scratch, pl, a, b, s, carry_out, m, batch, st);
}
