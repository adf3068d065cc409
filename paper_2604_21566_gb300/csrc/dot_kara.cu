// dot_kara.cu -- batched Karatsuba multiplication above the base-case size.
//
// The appendix's MPN-KARATSUBA (Karatsuba, or Toom-Cook 2-way; Sec. 2 notes
// that such recursions end in the same schoolbook base case that the column
// sums implement): with A = A_H b + A_L, B = B_H b + B_L, b = X^h,
//     P1 = A_H B_H,  P0 = A_L B_L,  P_D = |A_H - A_L| |B_H - B_L|,
//     P2 = sign(A_H - A_L) sign(B_H - B_L) P_D,
//     A B = P1 b^2 + (P1 + P0 - P2) b + P0.
// Every operation of a level is batched over all operations of the call:
//   * kara_split_kernel (one warp per op) writes A_L, A_H, |A_H - A_L| and the
//     same for B into three consecutive row blocks of a workspace, with the
//     sign of P2 per op: the comparison walks down from the top limb (it
//     almost always ends at the first), then one subtraction in the right
//     order with the warp lookahead;
//   * the three half-size products run as ONE batched product over 3x the
//     ops (the column-sum multiply at h <= KARA_BASE_LIMBS, else the next
//     level of this recursion);
//   * kara_combine_kernel (one warp per op) forms Q = P1 + P0 -/+ P_D
//     (2h limbs and a top word), then P = (P0 || P1) + Q b with the same
//     lookahead -- the additions and subtractions the paper notes multiply
//     with the recursion depth run on the add path.
// Odd m splits at h = ceil(m / 2); A_H and B_H are zero-padded to h limbs.
//
// Base case: up to 384 limbs, although dot_mul takes 512.  Between 385 and
// 512 limbs the column-sum multiply needs 16 columns per lane, the slowest of
// its shapes (5.4e12 limb products/s against 6.0e12-6.5e12 with 8 or 12), and
// one more level replaces each such product by three of at most 256 limbs
// (3/4 of the products) for some memory-bound split and combine work.
#include <string.h>

#include "dot_internal.cuh"
#include "dot_plan.h"
#include "dot_warp_op.cuh"

#define KARA_THREADS 256   // 8 warps, one op each
#define KARA_BASE_LIMBS 384

// The sign-and-magnitude difference |x - y| of two h-limb rows (x, y read
// through lx, ly), written through st; returns 1 when x < y.
template <typename LX, typename LY, typename ST>
__device__ __forceinline__ uint32_t kara_absdiff(LX lx, LY ly, ST st, size_t h)
{
    // most significant differing limb: chunks of 32 limbs from the top
    const int lane = (int)lane_id();
    uint32_t less = 0;
    for (size_t top = h; top > 0;) {
        const size_t n = top < 32 ? top : 32;
        const size_t i = top - 1 - (size_t)lane;   // lane 0 holds the highest limb of the chunk
        uint32_t xi = 0, yi = 0;
        if ((size_t)lane < n) {
            xi = lx(i);
            yi = ly(i);
        }
        const uint32_t diff = __ballot_sync(DOT_FULL, (size_t)lane < n && xi != yi);
        if (diff) {
            const int l = __ffs(diff) - 1;
            less = __shfl_sync(DOT_FULL, (uint32_t)(xi < yi), l);
            break;
        }
        top -= n;
    }
    if (less)
        addsub_warp_run<true>(ly, lx, st, h, 0u);
    else
        addsub_warp_run<true>(lx, ly, st, h, 0u);
    return less;
}

// a, b: [batch][m]; wa, wb: [3 batch][h] = rows A_L, then A_H, then |A_H - A_L|
// (B likewise); neg[k] = 1 when P2 < 0 (the differences have opposite signs).
__global__ void __launch_bounds__(KARA_THREADS)
kara_split_kernel(const uint32_t *a, const uint32_t *b, uint32_t *wa, uint32_t *wb, uint32_t *neg, size_t m,
                  size_t h, size_t batch)
{
    const size_t warp_global = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const int lane = (int)lane_id();
    const size_t mh = m - h;   // limbs of the high halves (<= h)
    for (size_t op = warp_global; op < batch; op += nwarps) {
        uint32_t s[2];
        for (int t = 0; t < 2; ++t) {
            const uint32_t *x = (t ? b : a) + op * m;
            uint32_t *w = t ? wb : wa;
            uint32_t *lo = w + op * h, *hi = w + (batch + op) * h, *df = w + (2 * batch + op) * h;
            for (size_t i = lane; i < h; i += 32) {
                lo[i] = ld_stream1(x + i);
                hi[i] = i < mh ? ld_stream1(x + h + i) : 0u;
            }
            // the halves just written are re-read from L2 by this warp
            __syncwarp();
            s[t] = kara_absdiff([=](size_t i) { return hi[i]; }, [=](size_t i) { return lo[i]; },
                                [=](size_t i, uint32_t v) { df[i] = v; }, h);
        }
        if (lane == 0) neg[op] = s[0] ^ s[1];
    }
}

// z: [3 batch][2h] = P0, P1, P_D rows; q: [batch][2h] scratch; p: [batch][2m].
// P = (P0 || P1) + (P1 + P0 -/+ P_D) X^h, exact in 2m limbs.
__global__ void __launch_bounds__(KARA_THREADS)
kara_combine_kernel(const uint32_t *z, const uint32_t *neg, uint32_t *q, uint32_t *p, size_t m, size_t h,
                    size_t batch)
{
    const size_t warp_global = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const size_t hh = 2 * h, mm = 2 * m;
    for (size_t op = warp_global; op < batch; op += nwarps) {
        const uint32_t *p0 = z + op * hh, *p1 = z + (batch + op) * hh, *pd = z + (2 * batch + op) * hh;
        uint32_t *qr = q + op * hh;
        uint32_t *pr = p + op * mm;
        // Q = P0 + P1 (top carry c1), then Q -/+ P_D (carry or borrow c2)
        const uint32_t c1 = addsub_warp_run<false>([=](size_t i) { return ld_stream1(p0 + i); },
                                                   [=](size_t i) { return ld_stream1(p1 + i); },
                                                   [=](size_t i, uint32_t v) { qr[i] = v; }, hh, 0u);
        __syncwarp();
        uint32_t top;
        if (neg[op]) {
            const uint32_t c2 = addsub_warp_run<false>([=](size_t i) { return qr[i]; },
                                                       [=](size_t i) { return ld_stream1(pd + i); },
                                                       [=](size_t i, uint32_t v) { qr[i] = v; }, hh, 0u);
            top = c1 + c2;
        } else {
            const uint32_t c2 = addsub_warp_run<true>([=](size_t i) { return qr[i]; },
                                                      [=](size_t i) { return ld_stream1(pd + i); },
                                                      [=](size_t i, uint32_t v) { qr[i] = v; }, hh, 0u);
            top = c1 - c2;   // the middle coefficient is nonnegative: never wraps
        }
        __syncwarp();
        // P = (P0 || P1) + (Q || top) X^h over 2m limbs (the carry out is 0)
        addsub_warp_run<false>(
            [=](size_t i) { return i < hh ? ld_stream1(p0 + i) : ld_stream1(p1 + (i - hh)); },
            [=](size_t i) { return i < h ? 0u : (i - h < hh ? qr[i - h] : (i - h == hh ? top : 0u)); },
            [=](size_t i, uint32_t v) { st_stream1(pr + i, v); }, mm, 0u);
    }
}

// Workspace words of one call on `batch` ops of m limbs (the levels below
// included): 3 batch h for each of wa and wb, 6 batch h for the three
// half-size products, 2 batch h for Q, batch for the signs.
static size_t kara_work_words(size_t m, size_t batch)
{
    if (m <= KARA_BASE_LIMBS) return 0;
    const size_t h = (m + 1) / 2;
    return 14 * batch * h + batch + 4 + kara_work_words(h, 3 * batch);
}

static unsigned kara_grid(dot_ctx_t ctx, const void *fn, size_t batch)
{
    const size_t need = dot_ceil_div(batch, (size_t)(KARA_THREADS / 32));
    const size_t cap = (size_t)ctx->num_sms * dot_blocks_per_sm(fn, KARA_THREADS, 0);
    return (unsigned)(need < cap ? need : cap);
}

static dot_status_t kara(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *p, size_t m, size_t batch,
                         uint32_t *work, cudaStream_t st)
{
    if (m <= KARA_BASE_LIMBS) return dot_mul(ctx, a, b, p, m, batch, (dot_stream_t)st);
    const size_t h = (m + 1) / 2;
    uint32_t *wa = work, *wb = wa + 3 * batch * h, *z = wb + 3 * batch * h, *q = z + 6 * batch * h;
    uint32_t *neg = q + 2 * batch * h;
    uint32_t *next = neg + batch;
    next += (4 - ((uintptr_t)next / 4) % 4) % 4;   // 16-byte alignment for the level below
    kara_split_kernel<<<kara_grid(ctx, (const void *)kara_split_kernel, batch), KARA_THREADS, 0, st>>>(
        a, b, wa, wb, neg, m, h, batch);
    if (cudaGetLastError() != cudaSuccess) return DOT_ECUDA;
    dot_status_t rc = kara(ctx, wa, wb, z, h, 3 * batch, next, st);
    if (rc != DOT_OK) return rc;
    kara_combine_kernel<<<kara_grid(ctx, (const void *)kara_combine_kernel, batch), KARA_THREADS, 0, st>>>(
        z, neg, q, p, m, h, batch);
    return cudaGetLastError() == cudaSuccess ? DOT_OK : DOT_ECUDA;
}

extern "C" {

DOT_API dot_status_t dot_mul_karatsuba(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *p,
                                       size_t m, size_t batch, dot_stream_t stream)
{
    DeviceScope scope;
    dot_status_t rc = dot_check_ctx(ctx, scope);
    if (rc != DOT_OK) return rc;
    if (batch == 0 || m == 0) return DOT_OK;
    if (!a || !b || !p) return DOT_EINVAL;
    if (m > DOT_KARA_MAX_LIMBS || batch > SIZE_MAX / 64 / m) return DOT_EINVAL;
    const size_t in = m * batch * 4, out = 2 * in;
    if (any_overlap(p, out, a, in) || any_overlap(p, out, b, in)) return DOT_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (m <= KARA_BASE_LIMBS) return dot_mul(ctx, a, b, p, m, batch, stream);
    uint32_t *work = nullptr;
    rc = dot_work(ctx, kara_work_words(m, batch) * 4, (void **)&work);
    if (rc != DOT_OK) return rc;
    return kara(ctx, a, b, p, m, batch, work, st);
}

}  // extern "C"
