// dot_tune.cu -- per-context tuning table and the autotuner.
//
// The tuned shapes are the ones the kernels take as template parameters:
// the columns per block R of the multiply (4, 8, 12, 16) and the segments per
// thread of the tiled look-back add/sub (1, 2, 4, i.e. 1024 to 4096-limb
// tiles).  A context keeps one choice per (op, bit length of m); the
// autotuner times every valid candidate on synthetic operands of the asked
// shape and keeps the fastest.  The table lives in the context; the Python
// layer persists it per GPU model and SM count.
#include "dot_internal.cuh"
#include "dot_plan.h"

// x[i] = 32 random bits from a counter hash (splitmix64 finaliser of i ^ seed)
__global__ void tune_fill_kernel(uint32_t *x, size_t n, uint64_t seed)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint64_t z = (uint64_t)i ^ seed;
        z += 0x9e3779b97f4a7c15ull;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        x[i] = (uint32_t)(z ^ (z >> 31));
    }
}

static int candidates(int op, size_t m, size_t batch, int *out)
{
    int n = 0;
    if (op == DOT_OP_MUL) {
        const int rs[4] = {4, 8, 12, 16};
        for (int r : rs)
            if (dot_knob_valid(op, m, r)) out[n++] = r;
        return n;
    }
    // only the tiled look-back kernel has a shape to choose
    dot_plan_t pl;
    if (dot_make_plan(op, m, batch, true, &pl) != DOT_OK || pl.kernel != DOT_K_ADDSUB_TILE) return 0;
    out[n++] = 1;
    out[n++] = 2;
    out[n++] = 4;
    return n;
}

extern "C" {

DOT_API dot_status_t dot_tune_set(dot_ctx_t ctx, int op, size_t m, int value)
{
    if (!ctx || op < DOT_OP_ADD || op > DOT_OP_MUL || m == 0) return DOT_EINVAL;
    if (value != 0 && !dot_knob_valid(op, m, value)) return DOT_EINVAL;
    ctx->tune[op][dot_tune_bucket(m)] = (unsigned char)value;
    return DOT_OK;
}

DOT_API dot_status_t dot_tune_get(dot_ctx_t ctx, int op, size_t m, int *value)
{
    if (!ctx || !value || op < DOT_OP_ADD || op > DOT_OP_MUL) return DOT_EINVAL;
    *value = ctx->tune[op][dot_tune_bucket(m)];
    return DOT_OK;
}

DOT_API dot_status_t dot_autotune(dot_ctx_t ctx, int op, size_t m, size_t batch, int *best, float *best_ms)
{
    DeviceScope scope;
    dot_status_t rc = dot_check_ctx(ctx, scope);
    if (rc != DOT_OK) return rc;
    if (!best || op < DOT_OP_ADD || op > DOT_OP_MUL || m == 0 || batch == 0) return DOT_EINVAL;
    if (m > SIZE_MAX / 16 / batch) return DOT_EINVAL;
    int cand[4];
    const int nc = candidates(op, m, batch, cand);
    *best = 0;
    if (best_ms) *best_ms = 0.f;
    if (nc == 0) return DOT_OK;   // nothing to choose for this size
    const size_t n = m * batch;
    const size_t out_limbs = op == DOT_OP_MUL ? 2 * n : n;
    uint32_t *a = nullptr, *b = nullptr, *r = nullptr, *c = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = ctx->side[0];
    const int bucket = dot_tune_bucket(m);
    const unsigned char saved = ctx->tune[op][bucket];
    int chosen = 0;
    float chosen_ms = 0.f;
    if (cudaMalloc((void **)&a, n * 4) != cudaSuccess || cudaMalloc((void **)&b, n * 4) != cudaSuccess ||
        cudaMalloc((void **)&r, out_limbs * 4) != cudaSuccess || cudaMalloc((void **)&c, batch * 4) != cudaSuccess) {
        rc = DOT_ENOMEM;
        goto done;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = DOT_ECUDA;
        goto done;
    }
    tune_fill_kernel<<<ctx->num_sms * 4, 256, 0, st>>>(a, n, 0x1234ull);
    tune_fill_kernel<<<ctx->num_sms * 4, 256, 0, st>>>(b, n, 0x5678ull);
    for (int k = 0; k < nc; ++k) {
        ctx->tune[op][bucket] = (unsigned char)cand[k];
        float ms = 0.f;
        for (int rep = 0; rep < 2 + 5 && rc == DOT_OK; ++rep) {
            if (rep == 2 && cudaEventRecord(e0, st) != cudaSuccess) rc = DOT_ECUDA;
            if (rc != DOT_OK) break;
            rc = op == DOT_OP_MUL ? dot_mul(ctx, a, b, r, m, batch, st)
               : op == DOT_OP_ADD ? dot_add(ctx, a, b, r, c, m, batch, st)
                                  : dot_sub(ctx, a, b, r, c, m, batch, st);
        }
        if (rc != DOT_OK) break;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = DOT_ECUDA;
            break;
        }
        ms /= 5.f;
        if (chosen == 0 || ms < chosen_ms) {
            chosen = cand[k];
            chosen_ms = ms;
        }
    }
done:
    if (rc == DOT_OK) {
        ctx->tune[op][bucket] = (unsigned char)chosen;
        *best = chosen;
        if (best_ms) *best_ms = chosen_ms;
        // a candidate that hit a device-side error shows in the sticky status
        rc = dot_ctx_check(ctx, st);
    } else {
        ctx->tune[op][bucket] = saved;
    }
    cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(a);
    cudaFree(b);
    cudaFree(r);
    cudaFree(c);
    return rc;
}

}  // extern "C"
