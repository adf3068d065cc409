// dot_ctx.cu -- context lifecycle, status codes, launch planning.
#include <stdlib.h>
#include <string.h>

#include "dot_internal.cuh"
#include "dot_plan.h"

dot_status_t dot_check_ctx(dot_ctx_t ctx, DeviceScope &scope)
{
    if (!ctx) return DOT_EINVAL;
    return scope.enter(ctx->device);
}

int dot_blocks_per_sm(const void *kernel, int threads, size_t smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

extern "C" {

DOT_API int dot_abi_version(void) { return DOT_ABI_VERSION; }

DOT_API const char *dot_status_str(dot_status_t s)
{
    switch (s) {
    case DOT_OK: return "ok";
    case DOT_EINVAL: return "invalid argument";
    case DOT_ECUDA: return "CUDA error";
    case DOT_ENOMEM: return "out of device memory";
    case DOT_ETIMEOUT: return "device-side wait ran out";
    case DOT_EUNSUPPORTED: return "unsupported size or mode";
    }
    return "unknown status";
}

DOT_API dot_status_t dot_ctx_create(dot_ctx_t *out, int device)
{
    if (!out) return DOT_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return DOT_ECUDA;
    if (device < 0 || device >= ndev) return DOT_EINVAL;
    DeviceScope scope;
    if (scope.enter(device) != DOT_OK) return DOT_ECUDA;
    dot_ctx_t c = (dot_ctx_t)calloc(1, sizeof(struct dot_ctx));
    if (!c) return DOT_ENOMEM;
    c->device = device;
    c->wait_limit_ns = 2000000000ull;
    c->debug_skip_tile = -1;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        free(c);
        return DOT_ECUDA;
    }
    dot_status_t st = DOT_OK;
    if (cudaMalloc((void **)&c->d_status, 256) != cudaSuccess ||
        cudaMalloc((void **)&c->d_counters, 256) != cudaSuccess) {
        st = DOT_ENOMEM;
    } else {
        // epoch starts at 1: zeroed tile states never look published
        unsigned long long init[4] = {0ull, 0ull, 1ull, 0ull};
        if (cudaMemset(c->d_status, 0, 256) != cudaSuccess ||
            cudaMemcpy(c->d_counters, init, sizeof init, cudaMemcpyHostToDevice) != cudaSuccess)
            st = DOT_ECUDA;
    }
    if (st == DOT_OK) {
        c->tile_state_cap = 1u << 16;
        if (cudaMalloc((void **)&c->d_tile_state, c->tile_state_cap * 8) != cudaSuccess ||
            cudaMemset(c->d_tile_state, 0, c->tile_state_cap * 8) != cudaSuccess)
            st = DOT_ENOMEM;
    }
    for (int i = 0; st == DOT_OK && i < 2; ++i)
        if (cudaStreamCreateWithFlags(&c->side[i], cudaStreamNonBlocking) != cudaSuccess) st = DOT_ECUDA;
    for (int i = 0; st == DOT_OK && i < 8; ++i)
        if (cudaEventCreateWithFlags(&c->ev[i], cudaEventDisableTiming) != cudaSuccess) st = DOT_ECUDA;
    if (st != DOT_OK) {
        dot_ctx_destroy(c);
        return st;
    }
    *out = c;
    return DOT_OK;
}

DOT_API void dot_ctx_destroy(dot_ctx_t c)
{
    if (!c) return;
    DeviceScope scope;
    scope.enter(c->device);
    cudaDeviceSynchronize();
    dot_mixed_release(c);
    for (int i = 0; i < 8; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    for (int i = 0; i < 2; ++i)
        if (c->side[i]) cudaStreamDestroy(c->side[i]);
    if (c->d_stage) cudaFree(c->d_stage);
    if (c->d_work) cudaFree(c->d_work);
    if (c->d_tile_state) cudaFree(c->d_tile_state);
    if (c->d_counters) cudaFree(c->d_counters);
    if (c->d_status) cudaFree(c->d_status);
    free(c);
}

DOT_API dot_status_t dot_ctx_check(dot_ctx_t c, dot_stream_t stream)
{
    DeviceScope scope;
    dot_status_t st = dot_check_ctx(c, scope);
    if (st != DOT_OK) return st;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return DOT_ECUDA;
    uint32_t h = 0;
    if (cudaMemcpy(&h, c->d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return DOT_ECUDA;
    if (h != DOT_OK && cudaMemset(c->d_status, 0, 4) != cudaSuccess) return DOT_ECUDA;
    return (dot_status_t)h;
}

DOT_API dot_status_t dot_ctx_set_wait_limit(dot_ctx_t c, uint64_t ns)
{
    if (!c || ns == 0) return DOT_EINVAL;
    c->wait_limit_ns = ns;
    return DOT_OK;
}

DOT_API dot_status_t dot_debug_skip_publish(dot_ctx_t c, int64_t tile)
{
    if (!c || tile < -1) return DOT_EINVAL;
    c->debug_skip_tile = tile;
    return DOT_OK;
}

DOT_API dot_status_t dot_plan_batched(int op, size_t m, size_t batch, int vector_ok, dot_plan_t *out)
{
    if (!out) return DOT_EINVAL;
    return dot_make_plan(op, m, batch, vector_ok != 0, out);
}

}  // extern "C"

// Make sure the look-back state array holds `tiles` entries.  Growing it
// allocates (outside any stream capture); states are epoch-tagged, so the
// array never needs clearing between launches.
dot_status_t dot_lookback_prepare(dot_ctx_t c, size_t tiles, LookbackArgs *out)
{
    if (tiles > c->tile_state_cap) {
        size_t cap = c->tile_state_cap;
        while (cap < tiles) cap *= 2;
        unsigned long long *p = nullptr;
        if (cudaDeviceSynchronize() != cudaSuccess) return DOT_ECUDA;
        if (cudaMalloc((void **)&p, cap * 8) != cudaSuccess) return DOT_ENOMEM;
        if (cudaMemset(p, 0, cap * 8) != cudaSuccess) {
            cudaFree(p);
            return DOT_ECUDA;
        }
        cudaFree(c->d_tile_state);
        c->d_tile_state = p;
        c->tile_state_cap = cap;
    }
    out->state = c->d_tile_state;
    out->counters = c->d_counters;
    out->status = c->d_status;
    out->wait_limit_ns = c->wait_limit_ns;
    out->skip_tile = c->debug_skip_tile;
    return DOT_OK;
}

dot_status_t dot_work(dot_ctx_t c, size_t bytes, void **out)
{
    if (bytes > c->work_bytes) {
        void *p = nullptr;
        if (cudaDeviceSynchronize() != cudaSuccess) return DOT_ECUDA;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return DOT_ENOMEM;
        if (c->d_work) cudaFree(c->d_work);
        c->d_work = p;
        c->work_bytes = bytes;
    }
    *out = c->d_work;
    return DOT_OK;
}
