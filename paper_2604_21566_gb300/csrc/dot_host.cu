// dot_host.cu -- host-buffer entry points: copy in, compute, copy out,
// chunk by chunk through two staging buffers.  Copies in run on one stream,
// the kernels on the caller's stream (in chunk order: they share the ctx
// look-back scratch) and copies out on another, ordered per buffer by events:
// a buffer's next copy-in waits only for the kernel that read it, and its next
// kernel for the copy-out of its previous results.  So the host-to-device
// direction keeps streaming while results flow back.
#include "dot_internal.cuh"
#include "dot_plan.h"

// Staged bytes per chunk (one of two staging buffers).  A call's first
// copy-in and its last copy-out overlap nothing, so chunks are kept small
// enough for that fill and drain to stay short (32 MB: about 0.1 ms of the
// link each), and large enough that a chunk's kernel is negligible next to
// its copies.
#define STAGE_BYTES_PER_BUFFER (32u << 20)

static dot_status_t ensure_stage(dot_ctx_t c, size_t bytes)
{
    if (c->stage_bytes >= bytes) return DOT_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return DOT_ECUDA;
    if (c->d_stage) cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_bytes = 0;
    if (cudaMalloc(&c->d_stage, bytes) != cudaSuccess) return DOT_ENOMEM;
    c->stage_bytes = bytes;
    return DOT_OK;
}

static size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }

// op: DOT_OP_ADD / SUB / MUL
static dot_status_t host_run(dot_ctx_t c, int op, const uint32_t *a, const uint32_t *b, uint32_t *r,
                             uint32_t *cout, size_t m, size_t batch, cudaStream_t user)
{
    DeviceScope scope;
    dot_status_t rc = dot_check_ctx(c, scope);
    if (rc != DOT_OK) return rc;
    if (batch == 0) return DOT_OK;
    const bool mul = op == DOT_OP_MUL;
    if (mul && m == 0) return DOT_OK;
    if (mul && m > DOT_MUL_MAX_LIMBS) return DOT_EUNSUPPORTED;
    if ((!mul && !cout) || (m && (!a || !b || !r))) return DOT_EINVAL;
    if (m > SIZE_MAX / 16 / batch) return DOT_EINVAL;
    const size_t rl = mul ? 2 * m : m;                        // result limbs per op
    const size_t per_op = 4 * (2 * m + rl) + (mul ? 0 : 4);   // staged bytes per op
    size_t chunk = STAGE_BYTES_PER_BUFFER / (per_op ? per_op : 4);
    if (chunk == 0) chunk = 1;
    if (chunk > batch) chunk = batch;
    const size_t a_bytes = round16(chunk * m * 4), r_bytes = round16(chunk * rl * 4);
    const size_t c_bytes = round16(chunk * 4);
    const size_t buf_bytes = 2 * a_bytes + r_bytes + c_bytes;
    rc = ensure_stage(c, 2 * buf_bytes);
    if (rc != DOT_OK) return rc;

    cudaStream_t in = c->side[0], out = c->side[1];
    cudaEvent_t *ev_in = c->ev, *ev_kern = c->ev + 2, *ev_out = c->ev + 4;
    // both copy streams start after the caller's earlier work
    if (cudaEventRecord(c->ev[6], user) != cudaSuccess || cudaStreamWaitEvent(in, c->ev[6], 0) != cudaSuccess ||
        cudaStreamWaitEvent(out, c->ev[6], 0) != cudaSuccess)
        return DOT_ECUDA;
    size_t k = 0;
    for (size_t lo = 0; lo < batch; lo += chunk, ++k) {
        const int j = (int)(k & 1);   // staging buffer
        const size_t n = (batch - lo < chunk) ? batch - lo : chunk;
        char *base = (char *)c->d_stage + j * buf_bytes;
        uint32_t *da = (uint32_t *)base, *db = (uint32_t *)(base + a_bytes);
        uint32_t *dr = (uint32_t *)(base + 2 * a_bytes), *dc = (uint32_t *)(base + 2 * a_bytes + r_bytes);
        // copy in once the buffer's previous inputs have been consumed
        if (k >= 2 && cudaStreamWaitEvent(in, ev_kern[j], 0) != cudaSuccess) return DOT_ECUDA;
        if (m) {
            if (cudaMemcpyAsync(da, a + lo * m, n * m * 4, cudaMemcpyHostToDevice, in) != cudaSuccess ||
                cudaMemcpyAsync(db, b + lo * m, n * m * 4, cudaMemcpyHostToDevice, in) != cudaSuccess)
                return DOT_ECUDA;
        }
        if (cudaEventRecord(ev_in[j], in) != cudaSuccess) return DOT_ECUDA;
        // compute once the inputs are in and the buffer's previous results are out
        if (cudaStreamWaitEvent(user, ev_in[j], 0) != cudaSuccess) return DOT_ECUDA;
        if (k >= 2 && cudaStreamWaitEvent(user, ev_out[j], 0) != cudaSuccess) return DOT_ECUDA;
        switch (op) {
        case DOT_OP_ADD: rc = dot_add(c, da, db, dr, dc, m, n, user); break;
        case DOT_OP_SUB: rc = dot_sub(c, da, db, dr, dc, m, n, user); break;
        default: rc = dot_mul(c, da, db, dr, m, n, user); break;
        }
        if (rc != DOT_OK) return rc;
        if (cudaEventRecord(ev_kern[j], user) != cudaSuccess) return DOT_ECUDA;
        // copy out
        if (cudaStreamWaitEvent(out, ev_kern[j], 0) != cudaSuccess) return DOT_ECUDA;
        if (rl && cudaMemcpyAsync(r + lo * rl, dr, n * rl * 4, cudaMemcpyDeviceToHost, out) != cudaSuccess)
            return DOT_ECUDA;
        if (!mul && cudaMemcpyAsync(cout + lo, dc, n * 4, cudaMemcpyDeviceToHost, out) != cudaSuccess)
            return DOT_ECUDA;
        if (cudaEventRecord(ev_out[j], out) != cudaSuccess) return DOT_ECUDA;
    }
    // the caller's later work sees every result on the host
    if (cudaEventRecord(c->ev[7], out) != cudaSuccess || cudaStreamWaitEvent(user, c->ev[7], 0) != cudaSuccess)
        return DOT_ECUDA;
    return DOT_OK;
}

extern "C" {

DOT_API dot_status_t dot_add_host(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *s,
                                  uint32_t *carry_out, size_t m, size_t batch, dot_stream_t stream)
{
    return host_run(ctx, DOT_OP_ADD, a, b, s, carry_out, m, batch, (cudaStream_t)stream);
}

DOT_API dot_status_t dot_sub_host(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *d,
                                  uint32_t *borrow_out, size_t m, size_t batch, dot_stream_t stream)
{
    return host_run(ctx, DOT_OP_SUB, a, b, d, borrow_out, m, batch, (cudaStream_t)stream);
}

DOT_API dot_status_t dot_mul_host(dot_ctx_t ctx, const uint32_t *a, const uint32_t *b, uint32_t *p,
                                  size_t m, size_t batch, dot_stream_t stream)
{
    return host_run(ctx, DOT_OP_MUL, a, b, p, nullptr, m, batch, (cudaStream_t)stream);
}

}  // extern "C"
