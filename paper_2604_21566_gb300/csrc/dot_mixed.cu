// dot_mixed.cu -- mixed ragged batches of add / sub / mul descriptors.
#include "dot_internal.cuh"
#include "dot_plan.h"

extern "C" {

DOT_API dot_status_t dot_mixed_ragged(dot_ctx_t ctx, const dot_desc_t *desc, size_t nops,
                                      const uint32_t *a, const uint32_t *b, uint32_t *r,
                                      uint32_t *carry, dot_stream_t stream)
{
    (void)desc; (void)a; (void)b; (void)r; (void)carry; (void)stream;
    dot_status_t rc = dot_check_ctx(ctx);
    if (rc != DOT_OK) return rc;
    if (nops == 0) return DOT_OK;
    return DOT_EUNSUPPORTED;
}

}  // extern "C"
