// BF16 / FP8 convolutions on tcgen05 tensor cores.
#include "conv.cuh"

namespace pgi {

pg_status tc_prepare(pg_ctx *, Net *, pg_precision) { return PG_ERR_UNSUPPORTED; }

pg_status forward_tc(pg_ctx *, const Net *, pg_precision, const float *, void *, uint32_t, int, int, float *,
                     cudaStream_t) {
  return PG_ERR_UNSUPPORTED;
}

}  // namespace pgi
