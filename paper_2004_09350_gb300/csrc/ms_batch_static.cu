// ms_batch_static.cu -- batched fragment kernels with the static per-CTA and the
// CTA-streamed schedules.
#include "ms_batch.cuh"

namespace ms {
#define MS_NONE
MS_BATCH_STATIC(MS_NONE)
MS_BATCH_CTA(MS_NONE)
#undef MS_NONE
}  // namespace ms
