// ms_batch_static.cu -- batched fragment kernels with the static per-CTA schedule.
#include "ms_batch.cuh"

namespace ms {
#define MS_NONE
MS_BATCH_STATIC(MS_NONE)
#undef MS_NONE
}  // namespace ms
