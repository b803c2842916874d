// ms_batch_d4.cu -- batched fragment kernels (dynamic schedule) with 4 chunks in flight per warp.
#include "ms_batch.cuh"

namespace ms {
#define MS_NONE
MS_BATCH_DYNAMIC(MS_NONE, 4)
#undef MS_NONE
}  // namespace ms
