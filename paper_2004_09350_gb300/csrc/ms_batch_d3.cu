// ms_batch_d3.cu -- batched fragment kernels (dynamic schedule) with 3 chunks in flight per warp.
#include "ms_batch.cuh"

namespace ms {
#define MS_NONE
MS_BATCH_DYNAMIC(MS_NONE, 3)
#undef MS_NONE
}  // namespace ms
