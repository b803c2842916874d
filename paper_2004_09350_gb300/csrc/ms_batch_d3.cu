// ms_batch_d3.cu -- batched fragment kernels with 3 chunks in flight per warp.
#include "ms_batch.cuh"

namespace ms {
MS_BATCH_INSTANTIATE(3)
}  // namespace ms
