// ms_batch_d2.cu -- batched fragment kernels with 2 chunks in flight per warp.
#include "ms_batch.cuh"

namespace ms {
MS_BATCH_INSTANTIATE(2)
}  // namespace ms
