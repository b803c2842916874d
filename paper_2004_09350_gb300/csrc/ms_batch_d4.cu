// ms_batch_d4.cu -- batched fragment kernels with 4 chunks in flight per warp.
#include "ms_batch.cuh"

namespace ms {
MS_BATCH_INSTANTIATE(4)
}  // namespace ms
