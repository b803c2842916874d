// ms_map_emit.cu -- k_map instantiation(s): OP_EMIT (compiled on its own for build parallelism).
#include "ms_launch.h"

namespace ms {

template <>
ms_status launch_map<OP_EMIT>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s) {
  return launch_map_impl<OP_EMIT>(c, a, n_max, s);
}
}  // namespace ms
