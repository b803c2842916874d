// ms_map_codec.cu -- k_map instantiation(s): OP_COMPRESS, OP_DECOMPRESS (compiled on its own for build parallelism).
#include "ms_launch.h"

namespace ms {

template <>
ms_status launch_map<OP_COMPRESS>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s) {
  return launch_map_impl<OP_COMPRESS>(c, a, n_max, s);
}

template <>
ms_status launch_map<OP_DECOMPRESS>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s) {
  return launch_map_impl<OP_DECOMPRESS>(c, a, n_max, s);
}
}  // namespace ms
