// ms_map_calc.cu -- k_map instantiation(s): OP_CALC (compiled on its own for build parallelism).
#include "ms_launch.h"

namespace ms {

template <>
ms_status launch_map<OP_CALC>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s) {
  return launch_map_impl<OP_CALC>(c, a, n_max, s);
}
}  // namespace ms
