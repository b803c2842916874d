// ms_map_project.cu -- k_map instantiations of project: OP_PROJECT (the CTA span gather) and OP_PROJECT_WARP (the per-warp gather), compiled on their own for build parallelism.
#include "ms_launch.h"

namespace ms {

template <>
ms_status launch_map<OP_PROJECT>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s) {
  return launch_map_impl<OP_PROJECT>(c, a, n_max, s);
}

template <>
ms_status launch_map<OP_PROJECT_WARP>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s) {
  return launch_map_impl<OP_PROJECT_WARP>(c, a, n_max, s);
}
}  // namespace ms
