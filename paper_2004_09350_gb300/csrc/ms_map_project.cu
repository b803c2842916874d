// ms_map_project.cu -- k_map instantiation(s): OP_PROJECT (random access) and OP_PROJECT_DELTA (compiled on its own for build parallelism).
#include "ms_launch.h"
#include "ms_project.cuh"

namespace ms {

template <>
ms_status launch_map<OP_PROJECT>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s) {
  return launch_map_impl<OP_PROJECT>(c, a, n_max, s);
}

template <>
ms_status launch_map<OP_PROJECT_DELTA>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s) {
  return launch_map_impl<OP_PROJECT_DELTA>(c, a, n_max, s);
}


template <>
ms_status launch_direct<OP_PROJECT>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s) {
  return launch_direct_impl<OP_PROJECT>(c, a, n_max, s);
}

template <>
ms_status launch_direct<OP_PROJECT_DELTA>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s) {
  return launch_direct_impl<OP_PROJECT_DELTA>(c, a, n_max, s);
}

ms_status launch_project_span(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s) {
  const uint64_t tiles = cdiv(cdiv(std::max<uint64_t>(n_max, 1), kBlock), kWarps);
  const int grid = grid_for(c, k_project_span, kSpanSmemBytes, tiles);
  ProfScope ps(c, MS_K_PROJECT, s);
  k_project_span<<<grid, kThreads, kSpanSmemBytes, s>>>(a);
  return cuda_status(cudaGetLastError());
}
}  // namespace ms
