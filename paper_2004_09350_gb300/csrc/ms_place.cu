// ms_place.cu -- placement of staged block-format outputs: one pass that scans the
// blocks' widths into payload offsets and headers and copies the payloads.
#include "ms_launch.h"

namespace ms {

ms_status launch_place(ms_ctx* c, const Work& w, DevMeta* out, uint64_t n_max, cudaStream_t s) {
  PlaceArgs a{};
  a.ctl = c->ctl;
  a.out_meta = out;
  a.stage_meta = w.stage_meta;
  a.status = w.status2;
  const uint64_t nb_max = std::max<uint64_t>(n_max / kBlock, 1);
  const int grid = grid_for(c, k_place<>, 0, cdiv(nb_max, (uint64_t)8));
  ProfScope ps(c, MS_K_PLACE, s);
  k_place<><<<grid, kThreads, 0, s>>>(a);
  return cuda_status(cudaGetLastError());
}

}  // namespace ms
