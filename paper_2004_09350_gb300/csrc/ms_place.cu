// ms_place.cu -- placement of staged block-format outputs: width scan (headers and
// payload offsets) and the payload copy.
#include "ms_launch.h"

namespace ms {

ms_status launch_place(ms_ctx* c, const Work& w, DevMeta* out, uint64_t n_max, cudaStream_t s) {
  PlaceArgs a{};
  a.ctl = c->ctl;
  a.out_meta = out;
  a.stage = w.stage;
  a.stage_meta = w.stage_meta;
  a.offsets = w.offsets;
  a.status = w.status2;
  const uint64_t nb_max = std::max<uint64_t>(n_max / kBlock, 1);
  {
    const int grid = grid_for(c, k_scan_widths<>, 0, cdiv(nb_max, (uint64_t)kThreads * 16));
    ProfScope ps(c, MS_K_PLACE_SCAN, s);
    k_scan_widths<><<<grid, kThreads, 0, s>>>(a);
    if (cuda_status(cudaGetLastError()) != MS_OK) return MS_ERR_CUDA;
  }
  const int grid = grid_for(c, k_copy_blocks<>, 0, cdiv(nb_max + 1, kWarps));
  ProfScope ps(c, MS_K_PLACE_COPY, s);
  k_copy_blocks<><<<grid, kThreads, 0, s>>>(a);
  return cuda_status(cudaGetLastError());
}

}  // namespace ms
