// ms_launch.h -- scratch layout and kernel launchers shared by the host-side
// translation units of libms.
#pragma once
#include <algorithm>

#include "ms_host.h"
#include "ms_kernels.cuh"

namespace ms {

// Scratch carved from the context's work area for one operator on <= n_max rows.
struct Work {
  uint64_t* status;      // look-back status of the count scan
  uint64_t* status2;     // look-back status of the width scan
  uint16_t* bitmap;      // match bitmap, 32 halfwords per 512-row chunk
  uint64_t* coff;        // per-chunk exclusive output offsets (+ total)
  uint64_t* bstart;      // per-output-block first chunk
  uint32_t* counts;      // per-chunk match counts
  uint32_t* keybits;     // semi-join membership bitmap
  uint64_t* stage_meta;  // {(stage offset << 8) | width, reference} per output block
};

ms_status carve(ms_ctx* c, uint64_t n_max, uint64_t key_domain, Work* w, cudaStream_t s);

// Every select predicate as one range test (ms_ops.cu).
void predicate_as_range(int cmp, uint64_t c1, uint64_t c2, MarkArgs* m);

template <class K>
int grid_for(ms_ctx* c, K kernel, size_t smem, uint64_t tiles, int threads = kThreads) {
  if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess || occ < 1)
    occ = 1;
  const uint64_t full = (uint64_t)occ * (uint64_t)c->sms;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(full, tiles));
}

// consumers (ms_consume.cu)
ms_status launch_mark_scan(ms_ctx* c, MarkArgs& a, const Work& w, uint64_t n_max, cudaStream_t s);
// the count scan alone
ms_status launch_scan(ms_ctx* c, const MarkArgs& a, const Work& w, uint64_t n_max, cudaStream_t s);
// the specialized select on packed block formats (ms_select_packed.cu): mark + scan
ms_status launch_select_packed(ms_ctx* c, MarkArgs& a, const Work& w, uint64_t n_max, cudaStream_t s);
// rle: the column is RLE (summed on its runs)
ms_status launch_agg_sum(ms_ctx* c, const DevMeta* in, uint64_t* d_result, uint64_t n_max, cudaStream_t s,
                         bool rle = false);
ms_status launch_group_sum(ms_ctx* c, const DevMeta* gid, const DevMeta* val, uint64_t G, uint64_t* d_sums,
                           uint64_t n_max, cudaStream_t s);
// rle: the input column is RLE (the kernels' RLE instantiation)
ms_status launch_build_keys(ms_ctx* c, const DevMeta* keys, uint64_t domain, uint32_t* bits, uint64_t n_max,
                            cudaStream_t s, bool rle);
ms_status launch_stats(ms_ctx* c, const DevMeta* in, uint64_t* d_stats, uint64_t n_max, cudaStream_t s, bool rle);
ms_status launch_selftest_wait(ms_ctx* c, cudaStream_t s);

// producers (ms_map_*.cu): one warp-independent k_map<OP> launch
template <int OP>
ms_status launch_map(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s);
template <>
ms_status launch_map<OP_COMPRESS>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s);
template <>
ms_status launch_map<OP_DECOMPRESS>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s);
template <>
ms_status launch_map<OP_PROJECT>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s);
template <>
ms_status launch_map<OP_CALC>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s);
template <>
ms_status launch_map<OP_EMIT>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s);
template <>
ms_status launch_map<OP_PROJECT_WARP>(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s);

// run-length encoding of a column (ms_rle.cu); `in` null: raw uint64 input (raw, n_max);
// in_rle: the input is itself RLE
ms_status rle_encode(ms_ctx* c, const DevMeta* in, const uint64_t* raw, uint64_t n_max, const Work& w,
                     ms_column** out, cudaStream_t s, bool in_rle = false);

// placement of a staged block-format output (ms_place.cu)
ms_status launch_place(ms_ctx* c, const Work& w, DevMeta* out, uint64_t n_max, cudaStream_t s);

// Shared body of the launch_map instantiations.
constexpr int kMapKernel[6] = {MS_K_COMPRESS, MS_K_DECOMPRESS, MS_K_PROJECT, MS_K_CALC, MS_K_EMIT, MS_K_PROJECT};

template <int OP>
ms_status launch_map_impl(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s) {
  const size_t smem = sizeof(typename ProducePlan<OP>::Smem) * kWarps + ProducePlan<OP>::kCtaBytes;
  const uint64_t tiles = cdiv(cdiv(std::max<uint64_t>(n_max, 1), kBlock), kWarps);
  const int grid = grid_for(c, k_map<OP>, smem, tiles);
  ProfScope ps(c, kMapKernel[OP], s);
  k_map<OP><<<grid, kThreads, smem, s>>>(a);
  return cuda_status(cudaGetLastError());  // records the failing code
}


}  // namespace ms
