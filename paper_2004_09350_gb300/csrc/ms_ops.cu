// ms_ops.cu -- operator entry points of libms: argument checks, scratch layout and
// kernel launches.  Every launch is asynchronous on the caller's stream.
#include <algorithm>

#include "ms_host.h"
#include "ms_kernels.cuh"

namespace ms {
namespace {

// Scratch carved from the context's work area for one operator on <= n_max rows.
struct Work {
  uint64_t* status;   // look-back status of the first kernel
  uint64_t* status2;  // look-back status of the second kernel
  uint16_t* bitmap;   // match bitmap, 32 halfwords per 512-row chunk
  uint64_t* coff;     // per-chunk exclusive output offsets (+ total)
  uint64_t* bstart;   // per-output-block first chunk
  uint32_t* keybits;  // semi-join membership bitmap
};

ms_status carve(ms_ctx* c, uint64_t n_max, uint64_t key_domain, Work* w, cudaStream_t s) {
  const uint64_t nch = std::max<uint64_t>(cdiv(n_max, kBlock), 1);
  const uint64_t ntiles = cdiv(nch, kWarps);
  const uint64_t st_b = align_up(8 * (ntiles + 1), 256);
  const uint64_t bm_b = align_up(64 * nch, 256);
  const uint64_t co_b = align_up(8 * (nch + 2), 256);
  const uint64_t kb_b = align_up(4 * cdiv(std::max<uint64_t>(key_domain, 1), 32), 256);
  const uint64_t total = 2 * st_b + bm_b + 2 * co_b + kb_b;
  ms_status st = ensure_work(c, total);
  if (st != MS_OK) return st;
  uint8_t* p = c->work;
  w->status = reinterpret_cast<uint64_t*>(p);
  w->status2 = reinterpret_cast<uint64_t*>(p + st_b);
  w->bitmap = reinterpret_cast<uint16_t*>(p + 2 * st_b);
  w->coff = reinterpret_cast<uint64_t*>(p + 2 * st_b + bm_b);
  w->bstart = reinterpret_cast<uint64_t*>(p + 2 * st_b + bm_b + co_b);
  w->keybits = reinterpret_cast<uint32_t*>(p + 2 * st_b + bm_b + 2 * co_b);
  return cuda_status(cudaMemsetAsync(p, 0, 2 * st_b, s));
}

template <class K>
int grid_for(ms_ctx* c, K kernel, size_t smem, uint64_t tiles) {
  if (smem > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, smem) != cudaSuccess || occ < 1)
    occ = 1;
  const uint64_t full = (uint64_t)occ * (uint64_t)c->sms;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(full, tiles));
}

bool owned(ms_ctx* c, const ms_column* col) { return col && col->ctx == c && !col->freed; }

constexpr int kProduceKernel[5] = {MS_K_COMPRESS, MS_K_DECOMPRESS, MS_K_PROJECT, MS_K_CALC, MS_K_EMIT};

template <int OP>
ms_status launch_produce(ms_ctx* c, ProduceArgs& a, uint64_t n_max, cudaStream_t s) {
  const size_t smem = (size_t)SmemPlan<OP>::kPerWarp * kWarps;
  const uint64_t tiles = cdiv(cdiv(std::max<uint64_t>(n_max, 1), kBlock), kWarps);
  const int grid = grid_for(c, k_produce<OP>, smem, tiles);
  ProfScope ps(c, kProduceKernel[OP], s);
  k_produce<OP><<<grid, kThreads, smem, s>>>(a);
  return cuda_status(cudaGetLastError());
}

ms_status launch_mark(ms_ctx* c, MarkArgs& a, uint64_t n_max, cudaStream_t s) {
  const size_t smem = 4096 * kWarps;
  const uint64_t tiles = cdiv(cdiv(std::max<uint64_t>(n_max, 1), kBlock), kWarps);
  const int grid = grid_for(c, k_mark, smem, tiles);
  ProfScope ps(c, MS_K_MARK, s);
  k_mark<<<grid, kThreads, smem, s>>>(a);
  return cuda_status(cudaGetLastError());
}

// Second step of select / semi-join: match bitmap -> positions column in out_fmt.
ms_status emit_positions(ms_ctx* c, const Work& w, uint64_t n_max, int fmt, int bw, ms_column** out,
                         cudaStream_t s) {
  ms_column* col = new_arena_column(c, fmt, bw, n_max);
  if (!col) return MS_ERR_NOMEM;
  ProduceArgs a{};
  a.ctl = c->ctl;
  a.bitmap = w.bitmap;
  a.coff = w.coff;
  a.bstart = w.bstart;
  a.emit_nch = std::max<uint64_t>(cdiv(n_max, kBlock), 1);
  a.out_meta = c->metas + col->slot;
  a.fmt = fmt;
  a.bw = bw;
  a.status = w.status2;
  ms_status st = launch_produce<OP_EMIT>(c, a, n_max, s);
  if (st != MS_OK) {
    drop_new_column(c, col);
    return st;
  }
  *out = col;
  return MS_OK;
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" {

ms_status ms_compress(ms_ctx* c, const uint64_t* d_in, uint64_t n, int fmt, int bw, ms_column** out,
                      void* stream) {
  if (!c || !out || (!d_in && n) || !valid_format(fmt, bw)) return MS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_in) % 16) return MS_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w;
  ms_status st = carve(c, n, 0, &w, s);
  if (st != MS_OK) return st;
  ms_column* col = new_arena_column(c, fmt, bw, n);
  if (!col) return MS_ERR_NOMEM;
  ProduceArgs a{};
  a.ctl = c->ctl;
  a.raw_in = d_in;
  a.raw_n = n;
  a.out_meta = c->metas + col->slot;
  a.fmt = fmt;
  a.bw = bw;
  a.status = w.status;
  st = launch_produce<OP_COMPRESS>(c, a, n, s);
  if (st != MS_OK) {
    drop_new_column(c, col);
    return st;
  }
  *out = col;
  return MS_OK;
}

ms_status ms_decompress(ms_ctx* c, const ms_column* col, uint64_t* d_out, uint64_t cap, void* stream) {
  if (!c || !owned(c, col) || (!d_out && cap)) return MS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_out) % 16) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ProduceArgs a{};
  a.ctl = c->ctl;
  a.in0 = c->metas + col->slot;
  a.raw_out = d_out;
  a.raw_cap = cap;
  a.fmt = MS_UNCOMPR;
  return launch_produce<OP_DECOMPRESS>(c, a, std::min(col->n_max, cap), s);
}

ms_status ms_select(ms_ctx* c, const ms_column* in, int cmp, uint64_t c1, uint64_t c2, int fmt, int bw,
                    ms_column** out, void* stream) {
  if (!c || !out || !owned(c, in) || !valid_format(fmt, bw) || cmp < MS_EQ || cmp > MS_BETWEEN)
    return MS_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w;
  ms_status st = carve(c, in->n_max, 0, &w, s);
  if (st != MS_OK) return st;
  MarkArgs m{};
  m.in = c->metas + in->slot;
  m.ctl = c->ctl;
  m.cmp = cmp;
  m.c1 = c1;
  m.c2 = c2;
  m.bitmap = w.bitmap;
  m.coff = w.coff;
  m.bstart = w.bstart;
  m.status = w.status;
  st = launch_mark(c, m, in->n_max, s);
  if (st != MS_OK) return st;
  return emit_positions(c, w, in->n_max, fmt, bw, out, s);
}

ms_status ms_project(ms_ctx* c, const ms_column* data, const ms_column* pos, int fmt, int bw,
                     ms_column** out, void* stream) {
  if (!c || !out || !owned(c, data) || !owned(c, pos) || !valid_format(fmt, bw)) return MS_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w;
  ms_status st = carve(c, pos->n_max, 0, &w, s);
  if (st != MS_OK) return st;
  ms_column* col = new_arena_column(c, fmt, bw, pos->n_max);
  if (!col) return MS_ERR_NOMEM;
  ProduceArgs a{};
  a.ctl = c->ctl;
  a.in0 = c->metas + data->slot;
  a.in1 = c->metas + pos->slot;
  a.out_meta = c->metas + col->slot;
  a.fmt = fmt;
  a.bw = bw;
  a.status = w.status;
  st = launch_produce<OP_PROJECT>(c, a, pos->n_max, s);
  if (st != MS_OK) {
    drop_new_column(c, col);
    return st;
  }
  *out = col;
  return MS_OK;
}

ms_status ms_calc(ms_ctx* c, int op, const ms_column* x, const ms_column* y, uint64_t scalar, int fmt,
                  int bw, ms_column** out, void* stream) {
  if (!c || !out || !owned(c, x) || (y && !owned(c, y)) || !valid_format(fmt, bw) || op < MS_ADD ||
      op > MS_MUL)
    return MS_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t n_max = y ? std::min(x->n_max, y->n_max) : x->n_max;
  Work w;
  ms_status st = carve(c, n_max, 0, &w, s);
  if (st != MS_OK) return st;
  ms_column* col = new_arena_column(c, fmt, bw, n_max);
  if (!col) return MS_ERR_NOMEM;
  ProduceArgs a{};
  a.ctl = c->ctl;
  a.in0 = c->metas + x->slot;
  a.in1 = y ? c->metas + y->slot : nullptr;
  a.arith = op;
  a.scalar = scalar;
  a.out_meta = c->metas + col->slot;
  a.fmt = fmt;
  a.bw = bw;
  a.status = w.status;
  st = launch_produce<OP_CALC>(c, a, n_max, s);
  if (st != MS_OK) {
    drop_new_column(c, col);
    return st;
  }
  *out = col;
  return MS_OK;
}

ms_status ms_agg_sum(ms_ctx* c, const ms_column* in, uint64_t* d_result, void* stream) {
  if (!c || !owned(c, in) || !d_result) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_result, 0, 8, s) != cudaSuccess) return MS_ERR_CUDA;
  const size_t smem = 4096 * kWarps;
  const uint64_t tiles = cdiv(cdiv(std::max<uint64_t>(in->n_max, 1), kBlock), kWarps);
  const int grid = grid_for(c, k_agg_sum, smem, tiles);
  ProfScope ps(c, MS_K_AGG_SUM, s);
  k_agg_sum<<<grid, kThreads, smem, s>>>(c->metas + in->slot, d_result, c->ctl);
  return cuda_status(cudaGetLastError());
}

ms_status ms_group_sum(ms_ctx* c, const ms_column* gid, const ms_column* val, uint64_t G, uint64_t* d_sums,
                       void* stream) {
  if (!c || !owned(c, gid) || !owned(c, val) || (!d_sums && G)) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (G && cudaMemsetAsync(d_sums, 0, 8 * G, s) != cudaSuccess) return MS_ERR_CUDA;
  const size_t smem = 4096 * kWarps + (G <= (uint64_t)kSmemGroups ? 8 * kSmemGroups : 0);
  const uint64_t n_max = std::min(gid->n_max, val->n_max);
  const uint64_t tiles = cdiv(cdiv(std::max<uint64_t>(n_max, 1), kBlock), kWarps);
  const int grid = grid_for(c, k_group_sum, 4096 * kWarps + 8 * kSmemGroups, tiles);
  ProfScope ps(c, MS_K_GROUP_SUM, s);
  k_group_sum<<<grid, kThreads, smem, s>>>(c->metas + gid->slot, c->metas + val->slot, G, d_sums, c->ctl);
  return cuda_status(cudaGetLastError());
}

ms_status ms_semijoin(ms_ctx* c, const ms_column* probe, const ms_column* keys, uint64_t domain, int fmt,
                      int bw, ms_column** out, void* stream) {
  if (!c || !out || !owned(c, probe) || !owned(c, keys) || !valid_format(fmt, bw) || domain == 0)
    return MS_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w;
  ms_status st = carve(c, std::max(probe->n_max, keys->n_max), domain, &w, s);
  if (st != MS_OK) return st;
  if (cudaMemsetAsync(w.keybits, 0, 4 * cdiv(domain, 32), s) != cudaSuccess) return MS_ERR_CUDA;
  {
    const size_t smem = 4096 * kWarps;
    const uint64_t tiles = cdiv(cdiv(std::max<uint64_t>(keys->n_max, 1), kBlock), kWarps);
    const int grid = grid_for(c, k_build_keys, smem, tiles);
    ProfScope ps(c, MS_K_BUILD_KEYS, s);
    k_build_keys<<<grid, kThreads, smem, s>>>(c->metas + keys->slot, domain, w.keybits, c->ctl);
    if (cudaGetLastError() != cudaSuccess) return MS_ERR_CUDA;
  }
  MarkArgs m{};
  m.in = c->metas + probe->slot;
  m.ctl = c->ctl;
  m.keybits = w.keybits;
  m.domain = domain;
  m.bitmap = w.bitmap;
  m.coff = w.coff;
  m.bstart = w.bstart;
  m.status = w.status;
  st = launch_mark(c, m, probe->n_max, s);
  if (st != MS_OK) return st;
  return emit_positions(c, w, probe->n_max, fmt, bw, out, s);
}

}  // extern "C"
