// ms_batch.cu -- batched fragments: binding fragments to columns, running them in
// one persistent launch (or one launch each), and CUDA graph capture.
#include <algorithm>
#include <vector>

#include "ms_batch.cuh"
#include "ms_launch.h"

struct ms_batch {
  ms_ctx* ctx;
  uint32_t n;
  ms::BatchFrag* d_frags;
  uint64_t* d_cs;
  ms::ChunkRec* d_dir;            // one record per chunk
  unsigned long long* d_counter;  // [0] work counter, [1] finished CTAs
  std::vector<uint64_t> cs;       // host copy of the chunk prefix
  uint64_t rows, bytes;
};

struct ms_graph {
  cudaGraphExec_t exec;
};

namespace ms {

#define MS_EXTERN extern
MS_BATCH_DYNAMIC(MS_EXTERN, 2)
MS_BATCH_DYNAMIC(MS_EXTERN, 3)
MS_BATCH_DYNAMIC(MS_EXTERN, 4)
MS_BATCH_STATIC(MS_EXTERN)
MS_BATCH_CTA(MS_EXTERN)
#undef MS_EXTERN

// Host-built part of a fragment: the column slots and the predicate.
struct BatchInit {
  int32_t xslot, yslot;
  uint64_t lo, span;
  uint32_t negate, empty;
};

// Per-fragment lengths and sizes read back by the host.
struct BatchSizes {
  uint64_t nx, ny, sx, sy;
};

__global__ void k_batch_bind(const BatchInit* init, uint32_t n, const DevMeta* metas, BatchFrag* frags,
                             BatchSizes* sizes) {
  for (uint32_t f = blockIdx.x * blockDim.x + threadIdx.x; f < n; f += gridDim.x * blockDim.x) {
    const BatchInit in = init[f];
    BatchFrag fr{};
    fr.x = view_of(metas + in.xslot);
    fr.y = view_of(metas + in.yslot);
    fr.lo = in.lo;
    fr.span = in.span;
    fr.negate = in.negate;
    fr.empty = in.empty;
    frags[f] = fr;
    sizes[f] = BatchSizes{fr.x.n, fr.y.n, fr.x.size, fr.y.size};
  }
}

// Builds the chunk directory: one thread per chunk, its fragment by binary search.
__global__ void k_batch_dir(const BatchFrag* frags, const uint64_t* cs, uint32_t n_frags, ChunkRec* dir,
                            DevCtl* ctl) {
  const uint64_t total = cs[n_frags];
  for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total;
       g += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = n_frags;  // cs[lo] <= g < cs[hi]
    while (hi - lo > 1) {
      const uint32_t mid = lo + ((hi - lo) >> 1);
      if (cs[mid] <= g) lo = mid;
      else hi = mid;
    }
    const BatchFrag fr = frags[lo];
    const uint64_t lg = g - cs[lo];
    ChunkRec r;
    resolve_chunk(fr.x, lg, &r.addr[0], &r.ref[0], &r.code[0], ctl);
    resolve_chunk(fr.y, lg, &r.addr[1], &r.ref[1], &r.code[1], ctl);
    r.lo = fr.lo;
    r.span = fr.span;
    r.frag = lo;
    r.meta = (uint32_t)min((uint64_t)kBlock, fr.x.n - lg * kBlock) | fr.negate << 16 | fr.empty << 17;
    dir[g] = r;
  }
}

BatchLauncher batch_launcher(uint32_t warps, uint32_t depth, bool compact, uint32_t schedule) {
  if (schedule == 0) {
#define MS_PICK(W, D)                                                                                   \
  if (warps == W && depth == D)                                                                         \
    return compact ? &launch_batch_kernel<W, D, true, false> : &launch_batch_kernel<W, D, false, false>;
    MS_PICK(4, 2) MS_PICK(8, 2) MS_PICK(4, 3) MS_PICK(8, 3) MS_PICK(4, 4) MS_PICK(8, 4)
#undef MS_PICK
  } else if (schedule == 1 && !compact) {
#define MS_PICK(W, D) \
  if (warps == W && depth == D) return &launch_batch_kernel<W, D, false, true>;
    MS_PICK(4, 2) MS_PICK(8, 2) MS_PICK(16, 2) MS_PICK(4, 3) MS_PICK(8, 3)
#undef MS_PICK
  } else if (schedule == 2 && !compact && warps == 8) {  // depth selects the buffers: 8 KB x depth per column
    if (depth == 2) return &launch_batch_cta<16384, false>;
    if (depth == 3) return &launch_batch_cta<24576, false>;
    if (depth == 4) return &launch_batch_cta<32768, false>;
  }
  return nullptr;
}

namespace {

bool owned_column(ms_ctx* c, const ms_column* col) { return col && col->ctx == c && !col->freed; }

int log2_exact(uint32_t v) {
  if (v == 0 || (v & (v - 1))) return -1;
  int k = 0;
  while ((1u << k) < v) k++;
  return k;
}

// Launches fragments [f0, f1) as one persistent run.
ms_status run_range(ms_batch* b, uint32_t f0, uint32_t f1, BatchLauncher launch, const ms_batch_config& cfg,
                    int lt, uint64_t* d_sums, cudaStream_t s) {
  const uint64_t c0 = b->cs[f0], c1 = b->cs[f1];
  if (c1 == c0) return MS_OK;
  BatchArgs a{};
  a.dir = b->d_dir;
  a.c0 = c0;
  a.c1 = c1;
  a.log2_tile = (uint32_t)lt;
  a.ntiles = cdiv(c1 - c0, 1ull << lt);
  a.counter = b->d_counter;
  a.done = reinterpret_cast<unsigned int*>(b->d_counter + 1);
  a.sums = reinterpret_cast<unsigned long long*>(d_sums);
  a.ctl = b->ctx->ctl;
  ProfScope ps(b->ctx, MS_K_BATCH, s);
  return launch(b->ctx, a, cfg.ctas_per_sm, s);
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" {

ms_status ms_batch_create(ms_ctx* c, uint32_t n, ms_column* const* x, ms_column* const* y, const int32_t* cmp,
                          const uint64_t* c1, const uint64_t* c2, ms_batch** out, void* stream) {
  MS_TRACE();
  if (!c || !out || !x || !y || !cmp || !c1 || n == 0) return MS_ERR_INVALID_ARG;
  *out = nullptr;
  std::vector<BatchInit> init(n);
  for (uint32_t f = 0; f < n; f++) {
    if (!owned_column(c, x[f]) || !owned_column(c, y[f]) || cmp[f] < MS_EQ || cmp[f] > MS_BETWEEN)
      return MS_ERR_INVALID_ARG;
    if (x[f]->fmt > MS_FOR_BP || y[f]->fmt > MS_FOR_BP) return MS_ERR_FORMAT;  // the five base formats only
    MarkArgs m{};
    predicate_as_range(cmp[f], c1[f], c2 ? c2[f] : 0, &m);
    init[f] = BatchInit{x[f]->slot, y[f]->slot, m.lo, m.span, m.negate, m.empty};
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ms_batch* b = new ms_batch{};
  b->ctx = c;
  b->n = n;
  b->d_frags = static_cast<BatchFrag*>(dev_alloc(c, sizeof(BatchFrag) * n));
  b->d_cs = static_cast<uint64_t*>(dev_alloc(c, sizeof(uint64_t) * (n + 1)));
  b->d_counter = static_cast<unsigned long long*>(dev_alloc(c, 256));
  void* d_init = dev_alloc(c, sizeof(BatchInit) * n);
  void* d_sizes = dev_alloc(c, sizeof(BatchSizes) * n);
  std::vector<BatchSizes> sizes(n);
  ms_status st = MS_OK;
  if (!b->d_frags || !b->d_cs || !b->d_counter || !d_init || !d_sizes) {
    st = MS_ERR_NOMEM;
  } else {
    st = cuda_status(cudaMemcpyAsync(d_init, init.data(), sizeof(BatchInit) * n, cudaMemcpyHostToDevice, s));
    if (st == MS_OK) st = cuda_status(cudaMemsetAsync(b->d_counter, 0, 256, s));
    if (st == MS_OK) {
      const int grid = (int)std::min<uint64_t>(cdiv(n, 256), 1024);
      k_batch_bind<<<grid, 256, 0, s>>>(static_cast<const BatchInit*>(d_init), n, c->metas, b->d_frags,
                                        static_cast<BatchSizes*>(d_sizes));
      st = cuda_status(cudaGetLastError());
    }
    if (st == MS_OK)
      st = cuda_status(cudaMemcpyAsync(sizes.data(), d_sizes, sizeof(BatchSizes) * n, cudaMemcpyDeviceToHost, s));
    if (st == MS_OK) st = cuda_status(cudaStreamSynchronize(s));
  }
  if (st == MS_OK) {
    b->cs.assign(n + 1, 0);
    for (uint32_t f = 0; f < n && st == MS_OK; f++) {
      if (sizes[f].nx != sizes[f].ny) st = MS_ERR_INVALID_ARG;
      b->cs[f + 1] = b->cs[f] + cdiv(sizes[f].nx, kBlock);
      b->rows += sizes[f].nx;
      b->bytes += sizes[f].sx + sizes[f].sy;
    }
    if (st == MS_OK && b->cs[n] >= (1ull << 31)) st = MS_ERR_INVALID_ARG;
  }
  if (st == MS_OK)
    st = cuda_status(cudaMemcpyAsync(b->d_cs, b->cs.data(), sizeof(uint64_t) * (n + 1), cudaMemcpyHostToDevice, s));
  if (st == MS_OK) {
    b->d_dir = static_cast<ChunkRec*>(dev_alloc(c, sizeof(ChunkRec) * std::max<uint64_t>(b->cs[n], 1)));
    if (!b->d_dir) st = MS_ERR_NOMEM;
  }
  if (st == MS_OK && b->cs[n]) {
    const int grid = (int)std::min<uint64_t>(cdiv(b->cs[n], 256), 65536);
    k_batch_dir<<<grid, 256, 0, s>>>(b->d_frags, b->d_cs, n, b->d_dir, c->ctl);
    st = cuda_status(cudaGetLastError());
  }
  if (st == MS_OK) st = cuda_status(cudaStreamSynchronize(s));
  else cudaStreamSynchronize(s);
  dev_free(c, d_init);
  dev_free(c, d_sizes);
  if (st != MS_OK) {
    ms_batch_destroy(b);
    return st;
  }
  *out = b;
  return MS_OK;
}

ms_status ms_batch_info(const ms_batch* b, uint64_t* rows, uint64_t* chunks, uint64_t* bytes) {
  if (!b) return MS_ERR_INVALID_ARG;
  if (rows) *rows = b->rows;
  if (chunks) *chunks = b->cs[b->n];
  if (bytes) *bytes = b->bytes;
  return MS_OK;
}

ms_status ms_batch_run(ms_batch* b, uint32_t f0, uint32_t f1, const ms_batch_config* cfg_in, uint32_t flags,
                       uint64_t* d_sums, void* stream) {
  MS_TRACE();
  if (!b || !d_sums || f0 > f1 || f1 > b->n || (flags & ~(MS_BATCH_ZERO | MS_BATCH_PER_FRAGMENT)))
    return MS_ERR_INVALID_ARG;
  const ms_batch_config cfg = cfg_in ? *cfg_in : ms_batch_config{8, 2, 32, 0, 0, 1};
  const BatchLauncher launch = batch_launcher(cfg.warps, cfg.depth, cfg.compact != 0, cfg.schedule);
  const int lt = log2_exact(cfg.tile_chunks);
  if (!launch || lt < 3 || lt > 10 || cfg.compact > 1) return MS_ERR_INVALID_ARG;
  if (cfg.schedule == 0 && cfg.tile_chunks < 2 * cfg.depth) return MS_ERR_INVALID_ARG;
  if (cfg.schedule == 1 && cfg.tile_chunks < cfg.warps) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (f0 == f1) return MS_OK;
  if ((flags & MS_BATCH_ZERO) &&
      cuda_status(cudaMemsetAsync(d_sums + f0, 0, sizeof(uint64_t) * (f1 - f0), s)) != MS_OK)
    return MS_ERR_CUDA;
  if (!(flags & MS_BATCH_PER_FRAGMENT)) return run_range(b, f0, f1, launch, cfg, lt, d_sums, s);
  for (uint32_t f = f0; f < f1; f++) {
    const ms_status st = run_range(b, f, f + 1, launch, cfg, lt, d_sums, s);
    if (st != MS_OK) return st;
  }
  return MS_OK;
}

ms_status ms_batch_graph(ms_batch* b, uint32_t f0, uint32_t f1, const ms_batch_config* cfg, uint32_t flags,
                         uint64_t* d_sums, ms_graph** out) {
  MS_TRACE();
  if (!b || !out) return MS_ERR_INVALID_ARG;
  *out = nullptr;
  const ms_batch_config conf = cfg ? *cfg : ms_batch_config{8, 2, 32, 0, 0, 1};
  const BatchLauncher launch = batch_launcher(conf.warps, conf.depth, conf.compact != 0, conf.schedule);
  if (!launch) return MS_ERR_INVALID_ARG;
  // kernel attributes are set outside the capture
  BatchArgs none{};
  if (launch(b->ctx, none, 0, nullptr) != MS_OK) return MS_ERR_CUDA;
  cudaStream_t s = nullptr;
  if (cuda_status(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != MS_OK) return MS_ERR_CUDA;
  ms_status st = MS_OK;
  cudaGraph_t graph = nullptr;
  if (st == MS_OK) st = cuda_status(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  if (st == MS_OK) {
    const bool prof = b->ctx->prof_on;
    b->ctx->prof_on = false;  // no profiling events inside a graph
    const ms_status run = ms_batch_run(b, f0, f1, cfg, flags, d_sums, s);
    b->ctx->prof_on = prof;
    const ms_status end = cuda_status(cudaStreamEndCapture(s, &graph));
    st = run != MS_OK ? run : end;
  }
  cudaGraphExec_t exec = nullptr;
  if (st == MS_OK) st = cuda_status(cudaGraphInstantiate(&exec, graph, 0));
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(s);
  if (st != MS_OK) return st;
  *out = new ms_graph{exec};
  return MS_OK;
}

ms_status ms_graph_launch(ms_graph* g, void* stream) {
  MS_TRACE();
  if (!g) return MS_ERR_INVALID_ARG;
  return cuda_status(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
}

ms_status ms_graph_destroy(ms_graph* g) {
  if (!g) return MS_ERR_INVALID_ARG;
  cudaGraphExecDestroy(g->exec);
  delete g;
  return MS_OK;
}

ms_status ms_batch_destroy(ms_batch* b) {
  if (!b) return MS_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  dev_free(b->ctx, b->d_frags);
  dev_free(b->ctx, b->d_cs);
  dev_free(b->ctx, b->d_dir);
  dev_free(b->ctx, b->d_counter);
  delete b;
  return MS_OK;
}

}  // extern "C"
