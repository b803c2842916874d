// ms_batch.cuh -- the batched fragment kernel (select -> project -> agg_sum fused
// per chunk, Sec. 5.1 "Simple Query" shape) and its launcher template.  The
// instantiations live in ms_batch_d{2,3,4}.cu, one translation unit per depth.
#pragma once
#include <algorithm>

#include "ms_host.h"

namespace ms {

// Staging width of a payload slot: chunks packed at up to kBatchSlotW bits are
// copied into shared memory ahead of use; wider ones (and full uncompressed
// chunks) are decoded in place from global memory.
constexpr int kBatchSlotW = 40;
constexpr int kBatchUnits = 4 * kBatchSlotW;  // 16-byte units per slot

// One fragment as the kernel sees it (128 bytes).
struct BatchFrag {
  ColView x, y;
  uint64_t lo, span;  // predicate as one range test: ((x - lo) <= span) != negate
  uint32_t negate, empty;
  uint64_t pad;
};
static_assert(sizeof(BatchFrag) == 128, "fragment descriptor size");

struct BatchArgs {
  const BatchFrag* frags;
  const uint64_t* cs;  // cs[f] = first chunk of fragment f; cs[n_frags] = all chunks
  uint32_t f0, f1;     // fragments of this run
  uint64_t c0, c1;     // their chunks: [cs[f0], cs[f1])
  uint64_t ntiles;     // ceil((c1 - c0) / tile_chunks)
  uint32_t log2_tile;  // tile_chunks = 1 << log2_tile
  unsigned long long* counter;  // work counter (0 between runs)
  unsigned int* done;           // CTAs finished (0 between runs)
  unsigned long long* sums;     // indexed by fragment id
  DevCtl* ctl;
};

template <int D>
struct BatchSmem {
  uint16_t xs[D][32 * kBatchSlotW];
  uint16_t ys[D][32 * kBatchSlotW];
  uint64_t xh[2 * D][2];
  uint64_t yh[2 * D][2];
};

// The fragment that owns chunk g, found from the cursor's last fragment forward.
struct FragCursor {
  uint32_t f;
  uint64_t beg, end;  // chunk range of fragment f

  MS_DEV void seek(uint64_t g, const uint64_t* cs, uint32_t f_hi) {
    if (g < end) return;
    // cs[lo] <= g < cs[hi]: the owner is the last fragment starting at or before g
    // (empty fragments start where their successor does).
    uint32_t lo = f + 1, hi = f_hi;
    while (hi - lo > 1) {
      const uint32_t mid = lo + ((hi - lo) >> 1);
      if (__ldg(reinterpret_cast<const unsigned long long*>(cs) + mid) <= g) lo = mid;
      else hi = mid;
    }
    f = lo;
    beg = __ldg(reinterpret_cast<const unsigned long long*>(cs) + lo);
    end = __ldg(reinterpret_cast<const unsigned long long*>(cs) + lo + 1);
  }
};

MS_DEV ColView load_view(const ColView* p) {
  ColView c;
  c.p = reinterpret_cast<const uint8_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&p->p)));
  c.n = __ldg(reinterpret_cast<const unsigned long long*>(&p->n));
  c.nb = __ldg(reinterpret_cast<const unsigned long long*>(&p->nb));
  c.pwords = __ldg(reinterpret_cast<const unsigned long long*>(&p->pwords));
  c.size = __ldg(reinterpret_cast<const unsigned long long*>(&p->size));
  c.fmt = __ldg(&p->fmt);
  c.bw = __ldg(&p->bw);
  return c;
}

constexpr uint64_t kNoChunk = ~0ull;

// Persistent kernel: every warp grabs tiles of 2^log2_tile consecutive chunks of
// the batch's chunk space and streams both columns of each chunk with `D` chunks
// in flight.  Positions s = 0, 1, ... of a warp's stream map to tile ring[(s >>
// log2_tile) & 1]; the issue stages run at most 2D-1 positions ahead, so two
// tiles (the current and the next) cover them when the tile holds >= 2D chunks.
template <int WARPS, int D, bool kCompact>
__global__ void __launch_bounds__(32 * WARPS) k_batch(BatchArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  BatchSmem<D>* sm = reinterpret_cast<BatchSmem<D>*>(smem_raw) + warp;
  const uint32_t lt = a.log2_tile;
  const uint64_t kmask = (1ull << lt) - 1;

  auto grab = [&]() -> uint64_t {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1ull);
    return __shfl_sync(kFull, (uint64_t)t, 0);
  };
  uint64_t ring0 = grab(), ring1 = a.ntiles;
  auto chunk_at = [&](uint64_t s) -> uint64_t {
    const uint64_t t = ((s >> lt) & 1) ? ring1 : ring0;
    if (t >= a.ntiles) return kNoChunk;
    const uint64_t g = a.c0 + (t << lt) + (s & kmask);
    return g < a.c1 ? g : kNoChunk;
  };
  const uint64_t cs0 = __ldg(reinterpret_cast<const unsigned long long*>(a.cs) + a.f0);
  const uint64_t cs1 = __ldg(reinterpret_cast<const unsigned long long*>(a.cs) + a.f0 + 1);
  FragCursor hc{a.f0, cs0, cs1}, pc = hc, dc = hc;

  auto issue_header = [&](uint64_t s) {
    const uint64_t g = chunk_at(s);
    if (g == kNoChunk) return;
    hc.seek(g, a.cs, a.f1);
    const BatchFrag* fr = a.frags + hc.f;
    const int h = (int)(s % (2 * D));
    stage_header(load_view(&fr->x), g - hc.beg, sm->xh[h], lane);
    stage_header(load_view(&fr->y), g - hc.beg, sm->yh[h], lane);
  };
  auto issue_payload = [&](uint64_t s) {
    const uint64_t g = chunk_at(s);
    if (g == kNoChunk) return;
    pc.seek(g, a.cs, a.f1);
    const BatchFrag* fr = a.frags + pc.f;
    const int h = (int)(s % (2 * D)), p = (int)(s % D);
    stage_payload(load_view(&fr->x), g - pc.beg, sm->xh[h], sm->xs[p], lane, kBatchUnits);
    stage_payload(load_view(&fr->y), g - pc.beg, sm->yh[h], sm->ys[p], lane, kBatchUnits);
  };

  uint64_t acc = 0;          // this lane's part of fragment acc_f's sum
  uint32_t acc_f = ~0u;
  auto flush = [&]() {
    const uint64_t t = warp_sum(acc);
    if (lane == 0 && acc_f != ~0u && t) atomicAdd(a.sums + acc_f, (unsigned long long)t);
    acc = 0;
  };

  if (ring0 < a.ntiles) {
    for (int i = 0; i < D; i++) issue_header(i);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    for (int j = 0; j < D - 1; j++) {
      issue_header(j + D);
      issue_payload(j);
      cp_async_commit();
    }
    for (uint64_t s = 0;; s++) {
      if ((s & kmask) == 0) {
        // entering tile s >> lt: stop at a dead tile, else fetch the one after it
        if ((((s >> lt) & 1) ? ring1 : ring0) >= a.ntiles) break;
        const uint64_t nxt = grab();
        if ((s >> lt) & 1) ring0 = nxt;
        else ring1 = nxt;
      }
      cp_async_wait<D - 2>();
      __syncwarp();
      issue_header(s + 2 * D - 1);
      issue_payload(s + D - 1);
      cp_async_commit();
      const uint64_t g = chunk_at(s);
      if (g != kNoChunk) {
        dc.seek(g, a.cs, a.f1);
        if (dc.f != acc_f) {
          flush();
          acc_f = dc.f;
        }
        const BatchFrag* fr = a.frags + dc.f;
        const uint64_t lg = g - dc.beg;
        const int h = (int)(s % (2 * D)), p = (int)(s % D);
        const uint64_t lo = __ldg(reinterpret_cast<const unsigned long long*>(&fr->lo));
        const uint64_t span = __ldg(reinterpret_cast<const unsigned long long*>(&fr->span));
        const uint32_t negate = __ldg(&fr->negate) ? 0xffffu : 0u;
        const uint32_t live = __ldg(&fr->empty) ? 0u : 0xffffu;
        uint32_t m16 = 0;
        // one decoder instance for both columns keeps the instruction footprint small
#pragma unroll 1
        for (int col = 0; col < 2; col++) {
          uint64_t v[16];
          const int valid = decode_staged<kCompact>(load_view(col ? &fr->y : &fr->x), lg, col ? sm->yh[h] : sm->xh[h],
                                                    col ? sm->ys[p] : sm->xs[p], lane, v, a.ctl, kBatchUnits);
          if (col == 0) {
#pragma unroll
            for (int k = 0; k < 16; k++) m16 |= (uint32_t)(v[k] - lo <= span) << k;
            const int first = 16 * lane;
            m16 = (m16 ^ negate) & live &
                  (valid >= first + 16 ? 0xffffu : (valid > first ? (1u << (valid - first)) - 1u : 0u));
          } else {
#pragma unroll
            for (int k = 0; k < 16; k++) acc += ((m16 >> k) & 1u) ? v[k] : 0ull;
          }
        }
      }
      __syncwarp();
    }
    cp_async_wait<0>();
    flush();
  }
  // the last CTA to finish resets the work counter for the next run
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(a.done, 1u) == gridDim.x - 1) {
      *a.counter = 0;
      *a.done = 0;
      __threadfence();
    }
  }
}

// Launches k_batch<WARPS, D, kCompact> over a.ntiles tiles; grid capped at the
// resident CTAs (ctas_per_sm per SM when nonzero).  With a.ntiles == 0 it only sets
// the kernel's shared-memory attribute and caches its occupancy (done before a
// stream capture).
template <int WARPS, int D, bool kCompact>
ms_status launch_batch_kernel(ms_ctx* c, const BatchArgs& a, uint32_t ctas_per_sm, cudaStream_t s) {
  static int occ_cache[16];  // per device; 0 = not yet known
  const size_t smem = sizeof(BatchSmem<D>) * WARPS;
  const int dev = c->device;
  int occ = (dev >= 0 && dev < 16) ? occ_cache[dev] : 0;
  if (occ == 0) {
    if (smem > 48 * 1024 &&
        cuda_status(cudaFuncSetAttribute(k_batch<WARPS, D, kCompact>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem)) != MS_OK)
      return MS_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<WARPS, D, kCompact>, 32 * WARPS, smem) !=
            cudaSuccess ||
        occ < 1)
      occ = 1;
    if (dev >= 0 && dev < 16) occ_cache[dev] = occ;
  }
  if (a.ntiles == 0) return MS_OK;
  if (ctas_per_sm) occ = std::min<int>(occ, (int)ctas_per_sm);
  const uint64_t full = (uint64_t)occ * (uint64_t)c->sms;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(full, cdiv(a.ntiles, WARPS)));
  k_batch<WARPS, D, kCompact><<<grid, 32 * WARPS, smem, s>>>(a);
  return cuda_status(cudaGetLastError());
}

using BatchLauncher = ms_status (*)(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t);

// Launcher of (warps, depth, compact), or nullptr for an unsupported combination.
BatchLauncher batch_launcher(uint32_t warps, uint32_t depth, bool compact);

#define MS_BATCH_DECLARE(D)                                                                                  \
  extern template ms_status launch_batch_kernel<4, D, false>(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t); \
  extern template ms_status launch_batch_kernel<8, D, false>(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t); \
  extern template ms_status launch_batch_kernel<4, D, true>(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t);  \
  extern template ms_status launch_batch_kernel<8, D, true>(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t);
#define MS_BATCH_INSTANTIATE(D)                                                                       \
  template ms_status launch_batch_kernel<4, D, false>(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t); \
  template ms_status launch_batch_kernel<8, D, false>(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t); \
  template ms_status launch_batch_kernel<4, D, true>(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t);  \
  template ms_status launch_batch_kernel<8, D, true>(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t);

}  // namespace ms
