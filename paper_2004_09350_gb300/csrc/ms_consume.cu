// ms_consume.cu -- consuming kernels (no output column): the select / semi-join
// mark step and its count scan, agg_sum, group_sum and the semi-join build side,
// plus their launchers.
#include "ms_launch.h"

namespace ms {

// Mark kernel of select: the CTA streams its claims of the column (cta_stream) and
// writes per 512-row chunk a 512-bit match bitmap (lane j's 16 rows -> halfword j)
// and the chunk's match count.


template <int BUF, bool kRle>
__global__ void __launch_bounds__(kTileThreads, kRle ? 2 : kTileMinBlocks) k_mark_t(MarkArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int lane = threadIdx.x & 31;
  auto* sm = reinterpret_cast<TileSmem<BUF>*>(smem_raw);
  const ColView c = view_of(a.in);
  const uint64_t lo = a.lo, span = a.span;
  const uint32_t negate = a.negate ? 0xffffu : 0u, live = a.empty ? 0u : 0xffffu;
  cta_stream<BUF, kRle>(c, sm, a.ctl, [&](uint64_t g, const uint64_t* v, int valid, bool narrow) {
    uint32_t m16 = 0;
    if (a.keybits) {  // semi-join probe against a key bitmap read through the caches
#pragma unroll
      for (int k = 0; k < 16; k++) {
        const uint64_t x = v[k];
        const bool hit = x < a.domain && ((__ldg(a.keybits + (x >> 5)) >> (x & 31)) & 1u);
        m16 |= (uint32_t)hit << k;
      }
    } else if (narrow) {  // 32-bit compares
      if (a.mode32 == 0) {
#pragma unroll
        for (int k = 0; k < 16; k++) m16 |= (uint32_t)((uint32_t)v[k] - a.lo32 <= a.span32) << k;
      } else {
        m16 = a.mode32 == 2 ? 0xffffu : 0u;
      }
      m16 = (m16 ^ negate) & live;
    } else {
#pragma unroll
      for (int k = 0; k < 16; k++) m16 |= (uint32_t)(v[k] - lo <= span) << k;
      m16 = (m16 ^ negate) & live;
    }
    // rows past the column's end never match
    const int first = 16 * lane;
    m16 &= valid >= first + 16 ? 0xffffu : (valid > first ? (1u << (valid - first)) - 1u : 0u);
    a.bitmap[g * 32 + lane] = (uint16_t)m16;
    const uint32_t cnt = __reduce_add_sync(kFull, (uint32_t)__popc(m16));
    if (lane == 0) a.counts[g] = cnt;
  });
}

// k_mark: the tile stream's usual 2 x 32 KB buffers.  k_mark_l1: 2 x 8 KB buffers
// and a small shared-memory carve-out, so that most of the SM's unified L1 caches
// the key bitmap of a semi-join probe.
template <bool kRle>
constexpr auto k_mark = k_mark_t<kTileBuf, kRle>;
constexpr int kMarkL1Buf = 8192;
template <bool kRle>
constexpr auto k_mark_l1 = k_mark_t<kMarkL1Buf, kRle>;

// Semi-join probe with the key bitmap in shared memory, for key domains whose
// bitmap fits one CTA (up to about 1.5 million keys: 2e5 takes 25 KB).  Probing a
// bitmap in L2 leaves the probe latency-bound on scattered 32-byte sector reads;
// from shared memory a lookup costs a few bank wavefronts.  Compiled for the tile
// stream's three CTAs per SM, which a small bitmap leaves room for (a bitmap that
// takes most of shared memory runs one).
constexpr int kKeyTileBuf = 16384;
constexpr size_t kKeyTileSmemBytes = sizeof(TileSmem<kKeyTileBuf>);

template <bool kRle>
__global__ void __launch_bounds__(kTileThreads, kRle ? 2 : kTileMinBlocks) k_mark_keys(MarkArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int lane = threadIdx.x & 31;
  auto* sm = reinterpret_cast<TileSmem<kKeyTileBuf>*>(smem_raw);
  uint32_t* kb = reinterpret_cast<uint32_t*>(smem_raw + kKeyTileSmemBytes);
  const uint64_t nw = (a.domain + 31) / 32;
  for (uint64_t i = threadIdx.x; i < nw; i += blockDim.x) kb[i] = __ldg(a.keybits + i);
  __syncthreads();
  const ColView c = view_of(a.in);
  cta_stream<kKeyTileBuf, kRle>(c, sm, a.ctl, [&](uint64_t g, const uint64_t* v, int valid, bool) {
    uint32_t m16 = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const uint64_t x = v[k];
      const bool hit = x < a.domain && ((kb[x >> 5] >> (x & 31)) & 1u);
      m16 |= (uint32_t)hit << k;
    }
    const int first = 16 * lane;
    m16 &= valid >= first + 16 ? 0xffffu : (valid > first ? (1u << (valid - first)) - 1u : 0u);
    a.bitmap[g * 32 + lane] = (uint16_t)m16;
    const uint32_t cnt = __reduce_add_sync(kFull, (uint32_t)__popc(m16));
    if (lane == 0) a.counts[g] = cnt;
  });
}

// Exclusive scan of the per-chunk match counts (decoupled look-back over tiles of
// 4096 chunks).  Writes coff (with coff[nchunks] = total), the first chunk of every
// output block (bstart) and the total into ctl->op_n.

__global__ void __launch_bounds__(kThreads) k_scan_counts(ScanArgs a) {
  __shared__ uint64_t s_warp[kWarps];
  __shared__ uint64_t s_excl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint64_t nch = (a.in->n + kBlock - 1) / kBlock;
  constexpr int kPer = 16;
  const uint64_t per_tile = (uint64_t)kThreads * kPer;
  const uint64_t ntiles = (nch + per_tile - 1) / per_tile;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctl->op_nch = nch;
    if (nch == 0) {
      a.coff[0] = 0;
      a.ctl->op_n = 0;
    }
  }
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t g0 = tile * per_tile + (uint64_t)threadIdx.x * kPer;
    uint32_t cnt[kPer];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
      cnt[k] = (g0 + k < nch) ? a.counts[g0 + k] : 0;
      sum += cnt[k];
    }
    const uint32_t texcl = warp_excl_scan32(sum, lane);
    if (lane == 31) s_warp[warp] = texcl + sum;
    __syncthreads();
    if (warp == 0) {
      const uint64_t wt = lane < kWarps ? s_warp[lane] : 0;
      const uint64_t wex = warp_excl_scan(wt, lane);
      const uint64_t agg = warp_sum(wt);
      const uint64_t ex = lookback(a.status, tile, agg, lane, a.ctl);
      if (lane < kWarps) s_warp[lane] = wex;
      if (lane == 0) s_excl = ex;
    }
    __syncthreads();
    uint64_t o = s_excl + s_warp[warp] + texcl;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
      const uint64_t g = g0 + k;
      if (g < nch) {
        a.coff[g] = o;
        if (cnt[k]) {
          for (uint64_t h = (o + kBlock - 1) / kBlock; h <= (o + cnt[k] - 1) / kBlock; h++) a.bstart[h] = g;
        }
        o += cnt[k];
        if (g == nch - 1) {
          a.coff[nch] = o;
          a.ctl->op_n = o;
        }
      }
    }
    __syncthreads();
  }
}


// ----------------------------------------------------------------- aggregates

// agg_sum of an RLE column on its runs (Sec. 3.2, an operator on the compressed
// form): the sum of run value x (run length) over the runs, modulo 2^64 as the sum
// of the values is.
__global__ void __launch_bounds__(256) k_agg_sum_rle(const DevMeta* in, uint64_t* result, DevCtl* ctl) {
  const ColView c = view_of(in);
  if (!rle_sound(c)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_error(ctl, MS_ERR_FORMAT, c.size);
    return;
  }
  const uint64_t R = c.nb;
  const uint64_t* val = reinterpret_cast<const uint64_t*>(c.p);
  const uint64_t* ends = val + R;
  uint64_t s = 0;
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t start = r ? ldg64(ends + r - 1) : 0;
    s += ldg64(val + r) * (ldg64(ends + r) - start);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(reinterpret_cast<unsigned long long*>(result), (unsigned long long)s);
}

__global__ void __launch_bounds__(kTileThreads, kTileMinBlocks) k_agg_sum(const DevMeta* in, uint64_t* result,
                                                                          DevCtl* ctl) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int lane = threadIdx.x & 31;
  auto* sm = reinterpret_cast<TileSmem<kTileBuf>*>(smem_raw);
  const ColView c = view_of(in);
  uint64_t acc = 0;
  cta_stream<kTileBuf>(c, sm, ctl, [&](uint64_t, const uint64_t* v, int, bool) {
#pragma unroll
    for (int k = 0; k < 16; k++) acc += v[k];  // zero past the column's end
  });
  acc = warp_sum(acc);
  if (lane == 0 && acc) atomicAdd(reinterpret_cast<unsigned long long*>(result), (unsigned long long)acc);
}


__global__ void __launch_bounds__(32 * kPairWarps, 4) k_group_sum(const DevMeta* gid, const DevMeta* val, uint64_t G,
                                                               uint64_t* sums, DevCtl* ctl) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto* rings = reinterpret_cast<StreamSmem<kPairDepth>*>(smem_raw);
  unsigned long long* hist =
      reinterpret_cast<unsigned long long*>(smem_raw + 2 * kPairWarps * sizeof(StreamSmem<kPairDepth>));
  const bool local = G <= kSmemGroups;
  if (local)
    for (uint64_t k = threadIdx.x; k < G; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  const ColView cg = view_of(gid), cv = view_of(val);
  if (blockIdx.x == 0 && threadIdx.x == 0 && cg.n != cv.n) set_error(ctl, MS_ERR_INVALID_ARG, cv.n);
  const uint64_t n = min(cg.n, cv.n);
  const uint64_t gw = (uint64_t)blockIdx.x * kPairWarps + warp, W = (uint64_t)gridDim.x * kPairWarps;
  stream_pairs(cg, cv, n, gw, W, rings + 2 * warp, rings + 2 * warp + 1, lane, ctl,
               [&](uint64_t, const uint64_t* g8, const uint64_t* v, int valid) {
#pragma unroll
                 for (int k = 0; k < 16; k++) {
                   if (16 * lane + k < valid) {
                     if (g8[k] < G) {
                       if (local) atomicAdd(hist + g8[k], (unsigned long long)v[k]);
                       else atomicAdd(reinterpret_cast<unsigned long long*>(sums) + g8[k], (unsigned long long)v[k]);
                     } else {
                       set_error(ctl, MS_ERR_OUT_OF_RANGE, g8[k]);
                     }
                   }
                 }
               });
  if (!local) return;
  __syncthreads();
  for (uint64_t k = threadIdx.x; k < G; k += blockDim.x)
    if (hist[k]) atomicAdd(reinterpret_cast<unsigned long long*>(sums) + k, hist[k]);
}

// Failure-detection self-test: tile 1 of a look-back whose tile 0 never publishes.
__global__ void k_selftest_wait(uint64_t* status, DevCtl* ctl) {
  lookback(status, 1, 0, threadIdx.x & 31, ctl);
}

ms_status launch_selftest_wait(ms_ctx* c, cudaStream_t s) {
  uint64_t* status = reinterpret_cast<uint64_t*>(c->work);
  if (cuda_status(cudaMemsetAsync(status, 0, 2 * sizeof(uint64_t), s)) != MS_OK) return MS_ERR_CUDA;
  k_selftest_wait<<<1, 32, 0, s>>>(status, c->ctl);
  return cuda_status(cudaGetLastError());
}

// Semi-join build side: set bit key for every key of the build column.
template <bool kRle>
__global__ void __launch_bounds__(kTileThreads, kRle ? 2 : kTileMinBlocks) k_build_keys(const DevMeta* keys, uint64_t domain,
                                                                             uint32_t* bits, DevCtl* ctl) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int lane = threadIdx.x & 31;
  auto* sm = reinterpret_cast<TileSmem<kTileBuf>*>(smem_raw);
  const ColView c = view_of(keys);
  cta_stream<kTileBuf, kRle>(c, sm, ctl, [&](uint64_t, const uint64_t* v, int valid, bool) {
#pragma unroll
    for (int k = 0; k < 16; k++) {
      if (16 * lane + k < valid) {
        if (v[k] < domain) atomicOr(bits + (v[k] >> 5), 1u << (v[k] & 31));
        else set_error(ctl, MS_ERR_OUT_OF_RANGE, v[k]);
      }
    }
  });
}


// Column statistics for the format selector (see ms_column_stats): one decoding
// pass, per chunk reductions, block-level accumulation in shared memory, one
// global atomic per statistic per CTA.
template <bool kRle>
__global__ void __launch_bounds__(kTileThreads, kRle ? 2 : kTileMinBlocks) k_stats(const DevMeta* in, uint64_t* stats,
                                                                        DevCtl* ctl) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ unsigned long long s_acc[MS_STATS_WORDS];
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < MS_STATS_WORDS; i += blockDim.x) s_acc[i] = 0;
  __syncthreads();
  auto* sm = reinterpret_cast<TileSmem<kTileBuf>*>(smem_raw);
  const ColView c = view_of(in);
  cta_stream<kTileBuf, kRle>(c, sm, ctl, [&](uint64_t, const uint64_t* v, int valid, bool) {
    uint64_t mx = 0, mn = ~0ull, dmax = 0;
    uint32_t sorted = 0, runs = 0;
    const uint64_t prev_last = __shfl_up_sync(kFull, v[15], 1);
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const int i = 16 * lane + k;
      if (i < valid) {
        mx = max(mx, v[k]);
        mn = min(mn, v[k]);
        if (i > 0) {
          const uint64_t prev = k ? v[k - 1] : prev_last;
          dmax = max(dmax, v[k] - prev);
          sorted += v[k] >= prev;
          runs += v[k] != prev;
        }
      }
    }
    uint64_t cmx = mx;
#pragma unroll
    for (int d = 16; d; d >>= 1) cmx = max(cmx, __shfl_xor_sync(kFull, cmx, d));
    const uint64_t cmn = warp_min(mn);
    uint64_t cdm = dmax;
#pragma unroll
    for (int d = 16; d; d >>= 1) cdm = max(cdm, __shfl_xor_sync(kFull, cdm, d));
    const uint32_t s_sorted = __reduce_add_sync(kFull, sorted), s_runs = __reduce_add_sync(kFull, runs);
    if (lane == 0 && valid > 0) {
      atomicMax(&s_acc[1], (unsigned long long)cmx);
      atomicAdd(&s_acc[2], 1ull);
      atomicAdd(&s_acc[3], (unsigned long long)bw64(cmx - cmn));
      atomicAdd(&s_acc[4], (unsigned long long)bw64(cdm));
      atomicAdd(&s_acc[5], (unsigned long long)s_sorted);
      atomicAdd(&s_acc[6], (unsigned long long)s_runs);
      atomicAdd(&s_acc[8 + bw64(cmx)], 1ull);
    }
  });
  __syncthreads();
  for (int i = threadIdx.x; i < MS_STATS_WORDS; i += blockDim.x) {
    if (i == 1) atomicMax(reinterpret_cast<unsigned long long*>(stats) + 1, s_acc[1]);
    else if (i != 0 && s_acc[i]) atomicAdd(reinterpret_cast<unsigned long long*>(stats) + i, s_acc[i]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) stats[0] = c.n;
}

constexpr size_t kTileSmemBytes = sizeof(TileSmem<kTileBuf>);

// grid of a tile-stream kernel over a column of at most n_max rows: one CTA per
// claim, at most the resident CTAs
template <class K>
int tile_grid(ms_ctx* c, K kernel, uint64_t n_max) {
  return grid_for(c, kernel, kTileSmemBytes, cdiv(cdiv(std::max<uint64_t>(n_max, 1), kBlock), kClaim), kTileThreads);
}

ms_status launch_stats(ms_ctx* c, const DevMeta* in, uint64_t* d_stats, uint64_t n_max, cudaStream_t s, bool rle) {
  auto kernel = rle ? k_stats<true> : k_stats<false>;
  const int grid = tile_grid(c, kernel, n_max);
  ProfScope ps(c, MS_K_STATS, s);
  kernel<<<grid, kTileThreads, kTileSmemBytes, s>>>(in, d_stats, c->ctl);
  return cuda_status(cudaGetLastError());
}

// Shared memory the key bitmap of a semi-join probe may take per CTA.
constexpr size_t kKeySmemBudget = 224 * 1024 - kKeyTileSmemBytes;

ms_status launch_mark_scan(ms_ctx* c, MarkArgs& a, const Work& w, uint64_t n_max, cudaStream_t s) {
  a.bitmap = w.bitmap;
  a.counts = w.counts;
  const uint64_t key_bytes = a.keybits ? 4 * cdiv(a.domain, 32) : 0;
  if (a.keybits && key_bytes <= kKeySmemBudget) {  // key bitmap in shared memory
    auto kernel = a.rle ? k_mark_keys<true> : k_mark_keys<false>;
    const size_t smem = kKeyTileSmemBytes + key_bytes;
    const int grid = grid_for(c, kernel, smem, cdiv(cdiv(std::max<uint64_t>(n_max, 1), kBlock), kClaim),
                              kTileThreads);
    ProfScope ps(c, MS_K_MARK, s);
    kernel<<<grid, kTileThreads, smem, s>>>(a);
    if (cuda_status(cudaGetLastError()) != MS_OK) return MS_ERR_CUDA;
  } else if (a.keybits) {  // a larger key bitmap: probed through L1 and L2 (k_mark_l1)
    auto kernel = a.rle ? k_mark_l1<true> : k_mark_l1<false>;
    const size_t smem = sizeof(TileSmem<kMarkL1Buf>);
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 25);
    const int grid = grid_for(c, kernel, smem,
                              cdiv(cdiv(std::max<uint64_t>(n_max, 1), kBlock), kClaim), kTileThreads);
    ProfScope ps(c, MS_K_MARK, s);
    kernel<<<grid, kTileThreads, smem, s>>>(a);
    if (cuda_status(cudaGetLastError()) != MS_OK) return MS_ERR_CUDA;
  } else {  // select
    auto kernel = a.rle ? k_mark<true> : k_mark<false>;
    const int grid = tile_grid(c, kernel, n_max);
    ProfScope ps(c, MS_K_MARK, s);
    kernel<<<grid, kTileThreads, kTileSmemBytes, s>>>(a);
    if (cuda_status(cudaGetLastError()) != MS_OK) return MS_ERR_CUDA;
  }
  return launch_scan(c, a, w, n_max, s);
}

ms_status launch_scan(ms_ctx* c, const MarkArgs& a, const Work& w, uint64_t n_max, cudaStream_t s) {
  ScanArgs sa{};
  sa.in = a.in;
  sa.ctl = c->ctl;
  sa.counts = w.counts;
  sa.coff = w.coff;
  sa.bstart = w.bstart;
  sa.status = w.status;
  const uint64_t stiles = cdiv(cdiv(std::max<uint64_t>(n_max, 1), kBlock), (uint64_t)kThreads * 16);
  const int grid = grid_for(c, k_scan_counts, 0, stiles);
  ProfScope ps(c, MS_K_SCAN, s);
  k_scan_counts<<<grid, kThreads, 0, s>>>(sa);
  return cuda_status(cudaGetLastError());
}

ms_status launch_agg_sum(ms_ctx* c, const DevMeta* in, uint64_t* d_result, uint64_t n_max, cudaStream_t s,
                         bool rle) {
  if (rle) {  // runs at most n_max
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(cdiv(n_max, 256), 4ull * c->sms));
    ProfScope ps(c, MS_K_AGG_SUM, s);
    k_agg_sum_rle<<<grid, 256, 0, s>>>(in, d_result, c->ctl);
    return cuda_status(cudaGetLastError());
  }
  const int grid = tile_grid(c, k_agg_sum, n_max);
  ProfScope ps(c, MS_K_AGG_SUM, s);
  k_agg_sum<<<grid, kTileThreads, kTileSmemBytes, s>>>(in, d_result, c->ctl);
  return cuda_status(cudaGetLastError());
}

ms_status launch_group_sum(ms_ctx* c, const DevMeta* gid, const DevMeta* val, uint64_t G, uint64_t* d_sums,
                           uint64_t n_max, cudaStream_t s) {
  const size_t smem = 2 * kPairWarps * sizeof(StreamSmem<kPairDepth>) +
                      (G <= (uint64_t)kSmemGroups ? 8 * std::max<uint64_t>(G, 1) : 0);
  const uint64_t tiles = cdiv(cdiv(std::max<uint64_t>(n_max, 1), kBlock), kPairWarps);
  const int grid = grid_for(c, k_group_sum, smem, tiles, 32 * kPairWarps);
  ProfScope ps(c, MS_K_GROUP_SUM, s);
  k_group_sum<<<grid, 32 * kPairWarps, smem, s>>>(gid, val, G, d_sums, c->ctl);
  return cuda_status(cudaGetLastError());
}

ms_status launch_build_keys(ms_ctx* c, const DevMeta* keys, uint64_t domain, uint32_t* bits, uint64_t n_max,
                            cudaStream_t s, bool rle) {
  auto kernel = rle ? k_build_keys<true> : k_build_keys<false>;
  const int grid = tile_grid(c, kernel, n_max);
  ProfScope ps(c, MS_K_BUILD_KEYS, s);
  kernel<<<grid, kTileThreads, kTileSmemBytes, s>>>(keys, domain, bits, c->ctl);
  return cuda_status(cudaGetLastError());
}

}  // namespace ms
