// ms_rle.cu -- run-length encoding of a column in any format (Sec. 2.1, RLE).
//
// A run is a maximal stretch of equal consecutive values; value t starts a run (is
// a head) when t = 0 or x[t] != x[t-1].  The encoder makes three passes over the
// input, each a tile stream of 512-value chunks decoded in registers:
//   1. k_rle_count: per chunk, the heads after its first value, and its first and
//      last values;
//   2. k_rle_bounds adds the chunk's first value as a head where it differs from
//      the previous chunk's last, and k_scan_counts turns the per-chunk head counts
//      into run offsets (decoupled look-back);
//   3. k_rle_write decodes the chunk again and writes every head's run value and the
//      end of the run before it, and the chunk's directory entry.
// The output (R values, R ends, ceil(n/512) directory entries) goes straight to the
// arena top; the last CTA to finish records the column.
#include "ms_launch.h"

namespace ms {

struct RleArgs {
  const DevMeta* in;
  DevCtl* ctl;
  DevMeta* out_meta;
  uint32_t* counts;      // per chunk: heads (passes 1-2)
  uint64_t* fl;          // per chunk: {first value, last value}
  const uint64_t* coff;  // per chunk: heads before it; coff[nch] = R (pass 3)
};

// Heads among the chunk's values after its first: bit k of the lane's mask is set
// when value t = 16*lane + k (0 < t < valid) differs from value t - 1.
MS_DEV uint32_t rle_inner_heads(const uint64_t* v, int valid, int lane) {
  const uint64_t prev = __shfl_up_sync(kFull, v[15], 1);
  uint32_t m = 0;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    const int t = 16 * lane + k;
    const uint64_t before = k ? v[k - 1] : prev;
    if (t > 0 && t < valid && v[k] != before) m |= 1u << k;
  }
  return m;
}

// The chunk's last value (value valid - 1), on every lane.  The lane's value at
// index t % 16 is picked by a selection tree over its bits, which keeps v in registers.
MS_DEV uint64_t rle_last_value(const uint64_t* v, int valid) {
  const int t = valid - 1, i = t & 15;
  uint64_t w8[8], w4[4], w2[2];
#pragma unroll
  for (int j = 0; j < 8; j++) w8[j] = (i & 8) ? v[j + 8] : v[j];
#pragma unroll
  for (int j = 0; j < 4; j++) w4[j] = (i & 4) ? w8[j + 4] : w8[j];
#pragma unroll
  for (int j = 0; j < 2; j++) w2[j] = (i & 2) ? w4[j + 2] : w4[j];
  return __shfl_sync(kFull, (i & 1) ? w2[1] : w2[0], t >> 4);
}

template <bool kRle>
__global__ void __launch_bounds__(kTileThreads, kRle ? 2 : kTileMinBlocks) k_rle_count(RleArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  auto* sm = reinterpret_cast<TileSmem<kTileBuf>*>(smem_raw);
  const int lane = threadIdx.x & 31;
  const ColView c = view_of(a.in);
  cta_stream<kTileBuf, kRle>(c, sm, a.ctl, [&](uint64_t g, const uint64_t* v, int valid, bool) {
    const uint32_t heads = __reduce_add_sync(kFull, (unsigned)__popc(rle_inner_heads(v, valid, lane)));
    const uint64_t first = __shfl_sync(kFull, v[0], 0);
    const uint64_t last = rle_last_value(v, valid);
    if (lane == 0) {
      a.counts[g] = heads;
      a.fl[2 * g] = first;
      a.fl[2 * g + 1] = last;
    }
  });
}

// Chunk g's first value is a head when g = 0 or it differs from chunk g-1's last.
__global__ void k_rle_bounds(RleArgs a) {
  const uint64_t nch = (a.in->n + kBlock - 1) / kBlock;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nch; g += (uint64_t)gridDim.x * blockDim.x)
    if (g == 0 || a.fl[2 * g] != a.fl[2 * g - 1]) a.counts[g] += 1;
}

template <bool kRle>
__global__ void __launch_bounds__(kTileThreads, kRle ? 2 : kTileMinBlocks) k_rle_write(RleArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  auto* sm = reinterpret_cast<TileSmem<kTileBuf>*>(smem_raw);
  const int lane = threadIdx.x & 31;
  DevCtl* ctl = a.ctl;
  const ColView c = view_of(a.in);
  const uint64_t n = c.n, nch = (n + kBlock - 1) / kBlock;
  const uint64_t R = ldg64(a.coff + nch);
  // the arena top changes only in the last CTA to finish, after every CTA read it
  const uint64_t top = ldg64(&ctl->top);
  const uint64_t size = 16 * R + 8 * nch;
  const bool fits = R <= n && size <= ctl->cap - top;
  uint64_t* vals = reinterpret_cast<uint64_t*>(ctl->arena + top);
  uint64_t* ends = vals + R;
  uint64_t* dir = ends + R;
  if (fits) {
    cta_stream<kTileBuf, kRle>(c, sm, ctl, [&](uint64_t g, const uint64_t* v, int valid, bool) {
      const uint64_t first = __shfl_sync(kFull, v[0], 0);
      const bool h0 = g == 0 || first != ldg64(a.fl + 2 * g - 1);
      uint32_t m = rle_inner_heads(v, valid, lane);
      if (lane == 0 && h0) m |= 1u;
      const uint32_t cnt = (uint32_t)__popc(m);
      const uint64_t c0 = ldg64(a.coff + g);
      uint64_t r = c0 + warp_excl_scan32(cnt, lane);
      const uint64_t row0 = g * kBlock + 16 * (uint64_t)lane;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        if ((m >> k) & 1u) {
          if (r < R) vals[r] = v[k];
          if (r > 0 && r <= R) ends[r - 1] = row0 + k;  // the run before ends here
          r++;
        }
      }
      if (lane == 0) {
        dir[g] = c0 + (h0 ? 1 : 0) - 1;  // the run that holds value 512 g
        if (g == nch - 1 && R > 0) ends[R - 1] = n;
      }
    });
  }
  // epilogue: the last CTA to finish records the column
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      DevMeta* m = a.out_meta;
      m->ptr = reinterpret_cast<uint64_t>(vals);
      m->fmt = (uint32_t)MS_RLE;
      m->bw = 0;
      m->pwords = 0;
      if (fits) {
        m->n = n;
        m->size = size;
        m->nb = R;
        const uint64_t grow = (size + 255) / 256 * 256;
        ctl->top = top + grow;
        if (top + grow > ctl->high) ctl->high = top + grow;
      } else {  // published empty, so that no reader leaves the arena
        set_error(ctl, R > n ? MS_ERR_FORMAT : MS_ERR_NOMEM, size);
        m->n = 0;
        m->size = 0;
        m->nb = 0;
      }
      ctl->done = 0;
      __threadfence();
    }
  }
}

__global__ void k_rle_raw_meta(DevMeta* m, const uint64_t* p, uint64_t n) {
  DevMeta v{};
  v.n = n;
  v.ptr = reinterpret_cast<uint64_t>(p);
  v.size = 8 * n;
  v.fmt = MS_UNCOMPR;
  *m = v;
}

namespace {
constexpr size_t kRleSmem = sizeof(TileSmem<kTileBuf>);

template <class K>
int rle_grid(ms_ctx* c, K kernel, uint64_t n_max) {
  return grid_for(c, kernel, kRleSmem, cdiv(cdiv(std::max<uint64_t>(n_max, 1), kBlock), kClaim), kTileThreads);
}
}  // namespace

// `in` may be null for raw uint64 input (raw, n); the scratch comes from w.
ms_status rle_encode(ms_ctx* c, const DevMeta* in, const uint64_t* raw, uint64_t n_max, const Work& w,
                     ms_column** out, cudaStream_t s, bool in_rle) {
  auto count = in_rle ? k_rle_count<true> : k_rle_count<false>;
  auto write = in_rle ? k_rle_write<true> : k_rle_write<false>;
  if (!in) {  // a column record for the raw input, in scratch the encoder does not use
    DevMeta* m = reinterpret_cast<DevMeta*>(w.status2);
    k_rle_raw_meta<<<1, 1, 0, s>>>(m, raw, n_max);
    if (cuda_status(cudaGetLastError()) != MS_OK) return MS_ERR_CUDA;
    in = m;
  }
  ms_column* col = new_arena_column(c, MS_RLE, 0, n_max);
  if (!col) return MS_ERR_NOMEM;
  RleArgs a{in, c->ctl, c->metas + col->slot, w.counts, w.stage_meta, w.coff};
  ms_status st = MS_OK;
  {
    ProfScope ps(c, MS_K_RLE, s);
    count<<<rle_grid(c, count, n_max), kTileThreads, kRleSmem, s>>>(a);
    st = cuda_status(cudaGetLastError());
    if (st == MS_OK) {
      const uint64_t nch = cdiv(n_max, kBlock);
      const int g = (int)std::max<uint64_t>(1, std::min<uint64_t>(cdiv(nch, 256), 4ull * c->sms));
      k_rle_bounds<<<g, 256, 0, s>>>(a);
      st = cuda_status(cudaGetLastError());
    }
  }
  if (st == MS_OK) {
    MarkArgs m{};
    m.in = in;
    m.ctl = c->ctl;
    st = launch_scan(c, m, w, n_max, s);
  }
  if (st == MS_OK) {
    ProfScope ps(c, MS_K_RLE, s);
    write<<<rle_grid(c, write, n_max), kTileThreads, kRleSmem, s>>>(a);
    st = cuda_status(cudaGetLastError());
  }
  if (st != MS_OK) {
    drop_new_column(c, col);
    return st;
  }
  *out = col;
  return MS_OK;
}

}  // namespace ms
