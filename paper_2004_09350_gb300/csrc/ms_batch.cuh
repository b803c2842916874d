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

// One 512-row chunk of a fragment, resolved once when the batch is bound (64 bytes).
// The hot loop reads this record instead of the columns' metadata and block
// headers: where each column's chunk lives, how it is coded, and the fragment's
// predicate.
//   code[c] = b | kind << 8 | fmt << 12 for column c (0 = x, 1 = y):
//     kind 0: a packed block of width b at addr (64*b bytes; FOR/DELTA use ref),
//     kind 1: raw uint64 values at addr (uncompressed chunk or block-format remainder),
//     kind 2: the horizontally packed tail of a static-BP column at width b.
//   meta = valid rows (1..512) | negate << 16 | empty << 17.
struct ChunkRec {
  uint64_t addr[2];
  uint64_t ref[2];
  uint64_t lo, span;  // predicate: ((x - lo) <= span) != negate, never if empty
  uint32_t code[2];
  uint32_t frag;
  uint32_t meta;
};
static_assert(sizeof(ChunkRec) == 64, "chunk record size");

constexpr int kKindPacked = 0, kKindRaw = 1, kKindTail = 2;

struct BatchArgs {
  const ChunkRec* dir;
  uint64_t c0, c1;     // chunks of this run: [c0, c1)
  uint64_t ntiles;     // ceil((c1 - c0) / tile_chunks)
  uint32_t log2_tile;  // tile_chunks = 1 << log2_tile
  unsigned long long* counter;  // work counter (0 between runs)
  unsigned int* done;           // CTAs finished (0 between runs)
  unsigned long long* sums;     // indexed by fragment id
  DevCtl* ctl;
};

template <int D>
struct BatchSmem {
  uint16_t slot[D][2][32 * kBatchSlotW];
  ChunkRec rec[2 * D];
};

constexpr uint32_t kNoChunk = ~0u;

// Record of chunk g of column c (the directory builder's per-column part).
MS_DEV void resolve_chunk(const ColView& c, uint64_t g, uint64_t* addr, uint64_t* ref, uint32_t* code,
                          DevCtl* ctl) {
  const uint64_t base = (uint64_t)c.p;
  *ref = 0;
  if (c.fmt == MS_UNCOMPR) {
    *addr = base + 4096 * g;
    *code = (uint32_t)kKindRaw << 8 | (uint32_t)MS_UNCOMPR << 12 | 64;
  } else if (c.fmt == MS_STATIC_BP) {
    const uint64_t full = c.n / kBlock;
    *addr = base + 64ull * c.bw * min(g, full);
    *code = (uint32_t)(g < full ? kKindPacked : kKindTail) << 8 | (uint32_t)MS_STATIC_BP << 12 | (uint32_t)c.bw;
  } else if (g < c.nb) {
    uint64_t w0 = 0, r = 0;
    if (16 * (g + 1) <= c.size) {
      w0 = ldg64(c.p + 16 * g);
      r = ldg64(c.p + 16 * g + 8);
    }
    uint32_t b = (uint32_t)(w0 & 255);
    if (16 * (g + 1) > c.size || b > 64 || 16 * c.nb + 8 * ((w0 >> 8) + 8ull * b) > c.size) {
      set_error(ctl, MS_ERR_FORMAT, g);
      b = 0;
      w0 = 0;
    }
    *addr = base + 16 * c.nb + 8 * (w0 >> 8);
    *ref = r;
    *code = (uint32_t)kKindPacked << 8 | (uint32_t)c.fmt << 12 | b;
  } else {
    *addr = base + 16 * c.nb + 8 * c.pwords;
    const uint64_t valid = min((uint64_t)kBlock, c.n - g * kBlock);
    if (16 * c.nb + 8 * (c.pwords + valid) > c.size) set_error(ctl, MS_ERR_FORMAT, g);
    *code = (uint32_t)kKindRaw << 8 | (uint32_t)c.fmt << 12 | 64;
  }
}

// Decodes one column's chunk from its record into lane registers.
template <bool kCompact>
MS_DEV void decode_rec(uint64_t addr, uint64_t ref, uint32_t code, int valid, const uint16_t* slot, int lane,
                       uint64_t v[16]) {
  const int b = (int)(code & 255), kind = (int)((code >> 8) & 15), fmt = (int)(code >> 12);
  if (kind == kKindPacked) {
    const uint16_t* src = b <= kBatchSlotW ? slot : reinterpret_cast<const uint16_t*>(addr);
    read_lane_stream_as<kCompact>(src, lane, b, v);
    if (fmt == MS_FOR_BP) {
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] += ref;
    } else if (fmt == MS_DELTA_BP && b <= 23) {  // 512 residuals < 2^23 sum below 2^32
      uint32_t s = 0;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        s += (uint32_t)v[k];
        v[k] = s;
      }
      const uint64_t excl = (uint64_t)warp_excl_scan32(s, lane) + ref;
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] += excl;
    } else if (fmt == MS_DELTA_BP) {
      uint64_t s = 0;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        s += v[k];
        v[k] = s;
      }
      const uint64_t excl = warp_excl_scan(s, lane) + ref;
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] += excl;
    }
  } else if (kind == kKindRaw) {
    const uint64_t* src = reinterpret_cast<const uint64_t*>(addr) + 16 * lane;
    if (valid == kBlock) {
#pragma unroll
      for (int cc = 0; cc < 8; cc++) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(src) + cc);
        v[2 * cc] = (uint64_t)q.x | ((uint64_t)q.y << 32);
        v[2 * cc + 1] = (uint64_t)q.z | ((uint64_t)q.w << 32);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] = (16 * lane + k < valid) ? ldg64(src + k) : 0;
    }
  } else {  // static-BP tail: values one after the other at width b
    const uint64_t* tail = reinterpret_cast<const uint64_t*>(addr);
    const uint64_t mask = lowmask(b);
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const int t = 16 * lane + k;
      uint64_t x = 0;
      if (t < valid && b) {
        const uint64_t bit = (uint64_t)t * b;
        const int sh = (int)(bit & 63);
        x = ldg64(tail + (bit >> 6)) >> sh;
        if (sh + b > 64) x |= ldg64(tail + (bit >> 6) + 1) << (64 - sh);
        x &= mask;
      }
      v[k] = x;
    }
  }
}

// Persistent kernel over the batch's chunk space, tiles of 2^log2_tile chunks,
// both columns of each chunk streamed with `D` chunks in flight per warp: chunk
// records travel 2D-1 positions ahead of use, payloads D-1 positions ahead.
//
// Dynamic schedule (kStatic false): every warp grabs whole tiles from the work
// counter.  Positions s = 0, 1, ... of a warp's stream map to tile ring[(s >>
// log2_tile) & 1]; the issue stages run at most 2D-1 positions ahead, so two
// tiles (the current and the next) cover them when the tile holds >= 2D chunks.
//
// Static schedule (kStatic true): CTA b owns tiles b, b + gridDim.x, ... and its
// warps share each tile (warp w takes chunks w, w + WARPS, ...).  All warps of a
// CTA then decode the same fragment, so the few width-specialised decoders it
// needs stay in the instruction cache.
template <int WARPS, int D, bool kCompact, bool kStatic>
__global__ void __launch_bounds__(32 * WARPS) k_batch(BatchArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  BatchSmem<D>* sm = reinterpret_cast<BatchSmem<D>*>(smem_raw) + warp;
  const uint32_t lt = a.log2_tile;
  const uint32_t kmask = (1u << lt) - 1;
  // static schedule: 2^lp positions of a warp per tile
  constexpr int kLogW = WARPS == 16 ? 4 : (WARPS == 8 ? 3 : 2);
  const uint32_t lp = lt - kLogW;
  const uint32_t pmask = (1u << lp) - 1;
  const uint32_t span = (uint32_t)(a.c1 - a.c0);  // chunks of this run (< 2^32)

  auto grab = [&]() -> uint32_t {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(a.counter, 1ull);
    return (uint32_t)min((unsigned long long)__shfl_sync(kFull, t, 0), (unsigned long long)a.ntiles);
  };
  const uint32_t ntiles = (uint32_t)a.ntiles;
  uint32_t ring0 = kStatic ? blockIdx.x : grab(), ring1 = ntiles;
  auto tile_of = [&](uint32_t s) -> uint32_t {
    if constexpr (kStatic) return blockIdx.x + (s >> lp) * gridDim.x;
    return ((s >> lt) & 1) ? ring1 : ring0;
  };
  // run-relative chunk at stream position s, or kNoChunk
  auto chunk_at = [&](uint32_t s) -> uint32_t {
    const uint32_t t = tile_of(s);
    if (t >= ntiles) return kNoChunk;
    const uint32_t g = kStatic ? (t << lt) + warp + ((s & pmask) << kLogW) : (t << lt) + (s & kmask);
    return g < span ? g : kNoChunk;
  };
  const ChunkRec* dir = a.dir + a.c0;

  auto issue_rec = [&](uint32_t s) {
    const uint32_t g = chunk_at(s);
    if (g != kNoChunk && lane < 4)
      cp_async16(reinterpret_cast<uint4*>(&sm->rec[s % (2 * D)]) + lane, reinterpret_cast<const uint4*>(dir + g) + lane);
  };
  auto issue_payload = [&](uint32_t s) {
    if (chunk_at(s) == kNoChunk) return;
    const ChunkRec& r = sm->rec[s % (2 * D)];
#pragma unroll
    for (int col = 0; col < 2; col++) {
      const uint32_t code = r.code[col];
      const int b = (int)(code & 255);
      if (((code >> 8) & 15) != kKindPacked || b > kBatchSlotW) continue;
      const uint4* src = reinterpret_cast<const uint4*>(r.addr[col]);
      uint4* dst = reinterpret_cast<uint4*>(sm->slot[s % D][col]);
      for (int u = lane; u < 4 * b; u += 32) cp_async16(dst + u, src + u);
    }
  };

  uint64_t acc = 0;          // this lane's part of fragment acc_f's sum
  uint32_t acc_f = ~0u;
  auto flush = [&]() {
    const uint64_t t = warp_sum(acc);
    if (lane == 0 && acc_f != ~0u && t) atomicAdd(a.sums + acc_f, (unsigned long long)t);
    acc = 0;
  };

  if (ring0 < ntiles) {
    for (int i = 0; i < D; i++) issue_rec(i);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    for (int j = 0; j < D - 1; j++) {
      issue_rec(j + D);
      issue_payload(j);
      cp_async_commit();
    }
    for (uint32_t s = 0;; s++) {
      if constexpr (kStatic) {
        if ((s & pmask) == 0 && tile_of(s) >= ntiles) break;
      } else if ((s & kmask) == 0) {
        // entering tile s >> lt: stop at a dead tile, else fetch the one after it
        if ((((s >> lt) & 1) ? ring1 : ring0) >= ntiles) break;
        const uint32_t nxt = grab();
        if ((s >> lt) & 1) ring0 = nxt;
        else ring1 = nxt;
      }
      cp_async_wait<D - 2>();
      __syncwarp();
      issue_rec(s + 2 * D - 1);
      issue_payload(s + D - 1);
      cp_async_commit();
      if (chunk_at(s) != kNoChunk) {
        const ChunkRec& r = sm->rec[s % (2 * D)];
        const uint32_t f = r.frag;
        if (f != acc_f) {
          flush();
          acc_f = f;
        }
        const uint32_t meta = r.meta;
        const int valid = (int)(meta & 1023);
        const uint64_t lo = r.lo, pspan = r.span;
        uint32_t m16 = 0;
        // one decoder instance for both columns keeps the instruction footprint small
#pragma unroll 1
        for (int col = 0; col < 2; col++) {
          uint64_t v[16];
          decode_rec<kCompact>(r.addr[col], r.ref[col], r.code[col], valid, sm->slot[s % D][col], lane, v);
          if (col == 0) {
#pragma unroll
            for (int k = 0; k < 16; k++) m16 |= (uint32_t)(v[k] - lo <= pspan) << k;
            const int first = 16 * lane;
            m16 = (m16 ^ ((meta >> 16) & 1 ? 0xffffu : 0u)) & ((meta >> 17) & 1 ? 0u : 0xffffu) &
                  (valid >= first + 16 ? 0xffffu : (valid > first ? (1u << (valid - first)) - 1u : 0u));
          } else {
#pragma unroll
            for (int k = 0; k < 16; k++)
              if ((m16 >> k) & 1u) acc += v[k];
          }
        }
      }
      __syncwarp();
    }
    cp_async_wait<0>();
    flush();
  }
  if constexpr (kStatic) return;
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

// ------------------------------------------------------ CTA-streamed schedule

// Schedule 2: the CTA tile stream of the single-column consumers, extended to the
// batch.  A CTA claims kBClaim consecutive chunks (claims b, b + gridDim.x, ...);
// their directory records load one claim ahead.  Inside one fragment the x and y
// payloads of consecutive packed chunks are contiguous, so the CTA copies a run of
// chunks of one fragment (as many as fit in both buffers) with all its threads,
// and its warps decode the run from shared memory while the next run loads.
// Uncompressed chunks, remainders and static tails are read in place.
constexpr int kBClaim = 64;

template <int BUF>
struct BatchCtaSmem {
  uint8_t xbuf[2][BUF];
  uint8_t ybuf[2][BUF];
  ChunkRec rec[3][kBClaim];  // the decoded claim, the scheduled claim, the next claim
};

// end of a chunk's staged bytes (its start when it is read in place)
MS_DEV uint64_t staged_end(const ChunkRec& r, int col) {
  const uint32_t code = r.code[col];
  const bool packed = ((code >> 8) & 15) == kKindPacked;
  return r.addr[col] + (packed ? 64ull * (code & 255) : 0);
}

template <int BUF, bool kCompact>
__global__ void __launch_bounds__(256) k_batch_cta(BatchArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  auto* sm = reinterpret_cast<BatchCtaSmem<BUF>*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
  const uint64_t span = a.c1 - a.c0;
  const uint64_t nclaims = (span + kBClaim - 1) / kBClaim;
  const ChunkRec* dir = a.dir + a.c0;
  auto load_rec = [&](uint64_t claim, int rb) {
    if (claim >= nclaims) return;
    for (int u = tid; u < 4 * kBClaim; u += blockDim.x) {
      const uint64_t g = claim * kBClaim + (u >> 2);
      if (g < span)
        cp_async16(reinterpret_cast<uint4*>(&sm->rec[rb][u >> 2]) + (u & 3),
                   reinterpret_cast<const uint4*>(dir + g) + (u & 3));
    }
  };
  uint64_t claim = blockIdx.x;
  if (claim >= nclaims) return;
  int rb = 0;
  uint64_t cb = claim * kBClaim, ce = min(span, cb + kBClaim), g = cb;
  load_rec(claim, 0);
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  load_rec(claim + gridDim.x, 1);
  // the run in flight / being decoded: chunks [ga, gb) of claim (rb_s, cb_s), buffer bi
  uint64_t ga = 0, gb = 0, cb_s = cb, x0 = 0, y0 = 0;
  int rb_s = 0, bi = 0;
  auto schedule = [&](int nbi) -> bool {
    if (g >= ce) {  // next claim (its records landed with an earlier group)
      claim += gridDim.x;
      if (claim >= nclaims) return false;
      rb = rb == 2 ? 0 : rb + 1;
      cb = claim * kBClaim;
      ce = min(span, cb + kBClaim);
      g = cb;
      load_rec(claim + gridDim.x, rb == 2 ? 0 : rb + 1);
    }
    const ChunkRec& r0 = sm->rec[rb][g - cb];
    const uint32_t f0 = r0.frag;
    const uint64_t sx = r0.addr[0], sy = r0.addr[1];
    // chunks of the claim in g's fragment whose staged bytes end within both buffers
    bool fits = false;
    if ((uint64_t)tid < ce - g) {
      const ChunkRec& r = sm->rec[rb][g + tid - cb];
      fits = r.frag == f0 && staged_end(r, 0) - sx <= (uint64_t)BUF && staged_end(r, 1) - sy <= (uint64_t)BUF;
    }
    const uint64_t cnt = max(1, __syncthreads_count(fits));
    const ChunkRec& rl = sm->rec[rb][g + cnt - 1 - cb];
    const uint64_t bx = min(staged_end(rl, 0) - sx, (uint64_t)BUF) & ~15ull;
    const uint64_t by = min(staged_end(rl, 1) - sy, (uint64_t)BUF) & ~15ull;
    for (uint32_t u = tid; u < (uint32_t)(bx >> 4); u += blockDim.x)
      cp_async16(reinterpret_cast<uint4*>(sm->xbuf[nbi]) + u, reinterpret_cast<const uint4*>(sx) + u);
    for (uint32_t u = tid; u < (uint32_t)(by >> 4); u += blockDim.x)
      cp_async16(reinterpret_cast<uint4*>(sm->ybuf[nbi]) + u, reinterpret_cast<const uint4*>(sy) + u);
    ga = g;
    gb = g + cnt;
    cb_s = cb;
    rb_s = rb;
    x0 = sx;
    y0 = sy;
    g += cnt;
    return true;
  };
  bool live = schedule(0);
  cp_async_commit();
  while (live) {
    cp_async_wait<0>();
    __syncthreads();
    const uint64_t da = ga, db = gb, dcb = cb_s, dx0 = x0, dy0 = y0;
    const int drb = rb_s, dbi = bi;
    bi ^= 1;
    live = schedule(bi);
    cp_async_commit();
    uint64_t acc = 0;
    for (uint64_t k = da + warp; k < db; k += nwarps) {
      const ChunkRec& r = sm->rec[drb][k - dcb];
      const uint32_t meta = r.meta;
      const int valid = (int)(meta & 1023);
      const uint64_t lo = r.lo, pspan = r.span;
      uint32_t m16 = 0;
#pragma unroll 1
      for (int col = 0; col < 2; col++) {
        const uint32_t code = r.code[col];
        const bool packed = ((code >> 8) & 15) == kKindPacked;
        const uint8_t* base = col ? sm->ybuf[dbi] : sm->xbuf[dbi];
        const uint64_t start = col ? dy0 : dx0;
        // a staged chunk lies inside the copied run: its bytes were checked against
        // the buffer when the run was cut
        const bool staged = packed && r.addr[col] >= start && r.addr[col] + 64ull * (code & 255) - start <= BUF;
        uint64_t v[16];
        if (staged) {
          decode_rec<kCompact>(r.addr[col], r.ref[col], code, valid,
                               reinterpret_cast<const uint16_t*>(base + (r.addr[col] - start)), lane, v);
        } else {
          // in place: a raw chunk, or (never for a consistent directory) a packed one outside the run
          decode_rec<kCompact>(r.addr[col], r.ref[col], code, valid, reinterpret_cast<const uint16_t*>(r.addr[col]),
                               lane, v);
        }
        if (col == 0) {
#pragma unroll
          for (int q = 0; q < 16; q++) m16 |= (uint32_t)(v[q] - lo <= pspan) << q;
          const int first = 16 * lane;
          m16 = (m16 ^ ((meta >> 16) & 1 ? 0xffffu : 0u)) & ((meta >> 17) & 1 ? 0u : 0xffffu) &
                (valid >= first + 16 ? 0xffffu : (valid > first ? (1u << (valid - first)) - 1u : 0u));
        } else {
#pragma unroll
          for (int q = 0; q < 16; q++)
            if ((m16 >> q) & 1u) acc += v[q];
        }
      }
    }
    // every chunk of a run belongs to one fragment
    const uint64_t t = warp_sum(acc);
    if (lane == 0 && t && da + warp < db)
      atomicAdd(a.sums + sm->rec[drb][da - dcb].frag, (unsigned long long)t);
    __syncthreads();
  }
  cp_async_wait<0>();
}

template <int BUF, bool kCompact>
ms_status launch_batch_cta(ms_ctx* c, const BatchArgs& a, uint32_t ctas_per_sm, cudaStream_t s) {
  static int occ_cache[16];
  const size_t smem = sizeof(BatchCtaSmem<BUF>);
  const int dev = c->device;
  int occ = (dev >= 0 && dev < 16) ? occ_cache[dev] : 0;
  if (occ == 0) {
    if (cuda_status(cudaFuncSetAttribute(k_batch_cta<BUF, kCompact>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem)) != MS_OK)
      return MS_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_cta<BUF, kCompact>, 256, smem) != cudaSuccess ||
        occ < 1)
      occ = 1;
    if (dev >= 0 && dev < 16) occ_cache[dev] = occ;
  }
  if (a.ntiles == 0) return MS_OK;
  if (ctas_per_sm) occ = std::min<int>(occ, (int)ctas_per_sm);
  const uint64_t claims = cdiv(a.c1 - a.c0, kBClaim);
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)occ * (uint64_t)c->sms, claims));
  k_batch_cta<BUF, kCompact><<<grid, 256, smem, s>>>(a);
  return cuda_status(cudaGetLastError());
}

// Launches k_batch<WARPS, D, kCompact> over a.ntiles tiles; grid capped at the
// resident CTAs (ctas_per_sm per SM when nonzero).  With a.ntiles == 0 it only sets
// the kernel's shared-memory attribute and caches its occupancy (done before a
// stream capture).
template <int WARPS, int D, bool kCompact, bool kStatic>
ms_status launch_batch_kernel(ms_ctx* c, const BatchArgs& a, uint32_t ctas_per_sm, cudaStream_t s) {
  static int occ_cache[16];  // per device; 0 = not yet known, -1 = does not fit
  const size_t smem = sizeof(BatchSmem<D>) * WARPS;
  const int dev = c->device;
  int occ = (dev >= 0 && dev < 16) ? occ_cache[dev] : 0;
  if (occ == 0) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem > (size_t)optin) {
      occ = -1;
    } else {
      if (smem > 48 * 1024 &&
          cuda_status(cudaFuncSetAttribute(k_batch<WARPS, D, kCompact, kStatic>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != MS_OK)
        return MS_ERR_CUDA;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<WARPS, D, kCompact, kStatic>, 32 * WARPS,
                                                        smem) != cudaSuccess ||
          occ < 1)
        occ = 1;
    }
    if (dev >= 0 && dev < 16) occ_cache[dev] = occ;
  }
  if (occ < 0) return MS_ERR_INVALID_ARG;  // the configuration's shared memory does not fit
  if (a.ntiles == 0) return MS_OK;
  if (ctas_per_sm) occ = std::min<int>(occ, (int)ctas_per_sm);
  const uint64_t full = (uint64_t)occ * (uint64_t)c->sms;
  const uint64_t want = kStatic ? a.ntiles : cdiv(a.ntiles, WARPS);
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(full, want));
  k_batch<WARPS, D, kCompact, kStatic><<<grid, 32 * WARPS, smem, s>>>(a);
  return cuda_status(cudaGetLastError());
}

using BatchLauncher = ms_status (*)(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t);

// Launcher of (warps, depth, compact, schedule), or nullptr for an unsupported
// combination.
BatchLauncher batch_launcher(uint32_t warps, uint32_t depth, bool compact, uint32_t schedule);

#define MS_BATCH_LAUNCHER(W, D, C, S) \
  launch_batch_kernel<W, D, C, S>(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t);
// dynamic schedule: warps {4, 8} x depth D x both decoders
#define MS_BATCH_DYNAMIC(X, D) \
  X template ms_status MS_BATCH_LAUNCHER(4, D, false, false) X template ms_status MS_BATCH_LAUNCHER(8, D, false, false) \
  X template ms_status MS_BATCH_LAUNCHER(4, D, true, false) X template ms_status MS_BATCH_LAUNCHER(8, D, true, false)
#define MS_BATCH_CTA(X)                                                                          \
  X template ms_status launch_batch_cta<16384, false>(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t); \
  X template ms_status launch_batch_cta<24576, false>(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t); \
  X template ms_status launch_batch_cta<32768, false>(ms_ctx*, const BatchArgs&, uint32_t, cudaStream_t);
// static schedule: width-specialised decoders, warps {4, 8, 16} x depth {2, 3}
#define MS_BATCH_STATIC(X)                                                                                        \
  X template ms_status MS_BATCH_LAUNCHER(4, 2, false, true) X template ms_status MS_BATCH_LAUNCHER(8, 2, false, true) \
  X template ms_status MS_BATCH_LAUNCHER(16, 2, false, true) X template ms_status MS_BATCH_LAUNCHER(4, 3, false, true) \
  X template ms_status MS_BATCH_LAUNCHER(8, 3, false, true)

}  // namespace ms
