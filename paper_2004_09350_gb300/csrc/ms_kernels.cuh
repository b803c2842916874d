// ms_kernels.cuh -- operator kernels of libms (sm_103a).
//
// A warp owns one 512-value chunk at a time.  Input blocks are decoded into lane
// registers, the operator core runs on the uncompressed values, and output blocks
// are recompressed in shared memory before they are stored.  This is the
// on-the-fly de/re-compression degree of Sec. 3.2 at block granularity: only
// compressed bytes travel to and from device memory.
//   * Consumers (mark, agg_sum, semi-join build, statistics) read their column
//     through the CTA tile stream (cta_stream): runs of consecutive blocks copied
//     into shared memory with all the CTA's threads, double-buffered.
//   * Producers (k_map: compress, decompress, project, calc, emit) encode each
//     output block into a stage at the arena's free end; a placement pass
//     (k_place, ms_place.cu) turns the block widths into payload offsets with a
//     decoupled look-back and moves the payloads into place.  Project gathers a CTA tile of sorted positions from
//     the data blocks they span, staged the same way (gather_cta).
//   * k_produce is the direct-offset compress of the allocation-free path: payload
//     offsets from a decoupled look-back inside the kernel, no placement pass.
#pragma once
#include <type_traits>

#include "ms_device.cuh"

namespace ms {

// --------------------------------------------------- CTA tile streams

// A CTA's stream of one column through two large shared-memory buffers.  Block
// payloads of consecutive chunks are contiguous in every format, so the CTA
// copies a whole run of chunks (a sub-tile, as many as fit in one buffer) with
// all its threads at once, and its warps then decode the run's chunks from
// shared memory while the next run loads into the other buffer.  Per chunk this
// leaves a header read from shared memory: no per-chunk copy bookkeeping.
// Chunks come in claims of kClaim consecutive chunks, CTA b taking claims b,
// b + gridDim.x, ...; a claim's block headers are loaded one claim ahead into a
// ring of three header buffers.
constexpr int kClaim = 128;
#ifndef MS_TILE_BUF
#define MS_TILE_BUF 32768
#endif
#ifndef MS_TILE_THREADS
#define MS_TILE_THREADS 256
#endif
#ifndef MS_TILE_MINB
#define MS_TILE_MINB 3
#endif
constexpr int kTileBuf = MS_TILE_BUF;          // bytes per buffer (two per CTA)
constexpr int kTileThreads = MS_TILE_THREADS;  // threads per CTA of the tile-stream kernels
constexpr int kTileMinBlocks = MS_TILE_MINB;

template <int BUF>
struct TileSmem {
  uint8_t buf[2][BUF];
  uint4 hdr[3][kClaim];  // the decoded claim, the scheduled claim, the next claim
};

// Calls body(g, v, valid, narrow) for every chunk g of c; v is zero past `valid`,
// and narrow says that every value of the chunk is below 2^32 (a block or static
// width of at most 32 bits).  Every thread of the CTA must call it (it
// synchronises the CTA).
// The CTA takes claims claim0, claim0 + cstride, ... (by default blockIdx.x and
// gridDim.x).
// The tile stream of an RLE column: the CTA's warps expand its claims' blocks from
// the runs (rle_expand_at), each warp loading the directory entries of its next block
// one ahead.  Kernels instantiate it in place of cta_stream for RLE inputs (cta_stream's
// kRle), so that the other formats' kernels keep their registers.
template <class Body>
MS_DEV void rle_stream(const ColView& c, DevCtl* ctl, Body& body, uint64_t claim0, uint64_t cstride) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const uint64_t nch = (c.n + kBlock - 1) / kBlock;
  const uint64_t nclaims = (nch + kClaim - 1) / kClaim;
  const uint64_t R = c.nb;
  const uint64_t* val = reinterpret_cast<const uint64_t*>(c.p);
  // the runs of a block when at most 32 cover it (lane i: end and value of run r0 + i);
  // returns their count, or 0 when the block is expanded by a search instead
  auto load_runs = [&](uint64_t d, uint64_t& e, uint64_t& x) -> int {
    const uint64_t r0 = __shfl_sync(kFull, d, 0), r1 = __shfl_sync(kFull, d, 1);
    if (!rle_sound(c) || r0 >= R || r1 >= R || r1 < r0 || r1 - r0 >= 32) return 0;
    const int m = (int)(r1 - r0) + 1;
    if (lane < m) {
      e = ldg64(val + R + r0 + lane);
      x = ldg64(val + r0 + lane);
    }
    return m;
  };
  for (uint64_t cl = claim0; cl < nclaims; cl += cstride) {
    const uint64_t end = min(nch, (cl + 1) * kClaim);
    uint64_t k = cl * kClaim + warp;
    // block k: directory entries d0 and runs (m0, e0, x0); block k + nwarps: d1, its
    // runs loaded while block k is expanded; block k + 2 nwarps: d2
    uint64_t d0 = k < end ? rle_dir_load(c, k, lane) : 0;
    uint64_t d1 = k + nwarps < end ? rle_dir_load(c, k + nwarps, lane) : 0;
    uint64_t e0 = 0, x0 = 0;
    int m0 = k < end ? load_runs(d0, e0, x0) : 0;
    for (; k < end; k += nwarps) {
      const uint64_t d2 = k + 2 * nwarps < end ? rle_dir_load(c, k + 2 * nwarps, lane) : 0;
      uint64_t e1 = 0, x1 = 0;
      const int m1 = k + nwarps < end ? load_runs(d1, e1, x1) : 0;
      const int valid = (int)min((uint64_t)kBlock, c.n - k * kBlock);
      uint64_t v[16];
      if (m0 > 0) rle_values_from_runs(k * kBlock + 16 * (uint64_t)lane, lane, valid, m0, e0, x0, v);
      else rle_expand_at(c, k, lane, valid, d0, v, ctl);
      body(k, v, valid, false);
      d0 = d1;
      d1 = d2;
      e0 = e1;
      x0 = x1;
      m0 = m1;
    }
    __syncthreads();
  }
}

// kRle: the kernel's instantiation for RLE inputs (rle_stream); the other one reports
// an RLE input as a format error.
template <int BUF, bool kRle = false, class Body>
MS_DEV void cta_stream(const ColView& c, TileSmem<BUF>* sm, DevCtl* ctl, Body body, uint64_t claim0 = ~0ull,
                       uint64_t cstride = 0) {
  static_assert(BUF >= 4096 && BUF % 4096 == 0, "buffer size");
  const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
  const uint64_t nch = (c.n + kBlock - 1) / kBlock;
  const uint64_t nclaims = (nch + kClaim - 1) / kClaim;
  const bool blockfmt = is_block_fmt(c.fmt);
  const uint64_t full = blockfmt ? c.nb : c.n / kBlock;  // chunks held in the buffers
  // fixed bytes per chunk (static / uncompressed); 0 for block formats
  const uint32_t fixed = c.fmt == MS_UNCOMPR ? 4096u : (c.fmt == MS_STATIC_BP ? 64u * (uint32_t)c.bw : 0u);
  const uint64_t pay0 = 16 * c.nb;  // byte offset of the block payloads (block formats)

  if (kRle || c.fmt == MS_RLE) {  // runs are read from global memory: nothing to stage
    if constexpr (kRle) {
      if (claim0 == ~0ull) {
        claim0 = blockIdx.x;
        cstride = gridDim.x;
      }
      rle_stream(c, ctl, body, claim0, cstride);
    } else if (blockIdx.x == 0 && threadIdx.x == 0) {
      set_error(ctl, MS_ERR_FORMAT, c.n);
    }
    return;
  }

  auto load_hdr = [&](uint64_t claim, int hb) {
    if (!blockfmt || claim >= nclaims) return;
    for (int k = tid; k < kClaim; k += nthr) {
      const uint64_t g = claim * kClaim + k;
      if (g < c.nb && 16 * (g + 1) <= c.size) cp_async16(&sm->hdr[hb][k], reinterpret_cast<const uint4*>(c.p) + g);
    }
  };
  // payload word offset and width of chunk g of the claim in header buffer hb
  auto hdr_of = [&](uint64_t g, uint64_t cb, int hb, uint64_t* off, uint32_t* b, uint64_t* ref) {
    const uint4 h = sm->hdr[hb][g - cb];
    const uint64_t w0 = (uint64_t)h.x | (uint64_t)h.y << 32;
    *ref = (uint64_t)h.z | (uint64_t)h.w << 32;
    *off = w0 >> 8;
    *b = (uint32_t)(w0 & 255);
  };
  // end (exclusive) of chunk g's payload, in bytes from the payload start
  auto end_bytes = [&](uint64_t g, uint64_t cb, int hb) -> uint64_t {
    if (!blockfmt) return (uint64_t)fixed * (g + 1);
    if (g >= c.nb) return 8 * c.pwords;
    uint64_t off, ref;
    uint32_t b;
    hdr_of(g, cb, hb, &off, &b, &ref);
    return 8 * (off + 8ull * min(b, 64u));
  };
  auto start_bytes = [&](uint64_t g, uint64_t cb, int hb) -> uint64_t {
    if (!blockfmt) return (uint64_t)fixed * g;
    if (g >= c.nb) return 8 * c.pwords;
    uint64_t off, ref;
    uint32_t b;
    hdr_of(g, cb, hb, &off, &b, &ref);
    return 8 * off;
  };

  if (claim0 == ~0ull) {
    claim0 = blockIdx.x;
    cstride = gridDim.x;
  }
  uint64_t claim = claim0;
  if (claim >= nclaims) return;
  int hb = 0;
  uint64_t cb = claim * kClaim, ce = min(nch, cb + kClaim), g = cb;
  load_hdr(claim, 0);
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  load_hdr(claim + cstride, 1);  // one claim ahead (header buffers rotate 0, 1, 2)
  // the sub-tile in flight / being decoded: chunks [ga, gb) of claim (hb_s, cb_s) in buffer bi
  uint64_t ga = 0, gb = 0, base = 0, cb_s = cb;
  int hb_s = 0, bi = 0;
  bool live = false;
  // schedules the next sub-tile from the current claim into buffer nbi and issues its copy
  auto schedule = [&](int nbi) -> bool {
    if (g >= ce) {  // next claim (its headers landed with an earlier group)
      claim += cstride;
      if (claim >= nclaims) return false;
      hb = hb == 2 ? 0 : hb + 1;
      cb = claim * kClaim;
      ce = min(nch, cb + kClaim);
      g = cb;
      load_hdr(claim + cstride, hb == 2 ? 0 : hb + 1);
    }
    const uint64_t s0 = start_bytes(g, cb, hb);
    // chunks of the claim whose payload ends within one buffer from s0 (ends are monotone)
    uint64_t cnt;
    if (blockfmt) {
      const uint64_t k = g + tid;
      const bool fits = k < ce && end_bytes(k, cb, hb) - s0 <= (uint64_t)BUF;
      cnt = (uint64_t)__syncthreads_count(fits);
      cnt = max(cnt, (uint64_t)1);  // a corrupt header never stalls the stream
    } else {
      cnt = min(ce - g, (uint64_t)(BUF / max(fixed, 1u)));
    }
    const uint64_t e = g + cnt;
    uint64_t bytes = min(end_bytes(e - 1, cb, hb), blockfmt ? (uint64_t)(c.size - pay0) : (uint64_t)c.size) - s0;
    bytes = min(bytes, (uint64_t)BUF) & ~15ull;
    const uint8_t* src = c.p + (blockfmt ? pay0 : 0) + s0;
    uint4* dst = reinterpret_cast<uint4*>(sm->buf[nbi]);
    const uint32_t units = (uint32_t)(bytes >> 4);
    if (c.fmt == MS_UNCOMPR) {
      for (uint32_t u = tid; u < units; u += nthr)
        cp_async16(dst + (((u >> 3) << 3) | ((u & 7) ^ ((u >> 3) & 7))), reinterpret_cast<const uint4*>(src) + u);
    } else {
      for (uint32_t u = tid; u < units; u += nthr) cp_async16(dst + u, reinterpret_cast<const uint4*>(src) + u);
    }
    ga = g;
    gb = e;
    base = s0;
    cb_s = cb;
    hb_s = hb;
    g = e;
    return true;
  };
  live = schedule(0);
  cp_async_commit();
  while (live) {
    cp_async_wait<0>();
    __syncthreads();
    // this sub-tile (decoded below) and the next one (loading meanwhile)
    const uint64_t da = ga, db = gb, dbase = base, dcb = cb_s;
    const int dhb = hb_s, dbi = bi;
    bi ^= 1;
    live = schedule(bi);
    cp_async_commit();
    for (uint64_t k = da + warp; k < db; k += nwarps) {
      const int valid = (int)min((uint64_t)kBlock, c.n - k * kBlock);
      uint64_t v[16];
      bool narrow = c.fmt == MS_STATIC_BP && c.bw <= 32;
      if (k < full) {
        uint32_t b;
        uint64_t off, ref = 0;
        const uint8_t* at;
        if (blockfmt) {
          hdr_of(k, dcb, dhb, &off, &b, &ref);
          // a corrupt header can point outside the column or the staged run
          if (b > 64 || 8 * (off + 8ull * b) + pay0 > c.size || 8 * off < dbase ||
              8 * (off + 8ull * b) - dbase > (uint64_t)BUF) {
            if (lane == 0) set_error(ctl, MS_ERR_FORMAT, k);
            b = 0;
            off = dbase / 8;
          }
          at = sm->buf[dbi] + (8 * off - dbase);
        } else {
          b = (uint32_t)c.bw;
          at = sm->buf[dbi] + (uint64_t)fixed * k - dbase;
        }
        narrow = (c.fmt == MS_DYN_BP || c.fmt == MS_STATIC_BP) && b <= 32;
        if (c.fmt == MS_UNCOMPR) {
          const uint4* st = reinterpret_cast<const uint4*>(at);
#pragma unroll
          for (int cc = 0; cc < 8; cc++) {
            const uint4 q = st[lane * 8 + (cc ^ (lane & 7))];
            v[2 * cc] = (uint64_t)q.x | ((uint64_t)q.y << 32);
            v[2 * cc + 1] = (uint64_t)q.z | ((uint64_t)q.w << 32);
          }
        } else {
          read_lane_stream(reinterpret_cast<const uint16_t*>(at), lane, (int)b, v);
          if (c.fmt == MS_FOR_BP) {
#pragma unroll
            for (int q = 0; q < 16; q++) v[q] += ref;
          } else if (c.fmt == MS_DELTA_BP && b <= 23) {  // 32-bit prefix sums (see decode_staged)
            uint32_t sum = 0;
#pragma unroll
            for (int q = 0; q < 16; q++) {
              sum += (uint32_t)v[q];
              v[q] = sum;
            }
            const uint64_t excl = (uint64_t)warp_excl_scan32(sum, lane) + ref;
#pragma unroll
            for (int q = 0; q < 16; q++) v[q] += excl;
          } else if (c.fmt == MS_DELTA_BP) {
            uint64_t sum = 0;
#pragma unroll
            for (int q = 0; q < 16; q++) {
              sum += v[q];
              v[q] = sum;
            }
            const uint64_t excl = warp_excl_scan(sum, lane) + ref;
#pragma unroll
            for (int q = 0; q < 16; q++) v[q] += excl;
          }
        }
      } else if (c.fmt == MS_STATIC_BP) {  // horizontal tail
        const uint64_t* tailp = reinterpret_cast<const uint64_t*>(c.p + 64ull * c.bw * full);
        const int bw = c.bw;
        const uint64_t mask = lowmask(bw);
#pragma unroll
        for (int q = 0; q < 16; q++) {
          const int t = 16 * lane + q;
          uint64_t x = 0;
          if (t < valid) {
            const uint64_t bit = (uint64_t)t * bw;
            const int sh = (int)(bit & 63);
            x = ldg64(tailp + (bit >> 6)) >> sh;
            if (sh + bw > 64) x |= ldg64(tailp + (bit >> 6) + 1) << (64 - sh);
            x &= mask;
          }
          v[q] = x;
        }
      } else {  // raw values: a partial uncompressed chunk or the block formats' remainder
        const uint64_t* rawp = reinterpret_cast<const uint64_t*>(
            c.fmt == MS_UNCOMPR ? c.p + 4096 * k : c.p + pay0 + 8 * c.pwords);
        const bool inside = c.fmt == MS_UNCOMPR || pay0 + 8 * (c.pwords + (uint64_t)valid) <= c.size;
        if (!inside && lane == 0) set_error(ctl, MS_ERR_FORMAT, k);
#pragma unroll
        for (int q = 0; q < 16; q++) v[q] = (16 * lane + q < valid && inside) ? ldg64(rawp + 16 * lane + q) : 0;
      }
      body(k, v, valid, narrow);
    }
    __syncthreads();
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------- consumer kernel arguments

// Select / semi-join mark kernel arguments (kernel in ms_consume.cu).
struct MarkArgs {
  const DevMeta* in;
  DevCtl* ctl;
  int rle;  // the input is RLE (selects the kernels' RLE instantiation on the host)
  // the predicate as one range test: hit = ((x - lo) <= span) != negate, never if empty
  uint64_t lo, span;
  uint32_t negate, empty;
  // the same range restricted to x < 2^32, for chunks whose values all fit 32 bits:
  // hit = (uint32(x - lo32) <= span32) != negate; mode32 1 = no x < 2^32 is in the
  // range, 2 = every one is (negate and empty apply as above)
  uint32_t lo32, span32, mode32;
  const uint32_t* keybits;  // semi-join: membership bitmap over the key domain
  uint64_t domain;
  uint16_t* bitmap;
  uint32_t* counts;
};



// Scan of per-chunk match counts (kernel in ms_consume.cu).
struct ScanArgs {
  const DevMeta* in;
  DevCtl* ctl;
  const uint32_t* counts;
  uint64_t* coff;
  uint64_t* bstart;
  uint64_t* status;
};

constexpr int kSmemGroups = 4096;
constexpr int kPairDepth = 2;        // two columns per warp: shallower rings
constexpr int kPairWarps = 4;        // 128-thread CTAs for the two-column consumers

// Two-column consumer: gid and val chunks of the same index stream side by side.
template <class Body>
MS_DEV void stream_pairs(const ColView& c0, const ColView& c1, uint64_t n, uint64_t first, uint64_t stride,
                         StreamSmem<kPairDepth>* s0, StreamSmem<kPairDepth>* s1, int lane, DevCtl* ctl, Body body) {
  constexpr int D = kPairDepth;
  const uint64_t nch = (n + kBlock - 1) / kBlock;
  const uint64_t count = first < nch ? (nch - first + stride - 1) / stride : 0;
  ChunkStream<D> a{c0, first, stride, count, s0, lane};
  ChunkStream<D> b{c1, first, stride, count, s1, lane};
  if (count == 0) return;
  for (int i = 0; i < D; i++) {
    a.issue_header(i);
    b.issue_header(i);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncwarp();
  for (int j = 0; j < D - 1; j++) {
    a.prologue_step(j);
    b.prologue_step(j);
    cp_async_commit();
  }
  for (uint64_t i = 0; i < count; i++) {
    cp_async_wait<D - 2>();
    __syncwarp();
    a.step(i);
    b.step(i);
    cp_async_commit();
    uint64_t u[16], v[16];
    const int va = a.decode(i, u, ctl);
    const int vb = b.decode(i, v, ctl);
    body(a.chunk(i), u, v, min(va, vb));
    __syncwarp();
  }
  cp_async_wait<0>();
}


// ------------------------------------------------------- produce (map) kernel

enum ProduceOp { OP_COMPRESS = 0, OP_DECOMPRESS = 1, OP_PROJECT = 2, OP_CALC = 3, OP_EMIT = 4, OP_PROJECT_WARP = 5 };

struct ProduceArgs {
  DevCtl* ctl;
  // inputs
  const DevMeta* in0;      // decompress / calc a / project data
  const DevMeta* in1;      // calc b (NULL: scalar) / project positions
  const uint64_t* raw_in;  // compress input
  uint64_t raw_n;          // compress input length
  int arith;
  uint64_t scalar;
  // emit inputs
  const uint16_t* bitmap;
  const uint64_t* coff;
  const uint64_t* bstart;
  uint64_t emit_nch;       // input chunks of the mark step
  // output
  DevMeta* out_meta;       // arena output (NULL: raw output)
  uint64_t* raw_out;
  uint64_t raw_cap;
  int fmt, bw;
  uint64_t* status;
  // staged block-format output (k_map): per output block {(stage offset << 8) |
  // width, reference}; the payloads sit in the stage at the arena's end, and k_place
  // places them
  uint64_t* stage_meta;
};

// Per-warp shared memory of each producing operator.  The slot of the main input
// stream that a warp has just decoded doubles as its output stage.
constexpr int kProdDepth = 3;   // single-input producers
constexpr int kProdDepth2 = 2;  // two-input producers
constexpr int kEmitSpan = 32;   // bitmap chunks an emit warp stages at once

struct SmemSingle {
  StreamSmem<kProdDepth> s0;
};
struct SmemPair {
  StreamSmem<kProdDepth2> s0, s1;
};
struct SmemProjectRandom {
  StreamSmem<kProdDepth2> s0;  // positions
};
struct SmemProjectDelta {
  StreamSmem<kProdDepth2> s0;  // positions
  uint64_t aux[kBlock];        // the data block decoded last
};
// Shared by the CTA of a project kernel: a piece of consecutive data blocks (their
// payloads are contiguous) and the pieces' block headers.
// (36 KB, so that two CTAs fit an SM: one CTA's tile set-up and copy latency
// overlaps the other's extraction; a wide span takes several pieces)
constexpr int kCtaHdr = 256;
template <int kCtaBuf>
struct ProjectCta {
  static constexpr int kBuf = kCtaBuf;
  uint8_t buf[kCtaBuf];
  // per block of the piece: {halfword offset of its payload in buf, width b, mask of
  // b bits (low word, high word)}; the value extraction reads up to 320 bytes past
  // the end of buf, into hdr
  uint4 hdr[kCtaHdr];
  uint64_t ref[kCtaHdr];  // the blocks' reference values
  static_assert(kCtaBuf % 16 == 0 && sizeof(uint4) * kCtaHdr >= 320, "extraction over-read must stay in hdr");
  uint64_t lo[kWarps], hi[kWarps];
  uint32_t ok[kWarps], nv[kWarps];
  uint64_t off_lo;
  uint64_t mbar;   // completion barrier of the piece's bulk copy
  uint32_t phase;  // its current phase parity
  uint32_t dead;   // a wait on the barrier gave up: no further copies into buf
};
struct SmemEmit {
  uint32_t bits[kEmitSpan * 16];
  uint64_t coff[kEmitSpan + 2];
  uint64_t aux[kBlock];  // the block's positions; then, once they are in registers, its encoding
  uint32_t bits2[kEmitSpan * 16];  // the next block's first span (pipelined emit)
  uint64_t coff2[kEmitSpan + 2];
};

#ifndef MS_EMIT_MIN_BLOCKS
#define MS_EMIT_MIN_BLOCKS 3  // resident CTAs per SM the emit kernel is compiled for
#endif
#ifndef MS_PROJECT_MIN_BLOCKS
#define MS_PROJECT_MIN_BLOCKS 2  // resident CTAs per SM the project kernel is compiled for
#endif
#ifndef MS_PROJECT_CTA_BUF
#define MS_PROJECT_CTA_BUF (36 * 1024)  // staged data blocks per CTA (DYN / FOR / static data)
#endif
#ifndef MS_PROJECT_SPAN_DENSITY
#define MS_PROJECT_SPAN_DENSITY 16  // a tile is staged when it has this many positions per spanned block
#endif
#ifndef MS_PROJECT_BULK
#define MS_PROJECT_BULK 1  // project copies its data pieces with the bulk-copy engine
#endif
#ifndef MS_PROJECT_DELTA_CTA_BUF
#define MS_PROJECT_DELTA_CTA_BUF (96 * 1024)  // staged data blocks per CTA (DELTA data)
#endif

template <int OP>
struct ProducePlan {
  using Smem = typename std::conditional<
      OP == OP_CALC, SmemPair,
      typename std::conditional<
          OP == OP_PROJECT, SmemProjectRandom,
          typename std::conditional<
              OP == OP_PROJECT_WARP, SmemProjectDelta,
              typename std::conditional<OP == OP_EMIT, SmemEmit, SmemSingle>::type>::type>::type>::type;
  static constexpr int kMinBlocks =
      OP == OP_PROJECT ? MS_PROJECT_MIN_BLOCKS : (OP == OP_CALC ? 1 : (OP == OP_EMIT ? MS_EMIT_MIN_BLOCKS : 2));
  // CTA-shared shared memory behind the per-warp plans (the CTA span copy of project)
  using Cta = ProjectCta<MS_PROJECT_CTA_BUF>;
  static constexpr size_t kCtaBytes = OP == OP_PROJECT ? sizeof(Cta) : 0;
};

// Output length of the operator (device-side, may depend on previous kernels).
template <int OP>
MS_DEV uint64_t produce_n(const ProduceArgs& a) {
  if (OP == OP_COMPRESS) return a.raw_n;
  if (OP == OP_DECOMPRESS) return min(a.in0->n, a.raw_cap);
  if (OP == OP_PROJECT || OP == OP_PROJECT_WARP) return a.in1->n;
  if (OP == OP_CALC) return a.in1 ? min(a.in0->n, a.in1->n) : a.in0->n;
  return *reinterpret_cast<volatile uint64_t*>(&a.ctl->op_n);  // OP_EMIT
}

MS_DEV uint64_t arith(int op, uint64_t x, uint64_t y) {
  return op == MS_ADD ? x + y : op == MS_SUB ? x - y : x * y;
}

// project core for non-DELTA data read in place (defined with the other project
// cores below); the CTA span gather falls back to it.
MS_DEV void project_direct(const ProduceArgs& a, const ColView& d, const uint64_t p[16], int valid, int lane,
                           uint64_t v[16], uint64_t* stage);

// Pipelined emit (the staged producer): while a warp expands output block g, the
// bitmap words and offsets of its next block are already on their way, and the
// next block's first input chunk (bstart) was read one block earlier still, so the
// per-block chain of dependent loads is off the critical path.
struct EmitPlan {
  uint64_t lo, cfirst, clast;
  int valid;
};


// bs0 = bstart[g], bs1 = bstart[g + 1] (or anything when g is the last block).
MS_DEV EmitPlan emit_plan(const ProduceArgs& a, uint64_t n_out, uint64_t g, uint64_t bs0, uint64_t bs1) {
  EmitPlan e;
  e.lo = g * kBlock;
  e.valid = (int)min((uint64_t)kBlock, n_out - e.lo);
  const uint64_t hi = e.lo + e.valid;
  const uint64_t nch_in =
      max((uint64_t)1, min(a.emit_nch, *reinterpret_cast<volatile const uint64_t*>(&a.ctl->op_nch)));
  e.cfirst = min(bs0, nch_in - 1);
  e.clast = max(e.cfirst, min((hi < n_out) ? bs1 : nch_in - 1, nch_in - 1));
  return e;
}

// Issues the copies of the bitmap words and offsets of chunks c0 .. c0 + nc - 1 (and
// the offset behind them) into bits / coff (one commit group).
MS_DEV void emit_stage(const ProduceArgs& a, uint64_t c0, int nc, uint32_t* bits, uint64_t* coff, int lane) {
  for (int u = lane; u < nc * 4; u += 32)
    cp_async16(bits + 4 * u, reinterpret_cast<const uint4*>(a.bitmap + c0 * 32) + u);
  for (int u = lane; u <= nc; u += 32) cp_async8(coff + u, a.coff + c0 + u);
  cp_async_commit();
}

// Positions of output block e (lane-blocked in v) from its staged first span in
// bits / coff; later spans (blocks spread over more than kEmitSpan chunks) are
// staged and waited for here.  The caller waited for the first span.
MS_DEV int emit_expand(const ProduceArgs& a, const EmitPlan& e, int lane, uint64_t v[16], SmemEmit* sm,
                       uint32_t* bits, uint64_t* coff) {
  const uint64_t lo = e.lo, hi = e.lo + e.valid;
  const bool dense = e.clast - e.cfirst < 64;
  for (uint64_t c0 = e.cfirst; c0 <= e.clast; c0 += kEmitSpan) {
    const int nc = (int)min((uint64_t)kEmitSpan, e.clast - c0 + 1);
    if (c0 != e.cfirst) {
      emit_stage(a, c0, nc, bits, coff, lane);
      cp_async_wait<0>();
      __syncwarp();
    }
    if (dense) {  // each lane expands its 16 rows of the chunk
      for (int ci = 0; ci < nc; ci++) {
        uint32_t hw = (bits[ci * 16 + (lane >> 1)] >> (16 * (lane & 1))) & 0xffffu;
        uint64_t o = coff[ci] + warp_excl_scan32(__popc(hw), lane);
        const uint64_t ch = c0 + ci;
        while (hw) {
          const int bb = __ffs(hw) - 1;
          hw &= hw - 1;
          if (o >= lo && o < hi) sm->aux[swz((int)(o - lo))] = ch * kBlock + 16 * lane + bb;
          o++;
        }
      }
    } else if (lane < nc) {  // sparse: a lane per chunk
      uint64_t o = coff[lane];
      const uint64_t end = coff[lane + 1];
      const uint64_t ch = c0 + lane;
      if (end > o && end > lo && o < hi) {
        for (int w = 0; w < 16 && o < hi; w++) {
          uint32_t bb32 = bits[lane * 16 + w];
          while (bb32) {
            const int bb = __ffs(bb32) - 1;
            bb32 &= bb32 - 1;
            if (o >= lo && o < hi) sm->aux[swz((int)(o - lo))] = ch * kBlock + 32 * w + bb;
            o++;
          }
        }
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int k = 0; k < 16; k++) {
    const int t = 16 * lane + k;
    v[k] = t < e.valid ? sm->aux[swz(t)] : 0;
  }
  __syncwarp();
  return e.valid;
}

// Sorted positions of a whole CTA tile (8 consecutive output chunks) into DYN /
// FOR / static-BP data.  The data blocks the tile's positions span have contiguous
// payloads, so the CTA copies them into shared memory in pieces of up to kCtaBuf
// bytes (one bulk copy per piece, issued by one thread), and each warp then cuts
// its values out of their blocks there.  A read per position in place would touch
// two or three scattered 64-byte rows of a block per value.  Unsorted or
// out-of-range positions, and tiles with fewer than MS_PROJECT_SPAN_DENSITY
// positions per spanned block, are read in place (project_direct).  Every thread of
// the CTA calls this once per tile (it synchronises the CTA).
template <class Cta>
MS_DEV void gather_cta(const ProduceArgs& a, const ColView& d, const uint64_t p[16], int valid, int warp, int lane,
                       uint64_t v[16], Cta* cs) {
  constexpr int kCtaBuf = Cta::kBuf;
  const int tid = threadIdx.x;
  const int nv = max(0, min(16, valid - 16 * lane));
  bool ok = d.fmt != MS_UNCOMPR;
  uint64_t mn = ~0ull, mx = 0;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    if (k < nv) {
      ok &= p[k] < d.n;
      if (k) ok &= p[k - 1] <= p[k];
      mn = min(mn, p[k]);
      mx = max(mx, p[k]);
    }
  }
  const uint64_t prev_mx = __shfl_up_sync(kFull, mx, 1);
  if (lane > 0 && nv > 0 && prev_mx > mn) ok = false;
  const bool wok = __all_sync(kFull, ok);
  uint64_t wmx = mx;
#pragma unroll
  for (int dd = 16; dd; dd >>= 1) wmx = max(wmx, __shfl_xor_sync(kFull, wmx, dd));
  if (lane == 0) {
    cs->lo[warp] = valid > 0 ? mn : ~0ull;
    cs->hi[warp] = wmx;
    cs->ok[warp] = wok;
    cs->nv[warp] = (uint32_t)max(valid, 0);
  }
  __syncthreads();
  bool tile_ok = true, any = false;
  uint64_t lo = ~0ull, hi = 0, prev_hi = 0, npos = 0;
  for (int w = 0; w < kWarps; w++) {
    tile_ok &= cs->ok[w] != 0;
    if (cs->nv[w]) {
      if (any) tile_ok &= prev_hi <= cs->lo[w];
      lo = min(lo, cs->lo[w]);
      hi = max(hi, cs->hi[w]);
      prev_hi = cs->hi[w];
      npos += cs->nv[w];
      any = true;
    }
  }
  const uint64_t B_lo = lo >> 9, B_hi = hi >> 9;
  // sparser tiles read their values in place: staging whole blocks for a few
  // positions each costs more than the scattered sector reads
  tile_ok &= any && (B_hi - B_lo + 1) * (uint64_t)MS_PROJECT_SPAN_DENSITY <= npos;
  __syncthreads();  // every thread has read the summaries
  if (!tile_ok) {  // gather in place, striped (the warp's 4 KB of the CTA buffer as its stage)
    project_direct(a, d, p, valid, lane, v, reinterpret_cast<uint64_t*>(cs->buf + 4096 * warp));
    __syncthreads();
    return;
  }
#pragma unroll
  for (int k = 0; k < 16; k++) v[k] = 0;
  const bool blockfmt = d.fmt != MS_STATIC_BP;
  const uint64_t nfull = blockfmt ? d.nb : d.n / kBlock;  // blocks with a packed payload
  const uint64_t pay0 = blockfmt ? 16 * d.nb : 0;
  const uint64_t last = min(B_hi, nfull - 1);
  // Positions relative to the tile's first block fit 32 bits (the tile spans at most
  // npos <= 4096 blocks), so the per-value work below is 32-bit.  Slots past the
  // warp's valid count get ~0, whose block lies in no piece.
  const uint64_t base = B_lo << 9;
  uint32_t rel[16];
#pragma unroll
  for (int k = 0; k < 16; k++) rel[k] = k < nv ? (uint32_t)(p[k] - base) : ~0u;
  for (uint64_t lo_blk = B_lo; nfull > 0 && lo_blk <= last;) {
    // thread t: block lo_blk + t
    const uint64_t hb = lo_blk + tid;
    const bool here = tid < kCtaHdr && hb <= last;
    uint64_t off = 0, ref = 0;
    uint32_t b = 0;
    if (here) {
      if (blockfmt) {
        const bool inh = 16 * (hb + 1) <= d.size;
        const uint64_t w0 = inh ? ldg64(d.p + 16 * hb) : 0;
        ref = inh ? ldg64(d.p + 16 * hb + 8) : 0;
        off = w0 >> 8;
        b = (uint32_t)(w0 & 255);
        // every payload starts on an 8-word boundary (its predecessors are 8b words
        // each); another offset is a corrupt chain and would misalign the copy
        if (!inh || b > 64 || (off & 7) || pay0 + 8 * (off + 8ull * b) > d.size) {
          set_error(a.ctl, MS_ERR_FORMAT, hb);
          b = 0;
          off = 0;
        }
      } else {
        b = (uint32_t)d.bw;
        off = 8ull * b * hb;
      }
    }
    if (tid == 0) cs->off_lo = off;
#if MS_PROJECT_BULK
    // Every thread's earlier generic-proxy accesses to buf (reads of the previous
    // piece, a fallback tile's staging stores) are ordered before the async-proxy
    // write of the bulk copy below: a proxy fence by each thread, then the barrier.
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
#endif
    __syncthreads();
    const uint64_t off_lo = cs->off_lo;
    const uint64_t end = off + 8ull * b;
    // blocks whose payload ends within one buffer (ends are monotone); a corrupt
    // header makes an empty block and never stalls the loop
    const bool fits = here && off >= off_lo && 8 * (end - off_lo) <= (uint64_t)kCtaBuf;
    if (fits) {
      cs->hdr[tid] = make_uint4((uint32_t)(4 * (off - off_lo)), b, b >= 32 ? ~0u : (1u << b) - 1u,
                                b <= 32 ? 0u : (b >= 64 ? ~0u : (1u << (b - 32)) - 1u));
      cs->ref[tid] = ref;
    }
    const int cnt = max(1, __syncthreads_count(fits));
    const uint4 hl = cs->hdr[cnt - 1];
    // (a stale entry from a corrupt chain only shortens or clamps the copy, which
    // never runs past the column's buffer)
    const uint64_t at = pay0 + 8 * off_lo;
    const uint64_t room = d.size > at ? d.size - at : 0;
    uint32_t bytes = (uint32_t)min(min((uint64_t)(2ull * hl.x + 64ull * hl.y), (uint64_t)kCtaBuf), room) & ~15u;
#if MS_PROJECT_BULK
    // One thread hands the piece to the bulk-copy engine and the CTA waits on the
    // barrier.  Payloads start on 64-byte boundaries of a 256-byte aligned column;
    // a column that breaks this (it can only be corrupt) copies nothing.
    if (reinterpret_cast<uintptr_t>(d.p + at) & 15) {
      if (tid == 0) set_error(a.ctl, MS_ERR_FORMAT, lo_blk);
      bytes = 0;
    }
    // After a wait that gave up, the CTA issues no further copy and decodes nothing
    // from buf (a copy may still be landing there); the barrier phase stays as it was.
    if (cs->dead) bytes = 0;
    const uint32_t par = cs->phase;
    if (bytes) {
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_expect_tx(&cs->mbar, bytes);
        bulk_copy_g2s(cs->buf, d.p + at, bytes, &cs->mbar);
      }
      if (!mbar_wait(&cs->mbar, par)) {
        cs->dead = 1;
        if (tid == 0) set_error(a.ctl, MS_ERR_TIMEOUT, lo_blk);
      }
    }
    __syncthreads();
    if (cs->dead) bytes = 0;
    if (tid == 0 && bytes) cs->phase = par ^ 1;
#else
    const uint4* src = reinterpret_cast<const uint4*>(d.p + at);
    for (uint32_t u = tid; u < (bytes >> 4); u += blockDim.x) cp_async16(reinterpret_cast<uint4*>(cs->buf) + u, src + u);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
#endif
    const uint32_t lo_r = (uint32_t)(lo_blk - B_lo);  // the piece's first block, tile-relative
    {
      // Value r of a block is bits [kk*b, kk*b + b) of lane stream j = r/16 (kk = r%16),
      // and stream halfword i of lane j is payload halfword 32i + j.  Five halfwords
      // cover a value of up to 64 bits at any of the 16 bit phases; the bits past the
      // value are masked off.  The last of them may lie up to 320 bytes past the
      // piece's end, which is still inside the shared buffer: `hdr` follows `buf`.
      const uint16_t* s16 = reinterpret_cast<const uint16_t*>(cs->buf);
      const bool add_ref = d.fmt == MS_FOR_BP;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        const uint32_t q = (rel[k] >> 9) - lo_r;
        if (q < (uint32_t)cnt) {
          const uint4 h = cs->hdr[q];
          if (2 * h.x + 64 * h.y > bytes) {  // never read past the copy
            set_error(a.ctl, MS_ERR_FORMAT, B_lo + lo_r + q);
          } else {
            const uint32_t r = rel[k] & 511, bit = (r & 15) * h.y;
            const uint32_t h0 = h.x + 32 * (bit >> 4) + (r >> 4);
            const uint32_t w0 = (uint32_t)s16[h0] | (uint32_t)s16[h0 + 32] << 16;
            const uint32_t w1 = (uint32_t)s16[h0 + 64] | (uint32_t)s16[h0 + 96] << 16;
            const uint32_t w2 = s16[h0 + 128];
            const uint32_t xl = __funnelshift_r(w0, w1, bit & 15) & h.z;
            const uint32_t xh = __funnelshift_r(w1, w2, bit & 15) & h.w;
            v[k] = ((uint64_t)xh << 32 | xl) + (add_ref ? cs->ref[q] : 0ull);
          }
        }
      }
    }
    __syncthreads();  // the next piece overwrites the buffer
    lo_blk += (uint64_t)cnt;
  }
  // positions in the uncompressed remainder (block formats) or the horizontal tail (static BP)
  const uint32_t nfull_r = nfull > B_lo ? (uint32_t)min(nfull - B_lo, (uint64_t)1 << 23) : 0u;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    if (k < nv && (rel[k] >> 9) >= nfull_r) {
      const uint64_t pk = base + rel[k];
      if (blockfmt) {
        const uint64_t at = pay0 + 8 * d.pwords + 8 * (pk - kBlock * d.nb);
        v[k] = at + 8 <= d.size ? ldg64(d.p + at) : 0;
      } else {
        const uint64_t* tail = reinterpret_cast<const uint64_t*>(d.p + 64ull * d.bw * nfull);
        const uint64_t bit = (pk - kBlock * nfull) * (uint64_t)d.bw;
        const int sh = (int)(bit & 63);
        uint64_t x = ldg64(tail + (bit >> 6)) >> sh;
        if (sh + d.bw > 64) x |= ldg64(tail + (bit >> 6) + 1) << (64 - sh);
        v[k] = x & lowmask(d.bw);
      }
    }
  }
  __syncthreads();
}

// Residual transform of a full block (Sec. 2.1): FOR subtracts the block minimum,
// DELTA takes differences to the predecessor (first residual 0, reference = first
// value).  Returns the block's bit width; v becomes the residuals.
MS_DEV int encode_block(int fmt, uint64_t v[16], int lane, uint64_t* ref_out) {
  uint64_t ref = 0;
  if (fmt == MS_FOR_BP) {
    uint64_t mn = v[0];
#pragma unroll
    for (int k = 1; k < 16; k++) mn = min(mn, v[k]);
    ref = warp_min(mn);
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] -= ref;
  } else if (fmt == MS_DELTA_BP) {
    const uint64_t prev = __shfl_up_sync(kFull, v[15], 1);
    ref = __shfl_sync(kFull, v[0], 0);
#pragma unroll
    for (int k = 15; k > 0; k--) v[k] -= v[k - 1];
    v[0] = lane ? v[0] - prev : 0;
  }
  uint64_t o = 0;
#pragma unroll
  for (int k = 0; k < 16; k++) o |= v[k];
  *ref_out = ref;
  return bw64(warp_or(o));
}

// ------------------------------------------------ project cores (direct producer)

// Values of a non-DELTA column at the warp's positions, read in place (Sec. 4.2
// random access; the block header doubles as a directory for DYN / FOR).  `stage`
// holds the warp's 512 positions (swizzled, index o = position o of the chunk) and
// receives the values in their place; bit i of `ok` says that position lane + 32i
// is valid and inside the column.  Lane t takes positions t, t + 32, ... (striped),
// so with sorted positions the 32 lanes of one load read neighbouring values of
// one block: the loads coalesce when positions are dense, and only the touched
// sectors are read when they are sparse.  kGatherGroup positions at a time: their
// header loads, then all their payload halfword loads, are in flight together.
#ifndef MS_GATHER_GROUP
#define MS_GATHER_GROUP 4
#endif
constexpr int kGatherGroup = MS_GATHER_GROUP;
MS_DEV void gather_values(const ColView& d, uint64_t* stage, uint32_t ok, int lane) {
  if (d.fmt == MS_RLE) {  // the run of each position: directory, then a short search
#pragma unroll
    for (int i = 0; i < 16; i++) {
      const uint64_t q = stage[swz(lane + 32 * i)];
      stage[swz(lane + 32 * i)] = ((ok >> i) & 1u) ? rle_read_at(d, q) : 0;
    }
    return;
  }
  if (d.fmt == MS_UNCOMPR) {
#pragma unroll
    for (int half = 0; half < 2; half++) {
      uint64_t x[8];
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const int i = 8 * half + u;
        const uint64_t q = stage[swz(lane + 32 * i)];
        x[u] = ((ok >> i) & 1u) ? ldg64(d.p + 8 * q) : 0;
      }
#pragma unroll
      for (int u = 0; u < 8; u++) stage[swz(lane + 32 * (8 * half + u))] = x[u];
    }
    return;
  }
  const bool stat = d.fmt == MS_STATIC_BP;
  const uint64_t nb = stat ? d.n / kBlock : d.nb;
  const uint64_t pay0 = stat ? 0 : 16 * nb;
  const uint64_t rem0 = stat ? 64ull * (uint64_t)d.bw * nb : 16 * nb + 8 * d.pwords;
  if (stat && d.bw <= 33) {
    // static BP up to 33 bits: no header, and three halfwords cover a value at any
    // bit phase, so eight positions' loads are in flight at once
    const int b = d.bw;
#pragma unroll
    for (int half = 0; half < 2; half++) {
      uint32_t h[8][3];
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const int i = 8 * half + u;
        const uint64_t q = stage[swz(lane + 32 * i)];
        const uint64_t g = q >> 9;
        const int r = (int)(q & 511), bit0 = (r & 15) * b;
        const bool in = ((ok >> i) & 1u) && g < nb && 64ull * b * (g + 1) <= d.size;
        const int nq = in ? (((bit0 & 15) + b + 15) >> 4) : 0;
        const uint16_t* hw = reinterpret_cast<const uint16_t*>(d.p + (in ? 64ull * b * g : 0)) + 32 * (bit0 >> 4) +
                             (r >> 4);
#pragma unroll
        for (int t = 0; t < 3; t++) h[u][t] = t < nq ? (uint32_t)__ldg(hw + 32 * t) : 0u;
      }
#pragma unroll
      for (int u = 0; u < 8; u++) {
        const int i = 8 * half + u;
        const uint64_t q = stage[swz(lane + 32 * i)];  // re-read: fewer live registers
        const int r = (int)(q & 511);
        const int sh = ((r & 15) * b) & 15;
        const uint64_t w = (uint64_t)h[u][0] | ((uint64_t)h[u][1] << 16) | ((uint64_t)h[u][2] << 32);
        uint64_t v = (w >> sh) & lowmask(b);
        if ((q >> 9) >= nb) {  // the horizontal tail
          const uint64_t bit = (uint64_t)r * (uint64_t)b;
          const int s2 = (int)(bit & 63);
          const uint64_t at = rem0 + 8 * (bit >> 6);
          uint64_t y = at + 8 <= d.size ? ldg64(d.p + at) >> s2 : 0;
          if (s2 + b > 64 && at + 16 <= d.size) y |= ldg64(d.p + at + 8) << (64 - s2);
          v = y & lowmask(b);
        }
        stage[swz(lane + 32 * i)] = ((ok >> i) & 1u) ? v : 0;
      }
    }
    return;
  }
#pragma unroll
  for (int half = 0; half < 16 / kGatherGroup; half++) {
    uint64_t q[kGatherGroup], w0[kGatherGroup], ref[kGatherGroup];
#pragma unroll
    for (int u = 0; u < kGatherGroup; u++) {  // headers (or the fixed static width)
      const int i = kGatherGroup * half + u;
      q[u] = stage[swz(lane + 32 * i)];
      const uint64_t g = q[u] >> 9;
      const bool in = ((ok >> i) & 1u) && g < nb;
      if (stat) {
        w0[u] = ((8ull * (uint64_t)d.bw * g) << 8) | (uint64_t)d.bw;
        ref[u] = 0;
      } else if (in && 16 * (g + 1) <= d.size) {
        const ulonglong2 h = __ldg(reinterpret_cast<const ulonglong2*>(d.p) + g);
        w0[u] = h.x;
        ref[u] = h.y;
      } else {
        w0[u] = 0;
        ref[u] = 0;
      }
    }
    uint32_t h[kGatherGroup][5];
#pragma unroll
    for (int u = 0; u < kGatherGroup; u++) {  // payload halfwords: up to five cover a value at any bit phase
      const int i = kGatherGroup * half + u;
      const uint64_t g = q[u] >> 9;
      const int r = (int)(q[u] & 511);
      const int b = (int)min((uint64_t)64, w0[u] & 255);
      const uint64_t pay = pay0 + 8 * (w0[u] >> 8);
      const bool in = ((ok >> i) & 1u) && g < nb && b > 0 && pay + 64ull * b <= d.size;
      const int bit0 = (r & 15) * b;
      const int nq = in ? (((bit0 & 15) + b + 15) >> 4) : 0;
      const uint16_t* hw = reinterpret_cast<const uint16_t*>(d.p + (in ? pay : 0)) + 32 * (bit0 >> 4) + (r >> 4);
#pragma unroll
      for (int t = 0; t < 5; t++) h[u][t] = t < nq ? (uint32_t)__ldg(hw + 32 * t) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kGatherGroup; u++) {
      const int i = kGatherGroup * half + u;
      const uint64_t g = q[u] >> 9;
      const int r = (int)(q[u] & 511);
      const int b = (int)min((uint64_t)64, w0[u] & 255);
      const int sh = ((r & 15) * b) & 15;
      const uint64_t lo = (uint64_t)h[u][0] | ((uint64_t)h[u][1] << 16) | ((uint64_t)h[u][2] << 32) |
                          ((uint64_t)h[u][3] << 48);
      uint64_t v = ((lo >> sh) | (sh ? ((uint64_t)h[u][4] << (64 - sh)) : 0)) & lowmask(b);
      v += ref[u];
      if (g >= nb) {  // the raw remainder, or static BP's horizontal tail
        if (stat) {
          const uint64_t bit = (uint64_t)r * (uint64_t)d.bw;
          const int s2 = (int)(bit & 63);
          const uint64_t at = rem0 + 8 * (bit >> 6);
          uint64_t y = at + 8 <= d.size ? ldg64(d.p + at) >> s2 : 0;
          if (s2 + d.bw > 64 && at + 16 <= d.size) y |= ldg64(d.p + at + 8) << (64 - s2);
          v = y & lowmask(d.bw);
        } else {
          const uint64_t at = rem0 + 8 * (uint64_t)r;
          v = at + 8 <= d.size ? ldg64(d.p + at) : 0;
        }
      }
      stage[swz(lane + 32 * i)] = ((ok >> i) & 1u) ? v : 0;
    }
  }
}

// project core, non-DELTA data: the warp's positions (lane-blocked, p[k] is output
// value 16*lane + k) go to the warp's 4 KB stage, are gathered striped in place by
// gather_values, and come back lane-blocked in v.  Positions >= n(data) raise
// MS_ERR_OUT_OF_RANGE and give 0.
MS_DEV void project_direct(const ProduceArgs& a, const ColView& d, const uint64_t p[16], int valid, int lane,
                           uint64_t v[16], uint64_t* stage) {
#pragma unroll
  for (int k = 0; k < 16; k++) stage[swz(16 * lane + k)] = p[k];
  __syncwarp();
  uint32_t ok = 0;
#pragma unroll
  for (int i = 0; i < 16; i++) {
    const int o = lane + 32 * i;
    const uint64_t q = stage[swz(o)];
    const bool in = o < valid;
    if (in && q >= d.n) set_error(a.ctl, MS_ERR_OUT_OF_RANGE, q);
    ok |= (uint32_t)(in && q < d.n) << i;
  }
  gather_values(d, stage, ok, lane);
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 16; k++) v[k] = stage[swz(16 * lane + k)];
  __syncwarp();
}

// Decodes block B (< nb) of a DELTA column straight from global memory (each lane
// reads its own stream; a warp load covers 64 contiguous bytes) into lane
// registers: residuals, then the in-lane prefix sums and one warp scan.
MS_DEV void decode_delta_block(const ColView& d, uint64_t B, uint64_t w0, uint64_t ref, int lane, uint64_t t[16],
                               DevCtl* ctl) {
  int b = (int)(w0 & 255);
  const uint64_t pay = 16 * d.nb + 8 * (w0 >> 8);
  if (b > 64 || pay + 64ull * b > d.size) {
    if (lane == 0) set_error(ctl, MS_ERR_FORMAT, B);
    b = 0;
  }
  read_lane_stream(reinterpret_cast<const uint16_t*>(d.p + (b ? pay : 0)), lane, b, t);
  if (b <= 23) {  // 512 residuals below 2^23 sum below 2^32
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      sum += (uint32_t)t[k];
      t[k] = sum;
    }
    const uint64_t excl = (uint64_t)warp_excl_scan32(sum, lane) + ref;
#pragma unroll
    for (int k = 0; k < 16; k++) t[k] += excl;
  } else {
    uint64_t sum = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      sum += t[k];
      t[k] = sum;
    }
    const uint64_t excl = warp_excl_scan(sum, lane) + ref;
#pragma unroll
    for (int k = 0; k < 16; k++) t[k] += excl;
  }
}

// project core, DELTA data, sorted positions (the usual case: the positions come
// from a select or a semi-join).  The warp's positions span blocks Bf..Bl; taken
// relative to block Bf they fit 32 bits, and every touched block is visited once,
// in order: a block of width 0 answers its positions with its reference, any other
// is decoded straight from global memory into `aux` as prefix sums relative to its
// reference (32-bit when the block is at most 23 bits wide: 511 residuals below
// 2^23 sum below 2^32), and its positions are read from there.  Returns false, with
// v untouched, when the positions are unsorted, out of range or span 2^31 rows or
// more (project_delta handles those).  The values collect in `ob` (lane-private
// slots 32k + lane, conflict-free) and come back to v at the end, so they do not hold
// registers during the walk.
MS_DEV bool project_delta_sorted(const ProduceArgs& a, const ColView& d, const uint64_t p[16], int valid, int lane,
                                 uint64_t v[16], uint64_t* aux, uint64_t* ob) {
  const int nv = max(0, min(16, valid - 16 * lane));
  bool ok = valid > 0;
  uint64_t mx = 0;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    if (k < nv) {
      ok &= p[k] < d.n;
      if (k) ok &= p[k - 1] <= p[k];
      mx = p[k];
    }
  }
  const uint64_t prev_mx = __shfl_up_sync(kFull, mx, 1);
  if (lane > 0 && nv > 0 && prev_mx > p[0]) ok = false;
  if (!__all_sync(kFull, ok)) return false;
  const uint64_t first = __shfl_sync(kFull, p[0], 0);
  const uint64_t last = __shfl_sync(kFull, mx, (valid - 1) >> 4);
  if (last - first >= (1ull << 31)) return false;
  const uint64_t Bf = first >> 9, base = Bf << 9;
  uint32_t rel[16];
#pragma unroll
  for (int k = 0; k < 16; k++) rel[k] = (uint32_t)(p[k] - base);
  uint32_t pend = nv >= 16 ? 0xffffu : (1u << nv) - 1u;
  if ((last >> 9) - Bf >= 32) {
    // sparse positions (16 or fewer per spanned block): those in blocks of width 0
    // are answered from their headers first (one load per position, mostly L1
    // hits), so that the block walk below visits only blocks that need decoding
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const uint64_t B = Bf + (rel[k] >> 9);
      if (((pend >> k) & 1u) && B < d.nb && 16 * (B + 1) <= d.size) {
        const ulonglong2 h = __ldg(reinterpret_cast<const ulonglong2*>(d.p) + B);
        if ((h.x & 255) == 0) {
          ob[32 * k + lane] = h.y;
          pend &= ~(1u << k);
        }
      }
    }
  }
  uint32_t* aux32 = reinterpret_cast<uint32_t*>(aux);
  while (__any_sync(kFull, pend != 0)) {
    // the next touched block: the smallest block among the lanes' pending positions
    uint32_t m = 0xffffffffu;
#pragma unroll
    for (int k = 0; k < 16; k++) m = min(m, ((pend >> k) & 1u) ? rel[k] : 0xffffffffu);
    const uint32_t blk = __reduce_min_sync(kFull, m >> 9);
    uint32_t hit = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) hit |= (uint32_t)(((pend >> k) & 1u) && (rel[k] >> 9) == blk) << k;
    const uint64_t B = Bf + blk;
    if (B >= d.nb) {  // the raw remainder behind the payload
      const uint64_t at = 16 * d.nb + 8 * d.pwords;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        const uint64_t o = rel[k] & 511;
        if ((hit >> k) & 1u) ob[32 * k + lane] = at + 8 * (o + 1) <= d.size ? ldg64(d.p + at + 8 * o) : 0;
      }
    } else {
      ulonglong2 h = make_ulonglong2(0, 0);
      if (16 * (B + 1) <= d.size) h = __ldg(reinterpret_cast<const ulonglong2*>(d.p) + B);
      else if (lane == 0) set_error(a.ctl, MS_ERR_FORMAT, B);
      int b = (int)(h.x & 255);
      const uint64_t pay = 16 * d.nb + 8 * (h.x >> 8);
      if (b > 64 || pay + 64ull * b > d.size) {
        if (lane == 0) set_error(a.ctl, MS_ERR_FORMAT, B);
        b = 0;
      }
      if (b == 0) {  // 512 copies of the reference
#pragma unroll
        for (int k = 0; k < 16; k++)
          if ((hit >> k) & 1u) ob[32 * k + lane] = h.y;
      } else {
        uint64_t t[16];
        read_lane_stream(reinterpret_cast<const uint16_t*>(d.p + pay), lane, b, t);
        // value i of the block is ref + (residuals 0..i summed); residual 0 is 0.
        // Stored transposed (slot 32k + lane for value 16 lane + k): the stores are
        // conflict-free
        if (b <= 23) {
          uint32_t sum = 0;
#pragma unroll
          for (int k = 0; k < 16; k++) {
            sum += (uint32_t)t[k];
            t[k] = sum;
          }
          const uint32_t ex = warp_excl_scan32(sum, lane);
#pragma unroll
          for (int k = 0; k < 16; k++) aux32[32 * k + lane] = (uint32_t)t[k] + ex;
          __syncwarp();
#pragma unroll
          for (int k = 0; k < 16; k++) {
            const uint32_t o = rel[k] & 511;
            if ((hit >> k) & 1u) ob[32 * k + lane] = h.y + aux32[32 * (o & 15) + (o >> 4)];
          }
        } else {
          uint64_t sum = 0;
#pragma unroll
          for (int k = 0; k < 16; k++) {
            sum += t[k];
            t[k] = sum;
          }
          const uint64_t ex = warp_excl_scan(sum, lane);
#pragma unroll
          for (int k = 0; k < 16; k++) aux[32 * k + lane] = t[k] + ex;
          __syncwarp();
#pragma unroll
          for (int k = 0; k < 16; k++) {
            const uint32_t o = rel[k] & 511;
            if ((hit >> k) & 1u) ob[32 * k + lane] = h.y + aux[32 * (o & 15) + (o >> 4)];
          }
        }
        __syncwarp();  // aux is rewritten by the next block
      }
    }
    pend &= ~hit;
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 16; k++) v[k] = k < nv ? ob[32 * k + lane] : 0;
  __syncwarp();
  return true;
}

// project core, DELTA data: values need their block's prefix sums.  First every
// position's block header is read (sixteen independent loads per lane, nearly all
// hits in L1): a block of width 0 holds 512 copies of its reference, and its
// positions are answered at once.  Then every other distinct block the warp's
// positions touch is decoded once (in ascending order) into `aux`, and the positions
// in it are read from there.  The positions wait in `stage` (lane-private slots).
// Works for unsorted positions.
MS_DEV void project_delta(const ProduceArgs& a, const ColView& d, const uint64_t p[16], int valid, int lane,
                          uint64_t v[16], uint64_t* stage, uint64_t* aux) {
  uint32_t pending = 0;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    v[k] = 0;
    stage[swz(16 * lane + k)] = p[k];
    const bool in = 16 * lane + k < valid;
    if (in && p[k] >= d.n) set_error(a.ctl, MS_ERR_OUT_OF_RANGE, p[k]);
    if (in && p[k] < d.n) {
      const uint64_t B = p[k] >> 9;
      bool flat = false;
      if (B < d.nb && 16 * (B + 1) <= d.size) {
        const ulonglong2 h = __ldg(reinterpret_cast<const ulonglong2*>(d.p) + B);
        flat = (h.x & 255) == 0;
        v[k] = h.y;
      }
      pending |= (uint32_t)!flat << k;
    }
  }
  while (__ballot_sync(kFull, pending) != 0) {
    uint64_t mb = ~0ull;
#pragma unroll
    for (int k = 0; k < 16; k++)
      if (pending & (1u << k)) mb = min(mb, stage[swz(16 * lane + k)] >> 9);
    const uint64_t B = warp_min(mb);
    if (B < d.nb) {
      ulonglong2 h = make_ulonglong2(0, 0);
      if (16 * (B + 1) <= d.size) h = __ldg(reinterpret_cast<const ulonglong2*>(d.p) + B);
      else if (lane == 0) set_error(a.ctl, MS_ERR_FORMAT, B);
      uint64_t t[16];
      decode_delta_block(d, B, h.x, h.y, lane, t, a.ctl);
#pragma unroll
      for (int k = 0; k < 16; k++) aux[swz(16 * lane + k)] = t[k];
    } else {  // the raw remainder
      const uint64_t at = 16 * d.nb + 8 * d.pwords;
      const int rem = (int)(d.n - B * kBlock);
#pragma unroll
      for (int k = 0; k < 16; k++) {
        const int o = 16 * lane + k;
        aux[swz(o)] = (o < rem && at + 8 * (uint64_t)(o + 1) <= d.size) ? ldg64(d.p + at + 8 * o) : 0;
      }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const uint64_t q = stage[swz(16 * lane + k)];
      if ((pending & (1u << k)) && (q >> 9) == B) {
        v[k] = aux[swz((int)(q & 511))];
        pending &= ~(1u << k);
      }
    }
    __syncwarp();
  }
}

// Per-warp shared memory and occupancy of the direct-offset producer.
template <int OP>
struct DirectPlan {
  struct Smem {
    StreamSmem<kProdDepth> s0;
  };
  static constexpr int kMinBlocks = 2;
};

// Direct-offset producer of the allocation-free compress path: payload offsets come
// from a decoupled look-back inside the kernel instead of a placement pass.
template <int OP>
__global__ void __launch_bounds__(kThreads, DirectPlan<OP>::kMinBlocks) k_produce(ProduceArgs a) {
  static_assert(OP == OP_COMPRESS, "the direct-offset producer serves the allocation-free compress only");
  using Smem = typename DirectPlan<OP>::Smem;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ uint64_t s_words[2][kWarps];  // by tile parity: payload words of each warp's block
  __shared__ uint64_t s_agg[2];
  __shared__ uint64_t s_excl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Smem* sm = reinterpret_cast<Smem*>(smem_raw) + warp;

  DevCtl* ctl = a.ctl;
  const bool raw = a.out_meta == nullptr;
  const uint64_t top = raw ? 0 : *reinterpret_cast<volatile uint64_t*>(&ctl->top);
  const uint64_t avail = raw ? 8 * a.raw_cap : ctl->cap - top;
  uint8_t* base = raw ? reinterpret_cast<uint8_t*>(a.raw_out) : reinterpret_cast<uint8_t*>(ctl->arena + top);

  const ColView c0 = view_raw(a.raw_in, a.raw_n);
  const uint64_t n_out = a.raw_n;
  const int fmt = a.fmt, bw = a.bw;
  const bool blockfmt = is_block_fmt(fmt);
  const uint64_t nch = (n_out + kBlock - 1) / kBlock, ntiles = (nch + kWarps - 1) / kWarps;
  const uint64_t nb_out = blockfmt ? n_out / kBlock : 0;
  const uint64_t static_chunks = n_out / kBlock;
  const uint64_t G = gridDim.x;
  const uint64_t my_tiles = blockIdx.x < ntiles ? (ntiles - blockIdx.x + G - 1) / G : 0;
  const uint64_t first = (uint64_t)blockIdx.x * kWarps + warp, stride = kWarps * G;

  // input streams: chunk i of a warp is first + i*stride, for every tile of the CTA
  constexpr int D = kProdDepth;
  StreamSmem<D>* ring0 = &sm->s0;
  ChunkStream<D> st0{c0, first, stride, my_tiles, ring0, lane};
  if (my_tiles) {
    for (int i = 0; i < D; i++) st0.issue_header(i);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    for (int j = 0; j < D - 1; j++) {
      st0.prologue_step(j);
      cp_async_commit();
    }
  }

  // A block-format tile is published and stored one iteration late: after encoding
  // tile i the CTA publishes its aggregate (payload words) and moves on; the
  // look-back of tile i and the store of its blocks from the stage slots happen at
  // the top of iteration i + 1, before that iteration's prefetch refills the slot.
  // By then the tile's predecessors have had a whole tile's time to publish, so the
  // look-back rarely waits.  Per warp, the pending block: its stage, width,
  // reference, valid count and chunk.
  bool pend = false;
  uint64_t pend_tile = 0, pend_g = 0, pend_ref = 0;
  int pend_b = 0, pend_valid = 0, par = 0;
  uint16_t* pend_stage = nullptr;
  auto finish = [&]() {  // every thread of the CTA calls it
    if (warp == 0) {
      const uint64_t agg = s_agg[par];
      const uint64_t ex = lookback_resolve(a.status, pend_tile, agg, lane, ctl);
      if (lane == 0) {
        s_excl = ex;
        if (pend_tile == ntiles - 1) ctl->op_words = ex + agg;
      }
    }
    __syncthreads();
    if (pend_valid > 0) {
      uint64_t off = s_excl;
      for (int w = 0; w < warp; w++) off += s_words[par][w];
      if (pend_valid == kBlock) {
        const uint64_t pay = 16 * nb_out + 8 * off;
        if (16 * (pend_g + 1) <= avail && pay + 64ull * pend_b <= avail) {
          if (lane == 0) {
            uint64_t* h = reinterpret_cast<uint64_t*>(base) + 2 * pend_g;
            h[0] = (off << 8) | (uint64_t)pend_b;
            h[1] = pend_ref;
          }
          uint4* dst = reinterpret_cast<uint4*>(base + pay);
          const uint4* src = reinterpret_cast<const uint4*>(pend_stage);
          for (int t = lane; t < 4 * pend_b; t += 32) dst[t] = src[t];
        } else if (lane == 0) {
          set_error(ctl, MS_ERR_NOMEM, pend_g);
        }
      } else {  // remainder: raw values behind the whole payload
        const uint64_t rem = 16 * nb_out + 8 * off;
        if (rem + 8ull * pend_valid <= avail) {
          uint64_t* dst = reinterpret_cast<uint64_t*>(base + rem);
          const uint64_t* src = reinterpret_cast<const uint64_t*>(pend_stage);
          for (int t = lane; t < pend_valid; t += 32) dst[t] = src[t];
        } else if (lane == 0) {
          set_error(ctl, MS_ERR_NOMEM, pend_g);
        }
      }
    }
    __syncwarp();
    pend = false;
  };

  for (uint64_t i = 0; i < my_tiles; i++) {
    const uint64_t tile = blockIdx.x + i * G;
    const uint64_t g = tile * kWarps + warp;
    uint64_t v[16];
    int valid = 0;
    uint16_t* out_stage;
    cp_async_wait<D - 2>();
    __syncwarp();
    if (pend) finish();  // before step(i) refills the pending tile's slot
    st0.step(i);
    cp_async_commit();
    out_stage = ring0->slot[i % D];
    valid = st0.decode(i, v, ctl);
    valid = (int)min((uint64_t)valid, g * kBlock < n_out ? n_out - g * kBlock : 0);
    __syncwarp();
    if (blockfmt) {
      // ---- encode into the warp's stage (the remainder as raw values) and publish
      // the tile's aggregate; the look-back and the store wait for the next iteration
      int b = 0;
      uint64_t ref = 0;
      if (valid == kBlock) {
        b = encode_block(fmt, v, lane, &ref);
        write_lane_stream(out_stage, lane, b, v);
      } else if (valid > 0) {
        uint64_t* st64 = reinterpret_cast<uint64_t*>(out_stage);
#pragma unroll
        for (int k = 0; k < 16; k++)
          if (16 * lane + k < valid) st64[16 * lane + k] = v[k];
      }
      par = (int)(i & 1);
      if (lane == 0) s_words[par][warp] = valid == kBlock ? 8ull * b : 0;
      __syncthreads();
      if (warp == 0) {
        const uint64_t agg = warp_sum(lane < kWarps ? s_words[par][lane] : 0);
        if (lane == 0) s_agg[par] = agg;
        lookback_publish(a.status, tile, agg, lane);
      }
      __syncwarp();
      pend = true;
      pend_tile = tile;
      pend_g = g;
      pend_b = b;
      pend_ref = ref;
      pend_valid = valid;
      pend_stage = out_stage;
      continue;
    }
    // ---- fixed-offset formats: encode and store in place
    if (fmt == MS_STATIC_BP && valid > 0) {
      uint64_t o = 0;
#pragma unroll
      for (int k = 0; k < 16; k++) o |= (16 * lane + k < valid) ? v[k] : 0;
      o = warp_or(o);
      if (bw64(o) > bw && lane == 0) set_error(ctl, MS_ERR_VALUE_TOO_WIDE, g);
      const uint64_t mask = lowmask(bw);
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] &= mask;
      if (g < static_chunks) {
        write_lane_stream(out_stage, lane, bw, v);
        __syncwarp();
        const uint64_t pay = 64ull * bw * g;
        if (pay + 64ull * bw <= avail) {
          uint4* dst = reinterpret_cast<uint4*>(base + pay);
          const uint4* src = reinterpret_cast<const uint4*>(out_stage);
          for (int t = lane; t < 4 * bw; t += 32) dst[t] = src[t];
        } else if (lane == 0) {
          set_error(ctl, MS_ERR_NOMEM, g);
        }
      } else {  // horizontal tail
        uint32_t* w32 = reinterpret_cast<uint32_t*>(out_stage);
        for (int t = lane; t < 1024; t += 32) w32[t] = 0;
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 16; k++) {
          const int t = 16 * lane + k;
          if (t < valid && v[k]) {
            const uint64_t bit = (uint64_t)t * bw;
            const int sh = (int)(bit & 31);
            const uint64_t x = v[k];
            int wi = (int)(bit >> 5);
            atomicOr(w32 + wi, (uint32_t)(x << sh));
            uint64_t rest = (sh == 0) ? (x >> 32) : (x >> (32 - sh));
            int have = 32 - sh;
            while (have < bw && rest) {
              atomicOr(w32 + (++wi), (uint32_t)rest);
              rest >>= 32;
              have += 32;
            }
          }
        }
        __syncwarp();
        const uint64_t pay = 64ull * bw * static_chunks;
        const int nw = (int)(((uint64_t)valid * bw + 63) / 64);
        if (pay + 8ull * nw <= avail) {
          uint64_t* dst = reinterpret_cast<uint64_t*>(base + pay);
          const uint64_t* src = reinterpret_cast<const uint64_t*>(out_stage);
          for (int t = lane; t < nw; t += 32) dst[t] = src[t];
        } else if (lane == 0) {
          set_error(ctl, MS_ERR_NOMEM, g);
        }
      }
    } else if (fmt == MS_UNCOMPR && valid > 0) {  // arena column or caller buffer
      const uint64_t pay = 8ull * kBlock * g;
      if (pay + 8ull * valid <= avail) {
        uint64_t* dst = reinterpret_cast<uint64_t*>(base + pay);
        if (valid == kBlock) {
          uint4* stg = reinterpret_cast<uint4*>(out_stage);
#pragma unroll
          for (int cc = 0; cc < 8; cc++)
            stg[lane * 8 + (cc ^ (lane & 7))] = make_uint4((uint32_t)v[2 * cc], (uint32_t)(v[2 * cc] >> 32),
                                                          (uint32_t)v[2 * cc + 1], (uint32_t)(v[2 * cc + 1] >> 32));
          __syncwarp();
#pragma unroll
          for (int it = 0; it < 8; it++) {
            const int ci = lane + 32 * it, L = ci >> 3, cc = ci & 7;
            reinterpret_cast<uint4*>(dst)[ci] = stg[L * 8 + (cc ^ (L & 7))];
          }
        } else {
#pragma unroll
          for (int k = 0; k < 16; k++)
            if (16 * lane + k < valid) dst[16 * lane + k] = v[k];
        }
      } else if (lane == 0) {
        set_error(ctl, MS_ERR_NOMEM, g);
      }
    }
    __syncwarp();
  }
  if (pend) finish();
  cp_async_wait<0>();

  // ---- epilogue: the last CTA to finish describes the output column and moves
  // the arena's top past it.
  if (raw) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&ctl->done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      uint64_t size, pwords = 0;
      if (fmt == MS_UNCOMPR) {
        size = 8 * n_out;
      } else if (fmt == MS_STATIC_BP) {
        size = 8 * ((n_out * (uint64_t)bw + 63) / 64);
      } else {
        pwords = nb_out ? *reinterpret_cast<volatile uint64_t*>(&ctl->op_words) : 0;
        size = 16 * nb_out + 8 * pwords + 8 * (n_out % kBlock);
      }
      DevMeta* m = a.out_meta;
      m->n = n_out;
      m->ptr = reinterpret_cast<uint64_t>(base);
      m->size = size;
      m->nb = nb_out;
      m->pwords = pwords;
      m->fmt = (uint32_t)fmt;
      m->bw = (uint32_t)(fmt == MS_STATIC_BP ? bw : 0);
      const uint64_t grow = (size + 255) / 256 * 256;
      if (size > avail) {
        // the column did not fit: publish it empty so no reader leaves the buffer
        set_error(ctl, MS_ERR_NOMEM, size);
        m->n = 0;
        m->size = 0;
        m->nb = 0;
        m->pwords = 0;
      } else {
        ctl->top = top + grow;
        if (top + grow > ctl->high) ctl->high = top + grow;
      }
      ctl->done = 0;
      __threadfence();
    }
  }
}

// The output stage of a block-format producer.  Encoded blocks wait there until
// the placement pass knows their final offsets.  It is taken from the free end of
// the arena, growing down from (cap & ~255) towards the columns at the arena top, so
// it holds the output's actual payload bytes (plus each warp's unused tail), not a
// worst-case slot per block.  A warp takes a piece of up to kStagePiece bytes with
// one atomic and fills it with its consecutive blocks.
constexpr uint64_t kStagePiece = 16384;

struct StageCursor {
  uint64_t at;    // arena offset of the warp's next free stage byte
  uint64_t left;  // free bytes left in the warp's piece
};

MS_DEV uint64_t stage_end(const DevCtl* ctl) { return ctl->cap & ~255ull; }

// Reserves `need` bytes (a multiple of 64) of the stage for the calling warp (every
// lane calls it with the same arguments); `remaining` is the number of output chunks
// the warp has left, the current one included.  Returns the arena offset, or
// ~0 when the stage would reach the columns below it (MS_ERR_NOMEM is raised).
MS_DEV uint64_t stage_take(DevCtl* ctl, uint64_t top, uint64_t need, uint64_t remaining, StageCursor& sc,
                           uint64_t g, int lane) {
  if (sc.left < need) {
    const uint64_t piece = remaining * (uint64_t)2048;
    const uint64_t want = max(need, piece < kStagePiece ? piece : kStagePiece);
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->stage), (unsigned long long)want);
    old = __shfl_sync(kFull, old, 0);
    const uint64_t end = stage_end(ctl);
    if (old + want > end - top) {
      if (lane == 0) set_error(ctl, MS_ERR_NOMEM, g);
      sc.left = 0;
      return ~0ull;
    }
    sc.at = end - (old + want);
    sc.left = want;
  }
  const uint64_t at = sc.at;
  sc.at += need;
  sc.left -= need;
  return at;
}

// Stores output chunk g (lane-blocked values v, `valid` of them) of a staged
// producer: a block-format block is encoded into the warp's stage slot in shared
// memory and copied into the arena's stage with its {stage offset, width,
// reference} (the placement pass moves it to its final offset); static BP and
// uncompressed chunks have fixed offsets and are stored in place.  `remaining`
// counts the warp's output chunks left, this one included.
MS_DEV void store_staged(const ProduceArgs& a, int fmt, int bw, bool blockfmt, uint64_t g, uint64_t v[16], int valid,
                         uint16_t* out_stage, uint8_t* base, uint64_t avail, uint64_t static_chunks, DevCtl* ctl,
                         int lane, uint64_t top, StageCursor& sc, uint64_t remaining) {
    if (blockfmt) {
      uint8_t* arena = reinterpret_cast<uint8_t*>(ctl->arena);
      if (valid == kBlock) {
        uint64_t ref;
        int b = encode_block(layout_fmt(fmt), v, lane, &ref);
        if (is_static_cascade(fmt)) {  // every block at the column's width
          if (b > bw) {
            if (lane == 0) set_error(ctl, MS_ERR_VALUE_TOO_WIDE, g);
            const uint64_t mask = lowmask(bw);
#pragma unroll
            for (int k = 0; k < 16; k++) v[k] &= mask;
          }
          b = bw;
        }
        write_lane_stream(out_stage, lane, b, v);
        __syncwarp();
        uint64_t at = 0;
        if (b > 0) {
          at = stage_take(ctl, top, 64ull * b, remaining, sc, g, lane);
          if (at != ~0ull) {
            uint4* dst = reinterpret_cast<uint4*>(arena + at);
            const uint4* src = reinterpret_cast<const uint4*>(out_stage);
            for (int t = lane; t < 4 * b; t += 32) dst[t] = src[t];
          }
        }
        if (lane == 0) {
          a.stage_meta[2 * g] = (at << 8) | (uint64_t)b;
          a.stage_meta[2 * g + 1] = ref;
        }
      } else if (valid > 0) {  // remainder: raw values, placed behind the payload later
        const uint64_t at = stage_take(ctl, top, (8ull * valid + 63) & ~63ull, remaining, sc, g, lane);
        if (at != ~0ull) {
          uint64_t* dst = reinterpret_cast<uint64_t*>(arena + at);
#pragma unroll
          for (int k = 0; k < 16; k++)
            if (16 * lane + k < valid) dst[16 * lane + k] = v[k];
        }
        if (lane == 0) a.stage_meta[2 * g] = at << 8;
      }
    } else if (fmt == MS_STATIC_BP) {
      uint64_t o = 0;
#pragma unroll
      for (int k = 0; k < 16; k++) o |= (16 * lane + k < valid) ? v[k] : 0;
      o = warp_or(o);
      if (bw64(o) > bw && lane == 0) set_error(ctl, MS_ERR_VALUE_TOO_WIDE, g);
      const uint64_t mask = lowmask(bw);
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] &= mask;
      if (g < static_chunks) {
        write_lane_stream(out_stage, lane, bw, v);
        __syncwarp();
        const uint64_t pay = 64ull * bw * g;
        if (pay + 64ull * bw <= avail) {
          uint4* dst = reinterpret_cast<uint4*>(base + pay);
          const uint4* src = reinterpret_cast<const uint4*>(out_stage);
          for (int t = lane; t < 4 * bw; t += 32) dst[t] = src[t];
        } else if (lane == 0) {
          set_error(ctl, MS_ERR_NOMEM, g);
        }
      } else {  // horizontal tail
        uint32_t* w32 = reinterpret_cast<uint32_t*>(out_stage);
        for (int t = lane; t < 1024; t += 32) w32[t] = 0;
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 16; k++) {
          const int t = 16 * lane + k;
          if (t < valid && v[k]) {
            const uint64_t bit = (uint64_t)t * bw;
            const int sh = (int)(bit & 31);
            const uint64_t x = v[k];
            int wi = (int)(bit >> 5);
            atomicOr(w32 + wi, (uint32_t)(x << sh));
            uint64_t rest = (sh == 0) ? (x >> 32) : (x >> (32 - sh));
            int have = 32 - sh;
            while (have < bw && rest) {
              atomicOr(w32 + (++wi), (uint32_t)rest);
              rest >>= 32;
              have += 32;
            }
          }
        }
        __syncwarp();
        const uint64_t pay = 64ull * bw * static_chunks;
        const int nw = (int)(((uint64_t)valid * bw + 63) / 64);
        if (pay + 8ull * nw <= avail) {
          uint64_t* dst = reinterpret_cast<uint64_t*>(base + pay);
          const uint64_t* src = reinterpret_cast<const uint64_t*>(out_stage);
          for (int t = lane; t < nw; t += 32) dst[t] = src[t];
        } else if (lane == 0) {
          set_error(ctl, MS_ERR_NOMEM, g);
        }
      }
    } else if (valid > 0) {  // uncompressed output (arena column or caller buffer)
      const uint64_t pay = 8ull * kBlock * g;
      if (pay + 8ull * valid <= avail) {
        uint64_t* dst = reinterpret_cast<uint64_t*>(base + pay);
        if (valid == kBlock) {
          uint4* stg = reinterpret_cast<uint4*>(out_stage);
#pragma unroll
          for (int cc = 0; cc < 8; cc++)
            stg[lane * 8 + (cc ^ (lane & 7))] = make_uint4((uint32_t)v[2 * cc], (uint32_t)(v[2 * cc] >> 32),
                                                          (uint32_t)v[2 * cc + 1], (uint32_t)(v[2 * cc + 1] >> 32));
          __syncwarp();
#pragma unroll
          for (int it = 0; it < 8; it++) {
            const int ci = lane + 32 * it, L = ci >> 3, cc = ci & 7;
            reinterpret_cast<uint4*>(dst)[ci] = stg[L * 8 + (cc ^ (L & 7))];
          }
        } else {
#pragma unroll
          for (int k = 0; k < 16; k++)
            if (16 * lane + k < valid) dst[16 * lane + k] = v[k];
        }
      } else if (lane == 0) {
        set_error(ctl, MS_ERR_NOMEM, g);
      }
    }
}

// Epilogue of a staged producer: the last CTA to finish records the output column
// (fixed-offset formats are complete here; block formats are completed by the
// placement pass).  Every thread of every CTA calls it.
MS_DEV void publish_staged(const ProduceArgs& a, uint64_t n_out, int fmt, int bw, bool blockfmt, uint8_t* base,
                           uint64_t top, uint64_t avail) {
  DevCtl* ctl = a.ctl;
  // The last CTA reads nothing that another CTA wrote (later kernels see the output
  // through the kernel boundary), so only the counter needs ordering.
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      DevMeta* m = a.out_meta;
      m->n = n_out;
      m->ptr = reinterpret_cast<uint64_t>(base);
      m->fmt = (uint32_t)fmt;
      m->bw = (uint32_t)((fmt == MS_STATIC_BP || is_static_cascade(fmt)) ? bw : 0);
      m->nb = blockfmt ? n_out / kBlock : 0;
      if (!blockfmt) {
        const uint64_t size = fmt == MS_UNCOMPR ? 8 * n_out : 8 * ((n_out * (uint64_t)bw + 63) / 64);
        m->size = size;
        m->pwords = 0;
        const uint64_t grow = (size + 255) / 256 * 256;
        if (size > avail) {
          // the column did not fit: publish it empty so no reader leaves the arena
          set_error(ctl, MS_ERR_NOMEM, size);
          m->n = 0;
          m->size = 0;
          m->nb = 0;
        } else {
          ctl->top = top + grow;
          if (top + grow > ctl->high) ctl->high = top + grow;
        }
      }
      ctl->done = 0;
      __threadfence();
    }
  }
}

// Warp-independent producing kernel.  Every warp streams its own chunks (chunk
// gw, gw + W, ... for warp gw of W), runs the operator and encodes each output
// block.  Uncompressed and static-BP outputs have fixed offsets and are stored in
// place.  A block-format output block goes to the output stage at the arena's end,
// and its {stage offset, width, reference} to stage_meta.  k_place then computes
// the payload offsets and moves the compressed bytes into place.  No block
// barrier and no look-back, so no warp waits for another.
template <int OP>
__global__ void __launch_bounds__(kThreads, ProducePlan<OP>::kMinBlocks) k_map(ProduceArgs a) {
  using Smem = typename ProducePlan<OP>::Smem;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Smem* sm = reinterpret_cast<Smem*>(smem_raw) + warp;

  DevCtl* ctl = a.ctl;
  const bool raw = a.out_meta == nullptr;
  // the arena top changes only in the last CTA to finish, after every CTA read it
  const uint64_t top = raw ? 0 : ldg64(&ctl->top);
  const uint64_t avail = raw ? 8 * a.raw_cap : ctl->cap - top;
  uint8_t* base = raw ? reinterpret_cast<uint8_t*>(a.raw_out) : reinterpret_cast<uint8_t*>(ctl->arena + top);

  ColView c0{}, c1{};
  if (OP == OP_COMPRESS) c0 = view_raw(a.raw_in, a.raw_n);
  constexpr bool kProject = OP == OP_PROJECT || OP == OP_PROJECT_WARP;
  if (OP == OP_DECOMPRESS || OP == OP_CALC || kProject) c0 = view_of(a.in0);
  if ((OP == OP_CALC || kProject) && a.in1) c1 = view_of(a.in1);
  const uint64_t n_out = produce_n<OP>(a);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (OP == OP_DECOMPRESS && a.in0->n > a.raw_cap) set_error(ctl, MS_ERR_INVALID_ARG, a.in0->n);
    if (OP == OP_CALC && a.in1 && a.in0->n != a.in1->n) set_error(ctl, MS_ERR_INVALID_ARG, a.in1->n);
  }
  const int fmt = a.fmt, bw = a.bw;
  const bool blockfmt = is_block_fmt(fmt);
  const uint64_t nch = (n_out + kBlock - 1) / kBlock;
  const uint64_t static_chunks = n_out / kBlock;
  const uint64_t gw = (uint64_t)blockIdx.x * kWarps + warp, W = (uint64_t)gridDim.x * kWarps;
  // chunk i of a warp: gw + i*W.  A project from compressed data gathers a CTA tile
  // at a time: the CTA's warps take the 8 chunks of one tile together (tiles
  // blockIdx.x, blockIdx.x + gridDim.x, ...) and every warp runs the CTA's tile
  // count, since the gather synchronises the CTA.  A project from uncompressed data
  // reads at random: each warp takes a contiguous segment of output chunks so that
  // its reads move forward through the data column.
  const bool cta_gather = OP == OP_PROJECT && c0.fmt != MS_UNCOMPR;
  const uint64_t seg = (nch + W - 1) / W;
  const bool segmented = kProject && !cta_gather;
  const uint64_t first = segmented ? gw * seg : gw, stride = segmented ? 1 : W;
  const uint64_t count =
      segmented ? (first < nch ? min(seg, nch - first) : 0) : (gw < nch ? (nch - gw + W - 1) / W : 0);
  const uint64_t ntile = (nch + kWarps - 1) / kWarps;
  const uint64_t loop_n =
      cta_gather ? (blockIdx.x < ntile ? (ntile - blockIdx.x + gridDim.x - 1) / gridDim.x : 0) : count;

  constexpr int D = (OP == OP_CALC || kProject) ? kProdDepth2 : kProdDepth;
  StreamSmem<D>* ring0 = nullptr;
  StreamSmem<D>* ring1 = nullptr;
  if constexpr (OP == OP_COMPRESS || OP == OP_DECOMPRESS || kProject) ring0 = &sm->s0;
  if constexpr (OP == OP_CALC) {
    ring0 = &sm->s0;
    ring1 = &sm->s1;
  }
  const ColView main_col = kProject ? c1 : c0;
  ChunkStream<D> st0{main_col, first, stride, (OP == OP_EMIT) ? 0 : count, ring0, lane};
  ChunkStream<D> st1{c1, first, stride, (OP == OP_CALC && a.in1) ? count : 0, ring1, lane};
  if (OP != OP_EMIT && count) {
    for (int i = 0; i < D; i++) {
      st0.issue_header(i);
      st1.issue_header(i);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    for (int j = 0; j < D - 1; j++) {
      st0.prologue_step(j);
      st1.prologue_step(j);
      cp_async_commit();
    }
  }

  auto* pcta = reinterpret_cast<typename ProducePlan<OP>::Cta*>(smem_raw + sizeof(Smem) * kWarps);
  if constexpr (OP == OP_PROJECT) {  // the CTA span copy's shared state (only OP_PROJECT has it)
    // piece headers start zeroed: a slot that a corrupt chain skips then reads as an
    // empty block at offset 0, never as an offset outside the buffer
    for (int t = threadIdx.x; t < kCtaHdr; t += blockDim.x) pcta->hdr[t] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
      mbar_init(&pcta->mbar, 1);
      pcta->phase = 0;
      pcta->dead = 0;
    }
    __syncthreads();
  }
  // pipelined emit: the first block's plan and span, the second block's first chunks
  EmitPlan eplan{};
  uint64_t nbs0 = 0, nbs1 = 0;
  if constexpr (OP == OP_EMIT) {
    if (loop_n > 0) {
      const uint64_t g0 = first;
      eplan = emit_plan(a, n_out, g0, a.bstart[g0], g0 + 1 < nch ? a.bstart[g0 + 1] : 0);
      emit_stage(a, eplan.cfirst, (int)min((uint64_t)kEmitSpan, eplan.clast - eplan.cfirst + 1), sm->bits,
                 sm->coff, lane);
      if (loop_n > 1) {
        const uint64_t g1 = first + stride;
        nbs0 = a.bstart[g1];
        nbs1 = g1 + 1 < nch ? a.bstart[g1 + 1] : 0;
      }
    }
  }
  StageCursor sc{0, 0};
  for (uint64_t i = 0; i < loop_n; i++) {
    const uint64_t g = first + i * stride;
    uint64_t v[16];
    int valid = 0;
    uint16_t* out_stage;
    if constexpr (OP == OP_EMIT) {
      out_stage = reinterpret_cast<uint16_t*>(sm->aux);  // free once emit_expand returned
      uint32_t* cbits = (i & 1) ? sm->bits2 : sm->bits;
      uint64_t* ccoff = (i & 1) ? sm->coff2 : sm->coff;
      const EmitPlan cur = eplan;
      if (i + 1 < loop_n) {  // the next block: plan it and start its first span
        const uint64_t gn = g + stride;
        eplan = emit_plan(a, n_out, gn, nbs0, nbs1);
        emit_stage(a, eplan.cfirst, (int)min((uint64_t)kEmitSpan, eplan.clast - eplan.cfirst + 1),
                   (i & 1) ? sm->bits : sm->bits2, (i & 1) ? sm->coff : sm->coff2, lane);
        if (i + 2 < loop_n) {  // the block after: its first chunks, for the next plan
          const uint64_t g2 = gn + stride;
          nbs0 = a.bstart[g2];
          nbs1 = g2 + 1 < nch ? a.bstart[g2 + 1] : 0;
        }
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
      valid = emit_expand(a, cur, lane, v, sm, cbits, ccoff);
    } else {
      cp_async_wait<D - 2>();
      __syncwarp();
      st0.step(i);
      st1.step(i);
      cp_async_commit();
      out_stage = ring0->slot[i % D];
      if constexpr (OP == OP_COMPRESS || OP == OP_DECOMPRESS) {
        valid = st0.template decode<kCompactCodec, OP == OP_DECOMPRESS>(i, v, ctl);
        valid = (int)min((uint64_t)valid, n_out - g * kBlock);
      } else if constexpr (OP == OP_CALC) {
        valid = st0.decode(i, v, ctl);
        if (a.in1) {
          uint64_t w[16];
          valid = min(valid, st1.decode(i, w, ctl));
#pragma unroll
          for (int k = 0; k < 16; k++) v[k] = arith(a.arith, v[k], w[k]);
        } else {
#pragma unroll
          for (int k = 0; k < 16; k++) v[k] = arith(a.arith, v[k], a.scalar);
        }
      } else if constexpr (OP == OP_PROJECT) {  // c0 = data, st0 streams the positions (c1)
        uint64_t p[16];
        valid = st0.decode(i, p, ctl);
        __syncwarp();
        if (cta_gather) gather_cta(a, c0, p, valid, warp, lane, v, pcta);
        else project_direct(a, c0, p, valid, lane, v, reinterpret_cast<uint64_t*>(out_stage));
      } else {  // OP_PROJECT_WARP: per-warp gather (no CTA tile): DELTA data by block decode, others in place
        uint64_t p[16];
        valid = st0.decode(i, p, ctl);
        __syncwarp();
        if (c0.fmt != MS_DELTA_BP) {
          project_direct(a, c0, p, valid, lane, v, reinterpret_cast<uint64_t*>(out_stage));
        } else if (!project_delta_sorted(a, c0, p, valid, lane, v, sm->aux, reinterpret_cast<uint64_t*>(out_stage))) {
          project_delta(a, c0, p, valid, lane, v, reinterpret_cast<uint64_t*>(out_stage), sm->aux);
        }
      }
      __syncwarp();
    }
    store_staged(a, fmt, bw, blockfmt, g, v, valid, out_stage, base, avail, static_chunks, ctl, lane, top, sc,
                 loop_n - i);
    __syncwarp();
  }
  cp_async_wait<0>();

  // ---- epilogue: the last CTA to finish records the output column
  if (raw) return;
  publish_staged(a, n_out, fmt, bw, blockfmt, base, top, avail);
}

// Placement of a staged block-format column, in one pass over tiles of T
// consecutive blocks (tile t on CTA t mod grid; the grid never exceeds the CTAs that
// fit the GPU at once, so a tile's predecessors are always in progress).  T is the
// output's block count spread evenly over whole rounds of one tile per CTA, between 8
// and kPlaceTile, so that a small output still reaches every CTA and a large one
// resolves few look-backs per CTA, with every CTA copying a like share.  Per tile: the blocks' widths come from
// stage_meta, a CTA scan and a decoupled look-back over the tiles give every
// block's payload word offset, the final headers {(offset << 8) | width, ref} go to
// the arena top, and the CTA's warps copy the tile's payloads out of the stage, a
// block per warp with all its loads in flight at once.  The CTA of the last tile
// records the total payload words and places the raw remainder behind the payload;
// the last CTA to finish completes the column record, moves the arena top past the
// column and releases the stage.
struct PlaceArgs {
  DevCtl* ctl;
  DevMeta* out_meta;
  const uint64_t* stage_meta;
  uint64_t* status;  // look-back status words, one per tile, zeroed
};

constexpr int kPlacePer = 4;                      // blocks per thread in the width scan
constexpr int kPlaceTile = kThreads * kPlacePer;  // largest tile

// Bytes free for the output column between the arena top and the stage below the
// arena's end, and the stage's start (an arena offset).
struct PlaceRoom {
  uint64_t avail, lo;
};

// (The stage size and the arena top were set by earlier kernels and change only in
// the last CTA to finish, after every CTA read them: cached loads, so that the CTAs
// do not all queue on the control block's line in L2.)
MS_DEV PlaceRoom place_room(const DevCtl* ctl, uint64_t top) {
  const uint64_t end = stage_end(ctl);
  const uint64_t used = min(ldg64(&ctl->stage), end - top);
  return PlaceRoom{end - used - top, end - used};
}

template <int kUnused = 0>
__global__ void __launch_bounds__(kThreads) k_place(PlaceArgs a) {
  __shared__ uint64_t s_warp[kWarps];
  __shared__ uint64_t s_excl;
  __shared__ uint32_t s_off[kPlaceTile];  // payload words before the block, within its tile
  __shared__ uint64_t s_at[kPlaceTile];   // the block's stage offset, ~0 if it never reached the stage
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  DevCtl* ctl = a.ctl;
  const uint64_t n = ldg64(&a.out_meta->n), nb = n / kBlock, r = n % kBlock;
  const uint64_t top = ldg64(&ctl->top);
  const PlaceRoom room = place_room(ctl, top);
  const uint64_t avail = room.avail, send = stage_end(ctl);
  uint8_t* arena = reinterpret_cast<uint8_t*>(ctl->arena);
  uint8_t* base = arena + top;
  uint64_t* hdr = reinterpret_cast<uint64_t*>(base);
  // rounds of one tile per CTA, then tiles that fill those rounds evenly
  const uint64_t G = gridDim.x, rounds = max((uint64_t)1, (nb + (uint64_t)kPlaceTile * G - 1) / ((uint64_t)kPlaceTile * G));
  const uint64_t spread = (nb + rounds * G - 1) / (rounds * G);
  const int T = (int)min((uint64_t)kPlaceTile, max((uint64_t)8, (spread + 7) / 8 * 8));
  const uint64_t ntiles = (nb + T - 1) / T;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t t0 = tile * T;
    const int nt = (int)min((uint64_t)T, nb - t0);
    const int jb = kPlacePer * threadIdx.x;  // this thread's first block of the tile
    uint32_t b[kPlacePer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPlacePer; k++) {
      b[k] = jb + k < nt ? (uint32_t)min((uint64_t)64, a.stage_meta[2 * (t0 + jb + k)] & 255) : 0;
      sum += 8 * b[k];
    }
    const uint32_t texcl = warp_excl_scan32(sum, lane);
    if (lane == 31) s_warp[warp] = texcl + sum;
    __syncthreads();
    if (warp == 0) {
      const uint64_t wt = lane < kWarps ? s_warp[lane] : 0;
      const uint64_t wex = warp_excl_scan(wt, lane);
      const uint64_t agg = warp_sum(wt);
      const uint64_t ex = lookback(a.status, tile, agg, lane, ctl);
      if (lane < kWarps) s_warp[lane] = wex;
      if (lane == 0) {
        s_excl = ex;
        if (tile == ntiles - 1) ctl->op_words = ex + agg;
      }
    }
    __syncthreads();
    const uint64_t tex = s_excl;
    uint32_t o = (uint32_t)s_warp[warp] + texcl;  // words before the block within the tile: 32 bits
#pragma unroll
    for (int k = 0; k < kPlacePer; k++) {
      const int j = jb + k;
      if (j < nt) {
        const uint64_t g = t0 + j;
        s_off[j] = o;
        const uint64_t at = a.stage_meta[2 * g] >> 8;
        s_at[j] = (b[k] == 0 || (at >= room.lo && at + 64ull * b[k] <= send)) ? at : ~0ull;
        if (b[k] && s_at[j] == ~0ull) set_error(ctl, MS_ERR_NOMEM, g);  // the block never reached the stage
        if (16 * (g + 1) <= avail) {
          hdr[2 * g] = ((tex + o) << 8) | b[k];
          hdr[2 * g + 1] = a.stage_meta[2 * g + 1];
        } else {
          set_error(ctl, MS_ERR_NOMEM, g);
        }
        o += 8 * b[k];
      }
    }
    __syncthreads();
    // Copy: warp w moves the payloads of the tile's blocks [j0, j1), which are
    // consecutive in the output, as one run of 16-byte units with eight units per
    // lane in flight (blocks of a few bits hold only 16-64 units, so a block at a
    // time would wait one memory round trip per few hundred bytes).  A unit's block
    // is found by binary search over the blocks' unit offsets.
    const int per = (nt + kWarps - 1) / kWarps;
    const int j0 = min(nt, warp * per), j1 = min(nt, j0 + per);
    if (j0 < j1) {
      const uint32_t w0 = s_off[j0];
      const uint32_t total = (s_off[j1 - 1] - w0) / 2 + 4 * (uint32_t)min((uint64_t)64, a.stage_meta[2 * (t0 + j1 - 1)] & 255);
      const uint64_t pay = 16 * nb + 8 * (tex + w0);
      if (16 * (t0 + j1) <= avail && pay + 16ull * total <= avail) {
        uint4* dst = reinterpret_cast<uint4*>(base + pay);
        for (uint32_t u0 = 0; u0 < total; u0 += 256) {
          uint4 q[8];
          bool ok[8];
#pragma unroll
          for (int i = 0; i < 8; i++) {
            const uint32_t u = u0 + 32 * i + lane;
            ok[i] = false;
            if (u < total) {
              int lo = j0, hi = j1 - 1;  // the last block whose first unit is <= u
              while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((s_off[mid] - w0) / 2 <= u) lo = mid;
                else hi = mid - 1;
              }
              const uint64_t at = s_at[lo];
              if (at != ~0ull) {
                q[i] = reinterpret_cast<const uint4*>(arena + at)[u - (s_off[lo] - w0) / 2];
                ok[i] = true;
              }
            }
          }
#pragma unroll
          for (int i = 0; i < 8; i++)
            if (ok[i]) dst[u0 + 32 * i + lane] = q[i];
        }
      } else if (lane == 0) {  // no room for the headers or the payload (NOMEM, also raised above)
        set_error(ctl, MS_ERR_NOMEM, t0 + j0);
      }
    }
    __syncthreads();  // s_off / s_at are reused by the next tile
  }
  // the remainder, by the CTA of the last tile (CTA 0 when there is no block): that
  // CTA's warp 0 wrote the total payload words
  if (r && warp == 0 && blockIdx.x == (ntiles ? (ntiles - 1) % gridDim.x : 0)) {
    const uint64_t pwords = nb ? *reinterpret_cast<volatile uint64_t*>(&ctl->op_words) : 0;
    const uint64_t rem = 16 * nb + 8 * pwords, at = a.stage_meta[2 * nb] >> 8;
    if (rem + 8 * r <= avail && at >= room.lo && at + 8 * r <= send) {
      const uint64_t* src = reinterpret_cast<const uint64_t*>(arena + at);
      uint64_t* dst = reinterpret_cast<uint64_t*>(base + rem);
      for (uint64_t t = lane; t < r; t += 32) dst[t] = src[t];
    } else if (lane == 0) {
      set_error(ctl, MS_ERR_NOMEM, nb);
    }
  }
  // The last CTA reads only the total payload words, which thread 0 of the last
  // tile's CTA wrote before its fence and increment below.
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      const uint64_t pwords = nb ? *reinterpret_cast<volatile uint64_t*>(&ctl->op_words) : 0;
      const uint64_t size = 16 * nb + 8 * pwords + 8 * r;
      DevMeta* m = a.out_meta;
      m->ptr = reinterpret_cast<uint64_t>(base);
      m->size = size;
      m->nb = nb;
      m->pwords = pwords;
      const uint64_t grow = (size + 255) / 256 * 256;
      if (size > avail) {
        // the column did not fit: publish it empty so no reader leaves the arena
        set_error(ctl, MS_ERR_NOMEM, size);
        m->n = 0;
        m->size = 0;
        m->nb = 0;
        m->pwords = 0;
      } else {
        ctl->top = top + grow;
        // the stage below the arena's end was in use beside the new column
        const uint64_t peak = top + grow + (send - room.lo);
        if (peak > ctl->high) ctl->high = peak;
      }
      ctl->stage = 0;
      ctl->done = 0;
      __threadfence();
    }
  }
}


}  // namespace ms
