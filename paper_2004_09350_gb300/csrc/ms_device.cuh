// ms_device.cuh -- device-side building blocks of libms (sm_103a).
//
// Register arrangement used by every kernel: a warp owns one 512-value chunk of a
// column.  Lane j holds that chunk's values 16j .. 16j+15 in v[0..15].  This is the
// order in which the block layout packs them: lane j's values form lane j's
// 16-bit-interleaved stream.  So decoding and encoding a block are sequential,
// per-lane bit-stream loops over conflict-free shared-memory halfwords.  DELTA
// decoding is an in-lane prefix sum plus one warp scan of the 32 lane totals.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "morphstore.h"

#define MS_DEV __device__ __forceinline__

namespace ms {

constexpr int kBlock = 512;             // values per format block (SIMD-BP512, Sec. 4.1)
constexpr int kWarps = 8;               // warps per CTA; one chunk per warp per tile
constexpr int kThreads = 32 * kWarps;
constexpr int kTile = kBlock * kWarps;  // 4096 values per CTA tile
constexpr int kMaxSlots = 1 << 16;      // column metadata slots per context
constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kSpinLimit = 1u << 20;  // bounded waits (about a second with back-off)

// Per-column metadata, device resident (64 bytes).
struct DevMeta {
  uint64_t n;       // logical values
  uint64_t ptr;     // device address of the column buffer
  uint64_t size;    // physical bytes
  uint64_t nb;      // blocks of the main part (block formats), else 0
  uint64_t pwords;  // packed payload words (block formats), else 0
  uint32_t fmt, bw;
  uint64_t rsv[2];
};

// Per-context control block, device resident.
struct DevCtl {
  uint64_t arena;     // device address of the arena
  uint64_t cap;       // arena bytes
  uint64_t top;       // bytes in use (bump offset)
  uint64_t high;      // high-water mark of top
  uint32_t err;       // sticky ms_status of the first device error
  uint32_t done;      // last-CTA-done counter (reset by the last CTA)
  uint64_t err_info;  // detail of the first device error
  uint64_t op_n;      // element count produced by the last mark kernel
  uint64_t op_words;  // payload words published by an op's final tile
  uint64_t op_nch;    // input chunks of the last mark step (its real length, not a bound)
  uint64_t stage;     // bytes of the transient output stage, taken from the arena's end
  uint64_t rsv[6];
};

// Read-only view of a column inside a kernel.
struct ColView {
  const uint8_t* p;
  uint64_t n, nb, pwords, size;
  int fmt, bw;
};

// FOR / DELTA cascaded with static BP are stored in the FOR+BP / DELTA+BP layout
// (every block at one width), so readers see them as those formats.
MS_DEV int layout_fmt(int f) { return f == MS_FOR_STATIC_BP ? MS_FOR_BP : (f == MS_DELTA_STATIC_BP ? MS_DELTA_BP : f); }
MS_DEV bool is_static_cascade(int f) { return f == MS_FOR_STATIC_BP || f == MS_DELTA_STATIC_BP; }

MS_DEV ColView view_of(const DevMeta* m) {
  ColView c;
  c.p = reinterpret_cast<const uint8_t*>(m->ptr);
  c.n = m->n;
  c.nb = m->nb;
  c.pwords = m->pwords;
  c.size = m->size;
  c.fmt = layout_fmt((int)m->fmt);
  c.bw = is_static_cascade((int)m->fmt) ? 0 : (int)m->bw;
  return c;
}

MS_DEV ColView view_raw(const uint64_t* p, uint64_t n) {
  ColView c;
  c.p = reinterpret_cast<const uint8_t*>(p);
  c.n = n;
  c.nb = 0;
  c.pwords = 0;
  c.size = 8 * n;
  c.fmt = MS_UNCOMPR;
  c.bw = 64;
  return c;
}

MS_DEV bool is_block_fmt(int f) {
  return f == MS_DYN_BP || f == MS_DELTA_BP || f == MS_FOR_BP || f == MS_FOR_STATIC_BP || f == MS_DELTA_STATIC_BP;
}

MS_DEV int bw64(uint64_t x) { return x ? 64 - __clzll((long long)x) : 0; }
MS_DEV uint64_t lowmask(int b) { return b >= 64 ? ~0ull : ((1ull << b) - 1ull); }

MS_DEV void set_error(DevCtl* c, uint32_t code, uint64_t info) {
  if (atomicCAS(&c->err, 0u, code) == 0u) {
    c->err_info = info;
    __threadfence();
  }
}

// ------------------------------------------------------------- warp helpers

MS_DEV uint64_t warp_sum(uint64_t x) {
#pragma unroll
  for (int d = 16; d; d >>= 1) x += __shfl_xor_sync(kFull, x, d);
  return x;
}

MS_DEV uint64_t warp_excl_scan(uint64_t x, int lane) {
  uint64_t s = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t y = __shfl_up_sync(kFull, s, d);
    if (lane >= d) s += y;
  }
  return s - x;
}

MS_DEV uint32_t warp_excl_scan32(uint32_t x, int lane) {
  uint32_t s = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(kFull, s, d);
    if (lane >= d) s += y;
  }
  return s - x;
}

MS_DEV uint64_t warp_or(uint64_t x) {
  uint32_t lo = __reduce_or_sync(kFull, (uint32_t)x);
  uint32_t hi = __reduce_or_sync(kFull, (uint32_t)(x >> 32));
  return ((uint64_t)hi << 32) | lo;
}

MS_DEV uint64_t warp_min(uint64_t x) {
  uint32_t hi = __reduce_min_sync(kFull, (uint32_t)(x >> 32));
  uint32_t lo = __reduce_min_sync(kFull, (uint32_t)(x >> 32) == hi ? (uint32_t)x : kFull);
  return ((uint64_t)hi << 32) | lo;
}

MS_DEV uint64_t ldg64(const void* p) { return __ldg(reinterpret_cast<const unsigned long long*>(p)); }

// Warp copy of n16 (<= 256) 16-byte units from global to shared memory.  All loads
// are issued before the first store so that a warp keeps up to 4 KB in flight.
MS_DEV void warp_stage(uint4* dst, const uint4* src, int n16, int lane) {
  uint4 r[8];
#pragma unroll
  for (int it = 0; it < 8; it++) {
    int i = lane + 32 * it;
    if (i < n16) r[it] = __ldg(src + i);
  }
#pragma unroll
  for (int it = 0; it < 8; it++) {
    int i = lane + 32 * it;
    if (i < n16) dst[i] = r[it];
  }
}

// Swizzled slot of value o (0..511) of a chunk held as 512 uint64 in shared
// memory.  Lane j's 16 values stay inside slots 16j..16j+15 and a half-warp
// reading "its k-th value" touches 16 distinct banks.
MS_DEV int swz(int o) { return o ^ ((o >> 4) & 15); }

// ------------------------------------------------------- lane bit streams

// Width-specialised lane-stream codecs.  Lane `lane`'s stream at width B is B
// halfwords (s[32*q + lane], q < B); its 16 values sit at stream bits [k*B, k*B+B).
// The halfwords are gathered into 32-bit words once and every value is cut out
// with compile-time shifts.
template <int B>
MS_DEV void unpack16(const uint16_t* s, int lane, uint64_t v[16]) {
  if constexpr (B == 0) {
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = 0;
  } else {
    constexpr int NW = (B + 1) / 2;  // 32-bit words of the lane stream
    uint32_t w[NW + 1];
#pragma unroll
    for (int i = 0; i < NW; i++) {
      const uint32_t lo = s[32 * (2 * i) + lane];
      const uint32_t hi = (2 * i + 1 < B) ? (uint32_t)s[32 * (2 * i + 1) + lane] : 0u;
      w[i] = lo | (hi << 16);
    }
    w[NW] = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      constexpr uint64_t kMask = B >= 64 ? ~0ull : ((1ull << (B & 63)) - 1ull);
      const int bit = k * B, wi = bit >> 5, sh = bit & 31;
      if constexpr (B <= 32) {
        uint32_t x = sh ? __funnelshift_r(w[wi], w[wi + 1], sh) : w[wi];
        v[k] = (uint64_t)(B == 32 ? x : (x & (uint32_t)kMask));
      } else {
        const uint32_t x0 = sh ? __funnelshift_r(w[wi], w[wi + 1], sh) : w[wi];
        const uint32_t x1 = sh ? __funnelshift_r(w[wi + 1], (wi + 2 <= NW) ? w[wi + 2] : 0u, sh) : w[wi + 1];
        v[k] = (((uint64_t)x1 << 32) | x0) & kMask;
      }
    }
  }
}

template <int B>
MS_DEV void pack16(uint16_t* s, int lane, const uint64_t r[16]) {
  if constexpr (B > 0) {
    constexpr int NW = (B + 1) / 2;
    uint32_t w[NW + 1];
#pragma unroll
    for (int i = 0; i <= NW; i++) w[i] = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const int bit = k * B, wi = bit >> 5, sh = bit & 31;
      const uint64_t x = r[k];
      w[wi] |= (uint32_t)(x << sh);
      if (sh + B > 32) w[wi + 1] |= (uint32_t)(x >> (32 - sh));
      if (sh + B > 64) w[wi + 2] |= (uint32_t)(x >> (64 - sh));
    }
#pragma unroll
    for (int i = 0; i < NW; i++) {
      s[32 * (2 * i) + lane] = (uint16_t)w[i];
      if (2 * i + 1 < B) s[32 * (2 * i + 1) + lane] = (uint16_t)(w[i] >> 16);
    }
  }
}

#define MS_WIDTH_CASES(M)                                                                                       \
  M(0) M(1) M(2) M(3) M(4) M(5) M(6) M(7) M(8) M(9) M(10) M(11) M(12) M(13) M(14) M(15) M(16) M(17) M(18) M(19) \
  M(20) M(21) M(22) M(23) M(24) M(25) M(26) M(27) M(28) M(29) M(30) M(31) M(32) M(33) M(34) M(35) M(36) M(37)  \
  M(38) M(39) M(40) M(41) M(42) M(43) M(44) M(45) M(46) M(47) M(48) M(49) M(50) M(51) M(52) M(53) M(54) M(55)  \
  M(56) M(57) M(58) M(59) M(60) M(61) M(62) M(63) M(64)

// Compact lane-stream codec: one loop for every width (a running 64-bit window).
// Slower per value than the width-specialised one but a fraction of its code;
// translation units whose kernels juggle several streams can build with
// MS_COMPACT_CODEC to keep their instruction footprint small.
MS_DEV void read_lane_stream_compact(const uint16_t* s, int lane, int b, uint64_t v[16]) {
  const uint64_t mask = lowmask(b);
  uint64_t acc = 0;
  int have = 0, q = 0;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    uint64_t x = 0;
    if (b) {
      while (have < b && have <= 48) {
        acc |= (uint64_t)s[32 * q + lane] << have;
        have += 16;
        q++;
      }
      if (have >= b) {
        x = acc & mask;
        acc = (b == 64) ? 0 : (acc >> b);
        have -= b;
      } else {  // b > 48: the value continues in the next halfword
        const uint64_t h = s[32 * q + lane];
        q++;
        x = (acc | (h << have)) & mask;
        const int used = b - have;
        acc = h >> used;
        have = 16 - used;
      }
    }
    v[k] = x;
  }
}

// Reads lane `lane`'s 16 values of width b (0..64) from a block payload (stream
// halfword q of the lane at s[32*q + lane]; shared or global memory).
template <bool kCompact>
MS_DEV void read_lane_stream_as(const uint16_t* s, int lane, int b, uint64_t v[16]) {
  if constexpr (kCompact) {
    read_lane_stream_compact(s, lane, b, v);
    return;
  }
  switch (b) {
#define MS_UNPACK_CASE(B) \
  case B:                 \
    unpack16<B>(s, lane, v); \
    break;
    MS_WIDTH_CASES(MS_UNPACK_CASE)
#undef MS_UNPACK_CASE
    default:
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] = 0;
  }
}

#ifdef MS_COMPACT_CODEC
constexpr bool kCompactCodec = true;
#else
constexpr bool kCompactCodec = false;
#endif

MS_DEV void read_lane_stream(const uint16_t* s, int lane, int b, uint64_t v[16]) {
  read_lane_stream_as<kCompactCodec>(s, lane, b, v);
}

// Writes lane `lane`'s 16 residuals (each < 2^b) as its stream into shared memory.
MS_DEV void write_lane_stream(uint16_t* s, int lane, int b, const uint64_t r[16]) {
  switch (b) {
#define MS_PACK_CASE(B) \
  case B:               \
    pack16<B>(s, lane, r); \
    break;
    MS_WIDTH_CASES(MS_PACK_CASE)
#undef MS_PACK_CASE
    default:
      break;
  }
}

// ------------------------------------------------------------ RLE (Sec. 2.1)
// An RLE column holds R run values, R exclusive run ends (the last is n) and a
// directory of ceil(n/512) entries, entry g = the run that holds value 512*g
// (ColView.nb = R).

// True when the column's size holds its R runs and its directory.
MS_DEV bool rle_sound(const ColView& c) {
  const uint64_t nch = (c.n + kBlock - 1) / kBlock;
  return (c.n == 0 || c.nb > 0) && c.nb <= c.size / 16 && 16 * c.nb + 8 * nch <= c.size;
}

// The run that holds value i: the least r with ends[r] > i.  `lo` is a run known
// to start at or before i (ends[lo-1] <= i; 0 always is).  The search gallops
// forward from lo and then bisects, so a run near lo is found in a few loads.
// Every index read stays in [0, R) whatever the ends hold.
MS_DEV uint64_t rle_run_of(const uint64_t* ends, uint64_t R, uint64_t i, uint64_t lo) {
  if (lo >= R) lo = 0;
  uint64_t hi = lo, step = 1;
  while (hi < R - 1 && ldg64(ends + hi) <= i) {
    lo = hi + 1;
    hi = min(R - 1, hi + step);
    step <<= 1;
  }
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (ldg64(ends + mid) > i) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// The directory entries that bound block g's runs, on lanes 0 and 1: the run that
// holds the block's first value and the one that holds the next block's first value
// (the last run past the last block).  Other lanes get 0.
MS_DEV uint64_t rle_dir_load(const ColView& c, uint64_t g, int lane) {
  const uint64_t R = c.nb, nch = (c.n + kBlock - 1) / kBlock;
  if (lane >= 2 || !rle_sound(c) || R == 0 || g >= nch) return 0;
  const uint64_t* dir = reinterpret_cast<const uint64_t*>(c.p) + 2 * R;
  return g + lane < nch ? ldg64(dir + g + lane) : R - 1;
}

// Values of the block from its m <= 32 runs r0 .. r0+m-1 held one per lane (lane i:
// end e and value x of run r0 + i): the run of value t is r0 + the number of these
// runs that end at or before t.
MS_DEV void rle_values_from_runs(uint64_t row0, int lane, int valid, int m, uint64_t e, uint64_t x, uint64_t v[16]) {
  int j[16];
#pragma unroll
  for (int k = 0; k < 16; k++) j[k] = 0;
  for (int i = 0; i < m; i++) {
    const uint64_t ei = __shfl_sync(kFull, e, i);
#pragma unroll
    for (int k = 0; k < 16; k++) j[k] += ei <= row0 + k;
  }
#pragma unroll
  for (int k = 0; k < 16; k++) {
    const uint64_t xk = __shfl_sync(kFull, x, min(j[k], m - 1));
    v[k] = 16 * lane + k < valid ? xk : 0;
  }
}

// Values of block g of an RLE column into lane registers (value 16*lane + k of the
// block in v[k], zero past `valid`); d is this lane's rle_dir_load(c, g, lane).  When
// at most 32 runs cover the block (runs longer than 16 values on average), lane i
// loads run r0 + i and every value takes its run from the warp's registers.
// Otherwise each lane finds the run of its first value by a search from r0 and walks
// forward.
MS_DEV void rle_expand_at(const ColView& c, uint64_t g, int lane, int valid, uint64_t d, uint64_t v[16],
                          DevCtl* ctl) {
  const uint64_t R = c.nb;
  const uint64_t* val = reinterpret_cast<const uint64_t*>(c.p);
  const uint64_t* ends = val + R;
  if (!rle_sound(c) || valid <= 0) {
    if (lane == 0 && valid > 0) set_error(ctl, MS_ERR_FORMAT, g);
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = 0;
    return;
  }
  uint64_t r0 = __shfl_sync(kFull, d, 0);
  const uint64_t r1 = __shfl_sync(kFull, d, 1);
  if (r0 >= R) r0 = 0;
  const uint64_t row0 = g * kBlock + 16 * (uint64_t)lane;
  if (r1 < R && r1 >= r0 && r1 - r0 < 32) {
    const int m = (int)(r1 - r0) + 1;
    uint64_t e = 0, x = 0;
    if (lane < m) {
      e = ldg64(ends + r0 + lane);
      x = ldg64(val + r0 + lane);
    }
    rle_values_from_runs(row0, lane, valid, m, e, x, v);
    return;
  }
  uint64_t r = rle_run_of(ends, R, row0, r0);
  uint64_t e = ldg64(ends + r), x = ldg64(val + r);
#pragma unroll
  for (int k = 0; k < 16; k++) {
    if (16 * lane + k < valid) {
      while (row0 + k >= e && r + 1 < R) {
        r++;
        e = ldg64(ends + r);
        x = ldg64(val + r);
      }
      v[k] = x;
    } else {
      v[k] = 0;
    }
  }
}

MS_DEV void rle_expand(const ColView& c, uint64_t g, int lane, int valid, uint64_t v[16], DevCtl* ctl) {
  rle_expand_at(c, g, lane, valid, rle_dir_load(c, g, lane), v, ctl);
}

// Value i (< n) of an RLE column; 0 for a column whose size cannot hold its runs.
MS_DEV uint64_t rle_read_at(const ColView& c, uint64_t i) {
  if (!rle_sound(c) || c.nb == 0) return 0;
  const uint64_t R = c.nb;
  const uint64_t* val = reinterpret_cast<const uint64_t*>(c.p);
  const uint64_t* ends = val + R;
  const uint64_t* dir = ends + R;
  return ldg64(val + rle_run_of(ends, R, i, ldg64(dir + i / kBlock)));
}

// ------------------------------------------------------------- chunk decode

// Decodes chunk g (values 512g .. 512g+511) of column c into lane registers.  Returns
// the number of valid values in the chunk (0 past the end).  `stage` is the
// warp's 4 KB shared buffer.
MS_DEV int decode_chunk(const ColView& c, uint64_t g, int lane, uint64_t v[16], uint16_t* stage,
                        DevCtl* ctl) {
  const uint64_t base = g * kBlock;
  if (base >= c.n) {
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = 0;
    return 0;
  }
  const int valid = (int)min((uint64_t)kBlock, c.n - base);
  if (c.fmt == MS_RLE) {
    rle_expand(c, g, lane, valid, v, ctl);
    return valid;
  }
  if (c.fmt == MS_UNCOMPR) {
    const uint64_t* src = reinterpret_cast<const uint64_t*>(c.p) + base;
    if (valid == kBlock) {
      uint4* st = reinterpret_cast<uint4*>(stage);
      uint4 r[8];
#pragma unroll
      for (int it = 0; it < 8; it++) r[it] = __ldg(reinterpret_cast<const uint4*>(src) + lane + 32 * it);
#pragma unroll
      for (int it = 0; it < 8; it++) {
        int ci = lane + 32 * it, L = ci >> 3, cc = ci & 7;
        st[L * 8 + (cc ^ (L & 7))] = r[it];
      }
      __syncwarp();
#pragma unroll
      for (int cc = 0; cc < 8; cc++) {
        uint4 q = st[lane * 8 + (cc ^ (lane & 7))];
        v[2 * cc] = (uint64_t)q.x | ((uint64_t)q.y << 32);
        v[2 * cc + 1] = (uint64_t)q.z | ((uint64_t)q.w << 32);
      }
      __syncwarp();
    } else {
#pragma unroll
      for (int k = 0; k < 16; k++) {
        int i = 16 * lane + k;
        v[k] = i < valid ? ldg64(src + i) : 0;
      }
    }
    return valid;
  }
  if (c.fmt == MS_STATIC_BP) {
    const int b = c.bw;
    const uint64_t C = c.n / kBlock;
    if (g < C) {
      warp_stage(reinterpret_cast<uint4*>(stage),
                 reinterpret_cast<const uint4*>(c.p + 64ull * b * g), 4 * b, lane);
      __syncwarp();
      read_lane_stream(stage, lane, b, v);
      __syncwarp();
    } else {  // horizontal tail
      const uint64_t* tail = reinterpret_cast<const uint64_t*>(c.p + 64ull * b * C);
      const uint64_t mask = lowmask(b);
#pragma unroll
      for (int k = 0; k < 16; k++) {
        int t = 16 * lane + k;
        uint64_t x = 0;
        if (t < valid) {
          uint64_t bit = (uint64_t)t * b;
          int s = (int)(bit & 63);
          x = ldg64(tail + (bit >> 6)) >> s;
          if (s + b > 64) x |= ldg64(tail + (bit >> 6) + 1) << (64 - s);
          x &= mask;
        }
        v[k] = x;
      }
    }
    return valid;
  }
  // block formats
  if (g < c.nb) {
    const uint64_t* hdr = reinterpret_cast<const uint64_t*>(c.p) + 2 * g;
    const uint64_t w0 = ldg64(hdr), ref = ldg64(hdr + 1);
    int b = (int)(w0 & 255);
    const uint64_t off = w0 >> 8;
    if (b > 64) {
      if (lane == 0) set_error(ctl, MS_ERR_FORMAT, g);
      b = 0;
    }
    warp_stage(reinterpret_cast<uint4*>(stage),
               reinterpret_cast<const uint4*>(c.p + 16 * c.nb + 8 * off), 4 * b, lane);
    __syncwarp();
    read_lane_stream(stage, lane, b, v);
    __syncwarp();
    if (c.fmt == MS_FOR_BP) {
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] += ref;
    } else if (c.fmt == MS_DELTA_BP && b <= 23) {
      // 512 residuals below 2^23 sum below 2^32: prefix sums in 32 bits (b is the
      // block's width, so the warp branches together)
      uint32_t s = 0;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        s += (uint32_t)v[k];
        v[k] = s;
      }
      const uint64_t excl = (uint64_t)warp_excl_scan32(s, lane) + ref;
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] += excl;
    } else if (c.fmt == MS_DELTA_BP) {
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
  } else {  // uncompressed remainder behind the payload
    const uint64_t* rem = reinterpret_cast<const uint64_t*>(c.p + 16 * c.nb + 8 * c.pwords);
#pragma unroll
    for (int k = 0; k < 16; k++) {
      int t = 16 * lane + k;
      v[k] = t < valid ? ldg64(rem + t) : 0;
    }
  }
  return valid;
}

// ------------------------------------------------ asynchronous chunk streams

MS_DEV void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
MS_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
MS_DEV void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One-shot bulk copies (the TMA engine's 1-D form): a single thread moves a run of
// 16-byte units from global into shared memory, and the CTA waits on an mbarrier
// whose transaction count the copy decrements.  Both addresses and the size must be
// multiples of 16 bytes; the callers check that before issuing.
MS_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
MS_DEV void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
MS_DEV void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
MS_DEV void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Waits for phase `parity` of the barrier to complete; false after kSpinLimit polls.
MS_DEV bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t spins = 0; spins < kSpinLimit; spins++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// Per-warp shared memory of one column stream: D payload slots of 4 KB (a 512-value
// block at up to 64 bits) and 2D header slots.
template <int D, int SW = 64>
struct StreamSmem {
  uint16_t slot[D][32 * SW];
  uint64_t hdr[2 * D][2];
};

// A warp walks chunks first, first+stride, ... (count of them) of one column and
// keeps kDepth chunk payloads in flight with cp.async.  Block headers travel one
// level further ahead, so issuing a payload copy never waits on a header load.
// Groups: the prologue fetches the first kDepth headers synchronously, then
// commits P_j = {header j+D, payload j} for j < D-1, and iteration i commits
// G_i = {header i+2D-1, payload i+D-1}.  After cp.async.wait_group(D-2) at the
// top of iteration i, the payload of chunk i and every header up to chunk
// i+D-1 have landed.
// Staging of one chunk g of column c (used by the streams below): the block header
// (16 bytes, one lane) and the chunk's packed payload (16-byte cp.async units,
// swizzled for uncompressed chunks so that blocked reads are conflict-free).
MS_DEV void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// RLE: the "header" of block g is its two directory entries (rle_dir_load); the
// "payload" is the block's runs when at most 32 cover it: ends in slot words 0..31,
// values in words 32..63.
static __device__ __noinline__ void stage_rle_header(const ColView c, uint64_t g, uint64_t* hdr, int lane) {
  const uint64_t R = c.nb, nch = (c.n + kBlock - 1) / kBlock;
  if (lane >= 2 || !rle_sound(c) || R == 0 || g >= nch) return;
  const uint64_t* dir = reinterpret_cast<const uint64_t*>(c.p) + 2 * R;
  if (g + lane < nch) cp_async8(hdr + lane, dir + g + lane);
  else hdr[lane] = R - 1;
}
MS_DEV bool rle_window(const ColView& c, const uint64_t* hdr, uint64_t* r0, int* m) {
  const uint64_t R = c.nb, a = hdr[0], b = hdr[1];
  if (!rle_sound(c) || a >= R || b >= R || b < a || b - a >= 32) return false;
  *r0 = a;
  *m = (int)(b - a) + 1;
  return true;
}
static __device__ __noinline__ void stage_rle_payload(const ColView c, uint64_t g, const uint64_t* hdr, uint16_t* slot,
                                                      int lane) {
  uint64_t r0;
  int m;
  if (g >= (c.n + kBlock - 1) / kBlock || !rle_window(c, hdr, &r0, &m) || lane >= m) return;
  const uint64_t* val = reinterpret_cast<const uint64_t*>(c.p);
  uint64_t* w = reinterpret_cast<uint64_t*>(slot);
  cp_async8(w + lane, val + c.nb + r0 + lane);
  cp_async8(w + 32 + lane, val + r0 + lane);
}

// Block g of an RLE column from its staged runs (at most 32 cover it), else read in
// place; returned by value so that the caller's registers stay its own.
struct Values16 {
  uint64_t v[16];
};
static __device__ __noinline__ Values16 rle_decode_staged(const ColView c, uint64_t g, const uint64_t* hdr,
                                                  const uint16_t* slot, int lane, int valid, DevCtl* ctl) {
  Values16 r;
  uint64_t r0;
  int m;
  if (rle_window(c, hdr, &r0, &m)) {
    const uint64_t* w = reinterpret_cast<const uint64_t*>(slot);
    rle_values_from_runs(g * kBlock + 16 * (uint64_t)lane, lane, valid, m, lane < m ? w[lane] : 0,
                         lane < m ? w[32 + lane] : 0, r.v);
  } else {
    rle_expand(c, g, lane, valid, r.v, ctl);
  }
  return r;
}

MS_DEV void stage_header(const ColView& c, uint64_t g, uint64_t* hdr, int lane) {
  if (c.fmt == MS_RLE) {
    stage_rle_header(c, g, hdr, lane);
    return;
  }
  if (lane != 0 || !is_block_fmt(c.fmt)) return;
  if (g < c.nb && 16 * (g + 1) <= c.size) cp_async16(hdr, c.p + 16 * g);
}

// A payload of more than max_units 16-byte units is not staged; decode_staged with
// the same max_units then reads it in place from global memory.
MS_DEV void stage_payload(const ColView& c, uint64_t g, const uint64_t* hdr, uint16_t* slot, int lane,
                          int max_units = 256) {
  if (c.fmt == MS_RLE) {
    stage_rle_payload(c, g, hdr, slot, lane);
    return;
  }
  const uint8_t* src = nullptr;
  int units = 0;
  bool swizzle = false;
  if (c.fmt == MS_UNCOMPR) {
    if ((g + 1) * kBlock <= c.n) {
      src = c.p + 4096 * g;
      units = 256;
      swizzle = true;
    }
  } else if (c.fmt == MS_STATIC_BP) {
    if (g < c.n / kBlock) {
      src = c.p + 64ull * c.bw * g;
      units = 4 * c.bw;
    }
  } else if (g < c.nb) {
    const uint64_t w0 = hdr[0];
    const int b = (int)min((uint64_t)64, w0 & 255);
    // a payload outside the column (corrupt metadata) is never read
    if (16 * c.nb + 8 * ((w0 >> 8) + 8ull * b) <= c.size) {
      src = c.p + 16 * c.nb + 8 * (w0 >> 8);
      units = 4 * b;
    }
  }
  if (units > max_units) return;
  uint4* dst = reinterpret_cast<uint4*>(slot);
  for (int u = lane; u < units; u += 32) {
    const int d = swizzle ? (((u >> 3) << 3) | ((u & 7) ^ ((u >> 3) & 7))) : u;
    cp_async16(dst + d, reinterpret_cast<const uint4*>(src) + u);
  }
}

// Decodes staged chunk g of column c into lane registers; returns its valid count.
// Payloads above max_units 16-byte units (not staged) are read from global memory.
// kRleInline: RLE blocks decoded in line (the decompress / morph producer, where RLE
// input is the common case); elsewhere out of line, so that the kernel keeps its registers.
template <bool kCompact = kCompactCodec, bool kRleInline = false>
MS_DEV int decode_staged(const ColView& c, uint64_t g, const uint64_t* hdr, const uint16_t* slot, int lane,
                         uint64_t v[16], DevCtl* ctl, int max_units = 256) {
  const uint64_t base = g * kBlock;
  if (base >= c.n) {
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = 0;
    return 0;
  }
  const int valid = (int)min((uint64_t)kBlock, c.n - base);
  if (c.fmt == MS_RLE) {
    if constexpr (kRleInline) {
      uint64_t r0;
      int m;
      if (rle_window(c, hdr, &r0, &m)) {
        const uint64_t* w = reinterpret_cast<const uint64_t*>(slot);
        rle_values_from_runs(base + 16 * (uint64_t)lane, lane, valid, m, lane < m ? w[lane] : 0,
                             lane < m ? w[32 + lane] : 0, v);
      } else {
        rle_expand(c, g, lane, valid, v, ctl);
      }
    } else {
      const Values16 r = rle_decode_staged(c, g, hdr, slot, lane, valid, ctl);
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] = r.v[k];
    }
    return valid;
  }
  if (c.fmt == MS_UNCOMPR) {
    if (valid == kBlock && max_units >= 256) {
      const uint4* st = reinterpret_cast<const uint4*>(slot);
#pragma unroll
      for (int cc = 0; cc < 8; cc++) {
        const uint4 q = st[lane * 8 + (cc ^ (lane & 7))];
        v[2 * cc] = (uint64_t)q.x | ((uint64_t)q.y << 32);
        v[2 * cc + 1] = (uint64_t)q.z | ((uint64_t)q.w << 32);
      }
    } else if (valid == kBlock) {
      const uint4* src = reinterpret_cast<const uint4*>(c.p + 4096 * g) + 8 * lane;
#pragma unroll
      for (int cc = 0; cc < 8; cc++) {
        const uint4 q = __ldg(src + cc);
        v[2 * cc] = (uint64_t)q.x | ((uint64_t)q.y << 32);
        v[2 * cc + 1] = (uint64_t)q.z | ((uint64_t)q.w << 32);
      }
    } else {
      const uint64_t* src = reinterpret_cast<const uint64_t*>(c.p) + base;
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] = (16 * lane + k < valid) ? ldg64(src + 16 * lane + k) : 0;
    }
    return valid;
  }
  if (c.fmt == MS_STATIC_BP) {
    const int b = c.bw;
    const uint64_t C = c.n / kBlock;
    if (g < C) {
      const bool staged = 4 * b <= max_units;
      read_lane_stream_as<kCompact>(staged ? slot : reinterpret_cast<const uint16_t*>(c.p + 64ull * b * g), lane, b,
                                    v);
    } else {
      const uint64_t* tail = reinterpret_cast<const uint64_t*>(c.p + 64ull * b * C);
      const uint64_t mask = lowmask(b);
#pragma unroll
      for (int k = 0; k < 16; k++) {
        const int t = 16 * lane + k;
        uint64_t x = 0;
        if (t < valid) {
          const uint64_t bit = (uint64_t)t * b;
          const int s = (int)(bit & 63);
          x = ldg64(tail + (bit >> 6)) >> s;
          if (s + b > 64) x |= ldg64(tail + (bit >> 6) + 1) << (64 - s);
          x &= mask;
        }
        v[k] = x;
      }
    }
    return valid;
  }
  if (g < c.nb) {
    const uint64_t w0 = hdr[0], ref = hdr[1];
    int b = (int)(w0 & 255);
    if (b > 64 || 16 * (g + 1) > c.size || 16 * c.nb + 8 * ((w0 >> 8) + 8ull * b) > c.size) {
      if (lane == 0) set_error(ctl, MS_ERR_FORMAT, g);
      b = 0;
    }
    const bool staged = 4 * b <= max_units;
    read_lane_stream_as<kCompact>(
        staged ? slot : reinterpret_cast<const uint16_t*>(c.p + 16 * c.nb + 8 * (w0 >> 8)), lane, b, v);
    if (c.fmt == MS_FOR_BP) {
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] += ref;
    } else if (c.fmt == MS_DELTA_BP && b <= 23) {
      // 512 residuals below 2^23 sum below 2^32: prefix sums in 32 bits (b is the
      // block's width, so the warp branches together)
      uint32_t s = 0;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        s += (uint32_t)v[k];
        v[k] = s;
      }
      const uint64_t excl = (uint64_t)warp_excl_scan32(s, lane) + ref;
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] += excl;
    } else if (c.fmt == MS_DELTA_BP) {
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
  } else {
    const uint64_t* rem = reinterpret_cast<const uint64_t*>(c.p + 16 * c.nb + 8 * c.pwords);
    const bool inside = 16 * c.nb + 8 * (c.pwords + (uint64_t)valid) <= c.size;
    if (!inside && lane == 0) set_error(ctl, MS_ERR_FORMAT, g);
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const int t = 16 * lane + k;
      v[k] = (t < valid && inside) ? ldg64(rem + t) : 0;
    }
  }
  return valid;
}

template <int kDepth, int SW = 64>
struct ChunkStream {
  ColView c;
  uint64_t first, stride, count;
  StreamSmem<kDepth, SW>* sm;
  int lane;
  const uint32_t* list = nullptr;  // when set: chunk i is first + list[i] (ascending)

  MS_DEV uint64_t chunk(uint64_t i) const { return list ? first + list[i] : first + i * stride; }

  MS_DEV void issue_header(uint64_t i) {
    if (i < count) stage_header(c, chunk(i), sm->hdr[i % (2 * kDepth)], lane);
  }
  MS_DEV void issue_payload(uint64_t i) {
    if (i < count) stage_payload(c, chunk(i), sm->hdr[i % (2 * kDepth)], sm->slot[i % kDepth], lane, 4 * SW);
  }

  MS_DEV void prologue() {
    for (int i = 0; i < kDepth; i++) issue_header(i);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
  }
  MS_DEV void prologue_step(int j) {  // j < kDepth-1, commit by the caller
    issue_header(j + kDepth);
    issue_payload(j);
  }
  MS_DEV void step(uint64_t i) {  // at iteration i, commit by the caller
    issue_header(i + 2 * kDepth - 1);
    issue_payload(i + kDepth - 1);
  }

  // Decodes chunk i (already landed) into lane registers; returns its valid count.
  // kC selects the compact (one loop for every width) lane-stream decoder.
  template <bool kC = kCompactCodec, bool kRleInline = false>
  MS_DEV int decode(uint64_t i, uint64_t v[16], DevCtl* ctl) const {
    if (i >= count) {
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] = 0;
      return 0;
    }
    return decode_staged<kC, kRleInline>(c, chunk(i), sm->hdr[i % (2 * kDepth)], sm->slot[i % kDepth], lane, v,
                                         ctl, 4 * SW);
  }
};

// Random read of value i (< c.n) of a non-DELTA column (Sec. 4.2 random access).
MS_DEV uint64_t read_at(const ColView& c, uint64_t i) {
  if (c.fmt == MS_UNCOMPR) return ldg64(c.p + 8 * i);
  if (c.fmt == MS_RLE) return rle_read_at(c, i);
  const uint64_t g = i / kBlock;
  const int r = (int)(i % kBlock);
  int b;
  uint64_t ref = 0;
  const uint8_t* payload;
  if (c.fmt == MS_STATIC_BP) {
    b = c.bw;
    const uint64_t C = c.n / kBlock;
    if (g >= C) {
      const uint64_t* tail = reinterpret_cast<const uint64_t*>(c.p + 64ull * b * C);
      uint64_t bit = (uint64_t)r * b;
      int s = (int)(bit & 63);
      uint64_t x = ldg64(tail + (bit >> 6)) >> s;
      if (s + b > 64) x |= ldg64(tail + (bit >> 6) + 1) << (64 - s);
      return x & lowmask(b);
    }
    payload = c.p + 64ull * b * g;
  } else {
    if (g >= c.nb) {
      const uint64_t at = 16 * c.nb + 8 * c.pwords + 8 * (uint64_t)r;
      return at + 8 <= c.size ? ldg64(c.p + at) : 0;
    }
    const uint64_t* hdr = reinterpret_cast<const uint64_t*>(c.p) + 2 * g;
    const uint64_t w0 = ldg64(hdr);
    b = (int)min((uint64_t)64, w0 & 255);
    ref = ldg64(hdr + 1);
    if (16 * c.nb + 8 * ((w0 >> 8) + 8ull * b) > c.size) return 0;  // corrupt metadata: never read outside
    payload = c.p + 16 * c.nb + 8 * (w0 >> 8);
  }
  if (b == 0) return ref;
  const int j = r >> 4, k = r & 15;
  const int bit0 = k * b;
  const uint16_t* hw = reinterpret_cast<const uint16_t*>(payload);
  uint64_t x = 0;
  int got = 0;
  int q = bit0 >> 4, s = bit0 & 15;
  // gather up to five halfwords of lane j's stream
  x = (uint64_t)__ldg(hw + 32 * q + j) >> s;
  got = 16 - s;
  q++;
  while (got < b) {
    x |= (uint64_t)__ldg(hw + 32 * q + j) << got;
    got += 16;
    q++;
  }
  return (x & lowmask(b)) + ref;
}

// ----------------------------------------------- decoupled look-back (bounded)

// Status word per tile: bits 62-63 flag (0 none, 1 aggregate, 2 inclusive prefix),
// bits 0-61 value.  Executed by one whole warp.  Returns the exclusive prefix of
// tile `tile`.  A wait that exceeds the spin limit raises MS_ERR_TIMEOUT and
// treats the missing predecessors as zero.
#define MS_FLAG_AGG (1ull << 62)
#define MS_FLAG_PRE (2ull << 62)
#define MS_VAL_MASK ((1ull << 62) - 1)

MS_DEV void publish(uint64_t* st, uint64_t flag_val) {
  __threadfence();
  *reinterpret_cast<volatile uint64_t*>(st) = flag_val;
}

// First half of a split look-back: publish tile's aggregate (its inclusive prefix if
// it is tile 0).  Executed by one whole warp.
MS_DEV void lookback_publish(uint64_t* status, uint64_t tile, uint64_t agg, int lane) {
  if (lane == 0) publish(status + tile, (tile == 0 ? MS_FLAG_PRE : MS_FLAG_AGG) | agg);
}

// Second half: wait for the predecessors, publish the inclusive prefix and return the
// exclusive prefix (the aggregate was published by lookback_publish).
MS_DEV uint64_t lookback_resolve(uint64_t* status, uint64_t tile, uint64_t agg, int lane, DevCtl* ctl);

MS_DEV uint64_t lookback(uint64_t* status, uint64_t tile, uint64_t agg, int lane, DevCtl* ctl) {
  lookback_publish(status, tile, agg, lane);
  return lookback_resolve(status, tile, agg, lane, ctl);
}

MS_DEV uint64_t lookback_resolve(uint64_t* status, uint64_t tile, uint64_t agg, int lane, DevCtl* ctl) {
  if (tile == 0) return 0;
  // Each round reads a window of 256 predecessors, 8 consecutive ones per lane (lane
  // l: tiles hi - 8l - j, j = 0..7, newest first), so a look-back that has to walk
  // back over a whole round of CTAs (tiles whose inclusive prefix is not out yet)
  // takes one or two memory round trips instead of one per 32 tiles.
  constexpr int kPer = 8;
  uint64_t excl = 0;
  int64_t hi = (int64_t)tile - 1;
  uint32_t spins = 0;
  while (true) {
    uint64_t st[kPer];
#pragma unroll
    for (int j = 0; j < kPer; j++) {
      const int64_t t = hi - kPer * lane - j;
      st[j] = t >= 0 ? *reinterpret_cast<volatile uint64_t*>(status + t) : MS_FLAG_PRE;
    }
    int jp = kPer;  // the lane's newest inclusive prefix
    bool lnone = false;
    uint64_t lsum = 0;
#pragma unroll
    for (int j = 0; j < kPer; j++) {
      if (jp == kPer) {
        const uint32_t f = (uint32_t)(st[j] >> 62);
        lnone |= f == 0;
        lsum += st[j] & MS_VAL_MASK;
        if (f == 2) jp = j;
      }
    }
    const uint32_t pre = __ballot_sync(kFull, jp < kPer);
    const int first = pre ? __ffs(pre) - 1 : 31;
    const uint32_t need = first == 31 ? kFull : ((2u << first) - 1u);
    if (__ballot_sync(kFull, lnone) & need) {
      if (++spins > kSpinLimit) {
        if (lane == 0) set_error(ctl, MS_ERR_TIMEOUT, tile);
        break;
      }
      __nanosleep(64);
      continue;
    }
    __threadfence();
    excl += warp_sum(lane <= first ? lsum : 0);
    if (pre) break;
    hi -= 32 * kPer;
  }
  if (lane == 0) publish(status + tile, MS_FLAG_PRE | (excl + agg));
  return excl;
}

}  // namespace ms
