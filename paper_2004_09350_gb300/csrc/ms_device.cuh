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
  uint64_t rsv[8];
};

// Read-only view of a column inside a kernel.
struct ColView {
  const uint8_t* p;
  uint64_t n, nb, pwords, size;
  int fmt, bw;
};

MS_DEV ColView view_of(const DevMeta* m) {
  ColView c;
  c.p = reinterpret_cast<const uint8_t*>(m->ptr);
  c.n = m->n;
  c.nb = m->nb;
  c.pwords = m->pwords;
  c.size = m->size;
  c.fmt = (int)m->fmt;
  c.bw = (int)m->bw;
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

MS_DEV bool is_block_fmt(int f) { return f == MS_DYN_BP || f == MS_DELTA_BP || f == MS_FOR_BP; }

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

// Reads lane `lane`'s 16 values of width b from a block payload in shared memory
// (stream halfword q of the lane at s[32*q + lane]).
MS_DEV void read_lane_stream(const uint16_t* s, int lane, int b, uint64_t v[16]) {
  if (b == 0) {
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = 0;
    return;
  }
  const uint64_t mask = lowmask(b);
  uint64_t acc = 0;
  int have = 0, q = 0;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    while (have < b && have <= 48) {
      acc |= (uint64_t)s[32 * q + lane] << have;
      have += 16;
      q++;
    }
    uint64_t x;
    if (have >= b) {
      x = acc & mask;
      acc = (b == 64) ? 0 : (acc >> b);
      have -= b;
    } else {  // b > 48 and 48 < have < b: the value continues in the next halfword
      uint64_t h = s[32 * q + lane];
      q++;
      x = (acc | (h << have)) & mask;
      int used = b - have;
      acc = h >> used;
      have = 16 - used;
    }
    v[k] = x;
  }
}

// Writes lane `lane`'s 16 residuals (each < 2^b) as its stream into shared memory.
MS_DEV void write_lane_stream(uint16_t* s, int lane, int b, const uint64_t r[16]) {
  if (b == 0) return;
  uint64_t acc = 0;
  int have = 0, q = 0;
#pragma unroll
  for (int k = 0; k < 16; k++) {
    uint64_t x = r[k];
    if (have + b <= 64) {
      acc |= x << have;  // have <= 15 < 64
      have += b;
    } else {  // the value straddles the 64-bit accumulator: flush four halfwords
      acc |= x << have;
#pragma unroll
      for (int t = 0; t < 4; t++) {
        s[32 * q + lane] = (uint16_t)acc;
        acc >>= 16;
        q++;
      }
      int fit = 64 - have;
      acc = x >> fit;
      have = b - fit;
    }
    while (have >= 16) {
      s[32 * q + lane] = (uint16_t)acc;
      acc >>= 16;
      have -= 16;
      q++;
    }
  }
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

// Random read of value i (< c.n) of a non-DELTA column (Sec. 4.2 random access).
MS_DEV uint64_t read_at(const ColView& c, uint64_t i) {
  if (c.fmt == MS_UNCOMPR) return ldg64(c.p + 8 * i);
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
    if (g >= c.nb) return ldg64(c.p + 16 * c.nb + 8 * c.pwords + 8 * (uint64_t)r);
    const uint64_t* hdr = reinterpret_cast<const uint64_t*>(c.p) + 2 * g;
    const uint64_t w0 = ldg64(hdr);
    b = (int)min((uint64_t)64, w0 & 255);
    ref = ldg64(hdr + 1);
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

MS_DEV uint64_t lookback(uint64_t* status, uint64_t tile, uint64_t agg, int lane, DevCtl* ctl) {
  if (tile == 0) {
    if (lane == 0) publish(status, MS_FLAG_PRE | agg);
    return 0;
  }
  if (lane == 0) publish(status + tile, MS_FLAG_AGG | agg);
  uint64_t excl = 0;
  int64_t hi = (int64_t)tile - 1;
  uint32_t spins = 0;
  while (true) {
    const int64_t t = hi - lane;
    uint64_t s = t >= 0 ? *reinterpret_cast<volatile uint64_t*>(status + t) : MS_FLAG_PRE;
    const uint32_t flag = (uint32_t)(s >> 62);
    const uint32_t pre = __ballot_sync(kFull, flag == 2);
    const uint32_t none = __ballot_sync(kFull, flag == 0);
    const int first = pre ? __ffs(pre) - 1 : 31;
    const uint32_t need = first == 31 ? kFull : ((2u << first) - 1u);
    if (none & need) {
      if (++spins > kSpinLimit) {
        if (lane == 0) set_error(ctl, MS_ERR_TIMEOUT, tile);
        break;
      }
      __nanosleep(64);
      continue;
    }
    __threadfence();
    excl += warp_sum(lane <= first ? (s & MS_VAL_MASK) : 0);
    if (pre) break;
    hi -= 32;
  }
  if (lane == 0) publish(status + tile, MS_FLAG_PRE | (excl + agg));
  return excl;
}

}  // namespace ms
