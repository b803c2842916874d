// ms_select_packed.cu -- the specialized select of Sec. 3.2 ("Specialized
// Operators"): a select that works on the compressed representation of its input
// instead of decompressing it.
//
// It is tailored to the block formats (dynamic BP, FOR+BP, DELTA+BP) and static
// BP, and uses what those formats know about each block:
//   * The header bounds every value of a block: [0, 2^b - 1] for dynamic BP,
//     [ref, ref + 2^b - 1] for FOR, [ref, ref + 511 * (2^b - 1)] for DELTA (the
//     first value plus at most 511 residuals below 2^b), [0, 2^bw - 1] for static
//     BP.  A block whose bound lies wholly inside the predicate's range matches
//     entirely, one wholly outside matches nowhere: neither is read or decoded,
//     only its 16-byte header.
//   * For the other blocks the predicate is moved into the residual domain once per
//     block (x = ref + r, so lo <= x <= hi becomes lo - ref <= r <= hi - ref), and
//     the b-bit residuals are compared as they come out of the packed lane stream,
//     in 32-bit arithmetic when b <= 32; FOR's reference is never added back.
//     DELTA residuals are prefix-summed (32-bit sums while the block's bound fits
//     32 bits) and compared relative to the block's first value.
// The output is the same per-chunk match bitmap and counts the general select's
// mark step writes, so the same scan and emit produce the positions column.
#include "ms_launch.h"

namespace ms {
namespace {

// The predicate as a linear interval [A, B] of uint64 plus a negation: the cyclic
// range test ((x - lo) <= span) != negate of MarkArgs, whose wrapped ranges become
// the complement of the gap they leave.
struct Interval {
  uint64_t A, B;
  bool neg, none;
};

MS_DEV Interval as_interval(const MarkArgs& a) {
  Interval iv;
  iv.none = a.empty != 0;
  iv.neg = a.negate != 0;
  const uint64_t hi = a.lo + a.span;
  if (hi >= a.lo) {
    iv.A = a.lo;
    iv.B = hi;
  } else {  // [lo, 2^64) and [0, hi]: the complement of (hi, lo)
    iv.A = hi + 1;
    iv.B = a.lo - 1;
    iv.neg = !iv.neg;
  }
  return iv;
}

// Lane `lane`'s 16-bit match mask for the residuals r[k] of a block whose values are
// R0 + r[k], given the interval [ra, rb] of matching residuals.
MS_DEV uint32_t residual_mask(const uint64_t r[16], uint64_t ra, uint64_t rb, int b) {
  uint32_t m = 0;
  if (b <= 32) {
    const uint32_t lo = (uint32_t)ra, span = (uint32_t)(rb - ra);
#pragma unroll
    for (int k = 0; k < 16; k++) m |= (uint32_t)((uint32_t)r[k] - lo <= span) << k;
  } else {
    const uint64_t span = rb - ra;
#pragma unroll
    for (int k = 0; k < 16; k++) m |= (uint32_t)(r[k] - ra <= span) << k;
  }
  return m;
}

__global__ void __launch_bounds__(kThreads, 2) k_select_packed(MarkArgs a) {
  const int lane = threadIdx.x & 31;
  const ColView c = view_of(a.in);
  const Interval iv = as_interval(a);
  const uint64_t nch = (c.n + kBlock - 1) / kBlock;
  const bool stat = c.fmt == MS_STATIC_BP;
  const uint64_t nfull = stat ? c.n / kBlock : c.nb;  // chunks with a packed payload
  const uint64_t W = (uint64_t)gridDim.x * kWarps;
  for (uint64_t g = (uint64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); g < nch; g += W) {
    const int valid = (int)min((uint64_t)kBlock, c.n - g * kBlock);
    uint32_t m16 = 0;
    if (iv.none) {
      m16 = 0;
    } else if (g < nfull) {
      int b;
      uint64_t ref = 0, pay = 0;
      if (stat) {
        b = c.bw;
        pay = 64ull * (uint64_t)b * g;
      } else {
        ulonglong2 h = make_ulonglong2(0, 0);
        if (16 * (g + 1) <= c.size) h = __ldg(reinterpret_cast<const ulonglong2*>(c.p) + g);
        b = (int)(h.x & 255);
        ref = c.fmt == MS_DYN_BP ? 0 : h.y;
        pay = 16 * c.nb + 8 * (h.x >> 8);
        if (b > 64 || pay + 64ull * b > c.size) {
          if (lane == 0) set_error(a.ctl, MS_ERR_FORMAT, g);
          b = 0;
        }
      }
      // bound of the block's values: [R0, R1]
      const uint64_t rmax = lowmask(b);
      const bool delta = c.fmt == MS_DELTA_BP;
      uint64_t R0 = ref, R1;
      bool bounded = true;
      if (delta) {
        const unsigned __int128 top = (unsigned __int128)ref + (unsigned __int128)rmax * 511u;
        bounded = (top >> 64) == 0;
        R1 = bounded ? (uint64_t)top : ~0ull;
      } else {
        // x = ref + r with no wrap (FOR's residual is x minus the block minimum), so
        // the bound saturates at 2^64 - 1 (FOR blocks of width 64 reach it)
        R1 = ref + rmax;
        if (R1 < ref) R1 = ~0ull;
      }
      const bool inside = bounded && iv.A <= R0 && R1 <= iv.B;
      const bool outside = bounded && (R1 < iv.A || R0 > iv.B);
      if (inside || outside) {
        m16 = inside ? 0xffffu : 0u;  // header only: the payload is not read
      } else {
        uint64_t r[16];
        read_lane_stream(reinterpret_cast<const uint16_t*>(c.p + (b ? pay : 0)), lane, b, r);
        if (!delta) {
          const uint64_t ra = iv.A > R0 ? iv.A - R0 : 0;
          const uint64_t rb = min(iv.B, R1) - R0;
          m16 = residual_mask(r, ra, rb, b);
        } else {
          // values relative to the block's first value: prefix sums of the residuals
          const uint64_t ra = iv.A > R0 ? iv.A - R0 : 0;
          const uint64_t rb = min(iv.B, R1) - R0;
          if (bounded && (R1 - R0) <= 0xffffffffull) {
            uint32_t s = 0;
#pragma unroll
            for (int k = 0; k < 16; k++) {
              s += (uint32_t)r[k];
              r[k] = s;
            }
            const uint32_t ex = warp_excl_scan32(s, lane);
#pragma unroll
            for (int k = 0; k < 16; k++) r[k] = (uint32_t)(r[k] + ex);
            m16 = residual_mask(r, ra, rb, 32);
          } else {
            uint64_t s = 0;
#pragma unroll
            for (int k = 0; k < 16; k++) {
              s += r[k];
              r[k] = s;
            }
            const uint64_t ex = warp_excl_scan(s, lane);
#pragma unroll
            for (int k = 0; k < 16; k++) r[k] += ex;  // values relative to the first
            if (bounded) {
              m16 = residual_mask(r, ra, rb, 64);
            } else {  // the sums may wrap: compare the absolute values
              const uint64_t span = iv.B - iv.A;
#pragma unroll
              for (int k = 0; k < 16; k++) m16 |= (uint32_t)(r[k] + ref - iv.A <= span) << k;
            }
          }
        }
      }
      if (iv.neg) m16 ^= 0xffffu;
    } else {  // raw remainder (block formats) or static BP's horizontal tail
      uint64_t x[16];
      if (stat) {
        const uint64_t* tail = reinterpret_cast<const uint64_t*>(c.p + 64ull * (uint64_t)c.bw * nfull);
        const uint64_t mask = lowmask(c.bw);
#pragma unroll
        for (int k = 0; k < 16; k++) {
          const int t = 16 * lane + k;
          uint64_t y = 0;
          if (t < valid) {
            const uint64_t bit = (uint64_t)t * (uint64_t)c.bw;
            const int s = (int)(bit & 63);
            y = ldg64(tail + (bit >> 6)) >> s;
            if (s + c.bw > 64) y |= ldg64(tail + (bit >> 6) + 1) << (64 - s);
            y &= mask;
          }
          x[k] = y;
        }
      } else {
        const uint64_t at = 16 * c.nb + 8 * c.pwords;
        const bool inside = at + 8 * (uint64_t)valid <= c.size;
        if (!inside && lane == 0) set_error(a.ctl, MS_ERR_FORMAT, g);
#pragma unroll
        for (int k = 0; k < 16; k++) {
          const int t = 16 * lane + k;
          x[k] = (t < valid && inside) ? ldg64(c.p + at + 8 * (uint64_t)t) : 0;
        }
      }
      const uint64_t span = iv.B - iv.A;
#pragma unroll
      for (int k = 0; k < 16; k++) m16 |= (uint32_t)(x[k] - iv.A <= span) << k;
      if (iv.neg) m16 ^= 0xffffu;
    }
    const int first = 16 * lane;
    m16 &= valid >= first + 16 ? 0xffffu : (valid > first ? (1u << (valid - first)) - 1u : 0u);
    a.bitmap[g * 32 + lane] = (uint16_t)m16;
    const uint32_t cnt = __reduce_add_sync(kFull, (uint32_t)__popc(m16));
    if (lane == 0) a.counts[g] = cnt;
  }
}

}  // namespace

ms_status launch_select_packed(ms_ctx* c, MarkArgs& a, const Work& w, uint64_t n_max, cudaStream_t s) {
  a.bitmap = w.bitmap;
  a.counts = w.counts;
  const uint64_t chunks = cdiv(std::max<uint64_t>(n_max, 1), kBlock);
  {
    const int grid = grid_for(c, k_select_packed, 0, cdiv(chunks, kWarps));
    ProfScope ps(c, MS_K_SELECT_PACKED, s);
    k_select_packed<<<grid, kThreads, 0, s>>>(a);
    if (cuda_status(cudaGetLastError()) != MS_OK) return MS_ERR_CUDA;
  }
  return launch_scan(c, a, w, n_max, s);
}

}  // namespace ms
