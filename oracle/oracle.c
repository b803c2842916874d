/*
 * oracle.c -- plain CPU oracle (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Written from the paper's definitions, one obvious loop per definition, bit by
 * bit where bits are placed.  No blocking, fusion or reordering beyond what the
 * definitions state.
 *
 * Byte layout (the paper fixes the techniques but prints no bit layout; this is
 * the reading the whole project uses):
 *
 *  bw(x)       = number of significant bits of x, bw(0) = 0 (Sec. 2.1, BP: "the
 *                effective bit width of the largest value in the block").
 *  block       = 512 consecutive logical values (SIMD-BP512, Sec. 4).
 *  lane stream = inside a block, value i belongs to lane j = i / 16 as its
 *                k = i % 16-th value; lane j's 16 values are packed LSB-first,
 *                value k at stream bits [k*b, k*b+b).  Stream bit t lies in
 *                stream halfword q = t / 16, bit t % 16.  Stream halfword q of
 *                lane j is stored at halfword 32*q + j of the block payload
 *                (halfword h = bytes 2h, 2h+1, little-endian).  A block packed at
 *                width b therefore occupies 32*b halfwords = 64*b bytes.  This is
 *                SIMD-BP's vertical layout with 32 lanes of 16-bit units.
 *  UNCOMPR     = n little-endian uint64 words.                      size 8n
 *  STATIC_BP b = the first C = n / 512 chunks of 512 values as blocks packed at
 *                width b (chunk c at byte 64*b*c), then the r = n % 512 tail
 *                values packed LSB-first one after another (tail value t at tail
 *                bits [t*b, t*b+b), bit s of the tail at byte s/8, bit s%8),
 *                padded to whole uint64 words.          size ceil(n*b/64)*8
 *  DYN_BP / DELTA_BP / FOR_BP (Sec. 4, main part + uncompressed remainder):
 *                nb = n / 512 blocks, r = n % 512.
 *                header: nb entries of two uint64 words
 *                   word0 = (payload word offset of the block << 8) | b_k
 *                   word1 = reference value of the block (0 for DYN_BP)
 *                payload: block k's 512 residuals packed at width b_k (layout
 *                   above), starting at payload uint64 word offset
 *                   off_k = sum_{i<k} 8*b_i; payload starts at byte 16*nb.
 *                remainder: the last r values as raw uint64, right after the
 *                   payload (Sec. 4: "stored directly behind the compressed
 *                   data").
 *                size = 16*nb + 8*sum_k 8*b_k + 8*r
 *     DYN_BP   residual = value,                                ref = 0
 *     FOR_BP   residual = value - min(block),                   ref = min(block)
 *              (Sec. 2.1: FOR = difference to a reference value; the reference
 *               is read as the block minimum so that residuals are >= 0)
 *     DELTA_BP residual_0 = 0, residual_i = x_i - x_{i-1} mod 2^64, ref = x_0
 *              (Sec. 2.1: DELTA = difference to the predecessor; the chain
 *               restarts at every block so that blocks decode independently)
 *     b_k = bw(max residual of block k), 0..64.
 *  RLE (Sec. 2.1: RLE records each run of equal consecutive values once, with its
 *                repetition; the repetition is recorded here as the position where
 *                the run ends, so that a run's length is the difference of two
 *                consecutive ends):
 *                R runs, run r = the r-th maximal stretch of equal consecutive
 *                values; nch = ceil(n / 512).
 *                values: R uint64, value of run r at byte 8*r
 *                ends:   R uint64, end_r = index of the first value after run r
 *                        (exclusive; end_{R-1} = n), at byte 8*R + 8*r
 *                directory: nch uint64, entry g = index of the run that holds
 *                        value 512*g, at byte 16*R + 8*g (the block directory of
 *                        Sec. 4.2's random access: a block's first run without a
 *                        search)
 *                size = 16*R + 8*nch; n = 0 gives R = 0 and size 0.
 *  FOR_STATIC_BP / DELTA_STATIC_BP b (Sec. 2.1: FOR and DELTA cascaded with the
 *                NS algorithm static BP, "one block and fixed bit width" for the
 *                residuals): the layout of FOR_BP / DELTA_BP (same residuals,
 *                references, headers and remainder) with b_k = b for every block,
 *                b given by the caller (1..64); a residual wider than b is an error.
 *                size = 16*nb + 64*b*nb + 8*r
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

#define ORC_BLOCK 512u

int orc_bitwidth(uint64_t x) {
  int b = 0;
  while (x) {
    b++;
    x >>= 1;
  }
  return b;
}

/* ------------------------------------------------------------------ bits */

static void set_byte_bit(uint8_t *buf, uint64_t bitpos, int v) {
  if (v) buf[bitpos / 8] |= (uint8_t)(1u << (bitpos % 8));
}
static int get_byte_bit(const uint8_t *buf, uint64_t bitpos) {
  return (buf[bitpos / 8] >> (bitpos % 8)) & 1;
}

/* byte-level bit position of stream bit t of lane j in a vertical block */
static uint64_t lane_bit_address(int lane, uint64_t t) {
  uint64_t q = t / 16, within = t % 16;
  uint64_t halfword = 32 * q + (uint64_t)lane;
  return halfword * 16 + within;
}

/* pack 512 residuals at width b into blk (64*b bytes, zeroed by the caller) */
static void pack_block(const uint64_t *res, int b, uint8_t *blk) {
  for (int i = 0; i < (int)ORC_BLOCK; i++) {
    int lane = i / 16, k = i % 16;
    for (int s = 0; s < b; s++)
      set_byte_bit(blk, lane_bit_address(lane, (uint64_t)k * b + s),
                   (int)((res[i] >> s) & 1));
  }
}

static void unpack_block(const uint8_t *blk, int b, uint64_t *res) {
  for (int i = 0; i < (int)ORC_BLOCK; i++) {
    int lane = i / 16, k = i % 16;
    uint64_t v = 0;
    for (int s = 0; s < b; s++)
      v |= (uint64_t)get_byte_bit(blk, lane_bit_address(lane, (uint64_t)k * b + s)) << s;
    res[i] = v;
  }
}

/* ------------------------------------------------------- block transforms */

static int is_block_fmt(int fmt) {
  return fmt == ORC_DYN_BP || fmt == ORC_DELTA_BP || fmt == ORC_FOR_BP || fmt == ORC_FOR_STATIC_BP ||
         fmt == ORC_DELTA_STATIC_BP;
}

/* the cascades with static BP: every block at the caller's width */
static int is_static_cascade(int fmt) { return fmt == ORC_FOR_STATIC_BP || fmt == ORC_DELTA_STATIC_BP; }

/* residuals and reference of one block per the format definitions */
static void block_residuals(int fmt, const uint64_t *x, uint64_t *res, uint64_t *ref) {
  if (fmt == ORC_DYN_BP) {
    for (unsigned i = 0; i < ORC_BLOCK; i++) res[i] = x[i];
    *ref = 0;
  } else if (fmt == ORC_FOR_BP || fmt == ORC_FOR_STATIC_BP) {
    uint64_t mn = x[0];
    for (unsigned i = 1; i < ORC_BLOCK; i++)
      if (x[i] < mn) mn = x[i];
    for (unsigned i = 0; i < ORC_BLOCK; i++) res[i] = x[i] - mn;
    *ref = mn;
  } else { /* DELTA */
    res[0] = 0;
    for (unsigned i = 1; i < ORC_BLOCK; i++) res[i] = x[i] - x[i - 1];
    *ref = x[0];
  }
}

static int max_width(const uint64_t *res, unsigned cnt) {
  int b = 0;
  for (unsigned i = 0; i < cnt; i++) {
    int w = orc_bitwidth(res[i]);
    if (w > b) b = w;
  }
  return b;
}

void orc_block_widths(int fmt, const uint64_t *x, uint64_t n, uint8_t *widths) {
  uint64_t res[ORC_BLOCK], ref;
  for (uint64_t k = 0; k < n / ORC_BLOCK; k++) {
    block_residuals(fmt, x + k * ORC_BLOCK, res, &ref);
    widths[k] = (uint8_t)max_width(res, ORC_BLOCK);
  }
}

/* --------------------------------------------------------------- sizes */

/* number of runs of x[0..n): 1 + the number of i >= 1 with x[i] != x[i-1] */
static uint64_t run_count(const uint64_t *x, uint64_t n) {
  if (n == 0) return 0;
  uint64_t R = 1;
  for (uint64_t i = 1; i < n; i++)
    if (x[i] != x[i - 1]) R++;
  return R;
}

uint64_t orc_size(int fmt, int bw, const uint64_t *x, uint64_t n) {
  if (fmt == ORC_UNCOMPR) return 8 * n;
  if (fmt == ORC_RLE) return 16 * run_count(x, n) + 8 * ((n + ORC_BLOCK - 1) / ORC_BLOCK);
  if (fmt == ORC_STATIC_BP) {
    if (bw < 1 || bw > 64) return 0;
    uint64_t chunks = n / ORC_BLOCK, r = n % ORC_BLOCK;
    return chunks * 64 * (uint64_t)bw + 8 * ((r * (uint64_t)bw + 63) / 64);
  }
  if (!is_block_fmt(fmt)) return 0;
  uint64_t nb = n / ORC_BLOCK, r = n % ORC_BLOCK, words = 0;
  if (is_static_cascade(fmt)) return (bw < 1 || bw > 64) ? 0 : 16 * nb + 64 * (uint64_t)bw * nb + 8 * r;
  uint64_t res[ORC_BLOCK], ref;
  for (uint64_t k = 0; k < nb; k++) {
    block_residuals(fmt, x + k * ORC_BLOCK, res, &ref);
    words += 8 * (uint64_t)max_width(res, ORC_BLOCK);
  }
  return 16 * nb + 8 * words + 8 * r;
}

/* ------------------------------------------------------------ compress */

static void put_u64(uint8_t *p, uint64_t v) {
  for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static uint64_t get_u64(const uint8_t *p) {
  uint64_t v = 0;
  for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i);
  return v;
}

int orc_compress(int fmt, int bw, const uint64_t *x, uint64_t n, uint8_t *out,
                 uint64_t cap, uint64_t *size_out) {
  if (fmt < ORC_UNCOMPR || fmt > ORC_DELTA_STATIC_BP) return ORC_BAD_ARG;
  if ((fmt == ORC_STATIC_BP || is_static_cascade(fmt)) && (bw < 1 || bw > 64)) return ORC_BAD_ARG;
  uint64_t size = orc_size(fmt, bw, x, n);
  if (size > cap) return ORC_BAD_ARG;
  memset(out, 0, size);
  *size_out = size;

  if (fmt == ORC_RLE) {
    uint64_t R = run_count(x, n), r = 0;
    uint8_t *vals = out, *ends = out + 8 * R, *dir = out + 16 * R;
    for (uint64_t i = 0; i < n; i++) {
      if (i > 0 && x[i] != x[i - 1]) {
        put_u64(ends + 8 * r, i); /* run r ends where run r+1 starts */
        r++;
      }
      if (i == 0 || x[i] != x[i - 1]) put_u64(vals + 8 * r, x[i]);
      if (i % ORC_BLOCK == 0) put_u64(dir + 8 * (i / ORC_BLOCK), r);
    }
    if (n > 0) put_u64(ends + 8 * r, n);
    return ORC_OK;
  }

  if (fmt == ORC_UNCOMPR) {
    for (uint64_t i = 0; i < n; i++) put_u64(out + 8 * i, x[i]);
    return ORC_OK;
  }
  if (fmt == ORC_STATIC_BP) {
    for (uint64_t i = 0; i < n; i++)
      if (orc_bitwidth(x[i]) > bw) return ORC_TOO_WIDE;
    uint64_t chunks = n / ORC_BLOCK;
    for (uint64_t c = 0; c < chunks; c++)
      pack_block(x + c * ORC_BLOCK, bw, out + c * 64 * (uint64_t)bw);
    uint8_t *tail = out + chunks * 64 * (uint64_t)bw;
    for (uint64_t t = 0; t < n % ORC_BLOCK; t++) {
      uint64_t v = x[chunks * ORC_BLOCK + t];
      for (int s = 0; s < bw; s++)
        set_byte_bit(tail, t * (uint64_t)bw + s, (int)((v >> s) & 1));
    }
    return ORC_OK;
  }
  /* block formats */
  uint64_t nb = n / ORC_BLOCK, r = n % ORC_BLOCK;
  uint64_t res[ORC_BLOCK], ref, off = 0;
  uint8_t *payload = out + 16 * nb;
  for (uint64_t k = 0; k < nb; k++) {
    block_residuals(fmt, x + k * ORC_BLOCK, res, &ref);
    int b = max_width(res, ORC_BLOCK);
    if (is_static_cascade(fmt)) {
      if (b > bw) return ORC_TOO_WIDE;
      b = bw;
    }
    put_u64(out + 16 * k, (off << 8) | (uint64_t)b);
    put_u64(out + 16 * k + 8, ref);
    pack_block(res, b, payload + 8 * off);
    off += 8 * (uint64_t)b;
  }
  uint8_t *rem = payload + 8 * off;
  for (uint64_t t = 0; t < r; t++) put_u64(rem + 8 * t, x[nb * ORC_BLOCK + t]);
  return ORC_OK;
}

/* ---------------------------------------------------------- decompress */

int orc_decompress(int fmt, int bw, uint64_t n, const uint8_t *buf, uint64_t size,
                   uint64_t *out) {
  if (fmt == ORC_RLE) {
    uint64_t nch = (n + ORC_BLOCK - 1) / ORC_BLOCK;
    if (size < 8 * nch || (size - 8 * nch) % 16) return ORC_BAD_FORMAT;
    uint64_t R = (size - 8 * nch) / 16;
    if ((n == 0) != (R == 0)) return ORC_BAD_FORMAT;
    const uint8_t *vals = buf, *ends = buf + 8 * R, *dir = buf + 16 * R;
    uint64_t start = 0;
    for (uint64_t r = 0; r < R; r++) {
      uint64_t end = get_u64(ends + 8 * r), v = get_u64(vals + 8 * r);
      if (end <= start || end > n) return ORC_BAD_FORMAT;
      for (uint64_t i = start; i < end; i++) {
        out[i] = v;
        if (i % ORC_BLOCK == 0 && get_u64(dir + 8 * (i / ORC_BLOCK)) != r) return ORC_BAD_FORMAT;
      }
      start = end;
    }
    if (start != n) return ORC_BAD_FORMAT;
    return ORC_OK;
  }
  if (fmt == ORC_UNCOMPR) {
    if (size < 8 * n) return ORC_BAD_FORMAT;
    for (uint64_t i = 0; i < n; i++) out[i] = get_u64(buf + 8 * i);
    return ORC_OK;
  }
  if (fmt == ORC_STATIC_BP) {
    if (bw < 1 || bw > 64) return ORC_BAD_ARG;
    uint64_t chunks = n / ORC_BLOCK;
    uint64_t need = chunks * 64 * (uint64_t)bw + 8 * (((n % ORC_BLOCK) * (uint64_t)bw + 63) / 64);
    if (size < need) return ORC_BAD_FORMAT;
    for (uint64_t c = 0; c < chunks; c++)
      unpack_block(buf + c * 64 * (uint64_t)bw, bw, out + c * ORC_BLOCK);
    const uint8_t *tail = buf + chunks * 64 * (uint64_t)bw;
    for (uint64_t t = 0; t < n % ORC_BLOCK; t++) {
      uint64_t v = 0;
      for (int s = 0; s < bw; s++)
        v |= (uint64_t)get_byte_bit(tail, t * (uint64_t)bw + s) << s;
      out[chunks * ORC_BLOCK + t] = v;
    }
    return ORC_OK;
  }
  if (!is_block_fmt(fmt)) return ORC_BAD_ARG;
  if (is_static_cascade(fmt) && (bw < 1 || bw > 64)) return ORC_BAD_ARG;
  uint64_t nb = n / ORC_BLOCK, r = n % ORC_BLOCK;
  if (size < 16 * nb) return ORC_BAD_FORMAT;
  const uint8_t *payload = buf + 16 * nb;
  uint64_t expect_off = 0, res[ORC_BLOCK];
  for (uint64_t k = 0; k < nb; k++) {
    uint64_t w0 = get_u64(buf + 16 * k), ref = get_u64(buf + 16 * k + 8);
    int b = (int)(w0 & 0xff);
    uint64_t off = w0 >> 8;
    if (b > 64 || off != expect_off) return ORC_BAD_FORMAT;
    if (is_static_cascade(fmt) && b != bw) return ORC_BAD_FORMAT;
    if (16 * nb + 8 * (off + 8 * (uint64_t)b) > size) return ORC_BAD_FORMAT;
    unpack_block(payload + 8 * off, b, res);
    uint64_t *x = out + k * ORC_BLOCK;
    if (fmt == ORC_DYN_BP) {
      for (unsigned i = 0; i < ORC_BLOCK; i++) x[i] = res[i];
    } else if (fmt == ORC_FOR_BP || fmt == ORC_FOR_STATIC_BP) {
      for (unsigned i = 0; i < ORC_BLOCK; i++) x[i] = ref + res[i];
    } else { /* DELTA: x_0 = ref, x_i = x_{i-1} + residual_i */
      x[0] = ref + res[0];
      for (unsigned i = 1; i < ORC_BLOCK; i++) x[i] = x[i - 1] + res[i];
    }
    expect_off += 8 * (uint64_t)b;
  }
  if (16 * nb + 8 * expect_off + 8 * r > size) return ORC_BAD_FORMAT;
  const uint8_t *rem = payload + 8 * expect_off;
  for (uint64_t t = 0; t < r; t++) out[nb * ORC_BLOCK + t] = get_u64(rem + 8 * t);
  return ORC_OK;
}

/* ----------------------------------------------------------- operators */

/* select (Sec. 5.1 "Single Operator"): ascending positions of matching values */
static int pred(int cmp, uint64_t x, uint64_t c1, uint64_t c2) {
  switch (cmp) {
    case ORC_EQ: return x == c1;
    case ORC_NE: return x != c1;
    case ORC_LT: return x < c1;
    case ORC_LE: return x <= c1;
    case ORC_GT: return x > c1;
    case ORC_GE: return x >= c1;
    case ORC_BETWEEN: return x >= c1 && x <= c2;
  }
  return 0;
}

int orc_select(const uint64_t *x, uint64_t n, int cmp, uint64_t c1, uint64_t c2,
               uint64_t *pos, uint64_t *m_out) {
  if (cmp < ORC_EQ || cmp > ORC_BETWEEN) return ORC_BAD_ARG;
  uint64_t m = 0;
  for (uint64_t i = 0; i < n; i++)
    if (pred(cmp, x[i], c1, c2)) pos[m++] = i;
  *m_out = m;
  return ORC_OK;
}

/* project (Sec. 4 "Query Operators"): values of d at the given positions */
int orc_project(const uint64_t *d, uint64_t nd, const uint64_t *pos, uint64_t m,
                uint64_t *out) {
  for (uint64_t j = 0; j < m; j++) {
    if (pos[j] >= nd) return ORC_OUT_OF_RANGE;
    out[j] = d[pos[j]];
  }
  return ORC_OK;
}

/* calc: element-wise binary arithmetic modulo 2^64; b == NULL uses the scalar c */
int orc_calc(int op, const uint64_t *a, const uint64_t *b, uint64_t c, uint64_t n,
             uint64_t *out) {
  if (op < ORC_ADD || op > ORC_MUL) return ORC_BAD_ARG;
  for (uint64_t i = 0; i < n; i++) {
    uint64_t y = b ? b[i] : c;
    out[i] = op == ORC_ADD ? a[i] + y : op == ORC_SUB ? a[i] - y : a[i] * y;
  }
  return ORC_OK;
}

/* sum (Sec. 5.1 "Simple Query"): whole-column sum modulo 2^64 */
uint64_t orc_agg_sum(const uint64_t *x, uint64_t n) {
  uint64_t s = 0;
  for (uint64_t i = 0; i < n; i++) s += x[i];
  return s;
}

/* grouped sum into an uncompressed result (Sec. 4, random write access) */
int orc_group_sum(const uint64_t *g, const uint64_t *v, uint64_t n, uint64_t G,
                  uint64_t *sums) {
  for (uint64_t k = 0; k < G; k++) sums[k] = 0;
  for (uint64_t i = 0; i < n; i++) {
    if (g[i] >= G) return ORC_OUT_OF_RANGE;
    sums[g[i]] += v[i];
  }
  return ORC_OK;
}

/* semi-join: ascending positions of probe values that occur among the keys */
static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : x > y;
}

int orc_semijoin(const uint64_t *probe, uint64_t n, const uint64_t *keys,
                 uint64_t nk, uint64_t key_domain, uint64_t *pos, uint64_t *m_out) {
  uint64_t *sorted = (uint64_t *)malloc((nk ? nk : 1) * sizeof(uint64_t));
  if (!sorted) return ORC_BAD_ARG;
  for (uint64_t i = 0; i < nk; i++) {
    if (keys[i] >= key_domain) {
      free(sorted);
      return ORC_OUT_OF_RANGE;
    }
    sorted[i] = keys[i];
  }
  qsort(sorted, nk, sizeof(uint64_t), cmp_u64);
  uint64_t m = 0;
  for (uint64_t i = 0; i < n; i++) {
    uint64_t lo = 0, hi = nk; /* binary search for probe[i] */
    while (lo < hi) {
      uint64_t mid = lo + (hi - lo) / 2;
      if (sorted[mid] < probe[i]) lo = mid + 1; else hi = mid;
    }
    if (lo < nk && sorted[lo] == probe[i]) pos[m++] = i;
  }
  free(sorted);
  *m_out = m;
  return ORC_OK;
}
