// ms_ops.cu -- operator entry points of libms: argument checks, scratch layout and
// the launch sequence of each operator.  Every launch is asynchronous on the
// caller's stream.
#include <algorithm>

#include "ms_launch.h"

namespace ms {

ms_status carve(ms_ctx* c, uint64_t n_max, uint64_t key_domain, Work* w, cudaStream_t s) {
  const uint64_t nch = std::max<uint64_t>(cdiv(n_max, kBlock), 1);
  const uint64_t ntiles = cdiv(nch, kWarps);
  const uint64_t st_b = align_up(8 * (ntiles + 1), 256);
  const uint64_t bm_b = align_up(64 * nch, 256);
  const uint64_t co_b = align_up(8 * (nch + 2), 256);
  const uint64_t kb_b = align_up(4 * cdiv(std::max<uint64_t>(key_domain, 1), 32), 256);
  const uint64_t cn_b = align_up(4 * (nch + 1), 256);
  const uint64_t sm_b = align_up(16 * (nch + 1), 256);
  // about 102 bytes per 512 rows; block payloads are staged in the arena
  const uint64_t total = 2 * st_b + bm_b + 2 * co_b + kb_b + cn_b + sm_b;
  ms_status st = ensure_work(c, total);
  if (st != MS_OK) return st;
  uint8_t* p = c->work;
  w->status = reinterpret_cast<uint64_t*>(p);
  w->status2 = reinterpret_cast<uint64_t*>(p + st_b);
  p += 2 * st_b;
  w->bitmap = reinterpret_cast<uint16_t*>(p);
  p += bm_b;
  w->coff = reinterpret_cast<uint64_t*>(p);
  p += co_b;
  w->bstart = reinterpret_cast<uint64_t*>(p);
  p += co_b;
  w->keybits = reinterpret_cast<uint32_t*>(p);
  p += kb_b;
  w->counts = reinterpret_cast<uint32_t*>(p);
  p += cn_b;
  w->stage_meta = reinterpret_cast<uint64_t*>(p);
  return cuda_status(cudaMemsetAsync(c->work, 0, 2 * st_b, s));
}

// Every select predicate as one range test over uint64 (Sec. 5.1 point and range
// predicates): x matches iff ((x - lo) <= span) != negate, and never if empty.
void predicate_as_range(int cmp, uint64_t c1, uint64_t c2, MarkArgs* m) {
  const uint64_t kMax = ~0ull;
  m->negate = 0;
  m->empty = 0;
  switch (cmp) {
    case MS_EQ: m->lo = c1; m->span = 0; break;
    case MS_NE: m->lo = c1; m->span = 0; m->negate = 1; break;
    case MS_LT: m->lo = 0; m->span = c1 - 1; m->empty = c1 == 0; break;
    case MS_LE: m->lo = 0; m->span = c1; break;
    case MS_GT: m->lo = c1 + 1; m->span = kMax - c1 - 1; m->empty = c1 == kMax; break;
    case MS_GE: m->lo = c1; m->span = kMax - c1; break;
    default: m->lo = c1; m->span = c2 - c1; m->empty = c2 < c1; break;  // MS_BETWEEN
  }
  // The range {x : (x - lo) mod 2^64 <= span} is a cyclic interval; its part below
  // 2^32 is again one cyclic interval of the 32-bit values (or none, or all).
  const uint64_t M = 0xffffffffull, lo = m->lo, span = m->span;
  m->lo32 = 0;
  m->span32 = 0;
  m->mode32 = 0;
  if (span == kMax) {  // every value
    m->mode32 = 2;
  } else if (lo + span >= lo) {  // no wrap: [lo, lo + span]
    if (lo > M) {
      m->mode32 = 1;
    } else {
      m->lo32 = (uint32_t)lo;
      m->span32 = (uint32_t)(std::min(lo + span, M) - lo);
    }
  } else {  // wraps: [lo, 2^64) and [0, lo + span - 2^64]
    const uint64_t hi = lo + span;  // mod 2^64
    if (lo > M) {  // only [0, hi] reaches below 2^32
      m->lo32 = 0;
      m->span32 = (uint32_t)std::min(hi, M);
    } else if (hi >= M || hi + 1 >= lo) {  // the two pieces cover [0, 2^32)
      m->mode32 = 2;
    } else {  // [lo, 2^32) and [0, hi]: the 32-bit interval from lo around to hi
      m->lo32 = (uint32_t)lo;
      m->span32 = (uint32_t)(hi - lo);  // mod 2^32
    }
  }
}

namespace {

bool owned(ms_ctx* c, const ms_column* col) { return col && col->ctx == c && !col->freed; }


// Launches k_map<OP> into a new arena column and, for block formats, places the
// staged blocks.
template <int OP>
ms_status produce_column(ms_ctx* c, ProduceArgs& a, const Work& w, uint64_t n_max, int fmt, int bw,
                         ms_column** out, cudaStream_t s) {
  ms_column* col = new_arena_column(c, fmt, bw, n_max);
  if (!col) return MS_ERR_NOMEM;
  a.ctl = c->ctl;
  a.out_meta = c->metas + col->slot;
  a.fmt = fmt;
  a.bw = has_static_bw(fmt) ? bw : 0;
  a.stage_meta = w.stage_meta;
  ms_status st = launch_map<OP>(c, a, n_max, s);
  if (st == MS_OK && host_block_fmt(fmt)) st = launch_place(c, w, a.out_meta, n_max, s);
  if (st != MS_OK) {
    // a producer that ran without its placement leaves stage bytes taken
    cudaMemsetAsync(&c->ctl->stage, 0, 8, s);
    drop_new_column(c, col);
    return st;
  }
  *out = col;
  return MS_OK;
}

// Second step of select / semi-join: match bitmap -> positions column.
ms_status emit_positions(ms_ctx* c, const Work& w, uint64_t n_max, int fmt, int bw, ms_column** out,
                         cudaStream_t s) {
  ProduceArgs a{};
  a.bitmap = w.bitmap;
  a.coff = w.coff;
  a.bstart = w.bstart;
  a.emit_nch = std::max<uint64_t>(cdiv(n_max, kBlock), 1);
  return produce_column<OP_EMIT>(c, a, w, n_max, fmt, bw, out, s);
}

}  // namespace
}  // namespace ms

using namespace ms;

extern "C" {

ms_status ms_compress(ms_ctx* c, const uint64_t* d_in, uint64_t n, int fmt, int bw, ms_column** out,
                      void* stream) {
  MS_TRACE();
  if (!c || !out || (!d_in && n) || !valid_format(fmt, bw)) return MS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_in) % 16) return MS_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w;
  ms_status st = carve(c, n, 0, &w, s);
  if (st != MS_OK) return st;
  if (fmt == MS_RLE) return rle_encode(c, nullptr, d_in, n, w, out, s);
  ProduceArgs a{};
  a.raw_in = d_in;
  a.raw_n = n;
  return produce_column<OP_COMPRESS>(c, a, w, n, fmt, bw, out, s);
}

ms_status ms_decompress(ms_ctx* c, const ms_column* col, uint64_t* d_out, uint64_t cap, void* stream) {
  MS_TRACE();
  if (!c || !owned(c, col) || (!d_out && cap)) return MS_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_out) % 16) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ProduceArgs a{};
  a.ctl = c->ctl;
  a.in0 = c->metas + col->slot;
  a.raw_out = d_out;
  a.raw_cap = cap;
  a.fmt = MS_UNCOMPR;
  return launch_map<OP_DECOMPRESS>(c, a, std::min(col->n_max, cap), s);
}

ms_status ms_morph(ms_ctx* c, const ms_column* col, int fmt, int bw, ms_column** out, void* stream) {
  MS_TRACE();
  if (!c || !out || !owned(c, col) || !valid_format(fmt, bw)) return MS_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w;
  ms_status st = carve(c, col->n_max, 0, &w, s);
  if (st != MS_OK) return st;
  if (fmt == MS_RLE) return rle_encode(c, c->metas + col->slot, nullptr, col->n_max, w, out, s, col->fmt == MS_RLE);
  ProduceArgs a{};
  a.in0 = c->metas + col->slot;
  a.raw_cap = ~0ull;
  return produce_column<OP_DECOMPRESS>(c, a, w, col->n_max, fmt, bw, out, s);
}

ms_status ms_select(ms_ctx* c, const ms_column* in, int cmp, uint64_t c1, uint64_t c2, int fmt, int bw,
                    ms_column** out, void* stream) {
  MS_TRACE();
  if (!c || !out || !owned(c, in) || !valid_format(fmt, bw) || cmp < MS_EQ || cmp > MS_BETWEEN)
    return MS_ERR_INVALID_ARG;
  *out = nullptr;
  if (fmt == MS_RLE) return MS_ERR_FORMAT;  // RLE comes from ms_compress / ms_morph
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w;
  ms_status st = carve(c, in->n_max, 0, &w, s);
  if (st != MS_OK) return st;
  MarkArgs m{};
  m.in = c->metas + in->slot;
  m.ctl = c->ctl;
  m.rle = in->fmt == MS_RLE;
  predicate_as_range(cmp, c1, c2, &m);
  st = launch_mark_scan(c, m, w, in->n_max, s);
  if (st != MS_OK) return st;
  return emit_positions(c, w, in->n_max, fmt, bw, out, s);
}

ms_status ms_select_packed(ms_ctx* c, const ms_column* in, int cmp, uint64_t c1, uint64_t c2, int fmt, int bw,
                           ms_column** out, void* stream) {
  MS_TRACE();
  if (!c || !out || !owned(c, in) || !valid_format(fmt, bw) || cmp < MS_EQ || cmp > MS_BETWEEN)
    return MS_ERR_INVALID_ARG;
  *out = nullptr;
  if (fmt == MS_RLE) return MS_ERR_FORMAT;  // RLE comes from ms_compress / ms_morph
  if (in->fmt == MS_UNCOMPR || in->fmt == MS_RLE) return MS_ERR_FORMAT;  // no bit-packed codes to work on
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w;
  ms_status st = carve(c, in->n_max, 0, &w, s);
  if (st != MS_OK) return st;
  MarkArgs m{};
  m.in = c->metas + in->slot;
  m.ctl = c->ctl;
  predicate_as_range(cmp, c1, c2, &m);
  st = launch_select_packed(c, m, w, in->n_max, s);
  if (st != MS_OK) return st;
  return emit_positions(c, w, in->n_max, fmt, bw, out, s);
}

ms_status ms_project(ms_ctx* c, const ms_column* data, const ms_column* pos, int fmt, int bw,
                     ms_column** out, void* stream) {
  MS_TRACE();
  if (!c || !out || !owned(c, data) || !owned(c, pos) || !valid_format(fmt, bw)) return MS_ERR_INVALID_ARG;
  *out = nullptr;
  if (fmt == MS_RLE) return MS_ERR_FORMAT;  // RLE comes from ms_compress / ms_morph
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w;
  ms_status st = carve(c, pos->n_max, 0, &w, s);
  if (st != MS_OK) return st;
  ProduceArgs a{};
  a.in0 = c->metas + data->slot;
  a.in1 = c->metas + pos->slot;
  // DELTA data needs whole-block decoding (prefix sums) and uncompressed data is read
  // in place, both by the per-warp gather.  DYN / FOR / static-BP data goes through the
  // CTA span gather when the positions are a DELTA column (sorted position lists are
  // kept as DELTA); other position columns (values used as keys, in any order) are
  // read in place by the per-warp gather, which keeps more warps per SM.  RLE data is
  // read by the per-warp gather too (directory, then a short search per position).
  // Both paths give the same values for any positions.
  const int dl = host_layout_fmt(data->fmt), pl = host_layout_fmt(pos->fmt);
  if (dl == MS_DELTA_BP || dl == MS_UNCOMPR || dl == MS_RLE || pl != MS_DELTA_BP)
    return produce_column<OP_PROJECT_WARP>(c, a, w, pos->n_max, fmt, bw, out, s);
  return produce_column<OP_PROJECT>(c, a, w, pos->n_max, fmt, bw, out, s);
}

ms_status ms_calc(ms_ctx* c, int op, const ms_column* x, const ms_column* y, uint64_t scalar, int fmt,
                  int bw, ms_column** out, void* stream) {
  MS_TRACE();
  if (!c || !out || !owned(c, x) || (y && !owned(c, y)) || !valid_format(fmt, bw) || op < MS_ADD ||
      op > MS_MUL)
    return MS_ERR_INVALID_ARG;
  *out = nullptr;
  if (fmt == MS_RLE) return MS_ERR_FORMAT;  // RLE comes from ms_compress / ms_morph
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t n_max = y ? std::min(x->n_max, y->n_max) : x->n_max;
  Work w;
  ms_status st = carve(c, n_max, 0, &w, s);
  if (st != MS_OK) return st;
  ProduceArgs a{};
  a.in0 = c->metas + x->slot;
  a.in1 = y ? c->metas + y->slot : nullptr;
  a.arith = op;
  a.scalar = scalar;
  return produce_column<OP_CALC>(c, a, w, n_max, fmt, bw, out, s);
}

ms_status ms_agg_sum(ms_ctx* c, const ms_column* in, uint64_t* d_result, void* stream) {
  MS_TRACE();
  if (!c || !owned(c, in) || !d_result) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cuda_status(cudaMemsetAsync(d_result, 0, 8, s)) != MS_OK) return MS_ERR_CUDA;
  return launch_agg_sum(c, c->metas + in->slot, d_result, in->n_max, s, in->fmt == MS_RLE);
}

ms_status ms_group_sum(ms_ctx* c, const ms_column* gid, const ms_column* val, uint64_t G, uint64_t* d_sums,
                       void* stream) {
  MS_TRACE();
  if (!c || !owned(c, gid) || !owned(c, val) || (!d_sums && G)) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (G && cuda_status(cudaMemsetAsync(d_sums, 0, 8 * G, s)) != MS_OK) return MS_ERR_CUDA;
  return launch_group_sum(c, c->metas + gid->slot, c->metas + val->slot, G, d_sums,
                          std::min(gid->n_max, val->n_max), s);
}

ms_status ms_semijoin(ms_ctx* c, const ms_column* probe, const ms_column* keys, uint64_t domain, int fmt,
                      int bw, ms_column** out, void* stream) {
  MS_TRACE();
  if (!c || !out || !owned(c, probe) || !owned(c, keys) || !valid_format(fmt, bw) || domain == 0)
    return MS_ERR_INVALID_ARG;
  *out = nullptr;
  if (fmt == MS_RLE) return MS_ERR_FORMAT;  // RLE comes from ms_compress / ms_morph
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Work w;
  ms_status st = carve(c, std::max(probe->n_max, keys->n_max), domain, &w, s);
  if (st != MS_OK) return st;
  if (cuda_status(cudaMemsetAsync(w.keybits, 0, 4 * cdiv(domain, 32), s)) != MS_OK) return MS_ERR_CUDA;
  st = launch_build_keys(c, c->metas + keys->slot, domain, w.keybits, keys->n_max, s, keys->fmt == MS_RLE);
  if (st != MS_OK) return st;
  MarkArgs m{};
  m.in = c->metas + probe->slot;
  m.ctl = c->ctl;
  m.keybits = w.keybits;
  m.domain = domain;
  m.rle = probe->fmt == MS_RLE;
  st = launch_mark_scan(c, m, w, probe->n_max, s);
  if (st != MS_OK) return st;
  return emit_positions(c, w, probe->n_max, fmt, bw, out, s);
}

ms_status ms_column_stats(ms_ctx* c, const ms_column* col, uint64_t* d_stats, void* stream) {
  MS_TRACE();
  if (!c || !owned(c, col) || !d_stats) return MS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cuda_status(cudaMemsetAsync(d_stats, 0, 8 * MS_STATS_WORDS, s)) != MS_OK) return MS_ERR_CUDA;
  return launch_stats(c, c->metas + col->slot, d_stats, col->n_max, s, col->fmt == MS_RLE);
}

ms_status ms_selftest_wait_timeout(ms_ctx* c, void* stream) {
  MS_TRACE();
  if (!c) return MS_ERR_INVALID_ARG;
  return launch_selftest_wait(c, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
