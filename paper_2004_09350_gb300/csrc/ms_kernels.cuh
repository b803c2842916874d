// ms_kernels.cuh -- operator kernels of libms (sm_103a).
//
// Every operator is one or two persistent kernels that loop over 4096-value tiles
// (8 warps x one 512-value chunk each).  Input blocks are decoded into lane
// registers, the operator core runs on the uncompressed values, and output blocks
// are recompressed in shared memory before they are stored.  This is the
// on-the-fly de/re-compression degree of Sec. 3.2 at block granularity: only
// compressed bytes travel to and from device memory.  The payload offsets of
// dynamically sized output blocks come from a decoupled look-back over tiles.
#pragma once
#include "ms_device.cuh"

namespace ms {

// ------------------------------------------------------------------ select core

MS_DEV bool pred(int cmp, uint64_t x, uint64_t c1, uint64_t c2) {
  switch (cmp) {
    case MS_EQ: return x == c1;
    case MS_NE: return x != c1;
    case MS_LT: return x < c1;
    case MS_LE: return x <= c1;
    case MS_GT: return x > c1;
    case MS_GE: return x >= c1;
    default: return x >= c1 && x <= c2;
  }
}

// Mark kernel of select / semi-join.  Writes, per 512-row chunk of the input, a
// 512-bit match bitmap (lane j's 16 rows -> halfword j), the exclusive output offset
// of the chunk (coff, with coff[nchunks] = total), and for every output block h
// the chunk holding output element 512h (bstart).  The total goes to ctl->op_n.
struct MarkArgs {
  const DevMeta* in;
  DevCtl* ctl;
  int cmp;
  uint64_t c1, c2;
  const uint32_t* keybits;  // semi-join: membership bitmap over the key domain
  uint64_t domain;
  uint16_t* bitmap;
  uint64_t* coff;
  uint64_t* bstart;
  uint64_t* status;
};

#ifndef MS_PRODUCE_ONLY  // translation units that only instantiate k_produce
__global__ void __launch_bounds__(kThreads) k_mark(MarkArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ uint64_t s_cnt[kWarps];
  __shared__ uint64_t s_excl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint16_t* stage = reinterpret_cast<uint16_t*>(smem_raw) + warp * 2048;
  const ColView c = view_of(a.in);
  const uint64_t nch = (c.n + kBlock - 1) / kBlock, ntiles = (nch + kWarps - 1) / kWarps;
  if (c.n == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    a.coff[0] = 0;
    a.ctl->op_n = 0;
  }
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t g = tile * kWarps + warp;
    uint64_t v[16];
    const int valid = decode_chunk(c, g, lane, v, stage, a.ctl);
    uint32_t m16 = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      bool hit;
      if (a.keybits) {
        const uint64_t x = v[k];
        hit = x < a.domain && ((__ldg(a.keybits + (x >> 5)) >> (x & 31)) & 1u);
      } else {
        hit = pred(a.cmp, v[k], a.c1, a.c2);
      }
      if (hit && 16 * lane + k < valid) m16 |= 1u << k;
    }
    if (g < nch) a.bitmap[g * 32 + lane] = (uint16_t)m16;
    const uint64_t cnt = warp_sum(__popc(m16));
    if (lane == 0) s_cnt[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
      const uint64_t agg = warp_sum(lane < kWarps ? s_cnt[lane] : 0);
      const uint64_t ex = lookback(a.status, tile, agg, lane, a.ctl);
      if (lane == 0) s_excl = ex;
    }
    __syncthreads();
    if (g < nch && lane == 0) {
      uint64_t o0 = s_excl;
      for (int w = 0; w < warp; w++) o0 += s_cnt[w];
      a.coff[g] = o0;
      if (cnt) {
        for (uint64_t h = (o0 + kBlock - 1) / kBlock; h <= (o0 + cnt - 1) / kBlock; h++) a.bstart[h] = g;
      }
      if (g == nch - 1) {
        a.coff[nch] = o0 + cnt;
        a.ctl->op_n = o0 + cnt;
      }
    }
    __syncthreads();
  }
}

#endif  // MS_PRODUCE_ONLY

// ------------------------------------------------------- produce (map) kernel

enum ProduceOp { OP_COMPRESS = 0, OP_DECOMPRESS = 1, OP_PROJECT = 2, OP_CALC = 3, OP_EMIT = 4 };

struct ProduceArgs {
  DevCtl* ctl;
  // inputs
  const DevMeta* in0;      // compress: unused; decompress/calc a/project data
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
};

template <int OP>
struct SmemPlan {
  static constexpr int kPerWarp = (OP == OP_PROJECT || OP == OP_EMIT) ? 12288 : 8192;
};

// Output length of the operator (device-side, may depend on previous kernels).
template <int OP>
MS_DEV uint64_t produce_n(const ProduceArgs& a) {
  if (OP == OP_COMPRESS) return a.raw_n;
  if (OP == OP_DECOMPRESS) return min(a.in0->n, a.raw_cap);
  if (OP == OP_PROJECT) return a.in1->n;
  if (OP == OP_CALC) return a.in1 ? min(a.in0->n, a.in1->n) : a.in0->n;
  return *reinterpret_cast<volatile uint64_t*>(&a.ctl->op_n);  // OP_EMIT
}

MS_DEV uint64_t arith(int op, uint64_t x, uint64_t y) {
  return op == MS_ADD ? x + y : op == MS_SUB ? x - y : x * y;
}

// Produces output chunk g into v; returns its valid count.
template <int OP>
MS_DEV int produce_chunk(const ProduceArgs& a, const ColView& c0, const ColView& c1, uint64_t n_out,
                         uint64_t g, int lane, uint64_t v[16], uint16_t* in_stage, uint64_t* aux) {
  if (g * kBlock >= n_out) {
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = 0;
    return 0;
  }
  if (OP == OP_COMPRESS || OP == OP_DECOMPRESS) {
    const int valid = decode_chunk(c0, g, lane, v, in_stage, a.ctl);
    return (int)min((uint64_t)valid, n_out - g * kBlock);
  }
  if (OP == OP_CALC) {
    int valid = decode_chunk(c0, g, lane, v, in_stage, a.ctl);
    if (a.in1) {
      uint64_t w[16];
      const int v2 = decode_chunk(c1, g, lane, w, in_stage, a.ctl);
      valid = min(valid, v2);
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] = arith(a.arith, v[k], w[k]);
    } else {
#pragma unroll
      for (int k = 0; k < 16; k++) v[k] = arith(a.arith, v[k], a.scalar);
    }
    return valid;
  }
  if (OP == OP_PROJECT) {
    // c0 = data column, c1 = positions column
    uint64_t p[16];
    const int valid = decode_chunk(c1, g, lane, p, in_stage, a.ctl);
    uint32_t pending = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) {
      v[k] = 0;
      if (16 * lane + k < valid) {
        if (p[k] < c0.n) {
          pending |= 1u << k;
        } else {
          set_error(a.ctl, MS_ERR_OUT_OF_RANGE, p[k]);
        }
      }
    }
    if (c0.fmt != MS_DELTA_BP) {
#pragma unroll
      for (int k = 0; k < 16; k++)
        if (pending & (1u << k)) v[k] = read_at(c0, p[k]);
      return valid;
    }
    // DELTA data: decode each distinct block touched by the warp once (in order)
    while (true) {
      uint64_t mb = ~0ull;
#pragma unroll
      for (int k = 0; k < 16; k++)
        if (pending & (1u << k)) mb = min(mb, p[k] / kBlock);
      const uint64_t B = warp_min(mb);
      if (B == ~0ull) break;
      uint64_t t[16];
      decode_chunk(c0, B, lane, t, in_stage, a.ctl);
#pragma unroll
      for (int k = 0; k < 16; k++) aux[swz(16 * lane + k)] = t[k];
      __syncwarp();
#pragma unroll
      for (int k = 0; k < 16; k++) {
        if ((pending & (1u << k)) && p[k] / kBlock == B) {
          v[k] = aux[swz((int)(p[k] % kBlock))];
          pending &= ~(1u << k);
        }
      }
      __syncwarp();
    }
    return valid;
  }
  // OP_EMIT: positions of output block g from the match bitmap
  const uint64_t lo = g * kBlock;
  const int valid = (int)min((uint64_t)kBlock, n_out - lo);
  const uint64_t hi = lo + valid;
  // chunk range holding the block's outputs (clamped: scratch is never trusted blindly)
  const uint64_t cfirst = min(a.bstart[g], a.emit_nch - 1);
  const uint64_t clast = max(cfirst, min((hi < n_out) ? a.bstart[g + 1] : a.emit_nch - 1, a.emit_nch - 1));
  if (clast - cfirst < 32) {
    for (uint64_t ch = cfirst; ch <= clast; ch++) {
      uint32_t hw = a.bitmap[ch * 32 + lane];
      uint64_t o = a.coff[ch] + warp_excl_scan32(__popc(hw), lane);
      while (hw) {
        const int bb = __ffs(hw) - 1;
        hw &= hw - 1;
        if (o >= lo && o < hi) aux[swz((int)(o - lo))] = ch * kBlock + 16 * lane + bb;
        o++;
      }
    }
  } else {
    for (uint64_t ch = cfirst + lane; ch <= clast; ch += 32) {
      uint64_t o = a.coff[ch];
      const uint64_t e = a.coff[ch + 1];
      if (e <= o || e <= lo || o >= hi) continue;
      const uint32_t* w32 = reinterpret_cast<const uint32_t*>(a.bitmap + ch * 32);
      for (int w = 0; w < 16 && o < hi; w++) {
        uint32_t bits = w32[w];
        while (bits) {
          const int bb = __ffs(bits) - 1;
          bits &= bits - 1;
          if (o >= lo && o < hi) aux[swz((int)(o - lo))] = ch * kBlock + 32 * w + bb;
          o++;
        }
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 16; k++) {
    const int t = 16 * lane + k;
    v[k] = t < valid ? aux[swz(t)] : 0;
  }
  __syncwarp();
  return valid;
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

template <int OP>
__global__ void __launch_bounds__(kThreads) k_produce(ProduceArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ uint64_t s_words[kWarps];
  __shared__ uint64_t s_excl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* ws = smem_raw + warp * SmemPlan<OP>::kPerWarp;
  uint16_t* in_stage = reinterpret_cast<uint16_t*>(ws);
  uint16_t* out_stage = reinterpret_cast<uint16_t*>(ws + 4096);
  uint64_t* aux = reinterpret_cast<uint64_t*>(ws + 8192);

  DevCtl* ctl = a.ctl;
  const bool raw = a.out_meta == nullptr;
  const uint64_t top = raw ? 0 : *reinterpret_cast<volatile uint64_t*>(&ctl->top);
  const uint64_t avail = raw ? 8 * a.raw_cap : ctl->cap - top;
  uint8_t* base = raw ? reinterpret_cast<uint8_t*>(a.raw_out) : reinterpret_cast<uint8_t*>(ctl->arena + top);

  ColView c0{}, c1{};
  if (OP == OP_COMPRESS) c0 = view_raw(a.raw_in, a.raw_n);
  if (OP == OP_DECOMPRESS || OP == OP_CALC || OP == OP_PROJECT) c0 = view_of(a.in0);
  if ((OP == OP_CALC || OP == OP_PROJECT) && a.in1) c1 = view_of(a.in1);
  const uint64_t n_out = produce_n<OP>(a);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (OP == OP_DECOMPRESS && a.in0->n > a.raw_cap) set_error(ctl, MS_ERR_INVALID_ARG, a.in0->n);
    if (OP == OP_CALC && a.in1 && a.in0->n != a.in1->n) set_error(ctl, MS_ERR_INVALID_ARG, a.in1->n);
  }
  const int fmt = a.fmt, bw = a.bw;
  const bool blockfmt = is_block_fmt(fmt);
  const uint64_t nch = (n_out + kBlock - 1) / kBlock, ntiles = (nch + kWarps - 1) / kWarps;
  const uint64_t nb_out = blockfmt ? n_out / kBlock : 0;
  const uint64_t static_chunks = n_out / kBlock;

  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t g = tile * kWarps + warp;
    uint64_t v[16];
    const int valid = produce_chunk<OP>(a, c0, c1, n_out, g, lane, v, in_stage, aux);
    // ---- encode into the warp's shared stage
    int b = 0;
    uint64_t ref = 0, words = 0;
    if (blockfmt) {
      if (valid == kBlock) {
        b = encode_block(fmt, v, lane, &ref);
        write_lane_stream(out_stage, lane, b, v);
        words = 8ull * b;
      }
    } else if (fmt == MS_STATIC_BP && valid > 0) {
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
      } else {  // horizontal tail
        uint32_t* w32 = reinterpret_cast<uint32_t*>(out_stage);
        for (int i = lane; i < 1024; i += 32) w32[i] = 0;
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 16; k++) {
          const int t = 16 * lane + k;
          if (t < valid && v[k]) {
            const uint64_t bit = (uint64_t)t * bw;
            const int s = (int)(bit & 31);
            const uint64_t x = v[k];
            int wi = (int)(bit >> 5);
            atomicOr(w32 + wi, (uint32_t)(x << s));
            uint64_t rest = (s == 0) ? (x >> 32) : (x >> (32 - s));
            int have = 32 - s;
            while (have < bw && rest) {
              atomicOr(w32 + (++wi), (uint32_t)rest);
              rest >>= 32;
              have += 32;
            }
          }
        }
      }
      __syncwarp();
    }
    if (blockfmt) {
      if (lane == 0) s_words[warp] = words;
      __syncthreads();
      if (warp == 0) {
        const uint64_t agg = warp_sum(lane < kWarps ? s_words[lane] : 0);
        const uint64_t ex = lookback(a.status, tile, agg, lane, ctl);
        if (lane == 0) {
          s_excl = ex;
          if (tile == ntiles - 1) ctl->op_words = ex + agg;
        }
      }
      __syncthreads();
    }
    // ---- store
    if (valid > 0) {
      if (blockfmt) {
        uint64_t off = s_excl;
        for (int w = 0; w < warp; w++) off += s_words[w];
        if (valid == kBlock) {
          const uint64_t pay = 16 * nb_out + 8 * off;
          if (16 * (g + 1) <= avail && pay + 64ull * b <= avail) {
            if (lane == 0) {
              uint64_t* h = reinterpret_cast<uint64_t*>(base) + 2 * g;
              h[0] = (off << 8) | (uint64_t)b;
              h[1] = ref;
            }
            uint4* dst = reinterpret_cast<uint4*>(base + pay);
            const uint4* src = reinterpret_cast<const uint4*>(out_stage);
            for (int i = lane; i < 4 * b; i += 32) dst[i] = src[i];
          } else if (lane == 0) {
            set_error(ctl, MS_ERR_NOMEM, g);
          }
        } else {  // remainder: raw values behind the whole payload
          const uint64_t rem = 16 * nb_out + 8 * off;
          if (rem + 8ull * valid <= avail) {
            uint64_t* dst = reinterpret_cast<uint64_t*>(base + rem);
#pragma unroll
            for (int k = 0; k < 16; k++)
              if (16 * lane + k < valid) dst[16 * lane + k] = v[k];
          } else if (lane == 0) {
            set_error(ctl, MS_ERR_NOMEM, g);
          }
        }
      } else if (fmt == MS_STATIC_BP) {
        if (g < static_chunks) {
          const uint64_t pay = 64ull * bw * g;
          if (pay + 64ull * bw <= avail) {
            uint4* dst = reinterpret_cast<uint4*>(base + pay);
            const uint4* src = reinterpret_cast<const uint4*>(out_stage);
            for (int i = lane; i < 4 * bw; i += 32) dst[i] = src[i];
          } else if (lane == 0) {
            set_error(ctl, MS_ERR_NOMEM, g);
          }
        } else {
          const uint64_t pay = 64ull * bw * static_chunks;
          const int nw = (int)(((uint64_t)valid * bw + 63) / 64);
          if (pay + 8ull * nw <= avail) {
            uint64_t* dst = reinterpret_cast<uint64_t*>(base + pay);
            const uint64_t* src = reinterpret_cast<const uint64_t*>(out_stage);
            for (int i = lane; i < nw; i += 32) dst[i] = src[i];
          } else if (lane == 0) {
            set_error(ctl, MS_ERR_NOMEM, g);
          }
        }
      } else {  // uncompressed output (arena column or caller buffer)
        const uint64_t pay = 8ull * kBlock * g;
        if (pay + 8ull * valid <= avail) {
          uint64_t* dst = reinterpret_cast<uint64_t*>(base + pay);
          if (valid == kBlock) {
            uint4* st = reinterpret_cast<uint4*>(out_stage);
#pragma unroll
            for (int cc = 0; cc < 8; cc++)
              st[lane * 8 + (cc ^ (lane & 7))] =
                  make_uint4((uint32_t)v[2 * cc], (uint32_t)(v[2 * cc] >> 32), (uint32_t)v[2 * cc + 1],
                             (uint32_t)(v[2 * cc + 1] >> 32));
            __syncwarp();
#pragma unroll
            for (int it = 0; it < 8; it++) {
              const int ci = lane + 32 * it, L = ci >> 3, cc = ci & 7;
              reinterpret_cast<uint4*>(dst)[ci] = st[L * 8 + (cc ^ (L & 7))];
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
    __syncwarp();
    if (blockfmt) __syncthreads();
  }

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
        set_error(ctl, MS_ERR_NOMEM, size);
      } else {
        ctl->top = top + grow;
        if (top + grow > ctl->high) ctl->high = top + grow;
      }
      ctl->done = 0;
      __threadfence();
    }
  }
}

#ifndef MS_PRODUCE_ONLY
// ----------------------------------------------------------------- aggregates

__global__ void __launch_bounds__(kThreads) k_agg_sum(const DevMeta* in, uint64_t* result, DevCtl* ctl) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  __shared__ uint64_t s_part[kWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint16_t* stage = reinterpret_cast<uint16_t*>(smem_raw) + warp * 2048;
  const ColView c = view_of(in);
  const uint64_t nch = (c.n + kBlock - 1) / kBlock, ntiles = (nch + kWarps - 1) / kWarps;
  uint64_t acc = 0;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    uint64_t v[16];
    const int valid = decode_chunk(c, tile * kWarps + warp, lane, v, stage, ctl);
#pragma unroll
    for (int k = 0; k < 16; k++) acc += (16 * lane + k < valid) ? v[k] : 0;
  }
  acc = warp_sum(acc);
  if (lane == 0) s_part[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < kWarps; w++) t += s_part[w];
    if (t) atomicAdd(reinterpret_cast<unsigned long long*>(result), (unsigned long long)t);
  }
}

constexpr int kSmemGroups = 4096;

__global__ void __launch_bounds__(kThreads) k_group_sum(const DevMeta* gid, const DevMeta* val, uint64_t G,
                                                         uint64_t* sums, DevCtl* ctl) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint16_t* stage = reinterpret_cast<uint16_t*>(smem_raw) + warp * 2048;
  unsigned long long* hist = reinterpret_cast<unsigned long long*>(smem_raw + kWarps * 4096);
  const bool local = G <= kSmemGroups;
  if (local)
    for (uint64_t k = threadIdx.x; k < G; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  const ColView cg = view_of(gid), cv = view_of(val);
  if (blockIdx.x == 0 && threadIdx.x == 0 && cg.n != cv.n) set_error(ctl, MS_ERR_INVALID_ARG, cv.n);
  const uint64_t n = min(cg.n, cv.n);
  const uint64_t nch = (n + kBlock - 1) / kBlock, ntiles = (nch + kWarps - 1) / kWarps;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t g = tile * kWarps + warp;
    uint64_t k8[16], v[16];
    int valid = decode_chunk(cg, g, lane, k8, stage, ctl);
    valid = min(valid, decode_chunk(cv, g, lane, v, stage, ctl));
#pragma unroll
    for (int k = 0; k < 16; k++) {
      if (16 * lane + k < valid) {
        if (k8[k] < G) {
          if (local) atomicAdd(hist + k8[k], (unsigned long long)v[k]);
          else atomicAdd(reinterpret_cast<unsigned long long*>(sums) + k8[k], (unsigned long long)v[k]);
        } else {
          set_error(ctl, MS_ERR_OUT_OF_RANGE, k8[k]);
        }
      }
    }
  }
  if (!local) return;
  __syncthreads();
  for (uint64_t k = threadIdx.x; k < G; k += blockDim.x)
    if (hist[k]) atomicAdd(reinterpret_cast<unsigned long long*>(sums) + k, hist[k]);
}

// Semi-join build side: set bit key for every key of the build column.
__global__ void __launch_bounds__(kThreads) k_build_keys(const DevMeta* keys, uint64_t domain, uint32_t* bits,
                                                          DevCtl* ctl) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint16_t* stage = reinterpret_cast<uint16_t*>(smem_raw) + warp * 2048;
  const ColView c = view_of(keys);
  const uint64_t nch = (c.n + kBlock - 1) / kBlock, ntiles = (nch + kWarps - 1) / kWarps;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    uint64_t v[16];
    const int valid = decode_chunk(c, tile * kWarps + warp, lane, v, stage, ctl);
#pragma unroll
    for (int k = 0; k < 16; k++) {
      if (16 * lane + k < valid) {
        if (v[k] < domain) atomicOr(bits + (v[k] >> 5), 1u << (v[k] & 31));
        else set_error(ctl, MS_ERR_OUT_OF_RANGE, v[k]);
      }
    }
  }
}

#endif  // MS_PRODUCE_ONLY

}  // namespace ms
