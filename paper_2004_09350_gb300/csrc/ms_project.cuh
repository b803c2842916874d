// ms_project.cuh -- project (Sec. 4.2, random read access by sorted positions) from
// DYN / FOR / static-BP data: the span-streaming gather.
//
// A CTA takes a tile of 8 consecutive output chunks (4096 positions).  When the
// tile's positions are sorted, the data blocks they touch are listed once, their
// payloads are cut into pieces of at most kSpanPiece bytes, and the pieces stream
// through a two-slot ring in shared memory: one thread hands each run of touched
// blocks that are contiguous in device memory to the bulk-copy engine
// (cp.async.bulk, completion on the slot's mbarrier), and while the next piece
// lands, all 256 threads cut the values of the current piece's positions out of
// shared memory, position i by thread i mod 256 (the positions of a piece are a
// contiguous index range).  Untouched blocks are never read, and each touched
// block is read once, whole and coalesced.  Values go to the warps' 4 KB buffers at
// their output index; each warp then encodes its chunk (store_staged).  Unsorted
// or out-of-range positions, tiles whose positions lie more than 2^32 rows apart
// and tiles that touch more than kSpanTouch blocks are gathered in place instead
// (project_direct).  About 112 KB of shared memory: two CTAs per SM, so one CTA's
// tile set-up overlaps the other's streaming.
#pragma once

#include "ms_kernels.cuh"

namespace ms {

constexpr int kSpanPiece = 15360;               // bytes per ring slot
constexpr int kSpanPack = kSpanPiece - 4096;    // a piece starts a new block below this fill
constexpr int kSpanSlots = 2;
constexpr int kSpanTouch = 1024;                // touched data blocks per tile, at most
constexpr uint32_t kRemBlock = 0xffu;           // width tag of a block past the packed part

// 16-byte aligned size: the per-warp buffers behind it take 16-byte accesses
struct alignas(16) SpanCta {
  uint8_t slot[kSpanSlots][kSpanPiece];
  uint64_t ref[kSpanTouch];         // reference of each touched block (FOR), else 0
  uint32_t info[kSpanTouch];        // (halfword offset of the block in its slot << 8) | width
  uint32_t tb[kSpanTouch];          // touched block, relative to the tile's first block
  uint32_t goff[kSpanTouch];        // its payload offset in the column (words; bytes / 8)
  uint16_t upiece[kSpanTouch];      // its piece
  uint16_t pstart[kSpanTouch + 1];  // first touched block of each piece
  uint16_t pfirst[kSpanTouch + 1];  // first position (tile index) of each piece
  uint32_t pos[kTile];              // tile-relative positions (~0 past the tile's end)
  uint16_t tidx[kTile];             // touched-block index of each position
  uint64_t wlo[kWarps], whi[kWarps];
  uint32_t wok[kWarps], wnv[kWarps], wsum[kWarps];
  uint64_t mbar[kSpanSlots];
  uint32_t phase;                   // parity of each slot's barrier (bit s)
  uint32_t dead;                    // a wait gave up: no further copies
  uint32_t ntouch, npieces;
};

// Per-warp buffer: the position chunk's decode stage, then the chunk's values, then
// its encoded output.
struct SpanWarp {
  uint16_t buf[32 * 64];
};

constexpr size_t kSpanSmemBytes = sizeof(SpanCta) + kWarps * sizeof(SpanWarp);
static_assert(sizeof(SpanCta) % 16 == 0 && sizeof(SpanWarp) % 16 == 0, "16-byte aligned warp buffers");
static_assert(kSpanSmemBytes + 1024 <= 228 * 1024 / 2, "two CTAs per SM");

// CTA-wide exclusive scan of one value per thread (kThreads threads).  Returns the
// thread's exclusive prefix; *total receives the sum.
MS_DEV uint32_t cta_excl_scan(uint32_t x, uint32_t* wsum, uint32_t* total) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ex = warp_excl_scan32(x, lane);
  if (lane == 31) wsum[warp] = ex + x;
  __syncthreads();
  uint32_t base = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kWarps; w++) {
    const uint32_t s = wsum[w];
    base += w < warp ? s : 0;
    tot += s;
  }
  __syncthreads();
  *total = tot;
  return base + ex;
}

__global__ void __launch_bounds__(kThreads, 2) k_project_span(ProduceArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  SpanCta* cs = reinterpret_cast<SpanCta*>(smem_raw);
  SpanWarp* sw = reinterpret_cast<SpanWarp*>(smem_raw + sizeof(SpanCta));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  DevCtl* ctl = a.ctl;
  const uint64_t top = *reinterpret_cast<volatile uint64_t*>(&ctl->top);
  const uint64_t avail = ctl->cap - top;
  uint8_t* base = reinterpret_cast<uint8_t*>(ctl->arena + top);
  const ColView d = view_of(a.in0), pc = view_of(a.in1);
  const uint64_t n_out = pc.n;
  const int fmt = a.fmt, bw = a.bw;
  const bool blockfmt = is_block_fmt(fmt);
  const uint64_t nch = (n_out + kBlock - 1) / kBlock, static_chunks = n_out / kBlock;
  const uint64_t ntile = (nch + kWarps - 1) / kWarps;
  const bool stat = d.fmt == MS_STATIC_BP;
  const uint64_t nfull = stat ? d.n / kBlock : d.nb;  // data blocks with a packed payload
  const uint64_t pay0 = stat ? 0 : 16 * d.nb;         // byte offset of the payloads
  const uint64_t rem0 = stat ? 64ull * (uint64_t)d.bw * nfull : 16 * d.nb + 8 * d.pwords;
  const bool add_ref = d.fmt == MS_FOR_BP;
  uint16_t* wbuf16 = sw[warp].buf;
  uint64_t* wbuf64 = reinterpret_cast<uint64_t*>(sw[warp].buf);
  if (tid == 0) {
    for (int s = 0; s < kSpanSlots; s++) mbar_init(&cs->mbar[s], 1);
    cs->phase = 0;
    cs->dead = 0;
  }
  __syncthreads();

  for (uint64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const uint64_t g = tile * kWarps + warp;
    // ---- A. the warp's positions (lane-blocked) and the tile's summary
    uint64_t p[16];
    int valid = decode_chunk(pc, g, lane, p, wbuf16, ctl);
    const int nv = max(0, min(16, valid - 16 * lane));
    bool ok = true;
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
    const int prev_nv = __shfl_up_sync(kFull, nv, 1);
    if (lane > 0 && nv > 0 && prev_nv > 0 && prev_mx > mn) ok = false;
    const bool wok = __all_sync(kFull, ok);
    uint64_t wmx = mx, wmn = mn;
#pragma unroll
    for (int dd = 16; dd; dd >>= 1) {
      wmx = max(wmx, __shfl_xor_sync(kFull, wmx, dd));
      wmn = min(wmn, __shfl_xor_sync(kFull, wmn, dd));
    }
    if (lane == 0) {
      cs->wlo[warp] = wmn;
      cs->whi[warp] = wmx;
      cs->wok[warp] = wok;
      cs->wnv[warp] = (uint32_t)max(valid, 0);
    }
    __syncthreads();
    bool tile_ok = true, any = false;
    uint64_t lo = ~0ull, hi = 0, prev_hi = 0;
    uint32_t npos = 0;
    for (int w = 0; w < kWarps; w++) {
      tile_ok &= cs->wok[w] != 0;
      if (cs->wnv[w]) {
        if (any) tile_ok &= prev_hi <= cs->wlo[w];
        lo = min(lo, cs->wlo[w]);
        hi = max(hi, cs->whi[w]);
        prev_hi = cs->whi[w];
        npos += cs->wnv[w];
        any = true;
      }
    }
    const uint64_t B_lo = lo >> 9;
    tile_ok &= any && hi - (B_lo << 9) < 0xffffffffull;
    // ---- B. tile-relative positions, then C. the touched blocks
    uint32_t ntouch = 0;
    if (tile_ok) {
#pragma unroll
      for (int k = 0; k < 16; k++)
        cs->pos[512 * warp + 16 * lane + k] = k < nv ? (uint32_t)(p[k] - (B_lo << 9)) : ~0u;
      __syncthreads();
      // thread t: positions 16t .. 16t+15 (in tile order)
      uint32_t newb = 0;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        const int i = 16 * tid + k;
        const uint32_t r = cs->pos[i];
        const uint32_t pr = i ? cs->pos[i - 1] : ~0u;
        newb += (r != ~0u && (i == 0 || (r >> 9) != (pr >> 9))) ? 1u : 0u;
      }
      uint32_t u = cta_excl_scan(newb, cs->wsum, &ntouch);
      if (ntouch <= (uint32_t)kSpanTouch) {
#pragma unroll
        for (int k = 0; k < 16; k++) {
          const int i = 16 * tid + k;
          const uint32_t r = cs->pos[i];
          if (r == ~0u) continue;
          const uint32_t pr = i ? cs->pos[i - 1] : ~0u;
          if (i == 0 || (r >> 9) != (pr >> 9)) {
            cs->tb[u] = r >> 9;
            u++;
          }
          cs->tidx[i] = (uint16_t)(u - 1);
        }
      }
      __syncthreads();
      tile_ok = ntouch <= (uint32_t)kSpanTouch && ntouch > 0;
    }
    if (!tile_ok) {  // gather in place (also keeps the barriers of every thread in step)
      uint64_t v[16];
      project_direct(a, d, p, valid, lane, v, wbuf64);
      store_staged(a, fmt, bw, blockfmt, g, v, valid, wbuf16, base, avail, static_chunks, ctl, lane);
      __syncthreads();
      continue;
    }
    // ---- D. headers of the touched blocks, pieces
    // thread t: touched blocks 4t .. 4t+3 (ntouch <= 1024 = 4 * 256)
    uint32_t sz[4], bb[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint32_t uu = 4 * tid + q;
      sz[q] = 0;
      bb[q] = kRemBlock;
      if (uu < ntouch) {
        const uint64_t B = B_lo + cs->tb[uu];
        uint64_t off = 0, ref = 0;
        uint32_t b = kRemBlock;
        if (B < nfull) {
          if (stat) {
            b = (uint32_t)d.bw;
            off = 8ull * b * B;
            if (off > 0xffffffffull) {  // beyond the 32-bit offsets of the piece table
              set_error(ctl, MS_ERR_FORMAT, B);
              b = 0;
              off = 0;
            }
          } else {
            const bool inh = 16 * (B + 1) <= d.size;
            const ulonglong2 h = inh ? __ldg(reinterpret_cast<const ulonglong2*>(d.p) + B) : make_ulonglong2(0, 0);
            off = h.x >> 8;
            b = (uint32_t)(h.x & 255);
            ref = add_ref ? h.y : 0;
            // payloads start on 8-word boundaries; anything else is a corrupt chain
            if (!inh || b > 64 || (off & 7) || pay0 + 8 * (off + 8ull * b) > d.size || off > 0xffffffffull) {
              set_error(ctl, MS_ERR_FORMAT, B);
              b = 0;
              off = 0;
            }
          }
          sz[q] = 64 * b;
        }
        bb[q] = b;
        cs->ref[uu] = ref;
        cs->goff[uu] = (uint32_t)off;
      }
    }
    uint32_t tot;
    const uint32_t c0 = cta_excl_scan(sz[0] + sz[1] + sz[2] + sz[3], cs->wsum, &tot);
    {
      uint32_t c = c0;
#pragma unroll
      for (int q = 0; q < 4; q++) {  // piece = cumulative bytes / kSpanPack: a piece's
        const uint32_t uu = 4 * tid + q;  // blocks start below kSpanPack, end below kSpanPiece
        if (uu < ntouch) {
          cs->upiece[uu] = (uint16_t)(c / kSpanPack);
          cs->info[uu] = c;  // cumulative bytes for now
        }
        c += sz[q];
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint32_t uu = 4 * tid + q;
      if (uu < ntouch && (uu == 0 || cs->upiece[uu] != cs->upiece[uu - 1])) cs->pstart[cs->upiece[uu]] = (uint16_t)uu;
    }
    if (tid == 0) {
      cs->npieces = (uint32_t)cs->upiece[ntouch - 1] + 1;
      cs->ntouch = ntouch;
    }
    __syncthreads();
    const uint32_t npieces = cs->npieces;
    uint32_t cum_piece[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint32_t uu = 4 * tid + q;
      cum_piece[q] = uu < ntouch ? cs->info[cs->pstart[cs->upiece[uu]]] : 0;
    }
    __syncthreads();  // every start offset is read before info is overwritten
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint32_t uu = 4 * tid + q;
      if (uu < ntouch) cs->info[uu] = (((cs->info[uu] - cum_piece[q]) >> 1) << 8) | bb[q];
    }
    // the first position of each piece
#pragma unroll
    for (int k = 0; k < 16; k++) {
      const int i = 16 * tid + k;
      if (cs->pos[i] == ~0u) continue;
      const uint32_t pp = cs->upiece[cs->tidx[i]];
      if (i == 0 || pp != cs->upiece[cs->tidx[i - 1]]) cs->pfirst[pp] = (uint16_t)i;
    }
    if (tid == 0) {
      cs->pstart[npieces] = (uint16_t)ntouch;
      cs->pfirst[npieces] = (uint16_t)npos;
    }
    // every thread's generic-proxy accesses to the slots are ordered before the
    // bulk copies that refill them
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    // ---- E. stream the pieces
    auto issue = [&](uint32_t j) {  // thread 0: the piece's runs into slot j % S
      if (cs->dead) return;
      const int sl = (int)(j % kSpanSlots);
      const uint32_t u0 = cs->pstart[j], u1 = cs->pstart[j + 1];
      uint32_t bytes = 0;
      for (uint32_t uu = u0; uu < u1; uu++) bytes += 64 * min(cs->info[uu] & 255, 64u) * ((cs->info[uu] & 255) != kRemBlock);
      if (bytes == 0) return;
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_expect_tx(&cs->mbar[sl], bytes);
      uint32_t uu = u0;
      while (uu < u1) {
        const uint32_t b0 = cs->info[uu] & 255;
        if (b0 == kRemBlock || b0 == 0) {
          uu++;
          continue;
        }
        // a run: touched blocks adjacent in the column (their payloads are contiguous)
        uint32_t ue = uu + 1, run = 64 * b0;
        while (ue < u1 && cs->tb[ue] == cs->tb[ue - 1] + 1 && (cs->info[ue] & 255) != kRemBlock) {
          run += 64 * (cs->info[ue] & 255);
          ue++;
        }
        bulk_copy_g2s(cs->slot[sl] + 2 * (cs->info[uu] >> 8), d.p + pay0 + 8ull * cs->goff[uu], run, &cs->mbar[sl]);
        uu = ue;
      }
    };
    if (tid == 0)
      for (uint32_t j = 0; j < min(npieces, (uint32_t)kSpanSlots); j++) issue(j);
    for (uint32_t j = 0; j < npieces; j++) {
      const int sl = (int)(j % kSpanSlots);
      // wait for the piece (a piece of empty or remainder blocks copies nothing)
      uint32_t bytes_here = 0;
      for (uint32_t uu = cs->pstart[j]; uu < cs->pstart[j + 1]; uu++)
        bytes_here |= ((cs->info[uu] & 255) != kRemBlock && (cs->info[uu] & 255) != 0) ? 1u : 0u;
      const uint32_t par = (cs->phase >> sl) & 1u;
      if (bytes_here && !cs->dead) {
        if (!mbar_wait(&cs->mbar[sl], par)) {
          cs->dead = 1;
          if (tid == 0) set_error(ctl, MS_ERR_TIMEOUT, tile);
        }
      }
      __syncthreads();
      const bool live = !cs->dead;
      // extract the piece's positions, thread i mod 256 takes position i
      const uint16_t* s16 = reinterpret_cast<const uint16_t*>(cs->slot[sl]);
      for (uint32_t i = cs->pfirst[j] + tid; i < cs->pfirst[j + 1]; i += kThreads) {
        const uint32_t rel = cs->pos[i];
        const uint32_t uu = cs->tidx[i];
        const uint32_t inf = cs->info[uu];
        const uint32_t b = inf & 255;
        const uint32_t r = rel & 511;
        uint64_t x = 0;
        if (b == kRemBlock) {  // the raw remainder, or static BP's horizontal tail
          if (stat) {
            const uint64_t bit = (uint64_t)r * (uint64_t)d.bw;
            const int s2 = (int)(bit & 63);
            const uint64_t at = rem0 + 8 * (bit >> 6);
            uint64_t y = at + 8 <= d.size ? ldg64(d.p + at) >> s2 : 0;
            if (s2 + d.bw > 64 && at + 16 <= d.size) y |= ldg64(d.p + at + 8) << (64 - s2);
            x = y & lowmask(d.bw);
          } else {
            const uint64_t at = rem0 + 8 * (uint64_t)r;
            x = at + 8 <= d.size ? ldg64(d.p + at) : 0;
          }
        } else if (b > 0 && live) {
          // value r of a block: bits [k*b, k*b + b) of lane stream r / 16 (k = r % 16);
          // stream halfword q of lane j is block halfword 32q + j
          const uint32_t bit0 = (r & 15) * b;
          const uint32_t h0 = (inf >> 8) + 32 * (bit0 >> 4) + (r >> 4);
          const uint32_t nq = ((bit0 & 15) + b + 15) >> 4;
          uint64_t w = 0;
          uint32_t top16 = 0;
#pragma unroll
          for (int t = 0; t < 4; t++)
            if ((uint32_t)t < nq) w |= (uint64_t)s16[h0 + 32 * t] << (16 * t);
          if (nq > 4) top16 = s16[h0 + 128];
          const int sh = (int)(bit0 & 15);
          x = ((w >> sh) | (sh ? ((uint64_t)top16 << (64 - sh)) : 0)) & lowmask((int)b);
        }
        x += cs->ref[uu];
        reinterpret_cast<uint64_t*>(sw[i >> 9].buf)[swz((int)(i & 511))] = x;
      }
      // the slot is free again: order the reads before the refill, then refill
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        if (bytes_here && live) cs->phase ^= 1u << sl;
        if (j + kSpanSlots < npieces) issue(j + kSpanSlots);
      }
      __syncthreads();
    }
    // ---- F. each warp encodes its chunk
    uint64_t v[16];
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = 16 * lane + k < valid ? wbuf64[swz(16 * lane + k)] : 0;
    __syncwarp();
    store_staged(a, fmt, bw, blockfmt, g, v, valid, wbuf16, base, avail, static_chunks, ctl, lane);
    __syncthreads();  // the warp buffers and the tile state are reused by the next tile
  }
  publish_staged(a, n_out, fmt, bw, blockfmt, base, top, avail);
}

}  // namespace ms
