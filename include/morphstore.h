/*
 * morphstore.h -- C ABI of libms, a GB300 (sm_103a) implementation of the
 * compression-enabled processing model of MorphStore (Damme et al., VLDB 2020,
 * arXiv 2004.09350).
 *
 * Model (Sec. 3, Sec. 4).  Base data, intermediates and results are columns of
 * unsigned 64-bit integers.  Every column is stored in exactly one format
 * ("Foundations", Sec. 3.1; "Column Storage", Sec. 4.1).  Operators follow the
 * operator-at-a-time model: each runs to completion and materialises its output
 * column.  Each operator takes the formats of its inputs from the columns and a
 * caller-chosen output format.  It decompresses input blocks on the fly, runs its
 * core on the uncompressed values in registers, and recompresses the output
 * block by block.  This is the "on-the-fly de/re-compression" degree of Sec. 3.2,
 * fused into one kernel per operator.  No uncompressed intermediate is written
 * to device memory.
 *
 * Formats and byte layout (Sec. 2.1 techniques; Sec. 4.1 main part of 512-value
 * blocks plus an uncompressed remainder behind it):
 *   bw(x)        number of significant bits of x; bw(0) = 0.
 *   block        512 consecutive values.  Value i of a block is value k = i%16 of
 *                lane j = i/16.  Lane j's 16 values are packed LSB-first at b bits:
 *                value k sits at stream bits [k*b, k*b+b).  Stream halfword q of
 *                lane j is stored at payload halfword 32*q + j.  A block of width b
 *                therefore takes 64*b bytes.
 *   MS_UNCOMPR   n raw little-endian uint64 values; size 8n.
 *   MS_STATIC_BP every full 512-value chunk is packed as a block at the fixed
 *                width b (chunk c at byte 64*b*c).  The n%512 tail values follow,
 *                packed LSB-first one after the other, padded to whole words.
 *                size = ceil(n*b/64)*8.  Random access needs no directory.
 *   MS_DYN_BP    header of n/512 entries {(payload word offset << 8) | b_k, ref_k},
 *                then the block payloads, then the n%512 remainder values as raw
 *                uint64.  b_k = bw(max residual), residual = value, ref = 0
 *                (SIMD-BP512, Sec. 4.1).
 *   MS_DELTA_BP  as DYN_BP with residual_0 = 0, residual_i = x_i - x_{i-1}
 *                (mod 2^64), ref = the block's first value.  DELTA is the
 *                difference to the predecessor, restarted at every block.
 *   MS_FOR_BP    as DYN_BP with residual = x - ref, ref = the block minimum.  FOR
 *                is the difference to a reference value.
 *   MS_RLE       run-length encoding (Sec. 2.1: a run of equal consecutive
 *                values is stored once, with its repetition).  R runs; the
 *                repetition is recorded as the position where the run ends:
 *                R run values (uint64), then R run ends (uint64, exclusive; the
 *                last is n), then a directory of ceil(n/512) uint64 entries, entry
 *                g = the run that holds value 512*g, so that a block's runs are
 *                found without a search (random access, Sec. 4.2).
 *                size = 16*R + 8*ceil(n/512); n_blocks (ms_column_meta) = R.
 *                Produced by ms_compress and ms_morph only; read by every
 *                operator but ms_select_packed and the batched fragments (which
 *                return MS_ERR_FORMAT for it at once).  Other operators with
 *                out_fmt MS_RLE return MS_ERR_FORMAT at once: morph their output.
 *   MS_FOR_STATIC_BP, MS_DELTA_STATIC_BP
 *                FOR and DELTA cascaded with static BP (Sec. 2.1 cascades; static
 *                BP's "one fixed bit width" for the residuals): the byte layout of
 *                MS_FOR_BP / MS_DELTA_BP with every block packed at the caller's
 *                static_bw (1..64), so block k's payload sits at word 8*b*k.  A
 *                residual wider than static_bw raises MS_ERR_VALUE_TOO_WIDE
 *                (device).  Every operator reads them as it reads MS_FOR_BP /
 *                MS_DELTA_BP; ms_compress_noalloc does not write them.
 *   A column buffer starts on a 256-byte boundary.  The header is 16 bytes per
 *   block, so every block payload starts on a 64-byte boundary.
 *
 * Memory and ownership.  A context owns an arena of device memory.  Operator
 * outputs are carved from it at a device-side top-of-arena offset.  The
 * output's size is therefore decided on the GPU and the host never waits for
 * it.  Column metadata (length, size, ...) lives in device memory.
 * ms_column_info() is the one call that copies it to the host, and it
 * synchronises the stream.  Arena columns are released in LIFO order: freeing a
 * column that is not the most recent one only marks it, and its space comes
 * back when every column allocated after it is freed too.  A block-format
 * output (dynamic BP, DELTA+BP, FOR+BP) is first encoded into a stage taken
 * from the arena's free end and then placed behind its block headers at the
 * top, so while its operator runs it needs room for its payload twice; an output
 * that does not fit is published empty and MS_ERR_NOMEM is raised.  Imported
 * columns are allocated with the context's allocator callbacks (cudaMalloc when
 * none are given).
 *
 * Streams and errors.  Operators are asynchronous on the given stream.
 * `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 * stream.  Operators on one context must be ordered on one stream.
 * Host-detectable errors (NULL pointers, unknown formats, static_bw outside
 * 1..64) return immediately with nothing enqueued.  Device-detected errors are
 * stored in a sticky device error word: a value too wide for static BP, a
 * position >= n, a group id >= G, a corrupt header, a length mismatch, arena
 * exhaustion, or a bounded spin running out.  The next ms_get_error() returns
 * that word and clears it.  After a device error the outputs are unspecified
 * but every write stayed in bounds.  No exception crosses this interface.
 *
 * Final query results are uncompressed (Sec. 3.3).  They come out through
 * ms_decompress, ms_agg_sum or ms_group_sum into caller-owned device memory.
 */
#ifndef MORPHSTORE_H
#define MORPHSTORE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MS_UNCOMPR = 0,
  MS_STATIC_BP = 1,
  MS_DYN_BP = 2,
  MS_DELTA_BP = 3,
  MS_FOR_BP = 4,
  MS_RLE = 5,
  MS_FOR_STATIC_BP = 6,
  MS_DELTA_STATIC_BP = 7
} ms_fmt;

typedef enum {
  MS_OK = 0,
  MS_ERR_INVALID_ARG = 1,
  MS_ERR_FORMAT = 2,
  MS_ERR_VALUE_TOO_WIDE = 3,
  MS_ERR_OUT_OF_RANGE = 4,
  MS_ERR_NOMEM = 5,
  MS_ERR_TIMEOUT = 6,
  MS_ERR_CUDA = 7
} ms_status;

/* select predicates against constants (Sec. 5.1 uses a point predicate) */
typedef enum {
  MS_EQ = 0, MS_NE = 1, MS_LT = 2, MS_LE = 3, MS_GT = 4, MS_GE = 5,
  MS_BETWEEN = 6 /* c1 <= x <= c2 */
} ms_cmp;

typedef enum { MS_ADD = 0, MS_SUB = 1, MS_MUL = 2 } ms_arith;

typedef struct ms_ctx ms_ctx;
typedef struct ms_column ms_column;

/* Allocator callbacks.  Must return device memory that is at least 256-byte
   aligned, or NULL on failure. */
typedef void *(*ms_alloc_fn)(size_t bytes, void *user);
typedef void (*ms_free_fn)(void *ptr, void *user);

/* Host copy of a column's metadata (filled by ms_column_info). */
typedef struct {
  uint64_t n;             /* logical values */
  int32_t fmt;            /* ms_fmt */
  int32_t static_bw;      /* width of MS_STATIC_BP, else 0 */
  uint64_t size_bytes;    /* physical size (the paper's footprint measure, Sec. 5) */
  uint64_t n_blocks;      /* 512-value blocks in the main part (block formats) */
  uint64_t payload_words; /* packed payload size in uint64 words (block formats) */
  uint64_t device_ptr;    /* device address of the column buffer */
} ms_column_meta;

/* ---------------------------------------------------------------- context */

/* Creates a context on `device`.  The context owns an arena of `arena_bytes`
   for operator outputs and scratch space for columns of up to `max_rows`
   values.  Scratch grows on demand for longer columns; growing synchronises the
   device.  alloc/free may be NULL, which means cudaMalloc/cudaFree.
   Errors: MS_ERR_INVALID_ARG, MS_ERR_NOMEM, MS_ERR_CUDA. */
ms_status ms_ctx_create(ms_ctx **out, int device, uint64_t arena_bytes,
                        uint64_t max_rows, ms_alloc_fn alloc, ms_free_fn free_fn,
                        void *user);
/* Synchronises the device, frees every column and the context's memory. */
ms_status ms_ctx_destroy(ms_ctx *ctx);

/* Reads and clears the sticky device error word; synchronises `stream`. */
ms_status ms_get_error(ms_ctx *ctx, void *stream);
/* Details of the last device error (an offending index or value), 0 if none;
   valid after ms_get_error returned an error. */
uint64_t ms_last_error_info(ms_ctx *ctx);

/* The cudaError_t of the last CUDA call that made an entry point return
   MS_ERR_CUDA (0 if none), and its description. */
int ms_last_cuda_error(void);
const char *ms_cuda_error_string(int code);

/* Arena bytes in use (current) and the high-water mark since the last reset;
   both synchronise `stream`.  The high-water mark is the peak footprint of the
   operator outputs, the transient stage of a block-format output included. */
ms_status ms_arena_usage(ms_ctx *ctx, uint64_t *in_use, uint64_t *high_water,
                         void *stream);
ms_status ms_arena_reset_high_water(ms_ctx *ctx, void *stream);
/* Bytes of the context's work area: the scratch its operators carve for
   look-back status words, match bitmaps, per-chunk offsets, per-block stage
   records (about 0.2 bytes per row in all) and key bitmaps.  It
   is allocated on demand and grows with the longest column seen; together with
   the arena's high-water mark it is the device memory a plan needs beyond its
   base columns.  0 for a NULL context.  No synchronisation. */
uint64_t ms_work_bytes(const ms_ctx *ctx);

/* ---------------------------------------------------------------- columns */

/* Copies n values' worth of bytes in `fmt` (layout above) from `src` (host or
   device memory, `size` bytes) into a new column allocated with the allocator
   callbacks.  The header chain of block formats is checked on the device
   (MS_ERR_FORMAT).  `static_bw` is used by MS_STATIC_BP only. */
ms_status ms_column_import(ms_ctx *ctx, int fmt, int static_bw, uint64_t n,
                           const void *src, uint64_t size, ms_column **out,
                           void *stream);
/* Copies the column's bytes to `dst` (host or device, `cap` bytes) and returns
   the size; synchronises `stream`.  MS_ERR_INVALID_ARG if cap is too small. */
ms_status ms_column_export(ms_ctx *ctx, const ms_column *col, void *dst, uint64_t cap,
                           uint64_t *size_out, void *stream);
/* Copies the column's metadata to the host; synchronises `stream`. */
ms_status ms_column_info(ms_ctx *ctx, const ms_column *col, ms_column_meta *out,
                         void *stream);
/* Upper bound on the column's length known on the host without a sync. */
uint64_t ms_column_max_rows(const ms_column *col);
/* Releases a column (LIFO for arena columns, see above).  Enqueued on `stream`. */
ms_status ms_column_free(ms_ctx *ctx, ms_column *col, void *stream);

/* -------------------------------------------------------------- operators */

/* compress (Sec. 4.1): n uncompressed values at device address d_in (16-byte
   aligned) -> new column in `fmt` (any format, MS_RLE included).
   MS_ERR_VALUE_TOO_WIDE (device) if a value needs more than static_bw bits under
   MS_STATIC_BP, or a residual under MS_FOR_STATIC_BP / MS_DELTA_STATIC_BP. */
ms_status ms_compress(ms_ctx *ctx, const uint64_t *d_in, uint64_t n, int fmt,
                      int static_bw, ms_column **out, void *stream);

/* decompress: column -> uncompressed values at d_out (16-byte aligned, room for
   `cap` values).  MS_ERR_INVALID_ARG (device) if the column holds more than cap
   values; nothing past cap is written. */
ms_status ms_decompress(ms_ctx *ctx, const ms_column *col, uint64_t *d_out,
                        uint64_t cap, void *stream);

/* specialized select (Sec. 3.2, "Specialized Operators"): the positions ms_select
   returns, computed on the compressed representation.  Only for inputs in
   MS_DYN_BP, MS_FOR_BP, MS_DELTA_BP or MS_STATIC_BP (MS_ERR_FORMAT otherwise, at
   once).  A block whose header bounds its values wholly inside or outside the
   predicate's range is decided from its 16-byte header without reading or
   decoding its payload; the others are compared in the residual domain as they
   are unpacked (the predicate is shifted by the block's reference once, so FOR
   and DELTA references are never added back, and b <= 32 compares in 32 bits). */
ms_status ms_select_packed(ms_ctx *ctx, const ms_column *in, int cmp, uint64_t c1,
                           uint64_t c2, int out_fmt, int out_static_bw, ms_column **out,
                           void *stream);

/* morph (Sec. 3.2, "On-the-Fly Morphing"): the column's values as a new column in
   out_fmt, with no uncompressed intermediate in device memory.  Each 512-value
   block is decoded into registers and re-encoded in out_fmt by the same warp (a
   direct morphing algorithm for every ordered pair of the five block and
   fixed-width formats: n^2 - n = 20 of them, and the identity; the static
   cascades likewise).  Into MS_RLE the column is decoded twice, block by block:
   once to count the runs of every block, once to write them (sizes from a scan of
   the counts).  MS_ERR_VALUE_TOO_WIDE (device) for a value or residual wider than
   out_static_bw under MS_STATIC_BP, MS_FOR_STATIC_BP or MS_DELTA_STATIC_BP. */
ms_status ms_morph(ms_ctx *ctx, const ms_column *col, int out_fmt, int out_static_bw,
                   ms_column **out, void *stream);

/* select (Sec. 5.1 "Single Operator"): ascending 0-based positions i with
   x_i <cmp> c1 (MS_BETWEEN: c1 <= x_i <= c2), as a new column in out_fmt. */
ms_status ms_select(ms_ctx *ctx, const ms_column *in, int cmp, uint64_t c1,
                    uint64_t c2, int out_fmt, int out_static_bw, ms_column **out,
                    void *stream);

/* project (Sec. 4.2, random read access): out_j = data[pos_j].  Any data format
   is accepted; random access into the block formats goes through the block
   header, which doubles as a directory.  MS_ERR_OUT_OF_RANGE (device) for
   pos_j >= n(data). */
ms_status ms_project(ms_ctx *ctx, const ms_column *data, const ms_column *pos,
                     int out_fmt, int out_static_bw, ms_column **out, void *stream);

/* calc: out_i = a_i <op> b_i modulo 2^64, or a_i <op> c when b is NULL.
   MS_ERR_INVALID_ARG (device) if n(a) != n(b); the output then has min(n(a),
   n(b)) values. */
ms_status ms_calc(ms_ctx *ctx, int op, const ms_column *a, const ms_column *b,
                  uint64_t c, int out_fmt, int out_static_bw, ms_column **out,
                  void *stream);

/* sum (Sec. 5.1 "Simple Query"): *d_result = sum of all values modulo 2^64
   (0 for an empty column).  d_result is caller-owned device memory.  An MS_RLE
   column is summed on its runs (value x run length), without expanding them. */
ms_status ms_agg_sum(ms_ctx *ctx, const ms_column *in, uint64_t *d_result,
                     void *stream);

/* grouped sum (Sec. 4.2: random writes go to an uncompressed result):
   d_sums[k] = sum of val_i over gid_i == k, for k < n_groups, modulo 2^64.
   d_sums (n_groups values) is caller-owned and is overwritten.
   MS_ERR_OUT_OF_RANGE (device) for gid_i >= n_groups. */
ms_status ms_group_sum(ms_ctx *ctx, const ms_column *gid, const ms_column *val,
                       uint64_t n_groups, uint64_t *d_sums, void *stream);

/* semi-join: ascending positions i with probe_i in the set of build_keys, as a
   new column in out_fmt.  Keys index a dimension of `key_domain` rows;
   MS_ERR_OUT_OF_RANGE (device) for a key >= key_domain.  Probe values >=
   key_domain simply do not match.  Duplicate keys are allowed. */
ms_status ms_semijoin(ms_ctx *ctx, const ms_column *probe, const ms_column *build_keys,
                      uint64_t key_domain, int out_fmt, int out_static_bw,
                      ms_column **out, void *stream);

/* ------------------------------------------------------- no-allocation use */

/* Largest column ms_compress_noalloc accepts (16 Mi values). */
#define MS_NOALLOC_MAX_ROWS (1ull << 24)

/* Compression for callers that cannot allocate device memory.  The paper has no
   counterpart: this serves embedding hosts.  Some callers cannot call cudaMalloc:
   a memory manager compressing a buffer while it serves an allocation request
   (it must not re-enter the allocator), a host whose device memory is all handed
   out by its own pool, or a latency-critical path that cannot take the implicit
   synchronisation a driver allocation may cause.
   It does what ms_compress does for the n uncompressed values at d_in (16-byte
   aligned).  It writes the column's bytes, in the layout above, to d_out
   (16-byte aligned, out_cap bytes) instead of a context's arena.  d_result
   (device, 2 uint64 words) receives the column's size in bytes and the device
   status (an ms_status: MS_ERR_NOMEM if out_cap is too small,
   MS_ERR_VALUE_TOO_WIDE for static BP).  Neither this call nor anything it
   starts allocates: its scratch (look-back status words and a control block,
   about 33 KB) is a fixed device array in the library.  n above
   MS_NOALLOC_MAX_ROWS is rejected with MS_ERR_INVALID_ARG.
   The first call on a device (with that device current) looks the array's
   device address up, sets the kernel's attributes and caches both; this set-up
   runs once per device even when several host threads make their first call
   together.  Make that first call before any stream capture.  Every call shares the array: calls that
   overlap on the GPU (different streams or host threads) race and must be
   serialised by the caller.  No context is needed.  Asynchronous on `stream`. */
ms_status ms_compress_noalloc(const uint64_t *d_in, uint64_t n, int fmt, int static_bw,
                              void *d_out, uint64_t out_cap, uint64_t *d_result,
                              void *stream);

/* ------------------------------------------------------ format selector */

/* The paper chooses formats with a gray-box cost model (Sec. 5.2, "Determining a
   good format combination") that it does not print.  This library learns one
   instead.  A small MLP maps 16 statistics of an intermediate to the predicted
   log2 bytes per value and log2 nanoseconds per value of each of the five formats
   (outputs 0..4: size, 5..9: time, in ms_fmt order).  Labels come from the engine
   itself, by compressing every intermediate into every format (the exhaustive
   try-all choice, against which the selector's regret is measured).

   Network: 16 -> 64 -> 64 -> 10, ReLU between layers, fp32.  Parameters are
   one packed array: W1[16][64], b1[64], W2[64][64], b2[64], W3[64][10], b3[10],
   row-major with the input index first (MS_MLP_PARAMS floats). */
#define MS_MLP_PARAMS 5898

/* y[n][10] = MLP(x[n][16]) (all device memory). */
ms_status ms_mlp_forward(const float *d_params, const float *d_x, uint64_t n, float *d_y,
                         void *stream);
/* Loss L = inv_count * sum over samples r and outputs o of mask[r][o] *
   (y_hat[r][o] - y[r][o])^2, and its gradient dL/dparams into d_grad
   (MS_MLP_PARAMS floats) and L into *d_loss.  d_partials is caller scratch of
   partials_floats floats (at least MS_MLP_PARAMS + 1).  More scratch lets more
   CTAs share the samples.  The result is deterministic: partial gradients are
   summed in a fixed order. */
ms_status ms_mlp_loss_grad(const float *d_params, const float *d_x, const float *d_y,
                           const float *d_mask, uint64_t n, float inv_count, float *d_grad,
                           float *d_loss, float *d_partials, uint64_t partials_floats,
                           void *stream);
/* One Adam step (Kingma & Ba 2015) on d_params with moments d_m, d_v; step >= 1. */
ms_status ms_mlp_adam(float *d_params, const float *d_grad, float *d_m, float *d_v, uint64_t step,
                      float lr, float beta1, float beta2, float eps, void *stream);

/* Statistics of a column, one decoding pass, into d_stats (MS_STATS_WORDS device
   words, overwritten).  For 512-value chunks (the last may be partial):
   [0] n, [1] maximum value, [2] chunks, [3] sum of bw(max - min) per chunk,
   [4] sum of bw(largest difference to the predecessor) per chunk,
   [5] pairs with x_i >= x_{i-1} inside chunks, [6] pairs with x_i != x_{i-1}
   inside chunks, [8 + b] chunks whose maximum has bit width b (b = 0..64). */
#define MS_STATS_WORDS 80
ms_status ms_column_stats(ms_ctx *ctx, const ms_column *col, uint64_t *d_stats, void *stream);

/* ----------------------------------------------------- batched fragments */

/* Many small queries in one launch.  The paper runs one query at a time.  Serving
   thousands of short query fragments over columns of uneven length one launch
   each leaves the GPU idle between launches, so a batch runs them all in one
   persistent kernel.

   Fragment f is the Sec. 5.1 "Simple Query" shape select -> project -> agg_sum
   over two columns x_f and y_f of equal length:
       sum_f = sum of y_f[i] over the rows i with x_f[i] <cmp_f> c1_f (c2_f),
   modulo 2^64.  This is the value of ms_select(x_f) -> ms_project(y_f, positions)
   -> ms_agg_sum.  The select's positions inside one 512-row chunk of x index the
   same chunk of y.  So the three operators fuse per chunk: decode the chunk of x,
   test the predicate, decode the chunk of y, and add the matching values.  Sums
   modulo 2^64 do not depend on the order of the additions, so every
   configuration gives the same bits.

   The batch numbers the chunks of all fragments consecutively (fragment f owns
   chunks cs[f] .. cs[f+1]-1) and cuts them into tiles of `tile_chunks` chunks.
   Tiles go to warps from a device work counter (the last CTA resets it, so a
   run needs no set-up launch) or round-robin to CTAs.  Each warp keeps `depth`
   chunks of both columns in flight with asynchronous copies. */
typedef struct ms_batch ms_batch;
typedef struct ms_graph ms_graph;

typedef struct {
  uint32_t warps;       /* warps per CTA */
  uint32_t depth;       /* chunks in flight per warp */
  uint32_t tile_chunks; /* chunks per tile: a power of two in 8..1024, at least
                           2*depth (schedule 0) or warps (schedule 1) */
  uint32_t ctas_per_sm; /* CTAs per SM, 0 = as many as fit */
  uint32_t compact;     /* 1: one decoding loop for every width (small code);
                           0: width-specialised decoders */
  uint32_t schedule;    /* 0: each warp takes whole tiles from the work counter;
                           1: CTA b takes tiles b, b + grid, ... and its warps
                           share each tile (one fragment per CTA at a time);
                           2: CTA b takes 64-chunk claims b, b + grid, ... and
                           copies runs of one fragment's chunks into two
                           shared buffers of 8 KB x depth per column, which
                           its warps decode (tile_chunks is not used) */
} ms_batch_config;
/* Supported (warps, depth, compact, schedule): schedule 0 with warps 4 or 8,
   depth 2..4, either decoder; schedule 1 with warps 4, 8 (depth 2 or 3) or 16
   (depth 2) and the width-specialised decoders; schedule 2 with warps 8, depth
   2..4 and the width-specialised decoders. */

/* ms_batch_run flags */
#define MS_BATCH_ZERO 1u         /* zero d_sums[f0..f1) first (one memset) */
#define MS_BATCH_PER_FRAGMENT 2u /* one launch per fragment instead of one in all */

/* Binds n_frags fragments: x[f], y[f] (columns of ctx, equal lengths), cmp[f]
   (ms_cmp) and c1[f], c2[f] (c2 is used by MS_BETWEEN only; c2 may be NULL).
   Host arrays.  Reads the columns' device metadata and synchronises `stream`.
   The columns must outlive the batch and must not be freed before it.
   Errors: MS_ERR_INVALID_ARG (NULL pointers, n_frags == 0, a foreign or freed
   column, an unknown cmp, x and y of unequal length, 2^31 chunks or more),
   MS_ERR_FORMAT (a column in MS_RLE or a static cascade: the batch kernels take
   the five base formats), MS_ERR_NOMEM, MS_ERR_CUDA. */
ms_status ms_batch_create(ms_ctx *ctx, uint32_t n_frags, ms_column *const *x,
                          ms_column *const *y, const int32_t *cmp, const uint64_t *c1,
                          const uint64_t *c2, ms_batch **out, void *stream);
/* Totals over the fragments: rows (of x), 512-row chunks, and compressed bytes of
   the x and y columns (the bytes a run reads).  Any pointer may be NULL. */
ms_status ms_batch_info(const ms_batch *b, uint64_t *rows, uint64_t *chunks,
                        uint64_t *bytes);
/* Computes fragments f0 .. f1-1 (f0 <= f1 <= n_frags) into d_sums[f] (device
   memory with n_frags words, indexed by fragment; other entries untouched).
   Without MS_BATCH_ZERO the sums are added to d_sums.  cfg NULL means the
   default configuration {8, 2, 32, 0, 0, 1}; MS_ERR_INVALID_ARG for an
   unsupported configuration (including one whose shared memory does not fit).  Asynchronous on `stream`; runs of one batch share
   its work counter and must be ordered on one stream.  Allocates nothing and does
   not synchronise, so it can be captured in a CUDA graph. */
ms_status ms_batch_run(ms_batch *b, uint32_t f0, uint32_t f1, const ms_batch_config *cfg,
                       uint32_t flags, uint64_t *d_sums, void *stream);
/* Captures ms_batch_run(b, f0, f1, cfg, flags, d_sums) into an instantiated CUDA
   graph (on a private stream).  The graph replays it with ms_graph_launch. */
ms_status ms_batch_graph(ms_batch *b, uint32_t f0, uint32_t f1, const ms_batch_config *cfg,
                         uint32_t flags, uint64_t *d_sums, ms_graph **out);
ms_status ms_graph_launch(ms_graph *g, void *stream);
ms_status ms_graph_destroy(ms_graph *g);
ms_status ms_batch_destroy(ms_batch *b);

/* ------------------------------------------------------------- self-test */

/* Failure-detection self-test: one bounded device-side wait that nothing ever
   satisfies (a look-back whose predecessor tile never publishes).  The wait gives
   up after its iteration limit (about 2^20 polls with back-off), records
   MS_ERR_TIMEOUT in the device error word and returns.  Nothing faults or traps;
   the context stays usable, and the next ms_get_error returns MS_ERR_TIMEOUT.
   Uses the context's scratch; asynchronous on `stream`. */
ms_status ms_selftest_wait_timeout(ms_ctx *ctx, void *stream);

/* ------------------------------------------------------------ profiling */

/* Kernels of the library, as reported by ms_profile_collect. */
typedef enum {
  MS_K_MARK = 0,       /* select / semi-join: decode + predicate -> match bitmap */
  MS_K_EMIT = 1,       /* select / semi-join: match bitmap -> positions column */
  MS_K_COMPRESS = 2,
  MS_K_DECOMPRESS = 3,
  MS_K_PROJECT = 4,
  MS_K_CALC = 5,
  MS_K_AGG_SUM = 6,
  MS_K_GROUP_SUM = 7,
  MS_K_BUILD_KEYS = 8, /* semi-join build side */
  MS_K_VALIDATE = 9,   /* header check of imported columns */
  MS_K_SCAN = 10,      /* select / semi-join: exclusive scan of per-chunk match counts */
  MS_K_PLACE = 11,      /* block-format outputs: payload offsets, headers and payload copy */
  MS_K_STATS = 12,      /* column statistics for the format selector */
  MS_K_BATCH = 13,      /* batched select -> project -> agg_sum fragments */
  MS_K_SELECT_PACKED = 14, /* specialized select on packed codes -> match bitmap */
  MS_K_ARENA = 15,      /* arena bookkeeping: top reset after ms_column_free, metadata writes */
  MS_K_RLE = 16,        /* RLE encoding: run heads per block, their scan, run records */
  MS_K_COUNT = 17
} ms_kernel;

typedef struct {
  int32_t kernel;    /* ms_kernel */
  uint32_t launches; /* launches recorded since the last collect */
  double total_ms;   /* summed device time between the events around each launch */
} ms_kernel_time;

/* When on, every kernel launch is bracketed by two CUDA events on its stream. */
ms_status ms_profile_enable(ms_ctx *ctx, int on);
/* Synchronises the device, sums the recorded launches per kernel into out[0..*n_out)
   (at most `max` entries, kernels without launches omitted) and clears the record. */
ms_status ms_profile_collect(ms_ctx *ctx, ms_kernel_time *out, int max, int *n_out);
/* Static name of a kernel id ("mark", "emit", ...), "?" when unknown. */
const char *ms_kernel_name(int kernel);

#ifdef __cplusplus
}
#endif
#endif /* MORPHSTORE_H */
