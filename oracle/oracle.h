/*
 * oracle.h -- plain, slow, single-threaded CPU oracle for the compression-enabled
 * processing model of MorphStore (Damme et al., VLDB 2020).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load
 * this code: only the test-suite, the smoke check and the bench's CPU-baseline
 * leg use it.  It shares no code, header, table or constant with the CUDA
 * library; both sides follow the same written format definitions.
 *
 * Everything here is integer arithmetic on unsigned 64-bit values; sums and
 * products wrap modulo 2^64.
 *
 * Formats (Sec. 4 "Column Storage"; Sec. 2.1 "Techniques"/"Algorithms"):
 *   0 UNCOMPR   raw little-endian uint64 values.
 *   1 STATIC_BP all values packed at one caller-chosen width b in [1,64]
 *               ("one block and fixed bit width").  No remainder.
 *   2 DYN_BP    512-value blocks, each packed at the effective bit width of its
 *               largest value (SIMD-BP512); n mod 512 values stay uncompressed.
 *   3 DELTA_BP  DELTA (difference to the predecessor) cascaded with DYN_BP.
 *   4 FOR_BP    FOR (difference to a reference value) cascaded with DYN_BP.
 *   5 RLE       run-length encoding: every run of equal consecutive values is
 *               recorded once, with the position where it ends.
 *   6 FOR_STATIC_BP    FOR cascaded with static BP: FOR_BP's layout with every
 *               block's residuals packed at the one caller-chosen width b.
 *   7 DELTA_STATIC_BP  DELTA cascaded with static BP, likewise.
 * The bit layout is not printed in the paper; the reading used here is spelled
 * out in oracle.c's header comment and is the one the CUDA library implements.
 */
#ifndef MS_ORACLE_H
#define MS_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* oracle status codes (its own numbering) */
enum { ORC_OK = 0, ORC_BAD_ARG = 1, ORC_BAD_FORMAT = 2, ORC_TOO_WIDE = 3,
       ORC_OUT_OF_RANGE = 4 };

enum { ORC_UNCOMPR = 0, ORC_STATIC_BP = 1, ORC_DYN_BP = 2, ORC_DELTA_BP = 3,
       ORC_FOR_BP = 4, ORC_RLE = 5, ORC_FOR_STATIC_BP = 6, ORC_DELTA_STATIC_BP = 7 };

enum { ORC_EQ = 0, ORC_NE = 1, ORC_LT = 2, ORC_LE = 3, ORC_GT = 4, ORC_GE = 5,
       ORC_BETWEEN = 6 };

enum { ORC_ADD = 0, ORC_SUB = 1, ORC_MUL = 2 };

/* effective bit width: number of significant bits, 0 for the value 0 */
int orc_bitwidth(uint64_t x);

/* physical size in bytes of x[0..n) stored in format fmt (bw used by STATIC_BP) */
uint64_t orc_size(int fmt, int bw, const uint64_t *x, uint64_t n);

/* writes exactly orc_size(...) bytes into out (cap bytes available) */
int orc_compress(int fmt, int bw, const uint64_t *x, uint64_t n, uint8_t *out,
                 uint64_t cap, uint64_t *size_out);

/* reads a column of n logical values from buf (size bytes) into out[0..n) */
int orc_decompress(int fmt, int bw, uint64_t n, const uint8_t *buf, uint64_t size,
                   uint64_t *out);

/* per-block widths of a DYN/DELTA/FOR column (nb = n/512 entries) */
void orc_block_widths(int fmt, const uint64_t *x, uint64_t n, uint8_t *widths);

/* ---- operators on uncompressed columns ---- */
int orc_select(const uint64_t *x, uint64_t n, int cmp, uint64_t c1, uint64_t c2,
               uint64_t *pos, uint64_t *m_out);
int orc_project(const uint64_t *d, uint64_t nd, const uint64_t *pos, uint64_t m,
                uint64_t *out);
int orc_calc(int op, const uint64_t *a, const uint64_t *b, uint64_t c, uint64_t n,
             uint64_t *out);
uint64_t orc_agg_sum(const uint64_t *x, uint64_t n);
int orc_group_sum(const uint64_t *g, const uint64_t *v, uint64_t n, uint64_t G,
                  uint64_t *sums);
int orc_semijoin(const uint64_t *probe, uint64_t n, const uint64_t *keys,
                 uint64_t nk, uint64_t key_domain, uint64_t *pos, uint64_t *m_out);

#ifdef __cplusplus
}
#endif
#endif
