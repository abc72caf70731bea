/*
 * sz3o.h -- serial CPU oracle of the SZ3-Interp hot path (TEST INFRASTRUCTURE).
 *
 * This library exists only to check the CUDA implementation.  It is called by
 * the tests, by the smoke check and by the CPU-baseline leg of the benchmark;
 * the product path never links, loads or calls it.  It shares no source, header,
 * table or helper with the CUDA library: the only thing the two have in common
 * is the written stream format and the parameter block layout.
 *
 * What it computes (SZ3 paper, arXiv 2111.02925):
 *   - Alg. 1 (general compressor): per point, predict then quantize, save the
 *     quantizer's unpredictable values, Huffman-encode the codes.  The
 *     preprocessor and the lossless stage are bypassed (module bypass, Sec. 1).
 *   - Sec. 6.2 "SZ3-Interp": multilevel linear / cubic interpolation predictor
 *     with constant coefficients (no stored coefficients).
 *   - Sec. 3.2 Quantizer: linear-scaling quantizer, bins of width 2*eb, the
 *     prediction error mapped to the index of the bin holding it; errors out of
 *     range are "unpredictable" and stored raw.  recover() reverses quantize().
 *   - Sec. 3.2 Encoder: Huffman tree built greedily from the code frequencies,
 *     codebook from the tree, codes encoded with it; save/load of the tree.
 *
 * The paper gives no formulas for the interpolation, no traversal order, no
 * rounding rule and no Huffman tie-break; this oracle implements one written
 * reading of each (listed in the design notes) and the CUDA path implements the
 * same reading, so the two agree bit for bit.
 *
 * Floating point: every arithmetic step is one IEEE-754 round-to-nearest-even
 * operation in the field's own type T (float or double), which is the type the
 * paper's quantizer interface takes (quantize(T data, T pred), Appendix A.3).
 * Compiled with -O2 -ffp-contract=off -fno-fast-math.
 *
 * All functions return 0 on success or a negative SZ3O_E_* code; none aborts.
 * All pointers are host pointers owned by the caller.
 */
#ifndef SZ3O_H
#define SZ3O_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SZ3O_OK = 0,
  SZ3O_E_INVAL = -1,          /* bad dims / eb / radius / order / chunk size   */
  SZ3O_E_NONFINITE = -2,      /* NaN or Inf in the input field                 */
  SZ3O_E_ZERO_RANGE_REL = -3, /* REL bound on a field whose value range is 0   */
  SZ3O_E_CAPACITY = -4,       /* output buffer too small                       */
  SZ3O_E_CORRUPT = -5,        /* stream fails a magic/version/length check     */
  SZ3O_E_NOMEM = -7           /* host allocation failed                        */
};

enum { SZ3O_F32 = 0, SZ3O_F64 = 1 };
enum { SZ3O_EB_ABS = 0, SZ3O_EB_REL = 1 };
enum { SZ3O_LINEAR = 0, SZ3O_CUBIC = 1 };

#define SZ3O_MAX_LEVELS 32
#define SZ3O_LMAX 24          /* longest Huffman code the format allows */
#define SZ3O_HEADER_BYTES 288
#define SZ3O_SUBBLOCK 512     /* codes per decode sub-block inside a chunk */

/* Parameter block.  Same byte layout as the CUDA library's sz3g_params. */
typedef struct sz3o_params {
  uint32_t dtype;          /* SZ3O_F32 / SZ3O_F64                          */
  uint32_t ndim;           /* 1..4                                         */
  uint64_t dims[4];        /* extents, slowest axis first; unused = 1;
                              the product N must be in [1, 2^31]           */
  uint32_t eb_mode;        /* SZ3O_EB_ABS / SZ3O_EB_REL                    */
  uint32_t interp;         /* SZ3O_LINEAR / SZ3O_CUBIC (all levels)        */
  double eb;               /* > 0; REL: fraction of (max - min)            */
  uint8_t dim_order[4];    /* permutation of 0..ndim-1 (all levels)        */
  uint8_t per_level;       /* 1: level_interp / level_order override       */
  uint8_t reserved[3];
  uint32_t radius;         /* 2..32768; codes are uint16 in [0, 2*radius)  */
  uint32_t chunk_codes;    /* Huffman chunk, multiple of 8 in [8, 65536]   */
  uint8_t level_interp[SZ3O_MAX_LEVELS];   /* index = level l (1..L)     */
  uint8_t level_order[SZ3O_MAX_LEVELS][4]; /* index = level l (1..L)     */
} sz3o_params;

/* Number of points N and number of levels L = ceil(log2(max extent)). */
int sz3o_shape(const sz3o_params* p, uint64_t* n_points, uint32_t* n_levels);

/* Error bound (REL: eb * (max - min) in double).  eb_T receives the bound
 * rounded toward zero into T (4 or 8 bytes). */
int sz3o_error_bound(const sz3o_params* p, const void* x, double* eb_abs, void* eb_T);

/* Traversal order: spatial (row-major) index of the point behind each code. */
int sz3o_traversal(const sz3o_params* p, uint64_t* spatial, uint64_t n);

/* Quantizer on one (value, prediction) pair: code in [0, 2*radius), 0 means
 * unpredictable; *recon receives the reconstructed value (x if unpredictable). */
int sz3o_quantize1(uint32_t dtype, const void* x, const void* pred, const void* eb_T,
                   uint32_t radius, uint32_t* code, void* recon);

/* predict_quantize over the whole field (Alg. 1 lines 2-4).
 * codes: N uint16 in traversal order; unpred: up to N values of T;
 * recon: N values of T (the decompressed field); eb_T: T. */
int sz3o_quantize(const sz3o_params* p, const void* x, uint16_t* codes, void* unpred,
                  uint64_t* n_unpred, void* recon, void* eb_T);

/* recover() over the whole field: inverse of sz3o_quantize given eb_T. */
int sz3o_recover(const sz3o_params* p, const void* eb_T, const uint16_t* codes,
                 const void* unpred, uint64_t n_unpred, void* out);

/* Histogram of n codes into 65536 uint64 bins. */
int sz3o_histogram(const uint16_t* codes, uint64_t n, uint64_t* hist);

/* Huffman code lengths (0 = unused symbol) for nsym symbols, lengths <= lmax. */
int sz3o_huffman_lengths(const uint64_t* freq, uint32_t nsym, uint32_t lmax, uint8_t* len);

/* Canonical codes from lengths. */
int sz3o_canonical_codes(const uint8_t* len, uint32_t nsym, uint32_t* code);

/* Chunked encode: chunk j covers codes [chunk*j, chunk*(j+1)).  Writes the
 * payload words, the word count of every chunk and (sub_bits, may be NULL)
 * the bit lengths of each chunk's 512-code sub-blocks but the last,
 * ceil(chunk/512) - 1 per chunk. */
int sz3o_huffman_encode(const uint16_t* codes, uint64_t n, const uint8_t* len,
                        const uint32_t* code, uint32_t chunk, uint32_t* words,
                        uint64_t cap_words, uint32_t* chunk_words, uint16_t* sub_bits,
                        uint64_t* n_words);

/* Chunked decode of n codes; sub_bits (may be NULL) is checked against the
 * decoded sub-block boundaries. */
int sz3o_huffman_decode(const uint32_t* words, uint64_t n_words, const uint32_t* chunk_words,
                        const uint16_t* sub_bits, uint32_t chunk, const uint8_t* len,
                        uint32_t nsym, uint16_t* codes, uint64_t n);

int sz3o_compress_bound(const sz3o_params* p, uint64_t* max_bytes);
int sz3o_compress(const sz3o_params* p, const void* x, void* out, uint64_t capacity,
                  uint64_t* out_bytes);
int sz3o_read_header(const void* stream, uint64_t bytes, sz3o_params* p, uint64_t* n_points);
int sz3o_decompress(const void* stream, uint64_t bytes, void* out, uint64_t capacity);

/* Per-level selection of interpolation and axis order (rank <= 3).
 * Candidate c = 2 o + interp over the axis orders (0,1,2), (1,2,0), (2,0,1),
 * (2,1,0) (2-D: (0,1), (1,0), (0,1), (1,0); 1-D: (0)).  cost[8]: estimated
 * bits of level `level` (1..L) under each candidate, from all points of the
 * level (nblocks = 0) or those inside nblocks seeded 16-point sample blocks.
 * feat[16]: the level's features.  p's interp / order are not used. */
#define SZ3O_SEL_CANDIDATES 8
int sz3o_select_costs(const sz3o_params* p, const void* x, uint32_t level, uint32_t nblocks, uint64_t seed,
                      double* cost);
int sz3o_select_features(const sz3o_params* p, const void* x, uint32_t level, uint32_t nblocks, uint64_t seed,
                         double* feat);
/* The SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014): the
 * first output of the generator whose state is `key`. */
uint64_t sz3o_splitmix64(uint64_t key);
/* The sample blocks of level `level`: block b covers grid coordinates
 * [lo[4b+d], hi[4b+d]) of G_{level-1} on axis d (d < ndim).  nblocks is
 * capped at 1024; returns the number of blocks written. */
uint32_t sz3o_select_blocks(const sz3o_params* p, uint32_t level, uint32_t nblocks, uint64_t seed, uint64_t* lo,
                            uint64_t* hi);

/* Optional lossless stage after the Huffman coder (szlz.c): byte-level LZ77
 * of our own definition over independent blocks of SZLZ_BLOCK bytes.
 * Stream (little-endian): "SZLZ", u32 block size, u64 n (input bytes),
 * u32 n_blocks = ceil(n / block), u32 0; then u32 size[n_blocks] (payload
 * bytes of block b; bit 31 set: stored raw); then, from the next 8-byte
 * boundary, the payloads in block order, each padded with zeros to 4 bytes.
 * A coded payload is a run of sequences: token (literal count, max 15) << 4 |
 * (match length - 4, max 15); when the literal nibble is 15, the rest of the
 * count as 255-bytes and a last byte < 255; the literals; then, unless the
 * payload ends there (the last sequence: literals only, match nibble 0), a
 * u16 distance back (1..65535) and, when the match nibble is 15, the rest of
 * the length the same way.  Matches may overlap their own output. */
#define SZLZ_BLOCK 32768
#define SZLZ_HEADER 24
uint64_t sz3o_lz_bound(uint64_t n);
int sz3o_lz_compress(const void* in, uint64_t n, void* out, uint64_t capacity, uint64_t* out_bytes);
int sz3o_lz_decompress(const void* in, uint64_t bytes, void* out, uint64_t capacity, uint64_t* out_n);

/* ---- SZ3-Pastri modules (szpastri.c) -------------------------------------
 * Unpred-aware quantizer (Sec. 4.2): values of T (dtype 0 float, 1 double)
 * aligned to the exponent e = floor(log2(eb)) of the bound, q = trunc(v /
 * 2^e), stored as planes of bits.  Stream (little-endian): "SZBP", u32 dtype,
 * u64 n, i32 e, u32 B (bit length of max |q|, <= 62), u64 W = ceil(n / 32);
 * then W u32 words of signs (bit j of word w: q[32w + j] < 0), then B planes
 * of W words, the plane of bit B-1 first and of bit 0 last (bit j of word w:
 * that bit of |q[32w + j]|); bits past n are 0.  Decodes to q 2^e.
 * Errors: SZ3O_E_INVAL (eb not finite and > 0, a |v / 2^e| >= 2^62),
 * SZ3O_E_NONFINITE, SZ3O_E_CAPACITY; decode SZ3O_E_CORRUPT. */
#define SZBP_HEADER 32
int sz3o_bitplane_exponent(double eb, int32_t* e);
uint64_t sz3o_bitplane_bound(uint64_t n);
int sz3o_bitplane_encode(uint32_t dtype, const void* v, uint64_t n, double eb, void* out, uint64_t capacity,
                         uint64_t* out_bytes);
int sz3o_bitplane_decode(const void* in, uint64_t bytes, void* out, uint64_t capacity, uint64_t* n_out);
/* Fixed Huffman code lengths over the 2 radius quantization codes (Sec. 3.2
 * Encoder, the predefined tree of SZ-Pastri): len[r] = 1; a code at distance
 * k >= 1 from r, with c the bit length of k, 2c + 2 bits when c <= 10, else
 * 24; len[0] (unpredictable) = 24.  Codewords: sz3o_canonical_codes. */
int sz3o_huffman_fixed_lengths(uint32_t radius, uint8_t* len);

#ifdef __cplusplus
}
#endif
#endif
