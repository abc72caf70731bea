/*
 * sz3g.h -- C ABI of the GB300 (sm_103a) implementation of the SZ3-Interp
 * compression hot path: multilevel interpolation prediction fused with the
 * linear-scaling quantizer, the quantization-code histogram, and chunked
 * canonical Huffman encode / decode (SZ3 paper, arXiv 2111.02925).
 *
 * Conventions for every function below:
 *  - Return value: 0 (SZ3G_OK) or a negative SZ3G_E_* status.  No function
 *    aborts, throws or exits; a CUDA failure is reported as SZ3G_E_CUDA.
 *  - Buffers named d_* are device pointers, h_* host pointers, owned by the
 *    caller, never freed or kept by the library after the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Kernels run on that stream; where a function returns a value
 *    computed on the GPU (sizes, statuses) it synchronises that stream before
 *    returning, and says so.
 *  - Workspace: `d_workspace` may be NULL, in which case the library takes
 *    the scratch it needs from its own stream-ordered memory pool
 *    (cudaMallocFromPoolAsync / cudaFreeAsync on `stream`) and returns it to
 *    the pool before returning; the pool keeps freed memory reserved for the
 *    process, so repeated calls reuse it without mapping it again.  Otherwise it must be at least sz3g_workspace_size() bytes,
 *    256-byte aligned, and is not read before it is written.
 *  - Data layout: a field is a dense row-major (C order) array of N = prod(dims)
 *    values of float (SZ3G_F32) or double (SZ3G_F64), slowest axis first.
 */
#ifndef SZ3G_H
#define SZ3G_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SZ3G_OK = 0,
  SZ3G_E_INVAL = -1,          /* bad dims / eb / radius / order / chunk / pointer alignment */
  SZ3G_E_NONFINITE = -2,      /* NaN or Inf in the input field                 */
  SZ3G_E_ZERO_RANGE_REL = -3, /* REL bound on a field whose value range is 0   */
  SZ3G_E_CAPACITY = -4,       /* output buffer or workspace too small          */
  SZ3G_E_CORRUPT = -5,        /* stream fails a magic/version/length/decode check */
  SZ3G_E_CUDA = -6,           /* a CUDA runtime call failed                    */
  SZ3G_E_NOMEM = -7,          /* device allocation failed                      */
  SZ3G_E_TIMEOUT = -8,        /* a bounded wait inside a kernel gave up        */
  SZ3G_E_CHECK = -9           /* checking build only: an index check inside a kernel failed */
};

enum { SZ3G_F32 = 0, SZ3G_F64 = 1 };
enum { SZ3G_EB_ABS = 0, SZ3G_EB_REL = 1 };
enum { SZ3G_LINEAR = 0, SZ3G_CUBIC = 1 };

#define SZ3G_MAX_LEVELS 32
#define SZ3G_LMAX 24        /* longest Huffman code in a stream            */
#define SZ3G_HEADER_BYTES 288
#define SZ3G_LZ_BLOCK 32768   /* bytes per block of the lossless stage */
#define SZ3G_LZ_HEADER 24     /* its header, before the block size table */

/*
 * Compression parameters (the paper's Config<T,N>, Appendix A.1 / Alg. 1
 * input `conf`).  232 bytes, 8-byte aligned, no implicit padding.
 *   dims        extents, slowest first, entries >= ndim ignored; every extent
 *               >= 1 and N = prod(dims) <= 2^31.
 *   eb_mode/eb  ABS: eb is the absolute bound.  REL: the bound is eb times the
 *               value range max - min (Sec. 6.2, throughput figure caption).
 *   interp      SZ3G_LINEAR or SZ3G_CUBIC (Sec. 6.2, SZ3-Interp).
 *   dim_order   permutation of 0..ndim-1: the order in which a level refines
 *               the axes.
 *   per_level   1: level l (1..L, L = ceil(log2 max dim)) uses
 *               level_interp[l] / level_order[l] instead.
 *   radius      quantization radius r in [2, 32768]: codes are uint16 in
 *               [0, 2r), 0 marks an unpredictable value (Sec. 3.2 Quantizer).
 *   chunk_codes Huffman chunk length, a multiple of 8 in [8, 65536]; every
 *               chunk starts on a fresh 32-bit word so chunks decode in parallel.
 */
typedef struct sz3g_params {
  uint32_t dtype;
  uint32_t ndim;
  uint64_t dims[4];
  uint32_t eb_mode;
  uint32_t interp;
  double eb;
  uint8_t dim_order[4];
  uint8_t per_level;
  uint8_t reserved[3];
  uint32_t radius;
  uint32_t chunk_codes;
  uint8_t level_interp[SZ3G_MAX_LEVELS];
  uint8_t level_order[SZ3G_MAX_LEVELS][4];
} sz3g_params;

/* Human-readable text of a status code (static storage). */
const char* sz3g_strerror(int status);

/* Largest stream sz3g_compress can write for these parameters (header +
 * every value unpredictable + longest codes).  No GPU work. */
int sz3g_compress_bound(const sz3g_params* p, size_t* max_bytes);

/* Scratch bytes sz3g_compress (for_decompress = 0) or sz3g_decompress
 * (for_decompress = 1) needs for these parameters.  No GPU work. */
int sz3g_workspace_size(const sz3g_params* p, int for_decompress, size_t* bytes);

/*
 * Compress one field: Alg. 1 of the paper without its preprocessor and
 * lossless stages -- predict (multilevel interpolation, Sec. 6.2) and quantize
 * (linear-scaling quantizer, Sec. 3.2) every point, save the unpredictable
 * values, histogram the codes, build a Huffman code from the histogram and
 * encode the codes (Sec. 3.2 Encoder), chunk by chunk.
 *   d_in         N values of T (device, 16-byte aligned), not modified.
 *   d_out        device buffer of out_capacity bytes (>= sz3g_compress_bound
 *                is always enough), 16-byte aligned.  Receives the stream.
 *   out_bytes    host; receives the stream length.  This needs the result of
 *                the GPU work, so the call synchronises `stream` before return.
 * Errors: SZ3G_E_INVAL, SZ3G_E_NONFINITE, SZ3G_E_ZERO_RANGE_REL,
 * SZ3G_E_CAPACITY (the stream did not fit; d_out contents undefined),
 * SZ3G_E_TIMEOUT, SZ3G_E_CUDA, SZ3G_E_NOMEM.
 */
int sz3g_compress(const sz3g_params* p, const void* d_in, void* d_out, size_t out_capacity,
                  size_t* out_bytes, void* d_workspace, size_t ws_bytes, void* stream);

/*
 * Graph cache (on by default): sz3g_compress / sz3g_decompress calls given a
 * caller-owned workspace replay, as one CUDA graph launch, the pipeline
 * captured by an earlier call with the same parameters (stream header) and
 * the same buffers and workspace -- the per-kernel host work between the
 * kernels is then skipped.  Up to 8 pipelines are kept (least recently used
 * replaced); not used while profiling is on.  on = 0 turns it off and frees
 * the cached graphs.
 */
int sz3g_graph_cache(int on);

/*
 * Failure injection, for tests of the library's failure handling (the paper
 * has no counterpart).  Process-wide settings read by the host when a call
 * enqueues its kernels (a pipeline replayed from the graph cache, or a batch
 * captured earlier, keeps the settings it was built with); not thread-safe.
 * Nothing here makes a GPU fault: every injected failure ends a bounded wait
 * or refuses an allocation, and the call returns its status.
 *   SZ3G_DEBUG_RESET        all settings back to normal (value ignored)
 *   SZ3G_DEBUG_WAIT_LIMIT   value = spin limit of the level queue's dependency
 *                           waits and of the encoder's and scans' look-backs
 *                           (0: the built-in limits)
 *   SZ3G_DEBUG_QUEUE_STALL  value = v: the first level of a batch's level
 *                           queue at or after index v that waits on another
 *                           level waits for one chunk more than that level
 *                           has (-1: none); the wait gives up and the run
 *                           reports SZ3G_E_TIMEOUT
 *   SZ3G_DEBUG_SILENT_CHUNK value = chunk that never publishes its look-back
 *                           state in the one-pass encoder (fields of at most
 *                           1024 chunks; -1: none); the chunks after it give
 *                           up and the call reports SZ3G_E_TIMEOUT
 *   SZ3G_DEBUG_ALLOC_FAIL   value = number of the library's following
 *                           workspace allocations that fail (SZ3G_E_NOMEM)
 * Returns SZ3G_OK, or SZ3G_E_INVAL for an unknown kind or a value out of range.
 */
enum {
  SZ3G_DEBUG_RESET = 0,
  SZ3G_DEBUG_WAIT_LIMIT = 1,
  SZ3G_DEBUG_QUEUE_STALL = 2,
  SZ3G_DEBUG_SILENT_CHUNK = 3,
  SZ3G_DEBUG_ALLOC_FAIL = 4
};
int sz3g_debug_inject(int kind, long long value);

/* ---------------------------------------------------------------------------
 * Optional lossless stage after the Huffman coder (SZ3 ends its pipelines in
 * a dictionary coder): byte-level LZ77 over independent SZ3G_LZ_BLOCK-byte
 * blocks, for any byte buffer (e.g. a stream of sz3g_compress).  Format
 * (little-endian): "SZLZ", u32 block size, u64 n, u32 n_blocks =
 * ceil(n / block), u32 0; u32 size[n_blocks] (payload bytes of block b; bit
 * 31: stored raw); from the next 8-byte boundary the payloads in block order,
 * each padded with zeros to 4 bytes.  A coded payload is a run of sequences:
 * token = (literal count, max 15) << 4 | (match length - 4, max 15); the rest
 * of a count of 15 or more as 255-bytes ending in a byte < 255; the literals;
 * unless the payload ends there (the last sequence: literals only, match
 * nibble 0), a u16 distance back (1..65535) and the rest of a match nibble
 * 15 the same way.  Matches may overlap their output.  The encoder's parse:
 * h(i) = (u32 at i) * 2654435761 >> 20 (mod 2^32); the candidate of position
 * i is the last earlier position of the block with the same hash (over every
 * position, not only the ones the parse visits); from `pos` the first
 * position whose candidate matches in four bytes starts a match, extended
 * while the next byte equals; a block whose coded form is not shorter is
 * stored raw.  Device pointers 16-byte aligned; the workspace comes from the
 * library's pool; synchronise `stream`.
 * ------------------------------------------------------------------------- */
int sz3g_lossless_bound(uint64_t n, uint64_t* max_bytes);
int sz3g_lossless_compress(const void* d_in, uint64_t n, void* d_out, size_t out_capacity, size_t* out_bytes,
                           void* stream);
/* *n_out: decoded bytes (the header's n); out_capacity >= n, else SZ3G_E_CAPACITY */
int sz3g_lossless_decompress(const void* d_stream, size_t bytes, void* d_out, size_t out_capacity, uint64_t* n_out,
                             void* stream);

/* ---------------------------------------------------------------------------
 * SZ3-Pastri modules on the quantize / encode path.
 *
 * Unpred-aware quantizer (Sec. 4.2): n values of T (dtype SZ3G_F32 / F64,
 * device, aligned to T) are aligned to the exponent e = floor(log2(eb)) of
 * the absolute bound eb, q = trunc(v / 2^e) (so |v - q 2^e| < 2^e <= eb), and
 * stored by bitplane.  Stream (little-endian, d_out 16-byte aligned, at most
 * sz3g_bitplane_bound bytes): "SZBP", u32 dtype, u64 n, i32 e, u32 B (bit
 * length of max |q|, <= 62), u64 W = ceil(n / 32); then W u32 words of signs
 * (bit j of word w: q[32w + j] < 0); then B planes of W words each, the plane
 * of bit B-1 first and of bit 0 last (bit j of word w: that bit of
 * |q[32w + j]|); bits past n are 0.  Decodes to q 2^e in T (exact).
 * Encode errors: SZ3G_E_INVAL (eb not finite and > 0, some |v / 2^e| >= 2^62),
 * SZ3G_E_NONFINITE, SZ3G_E_CAPACITY; decode: SZ3G_E_CORRUPT (header or
 * length), SZ3G_E_CAPACITY.  Both synchronise `stream`.
 *
 * Fixed Huffman (Sec. 3.2 Encoder, the predefined tree of SZ-Pastri): the
 * code lengths (d_len, 2 radius uint8) and canonical codewords (d_code, 2
 * radius uint32) of a code fixed in advance, for sz3g_huffman_encode /
 * sz3g_huffman_decode with nsym = 2 radius: code r 1 bit; a code at distance
 * k >= 1 from r, c = bit length of k, 2c + 2 bits when c <= 10, else 24; code 0
 * (unpredictable) 24 bits.  Asynchronous; radius in [2, 32768].
 * ------------------------------------------------------------------------- */
#define SZ3G_BP_HEADER 32
int sz3g_bitplane_bound(uint64_t n, uint64_t* max_bytes);
int sz3g_bitplane_encode(uint32_t dtype, const void* d_values, uint64_t n, double eb, void* d_out,
                         size_t out_capacity, size_t* out_bytes, void* stream);
int sz3g_bitplane_decode(const void* d_stream, size_t bytes, void* d_out, size_t out_capacity, uint64_t* n_out,
                         void* stream);
int sz3g_huffman_fixed(uint32_t radius, uint8_t* d_len, uint32_t* d_code, void* stream);

/*
 * Parse and validate a stream header.  `stream` is a host pointer
 * (stream_on_device = 0) or a device pointer (1: the 288 header bytes are
 * copied to the host with a synchronous cudaMemcpy).  Fills *p and the point
 * count.  Errors: SZ3G_E_CORRUPT, SZ3G_E_INVAL (NULL pointers), SZ3G_E_CUDA.
 */
int sz3g_read_header(const void* stream, size_t bytes, int stream_on_device, sz3g_params* p,
                     uint64_t* n_points);

/*
 * Decompress one stream: decode the chunks, then recover every point in the
 * traversal order of the compressor (recover(), Sec. 3.2; decode(), Sec. 3.2
 * Encoder).
 *   d_stream     device, `bytes` long, 16-byte aligned.
 *   d_out        device, out_capacity >= N * sizeof(T) bytes, 16-byte aligned.
 * Reads the header to the host first (synchronous) and synchronises `stream`
 * at the end to report decode errors.
 * Errors: SZ3G_E_CORRUPT, SZ3G_E_CAPACITY, SZ3G_E_INVAL, SZ3G_E_TIMEOUT,
 * SZ3G_E_CUDA, SZ3G_E_NOMEM.
 */
int sz3g_decompress(const void* d_stream, size_t bytes, void* d_out, size_t out_capacity,
                    void* d_workspace, size_t ws_bytes, void* stream);

/*
 * Asynchronous forms for stream-ordered use and CUDA-graph capture: the
 * pipeline is enqueued on `stream` and the call returns without
 * synchronising; nothing is allocated and nothing is read back to the host.
 * The result is written on the device when the pipeline ends:
 *   *d_status      int32, SZ3G_OK or the error code the synchronous form
 *                  would have returned for a run-time failure (non-finite
 *                  input, zero range with REL, capacity, corrupt stream,
 *                  timeout);
 *   *d_out_bytes   (compress, may be NULL) u64 stream length, 0 on error.
 * The workspace is required (sz3g_workspace_size bytes, 256-byte aligned) and
 * must not be shared with a run still in flight.  Host-side checks (params,
 * pointers, alignment, workspace size, header) are reported by the return
 * value, as SZ3G_E_INVAL / SZ3G_E_CAPACITY / SZ3G_E_CORRUPT; SZ3G_OK means the
 * work is enqueued.  A capture replays with the buffers, parameters (and, for
 * decompress, the header) given at capture time.
 *   h_header  (decompress) host copy of the stream's SZ3G_HEADER_BYTES bytes.
 */
int sz3g_compress_async(const sz3g_params* p, const void* d_in, void* d_out, size_t out_capacity,
                        unsigned long long* d_out_bytes, int* d_status, void* d_workspace, size_t ws_bytes,
                        void* stream);
int sz3g_decompress_async(const void* h_header, const void* d_stream, size_t bytes, void* d_out,
                          size_t out_capacity, int* d_status, void* d_workspace, size_t ws_bytes,
                          void* stream);

/*
 * End-to-end forms on HOST buffers: copy h_in to the device, compress, copy
 * the stream back (and the reverse for decompress), all on `stream`.  The
 * device copies of input, output and workspace are one staging set per
 * device, kept by the library between calls and grown on demand (so repeated
 * calls on one field shape replay the cached graph of the pipeline, see
 * sz3g_graph_cache); a call made while another thread holds the set stages
 * through memory of the library's stream-ordered pool instead.  Both return
 * after synchronising `stream`.  h_* may be pageable or pinned; pinned memory
 * makes the copies asynchronous and faster.  Decompressing into page-locked
 * h_out a 3-D field whose finest level runs on the register-blocked kernel,
 * that level runs in slabs of planes and each slab is copied out (on a
 * library stream) while the next ones are computed.  Same errors as the
 * device forms; on an error the contents of h_out are unspecified.
 */
int sz3g_compress_host(const sz3g_params* p, const void* h_in, void* h_out, size_t out_capacity,
                       size_t* out_bytes, void* stream);
int sz3g_decompress_host(const void* h_stream, size_t bytes, void* h_out, size_t out_capacity,
                         void* stream);

/*
 * Frees what the library keeps between calls: the cached graphs, the staging
 * sets of the host-buffer forms, and the free memory of its pool on the
 * devices that held a staging set.  Synchronises those devices.  Not to be
 * called while another thread is inside a call of this library.
 */
int sz3g_trim(void);

/* ---------------------------------------------------------------------------
 * Stage entry points: the steps of the hot path one at a time, with their
 * intermediate results exposed (used to check each step on its own).
 * ------------------------------------------------------------------------- */

/*
 * predict_quantize (Appendix A.7, Alg. 1 lines 2-4) over the whole field.
 *   d_codes   N uint16 codes in traversal order (0 = unpredictable).
 *   d_unpred  up to N values of T: the unpredictable values in traversal
 *             order (Sec. 3.2 Quantizer save()).
 *   d_hist    65536 uint32 bins: histogram of d_codes.
 *   h_n_unpred, h_ebT (host, 8 bytes: the bound rounded into T, as its T
 *             bits) are written after a stream synchronisation.
 */
int sz3g_predict_quantize(const sz3g_params* p, const void* d_in, uint16_t* d_codes, void* d_unpred,
                          uint32_t* d_hist, uint64_t* h_n_unpred, void* h_ebT, void* d_workspace,
                          size_t ws_bytes, void* stream);

/*
 * recover() (Sec. 3.2) over the whole field: inverse of sz3g_predict_quantize.
 *   h_ebT     host, the T value of the bound.  d_codes / d_unpred as above.
 *   d_out     N values of T.
 * Errors: SZ3G_E_CORRUPT when a code is outside [0, 2r) or the number of zero
 * codes differs from n_unpred (after a stream synchronisation).
 */
int sz3g_recover(const sz3g_params* p, const void* h_ebT, const uint16_t* d_codes,
                 const void* d_unpred, uint64_t n_unpred, void* d_out, void* d_workspace,
                 size_t ws_bytes, void* stream);

/*
 * Huffman code lengths from a histogram (Sec. 3.2 Encoder: tree built
 * greedily from frequencies): d_hist 65536 uint32 bins -> d_len 65536 uint8
 * (0 = unused), every length <= SZ3G_LMAX.  d_code receives the canonical
 * codewords (uint32, right-aligned).  One CTA; synchronises `stream` to
 * report errors.
 */
int sz3g_huffman_build(const uint32_t* d_hist, uint32_t nsym, uint8_t* d_len, uint32_t* d_code,
                       void* stream);

/*
 * Chunked Huffman encode of n codes with the lengths / codewords above.
 * Chunk j covers codes [chunk*j, chunk*(j+1)); it starts on a fresh word,
 * bits most significant first, tail zero.
 *   d_words        payload capacity cap_words uint32.
 *   d_chunk_words  ceil(n/chunk) uint32: words of every chunk.
 *   d_sub_bits     NULL, or ceil(n/chunk) * (ceil(chunk/512) - 1) uint16: bit
 *                  lengths of each chunk's 512-code sub-blocks but the last
 *                  (0 past the end of a short last chunk).
 *   h_n_words      host, total words (after a stream synchronisation).
 */
int sz3g_huffman_encode(const uint16_t* d_codes, uint64_t n, const uint8_t* d_len,
                        const uint32_t* d_code, uint32_t nsym, uint32_t chunk, uint32_t* d_words,
                        uint64_t cap_words, uint32_t* d_chunk_words, uint16_t* d_sub_bits,
                        uint64_t* h_n_words, void* stream);

/*
 * Chunked Huffman decode of n codes (Sec. 3.2 Encoder decode()).  d_len are
 * the code lengths of nsym symbols: any prefix code with lengths <= LMAX
 * (Kraft sum <= 1; an incomplete one such as sz3g_huffman_fixed's too).  With d_sub_bits (as written by
 * sz3g_huffman_encode) every 512-code sub-block decodes on its own thread and
 * must end exactly where the table says; with NULL one thread decodes a
 * chunk.  SZ3G_E_CORRUPT when a chunk runs out of bits, holds a bit pattern
 * that is no codeword or contradicts the sub-block table (after a
 * synchronisation).
 */
int sz3g_huffman_decode(const uint32_t* d_words, uint64_t n_words, const uint32_t* d_chunk_words,
                        const uint16_t* d_sub_bits, uint32_t chunk, const uint8_t* d_len,
                        uint32_t nsym, uint16_t* d_codes, uint64_t n, void* stream);

/*
 * sz3g_huffman_decode without any device allocation (the paper has no
 * counterpart: this serves callers that must not allocate device memory,
 * such as a process whose device memory is owned by another allocator's pool,
 * or a latency-sensitive path where an allocation may block or fail).  Same
 * arguments and results as sz3g_huffman_decode; its scratch is a fixed 4 MiB
 * array built into the library (held on every GPU that loads the library
 * until the process exits).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current.
 *  - Synchronous: every call waits for its own GPU work (also on the error
 *    paths), so it cannot be recorded into a CUDA graph.
 *  - All calls share the array and each call resets the parts that must start
 *    at zero; calls whose GPU work overlaps race on it, so do not run two at
 *    once.
 *  - SZ3G_E_CAPACITY when the stream needs more scratch than the array holds
 *    (about 32 bytes per 4096-code chunk plus 0.7 MiB of decode tables,
 *    i.e. n up to roughly 4.3e8 codes at 4096-code chunks); nothing is
 *    launched then.
 *  - Statuses as sz3g_huffman_decode (the same mapping of device flags).
 */
int sz3g_huffman_decode_static(const uint32_t* d_words, uint64_t n_words, const uint32_t* d_chunk_words,
                               const uint16_t* d_sub_bits, uint32_t chunk, const uint8_t* d_len,
                               uint32_t nsym, uint16_t* d_codes, uint64_t n, void* stream);

/* ---------------------------------------------------------------------------
 * Batches (no counterpart in the paper: its compressor handles one field per
 * call).  Many fields of uneven shape and error bound are compressed, or
 * decompressed, by one graph launch.  A batch is planned once for a fixed set
 * of buffers: its fields are spread over parallel branches, each branch runs
 * its fields' pipelines one after another in a workspace the batch owns, and
 * every launch of every field is captured once into a CUDA graph that each
 * run replays.  The results are bit-identical to one sz3g_compress /
 * sz3g_decompress call per field.
 * ------------------------------------------------------------------------- */
typedef struct sz3g_batch sz3g_batch;

/*
 * Plans a batch of n fields and captures its graph (8 branches, no CTA cap).
 *   decompress = 0: params[i] and d_in[i] (device, 16-byte aligned) describe
 *     field i, d_out[i] receives its stream (out_capacity[i] >= its
 *     sz3g_compress_bound); in_bytes may be NULL.
 *   decompress = 1: d_in[i] holds a stream of in_bytes[i] bytes, d_out[i]
 *     (out_capacity[i] bytes) receives the field; params may be NULL.  The
 *     stream headers are read here (synchronises).
 * Buffers stay owned by the caller and must outlive the batch; the batch
 * allocates its workspaces and a result array.  Errors as for the single-
 * field calls (the first failing field decides).
 */
int sz3g_batch_create(int n, int decompress, const sz3g_params* params, const void* const* d_in,
                      const size_t* in_bytes, void* const* d_out, const size_t* out_capacity,
                      sz3g_batch** batch);

/* Replays the batch's graph on `stream` (asynchronous). */
int sz3g_batch_run(sz3g_batch* batch, void* stream);

/*
 * Synchronises the device and reads the results of the last run: h_bytes[i]
 * the stream length of field i (compress), h_status[i] its status (either may
 * be NULL).  Returns the first non-OK status, else SZ3G_OK.
 */
int sz3g_batch_results(sz3g_batch* batch, uint64_t* h_bytes, int* h_status);

/*
 * Rebuilds the graph with `branches` parallel branches (clamped to [1, n])
 * and at most `cta_cap` CTAs per level-kernel launch (0: a full wave).
 */
int sz3g_batch_configure(sz3g_batch* batch, int branches, int cta_cap);

/*
 * Level-queue mode (on = 1): every field gets its own workspace; the branches
 * run each field's steps up to its grid levels, then one persistent kernel
 * launch per element type runs the levels of all fields from a cross-field
 * work queue -- tiles of every (field, level) in coarse-to-fine order, each
 * level waiting (bounded) on a completion counter of its field's next
 * coarser level -- then the branches run the encoders.  Rebuilds the graph;
 * results stay bit-identical.  on = 0: every field's levels are launched in
 * its own branch (the default).
 */
int sz3g_batch_set_queue(sz3g_batch* batch, int on);

/* Whether the level queue is used, and the grid levels it holds. */
int sz3g_batch_queue_info(const sz3g_batch* batch, int* on, int* levels);

/*
 * Autotuner: runs the batch (three times after two warm-ups, keeping the
 * fastest of the three) under every combination
 * of 1..256 branches and CTA caps of none, 1, 1/2 and 1/4 of the SMs, and
 * in level-queue mode under every branch count, keeps the fastest and
 * reports it.  Overwrites the batch's outputs; synchronises.
 */
int sz3g_batch_tune(sz3g_batch* batch, void* stream, int* h_branches, int* h_cta_cap);

/* Current configuration and the number of nodes of the captured graph. */
int sz3g_batch_info(const sz3g_batch* batch, int* branches, int* cta_cap, uint64_t* graph_nodes);

/* Frees the batch's graph, workspaces and result array (NULL is accepted). */
int sz3g_batch_destroy(sz3g_batch* batch);

/* ---------------------------------------------------------------------------
 * Per-level choice of interpolation and axis order (the paper's best-fit /
 * composite predictor idea, Sec. 3.1, and the per-level interpolation of
 * SZ3-Interp, Sec. 6.2; fields of rank <= 3).  Candidate c = 2 o + interp
 * over the axis orders (0,1,2), (1,2,0), (2,0,1), (2,1,0) (2-D: (0,1), (1,0),
 * then the same two again, never chosen on a tie; 1-D: (0)).  For level l the
 * estimate predicts every point of the level from the original values along
 * its pass axis (the last axis of the order on which its coordinate at
 * stride 2^(l-1) is odd), quantizes it with p's bound and radius, and costs
 * the codes by their Shannon bits plus 8 sizeof(T) bits per unpredictable
 * value -- over all points of the level (nblocks = 0) or those inside
 * nblocks seeded sample blocks of up to 16 grid points per axis (block b of
 * level l starts on axis d at SplitMix64(seed ^ l << 48 ^ b << 8 ^ d) mod
 * (m_d - span_d + 1); a point in several blocks counts once).  p's interp /
 * dim_order are not used.  All of these synchronise `stream`.
 * ------------------------------------------------------------------------- */

/* h_cost[(l - 1) * 8 + c]: estimated bits of level l (1..L) under candidate c. */
int sz3g_select_costs(const sz3g_params* p, const void* d_x, uint32_t nblocks, uint64_t seed, double* h_cost,
                      void* stream);

/*
 * h_feat[(l - 1) * 16 + k]: 16 features of level l from the same sample
 * blocks: per axis d = 0..2 (0 for missing axes) log2(1 + mean |linear
 * error| / eb), log2(1 + mean |cubic error| / eb) and the log2 ratio of mean
 * squared lag-2 to lag-1 differences; l / L; l - 1; log10(eb / (max - min));
 * the fraction of points whose differences to their +1 neighbours are all
 * within eb; the fractions of the level's points (order (0,1,2)) whose linear
 * and cubic errors exceed 64 eb; log2 of the last over the first extent.
 */
int sz3g_select_features(const sz3g_params* p, const void* d_x, uint32_t nblocks, uint64_t seed, double* h_feat,
                         void* stream);

/* Sampling selector: h_choice[l] = the candidate of least estimated bits for
 * level l = 1..L (ties: the lower index); h_choice[0] = 0. */
int sz3g_select_sampled(const sz3g_params* p, const void* d_x, uint32_t nblocks, uint64_t seed, uint8_t* h_choice,
                        void* stream);

/* Learned selector: h_choice[l] = argmax of the network's logits on level l's
 * features (d_w: SZ3G_MLP_WEIGHTS floats on the device). */
int sz3g_select_learned(const sz3g_params* p, const void* d_x, const float* d_w, uint32_t nblocks, uint64_t seed,
                        uint8_t* h_choice, void* stream);

/*
 * The selector's network: 16 features, standardised by (f - mu) / sd, -> 64
 * hidden units (ReLU) -> 8 logits; masked softmax cross-entropy.  Weights, as
 * SZ3G_MLP_WEIGHTS floats: mu[16], sd[16], W1[64][16], b1[64], W2[8][64],
 * b2[8].  d_feat: n x 16 floats; d_mask: n x 8 bytes (1: candidate allowed);
 * d_label: n int32 (an allowed candidate).
 */
#define SZ3G_MLP_WEIGHTS 1640
/* d_logits: n x 8 (masked: -inf). */
int sz3g_mlp_forward(const float* d_w, const float* d_feat, const uint8_t* d_mask, uint32_t n, float* d_logits,
                     void* stream);
/* d_grad: SZ3G_MLP_WEIGHTS floats, the gradient of the mean loss (zero for
 * mu / sd); h_loss: the mean loss.  Synchronises. */
int sz3g_mlp_gradient(const float* d_w, const float* d_feat, const uint8_t* d_mask, const int32_t* d_label,
                      uint32_t n, float* d_grad, float* h_loss, void* stream);
/* `steps` full-batch gradient steps of size lr on d_w; h_loss: the mean loss
 * before the last step.  Synchronises. */
int sz3g_mlp_train(float* d_w, const float* d_feat, const uint8_t* d_mask, const int32_t* d_label, uint32_t n,
                   float lr, uint32_t steps, float* h_loss, void* stream);

/* ---------------------------------------------------------------------------
 * Diagnostics (no counterpart in the paper): launch accounting and per-kernel
 * timing with CUDA events, used by the benchmark to attribute time to kernels.
 * ------------------------------------------------------------------------- */

/* Total kernel launches issued by the library since it was loaded. */
int sz3g_launch_count(uint64_t* launches);

/* on != 0: from now on bracket every launch with CUDA events on its stream
 * (and drop earlier records); on == 0: stop recording.  Host-side only. */
int sz3g_profile_enable(int on);

/* Sum of the recorded durations of one kernel (name from
 * sz3g_profile_kernel_name) and the number of recorded launches.  Waits for
 * the recorded events.  SZ3G_E_INVAL for an unknown name. */
int sz3g_profile_read(const char* kernel, double* total_ms, uint64_t* launches);

/* Name of kernel `index` (0, 1, ...), or NULL past the last one. */
const char* sz3g_profile_kernel_name(int index);

#ifdef __cplusplus
}
#endif
#endif
