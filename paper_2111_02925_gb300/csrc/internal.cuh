// internal.cuh -- shared definitions of the sm_103a implementation (not part of
// the public ABI).  Every floating-point step of the prediction and of the
// quantizer is one IEEE round-to-nearest-even operation in the field type T;
// the library is compiled with -fmad=false so no multiply-add is contracted.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sz3g.h"

namespace sz3g {

constexpr int kMaxPasses = 1 + 4 * 31;  // anchor + up to 4 passes on each of 31 levels
constexpr int kSyms = 65536;            // alphabet of uint16 codes
constexpr int kLutBits = 13;            // direct decode table: first 13 bits of a codeword
#define SZ3G_SUBBLOCK 512               // codes per decode sub-block inside a chunk

// Status bits raised on the device and read back once per call.
enum : uint32_t {
  kFlagNonFinite = 1u << 0,
  kFlagZeroRange = 1u << 1,
  kFlagBadBound = 1u << 2,
  kFlagCapacity = 1u << 3,
  kFlagCorrupt = 1u << 4,
  kFlagTimeout = 1u << 5,
  kFlagCheck = 1u << 6,  // checking build: an index check failed
};

// Small block of device state at the start of every workspace.
struct DevState {
  uint32_t flags;        // kFlag* bits
  uint32_t n_used;       // symbols with a code
  uint32_t ticket;       // dynamic chunk counter of the encoder
  uint32_t range_ticket;  // blocks of the range kernel that have finished
  unsigned long long n_unpred;     // unpredictable values
  unsigned long long n_words;      // payload words
  unsigned long long out_bytes;    // stream length
  double eb_abs;         // absolute bound (double)
  double ebT_bits_d;     // unused padding slot
  unsigned long long ebT_bits;     // bound rounded into T, as T bits
  unsigned long long ebr_bits;     // fl_T(1 / eb_T), as T bits
  unsigned long long zeros_total;  // decompress: zero codes seen by the decoder
  unsigned long long pad[6];
};
static_assert(sizeof(DevState) <= 256, "DevState must fit its 256-byte slot");

// One pass of the interpolation schedule on the compact grid G_k (level
// l = k + 1): the sub-lattice of points whose coordinate on the pass axis is
// odd, on axes refined earlier in this level any, on later axes even.
// Coordinates are padded to 4 axes (leading unit axes).
struct PassDesc {
  unsigned long long off;      // code index of the pass's first point
  unsigned long long count;    // points in the pass
  uint32_t E[4];               // lattice extents
  uint32_t start[4], step[4];  // grid coordinate = start + step * lattice coordinate
  uint32_t m[4];               // extents of the grid G_k
  unsigned long long gstride[4];  // element strides of G_k (compact, row-major)
  unsigned long long xstride[4];  // strides in the full-resolution input for one G_k step
  int axis;                    // pass axis 0..3
  int interp;                  // SZ3G_LINEAR / SZ3G_CUBIC
  int grid;                    // k
  int pad;
};

// Inverse map code index -> input index for every pass (used by the encoder
// to fetch unpredictable values).  Entry 0 is the anchor.
struct PassMapEntry {
  unsigned long long off;
  uint32_t E[4];
  unsigned long long xstart;      // input index of lattice coordinate 0
  unsigned long long xls[4];      // input stride of one lattice step per axis
};
struct PassMap {
  int n;
  int pad;
  PassMapEntry e[kMaxPasses];
};

// Host-side plan of one field.
struct Plan {
  int dtype;                 // SZ3G_F32 / SZ3G_F64
  int esz;                   // 4 / 8
  int ndim;                  // as given
  int L;                     // levels
  uint32_t radius, chunk;
  unsigned long long N;
  unsigned long long n[4];   // padded to 4 axes
  unsigned long long fstride[4];
  unsigned long long gm[33][4];   // extents of G_k, k = 0..L
  unsigned long long gsize[33];   // points of G_k
  int n_pass;                // passes excluding the anchor
  PassDesc pass[kMaxPasses]; // in traversal order (level L first)
  unsigned long long n_chunks;
  uint32_t nsub;             // 512-code sub-blocks per chunk
};

// Failure injection for tests (set by sz3g_debug_inject, read on the host by
// the launchers, which pass the values to their kernels; process-wide).
struct DebugInject {
  uint32_t wait_limit;     // spin limit of the dependency waits and look-backs (0: the built-in limits)
  long long queue_stall;   // level-queue entry whose dependency can never be met (-1: none)
  long long silent_chunk;  // chunk that never publishes its look-back state in the one-pass encoder (-1: none)
  int alloc_fail;          // library allocations still to fail
};
extern DebugInject g_debug;

// Kernels known to the launch accounting (names in prof.cu).
enum KernelId {
  kKRange, kKEb, kKAnchor, kKLift, kKPassQuantize, kKPassRecover, kKCodebook, kKEncode, kKFinalize,
  kKDecodeTables, kKDecode, kKScan, kKZeroCount, kKPackTable, kKLevelQuantize, kKLevelRecover,
  kKCoarseQuantize, kKCoarseRecover, kKDecimate, kKPublish, kKSelect, kKMlp, kKLossless, kKReport, kKBitplane, kKFixedTable, kKernelCount
};

// prof.cu: whether per-launch timing is on; launches replayed inside a graph
// are added to the launch count by the replaying code.
bool profiling_on();
void count_launches(unsigned long long n);
unsigned long long launch_total();

// Named ranges on the host timeline (NVTX, header-only; free unless a
// profiler attached its collector): every C-ABI entry point opens one.
class TraceRange {
 public:
  explicit TraceRange(const char* name);
  ~TraceRange();
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};
#define SZ3G_TRACE(name) ::sz3g::TraceRange sz3g_trace_range_(name)

// Index checks of the checking build (compiled with -DSZ3G_CHECK): a failed
// check raises kFlagCheck (the call then reports SZ3G_E_CHECK) and the
// access it guards is skipped.  In the ordinary build every check is the
// constant true and compiles away.
#ifdef SZ3G_CHECK
__device__ __forceinline__ bool index_ok(bool ok, DevState* st) {
  if (!ok) atomicOr(&st->flags, kFlagCheck);
  return ok;
}
#define SZ3G_IN(cond, st) ::sz3g::index_ok((cond), (st))
#else
#define SZ3G_IN(cond, st) true
#endif

// Counts a launch and, while profiling is on, brackets it with CUDA events.
class LaunchScope {
 public:
  LaunchScope(int kid, cudaStream_t s);
  ~LaunchScope();
  LaunchScope(const LaunchScope&) = delete;
  LaunchScope& operator=(const LaunchScope&) = delete;

 private:
  int kid_;
  cudaStream_t s_;
  void* a_;
};
#define SZ3G_LAUNCH(kid, s, ...)                    \
  do {                                              \
    ::sz3g::LaunchScope sz3g_launch_scope_((kid), (s)); \
    __VA_ARGS__;                                    \
  } while (0)

// Builds the plan; returns SZ3G_OK or SZ3G_E_INVAL.  Shared by all entry points.
int make_plan(const sz3g_params* p, Plan* plan);
void make_pass_map(const Plan& plan, PassMap* map);

// ---------------------------------------------------------------------------
// Device arithmetic of the method.
// ---------------------------------------------------------------------------

// Interpolation predictor (Sec. 6.2): a, b at -1 / +1 and c, d at -3 / +3 on
// the pass axis of the compact grid; has_* say which of b, c, d exist.
template <typename T>
__device__ __forceinline__ T interp_predict(T a, T b, T c, T d, bool has_b, bool has_c, bool has_d,
                                            int interp) {
  if (interp == SZ3G_CUBIC) {
    if (has_c && has_d) {
      T ab = a + b;
      T nine = T(9) * ab;
      T cd = c + d;
      T num = nine - cd;
      return num * T(0.0625);
    }
    if (!has_c && has_d) {
      T a3 = T(3) * a;
      T b6 = T(6) * b;
      T sum = a3 + b6;
      T num = sum - d;
      return num * T(0.125);
    }
    if (has_c && has_b) {
      T a6 = T(6) * a;
      T b3 = T(3) * b;
      T sum = a6 + b3;
      T num = sum - c;
      return num * T(0.125);
    }
  }
  if (has_b) {
    T ab = a + b;
    return ab * T(0.5);
  }
  if (has_c) {
    T a15 = T(1.5) * a;
    T c05 = T(0.5) * c;
    return a15 - c05;
  }
  return a;
}

// Truncation toward zero of a value the caller only uses when 0 <= v < 2^22
// (any other input gives an unspecified result that the caller discards).
// FP32: the sum v + 2^23 rounded toward zero is 2^23 + trunc(v), whose bits
// hold trunc(v) in the mantissa -- one full-rate add instead of a conversion.
__device__ __forceinline__ int to_int_rz(float v) { return __float_as_int(__fadd_rz(v, 8388608.0f)) - 0x4B000000; }
__device__ __forceinline__ int to_int_rz(double v) { return __double2int_rz(v); }

// (T)v for an integer |v| < 2^22, exactly.  FP32: the float whose bits are
// those of 1.5 * 2^23 plus v is 1.5 * 2^23 + v (v lands in the mantissa), so
// subtracting 1.5 * 2^23 leaves v -- integer and float adds instead of a
// conversion.
template <typename T>
__device__ __forceinline__ T small_int_to(int v) {
  if constexpr (sizeof(T) == 4) return __int_as_float(0x4B400000 + v) - 12582912.0f;
  else return T(v);
}

// Linear-scaling quantizer (Sec. 3.2): code radius + q with q the index of the
// width-2*eb bin holding x - pred (half-up), or 0 when |q| would reach the
// radius or the reconstruction misses the bound.  Evaluated without branches:
// every candidate value is computed and the result selected, so the rounding
// of each step is the same as in the sequential form
//   d = x - pred; t = |d| * ebr; if !(t < 2r - 1) -> 0;
//   h = (trunc(t) + 1) >> 1; q = sign(d) h; r = pred + (2q) * eb;
//   if !(|r - x| <= eb) -> 0; else radius + q.
template <typename T>
__device__ __forceinline__ uint32_t quantize_point(T x, T pred, T ebT, T ebr, int radius, T& recon) {
  const T d = x - pred;
  const T t = fabs(d) * ebr;
  const bool in = t < T(2 * radius - 1);  // false for NaN
  const int m = to_int_rz(t);
  const int h = (int)(((unsigned)m + 1u) >> 1);
  const int q = d < T(0) ? -h : h;
  const T q2 = small_int_to<T>((int)((unsigned)q << 1));
  const T step = q2 * ebT;
  const T r = pred + step;
  const bool ok = in && fabs(r - x) <= ebT;
  recon = ok ? r : x;
  return ok ? (uint32_t)(radius + q) : 0u;
}

// recover() (Sec. 3.2): pred + 2 (code - radius) eb.
template <typename T>
__device__ __forceinline__ T recover_point(T pred, uint32_t code, int radius, T ebT) {
  int q = (int)code - radius;
  T q2 = small_int_to<T>(2 * q);
  T step = q2 * ebT;
  return pred + step;
}

template <typename T>
__device__ __forceinline__ T bits_to(unsigned long long b);
template <>
__device__ __forceinline__ float bits_to<float>(unsigned long long b) {
  return __uint_as_float((uint32_t)b);
}
template <>
__device__ __forceinline__ double bits_to<double>(unsigned long long b) {
  return __longlong_as_double((long long)b);
}

// ---------------------------------------------------------------------------
// Launchers (host functions, defined in the .cu files).
// ---------------------------------------------------------------------------
// k_interp.cu
size_t range_scratch_bytes(const Plan& pl);
// REL with X1 (the decimated pyramid): the range pass also writes X_1 ..
// X_{kc-1}, every copy the levels read, when the field's rows allow it
// (*wrote_pyr).
int launch_range_eb(const Plan& pl, const void* d_in, DevState* st, void* scratch, size_t scratch_bytes,
                    int eb_mode, double eb, cudaStream_t s, void* X1 = nullptr, bool* wrote_pyr = nullptr);
// The grid of the coarse group (levels on it and coarser run in one CTA).
int coarse_grid(const Plan& pl);
// Cross-field work queue of grid levels (k_level.cu): with a queue, the
// level paths below launch the coarse group (and the decimated pyramid) and
// collect the finer levels of the field into the queue instead of launching
// them; level_queue_launch then runs every collected level in one
// persistent launch per type.
struct LevelQueue;
LevelQueue* level_queue_new(bool comp);
void level_queue_free(LevelQueue* q);
int level_queue_reserve(LevelQueue* q, size_t max_levels);  // device descriptors; before graph capture
int level_queue_count(const LevelQueue* q);
int level_queue_launch(LevelQueue* q, cudaStream_t s);       // descriptors built on the host, kernels on s
int level_queue_upload(LevelQueue* q);                        // descriptors to the device, before a run

int launch_quantize_levels(const Plan& pl, const void* d_in, uint16_t* codes, void* const* R,
                           uint32_t* hist, DevState* st, void* X1, bool pyr_ready, cudaStream_t s,
                           LevelQueue* lq = nullptr, int field = 0);
int launch_recover_levels(const Plan& pl, const uint16_t* codes, const void* unpred,
                          unsigned long long n_unpred, const unsigned long long* zunit,
                          void* const* R, void* d_out, DevState* st, unsigned long long ebT_bits,
                          bool codes_padded, cudaStream_t s, LevelQueue* lq = nullptr, int field = 0);

// k_level.cu (fields of rank <= 3)
// Upper bound on the CTAs of one level-kernel launch (0: one wave of the whole
// GPU).  Set while a batch graph is built, so that concurrent fields share the
// SMs; read on the host at launch time.
extern int g_level_cta_cap;
bool level_path_ok(const Plan& pl);
// Whether decompressing writes the field only from the finest level's
// register-blocked kernel, in plane-group order (3-D, rows of 16 bytes, a
// 16-byte aligned output): the field can then leave for the host in slabs.
bool recover_writes_out_once(const Plan& pl, const void* d_out);
// Copies of the field to page-locked host memory, issued on `copy` as each
// slab of the finest level's planes is done (set by the host-buffer
// decompress around its enqueue; read on the same thread).
struct SlabSink {
  void* h_out;
  cudaStream_t copy;
  int slabs;
};
extern thread_local const SlabSink* g_slab_sink;
int launch_quantize_fused(const Plan& pl, const void* d_in, uint16_t* codes, void* const* R, uint32_t* hist,
                          DevState* st, void* X1, bool pyr_ready, cudaStream_t s, LevelQueue* lq = nullptr,
                          int field = 0);
// Decimated copies of the field X_k = x[::2^k, ::2^k, ::2^k] over G_k, k >= 1
// (rows pitched to 16 bytes, one after another): the inputs of the coarser
// levels; xpyr_bytes is 0 when the level path does not use them.
inline unsigned long long xk_pitch(const Plan& pl, int k) {
  const unsigned long long al = 16 / pl.esz;
  return (pl.gm[k][3] + al - 1) / al * al;
}
inline unsigned long long xk_bytes(const Plan& pl, int k) {
  return ((xk_pitch(pl, k) * pl.gm[k][2] * pl.gm[k][1] * pl.esz) + 255) & ~255ull;
}
inline unsigned long long xpyr_offset(const Plan& pl, int k) {  // byte offset of X_k
  unsigned long long o = 0;
  for (int q = 1; q < k; ++q) o += xk_bytes(pl, q);
  return o;
}
inline unsigned long long xpyr_bytes(const Plan& pl) {
  if (pl.n[0] != 1 || pl.L < 1) return 0;
  return xpyr_offset(pl, pl.L + 1);
}
int launch_recover_fused(const Plan& pl, const uint16_t* codes, const void* unpred, unsigned long long n_unpred,
                         const unsigned long long* zunit, void* const* R, void* d_out,
                         DevState* st, unsigned long long ebT_bits, bool codes_padded, cudaStream_t s,
                         LevelQueue* lq = nullptr, int field = 0);

// k_huffman.cu: device-wide exclusive prefix sum (u32 -> u64) by decoupled look-back
size_t scan_state_bytes(unsigned long long n);
int launch_scan(const uint32_t* in, unsigned long long n, unsigned long long* out, uint32_t limit,
                unsigned long long expect, int check_expect, void* state, DevState* st, cudaStream_t s,
                bool state_zeroed);

// k_lz.cu: the optional lossless stage (byte-level LZ77 over 32 KiB blocks)
// k_pastri.cu: unpred-aware quantizer (bitplanes) and the fixed Huffman table
int bitplane_exponent(double eb, int* e);
size_t bp_state_bytes();
int launch_bitplane_encode(uint32_t dtype, const void* d_values, unsigned long long n, int e, void* d_out,
                           unsigned long long cap, void* d_state, cudaStream_t s);
int read_bitplane_state(const void* d_state, uint32_t* flags, unsigned long long* out_bytes, cudaStream_t s);
int launch_bitplane_decode(uint32_t dtype, const void* d_stream, unsigned long long n, unsigned long long W,
                           uint32_t B, int e, void* d_out, cudaStream_t s);
int launch_huffman_fixed(uint32_t radius, uint8_t* d_len, uint32_t* d_code, cudaStream_t s);
size_t lz_workspace_bytes(unsigned long long n);
int launch_lz_compress(const void* d_in, unsigned long long n, void* d_out, unsigned char* ws, cudaStream_t s,
                       DevState** st);
int launch_lz_decompress(const void* d_stream, unsigned long long bytes, unsigned long long n, void* d_out,
                         unsigned char* ws, cudaStream_t s, DevState** st);

// api.cu: the pipelines without synchronisation (also used by the batch).
struct Header {  // a parsed stream header
  sz3g_params p;
  Plan plan;
  unsigned long long n_unpred, n_words, ebT_bits;
  uint32_t n_used;
  unsigned long long off_table, off_chunks, off_sub, off_payload, end;
};
size_t compress_ws_bytes(const Plan& pl);
size_t decompress_ws_bytes(const Plan& pl);
int stream_status(uint32_t flags);
int parse_stream_header(const unsigned char* hb, size_t bytes, Header* h);
// rounds: the workspace holds the codebook's parallel-rounds scratch
// (compress_layout(pl, true)); the batch's workspaces do not
int compress_enqueue(const sz3g_params* p, const Plan& pl, const void* d_in, void* d_out, size_t out_capacity,
                     unsigned char* ws, cudaStream_t s, DevState** st, bool rounds = false);
// compress_enqueue in two parts: up to the levels (collected into lq when
// given), then the encoder.
int compress_enqueue_pre(const sz3g_params* p, const Plan& pl, const void* d_in, unsigned char* ws, cudaStream_t s,
                         DevState** st, LevelQueue* lq, int field);
int compress_enqueue_post(const sz3g_params* p, const Plan& pl, const void* d_in, void* d_out, size_t out_capacity,
                          unsigned char* ws, cudaStream_t s, bool rounds = false);
// with lq: everything but the levels collected into lq
int decompress_enqueue(const Header& h, const void* d_stream, void* d_out, unsigned char* ws, cudaStream_t s,
                       DevState** st, LevelQueue* lq = nullptr, int field = 0);

// k_huffman.cu
size_t codebook_scratch_bytes();
// rounds: scratch of the parallel length-limit rounds (codebook_rounds_bytes),
// or null for the rounds one after another
int launch_codebook(const uint32_t* hist, uint32_t nsym, uint32_t* table, uint8_t* len_out,
                    uint32_t* code_out, DevState* st, void* scratch, unsigned char* d_out,
                    unsigned long long out_capacity, int esz, cudaStream_t s, void* rounds = nullptr);
size_t codebook_rounds_bytes(unsigned long long max_symbols);  // 0: never needed
int launch_finalize(const Plan& pl, const sz3g_params* p, DevState* st, unsigned char* d_out,
                    unsigned long long out_capacity, cudaStream_t s);

// Encoder modes.
enum { kEncodeStream = 0, kEncodeRaw = 1 };

__host__ __device__ __forceinline__ unsigned long long pad8(unsigned long long x) { return (x + 7) & ~7ull; }

}  // namespace sz3g
