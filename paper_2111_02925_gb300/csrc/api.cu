// api.cu -- the extern "C" entry points declared in include/sz3g.h: argument
// checks, workspace layout, the launch sequence of compress / decompress and
// the stage entry points, and the mapping of device status bits to statuses.
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace sz3g {

DebugInject g_debug = {0u, -1, -1, 0};

// Launchers defined in k_huffman.cu that are used only here.
int launch_encode(const Plan& pl, const uint16_t* codes, const uint32_t* table, const void* d_in, const PassMap* map,
                  void* scratch, DevState* st, unsigned char* d_out, unsigned long long out_capacity, int mode,
                  uint32_t* words_out, uint32_t* chunk_words_out, uint16_t* sub_out, unsigned long long cap_words,
                  cudaStream_t s, const sz3g_params* header_p = nullptr, bool* header_written = nullptr);
int launch_compact_unpred(const Plan& pl, const uint16_t* codes, const void* d_in, const PassMap* map, void* scratch,
                          const uint32_t* table, void* d_unpred, DevState* st, cudaStream_t s);
size_t encode_scratch_bytes(unsigned long long n_chunks);
int launch_decode_tables(const unsigned char* tab, uint32_t n_used, const uint8_t* len, uint32_t nsym,
                         void* tables, DevState* st, cudaStream_t s);
int launch_decode_chunks(const uint32_t* words, unsigned long long n_words, const uint32_t* chunk_words,
                         const uint16_t* sub_bits, unsigned long long n_chunks, uint32_t chunk, unsigned long long n,
                         const void* tables, uint16_t* codes, uint32_t* zcnt, void* state, DevState* st,
                         cudaStream_t s, bool state_zeroed = false);
size_t decode_state_bytes(unsigned long long n_chunks, uint32_t chunk);
int launch_zero_counts(const uint16_t* codes, unsigned long long n, uint32_t chunk, unsigned long long n_chunks,
                       uint32_t* zcnt, cudaStream_t s);

int launch_pack_table(const uint8_t* len, const uint32_t* code, uint32_t nsym, uint32_t* table, cudaStream_t s);
size_t dec_tables_bytes();

namespace {

constexpr size_t kAlign = 256;

inline size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Bump layout of a workspace.
struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off += up(bytes);
    return o;
  }
};

struct CompressWs {
  size_t st, hist, table, range, cb, enc, codes, x1, R[34], rounds, total;
};

// rounds: room for the codebook's parallel length-limit rounds at the end
// (the single-field forms; a batch's per-field workspaces leave it out).
CompressWs compress_layout(const Plan& pl, bool rounds = true) {
  CompressWs w{};
  Layout l;
  w.st = l.take(sizeof(DevState));
  w.hist = l.take(kSyms * 4);
  w.table = l.take(kSyms * 4);
  w.range = l.take(range_scratch_bytes(pl));
  w.enc = l.take(encode_scratch_bytes(pl.n_chunks));
  // cleared at the start of every call up to here; the codebook scratch
  // needs no clearing
  w.cb = l.take(codebook_scratch_bytes());
  w.codes = l.take(pl.N * 2);
  w.x1 = l.take(xpyr_bytes(pl));
  // the fused level path never stores the finest grid's reconstruction
  for (int k = level_path_ok(pl) ? 1 : 0; k <= pl.L; ++k) w.R[k] = l.take(pl.gsize[k] * pl.esz);
  const unsigned long long max_sym = pl.N < 2ull * pl.radius ? pl.N : 2ull * pl.radius;
  const size_t rb = rounds ? codebook_rounds_bytes(max_sym) : 0;
  w.rounds = rb ? l.take(rb) : 0;
  w.total = l.off;
  return w;
}

struct DecompressWs {
  size_t st, dstate, scan2, tables, zcnt, zunit, codes, R[34], total;
};

DecompressWs decompress_layout(const Plan& pl) {
  DecompressWs w{};
  Layout l;
  w.st = l.take(sizeof(DevState));
  // the scans' look-back states next to the status block: one clear covers all three
  w.dstate = l.take(decode_state_bytes(pl.n_chunks, pl.chunk));
  w.scan2 = l.take(scan_state_bytes(pl.n_chunks * pl.nsub));
  w.tables = l.take(dec_tables_bytes());
  w.zcnt = l.take(pl.n_chunks * pl.nsub * 4);
  w.zunit = l.take(pl.n_chunks * pl.nsub * 8);
  w.codes = l.take(pl.N * 2 + 256);  // the level kernels copy whole 16-byte blocks of codes
  for (int k = 1; k <= pl.L; ++k) w.R[k] = l.take(pl.gsize[k] * pl.esz);
  w.R[0] = 0;
  w.total = l.off;
  return w;
}

// The library's stream-ordered memory pool on the current device: memory
// freed into it stays reserved for the process (release threshold: never),
// so the scratch of repeated calls is not mapped and unmapped every time.
cudaMemPool_t lib_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pl = nullptr;
    if (cudaMemPoolCreate(&pl, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    unsigned long long keep = ~0ull;
    cudaMemPoolSetAttribute(pl, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaGetLastError();
    pools[dev] = pl;
  }
  return pools[dev];
}

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s) {
  if (g_debug.alloc_fail > 0) {  // injected failure (tests)
    --g_debug.alloc_fail;
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  cudaMemPool_t pl = lib_pool();
  return pl ? cudaMallocFromPoolAsync(p, bytes, pl, s) : cudaMallocAsync(p, bytes, s);
}

// Workspace owned for the duration of one call when the caller passes none.
struct Scratch {
  void* ptr = nullptr;
  cudaStream_t s = nullptr;
  ~Scratch() {
    if (ptr) cudaFreeAsync(ptr, s);
  }
};

int get_ws(void* user, size_t user_bytes, size_t need, cudaStream_t s, Scratch& own, unsigned char** base) {
  if (user) {
    if (user_bytes < need) return SZ3G_E_CAPACITY;
    if ((uintptr_t)user % kAlign) return SZ3G_E_INVAL;
    *base = (unsigned char*)user;
    return SZ3G_OK;
  }
  own.s = s;
  if (pool_alloc(&own.ptr, need ? need : kAlign, s) != cudaSuccess) {
    cudaGetLastError();
    own.ptr = nullptr;
    return SZ3G_E_NOMEM;
  }
  *base = (unsigned char*)own.ptr;
  return SZ3G_OK;
}

__host__ __device__ inline int flags_status(uint32_t f) {
  if (f & kFlagCheck) return SZ3G_E_CHECK;  // checking build: an index went out of range
  if (f & kFlagBadBound) return SZ3G_E_INVAL;
  if (f & kFlagNonFinite) return SZ3G_E_NONFINITE;
  if (f & kFlagZeroRange) return SZ3G_E_ZERO_RANGE_REL;
  if (f & kFlagCapacity) return SZ3G_E_CAPACITY;
  if (f & kFlagTimeout) return SZ3G_E_TIMEOUT;
  if (f & kFlagCorrupt) return SZ3G_E_CORRUPT;
  return SZ3G_OK;
}

int status_of(uint32_t f) { return flags_status(f); }

// The asynchronous forms' result on the device: the run's status and (a
// compress) the stream length, 0 unless the status is SZ3G_OK.
__global__ void report_kernel(const DevState* st, unsigned long long* out_bytes, int* status) {
  if (threadIdx.x != 0) return;
  const int r = flags_status(st->flags);
  if (status) *status = r;
  if (out_bytes) *out_bytes = r == SZ3G_OK ? st->out_bytes : 0ull;
}

int launch_report(const DevState* st, unsigned long long* out_bytes, int* status, cudaStream_t s) {
  SZ3G_LAUNCH(kKReport, s, report_kernel<<<1, 32, 0, s>>>(st, out_bytes, status));
  return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
}

int read_state(const DevState* d, DevState* h, cudaStream_t s) {
  if (cudaMemcpyAsync(h, d, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess) return SZ3G_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SZ3G_E_CUDA;
  return SZ3G_OK;
}

#define SZ3G_TRY(x)                 \
  do {                              \
    int _rc = (x);                  \
    if (_rc != SZ3G_OK) return _rc; \
  } while (0)
#define SZ3G_CUDA(x)                              \
  do {                                            \
    if ((x) != cudaSuccess) {                     \
      cudaGetLastError();                         \
      return SZ3G_E_CUDA;                         \
    }                                             \
  } while (0)

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// ---- stream header parse (host) -------------------------------------------
uint64_t get_le(const unsigned char* b, int n) {
  uint64_t v = 0;
  for (int i = n - 1; i >= 0; --i) v = (v << 8) | b[i];
  return v;
}


int parse_header(const unsigned char* s, size_t bytes, Header* h) {
  std::memset(h, 0, sizeof(*h));
  if (bytes < SZ3G_HEADER_BYTES) return SZ3G_E_CORRUPT;
  if (s[0] != 'S' || s[1] != 'Z' || s[2] != '3' || s[3] != 'G') return SZ3G_E_CORRUPT;
  if (get_le(s + 4, 2) != 1) return SZ3G_E_CORRUPT;
  sz3g_params& p = h->p;
  p.dtype = s[6];
  p.ndim = s[7];
  if (p.ndim < 1 || p.ndim > 4) return SZ3G_E_CORRUPT;
  for (int i = 0; i < 4; ++i) p.dims[i] = get_le(s + 8 + 8 * i, 8);
  p.eb_mode = s[40];
  p.interp = s[41];
  p.per_level = s[42];
  p.radius = (uint32_t)get_le(s + 44, 4);
  uint64_t ebb = get_le(s + 48, 8);
  std::memcpy(&p.eb, &ebb, 8);
  p.chunk_codes = (uint32_t)get_le(s + 72, 4);
  for (int l = 0; l < SZ3G_MAX_LEVELS; ++l) {
    p.level_interp[l] = s[112 + l];
    for (int i = 0; i < 4; ++i) p.level_order[l][i] = s[144 + 4 * l + i];
  }
  for (int i = 0; i < 4; ++i) p.dim_order[i] = s[272 + i];
  if (make_plan(&p, &h->plan) != SZ3G_OK) return SZ3G_E_CORRUPT;
  const Plan& pl = h->plan;
  if ((int)s[43] != pl.L) return SZ3G_E_CORRUPT;
  h->ebT_bits = get_le(s + 64, 8);
  if (pl.esz == 4) {
    if (h->ebT_bits >> 32) return SZ3G_E_CORRUPT;
    float e;
    uint32_t u = (uint32_t)h->ebT_bits;
    std::memcpy(&e, &u, 4);
    if (!std::isnormal(e) || !(e > 0) || !std::isnormal(1.0f / e)) return SZ3G_E_CORRUPT;
  } else {
    double e;
    std::memcpy(&e, &h->ebT_bits, 8);
    if (!std::isnormal(e) || !(e > 0) || !std::isnormal(1.0 / e)) return SZ3G_E_CORRUPT;
  }
  h->n_used = (uint32_t)get_le(s + 76, 4);
  if (get_le(s + 80, 8) != pl.N) return SZ3G_E_CORRUPT;
  h->n_unpred = get_le(s + 88, 8);
  const unsigned long long nch = get_le(s + 96, 8);
  h->n_words = get_le(s + 104, 8);
  if (h->n_unpred > pl.N || nch != pl.n_chunks) return SZ3G_E_CORRUPT;
  if (h->n_used < 1 || h->n_used > 2 * pl.radius) return SZ3G_E_CORRUPT;
  if (h->n_words > pl.n_chunks * (((unsigned long long)pl.chunk * SZ3G_LMAX + 31) / 32)) return SZ3G_E_CORRUPT;
  h->off_table = SZ3G_HEADER_BYTES + pad8(h->n_unpred * pl.esz);
  h->off_chunks = h->off_table + pad8(3ull * h->n_used);
  h->off_sub = h->off_chunks + pad8(pl.n_chunks * 4);
  h->off_payload = h->off_sub + pad8(pl.n_chunks * (pl.nsub - 1) * 2);
  h->end = h->off_payload + pad8(h->n_words * 4);
  if (h->end > bytes) return SZ3G_E_CORRUPT;
  return SZ3G_OK;
}

}  // namespace

size_t compress_ws_bytes(const Plan& pl) { return compress_layout(pl, false).total; }
size_t decompress_ws_bytes(const Plan& pl) { return decompress_layout(pl).total; }
int stream_status(uint32_t flags) { return status_of(flags); }
int parse_stream_header(const unsigned char* hb, size_t bytes, Header* h) { return parse_header(hb, bytes, h); }

// The compress pipeline on stream s, without synchronising: on completion the
// status block *st holds the flags and the stream length.
int compress_enqueue_pre(const sz3g_params* p, const Plan& pl, const void* d_in, unsigned char* ws, cudaStream_t s,
                         DevState** st_out, LevelQueue* lq, int field) {
  const CompressWs L = compress_layout(pl);
  DevState* st = (DevState*)(ws + L.st);
  *st_out = st;
  SZ3G_CUDA(cudaMemsetAsync(ws, 0, L.cb, s));  // state, histogram, tables, look-back status
  void* X = xpyr_bytes(pl) ? ws + L.x1 : nullptr;
  bool pyr_ready = false;
  SZ3G_TRY(launch_range_eb(pl, d_in, st, ws + L.range, range_scratch_bytes(pl), (int)p->eb_mode, p->eb, s, X,
                           &pyr_ready));
  void* R[34];
  for (int k = 0; k <= pl.L; ++k) R[k] = (k == 0 && level_path_ok(pl)) ? nullptr : ws + L.R[k];
  uint16_t* codes = (uint16_t*)(ws + L.codes);
  uint32_t* hist = (uint32_t*)(ws + L.hist);
  SZ3G_TRY(launch_quantize_levels(pl, d_in, codes, R, hist, st, X, pyr_ready, s, lq, field));
  return SZ3G_OK;
}

int compress_enqueue_post(const sz3g_params* p, const Plan& pl, const void* d_in, void* d_out, size_t out_capacity,
                          unsigned char* ws, cudaStream_t s, bool rounds) {
  const CompressWs L = compress_layout(pl, rounds);
  DevState* st = (DevState*)(ws + L.st);
  uint16_t* codes = (uint16_t*)(ws + L.codes);
  uint32_t* hist = (uint32_t*)(ws + L.hist);
  uint32_t* table = (uint32_t*)(ws + L.table);
  SZ3G_TRY(launch_codebook(hist, 2 * pl.radius, table, nullptr, nullptr, st, ws + L.cb, (unsigned char*)d_out,
                           out_capacity, pl.esz, s, L.rounds ? ws + L.rounds : nullptr));
  PassMap map;  // kernel parameter, copied at launch
  make_pass_map(pl, &map);
  // the one-pass encoder writes the header from its last tile; otherwise a
  // finalize launch does
  bool header_written = false;
  SZ3G_TRY(launch_encode(pl, codes, table, d_in, &map, ws + L.enc, st, (unsigned char*)d_out, out_capacity,
                         kEncodeStream, nullptr, nullptr, nullptr, 0, s, p, &header_written));
  if (!header_written) SZ3G_TRY(launch_finalize(pl, p, st, (unsigned char*)d_out, out_capacity, s));
  return SZ3G_OK;
}

// The compress pipeline on s, without synchronising.
int compress_enqueue(const sz3g_params* p, const Plan& pl, const void* d_in, void* d_out, size_t out_capacity,
                     unsigned char* ws, cudaStream_t s, DevState** st_out, bool rounds) {
  SZ3G_TRY(compress_enqueue_pre(p, pl, d_in, ws, s, st_out, nullptr, 0));
  return compress_enqueue_post(p, pl, d_in, d_out, out_capacity, ws, s, rounds);
}

// The decompress pipeline of a parsed stream on s, without synchronising.
int decompress_enqueue(const Header& h, const void* d_stream, void* d_out, unsigned char* ws, cudaStream_t s,
                       DevState** st_out, LevelQueue* lq, int field) {
  const Plan& pl = h.plan;
  const DecompressWs L = decompress_layout(pl);
  DevState* st = (DevState*)(ws + L.st);
  *st_out = st;
  SZ3G_CUDA(cudaMemsetAsync(ws, 0, L.tables, s));  // status block and the scans' look-back states
  const unsigned char* base = (const unsigned char*)d_stream;
  SZ3G_TRY(launch_decode_tables(base + h.off_table, h.n_used, nullptr, 2 * pl.radius, ws + L.tables, st, s));
  uint16_t* codes = (uint16_t*)(ws + L.codes);
  SZ3G_TRY(launch_decode_chunks((const uint32_t*)(base + h.off_payload), h.n_words,
                                (const uint32_t*)(base + h.off_chunks),
                                pl.nsub > 1 ? (const uint16_t*)(base + h.off_sub) : nullptr, pl.n_chunks, pl.chunk,
                                pl.N, ws + L.tables, codes, (uint32_t*)(ws + L.zcnt), ws + L.dstate, st, s, true));
  SZ3G_TRY(launch_scan((uint32_t*)(ws + L.zcnt), pl.n_chunks * pl.nsub, (unsigned long long*)(ws + L.zunit), 0,
                       h.n_unpred, 1, ws + L.scan2, st, s, true));
  void* R[34];
  for (int k = 0; k <= pl.L; ++k) R[k] = k == 0 ? d_out : ws + L.R[k];
  SZ3G_TRY(launch_recover_levels(pl, codes, base + SZ3G_HEADER_BYTES, h.n_unpred, (unsigned long long*)(ws + L.zunit),
                                 R, d_out, st, h.ebT_bits, true, s, lq, field));
  return SZ3G_OK;
}

// ---------------------------------------------------------------------------
// Graph cache: a compress or decompress call whose workspace is the
// caller's replays the pipeline captured by an earlier call with the same
// parameters (or stream header) and buffers -- everything the host-side
// enqueue reads -- as one graph launch, without the per-kernel host work
// (tensor maps, launch configuration) between the kernels.  Not used while
// per-launch profiling is on.
// ---------------------------------------------------------------------------
namespace {

struct GraphEntry {
  std::vector<unsigned char> key;
  cudaGraphExec_t exec = nullptr;
  DevState* st = nullptr;
  unsigned long long launches = 0, tick = 0;
};

constexpr int kGraphCacheEntries = 8;
std::mutex g_gmu;
GraphEntry g_graphs[kGraphCacheEntries];
unsigned long long g_gtick = 0;
bool g_gcache_on = true;

template <typename T>
void key_add(std::vector<unsigned char>& k, const T& v) {
  const unsigned char* b = reinterpret_cast<const unsigned char*>(&v);
  k.insert(k.end(), b, b + sizeof(T));
}

// Runs `enqueue(stream, &st)` on s through the cache.
template <typename F>
int run_cached(const std::vector<unsigned char>& key, cudaStream_t s, F enqueue, DevState** st_out) {
  std::lock_guard<std::mutex> lk(g_gmu);
  for (GraphEntry& e : g_graphs)
    if (e.exec && e.key == key) {
      e.tick = ++g_gtick;
      if (cudaGraphLaunch(e.exec, s) != cudaSuccess) {
        cudaGetLastError();
        return SZ3G_E_CUDA;
      }
      count_launches(e.launches);
      *st_out = e.st;
      return SZ3G_OK;
    }
  // capture on a private stream (nothing runs), then replay on s
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return enqueue(s, st_out);
  }
  const unsigned long long l0 = launch_total();
  DevState* st = nullptr;
  int rc = SZ3G_OK;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    rc = SZ3G_E_CUDA;
  } else {
    rc = enqueue(cs, &st);
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess) rc = rc == SZ3G_OK ? SZ3G_E_CUDA : rc;
  }
  cudaStreamDestroy(cs);
  const unsigned long long launches = launch_total() - l0;
  cudaGraphExec_t exec = nullptr;
  if (rc == SZ3G_OK && g && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) exec = nullptr;
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  if (rc != SZ3G_OK || !exec) {  // not capturable: launch directly
    if (exec) cudaGraphExecDestroy(exec);
    return rc != SZ3G_OK ? rc : enqueue(s, st_out);
  }
  GraphEntry* slot = &g_graphs[0];
  for (GraphEntry& e : g_graphs)
    if (!e.exec || e.tick < slot->tick) slot = &e;
  if (slot->exec) cudaGraphExecDestroy(slot->exec);
  slot->key = key;
  slot->exec = exec;
  slot->st = st;
  slot->launches = launches;
  slot->tick = ++g_gtick;
  if (cudaGraphLaunch(exec, s) != cudaSuccess) {
    cudaGetLastError();
    return SZ3G_E_CUDA;
  }
  *st_out = st;
  return SZ3G_OK;
}

bool use_graph_cache(const void* user_ws) { return user_ws && g_gcache_on && !profiling_on(); }

void sz3g_graph_cache_clear() {
  std::lock_guard<std::mutex> lk(g_gmu);
  for (GraphEntry& e : g_graphs) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    e = GraphEntry{};
  }
}

// Decompress with the header bytes `hb` already on the host (the device
// stream holds the same bytes at its start).
int decompress_parsed(const unsigned char* hb, const void* d_stream, size_t bytes, void* d_out, size_t out_capacity,
                      void* d_workspace, size_t ws_bytes, cudaStream_t s) {
  Header h;
  SZ3G_TRY(parse_header(hb, bytes, &h));
  const Plan& pl = h.plan;
  if (out_capacity < pl.N * pl.esz) return SZ3G_E_CAPACITY;
  const DecompressWs L = decompress_layout(pl);
  Scratch own;
  unsigned char* ws;
  SZ3G_TRY(get_ws(d_workspace, ws_bytes, L.total, s, own, &ws));
  DevState* st = nullptr;
  if (use_graph_cache(d_workspace)) {
    std::vector<unsigned char> key;
    int dev = 0;
    cudaGetDevice(&dev);
    key_add(key, 'D');
    key_add(key, dev);
    key.insert(key.end(), hb, hb + SZ3G_HEADER_BYTES);
    key_add(key, bytes);
    key_add(key, d_stream);
    key_add(key, d_out);
    key_add(key, out_capacity);
    key_add(key, d_workspace);
    key_add(key, ws_bytes);
    if (g_slab_sink) {  // the graph holds the copies to this host buffer
      key_add(key, g_slab_sink->h_out);
      key_add(key, g_slab_sink->slabs);
    }
    SZ3G_TRY(run_cached(
        key, s, [&](cudaStream_t es, DevState** sto) { return decompress_enqueue(h, d_stream, d_out, ws, es, sto); },
        &st));
  } else {
    SZ3G_TRY(decompress_enqueue(h, d_stream, d_out, ws, s, &st));
  }
  DevState hs;
  SZ3G_TRY(read_state(st, &hs, s));
  return status_of(hs.flags);
}

// Device buffers the host-buffer entry points stage through: one set per
// device, kept between calls and grown on demand, so that repeated calls on
// fields of one shape reuse the same addresses and with them the cached graph
// of the pipeline.  A call that finds the set in use by another thread stages
// through pool memory of its own instead.
struct Staging {
  std::mutex mu;
  void* buf[3] = {nullptr, nullptr, nullptr};
  size_t cap[3] = {0, 0, 0};
};
constexpr int kStageDevices = 64;
constexpr int kOutputSlabs = 8;  // slabs of planes the host-buffer decompress copies out one by one
Staging g_stage[kStageDevices];

Staging* staging_of_current() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStageDevices) {
    cudaGetLastError();
    return nullptr;
  }
  return &g_stage[dev];
}

// Slot i of a held set with at least `bytes` (rounded up to 2 MiB); the old
// buffer is released in stream order on s.
int stage_reserve(Staging& g, int i, size_t bytes, cudaStream_t s, void** out) {
  bytes = (bytes + (2u << 20) - 1) & ~(size_t)((2u << 20) - 1);
  if (g.cap[i] < bytes) {
    if (g.buf[i]) cudaFreeAsync(g.buf[i], s);
    g.buf[i] = nullptr;
    g.cap[i] = 0;
    if (pool_alloc(&g.buf[i], bytes, s) != cudaSuccess) {
      cudaGetLastError();
      g.buf[i] = nullptr;
      return SZ3G_E_NOMEM;
    }
    g.cap[i] = bytes;
  }
  *out = g.buf[i];
  return SZ3G_OK;
}

// Releases every staging set and returns the pool's free memory of each
// device that held one.
void staging_release_all() {
  int cur = 0;
  cudaGetDevice(&cur);
  for (int d = 0; d < kStageDevices; ++d) {
    Staging& g = g_stage[d];
    std::lock_guard<std::mutex> lk(g.mu);
    if (!g.buf[0] && !g.buf[1] && !g.buf[2]) continue;
    if (cudaSetDevice(d) != cudaSuccess) continue;
    cudaDeviceSynchronize();
    for (int i = 0; i < 3; ++i) {
      if (g.buf[i]) cudaFreeAsync(g.buf[i], 0);
      g.buf[i] = nullptr;
      g.cap[i] = 0;
    }
    cudaDeviceSynchronize();
    if (cudaMemPool_t pl = lib_pool()) cudaMemPoolTrimTo(pl, 0);
  }
  cudaSetDevice(cur);
  cudaGetLastError();
}

}  // namespace

}  // namespace sz3g

using namespace sz3g;

extern "C" {

const char* sz3g_strerror(int status) {
  switch (status) {
    case SZ3G_OK: return "ok";
    case SZ3G_E_INVAL: return "invalid argument (dims, error bound, radius, order, chunk or alignment)";
    case SZ3G_E_NONFINITE: return "input field holds NaN or Inf";
    case SZ3G_E_ZERO_RANGE_REL: return "relative error bound on a field whose value range is zero";
    case SZ3G_E_CAPACITY: return "output buffer or workspace too small";
    case SZ3G_E_CORRUPT: return "stream is corrupt or truncated";
    case SZ3G_E_CUDA: return "a CUDA runtime call failed";
    case SZ3G_E_NOMEM: return "device allocation failed";
    case SZ3G_E_TIMEOUT: return "a bounded wait inside a kernel gave up";
    case SZ3G_E_CHECK: return "an index check inside a kernel failed (checking build)";
    default: return "unknown status";
  }
}

int sz3g_compress_bound(const sz3g_params* p, size_t* max_bytes) {
  Plan pl;
  SZ3G_TRY(make_plan(p, &pl));
  if (!max_bytes) return SZ3G_E_INVAL;
  const unsigned long long maxw = ((unsigned long long)pl.chunk * SZ3G_LMAX + 31) / 32;
  *max_bytes = SZ3G_HEADER_BYTES + pad8(pl.N * pl.esz) + pad8(2ull * pl.radius * 3) + pad8(pl.n_chunks * 4) +
               pad8(pl.n_chunks * (pl.nsub - 1) * 2) + pad8(pl.n_chunks * maxw * 4);
  return SZ3G_OK;
}

int sz3g_workspace_size(const sz3g_params* p, int for_decompress, size_t* bytes) {
  Plan pl;
  SZ3G_TRY(make_plan(p, &pl));
  if (!bytes) return SZ3G_E_INVAL;
  *bytes = for_decompress ? decompress_layout(pl).total : compress_layout(pl).total;
  return SZ3G_OK;
}

int sz3g_compress(const sz3g_params* p, const void* d_in, void* d_out, size_t out_capacity, size_t* out_bytes,
                  void* d_workspace, size_t ws_bytes, void* stream) {
  SZ3G_TRACE("sz3g_compress");
  Plan pl;
  SZ3G_TRY(make_plan(p, &pl));
  if (!d_in || !d_out || !out_bytes || !aligned(d_in, 16) || !aligned(d_out, 16)) return SZ3G_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const CompressWs L = compress_layout(pl);
  Scratch own;
  unsigned char* ws;
  SZ3G_TRY(get_ws(d_workspace, ws_bytes, L.total, s, own, &ws));
  DevState* st = nullptr;
  if (use_graph_cache(d_workspace)) {
    std::vector<unsigned char> key;
    int dev = 0;
    cudaGetDevice(&dev);
    key_add(key, 'C');
    key_add(key, dev);
    key_add(key, *p);
    key_add(key, d_in);
    key_add(key, d_out);
    key_add(key, out_capacity);
    key_add(key, d_workspace);
    key_add(key, ws_bytes);
    SZ3G_TRY(run_cached(
        key, s,
        [&](cudaStream_t es, DevState** sto) {
          return compress_enqueue(p, pl, d_in, d_out, out_capacity, ws, es, sto, true);
        },
        &st));
  } else {
    SZ3G_TRY(compress_enqueue(p, pl, d_in, d_out, out_capacity, ws, s, &st, true));
  }
  DevState h;
  SZ3G_TRY(read_state(st, &h, s));
  SZ3G_TRY(status_of(h.flags));
  *out_bytes = (size_t)h.out_bytes;
  return SZ3G_OK;
}

int sz3g_lossless_bound(uint64_t n, uint64_t* max_bytes) {
  if (!max_bytes) return SZ3G_E_INVAL;
  const uint64_t nb = (n + SZ3G_LZ_BLOCK - 1) / SZ3G_LZ_BLOCK;
  *max_bytes = SZ3G_LZ_HEADER + 8 * nb + 8 + n;
  return SZ3G_OK;
}

int sz3g_lossless_compress(const void* d_in, uint64_t n, void* d_out, size_t out_capacity, size_t* out_bytes,
                           void* stream) {
  if (!d_out || !out_bytes || (n && !d_in) || !aligned(d_out, 16) || (n && !aligned(d_in, 16)) ||
      (n + SZ3G_LZ_BLOCK - 1) / SZ3G_LZ_BLOCK > 0x7fffffffull)
    return SZ3G_E_INVAL;
  uint64_t bound = 0;
  sz3g_lossless_bound(n, &bound);
  if (out_capacity < bound) return SZ3G_E_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch own;
  unsigned char* ws;
  SZ3G_TRY(get_ws(nullptr, 0, lz_workspace_bytes(n), s, own, &ws));
  DevState* st = nullptr;
  SZ3G_TRY(launch_lz_compress(d_in, n, d_out, ws, s, &st));
  DevState h;
  SZ3G_TRY(read_state(st, &h, s));
  SZ3G_TRY(status_of(h.flags));
  *out_bytes = (size_t)h.out_bytes;
  return SZ3G_OK;
}

int sz3g_lossless_decompress(const void* d_stream, size_t bytes, void* d_out, size_t out_capacity, uint64_t* n_out,
                             void* stream) {
  if (!d_stream || !d_out || !aligned(d_stream, 16) || !aligned(d_out, 16)) return SZ3G_E_INVAL;
  if (bytes < SZ3G_LZ_HEADER) return SZ3G_E_CORRUPT;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char hb[SZ3G_LZ_HEADER];
  SZ3G_CUDA(cudaMemcpyAsync(hb, d_stream, SZ3G_LZ_HEADER, cudaMemcpyDeviceToHost, s));
  SZ3G_CUDA(cudaStreamSynchronize(s));
  uint32_t bs = 0, nblk = 0;
  uint64_t n = 0;
  std::memcpy(&bs, hb + 4, 4);
  std::memcpy(&n, hb + 8, 8);
  std::memcpy(&nblk, hb + 16, 4);
  if (std::memcmp(hb, "SZLZ", 4) != 0 || bs != SZ3G_LZ_BLOCK || nblk != (n + SZ3G_LZ_BLOCK - 1) / SZ3G_LZ_BLOCK ||
      ((SZ3G_LZ_HEADER + 4ull * nblk + 7) & ~7ull) > bytes)
    return SZ3G_E_CORRUPT;
  if (n > out_capacity) return SZ3G_E_CAPACITY;
  Scratch own;
  unsigned char* ws;
  SZ3G_TRY(get_ws(nullptr, 0, lz_workspace_bytes(n), s, own, &ws));
  DevState* st = nullptr;
  SZ3G_TRY(launch_lz_decompress(d_stream, bytes, n, d_out, ws, s, &st));
  DevState h;
  SZ3G_TRY(read_state(st, &h, s));
  SZ3G_TRY(status_of(h.flags));
  if (n_out) *n_out = n;
  return SZ3G_OK;
}

int sz3g_bitplane_bound(uint64_t n, uint64_t* max_bytes) {
  if (!max_bytes) return SZ3G_E_INVAL;
  *max_bytes = SZ3G_BP_HEADER + 4ull * ((n + 31) / 32) * 64ull;
  return SZ3G_OK;
}

int sz3g_bitplane_encode(uint32_t dtype, const void* d_values, uint64_t n, double eb, void* d_out,
                         size_t out_capacity, size_t* out_bytes, void* stream) {
  int e = 0;
  if (dtype > SZ3G_F64 || !d_out || !out_bytes || (n && !d_values) || !aligned(d_out, 16) ||
      (n && !aligned(d_values, dtype == SZ3G_F32 ? 4 : 8)) || n > (1ull << 40))
    return SZ3G_E_INVAL;
  SZ3G_TRY(bitplane_exponent(eb, &e));
  cudaStream_t s = (cudaStream_t)stream;
  Scratch own;
  unsigned char* ws;
  SZ3G_TRY(get_ws(nullptr, 0, bp_state_bytes(), s, own, &ws));
  SZ3G_TRY(launch_bitplane_encode(dtype, d_values, n, e, d_out, out_capacity, ws, s));
  uint32_t flags = 0;
  unsigned long long nb = 0;
  SZ3G_TRY(read_bitplane_state(ws, &flags, &nb, s));
  if (flags & kFlagNonFinite) return SZ3G_E_NONFINITE;  // before a too-wide value
  SZ3G_TRY(status_of(flags));
  *out_bytes = (size_t)nb;
  return SZ3G_OK;
}

int sz3g_bitplane_decode(const void* d_stream, size_t bytes, void* d_out, size_t out_capacity, uint64_t* n_out,
                         void* stream) {
  if (!d_stream || !aligned(d_stream, 16)) return SZ3G_E_INVAL;
  if (bytes < SZ3G_BP_HEADER) return SZ3G_E_CORRUPT;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char hb[SZ3G_BP_HEADER];
  SZ3G_CUDA(cudaMemcpyAsync(hb, d_stream, SZ3G_BP_HEADER, cudaMemcpyDeviceToHost, s));
  SZ3G_CUDA(cudaStreamSynchronize(s));
  uint32_t dtype = 0, B = 0, eu = 0;
  uint64_t n = 0, W = 0;
  std::memcpy(&dtype, hb + 4, 4);
  std::memcpy(&n, hb + 8, 8);
  std::memcpy(&eu, hb + 16, 4);
  std::memcpy(&B, hb + 20, 4);
  std::memcpy(&W, hb + 24, 8);
  if (std::memcmp(hb, "SZBP", 4) != 0 || dtype > SZ3G_F64 || B > 62 || n > (1ull << 40) || W != (n + 31) / 32 ||
      bytes < SZ3G_BP_HEADER + 4ull * W * (1ull + B))
    return SZ3G_E_CORRUPT;
  const size_t esz = dtype == SZ3G_F32 ? 4 : 8;
  if (n * esz > out_capacity || (n && !d_out)) return SZ3G_E_CAPACITY;
  if (n && !aligned(d_out, esz)) return SZ3G_E_INVAL;
  SZ3G_TRY(launch_bitplane_decode(dtype, d_stream, n, W, B, (int)(int32_t)eu, d_out, s));
  SZ3G_CUDA(cudaStreamSynchronize(s));
  if (n_out) *n_out = n;
  return SZ3G_OK;
}

int sz3g_huffman_fixed(uint32_t radius, uint8_t* d_len, uint32_t* d_code, void* stream) {
  if (radius < 2 || radius > 32768 || !d_len || !d_code) return SZ3G_E_INVAL;
  SZ3G_TRY(launch_huffman_fixed(radius, d_len, d_code, (cudaStream_t)stream));
  return SZ3G_OK;
}

int sz3g_debug_inject(int kind, long long value) {
  switch (kind) {
    case SZ3G_DEBUG_RESET:
      g_debug = DebugInject{0u, -1, -1, 0};
      return SZ3G_OK;
    case SZ3G_DEBUG_WAIT_LIMIT:
      if (value < 0 || value > 0x7fffffffll) return SZ3G_E_INVAL;
      g_debug.wait_limit = (uint32_t)value;
      return SZ3G_OK;
    case SZ3G_DEBUG_QUEUE_STALL:
      g_debug.queue_stall = value < 0 ? -1 : value;
      return SZ3G_OK;
    case SZ3G_DEBUG_SILENT_CHUNK:
      g_debug.silent_chunk = value < 0 ? -1 : value;
      return SZ3G_OK;
    case SZ3G_DEBUG_ALLOC_FAIL:
      if (value < 0 || value > 0x7fffffffll) return SZ3G_E_INVAL;
      g_debug.alloc_fail = (int)value;
      return SZ3G_OK;
    default:
      return SZ3G_E_INVAL;
  }
}

int sz3g_graph_cache(int on) {
  {
    std::lock_guard<std::mutex> lk(g_gmu);
    g_gcache_on = on != 0;
  }
  if (!on) sz3g_graph_cache_clear();
  return SZ3G_OK;
}

int sz3g_read_header(const void* stream, size_t bytes, int stream_on_device, sz3g_params* p, uint64_t* n_points) {
  if (!stream || !p) return SZ3G_E_INVAL;
  unsigned char hb[SZ3G_HEADER_BYTES];
  if (bytes < SZ3G_HEADER_BYTES) return SZ3G_E_CORRUPT;
  if (stream_on_device) {
    SZ3G_CUDA(cudaMemcpy(hb, stream, SZ3G_HEADER_BYTES, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(hb, stream, SZ3G_HEADER_BYTES);
  }
  Header h;
  SZ3G_TRY(parse_header(hb, bytes, &h));
  *p = h.p;
  if (n_points) *n_points = h.plan.N;
  return SZ3G_OK;
}

int sz3g_decompress(const void* d_stream, size_t bytes, void* d_out, size_t out_capacity, void* d_workspace,
                    size_t ws_bytes, void* stream) {
  SZ3G_TRACE("sz3g_decompress");
  if (!d_stream || !d_out || !aligned(d_stream, 16) || !aligned(d_out, 16)) return SZ3G_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char hb[SZ3G_HEADER_BYTES];
  if (bytes < SZ3G_HEADER_BYTES) return SZ3G_E_CORRUPT;
  SZ3G_CUDA(cudaMemcpyAsync(hb, d_stream, SZ3G_HEADER_BYTES, cudaMemcpyDeviceToHost, s));
  SZ3G_CUDA(cudaStreamSynchronize(s));
  return decompress_parsed(hb, d_stream, bytes, d_out, out_capacity, d_workspace, ws_bytes, s);
}

namespace {

// The library's stream for copies that overlap a pipeline, one per device.
cudaStream_t copy_stream_of_current() {
  static std::mutex mu;
  static cudaStream_t streams[kStageDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStageDevices) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    streams[dev] = nullptr;
  }
  return streams[dev];
}

// Whether [h, h + n) is page-locked host memory (copies from the device into
// it can run asynchronously and inside a graph).
bool host_locked(const void* h, size_t n) {
  if (!h || !n) return false;
  cudaPointerAttributes a0, a1;
  if (cudaPointerGetAttributes(&a0, h) != cudaSuccess ||
      cudaPointerGetAttributes(&a1, (const unsigned char*)h + (n - 1)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a0.type == cudaMemoryTypeHost && a1.type == cudaMemoryTypeHost;
}

// Holds the current device's staging set for one host-buffer call, if no
// other thread has it; on release the stream is synchronised first, so that
// no copy or kernel of an abandoned call still touches the buffers.
struct StageHold {
  Staging* g = nullptr;
  cudaStream_t s = nullptr;
  explicit StageHold(cudaStream_t st) : s(st) {
    Staging* c = staging_of_current();
    if (c && c->mu.try_lock()) g = c;
  }
  ~StageHold() {
    if (!g) return;
    cudaStreamSynchronize(s);
    g->mu.unlock();
  }
};

}  // namespace

int sz3g_compress_async(const sz3g_params* p, const void* d_in, void* d_out, size_t out_capacity,
                        unsigned long long* d_out_bytes, int* d_status, void* d_workspace, size_t ws_bytes,
                        void* stream) {
  SZ3G_TRACE("sz3g_compress_async");
  Plan pl;
  SZ3G_TRY(make_plan(p, &pl));
  if (!d_in || !d_out || !d_status || !d_workspace || !aligned(d_in, 16) || !aligned(d_out, 16) ||
      !aligned(d_workspace, kAlign) || (d_out_bytes && !aligned(d_out_bytes, 8)) || !aligned(d_status, 4))
    return SZ3G_E_INVAL;
  const CompressWs L = compress_layout(pl);
  if (ws_bytes < L.total) return SZ3G_E_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  DevState* st = nullptr;
  SZ3G_TRY(compress_enqueue(p, pl, d_in, d_out, out_capacity, (unsigned char*)d_workspace, s, &st, true));
  return launch_report(st, d_out_bytes, d_status, s);
}

int sz3g_decompress_async(const void* h_header, const void* d_stream, size_t bytes, void* d_out,
                          size_t out_capacity, int* d_status, void* d_workspace, size_t ws_bytes, void* stream) {
  SZ3G_TRACE("sz3g_decompress_async");
  if (!h_header || !d_stream || !d_out || !d_status || !d_workspace || !aligned(d_stream, 16) ||
      !aligned(d_out, 16) || !aligned(d_workspace, kAlign) || !aligned(d_status, 4))
    return SZ3G_E_INVAL;
  if (bytes < SZ3G_HEADER_BYTES) return SZ3G_E_CORRUPT;
  Header h;
  SZ3G_TRY(parse_header((const unsigned char*)h_header, bytes, &h));
  if (out_capacity < h.plan.N * h.plan.esz) return SZ3G_E_CAPACITY;
  if (ws_bytes < decompress_layout(h.plan).total) return SZ3G_E_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  DevState* st = nullptr;
  SZ3G_TRY(decompress_enqueue(h, d_stream, d_out, (unsigned char*)d_workspace, s, &st));
  return launch_report(st, nullptr, d_status, s);
}

int sz3g_compress_host(const sz3g_params* p, const void* h_in, void* h_out, size_t out_capacity, size_t* out_bytes,
                       void* stream) {
  SZ3G_TRACE("sz3g_compress_host");
  Plan pl;
  SZ3G_TRY(make_plan(p, &pl));
  if (!h_in || !h_out || !out_bytes) return SZ3G_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  size_t bound;
  SZ3G_TRY(sz3g_compress_bound(p, &bound));
  const size_t in_bytes = pl.N * pl.esz, ws_bytes = compress_layout(pl).total;
  StageHold hold(s);
  Scratch din, dout;
  void *d_in = nullptr, *d_out = nullptr, *d_ws = nullptr;
  if (hold.g) {
    SZ3G_TRY(stage_reserve(*hold.g, 0, in_bytes, s, &d_in));
    SZ3G_TRY(stage_reserve(*hold.g, 1, bound, s, &d_out));
    SZ3G_TRY(stage_reserve(*hold.g, 2, ws_bytes, s, &d_ws));
  } else {
    din.s = dout.s = s;
    if (pool_alloc(&din.ptr, in_bytes, s) != cudaSuccess || pool_alloc(&dout.ptr, bound, s) != cudaSuccess) {
      cudaGetLastError();
      return SZ3G_E_NOMEM;
    }
    d_in = din.ptr;
    d_out = dout.ptr;
  }
  SZ3G_CUDA(cudaMemcpyAsync(d_in, h_in, in_bytes, cudaMemcpyHostToDevice, s));
  size_t nb = 0;
  SZ3G_TRY(sz3g_compress(p, d_in, d_out, bound, &nb, d_ws, d_ws ? hold.g->cap[2] : 0, stream));
  if (nb > out_capacity) return SZ3G_E_CAPACITY;
  SZ3G_CUDA(cudaMemcpyAsync(h_out, d_out, nb, cudaMemcpyDeviceToHost, s));
  SZ3G_CUDA(cudaStreamSynchronize(s));
  *out_bytes = nb;
  return SZ3G_OK;
}

int sz3g_decompress_host(const void* h_stream, size_t bytes, void* h_out, size_t out_capacity, void* stream) {
  SZ3G_TRACE("sz3g_decompress_host");
  if (!h_stream || !h_out) return SZ3G_E_INVAL;
  if (bytes < SZ3G_HEADER_BYTES) return SZ3G_E_CORRUPT;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char hb[SZ3G_HEADER_BYTES];
  std::memcpy(hb, h_stream, SZ3G_HEADER_BYTES);
  Header h;
  SZ3G_TRY(parse_header(hb, bytes, &h));
  const size_t out_bytes = h.plan.N * h.plan.esz, ws_bytes = decompress_layout(h.plan).total;
  if (out_capacity < out_bytes) return SZ3G_E_CAPACITY;
  StageHold hold(s);
  Scratch dst, dout;
  void *d_st = nullptr, *d_out = nullptr, *d_ws = nullptr;
  if (hold.g) {
    SZ3G_TRY(stage_reserve(*hold.g, 0, out_bytes, s, &d_out));
    SZ3G_TRY(stage_reserve(*hold.g, 1, bytes, s, &d_st));
    SZ3G_TRY(stage_reserve(*hold.g, 2, ws_bytes, s, &d_ws));
  } else {
    dst.s = dout.s = s;
    if (pool_alloc(&dst.ptr, bytes, s) != cudaSuccess || pool_alloc(&dout.ptr, out_bytes, s) != cudaSuccess) {
      cudaGetLastError();
      return SZ3G_E_NOMEM;
    }
    d_st = dst.ptr;
    d_out = dout.ptr;
  }
  SZ3G_CUDA(cudaMemcpyAsync(d_st, h_stream, bytes, cudaMemcpyHostToDevice, s));
  // A page-locked output of a field whose finest level runs on the
  // register-blocked kernel leaves in slabs of planes, each copied while the
  // later slabs are still computed.  Only the holder of the staging set uses
  // the copy stream, so no two calls ever share it (one may be capturing).
  cudaStream_t cs = nullptr;
  const bool slabbed = hold.g && recover_writes_out_once(h.plan, d_out) && host_locked(h_out, out_bytes) &&
                       (cs = copy_stream_of_current()) != nullptr;
  SlabSink sink{h_out, cs, kOutputSlabs};
  g_slab_sink = slabbed ? &sink : nullptr;
  const int rc = decompress_parsed(hb, d_st, bytes, d_out, out_bytes, d_ws, d_ws ? hold.g->cap[2] : 0, s);
  g_slab_sink = nullptr;
  SZ3G_TRY(rc);
  if (!slabbed) SZ3G_CUDA(cudaMemcpyAsync(h_out, d_out, out_bytes, cudaMemcpyDeviceToHost, s));
  SZ3G_CUDA(cudaStreamSynchronize(s));
  return SZ3G_OK;
}

int sz3g_trim(void) {
  sz3g_graph_cache_clear();
  staging_release_all();
  return SZ3G_OK;
}

int sz3g_predict_quantize(const sz3g_params* p, const void* d_in, uint16_t* d_codes, void* d_unpred,
                          uint32_t* d_hist, uint64_t* h_n_unpred, void* h_ebT, void* d_workspace, size_t ws_bytes,
                          void* stream) {
  SZ3G_TRACE("sz3g_predict_quantize");
  Plan pl;
  SZ3G_TRY(make_plan(p, &pl));
  if (!d_in || !d_codes || !d_unpred || !d_hist || !aligned(d_in, 16) || !aligned(d_codes, 16)) return SZ3G_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const CompressWs L = compress_layout(pl);
  Scratch own;
  unsigned char* ws;
  SZ3G_TRY(get_ws(d_workspace, ws_bytes, L.total, s, own, &ws));
  DevState* st = (DevState*)(ws + L.st);
  SZ3G_CUDA(cudaMemsetAsync(ws, 0, L.cb, s));
  SZ3G_CUDA(cudaMemsetAsync(d_hist, 0, kSyms * 4, s));
  SZ3G_TRY(launch_range_eb(pl, d_in, st, ws + L.range, range_scratch_bytes(pl), (int)p->eb_mode, p->eb, s));
  void* R[34];
  for (int k = 0; k <= pl.L; ++k) R[k] = (k == 0 && level_path_ok(pl)) ? nullptr : ws + L.R[k];
  SZ3G_TRY(launch_quantize_levels(pl, d_in, d_codes, R, d_hist, st, xpyr_bytes(pl) ? ws + L.x1 : nullptr, false, s));
  PassMap map;
  make_pass_map(pl, &map);
  SZ3G_TRY(launch_compact_unpred(pl, d_codes, d_in, &map, ws + L.enc, (uint32_t*)(ws + L.table), d_unpred, st, s));
  DevState h;
  SZ3G_TRY(read_state(st, &h, s));
  SZ3G_TRY(status_of(h.flags));
  if (h_n_unpred) *h_n_unpred = h.n_unpred;
  if (h_ebT) std::memcpy(h_ebT, &h.ebT_bits, 8);
  return SZ3G_OK;
}

int sz3g_recover(const sz3g_params* p, const void* h_ebT, const uint16_t* d_codes, const void* d_unpred,
                 uint64_t n_unpred, void* d_out, void* d_workspace, size_t ws_bytes, void* stream) {
  SZ3G_TRACE("sz3g_recover");
  Plan pl;
  SZ3G_TRY(make_plan(p, &pl));
  if (!h_ebT || !d_codes || !d_out || (n_unpred && !d_unpred) || !aligned(d_codes, 16)) return SZ3G_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const DecompressWs L = decompress_layout(pl);
  Scratch own;
  unsigned char* ws;
  SZ3G_TRY(get_ws(d_workspace, ws_bytes, L.total, s, own, &ws));
  DevState* st = (DevState*)(ws + L.st);
  SZ3G_CUDA(cudaMemsetAsync(st, 0, sizeof(DevState), s));
  SZ3G_TRY(launch_zero_counts(d_codes, pl.N, pl.chunk, pl.n_chunks, (uint32_t*)(ws + L.zcnt), s));
  SZ3G_TRY(launch_scan((uint32_t*)(ws + L.zcnt), pl.n_chunks * pl.nsub, (unsigned long long*)(ws + L.zunit), 0,
                       n_unpred, 1, ws + L.scan2, st, s, false));
  unsigned long long eb_bits = 0;
  std::memcpy(&eb_bits, h_ebT, pl.esz);
  void* R[34];
  for (int k = 0; k <= pl.L; ++k) R[k] = k == 0 ? d_out : ws + L.R[k];
  SZ3G_TRY(launch_recover_levels(pl, d_codes, d_unpred, n_unpred, (unsigned long long*)(ws + L.zunit), R, d_out,
                                 st, eb_bits, false, s));
  DevState h;
  SZ3G_TRY(read_state(st, &h, s));
  return status_of(h.flags);
}

int sz3g_huffman_build(const uint32_t* d_hist, uint32_t nsym, uint8_t* d_len, uint32_t* d_code, void* stream) {
  SZ3G_TRACE("sz3g_huffman_build");
  if (!d_hist || !d_len || !d_code || nsym < 1 || nsym > (uint32_t)kSyms) return SZ3G_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Layout l;
  const size_t o_st = l.take(sizeof(DevState)), o_tab = l.take(kSyms * 4), o_cb = l.take(codebook_scratch_bytes());
  const size_t rb = codebook_rounds_bytes(nsym), o_rounds = rb ? l.take(rb) : 0;
  Scratch own;
  unsigned char* ws;
  SZ3G_TRY(get_ws(nullptr, 0, l.off, s, own, &ws));
  DevState* st = (DevState*)(ws + o_st);
  SZ3G_CUDA(cudaMemsetAsync(st, 0, sizeof(DevState), s));
  SZ3G_TRY(launch_codebook(d_hist, nsym, (uint32_t*)(ws + o_tab), d_len, d_code, st, ws + o_cb, nullptr, 0, 4, s,
                           rb ? ws + o_rounds : nullptr));
  DevState h;
  SZ3G_TRY(read_state(st, &h, s));
  return status_of(h.flags);
}

int sz3g_huffman_encode(const uint16_t* d_codes, uint64_t n, const uint8_t* d_len, const uint32_t* d_code,
                        uint32_t nsym, uint32_t chunk, uint32_t* d_words, uint64_t cap_words,
                        uint32_t* d_chunk_words, uint16_t* d_sub_bits, uint64_t* h_n_words, void* stream) {
  SZ3G_TRACE("sz3g_huffman_encode");
  if (!d_codes || !d_len || !d_code || !d_words || !d_chunk_words || n < 1 || nsym < 1 || nsym > (uint32_t)kSyms ||
      chunk < 8 || chunk > 65536 || chunk % 8 || !aligned(d_codes, 16))
    return SZ3G_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Plan pl;
  std::memset(&pl, 0, sizeof(pl));
  pl.N = n;
  pl.chunk = chunk;
  pl.n_chunks = (n + chunk - 1) / chunk;
  pl.nsub = (chunk + SZ3G_SUBBLOCK - 1) / SZ3G_SUBBLOCK;
  pl.esz = 4;
  Layout l;
  const size_t o_st = l.take(sizeof(DevState)), o_tab = l.take(kSyms * 4),
               o_enc = l.take(encode_scratch_bytes(pl.n_chunks));
  Scratch own;
  unsigned char* ws;
  SZ3G_TRY(get_ws(nullptr, 0, l.off, s, own, &ws));
  DevState* st = (DevState*)(ws + o_st);
  SZ3G_CUDA(cudaMemsetAsync(ws, 0, l.off, s));
  SZ3G_TRY(launch_pack_table(d_len, d_code, nsym, (uint32_t*)(ws + o_tab), s));
  PassMap map;  // unused in this mode
  std::memset(&map, 0, sizeof(map));
  map.n = 1;
  for (int d = 0; d < 4; ++d) map.e[0].E[d] = 1;
  SZ3G_TRY(launch_encode(pl, d_codes, (uint32_t*)(ws + o_tab), nullptr, &map, ws + o_enc, st, nullptr, 0, kEncodeRaw,
                         d_words, d_chunk_words, d_sub_bits, cap_words, s));
  DevState h;
  SZ3G_TRY(read_state(st, &h, s));
  SZ3G_TRY(status_of(h.flags));
  if (h_n_words) *h_n_words = h.n_words;
  return SZ3G_OK;
}

int sz3g_huffman_decode(const uint32_t* d_words, uint64_t n_words, const uint32_t* d_chunk_words,
                        const uint16_t* d_sub_bits, uint32_t chunk, const uint8_t* d_len, uint32_t nsym,
                        uint16_t* d_codes, uint64_t n, void* stream) {
  SZ3G_TRACE("sz3g_huffman_decode");
  if (!d_words || !d_chunk_words || !d_len || !d_codes || n < 1 || nsym < 1 || nsym > (uint32_t)kSyms || chunk < 8 ||
      chunk > 65536 || chunk % 8 || !aligned(d_codes, 16))
    return SZ3G_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned long long nch = (n + chunk - 1) / chunk, nsb = (chunk + SZ3G_SUBBLOCK - 1) / SZ3G_SUBBLOCK;
  Layout l;
  const size_t o_st = l.take(sizeof(DevState)), o_t = l.take(dec_tables_bytes()), o_zc = l.take(nch * nsb * 4),
               o_sc = l.take(decode_state_bytes(nch, chunk));
  Scratch own;
  unsigned char* ws;
  SZ3G_TRY(get_ws(nullptr, 0, l.off, s, own, &ws));
  DevState* st = (DevState*)(ws + o_st);
  SZ3G_CUDA(cudaMemsetAsync(st, 0, sizeof(DevState), s));
  SZ3G_TRY(launch_decode_tables(nullptr, 0, d_len, nsym, ws + o_t, st, s));
  SZ3G_TRY(launch_decode_chunks(d_words, n_words, d_chunk_words, d_sub_bits, nch, chunk, n, ws + o_t, d_codes,
                                (uint32_t*)(ws + o_zc), ws + o_sc, st, s));
  DevState h;
  SZ3G_TRY(read_state(st, &h, s));
  return status_of(h.flags);
}

}  // extern "C"
