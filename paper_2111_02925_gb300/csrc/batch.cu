// batch.cu -- many fields of uneven shape and error bound compressed (or
// decompressed) by one call.
//
// A batch is planned once for a fixed set of buffers.  Fields are spread over
// B branches (largest first, each to the branch with the least work so far);
// each branch owns one workspace sized for its largest field and runs its
// fields one after another; the branches run concurrently.  Every launch of
// every field -- the whole pipeline, with no host synchronisation between
// fields -- is captured once into a CUDA graph that each run replays, and a
// small kernel after each field copies its status block into a per-field
// result array.  The number of branches and the CTA cap of the level kernels
// (so that concurrent fields share the SMs) are chosen by sz3g_batch_tune,
// which times every candidate on the batch itself.
//
// Level-queue mode: every field has its own workspace; the branches run each
// field's steps up to its levels, then one persistent launch per type runs
// the grid levels of all fields from a cross-field work queue (tiles of
// every (field, level), each level waiting on its field's next coarser level
// through a completion counter), then the branches run the encoders (or, for
// decompression, only the status copies).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.cuh"

namespace sz3g {

// Status of a finished field: flags and stream length.
__global__ void publish_kernel(const DevState* st, unsigned long long* res) {
  if (threadIdx.x == 0) {
    res[0] = st->flags;
    res[1] = st->out_bytes;
  }
}

}  // namespace sz3g

using namespace sz3g;

struct sz3g_batch {
  int n = 0;
  int decompress = 0;
  std::vector<sz3g_params> params;
  std::vector<Plan> plans;
  std::vector<Header> headers;          // decompress
  std::vector<const void*> in;
  std::vector<void*> out;
  std::vector<size_t> out_cap;
  std::vector<size_t> ws_need;          // per field
  int branches = 0, cta_cap = 0;
  int queue = 0;                        // level-queue mode
  std::vector<void*> ws;                // per branch (queue mode: one block holding every field's)
  std::vector<size_t> ws_off;           // queue mode: offset of each field's workspace
  LevelQueue* lq = nullptr;
  unsigned long long* d_res = nullptr;  // 2 per field
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t nodes = 0;
};

namespace {

void release_graph(sz3g_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  for (void* p : b->ws)
    if (p) cudaFree(p);
  b->ws.clear();
  level_queue_free(b->lq);
  b->lq = nullptr;
}

// Captures the batch with the given number of branches and CTA cap.
int build_graph(sz3g_batch* b, int branches, int cta_cap) {
  release_graph(b);
  branches = std::max(1, std::min(branches, b->n));
  // largest field first, to the least loaded branch
  std::vector<int> order(b->n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->plans[x].N > b->plans[y].N; });
  std::vector<unsigned long long> load(branches, 0);
  std::vector<std::vector<int>> lists(branches);
  std::vector<size_t> need(branches, 0);
  for (int f : order) {
    const int br = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[br] += b->plans[f].N;
    lists[br].push_back(f);
    need[br] = std::max(need[br], b->ws_need[f]);
  }
  if (!b->queue) {
    b->ws.assign(branches, nullptr);
    for (int br = 0; br < branches; ++br) {
      if (lists[br].empty()) continue;
      if (cudaMalloc(&b->ws[br], need[br] ? need[br] : 256) != cudaSuccess) {
        cudaGetLastError();
        release_graph(b);
        return SZ3G_E_NOMEM;
      }
    }
  } else {
    b->ws_off.assign(b->n, 0);
    size_t tot = 0, max_levels = 0;
    for (int f = 0; f < b->n; ++f) {
      b->ws_off[f] = tot;
      tot += (b->ws_need[f] + 255) & ~(size_t)255;
      max_levels += (size_t)b->plans[f].L + 1;
    }
    b->ws.assign(1, nullptr);
    b->lq = level_queue_new(!b->decompress);
    if (cudaMalloc(&b->ws[0], tot ? tot : 256) != cudaSuccess) {
      cudaGetLastError();
      release_graph(b);
      return SZ3G_E_NOMEM;
    }
    const int r = level_queue_reserve(b->lq, max_levels);
    if (r != SZ3G_OK) {
      release_graph(b);
      return r;
    }
  }
  cudaStream_t cs = nullptr;
  std::vector<cudaStream_t> bs(branches, nullptr);
  std::vector<cudaEvent_t> ev(2 * branches + 2, nullptr);
  int rc = SZ3G_OK;
  auto fail = [&](int code) {
    if (rc == SZ3G_OK) rc = code;
  };
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) fail(SZ3G_E_CUDA);
  for (int i = 0; i < branches && rc == SZ3G_OK; ++i)
    if (cudaStreamCreateWithFlags(&bs[i], cudaStreamNonBlocking) != cudaSuccess) fail(SZ3G_E_CUDA);
  for (size_t i = 0; i < ev.size() && rc == SZ3G_OK; ++i)
    if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) fail(SZ3G_E_CUDA);
  const int saved_cap = g_level_cta_cap;
  if (rc == SZ3G_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) fail(SZ3G_E_CUDA);
  bool capturing = rc == SZ3G_OK;
  if (capturing) {
    g_level_cta_cap = cta_cap;
    std::vector<DevState*> sts(b->n, nullptr);
    // one fan-out of the branches from cs and back: step(br, f) for the
    // fields of every branch, in order
    auto fan = [&](cudaEvent_t root, cudaEvent_t* done, auto&& step) {
      if (rc == SZ3G_OK && cudaEventRecord(root, cs) != cudaSuccess) fail(SZ3G_E_CUDA);
      for (int br = 0; br < branches && rc == SZ3G_OK; ++br) {
        if (lists[br].empty()) continue;
        if (cudaStreamWaitEvent(bs[br], root, 0) != cudaSuccess) {
          fail(SZ3G_E_CUDA);
          break;
        }
        for (int f : lists[br]) {
          const int r = step(br, f);
          if (r != SZ3G_OK) {
            fail(r);
            break;
          }
        }
        if (rc == SZ3G_OK && cudaEventRecord(done[br], bs[br]) != cudaSuccess) fail(SZ3G_E_CUDA);
        if (rc == SZ3G_OK && cudaStreamWaitEvent(cs, done[br], 0) != cudaSuccess) fail(SZ3G_E_CUDA);
      }
    };
    auto publish = [&](int br, int f) -> int {
      SZ3G_LAUNCH(kKPublish, bs[br], publish_kernel<<<1, 32, 0, bs[br]>>>(sts[f], b->d_res + 2 * f));
      return cudaGetLastError() == cudaSuccess ? SZ3G_OK : SZ3G_E_CUDA;
    };
    if (!b->queue) {
      fan(ev[2 * branches], ev.data(), [&](int br, int f) -> int {
        int r;
        if (b->decompress)
          r = decompress_enqueue(b->headers[f], b->in[f], b->out[f], (unsigned char*)b->ws[br], bs[br], &sts[f]);
        else
          r = compress_enqueue(&b->params[f], b->plans[f], b->in[f], b->out[f], b->out_cap[f],
                               (unsigned char*)b->ws[br], bs[br], &sts[f]);
        return r != SZ3G_OK ? r : publish(br, f);
      });
    } else {
      auto wsf = [&](int f) { return (unsigned char*)b->ws[0] + b->ws_off[f]; };
      fan(ev[2 * branches], ev.data(), [&](int br, int f) -> int {
        if (b->decompress)
          return decompress_enqueue(b->headers[f], b->in[f], b->out[f], wsf(f), bs[br], &sts[f], b->lq, f);
        return compress_enqueue_pre(&b->params[f], b->plans[f], b->in[f], wsf(f), bs[br], &sts[f], b->lq, f);
      });
      if (rc == SZ3G_OK) fail(level_queue_launch(b->lq, cs));
      fan(ev[2 * branches + 1], ev.data() + branches, [&](int br, int f) -> int {
        if (!b->decompress) {
          const int r = compress_enqueue_post(&b->params[f], b->plans[f], b->in[f], b->out[f], b->out_cap[f],
                                              wsf(f), bs[br]);
          if (r != SZ3G_OK) return r;
        }
        return publish(br, f);
      });
    }
    g_level_cta_cap = saved_cap;
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &g);
    if (ec != cudaSuccess || !g) {
      cudaGetLastError();
      fail(SZ3G_E_CUDA);
    } else if (rc != SZ3G_OK) {
      cudaGraphDestroy(g);
    } else {
      b->graph = g;
      if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
        cudaGetLastError();
        fail(SZ3G_E_CUDA);
      }
      size_t nn = 0;
      if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess) b->nodes = nn;
      if (rc == SZ3G_OK && b->queue) fail(level_queue_upload(b->lq));
    }
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : bs)
    if (s) cudaStreamDestroy(s);
  if (cs) cudaStreamDestroy(cs);
  if (rc != SZ3G_OK) {
    release_graph(b);
    return rc;
  }
  b->branches = branches;
  b->cta_cap = cta_cap;
  return SZ3G_OK;
}

}  // namespace

extern "C" {

int sz3g_batch_create(int n, int decompress, const sz3g_params* params, const void* const* d_in,
                      const size_t* in_bytes, void* const* d_out, const size_t* out_capacity, sz3g_batch** out) {
  if (!out || n < 1 || !d_in || !d_out || !out_capacity || (!decompress && !params) || (decompress && !in_bytes))
    return SZ3G_E_INVAL;
  *out = nullptr;
  sz3g_batch* b = new sz3g_batch;
  b->n = n;
  b->decompress = decompress != 0;
  b->plans.resize(n);
  b->in.assign(d_in, d_in + n);
  b->out.assign(d_out, d_out + n);
  b->out_cap.assign(out_capacity, out_capacity + n);
  b->ws_need.resize(n);
  int rc = SZ3G_OK;
  if (!decompress) {
    b->params.assign(params, params + n);
    for (int f = 0; f < n && rc == SZ3G_OK; ++f) {
      rc = make_plan(&b->params[f], &b->plans[f]);
      if (rc == SZ3G_OK && (!d_in[f] || !d_out[f] || ((uintptr_t)d_in[f] % 16) || ((uintptr_t)d_out[f] % 16)))
        rc = SZ3G_E_INVAL;
      size_t bound = 0;
      if (rc == SZ3G_OK) rc = sz3g_compress_bound(&b->params[f], &bound);
      if (rc == SZ3G_OK && out_capacity[f] < bound) rc = SZ3G_E_CAPACITY;
      if (rc == SZ3G_OK) b->ws_need[f] = compress_ws_bytes(b->plans[f]);
    }
  } else {
    b->headers.resize(n);
    for (int f = 0; f < n && rc == SZ3G_OK; ++f) {
      unsigned char hb[SZ3G_HEADER_BYTES];
      if (!d_in[f] || !d_out[f] || ((uintptr_t)d_in[f] % 16) || ((uintptr_t)d_out[f] % 16)) rc = SZ3G_E_INVAL;
      else if (in_bytes[f] < SZ3G_HEADER_BYTES) rc = SZ3G_E_CORRUPT;
      else if (cudaMemcpy(hb, d_in[f], SZ3G_HEADER_BYTES, cudaMemcpyDeviceToHost) != cudaSuccess) rc = SZ3G_E_CUDA;
      if (rc == SZ3G_OK) rc = parse_stream_header(hb, in_bytes[f], &b->headers[f]);
      if (rc == SZ3G_OK) {
        b->plans[f] = b->headers[f].plan;
        if (out_capacity[f] < b->plans[f].N * b->plans[f].esz) rc = SZ3G_E_CAPACITY;
        b->ws_need[f] = decompress_ws_bytes(b->plans[f]);
      }
    }
  }
  if (rc == SZ3G_OK && cudaMalloc(&b->d_res, 16 * (size_t)n) != cudaSuccess) rc = SZ3G_E_NOMEM;
  if (rc == SZ3G_OK) rc = build_graph(b, std::min(n, 8), 0);
  if (rc != SZ3G_OK) {
    cudaGetLastError();
    sz3g_batch_destroy(b);
    return rc;
  }
  *out = b;
  return SZ3G_OK;
}

int sz3g_batch_configure(sz3g_batch* b, int branches, int cta_cap) {
  if (!b || branches < 1 || cta_cap < 0) return SZ3G_E_INVAL;
  return build_graph(b, branches, cta_cap);
}

int sz3g_batch_set_queue(sz3g_batch* b, int on) {
  if (!b) return SZ3G_E_INVAL;
  b->queue = on != 0;
  return build_graph(b, b->branches ? b->branches : std::min(b->n, 8), b->cta_cap);
}

int sz3g_batch_queue_info(const sz3g_batch* b, int* on, int* levels) {
  if (!b) return SZ3G_E_INVAL;
  if (on) *on = b->queue;
  if (levels) *levels = b->lq ? level_queue_count(b->lq) : 0;
  return SZ3G_OK;
}

int sz3g_batch_run(sz3g_batch* b, void* stream) {
  SZ3G_TRACE("sz3g_batch_run");
  if (!b || !b->exec) return SZ3G_E_INVAL;
  if (cudaGraphLaunch(b->exec, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return SZ3G_E_CUDA;
  }
  return SZ3G_OK;
}

int sz3g_batch_results(sz3g_batch* b, uint64_t* h_bytes, int* h_status) {
  if (!b) return SZ3G_E_INVAL;
  std::vector<unsigned long long> r(2 * (size_t)b->n);
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(r.data(), b->d_res, 16 * (size_t)b->n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return SZ3G_E_CUDA;
  }
  int worst = SZ3G_OK;
  for (int f = 0; f < b->n; ++f) {
    const int st = stream_status((uint32_t)r[2 * f]);
    if (h_status) h_status[f] = st;
    if (h_bytes) h_bytes[f] = r[2 * f + 1];
    if (st != SZ3G_OK && worst == SZ3G_OK) worst = st;
  }
  return worst;
}

int sz3g_batch_info(const sz3g_batch* b, int* branches, int* cta_cap, uint64_t* graph_nodes) {
  if (!b) return SZ3G_E_INVAL;
  if (branches) *branches = b->branches;
  if (cta_cap) *cta_cap = b->cta_cap;
  if (graph_nodes) *graph_nodes = b->nodes;
  return SZ3G_OK;
}

int sz3g_batch_tune(sz3g_batch* b, void* stream, int* h_branches, int* h_cta_cap) {
  if (!b) return SZ3G_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int br_cand[] = {1, 2, 4, 8, 16, 32, 64, 128, 256};
  const int cap_cand[] = {0, nsm, nsm / 2, nsm / 4};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return SZ3G_E_CUDA;
  }
  float best = -1.0f;
  int best_br = b->branches, best_cap = b->cta_cap, best_q = b->queue;
  int rc = SZ3G_OK;
  for (int qm = 0; qm < 2 && rc == SZ3G_OK; ++qm)
  for (int br : br_cand) {
    if (br > b->n && br != 1) continue;
    for (int cap : cap_cand) {
      if (qm && cap != 0) continue;  // the queue's launch takes the whole GPU
      b->queue = qm;
      rc = build_graph(b, br, cap);
      if (rc != SZ3G_OK) break;
      float t = -1.0f, ms = 0.0f;
      cudaGraphLaunch(b->exec, s);  // warm-up (first launch of a new graph, first touch of its workspaces)
      cudaGraphLaunch(b->exec, s);
      for (int rep = 0; rep < 3; ++rep) {  // the fastest of three replays
        cudaEventRecord(e0, s);
        cudaGraphLaunch(b->exec, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          rc = SZ3G_E_CUDA;
          break;
        }
        if (t < 0 || ms < t) t = ms;
      }
      if (rc != SZ3G_OK) break;
      if (best < 0 || t < best) {
        best = t;
        best_br = br;
        best_cap = cap;
        best_q = qm;
      }
    }
    if (rc != SZ3G_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  if (rc != SZ3G_OK) return rc;
  b->queue = best_q;
  rc = build_graph(b, best_br, best_cap);
  if (h_branches) *h_branches = b->branches;
  if (h_cta_cap) *h_cta_cap = b->cta_cap;
  return rc;
}

int sz3g_batch_destroy(sz3g_batch* b) {
  if (!b) return SZ3G_OK;
  release_graph(b);
  if (b->d_res) cudaFree(b->d_res);
  delete b;
  return SZ3G_OK;
}

}  // extern "C"
