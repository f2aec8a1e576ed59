// graph.cu -- a solve as one CUDA-graph launch, and the read-backs that
// steer a plain solve.
//
// A plain solve reads a few device values back to the host (the octree's
// level counts, the number of leaves, the walk's list lengths, the near
// field's slot and work-item totals) and sizes the launches after them.  A
// graph cannot wait for the host, so the solve is captured in two passes:
//   1. a plain solve that keeps every value it reads back (the plan);
//   2. the same host code under stream capture, taking the planned values
//      instead of reading them.  At each read-back point the graph gets a
//      check kernel that compares the device words with the planned values
//      and sets the condition of an IF node; the rest of the solve is
//      captured into that node's body.
// A replay therefore runs the whole solve, as captured, exactly when every
// steering value equals the plan (same tree shape, list lengths and
// totals), and otherwise skips what follows the first differing check.
// The innermost body ends by marking the replay record done; the host reads
// the record after the launch and re-solves plainly (and re-captures) when
// it is not.  Every kernel reads its data from the device, so a replay with
// new coordinates or masses but the planned sizes computes the new solve.
#include <string.h>

#include "internal.cuh"

namespace amfmm {

namespace {

__global__ void k_expect(Expect e, cudaGraphConditionalHandle h) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < e.n; i += blockDim.x)
    if (*e.addr[i] != e.val[i]) bad = 1;
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(h, bad ? 0u : 1u);
}

__global__ void k_rec_bbox(const double *__restrict__ bbox, GraphRec *rec) {
  const int t = threadIdx.x;
  if (t < 3) rec->lo[t] = bbox[t];
  if (t == 3) rec->scale = bbox[3];
}

__global__ void k_rec_clear(GraphRec *rec) {
  if (threadIdx.x == 0) rec->done = 0u;
}

__global__ void k_rec_done(GraphRec *rec) {
  if (threadIdx.x == 0) rec->done = 1u;
}

GraphKey key_of(const fmm_ctx *c, const double *ax, const double *ay, const double *az) {
  GraphKey k;
  const void *p[7] = {c->x, c->y, c->z, c->m, ax, ay, az};
  for (int i = 0; i < 7; ++i) k.p[i] = p[i];
  k.n = c->sz.n;
  k.nsys = c->sz.nsys;
  k.theta = c->theta;
  k.eps2 = c->eps2;
  k.G = c->opts.G;
  k.n_crit = c->opts.n_crit;
  k.order_P = c->opts.order_P;
  k.variant = c->opts.variant;
  k.precision = c->opts.precision;
  k.rows = c->p2p_rows;
  k.alloc_gen = c->alloc_gen;
  return k;
}

// Pass 2: the solve's launches captured into a graph (nothing runs).
int capture(fmm_ctx *c, int depth0, double *ax, double *ay, double *az) {
  for (int d = 0; d < kMaxGraphDepth; ++d)
    if (!c->gstream[d]) AMFMM_CUDA(c, cudaStreamCreateWithFlags(&c->gstream[d], cudaStreamNonBlocking));
  if (c->gexec) {
    AMFMM_CUDA(c, cudaGraphExecDestroy(c->gexec));
    c->gexec = nullptr;
  }
  const cudaStream_t user = c->stream;
  const bool timing = c->timing;
  const int64_t n = c->sz.n;
  const int nsys = c->sz.nsys;
  c->sz = Sizes();
  c->sz.n = n;
  c->sz.nsys = nsys;
  c->launches = 0;
  c->last_depth = depth0;
  c->gplan_pos = 0;
  c->gdepth = 0;
  c->stream = c->gstream[0];
  GraphRec *rec = ptr<GraphRec>(c->grec);
  int rc = FMM_OK;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    c->stream = user;
    cudaGetLastError();
    return set_error(c, FMM_ECUDA, "cudaStreamBeginCapture failed: %s", cudaGetErrorString(e));
  }
  c->gmode = kGraphCapture;
  c->timing = false;
  k_rec_clear<<<1, 32, 0, c->stream>>>(rec);
  rc = launched(c, "graph_rec_clear");
  if (rc == FMM_OK) rc = run_stages(c, ax, ay, az);
  if (rc == FMM_OK && c->gplan_pos != c->gplan.size())
    rc = set_error(c, FMM_ECUDA, "graph capture: the solve read back less than its plan");
  if (rc == FMM_OK) {
    k_rec_done<<<1, 32, 0, c->stream>>>(rec);
    rc = launched(c, "graph_rec_done");
  }
  // close the bodies, innermost first, then the graph itself
  for (int d = c->gdepth; d >= 1; --d) {
    cudaGraph_t body = nullptr;
    e = cudaStreamEndCapture(c->gstream[d], &body);  // the body stays owned by its node
    if (e != cudaSuccess && rc == FMM_OK)
      rc = set_error(c, FMM_ECUDA, "ending the capture of a graph body failed: %s", cudaGetErrorString(e));
  }
  c->stream = c->gstream[0];
  if (rc == FMM_OK) {
    e = cudaMemcpyAsync(static_cast<char *>(c->hpin) + kGraphRecHostOff, rec, sizeof(GraphRec),
                        cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) rc = set_error(c, FMM_ECUDA, "capturing the record copy failed: %s", cudaGetErrorString(e));
  }
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->stream, &g);
  if (e != cudaSuccess && rc == FMM_OK)
    rc = set_error(c, FMM_ECUDA, "ending the capture failed: %s", cudaGetErrorString(e));
  c->gmode = kGraphOff;
  c->timing = timing;
  c->stream = user;
  c->gdepth = 0;
  if (rc == FMM_OK) {
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    if (e != cudaSuccess) {
      c->gexec = nullptr;
      rc = set_error(c, FMM_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
    }
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  if (rc == FMM_OK) c->glaunches = c->launches;
  return rc;
}

}  // namespace

int read_back(fmm_ctx *c, const HostRead *r, int nr) {
  if (c->gmode == kGraphCapture) {
    for (int k = 0; k < nr; ++k) {
      if (c->gplan_pos >= c->gplan.size() || c->gplan[c->gplan_pos].size() != r[k].bytes)
        return set_error(c, FMM_ECUDA, "graph capture: the solve took another path than its plan");
      memcpy(r[k].host, c->gplan[c->gplan_pos].data(), r[k].bytes);
      ++c->gplan_pos;
    }
    return FMM_OK;
  }
  for (int k = 0; k < nr; ++k)
    AMFMM_CUDA(c, cudaMemcpyAsync(r[k].host, r[k].dev, r[k].bytes, cudaMemcpyDeviceToHost, c->stream));
  AMFMM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (c->gmode == kGraphRecord)
    for (int k = 0; k < nr; ++k) {
      const unsigned char *h = static_cast<const unsigned char *>(r[k].host);
      c->gplan.emplace_back(h, h + r[k].bytes);
    }
  return FMM_OK;
}

int graph_expect(fmm_ctx *c, const Expect &ex) {
  if (c->gmode != kGraphCapture) return FMM_OK;
  if (c->gdepth + 1 >= kMaxGraphDepth) return set_error(c, FMM_ECUDA, "graph capture: too many nested checks");
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  AMFMM_CUDA(c, cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive || !g) return set_error(c, FMM_ECUDA, "graph capture: stream not capturing");
  cudaGraphConditionalHandle h;
  AMFMM_CUDA(c, cudaGraphConditionalHandleCreate(&h, g, 0u, cudaGraphCondAssignDefault));
  k_expect<<<1, 128, 0, c->stream>>>(ex, h);
  AMFMM_TRY(launched(c, "graph_expect"));
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  AMFMM_CUDA(c, cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  // (the struct holds a union without a default constructor)
  alignas(cudaGraphNodeParams) unsigned char pbuf[sizeof(cudaGraphNodeParams)];
  memset(pbuf, 0, sizeof(pbuf));
  cudaGraphNodeParams &p = *reinterpret_cast<cudaGraphNodeParams *>(pbuf);
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeIf;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  AMFMM_CUDA(c, cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  AMFMM_CUDA(c, cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaStream_t next = c->gstream[c->gdepth + 1];
  AMFMM_CUDA(c, cudaStreamBeginCaptureToGraph(next, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed));
  ++c->gdepth;
  c->stream = next;
  return FMM_OK;
}

int graph_record_bbox(fmm_ctx *c, const double *bbox) {
  if (c->gmode != kGraphCapture) return FMM_OK;
  k_rec_bbox<<<1, 32, 0, c->stream>>>(bbox, ptr<GraphRec>(c->grec));
  return launched(c, "graph_rec_bbox");
}

bool graph_usable(const fmm_ctx *c) {
  return c->graph_enabled && c->opts.order_P == 3 && !c->sel_enabled;
}

// Capture policy: the first solve of a key is captured.  A replay that
// finds other sizes drops the graph, and the following solves run plainly
// (recording their plans) until one plan repeats the one before it: a
// system whose tree changes every step (an integration) then costs no
// replays that would stop half-way.
int graph_solve(fmm_ctx *c, double *ax, double *ay, double *az) {
  AMFMM_TRY(ensure_bytes(c, c->grec, sizeof(GraphRec)));
  const GraphKey key = key_of(c, ax, ay, az);
  if (c->gexec && key == c->gkey) {
    AMFMM_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
    AMFMM_CUDA(c, cudaStreamSynchronize(c->stream));
    const GraphRec *r = reinterpret_cast<const GraphRec *>(static_cast<const char *>(c->hpin) + kGraphRecHostOff);
    if (r->done == 1u) {
      c->sz = c->gsz;
      for (int d = 0; d < 3; ++d) c->sz.lo[d] = r->lo[d];
      c->sz.scale = r->scale;
      c->stage = kDown;
      c->launches_last = c->glaunches;
      c->last_replay = true;
      ++c->g_replays;
      return FMM_OK;
    }
    // the sizes changed (or an input is invalid): solve plainly
    ++c->g_fallbacks;
    c->gwait = true;
  } else if (!(key == c->gkey)) {
    c->gwait = false;  // a new configuration is captured at once
  }
  if (c->gexec) {
    AMFMM_CUDA(c, cudaGraphExecDestroy(c->gexec));
    c->gexec = nullptr;
  }
  // pass 1: a plain solve that keeps its read-backs.  A solve that had to
  // grow a buffer took a path (a retry) that a capture cannot repeat: the
  // first solve of a context is then planned once more, on grown buffers.
  int depth0 = c->last_depth;
  for (int attempt = 0; attempt < 2; ++attempt) {
    depth0 = c->last_depth;
    const int64_t gen0 = c->alloc_gen;
    c->gplan.clear();
    c->gmode = kGraphRecord;
    const int rc = run_stages(c, ax, ay, az);
    c->gmode = kGraphOff;
    if (rc != FMM_OK) return rc;
    if (c->alloc_gen == gen0) break;
  }
  const bool repeat = c->gplan == c->gplan_prev;
  c->gplan_prev = c->gplan;
  c->gkey = key;
  if (c->gwait && !repeat) return FMM_OK;
  const Sizes plan = c->sz;
  const int depth1 = c->last_depth;
  const int64_t launches = c->launches_last;
  // pass 2: the same solve captured; its results are those of pass 1
  if (capture(c, depth0, ax, ay, az) == FMM_OK) {
    c->gsz = plan;
    c->gkey = key_of(c, ax, ay, az);
    c->gwait = false;
    ++c->g_captures;
  } else {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    ++c->g_capture_failures;
    snprintf(c->gerrbuf, sizeof(c->gerrbuf), "%s", c->errbuf);
    c->errbuf[0] = 0;
  }
  c->sz = plan;
  c->last_depth = depth1;
  c->stage = kDown;
  c->launches_last = launches;
  return FMM_OK;
}

}  // namespace amfmm

extern "C" const char *fmm_graph_error(const fmm_ctx *c) { return c ? c->gerrbuf : "NULL context"; }
