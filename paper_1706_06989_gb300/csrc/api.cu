// api.cu -- the C ABI declared in include/amfmm.h: context, validation,
// stage sequencing, buffers, statistics and exports.
#include <stdarg.h>
#include <string.h>

#include "internal.cuh"

namespace amfmm {

int set_error(fmm_ctx *c, int code, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->errbuf, sizeof(c->errbuf), fmt, ap);
    va_end(ap);
  }
  return code;
}

int ensure_bytes(fmm_ctx *c, DBuf &b, size_t bytes) {
  if (bytes <= b.cap) return FMM_OK;
  // a captured solve runs on the buffers its planning solve sized
  if (c->gmode == kGraphCapture) return set_error(c, FMM_ECUDA, "graph capture: a buffer would grow");
  ++c->alloc_gen;
  size_t cap = std::max(bytes, b.cap + b.cap / 2);
  cap = (cap + 255) & ~static_cast<size_t>(255);
  if (b.p) {
    // the old buffer may still be read by work queued on the stream
    cudaStreamSynchronize(c->stream);
    cudaError_t e = cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    if (e != cudaSuccess) return set_error(c, FMM_ECUDA, "cudaFree failed: %s", cudaGetErrorString(e));
  }
  cudaError_t e = cudaMalloc(&b.p, cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return set_error(c, FMM_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", cap, cudaGetErrorString(e));
  }
  b.cap = cap;
  return FMM_OK;
}

int ensure_keep_bytes(fmm_ctx *c, DBuf &b, size_t bytes, size_t used) {
  if (bytes <= b.cap) return FMM_OK;
  if (c->gmode == kGraphCapture) return set_error(c, FMM_ECUDA, "graph capture: a buffer would grow");
  ++c->alloc_gen;
  size_t cap = std::max(bytes, b.cap * 2);
  cap = (cap + 255) & ~static_cast<size_t>(255);
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, cap);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(c, FMM_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", cap, cudaGetErrorString(e));
  }
  if (b.p && used)
    AMFMM_CUDA(c, cudaMemcpyAsync(p, b.p, std::min(used, b.cap), cudaMemcpyDeviceToDevice, c->stream));
  if (b.p) {
    AMFMM_CUDA(c, cudaStreamSynchronize(c->stream));
    AMFMM_CUDA(c, cudaFree(b.p));
  }
  b.p = p;
  b.cap = cap;
  return FMM_OK;
}

int launched(fmm_ctx *c, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(c, FMM_ECUDA, "launch of %s failed: %s", what, cudaGetErrorString(e));
  ++c->launches;
  return FMM_OK;
}

void timer(fmm_ctx *c, int slot) {
  // (event records are not allowed in the conditional bodies of a graph)
  if (c->timing && c->gmode != kGraphCapture) cudaEventRecord(c->ev[slot], c->stream);
}

}  // namespace amfmm

using namespace amfmm;

namespace {

void free_buf(DBuf &b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
}

int check_opts(fmm_ctx *c, const fmm_opts *o) {
  if (!o) return set_error(c, FMM_EINVAL, "opts is NULL");
  if (!(o->theta > 0.0 && o->theta <= 1.0))
    return set_error(c, FMM_EINVAL, "theta must satisfy 0 < theta <= 1 (got %g)", o->theta);
  if (o->n_crit < 1) return set_error(c, FMM_EINVAL, "n_crit must be >= 1 (got %d)", o->n_crit);
  if (o->order_P < 3 || o->order_P > 8)
    return set_error(c, FMM_EUNSUPPORTED, "order_P %d is not built (3 to 8 are)", o->order_P);
  if (o->order_P != 3 && o->precision != FMM_FP64)
    return set_error(c, FMM_EUNSUPPORTED, "orders above 3 are built in FP64 only");
  if (o->variant < FMM_UC || o->variant > FMM_TCO)
    return set_error(c, FMM_EINVAL, "variant must be FMM_UC, FMM_TC or FMM_TCO");
  if (o->precision != FMM_FP64 && o->precision != FMM_MIXED)
    return set_error(c, FMM_EINVAL, "precision must be FMM_FP64 or FMM_MIXED");
  if (!(o->G == o->G)) return set_error(c, FMM_EINVAL, "G is NaN");
  return FMM_OK;
}

int need_stage(fmm_ctx *c, int stage, const char *what) {
  if (c->stage < stage) return set_error(c, FMM_EORDER, "%s called out of sequence", what);
  return FMM_OK;
}

}  // namespace

extern "C" {

int fmm_create(fmm_ctx **out, const fmm_opts *opts, void *cuda_stream) {
  if (!out) return FMM_EINVAL;
  *out = nullptr;
  fmm_ctx *c = new (std::nothrow) fmm_ctx();
  if (!c) return FMM_ENOMEM;
  int rc = check_opts(c, opts);
  if (rc != FMM_OK) {
    delete c;
    return rc;
  }
  c->opts = *opts;
  c->theta = opts->theta;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess ||
      cudaMallocHost(&c->hpin, 16384) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return FMM_ECUDA;
  }
  for (int k = 0; k < kNumTimers; ++k) {
    if (cudaEventCreate(&c->ev[k]) != cudaSuccess) {
      cudaGetLastError();
      fmm_destroy(c);
      return FMM_ECUDA;
    }
  }
  if (ensure_bytes(c, c->totals, 1024) != FMM_OK) {
    fmm_destroy(c);
    return FMM_ENOMEM;
  }
  *out = c;
  return FMM_OK;
}

void fmm_destroy(fmm_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  DBuf *all[] = {&c->key[0], &c->key[1], &c->idx[0], &c->idx[1], &c->order, &c->X, &c->Y, &c->Zb, &c->Mb,
                 &c->cur, &c->flag, &c->incl, &c->lcp, &c->leaf_of, &c->cell_at, &c->near, &c->acc,
                 &c->status, &c->bbox_part, &c->bbox, &c->sys_off, &c->sysid, &c->sbox, &c->begin, &c->count, &c->level, &c->parent,
                 &c->first_child, &c->nchild, &c->S, &c->M, &c->Z, &c->invM, &c->Rmax, &c->rmax2, &c->mom,
                 &c->loc, &c->leaves, &c->front[0], &c->front[1],
                 &c->m2l, &c->p2p, &c->self_list, &c->walk_zr, &c->walk_zf, &c->walk_nl, &c->walk_state, &c->walk_lb, &c->ekey[0], &c->ekey[1], &c->eval[0], &c->eval[1],
                 &c->m2l_pos, &c->m2l_off, &c->m2l_slots, &c->cell32, &c->qoh, &c->pkey[0], &c->pkey[1], &c->pval[0],
                 &c->pval[1], &c->p2p_A, &c->p2p_offA, &c->p2p_offB, &c->p2p_pos, &c->p2p_poff,
                 &c->p2p_len, &c->p2p_slots, &c->p2p_colOff, &c->p2p_cols, &c->p2p_nb, &c->p2p_pre, &c->p2p_bodyf, &c->p2p_items, &c->p2p_itemOff, &c->p2p_extraOff, &c->p2p_extra, &c->scan_tmp, &c->sort_hist, &c->totals, &c->diag, &c->sel_params, &c->sel_cellfeat, &c->sel_cand, &c->sel_lga, &c->sel_scratch, &c->sel_part, &c->sel_score, &c->sel_grad, &c->sel_perm, &c->sel_xb, &c->sel_yb, &c->gen_tab, &c->hx, &c->hy,
                 &c->hz, &c->hm, &c->hax, &c->hay, &c->haz};
  for (DBuf *b : all) free_buf(*b);
  free_buf(c->grec);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  for (cudaStream_t s : c->gstream)
    if (s) cudaStreamDestroy(s);
  for (int k = 0; k < kNumTimers; ++k)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  if (c->hpin) cudaFreeHost(c->hpin);
  delete c;
}

const char *fmm_last_error(const fmm_ctx *c) { return c ? c->errbuf : "NULL context"; }

int fmm_set_opts(fmm_ctx *c, const fmm_opts *opts) {
  if (!c) return FMM_EINVAL;
  AMFMM_TRY(check_opts(c, opts));
  c->opts = *opts;
  c->theta = opts->theta;
  c->stage = kNone;
  return FMM_OK;
}

int fmm_set_tile(fmm_ctx *c, int rows) {
  if (!c) return FMM_EINVAL;
  if (rows != 8 && rows != 16 && rows != 32) return set_error(c, FMM_EINVAL, "leaf tile must be 8, 16 or 32 (got %d)", rows);
  c->p2p_rows = rows;
  return FMM_OK;
}

int fmm_set_softening(fmm_ctx *c, double eps) {
  if (!c) return FMM_EINVAL;
  if (!(eps >= 0.0) || !(eps < 1e300)) return set_error(c, FMM_EINVAL, "softening must be finite and >= 0 (got %g)", eps);
  c->eps2 = eps * eps;
  c->stage = kNone;
  return FMM_OK;
}

int fmm_set_timing(fmm_ctx *c, int enable) {
  if (!c) return FMM_EINVAL;
  c->timing = enable != 0;
  return FMM_OK;
}

int fmm_set_graph(fmm_ctx *c, int enable) {
  if (!c) return FMM_EINVAL;
  c->graph_enabled = enable != 0;
  return FMM_OK;
}

int fmm_graph_stats(const fmm_ctx *c, int64_t *out) {
  if (!c || !out) return FMM_EINVAL;
  out[0] = c->g_replays;
  out[1] = c->g_captures;
  out[2] = c->g_fallbacks;
  out[3] = c->g_capture_failures;
  out[4] = c->gexec ? c->glaunches : 0;
  return FMM_OK;
}

}  // extern "C"

namespace {

// Common start of a solve of nsys >= 1 independent systems; offsets (host,
// nsys + 1 entries) or NULL for a single system of n bodies: checks the
// arguments and puts the system offsets on the device (synchronously).
int begin_solve(fmm_ctx *c, const double *x, const double *y, const double *z, const double *m, int64_t n,
                double theta, const int64_t *offsets, int nsys) {
  if (!c) return FMM_EINVAL;
  c->stage = kNone;
  c->errbuf[0] = 0;
  if (n < 1) return set_error(c, FMM_EINVAL, "n must be >= 1 (got %lld)", static_cast<long long>(n));
  if (n > 0x7fffffffLL) return set_error(c, FMM_EINVAL, "n must be < 2^31");
  if (!x || !y || !z || !m) return set_error(c, FMM_EINVAL, "NULL body array");
  if (theta != 0.0) {
    if (!(theta > 0.0 && theta <= 1.0))
      return set_error(c, FMM_EINVAL, "theta must satisfy 0 < theta <= 1 (got %g)", theta);
    c->theta = theta;
  } else {
    c->theta = c->opts.theta;
  }
  if (nsys < 1) return set_error(c, FMM_EINVAL, "nsys must be >= 1");
  c->x = x;
  c->y = y;
  c->z = z;
  c->m = m;
  c->sz = Sizes();
  c->sz.n = n;
  c->sz.nsys = nsys;
  c->launches = 0;
  // system offsets on the device
  AMFMM_TRY(ensure<int64_t>(c, c->sys_off, static_cast<size_t>(nsys) + 1));
  if (offsets) {
    AMFMM_CUDA(c, cudaStreamSynchronize(c->stream));  // the pinned staging buffer is reused
    int64_t *h = static_cast<int64_t *>(c->hpin);
    const size_t cap = 4096 / sizeof(int64_t);
    for (size_t b = 0; b < static_cast<size_t>(nsys) + 1; b += cap) {
      const size_t cnt = std::min(cap, static_cast<size_t>(nsys) + 1 - b);
      for (size_t k = 0; k < cnt; ++k) h[k] = offsets[b + k];
      AMFMM_CUDA(c, cudaMemcpyAsync(ptr<int64_t>(c->sys_off) + b, h, cnt * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, c->stream));
      AMFMM_CUDA(c, cudaStreamSynchronize(c->stream));
    }
  } else {
    int64_t *h = static_cast<int64_t *>(c->hpin);
    AMFMM_CUDA(c, cudaStreamSynchronize(c->stream));
    h[0] = 0;
    h[1] = n;
    AMFMM_CUDA(c, cudaMemcpyAsync(c->sys_off.p, h, 2 * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  }
  c->last_replay = false;
  return FMM_OK;
}

int tree_stage(fmm_ctx *c) {
  timer(c, kTreeBeg);
  AMFMM_TRY(build_tree(c));
  timer(c, kTreeEnd);
  c->stage = kTree;
  return FMM_OK;
}

int start_solve(fmm_ctx *c, const double *x, const double *y, const double *z, const double *m, int64_t n,
                double theta, const int64_t *offsets, int nsys) {
  AMFMM_TRY(begin_solve(c, x, y, z, m, n, theta, offsets, nsys));
  return tree_stage(c);
}

}  // namespace

namespace amfmm {

// The stages of a solve after begin_solve.
int run_stages(fmm_ctx *c, double *ax, double *ay, double *az) {
  AMFMM_TRY(tree_stage(c));
  AMFMM_TRY(fmm_upward(c));
  AMFMM_TRY(fmm_interact(c));
  AMFMM_TRY(fmm_downward(c));
  return fmm_forces(c, ax, ay, az);
}

}  // namespace amfmm

extern "C" {

int fmm_build_tree(fmm_ctx *c, const double *x, const double *y, const double *z, const double *m,
                   int64_t n, double theta) {
  return start_solve(c, x, y, z, m, n, theta, nullptr, 1);
}

int fmm_solve_batch(fmm_ctx *c, const double *x, const double *y, const double *z, const double *m,
                    const int64_t *offsets, int nsys, double *ax, double *ay, double *az) {
  if (!c) return FMM_EINVAL;
  if (!offsets || nsys < 1) return set_error(c, FMM_EINVAL, "offsets must list nsys >= 1 systems");
  if (offsets[0] != 0) return set_error(c, FMM_EINVAL, "offsets[0] must be 0");
  for (int s = 0; s < nsys; ++s)
    if (offsets[s + 1] <= offsets[s]) return set_error(c, FMM_EINVAL, "system %d is empty or offsets decrease", s);
  AMFMM_TRY(begin_solve(c, x, y, z, m, offsets[nsys], 0.0, offsets, nsys));
  if (!ax || !ay || !az) return set_error(c, FMM_EINVAL, "NULL output array");
  if (graph_usable(c)) return graph_solve(c, ax, ay, az);
  return run_stages(c, ax, ay, az);
}

int fmm_upward(fmm_ctx *c) {
  if (!c) return FMM_EINVAL;
  AMFMM_TRY(need_stage(c, kTree, "fmm_upward"));
  timer(c, kUpBeg);
  AMFMM_TRY(upward(c));
  timer(c, kUpEnd);
  c->stage = kUp;
  return FMM_OK;
}

int fmm_interact(fmm_ctx *c) {
  if (!c) return FMM_EINVAL;
  AMFMM_TRY(need_stage(c, kUp, "fmm_interact"));
  if (c->eps2 > 0.0 && c->opts.order_P != 3)
    return set_error(c, FMM_EUNSUPPORTED, "softening is built at order 3 only (order_P = %d)", c->opts.order_P);
  timer(c, kWalkBeg);
  AMFMM_TRY(walk(c));
  AMFMM_TRY(m2l_prepare(c));
  AMFMM_TRY(p2p_prepare(c));
  timer(c, kWalkEnd);
  timer(c, kM2LBeg);
  AMFMM_TRY(m2l_run(c));
  timer(c, kM2LEnd);
  timer(c, kP2PBeg);
  AMFMM_TRY(p2p_run(c));
  timer(c, kP2PEnd);
  timer(c, kRedBeg);
  AMFMM_TRY(m2l_reduce(c));
  AMFMM_TRY(p2p_reduce(c));
  timer(c, kRedEnd);
  c->stage = kInteract;
  return FMM_OK;
}

int fmm_downward(fmm_ctx *c) {
  if (!c) return FMM_EINVAL;
  AMFMM_TRY(need_stage(c, kInteract, "fmm_downward"));
  timer(c, kDownBeg);
  AMFMM_TRY(downward(c));
  c->stage = kDown;
  return FMM_OK;
}

int fmm_forces(fmm_ctx *c, double *ax, double *ay, double *az) {
  if (!c) return FMM_EINVAL;
  AMFMM_TRY(need_stage(c, kDown, "fmm_forces"));
  if (!ax || !ay || !az) return set_error(c, FMM_EINVAL, "NULL output array");
  AMFMM_TRY(forces(c, ax, ay, az));
  timer(c, kDownEnd);
  c->launches_last = c->launches;
  return FMM_OK;
}

int fmm_solve(fmm_ctx *c, const double *x, const double *y, const double *z, const double *m, int64_t n,
              double *ax, double *ay, double *az) {
  AMFMM_TRY(begin_solve(c, x, y, z, m, n, 0.0, nullptr, 1));
  if (!ax || !ay || !az) return set_error(c, FMM_EINVAL, "NULL output array");
  if (graph_usable(c)) return graph_solve(c, ax, ay, az);
  return run_stages(c, ax, ay, az);
}

int fmm_solve_host(fmm_ctx *c, const double *x, const double *y, const double *z, const double *m, int64_t n,
                   double *ax, double *ay, double *az) {
  if (!c) return FMM_EINVAL;
  if (n < 1) return set_error(c, FMM_EINVAL, "n must be >= 1");
  if (!x || !y || !z || !m || !ax || !ay || !az) return set_error(c, FMM_EINVAL, "NULL host array");
  const size_t b = sizeof(double) * static_cast<size_t>(n);
  DBuf *in[] = {&c->hx, &c->hy, &c->hz, &c->hm, &c->hax, &c->hay, &c->haz};
  for (DBuf *d : in) AMFMM_TRY(ensure_bytes(c, *d, b));
  const double *src[] = {x, y, z, m};
  for (int k = 0; k < 4; ++k)
    AMFMM_CUDA(c, cudaMemcpyAsync(in[k]->p, src[k], b, cudaMemcpyHostToDevice, c->stream));
  AMFMM_TRY(fmm_solve(c, ptr<double>(c->hx), ptr<double>(c->hy), ptr<double>(c->hz), ptr<double>(c->hm), n,
                      ptr<double>(c->hax), ptr<double>(c->hay), ptr<double>(c->haz)));
  double *dst[] = {ax, ay, az};
  for (int k = 0; k < 3; ++k)
    AMFMM_CUDA(c, cudaMemcpyAsync(dst[k], in[4 + k]->p, b, cudaMemcpyDeviceToHost, c->stream));
  AMFMM_CUDA(c, cudaStreamSynchronize(c->stream));
  return FMM_OK;
}

int fmm_get_stats(fmm_ctx *c, fmm_stats *s) {
  if (!c || !s) return FMM_EINVAL;
  AMFMM_CUDA(c, cudaStreamSynchronize(c->stream));
  memset(s, 0, sizeof(*s));
  s->n = c->sz.n;
  s->ncell = c->sz.ncell;
  s->nleaf = c->sz.nleaf;
  s->depth = c->sz.depth;
  s->n_m2l = c->sz.n_m2l;
  s->n_p2p = c->sz.n_p2p;
  s->n_self = c->sz.n_self;
  s->launches = c->launches_last;
  for (int d = 0; d < 3; ++d) s->lo[d] = c->sz.lo[d];
  s->scale = c->sz.scale;
  if (c->stage >= kInteract && c->totals.p) {
    long long v = 0;
    AMFMM_CUDA(c, cudaMemcpy(&v, ptr<int64_t>(c->totals) + 8, sizeof(v), cudaMemcpyDeviceToHost));
    s->p2p_body_pairs = v;
    if (c->sel_enabled) {
      AMFMM_CUDA(c, cudaMemcpy(&v, ptr<int64_t>(c->totals) + 10, sizeof(v), cudaMemcpyDeviceToHost));
      s->n_scored = v;
    }
  }
  if (c->timing && c->stage >= kDown && !c->last_replay) {
    float *ms[] = {&s->ms_tree, &s->ms_upward, &s->ms_walk, &s->ms_m2l, &s->ms_p2p, &s->ms_reduce, &s->ms_downward};
    const int beg[] = {kTreeBeg, kUpBeg, kWalkBeg, kM2LBeg, kP2PBeg, kRedBeg, kDownBeg};
    for (int k = 0; k < 7; ++k) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, c->ev[beg[k]], c->ev[beg[k] + 1]) != cudaSuccess) {
        cudaGetLastError();
        t = -1.f;
      }
      *ms[k] = t;
    }
  }
  return FMM_OK;
}

int fmm_export_keys(fmm_ctx *c, uint64_t *keys, int32_t *order) {
  if (!c || !keys || !order) return FMM_EINVAL;
  AMFMM_TRY(need_stage(c, kTree, "fmm_export_keys"));
  const size_t n = static_cast<size_t>(c->sz.n);
  AMFMM_CUDA(c, cudaMemcpyAsync(keys, c->key[c->sz.key_which].p, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, c->stream));
  AMFMM_CUDA(c, cudaMemcpyAsync(order, c->order.p, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
  return FMM_OK;
}

int fmm_export_tree(fmm_ctx *c, int32_t *begin, int32_t *count, int32_t *level, int32_t *parent,
                    int32_t *first_child, int32_t *nchild, double *M, double *Z, double *Rmax) {
  if (!c) return FMM_EINVAL;
  AMFMM_TRY(need_stage(c, kTree, "fmm_export_tree"));
  const size_t nc = static_cast<size_t>(c->sz.ncell);
  int32_t *dst[] = {begin, count, level, parent, first_child, nchild};
  DBuf *src[] = {&c->begin, &c->count, &c->level, &c->parent, &c->first_child, &c->nchild};
  for (int k = 0; k < 6; ++k)
    if (dst[k]) AMFMM_CUDA(c, cudaMemcpyAsync(dst[k], src[k]->p, nc * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
  if (M || Z || Rmax) AMFMM_TRY(need_stage(c, kUp, "fmm_export_tree (geometry)"));
  if (M) AMFMM_CUDA(c, cudaMemcpyAsync(M, c->M.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  if (Z) AMFMM_CUDA(c, cudaMemcpyAsync(Z, c->Z.p, 3 * nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  if (Rmax) AMFMM_CUDA(c, cudaMemcpyAsync(Rmax, c->Rmax.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  return FMM_OK;
}

int fmm_export_moments(fmm_ctx *c, double *mom) {
  if (!c || !mom) return FMM_EINVAL;
  AMFMM_TRY(need_stage(c, kUp, "fmm_export_moments"));
  AMFMM_CUDA(c, cudaMemcpyAsync(mom, c->mom.p,
                                static_cast<size_t>(c->sz.ncell) * mom_stride(c->opts.order_P) * sizeof(double),
                                cudaMemcpyDeviceToDevice, c->stream));
  return FMM_OK;
}

int fmm_export_lists(fmm_ctx *c, int32_t *m2l, int32_t *p2p, int32_t *self) {
  if (!c) return FMM_EINVAL;
  AMFMM_TRY(need_stage(c, kInteract, "fmm_export_lists"));
  if (m2l && c->sz.n_m2l)
    AMFMM_CUDA(c, cudaMemcpyAsync(m2l, c->m2l.p, 2 * c->sz.n_m2l * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
  if (p2p && c->sz.n_p2p)
    AMFMM_CUDA(c, cudaMemcpyAsync(p2p, c->p2p.p, 2 * c->sz.n_p2p * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
  if (self && c->sz.n_self)
    AMFMM_CUDA(c, cudaMemcpyAsync(self, c->self_list.p, c->sz.n_self * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
  return FMM_OK;
}

int fmm_export_locals(fmm_ctx *c, double *C) {
  if (!c || !C) return FMM_EINVAL;
  AMFMM_TRY(need_stage(c, kDown, "fmm_export_locals"));
  AMFMM_CUDA(c, cudaMemcpyAsync(C, c->loc.p,
                                static_cast<size_t>(c->sz.ncell) * loc_stride(c->opts.order_P) * sizeof(double),
                                cudaMemcpyDeviceToDevice, c->stream));
  return FMM_OK;
}

}  // extern "C"
