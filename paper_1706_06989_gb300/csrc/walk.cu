// walk.cu -- a5, a6: the dual-tree walk of Dehnen (2000) under the opening
// criterion of Sec. 2,
//     |Z_A - Z_B| >= (R_A,max + R_B,max) / theta,
// evaluated as theta^2 |Z_A - Z_B|^2 >= (R_A,max + R_B,max)^2 (equality
// accepted) with explicitly rounded FP64 operations, so that the GPU and any
// serial evaluation of the same expression agree bit for bit.
//
// Rules for a pair of cells (A, B):
//   A == B, leaf        -> the leaf is summed directly with itself;
//   A == B, not a leaf  -> (c_i, c_i) for every child and (c_i, c_j), i < j;
//   accepted            -> one mutual M2L interaction;
//   both leaves         -> one mutual P2P interaction;
//   otherwise           -> split one cell (the non-leaf if only one is; else
//                          the larger R_max, then the shallower, then the
//                          smaller id) and visit (child, other) for each child.
// The set of emitted pairs depends only on these per-pair decisions, so it is
// independent of the traversal order.  The walk proceeds one generation of
// pairs at a time; an exclusive scan of the per-pair output counts places
// every output, which makes the list order deterministic.
#include "internal.cuh"

namespace amfmm {
namespace {

constexpr int kBlock = 256;

enum Action : int32_t { kSelfLeaf = 0, kSelfSplit = 1, kAccept = 2, kNear = 3, kSplitA = 4, kSplitB = 5 };

// per cell {Z_x, Z_y, Z_z, R_max}, one 32-byte load
__device__ __forceinline__ bool well_separated(const double4_32a a, const double4_32a b, double theta) {
  const double dx = __dsub_rn(a.x, b.x);
  const double dy = __dsub_rn(a.y, b.y);
  const double dz = __dsub_rn(a.z, b.z);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double th2 = __dmul_rn(theta, theta);
  const double s = __dadd_rn(a.w, b.w);
  return __dmul_rn(th2, d2) >= __dmul_rn(s, s);
}

// packs the walk's per-cell inputs: {Z, R_max} and {nchild, level}
__global__ void k_pack_cells(int32_t ncell, const double *__restrict__ Z, const double *__restrict__ Rmax,
                             const int32_t *__restrict__ nchild, const int32_t *__restrict__ level,
                             double4_32a *__restrict__ zr, int2 *__restrict__ nl) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  zr[c] = make_double4_32a(Z[3 * c], Z[3 * c + 1], Z[3 * c + 2], Rmax[c]);
  nl[c] = make_int2(nchild[c], level[c]);
}

// score (may be NULL): the learned selector's prediction for every frontier
// pair (+inf where the safety bound fails); with it, a pair is accepted when
// the opening criterion accepts it (theta is then a floor on the accepted
// set, which bounds the work of a strict target) or when score < target.
__global__ void k_classify(int64_t nf, const int2 *__restrict__ front, const int2 *__restrict__ nl,
                           const double4_32a *__restrict__ zr, double theta, const float *__restrict__ score,
                           float target, int32_t *__restrict__ action, int4 *__restrict__ counts) {
  int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= nf) return;
  const int A = front[t].x, B = front[t].y;
  int act;
  int4 cnt = make_int4(0, 0, 0, 0);
  const int2 nlA = nl[A];
  if (A == B) {
    const int k = nlA.x;
    if (k == 0) {
      act = kSelfLeaf;
      cnt.w = 1;
    } else {
      act = kSelfSplit;
      cnt.x = k + k * (k - 1) / 2;
    }
  } else if (well_separated(zr[A], zr[B], theta) || (score && score[t] < target)) {
    act = kAccept;
    cnt.y = 1;
  } else {
    const int2 nlB = nl[B];
    const int ka = nlA.x, kb = nlB.x;
    if (ka == 0 && kb == 0) {
      act = kNear;
      cnt.z = 1;
    } else {
      bool pickA;
      if (kb == 0) pickA = true;
      else if (ka == 0) pickA = false;
      else {
        const double ra = zr[A].w, rb = zr[B].w;
        if (ra != rb) pickA = ra > rb;
        else if (nlA.y != nlB.y) pickA = nlA.y < nlB.y;
        else pickA = A < B;
      }
      act = pickA ? kSplitA : kSplitB;
      cnt.x = pickA ? ka : kb;
    }
  }
  action[t] = act;
  counts[t] = cnt;
}

__global__ void k_emit(int64_t nf, const int2 *__restrict__ front, const int32_t *__restrict__ action,
                       const int4 *__restrict__ offs, const int32_t *__restrict__ first_child,
                       const int32_t *__restrict__ nchild, int2 *__restrict__ next,
                       int2 *__restrict__ m2l, int64_t m2l_base, int2 *__restrict__ p2p,
                       int64_t p2p_base, int32_t *__restrict__ self, int64_t self_base) {
  int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= nf) return;
  const int A = front[t].x, B = front[t].y;
  const int4 o = offs[t];
  switch (action[t]) {
    case kSelfLeaf:
      self[self_base + o.w] = A;
      break;
    case kSelfSplit: {
      const int f = first_child[A], k = nchild[A];
      int q = o.x;
      for (int i = 0; i < k; ++i) next[q++] = make_int2(f + i, f + i);
      for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j) next[q++] = make_int2(f + i, f + j);
      break;
    }
    case kAccept:
      m2l[m2l_base + o.y] = make_int2(min(A, B), max(A, B));
      break;
    case kNear:
      p2p[p2p_base + o.z] = make_int2(min(A, B), max(A, B));
      break;
    case kSplitA: {
      const int f = first_child[A], k = nchild[A];
      for (int i = 0; i < k; ++i) next[o.x + i] = make_int2(f + i, B);
      break;
    }
    default: {
      const int f = first_child[B], k = nchild[B];
      for (int i = 0; i < k; ++i) next[o.x + i] = make_int2(A, f + i);
      break;
    }
  }
}

__global__ void k_roots_front(int32_t nsys, int2 *__restrict__ front) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nsys) front[s] = make_int2(s, s);
}

}  // namespace

int walk(fmm_ctx *c) {
  cudaStream_t st = c->stream;
  const int64_t n = c->sz.n;
  int64_t cap_front = std::max<int64_t>(4096, n / 4);
  AMFMM_TRY(ensure<int2>(c, c->front[0], cap_front));
  AMFMM_TRY(ensure<int2>(c, c->front[1], cap_front));
  int64_t cap_m2l = c->m2l.cap / sizeof(int2), cap_p2p = c->p2p.cap / sizeof(int2),
          cap_self = c->self_list.cap / sizeof(int32_t);
  if (cap_m2l < 1024) {
    cap_m2l = std::max<int64_t>(1024, 8 * n);
    AMFMM_TRY(ensure<int2>(c, c->m2l, cap_m2l));
  }
  if (cap_p2p < 1024) {
    cap_p2p = std::max<int64_t>(1024, 2 * n);
    AMFMM_TRY(ensure<int2>(c, c->p2p, cap_p2p));
  }
  if (cap_self < 1024) {
    cap_self = std::max<int64_t>(1024, n / 4 + 64);
    AMFMM_TRY(ensure<int32_t>(c, c->self_list, cap_self));
  }

  int4 *total = ptr<int4>(c->totals);
  const int64_t nc = c->sz.ncell;
  AMFMM_TRY(ensure<double4_32a>(c, c->walk_zr, nc));
  AMFMM_TRY(ensure<int2>(c, c->walk_nl, nc));
  k_pack_cells<<<grid_for(nc, kBlock), kBlock, 0, st>>>(static_cast<int32_t>(nc), ptr<double>(c->Z), ptr<double>(c->Rmax),
                                                       ptr<int32_t>(c->nchild), ptr<int32_t>(c->level),
                                                       ptr<double4_32a>(c->walk_zr), ptr<int2>(c->walk_nl));
  AMFMM_TRY(launched(c, "walk_pack"));
  // one self pair per root: systems of a forest never interact
  const int64_t nsys = c->sz.nsys;
  if (nsys > static_cast<int64_t>(c->front[0].cap / sizeof(int2))) AMFMM_TRY(ensure<int2>(c, c->front[0], nsys));
  k_roots_front<<<grid_for(nsys, kBlock), kBlock, 0, st>>>(static_cast<int32_t>(nsys), ptr<int2>(c->front[0]));
  AMFMM_TRY(launched(c, "walk_roots"));
  int64_t nf = nsys, n_m2l = 0, n_p2p = 0, n_self = 0;
  int cur = 0;
  while (nf > 0) {
    AMFMM_TRY(ensure<int32_t>(c, c->action, nf));
    AMFMM_TRY(ensure<int4>(c, c->wcount, nf));
    AMFMM_TRY(ensure<int4>(c, c->woff, nf));
    const float *score = nullptr;
    if (c->sel_enabled) {
      AMFMM_TRY(ensure<float>(c, c->sel_score, nf));
      AMFMM_TRY(walk_scores(c, nf, ptr<int2>(c->front[cur]), ptr<float>(c->sel_score)));
      score = ptr<float>(c->sel_score);
    }
    k_classify<<<grid_for(nf, kBlock), kBlock, 0, st>>>(
        nf, ptr<int2>(c->front[cur]), ptr<int2>(c->walk_nl), ptr<double4_32a>(c->walk_zr), c->theta, score,
        static_cast<float>(c->sel_log10_target), ptr<int32_t>(c->action), ptr<int4>(c->wcount));
    AMFMM_TRY(launched(c, "walk_classify"));
    AMFMM_TRY(exclusive_scan_i4(c, ptr<int4>(c->wcount), ptr<int4>(c->woff), nf, total));
    int4 *h = static_cast<int4 *>(c->hpin);
    AMFMM_CUDA(c, cudaMemcpyAsync(h, total, sizeof(int4), cudaMemcpyDeviceToHost, st));
    AMFMM_CUDA(c, cudaStreamSynchronize(st));
    const int4 tot = *h;
    if (tot.x > 0 && tot.x > static_cast<int64_t>(c->front[cur ^ 1].cap / sizeof(int2)))
      AMFMM_TRY(ensure<int2>(c, c->front[cur ^ 1], std::max<int64_t>(tot.x, 2 * (c->front[cur ^ 1].cap / sizeof(int2)))));
    if (n_m2l + tot.y > cap_m2l) {
      cap_m2l = std::max<int64_t>(2 * cap_m2l, n_m2l + tot.y);
      AMFMM_TRY(ensure_keep_bytes(c, c->m2l, cap_m2l * sizeof(int2), n_m2l * sizeof(int2)));
    }
    if (n_p2p + tot.z > cap_p2p) {
      cap_p2p = std::max<int64_t>(2 * cap_p2p, n_p2p + tot.z);
      AMFMM_TRY(ensure_keep_bytes(c, c->p2p, cap_p2p * sizeof(int2), n_p2p * sizeof(int2)));
    }
    if (n_self + tot.w > cap_self) {
      cap_self = std::max<int64_t>(2 * cap_self, n_self + tot.w);
      AMFMM_TRY(ensure_keep_bytes(c, c->self_list, cap_self * sizeof(int32_t), n_self * sizeof(int32_t)));
    }
    k_emit<<<grid_for(nf, kBlock), kBlock, 0, st>>>(
        nf, ptr<int2>(c->front[cur]), ptr<int32_t>(c->action), ptr<int4>(c->woff),
        ptr<int32_t>(c->first_child), ptr<int32_t>(c->nchild), ptr<int2>(c->front[cur ^ 1]),
        ptr<int2>(c->m2l), n_m2l, ptr<int2>(c->p2p), n_p2p, ptr<int32_t>(c->self_list), n_self);
    AMFMM_TRY(launched(c, "walk_emit"));
    n_m2l += tot.y;
    n_p2p += tot.z;
    n_self += tot.w;
    nf = tot.x;
    cur ^= 1;
  }
  c->sz.n_m2l = n_m2l;
  c->sz.n_p2p = n_p2p;
  c->sz.n_self = n_self;
  return FMM_OK;
}

}  // namespace amfmm
