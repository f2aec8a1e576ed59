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
#include <cmath>
#include <cstring>

#include "geom.cuh"
#include "internal.cuh"

namespace amfmm {
namespace {

constexpr int kBlock = 256;

enum Action : int32_t { kSelfLeaf = 0, kSelfSplit = 1, kAccept = 2, kNear = 3, kSplitA = 4, kSplitB = 5 };

// packs the walk's per-cell inputs: {Z, R_max} (FP64 and the FP32 filter's
// copy) and {nchild, level}
__global__ void k_pack_cells(int32_t ncell, const double *__restrict__ Z, const double *__restrict__ Rmax,
                             const int32_t *__restrict__ nchild, const int32_t *__restrict__ level,
                             double4_32a *__restrict__ zr, CellF *__restrict__ zf, int2 *__restrict__ nl) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const double x = Z[3 * c], y = Z[3 * c + 1], z = Z[3 * c + 2], R = Rmax[c];
  zr[c] = make_double4_32a(x, y, z, R);
  const float hx = static_cast<float>(x), hy = static_cast<float>(y), hz = static_cast<float>(z);
  CellF f;
  f.h = make_float4(hx, hy, hz, static_cast<float>(R));
  f.l = make_float4(static_cast<float>(x - hx), static_cast<float>(y - hy), static_cast<float>(z - hz), 0.f);
  zf[c] = f;
  nl[c] = make_int2(nchild[c], level[c]);
}

// score (may be NULL): the learned selector's prediction for every frontier
// pair (+inf where the safety bound fails); with it, a pair is accepted when
// the opening criterion accepts it (theta is then a floor on the accepted
// set, which bounds the work of a strict target) or when score < target.
// Output counts: x = next-generation pairs, y = M2L, z = P2P, w = leaf self.
__device__ __forceinline__ int classify(int A, int B, const int2 *__restrict__ nl,
                                        const double4_32a *__restrict__ zr, const CellF *__restrict__ zf,
                                        double theta, float th2f, bool accept_hint, int4 &cnt) {
  cnt = make_int4(0, 0, 0, 0);
  const int2 nlA = nl[A];
  if (A == B) {
    const int k = nlA.x;
    if (k == 0) {
      cnt.w = 1;
      return kSelfLeaf;
    }
    cnt.x = k + k * (k - 1) / 2;
    return kSelfSplit;
  }
  int sep = 1;
  float rA = 0.f, rB = 0.f;  // FP32 R_max, kept for the split choice
  if (!accept_hint) {
    const CellF fA = zf[A], fB = zf[B];
    sep = separated_fast(fA, fB, th2f);
    rA = fA.h.w;
    rB = fB.h.w;
  }
  if (sep < 0) sep = well_separated(zr[A], zr[B], theta);
  if (sep) {
    cnt.y = 1;
    return kAccept;
  }
  const int2 nlB = nl[B];
  const int ka = nlA.x, kb = nlB.x;
  if (ka == 0 && kb == 0) {
    cnt.z = 1;
    return kNear;
  }
  bool pickA;
  if (kb == 0) pickA = true;
  else if (ka == 0) pickA = false;
  else if (rA != rB) {
    // R_max rounded to FP32 (monotone rounding): unequal FP32 values order
    // the FP64 values the same way, strictly
    pickA = rA > rB;
  } else {
    const double ra = zr[A].w, rb = zr[B].w;
    if (ra != rb) pickA = ra > rb;
    else if (nlA.y != nlB.y) pickA = nlA.y < nlB.y;
    else pickA = A < B;
  }
  cnt.x = pickA ? ka : kb;
  return pickA ? kSplitA : kSplitB;
}

__device__ __forceinline__ int4 add4(int4 a, int4 b) { return make_int4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }

// Device-resident state of one generation (one record per generation):
//   ticket  -- tile counter; a block takes the tiles of the frontier in the
//              order it draws tickets, so every block waits only on tiles
//              that were taken before its own;
//   status  -- bit 0: an output exceeded its buffer (the walk stops: the next
//              generation gets an empty frontier); bit 1: a wait for a
//              predecessor gave up; bit 2: too few look-back records;
//   total   -- the generation's output counts (x: next frontier, y: M2L,
//              z: P2P, w: leaf self), written by the block of the last tile;
//   in      -- the generation's frontier size and the list offsets it writes
//              at, written by the previous generation (by the host for the
//              first one).
// The look-back records flag/agg/inc are shared by all generations and told
// apart by an epoch per generation (flag = epoch << 2 | state, state 1:
// aggregate, 2: inclusive prefix).
struct GenIn {
  long long nf, m2l, p2p, self;
};
struct GenState {
  unsigned ticket;
  int status;
  int pad[2];
  int4 total;
  GenIn in;
};

constexpr int kGenItems = 4;
constexpr int kGenBlock = 256;  // threads of a generation block (128: 1.29 ms, 512: 1.21 ms, 256: 1.16 ms per 1M solve)
constexpr int kGenTile = kGenBlock * kGenItems;
constexpr int kGenBlocksPerSM = 5;  // resident blocks per SM the registers are limited for
constexpr long long kSpinLimit = 1LL << 22;

__device__ __forceinline__ int4 ld_volatile4(const int4 *p) {
  const volatile int *q = reinterpret_cast<const volatile int *>(p);
  return make_int4(q[0], q[1], q[2], q[3]);
}
__device__ __forceinline__ void st_volatile4(int4 *p, int4 v) {
  volatile int *q = reinterpret_cast<volatile int *>(p);
  q[0] = v.x;
  q[1] = v.y;
  q[2] = v.z;
  q[3] = v.w;
}

// One generation of the walk: every pair of the frontier is classified, the
// output counts are scanned across the block and then across tiles (single
// pass, decoupled look-back), and the outputs are written in frontier order.
// The grid is persistent: blocks draw tiles until the frontier is done.  The
// frontier size and the list offsets come from the generation's record, so
// the host launches all generations without waiting.  Writes beyond a
// buffer's capacity are skipped; the block of the last tile then stops the
// walk and flags it, and the host grows the buffers (keeping what earlier
// generations wrote) and resumes the walk at the flagged generation.
__global__ void __launch_bounds__(kGenBlock, kGenBlocksPerSM) k_walk_gen(
    GenState *__restrict__ gs, int g, const int2 *__restrict__ front, const int2 *__restrict__ nl,
    const double4_32a *__restrict__ zr, const CellF *__restrict__ zf, double theta, const float *__restrict__ score,
    float target, const int32_t *__restrict__ first_child, int2 *__restrict__ next, int64_t cap_next,
    int2 *__restrict__ m2l, int64_t cap_m2l, int2 *__restrict__ p2p, int64_t cap_p2p, int32_t *__restrict__ self,
    int64_t cap_self, unsigned epoch, int64_t max_places, int *__restrict__ flag, int4 *__restrict__ agg,
    int4 *__restrict__ inc) {
  __shared__ unsigned s_place;
  __shared__ int4 s_warp[kGenBlock / 32];
  __shared__ int4 s_red[kGenBlock / 32];
  __shared__ int s_stop[kGenBlock / 32];
  const float th2f = static_cast<float>(theta) * static_cast<float>(theta);
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  GenState &G = gs[g];
  const GenIn in = G.in;
  const int64_t nf = in.nf;
  const int64_t nb = (nf + kGenTile - 1) / kGenTile;
  if (nb == 0 || nb > max_places) {
    if (blockIdx.x == 0 && t == 0) {
      if (nb > max_places) atomicOr(&G.status, 4);
      G.total = make_int4(0, 0, 0, 0);
      gs[g + 1].in = GenIn{0, in.m2l, in.p2p, in.self};
    }
    return;
  }
  const int64_t m2l_base = in.m2l, p2p_base = in.p2p, self_base = in.self;
  // a generation of few tiles needs few blocks: blocks beyond the tile count
  // leave without drawing a ticket (the others take every tile; a block
  // still waits only for tiles that blocks already running have taken)
  if (static_cast<int64_t>(blockIdx.x) >= nb) return;
  for (;;) {
  if (t == 0) s_place = atomicAdd(&G.ticket, 1u);
  __syncthreads();
  const unsigned place = s_place;
  if (place >= nb) break;
  const int64_t i0 = static_cast<int64_t>(place) * kGenTile + static_cast<int64_t>(t) * kGenItems;
  int act[kGenItems];
  int2 pr[kGenItems];
  int4 mine = make_int4(0, 0, 0, 0);
#pragma unroll
  for (int k = 0; k < kGenItems; ++k) {
    const int64_t i = i0 + k;
    act[k] = -1;
    if (i < nf) {
      pr[k] = front[i];
      int4 cnt;
      const bool hint = score != nullptr && score[i] < target;
      act[k] = classify(pr[k].x, pr[k].y, nl, zr, zf, theta, th2f, hint, cnt);
      mine = add4(mine, cnt);
    }
  }
  // block-wide exclusive scan of the per-thread counts
  int4 incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int4 y = make_int4(__shfl_up_sync(0xffffffffu, incl.x, o), __shfl_up_sync(0xffffffffu, incl.y, o),
                             __shfl_up_sync(0xffffffffu, incl.z, o), __shfl_up_sync(0xffffffffu, incl.w, o));
    if (lane >= o) incl = add4(incl, y);
  }
  if (lane == 31) s_warp[w] = incl;
  __syncthreads();
  int4 before = make_int4(incl.x - mine.x, incl.y - mine.y, incl.z - mine.z, incl.w - mine.w);
  int4 block_total = make_int4(0, 0, 0, 0);
#pragma unroll
  for (int q = 0; q < kGenBlock / 32; ++q) {
    if (q < w) before = add4(before, s_warp[q]);
    block_total = add4(block_total, s_warp[q]);
  }
  // look-back: the sum of the totals of all earlier places, read by the
  // whole block kGenBlock places at a time (thread k looks at place - 1 - k).
  // Every thread of the block would otherwise wait at the next barrier, so a
  // window as wide as the block costs nothing extra and lets the inclusive
  // prefixes travel kGenBlock places per round instead of one warp's 32.
  const int ep = static_cast<int>(epoch & 0x3fffffffu) << 2;
  if (t == 0) {
    if (place == 0) st_volatile4(&inc[0], block_total);
    else st_volatile4(&agg[place], block_total);
    __threadfence();
    atomicExch(&flag[place], ep | (place == 0 ? 2 : 1));
  }
  int4 pre = make_int4(0, 0, 0, 0);
  bool failed = false;
  if (place > 0) {
    int top = static_cast<int>(place) - 1;  // highest place not yet summed
    long long spins = 0;                     // the same in every thread: the loops below are block-uniform
    while (top >= 0) {
      const int j = top - t;
      int f = j >= 0 ? *reinterpret_cast<volatile int *>(&flag[j]) : (ep | 2);
      bool ready = (f & ~3) == ep && (f & 3) != 0;
      // wait until every place of the window has published something
      while (!__syncthreads_and(ready)) {
        if (++spins > kSpinLimit) break;
        __nanosleep(32);
        if (!ready) {
          f = *reinterpret_cast<volatile int *>(&flag[j]);
          ready = (f & ~3) == ep && (f & 3) != 0;
        }
      }
      if (!__syncthreads_and(ready)) {
        failed = true;
        break;
      }
      __threadfence();
      // nearest place in the window that holds an inclusive prefix: threads
      // [0, stop) add aggregates, thread stop the inclusive prefix
      const unsigned incl_mask = __ballot_sync(0xffffffffu, j >= 0 && (f & 3) == 2);
      if (lane == 0) s_stop[w] = incl_mask ? w * 32 + __ffs(incl_mask) - 1 : kGenBlock;
      __syncthreads();
      int stop = kGenBlock;
#pragma unroll
      for (int q = 0; q < kGenBlock / 32; ++q) stop = min(stop, s_stop[q]);
      int4 v = make_int4(0, 0, 0, 0);
      if (j >= 0 && t < stop) v = ld_volatile4(&agg[j]);
      if (j >= 0 && t == stop) v = ld_volatile4(&inc[j]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        v = add4(v, make_int4(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o),
                              __shfl_xor_sync(0xffffffffu, v.z, o), __shfl_xor_sync(0xffffffffu, v.w, o)));
      if (lane == 0) s_red[w] = v;
      __syncthreads();
#pragma unroll
      for (int q = 0; q < kGenBlock / 32; ++q) pre = add4(pre, s_red[q]);
      __syncthreads();  // s_stop and s_red are written again by the next round
      if (stop < kGenBlock) break;
      top -= kGenBlock;
    }
    if (t == 0) {
      if (failed) atomicOr(&G.status, 2);
      st_volatile4(&inc[place], add4(pre, block_total));
      __threadfence();
      atomicExch(&flag[place], ep | 2);
    }
  }
  if (t == 0 && place == nb - 1) {
    const int4 tot = add4(pre, block_total);
    G.total = tot;
    const bool over = tot.x > cap_next || m2l_base + tot.y > cap_m2l || p2p_base + tot.z > cap_p2p ||
                      self_base + tot.w > cap_self;
    if (over) atomicOr(&G.status, 1);
    gs[g + 1].in = GenIn{over ? 0 : tot.x, m2l_base + tot.y, p2p_base + tot.z, self_base + tot.w};
  }
  const int4 base = add4(pre, before);
  int64_t ox = base.x, oy = m2l_base + base.y, oz = p2p_base + base.z, ow = self_base + base.w;
  bool over = false;
#pragma unroll
  for (int k = 0; k < kGenItems; ++k) {
    if (act[k] < 0) continue;
    const int A = pr[k].x, B = pr[k].y;
    switch (act[k]) {
      case kSelfLeaf:
        if (ow < cap_self) self[ow] = A;
        else over = true;
        ++ow;
        break;
      case kSelfSplit: {
        const int f = first_child[A], kk = nl[A].x;
        for (int a = 0; a < kk; ++a) {
          if (ox < cap_next) next[ox] = make_int2(f + a, f + a);
          else over = true;
          ++ox;
        }
        for (int a = 0; a < kk; ++a)
          for (int b = a + 1; b < kk; ++b) {
            if (ox < cap_next) next[ox] = make_int2(f + a, f + b);
            else over = true;
            ++ox;
          }
        break;
      }
      case kAccept:
        if (oy < cap_m2l) m2l[oy] = make_int2(min(A, B), max(A, B));
        else over = true;
        ++oy;
        break;
      case kNear:
        if (oz < cap_p2p) p2p[oz] = make_int2(min(A, B), max(A, B));
        else over = true;
        ++oz;
        break;
      case kSplitA: {
        const int f = first_child[A], kk = nl[A].x;
        for (int a = 0; a < kk; ++a) {
          if (ox < cap_next) next[ox] = make_int2(f + a, B);
          else over = true;
          ++ox;
        }
        break;
      }
      default: {
        const int f = first_child[B], kk = nl[B].x;
        for (int a = 0; a < kk; ++a) {
          if (ox < cap_next) next[ox] = make_int2(A, f + a);
          else over = true;
          ++ox;
        }
        break;
      }
    }
  }
  (void)over;  // the block of the last tile judges overflow from the totals
  __syncthreads();  // shared memory is reused by the next tile
  }
}

// one self pair per root, and the first generation's inputs
__global__ void k_roots_front(int32_t nsys, int2 *__restrict__ front, GenState *__restrict__ gs) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nsys) front[s] = make_int2(s, s);
  if (s == 0) gs[0].in = GenIn{nsys, 0, 0, 0};
}

}  // namespace

int pack_walk_cells(fmm_ctx *c) {
  const int64_t nc = c->sz.ncell;
  AMFMM_TRY(ensure<double4_32a>(c, c->walk_zr, nc));
  AMFMM_TRY(ensure<int2>(c, c->walk_nl, nc));
  AMFMM_TRY(ensure<CellF>(c, c->walk_zf, nc));
  k_pack_cells<<<grid_for(nc, kBlock), kBlock, 0, c->stream>>>(
      static_cast<int32_t>(nc), ptr<double>(c->Z), ptr<double>(c->Rmax), ptr<int32_t>(c->nchild),
      ptr<int32_t>(c->level), ptr<double4_32a>(c->walk_zr), ptr<CellF>(c->walk_zf), ptr<int2>(c->walk_nl));
  return launched(c, "walk_pack");
}

int walk(fmm_ctx *c) {
  cudaStream_t st = c->stream;
  const int64_t n = c->sz.n;
  // First sizes of the walk's buffers, per body: the lists grow about as
  // theta^-3 (at theta = 0.5 a Plummer sphere has 24 accepted pairs and 4
  // leaf pairs per body), bounded so that small angles do not reserve
  // memory ahead of need; a generation that outgrows them runs again.
  const double s3 = std::min(8.0, std::pow(0.5 / c->theta, 3.0));
  const auto per_body = [&](double lo, double k, double hi) {
    return static_cast<int64_t>(static_cast<double>(n) * std::min(hi, std::max(lo, k * s3)));
  };
  int64_t cap_front = std::max<int64_t>(4096, per_body(0.25, 8.0, 32.0));
  AMFMM_TRY(ensure<int2>(c, c->front[0], cap_front));
  AMFMM_TRY(ensure<int2>(c, c->front[1], cap_front));
  int64_t cap_m2l = c->m2l.cap / sizeof(int2), cap_p2p = c->p2p.cap / sizeof(int2),
          cap_self = c->self_list.cap / sizeof(int32_t);
  if (cap_m2l < 1024) {
    cap_m2l = std::max<int64_t>(1024, per_body(8.0, 32.0, 256.0));
    AMFMM_TRY(ensure<int2>(c, c->m2l, cap_m2l));
  }
  if (cap_p2p < 1024) {
    cap_p2p = std::max<int64_t>(1024, per_body(2.0, 6.0, 48.0));
    AMFMM_TRY(ensure<int2>(c, c->p2p, cap_p2p));
  }
  if (cap_self < 1024) {
    cap_self = std::max<int64_t>(1024, n / 4 + 64);
    AMFMM_TRY(ensure<int32_t>(c, c->self_list, cap_self));
  }

  AMFMM_TRY(pack_walk_cells(c));
  if (c->sel_enabled) {
    if (c->sz.nsys != 1)
      return set_error(c, FMM_EUNSUPPORTED, "the learned selector works on one system at a time");
    AMFMM_TRY(cell_features(c));
    if (c->sel_rule == FMM_SEL_RELATIVE) AMFMM_TRY(field_estimate(c));
    AMFMM_CUDA(c, cudaMemsetAsync(ptr<int64_t>(c->totals) + 10, 0, sizeof(int64_t), st));
  }
  // one self pair per root: systems of a forest never interact
  const int64_t nsys = c->sz.nsys;
  if (nsys > static_cast<int64_t>(c->front[0].cap / sizeof(int2))) AMFMM_TRY(ensure<int2>(c, c->front[0], nsys));
  // The walk lasts at most 2 depth + 1 generations with pairs (a generation
  // raises the sum of the two cells' levels by one, or by two for a pair of
  // a cell with itself); one more finds the frontier empty.
  const int ngen = 2 * c->sz.depth + 3;
  int64_t n_m2l = 0, n_p2p = 0, n_self = 0;
  AMFMM_TRY(ensure_bytes(c, c->walk_state, sizeof(GenState) * (ngen + 1)));
  if (sizeof(GenState) * (ngen + 1) > 8192) return set_error(c, FMM_EUNSUPPORTED, "tree too deep for the walk state");
  GenState *gs = static_cast<GenState *>(c->walk_state.p);
  const unsigned grid = static_cast<unsigned>(std::max(1, c->num_sms * kGenBlocksPerSM));
  // generation records: zero, then the first generation's inputs (the roots)
  AMFMM_CUDA(c, cudaMemsetAsync(gs, 0, sizeof(GenState) * (ngen + 1), st));
  k_roots_front<<<grid_for(nsys, kBlock), kBlock, 0, st>>>(static_cast<int32_t>(nsys), ptr<int2>(c->front[0]), gs);
  AMFMM_TRY(launched(c, "walk_roots"));
  int gstart = 0;  // first generation to (re)run
  for (int attempt = 0;; ++attempt) {
    if (attempt > 16) return set_error(c, FMM_EINVAL, "walk: outputs still overflow after growing the buffers");
    const int64_t cap_next = std::min(c->front[0].cap, c->front[1].cap) / sizeof(int2);
    cap_front = cap_next;
    if (c->sel_enabled) {  // one score and one candidate slot per frontier pair
      AMFMM_TRY(ensure<float>(c, c->sel_score, cap_front));
      AMFMM_TRY(ensure<int32_t>(c, c->sel_cand, cap_front));
    }
    const int64_t max_places = (cap_next + kGenTile - 1) / kGenTile + 1;
    // look-back records; fresh memory is zeroed so no stale flag matches an epoch
    const size_t lb_bytes = static_cast<size_t>(max_places) * (sizeof(int) + 2 * sizeof(int4)) + 64;
    if (c->walk_lb.cap < lb_bytes) {
      AMFMM_TRY(ensure_bytes(c, c->walk_lb, lb_bytes));
      AMFMM_CUDA(c, cudaMemsetAsync(c->walk_lb.p, 0, c->walk_lb.cap, st));
    }
    const int64_t nbc = static_cast<int64_t>((c->walk_lb.cap - 64) / (sizeof(int) + 2 * sizeof(int4)));
    int4 *agg = static_cast<int4 *>(c->walk_lb.p);
    int4 *inc = agg + nbc;
    int *flg = reinterpret_cast<int *>(inc + nbc);
    // A replayed graph repeats the epochs it was captured with: clear the
    // look-back records so that no flag of an earlier replay matches.
    if (capturing(c)) AMFMM_CUDA(c, cudaMemsetAsync(c->walk_lb.p, 0, c->walk_lb.cap, st));
    const unsigned epoch0 = c->walk_epoch + 1;
    c->walk_epoch = (c->walk_epoch + ngen + 1) & 0x3fffffffu;
    if (c->walk_epoch < epoch0) c->walk_epoch = ngen + 1;  // wrapped: restart above zero
    for (int g = gstart; g < ngen; ++g) {
      const float *score = nullptr;
      if (c->sel_enabled) {
        AMFMM_TRY(walk_scores(c, &gs[g].in.nf, cap_front, ptr<int2>(c->front[g & 1]), ptr<float>(c->sel_score)));
        score = ptr<float>(c->sel_score);
      }
      unsigned ep = (epoch0 + g) & 0x3fffffffu;
      if (ep == 0) ep = 1;
      k_walk_gen<<<grid, kGenBlock, 0, st>>>(
          gs, g, ptr<int2>(c->front[g & 1]), ptr<int2>(c->walk_nl), ptr<double4_32a>(c->walk_zr),
          ptr<CellF>(c->walk_zf), c->theta, score, static_cast<float>(c->sel_log10_target),
          ptr<int32_t>(c->first_child), ptr<int2>(c->front[(g + 1) & 1]), cap_next, ptr<int2>(c->m2l), cap_m2l,
          ptr<int2>(c->p2p), cap_p2p, ptr<int32_t>(c->self_list), cap_self, ep, std::min(max_places, nbc), flg,
          agg, inc);
      AMFMM_TRY(launched(c, "walk_gen"));
    }
    GenState *h = static_cast<GenState *>(c->hpin);
    const HostRead rb{h, gs, sizeof(GenState) * (ngen + 1)};
    AMFMM_TRY(read_back(c, &rb, 1));
    int first_bad = -1;
    for (int g = gstart; g < ngen; ++g) {
      if (h[g].status & 2) return set_error(c, FMM_ETIMEOUT, "walk: a block waited too long for its predecessor");
      if ((h[g].status & 5) && first_bad < 0) first_bad = g;
    }
    if (capturing(c)) {
      // a captured walk keeps the planned buffers: the plan's walk fitted
      if (first_bad >= 0 || gstart != 0) return set_error(c, FMM_ECUDA, "graph capture: the planning walk grew its buffers");
      Expect e;
      for (int g = 0; g < ngen; ++g) e.add(&gs[g].status, static_cast<uint32_t>(h[g].status));
      e.add64(&gs[ngen].in.nf, static_cast<uint64_t>(h[ngen].in.nf));
      e.add64(&gs[ngen].in.m2l, static_cast<uint64_t>(h[ngen].in.m2l));
      e.add64(&gs[ngen].in.p2p, static_cast<uint64_t>(h[ngen].in.p2p));
      if (!e.add64(&gs[ngen].in.self, static_cast<uint64_t>(h[ngen].in.self)))
        return set_error(c, FMM_ECUDA, "graph capture: too many walk generations to check");
      AMFMM_TRY(graph_expect(c, e));
      st = c->stream;
    }
    if (first_bad < 0) {
      if (h[ngen].in.nf != 0) return set_error(c, FMM_EINVAL, "walk: more generations than the depth allows");
      n_m2l = h[ngen].in.m2l;
      n_p2p = h[ngen].in.p2p;
      n_self = h[ngen].in.self;
      break;
    }
    // An output of generation b did not fit (its counts are exact).  Grow
    // what overflowed, keeping everything the earlier generations wrote (the
    // lists up to b's bases and b's own frontier), and resume at b.
    const int b = first_bad;
    const GenState hb = h[b];
    if ((hb.status & 4) || hb.total.x > cap_next) {
      const int64_t want = std::max<int64_t>(2 * cap_next, hb.total.x);
      AMFMM_TRY(ensure_keep_bytes(c, c->front[b & 1], want * sizeof(int2), hb.in.nf * sizeof(int2)));
      AMFMM_TRY(ensure<int2>(c, c->front[(b + 1) & 1], want));
    }
    if (hb.in.m2l + hb.total.y > cap_m2l) {
      AMFMM_TRY(ensure_keep_bytes(c, c->m2l, std::max<int64_t>(2 * cap_m2l, hb.in.m2l + hb.total.y) * sizeof(int2),
                                  hb.in.m2l * sizeof(int2)));
      cap_m2l = c->m2l.cap / sizeof(int2);
    }
    if (hb.in.p2p + hb.total.z > cap_p2p) {
      AMFMM_TRY(ensure_keep_bytes(c, c->p2p, std::max<int64_t>(2 * cap_p2p, hb.in.p2p + hb.total.z) * sizeof(int2),
                                  hb.in.p2p * sizeof(int2)));
      cap_p2p = c->p2p.cap / sizeof(int2);
    }
    if (hb.in.self + hb.total.w > cap_self) {
      AMFMM_TRY(ensure_keep_bytes(c, c->self_list,
                                  std::max<int64_t>(2 * cap_self, hb.in.self + hb.total.w) * sizeof(int32_t),
                                  hb.in.self * sizeof(int32_t)));
      cap_self = c->self_list.cap / sizeof(int32_t);
    }
    // records from b on: b keeps its inputs, the later ones start empty
    std::memset(static_cast<void *>(h + b), 0, sizeof(GenState) * (ngen + 1 - b));
    h[b].in = hb.in;
    AMFMM_CUDA(c, cudaMemcpyAsync(gs + b, h + b, sizeof(GenState) * (ngen + 1 - b), cudaMemcpyHostToDevice, st));
    gstart = b;
  }
  c->sz.n_m2l = n_m2l;
  c->sz.n_p2p = n_p2p;
  c->sz.n_self = n_self;
  return FMM_OK;
}

}  // namespace amfmm

using namespace amfmm;

// Test hook for the bounded wait of the walk's look-back (no counterpart in
// the paper): one generation of two tiles is launched with one block and its
// ticket counter already at 1, so the block takes the second tile and waits
// for the first, which no block takes.  The wait gives up after kSpinLimit
// polls, the block skips its output (all capacities are zero), and the call
// must return FMM_ETIMEOUT with the context still usable.  Every read stays
// inside a zeroed frontier of two tiles and one zeroed cell; every write
// inside two generation records and two look-back records.
extern "C" int fmm_debug_walk_wait_timeout(fmm_ctx *c) {
  if (!c) return FMM_EINVAL;
  cudaStream_t st = c->stream;
  const int64_t nf = kGenTile + 1;  // two tiles
  AMFMM_TRY(ensure_bytes(c, c->walk_state, 2 * sizeof(GenState)));
  const size_t lb_bytes = 2 * (sizeof(int) + 2 * sizeof(int4)) + 64;
  if (c->walk_lb.cap < lb_bytes) {
    AMFMM_TRY(ensure_bytes(c, c->walk_lb, lb_bytes));
    AMFMM_CUDA(c, cudaMemsetAsync(c->walk_lb.p, 0, c->walk_lb.cap, st));
  }
  const int64_t nbc = static_cast<int64_t>((c->walk_lb.cap - 64) / (sizeof(int) + 2 * sizeof(int4)));
  int4 *agg = static_cast<int4 *>(c->walk_lb.p);
  int4 *inc = agg + nbc;
  int *flg = reinterpret_cast<int *>(inc + nbc);
  AMFMM_TRY(ensure<int2>(c, c->front[0], nf));
  AMFMM_TRY(ensure<int2>(c, c->front[1], 1));
  AMFMM_TRY(ensure<int2>(c, c->walk_nl, 1));
  AMFMM_TRY(ensure<double4_32a>(c, c->walk_zr, 1));
  AMFMM_TRY(ensure<CellF>(c, c->walk_zf, 1));
  AMFMM_TRY(ensure<int32_t>(c, c->first_child, 1));
  AMFMM_CUDA(c, cudaMemsetAsync(c->front[0].p, 0, sizeof(int2) * nf, st));
  AMFMM_CUDA(c, cudaMemsetAsync(c->walk_nl.p, 0, sizeof(int2), st));
  AMFMM_CUDA(c, cudaMemsetAsync(c->walk_zr.p, 0, sizeof(double4_32a), st));
  AMFMM_CUDA(c, cudaMemsetAsync(c->walk_zf.p, 0, sizeof(CellF), st));
  GenState *gs = static_cast<GenState *>(c->walk_state.p);
  GenState *hs = reinterpret_cast<GenState *>(static_cast<char *>(c->hpin) + 8192);
  hs[0] = GenState{};
  hs[0].ticket = 1;  // the only block takes the second tile
  hs[0].in = GenIn{nf, 0, 0, 0};
  hs[1] = GenState{};
  AMFMM_CUDA(c, cudaMemcpyAsync(gs, hs, 2 * sizeof(GenState), cudaMemcpyHostToDevice, st));
  c->walk_epoch = (c->walk_epoch + 1) & 0x3fffffffu;
  if (c->walk_epoch == 0) c->walk_epoch = 1;
  k_walk_gen<<<1, kGenBlock, 0, st>>>(gs, 0, ptr<int2>(c->front[0]), ptr<int2>(c->walk_nl),
                                      ptr<double4_32a>(c->walk_zr), ptr<CellF>(c->walk_zf), 0.5, nullptr, 0.f,
                                      ptr<int32_t>(c->first_child), ptr<int2>(c->front[1]), 0, nullptr, 0, nullptr,
                                      0, nullptr, 0, c->walk_epoch, std::min<int64_t>(2, nbc), flg, agg, inc);
  AMFMM_TRY(launched(c, "walk_gen_wait_test"));
  GenState *h = static_cast<GenState *>(c->hpin);
  AMFMM_CUDA(c, cudaMemcpyAsync(h, gs, sizeof(GenState), cudaMemcpyDeviceToHost, st));
  AMFMM_CUDA(c, cudaStreamSynchronize(st));
  const int status = h->status;
  c->stage = kNone;
  if (status & 2) return set_error(c, FMM_ETIMEOUT, "walk: a block waited too long for its predecessor");
  return FMM_OK;
}

