// internal.cuh -- context, device buffers and launch helpers shared by the
// translation units of libamfmm.so.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/amfmm.h"

namespace amfmm {

constexpr int kMaxLevel = 21;   // 63-bit Morton keys: 21 octal digits
constexpr int kMomStride = 20;  // M, dipole(3), Q(6), O(10)
constexpr int kLocStride = 20;  // C_i(3), C_ij(6), C_ijk(10), pad

// Growable device buffer; contents are discarded on growth.
struct DBuf {
  void *p = nullptr;
  size_t cap = 0;
};

struct Err {
  int code = FMM_OK;
  std::string msg;
};

// Per-solve sizes read back to the host.
struct Sizes {
  int64_t n = 0, ncell = 0, nleaf = 0, n_m2l = 0, n_p2p = 0, n_self = 0;
  int depth = 0;
  int key_which = 0;             // ping-pong slot holding the sorted keys
  int nsys = 1;                  // independent systems (roots) in the forest
  double lo[3] = {0, 0, 0}, scale = 0;
  int64_t p2p_body_pairs = 0;
  int64_t p2p_items = 0;         // near-field work items (chunks of the leaves' column streams)
  std::vector<int64_t> lvl_off;  // cells of level l are [lvl_off[l], lvl_off[l+1])
};

enum Stage { kNone = 0, kTree = 1, kUp = 2, kInteract = 3, kDown = 4 };

// Graph-captured solves (graph.cu).  kGraphRecord: a plain solve that keeps
// every value it reads back from the device; kGraphCapture: the same host
// code run again under stream capture, taking those values instead of
// reading them.
enum GraphMode { kGraphOff = 0, kGraphRecord = 1, kGraphCapture = 2 };
constexpr int kMaxGraphDepth = 24;  // capture streams: the graph and one per nested check
constexpr int kMaxExpect = 96;      // device words one check compares

// What a solve's graph was captured for: a replay is valid only for the
// same caller buffers, sizes and options, and only while no device buffer
// of the context has been reallocated since.
struct GraphKey {
  const void *p[7] = {};
  int64_t n = 0;
  int nsys = 0;
  double theta = 0, eps2 = 0, G = 0;
  int n_crit = 0, order_P = 0, variant = 0, precision = 0, rows = 0;
  int64_t alloc_gen = -1;
  bool operator==(const GraphKey &o) const {
    for (int k = 0; k < 7; ++k)
      if (p[k] != o.p[k]) return false;
    return n == o.n && nsys == o.nsys && theta == o.theta && eps2 == o.eps2 && G == o.G && n_crit == o.n_crit &&
           order_P == o.order_P && variant == o.variant && precision == o.precision && rows == o.rows &&
           alloc_gen == o.alloc_gen;
  }
};

// Device words with the values the planning solve read there: a captured
// check lets the rest of the graph run only if every word still holds its
// value (passed to the check kernel by value).
struct Expect {
  const uint32_t *addr[kMaxExpect];
  uint32_t val[kMaxExpect];
  int n = 0;
  bool add(const void *dev_word, uint32_t v) {
    if (n >= kMaxExpect) return false;
    addr[n] = static_cast<const uint32_t *>(dev_word);
    val[n++] = v;
    return true;
  }
  bool add64(const void *dev_dword, uint64_t v) {
    const uint32_t *w = static_cast<const uint32_t *>(dev_dword);
    return add(w, static_cast<uint32_t>(v)) && add(w + 1, static_cast<uint32_t>(v >> 32));
  }
};

// Result record of a replay: done = 1 once the innermost check passed and
// the solve's last kernel ran; the bounding cube for the statistics.
struct GraphRec {
  uint32_t done;
  uint32_t pad;
  double lo[3], scale;
};
constexpr size_t kGraphRecHostOff = 12288;  // its pinned host copy inside hpin

enum TimerSlot {
  kTreeBeg = 0, kTreeEnd, kUpBeg, kUpEnd, kWalkBeg, kWalkEnd, kM2LBeg, kM2LEnd,
  kP2PBeg, kP2PEnd, kRedBeg, kRedEnd, kDownBeg, kDownEnd, kNumTimers
};

}  // namespace amfmm

struct fmm_ctx {
  fmm_opts opts{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  char errbuf[512] = {0};
  int stage = amfmm::kNone;
  bool timing = false;
  cudaEvent_t ev[amfmm::kNumTimers] = {};
  int64_t launches = 0, launches_last = 0;
  float stage_ms[7] = {0, 0, 0, 0, 0, 0, 0};

  // solve inputs (caller-owned device memory)
  const double *x = nullptr, *y = nullptr, *z = nullptr, *m = nullptr;
  double theta = 0.5;
  double eps2 = 0.0;  // Plummer softening length squared (0: the paper's unsoftened 1/R)
  int p2p_rows = 16;  // leaf tile: rows of a leaf staged per pass of the near field (8, 16 or 32)
  amfmm::Sizes sz;
  int m2l_which = 0;  // which of the ekey/eval buffers holds the sorted M2L entries
  int p2p_order = -1;  // which pval buffer holds the near field's item order (-1: items in index order)

  // pinned host scratch for small read-backs
  void *hpin = nullptr;

  // ---- device buffers ----
  // bodies
  amfmm::DBuf key[2], idx[2], order, X, Y, Zb, Mb, cur, flag, incl, lcp, leaf_of, cell_at,
      near, acc, status, bbox_part, bbox, sys_off, sysid, sbox;
  // cells
  amfmm::DBuf begin, count, level, parent, first_child, nchild, S, M, Z, invM, Rmax,
      rmax2, mom, loc, leaves;
  // walk
  amfmm::DBuf front[2], m2l, p2p, self_list, walk_zr, walk_zf, walk_nl, walk_state, walk_lb;
  int last_depth = 0;        // depth of the previous tree: levels of the first batch of the next build
  unsigned walk_epoch = 0;  // epochs of the single-pass walk generations
  // M2L scatter
  amfmm::DBuf ekey[2], eval[2], m2l_pos, m2l_off, m2l_slots, cell32, qoh;
  // P2P grouping
  amfmm::DBuf pkey[2], pval[2], p2p_A, p2p_offA, p2p_offB, p2p_pos, p2p_poff, p2p_len,
      p2p_slots, p2p_colOff, p2p_cols, p2p_nb, p2p_pre, p2p_bodyf, p2p_items, p2p_itemOff, p2p_extraOff,
      p2p_extra;
  // scan / sort scratch; `totals` holds small device results (1 KiB):
  // [0,16) scan totals, [64,72) near-field body-pair count, [80,88) selector-scored pairs, [88,92) selector candidates, [96,104) slot total,
  // [128,140) near-field column, work-item and extra-partial totals, [160,168) work queues (near field, gathered far field)
  amfmm::DBuf scan_tmp, sort_hist, totals, diag;
  // learned pair selector
  amfmm::DBuf sel_params, sel_cellfeat, sel_cand, sel_lga, sel_scratch, sel_part, sel_score, sel_grad, sel_perm, sel_xb, sel_yb;
  bool sel_enabled = false;
  double sel_log10_target = -3.0;
  double sel_theta_max = 1.0;  // upper edge of the band the network decides
  int64_t sel_min_work = 256;  // pairs with n_A n_B below this are left to the floor
  int sel_rule = FMM_SEL_RELATIVE;  // acceptance rule of the learned selector
  // index tables of the table-driven general order (P = 6 .. 8)
  amfmm::DBuf gen_tab;
  // host-solve staging
  amfmm::DBuf hx, hy, hz, hm, hax, hay, haz;
  // graph-captured solves
  bool graph_enabled = false;
  int gmode = amfmm::kGraphOff;
  std::vector<std::vector<unsigned char>> gplan;  // read-backs of the planning solve, in order
  std::vector<std::vector<unsigned char>> gplan_prev;  // those of the solve before
  size_t gplan_pos = 0;
  bool gwait = false;  // after a failed replay: capture again only once a plan repeats
  char gerrbuf[512] = {0};  // why the last capture was abandoned
  cudaStream_t gstream[amfmm::kMaxGraphDepth] = {};  // [0] the graph, [d] the body of the d-th check
  int gdepth = 0;
  cudaGraphExec_t gexec = nullptr;
  amfmm::GraphKey gkey;
  amfmm::Sizes gsz;          // sizes of the captured solve
  int64_t glaunches = 0;     // kernels in the captured graph
  int64_t alloc_gen = 0;     // device (re)allocations so far
  int64_t g_replays = 0, g_captures = 0, g_fallbacks = 0, g_capture_failures = 0;
  bool last_replay = false;  // the last solve was a graph replay (no stage timers)
  amfmm::DBuf grec;          // GraphRec of the replays
};

namespace amfmm {

// ---------------------------------------------------------------------------
// errors and allocation
// ---------------------------------------------------------------------------
int set_error(fmm_ctx *c, int code, const char *fmt, ...);

#define AMFMM_CUDA(c, call)                                                              \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return ::amfmm::set_error((c), FMM_ECUDA, "%s failed: %s (%s:%d)", #call,          \
                                cudaGetErrorString(e_), __FILE__, __LINE__);             \
  } while (0)

#define AMFMM_TRY(expr)        \
  do {                         \
    int rc_ = (expr);          \
    if (rc_ != FMM_OK) return rc_; \
  } while (0)

int ensure_bytes(fmm_ctx *c, DBuf &b, size_t bytes);
// Grows keeping the first `used` bytes.
int ensure_keep_bytes(fmm_ctx *c, DBuf &b, size_t bytes, size_t used);

template <class T>
inline int ensure(fmm_ctx *c, DBuf &b, size_t count) {
  return ensure_bytes(c, b, count * sizeof(T));
}
template <class T>
inline T *ptr(DBuf &b) {
  return static_cast<T *>(b.p);
}

// Checks the last launch and counts it.
int launched(fmm_ctx *c, const char *what);

inline unsigned grid_for(int64_t n, int block) {
  return static_cast<unsigned>((n + block - 1) / block);
}

// ---------------------------------------------------------------------------
// primitives (sort.cu)
// ---------------------------------------------------------------------------
// Exclusive prefix sums; `total` (device, 1 element) receives the sum.
int exclusive_scan_i32(fmm_ctx *c, const int32_t *in, int32_t *out, int64_t n, int32_t *total);
int exclusive_scan_i64(fmm_ctx *c, const int64_t *in, int64_t *out, int64_t n, int64_t *total);
int exclusive_scan_i4(fmm_ctx *c, const int4 *in, int4 *out, int64_t n, int4 *total);
// Stable LSD radix sort of (key, value) pairs on the low `bits` key bits.
// Sorted data ends in buffer index *which (0 or 1) of the ping-pong pairs.
int radix_sort_u64(fmm_ctx *c, DBuf key[2], DBuf val[2], int64_t n, int bits, int *which);
int radix_sort_u32(fmm_ctx *c, DBuf key[2], DBuf val[2], int64_t n, int bits, int *which);

// ---------------------------------------------------------------------------
// stages
// ---------------------------------------------------------------------------
int build_tree(fmm_ctx *c);         // tree.cu
int upward(fmm_ctx *c);             // tree.cu
int walk(fmm_ctx *c);               // walk.cu
int pack_walk_cells(fmm_ctx *c);    // walk.cu: per-cell records of the criterion
int m2l_prepare(fmm_ctx *c);        // m2l.cu: slot positions (sort by cell)
int m2l_run(fmm_ctx *c);            // m2l.cu: mutual M2L into slots
int m2l_reduce(fmm_ctx *c);         // m2l.cu: per-cell fixed-order sums
// the mixed form at order 3 gathers each cell's partners (one-sided, no slots)
inline bool m2l_gathered(const fmm_ctx *c) { return c->opts.precision == FMM_MIXED && c->opts.order_P == 3; }
int p2p_prepare(fmm_ctx *c);        // p2p.cu: grouping by leaf, partial slots
int p2p_run(fmm_ctx *c);            // p2p.cu: mutual near field
int p2p_reduce(fmm_ctx *c);         // p2p.cu: per-body fixed-order sums
int downward(fmm_ctx *c);           // down.cu (L2L, L2P into sorted order)
int forces(fmm_ctx *c, double *ax, double *ay, double *az);  // down.cu (caller order)

// general order P (expansion.cu)
int mom_stride(int P);  // moments of order 0..P per cell
int loc_stride(int P);  // local coefficients per cell (order 3: 20 with padding)
int upward_general(fmm_ctx *c);
int m2l_general(fmm_ctx *c);
int reduce_general(fmm_ctx *c);
int downward_general(fmm_ctx *c);
// the same stages at P = 6 .. 8, table-driven (expansion_table.cu)
int upward_table(fmm_ctx *c);
int m2l_table(fmm_ctx *c);
int downward_table(fmm_ctx *c);

// learned selector (selector.cu, m2l.cu)
int cell_features(fmm_ctx *c);  // per-cell parts of the selector's features
int field_estimate(fmm_ctx *c);  // per-cell log10 |a| estimate of the selector's relative rule
int walk_scores(fmm_ctx *c, const long long *nf_dev, int64_t cap, const int2 *front, float *score);
int pair_locals_tc(fmm_ctx *c, const int2 *pairs, int64_t K, double *out);

void timer(fmm_ctx *c, int slot);

// ---------------------------------------------------------------------------
// read-backs and graph capture (graph.cu)
// ---------------------------------------------------------------------------
// Device values that steer the host's launches: copied and waited for in a
// plain solve (and kept when recording a plan); taken from the plan, in the
// same order, while capturing.  `host` must be pinned (hpin).
struct HostRead {
  void *host;
  const void *dev;
  size_t bytes;
};
int read_back(fmm_ctx *c, const HostRead *r, int nr);
inline bool capturing(const fmm_ctx *c) { return c->gmode == kGraphCapture; }
// While capturing: a check that the device words hold the planned values,
// and a conditional node under which the rest of the solve is captured
// (c->stream becomes the body's capture stream).  No-op otherwise.
int graph_expect(fmm_ctx *c, const Expect &e);
// Copies the bounding cube (4 doubles: lo, scale) into the replay record.
int graph_record_bbox(fmm_ctx *c, const double *bbox);
// The solve as one graph launch (graph.cu); begin_solve has run.
bool graph_usable(const fmm_ctx *c);
int graph_solve(fmm_ctx *c, double *ax, double *ay, double *az);
// The stages of a solve after begin_solve (api.cu).
int run_stages(fmm_ctx *c, double *ax, double *ay, double *az);

}  // namespace amfmm
