/*
 * amfmm.h -- C ABI of the GB300 (sm_103a) angular-momentum-conserving
 * Cartesian fast multipole method (Marcello 2017, arXiv:1706.06989, a
 * modification of Dehnen 2000).
 *
 * Problem (Sec. 2): N bodies with positions X_n and masses mu_n; find every
 * body's gravitational acceleration a_n = G sum_m mu_m (X_m - X_n)/|X_m - X_n|^3
 * approximated by a symmetric (mutual) cell-cell expansion to order P = 3
 * with the paper's torque-cancelling correction, so that the interactions
 * conserve linear momentum (Eq. "unit") and angular momentum (Eq. 7 / Eq. 8,
 * App. A) to rounding.
 *
 * Call sequence for one force solve (each call is enqueued on the context's
 * CUDA stream; calls that must learn a size synchronise that stream and say
 * so below):
 *     fmm_build_tree -> fmm_upward -> fmm_interact -> fmm_downward -> fmm_forces
 * A call out of this order returns FMM_EORDER.  fmm_solve runs all five.
 *
 * Memory: every pointer argument named "device" is CUDA device memory owned
 * by the caller; the library never frees or retains it beyond the call,
 * except that the body arrays given to fmm_build_tree are read again (not
 * copied) by fmm_upward .. fmm_forces of the same solve and must stay
 * unchanged until fmm_forces returns.  The context owns every internal
 * buffer (tree, lists, expansion slots) and grows them on demand with
 * cudaMalloc; they are released by fmm_destroy.
 *
 * Errors: every int-returning call returns FMM_OK (0) or a negative code;
 * fmm_last_error gives a one-line message.  A failed call leaves the
 * context usable for a new fmm_build_tree.  Input validation: n >= 1,
 * 0 < theta <= 1 (Sec. 2), n_crit >= 1, order_P in {3, 4, 5}; a body with a
 * non-finite coordinate or a mass that is not positive and finite is
 * detected on the device and reported as FMM_EINVAL by the next call that
 * synchronises (fmm_build_tree).
 *
 * Units and conventions: G from fmm_opts (1 for the paper's units); an
 * unsoftened 1/R potential; a pair of bodies (or cells) at zero separation
 * contributes nothing.
 */
#ifndef AMFMM_H
#define AMFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FMM_OK 0
#define FMM_EINVAL (-1)       /* bad argument or bad body data */
#define FMM_ENOMEM (-2)       /* device allocation failed */
#define FMM_ECUDA (-3)        /* a CUDA call or kernel launch failed */
#define FMM_ETIMEOUT (-4)     /* a bounded device wait expired */
#define FMM_EORDER (-5)       /* call out of sequence */
#define FMM_EUNSUPPORTED (-6) /* option not built */
#define FMM_ESIZE (-7)        /* input larger than a fixed capacity */

/* Variants of Sec. 3. */
#define FMM_UC 0  /* uncorrected Dehnen (2000) expansion */
#define FMM_TC 1  /* torque corrected with D_ijkl (Eq. 7) */
#define FMM_TCO 2 /* torque corrected with the reduced D'_ijkl (Eq. 8) */

/* Arithmetic of the interaction kernels. */
#define FMM_FP64 0  /* every stage in FP64 */
#define FMM_MIXED 1 /* near field and M2L in FP32 on cell-relative coordinates,
                       FP64 tree geometry, moments and accumulation */

typedef struct fmm_ctx fmm_ctx;

typedef struct {
  double theta;  /* opening angle, 0 < theta <= 1 (Sec. 2) */
  int n_crit;    /* a cell with at most n_crit bodies is a leaf (Sec. 2: 25) */
  int order_P;   /* expansion order: 3 (Eqs. 2-4), or 4, 5 (App. A; FP64 only) */
  int variant;   /* FMM_UC, FMM_TC or FMM_TCO */
  int precision; /* FMM_FP64 or FMM_MIXED */
  double G;      /* gravitational constant applied to the accelerations */
} fmm_opts;

typedef struct {
  int64_t n;          /* bodies */
  int64_t ncell;      /* cells of the octree */
  int64_t nleaf;      /* leaves */
  int32_t depth;      /* deepest level (root = 0, at most 21) */
  int64_t n_m2l;      /* accepted cell pairs (mutual M2L) */
  int64_t n_p2p;      /* leaf pairs summed directly (mutual P2P) */
  int64_t n_self;     /* leaves summed directly with themselves */
  int64_t p2p_body_pairs; /* sum over leaf pairs of n_A n_B plus n(n-1)/2 per self leaf */
  int64_t launches;   /* kernels launched by the last completed solve */
  double lo[3];       /* bounding-cube origin used for the Morton keys */
  double scale;       /* 2^21 / cube extent (0 for a cube of zero extent) */
  /* per-stage device time in ms of the last solve, when timing is enabled
     with fmm_set_timing: tree, upward, walk, m2l, p2p, reduce, downward */
  float ms_tree, ms_upward, ms_walk, ms_m2l, ms_p2p, ms_reduce, ms_downward;
  int64_t n_scored;   /* pairs the learned selector evaluated in the last solve (0 without it) */
} fmm_stats;

/* Creates a context bound to `cuda_stream` (a cudaStream_t; NULL = the
 * legacy default stream) on the current device.  *ctx is set on success. */
int fmm_create(fmm_ctx **ctx, const fmm_opts *opts, void *cuda_stream);
void fmm_destroy(fmm_ctx *ctx);
const char *fmm_last_error(const fmm_ctx *ctx);
/* Replaces the options between solves (theta, n_crit, variant, precision, G). */
int fmm_set_opts(fmm_ctx *ctx, const fmm_opts *opts);
/* 1: record CUDA events around every stage (fmm_get_stats reports them). */
int fmm_set_timing(fmm_ctx *ctx, int enable);
/* Plummer softening of the following solves and of fmm_direct: every
 * interaction (M2L, P2P) and the direct sums use G(R) = -1/sqrt(R^2 + eps^2)
 * instead of the paper's -1/R.  The paper notes (Sec. 4) that the
 * angular-momentum correction carries over to any Green's function of the
 * distance alone; it is applied unchanged (the derivative tensors keep their
 * form with R^2 -> R^2 + eps^2), so TC and TCO still cancel every pair's
 * torque.  The tree, the opening criterion and the lists do not depend on
 * eps.  eps = 0 (the default) is the unsoftened method.  Built at order
 * P = 3 (FP64 and mixed); a softened solve at P = 4, 5 returns
 * FMM_EUNSUPPORTED from fmm_interact.  FMM_EINVAL for eps < 0 or not finite.
 * The learned selector's training labels stay those of the unsoftened
 * expansion. */
int fmm_set_softening(fmm_ctx *ctx, double eps);
/* Leaf tile of the near field (a8): the number of a leaf's bodies (rows) the
 * mutual P2P kernel stages in shared memory per pass over the leaf's partner
 * columns, 8, 16 (the default) or 32.  Larger tiles take fewer passes over the
 * columns of big leaves; smaller ones fit more warps per SM.  The result is
 * the same sum in another order of the work: FP64 results differ from one
 * tile to another only by rounding.  FMM_EINVAL for other values. */
int fmm_set_tile(fmm_ctx *ctx, int rows);

/* a1-a3 (Sec. 2, first paragraph): bounding cube, 63-bit Morton keys, stable
 * radix sort by (key, index), octree whose leaves hold at most n_crit bodies
 * (or sit at level 21), numbered breadth first.  x, y, z, m: device, n
 * doubles each, caller order.  `theta` overrides opts.theta for this solve
 * (pass 0 to keep it).  Synchronises the stream (the level sizes are read
 * back). */
int fmm_build_tree(fmm_ctx *ctx, const double *x, const double *y, const double *z,
                   const double *m, int64_t n, double theta);

/* a4 (Eqs. 1-3 and the octupole definition): per cell mass M, centre of
 * mass Z, R_max (the largest body distance from Z) and moments about Z to
 * order P (leaf P2M from bodies, then M2M shifts).  Asynchronous. */
int fmm_upward(fmm_ctx *ctx);

/* a5-a8: dual-tree walk under the opening criterion
 * |Z_A - Z_B| >= (R_A,max + R_B,max)/theta (Sec. 2) producing the accepted
 * cell pairs and the leaf pairs; mutual M2L of every accepted pair with the
 * variant's corrective force (Eqs. 3, 4, 7, 8); mutual P2P of every leaf
 * pair and self leaf; fixed-order segmented sums.  Synchronises the stream
 * (list lengths are read back). */
int fmm_interact(fmm_ctx *ctx);

/* a9: L2L shift of the local expansions down the tree and L2P evaluation at
 * every body, plus the near-field sums.  Asynchronous. */
int fmm_downward(fmm_ctx *ctx);

/* Writes the accelerations in the caller's body order.  ax, ay, az: device,
 * n doubles each.  Asynchronous. */
int fmm_forces(fmm_ctx *ctx, double *ax, double *ay, double *az);

/* The five calls above in order (device pointers as above). */
int fmm_solve(fmm_ctx *ctx, const double *x, const double *y, const double *z, const double *m,
              int64_t n, double *ax, double *ay, double *az);

/* a13: one solve of nsys independent systems in one launch sequence.  The
 * bodies are concatenated: system s owns indices [offsets[s], offsets[s+1])
 * of x, y, z, m (device, offsets[nsys] doubles each); offsets is a HOST array
 * of nsys + 1 increasing entries with offsets[0] = 0 and no empty system.
 * Every system gets its own bounding cube, keys and octree (a forest with one
 * root per system); bodies of different systems never interact.  Outputs as
 * fmm_forces.  Synchronises the stream (like fmm_build_tree). */
int fmm_solve_batch(fmm_ctx *ctx, const double *x, const double *y, const double *z, const double *m,
                    const int64_t *offsets, int nsys, double *ax, double *ay, double *az);

/* a13: graph-captured solves.  With enable = 1, fmm_solve, fmm_solve_batch
 * and fmm_solve_host run each solve as one CUDA-graph launch on the
 * context's stream, no host round trip inside it:
 *  - The first solve (and any solve whose key differs from the captured
 *    one: caller buffers, n, nsys, options, softening, leaf tile, or a device
 *    buffer of the context reallocated since) is solved plainly, keeping
 *    every device value the host reads back to size its launches; the same
 *    host code then runs again under stream capture, taking those values
 *    instead of reading them.
 *  - Where a plain solve reads back (the octree's level counts, the leaf
 *    count, the walk's list lengths, the near field's totals) the graph holds
 *    a check kernel and an IF node: the rest of the solve runs only if the
 *    device values equal the captured ones.
 *  - Later solves with the same key replay the graph and read one record
 *    back.  Every kernel reads its data from the device, so new coordinates
 *    or masses with the same sizes are solved by the replay, bit-identical
 *    to a plain solve; when a size differs (or an input is invalid) the
 *    record says so and the call solves plainly and captures again.
 * Results, statistics and errors are those of a plain solve; a replay has no
 * stage timers.  Order 3 only, without the learned selector (other solves
 * run plainly).  Synchronises the stream.  enable = 0 (the default) keeps
 * the plain path. */
int fmm_set_graph(fmm_ctx *ctx, int enable);
/* Counters of the graph-captured solves: out[0] replays that completed,
 * out[1] captures, out[2] replays that found other sizes and fell back to a
 * plain solve, out[3] captures abandoned (the solve itself succeeded; e.g.
 * its planning solve had to grow a buffer), out[4] kernels in the current
 * graph (0 if none).  out: HOST, 5 entries. */
int fmm_graph_stats(const fmm_ctx *ctx, int64_t *out);
/* Why the last capture was abandoned ("" if none was). */
const char *fmm_graph_error(const fmm_ctx *ctx);

/* a13: picks the leaf size for an ensemble.  Runs fmm_solve_batch once per
 * candidate n_crit (warm-up) and then `reps` timed times (CUDA events on the
 * context's stream), writes the mean ms per candidate to ms_out (HOST, ncand
 * floats, may be NULL) and the fastest candidate to *best (HOST).  The
 * context's options are restored afterwards (set n_crit to *best with
 * fmm_set_opts to use it).  ax, ay, az receive the last solve's accelerations.
 * Synchronises the stream. */
int fmm_autotune_ncrit(fmm_ctx *ctx, const double *x, const double *y, const double *z, const double *m,
                       const int64_t *offsets, int nsys, const int *candidates, int ncand, int reps,
                       double *ax, double *ay, double *az, int *best, float *ms_out);

/* a13: picks the leaf size and the leaf tile together: every pair
 * (ncrit[a], tiles[b]) is timed as above; ms_out (HOST, nn x nt floats, row
 * a = ncrit[a], may be NULL) receives the mean ms of each pair, *best_ncrit
 * and *best_tile (HOST) the fastest.  Tiles are 8, 16 or 32 (fmm_set_tile).
 * The context's options and tile are restored afterwards.  Synchronises the
 * stream. */
int fmm_autotune(fmm_ctx *ctx, const double *x, const double *y, const double *z, const double *m,
                 const int64_t *offsets, int nsys, const int *ncrit, int nn, const int *tiles, int nt, int reps,
                 double *ax, double *ay, double *az, int *best_ncrit, int *best_tile, float *ms_out);

/* The same solve from HOST arrays (pageable or pinned): copies the bodies to
 * context-owned device buffers, solves, copies the accelerations back and
 * synchronises the stream before returning. */
int fmm_solve_host(fmm_ctx *ctx, const double *x, const double *y, const double *z,
                   const double *m, int64_t n, double *ax, double *ay, double *az);

/* a14: nsteps uniform kick-drift-kick leapfrog steps of length dt (uniform
 * steps are what conservation needs, Sec. 4).  Each step: v += a dt/2,
 * x += v dt, a = solve(x), v += a dt/2; the first acceleration is solved
 * before the loop.  x, y, z, vx, vy, vz: device, n doubles, updated in place
 * (caller order); m: device; ax, ay, az: device, n doubles, hold the
 * accelerations of the final positions on return.  mom: device, 6 (nsteps+1)
 * doubles or NULL: after step s (s = 0 before the first) the totals
 * P = sum m v and L = sum m x x v (about the origin), FP64 compensated in a
 * fixed order.  Synchronises the stream once per solve. */
int fmm_leapfrog(fmm_ctx *ctx, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                 const double *m, int64_t n, double dt, int nsteps, double *ax, double *ay, double *az,
                 double *mom);

/* ---- a12: learned pair selector ------------------------------------------ */
/* The paper allows any pair selection driven by an error estimate (Sec. 2,
 * after the opening criterion); every accepted pair still interacts mutually
 * with the correction, so conservation is unchanged.  The estimate is a
 * network of 8 pair features -> 3 x 64 SiLU -> 1 output, the predicted log10
 * of the pair's normalised M2L error; it runs in BF16 on the tensor cores
 * with FP32 accumulation.  Parameters: fmm_selector_nparams() floats (FP32):
 * W1[64][8], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], w4[64], b4,
 * feature mean[8], feature scale[8].  Features of a pair (ordered by R_max in FP32,
 * then id): log10 of |r|, R_A/|r|, R_B/|r|, M_A, M_B, |Q_A - tr/3|/(M_A R_A^2),
 * the same for B, and N_A + N_B; normalised as (f - mean) * scale. */
int fmm_selector_nparams(void);

/* Acceptance rules of the learned selector (see fmm_selector_set). */
#define FMM_SEL_ABSOLUTE 0 /* predicted absolute pair error below the target */
#define FMM_SEL_RELATIVE 1 /* ... below the target times the field at each side */

/* Enables (enable = 1) or disables the selector for the following solves.
 * params: HOST, fmm_selector_nparams() floats.  With it, the opening
 * criterion at the context's theta still accepts what it accepts; a pair it
 * rejects but that the criterion at theta_max (theta < theta_max <= 1;
 * theta_max = 1 is the safety bound |Z_A - Z_B| >= R_A + R_B) accepts, and
 * whose n_A n_B >= min_work, is scored: the network predicts the larger
 * side's error e in units of the partner's monopole field, so side A's error
 * is at most e M_B/r^2 and side B's e M_A/r^2.  The pair is accepted when
 *   FMM_SEL_ABSOLUTE:  e max(M_A, M_B) / r^2 < 10^log10_target (G = 1), or
 *   FMM_SEL_RELATIVE:  e max(M_B / (r^2 |a_A|), M_A / (r^2 |a_B|))
 *                      < 10^log10_target,
 * with |a| a per-cell estimate of the field from the softened monopoles of
 * one coarse level.  Pairs below min_work are not scored (opening a pair of
 * few bodies costs less than the network, about 18k flop).  Every other pair
 * is opened as usual.  The network only adds pairs, so the interaction lists
 * never grow beyond those of the plain criterion at theta.  One system per
 * solve (fmm_solve_batch with the selector on returns FMM_EUNSUPPORTED).
 * FMM_EINVAL if theta_max is outside (0, 1] or the rule is unknown. */
int fmm_selector_set(fmm_ctx *ctx, const float *params, double log10_target, double theta_max, int64_t min_work,
                     int rule, int enable);

/* Training samples for K given cell pairs of the current tree (after
 * fmm_upward, order 3): pairs: device, K x 2 int32; feat: device, K x 8 raw
 * features; label (device, K floats, may be NULL): log10 of the larger of
 * the two sides' errors, where a side's error is the rms over its bodies of
 * |a_M2L - a_direct| for the pair alone (torque-corrected order-3
 * expansion) divided by the other cell's monopole field M_other/|r|^2;
 * floored at -12 (the FP64 rounding level).  A side of n > 128 bodies is
 * represented by the 128 bodies at sorted positions floor(t n / 128) of the
 * cell.  Asynchronous. */
int fmm_selector_samples(fmm_ctx *ctx, const int32_t *pairs, int64_t K, float *feat, float *label);

/* Network output for K samples of raw features (device in, device out). */
int fmm_mlp_forward(fmm_ctx *ctx, const float *params, const float *feat, int64_t K, float *out);
/* Gradient (device, first 8961 entries of the parameter layout) and mean
 * squared error (device, 1 float, may be NULL) of a batch of B samples; sums
 * in a fixed order (reproducible). */
int fmm_mlp_grad(fmm_ctx *ctx, const float *params, const float *feat, const float *label, int64_t B,
                 float *grad, float *loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) of the network weights; m, v:
 * device moment buffers of the same layout; step counts from 1. */
int fmm_mlp_adam(fmm_ctx *ctx, float *params, float *m, float *v, const float *grad, float lr, int step);
/* `steps` Adam steps on minibatches of `batch` samples in the order of one
 * seeded permutation of the n samples (X: device n x 8 raw features, y:
 * device n labels; params: device, updated; adam: device, 2 x 8961 floats,
 * zeroed by the caller).  loss_out: HOST, steps floats or NULL.
 * Synchronises the stream. */
int fmm_selector_train(fmm_ctx *ctx, float *params, float *adam, const float *X, const float *y, int64_t n,
                       int batch, int steps, float lr, unsigned long long seed, float *loss_out);

/* ---- test hook (no counterpart in the paper) ------------------------------ */
/* Exercises the bounded wait of the walk's single-pass scan: launches one
 * walk generation of two tiles with one block whose tile counter already
 * stands at 1, so the block waits for a predecessor that no block takes.
 * The wait gives up after its poll limit (about a second), the block writes
 * nothing but its own scan records, and the call returns FMM_ETIMEOUT; the
 * context stays usable (the next call must be fmm_build_tree or fmm_solve).
 * Synchronises the stream. */
int fmm_debug_walk_wait_timeout(fmm_ctx *ctx);

/* ---- a10 diagnostics (Sec. 3) ---------------------------------------------- */

/* Exact accelerations of nt target bodies by direct summation over all n
 * bodies (Sec. 3: the reference of the error metric), softened as set by
 * fmm_set_softening, FP64 with Neumaier-compensated sums in a fixed
 * order (reproducible).  x, y, z, m: device, n doubles, any body order;
 * targets: device, nt int32 indices into them; ax, ay, az: device, nt
 * doubles (G = 1; the context's G is not applied).  A body at zero
 * separation from the target contributes nothing.  Asynchronous. */
int fmm_direct(fmm_ctx *ctx, const double *x, const double *y, const double *z, const double *m,
               int64_t n, const int32_t *targets, int64_t nt, double *ax, double *ay, double *az);

/* Net force and torque balance of Sec. 3,
 *   sqrt( sum_d (sum_n mu_n A_nd)^2 / sum_d (sum_n mu_n |A_nd|)^2 ),
 * with A = (ax, ay, az) for the force and A = X x a (about the origin) for the
 * torque.  All arrays device, n doubles; out: HOST, 2 doubles {force, torque}.
 * FP64, compensated, fixed order.  Synchronises the stream. */
int fmm_balance(fmm_ctx *ctx, const double *x, const double *y, const double *z, const double *m,
                const double *ax, const double *ay, const double *az, int64_t n, double *out);

/* The same balance check for callers that cannot allocate device memory: no
 * context, and no cudaMalloc, cudaFree or other allocating call.  Some callers
 * cannot allocate at the moment they want this check: codes whose device
 * memory is handed out by their own fixed pool or arena and may not grow it,
 * and time-step loops that must not stall on the device synchronisation that
 * cudaMalloc and cudaFree bring, or risk an allocation failure mid-run.  (The
 * paper has no counterpart; this is a library convenience.)
 *
 * x, y, z, m, ax, ay, az: device, n doubles; out: DEVICE, 2 doubles
 * {force, torque}, written by a kernel on `cuda_stream` (a cudaStream_t; NULL
 * = the legacy default stream); the call returns without synchronising.
 * Scratch is a fixed array in the library's device memory, one record per
 * 4,096 bodies, so n is limited to 4,194,304: a larger n returns FMM_ESIZE and
 * launches nothing.  The array (about 197 KB) stays allocated on every GPU
 * that loads the library until the process exits.  All calls share it: two
 * calls whose kernels overlap on the GPU race; issue them on one stream, or
 * order them.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process, so make
 * that first call before any stream capture, pass a stream of the current
 * device, and do not call cudaDeviceReset between calls (that releases the
 * library's device memory, and the kept address would be stale).
 * Returns FMM_EINVAL for n < 1 or a NULL pointer, FMM_ECUDA if a launch fails. */
int fmm_balance_noalloc(const double *x, const double *y, const double *z, const double *m,
                        const double *ax, const double *ay, const double *az, int64_t n, double *out,
                        void *cuda_stream);

/* Measured arithmetic peak of the GPU's plain FMA pipe (the pipe that bounds
 * the P2P and M2L kernels; no tensor cores), for the roofline of those
 * kernels: independent FMA chains on every SM of the current device, timed
 * with CUDA events on the legacy default stream; the best of `reps` timed
 * launches after one warm-up.  precision FMM_FP64: DFMA; FMM_MIXED: FFMA.
 * *tflops (HOST) receives TFLOP/s with an FMA counted as 2.  No context;
 * allocates nothing; synchronises the device's default stream.  (A
 * measurement aid; the paper has no counterpart.) */
int fmm_alu_peak(int precision, int reps, double *tflops);

/* Counts (and stage timings) of the last solve; synchronises the stream. */
int fmm_get_stats(fmm_ctx *ctx, fmm_stats *out);

/* ---- exports for bit-exact checks (device outputs, caller-sized from
 *      fmm_get_stats; synchronise nothing) ---------------------------------- */

/* keys: n uint64 (sorted); order: n int32 (sorted position -> caller index) */
int fmm_export_keys(fmm_ctx *ctx, uint64_t *keys, int32_t *order);
/* per cell (ncell each): begin, count, level, parent, first_child, nchild
 * (int32), M, Rmax (double), Z (ncell x 3 double, row major) */
int fmm_export_tree(fmm_ctx *ctx, int32_t *begin, int32_t *count, int32_t *level,
                    int32_t *parent, int32_t *first_child, int32_t *nchild, double *M,
                    double *Z, double *Rmax);
/* moments about Z: ncell x (P+1)(P+2)(P+3)/6 doubles (20 at P = 3), orders 0..P
 * by exponent triple (a,b,c), a = n..0 then b = n-a..0; at P = 3:
 * [M, Mx, My, Mz, Qxx, Qxy, Qxz, Qyy, Qyz, Qzz,
 *  Oxxx, Oxxy, Oxxz, Oxyy, Oxyz, Oxzz, Oyyy, Oyyz, Oyzz, Ozzz] */
int fmm_export_moments(fmm_ctx *ctx, double *mom);
/* m2l: n_m2l x 2, p2p: n_p2p x 2 (each pair (min, max)), self: n_self;
 * int32, in the library's processing order (sort them to compare) */
int fmm_export_lists(fmm_ctx *ctx, int32_t *m2l, int32_t *p2p, int32_t *self);
/* local expansion of every cell after the downward shift.  P = 3: ncell x 20
 * doubles [C_x, C_y, C_z, C_xx, C_xy, C_xz, C_yy, C_yz, C_zz, C_xxx, C_xxy,
 * C_xxz, C_xyy, C_xyz, C_xzz, C_yyy, C_yyz, C_yzz, C_zzz, 0]; a body at
 * offset x from Z receives a = -(C_i + C_ij x_j + C_ijk x_j x_k / 2) plus its
 * near-field sum.  P = 4, 5: ncell x ((P+1)(P+2)(P+3)/6 - 1) doubles, the
 * Taylor coefficients L^a of orders 1..P in the moments' multi-index order
 * (a body at x receives g_k = -sum_a L^(a+e_k) x^a / a!). */
int fmm_export_locals(fmm_ctx *ctx, double *C);

#ifdef __cplusplus
}
#endif
#endif
