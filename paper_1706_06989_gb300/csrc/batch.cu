// batch.cu -- a13: autotuner for batched ensembles.
//
// The forest solve (fmm_solve_batch) is timed with CUDA events on the
// context's stream for every candidate pair of leaf size n_crit (a leaf holds
// at most n_crit bodies, Sec. 2) and leaf tile (the rows of a leaf the near
// field stages per pass); the fastest pair is returned.  Every candidate
// gives a valid solve of the same method: n_crit changes the tree, the tile
// only the order of the near field's work.
#include "internal.cuh"

using namespace amfmm;

namespace {

// Mean ms of `reps` timed forest solves (after one untimed one) with the
// context's current options; a repetition that cannot be timed fails the call
// (counting it as zero would make the candidate look fast).
int time_batch(fmm_ctx *c, cudaEvent_t e0, cudaEvent_t e1, const double *x, const double *y, const double *z,
               const double *m, const int64_t *offsets, int nsys, int reps, double *ax, double *ay, double *az,
               float *ms) {
  int rc = fmm_solve_batch(c, x, y, z, m, offsets, nsys, ax, ay, az);  // warm-up and buffer growth
  float tot = 0.f;
  for (int r = 0; r < reps && rc == FMM_OK; ++r) {
    cudaError_t ce = cudaEventRecord(e0, c->stream);
    if (ce == cudaSuccess) rc = fmm_solve_batch(c, x, y, z, m, offsets, nsys, ax, ay, az);
    if (rc != FMM_OK) break;
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, c->stream);
    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
    float t = 0.f;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
    if (ce != cudaSuccess)
      rc = set_error(c, FMM_ECUDA, "timing n_crit %d, tile %d: %s", c->opts.n_crit, c->p2p_rows,
                     cudaGetErrorString(ce));
    tot += t;
  }
  *ms = tot / reps;
  return rc;
}

}  // namespace

extern "C" int fmm_autotune(fmm_ctx *c, const double *x, const double *y, const double *z, const double *m,
                            const int64_t *offsets, int nsys, const int *ncrit, int nn, const int *tiles, int nt,
                            int reps, double *ax, double *ay, double *az, int *best_ncrit, int *best_tile,
                            float *ms_out) {
  if (!c || !ncrit || !tiles || nn < 1 || nt < 1 || reps < 1 || !best_ncrit || !best_tile) return FMM_EINVAL;
  for (int k = 0; k < nn; ++k)
    if (ncrit[k] < 1) return set_error(c, FMM_EINVAL, "candidate n_crit must be >= 1");
  for (int k = 0; k < nt; ++k)
    if (tiles[k] != 8 && tiles[k] != 16 && tiles[k] != 32) return set_error(c, FMM_EINVAL, "leaf tile must be 8, 16 or 32");
  const fmm_opts saved = c->opts;
  const int saved_rows = c->p2p_rows;
  cudaEvent_t e0, e1;
  AMFMM_CUDA(c, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error(c, FMM_ECUDA, "cudaEventCreate failed");
  }
  int rc = FMM_OK;
  float best_ms = 0.f;
  *best_ncrit = ncrit[0];
  *best_tile = tiles[0];
  for (int a = 0; a < nn && rc == FMM_OK; ++a)
    for (int b = 0; b < nt && rc == FMM_OK; ++b) {
      c->opts.n_crit = ncrit[a];
      c->p2p_rows = tiles[b];
      float ms = 0.f;
      rc = time_batch(c, e0, e1, x, y, z, m, offsets, nsys, reps, ax, ay, az, &ms);
      if (ms_out) ms_out[a * nt + b] = ms;
      if (rc == FMM_OK && ((a == 0 && b == 0) || ms < best_ms)) {
        best_ms = ms;
        *best_ncrit = ncrit[a];
        *best_tile = tiles[b];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->opts = saved;
  c->p2p_rows = saved_rows;
  c->stage = kNone;
  return rc;
}

extern "C" int fmm_autotune_ncrit(fmm_ctx *c, const double *x, const double *y, const double *z,
                                  const double *m, const int64_t *offsets, int nsys, const int *candidates,
                                  int ncand, int reps, double *ax, double *ay, double *az, int *best,
                                  float *ms_out) {
  if (!c || !candidates || ncand < 1 || reps < 1 || !best) return FMM_EINVAL;
  int tile = 0;
  const int cur = c->p2p_rows;
  return fmm_autotune(c, x, y, z, m, offsets, nsys, candidates, ncand, &cur, 1, reps, ax, ay, az, best, &tile,
                      ms_out);
}
