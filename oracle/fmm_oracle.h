/*
 * fmm_oracle.h -- declarations of the FP64 CPU oracle (test infrastructure
 * only; see fmm_oracle.c).  Arrays are caller-owned host memory; cell and
 * body indices are 32-bit (n < 2^31).
 */
#ifndef FMM_ORACLE_H
#define FMM_ORACLE_H
#include <stdint.h>

#define ORC_OK 0
#define ORC_EINVAL -1

/* variants of Sec. 3: uncorrected, torque corrected (Eq. 7), optimised (Eq. 8) */
#define ORC_UC 0
#define ORC_TC 1
#define ORC_TCO 2

/* which parts orc_eval sums */
#define ORC_PART_FAR 1
#define ORC_PART_NEAR 2

typedef struct orc orc_t;

/* Bounding cube and 63-bit Morton keys (x in the lowest bit of each triple). */
int orc_morton(int n, const double *x, const double *y, const double *z, uint64_t *keys,
               double *lo, double *scale);

/* Sort, octree, centres of mass, R_max, moments to order P, dual-tree walk. */
orc_t *orc_create(int n, const double *x, const double *y, const double *z, const double *m,
                  int n_crit, double theta, int P, int *err);
void orc_destroy(orc_t *t);

/* out = {n, ncell, n_m2l, n_p2p, n_self, nmom} */
int orc_sizes(const orc_t *t, int *out);
int orc_get_keys(const orc_t *t, uint64_t *key, int *order, double *lo, double *scale);
int orc_get_cells(const orc_t *t, int *begin, int *count, int *level, int *parent,
                  int *first_child, int *nchild);
/* Z is [ncell][3]; mom is [ncell][nmom] by multi-index (a,b,c) */
int orc_get_geometry(const orc_t *t, double *M, double *Z, double *Rmax, double *mom);
int orc_get_lists(const orc_t *t, int *m2l, int *p2p, int *self);
/* Replaces the lists (e.g. by those of another pair selection); indices are
 * validated (P2P and self entries must be leaves). */
int orc_set_lists(orc_t *t, const int *m2l, int n_m2l, const int *p2p, int n_p2p, const int *self,
                  int n_self);

/* Accelerations in the caller's body order.  generic=0: order 3, Eqs. (3),
 * (4), (7), (8); generic=1: App. A at the order given to orc_create.
 * mask (caller order, may be NULL): only the flagged bodies receive their
 * full acceleration; entries of other bodies are partial and meaningless. */
int orc_eval(const orc_t *t, int variant, int generic, int parts, const unsigned char *mask,
             double *ax, double *ay, double *az);
/* Accelerations from one cell pair only (zero elsewhere), caller order. */
int orc_pair_accel(const orc_t *t, int A, int B, int variant, int generic, double *ax,
                   double *ay, double *az);

/* derivatives of G = -1/sqrt(R^2 + eps^2) (eps = 0: the paper's -1/R) */
int orc_dtensor_generic(const double *r, double eps, int n, double *out);
int orc_dtensor_p3(const double *r, double eps, double *d0, double *d1, double *d2, double *d3, double *d4,
                   double *d4prime);
/* Plummer softening of the evaluation (orc_eval, orc_pair_accel) */
int orc_set_softening(orc_t *t, double eps);

/* direct sums of G = -1/sqrt(R^2 + eps^2), Neumaier-compensated */
int orc_direct(int n, const double *x, const double *y, const double *z, const double *m, int nt,
               const int *targets, double eps, double *ax, double *ay, double *az);
int orc_balance(int n, const double *x, const double *y, const double *z, const double *m,
                const double *ax, const double *ay, const double *az, double *out);
#endif
