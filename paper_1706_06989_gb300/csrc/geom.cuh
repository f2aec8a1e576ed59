// geom.cuh -- centre of mass of a cell, shared by every expansion order.
//
// Sec. 2: the opening criterion compares centres of mass, so Z must come out
// identical wherever it is computed.  A leaf sums its bodies in sorted order,
// any other cell sums its children in octant order, Z = S / M, every step an
// explicitly rounded FP64 operation (no FMA contraction).
#pragma once

namespace amfmm {

__device__ __forceinline__ void leaf_com(int c, int b, int e, const double *__restrict__ X,
                                         const double *__restrict__ Y, const double *__restrict__ Zb,
                                         const double *__restrict__ Mb, double *__restrict__ S,
                                         double *__restrict__ M, double *__restrict__ Z,
                                         double *__restrict__ invM, double z[3]) {
  double sx = 0.0, sy = 0.0, sz = 0.0, mm = 0.0;
  for (int i = b; i < e; ++i) {
    const double mu = Mb[i];
    sx = __dadd_rn(sx, __dmul_rn(mu, X[i]));
    sy = __dadd_rn(sy, __dmul_rn(mu, Y[i]));
    sz = __dadd_rn(sz, __dmul_rn(mu, Zb[i]));
    mm = __dadd_rn(mm, mu);
  }
  z[0] = __ddiv_rn(sx, mm);
  z[1] = __ddiv_rn(sy, mm);
  z[2] = __ddiv_rn(sz, mm);
  S[3 * c] = sx;
  S[3 * c + 1] = sy;
  S[3 * c + 2] = sz;
  M[c] = mm;
  Z[3 * c] = z[0];
  Z[3 * c + 1] = z[1];
  Z[3 * c + 2] = z[2];
  invM[c] = 1.0 / mm;
}

__device__ __forceinline__ void parent_com(int c, int f, int nch, double *__restrict__ S, double *__restrict__ M,
                                           double *__restrict__ Z, double *__restrict__ invM, double z[3]) {
  double sx = 0.0, sy = 0.0, sz = 0.0, mm = 0.0;
  for (int k = f; k < f + nch; ++k) {
    sx = __dadd_rn(sx, S[3 * k]);
    sy = __dadd_rn(sy, S[3 * k + 1]);
    sz = __dadd_rn(sz, S[3 * k + 2]);
    mm = __dadd_rn(mm, M[k]);
  }
  z[0] = __ddiv_rn(sx, mm);
  z[1] = __ddiv_rn(sy, mm);
  z[2] = __ddiv_rn(sz, mm);
  S[3 * c] = sx;
  S[3 * c + 1] = sy;
  S[3 * c + 2] = sz;
  M[c] = mm;
  Z[3 * c] = z[0];
  Z[3 * c + 1] = z[1];
  Z[3 * c + 2] = z[2];
  invM[c] = 1.0 / mm;
}

}  // namespace amfmm
