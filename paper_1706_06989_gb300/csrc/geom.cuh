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

// ---- opening criterion (Sec. 2), shared by the walk and the learned selector ----
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

// FP32 filter of the criterion.  On this GPU an FP64 operation costs about
// as much as 64 FP32 ones, so the walk first evaluates theta^2 d^2 - (R_A +
// R_B)^2 in FP32, from Z split into hi + lo floats (d carries FP32 relative
// accuracy even for close centres).  Each side of the comparison then has a
// relative error below 1e-6 against its exact value, and so does the FP64
// expression; when the two sides differ by more than 1e-5 of their sum, the
// FP32 sign is therefore the FP64 decision.  The lo parts carry an absolute
// error of about 2^-48 |Z| each; for centres closer than ~2^-20 |Z| that term
// outgrows the relative bound, so the tolerance adds 3e-21 max|Z|^2, which
// covers it (2 d e <= 1e-6 d^2 + 1e6 e^2).  Closer calls, and values outside
// the comfortable FP32 range, return -1 and are decided in FP64.
struct CellF {
  float4 h;  // Z hi (x, y, z), R_max rounded to FP32
  float4 l;  // Z - hi (x, y, z), unused
};

__device__ __forceinline__ int separated_fast(const CellF &a, const CellF &b, float th2) {
  const float dx = (a.h.x - b.h.x) + (a.l.x - b.l.x);
  const float dy = (a.h.y - b.h.y) + (a.l.y - b.l.y);
  const float dz = (a.h.z - b.h.z) + (a.l.z - b.l.z);
  const float lhs = th2 * (dx * dx + dy * dy + dz * dz);
  const float sr = a.h.w + b.h.w;
  const float rhs = sr * sr;
  const float tot = lhs + rhs;
  if (!(tot > 1e-30f && tot < 1e30f)) return -1;
  const float m = fmaxf(fmaxf(fmaxf(fabsf(a.h.x), fabsf(a.h.y)), fabsf(a.h.z)),
                        fmaxf(fmaxf(fabsf(b.h.x), fabsf(b.h.y)), fabsf(b.h.z)));
  const float diff = lhs - rhs, tol = 1e-5f * tot + 3e-21f * m * m;
  if (diff > tol) return 1;
  if (diff < -tol) return 0;
  return -1;
}

}  // namespace amfmm
