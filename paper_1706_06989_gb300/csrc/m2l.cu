// m2l.cu -- a7: mutual cell-cell interactions at expansion order 3 with the
// torque-cancelling correction, and their fixed-order per-cell sums.
//
// For an accepted pair (A, B) with r = Z_A - Z_B (the vector from B's centre
// of mass to A's; the Taylor series of Eqs. 2-4 is an expansion about this r)
// and the derivatives of G = -1/R (Sec. 2)
//     D_i   = r_i / R^3
//     D_ij  = -3 r_i r_j / R^5 + d_ij / R^3
//     D_ijk = 15 r_i r_j r_k / R^7 - 3 (d_ij r_k + d_jk r_i + d_ki r_j) / R^5,
// Eq. (3) gives the acceleration of a body of A at offset x from Z_A as
//     g_i = -(C_i + C_ij x_j + C_ijk x_j x_k / 2)
// with C^A_i = M_B D_i + Q_B,jk D_ijk / 2, C^A_ij = M_B D_ij, C^A_ijk = M_B D_ijk,
// and Eq. (4) gives the same form for B with
//     C^B_i = -M_A D_i - Q_A,jk D_ijk / 2, C^B_ij = M_A D_ij, C^B_ijk = -M_A D_ijk.
// (Q is the extensive quadrupole of Eq. 3; dipoles about the centres of mass
// vanish and are dropped, as Sec. 2 notes.)  The contraction Q_jk D_ijk is
// taken through r:  Q_jk D_ijk = 15 r_i (r.Q.r)/R^7 - 3 (2 (Q r)_i + r_i tr Q)/R^5
// (evaluated below with the unit vector n = r/R).
//
// Torque correction (Eq. 7 with the coefficient of App. A at P = 3):
//     F_i = (1/6) (M_A O_B,jkl - O_A,jkl M_B) D_ijkl,
// applied as +F/M_A on A and -F/M_B on B (C^A_i -= F_i/M_A, C^B_i += F_i/M_B).
// With S = M_A O_B - M_B O_A, u_i = S_ikl r_k r_l, t_i = S_ijj and
// D_ijkl = -105 rrrr/R^9 + 15 (six d rr terms)/R^7 - 3 (three d d terms)/R^5,
//     D_ijkl S_jkl = -105 r_i (r.u)/R^9 + 45 (u_i + r_i (r.t))/R^7 - 9 t_i/R^5.
// The variant of Eq. (8) keeps only the terms of D'_ijkl (those without a
// factor r_i):  D'_ijkl S_jkl = 45 u_i/R^7 - 9 t_i/R^5.
//
// Softening (optional): with G = -1/sqrt(R^2 + eps^2) every derivative keeps
// the same form with R^2 -> R^2 + eps^2 (the derivatives act through
// u = r.r + eps^2 only), so the formulas below take R^2 + eps^2 and leave the
// components r_i alone; n = r/R is then no longer a unit vector, and nothing
// below assumes that it is.  The torque correction still cancels the pair's
// torque (the G is still a function of the distance only).
//
// Each pair writes its two local contributions into slots whose positions
// were fixed by a stable sort of (cell, 2k + side); every cell then sums its
// slots in that order.  No floating-point atomics: the result is
// reproducible bit for bit.
#include "internal.cuh"

namespace amfmm {
namespace {

// threads per block of the FP64 pair kernel (Plummer, FP64: 256 against 128
// took 6.90 against 7.17 ms at N = 1M, 27.6 against 28.7 ms at 4M; 512 was
// slower)
constexpr int kBlock = 256;
constexpr int kCell32 = 24;    // floats per cell in the mixed form's copy (raw moments)
constexpr int kCell32TF = 20;  // the same with trace-free moments (unsoftened UC and TC)
constexpr int kQOh = 16;     // doubles per cell of the FP64 form's quadrupole and octupole per mass
constexpr int kSlot64 = 24;  // doubles per slot of the FP64 order-3 M2L (21 used: m2l_pair's SLOT form)

__device__ __forceinline__ double rsqrt_t(double v) { return rsqrt(v); }
__device__ __forceinline__ float rsqrt_t(float v) { return rsqrtf(v); }

// Local layout: Cx Cy Cz | Cxx Cxy Cxz Cyy Cyz Czz | Cxxx Cxxy Cxxz Cxyy Cxyz Cxzz Cyyy Cyyz Cyzz Czzz
// Moment layout: M | Dx Dy Dz | Qxx Qxy Qxz Qyy Qyz Qzz | Oxxx ... Ozzz (same order as locals)
// Separations below which the FP32 form treats a pair as coincident (its
// r^-5 terms would leave the FP32 range); FP64 only skips r = 0.
template <class T>
__device__ __forceinline__ T min_r2();
template <>
__device__ __forceinline__ double min_r2<double>() { return 0.0; }
template <>
__device__ __forceinline__ float min_r2<float>() { return 1e-30f; }

// The pair in terms of the unit vector n = r/R: D_i = n_i R^-2,
// D_ij = (d_ij - 3 n_i n_j) R^-3, D_ijk = (15 n_i n_j n_k - 3 (d_ij n_k + d_jk n_i
// + d_ki n_j)) R^-4 and D_ijkl S_jkl = (-105 n_i (n.u) + 45 (u_i + n_i (n.t))
// - 9 t_i) R^-5 with u_i = S_ikl n_k n_l, t_i = S_ijj.  Powers of 1/R are
// applied one factor at a time to the mass- or moment-scaled terms, so no
// large power of 1/R is formed on its own (this keeps the FP32 form in range).
// The correction is formed from the octupoles per unit mass, Oh = O / M (a
// per-cell array): S = M_A O_B - M_B O_A = M_A M_B (Oh_B - Oh_A), and the
// two masses fold into the scale factors F / M_A = M_B (F / (M_A M_B)) and
// F / M_B = M_A (F / (M_A M_B)), so the pair needs 10 subtractions for S and
// no divisions.  (The FP64 form runs at the FP64 pipe's rate: every
// operation per pair counts.)
//
// HARM: the unsoftened 1/R is harmonic away from R = 0, so every D tensor is
// trace-free in any two indices and its contraction with the trace part of a
// moment vanishes.  With HARM the caller passes trace-free quadrupoles
// (Q - tr Q / 3 I), which drops the trace term of h, and for TC trace-free
// octupoles per unit mass (t = 0 for their difference), which drops every
// t term of the correction: F = R^-5 [7.5 u - 17.5 n (n.u)].  Same sums up
// to rounding, about 24 fewer FP64 operations per pair.  (Softened
// derivatives are not trace-free, and TCO's correction is not a contraction
// with the full D: both keep the raw moments.)
//
// SLOT: the pair's slot form for the FP64 reduction (kSlot64 values per
// side): C_i as above, then the unit tensors U2 and U3 themselves, then the
// side's scale factors of the two (C^A: M_B R^-3, M_B R^-4; C^B: M_A R^-3,
// -M_A R^-4), which the reduction applies with one FMA per value where it
// would otherwise add (32 products fewer per pair).
template <class T, int VARIANT, bool HARM = false, bool SLOT = false>
__device__ __forceinline__ void m2l_pair(const T r[3], T MA, T MB, const T *QA, const T *QB, const T *OhA,
                                         const T *OhB, T eps2, T *CA, T *CB) {
  const T r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  if (!(r2 > min_r2<T>())) {
#pragma unroll
    for (int q = 0; q < (SLOT ? 21 : 19); ++q) CA[q] = CB[q] = T(0);
    return;
  }
  const T Ri = rsqrt_t(r2 + eps2);
  const T x = r[0] * Ri, y = r[1] * Ri, z = r[2] * Ri;
  const T xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  // unit parts of D_ij and D_ijk
  const T U2[6] = {T(1) - T(3) * xx, T(-3) * xy, T(-3) * xz, T(1) - T(3) * yy, T(-3) * yz, T(1) - T(3) * zz};
  const T fx3 = T(15) * xx - T(3), fy3 = T(15) * yy - T(3), fz3 = T(15) * zz - T(3);
  const T U3[10] = {(fx3 - T(6)) * x, fx3 * y, fx3 * z, fy3 * x, T(15) * xy * z, fz3 * x, (fy3 - T(6)) * y,
                    fy3 * z, fz3 * y, (fz3 - T(6)) * z};
  // mass-scaled powers: M R^-2, M R^-3, M R^-4
  const T Ri2 = Ri * Ri;
  const T MB2 = MB * Ri2, MA2 = MA * Ri2;
  const T MB3 = MB2 * Ri, MA3 = MA2 * Ri;
  const T MB4 = MB3 * Ri, MA4 = MA3 * Ri;
  const T Ri4 = Ri2 * Ri2;
  // h = Q_jk D_ijk / 2 = R^-4 [n_i (15 n.Q.n - 3 trQ) - 6 (Q n)_i] / 2
  const T v = T(-3) * Ri4;
  const T c75 = T(7.5) * Ri4;
  T hA[3], hB[3];
  {
    const T *Q = QB;
    const T qx = Q[0] * x + Q[1] * y + Q[2] * z;
    const T qy = Q[1] * x + Q[3] * y + Q[4] * z;
    const T qz = Q[2] * x + Q[4] * y + Q[5] * z;
    const T w = HARM ? c75 * (x * qx + y * qy + z * qz)
                     : (T(7.5) * (x * qx + y * qy + z * qz) - T(1.5) * (Q[0] + Q[3] + Q[5])) * Ri4;
    hB[0] = w * x + v * qx;
    hB[1] = w * y + v * qy;
    hB[2] = w * z + v * qz;
  }
  {
    const T *Q = QA;
    const T qx = Q[0] * x + Q[1] * y + Q[2] * z;
    const T qy = Q[1] * x + Q[3] * y + Q[4] * z;
    const T qz = Q[2] * x + Q[4] * y + Q[5] * z;
    const T w = HARM ? c75 * (x * qx + y * qy + z * qz)
                     : (T(7.5) * (x * qx + y * qy + z * qz) - T(1.5) * (Q[0] + Q[3] + Q[5])) * Ri4;
    hA[0] = w * x + v * qx;
    hA[1] = w * y + v * qy;
    hA[2] = w * z + v * qz;
  }
  const T nv[3] = {x, y, z};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    CA[i] = MB2 * nv[i] + hB[i];
    CB[i] = -(MA2 * nv[i] + hA[i]);
  }
  if (SLOT) {
#pragma unroll
    for (int k = 0; k < 6; ++k) CA[3 + k] = CB[3 + k] = U2[k];
#pragma unroll
    for (int k = 0; k < 10; ++k) CA[9 + k] = CB[9 + k] = U3[k];
    CA[19] = MB3;
    CA[20] = MB4;
    CB[19] = MA3;
    CB[20] = -MA4;
  } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      CA[3 + k] = MB3 * U2[k];
      CB[3 + k] = MA3 * U2[k];
    }
#pragma unroll
    for (int k = 0; k < 10; ++k) {
      CA[9 + k] = MB4 * U3[k];
      CB[9 + k] = -(MA4 * U3[k]);
    }
  }
  if (VARIANT == FMM_TC && HARM) {
    // trace-free Sh: F = 7.5 R^-5 [u + (-7/3) n (n.u)], the 7.5 R^-5 folded
    // into the scale factors
    T S[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) S[k] = OhB[k] - OhA[k];
    const T xy2 = T(2) * xy, xz2 = T(2) * xz, yz2 = T(2) * yz;
    const T ux = S[0] * xx + S[3] * yy + S[5] * zz + S[1] * xy2 + S[2] * xz2 + S[4] * yz2;
    const T uy = S[1] * xx + S[6] * yy + S[8] * zz + S[3] * xy2 + S[4] * xz2 + S[7] * yz2;
    const T uz = S[2] * xx + S[7] * yy + S[9] * zz + S[4] * xy2 + S[5] * xz2 + S[8] * yz2;
    const T w = T(-7.0 / 3.0) * (x * ux + y * uy + z * uz);
    const T F[3] = {ux + w * x, uy + w * y, uz + w * z};
    const T c5 = c75 * Ri;
    const T sA = MB * c5, sB = MA * c5;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      CA[i] -= F[i] * sA;
      CB[i] += F[i] * sB;
    }
  } else if (VARIANT != FMM_UC) {
    // Sh = Oh_B - Oh_A = S / (M_A M_B) (xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz)
    T S[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) S[k] = OhB[k] - OhA[k];
    // u_i = S_ikl n_k n_l, t_i = S_ijj
    const T xy2 = T(2) * xy, xz2 = T(2) * xz, yz2 = T(2) * yz;
    const T ux = S[0] * xx + S[3] * yy + S[5] * zz + S[1] * xy2 + S[2] * xz2 + S[4] * yz2;
    const T uy = S[1] * xx + S[6] * yy + S[8] * zz + S[3] * xy2 + S[4] * xz2 + S[7] * yz2;
    const T uz = S[2] * xx + S[7] * yy + S[9] * zz + S[4] * xy2 + S[5] * xz2 + S[8] * yz2;
    const T tx = S[0] + S[3] + S[5];
    const T ty = S[1] + S[6] + S[8];
    const T tz = S[2] + S[7] + S[9];
    // F = (1/6) D_ijkl S_jkl = R^-5 [7.5 u - 1.5 t (+ n (-17.5 n.u + 7.5 n.t) for TC)]
    T F[3] = {T(7.5) * ux - T(1.5) * tx, T(7.5) * uy - T(1.5) * ty, T(7.5) * uz - T(1.5) * tz};
    if (VARIANT == FMM_TC) {
      const T w = T(-17.5) * (x * ux + y * uy + z * uz) + T(7.5) * (x * tx + y * ty + z * tz);
      F[0] += w * x;
      F[1] += w * y;
      F[2] += w * z;
    }
    // C^A_i -= F_i / M_A = M_B Fh_i R^-5,  C^B_i += F_i / M_B = M_A Fh_i R^-5
    const T Ri5 = Ri4 * Ri;
    const T sA = MB * Ri5, sB = MA * Ri5;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      CA[i] -= F[i] * sA;
      CB[i] += F[i] * sB;
    }
  }
}

// One thread per accepted pair.  Slots are kSlot64 wide (m2l_pair's SLOT
// form, 21 used).
// FP64 form: reads the FP64 cell data.
// qoh: per cell the quadrupole (6) and the octupole per unit mass (10) the
// pair function takes, trace-free where HARM allows (k_qoh).
template <int VARIANT, bool HARM>
__global__ void __launch_bounds__(kBlock) k_m2l64(int64_t K, const int2 *__restrict__ pairs,
                                                   const double *__restrict__ Z,
                                                   const double *__restrict__ M,
                                                   const double *__restrict__ qoh,
                                                   const int32_t *__restrict__ pos, double eps2,
                                                   double *__restrict__ slots) {
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= K) return;
  const int A = pairs[k].x, B = pairs[k].y;
  double CA[kSlot64], CB[kSlot64];
  const double r[3] = {Z[3 * A] - Z[3 * B], Z[3 * A + 1] - Z[3 * B + 1], Z[3 * A + 2] - Z[3 * B + 2]};
  const double *qA = qoh + static_cast<int64_t>(A) * kQOh;
  const double *qB = qoh + static_cast<int64_t>(B) * kQOh;
  m2l_pair<double, VARIANT, HARM, true>(r, M[A], M[B], qA, qB, qA + 6, qB + 6, eps2, CA, CB);
  CA[21] = CB[21] = CA[22] = CB[22] = CA[23] = CB[23] = 0.0;
  double *sa = slots + static_cast<int64_t>(pos[2 * k]) * kSlot64;
  double *sb = slots + static_cast<int64_t>(pos[2 * k + 1]) * kSlot64;
#pragma unroll
  for (int q = 0; q < kSlot64; q += 2) {
    *reinterpret_cast<double2 *>(sa + q) = make_double2(CA[q], CA[q + 1]);
    *reinterpret_cast<double2 *>(sb + q) = make_double2(CB[q], CB[q + 1]);
  }
}

// One side of the same interaction: the local of a target cell T from a
// source cell S, with r = Z_T - Z_S.  Written for T = A it is the C^A of
// m2l_pair; for T = B it is C^B, because every term of C^B is the C^A form
// with r -> -r and A <-> B: the odd terms (n D, U3, Q D_ijk) change sign with
// r, the even ones (U2, and F, whose S = M_T O_S - M_S O_T changes sign
// with the roles) pick up the sign of the role swap.  So a gather over each
// cell's partners evaluates the mutual interaction once from each side.
template <class T, int VARIANT>
__device__ __forceinline__ void m2l_one(const T r[3], T MT, T iMT, T MS, const T *QS, const T *OT, const T *OS,
                                        T eps2, T *C) {
  const T r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  if (!(r2 > min_r2<T>())) {
#pragma unroll
    for (int q = 0; q < 19; ++q) C[q] = T(0);
    return;
  }
  const T Ri = rsqrt_t(r2 + eps2);
  const T x = r[0] * Ri, y = r[1] * Ri, z = r[2] * Ri;
  const T xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  const T fxx = T(15) * xx, fyy = T(15) * yy, fzz = T(15) * zz;
  const T M2 = MS * Ri * Ri, M3 = M2 * Ri, M4 = M3 * Ri;
  const T Ri2 = Ri * Ri;
  const T qx = QS[0] * x + QS[1] * y + QS[2] * z;
  const T qy = QS[1] * x + QS[3] * y + QS[4] * z;
  const T qz = QS[2] * x + QS[4] * y + QS[5] * z;
  const T w = (T(7.5) * (x * qx + y * qy + z * qz) - T(1.5) * (QS[0] + QS[3] + QS[5])) * Ri2 * Ri2;
  const T v = T(-3) * Ri2 * Ri2;
  C[0] = M2 * x + (w * x + v * qx);
  C[1] = M2 * y + (w * y + v * qy);
  C[2] = M2 * z + (w * z + v * qz);
  C[3] = M3 * (T(1) - T(3) * xx);
  C[4] = M3 * (T(-3) * xy);
  C[5] = M3 * (T(-3) * xz);
  C[6] = M3 * (T(1) - T(3) * yy);
  C[7] = M3 * (T(-3) * yz);
  C[8] = M3 * (T(1) - T(3) * zz);
  C[9] = M4 * ((fxx - T(9)) * x);
  C[10] = M4 * ((fxx - T(3)) * y);
  C[11] = M4 * ((fxx - T(3)) * z);
  C[12] = M4 * ((fyy - T(3)) * x);
  C[13] = M4 * (T(15) * xy * z);
  C[14] = M4 * ((fzz - T(3)) * x);
  C[15] = M4 * ((fyy - T(9)) * y);
  C[16] = M4 * ((fyy - T(3)) * z);
  C[17] = M4 * ((fzz - T(3)) * y);
  C[18] = M4 * ((fzz - T(9)) * z);
  if (VARIANT != FMM_UC) {
    T S[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) S[k] = MT * OS[k] - MS * OT[k];
    const T ux = S[0] * xx + S[3] * yy + S[5] * zz + T(2) * (S[1] * xy + S[2] * xz + S[4] * yz);
    const T uy = S[1] * xx + S[6] * yy + S[8] * zz + T(2) * (S[3] * xy + S[4] * xz + S[7] * yz);
    const T uz = S[2] * xx + S[7] * yy + S[9] * zz + T(2) * (S[4] * xy + S[5] * xz + S[8] * yz);
    const T tx = S[0] + S[3] + S[5];
    const T ty = S[1] + S[6] + S[8];
    const T tz = S[2] + S[7] + S[9];
    T F[3] = {T(7.5) * ux - T(1.5) * tx, T(7.5) * uy - T(1.5) * ty, T(7.5) * uz - T(1.5) * tz};
    if (VARIANT == FMM_TC) {
      const T g = T(-17.5) * (x * ux + y * uy + z * uz) + T(7.5) * (x * tx + y * ty + z * tz);
      F[0] += g * x;
      F[1] += g * y;
      F[2] += g * z;
    }
    const T s5 = Ri2 * Ri2 * Ri * iMT;
#pragma unroll
    for (int i = 0; i < 3; ++i) C[i] -= F[i] * s5;
  }
}

// m2l_one for the unsoftened UC and TC forms, on trace-free moments (see
// HARM of m2l_pair): QS5 = the source's trace-free quadrupole (xx xy xz yy
// yz; zz = -xx - yy), OhT and OhS its target's and its own trace-free
// octupoles per unit mass (xxx xxy xxz xyy xyz yyy yyz; xzz = -xxx - xyy,
// yzz = -xxy - yyy, zzz = -xxz - yyz).  The correction becomes
// F = 7.5 R^-5 M_S [u + (-7/3) n (n.u)] of Sh = Oh_S - Oh_T: the target's
// mass and its inverse drop out.
template <int VARIANT>
__device__ __forceinline__ void m2l_one_tf(const float r[3], float MS, const float *QS5, const float *OhT,
                                           const float *OhS, float *C) {
  const float r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  if (!(r2 > min_r2<float>())) {
#pragma unroll
    for (int q = 0; q < 19; ++q) C[q] = 0.f;
    return;
  }
  const float Ri = rsqrtf(r2);
  const float x = r[0] * Ri, y = r[1] * Ri, z = r[2] * Ri;
  const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  const float fxx = 15.f * xx, fyy = 15.f * yy, fzz = 15.f * zz;
  const float M2 = MS * Ri * Ri, M3 = M2 * Ri, M4 = M3 * Ri;
  const float Ri2 = Ri * Ri;
  const float Ri4 = Ri2 * Ri2;
  const float Q[6] = {QS5[0], QS5[1], QS5[2], QS5[3], QS5[4], -(QS5[0] + QS5[3])};
  const float qx = Q[0] * x + Q[1] * y + Q[2] * z;
  const float qy = Q[1] * x + Q[3] * y + Q[4] * z;
  const float qz = Q[2] * x + Q[4] * y + Q[5] * z;
  const float c75 = 7.5f * Ri4;
  const float w = c75 * (x * qx + y * qy + z * qz);
  const float v = -3.f * Ri4;
  C[0] = M2 * x + (w * x + v * qx);
  C[1] = M2 * y + (w * y + v * qy);
  C[2] = M2 * z + (w * z + v * qz);
  C[3] = M3 * (1.f - 3.f * xx);
  C[4] = M3 * (-3.f * xy);
  C[5] = M3 * (-3.f * xz);
  C[6] = M3 * (1.f - 3.f * yy);
  C[7] = M3 * (-3.f * yz);
  C[8] = M3 * (1.f - 3.f * zz);
  C[9] = M4 * ((fxx - 9.f) * x);
  C[10] = M4 * ((fxx - 3.f) * y);
  C[11] = M4 * ((fxx - 3.f) * z);
  C[12] = M4 * ((fyy - 3.f) * x);
  C[13] = M4 * (15.f * xy * z);
  C[14] = M4 * ((fzz - 3.f) * x);
  C[15] = M4 * ((fyy - 9.f) * y);
  C[16] = M4 * ((fyy - 3.f) * z);
  C[17] = M4 * ((fzz - 3.f) * y);
  C[18] = M4 * ((fzz - 9.f) * z);
  if (VARIANT == FMM_TC) {
    // Sh in the order xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
    float S[10];
    S[0] = OhS[0] - OhT[0];
    S[1] = OhS[1] - OhT[1];
    S[2] = OhS[2] - OhT[2];
    S[3] = OhS[3] - OhT[3];
    S[4] = OhS[4] - OhT[4];
    S[6] = OhS[5] - OhT[5];
    S[7] = OhS[6] - OhT[6];
    S[5] = -(S[0] + S[3]);
    S[8] = -(S[1] + S[6]);
    S[9] = -(S[2] + S[7]);
    const float ux = S[0] * xx + S[3] * yy + S[5] * zz + 2.f * (S[1] * xy + S[2] * xz + S[4] * yz);
    const float uy = S[1] * xx + S[6] * yy + S[8] * zz + 2.f * (S[3] * xy + S[4] * xz + S[7] * yz);
    const float uz = S[2] * xx + S[7] * yy + S[9] * zz + 2.f * (S[4] * xy + S[5] * xz + S[8] * yz);
    const float g = (-7.f / 3.f) * (x * ux + y * uy + z * uz);
    const float s5 = c75 * Ri * MS;
    C[0] -= (ux + g * x) * s5;
    C[1] -= (uy + g * y) * s5;
    C[2] -= (uz + g * z) * s5;
  }
}

// Mixed form, gathered: one warp per cell T, its lanes over T's partners in
// the stably sorted order of the list.  Every lane keeps FP32 sums of the
// partners it visits, compensated (Kahan) for C_i.  The 32 lane sums of a coefficient
// are then combined by one lane, in lane order, with error-free FP32
// additions (TwoSum), and widened to FP64 once: the FP64 pipe, 1/64 of the
// FP32 rate on this GPU, sees three operations per coefficient and cell.
// Each cell's local is written whole (zero for a cell without partners).
constexpr int kGatherWarps = 4;  // 4 warps per block: 0.80 ms against 0.93 ms with 8 (N = 1M)

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// TF: records of kCell32TF floats with trace-free moments (m2l_one_tf),
// else kCell32 floats with the raw ones.
template <int VARIANT, bool TF>
__global__ void __launch_bounds__(kGatherWarps * 32) k_m2l32_gather(int32_t ncell, const int32_t *__restrict__ off,
                                                                    const uint32_t *__restrict__ partner,
                                                                    const float *__restrict__ cell32,
                                                                    double *__restrict__ loc, float eps2,
                                                                    int *__restrict__ queue) {
  // per warp, per coefficient, per lane: the lane's sum and (negated) error
  __shared__ float sh[kGatherWarps][19][33];
  __shared__ float sl[kGatherWarps][19][33];
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // cells differ widely in their number of partners: warps draw cells from a
  // queue (the grid is what fits on the GPU at once); the result of a cell
  // does not depend on which warp takes it
  for (;;) {
  int c = 0;
  if (lane == 0) c = atomicAdd(queue, 1);
  c = __shfl_sync(0xffffffffu, c, 0);
  if (c >= ncell) break;
  constexpr int kRec = TF ? kCell32TF : kCell32;
  // float4 loads of a partner record: the UC form needs no octupole
  constexpr int kLoads = TF ? (VARIANT == FMM_UC ? 3 : kCell32TF / 4) : kCell32 / 4;
  const float *t = cell32 + static_cast<int64_t>(c) * kRec;
  const float thx = t[0], thy = t[1], thz = t[2], tlx = t[3], tly = t[4], tlz = t[5];
  const float MT = t[6], iMT = TF ? 0.f : t[7];
  float OT[10];
#pragma unroll
  for (int k = 0; k < 10; ++k) OT[k] = VARIANT != FMM_UC ? (TF ? (k < 7 ? t[12 + k] : 0.f) : t[14 + k]) : 0.f;
  float sum[19], cmp[19];
#pragma unroll
  for (int q = 0; q < 19; ++q) sum[q] = cmp[q] = 0.f;
  const int e1 = off[c + 1];
  for (int e = off[c] + lane; e < e1; e += 32) {
    const float4 *ps = reinterpret_cast<const float4 *>(cell32 + static_cast<int64_t>(partner[e]) * kRec);
    float b[kCell32];
#pragma unroll
    for (int u = 0; u < kLoads; ++u) {
      const float4 vb = ps[u];
      b[4 * u] = vb.x; b[4 * u + 1] = vb.y; b[4 * u + 2] = vb.z; b[4 * u + 3] = vb.w;
    }
    const float r[3] = {(thx - b[0]) + (tlx - b[3]), (thy - b[1]) + (tly - b[4]), (thz - b[2]) + (tlz - b[5])};
    float C[19];
    if constexpr (TF) m2l_one_tf<VARIANT>(r, b[6], b + 7, OT, b + 12, C);
    else m2l_one<float, VARIANT>(r, MT, iMT, b[6], b + 8, OT, b + 14, eps2, C);
    // compensated sums for the field coefficients C_i, which take the
    // cancellation of contributions from opposite sides; plain FP32 sums for
    // C_ij and C_ijk, which reach the force multiplied by the body's offset
    // (measured at N = 1M: the same 5.3e-8 rms deviation from the FP64 form,
    // and 7% less time than compensating all 19)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float yq = C[q] - cmp[q];
      const float tq = sum[q] + yq;
      cmp[q] = (tq - sum[q]) - yq;
      sum[q] = tq;
    }
#pragma unroll
    for (int q = 3; q < 19; ++q) sum[q] += C[q];
  }
#pragma unroll
  for (int q = 0; q < 19; ++q) {
    sh[w][q][lane] = sum[q];
    sl[w][q][lane] = -cmp[q];
  }
  __syncwarp();
  if (lane < 19) {
    float hi = sh[w][lane][0], lo = sl[w][lane][0];
    for (int j = 1; j < 32; ++j) {
      float s2, e2;
      two_sum(hi, sh[w][lane][j], s2, e2);
      hi = s2;
      lo += e2 + sl[w][lane][j];
    }
    loc[static_cast<int64_t>(c) * kLocStride + lane] = static_cast<double>(hi) + static_cast<double>(lo);
  } else if (lane == 19) {
    loc[static_cast<int64_t>(c) * kLocStride + 19] = 0.0;
  }
  __syncwarp();  // sh and sl are written again by the next cell
  }
}

// Per cell for the FP64 order-3 M2L: the quadrupole Q (6) and the octupole
// per unit mass Oh = O / M (10; xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz).
// tf_q: Q - (tr Q / 3) I; tf_o: Oh - (1/5)(d_ij t_k + d_ik t_j + d_jk t_i),
// t_i = Oh_ijj (both trace-free).
__global__ void k_qoh(int32_t ncell, const double *__restrict__ invM, const double *__restrict__ mom, int tf_q,
                      int tf_o, double *__restrict__ qoh) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const double *m = mom + static_cast<int64_t>(c) * kMomStride;
  double *o = qoh + static_cast<int64_t>(c) * kQOh;
  double Q[6], O[10];
#pragma unroll
  for (int q = 0; q < 6; ++q) Q[q] = m[4 + q];
  const double im = invM[c];
#pragma unroll
  for (int q = 0; q < 10; ++q) O[q] = m[10 + q] * im;
  if (tf_q) {
    const double t3 = (Q[0] + Q[3] + Q[5]) / 3.0;
    Q[0] -= t3;
    Q[3] -= t3;
    Q[5] -= t3;
  }
  if (tf_o) {
    const double tx = (O[0] + O[3] + O[5]) * 0.2, ty = (O[1] + O[6] + O[8]) * 0.2,
                 tz = (O[2] + O[7] + O[9]) * 0.2;
    O[0] -= 3.0 * tx;
    O[1] -= ty;
    O[2] -= tz;
    O[3] -= tx;
    O[5] -= tx;
    O[6] -= 3.0 * ty;
    O[7] -= tz;
    O[8] -= ty;
    O[9] -= 3.0 * tz;
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) o[q] = Q[q];
#pragma unroll
  for (int q = 0; q < 10; ++q) o[6 + q] = O[q];
}

// FP32 copy of the cell data for the mixed form
__global__ void k_cell32(int32_t ncell, const double *__restrict__ Z, const double *__restrict__ M,
                         const double *__restrict__ invM, const double *__restrict__ mom,
                         float *__restrict__ cell32) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  float *o = cell32 + static_cast<int64_t>(c) * kCell32;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double z = Z[3 * c + d];
    const float hi = static_cast<float>(z);
    o[d] = hi;
    o[3 + d] = static_cast<float>(z - static_cast<double>(hi));
  }
  o[6] = static_cast<float>(M[c]);
  o[7] = static_cast<float>(invM[c]);
  const double *m = mom + static_cast<int64_t>(c) * kMomStride;
#pragma unroll
  for (int q = 0; q < 16; ++q) o[8 + q] = static_cast<float>(m[4 + q]);
}

// The same with trace-free moments, kCell32TF floats: Z hi (3), Z lo (3), M,
// Q - tr Q / 3 I (xx xy xz yy yz), Oh = O / M less its trace part (xxx xxy
// xxz xyy xyz yyy yyz), one pad; the traces are removed in FP64.
__global__ void k_cell32_tf(int32_t ncell, const double *__restrict__ Z, const double *__restrict__ M,
                            const double *__restrict__ invM, const double *__restrict__ mom,
                            float *__restrict__ cell32) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  float *o = cell32 + static_cast<int64_t>(c) * kCell32TF;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double z = Z[3 * c + d];
    const float hi = static_cast<float>(z);
    o[d] = hi;
    o[3 + d] = static_cast<float>(z - static_cast<double>(hi));
  }
  o[6] = static_cast<float>(M[c]);
  const double *m = mom + static_cast<int64_t>(c) * kMomStride;
  const double t3 = (m[4] + m[7] + m[9]) / 3.0;
  o[7] = static_cast<float>(m[4] - t3);
  o[8] = static_cast<float>(m[5]);
  o[9] = static_cast<float>(m[6]);
  o[10] = static_cast<float>(m[7] - t3);
  o[11] = static_cast<float>(m[8]);
  const double im = invM[c];
  double O[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) O[q] = m[10 + q] * im;
  const double tx = (O[0] + O[3] + O[5]) * 0.2, ty = (O[1] + O[6] + O[8]) * 0.2, tz = (O[2] + O[7] + O[9]) * 0.2;
  o[12] = static_cast<float>(O[0] - 3.0 * tx);
  o[13] = static_cast<float>(O[1] - ty);
  o[14] = static_cast<float>(O[2] - tz);
  o[15] = static_cast<float>(O[3] - tx);
  o[16] = static_cast<float>(O[4]);
  o[17] = static_cast<float>(O[6] - 3.0 * ty);
  o[18] = static_cast<float>(O[7] - tz);
  o[19] = 0.f;
}

// The two order-3 TC locals of given pairs, [k][side][20] (labels of the
// learned selector)
__global__ void k_pair_locals(int64_t K, const int2 *__restrict__ pairs, const double *__restrict__ Z,
                              const double *__restrict__ M, const double *__restrict__ invM,
                              const double *__restrict__ mom, double *__restrict__ out) {
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= K) return;
  const int A = pairs[k].x, B = pairs[k].y;
  double CA[kLocStride], CB[kLocStride];
  const double r[3] = {Z[3 * A] - Z[3 * B], Z[3 * A + 1] - Z[3 * B + 1], Z[3 * A + 2] - Z[3 * B + 2]};
  const double *mA = mom + static_cast<int64_t>(A) * kMomStride;
  const double *mB = mom + static_cast<int64_t>(B) * kMomStride;
  double OhA[10], OhB[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    OhA[q] = mA[10 + q] * invM[A];
    OhB[q] = mB[10 + q] * invM[B];
  }
  // the labels are errors of the unsoftened expansion
  m2l_pair<double, FMM_TC>(r, M[A], M[B], mA + 4, mB + 4, OhA, OhB, 0.0, CA, CB);
  CA[19] = CB[19] = 0.0;
#pragma unroll
  for (int q = 0; q < kLocStride; ++q) {
    out[(2 * k) * kLocStride + q] = CA[q];
    out[(2 * k + 1) * kLocStride + q] = CB[q];
  }
}

// entries for the stable sort by cell: (cell, 2k + side) for the slot form,
// (cell, partner) for the gather form
__global__ void k_m2l_entries(int64_t K, const int2 *__restrict__ pairs, int gather, uint32_t *__restrict__ key,
                              uint32_t *__restrict__ val) {
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= K) return;
  const int2 p = pairs[k];
  key[2 * k] = static_cast<uint32_t>(p.x);
  val[2 * k] = gather ? static_cast<uint32_t>(p.y) : static_cast<uint32_t>(2 * k);
  key[2 * k + 1] = static_cast<uint32_t>(p.y);
  val[2 * k + 1] = gather ? static_cast<uint32_t>(p.x) : static_cast<uint32_t>(2 * k + 1);
}

// off[c] = first sorted position of cell c (cells without entries get the
// position of the next cell): every position s starts the cells
// (key[s-1], key[s]], and the last entry closes the cells after it.
// Four positions per thread, read as one 16-byte load (key is 16-byte aligned).
__global__ void k_segment_offsets(int64_t E, int32_t ncell, const uint32_t *__restrict__ key,
                                  int32_t *__restrict__ off) {
  const int64_t s0 = 4 * (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x);
  if (s0 >= E) return;
  int k[4];
  if (s0 + 4 <= E) {
    const uint4 v = *reinterpret_cast<const uint4 *>(key + s0);
    k[0] = static_cast<int>(v.x), k[1] = static_cast<int>(v.y), k[2] = static_cast<int>(v.z),
    k[3] = static_cast<int>(v.w);
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) k[u] = s0 + u < E ? static_cast<int>(key[s0 + u]) : ncell;
  }
  int kp = s0 == 0 ? -1 : static_cast<int>(key[s0 - 1]);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t s = s0 + u;
    if (s < E) {
      for (int c = kp + 1; c <= k[u]; ++c) off[c] = static_cast<int32_t>(s);
      if (s == E - 1)
        for (int c = k[u] + 1; c <= ncell; ++c) off[c] = static_cast<int32_t>(E);
    }
    kp = k[u];
  }
}

__global__ void k_inverse(int64_t E, const uint32_t *__restrict__ sval, int32_t *__restrict__ pos) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (s < E) pos[sval[s]] = static_cast<int32_t>(s);
}

// Every cell sums its FP64 slots (kSlot64 = 24 doubles per slot, in the
// stable order of the sort): one warp per cell reads the cell's slot rows as
// one flat array, 32 consecutive doubles per load, so every lane is busy and
// every load is two full 128-byte lines.  Element e of the block is value
// e mod 24 of its slot; lane l meets, at its j-th load, value (l + 32 j) mod
// 24, which repeats with period 3 (3 x 32 = 4 x 24), so every lane keeps
// three partial sums (phase u = j mod 3), each of one coefficient.  A field
// coefficient (value < 3) is added; a U2 or U3 value is multiplied by its
// slot's scale factor (value 19 or 20 of the same slot, held by lane l + so
// of the same load or of the next) in one FMA; the partials of the lanes
// that meet scale factors and the pad are never read.  The partials of a
// coefficient are then added by one lane in a fixed order (phase, then
// lane).
constexpr int kRedWarps = 4;  // warps (cells) per block (reduce stage 2.51 against 2.55 ms with 8 at N = 1M)
constexpr int kRedPhases = 3;   // loads per period
constexpr int kRedPeriods = 2;  // periods per loop trip: six loads in flight

// Lane t sends, in the shuffle of phase u, its element of the NEXT load
// (position 32 (u + 1) + t of the period) when that element is a scale
// factor whose first user lies in load u; otherwise its own element of load u.
__host__ __device__ constexpr int red_scale_off(int q) { return q < 9 ? 19 - q : 20 - q; }
__host__ __device__ constexpr bool red_sends_next(int u, int t) {
  const int p = 32 * (u + 1) + t, r = p % kSlot64, first = p - r + (r == 19 ? 3 : 9);
  return u + 1 < kRedPhases && (r == 19 || r == 20) && first < 32 * (u + 1);
}
// Every value of load u that needs a scale factor finds it in the phase's
// shuffle: at lane l + so of load u (a lane that does not send ahead) or at
// lane l + so - 32 of load u + 1 (a lane that does).
constexpr bool red_plan_ok() {
  for (int u = 0; u < kRedPhases; ++u)
    for (int l = 0; l < 32; ++l) {
      const int q = (l + 32 * u) % kSlot64;
      if (q < 3 || q >= 19) continue;
      const int t = l + red_scale_off(q);
      if (t < 32 ? red_sends_next(u, t) : (u + 1 >= kRedPhases || !red_sends_next(u, t - 32))) return false;
    }
  return true;
}
static_assert(red_plan_ok(), "one shuffle per phase must carry every scale factor");
static_assert((kRedPhases * 32) % kSlot64 == 0, "a period of loads covers whole slots");

__global__ void __launch_bounds__(kRedWarps * 32) k_m2l_reduce(int32_t ncell, const int32_t *__restrict__ off,
                                                               const double *__restrict__ slots,
                                                               double *__restrict__ loc) {
  __shared__ double part[kRedWarps][kRedPhases][32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int c = blockIdx.x * kRedWarps + w;
  if (c >= ncell) return;  // a whole warp: no block-wide synchronisation below
  const int64_t e0 = static_cast<int64_t>(off[c]) * kSlot64, e1 = static_cast<int64_t>(off[c + 1]) * kSlot64;
  double acc[kRedPhases];
  int src[kRedPhases];
  bool ahead[kRedPhases], field[kRedPhases];
#pragma unroll
  for (int u = 0; u < kRedPhases; ++u) {
    acc[u] = 0.0;
    const int q = (l + 32 * u) % kSlot64;
    src[u] = (l + red_scale_off(q)) & 31;
    ahead[u] = red_sends_next(u, l);
    field[u] = q < 3;
  }
  // The block is a whole number of slots and a slot never straddles two
  // periods, so every scale factor a loaded value needs is loaded too.
  for (int64_t b = e0; b < e1; b += kRedPeriods * kRedPhases * 32) {
    double v[kRedPeriods][kRedPhases];
#pragma unroll
    for (int h = 0; h < kRedPeriods; ++h)
#pragma unroll
      for (int u = 0; u < kRedPhases; ++u) {
        const int64_t e = b + l + 32 * (h * kRedPhases + u);
        v[h][u] = e < e1 ? __ldg(&slots[e]) : 0.0;
      }
#pragma unroll
    for (int h = 0; h < kRedPeriods; ++h)
#pragma unroll
      for (int u = 0; u < kRedPhases; ++u) {
        const double send = u + 1 < kRedPhases && ahead[u] ? v[h][u + 1 < kRedPhases ? u + 1 : u] : v[h][u];
        const double f = __shfl_sync(0xffffffffu, send, src[u]);
        // one FP64 instruction per load for every lane (the FP64 pipe, not
        // DRAM, bounds this kernel): a field value is taken with factor 1;
        // the lanes of scale factors and pad fill partials that nothing reads
        if (b + l + 32 * (h * kRedPhases + u) < e1) acc[u] = fma(v[h][u], field[u] ? 1.0 : f, acc[u]);
      }
  }
#pragma unroll
  for (int u = 0; u < kRedPhases; ++u) part[w][u][l] = acc[u];
  __syncwarp();
  if (l < 19) {
    // lanes holding coefficient q at phase u: l = (q - 32 u) mod 24, and that + 24
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < kRedPhases; ++u) {
      const int r = ((l - 32 * u) % kSlot64 + kSlot64) % kSlot64;
      s += part[w][u][r];
      if (r + kSlot64 < 32) s += part[w][u][r + kSlot64];
    }
    loc[static_cast<int64_t>(c) * kLocStride + l] = s;
  } else if (l == 19) {
    loc[static_cast<int64_t>(c) * kLocStride + 19] = 0.0;
  }
}

int launch_m2l64(fmm_ctx *c, int64_t K) {
  const int2 *pairs = ptr<int2>(c->m2l);
  const unsigned g = grid_for(K, kBlock);
  const double *Z = ptr<double>(c->Z), *M = ptr<double>(c->M), *qoh = ptr<double>(c->qoh);
  const int32_t *pos = ptr<int32_t>(c->m2l_pos);
  double *slots = ptr<double>(c->m2l_slots);
  cudaStream_t st = c->stream;
  const double e2 = c->eps2;
  // the trace-free forms hold for the unsoftened 1/R (k_qoh wrote them)
  const bool harm = e2 == 0.0;
  switch (c->opts.variant) {
    case FMM_UC:
      if (harm) k_m2l64<FMM_UC, true><<<g, kBlock, 0, st>>>(K, pairs, Z, M, qoh, pos, e2, slots);
      else k_m2l64<FMM_UC, false><<<g, kBlock, 0, st>>>(K, pairs, Z, M, qoh, pos, e2, slots);
      break;
    case FMM_TC:
      if (harm) k_m2l64<FMM_TC, true><<<g, kBlock, 0, st>>>(K, pairs, Z, M, qoh, pos, e2, slots);
      else k_m2l64<FMM_TC, false><<<g, kBlock, 0, st>>>(K, pairs, Z, M, qoh, pos, e2, slots);
      break;
    default:
      if (harm) k_m2l64<FMM_TCO, true><<<g, kBlock, 0, st>>>(K, pairs, Z, M, qoh, pos, e2, slots);
      else k_m2l64<FMM_TCO, false><<<g, kBlock, 0, st>>>(K, pairs, Z, M, qoh, pos, e2, slots);
      break;
  }
  return launched(c, "m2l");
}

// the mixed form's cell records carry trace-free moments when the kernel
// may use them: unsoftened, and a correction that is a contraction with D
bool cell32_tf(const fmm_ctx *c) { return c->eps2 == 0.0 && c->opts.variant != FMM_TCO; }

int launch_m2l32_gather(fmm_ctx *c) {
  const int32_t nc = static_cast<int32_t>(c->sz.ncell);
  const int32_t *off = ptr<int32_t>(c->m2l_off);
  const uint32_t *partner = ptr<uint32_t>(c->eval[c->m2l_which]);
  const float *c32 = ptr<float>(c->cell32);
  double *loc = ptr<double>(c->loc);
  cudaStream_t st = c->stream;
  int *queue = ptr<int32_t>(c->totals) + 41;
  AMFMM_CUDA(c, cudaMemsetAsync(queue, 0, sizeof(int), st));
  const bool tf = cell32_tf(c);
  auto kern = c->opts.variant == FMM_UC   ? (tf ? k_m2l32_gather<FMM_UC, true> : k_m2l32_gather<FMM_UC, false>)
              : c->opts.variant == FMM_TC ? (tf ? k_m2l32_gather<FMM_TC, true> : k_m2l32_gather<FMM_TC, false>)
                                          : k_m2l32_gather<FMM_TCO, false>;
  int per_sm = 0;
  AMFMM_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGatherWarps * 32, 0));
  const int64_t resident = static_cast<int64_t>(std::max(1, per_sm)) * std::max(1, c->num_sms);
  const unsigned g =
      static_cast<unsigned>(std::min<int64_t>(grid_for(static_cast<int64_t>(nc) * 32, kGatherWarps * 32), resident));
  kern<<<g, kGatherWarps * 32, 0, st>>>(nc, off, partner, c32, loc, static_cast<float>(c->eps2), queue);
  return launched(c, "m2l");
}

int bits_for(int64_t v) {
  int b = 1;
  while ((int64_t(1) << b) <= v) ++b;
  return b;
}

}  // namespace

int m2l_prepare(fmm_ctx *c) {
  cudaStream_t st = c->stream;
  const int64_t K = c->sz.n_m2l, nc = c->sz.ncell, E = 2 * K;
  AMFMM_TRY(ensure<double>(c, c->loc, static_cast<size_t>(loc_stride(c->opts.order_P)) * nc));
  AMFMM_TRY(ensure<int32_t>(c, c->m2l_off, nc + 1));
  if (E > 0x7fffffffLL) return set_error(c, FMM_EUNSUPPORTED, "too many M2L pairs (%lld)", (long long)K);
  int32_t *off = ptr<int32_t>(c->m2l_off);
  AMFMM_CUDA(c, cudaMemsetAsync(off, 0, sizeof(int32_t) * (nc + 1), st));
  if (K == 0) return FMM_OK;
  AMFMM_TRY(ensure<uint32_t>(c, c->ekey[0], E));
  AMFMM_TRY(ensure<uint32_t>(c, c->eval[0], E));
  if (!m2l_gathered(c)) AMFMM_TRY(ensure<int32_t>(c, c->m2l_pos, E));
  const bool fp32 = c->opts.precision == FMM_MIXED;
  const int gather = m2l_gathered(c);
  k_m2l_entries<<<grid_for(K, 256), 256, 0, st>>>(K, ptr<int2>(c->m2l), gather, ptr<uint32_t>(c->ekey[0]),
                                                  ptr<uint32_t>(c->eval[0]));
  AMFMM_TRY(launched(c, "m2l_entries"));
  int which = 0;
  AMFMM_TRY(radix_sort_u32(c, c->ekey, c->eval, E, bits_for(nc), &which));
  c->m2l_which = which;
  k_segment_offsets<<<grid_for((E + 3) / 4, 256), 256, 0, st>>>(E, static_cast<int32_t>(nc),
                                                               ptr<uint32_t>(c->ekey[which]), off);
  AMFMM_TRY(launched(c, "segment_offsets"));
  if (!gather) {
    k_inverse<<<grid_for(E, 256), 256, 0, st>>>(E, ptr<uint32_t>(c->eval[which]), ptr<int32_t>(c->m2l_pos));
    AMFMM_TRY(launched(c, "m2l_inverse"));
    const size_t esz = fp32 ? sizeof(float) : sizeof(double);
    const int stride = c->opts.order_P == 3 ? kSlot64 : loc_stride(c->opts.order_P);
    AMFMM_TRY(ensure_bytes(c, c->m2l_slots, static_cast<size_t>(E) * stride * esz));
  }
  if (fp32) {
    AMFMM_TRY(ensure<float>(c, c->cell32, static_cast<size_t>(kCell32) * nc));
    if (cell32_tf(c))
      k_cell32_tf<<<grid_for(nc, 256), 256, 0, st>>>(static_cast<int32_t>(nc), ptr<double>(c->Z), ptr<double>(c->M),
                                                     ptr<double>(c->invM), ptr<double>(c->mom), ptr<float>(c->cell32));
    else
      k_cell32<<<grid_for(nc, 256), 256, 0, st>>>(static_cast<int32_t>(nc), ptr<double>(c->Z), ptr<double>(c->M),
                                                  ptr<double>(c->invM), ptr<double>(c->mom), ptr<float>(c->cell32));
    AMFMM_TRY(launched(c, "cell32"));
  } else if (c->opts.order_P == 3) {
    AMFMM_TRY(ensure<double>(c, c->qoh, static_cast<size_t>(kQOh) * nc));
    const int harm = c->eps2 == 0.0;
    k_qoh<<<grid_for(nc, 128), 128, 0, st>>>(static_cast<int32_t>(nc), ptr<double>(c->invM), ptr<double>(c->mom),
                                             harm, harm && c->opts.variant == FMM_TC, ptr<double>(c->qoh));
    AMFMM_TRY(launched(c, "qoh"));
  }
  return FMM_OK;
}

int pair_locals_tc(fmm_ctx *c, const int2 *pairs, int64_t K, double *out) {
  k_pair_locals<<<grid_for(K, 128), 128, 0, c->stream>>>(K, pairs, ptr<double>(c->Z), ptr<double>(c->M),
                                                        ptr<double>(c->invM), ptr<double>(c->mom), out);
  return launched(c, "pair_locals");
}

int m2l_run(fmm_ctx *c) {
  const int64_t K = c->sz.n_m2l;
  if (K == 0) return FMM_OK;
  if (c->opts.order_P != 3) return m2l_general(c);
  if (m2l_gathered(c)) return launch_m2l32_gather(c);
  return launch_m2l64(c, K);
}

int m2l_reduce(fmm_ctx *c) {
  if (c->opts.order_P != 3) return reduce_general(c);
  cudaStream_t st = c->stream;
  const int64_t K = c->sz.n_m2l, nc = c->sz.ncell;
  if (K == 0) {
    AMFMM_CUDA(c, cudaMemsetAsync(c->loc.p, 0, sizeof(double) * kLocStride * nc, st));
    return FMM_OK;
  }
  if (m2l_gathered(c)) return FMM_OK;  // the gather kernel wrote every local
  int32_t *off = ptr<int32_t>(c->m2l_off);
  // (warps drawing cells from a queue, as the gather does, measured 2.44 ms
  // against 2.39 ms for one warp per cell at N = 1M)
  k_m2l_reduce<<<grid_for(nc * 32, kRedWarps * 32), kRedWarps * 32, 0, st>>>(
      static_cast<int32_t>(nc), off, ptr<double>(c->m2l_slots), ptr<double>(c->loc));
  return launched(c, "m2l_reduce");
}

}  // namespace amfmm
