// down.cu -- a9: downward pass.  The local expansion of a cell, written about
// its centre of mass Z (Eqs. 3 and 4 are polynomials in the offset from Z), is
// the sum of its own interactions and its parent's expansion shifted to Z
// (L2L, exact for a polynomial): with s = Z_child - Z_parent,
//     C_i'   = C_i + C_ij s_j + C_ijk s_j s_k / 2
//     C_ij'  = C_ij + C_ijk s_k
//     C_ijk' = C_ijk.
// Every body of a leaf then receives a = -(C_i + C_ij x_j + C_ijk x_j x_k / 2)
// with x = X - Z_leaf (L2P), plus its near-field sum; fmm_forces scatters the
// result to the caller's order and multiplies by G.
#include "internal.cuh"

namespace amfmm {
namespace {

// symmetric index helpers for the local layout
// C_ij: xx xy xz yy yz zz -> 3..8 ; C_ijk: xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz -> 9..18
__device__ __forceinline__ int i2(int i, int j) {
  const int a = min(i, j), b = max(i, j);
  return a == 0 ? b : (a == 1 ? 2 + b : 5);
}
__device__ __forceinline__ int i3(int i, int j, int k) {
  // sort the three indices
  int a = i, b = j, c = k, t;
  if (a > b) { t = a; a = b; b = t; }
  if (b > c) { t = b; b = c; c = t; }
  if (a > b) { t = a; a = b; b = t; }
  if (a == 0) {
    if (b == 0) return c;          // xxx xxy xxz
    if (b == 1) return 2 + c;      // xyy xyz
    return 5;                      // xzz
  }
  if (a == 1) return b == 1 ? 5 + c : 8;  // yyy yyz | yzz
  return 9;                               // zzz
}

__global__ void k_l2l(int32_t c0, int32_t c1, const int32_t *__restrict__ parent,
                      const double *__restrict__ Z, double *__restrict__ loc) {
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c1) return;
  const int p = parent[c];
  const double s[3] = {Z[3 * c] - Z[3 * p], Z[3 * c + 1] - Z[3 * p + 1], Z[3 * c + 2] - Z[3 * p + 2]};
  const double *P = loc + static_cast<int64_t>(p) * kLocStride;
  double *C = loc + static_cast<int64_t>(c) * kLocStride;
  double Pl[19];
#pragma unroll
  for (int q = 0; q < 19; ++q) Pl[q] = P[q];
  // C_ijk' = C_ijk (shift adds nothing new)
#pragma unroll
  for (int q = 0; q < 10; ++q) C[9 + q] += Pl[9 + q];
  // C_ij' = C_ij + C_ijk s_k
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      double v = Pl[3 + i2(i, j)];
#pragma unroll
      for (int k = 0; k < 3; ++k) v += Pl[9 + i3(i, j, k)] * s[k];
      C[3 + i2(i, j)] += v;
    }
  // C_i' = C_i + C_ij s_j + C_ijk s_j s_k / 2
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double v = Pl[i], w = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      v += Pl[3 + i2(i, j)] * s[j];
#pragma unroll
      for (int k = 0; k < 3; ++k) w += Pl[9 + i3(i, j, k)] * s[j] * s[k];
    }
    C[i] += v + 0.5 * w;
  }
}

__global__ void k_l2p(int64_t n, const int32_t *__restrict__ leaf_of, const double *__restrict__ Z,
                      const double *__restrict__ loc, const double *__restrict__ X,
                      const double *__restrict__ Y, const double *__restrict__ Zb,
                      const double *__restrict__ near, double *__restrict__ acc) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const int L = leaf_of[i];
  const double x[3] = {X[i] - Z[3 * L], Y[i] - Z[3 * L + 1], Zb[i] - Z[3 * L + 2]};
  const double *C = loc + static_cast<int64_t>(L) * kLocStride;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double v = C[d], w = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      v += C[3 + i2(d, j)] * x[j];
#pragma unroll
      for (int k = 0; k < 3; ++k) w += C[9 + i3(d, j, k)] * x[j] * x[k];
    }
    acc[d * n + i] = near[d * n + i] - (v + 0.5 * w);
  }
}

__global__ void k_unpermute(int64_t n, const int32_t *__restrict__ order, const double *__restrict__ acc,
                            double G, double *__restrict__ ax, double *__restrict__ ay,
                            double *__restrict__ az) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const int o = order[i];
  ax[o] = G * acc[i];
  ay[o] = G * acc[n + i];
  az[o] = G * acc[2 * n + i];
}

}  // namespace

int downward(fmm_ctx *c) {
  cudaStream_t st = c->stream;
  const int64_t n = c->sz.n;
  AMFMM_TRY(ensure<double>(c, c->acc, 3 * n));
  if (c->opts.order_P != 3) return downward_general(c);
  for (int lev = 1; lev <= c->sz.depth; ++lev) {
    const int64_t c0 = c->sz.lvl_off[lev], c1 = c->sz.lvl_off[lev + 1];
    if (c1 <= c0) continue;
    k_l2l<<<grid_for(c1 - c0, 128), 128, 0, st>>>(static_cast<int32_t>(c0), static_cast<int32_t>(c1),
                                                   ptr<int32_t>(c->parent), ptr<double>(c->Z),
                                                   ptr<double>(c->loc));
    AMFMM_TRY(launched(c, "l2l"));
  }
  k_l2p<<<grid_for(n, 256), 256, 0, st>>>(n, ptr<int32_t>(c->leaf_of), ptr<double>(c->Z), ptr<double>(c->loc),
                                          ptr<double>(c->X), ptr<double>(c->Y), ptr<double>(c->Zb),
                                          ptr<double>(c->near), ptr<double>(c->acc));
  return launched(c, "l2p");
}

int forces(fmm_ctx *c, double *ax, double *ay, double *az) {
  const int64_t n = c->sz.n;
  k_unpermute<<<grid_for(n, 256), 256, 0, c->stream>>>(n, ptr<int32_t>(c->order), ptr<double>(c->acc),
                                                       c->opts.G, ax, ay, az);
  return launched(c, "unpermute");
}

}  // namespace amfmm
