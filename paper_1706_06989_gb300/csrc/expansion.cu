// expansion.cu -- a7': the general-order expansion of App. A on the GPU
// (orders P = 4 and 5 from generated code, FP64; P = 6 .. 8 from the
// table-driven kernels of expansion_table.cu), reusing the tree, walk and
// near field of the order-3 path.  The per-order arithmetic is generated (expansion_gen.cuh);
// this file holds the kernels and their launches:
//   P2M   moments of order 0..P about each leaf's centre of mass
//   M2M   shifted child moments, level by level
//   M2L   mutual interaction of every accepted pair: locals of order 1..P on
//         both sides and the corrective force (TC: App. A; TCO: its
//         projection perpendicular to r), written to slots
//   sums  fixed-order per-cell sums of the slots (as at order 3)
//   L2L / L2P  as at order 3, to order P
#include "internal.cuh"
#include "geom.cuh"

namespace amfmm {
namespace {

__device__ __forceinline__ double rsqrt_t(double v) { return rsqrt(v); }

#include "expansion_gen.cuh"

template <int P>
__global__ void k_leaf_upward_gen(int32_t nleaf, const int32_t *__restrict__ leaves,
                                  const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
                                  const double *__restrict__ X, const double *__restrict__ Y,
                                  const double *__restrict__ Zb, const double *__restrict__ Mb,
                                  double *__restrict__ S, double *__restrict__ M, double *__restrict__ Z,
                                  double *__restrict__ invM, double *__restrict__ mom) {
  using E = Expansion<P>;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nleaf) return;
  const int c = leaves[q];
  const int b = begin[c], e = b + count[c];
  double z[3];
  leaf_com(c, b, e, X, Y, Zb, Mb, S, M, Z, invM, z);
  double mo[E::kNM];
#pragma unroll
  for (int k = 0; k < E::kNM; ++k) mo[k] = 0.0;
  for (int i = b; i < e; ++i) E::p2m_add(mo, Mb[i], X[i] - z[0], Y[i] - z[1], Zb[i] - z[2]);
  mo[0] = M[c];
  double *out = mom + static_cast<int64_t>(c) * E::kNM;
#pragma unroll
  for (int k = 0; k < E::kNM; ++k) out[k] = mo[k];
}

template <int P>
__global__ void k_internal_upward_gen(int32_t c0, int32_t c1, const int32_t *__restrict__ first_child,
                                      const int32_t *__restrict__ nchild, double *__restrict__ S,
                                      double *__restrict__ M, double *__restrict__ Z, double *__restrict__ invM,
                                      double *__restrict__ mom) {
  using E = Expansion<P>;
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c1) return;
  const int nch = nchild[c];
  if (nch == 0) return;
  const int f = first_child[c];
  double z[3];
  parent_com(c, f, nch, S, M, Z, invM, z);
  double p[E::kNM];
#pragma unroll
  for (int k = 0; k < E::kNM; ++k) p[k] = 0.0;
  for (int k = f; k < f + nch; ++k) {
    const double s[3] = {Z[3 * k] - z[0], Z[3 * k + 1] - z[1], Z[3 * k + 2] - z[2]};
    E::m2m_add(p, mom + static_cast<int64_t>(k) * E::kNM, s);
  }
  p[0] = M[c];
  double *out = mom + static_cast<int64_t>(c) * E::kNM;
#pragma unroll
  for (int k = 0; k < E::kNM; ++k) out[k] = p[k];
}

// one thread per accepted pair; the two local contributions go straight to
// their slots (kNL doubles each)
template <int P, int VARIANT>
__global__ void __launch_bounds__(128) k_m2l_gen(int64_t K, const int2 *__restrict__ pairs,
                                                 const double *__restrict__ Z, const double *__restrict__ invM,
                                                 const double *__restrict__ mom, const int32_t *__restrict__ pos,
                                                 double *__restrict__ slots) {
  using E = Expansion<P>;
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= K) return;
  const int A = pairs[k].x, B = pairs[k].y;
  const double r[3] = {Z[3 * A] - Z[3 * B], Z[3 * A + 1] - Z[3 * B + 1], Z[3 * A + 2] - Z[3 * B + 2]};
  double *LA = slots + static_cast<int64_t>(pos[2 * k]) * E::kNL;
  double *LB = slots + static_cast<int64_t>(pos[2 * k + 1]) * E::kNL;
  E::template m2l<double, VARIANT>(r, mom + static_cast<int64_t>(A) * E::kNM, mom + static_cast<int64_t>(B) * E::kNM,
                                   invM[A], invM[B], LA, LB, 0.0);
}

// per-cell sums of the slots in sorted order; a warp per cell, lanes over
// the coefficients
__global__ void k_reduce_stride(int32_t ncell, int stride, const int32_t *__restrict__ off,
                                const double *__restrict__ slots, double *__restrict__ loc) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= ncell) return;
  const int s0 = off[c], s1 = off[c + 1];
  for (int q = lane; q < stride; q += 32) {
    double acc = 0.0;
    for (int s = s0; s < s1; ++s) acc += slots[static_cast<int64_t>(s) * stride + q];
    loc[static_cast<int64_t>(c) * stride + q] = acc;
  }
}

template <int P>
__global__ void k_l2l_gen(int32_t c0, int32_t c1, const int32_t *__restrict__ parent, const double *__restrict__ Z,
                          double *__restrict__ loc) {
  using E = Expansion<P>;
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c1) return;
  const int p = parent[c];
  const double s[3] = {Z[3 * c] - Z[3 * p], Z[3 * c + 1] - Z[3 * p + 1], Z[3 * c + 2] - Z[3 * p + 2]};
  double Lp[E::kNL], Lc[E::kNL];
#pragma unroll
  for (int q = 0; q < E::kNL; ++q) {
    Lp[q] = loc[static_cast<int64_t>(p) * E::kNL + q];
    Lc[q] = loc[static_cast<int64_t>(c) * E::kNL + q];
  }
  E::l2l_add(Lc, Lp, s);
#pragma unroll
  for (int q = 0; q < E::kNL; ++q) loc[static_cast<int64_t>(c) * E::kNL + q] = Lc[q];
}

template <int P>
__global__ void k_l2p_gen(int64_t n, const int32_t *__restrict__ leaf_of, const double *__restrict__ Z,
                          const double *__restrict__ loc, const double *__restrict__ X, const double *__restrict__ Y,
                          const double *__restrict__ Zb, const double *__restrict__ near, double *__restrict__ acc) {
  using E = Expansion<P>;
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const int L = leaf_of[i];
  const double x[3] = {X[i] - Z[3 * L], Y[i] - Z[3 * L + 1], Zb[i] - Z[3 * L + 2]};
  double g[3];
  E::l2p(loc + static_cast<int64_t>(L) * E::kNL, x, g);
#pragma unroll
  for (int d = 0; d < 3; ++d) acc[d * n + i] = near[d * n + i] + g[d];
}

template <int P>
int upward_p(fmm_ctx *c) {
  cudaStream_t st = c->stream;
  k_leaf_upward_gen<P><<<grid_for(c->sz.nleaf, 128), 128, 0, st>>>(
      static_cast<int32_t>(c->sz.nleaf), ptr<int32_t>(c->leaves), ptr<int32_t>(c->begin), ptr<int32_t>(c->count),
      ptr<double>(c->X), ptr<double>(c->Y), ptr<double>(c->Zb), ptr<double>(c->Mb), ptr<double>(c->S),
      ptr<double>(c->M), ptr<double>(c->Z), ptr<double>(c->invM), ptr<double>(c->mom));
  AMFMM_TRY(launched(c, "leaf_upward_gen"));
  for (int lev = c->sz.depth - 1; lev >= 0; --lev) {
    const int64_t c0 = c->sz.lvl_off[lev], c1 = c->sz.lvl_off[lev + 1];
    k_internal_upward_gen<P><<<grid_for(c1 - c0, 128), 128, 0, st>>>(
        static_cast<int32_t>(c0), static_cast<int32_t>(c1), ptr<int32_t>(c->first_child), ptr<int32_t>(c->nchild),
        ptr<double>(c->S), ptr<double>(c->M), ptr<double>(c->Z), ptr<double>(c->invM), ptr<double>(c->mom));
    AMFMM_TRY(launched(c, "internal_upward_gen"));
  }
  return FMM_OK;
}

template <int P>
int m2l_p(fmm_ctx *c) {
  const int64_t K = c->sz.n_m2l;
  const unsigned g = grid_for(K, 128);
  const int2 *pairs = ptr<int2>(c->m2l);
  const double *Z = ptr<double>(c->Z), *iM = ptr<double>(c->invM), *mom = ptr<double>(c->mom);
  const int32_t *pos = ptr<int32_t>(c->m2l_pos);
  double *slots = ptr<double>(c->m2l_slots);
  cudaStream_t st = c->stream;
  switch (c->opts.variant) {
    case FMM_UC: k_m2l_gen<P, FMM_UC><<<g, 128, 0, st>>>(K, pairs, Z, iM, mom, pos, slots); break;
    case FMM_TC: k_m2l_gen<P, FMM_TC><<<g, 128, 0, st>>>(K, pairs, Z, iM, mom, pos, slots); break;
    default: k_m2l_gen<P, FMM_TCO><<<g, 128, 0, st>>>(K, pairs, Z, iM, mom, pos, slots); break;
  }
  return launched(c, "m2l_gen");
}

template <int P>
int downward_p(fmm_ctx *c) {
  cudaStream_t st = c->stream;
  const int64_t n = c->sz.n;
  for (int lev = 1; lev <= c->sz.depth; ++lev) {
    const int64_t c0 = c->sz.lvl_off[lev], c1 = c->sz.lvl_off[lev + 1];
    if (c1 <= c0) continue;
    k_l2l_gen<P><<<grid_for(c1 - c0, 128), 128, 0, st>>>(static_cast<int32_t>(c0), static_cast<int32_t>(c1),
                                                         ptr<int32_t>(c->parent), ptr<double>(c->Z), ptr<double>(c->loc));
    AMFMM_TRY(launched(c, "l2l_gen"));
  }
  k_l2p_gen<P><<<grid_for(n, 256), 256, 0, st>>>(n, ptr<int32_t>(c->leaf_of), ptr<double>(c->Z), ptr<double>(c->loc),
                                                 ptr<double>(c->X), ptr<double>(c->Y), ptr<double>(c->Zb),
                                                 ptr<double>(c->near), ptr<double>(c->acc));
  return launched(c, "l2p_gen");
}

}  // namespace

int mom_stride(int P) { return (P + 1) * (P + 2) * (P + 3) / 6; }
int loc_stride(int P) { return P == 3 ? kLocStride : mom_stride(P) - 1; }

int upward_general(fmm_ctx *c) {
  switch (c->opts.order_P) {
    case 4: return upward_p<4>(c);
    case 5: return upward_p<5>(c);
    default: return upward_table(c);
  }
}

int m2l_general(fmm_ctx *c) {
  if (c->sz.n_m2l == 0) return FMM_OK;
  switch (c->opts.order_P) {
    case 4: return m2l_p<4>(c);
    case 5: return m2l_p<5>(c);
    default: return m2l_table(c);
  }
}

int reduce_general(fmm_ctx *c) {
  const int64_t nc = c->sz.ncell;
  const int stride = loc_stride(c->opts.order_P);
  if (c->sz.n_m2l == 0) {
    AMFMM_CUDA(c, cudaMemsetAsync(c->loc.p, 0, sizeof(double) * stride * nc, c->stream));
    return FMM_OK;
  }
  k_reduce_stride<<<grid_for(nc * 32, 256), 256, 0, c->stream>>>(static_cast<int32_t>(nc), stride,
                                                                  ptr<int32_t>(c->m2l_off), ptr<double>(c->m2l_slots),
                                                                  ptr<double>(c->loc));
  return launched(c, "reduce_general");
}

int downward_general(fmm_ctx *c) {
  switch (c->opts.order_P) {
    case 4: return downward_p<4>(c);
    case 5: return downward_p<5>(c);
    default: return downward_table(c);
  }
}

}  // namespace amfmm
