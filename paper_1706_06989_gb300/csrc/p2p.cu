// p2p.cu -- a8: mutual near-field sums (Sec. 2: "the force contributions from
// any remaining nearby particles are computed directly").
//
// For every leaf pair (A, B) each body pair (i in A, j in B) is evaluated
// once: with d = X_j - X_i and s = 1/|d|^3,
//     a_i += m_j s d,    a_j -= m_i s d,
// so the two contributions are equal and opposite (linear momentum is
// conserved pair by pair).  A leaf with itself sums every ordered pair i != j
// once on the side of i.  A pair at zero separation contributes nothing.
//
// Work layout: one warp per leaf A, over A's self interaction and every leaf
// pair whose smaller id is A (pairs sorted by A, stable).  Lane = (row body i
// of A, column phase g): with n_A rows, R = 32 / n_A lanes share a row and take
// every R-th body of the partner, so small leaves still fill the warp.  The
// A-side sum stays in registers across all partners; the B-side sums are
// column sums through shared memory, b_j = sum_i s_ij (x_i - x_j) written as
// T_j - x_j S_j with S_j = sum_i s_ij and T_j = sum_i s_ij x_i (x relative to
// Z_A), one partial per (pair, body of B).  Each body then adds its partials in
// the order of the stable sort.  Every sum has a fixed order; no atomics.
//
// FP64 form: everything in FP64.  Mixed form: coordinates relative to Z_A
// rounded to FP32, pair terms in FP32, the per-lane running sum over all
// partners compensated (Kahan) in FP32, lanes and partials combined in FP64.
#include "internal.cuh"

namespace amfmm {
namespace {

constexpr int kWarps = 4;
constexpr int kCH = 32;

__device__ __forceinline__ double rsqrt_t(double v) { return rsqrt(v); }
__device__ __forceinline__ float rsqrt_t(float v) { return rsqrtf(v); }

template <class T>
struct Acc3 {
  T s[3] = {T(0), T(0), T(0)};
  __device__ __forceinline__ void add(int d, T v) { s[d] += v; }
  __device__ __forceinline__ double get(int d) const { return static_cast<double>(s[d]); }
};
// compensated running sum for the FP32 form
template <>
struct Acc3<float> {
  float s[3] = {0.f, 0.f, 0.f}, c[3] = {0.f, 0.f, 0.f};
  __device__ __forceinline__ void add(int d, float v) {
    const float y = __fsub_rn(v, c[d]);
    const float t = __fadd_rn(s[d], y);
    c[d] = __fsub_rn(__fsub_rn(t, s[d]), y);
    s[d] = t;
  }
  __device__ __forceinline__ double get(int d) const {
    return static_cast<double>(s[d]) - static_cast<double>(c[d]);
  }
};

template <class T>
__global__ void __launch_bounds__(kWarps * 32) k_p2p(
    int32_t nleaf, int64_t n, const int32_t *__restrict__ leaves, const int32_t *__restrict__ begin,
    const int32_t *__restrict__ count, const double *__restrict__ Zc, const double *__restrict__ X,
    const double *__restrict__ Y, const double *__restrict__ Zb, const double *__restrict__ Mb,
    const int32_t *__restrict__ offA, const int2 *__restrict__ pairs, const int32_t *__restrict__ pos,
    const int64_t *__restrict__ poff, double *__restrict__ near, T *__restrict__ slots,
    unsigned long long *__restrict__ stat_pairs) {
  __shared__ T sS[kWarps][kCH][33];
  __shared__ T sX[kWarps][32][3];
  __shared__ double sR[kWarps][32][3];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int q = blockIdx.x * kWarps + w;
  if (q >= nleaf) return;
  const int L = leaves[q];
  const int bA = begin[L], nA = count[L];
  const double zx = Zc[3 * L], zy = Zc[3 * L + 1], zz = Zc[3 * L + 2];
  const int kb = offA[L], ke = offA[L + 1];
  unsigned long long npairs = static_cast<unsigned long long>(nA) * (nA - 1) / 2;

  for (int r0 = 0; r0 < nA; r0 += 32) {
    const int nrow = min(32, nA - r0);
    const int R = 32 / nrow;
    const int il = l / R, g = l % R;
    const bool active = il < nrow;
    T xi = T(0), yi = T(0), zi = T(0), mi = T(0);
    if (active) {
      const int i = bA + r0 + il;
      xi = T(X[i] - zx);
      yi = T(Y[i] - zy);
      zi = T(Zb[i] - zz);
      mi = T(Mb[i]);
      if (g == 0) {
        sX[w][il][0] = xi;
        sX[w][il][1] = yi;
        sX[w][il][2] = zi;
      }
    }
    Acc3<T> a;
    // self: ordered pairs i != j, one-sided
    if (active) {
      for (int j = g; j < nA; j += R) {
        const int jb = bA + j;
        const T dx = T(X[jb] - zx) - xi, dy = T(Y[jb] - zy) - yi, dz = T(Zb[jb] - zz) - zi;
        const T r2 = dx * dx + dy * dy + dz * dz;
        if (r2 > T(0)) {
          const T ri = rsqrt_t(r2);
          const T sj = T(Mb[jb]) * (ri * ri * ri);
          a.add(0, sj * dx);
          a.add(1, sj * dy);
          a.add(2, sj * dz);
        }
      }
    }
    // leaf pairs with A as the smaller id
    for (int k = kb; k < ke; ++k) {
      const int B = pairs[k].y;
      const int bB = begin[B], nB = count[B];
      if (r0 == 0 && l == 0) npairs += static_cast<unsigned long long>(nA) * nB;
      T *out = slots + poff[pos[k]];
      for (int j0 = 0; j0 < nB; j0 += kCH) {
        const int ncol = min(kCH, nB - j0);
        if (active) {
          for (int jj = g; jj < ncol; jj += R) {
            const int jb = bB + j0 + jj;
            const T dx = T(X[jb] - zx) - xi, dy = T(Y[jb] - zy) - yi, dz = T(Zb[jb] - zz) - zi;
            const T r2 = dx * dx + dy * dy + dz * dz;
            T si = T(0);
            if (r2 > T(0)) {
              const T ri = rsqrt_t(r2);
              const T r3 = ri * ri * ri;
              const T sj = T(Mb[jb]) * r3;
              a.add(0, sj * dx);
              a.add(1, sj * dy);
              a.add(2, sj * dz);
              si = mi * r3;
            }
            sS[w][jj][il] = si;
          }
        }
        __syncwarp();
        if (l < ncol) {
          const int jb = bB + j0 + l;
          const T xj = T(X[jb] - zx), yj = T(Y[jb] - zy), zj = T(Zb[jb] - zz);
          T S = T(0), Tx = T(0), Ty = T(0), Tz = T(0);
          for (int r = 0; r < nrow; ++r) {
            const T s = sS[w][l][r];
            S += s;
            Tx += s * sX[w][r][0];
            Ty += s * sX[w][r][1];
            Tz += s * sX[w][r][2];
          }
          T *o = out + 3 * (j0 + l);
          const T bx = Tx - xj * S, by = Ty - yj * S, bz = Tz - zj * S;
          if (r0 == 0) {
            o[0] = bx;
            o[1] = by;
            o[2] = bz;
          } else {
            o[0] += bx;
            o[1] += by;
            o[2] += bz;
          }
        }
        __syncwarp();
      }
    }
    sR[w][l][0] = a.get(0);
    sR[w][l][1] = a.get(1);
    sR[w][l][2] = a.get(2);
    __syncwarp();
    if (l < nrow) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      for (int t = 0; t < R; ++t) {
        s0 += sR[w][l * R + t][0];
        s1 += sR[w][l * R + t][1];
        s2 += sR[w][l * R + t][2];
      }
      const int64_t i = bA + r0 + l;
      near[i] = s0;
      near[n + i] = s1;
      near[2 * n + i] = s2;
    }
    __syncwarp();
  }
  if (l == 0) atomicAdd(stat_pairs, npairs);
}

// Each body adds, in sorted order, the partials that the pairs in which its
// leaf is the larger id left for it.
template <class T>
__global__ void k_p2p_reduce(int64_t n, const int32_t *__restrict__ leaf_of, const int32_t *__restrict__ begin,
                             const int32_t *__restrict__ offB, const int64_t *__restrict__ poff,
                             const T *__restrict__ slots, double *__restrict__ near) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const int L = leaf_of[i];
  const int t = static_cast<int>(i - begin[L]);
  double a0 = near[i], a1 = near[n + i], a2 = near[2 * n + i];
  for (int e = offB[L]; e < offB[L + 1]; ++e) {
    const T *p = slots + poff[e] + 3 * t;
    a0 += static_cast<double>(p[0]);
    a1 += static_cast<double>(p[1]);
    a2 += static_cast<double>(p[2]);
  }
  near[i] = a0;
  near[n + i] = a1;
  near[2 * n + i] = a2;
}

__global__ void k_pair_keys(int64_t K, const int2 *__restrict__ pairs, int side, uint32_t *__restrict__ key,
                            uint32_t *__restrict__ val, int32_t *__restrict__ cnt) {
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= K) return;
  const int c = side == 0 ? pairs[k].x : pairs[k].y;
  key[k] = static_cast<uint32_t>(c);
  val[k] = static_cast<uint32_t>(k);
  atomicAdd(&cnt[c], 1);
}

__global__ void k_gather_pairs(int64_t K, const int2 *__restrict__ in, const uint32_t *__restrict__ sval,
                               int2 *__restrict__ out) {
  const int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (s < K) out[s] = in[sval[s]];
}

// pos[s] = CSR position of sorted pair s on its B side; len[e] = 3 n_B
__global__ void k_b_positions(int64_t K, const uint32_t *__restrict__ sval, const int2 *__restrict__ pairs,
                              const int32_t *__restrict__ count, int32_t *__restrict__ pos,
                              int64_t *__restrict__ len) {
  const int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (e >= K) return;
  const uint32_t s = sval[e];
  pos[s] = static_cast<int32_t>(e);
  len[e] = 3 * static_cast<int64_t>(count[pairs[s].y]);
}

int bits_for(int64_t v) {
  int b = 1;
  while ((int64_t(1) << b) <= v) ++b;
  return b;
}

template <class T>
int launch_p2p(fmm_ctx *c, int64_t K) {
  cudaStream_t st = c->stream;
  const int64_t n = c->sz.n;
  const int32_t nleaf = static_cast<int32_t>(c->sz.nleaf);
  k_p2p<T><<<grid_for(nleaf, kWarps), kWarps * 32, 0, st>>>(
      nleaf, n, ptr<int32_t>(c->leaves), ptr<int32_t>(c->begin), ptr<int32_t>(c->count),
      ptr<double>(c->Z), ptr<double>(c->X), ptr<double>(c->Y), ptr<double>(c->Zb), ptr<double>(c->Mb),
      ptr<int32_t>(c->p2p_offA), ptr<int2>(c->p2p_A), ptr<int32_t>(c->p2p_pos), ptr<int64_t>(c->p2p_poff),
      ptr<double>(c->near), static_cast<T *>(c->p2p_slots.p),
      ptr<unsigned long long>(c->totals) + 8);
  AMFMM_TRY(launched(c, "p2p"));
  timer(c, kP2PEnd);
  if (K > 0) {
    k_p2p_reduce<T><<<grid_for(n, 256), 256, 0, st>>>(n, ptr<int32_t>(c->leaf_of), ptr<int32_t>(c->begin),
                                                       ptr<int32_t>(c->p2p_offB), ptr<int64_t>(c->p2p_poff),
                                                       static_cast<T *>(c->p2p_slots.p), ptr<double>(c->near));
    AMFMM_TRY(launched(c, "p2p_reduce"));
  }
  return FMM_OK;
}

}  // namespace

int p2p(fmm_ctx *c) {
  cudaStream_t st = c->stream;
  const int64_t K = c->sz.n_p2p, nc = c->sz.ncell, n = c->sz.n;
  const bool fp32 = c->opts.precision == FMM_MIXED;
  AMFMM_TRY(ensure<double>(c, c->near, 3 * n));
  AMFMM_TRY(ensure<int32_t>(c, c->p2p_offA, nc + 1));
  AMFMM_TRY(ensure<int32_t>(c, c->p2p_offB, nc + 1));
  AMFMM_TRY(ensure<int64_t>(c, c->p2p_poff, K + 1));
  AMFMM_TRY(ensure<int32_t>(c, c->p2p_pos, K + 1));
  AMFMM_TRY(ensure<int2>(c, c->p2p_A, K + 1));
  AMFMM_TRY(ensure<int32_t>(c, c->incl, std::max<int64_t>(nc + 1, n + 1)));
  int32_t *cnt = ptr<int32_t>(c->incl);
  int32_t *offA = ptr<int32_t>(c->p2p_offA), *offB = ptr<int32_t>(c->p2p_offB);
  int64_t *stat = ptr<int64_t>(c->totals) + 8;
  AMFMM_CUDA(c, cudaMemsetAsync(stat, 0, sizeof(int64_t), st));
  if (K > 0) {
    AMFMM_TRY(ensure<uint32_t>(c, c->pkey[0], K));
    AMFMM_TRY(ensure<uint32_t>(c, c->pval[0], K));
    // group by A (stable)
    AMFMM_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nc + 1), st));
    k_pair_keys<<<grid_for(K, 256), 256, 0, st>>>(K, ptr<int2>(c->p2p), 0, ptr<uint32_t>(c->pkey[0]),
                                                  ptr<uint32_t>(c->pval[0]), cnt);
    AMFMM_TRY(launched(c, "p2p_keysA"));
    AMFMM_TRY(exclusive_scan_i32(c, cnt, offA, nc + 1, nullptr));
    int which = 0;
    AMFMM_TRY(radix_sort_u32(c, c->pkey, c->pval, K, bits_for(nc), &which));
    k_gather_pairs<<<grid_for(K, 256), 256, 0, st>>>(K, ptr<int2>(c->p2p), ptr<uint32_t>(c->pval[which]),
                                                     ptr<int2>(c->p2p_A));
    AMFMM_TRY(launched(c, "p2p_gather"));
    // CSR on the B side
    AMFMM_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nc + 1), st));
    k_pair_keys<<<grid_for(K, 256), 256, 0, st>>>(K, ptr<int2>(c->p2p_A), 1, ptr<uint32_t>(c->pkey[0]),
                                                  ptr<uint32_t>(c->pval[0]), cnt);
    AMFMM_TRY(launched(c, "p2p_keysB"));
    AMFMM_TRY(exclusive_scan_i32(c, cnt, offB, nc + 1, nullptr));
    AMFMM_TRY(radix_sort_u32(c, c->pkey, c->pval, K, bits_for(nc), &which));
    // lengths into a temporary int64 array, then scanned into poff
    AMFMM_TRY(ensure<int64_t>(c, c->p2p_len, K + 1));
    int64_t *len = ptr<int64_t>(c->p2p_len);
    k_b_positions<<<grid_for(K, 256), 256, 0, st>>>(K, ptr<uint32_t>(c->pval[which]), ptr<int2>(c->p2p_A),
                                                    ptr<int32_t>(c->count), ptr<int32_t>(c->p2p_pos), len);
    AMFMM_TRY(launched(c, "p2p_bpos"));
    int64_t *ptot = ptr<int64_t>(c->totals) + 12;
    AMFMM_TRY(exclusive_scan_i64(c, len, ptr<int64_t>(c->p2p_poff), K, ptot));
    int64_t *h = static_cast<int64_t *>(c->hpin);
    AMFMM_CUDA(c, cudaMemcpyAsync(h, ptot, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    AMFMM_CUDA(c, cudaStreamSynchronize(st));
    AMFMM_TRY(ensure_bytes(c, c->p2p_slots, static_cast<size_t>(h[0] + 3) * (fp32 ? sizeof(float) : sizeof(double))));
  } else {
    AMFMM_CUDA(c, cudaMemsetAsync(offA, 0, sizeof(int32_t) * (nc + 1), st));
    AMFMM_CUDA(c, cudaMemsetAsync(offB, 0, sizeof(int32_t) * (nc + 1), st));
    AMFMM_TRY(ensure_bytes(c, c->p2p_slots, 64));
  }
  timer(c, kP2PBeg);
  if (fp32) return launch_p2p<float>(c, K);
  return launch_p2p<double>(c, K);
}

}  // namespace amfmm
