// expansion_table.cu -- a7' at orders P = 6 .. 8: the general-order
// expansion of App. A driven by index tables instead of generated
// straight-line code (which at these orders holds hundreds of values per
// thread and spills).  The formulas are those of the generated orders 4 and
// 5, in multi-index notation (alpha, beta, gamma exponent triples, |a| the
// order, a! the product of the factorials):
//   derivatives  D^g = d^g G(r), G = -1/R, written D^g = R^-(|g|+1) U^g(n),
//                n = r/R, U^g the polynomial in n of the chain rule on G(u),
//                u = r.r (every way of pairing equal indices through u's
//                second derivative, the other indices left as components of
//                r):  U^g = sum_{i,j,l} c_m K_a(i) K_b(j) K_c(l) nx^(a-2i) ny^(b-2j) nz^(c-2l),
//                m = |g| - i - j - l, c_m = -(-1)^m (2m-1)!!,
//                K_a(i) = a! / (2^i i! (a-2i)!)
//   field of B at A:  L_A^a = sum_b (-1)^|b| D^(a+b) M_B^b / b!,   |a| + |b| <= P
//   field of A at B:  L_B^b = (-1)^|b| sum_a D^(a+b) M_A^a / a!
//   correction:       F_k = - sum_{|a|+|b|=P} (-1)^|b| M_A^a M_B^b D^(a+b+e_k) / (a! b!),
//                     +F/M_A on A, -F/M_B on B; TCO: F - n (n.F)
//   P2M: M^a = sum mu x^a;  M2M: M^a += sum_{b<=a} C(a,b) M_child^b s^(a-b)
//   L2L: L'^a += sum_g L^(a+g) s^g / g!;  L2P: g_k = -sum_a L^(a+e_k) x^a / a!
// Multi-indices of order n are stored from offset n (n+1) (n+2) / 6, ordered
// a0 = n..0 and then a1 = n - a0 .. 0, so that the position of (a0, a1, a2)
// in its order is s (s+1) / 2 + a2 with s = a1 + a2.
//
// Work layout: one warp per accepted pair (lanes over the output
// coefficients, the derivatives and scaled moments of the pair staged in
// shared memory), one warp per cell for P2M, M2M and L2L, one thread per
// body for L2P.  FP64 throughout; every sum has a fixed order.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"
#include "geom.cuh"

namespace amfmm {
namespace {

constexpr int kTabMaxP = 8;
constexpr int kNUMax = (kTabMaxP + 2) * (kTabMaxP + 3) * (kTabMaxP + 4) / 6;  // orders 0..P+1: 220
constexpr int kNMMax = (kTabMaxP + 1) * (kTabMaxP + 2) * (kTabMaxP + 3) / 6;  // orders 0..P: 165
constexpr int kTabWarps = 4;

__host__ __device__ constexpr int mi_off(int n) { return n * (n + 1) * (n + 2) / 6; }
__device__ __forceinline__ int mi_idx(int a0, int a1, int a2) {
  const int n = a0 + a1 + a2, s = a1 + a2;
  return mi_off(n) + s * (s + 1) / 2 + a2;
}

// Index tables, built once on the host and copied to each context:
//   expo[i]  = (a0, a1, a2, |a|) of multi-index i (orders 0..kTabMaxP+1)
//   ifact[i] = 1 / a!
//   uoff[g] .. uoff[g+1]: the terms of U^g, each a coefficient and the
//   exponents of n packed as px | py << 8 | pz << 16
//   and per order P (3 .. kTabMaxP) the M2L's work split over a warp's 32
//   lanes: the derivatives U^g and the local coefficients assigned to lanes
//   largest first, each to the least loaded lane (their costs differ by an
//   order of magnitude), and the (a, b) products of the corrective force as
//   one flat list that the lanes stride through.
constexpr int kTabMinP = 3;
constexpr int kTabNP = kTabMaxP - kTabMinP + 1;
struct TabHost {
  std::vector<int4> expo;
  std::vector<double> ifact;
  std::vector<int> uoff;
  std::vector<double> ucoef;
  std::vector<int> uexp;
  std::vector<int> u_lane, l_lane;  // [P - kTabMinP][33]: lane ranges in u_items / l_items
  std::vector<int> u_items, l_items;
  std::vector<int> c_off;            // [P - kTabMinP + 1]: ranges in c_pairs
  std::vector<int2> c_pairs;         // (ia | ib << 16, U index of a + b + e_x | e_y << 8 | e_z << 16)
};

int mi_idx_host(int a0, int a1, int a2) {
  const int n = a0 + a1 + a2, s = a1 + a2;
  return n * (n + 1) * (n + 2) / 6 + s * (s + 1) / 2 + a2;
}

// items 0 .. n-1 with costs w, assigned largest first to the least loaded of
// 32 lanes (ties: lower item, lower lane); per lane in increasing item order
void lane_split(const std::vector<int> &w, std::vector<int> &lane_ranges, std::vector<int> &items) {
  const int n = static_cast<int>(w.size());
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return w[a] > w[b]; });
  std::vector<long long> load(32, 0);
  std::vector<std::vector<int>> per(32);
  for (int i : order) {
    int best = 0;
    for (int l = 1; l < 32; ++l)
      if (load[l] < load[best]) best = l;
    load[best] += w[i];
    per[best].push_back(i);
  }
  for (int l = 0; l < 32; ++l) {
    std::sort(per[l].begin(), per[l].end());
    lane_ranges.push_back(static_cast<int>(items.size()));
    items.insert(items.end(), per[l].begin(), per[l].end());
  }
  lane_ranges.push_back(static_cast<int>(items.size()));
}

double fact(int k) {
  double f = 1.0;
  for (int q = 2; q <= k; ++q) f *= q;
  return f;
}

const TabHost &tables() {
  static TabHost t;
  static std::once_flag once;
  std::call_once(once, [] {
    for (int n = 0; n <= kTabMaxP + 1; ++n)
      for (int a0 = n; a0 >= 0; --a0)
        for (int a1 = n - a0; a1 >= 0; --a1) {
          const int a2 = n - a0 - a1;
          t.expo.push_back(make_int4(a0, a1, a2, n));
          t.ifact.push_back(1.0 / (fact(a0) * fact(a1) * fact(a2)));
        }
    t.uoff.push_back(0);
    for (const int4 &g : t.expo) {
      const int a = g.x, b = g.y, c = g.z, n = g.w;
      for (int i = 0; 2 * i <= a; ++i)
        for (int j = 0; 2 * j <= b; ++j)
          for (int l = 0; 2 * l <= c; ++l) {
            const int m = n - i - j - l;
            double dfm = 1.0;  // (2m - 1)!!
            for (int k = 2 * m - 1; k > 1; k -= 2) dfm *= k;
            const double cm = (m % 2 == 0 ? -1.0 : 1.0) * dfm;
            const double ka = fact(a) / (std::pow(2.0, i) * fact(i) * fact(a - 2 * i));
            const double kb = fact(b) / (std::pow(2.0, j) * fact(j) * fact(b - 2 * j));
            const double kc = fact(c) / (std::pow(2.0, l) * fact(l) * fact(c - 2 * l));
            t.ucoef.push_back(cm * ka * kb * kc);
            t.uexp.push_back((a - 2 * i) | ((b - 2 * j) << 8) | ((c - 2 * l) << 16));
          }
      t.uoff.push_back(static_cast<int>(t.ucoef.size()));
    }
    for (int P = kTabMinP; P <= kTabMaxP; ++P) {
      const int NM = mi_off(P + 1), NU = mi_off(P + 2), NL = NM - 1;
      std::vector<int> wu(NU), wl(NL);
      for (int g = 0; g < NU; ++g) wu[g] = t.uoff[g + 1] - t.uoff[g];
      for (int o = 0; o < NL; ++o) wl[o] = mi_off(P - t.expo[o + 1].w + 1);
      lane_split(wu, t.u_lane, t.u_items);
      lane_split(wl, t.l_lane, t.l_items);
      t.c_off.push_back(static_cast<int>(t.c_pairs.size()));
      for (int ia = 0; ia < NM; ++ia) {
        const int4 a = t.expo[ia];
        const int nb = P - a.w;
        for (int ib = mi_off(nb); ib < mi_off(nb + 1); ++ib) {
          const int4 b = t.expo[ib];
          const int x = a.x + b.x, y = a.y + b.y, z = a.z + b.z;
          t.c_pairs.push_back(make_int2(ia | (ib << 16), mi_idx_host(x + 1, y, z) | (mi_idx_host(x, y + 1, z) << 8) |
                                                             (mi_idx_host(x, y, z + 1) << 16)));
        }
      }
    }
    t.c_off.push_back(static_cast<int>(t.c_pairs.size()));
  });
  return t;
}

struct TabDev {
  const int4 *expo;
  const double *ifact;
  const int *uoff;
  const double *ucoef;
  const int *uexp;
  const int *u_lane, *l_lane, *u_items, *l_items, *c_off;
  const int2 *c_pairs;
};

// the device copy of the tables, in one context-owned buffer
int device_tables(fmm_ctx *c, TabDev *out) {
  const TabHost &t = tables();
  auto up = [](size_t v) { return (v + 255) & ~size_t(255); };
  struct Part {
    const void *src;
    size_t bytes, off;
  };
  Part parts[] = {{t.expo.data(), t.expo.size() * sizeof(int4), 0},
                  {t.ifact.data(), t.ifact.size() * sizeof(double), 0},
                  {t.uoff.data(), t.uoff.size() * sizeof(int), 0},
                  {t.ucoef.data(), t.ucoef.size() * sizeof(double), 0},
                  {t.uexp.data(), t.uexp.size() * sizeof(int), 0},
                  {t.u_lane.data(), t.u_lane.size() * sizeof(int), 0},
                  {t.l_lane.data(), t.l_lane.size() * sizeof(int), 0},
                  {t.u_items.data(), t.u_items.size() * sizeof(int), 0},
                  {t.l_items.data(), t.l_items.size() * sizeof(int), 0},
                  {t.c_off.data(), t.c_off.size() * sizeof(int), 0},
                  {t.c_pairs.data(), t.c_pairs.size() * sizeof(int2), 0}};
  size_t total = 0;
  for (Part &q : parts) {
    q.off = total;
    total += up(q.bytes);
  }
  if (c->gen_tab.cap < total) {
    AMFMM_TRY(ensure_bytes(c, c->gen_tab, total));
    std::vector<char> h(total, 0);
    for (const Part &q : parts) memcpy(h.data() + q.off, q.src, q.bytes);
    // synchronous: the host vector goes out of scope afterwards
    AMFMM_CUDA(c, cudaMemcpy(c->gen_tab.p, h.data(), total, cudaMemcpyHostToDevice));
  }
  const char *base = static_cast<const char *>(c->gen_tab.p);
  out->expo = reinterpret_cast<const int4 *>(base + parts[0].off);
  out->ifact = reinterpret_cast<const double *>(base + parts[1].off);
  out->uoff = reinterpret_cast<const int *>(base + parts[2].off);
  out->ucoef = reinterpret_cast<const double *>(base + parts[3].off);
  out->uexp = reinterpret_cast<const int *>(base + parts[4].off);
  out->u_lane = reinterpret_cast<const int *>(base + parts[5].off);
  out->l_lane = reinterpret_cast<const int *>(base + parts[6].off);
  out->u_items = reinterpret_cast<const int *>(base + parts[7].off);
  out->l_items = reinterpret_cast<const int *>(base + parts[8].off);
  out->c_off = reinterpret_cast<const int *>(base + parts[9].off);
  out->c_pairs = reinterpret_cast<const int2 *>(base + parts[10].off);
  return FMM_OK;
}

// ---------------------------------------------------------------------------
// M2L: one warp per accepted pair
// ---------------------------------------------------------------------------
struct PairSmem {
  double U[kNUMax];
  // scaled moments with the 1/b! of the sums folded in: sA[b] = M_A^b R^-|b| / b!,
  // sB[b] = (-1)^|b| M_B^b R^-|b| / b!
  double sA[kNMMax], sB[kNMMax];
  double pw[3][kTabMaxP + 2];  // powers of the unit vector's components
  double F[3][32];
};

// per-block copy of the multi-index table: exponents packed a0 | a1 << 8 |
// a2 << 16 | |a| << 24 (orders 0 .. kTabMaxP + 1)
__device__ __forceinline__ void load_expo(int *dst, const int4 *__restrict__ expo) {
  for (int i = threadIdx.x; i < kNUMax; i += blockDim.x) {
    const int4 e = expo[i];
    dst[i] = e.x | (e.y << 8) | (e.z << 16) | (e.w << 24);
  }
}
__device__ __forceinline__ int mi_idx_sum(int pa, int pb) {
  // index of the multi-index a + b from the packed exponents of a and b
  const int s = pa + pb;  // no field exceeds 255
  return mi_idx(s & 255, (s >> 8) & 255, (s >> 16) & 255);
}

template <int VARIANT>
__global__ void __launch_bounds__(kTabWarps * 32) k_m2l_tab(int P, int64_t K, const int2 *__restrict__ pairs,
                                                            const double *__restrict__ Z,
                                                            const double *__restrict__ invM,
                                                            const double *__restrict__ mom,
                                                            const int32_t *__restrict__ pos, TabDev tab,
                                                            double *__restrict__ slots) {
  __shared__ PairSmem sm_all[kTabWarps];
  __shared__ int ex[kNUMax];
  __shared__ double ifa[kNUMax];
  load_expo(ex, tab.expo);
  for (int i = threadIdx.x; i < kNUMax; i += blockDim.x) ifa[i] = tab.ifact[i];
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  PairSmem &sm = sm_all[w];
  const int NM = mi_off(P + 1), NL = NM - 1;
  for (int64_t k = blockIdx.x * static_cast<int64_t>(kTabWarps) + w; k < K;
       k += static_cast<int64_t>(gridDim.x) * kTabWarps) {
    const int A = pairs[k].x, B = pairs[k].y;
    double *LA = slots + static_cast<int64_t>(pos[2 * k]) * NL;
    double *LB = slots + static_cast<int64_t>(pos[2 * k + 1]) * NL;
    const double r0 = Z[3 * A] - Z[3 * B], r1 = Z[3 * A + 1] - Z[3 * B + 1], r2 = Z[3 * A + 2] - Z[3 * B + 2];
    const double R2 = r0 * r0 + r1 * r1 + r2 * r2;
    if (!(R2 > 0.0)) {
      for (int q = lane; q < NL; q += 32) LA[q] = LB[q] = 0.0;
      continue;
    }
    const double Ri = rsqrt(R2);
    const double nx = r0 * Ri, ny = r1 * Ri, nz = r2 * Ri;
    double ri[kTabMaxP + 3];
    ri[0] = 1.0;
#pragma unroll
    for (int q = 1; q < kTabMaxP + 3; ++q) ri[q] = ri[q - 1] * Ri;
    if (lane < 3) {
      const double v = lane == 0 ? nx : (lane == 1 ? ny : nz);
      double p = 1.0;
      for (int q = 0; q < kTabMaxP + 2; ++q) {
        sm.pw[lane][q] = p;
        p *= v;
      }
    }
    // moments scaled by R^-|b| and divided by b!
    const double *mA = mom + static_cast<int64_t>(A) * NM, *mB = mom + static_cast<int64_t>(B) * NM;
    for (int i = lane; i < NM; i += 32) {
      const int o = ex[i] >> 24;
      const double f = ri[o] * ifa[i];
      sm.sA[i] = mA[i] * f;
      sm.sB[i] = (o % 2 == 0 ? f : -f) * mB[i];
    }
    __syncwarp();
    // U^g(n) for |g| <= P + 1, each lane its share of the terms
    const int sp = (P - kTabMinP) * 33;
    for (int it = tab.u_lane[sp + lane]; it < tab.u_lane[sp + lane + 1]; ++it) {
      const int g = tab.u_items[it];
      double u = 0.0;
      for (int t = tab.uoff[g]; t < tab.uoff[g + 1]; ++t) {
        const int e = tab.uexp[t];
        u += tab.ucoef[t] * (sm.pw[0][e & 255] * sm.pw[1][(e >> 8) & 255] * sm.pw[2][e >> 16]);
      }
      sm.U[g] = u;
    }
    __syncwarp();
    // corrective force: the lanes stride through the (a, b) products with
    // |a| + |b| = P
    double f0 = 0.0, f1 = 0.0, f2 = 0.0;
    if (VARIANT != FMM_UC) {
      const int c1 = tab.c_off[P - kTabMinP + 1];
      for (int it = tab.c_off[P - kTabMinP] + lane; it < c1; it += 32) {
        const int2 pq = tab.c_pairs[it];
        const double cb = -sm.sA[pq.x & 0xffff] * sm.sB[pq.x >> 16];  // (-1)^|b| / (a! b!) folded in
        f0 += cb * sm.U[pq.y & 255];
        f1 += cb * sm.U[(pq.y >> 8) & 255];
        f2 += cb * sm.U[pq.y >> 16];
      }
      // lane sums in a fixed order
      sm.F[0][lane] = f0;
      sm.F[1][lane] = f1;
      sm.F[2][lane] = f2;
      __syncwarp();
      if (lane < 3) {
        double s = 0.0;
        for (int q = 0; q < 32; ++q) s += sm.F[lane][q];
        sm.F[lane][0] = s;
      }
      __syncwarp();
      f0 = sm.F[0][0] * ri[2];
      f1 = sm.F[1][0] * ri[2];
      f2 = sm.F[2][0] * ri[2];
      if (VARIANT == FMM_TCO) {
        const double nf = nx * f0 + ny * f1 + nz * f2;
        f0 -= nx * nf;
        f1 -= ny * nf;
        f2 -= nz * nf;
      }
    }
    // locals of order 1..P on both sides, each lane its share of the outputs
    for (int it = tab.l_lane[sp + lane]; it < tab.l_lane[sp + lane + 1]; ++it) {
      const int o = tab.l_items[it];
      const int pq = ex[o + 1] & 0xffffff;
      const int nq = ex[o + 1] >> 24;
      double accA = 0.0, accB = 0.0;
      const int top = mi_off(P - nq + 1);
      for (int is = 0; is < top; ++is) {
        const double u = sm.U[mi_idx_sum(pq, ex[is] & 0xffffff)];
        accA += u * sm.sB[is];
        accB += u * sm.sA[is];
      }
      double la = ri[nq + 1] * accA;
      double lb = (nq % 2 == 0 ? 1.0 : -1.0) * ri[nq + 1] * accB;
      if (VARIANT != FMM_UC && o < 3) {
        const double f = o == 0 ? f0 : (o == 1 ? f1 : f2);
        la -= f * invM[A];
        lb += f * invM[B];
      }
      LA[o] = la;
      LB[o] = lb;
    }
    __syncwarp();  // the staged values are written again by the next pair
  }
}

// ---------------------------------------------------------------------------
// P2M (leaves), M2M (one level), L2L (one level), L2P
// ---------------------------------------------------------------------------
// one warp per leaf: centre of mass as at order 3, then lanes over the
// multi-indices, each summing mu x^a over the leaf's bodies in sorted order
__global__ void k_leaf_upward_tab(int P, int32_t nleaf, const int32_t *__restrict__ leaves,
                                  const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
                                  const double *__restrict__ X, const double *__restrict__ Y,
                                  const double *__restrict__ Zb, const double *__restrict__ Mb,
                                  double *__restrict__ S, double *__restrict__ M, double *__restrict__ Z,
                                  double *__restrict__ invM, double *__restrict__ mom, TabDev tab) {
  const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= nleaf) return;
  const int c = leaves[q];
  const int b = begin[c], e = b + count[c];
  double z[3];
  if (lane == 0) leaf_com(c, b, e, X, Y, Zb, Mb, S, M, Z, invM, z);
  z[0] = __shfl_sync(0xffffffffu, z[0], 0);
  z[1] = __shfl_sync(0xffffffffu, z[1], 0);
  z[2] = __shfl_sync(0xffffffffu, z[2], 0);
  const int NM = mi_off(P + 1);
  double *out = mom + static_cast<int64_t>(c) * NM;
  for (int i = lane; i < NM; i += 32) {
    const int4 a = tab.expo[i];
    double acc = 0.0;
    for (int j = b; j < e; ++j) {
      const double x = X[j] - z[0], y = Y[j] - z[1], zz = Zb[j] - z[2];
      double v = Mb[j];
      for (int t = 0; t < a.x; ++t) v *= x;
      for (int t = 0; t < a.y; ++t) v *= y;
      for (int t = 0; t < a.z; ++t) v *= zz;
      acc += v;
    }
    out[i] = acc;
  }
  __syncwarp();
  if (lane == 0) out[0] = M[c];
}

// one warp per cell of a level: centre of mass from the children (as at
// order 3), then lanes over a: M^a = sum over children in order of
// sum_{b <= a} C(a, b) M_child^b s^(a-b); binomials and the powers of each
// child's shift s from shared memory
constexpr int kTabLevelWarps = 4;

__global__ void __launch_bounds__(kTabLevelWarps * 32) k_internal_upward_tab(
    int P, int32_t c0, int32_t c1, const int32_t *__restrict__ first_child, const int32_t *__restrict__ nchild,
    double *__restrict__ S, double *__restrict__ M, double *__restrict__ Z, double *__restrict__ invM,
    double *__restrict__ mom, TabDev tab) {
  __shared__ double binom_t[kTabMaxP + 1][kTabMaxP + 1];
  __shared__ double pw[kTabLevelWarps][3][kTabMaxP + 1];
  __shared__ int ex[kNUMax];
  for (int q = threadIdx.x; q < (kTabMaxP + 1) * (kTabMaxP + 1); q += blockDim.x) {
    const int n = q / (kTabMaxP + 1), k = q % (kTabMaxP + 1);
    double r = 0.0;
    if (k <= n) {
      r = 1.0;
      for (int t = 1; t <= k; ++t) r = r * (n - k + t) / t;
    }
    binom_t[n][k] = r;
  }
  load_expo(ex, tab.expo);
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = c0 + blockIdx.x * kTabLevelWarps + w;
  if (c >= c1) return;
  const int nch = nchild[c];
  if (nch == 0) return;
  const int f = first_child[c];
  double z[3];
  if (lane == 0) parent_com(c, f, nch, S, M, Z, invM, z);
  z[0] = __shfl_sync(0xffffffffu, z[0], 0);
  z[1] = __shfl_sync(0xffffffffu, z[1], 0);
  z[2] = __shfl_sync(0xffffffffu, z[2], 0);
  const int NM = mi_off(P + 1);
  double acc[(kNMMax + 31) / 32];
#pragma unroll
  for (int u = 0; u < (kNMMax + 31) / 32; ++u) acc[u] = 0.0;
  for (int k = f; k < f + nch; ++k) {
    __syncwarp();
    if (lane < 3) {
      const double sv = Z[3 * k + lane] - z[lane];
      double p = 1.0;
      for (int q = 0; q <= kTabMaxP; ++q) {
        pw[w][lane][q] = p;
        p *= sv;
      }
    }
    __syncwarp();
    const double *mc = mom + static_cast<int64_t>(k) * NM;
#pragma unroll
    for (int u = 0; u < (kNMMax + 31) / 32; ++u) {
      const int i = lane + 32 * u;
      if (i >= NM) continue;
      const int e = ex[i];
      const int a0 = e & 255, a1 = (e >> 8) & 255, a2 = (e >> 16) & 255;
      double v = 0.0;
      for (int b0 = 0; b0 <= a0; ++b0) {
        const double f0 = binom_t[a0][b0] * pw[w][0][a0 - b0];
        for (int b1 = 0; b1 <= a1; ++b1) {
          const double f1 = f0 * binom_t[a1][b1] * pw[w][1][a1 - b1];
          for (int b2 = 0; b2 <= a2; ++b2)
            v += f1 * binom_t[a2][b2] * pw[w][2][a2 - b2] * mc[mi_idx(b0, b1, b2)];
        }
      }
      acc[u] += v;
    }
  }
  double *out = mom + static_cast<int64_t>(c) * NM;
#pragma unroll
  for (int u = 0; u < (kNMMax + 31) / 32; ++u) {
    const int i = lane + 32 * u;
    if (i < NM) out[i] = i == 0 ? M[c] : acc[u];
  }
}

// one warp per cell of a level: L^a(cell) += sum_g L^(a+g)(parent) s^g / g!
__global__ void __launch_bounds__(kTabLevelWarps * 32) k_l2l_tab(int P, int32_t c0, int32_t c1,
                                                                 const int32_t *__restrict__ parent,
                                                                 const double *__restrict__ Z,
                                                                 double *__restrict__ loc, TabDev tab) {
  __shared__ double pw[kTabLevelWarps][3][kTabMaxP + 1];
  __shared__ int ex[kNUMax];
  __shared__ double ifa[kNUMax];
  load_expo(ex, tab.expo);
  for (int i = threadIdx.x; i < kNUMax; i += blockDim.x) ifa[i] = tab.ifact[i];
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = c0 + blockIdx.x * kTabLevelWarps + w;
  if (c >= c1) return;
  const int p = parent[c];
  if (lane < 3) {
    const double sv = Z[3 * c + lane] - Z[3 * p + lane];
    double q = 1.0;
    for (int t = 0; t <= kTabMaxP; ++t) {
      pw[w][lane][t] = q;
      q *= sv;
    }
  }
  __syncwarp();
  const int NL = mi_off(P + 1) - 1;
  const double *Lp = loc + static_cast<int64_t>(p) * NL;
  double *Lc = loc + static_cast<int64_t>(c) * NL;
  for (int o = lane; o < NL; o += 32) {
    const int pa = ex[o + 1] & 0xffffff;
    const int na = ex[o + 1] >> 24;
    double acc = 0.0;
    const int top = mi_off(P - na + 1);
    for (int ig = 0; ig < top; ++ig) {
      const int eg = ex[ig];
      const double mono = pw[w][0][eg & 255] * pw[w][1][(eg >> 8) & 255] * pw[w][2][(eg >> 16) & 255];
      acc += Lp[mi_idx_sum(pa, eg & 0xffffff) - 1] * (ifa[ig] * mono);
    }
    Lc[o] += acc;
  }
}

// one thread per body: g_k = -sum_{|a| <= P-1} L^(a+e_k) x^a / a!
__global__ void k_l2p_tab(int P, int64_t n, const int32_t *__restrict__ leaf_of, const double *__restrict__ Z,
                          const double *__restrict__ loc, const double *__restrict__ X,
                          const double *__restrict__ Y, const double *__restrict__ Zb,
                          const double *__restrict__ near, double *__restrict__ acc, TabDev tab) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const int L = leaf_of[i];
  const double x = X[i] - Z[3 * L], y = Y[i] - Z[3 * L + 1], z = Zb[i] - Z[3 * L + 2];
  const int NL = mi_off(P + 1) - 1;
  const double *Lc = loc + static_cast<int64_t>(L) * NL;
  double px[kTabMaxP], py[kTabMaxP], pz[kTabMaxP];
  px[0] = py[0] = pz[0] = 1.0;
#pragma unroll
  for (int q = 1; q < kTabMaxP; ++q) {
    px[q] = px[q - 1] * x;
    py[q] = py[q - 1] * y;
    pz[q] = pz[q - 1] * z;
  }
  double g0 = 0.0, g1 = 0.0, g2 = 0.0;
  for (int ia = 0; ia < mi_off(P); ++ia) {
    const int4 a = tab.expo[ia];
    const double w = tab.ifact[ia] * (px[a.x] * py[a.y] * pz[a.z]);
    g0 += w * Lc[mi_idx(a.x + 1, a.y, a.z) - 1];
    g1 += w * Lc[mi_idx(a.x, a.y + 1, a.z) - 1];
    g2 += w * Lc[mi_idx(a.x, a.y, a.z + 1) - 1];
  }
  acc[i] = near[i] - g0;
  acc[n + i] = near[n + i] - g1;
  acc[2 * n + i] = near[2 * n + i] - g2;
}

}  // namespace

int upward_table(fmm_ctx *c) {
  TabDev tab;
  AMFMM_TRY(device_tables(c, &tab));
  cudaStream_t st = c->stream;
  const int P = c->opts.order_P;
  k_leaf_upward_tab<<<grid_for(c->sz.nleaf * 32, 128), 128, 0, st>>>(
      P, static_cast<int32_t>(c->sz.nleaf), ptr<int32_t>(c->leaves), ptr<int32_t>(c->begin), ptr<int32_t>(c->count),
      ptr<double>(c->X), ptr<double>(c->Y), ptr<double>(c->Zb), ptr<double>(c->Mb), ptr<double>(c->S),
      ptr<double>(c->M), ptr<double>(c->Z), ptr<double>(c->invM), ptr<double>(c->mom), tab);
  AMFMM_TRY(launched(c, "leaf_upward_tab"));
  for (int lev = c->sz.depth - 1; lev >= 0; --lev) {
    const int64_t c0 = c->sz.lvl_off[lev], c1 = c->sz.lvl_off[lev + 1];
    if (c1 <= c0) continue;
    k_internal_upward_tab<<<grid_for(c1 - c0, kTabLevelWarps), kTabLevelWarps * 32, 0, st>>>(
        P, static_cast<int32_t>(c0), static_cast<int32_t>(c1), ptr<int32_t>(c->first_child), ptr<int32_t>(c->nchild),
        ptr<double>(c->S), ptr<double>(c->M), ptr<double>(c->Z), ptr<double>(c->invM), ptr<double>(c->mom), tab);
    AMFMM_TRY(launched(c, "internal_upward_tab"));
  }
  return FMM_OK;
}

int m2l_table(fmm_ctx *c) {
  const int64_t K = c->sz.n_m2l;
  if (K == 0) return FMM_OK;
  TabDev tab;
  AMFMM_TRY(device_tables(c, &tab));
  const int P = c->opts.order_P;
  const unsigned g = static_cast<unsigned>(std::min<int64_t>((K + kTabWarps - 1) / kTabWarps,
                                                             static_cast<int64_t>(c->num_sms) * 16));
  const int2 *pairs = ptr<int2>(c->m2l);
  const double *Z = ptr<double>(c->Z), *iM = ptr<double>(c->invM), *mom = ptr<double>(c->mom);
  const int32_t *pos = ptr<int32_t>(c->m2l_pos);
  double *slots = ptr<double>(c->m2l_slots);
  cudaStream_t st = c->stream;
  switch (c->opts.variant) {
    case FMM_UC: k_m2l_tab<FMM_UC><<<g, kTabWarps * 32, 0, st>>>(P, K, pairs, Z, iM, mom, pos, tab, slots); break;
    case FMM_TC: k_m2l_tab<FMM_TC><<<g, kTabWarps * 32, 0, st>>>(P, K, pairs, Z, iM, mom, pos, tab, slots); break;
    default: k_m2l_tab<FMM_TCO><<<g, kTabWarps * 32, 0, st>>>(P, K, pairs, Z, iM, mom, pos, tab, slots); break;
  }
  return launched(c, "m2l_tab");
}

int downward_table(fmm_ctx *c) {
  TabDev tab;
  AMFMM_TRY(device_tables(c, &tab));
  cudaStream_t st = c->stream;
  const int P = c->opts.order_P;
  const int64_t n = c->sz.n;
  for (int lev = 1; lev <= c->sz.depth; ++lev) {
    const int64_t c0 = c->sz.lvl_off[lev], c1 = c->sz.lvl_off[lev + 1];
    if (c1 <= c0) continue;
    k_l2l_tab<<<grid_for(c1 - c0, kTabLevelWarps), kTabLevelWarps * 32, 0, st>>>(P, static_cast<int32_t>(c0), static_cast<int32_t>(c1),
                                                             ptr<int32_t>(c->parent), ptr<double>(c->Z),
                                                             ptr<double>(c->loc), tab);
    AMFMM_TRY(launched(c, "l2l_tab"));
  }
  k_l2p_tab<<<grid_for(n, 128), 128, 0, st>>>(P, n, ptr<int32_t>(c->leaf_of), ptr<double>(c->Z), ptr<double>(c->loc),
                                              ptr<double>(c->X), ptr<double>(c->Y), ptr<double>(c->Zb),
                                              ptr<double>(c->near), ptr<double>(c->acc), tab);
  return launched(c, "l2p_tab");
}

}  // namespace amfmm
