// p2p.cu -- a8: mutual near-field sums (Sec. 2: "the force contributions from
// any remaining nearby particles are computed directly").
//
// For every leaf pair (A, B) each body pair (i in A, j in B) is evaluated
// once: with d = X_j - X_i and s = 1/|d|^3,
//     a_i += m_j s d,    a_j -= m_i s d,
// so the two contributions are equal and opposite (linear momentum is
// conserved pair by pair).  With Plummer softening, s = 1/(|d|^2 + eps^2)^(3/2).  A leaf with itself sums every ordered pair i != j
// once on the side of i.  A pair at zero separation contributes nothing.
//
// Work layout: one warp per leaf A.  Its columns are A's own bodies (summed
// one-sided, i != j) followed by the bodies of every leaf B paired with A as
// the smaller id (pairs sorted by A, stable), packed 32 columns to a step so
// that small leaves still fill the warp.  Each lane owns one column body j and
// loops over the rows i of A: the B-side sum b_j = sum_i m_i s_ij (X_i - X_j)
// stays in a register and is complete when the loop ends; the A-side term
// -m_j s_ij (X_i - X_j) goes to a per-(row, lane) partial in shared memory,
// summed over the lanes in lane order once per leaf.  b_j is written to the
// slot of (pair, body j); each body then adds its slots in the order of the
// stable sort.  Every sum has a fixed order; no atomics.
//
// FP64 form: absolute coordinates, everything in FP64.  Mixed form:
// coordinates relative to Z_A computed in FP64 and rounded to FP32, pair terms
// and the short sums (over the rows of one leaf, over one lane's columns) in
// FP32, every longer sum (lanes, slots, partners) in FP64.
#include "internal.cuh"

namespace amfmm {
namespace {

constexpr int kWarps = 4;
// Rows of A held in shared memory per pass (the leaf tile): 8, 16 or 32,
// chosen per context (fmm_set_tile, fmm_autotune).  16 measured best in both
// forms on a Plummer sphere of N = 1M: against 32 it halves the shared memory
// per warp and doubles the resident warps (FP32 P2P 1.68 -> 1.10 ms, FP64
// 19.8 -> 18.2 ms); 8 costs more column passes than it gains (1.22 / 18.4
// ms).  Ensembles of small systems may prefer another tile.

// r^-3 from r^2 > 0, the factor of every pair force.
// FP32: the hardware reciprocal square root, cubed.
__device__ __forceinline__ float inv_r3(float r2) {
  const float ri = rsqrtf(r2);
  return ri * ri * ri;
}
// FP64, where the FP64 pipe bounds the kernel: a 24-bit seed y0 ~ r^-1 from
// the FP32 unit, then r^-3 = y0^3 (1 - e)^(-3/2) with e = 1 - r^2 y0^2,
// expanded by the binomial series to 1 + 3/2 e + 15/8 e^2 (|e| < 2^-21, so
// the first omitted term, 35/16 e^3, lies below 2^-60): six FP64 operations
// in all.  The seed comes from r^2 = m 4^k with m in [1, 4): m's leading 23
// bits make an FP32 number, and its reciprocal root scaled by 2^-k goes back
// to FP64 by integer operations on the bit patterns, not by conversions.
// y0 has 24 significant bits, so y0^2 is exact and e carries one rounding.
// Subnormal, infinite or NaN r^2 take the library's reciprocal square root.
__device__ __forceinline__ double inv_r3(double r2) {
  const long long bits = __double_as_longlong(r2);
  const int ex = static_cast<int>(bits >> 52);  // r2 >= 0: the biased exponent
  if (ex == 0 || ex == 0x7ff) {
    const double ri = rsqrt(r2);
    return ri * ri * ri;
  }
  const int E = ex - 1023, k = E >> 1;  // r2 = m 2^(2k), m in [1, 4)
  const unsigned mf = (static_cast<unsigned>(E - 2 * k + 127) << 23) | static_cast<unsigned>((bits >> 29) & 0x7fffff);
  const unsigned yf = __float_as_uint(rsqrtf(__uint_as_float(mf)));  // in (1/2, 1]
  const double y0 = __longlong_as_double((static_cast<long long>(static_cast<int>(yf >> 23) - 127 + 1023 - k) << 52) |
                                         (static_cast<long long>(yf & 0x7fffff) << 29));
  const double y2 = y0 * y0;
  const double e = fma(-r2, y2, 1.0);
  const double y3 = y2 * y0;
  return fma(y3, e * fma(e, 1.875, 1.5), y3);
}

// Shared memory per warp: the rows (bodies of A) and, per row and component,
// one running partial of the A-side sum for every lane.
template <class T, int ROWS>
struct P2PSmem {
  alignas(16) T row[ROWS][4];  // x, y, z, m of the current row chunk (16-byte loads)
  T acc[ROWS * 3][32];         // A-side partial sums, [3 i + d][lane]
};
template <class T, int ROWS>
__device__ __forceinline__ void acc_zero(P2PSmem<T, ROWS> &sm, int nr, int l) {
  for (int v = 0; v < 3 * nr; ++v) sm.acc[v][l] = T(0);
}
// partial of row i, lane l -= s (dx, dy, dz).  (One float4 per (row, lane)
// for the FP32 form, one 16-byte load and store per update, measured 1%
// slower at N = 1M than these three scalar updates.)
template <class T, int ROWS>
__device__ __forceinline__ void acc_sub(P2PSmem<T, ROWS> &sm, int i, int l, T s, T dx, T dy, T dz) {
  sm.acc[3 * i][l] -= s * dx;
  sm.acc[3 * i + 1][l] -= s * dy;
  sm.acc[3 * i + 2][l] -= s * dz;
}
// component v % 3 of row v / 3, lane t
template <class T, int ROWS>
__device__ __forceinline__ T acc_get(const P2PSmem<T, ROWS> &sm, int v, int t) { return sm.acc[v][t]; }

// Coordinates a lane works with: absolute in FP64; relative to Z_A (computed
// in FP64, rounded once) in the mixed form.
// below this squared separation the FP32 form treats two bodies as coincident
// (their 1/r^3 would leave the FP32 range); FP64 only skips r = 0
template <class T>
__device__ __forceinline__ T p2p_min_r2();
template <>
__device__ __forceinline__ float p2p_min_r2<float>() { return 1e-30f; }
// r2 above that bound; FP64 tests r2 != +0 on its bit pattern (r2 is a sum of
// squares, so never negative) to keep the comparison off the FP64 pipe
__device__ __forceinline__ bool p2p_apart(double r2) { return __double_as_longlong(r2) != 0; }
__device__ __forceinline__ bool p2p_apart(float r2) { return r2 > p2p_min_r2<float>(); }

// R consecutive rows i.. against one column body (FP32 form): the B-side sum
// in row order, then the A-side partials.
template <int R, int ROWS>
__device__ __forceinline__ void rows32(P2PSmem<float, ROWS> &sm, int i, int l, bool valid, bool mutual, float xj,
                                       float yj, float zj, float mj, float eps2, float &bx, float &by,
                                       float &bz) {
  float dx[R], dy[R], dz[R], r3[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const float4 rw = *reinterpret_cast<const float4 *>(sm.row[i + u]);
    dx[u] = rw.x - xj;
    dy[u] = rw.y - yj;
    dz[u] = rw.z - zj;
    const float r2 = fmaf(dz[u], dz[u], fmaf(dy[u], dy[u], fmaf(dx[u], dx[u], eps2)));
    const bool ok = valid && r2 > p2p_min_r2<float>();
    const float ri = ok ? rsqrtf(r2) : 0.f;
    r3[u] = ri * ri * ri;
    const float si = rw.w * r3[u];
    bx += si * dx[u];
    by += si * dy[u];
    bz += si * dz[u];
  }
  if (mutual) {
#pragma unroll
    for (int u = 0; u < R; ++u) acc_sub(sm, i + u, l, mj * r3[u], dx[u], dy[u], dz[u]);
  }
}

template <class T>
__device__ __forceinline__ T coord(double v, double z);
template <>
__device__ __forceinline__ double coord<double>(double v, double) { return v; }

// Mixed form: bodies and the leaf centre as hi + lo floats, so an offset
// (x_hi - z_hi) + (x_lo - z_lo) is formed with FP32 operations only (FP64
// costs 64 FP32 operations on this GPU) and keeps FP32 relative accuracy.
struct BodyF {
  float4 h;  // x, y, z hi; mass
  float4 l;  // x, y, z lo
};

__global__ void k_body32(int64_t n, const double *__restrict__ X, const double *__restrict__ Y,
                         const double *__restrict__ Zb, const double *__restrict__ Mb, BodyF *__restrict__ out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const double x = X[i], y = Y[i], z = Zb[i];
  const float hx = static_cast<float>(x), hy = static_cast<float>(y), hz = static_cast<float>(z);
  BodyF b;
  b.h = make_float4(hx, hy, hz, static_cast<float>(Mb[i]));
  b.l = make_float4(static_cast<float>(x - hx), static_cast<float>(y - hy), static_cast<float>(z - hz), 0.f);
  out[i] = b;
}

__device__ __forceinline__ float3 offset32(const BodyF &b, const float4 zh, const float4 zl) {
  return make_float3((b.h.x - zh.x) + (b.l.x - zl.x), (b.h.y - zh.y) + (b.l.y - zl.y),
                     (b.h.z - zh.z) + (b.l.z - zl.z));
}

// A column body as loaded: hi/lo floats in the mixed form, FP64 otherwise.
template <class T>
struct RawBody {
  double x, y, z, m;
};
template <>
struct RawBody<float> {
  BodyF b;
};

template <class T>
__device__ __forceinline__ RawBody<T> load_body(int j, bool valid, const BodyF *__restrict__ bodyf,
                                                const double *__restrict__ X, const double *__restrict__ Y,
                                                const double *__restrict__ Zb, const double *__restrict__ Mb) {
  RawBody<T> r{};
  if (valid) {
    if constexpr (sizeof(T) == sizeof(float)) {
      r.b = bodyf[j];
    } else {
      r.x = X[j];
      r.y = Y[j];
      r.z = Zb[j];
      r.m = Mb[j];
    }
  }
  return r;
}

template <class T, int ROWS>
__global__ void __launch_bounds__(kWarps * 32) k_p2p(
    int32_t nitem, int64_t n, const int4 *__restrict__ items, const int32_t *__restrict__ begin,
    const int32_t *__restrict__ count, const double *__restrict__ Zc, const double *__restrict__ X,
    const double *__restrict__ Y, const double *__restrict__ Zb, const double *__restrict__ Mb,
    const int2 *__restrict__ cols, double *__restrict__ near, double *__restrict__ extra,
    T *__restrict__ slots, const BodyF *__restrict__ bodyf, T eps2, const int32_t *__restrict__ order,
    int *__restrict__ queue) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  P2PSmem<T, ROWS> &sm = reinterpret_cast<P2PSmem<T, ROWS> *>(smem_raw)[w];
  // Work items differ in size by orders of magnitude, so warps draw them
  // from a queue until it is empty instead of taking a fixed one: a block's
  // warps then never wait for one another's items (the grid is as large as
  // fits on the GPU at once).  Which warp takes an item does not change what
  // it computes or where it writes.  order (FP64 form; may be NULL) hands the
  // items out largest first.
  for (;;) {
  int q = 0;
  if (l == 0) q = atomicAdd(queue, 1);
  q = __shfl_sync(0xffffffffu, q, 0);
  if (q >= nitem) break;
  // work item: leaf, column range; w < 0 marks the leaf's first chunk (which
  // owns the near-field sums of the leaf), w >= 0 the offset of a later
  // chunk's A-side partials in `extra`
  const int4 it = items[order ? order[q] : q];
  const int L = it.x;
  const bool first = it.w < 0;
  const int bA = begin[L], nA = count[L];
  const double zx = Zc[3 * L], zy = Zc[3 * L + 1], zz = Zc[3 * L + 2];
  float4 zh = make_float4(0.f, 0.f, 0.f, 0.f), zl = zh;
  if constexpr (sizeof(T) == sizeof(float)) {
    zh = make_float4(static_cast<float>(zx), static_cast<float>(zy), static_cast<float>(zz), 0.f);
    zl = make_float4(static_cast<float>(zx - zh.x), static_cast<float>(zy - zh.y), static_cast<float>(zz - zh.z), 0.f);
  }
  const int cb = it.y, ce = it.z;
  if (first) {
    for (int t = l; t < nA; t += 32) {
      near[bA + t] = 0.0;
      near[n + bA + t] = 0.0;
      near[2 * n + bA + t] = 0.0;
    }
  }
  __syncwarp();
  constexpr int kRows = ROWS;
  for (int r0 = 0; r0 < nA; r0 += kRows) {
    const int nr = min(kRows, nA - r0);
    if (l < nr) {
      const int i = bA + r0 + l;
      if constexpr (sizeof(T) == sizeof(float)) {
        const BodyF b = bodyf[i];
        const float3 o = offset32(b, zh, zl);
        sm.row[l][0] = o.x;
        sm.row[l][1] = o.y;
        sm.row[l][2] = o.z;
        sm.row[l][3] = b.h.w;
      } else {
        sm.row[l][0] = coord<T>(X[i], zx);
        sm.row[l][1] = coord<T>(Y[i], zy);
        sm.row[l][2] = coord<T>(Zb[i], zz);
        sm.row[l][3] = T(Mb[i]);
      }
    }
    acc_zero(sm, nr, l);
    __syncwarp();
    // columns: A's own bodies (one-sided, self) then the bodies of every
    // partner leaf B with A < B, packed 32 to a step.  Loads run ahead: the
    // column entry two steps ahead, the body of the next step.
    int2 colN = cb + l < ce ? cols[cb + l] : make_int2(0, -2);
    RawBody<T> rbN = load_body<T>(colN.x, cb + l < ce, bodyf, X, Y, Zb, Mb);
    int2 colNN = cb + 32 + l < ce ? cols[cb + 32 + l] : make_int2(0, -2);
    for (int c0 = cb; c0 < ce; c0 += 32) {
      const bool valid = c0 + l < ce;
      const int2 col = colN;
      const RawBody<T> rb = rbN;
      colN = colNN;
      rbN = load_body<T>(colN.x, c0 + 32 + l < ce, bodyf, X, Y, Zb, Mb);
      colNN = c0 + 64 + l < ce ? cols[c0 + 64 + l] : make_int2(0, -2);
      T xj = T(0), yj = T(0), zj = T(0), mj = T(0);
      if (valid) {
        if constexpr (sizeof(T) == sizeof(float)) {
          const float3 o = offset32(rb.b, zh, zl);
          xj = o.x;
          yj = o.y;
          zj = o.z;
          mj = rb.b.h.w;
        } else {
          xj = rb.x;
          yj = rb.y;
          zj = rb.z;
          mj = rb.m;
        }
      }
      const bool mutual = col.y >= 0;
      T bx = T(0), by = T(0), bz = T(0);
      // FP32: four rows per step, then two, independent dependency chains
      // for the pipelines and less loop control per pair (FP64 is bound by
      // its pipe and runs faster one row at a time)
      int i = 0;
      if constexpr (sizeof(T) == sizeof(float)) {
        for (; i + 7 < nr; i += 8) rows32<8, ROWS>(sm, i, l, valid, mutual, xj, yj, zj, mj, eps2, bx, by, bz);
        for (; i + 3 < nr; i += 4) rows32<4, ROWS>(sm, i, l, valid, mutual, xj, yj, zj, mj, eps2, bx, by, bz);
        for (; i + 1 < nr; i += 2) rows32<2, ROWS>(sm, i, l, valid, mutual, xj, yj, zj, mj, eps2, bx, by, bz);
      }
      for (; i < nr; ++i) {
        const T dx = sm.row[i][0] - xj, dy = sm.row[i][1] - yj, dz = sm.row[i][2] - zj;
        // softening enters as the addend of the first product (no extra
        // operation; eps2 = 0 gives the unsoftened sum)
        const T r2 = fma(dz, dz, fma(dy, dy, fma(dx, dx, eps2)));
        if (valid && p2p_apart(r2)) {
          const T r3 = inv_r3(r2);
          const T si = sm.row[i][3] * r3;
          bx += si * dx;
          by += si * dy;
          bz += si * dz;
          if (mutual) {
            const T sj = mj * r3;
            acc_sub(sm, i, l, sj, dx, dy, dz);
          }
        }
      }
      if (valid) {
        if (mutual) {
          T *o = slots + 3 * static_cast<int64_t>(col.y);
          if (r0 == 0) {
            o[0] = bx;
            o[1] = by;
            o[2] = bz;
          } else {
            o[0] += bx;
            o[1] += by;
            o[2] += bz;
          }
        } else {
          near[col.x] += static_cast<double>(bx);
          near[n + col.x] += static_cast<double>(by);
          near[2 * n + col.x] += static_cast<double>(bz);
        }
      }
    }
    __syncwarp();
    // A-side: every row's partials summed over the lanes in a fixed order
    // (FP64: sequential; mixed: pairwise in FP32 over the 32 lanes, then one
    // FP64 addition)
    for (int v = l; v < 3 * nr; v += 32) {
      double s = 0.0;
      if constexpr (sizeof(T) == sizeof(float)) {
        float g[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          float a[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) a[t] = acc_get(sm, v, 8 * h + t);
          g[h] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
        }
        s = static_cast<double>((g[0] + g[1]) + (g[2] + g[3]));
      } else {
#pragma unroll 8
        for (int t = 0; t < 32; ++t) s += static_cast<double>(acc_get(sm, v, t));
      }
      if (first) near[static_cast<int64_t>(v % 3) * n + bA + r0 + v / 3] += s;
      else extra[it.w + 3 * (r0 + v / 3) + v % 3] = s;
    }
    __syncwarp();
  }
  }
}

// A leaf whose column stream was split adds the A-side partials of its later
// chunks, in chunk order, once every chunk is done (one thread per body).
__global__ void k_p2p_chunks(int32_t nleaf, int64_t n, const int32_t *__restrict__ leaves,
                             const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
                             const int32_t *__restrict__ itemOff, const int4 *__restrict__ items,
                             const double *__restrict__ extra, double *__restrict__ near) {
  const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int l = threadIdx.x & 31;
  if (q >= nleaf) return;
  const int i0 = itemOff[q], i1 = itemOff[q + 1];
  if (i1 - i0 < 2) return;
  const int L = leaves[q];
  const int bA = begin[L], nA = count[L];
  for (int r = l; r < nA; r += 32) {
    double a0 = near[bA + r], a1 = near[n + bA + r], a2 = near[2 * n + bA + r];
    for (int k = i0 + 1; k < i1; ++k) {
      const double *e = extra + items[k].w + 3 * r;
      a0 += e[0];
      a1 += e[1];
      a2 += e[2];
    }
    near[bA + r] = a0;
    near[n + bA + r] = a1;
    near[2 * n + bA + r] = a2;
  }
}

// Work items: the column stream of a leaf is cut into chunks of at most
// `chunk` columns (the first chunk also holds all of the leaf's own bodies,
// so that the one-sided self sums stay in one warp).  One warp per chunk
// keeps a leaf that the walk paired with millions of bodies (a large sparse
// leaf next to a dense region) from serialising the kernel.  The FP64 form
// takes shorter chunks, whose items it hands out largest first (a short
// tail); the FP32 form keeps longer ones in leaf order, where neighbouring
// warps share partner columns in cache.
constexpr int kChunk64 = 2048;
constexpr int kChunk32 = 4096;

__device__ __forceinline__ int chunks_of(int ncol, int nself, int chunk) {
  const int first = max(chunk, nself);
  return ncol <= first ? 1 : 1 + (ncol - first + chunk - 1) / chunk;
}

__global__ void k_item_counts(int32_t nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ count,
                              const int32_t *__restrict__ colOff, int chunk, int32_t *__restrict__ nitems,
                              int32_t *__restrict__ nextra) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nleaf) return;
  const int L = leaves[q];
  const int k = chunks_of(colOff[L + 1] - colOff[L], count[L], chunk);
  nitems[q] = k;
  nextra[q] = (k - 1) * 3 * count[L];
}

__global__ void k_item_fill(int32_t nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ count,
                            const int32_t *__restrict__ colOff, int chunk, const int32_t *__restrict__ itemOff,
                            const int32_t *__restrict__ extraOff, int4 *__restrict__ items) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nleaf) return;
  const int L = leaves[q];
  const int cb = colOff[L], ce = colOff[L + 1], nA = count[L];
  const int k = chunks_of(ce - cb, nA, chunk);
  const int first = max(chunk, nA);
  int o = itemOff[q];
  items[o] = make_int4(L, cb, min(ce, cb + first), -1);
  for (int j = 1; j < k; ++j) {
    const int c0 = cb + first + (j - 1) * chunk;
    items[o + j] = make_int4(L, c0, min(ce, c0 + chunk), extraOff[q] + (j - 1) * 3 * nA);
  }
}

// Sort keys that hand the FP64 near field's work items out largest first
// (rows x columns, coarsened to 16 bits and complemented; the sort is stable,
// so equal keys keep the item order).  The last items a launch draws are
// then short, and its tail shrinks.
__global__ void k_item_keys(int32_t nitem, const int4 *__restrict__ items, const int32_t *__restrict__ count,
                            uint32_t *__restrict__ key, uint32_t *__restrict__ val) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nitem) return;
  const int4 it = items[q];
  const int64_t cost = static_cast<int64_t>(count[it.x]) * (it.z - it.y);
  const int64_t c8 = cost >> 3;
  key[q] = 0xffffu - static_cast<uint32_t>(c8 < 0xffff ? c8 : 0xffff);
  val[q] = static_cast<uint32_t>(q);
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
  int e = offB[L];
  const int e1 = offB[L + 1];
  if (sizeof(T) == sizeof(float)) {
    // FP32 partials: sums of eight in FP32 (fixed order), accumulated in FP64
    for (; e + 8 <= e1; e += 8) {
      T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const T *p = slots + poff[e + u] + 3 * t;
        s0 += p[0];
        s1 += p[1];
        s2 += p[2];
      }
      a0 += static_cast<double>(s0);
      a1 += static_cast<double>(s1);
      a2 += static_cast<double>(s2);
    }
  }
  for (; e < e1; ++e) {
    const T *p = slots + poff[e] + 3 * t;
    a0 += static_cast<double>(p[0]);
    a1 += static_cast<double>(p[1]);
    a2 += static_cast<double>(p[2]);
  }
  near[i] = a0;
  near[n + i] = a1;
  near[2 * n + i] = a2;
}

// Sort keys of the pairs by one side, the per-cell pair counts, and (if nb is
// given) every pair's column count n_B.
__global__ void k_pair_keys(int64_t K, const int2 *__restrict__ pairs, int side, uint32_t *__restrict__ key,
                            uint32_t *__restrict__ val, int32_t *__restrict__ cnt,
                            const int32_t *__restrict__ count, int32_t *__restrict__ nb) {
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= K) return;
  const int2 p = pairs[k];
  const int c = side == 0 ? p.x : p.y;
  key[k] = static_cast<uint32_t>(c);
  val[k] = static_cast<uint32_t>(k);
  atomicAdd(&cnt[c], 1);
  if (nb) nb[k] = count[p.y];
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

// Columns of every leaf: first its own bodies (marked -1: one-sided), then the
// bodies of its partner leaves in the A-sorted pair order, each with the slot
// that receives its B-side partial.
// Column count of every leaf A: its own bodies plus, from the prefix sums
// pre of the partners' sizes over the A-sorted pairs, the bodies of its
// partners.  Also the near-field work: n_A n_B per leaf pair plus
// n (n - 1) / 2 per leaf (one atomic per warp, integer: exact).
__global__ void k_leaf_cols(int32_t nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ count,
                            const int32_t *__restrict__ offA, const int32_t *__restrict__ pre,
                            int32_t *__restrict__ ccount, unsigned long long *__restrict__ work) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = 0;
  if (q < nleaf) {
    const int L = leaves[q];
    const int a = count[L];
    const int cols = pre ? pre[offA[L + 1]] - pre[offA[L]] : 0;
    ccount[L] = a + cols;
    v = static_cast<unsigned long long>(a) * cols + static_cast<unsigned long long>(a) * (a - 1) / 2;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(work, v);
}

__global__ void k_cols_self(int32_t nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ begin,
                            const int32_t *__restrict__ count, const int32_t *__restrict__ colOff,
                            int2 *__restrict__ cols) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nleaf) return;
  const int L = leaves[q];
  const int b = begin[L], c0 = colOff[L];
  for (int t = 0; t < count[L]; ++t) cols[c0 + t] = make_int2(b + t, -1);
}

__global__ void k_cols_pairs(int64_t K, const int2 *__restrict__ pairs, const int32_t *__restrict__ begin,
                             const int32_t *__restrict__ count, const int32_t *__restrict__ colOff,
                             const int32_t *__restrict__ offA, const int32_t *__restrict__ pre,
                             const int32_t *__restrict__ pos, const int64_t *__restrict__ poff,
                             int2 *__restrict__ cols) {
  // A warp writes the runs of its 32 pairs together: entry j of the warp's
  // concatenated runs goes to lane j mod 32, which finds the pair owning it
  // by a binary search over the warp's prefix sums, so consecutive lanes
  // store consecutive entries of a run.
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int nB = 0, base = 0, bB = 0;
  long long o = 0;
  if (k < K) {
    const int2 p = pairs[k];
    base = colOff[p.x] + count[p.x] + (pre[k] - pre[offA[p.x]]);
    bB = begin[p.y];
    o = poff[pos[k]];
    nB = count[p.y];
  }
  int incl = nB;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  const int excl = incl - nB;
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  for (int j0 = 0; j0 < total; j0 += 32) {
    const int j = j0 + lane;
    int own = 0;  // number of lanes whose run ends at or before j
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int e = __shfl_sync(0xffffffffu, incl, own + step - 1);
      if (e <= j) own += step;
    }
    own = min(own, 31);
    const int b = __shfl_sync(0xffffffffu, base, own), x = __shfl_sync(0xffffffffu, excl, own);
    const int bb = __shfl_sync(0xffffffffu, bB, own);
    const long long oo = __shfl_sync(0xffffffffu, o, own);
    if (j < total) {
      const int t = j - x;
      // the slot's index (its offset / 3): 3x the range of an int32 offset
      cols[b + t] = make_int2(bb + t, static_cast<int32_t>(oo / 3 + t));
    }
  }
}

template <class T, int ROWS>
int launch_p2p_rows(fmm_ctx *c) {
  const int64_t n = c->sz.n;
  const int32_t nleaf = static_cast<int32_t>(c->sz.nleaf);
  const size_t shm = kWarps * sizeof(P2PSmem<T, ROWS>);
  // per function and device, so set on every launch (a host-side call)
  AMFMM_CUDA(c, cudaFuncSetAttribute(k_p2p<T, ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(shm)));
  const int32_t nitem = static_cast<int32_t>(c->sz.p2p_items);
  int per_sm = 0;
  AMFMM_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_p2p<T, ROWS>, kWarps * 32, shm));
  const int64_t resident = static_cast<int64_t>(std::max(1, per_sm)) * std::max(1, c->num_sms);
  const unsigned grid = static_cast<unsigned>(std::min<int64_t>(grid_for(nitem, kWarps), resident));
  int *queue = ptr<int32_t>(c->totals) + 40;
  AMFMM_CUDA(c, cudaMemsetAsync(queue, 0, sizeof(int), c->stream));
  k_p2p<T, ROWS><<<grid, kWarps * 32, shm, c->stream>>>(
      nitem, n, ptr<int4>(c->p2p_items), ptr<int32_t>(c->begin), ptr<int32_t>(c->count),
      ptr<double>(c->Z), ptr<double>(c->X), ptr<double>(c->Y), ptr<double>(c->Zb), ptr<double>(c->Mb),
      ptr<int2>(c->p2p_cols), ptr<double>(c->near), ptr<double>(c->p2p_extra),
      static_cast<T *>(c->p2p_slots.p), sizeof(T) == sizeof(float) ? ptr<BodyF>(c->p2p_bodyf) : nullptr,
      static_cast<T>(c->eps2), c->p2p_order >= 0 ? ptr<int32_t>(c->pval[c->p2p_order]) : nullptr, queue);
  AMFMM_TRY(launched(c, "p2p"));
  if (nitem > nleaf) {
    k_p2p_chunks<<<grid_for(static_cast<int64_t>(nleaf) * 32, 256), 256, 0, c->stream>>>(
        nleaf, n, ptr<int32_t>(c->leaves), ptr<int32_t>(c->begin), ptr<int32_t>(c->count),
        ptr<int32_t>(c->p2p_itemOff), ptr<int4>(c->p2p_items), ptr<double>(c->p2p_extra), ptr<double>(c->near));
    AMFMM_TRY(launched(c, "p2p_chunks"));
  }
  return FMM_OK;
}

template <class T>
int launch_p2p(fmm_ctx *c) {
  switch (c->p2p_rows) {
    case 8: return launch_p2p_rows<T, 8>(c);
    case 32: return launch_p2p_rows<T, 32>(c);
    default: return launch_p2p_rows<T, 16>(c);
  }
}

template <class T>
int launch_p2p_reduce(fmm_ctx *c) {
  const int64_t n = c->sz.n;
  k_p2p_reduce<T><<<grid_for(n, 256), 256, 0, c->stream>>>(n, ptr<int32_t>(c->leaf_of), ptr<int32_t>(c->begin),
                                                           ptr<int32_t>(c->p2p_offB), ptr<int64_t>(c->p2p_poff),
                                                           static_cast<T *>(c->p2p_slots.p), ptr<double>(c->near));
  return launched(c, "p2p_reduce");
}

}  // namespace

int p2p_prepare(fmm_ctx *c) {
  cudaStream_t st = c->stream;
  const int64_t K = c->sz.n_p2p, nc = c->sz.ncell, n = c->sz.n;
  const int32_t nleaf = static_cast<int32_t>(c->sz.nleaf);
  const bool fp32 = c->opts.precision == FMM_MIXED;
  AMFMM_TRY(ensure<double>(c, c->near, 3 * n));
  AMFMM_TRY(ensure<int32_t>(c, c->p2p_offA, nc + 1));
  AMFMM_TRY(ensure<int32_t>(c, c->p2p_offB, nc + 1));
  AMFMM_TRY(ensure<int32_t>(c, c->p2p_colOff, nc + 1));
  AMFMM_TRY(ensure<int64_t>(c, c->p2p_poff, K + 1));
  AMFMM_TRY(ensure<int32_t>(c, c->p2p_pos, K + 1));
  AMFMM_TRY(ensure<int2>(c, c->p2p_A, K + 1));
  AMFMM_TRY(ensure<int32_t>(c, c->incl, std::max<int64_t>(nc + 1, n + 1)));
  int32_t *cnt = ptr<int32_t>(c->incl);
  int32_t *offA = ptr<int32_t>(c->p2p_offA), *offB = ptr<int32_t>(c->p2p_offB);
  int32_t *colOff = ptr<int32_t>(c->p2p_colOff);
  unsigned long long *stat = ptr<unsigned long long>(c->totals) + 8;
  int32_t *ctot = ptr<int32_t>(c->totals) + 32;
  AMFMM_CUDA(c, cudaMemsetAsync(stat, 0, sizeof(unsigned long long), st));
  if (fp32) {
    AMFMM_TRY(ensure<BodyF>(c, c->p2p_bodyf, n));
    k_body32<<<grid_for(n, 256), 256, 0, st>>>(n, ptr<double>(c->X), ptr<double>(c->Y), ptr<double>(c->Zb),
                                               ptr<double>(c->Mb), ptr<BodyF>(c->p2p_bodyf));
    AMFMM_TRY(launched(c, "p2p_body32"));
  }
  AMFMM_TRY(ensure<int32_t>(c, c->p2p_nb, K + 1));
  AMFMM_TRY(ensure<int32_t>(c, c->p2p_pre, K + 1));
  int32_t *nb = ptr<int32_t>(c->p2p_nb), *pre = ptr<int32_t>(c->p2p_pre);
  int64_t *h = static_cast<int64_t *>(c->hpin);
  h[0] = 0;
  if (K > 0) {
    AMFMM_TRY(ensure<uint32_t>(c, c->pkey[0], K));
    AMFMM_TRY(ensure<uint32_t>(c, c->pval[0], K));
    // group by A (stable)
    AMFMM_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nc + 1), st));
    k_pair_keys<<<grid_for(K, 256), 256, 0, st>>>(K, ptr<int2>(c->p2p), 0, ptr<uint32_t>(c->pkey[0]),
                                                  ptr<uint32_t>(c->pval[0]), cnt, nullptr, nullptr);
    AMFMM_TRY(launched(c, "p2p_keysA"));
    AMFMM_TRY(exclusive_scan_i32(c, cnt, offA, nc + 1, nullptr));
    int which = 0;
    AMFMM_TRY(radix_sort_u32(c, c->pkey, c->pval, K, bits_for(nc), &which));
    k_gather_pairs<<<grid_for(K, 256), 256, 0, st>>>(K, ptr<int2>(c->p2p), ptr<uint32_t>(c->pval[which]),
                                                     ptr<int2>(c->p2p_A));
    AMFMM_TRY(launched(c, "p2p_gather"));
    // CSR on the B side; column counts n_B in A-sorted order
    AMFMM_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nc + 1), st));
    k_pair_keys<<<grid_for(K, 256), 256, 0, st>>>(K, ptr<int2>(c->p2p_A), 1, ptr<uint32_t>(c->pkey[0]),
                                                  ptr<uint32_t>(c->pval[0]), cnt, ptr<int32_t>(c->count), nb);
    AMFMM_TRY(launched(c, "p2p_keysB"));
    AMFMM_TRY(exclusive_scan_i32(c, cnt, offB, nc + 1, nullptr));
    AMFMM_TRY(radix_sort_u32(c, c->pkey, c->pval, K, bits_for(nc), &which));
    // B-side slot offsets: 3 n_B doubles per pair, in B-CSR order
    AMFMM_TRY(ensure<int64_t>(c, c->p2p_len, K + 1));
    int64_t *len = ptr<int64_t>(c->p2p_len);
    k_b_positions<<<grid_for(K, 256), 256, 0, st>>>(K, ptr<uint32_t>(c->pval[which]), ptr<int2>(c->p2p_A),
                                                    ptr<int32_t>(c->count), ptr<int32_t>(c->p2p_pos), len);
    AMFMM_TRY(launched(c, "p2p_bpos"));
    int64_t *ptot = ptr<int64_t>(c->totals) + 12;
    AMFMM_TRY(exclusive_scan_i64(c, len, ptr<int64_t>(c->p2p_poff), K, ptot));
  }
  // column stream per leaf: pre = prefix sums of n_B over the A-sorted pairs
  // (K + 1 entries, so pre[K] is the total)
  if (K > 0) {
    AMFMM_CUDA(c, cudaMemsetAsync(nb + K, 0, sizeof(int32_t), st));
    AMFMM_TRY(exclusive_scan_i32(c, nb, pre, K + 1, nullptr));
  }
  AMFMM_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nc + 1), st));
  k_leaf_cols<<<grid_for(nleaf, 256), 256, 0, st>>>(nleaf, ptr<int32_t>(c->leaves), ptr<int32_t>(c->count), offA,
                                                    K > 0 ? pre : nullptr, cnt, stat);
  AMFMM_TRY(launched(c, "p2p_leaf_cols"));
  AMFMM_TRY(exclusive_scan_i32(c, cnt, colOff, nc + 1, ctot));
  // work items: chunks of the column streams
  AMFMM_TRY(ensure<int32_t>(c, c->p2p_itemOff, nleaf + 1));
  AMFMM_TRY(ensure<int32_t>(c, c->p2p_extraOff, nleaf + 1));
  int32_t *itemOff = ptr<int32_t>(c->p2p_itemOff), *extraOff = ptr<int32_t>(c->p2p_extraOff);
  // totals: [32] columns, [33] work items, [34] extra partials (int32 slots)
  int32_t *itot = ptr<int32_t>(c->totals) + 33, *etot = ptr<int32_t>(c->totals) + 34;
  int32_t *icnt = cnt, *ecnt = ptr<int32_t>(c->flag);  // free scratch of >= nleaf + 1
  AMFMM_CUDA(c, cudaMemsetAsync(icnt + nleaf, 0, sizeof(int32_t), st));
  AMFMM_CUDA(c, cudaMemsetAsync(ecnt + nleaf, 0, sizeof(int32_t), st));
  const int chunk = fp32 ? kChunk32 : kChunk64;
  k_item_counts<<<grid_for(nleaf, 256), 256, 0, st>>>(nleaf, ptr<int32_t>(c->leaves), ptr<int32_t>(c->count),
                                                      colOff, chunk, icnt, ecnt);
  AMFMM_TRY(launched(c, "p2p_item_counts"));
  AMFMM_TRY(exclusive_scan_i32(c, icnt, itemOff, nleaf + 1, itot));
  AMFMM_TRY(exclusive_scan_i32(c, ecnt, extraOff, nleaf + 1, etot));
  int32_t *hc = reinterpret_cast<int32_t *>(h + 1);
  {
    // (totals[12], the slot total, is not written after its scan)
    const int64_t *ptot = ptr<int64_t>(c->totals) + 12;
    HostRead rb[2];
    int nr = 0;
    if (K > 0) rb[nr++] = HostRead{h, ptot, sizeof(int64_t)};
    rb[nr++] = HostRead{hc, ctot, 3 * sizeof(int32_t)};
    AMFMM_TRY(read_back(c, rb, nr));
    if (capturing(c)) {
      Expect e;
      if (K > 0) e.add64(ptot, static_cast<uint64_t>(h[0]));
      for (int k = 0; k < 3; ++k) e.add(ctot + k, static_cast<uint32_t>(hc[k]));
      AMFMM_TRY(graph_expect(c, e));
      st = c->stream;
    }
  }
  const int64_t nslot = h[0], ncol = hc[0];
  const int64_t nitem = hc[1], nextra = hc[2];
  // the columns (one per body of A and per slot: n + nslot / 3) are counted
  // by int32 scans and a slot is named by its int32 index: refuse before
  // anything is sized or launched from these totals
  if (nslot / 3 + n + 1 > 0x7fffffffLL)
    return set_error(c, FMM_EUNSUPPORTED, "too many near-field slots (%lld values)", (long long)nslot);
  c->sz.p2p_items = nitem;
  AMFMM_TRY(ensure<int4>(c, c->p2p_items, nitem + 1));
  AMFMM_TRY(ensure<double>(c, c->p2p_extra, nextra + 1));
  k_item_fill<<<grid_for(nleaf, 256), 256, 0, st>>>(nleaf, ptr<int32_t>(c->leaves), ptr<int32_t>(c->count), colOff,
                                                    chunk, itemOff, extraOff, ptr<int4>(c->p2p_items));
  AMFMM_TRY(launched(c, "p2p_item_fill"));
  // FP64: the items largest first (the pair sort's buffers are free here).
  // (In the FP32 form the leaf order's cache sharing is worth more than a
  // shorter tail.)
  c->p2p_order = -1;
  if (!fp32 && nitem > 1) {
    AMFMM_TRY(ensure<uint32_t>(c, c->pkey[0], nitem));
    AMFMM_TRY(ensure<uint32_t>(c, c->pval[0], nitem));
    k_item_keys<<<grid_for(nitem, 256), 256, 0, st>>>(static_cast<int32_t>(nitem), ptr<int4>(c->p2p_items),
                                                      ptr<int32_t>(c->count), ptr<uint32_t>(c->pkey[0]),
                                                      ptr<uint32_t>(c->pval[0]));
    AMFMM_TRY(launched(c, "p2p_item_keys"));
    int which = 0;
    AMFMM_TRY(radix_sort_u32(c, c->pkey, c->pval, nitem, 16, &which));
    c->p2p_order = which;
  }
  AMFMM_TRY(ensure_bytes(c, c->p2p_slots, static_cast<size_t>(nslot + 3) * (fp32 ? sizeof(float) : sizeof(double))));
  AMFMM_TRY(ensure<int2>(c, c->p2p_cols, ncol + 1));
  k_cols_self<<<grid_for(nleaf, 256), 256, 0, st>>>(nleaf, ptr<int32_t>(c->leaves), ptr<int32_t>(c->begin),
                                                    ptr<int32_t>(c->count), colOff, ptr<int2>(c->p2p_cols));
  AMFMM_TRY(launched(c, "p2p_cols_self"));
  if (K > 0) {
    k_cols_pairs<<<grid_for(K, 256), 256, 0, st>>>(K, ptr<int2>(c->p2p_A), ptr<int32_t>(c->begin),
                                                   ptr<int32_t>(c->count), colOff, offA, pre,
                                                   ptr<int32_t>(c->p2p_pos), ptr<int64_t>(c->p2p_poff),
                                                   ptr<int2>(c->p2p_cols));
    AMFMM_TRY(launched(c, "p2p_cols_pairs"));
  }
  return FMM_OK;
}

int p2p_run(fmm_ctx *c) {
  if (c->opts.precision == FMM_MIXED) return launch_p2p<float>(c);
  return launch_p2p<double>(c);
}

int p2p_reduce(fmm_ctx *c) {
  if (c->sz.n_p2p == 0) return FMM_OK;
  if (c->opts.precision == FMM_MIXED) return launch_p2p_reduce<float>(c);
  return launch_p2p_reduce<double>(c);
}

}  // namespace amfmm
