// tree.cu -- a1-a4: bounding cube, Morton keys, sort, octree, centres of mass,
// R_max and moments.
//
// Sec. 2 of the paper: the bodies are decomposed into an oct-tree whose cells
// hold at most n_crit bodies; the opening criterion uses each cell's centre
// of mass Z and R_max, the largest distance from one of its bodies to Z.
// Because the interaction lists depend on exact comparisons of Z and R_max,
// every operation on that path is an explicitly rounded FP64 operation in a
// fixed order (no FMA contraction): leaf sums run over the bodies in sorted
// order, other cells sum their children in octant order, Z = S / M, and R_max
// is the exact maximum over the cell's bodies.
#include "internal.cuh"
#include "geom.cuh"

namespace amfmm {
namespace {

constexpr int kBlock = 256;

// ---------------------------------------------------------------------------
// a1: bounding cube and keys
// ---------------------------------------------------------------------------
__global__ void k_bbox_partial(const double *__restrict__ x, const double *__restrict__ y,
                               const double *__restrict__ z, const double *__restrict__ m,
                               int64_t n, double *__restrict__ part, int *__restrict__ status) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double p[3] = {x[i], y[i], z[i]};
    const double mi = m[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      bad |= !isfinite(p[d]);
      lo[d] = fmin(lo[d], p[d]);
      hi[d] = fmax(hi[d], p[d]);
    }
    bad |= !(mi > 0.0) || !isfinite(mi);
  }
  if (bad) atomicOr(status, 1);
  __shared__ double sh[6][kBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
    if (lane == 0) {
      sh[d][w] = lo[d];
      sh[3 + d][w] = hi[d];
    }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int k = threadIdx.x;
    double v = sh[k][0];
    for (int q = 1; q < kBlock / 32; ++q) v = k < 3 ? fmin(v, sh[k][q]) : fmax(v, sh[k][q]);
    part[blockIdx.x * 6 + k] = v;
  }
}

// bbox[0..2] = lo, bbox[3] = scale = 2^21 / ext (0 when ext == 0).  One block;
// min and max are exact, so the order of combination does not matter.
__global__ void k_bbox_final(const double *__restrict__ part, int nb, double *__restrict__ bbox) {
  __shared__ double sh[6][kBlock / 32];
  double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    for (int k = 0; k < 6; ++k) v[k] = k < 3 ? fmin(v[k], part[b * 6 + k]) : fmax(v[k], part[b * 6 + k]);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < 6; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      const double u = __shfl_xor_sync(0xffffffffu, v[k], o);
      v[k] = k < 3 ? fmin(v[k], u) : fmax(v[k], u);
    }
    if (lane == 0) sh[k][w] = v[k];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    lo[d] = sh[d][0];
    hi[d] = sh[3 + d][0];
    for (int q = 1; q < kBlock / 32; ++q) {
      lo[d] = fmin(lo[d], sh[d][q]);
      hi[d] = fmax(hi[d], sh[3 + d][q]);
    }
  }
  double ext = __dsub_rn(hi[0], lo[0]);
  ext = fmax(ext, __dsub_rn(hi[1], lo[1]));
  ext = fmax(ext, __dsub_rn(hi[2], lo[2]));
  for (int d = 0; d < 3; ++d) bbox[d] = lo[d];
  bbox[3] = ext > 0.0 ? __ddiv_rn(2097152.0, ext) : 0.0;
}

__device__ __forceinline__ uint64_t quantise(double v, double lo, double scale) {
  double t = __dmul_rn(__dsub_rn(v, lo), scale);
  double f = floor(t);
  f = fmin(f, 2097151.0);
  return static_cast<uint64_t>(f);
}

// bit b of q -> bit 3b
__device__ __forceinline__ uint64_t spread3(uint64_t q) {
  q &= 0x1fffffull;
  q = (q | (q << 32)) & 0x1f00000000ffffull;
  q = (q | (q << 16)) & 0x1f0000ff0000ffull;
  q = (q | (q << 8)) & 0x100f00f00f00f00full;
  q = (q | (q << 4)) & 0x10c30c30c30c30c3ull;
  q = (q | (q << 2)) & 0x1249249249249249ull;
  return q;
}

__global__ void k_keys(const double *__restrict__ x, const double *__restrict__ y,
                       const double *__restrict__ z, int64_t n, const double *__restrict__ bbox,
                       uint64_t *__restrict__ key, uint32_t *__restrict__ idx) {
  int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const double s = bbox[3];
  uint64_t qx = quantise(x[i], bbox[0], s), qy = quantise(y[i], bbox[1], s),
           qz = quantise(z[i], bbox[2], s);
  key[i] = spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
  idx[i] = static_cast<uint32_t>(i);
}

// ---------------------------------------------------------------------------
// a13: a forest of independent systems (concatenated, system s owns caller
// indices [off[s], off[s+1])).  Every system gets its own bounding cube and
// keys; a second stable sort pass groups the bodies by system, so each
// system's bodies stay in key order and every root covers one system.
// ---------------------------------------------------------------------------
// one block per system: its cube (lo, scale), the system id of its bodies and
// the bad-data flag
__global__ void k_bbox_sys(const double *__restrict__ x, const double *__restrict__ y,
                           const double *__restrict__ z, const double *__restrict__ m,
                           const int64_t *__restrict__ off, double *__restrict__ sbox,
                           int32_t *__restrict__ sysid, int *__restrict__ status) {
  const int s = blockIdx.x;
  const int64_t b = off[s], e = off[s + 1];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
    const double p[3] = {x[i], y[i], z[i]};
    const double mi = m[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      bad |= !isfinite(p[d]);
      lo[d] = fmin(lo[d], p[d]);
      hi[d] = fmax(hi[d], p[d]);
    }
    bad |= !(mi > 0.0) || !isfinite(mi);
    sysid[i] = s;
  }
  if (bad) atomicOr(status, 1);
  __shared__ double sh[6][kBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
    if (lane == 0) {
      sh[d][w] = lo[d];
      sh[3 + d][w] = hi[d];
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int d = 0; d < 3; ++d)
    for (int q = 1; q < kBlock / 32; ++q) {
      sh[d][0] = fmin(sh[d][0], sh[d][q]);
      sh[3 + d][0] = fmax(sh[3 + d][0], sh[3 + d][q]);
    }
  double ext = __dsub_rn(sh[3][0], sh[0][0]);
  ext = fmax(ext, __dsub_rn(sh[4][0], sh[1][0]));
  ext = fmax(ext, __dsub_rn(sh[5][0], sh[2][0]));
  for (int d = 0; d < 3; ++d) sbox[4 * s + d] = sh[d][0];
  sbox[4 * s + 3] = ext > 0.0 ? __ddiv_rn(2097152.0, ext) : 0.0;
}

__global__ void k_keys_sys(const double *__restrict__ x, const double *__restrict__ y,
                           const double *__restrict__ z, int64_t n, const double *__restrict__ sbox,
                           const int32_t *__restrict__ sysid, uint64_t *__restrict__ key,
                           uint32_t *__restrict__ idx) {
  int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const double *b = sbox + 4 * sysid[i];
  uint64_t qx = quantise(x[i], b[0], b[3]), qy = quantise(y[i], b[1], b[3]), qz = quantise(z[i], b[2], b[3]);
  key[i] = spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
  idx[i] = static_cast<uint32_t>(i);
}

// second pass: (system of the body at sorted position s, s)
__global__ void k_sys_keys(int64_t n, const uint32_t *__restrict__ idx, const int32_t *__restrict__ sysid,
                           uint32_t *__restrict__ skey, uint32_t *__restrict__ sval) {
  int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (s >= n) return;
  skey[s] = static_cast<uint32_t>(sysid[idx[s]]);
  sval[s] = static_cast<uint32_t>(s);
}

__global__ void k_gather_sorted(int64_t n, const uint32_t *__restrict__ perm, const uint64_t *__restrict__ k1,
                                const uint32_t *__restrict__ i1, uint64_t *__restrict__ k2,
                                uint32_t *__restrict__ i2) {
  int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n) return;
  k2[t] = k1[perm[t]];
  i2[t] = i1[perm[t]];
}

// level 0: one root per system
__global__ void k_roots(int32_t nsys, const int64_t *__restrict__ off, int32_t *__restrict__ begin,
                        int32_t *__restrict__ count, int32_t *__restrict__ level, int32_t *__restrict__ parent,
                        int32_t *__restrict__ first_child, int32_t *__restrict__ nchild, int32_t *__restrict__ lvl,
                        int *__restrict__ ovf) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) {
    lvl[0] = 0;
    lvl[1] = nsys;
    *ovf = 0;
  }
  if (s >= nsys) return;
  begin[s] = static_cast<int32_t>(off[s]);
  count[s] = static_cast<int32_t>(off[s + 1] - off[s]);
  level[s] = 0;
  parent[s] = -1;
  first_child[s] = -1;
  nchild[s] = 0;
}

// Gather the bodies into key order; lcp[s] = octal digits shared by keys s-1, s.
__global__ void k_permute(const double *__restrict__ x, const double *__restrict__ y,
                          const double *__restrict__ z, const double *__restrict__ m,
                          const uint64_t *__restrict__ key, const uint32_t *__restrict__ idx,
                          int64_t n, double *__restrict__ X, double *__restrict__ Y,
                          double *__restrict__ Zb, double *__restrict__ Mb,
                          int32_t *__restrict__ order, int32_t *__restrict__ lcp,
                          int32_t *__restrict__ cur, const int32_t *__restrict__ sysid) {
  int64_t s = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (s >= n) return;
  const uint32_t o = idx[s];
  X[s] = x[o];
  Y[s] = y[o];
  Zb[s] = z[o];
  Mb[s] = m[o];
  order[s] = static_cast<int32_t>(o);
  int l = 0;
  if (s > 0) {
    uint64_t d = key[s - 1] ^ key[s];
    l = d == 0 ? kMaxLevel : (__clzll(static_cast<long long>(d)) - 1) / 3;
  }
  lcp[s] = l;
  cur[s] = sysid ? sysid[o] : 0;  // root of the body's system
}

// ---------------------------------------------------------------------------
// a3: octree, one level per pass
// ---------------------------------------------------------------------------
// A body starts a child cell at level lev+1 when its cell at level lev is split
// and it is the cell's first body or its key differs from its predecessor's
// in digit lev+1.
// The level kernels read the level's first new cell id from lvl[lev + 1]
// (device-resident, so that several levels are enqueued before the host
// looks) and do nothing once a level has run out of cell capacity (*ovf).
// From the second level on it first moves every body to its cell of this
// level: -1 for a body of a leaf of the previous level (retired), else the
// child of its previous cell that starts at the last flagged body at or
// before it (same cell), from that level's flags and their exclusive sums.
__global__ void k_level_flags(int64_t n, int lev, int n_crit, const int32_t *__restrict__ lcp,
                              const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
                              int32_t *__restrict__ cur, int32_t *__restrict__ flag,
                              const int32_t *__restrict__ excl, const int32_t *__restrict__ lvl,
                              int32_t *__restrict__ cell_at_lev, int32_t *__restrict__ leaf_of,
                              const int *__restrict__ ovf) {
  int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n || *ovf) return;
  int c = cur[i];
  if (lev > 0 && c >= 0) {
    c = count[c] <= n_crit ? -1 : lvl[lev] + excl[i] + flag[i] - 1;
    cur[i] = c;
  }
  cell_at_lev[i] = c;
  int f = 0;
  if (c >= 0) {
    const bool leaf = count[c] <= n_crit || lev == kMaxLevel;
    if (leaf) leaf_of[i] = c;
    else f = (i == begin[c]) || (lcp[i] == lev);
  }
  flag[i] = f;
}

// Also closes the level: lvl[lev + 2] = lvl[lev + 1] + (new cells).
__global__ void k_make_cells(int64_t n, int lev, int32_t *__restrict__ lvl, const int32_t *__restrict__ ntot,
                             int64_t cap, const int32_t *__restrict__ flag, const int32_t *__restrict__ excl,
                             const int32_t *__restrict__ cur, int32_t *__restrict__ begin,
                             int32_t *__restrict__ level, int32_t *__restrict__ parent,
                             int32_t *__restrict__ first_child, int32_t *__restrict__ nchild, int *__restrict__ ovf) {
  int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int off = lvl[lev + 1];
  if (i == 0) {
    lvl[lev + 2] = off + *ntot;
    if (static_cast<int64_t>(off) + *ntot > cap) atomicOr(ovf, 1);
  }
  if (i >= n || !flag[i] || *ovf) return;
  const int c = cur[i];
  const int id = off + excl[i];
  if (id >= cap) return;  // flagged above; the tree is built again with more room
  begin[id] = static_cast<int32_t>(i);
  level[id] = lev + 1;
  parent[id] = c;
  first_child[id] = -1;
  nchild[id] = 0;
  if (i == begin[c]) first_child[c] = id;
}

__global__ void k_cell_counts(int lev, const int32_t *__restrict__ lvl, int32_t *__restrict__ begin,
                              int32_t *__restrict__ count, const int32_t *__restrict__ parent,
                              int32_t *__restrict__ nchild, const int *__restrict__ ovf) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int off = lvl[lev + 1], nnew = lvl[lev + 2] - off;
  if (k >= nnew || *ovf) return;
  const int id = off + k;
  const int p = parent[id];
  int end = begin[p] + count[p];
  if (k + 1 < nnew) end = min(end, begin[id + 1]);
  count[id] = end - begin[id];
  atomicAdd(&nchild[p], 1);
}

__global__ void k_leaf_flags(int32_t ncell, const int32_t *__restrict__ nchild, int32_t *__restrict__ f) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncell) f[c] = nchild[c] == 0;
}
__global__ void k_leaf_compact(int32_t ncell, const int32_t *__restrict__ nchild,
                               const int32_t *__restrict__ excl, int32_t *__restrict__ leaves) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncell && nchild[c] == 0) leaves[excl[c]] = c;
}

// ---------------------------------------------------------------------------
// a4: centres of mass, moments, R_max
// ---------------------------------------------------------------------------
// Moments about Z in the order M, x, y, z, xx, xy, xz, yy, yz, zz, xxx, xxy,
// xxz, xyy, xyz, xzz, yyy, yyz, yzz, zzz.
__device__ __forceinline__ void add_body_moments(double *mo, double mu, double x, double y, double z) {
  const double mx = mu * x, my = mu * y, mz = mu * z;
  mo[0] += mu;
  mo[1] += mx;
  mo[2] += my;
  mo[3] += mz;
  const double mxx = mx * x, mxy = mx * y, mxz = mx * z, myy = my * y, myz = my * z, mzz = mz * z;
  mo[4] += mxx;
  mo[5] += mxy;
  mo[6] += mxz;
  mo[7] += myy;
  mo[8] += myz;
  mo[9] += mzz;
  mo[10] += mxx * x;
  mo[11] += mxx * y;
  mo[12] += mxx * z;
  mo[13] += myy * x;
  mo[14] += mxy * z;
  mo[15] += mzz * x;
  mo[16] += myy * y;
  mo[17] += myy * z;
  mo[18] += mzz * y;
  mo[19] += mzz * z;
}

__global__ void k_leaf_upward(int32_t nleaf, const int32_t *__restrict__ leaves,
                              const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
                              const double *__restrict__ X, const double *__restrict__ Y,
                              const double *__restrict__ Zb, const double *__restrict__ Mb,
                              double *__restrict__ S, double *__restrict__ M, double *__restrict__ Z,
                              double *__restrict__ invM, double *__restrict__ mom) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nleaf) return;
  const int c = leaves[q];
  const int b = begin[c], e = b + count[c];
  double zc[3];
  leaf_com(c, b, e, X, Y, Zb, Mb, S, M, Z, invM, zc);
  const double zx = zc[0], zy = zc[1], zz = zc[2], mm = M[c];
  double mo[kMomStride];
#pragma unroll
  for (int k = 0; k < kMomStride; ++k) mo[k] = 0.0;
  for (int i = b; i < e; ++i) add_body_moments(mo, Mb[i], X[i] - zx, Y[i] - zy, Zb[i] - zz);
  mo[0] = mm;
  double *out = mom + static_cast<int64_t>(c) * kMomStride;
#pragma unroll
  for (int k = 0; k < kMomStride; ++k) out[k] = mo[k];
}

// One level of internal cells: S, M from the children in octant order, then
// the moments shifted from each child centre to Z (M2M, exact algebra for the
// raw moments Sum mu x^a): with s = Z_child - Z,
//   Q_ij  += Q_ij' + M' s_i s_j
//   O_ijk += O_ijk' + (Q_ij' s_k + Q_ik' s_j + Q_jk' s_i) + M' s_i s_j s_k
// The child dipoles D' (zero about a centre of mass up to rounding, Sec. 2)
// are left out of the shift; the parent's dipole is the shift of the child
// monopoles, D_i = Sum M' s_i.
__global__ void k_internal_upward(int32_t c0, int32_t c1, const int32_t *__restrict__ first_child,
                                  const int32_t *__restrict__ nchild, double *__restrict__ S,
                                  double *__restrict__ M, double *__restrict__ Z,
                                  double *__restrict__ invM, double *__restrict__ mom) {
  const int c = c0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= c1) return;
  const int nch = nchild[c];
  if (nch == 0) return;
  const int f = first_child[c];
  double zc[3];
  parent_com(c, f, nch, S, M, Z, invM, zc);
  const double zx = zc[0], zy = zc[1], zz = zc[2], mm = M[c];
  double p[kMomStride];
#pragma unroll
  for (int k = 0; k < kMomStride; ++k) p[k] = 0.0;
  for (int k = f; k < f + nch; ++k) {
    const double *q = mom + static_cast<int64_t>(k) * kMomStride;
    const double s[3] = {Z[3 * k] - zx, Z[3 * k + 1] - zy, Z[3 * k + 2] - zz};
    const double Mc = q[0];
    const double Ms[3] = {Mc * s[0], Mc * s[1], Mc * s[2]};
    // symmetric Q' as a full matrix
    const double Q[3][3] = {{q[4], q[5], q[6]}, {q[5], q[7], q[8]}, {q[6], q[8], q[9]}};
#pragma unroll
    for (int i = 0; i < 3; ++i) p[1 + i] += Ms[i];
    // Q: xx xy xz yy yz zz
    const int qi[6] = {0, 0, 0, 1, 1, 2}, qj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int t = 0; t < 6; ++t) p[4 + t] += Q[qi[t]][qj[t]] + Ms[qi[t]] * s[qj[t]];
    // O: xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
    const int oi[10] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 2};
    const int oj[10] = {0, 0, 0, 1, 1, 2, 1, 1, 2, 2};
    const int ok[10] = {0, 1, 2, 1, 2, 2, 1, 2, 2, 2};
#pragma unroll
    for (int t = 0; t < 10; ++t) {
      const int i = oi[t], j = oj[t], l = ok[t];
      p[10 + t] += q[10 + t] + (Q[i][j] * s[l] + Q[i][l] * s[j] + Q[j][l] * s[i]) + Ms[i] * s[j] * s[l];
    }
  }
  p[0] = mm;
  double *out = mom + static_cast<int64_t>(c) * kMomStride;
#pragma unroll
  for (int k = 0; k < kMomStride; ++k) out[k] = p[k];
}

// index tables of the symmetric moments: Q in the order xx xy xz yy yz zz,
// O in the order xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
__constant__ int c_q2i[6] = {0, 0, 0, 1, 1, 2}, c_q2j[6] = {0, 1, 2, 1, 2, 2};
__constant__ int c_o3i[10] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 2};
__constant__ int c_o3j[10] = {0, 0, 0, 1, 1, 2, 1, 1, 2, 2};
__constant__ int c_o3k[10] = {0, 1, 2, 1, 2, 2, 1, 2, 2, 2};
// position of Q_ab in that order
__device__ __forceinline__ int sym2(int a, int b) {
  const int lo = min(a, b), hi = max(a, b);
  return lo * 3 - lo * (lo - 1) / 2 + (hi - lo);
}

// The same level with one warp per cell, for levels of few cells.  With one
// thread per cell a small level is a single warp's chain of FP64 operations,
// and an FP64 warp instruction takes many cycles on this GPU (the top
// levels took 30-40 us each).  Here lane k loads child k, every lane forms
// the same octant-order sums of S and M from the shuffled child values (so Z
// is bit-identical to the one-thread form), and lane q then adds moment
// component q over the children in child order.
__global__ void k_internal_upward_warp(int32_t c0, int32_t c1, const int32_t *__restrict__ first_child,
                                       const int32_t *__restrict__ nchild, double *__restrict__ S,
                                       double *__restrict__ M, double *__restrict__ Z,
                                       double *__restrict__ invM, double *__restrict__ mom) {
  const int64_t wg = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t cc = c0 + wg;
  if (cc >= c1) return;  // whole warp
  const int c = static_cast<int>(cc);
  const int nch = nchild[c];
  if (nch == 0) return;  // whole warp
  const int f = first_child[c];
  double sx = 0.0, sy = 0.0, sz = 0.0, mc = 0.0;
  if (lane < nch) {
    sx = S[3 * (f + lane)];
    sy = S[3 * (f + lane) + 1];
    sz = S[3 * (f + lane) + 2];
    mc = M[f + lane];
  }
  double tx = 0.0, ty = 0.0, tz = 0.0, tm = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const double vx = __shfl_sync(0xffffffffu, sx, j), vy = __shfl_sync(0xffffffffu, sy, j);
    const double vz = __shfl_sync(0xffffffffu, sz, j), vm = __shfl_sync(0xffffffffu, mc, j);
    if (j < nch) {
      tx = __dadd_rn(tx, vx);
      ty = __dadd_rn(ty, vy);
      tz = __dadd_rn(tz, vz);
      tm = __dadd_rn(tm, vm);
    }
  }
  const double zx = __ddiv_rn(tx, tm), zy = __ddiv_rn(ty, tm), zz = __ddiv_rn(tz, tm);
  if (lane == 0) {
    S[3 * c] = tx;
    S[3 * c + 1] = ty;
    S[3 * c + 2] = tz;
    M[c] = tm;
    Z[3 * c] = zx;
    Z[3 * c + 1] = zy;
    Z[3 * c + 2] = zz;
    invM[c] = 1.0 / tm;
    mom[static_cast<int64_t>(c) * kMomStride] = tm;
  }
  const int q = lane;
  if (q < 1 || q >= kMomStride) return;
  // component q: 1..3 dipole (i), 4..9 Q (i, j), 10..19 O (i, j, l); the
  // indices of this lane, and the slots of the Q entries it needs
  int i = 0, j = 0, l = 0;
  if (q < 4) {
    i = q - 1;
  } else if (q < 10) {
    i = c_q2i[q - 4];
    j = c_q2j[q - 4];
  } else {
    i = c_o3i[q - 10];
    j = c_o3j[q - 10];
    l = c_o3k[q - 10];
  }
  const int qij = 4 + sym2(i, j), qil = 4 + sym2(i, l), qjl = 4 + sym2(j, l);
  double acc = 0.0;
  for (int k = f; k < f + nch; ++k) {
    const double *cq = mom + static_cast<int64_t>(k) * kMomStride;
    const double s0 = Z[3 * k] - zx, s1 = Z[3 * k + 1] - zy, s2 = Z[3 * k + 2] - zz;
    const double si = i == 0 ? s0 : (i == 1 ? s1 : s2);
    const double sj = j == 0 ? s0 : (j == 1 ? s1 : s2);
    const double sl = l == 0 ? s0 : (l == 1 ? s1 : s2);
    const double Msi = cq[0] * si;
    if (q < 4) acc += Msi;
    else if (q < 10) acc += cq[q] + Msi * sj;
    else acc += cq[q] + (cq[qij] * sl + cq[qil] * sj + cq[qjl] * si) + Msi * sj * sl;
  }
  mom[static_cast<int64_t>(c) * kMomStride + q] = acc;
}

// R_max^2 of every cell: for each level, each body's squared distance to the
// centre of its cell at that level; a segmented warp maximum (bodies of one
// cell are contiguous) and one atomicMax per segment, both on the bit pattern
// (monotone for non-negative doubles, and integer work, which keeps the
// maximum off the FP64 pipe).  max is exact, so the order of combination
// does not matter.
__global__ void k_rmax_bodies(int64_t n, const int32_t *__restrict__ cell_at,
                              const double *__restrict__ X, const double *__restrict__ Y,
                              const double *__restrict__ Zb, const double *__restrict__ Z,
                              unsigned long long *__restrict__ rmax2) {
  const int lev = blockIdx.y;
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int c = -1;
  unsigned long long d2 = 0;  // bit pattern of |X - Z|^2 >= +0
  if (i < n) {
    c = cell_at[static_cast<int64_t>(lev) * n + i];
    if (c >= 0) {
      const double dx = __dsub_rn(X[i], Z[3 * c]);
      const double dy = __dsub_rn(Y[i], Z[3 * c + 1]);
      const double dz = __dsub_rn(Zb[i], Z[3 * c + 2]);
      d2 = static_cast<unsigned long long>(
          __double_as_longlong(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz))));
    }
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_down_sync(0xffffffffu, d2, o);
    const int co = __shfl_down_sync(0xffffffffu, c, o);
    if (lane + o < 32 && co == c && v > d2) d2 = v;
  }
  const int cprev = __shfl_up_sync(0xffffffffu, c, 1);
  const bool head = (lane == 0) || (cprev != c);
  if (c >= 0 && head) atomicMax(&rmax2[c], d2);
}

__global__ void k_rmax_final(int32_t ncell, const unsigned long long *__restrict__ rmax2,
                             double *__restrict__ Rmax) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncell) Rmax[c] = __dsqrt_rn(__longlong_as_double(static_cast<long long>(rmax2[c])));
}

int ensure_cells(fmm_ctx *c, int64_t need, int64_t used) {
  DBuf *ib[] = {&c->begin, &c->count, &c->level, &c->parent, &c->first_child, &c->nchild};
  for (DBuf *b : ib) AMFMM_TRY(ensure_keep_bytes(c, *b, need * sizeof(int32_t), used * sizeof(int32_t)));
  return FMM_OK;
}

}  // namespace

int build_tree(fmm_ctx *c) {
  const int64_t n = c->sz.n;
  cudaStream_t st = c->stream;
  // body buffers
  AMFMM_TRY(ensure<uint64_t>(c, c->key[0], n));
  AMFMM_TRY(ensure<uint32_t>(c, c->idx[0], n));
  AMFMM_TRY(ensure<double>(c, c->X, n));
  AMFMM_TRY(ensure<double>(c, c->Y, n));
  AMFMM_TRY(ensure<double>(c, c->Zb, n));
  AMFMM_TRY(ensure<double>(c, c->Mb, n));
  AMFMM_TRY(ensure<int32_t>(c, c->order, n));
  AMFMM_TRY(ensure<int32_t>(c, c->cur, n));
  AMFMM_TRY(ensure<int32_t>(c, c->flag, n));
  AMFMM_TRY(ensure<int32_t>(c, c->incl, n + 1));
  AMFMM_TRY(ensure<int32_t>(c, c->leaf_of, n));
  AMFMM_TRY(ensure<int32_t>(c, c->cell_at, static_cast<size_t>(kMaxLevel + 1) * n));
  AMFMM_TRY(ensure<int>(c, c->status, 8 + kMaxLevel + 3));
  const int nbb = std::max(1, std::min<int>(c->num_sms * 4, static_cast<int>((n + kBlock - 1) / kBlock)));
  AMFMM_TRY(ensure<double>(c, c->bbox_part, 6 * nbb));
  AMFMM_TRY(ensure<double>(c, c->bbox, 8));
  

  int *status = ptr<int>(c->status);
  AMFMM_CUDA(c, cudaMemsetAsync(status, 0, sizeof(int) * (8 + kMaxLevel + 3), st));
  const int nsys = c->sz.nsys;
  int which = 0;
  if (nsys == 1) {
    k_bbox_partial<<<nbb, kBlock, 0, st>>>(c->x, c->y, c->z, c->m, n, ptr<double>(c->bbox_part), status);
    AMFMM_TRY(launched(c, "bbox_partial"));
    k_bbox_final<<<1, kBlock, 0, st>>>(ptr<double>(c->bbox_part), nbb, ptr<double>(c->bbox));
    AMFMM_TRY(launched(c, "bbox_final"));
    k_keys<<<grid_for(n, kBlock), kBlock, 0, st>>>(c->x, c->y, c->z, n, ptr<double>(c->bbox),
                                                   ptr<uint64_t>(c->key[0]), ptr<uint32_t>(c->idx[0]));
    AMFMM_TRY(launched(c, "keys"));
    AMFMM_TRY(radix_sort_u64(c, c->key, c->idx, n, 63, &which));
  } else {
    AMFMM_TRY(ensure<double>(c, c->sbox, 4 * static_cast<size_t>(nsys)));
    AMFMM_TRY(ensure<int32_t>(c, c->sysid, n));
    k_bbox_sys<<<nsys, kBlock, 0, st>>>(c->x, c->y, c->z, c->m, ptr<int64_t>(c->sys_off), ptr<double>(c->sbox),
                                        ptr<int32_t>(c->sysid), status);
    AMFMM_TRY(launched(c, "bbox_sys"));
    k_keys_sys<<<grid_for(n, kBlock), kBlock, 0, st>>>(c->x, c->y, c->z, n, ptr<double>(c->sbox),
                                                       ptr<int32_t>(c->sysid), ptr<uint64_t>(c->key[0]),
                                                       ptr<uint32_t>(c->idx[0]));
    AMFMM_TRY(launched(c, "keys_sys"));
    int w1 = 0;
    AMFMM_TRY(radix_sort_u64(c, c->key, c->idx, n, 63, &w1));
    AMFMM_TRY(ensure<uint32_t>(c, c->ekey[0], n));
    AMFMM_TRY(ensure<uint32_t>(c, c->eval[0], n));
    k_sys_keys<<<grid_for(n, kBlock), kBlock, 0, st>>>(n, ptr<uint32_t>(c->idx[w1]), ptr<int32_t>(c->sysid),
                                                       ptr<uint32_t>(c->ekey[0]), ptr<uint32_t>(c->eval[0]));
    AMFMM_TRY(launched(c, "sys_keys"));
    int w2 = 0, sbits = 1;
    while ((int64_t(1) << sbits) <= nsys) ++sbits;
    AMFMM_TRY(radix_sort_u32(c, c->ekey, c->eval, n, sbits, &w2));
    k_gather_sorted<<<grid_for(n, kBlock), kBlock, 0, st>>>(n, ptr<uint32_t>(c->eval[w2]), ptr<uint64_t>(c->key[w1]),
                                                            ptr<uint32_t>(c->idx[w1]), ptr<uint64_t>(c->key[w1 ^ 1]),
                                                            ptr<uint32_t>(c->idx[w1 ^ 1]));
    AMFMM_TRY(launched(c, "gather_sorted"));
    which = w1 ^ 1;
  }
  const uint64_t *skey = ptr<uint64_t>(c->key[which]);
  const uint32_t *sidx = ptr<uint32_t>(c->idx[which]);
  AMFMM_TRY(ensure<int32_t>(c, c->lcp, n));
  int32_t *lcp = ptr<int32_t>(c->lcp);
  c->sz.key_which = which;

  // Octree level by level, from one root per system.  The levels' first cell
  // ids live on the device (lvl), so levels are enqueued in batches and the
  // host reads the counts once per batch: the first batch runs as many
  // levels as the previous tree had (a repeated or slowly changing system
  // needs one round trip), later ones two at a time.  Levels past the last
  // find no body left and do nothing.  A level that runs out of cell room
  // stops the batch; the tree is then built again with twice the room.
  int *ovf = status + 1;
  int32_t *lvl = reinterpret_cast<int32_t *>(status + 8);  // kMaxLevel + 3 entries
  int32_t *flag = ptr<int32_t>(c->flag);
  int32_t *excl = ptr<int32_t>(c->incl);
  int32_t *total = ptr<int32_t>(c->totals);
  int64_t cap_cells = std::max<int64_t>(std::max<int64_t>(1024, n / 2 + 64), 2 * static_cast<int64_t>(nsys));
  int lev = 0;
  for (int attempt = 0;; ++attempt) {
    if (attempt > 16) return set_error(c, FMM_EINVAL, "octree: cell room still short after growing");
    AMFMM_TRY(ensure_cells(c, cap_cells, 0));
    const int64_t cap = static_cast<int64_t>(std::min({c->begin.cap, c->count.cap, c->level.cap, c->parent.cap,
                                                       c->first_child.cap, c->nchild.cap}) /
                                             sizeof(int32_t));
    k_permute<<<grid_for(n, kBlock), kBlock, 0, st>>>(c->x, c->y, c->z, c->m, skey, sidx, n,
                                                      ptr<double>(c->X), ptr<double>(c->Y),
                                                      ptr<double>(c->Zb), ptr<double>(c->Mb),
                                                      ptr<int32_t>(c->order), lcp, ptr<int32_t>(c->cur),
                                                      nsys == 1 ? nullptr : ptr<int32_t>(c->sysid));
    AMFMM_TRY(launched(c, "permute"));
    k_roots<<<grid_for(nsys, kBlock), kBlock, 0, st>>>(nsys, ptr<int64_t>(c->sys_off), ptr<int32_t>(c->begin),
                                                       ptr<int32_t>(c->count), ptr<int32_t>(c->level),
                                                       ptr<int32_t>(c->parent), ptr<int32_t>(c->first_child),
                                                       ptr<int32_t>(c->nchild), lvl, ovf);
    AMFMM_TRY(launched(c, "roots"));
    bool done = false, over = false;
    int32_t *h = static_cast<int32_t *>(c->hpin);
    for (lev = 0; !done;) {
      const int batch = lev == 0 ? std::max(1, c->last_depth + 1) : 2;
      const int lev_end = std::min(lev + batch, kMaxLevel + 1);
      for (int l = lev; l < lev_end; ++l) {
        k_level_flags<<<grid_for(n, kBlock), kBlock, 0, st>>>(
            n, l, c->opts.n_crit, lcp, ptr<int32_t>(c->begin), ptr<int32_t>(c->count), ptr<int32_t>(c->cur),
            flag, excl, lvl, ptr<int32_t>(c->cell_at) + static_cast<int64_t>(l) * n, ptr<int32_t>(c->leaf_of), ovf);
        AMFMM_TRY(launched(c, "level_flags"));
        AMFMM_TRY(exclusive_scan_i32(c, flag, excl, n, total));
        k_make_cells<<<grid_for(n, kBlock), kBlock, 0, st>>>(
            n, l, lvl, total, cap, flag, excl, ptr<int32_t>(c->cur), ptr<int32_t>(c->begin),
            ptr<int32_t>(c->level), ptr<int32_t>(c->parent), ptr<int32_t>(c->first_child),
            ptr<int32_t>(c->nchild), ovf);
        AMFMM_TRY(launched(c, "make_cells"));
        // no more new cells than bodies
        k_cell_counts<<<grid_for(n, kBlock), kBlock, 0, st>>>(l, lvl, ptr<int32_t>(c->begin), ptr<int32_t>(c->count),
                                                             ptr<int32_t>(c->parent), ptr<int32_t>(c->nchild), ovf);
        AMFMM_TRY(launched(c, "cell_counts"));
      }
      const HostRead rb{h, status, sizeof(int) * (8 + kMaxLevel + 3)};
      AMFMM_TRY(read_back(c, &rb, 1));
      if (capturing(c)) {
        // a captured solve keeps the planned cell room
        if (h[1]) return set_error(c, FMM_ECUDA, "graph capture: the planning solve grew the cell room");
        Expect e;
        for (int k = 0; k < 8 + kMaxLevel + 3; ++k) e.add(status + k, static_cast<uint32_t>(h[k]));
        AMFMM_TRY(graph_expect(c, e));
        st = c->stream;
      }
      const int32_t *hl = h + 8;
      if (h[1]) {  // out of cell room: grow beyond what the levels so far asked for
        int64_t need = cap;
        for (int l = 0; l < lev_end; ++l) need = std::max<int64_t>(need, hl[l + 2]);
        cap_cells = std::max<int64_t>(2 * cap, need + n / 2 + 64);
        over = true;
        break;
      }
      for (int l = lev; l < lev_end && !done; ++l)
        if (hl[l + 2] == hl[l + 1]) {  // level l made no new cells: the tree is complete
          done = true;
          lev = l;
        }
      if (!done) {
        if (lev_end > kMaxLevel) return set_error(c, FMM_EINVAL, "octree: cells below the deepest level");
        lev = lev_end;
      }
    }
    if (over) continue;
    c->sz.lvl_off.assign(h + 8, h + 8 + lev + 2);
    break;
  }
  c->last_depth = lev;
  c->sz.depth = lev;
  c->sz.ncell = c->sz.lvl_off.back();
  // leaves in id order
  const int64_t nc = c->sz.ncell;
  AMFMM_TRY(ensure<int32_t>(c, c->leaves, nc + 1));
  // a tree of single-child chains can have more cells than bodies
  AMFMM_TRY(ensure<int32_t>(c, c->flag, std::max(n, nc) + 1));
  AMFMM_TRY(ensure<int32_t>(c, c->incl, std::max(n, nc) + 1));
  flag = ptr<int32_t>(c->flag);
  excl = ptr<int32_t>(c->incl);
  k_leaf_flags<<<grid_for(nc, kBlock), kBlock, 0, st>>>(static_cast<int32_t>(nc), ptr<int32_t>(c->nchild), flag);
  AMFMM_TRY(launched(c, "leaf_flags"));
  AMFMM_TRY(exclusive_scan_i32(c, flag, excl, nc, total));
  k_leaf_compact<<<grid_for(nc, kBlock), kBlock, 0, st>>>(static_cast<int32_t>(nc), ptr<int32_t>(c->nchild),
                                                          excl, ptr<int32_t>(c->leaves));
  AMFMM_TRY(launched(c, "leaf_compact"));
  {
    int32_t *h = static_cast<int32_t *>(c->hpin);
    double *hb = reinterpret_cast<double *>(h + 4);
    const double *bbox = c->sz.nsys == 1 ? ptr<double>(c->bbox) : ptr<double>(c->sbox);
    const HostRead rb[3] = {{h, total, sizeof(int32_t)}, {h + 1, status, sizeof(int32_t)},
                            {hb, bbox, 4 * sizeof(double)}};
    AMFMM_TRY(read_back(c, rb, 3));
    if (capturing(c)) {
      AMFMM_TRY(graph_record_bbox(c, bbox));
      Expect e;
      e.add(total, static_cast<uint32_t>(h[0]));
      e.add(status, static_cast<uint32_t>(h[1]));
      AMFMM_TRY(graph_expect(c, e));
    }
    c->sz.nleaf = h[0];
    for (int d = 0; d < 3; ++d) c->sz.lo[d] = hb[d];
    c->sz.scale = hb[3];
    if (h[1] != 0)
      return set_error(c, FMM_EINVAL, "a body has a non-finite coordinate or a mass that is not positive and finite");
  }
  return FMM_OK;
}

int upward(fmm_ctx *c) {
  const int64_t n = c->sz.n, nc = c->sz.ncell;
  cudaStream_t st = c->stream;
  AMFMM_TRY(ensure<double>(c, c->S, 3 * nc));
  AMFMM_TRY(ensure<double>(c, c->M, nc));
  AMFMM_TRY(ensure<double>(c, c->Z, 3 * nc));
  AMFMM_TRY(ensure<double>(c, c->invM, nc));
  AMFMM_TRY(ensure<double>(c, c->Rmax, nc));
  AMFMM_TRY(ensure<unsigned long long>(c, c->rmax2, nc));
  AMFMM_TRY(ensure<double>(c, c->mom, static_cast<size_t>(mom_stride(c->opts.order_P)) * nc));
  if (c->opts.order_P != 3) {
    AMFMM_TRY(upward_general(c));
  } else {
  k_leaf_upward<<<grid_for(c->sz.nleaf, 128), 128, 0, st>>>(
      static_cast<int32_t>(c->sz.nleaf), ptr<int32_t>(c->leaves), ptr<int32_t>(c->begin),
      ptr<int32_t>(c->count), ptr<double>(c->X), ptr<double>(c->Y), ptr<double>(c->Zb),
      ptr<double>(c->Mb), ptr<double>(c->S), ptr<double>(c->M), ptr<double>(c->Z),
      ptr<double>(c->invM), ptr<double>(c->mom));
  AMFMM_TRY(launched(c, "leaf_upward"));
  for (int lev = c->sz.depth - 1; lev >= 0; --lev) {
    const int64_t c0 = c->sz.lvl_off[lev], c1 = c->sz.lvl_off[lev + 1];
    // few cells: a warp per cell; many: a thread per cell (throughput-bound)
    if (c1 - c0 < 8192)
      k_internal_upward_warp<<<grid_for(32 * (c1 - c0), 128), 128, 0, st>>>(
          static_cast<int32_t>(c0), static_cast<int32_t>(c1), ptr<int32_t>(c->first_child),
          ptr<int32_t>(c->nchild), ptr<double>(c->S), ptr<double>(c->M), ptr<double>(c->Z),
          ptr<double>(c->invM), ptr<double>(c->mom));
    else
      k_internal_upward<<<grid_for(c1 - c0, 128), 128, 0, st>>>(
          static_cast<int32_t>(c0), static_cast<int32_t>(c1), ptr<int32_t>(c->first_child),
          ptr<int32_t>(c->nchild), ptr<double>(c->S), ptr<double>(c->M), ptr<double>(c->Z),
          ptr<double>(c->invM), ptr<double>(c->mom));
    AMFMM_TRY(launched(c, "internal_upward"));
  }
  }
  AMFMM_CUDA(c, cudaMemsetAsync(c->rmax2.p, 0, sizeof(unsigned long long) * nc, st));
  dim3 g(grid_for(n, kBlock), static_cast<unsigned>(c->sz.depth + 1));
  k_rmax_bodies<<<g, kBlock, 0, st>>>(n, ptr<int32_t>(c->cell_at), ptr<double>(c->X), ptr<double>(c->Y),
                                      ptr<double>(c->Zb), ptr<double>(c->Z),
                                      ptr<unsigned long long>(c->rmax2));
  AMFMM_TRY(launched(c, "rmax_bodies"));
  k_rmax_final<<<grid_for(nc, kBlock), kBlock, 0, st>>>(static_cast<int32_t>(nc),
                                                        ptr<unsigned long long>(c->rmax2), ptr<double>(c->Rmax));
  return launched(c, "rmax_final");
}

}  // namespace amfmm
