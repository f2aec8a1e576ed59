// sort.cu -- device primitives: exclusive prefix sums and a stable LSD radix
// sort of (key, value) pairs.  Both are deterministic: integer arithmetic
// only, and a fixed assignment of keys to ranks.
#include "internal.cuh"

namespace amfmm {
namespace {

constexpr int kScanBlock = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;
constexpr int kRedundantTiles = 4096;  // up to 8M elements: two launches per scan

constexpr int kSortBlock = 256;
// keys per thread of a sort tile, per key type
template <class K>
struct SortCfg {
  static constexpr int kItems = 16;
};
template <class K>
constexpr int kSortItems = SortCfg<K>::kItems;
template <class K>
constexpr int kSortTile = kSortBlock * kSortItems<K>;
constexpr int kDigitBits = 9;
constexpr int kRadix = 1 << kDigitBits;  // 512 buckets per pass
constexpr unsigned kDigitMask = kRadix - 1;

// ---- element operations for the scans ----
__device__ __forceinline__ int32_t vadd(int32_t a, int32_t b) { return a + b; }
__device__ __forceinline__ int64_t vadd(int64_t a, int64_t b) { return a + b; }
__device__ __forceinline__ int4 vadd(int4 a, int4 b) {
  return make_int4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
template <class T> __device__ __forceinline__ T vzero();
template <> __device__ __forceinline__ int32_t vzero<int32_t>() { return 0; }
template <> __device__ __forceinline__ int64_t vzero<int64_t>() { return 0; }
template <> __device__ __forceinline__ int4 vzero<int4>() { return make_int4(0, 0, 0, 0); }

__device__ __forceinline__ int32_t shfl_up(int32_t v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ int64_t shfl_up(int64_t v, int d) {
  return static_cast<int64_t>(__shfl_up_sync(0xffffffffu, static_cast<long long>(v), d));
}
__device__ __forceinline__ int4 shfl_up(int4 v, int d) {
  return make_int4(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d),
                   __shfl_up_sync(0xffffffffu, v.z, d), __shfl_up_sync(0xffffffffu, v.w, d));
}

// Inclusive scan across the warp.
template <class T>
__device__ __forceinline__ T warp_inclusive(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T t = shfl_up(v, d);
    if (lane >= d) v = vadd(v, t);
  }
  return v;
}

// Exclusive scan of one value per thread over the block; returns the block total.
template <class T>
__device__ __forceinline__ T block_exclusive(T v, T *excl) {
  __shared__ T wtot[kScanBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T inc = warp_inclusive(v);
  if (lane == 31) wtot[w] = inc;
  __syncthreads();
  if (w == 0) {
    T s = lane < kScanBlock / 32 ? wtot[lane] : vzero<T>();
    s = warp_inclusive(s);
    if (lane < kScanBlock / 32) wtot[lane] = s;
  }
  __syncthreads();
  T before = w > 0 ? wtot[w - 1] : vzero<T>();
  T prev = shfl_up(inc, 1);
  if (lane == 0) prev = vzero<T>();
  *excl = vadd(before, prev);
  T total = wtot[kScanBlock / 32 - 1];
  __syncthreads();
  return total;
}

template <class T>
__global__ void k_tile_reduce(const T *__restrict__ in, int64_t n, T *__restrict__ sums) {
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
  T s = vzero<T>();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + static_cast<int64_t>(k) * kScanBlock + threadIdx.x;
    if (i < n) s = vadd(s, in[i]);
  }
  T excl;
  T tot = block_exclusive(s, &excl);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Exclusive scan of one tile; the tile's offset is offs[tile] when offs is
// given, else the sum of the tile sums sums[0, tile) taken by this block
// (integer addition: exact in any order), else zero.  The last tile writes
// the grand total.
template <class T>
__global__ void k_tile_scan(const T *__restrict__ in, T *__restrict__ out, int64_t n,
                            const T *__restrict__ offs, T *__restrict__ total,
                            const T *__restrict__ sums = nullptr) {
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
  T pre = vzero<T>();
  if (!offs && sums) {
    for (int q = threadIdx.x; q < static_cast<int>(blockIdx.x); q += kScanBlock) pre = vadd(pre, sums[q]);
    T ignore;
    pre = block_exclusive(pre, &ignore);  // the block total of the partial sums
  }
  // each thread owns kScanItems consecutive elements
  T v[kScanItems];
  const int64_t mybase = base + static_cast<int64_t>(threadIdx.x) * kScanItems;
  T s = vzero<T>();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = mybase + k;
    v[k] = i < n ? in[i] : vzero<T>();
    s = vadd(s, v[k]);
  }
  T excl;
  T tot = block_exclusive(s, &excl);
  T off = offs ? offs[blockIdx.x] : pre;
  T run = vadd(off, excl);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = mybase + k;
    if (i < n) out[i] = run;
    run = vadd(run, v[k]);
  }
  if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = vadd(off, tot);
}

template <class T>
int scan_impl(fmm_ctx *c, const T *in, T *out, int64_t n, T *total, size_t tmp_off) {
  if (n <= 0) {
    if (total) AMFMM_CUDA(c, cudaMemsetAsync(total, 0, sizeof(T), c->stream));
    return FMM_OK;
  }
  const int64_t nt = (n + kScanTile - 1) / kScanTile;
  if (nt == 1) {
    k_tile_scan<T><<<1, kScanBlock, 0, c->stream>>>(in, out, n, nullptr, total);
    return launched(c, "tile_scan");
  }
  // scratch: sums[nt], offs[nt], then the recursion's scratch
  size_t need = tmp_off + 2 * static_cast<size_t>(nt) * sizeof(T) + 256;
  if (need > c->scan_tmp.cap) {
    return set_error(c, FMM_ENOMEM, "scan scratch too small (%zu > %zu)", need, c->scan_tmp.cap);
  }
  char *base = static_cast<char *>(c->scan_tmp.p) + tmp_off;
  T *sums = reinterpret_cast<T *>(base);
  T *offs = sums + nt;
  size_t next = tmp_off + ((2 * static_cast<size_t>(nt) * sizeof(T) + 255) / 256) * 256;
  k_tile_reduce<T><<<static_cast<unsigned>(nt), kScanBlock, 0, c->stream>>>(in, n, sums);
  AMFMM_TRY(launched(c, "tile_reduce"));
  if (nt <= kRedundantTiles) {
    // few tiles: every block adds up the sums of the tiles before it (at
    // most kRedundantTiles reads, from L2) instead of a separate scan of them
    k_tile_scan<T><<<static_cast<unsigned>(nt), kScanBlock, 0, c->stream>>>(in, out, n, nullptr, total, sums);
    return launched(c, "tile_scan");
  }
  AMFMM_TRY(scan_impl<T>(c, sums, offs, nt, nullptr, next));
  k_tile_scan<T><<<static_cast<unsigned>(nt), kScanBlock, 0, c->stream>>>(in, out, n, offs, total);
  return launched(c, "tile_scan");
}

template <class T>
int scan_entry(fmm_ctx *c, const T *in, T *out, int64_t n, T *total) {
  // scratch bound: 2 * sizeof(T) * (n/tile + n/tile^2 + ...) + alignment
  size_t need = 0;
  for (int64_t m = (n + kScanTile - 1) / kScanTile; m > 1; m = (m + kScanTile - 1) / kScanTile)
    need += ((2 * static_cast<size_t>(m) * sizeof(T) + 255) / 256) * 256 + 256;
  AMFMM_TRY(ensure_bytes(c, c->scan_tmp, need + 1024));
  return scan_impl<T>(c, in, out, n, total, 0);
}

// ---- radix sort ----
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <class K>
__global__ void k_radix_hist(const K *__restrict__ key, int64_t n, int shift,
                             int32_t *__restrict__ hist, int ntiles) {
  __shared__ int cnt[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += kSortBlock) cnt[d] = 0;
  __syncthreads();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile<K>;
  if (base + kSortTile<K> <= n) {
    // whole tile: 16-byte loads (the tile starts 16-byte aligned), all in
    // flight before the counting
    constexpr int kPer = 16 / sizeof(K), kLoads = kSortItems<K> / kPer;
    using V = uint4;
    V v[kLoads];
    const V *kv = reinterpret_cast<const V *>(key + base);
#pragma unroll
    for (int k = 0; k < kLoads; ++k) v[k] = kv[k * kSortBlock + threadIdx.x];
#pragma unroll
    for (int k = 0; k < kLoads; ++k) {
      const K *e = reinterpret_cast<const K *>(&v[k]);
#pragma unroll
      for (int u = 0; u < kPer; ++u) atomicAdd(&cnt[static_cast<int>((e[u] >> shift) & kDigitMask)], 1);
    }
  } else {
    for (int k = 0; k < kSortItems<K>; ++k) {
      int64_t i = base + static_cast<int64_t>(k) * kSortBlock + threadIdx.x;
      if (i < n) atomicAdd(&cnt[static_cast<int>((key[i] >> shift) & kDigitMask)], 1);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortBlock)
    hist[static_cast<int64_t>(d) * ntiles + blockIdx.x] = cnt[d];
}

// Stable scatter of one tile of kSortTile keys.  Warp w owns the keys
// [w * 512, (w + 1) * 512) of the tile and takes them 32 at a time in index
// order: a key's rank among the warp's keys of its digit is the warp's running
// count of that digit (shared memory, updated by the first lane of each group
// of equal digits) plus its rank within the group.  One exclusive scan over
// (digit, warp) then gives every key its position in the tile's stably
// digit-sorted order; the tile is staged in that order in shared memory and
// written out so that consecutive threads store consecutive positions of a
// bucket (coalesced).
template <class K>
constexpr int kWarpKeys = kSortTile<K> / (kSortBlock / 32);  // 512 at 16 keys per thread
template <class K>
constexpr int kRounds = kWarpKeys<K> / 32;
static_assert(kRadix == 2 * kSortBlock, "the scan gives each thread two digits");

template <class K>
__global__ void __launch_bounds__(kSortBlock) k_radix_scatter(
    const K *__restrict__ key, const uint32_t *__restrict__ val, int64_t n, int shift,
    const int32_t *__restrict__ offs, int ntiles, K *__restrict__ okey, uint32_t *__restrict__ oval) {
  constexpr int kW = kSortBlock / 32;
  constexpr size_t kCntBytes = sizeof(int) * kW * (kRadix + 1);
  constexpr size_t kStageBytes = sizeof(K) * kSortTile<K>;
  constexpr int kRounds = ::amfmm::kRounds<K>;
  constexpr int kWarpKeys = ::amfmm::kWarpKeys<K>;
  constexpr int kSortTile = ::amfmm::kSortTile<K>;
  __shared__ __align__(16) unsigned char pool[kCntBytes > kStageBytes ? kCntBytes : kStageBytes];
  __shared__ int dstart[kRadix];
  __shared__ int goff[kRadix];
  __shared__ int wsum[kW];
  int(*cnt)[kRadix + 1] = reinterpret_cast<int(*)[kRadix + 1]>(pool);
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int64_t tile0 = static_cast<int64_t>(blockIdx.x) * kSortTile;
  const int nvalid = static_cast<int>(n - tile0 < kSortTile ? n - tile0 : kSortTile);
  for (int q = t; q < kW * (kRadix + 1); q += kSortBlock) (&cnt[0][0])[q] = 0;
  for (int d = t; d < kRadix; d += kSortBlock) goff[d] = offs[static_cast<int64_t>(d) * ntiles + blockIdx.x];
  __syncthreads();
  const unsigned lt = lanemask_lt();
  K k[kRounds];
  uint32_t v[kRounds];
  int lpos[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int li = w * kWarpKeys + r * 32 + lane;
    const bool valid = li < nvalid;
    k[r] = valid ? key[tile0 + li] : K(0);
    v[r] = valid ? val[tile0 + li] : 0u;
    const int d = valid ? static_cast<int>((k[r] >> shift) & kDigitMask) : kRadix;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int wrank = __popc(peers & lt);
    const int prev = cnt[w][d];
    __syncwarp();
    lpos[r] = prev + wrank;
    if (wrank == 0) cnt[w][d] = prev + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // exclusive scan over (digit, warp), digit-major: thread t owns digits
  // 2t and 2t + 1 (kRadix = 2 * kSortBlock)
  int own = 0;
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int q = 0; q < kW; ++q) own += cnt[q][2 * t + h];
  int incl = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  int before = incl - own;
  for (int q = 0; q < w; ++q) before += wsum[q];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int dd = 2 * t + h;
    dstart[dd] = before;
#pragma unroll
    for (int q = 0; q < kW; ++q) {
      const int cq = cnt[q][dd];
      cnt[q][dd] = before;
      before += cq;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int li = w * kWarpKeys + r * 32 + lane;
    if (li < nvalid) lpos[r] += cnt[w][static_cast<int>((k[r] >> shift) & kDigitMask)];
  }
  __syncthreads();  // the counts are dead from here; the pool stages the tile
  K *sk = reinterpret_cast<K *>(pool);
#pragma unroll
  for (int r = 0; r < kRounds; ++r)
    if (w * kWarpKeys + r * 32 + lane < nvalid) sk[lpos[r]] = k[r];
  __syncthreads();
  int dig[kRounds];
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int j = r * kSortBlock + t;
    dig[r] = 0;
    if (j < nvalid) {
      const K kk = sk[j];
      const int d = static_cast<int>((kk >> shift) & kDigitMask);
      dig[r] = d;
      okey[goff[d] + (j - dstart[d])] = kk;
    }
  }
  __syncthreads();
  uint32_t *sv = reinterpret_cast<uint32_t *>(pool);
#pragma unroll
  for (int r = 0; r < kRounds; ++r)
    if (w * kWarpKeys + r * 32 + lane < nvalid) sv[lpos[r]] = v[r];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRounds; ++r) {
    const int j = r * kSortBlock + t;
    if (j < nvalid) oval[goff[dig[r]] + (j - dstart[dig[r]])] = sv[j];
  }
}

template <class K>
int radix_sort(fmm_ctx *c, DBuf key[2], DBuf val[2], int64_t n, int bits, int *which) {
  *which = 0;
  if (n <= 1 || bits <= 0) return FMM_OK;
  if (n > 0x7fffffffLL) return set_error(c, FMM_EINVAL, "radix sort: n too large");
  const int ntiles = static_cast<int>((n + kSortTile<K> - 1) / kSortTile<K>);
  const int64_t nh = static_cast<int64_t>(kRadix) * ntiles;
  AMFMM_TRY(ensure<int32_t>(c, c->sort_hist, 2 * nh + 64));
  AMFMM_TRY(ensure<K>(c, key[1], n));
  AMFMM_TRY(ensure<uint32_t>(c, val[1], n));
  int32_t *hist = ptr<int32_t>(c->sort_hist);
  int32_t *offs = hist + nh;
  int cur = 0;
  // equal digit widths of at most kDigitBits bits
  const int passes = (bits + kDigitBits - 1) / kDigitBits;
  for (int p = 0, shift = 0; p < passes; ++p, shift += kDigitBits) {
    k_radix_hist<K><<<ntiles, kSortBlock, 0, c->stream>>>(ptr<K>(key[cur]), n, shift, hist, ntiles);
    AMFMM_TRY(launched(c, "radix_hist"));
    AMFMM_TRY(exclusive_scan_i32(c, hist, offs, nh, nullptr));
    k_radix_scatter<K><<<ntiles, kSortBlock, 0, c->stream>>>(
        ptr<K>(key[cur]), ptr<uint32_t>(val[cur]), n, shift, offs, ntiles, ptr<K>(key[cur ^ 1]),
        ptr<uint32_t>(val[cur ^ 1]));
    AMFMM_TRY(launched(c, "radix_scatter"));
    cur ^= 1;
  }
  *which = cur;
  return FMM_OK;
}

}  // namespace

int exclusive_scan_i32(fmm_ctx *c, const int32_t *in, int32_t *out, int64_t n, int32_t *total) {
  return scan_entry<int32_t>(c, in, out, n, total);
}
int exclusive_scan_i64(fmm_ctx *c, const int64_t *in, int64_t *out, int64_t n, int64_t *total) {
  return scan_entry<int64_t>(c, in, out, n, total);
}
int exclusive_scan_i4(fmm_ctx *c, const int4 *in, int4 *out, int64_t n, int4 *total) {
  return scan_entry<int4>(c, in, out, n, total);
}
int radix_sort_u64(fmm_ctx *c, DBuf key[2], DBuf val[2], int64_t n, int bits, int *which) {
  return radix_sort<uint64_t>(c, key, val, n, bits, which);
}
int radix_sort_u32(fmm_ctx *c, DBuf key[2], DBuf val[2], int64_t n, int bits, int *which) {
  return radix_sort<uint32_t>(c, key, val, n, bits, which);
}

}  // namespace amfmm
