// diag.cu -- a10: diagnostics.  Exact direct summation for a subset of bodies
// (Sec. 3 measures the method's error against the directly summed force) and
// the net force / torque balance of Sec. 3,
//     sqrt( sum_d (sum_n mu_n A_nd)^2 / sum_d (sum_n mu_n |A_nd|)^2 ),
// with A = a (force) and A = X x a (torque).  Both are FP64 with Neumaier
// compensated sums in a fixed order of combination, so they are
// reproducible bit for bit.
#include <mutex>

#include "internal.cuh"

namespace amfmm {
namespace {

constexpr int kBlock = 256;

struct Comp {
  double s, c;
};

__device__ __forceinline__ void nadd(Comp &a, double v) {
  const double t = a.s + v;
  if (fabs(a.s) >= fabs(v)) a.c += (a.s - t) + v;
  else a.c += (v - t) + a.s;
  a.s = t;
}

// combine two compensated partial sums (fixed order: a then b)
__device__ __forceinline__ Comp ncombine(Comp a, Comp b) {
  nadd(a, b.s);
  a.c += b.c;
  return a;
}

// Block-wide reduction of NV compensated sums in a fixed tree order; the
// result is valid in thread 0.
template <int NV>
__device__ void block_reduce(Comp (&v)[NV]) {
  __shared__ double sh[NV][2][kBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      Comp u{__shfl_down_sync(0xffffffffu, v[k].s, o), __shfl_down_sync(0xffffffffu, v[k].c, o)};
      if (lane < o) v[k] = ncombine(v[k], u);
    }
    if (lane == 0) {
      sh[k][0][w] = v[k].s;
      sh[k][1][w] = v[k].c;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      Comp a{sh[k][0][0], sh[k][1][0]};
      for (int q = 1; q < kBlock / 32; ++q) a = ncombine(a, Comp{sh[k][0][q], sh[k][1][q]});
      v[k] = a;
    }
  }
  __syncthreads();
}

// Arithmetic peak of the plain (non-tensor) FMA pipe: every thread runs
// kPeakChains independent chains a = a * b + c, kPeakUnroll steps per
// iteration, on a grid of kPeakBlocksPerSM blocks per SM.  The chains' sum is
// written only if it equals a value it cannot reach, which keeps them live
// without a store per thread.  The roofline of the interaction kernels
// (bound by this pipe, not by memory) is taken against what it measures.
constexpr int kPeakBlock = 256, kPeakBlocksPerSM = 8, kPeakChains = 8, kPeakUnroll = 16;

template <class T>
__global__ void __launch_bounds__(kPeakBlock) k_fma_peak(int iters, T *__restrict__ sink) {
  T a[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
  const T b = T(0.9999), c = T(1e-4);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) a[k] = fma(a[k], b, c);
    }
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += a[k];
  if (s == T(-12345.0) && sink) *sink = s;
}

// one block per target body
__global__ void __launch_bounds__(kBlock) k_direct(int64_t n, const double *__restrict__ x,
                                                   const double *__restrict__ y, const double *__restrict__ z,
                                                   const double *__restrict__ m, const int32_t *__restrict__ tg,
                                                   double eps2, double *__restrict__ ax, double *__restrict__ ay,
                                                   double *__restrict__ az) {
  const int i = tg[blockIdx.x];
  const double xi = x[i], yi = y[i], zi = z[i];
  Comp a[3] = {{0, 0}, {0, 0}, {0, 0}};
  for (int64_t j = threadIdx.x; j < n; j += kBlock) {
    const double dx = x[j] - xi, dy = y[j] - yi, dz = z[j] - zi;
    const double d2 = (dx * dx + dy * dy) + dz * dz;
    if (d2 > 0.0) {
      const double r2 = d2 + eps2;
      const double inv3 = 1.0 / (r2 * sqrt(r2));
      const double s = m[j] * inv3;
      nadd(a[0], s * dx);
      nadd(a[1], s * dy);
      nadd(a[2], s * dz);
    }
  }
  block_reduce<3>(a);
  if (threadIdx.x == 0) {
    ax[blockIdx.x] = a[0].s + a[0].c;
    ay[blockIdx.x] = a[1].s + a[1].c;
    az[blockIdx.x] = a[2].s + a[2].c;
  }
}

// per-block partials of sum mu A (compensated) and sum mu |A| for force and torque
__global__ void __launch_bounds__(kBlock) k_balance_partial(int64_t n, const double *__restrict__ x,
                                                            const double *__restrict__ y,
                                                            const double *__restrict__ z,
                                                            const double *__restrict__ m,
                                                            const double *__restrict__ ax,
                                                            const double *__restrict__ ay,
                                                            const double *__restrict__ az,
                                                            double *__restrict__ part) {
  Comp v[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = Comp{0, 0};
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = blockIdx.x * per, b1 = min(n, b0 + per);
  for (int64_t i = b0 + threadIdx.x; i < b1; i += kBlock) {
    const double mu = m[i];
    const double a[3] = {ax[i], ay[i], az[i]};
    const double t[3] = {y[i] * az[i] - z[i] * ay[i], z[i] * ax[i] - x[i] * az[i], x[i] * ay[i] - y[i] * ax[i]};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      nadd(v[d], mu * a[d]);
      nadd(v[3 + d], mu * fabs(a[d]));
      nadd(v[6 + d], mu * t[d]);
      nadd(v[9 + d], mu * fabs(t[d]));
    }
  }
  block_reduce<12>(v);
  if (threadIdx.x == 0)
    for (int k = 0; k < 12; ++k) {
      part[(blockIdx.x * 12 + k) * 2] = v[k].s;
      part[(blockIdx.x * 12 + k) * 2 + 1] = v[k].c;
    }
}

__global__ void k_balance_final(int nb, const double *__restrict__ part, double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Comp v[12];
  for (int k = 0; k < 12; ++k) v[k] = Comp{0, 0};
  for (int b = 0; b < nb; ++b)
    for (int k = 0; k < 12; ++k) v[k] = ncombine(v[k], Comp{part[(b * 12 + k) * 2], part[(b * 12 + k) * 2 + 1]});
  double fn = 0, fd = 0, tn = 0, td = 0;
  for (int d = 0; d < 3; ++d) {
    const double f = v[d].s + v[d].c, fa = v[3 + d].s + v[3 + d].c;
    const double t = v[6 + d].s + v[6 + d].c, ta = v[9 + d].s + v[9 + d].c;
    fn += f * f;
    fd += fa * fa;
    tn += t * t;
    td += ta * ta;
  }
  out[0] = fd > 0 ? sqrt(fn / fd) : 0.0;
  out[1] = td > 0 ? sqrt(tn / td) : 0.0;
}

}  // namespace
}  // namespace amfmm

using namespace amfmm;

extern "C" {

int fmm_direct(fmm_ctx *c, const double *x, const double *y, const double *z, const double *m, int64_t n,
               const int32_t *targets, int64_t nt, double *ax, double *ay, double *az) {
  if (!c) return FMM_EINVAL;
  if (n < 1 || nt < 0 || nt > 0x7fffffffLL) return set_error(c, FMM_EINVAL, "bad sizes for fmm_direct");
  if (nt == 0) return FMM_OK;
  if (!x || !y || !z || !m || !targets || !ax || !ay || !az) return set_error(c, FMM_EINVAL, "NULL array");
  k_direct<<<static_cast<unsigned>(nt), kBlock, 0, c->stream>>>(n, x, y, z, m, targets, c->eps2, ax, ay, az);
  return launched(c, "direct");
}

int fmm_alu_peak(int precision, int reps, double *tflops) {
  if (!tflops || reps < 1 || (precision != FMM_FP64 && precision != FMM_MIXED)) return FMM_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return FMM_ECUDA;
  }
  // FP64 runs at 1/64 of the FP32 rate: fewer iterations keep both launches
  // in the millisecond range
  const int iters = precision == FMM_FP64 ? 64 : 4096;
  const unsigned grid = static_cast<unsigned>(sms * kPeakBlocksPerSM);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double best = 0.0;
  int rc = FMM_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = FMM_ECUDA;
  for (int r = 0; r <= reps && rc == FMM_OK; ++r) {  // the first launch warms up
    cudaEventRecord(e0, 0);
    if (precision == FMM_FP64) k_fma_peak<double><<<grid, kPeakBlock>>>(iters, nullptr);
    else k_fma_peak<float><<<grid, kPeakBlock>>>(iters, nullptr);
    cudaEventRecord(e1, 0);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) {
      rc = FMM_ECUDA;
      break;
    }
    const double flops = 2.0 * kPeakChains * kPeakUnroll * static_cast<double>(iters) * grid * kPeakBlock;
    if (r > 0) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  if (rc == FMM_OK) *tflops = best;
  return rc;
}

int fmm_balance(fmm_ctx *c, const double *x, const double *y, const double *z, const double *m,
                const double *ax, const double *ay, const double *az, int64_t n, double *out) {
  if (!c || !out) return FMM_EINVAL;
  if (n < 1) return set_error(c, FMM_EINVAL, "n must be >= 1");
  const int nb = static_cast<int>(std::min<int64_t>(c->num_sms * 4, (n + kBlock - 1) / kBlock));
  AMFMM_TRY(ensure<double>(c, c->diag, static_cast<size_t>(nb) * 24 + 8));
  double *part = ptr<double>(c->diag);
  k_balance_partial<<<nb, kBlock, 0, c->stream>>>(n, x, y, z, m, ax, ay, az, part);
  AMFMM_TRY(launched(c, "balance_partial"));
  k_balance_final<<<1, 32, 0, c->stream>>>(nb, part, part + static_cast<size_t>(nb) * 24);
  AMFMM_TRY(launched(c, "balance_final"));
  AMFMM_CUDA(c, cudaMemcpyAsync(out, part + static_cast<size_t>(nb) * 24, 2 * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
  AMFMM_CUDA(c, cudaStreamSynchronize(c->stream));
  return FMM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Balance check without any allocation.
//
// The partial sums live in a file-scope device array instead of memory the
// library allocates: one record of 12 compensated sums (24 doubles) per tile
// of kNoAllocTile bodies, for at most kNoAllocMaxTiles tiles.  Every GPU that
// loads the library holds this array (about 197 KB) until the process exits.
// Each call overwrites the records it reads, so nothing needs clearing, but all
// calls share the one array: two calls whose kernels overlap on the GPU (for
// example on two streams) race and can return wrong values.
// ---------------------------------------------------------------------------
namespace amfmm {
namespace {

constexpr int64_t kNoAllocTile = 4096;
constexpr int64_t kNoAllocMaxTiles = 1024;  // at most 4,194,304 bodies
static __device__ __align__(256) double g_balance_scratch[kNoAllocMaxTiles * 24];

// same sums as k_balance_partial, over fixed tiles of kNoAllocTile bodies
__global__ void __launch_bounds__(kBlock) k_balance_tiles(int64_t n, const double *__restrict__ x,
                                                          const double *__restrict__ y,
                                                          const double *__restrict__ z,
                                                          const double *__restrict__ m,
                                                          const double *__restrict__ ax,
                                                          const double *__restrict__ ay,
                                                          const double *__restrict__ az,
                                                          double *__restrict__ part) {
  Comp v[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = Comp{0, 0};
  const int64_t b0 = blockIdx.x * kNoAllocTile, b1 = min(n, b0 + kNoAllocTile);
  for (int64_t i = b0 + threadIdx.x; i < b1; i += kBlock) {
    const double mu = m[i];
    const double a[3] = {ax[i], ay[i], az[i]};
    const double t[3] = {y[i] * az[i] - z[i] * ay[i], z[i] * ax[i] - x[i] * az[i], x[i] * ay[i] - y[i] * ax[i]};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      nadd(v[d], mu * a[d]);
      nadd(v[3 + d], mu * fabs(a[d]));
      nadd(v[6 + d], mu * t[d]);
      nadd(v[9 + d], mu * fabs(t[d]));
    }
  }
  block_reduce<12>(v);
  if (threadIdx.x == 0)
    for (int k = 0; k < 12; ++k) {
      part[(blockIdx.x * 12 + k) * 2] = v[k].s;
      part[(blockIdx.x * 12 + k) * 2 + 1] = v[k].c;
    }
}

// Device address of g_balance_scratch for the current device, looked up once
// per device (host code cannot use the symbol's name as a device pointer).
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double *g_scratch_ptr[kMaxDevices] = {};

int noalloc_scratch(double **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return FMM_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_balance_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return FMM_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return FMM_OK;
}

}  // namespace
}  // namespace amfmm

extern "C" int fmm_balance_noalloc(const double *x, const double *y, const double *z, const double *m,
                                   const double *ax, const double *ay, const double *az, int64_t n,
                                   double *out, void *cuda_stream) {
  using namespace amfmm;
  if (n < 1 || !x || !y || !z || !m || !ax || !ay || !az || !out) return FMM_EINVAL;
  if (n > kNoAllocTile * kNoAllocMaxTiles) return FMM_ESIZE;
  double *part = nullptr;
  const int rc = noalloc_scratch(&part);
  if (rc != FMM_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int nb = static_cast<int>((n + kNoAllocTile - 1) / kNoAllocTile);
  k_balance_tiles<<<nb, kBlock, 0, st>>>(n, x, y, z, m, ax, ay, az, part);
  if (cudaGetLastError() != cudaSuccess) return FMM_ECUDA;
  k_balance_final<<<1, 32, 0, st>>>(nb, part, out);
  if (cudaGetLastError() != cudaSuccess) return FMM_ECUDA;
  return FMM_OK;
}
