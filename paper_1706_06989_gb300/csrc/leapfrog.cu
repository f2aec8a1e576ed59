// leapfrog.cu -- a14: uniform kick-drift-kick leapfrog driven by the solver.
//
// Sec. 4 of the paper: momentum and angular momentum are conserved only when
// every body advances with the same time step.  With uniform steps the
// kick-drift-kick leapfrog changes the total linear momentum by
// dt * sum m a (zero when the forces balance, Eq. "unit") and the total
// angular momentum by dt * sum m X x a (zero when the torques balance, Eq. 7
// or 8); a drift leaves both unchanged (it adds V dt to X, and V x V = 0).
// The driver records both totals after every step so that their drift can
// be measured.
#include "internal.cuh"

namespace amfmm {
namespace {

constexpr int kBlock = 256;

__global__ void k_kick(int64_t n, double h, const double *__restrict__ ax, const double *__restrict__ ay,
                       const double *__restrict__ az, double *__restrict__ vx, double *__restrict__ vy,
                       double *__restrict__ vz) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  vx[i] += h * ax[i];
  vy[i] += h * ay[i];
  vz[i] += h * az[i];
}

__global__ void k_drift(int64_t n, double dt, const double *__restrict__ vx, const double *__restrict__ vy,
                        const double *__restrict__ vz, double *__restrict__ x, double *__restrict__ y,
                        double *__restrict__ z) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  x[i] += dt * vx[i];
  y[i] += dt * vy[i];
  z[i] += dt * vz[i];
}

struct Comp {
  double s, c;
};
__device__ __forceinline__ void nadd(Comp &a, double v) {
  const double t = a.s + v;
  if (fabs(a.s) >= fabs(v)) a.c += (a.s - t) + v;
  else a.c += (v - t) + a.s;
  a.s = t;
}

// per-block compensated partials of P = sum m V and L = sum m X x V
__global__ void __launch_bounds__(kBlock) k_momentum_partial(int64_t n, const double *__restrict__ x,
                                                             const double *__restrict__ y,
                                                             const double *__restrict__ z,
                                                             const double *__restrict__ vx,
                                                             const double *__restrict__ vy,
                                                             const double *__restrict__ vz,
                                                             const double *__restrict__ m,
                                                             double *__restrict__ part) {
  Comp v[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) v[k] = Comp{0, 0};
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = blockIdx.x * per, b1 = min(n, b0 + per);
  for (int64_t i = b0 + threadIdx.x; i < b1; i += kBlock) {
    const double mu = m[i];
    nadd(v[0], mu * vx[i]);
    nadd(v[1], mu * vy[i]);
    nadd(v[2], mu * vz[i]);
    nadd(v[3], mu * (y[i] * vz[i] - z[i] * vy[i]));
    nadd(v[4], mu * (z[i] * vx[i] - x[i] * vz[i]));
    nadd(v[5], mu * (x[i] * vy[i] - y[i] * vx[i]));
  }
  __shared__ double sh[6][2][kBlock];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    sh[k][0][threadIdx.x] = v[k].s;
    sh[k][1][threadIdx.x] = v[k].c;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int k = threadIdx.x;
    Comp a{0, 0};
    for (int t = 0; t < kBlock; ++t) {
      nadd(a, sh[k][0][t]);
      a.c += sh[k][1][t];
    }
    part[(blockIdx.x * 6 + k) * 2] = a.s;
    part[(blockIdx.x * 6 + k) * 2 + 1] = a.c;
  }
}

__global__ void k_momentum_final(int nb, const double *__restrict__ part, double *__restrict__ out) {
  if (threadIdx.x >= 6 || blockIdx.x != 0) return;
  const int k = threadIdx.x;
  Comp a{0, 0};
  for (int b = 0; b < nb; ++b) {
    nadd(a, part[(b * 6 + k) * 2]);
    a.c += part[(b * 6 + k) * 2 + 1];
  }
  out[k] = a.s + a.c;
}

int momentum(fmm_ctx *c, const double *x, const double *y, const double *z, const double *vx, const double *vy,
             const double *vz, const double *m, int64_t n, double *out) {
  const int nb = static_cast<int>(std::min<int64_t>(c->num_sms * 2, (n + kBlock - 1) / kBlock));
  AMFMM_TRY(ensure<double>(c, c->diag, static_cast<size_t>(nb) * 12 + 8));
  double *part = ptr<double>(c->diag);
  k_momentum_partial<<<nb, kBlock, 0, c->stream>>>(n, x, y, z, vx, vy, vz, m, part);
  AMFMM_TRY(launched(c, "momentum_partial"));
  k_momentum_final<<<1, 32, 0, c->stream>>>(nb, part, out);
  return launched(c, "momentum_final");
}

}  // namespace
}  // namespace amfmm

using namespace amfmm;

extern "C" int fmm_leapfrog(fmm_ctx *c, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                            const double *m, int64_t n, double dt, int nsteps, double *ax, double *ay,
                            double *az, double *mom) {
  if (!c) return FMM_EINVAL;
  if (n < 1 || nsteps < 0 || !(dt == dt)) return set_error(c, FMM_EINVAL, "bad leapfrog arguments");
  if (!x || !y || !z || !vx || !vy || !vz || !m || !ax || !ay || !az)
    return set_error(c, FMM_EINVAL, "NULL array");
  cudaStream_t st = c->stream;
  const unsigned g = grid_for(n, kBlock);
  const double h = 0.5 * dt;
  if (mom) AMFMM_TRY(momentum(c, x, y, z, vx, vy, vz, m, n, mom));
  AMFMM_TRY(fmm_solve(c, x, y, z, m, n, ax, ay, az));
  for (int s = 0; s < nsteps; ++s) {
    k_kick<<<g, kBlock, 0, st>>>(n, h, ax, ay, az, vx, vy, vz);
    AMFMM_TRY(launched(c, "kick"));
    k_drift<<<g, kBlock, 0, st>>>(n, dt, vx, vy, vz, x, y, z);
    AMFMM_TRY(launched(c, "drift"));
    AMFMM_TRY(fmm_solve(c, x, y, z, m, n, ax, ay, az));
    k_kick<<<g, kBlock, 0, st>>>(n, h, ax, ay, az, vx, vy, vz);
    AMFMM_TRY(launched(c, "kick"));
    if (mom) AMFMM_TRY(momentum(c, x, y, z, vx, vy, vz, m, n, mom + 6 * static_cast<int64_t>(s + 1)));
  }
  return FMM_OK;
}
