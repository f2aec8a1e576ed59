// selector.cu -- a12: a learned pair selector.
//
// The paper notes (Sec. 2) that the modification applies unchanged to pair
// selections driven by an error estimate (Dehnen 2014): every accepted pair
// still interacts mutually, so force and torque stay balanced.  Here the
// estimate is a small network: 8 pair features -> 3 x 64 SiLU -> 1, the
// predicted log10 of the pair's M2L error in units of the partner's monopole
// field (the worse side).  In the walk the opening criterion at theta keeps
// deciding, except in a band: a pair that the criterion rejects at theta but
// accepts at theta_max <= 1 (theta_max = 1 is the safety bound |Z_A - Z_B| >=
// R_A,max + R_B,max), and that holds enough bodies to be worth scoring, is
// accepted when its predicted error -- absolute, or relative to an estimate
// of the field at each side -- is below a target.
//
// Network arithmetic: BF16 inputs and weights on the tensor cores
// (mma.sync m16n8k16, FP32 accumulation); biases, SiLU and the output layer in
// FP32; each layer's FP32 accumulator fragment is re-packed in registers as
// the next layer's BF16 operand fragment.  Training: mean squared error,
// gradients of the inputs of each layer on the tensor cores, gradients of the
// weights in FP32 per block of 64 samples, summed over blocks in a fixed order,
// Adam update of the FP32 master weights.
//
// Parameter layout (FP32, kNParams): W1[64][8], b1[64], W2[64][64], b2[64],
// W3[64][64], b3[64], w4[64], b4, then the feature normalisation mean[8],
// scale[8] (x_norm = (x - mean) * scale).
#include <cuda_bf16.h>

#include <random>
#include <vector>

#include "geom.cuh"
#include "internal.cuh"

namespace amfmm {

constexpr int kH = 64;
constexpr int kF = 8;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kF, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH, kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kH,
              kNWeights = kOffB4 + 1, kOffMean = kNWeights, kOffScale = kOffMean + kF,
              kNParams = kOffScale + kF;

namespace {

// ---------------------------------------------------------------------------
// features and labels
// ---------------------------------------------------------------------------
// Per-cell parts of the features, once per tree: log10 R_max, log10 M,
// log10 of the trace-free quadrupole norm |Q - tr(Q)/3 I| / (M R_max^2) (plus
// 1e-12), and the body count.  A cell of one body, or of zero extent, has no
// quadrupole: its norm is 0.  The norm and its ratio are formed in FP64 (the
// trace removal cancels, and the squared norm of a small cell leaves the
// FP32 range); everything per pair is FP32 (FP64 costs 64 FP32 operations on
// this GPU, and the features only need BF16 accuracy).
__device__ __forceinline__ float lg(float v) { return __log2f(v) * 0.30102999566f; }

__global__ void k_cell_features(int32_t ncell, const double *__restrict__ Rmax, const double *__restrict__ M,
                                const double *__restrict__ mom, int mstride, const int32_t *__restrict__ count,
                                float4 *__restrict__ cf) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const double *q = mom + static_cast<int64_t>(c) * mstride + 4;
  const double tr = (q[0] + q[3] + q[5]) / 3.0;
  const double a = q[0] - tr, d = q[3] - tr, f = q[5] - tr;
  const double n2 = a * a + d * d + f * f + 2.0 * (q[1] * q[1] + q[2] * q[2] + q[4] * q[4]);
  const double den = M[c] * Rmax[c] * Rmax[c];
  const float qn = (count[c] > 1 && den > 0.0) ? static_cast<float>(sqrt(n2) / den) : 0.f;
  const float R = static_cast<float>(Rmax[c]), m = static_cast<float>(M[c]);
  cf[c] = make_float4(lg(R), lg(m), lg(qn + 1e-12f), static_cast<float>(count[c]));
}

// raw features of a pair: log10 of |r|, R_A/|r|, R_B/|r|, M_A, M_B, q_A, q_B,
// N_A + N_B, with the pair ordered by R_max (FP32, descending), then by id,
// so that (A, B) and (B, A) give the same features and decision.  |r| comes
// from the hi + lo float centres.
__device__ __forceinline__ void pair_features(int A, int B, const CellF *__restrict__ zf,
                                              const float4 *__restrict__ cf, float f[kF]) {
  CellF a = zf[A], b = zf[B];
  if (b.h.w > a.h.w || (b.h.w == a.h.w && B < A)) {
    const int t = A;
    A = B;
    B = t;
    const CellF u = a;
    a = b;
    b = u;
  }
  const float4 fa = cf[A], fb = cf[B];
  const float dx = (a.h.x - b.h.x) + (a.l.x - b.l.x);
  const float dy = (a.h.y - b.h.y) + (a.l.y - b.l.y);
  const float dz = (a.h.z - b.h.z) + (a.l.z - b.l.z);
  const float lr = 0.5f * lg(dx * dx + dy * dy + dz * dz + 1e-37f);
  f[0] = lr;
  f[1] = fmaxf(fa.x - lr, -12.f);
  f[2] = fmaxf(fb.x - lr, -12.f);
  f[3] = fa.y;
  f[4] = fb.y;
  f[5] = fa.z;
  f[6] = fb.z;
  f[7] = lg(fa.w + fb.w);
}

__global__ void k_features(int64_t K, const int2 *__restrict__ pairs, const CellF *__restrict__ zf,
                           const float4 *__restrict__ cf, float *__restrict__ feat) {
  const int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (k >= K) return;
  float f[kF];
  pair_features(pairs[k].x, pairs[k].y, zf, cf, f);
#pragma unroll
  for (int q = 0; q < kF; ++q) feat[k * kF + q] = f[q];
}

// Field at every cell for the relative acceptance rule: the monopoles of one
// coarse level (at most 2048 cells), each softened by its own R_max (the
// field of an extended mass, finite inside it), summed in FP32 at the cell's
// centre.  A rough estimate is enough: it only scales the error target.
// Stored as log10 |a|.
constexpr int kFieldTile = 256;

__global__ void __launch_bounds__(kFieldTile) k_field_estimate(int32_t ncell, const CellF *__restrict__ zf,
                                                              const double *__restrict__ M, int32_t k0,
                                                              int32_t k1, float *__restrict__ lga) {
  __shared__ float4 src[kFieldTile];
  __shared__ float eps2[kFieldTile];
  const int c = blockIdx.x * kFieldTile + threadIdx.x;
  float4 me = make_float4(0.f, 0.f, 0.f, 0.f);
  if (c < ncell) me = zf[c].h;
  float ax = 0.f, ay = 0.f, az = 0.f;
  for (int t0 = k0; t0 < k1; t0 += kFieldTile) {
    const int k = t0 + threadIdx.x;
    if (k < k1) {
      const float4 h = zf[k].h;
      src[threadIdx.x] = make_float4(h.x, h.y, h.z, static_cast<float>(M[k]));
      eps2[threadIdx.x] = h.w * h.w;
    }
    __syncthreads();
    const int nt = min(kFieldTile, k1 - t0);
    for (int j = 0; j < nt; ++j) {
      const float4 s = src[j];
      const float e2 = eps2[j];
      const float dx = s.x - me.x, dy = s.y - me.y, dz = s.z - me.z;
      const float r2 = dx * dx + dy * dy + dz * dz + e2;
      if (r2 > 0.f) {
        const float ri = rsqrtf(r2);
        const float w = s.w * ri * ri * ri;
        ax += w * dx;
        ay += w * dy;
        az += w * dz;
      }
    }
    __syncthreads();
  }
  if (c < ncell) lga[c] = lg(sqrtf(ax * ax + ay * ay + az * az) + 1e-30f);
}

// Label of one pair (block per pair): for each side, the rms over its bodies
// of |a_M2L - a_direct| for the interaction of A with B alone (order 3, the
// torque-corrected expansion of Eqs. 3, 4, 7), divided by the monopole field
// of the other cell at that distance (M_B/|r|^2 on A, M_A/|r|^2 on B); the
// label is log10 of the larger of the two, floored at -12.  Taking the worse
// side keeps a small cell's large error from being averaged away by the
// bodies of a big partner.  A side of more than kLabelTargets bodies is
// represented by kLabelTargets of them at evenly spaced sorted positions
// (t n / kLabelTargets), each still summed over every body of the partner,
// so that pairs of big cells can be labelled too.
constexpr int kLabelTargets = 128;

__device__ __forceinline__ int label_target(int t, int n) {
  return n <= kLabelTargets ? t : static_cast<int>((static_cast<int64_t>(t) * n) / kLabelTargets);
}
__global__ void __launch_bounds__(128) k_labels(int64_t K, const int2 *__restrict__ pairs,
                                                const int32_t *__restrict__ begin, const int32_t *__restrict__ count,
                                                const double *__restrict__ X, const double *__restrict__ Y,
                                                const double *__restrict__ Zb, const double *__restrict__ Mb,
                                                const double *__restrict__ Z, const double *__restrict__ loc_pair,
                                                float *__restrict__ label) {
  const int64_t k = blockIdx.x;
  if (k >= K) return;
  int A = pairs[k].x, B = pairs[k].y;
  const double *CA = loc_pair + (2 * k) * 20, *CB = loc_pair + (2 * k + 1) * 20;
  const int bA = begin[A], nA = count[A], bB = begin[B], nB = count[B];
  const int tA = min(nA, kLabelTargets), tB = min(nB, kLabelTargets);
  double errA = 0.0, errB = 0.0;
  for (int t = threadIdx.x; t < tA + tB; t += blockDim.x) {
    const bool onA = t < tA;
    const int i = onA ? bA + label_target(t, nA) : bB + label_target(t - tA, nB);
    const int c = onA ? A : B;
    const double *C = onA ? CA : CB;
    const int ob = onA ? bB : bA, on = onA ? nB : nA;
    const double x[3] = {X[i] - Z[3 * c], Y[i] - Z[3 * c + 1], Zb[i] - Z[3 * c + 2]};
    // order-3 local expansion: g_i = -(C_i + C_ij x_j + C_ijk x_j x_k / 2)
    const double Q[3][3] = {{C[3], C[4], C[5]}, {C[4], C[6], C[7]}, {C[5], C[7], C[8]}};
    const double O[3][3][3] = {{{C[9], C[10], C[11]}, {C[10], C[12], C[13]}, {C[11], C[13], C[14]}},
                               {{C[10], C[12], C[13]}, {C[12], C[15], C[16]}, {C[13], C[16], C[17]}},
                               {{C[11], C[13], C[14]}, {C[13], C[16], C[17]}, {C[14], C[17], C[18]}}};
    double g[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double v = C[d], w = 0.0;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        v += Q[d][j] * x[j];
#pragma unroll
        for (int l = 0; l < 3; ++l) w += O[d][j][l] * x[j] * x[l];
      }
      g[d] = -(v + 0.5 * w);
    }
    double a[3] = {0, 0, 0};
    for (int j = ob; j < ob + on; ++j) {
      const double d0 = X[j] - X[i], d1 = Y[j] - Y[i], d2 = Zb[j] - Zb[i];
      const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
      if (r2 > 0.0) {
        const double s = Mb[j] / (r2 * sqrt(r2));
        a[0] += s * d0;
        a[1] += s * d1;
        a[2] += s * d2;
      }
    }
    const double e0 = g[0] - a[0], e1 = g[1] - a[1], e2 = g[2] - a[2];
    (onA ? errA : errB) += e0 * e0 + e1 * e1 + e2 * e2;
  }
  __shared__ double sh[2][128];
  sh[0][threadIdx.x] = errA;
  sh[1][threadIdx.x] = errB;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double mA = 0, mB = 0;
    for (int j = bA; j < bA + nA; ++j) mA += Mb[j];
    for (int j = bB; j < bB + nB; ++j) mB += Mb[j];
    const double dx = Z[3 * A] - Z[3 * B], dy = Z[3 * A + 1] - Z[3 * B + 1], dz = Z[3 * A + 2] - Z[3 * B + 2];
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double eA = sqrt(sh[0][0] / tA) / (mB / r2), eB = sqrt(sh[1][0] / tB) / (mA / r2);
    // below 1e-12 of the monopole scale the error is FP64 rounding noise
    label[k] = static_cast<float>(fmax(log10(fmax(eA, eB) + 1e-300), -12.0));
  }
}

// ---------------------------------------------------------------------------
// the network on the tensor cores
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// SiLU z sigmoid(z) with sigmoid(z) = (1 + tanh(z/2))/2 on the hardware tanh
// (one special-function operation per activation)
__device__ __forceinline__ float tanh_hw(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sigm(float z) { return fmaf(0.5f, tanh_hw(0.5f * z), 0.5f); }
__device__ __forceinline__ float silu(float z) { return z * sigm(z); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = sigm(z);
  return s * (1.f + z * (1.f - s));
}

// Shared-memory copy of the network: BF16 weights, FP32 biases / output layer.
struct NetSmem {
  __nv_bfloat16 W1[kH][16];  // input width padded to 16
  __nv_bfloat16 W2[kH][kH];
  __nv_bfloat16 W3[kH][kH];
  float b1[kH], b2[kH], b3[kH], w4[kH], b4, mean[kF], scale[kF];
};

__device__ void load_net(NetSmem &s, const float *__restrict__ p) {
  for (int q = threadIdx.x; q < kH * 16; q += blockDim.x) {
    const int o = q / 16, i = q % 16;
    s.W1[o][i] = __float2bfloat16_rn(i < kF ? p[kOffW1 + o * kF + i] : 0.f);
  }
  for (int q = threadIdx.x; q < kH * kH; q += blockDim.x) {
    s.W2[q / kH][q % kH] = __float2bfloat16_rn(p[kOffW2 + q]);
    s.W3[q / kH][q % kH] = __float2bfloat16_rn(p[kOffW3 + q]);
  }
  for (int q = threadIdx.x; q < kH; q += blockDim.x) {
    s.b1[q] = p[kOffB1 + q];
    s.b2[q] = p[kOffB2 + q];
    s.b3[q] = p[kOffB3 + q];
    s.w4[q] = p[kOffW4 + q];
  }
  if (threadIdx.x < kF) {
    s.mean[threadIdx.x] = p[kOffMean + threadIdx.x];
    s.scale[threadIdx.x] = p[kOffScale + threadIdx.x];
  }
  if (threadIdx.x == 0) s.b4 = p[kOffB4];
}

// Per-warp state of 16 samples.  Fragment conventions (m16n8k16): lane =
// 4 g + t; an accumulator tile n holds rows g and g + 8, columns 8 n + 2 t and
// 8 n + 2 t + 1.
struct Act {
  float z[3][8][4];  // pre-activations of the three hidden layers
  float y[2];        // outputs of rows g and g + 8
};

// B fragment of W[o][i] used as B[k = i][n = o] (forward: out = in W^T)
__device__ __forceinline__ void bfrag_fwd(const __nv_bfloat16 (*W)[kH], int kb, int n, int g, int t, uint32_t &b0,
                                          uint32_t &b1) {
  b0 = *reinterpret_cast<const uint32_t *>(&W[8 * n + g][16 * kb + 2 * t]);
  b1 = *reinterpret_cast<const uint32_t *>(&W[8 * n + g][16 * kb + 2 * t + 8]);
}

// forward of 16 samples whose normalised features sit in xs[16][kF]
__device__ void forward16(const NetSmem &s, const float (*xs)[kF], Act &act) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t a[4];
  a[0] = pack_bf16(xs[g][2 * t], xs[g][2 * t + 1]);
  a[1] = pack_bf16(xs[g + 8][2 * t], xs[g + 8][2 * t + 1]);
  a[2] = 0u;
  a[3] = 0u;
  float h[8][4];
  // layer 1 (K = 8, padded to 16)
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    const uint32_t b0 = *reinterpret_cast<const uint32_t *>(&s.W1[8 * n + g][2 * t]);
    mma16816(c, a, b0, 0u);
    const float bb0 = s.b1[8 * n + 2 * t], bb1 = s.b1[8 * n + 2 * t + 1];
    act.z[0][n][0] = c[0] + bb0;
    act.z[0][n][1] = c[1] + bb1;
    act.z[0][n][2] = c[2] + bb0;
    act.z[0][n][3] = c[3] + bb1;
#pragma unroll
    for (int q = 0; q < 4; ++q) h[n][q] = silu(act.z[0][n][q]);
  }
  // layers 2 and 3
#pragma unroll
  for (int L = 1; L < 3; ++L) {
    const __nv_bfloat16(*W)[kH] = L == 1 ? s.W2 : s.W3;
    const float *bias = L == 1 ? s.b2 : s.b3;
    uint32_t A[4][4];
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
      A[kb][0] = pack_bf16(h[2 * kb][0], h[2 * kb][1]);
      A[kb][1] = pack_bf16(h[2 * kb][2], h[2 * kb][3]);
      A[kb][2] = pack_bf16(h[2 * kb + 1][0], h[2 * kb + 1][1]);
      A[kb][3] = pack_bf16(h[2 * kb + 1][2], h[2 * kb + 1][3]);
    }
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kb = 0; kb < 4; ++kb) {
        uint32_t b0, b1;
        bfrag_fwd(W, kb, n, g, t, b0, b1);
        mma16816(c, A[kb], b0, b1);
      }
      const float bb0 = bias[8 * n + 2 * t], bb1 = bias[8 * n + 2 * t + 1];
      act.z[L][n][0] = c[0] + bb0;
      act.z[L][n][1] = c[1] + bb1;
      act.z[L][n][2] = c[2] + bb0;
      act.z[L][n][3] = c[3] + bb1;
#pragma unroll
      for (int q = 0; q < 4; ++q) h[n][q] = silu(act.z[L][n][q]);
    }
  }
  // output layer in FP32: partial dots over this lane's columns, then the
  // four lanes of the row group in a fixed order
  float y0 = 0.f, y1 = 0.f;
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const float w0 = s.w4[8 * n + 2 * t], w1 = s.w4[8 * n + 2 * t + 1];
    y0 += h[n][0] * w0 + h[n][1] * w1;
    y1 += h[n][2] * w0 + h[n][3] * w1;
  }
  y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
  y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
  y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
  y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
  act.y[0] = y0 + s.b4;
  act.y[1] = y1 + s.b4;
}

// Inference forward with the tensor-core B fragments of all three layers in
// registers (loaded once per warp, reused for every group of 16 samples); the
// biases and the output layer stay in shared memory.  Same arithmetic as
// forward16, without keeping the pre-activations.
struct NetRegs {
  uint32_t w1[8];
  uint32_t w2[4][8][2];
  uint32_t w3[4][8][2];
};

__device__ __forceinline__ void load_regs(const NetSmem &s, NetRegs &r) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int n = 0; n < 8; ++n) r.w1[n] = *reinterpret_cast<const uint32_t *>(&s.W1[8 * n + g][2 * t]);
#pragma unroll
  for (int kb = 0; kb < 4; ++kb)
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      bfrag_fwd(s.W2, kb, n, g, t, r.w2[kb][n][0], r.w2[kb][n][1]);
      bfrag_fwd(s.W3, kb, n, g, t, r.w3[kb][n][0], r.w3[kb][n][1]);
    }
}

__device__ __forceinline__ void infer16(const NetSmem &s, const NetRegs &r, const float (*xs)[kF], float &y0,
                                        float &y1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t a[4];
  a[0] = pack_bf16(xs[g][2 * t], xs[g][2 * t + 1]);
  a[1] = pack_bf16(xs[g + 8][2 * t], xs[g + 8][2 * t + 1]);
  a[2] = 0u;
  a[3] = 0u;
  float h[8][4];
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    mma16816(c, a, r.w1[n], 0u);
    const float bb0 = s.b1[8 * n + 2 * t], bb1 = s.b1[8 * n + 2 * t + 1];
    h[n][0] = silu(c[0] + bb0);
    h[n][1] = silu(c[1] + bb1);
    h[n][2] = silu(c[2] + bb0);
    h[n][3] = silu(c[3] + bb1);
  }
#pragma unroll
  for (int L = 1; L < 3; ++L) {
    const float *bias = L == 1 ? s.b2 : s.b3;
    uint32_t A[4][4];
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
      A[kb][0] = pack_bf16(h[2 * kb][0], h[2 * kb][1]);
      A[kb][1] = pack_bf16(h[2 * kb][2], h[2 * kb][3]);
      A[kb][2] = pack_bf16(h[2 * kb + 1][0], h[2 * kb + 1][1]);
      A[kb][3] = pack_bf16(h[2 * kb + 1][2], h[2 * kb + 1][3]);
    }
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kb = 0; kb < 4; ++kb) {
        if (L == 1) mma16816(c, A[kb], r.w2[kb][n][0], r.w2[kb][n][1]);
        else mma16816(c, A[kb], r.w3[kb][n][0], r.w3[kb][n][1]);
      }
      const float bb0 = bias[8 * n + 2 * t], bb1 = bias[8 * n + 2 * t + 1];
      h[n][0] = silu(c[0] + bb0);
      h[n][1] = silu(c[1] + bb1);
      h[n][2] = silu(c[2] + bb0);
      h[n][3] = silu(c[3] + bb1);
    }
  }
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const float w0 = s.w4[8 * n + 2 * t], w1 = s.w4[8 * n + 2 * t + 1];
    s0 += h[n][0] * w0 + h[n][1] * w1;
    s1 += h[n][2] * w0 + h[n][3] * w1;
  }
  s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
  s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
  y0 = s0 + s.b4;
  y1 = s1 + s.b4;
}

// inference over K samples of raw features
__global__ void __launch_bounds__(128) k_mlp_infer(int64_t K, const float *__restrict__ params,
                                                   const float *__restrict__ feat, float *__restrict__ out) {
  __shared__ NetSmem s;
  __shared__ float xs[4][16][kF];
  load_net(s, params);
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (static_cast<int64_t>(blockIdx.x) * 4 + w) * 16;
  if (lane < 16) {
    const int64_t k = base + lane;
#pragma unroll
    for (int q = 0; q < kF; ++q)
      xs[w][lane][q] = k < K ? (feat[k * kF + q] - s.mean[q]) * s.scale[q] : 0.f;
  }
  __syncwarp();
  Act act;
  forward16(s, xs[w], act);
  const int g = lane >> 2;
  if ((lane & 3) == 0) {
    if (base + g < K) out[base + g] = act.y[0];
    if (base + g + 8 < K) out[base + g + 8] = act.y[1];
  }
}

// One minibatch: forward, backward, per-block gradient partials (64 samples a
// block); loss = mean over the batch of (y - label)^2.
struct TrainSmem {
  NetSmem net;
  float xs[4][16][kF];
  float dz[64][kH];   // dL/dz of the current layer, 64 samples
  float hin[64][kH];  // the BF16-rounded input of the current layer (as FP32)
};

__global__ void __launch_bounds__(128) k_mlp_grad(int64_t B, const float *__restrict__ params,
                                                  const float *__restrict__ feat, const float *__restrict__ lab,
                                                  float *__restrict__ part, float *__restrict__ loss_part) {
  extern __shared__ __align__(16) unsigned char raw[];
  TrainSmem &s = *reinterpret_cast<TrainSmem *>(raw);
  load_net(s.net, params);
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t base = static_cast<int64_t>(blockIdx.x) * 64 + w * 16;
  if (lane < 16) {
    const int64_t k = base + lane;
#pragma unroll
    for (int q = 0; q < kF; ++q)
      s.xs[w][lane][q] = k < B ? (feat[k * kF + q] - s.net.mean[q]) * s.net.scale[q] : 0.f;
  }
  __syncwarp();
  Act act;
  forward16(s.net, s.xs[w], act);
  // dL/dy = 2 (y - label) / B for real samples
  const int64_t r0 = base + g, r1 = base + g + 8;
  const float dy0 = r0 < B ? 2.f * (act.y[0] - lab[r0]) / static_cast<float>(B) : 0.f;
  const float dy1 = r1 < B ? 2.f * (act.y[1] - lab[r1]) / static_cast<float>(B) : 0.f;
  float lsum = 0.f;
  if (t == 0) {
    if (r0 < B) lsum += (act.y[0] - lab[r0]) * (act.y[0] - lab[r0]);
    if (r1 < B) lsum += (act.y[1] - lab[r1]) * (act.y[1] - lab[r1]);
  }
  // output layer: dw4 = sum dy h3, db4 = sum dy; dz3 = dy w4 silu'(z3)
  float dz[8][4];
  float* pp = part + static_cast<int64_t>(blockIdx.x) * kNWeights;
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const float w0 = s.net.w4[8 * n + 2 * t], w1 = s.net.w4[8 * n + 2 * t + 1];
    dz[n][0] = dy0 * w0 * silu_grad(act.z[2][n][0]);
    dz[n][1] = dy0 * w1 * silu_grad(act.z[2][n][1]);
    dz[n][2] = dy1 * w0 * silu_grad(act.z[2][n][2]);
    dz[n][3] = dy1 * w1 * silu_grad(act.z[2][n][3]);
  }
  // h3 values for dw4: stage in shared memory, reduce over 64 samples below
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    s.hin[w * 16 + g][8 * n + 2 * t] = silu(act.z[2][n][0]);
    s.hin[w * 16 + g][8 * n + 2 * t + 1] = silu(act.z[2][n][1]);
    s.hin[w * 16 + g + 8][8 * n + 2 * t] = silu(act.z[2][n][2]);
    s.hin[w * 16 + g + 8][8 * n + 2 * t + 1] = silu(act.z[2][n][3]);
  }
  // dy per sample (kept in dz row space: column 0 of a scratch row)
  if (t == 0) {
    s.dz[w * 16 + g][0] = dy0;
    s.dz[w * 16 + g + 8][0] = dy1;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kH + 1; q += blockDim.x) {
    float acc = 0.f;
    for (int r = 0; r < 64; ++r) acc += s.dz[r][0] * (q < kH ? s.hin[r][q] : 1.f);
    pp[q < kH ? kOffW4 + q : kOffB4] = acc;
  }
  __syncthreads();
  // hidden layers 3, 2, 1
#pragma unroll
  for (int L = 2; L >= 0; --L) {
    // stage dz (FP32) and the layer input (BF16-rounded) for the weight gradient
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      s.dz[w * 16 + g][8 * n + 2 * t] = dz[n][0];
      s.dz[w * 16 + g][8 * n + 2 * t + 1] = dz[n][1];
      s.dz[w * 16 + g + 8][8 * n + 2 * t] = dz[n][2];
      s.dz[w * 16 + g + 8][8 * n + 2 * t + 1] = dz[n][3];
    }
    if (L > 0) {
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        s.hin[w * 16 + g][8 * n + 2 * t] = bf16r(silu(act.z[L - 1][n][0]));
        s.hin[w * 16 + g][8 * n + 2 * t + 1] = bf16r(silu(act.z[L - 1][n][1]));
        s.hin[w * 16 + g + 8][8 * n + 2 * t] = bf16r(silu(act.z[L - 1][n][2]));
        s.hin[w * 16 + g + 8][8 * n + 2 * t + 1] = bf16r(silu(act.z[L - 1][n][3]));
      }
    } else if (lane < 16) {
#pragma unroll
      for (int q = 0; q < kF; ++q) s.hin[w * 16 + lane][q] = bf16r(s.xs[w][lane][q]);
    }
    __syncthreads();
    const int nin = L > 0 ? kH : kF;
    const int offW = L == 2 ? kOffW3 : (L == 1 ? kOffW2 : kOffW1);
    const int offB = L == 2 ? kOffB3 : (L == 1 ? kOffB2 : kOffB1);
    for (int q = threadIdx.x; q < kH * nin; q += blockDim.x) {
      const int o = q / nin, i = q % nin;
      float acc = 0.f;
      for (int r = 0; r < 64; ++r) acc += s.dz[r][o] * s.hin[r][i];
      pp[offW + q] = acc;
    }
    for (int o = threadIdx.x; o < kH; o += blockDim.x) {
      float acc = 0.f;
      for (int r = 0; r < 64; ++r) acc += s.dz[r][o];
      pp[offB + o] = acc;
    }
    __syncthreads();
    if (L > 0) {
      // dh_{L-1} = bf16(dz_L) W_L on the tensor cores, then dz_{L-1}
      const __nv_bfloat16(*W)[kH] = L == 2 ? s.net.W3 : s.net.W2;
      uint32_t A[4][4];
#pragma unroll
      for (int kb = 0; kb < 4; ++kb) {
        A[kb][0] = pack_bf16(dz[2 * kb][0], dz[2 * kb][1]);
        A[kb][1] = pack_bf16(dz[2 * kb][2], dz[2 * kb][3]);
        A[kb][2] = pack_bf16(dz[2 * kb + 1][0], dz[2 * kb + 1][1]);
        A[kb][3] = pack_bf16(dz[2 * kb + 1][2], dz[2 * kb + 1][3]);
      }
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
          // B[k = o][n = i] = W[o][i]
          const int o0 = 16 * kb + 2 * t, i0 = 8 * n + g;
          __nv_bfloat162 v0, v1;
          v0.x = W[o0][i0];
          v0.y = W[o0 + 1][i0];
          v1.x = W[o0 + 8][i0];
          v1.y = W[o0 + 9][i0];
          mma16816(c, A[kb], *reinterpret_cast<uint32_t *>(&v0), *reinterpret_cast<uint32_t *>(&v1));
        }
        dz[n][0] = c[0] * silu_grad(act.z[L - 1][n][0]);
        dz[n][1] = c[1] * silu_grad(act.z[L - 1][n][1]);
        dz[n][2] = c[2] * silu_grad(act.z[L - 1][n][2]);
        dz[n][3] = c[3] * silu_grad(act.z[L - 1][n][3]);
      }
    }
    __syncthreads();
  }
  // loss partial: lanes with t == 0 hold row losses; fixed-order sum
  lsum += __shfl_xor_sync(0xffffffffu, lsum, 4);
  lsum += __shfl_xor_sync(0xffffffffu, lsum, 8);
  lsum += __shfl_xor_sync(0xffffffffu, lsum, 16);
  __shared__ float ls[4];
  if (lane == 0) ls[w] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) loss_part[blockIdx.x] = ((ls[0] + ls[1]) + (ls[2] + ls[3]));
}

// gradient = sum of the block partials in block order; loss likewise
__global__ void k_grad_reduce(int nblk, const float *__restrict__ part, const float *__restrict__ loss_part,
                              int64_t B, float *__restrict__ grad, float *__restrict__ loss) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < kNWeights) {
    float acc = 0.f;
    for (int b = 0; b < nblk; ++b) acc += part[static_cast<int64_t>(b) * kNWeights + q];
    grad[q] = acc;
  }
  if (q == 0 && loss) {
    float acc = 0.f;
    for (int b = 0; b < nblk; ++b) acc += loss_part[b];
    *loss = acc / static_cast<float>(B);
  }
}

__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, float lr, float b1, float b2, float eps, int step) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= kNWeights) return;
  const float gg = g[q];
  const float mm = b1 * m[q] + (1.f - b1) * gg;
  const float vv = b2 * v[q] + (1.f - b2) * gg * gg;
  m[q] = mm;
  v[q] = vv;
  const float mh = mm / (1.f - powf(b1, static_cast<float>(step)));
  const float vh = vv / (1.f - powf(b2, static_cast<float>(step)));
  p[q] -= lr * mh / (sqrtf(vh) + eps);
}

// ---------------------------------------------------------------------------
// scoring of the walk's candidate pairs
// ---------------------------------------------------------------------------
// Scoring of the walk's frontier in two steps.  k_band_select marks the
// pairs the network decides: A != B, not accepted by the criterion at the
// floor theta_lo, and accepted by it at theta_hi <= 1 (theta_hi = 1 is the
// safety bound |Z_A - Z_B| >= R_A + R_B), with the walk's own criterion (FP32
// filter, exact FP64 for close calls).  It sets score = +inf for every pair
// and appends the marked ones to a candidate list (warp-aggregated).  The
// list's order varies from run to run, but a pair's score depends only on the
// pair (the rows of a tensor-core product are independent), so the walk does
// not.  k_walk_scores then runs the network on the candidates only.
__global__ void k_band_select(const long long *__restrict__ nf_dev, int64_t cap, const int2 *__restrict__ front,
                              const double4_32a *__restrict__ zr, const CellF *__restrict__ zf,
                              const int32_t *__restrict__ count, int64_t min_work, double th_lo, double th_hi,
                              float *__restrict__ score, int32_t *__restrict__ cand, unsigned *__restrict__ ncand) {
  // the frontier size comes from the walk's generation record; a frontier
  // beyond the buffers (the walk then stops and runs again) is not scored
  const int64_t nf = min(static_cast<int64_t>(*nf_dev), cap);
  const int lane = threadIdx.x & 31;
  for (int64_t base = blockIdx.x * static_cast<int64_t>(blockDim.x); base < nf;
       base += static_cast<int64_t>(gridDim.x) * blockDim.x) {
  const int64_t t = base + threadIdx.x;
  bool ok = false;
  if (t < nf) {
    score[t] = INFINITY;
    const int A = front[t].x, B = front[t].y;
    // a pair of few bodies costs less to open than to score
    if (A != B && static_cast<int64_t>(count[A]) * count[B] >= min_work) {
      const float th2f_lo = static_cast<float>(th_lo) * static_cast<float>(th_lo);
      const float th2f_hi = static_cast<float>(th_hi) * static_cast<float>(th_hi);
      const CellF fa = zf[A], fb = zf[B];
      int hi = separated_fast(fa, fb, th2f_hi);
      if (hi < 0) hi = well_separated(zr[A], zr[B], th_hi);
      if (hi) {
        int lo = separated_fast(fa, fb, th2f_lo);
        if (lo < 0) lo = well_separated(zr[A], zr[B], th_lo);
        ok = !lo;
      }
    }
  }
  const unsigned m = __ballot_sync(0xffffffffu, ok);
  if (m != 0u) {
    unsigned at = 0;
    if (lane == 0) at = atomicAdd(ncand, static_cast<unsigned>(__popc(m)));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (ok) cand[at + __popc(m & ((1u << lane) - 1u))] = static_cast<int32_t>(t);
  }
  }
}

// The network on the candidates, 16 per warp step; persistent blocks stage
// the network in shared memory once, every warp then holds its tensor-core
// fragments in registers.  The score is the predicted absolute error of the
// pair relative to the field at each side, in log10: the network predicts
// the larger side's error in units of the partner's monopole field M/r^2, so
// side A's error is at most 10^pred M_B/r^2, side B's 10^pred M_A/r^2, and
//   score = pred + log10 max(M_B / (r^2 |a_A|), M_A / (r^2 |a_B|)),
// compared by the walk with log10 of the relative target.
__global__ void __launch_bounds__(128) k_walk_scores(const int2 *__restrict__ front,
                                                     const int32_t *__restrict__ cand,
                                                     const unsigned *__restrict__ ncand,
                                                     const float *__restrict__ params,
                                                     const CellF *__restrict__ zf, const float4 *__restrict__ cf,
                                                     const float *__restrict__ lga, float *__restrict__ score,
                                                     unsigned long long *__restrict__ scored) {
  __shared__ NetSmem s;
  __shared__ float xs[4][16][kF];
  __shared__ float adj[4][16];
  const int64_t K = *ncand;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(scored, static_cast<unsigned long long>(K));
  // the grid is sized for the largest frontier: a block with no candidate
  // group leaves before it stages the network (36 KB per block, at every
  // generation of the walk)
  if (static_cast<int64_t>(blockIdx.x) * 4 * 16 >= K) return;
  load_net(s, params);
  __syncthreads();
  NetRegs wr;
  load_regs(s, wr);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2;
  for (int64_t grp = static_cast<int64_t>(blockIdx.x) * 4 + w; grp * 16 < K;
       grp += static_cast<int64_t>(gridDim.x) * 4) {
    const int64_t base = grp * 16;
    if (lane < 16) {
      float f[kF] = {0, 0, 0, 0, 0, 0, 0, 0};
      float ad = 0.f;
      if (base + lane < K) {
        const int2 pr = front[cand[base + lane]];
        pair_features(pr.x, pr.y, zf, cf, f);
        const float l2r = 2.f * f[0];
        ad = lga ? fmaxf(cf[pr.y].y - l2r - lga[pr.x], cf[pr.x].y - l2r - lga[pr.y])
                 : fmaxf(cf[pr.y].y, cf[pr.x].y) - l2r;
      }
      adj[w][lane] = ad;
#pragma unroll
      for (int q = 0; q < kF; ++q) xs[w][lane][q] = (f[q] - s.mean[q]) * s.scale[q];
    }
    __syncwarp();
    float y0, y1;
    infer16(s, wr, xs[w], y0, y1);
    if ((lane & 3) == 0) {
      if (base + g < K) score[cand[base + g]] = y0 + adj[w][g];
      if (base + g + 8 < K) score[cand[base + g + 8]] = y1 + adj[w][g + 8];
    }
    __syncwarp();
  }
}

__global__ void k_gather_batch(int64_t B, const int64_t *__restrict__ perm, int64_t start, int64_t n,
                               const float *__restrict__ X, const float *__restrict__ y, float *__restrict__ xb,
                               float *__restrict__ yb) {
  const int64_t b = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (b >= B) return;
  const int64_t i = perm[(start + b) % n];
#pragma unroll
  for (int q = 0; q < kF; ++q) xb[b * kF + q] = X[i * kF + q];
  yb[b] = y[i];
}

}  // namespace

int cell_features(fmm_ctx *c) {
  const int64_t nc = c->sz.ncell;
  AMFMM_TRY(ensure<float4>(c, c->sel_cellfeat, nc));
  k_cell_features<<<grid_for(nc, 256), 256, 0, c->stream>>>(static_cast<int32_t>(nc), ptr<double>(c->Rmax),
                                                           ptr<double>(c->M), ptr<double>(c->mom),
                                                           mom_stride(c->opts.order_P), ptr<int32_t>(c->count),
                                                           ptr<float4>(c->sel_cellfeat));
  return launched(c, "cell_features");
}

int field_estimate(fmm_ctx *c) {
  const int64_t nc = c->sz.ncell;
  // the coarse level: the last one before the first level with more than
  // 2048 cells (deep levels can be small again, but hold only a dense core)
  int L = 0;
  for (int l = 0; l <= c->sz.depth; ++l) {
    if (c->sz.lvl_off[l + 1] - c->sz.lvl_off[l] > 2048) break;
    L = l;
  }
  AMFMM_TRY(ensure<float>(c, c->sel_lga, nc));
  k_field_estimate<<<grid_for(nc, kFieldTile), kFieldTile, 0, c->stream>>>(
      static_cast<int32_t>(nc), ptr<CellF>(c->walk_zf), ptr<double>(c->M), static_cast<int32_t>(c->sz.lvl_off[L]),
      static_cast<int32_t>(c->sz.lvl_off[L + 1]), ptr<float>(c->sel_lga));
  return launched(c, "field_estimate");
}

int walk_scores(fmm_ctx *c, const long long *nf_dev, int64_t cap, const int2 *front, float *score) {
  cudaStream_t st = c->stream;
  unsigned *ncand = reinterpret_cast<unsigned *>(ptr<int64_t>(c->totals) + 11);
  AMFMM_CUDA(c, cudaMemsetAsync(ncand, 0, sizeof(unsigned), st));
  const double lo = c->opts.theta, hi = c->sel_theta_max;
  // persistent grids: the frontier size is only known on the device
  k_band_select<<<static_cast<unsigned>(c->num_sms * 8), 256, 0, st>>>(
      nf_dev, cap, front, ptr<double4_32a>(c->walk_zr), ptr<CellF>(c->walk_zf), ptr<int32_t>(c->count),
      c->sel_min_work, lo, hi, score, ptr<int32_t>(c->sel_cand), ncand);
  AMFMM_TRY(launched(c, "band_select"));
  const unsigned g = static_cast<unsigned>(c->num_sms * 4);
  k_walk_scores<<<g, 128, 0, st>>>(front, ptr<int32_t>(c->sel_cand), ncand, ptr<float>(c->sel_params),
                                   ptr<CellF>(c->walk_zf), ptr<float4>(c->sel_cellfeat),
                                   c->sel_rule == FMM_SEL_RELATIVE ? ptr<float>(c->sel_lga) : nullptr,
                                   score, ptr<unsigned long long>(c->totals) + 10);
  return launched(c, "walk_scores");
}

}  // namespace amfmm

using namespace amfmm;

extern "C" {

int fmm_selector_nparams(void) { return kNParams; }

int fmm_selector_set(fmm_ctx *c, const float *params, double log10_target, double theta_max, int64_t min_work,
                     int rule, int enable) {
  if (!c) return FMM_EINVAL;
  if (enable) {
    if (!params) return set_error(c, FMM_EINVAL, "NULL parameters");
    if (rule != FMM_SEL_ABSOLUTE && rule != FMM_SEL_RELATIVE)
      return set_error(c, FMM_EINVAL, "unknown selector rule %d", rule);
    if (!(theta_max > 0.0 && theta_max <= 1.0))
      return set_error(c, FMM_EINVAL, "theta_max must lie in (0, 1] (got %g)", theta_max);
    AMFMM_TRY(ensure<float>(c, c->sel_params, kNParams));
    AMFMM_CUDA(c, cudaMemcpyAsync(c->sel_params.p, params, sizeof(float) * kNParams, cudaMemcpyHostToDevice,
                                  c->stream));
    AMFMM_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  c->sel_enabled = enable != 0;
  c->sel_log10_target = log10_target;
  if (enable) {
    c->sel_theta_max = theta_max;
    c->sel_min_work = min_work < 0 ? 0 : min_work;
    c->sel_rule = rule;
  }
  c->stage = kNone;
  return FMM_OK;
}

int fmm_selector_samples(fmm_ctx *c, const int32_t *pairs, int64_t K, float *feat, float *label) {
  if (!c) return FMM_EINVAL;
  if (c->stage < kUp) return set_error(c, FMM_EORDER, "fmm_selector_samples needs fmm_upward first");
  if (c->opts.order_P != 3) return set_error(c, FMM_EUNSUPPORTED, "samples are built at order 3");
  if (K < 0 || (K > 0 && (!pairs || !feat))) return set_error(c, FMM_EINVAL, "bad sample arguments");
  if (K == 0) return FMM_OK;
  cudaStream_t st = c->stream;
  const int2 *pp = reinterpret_cast<const int2 *>(pairs);
  AMFMM_TRY(pack_walk_cells(c));
  AMFMM_TRY(cell_features(c));
  k_features<<<grid_for(K, 256), 256, 0, st>>>(K, pp, ptr<CellF>(c->walk_zf), ptr<float4>(c->sel_cellfeat), feat);
  AMFMM_TRY(launched(c, "features"));
  if (label) {
    // the pairs' order-3 TC locals, then the per-pair errors
    AMFMM_TRY(ensure<double>(c, c->sel_scratch, static_cast<size_t>(K) * 40));
    AMFMM_TRY(pair_locals_tc(c, pp, K, ptr<double>(c->sel_scratch)));
    k_labels<<<static_cast<unsigned>(K), 128, 0, st>>>(K, pp, ptr<int32_t>(c->begin), ptr<int32_t>(c->count),
                                                         ptr<double>(c->X), ptr<double>(c->Y), ptr<double>(c->Zb),
                                                         ptr<double>(c->Mb), ptr<double>(c->Z),
                                                         ptr<double>(c->sel_scratch), label);
    AMFMM_TRY(launched(c, "labels"));
  }
  return FMM_OK;
}

int fmm_mlp_forward(fmm_ctx *c, const float *params, const float *feat, int64_t K, float *out) {
  if (!c || !params || K < 0) return FMM_EINVAL;
  if (K == 0) return FMM_OK;
  k_mlp_infer<<<grid_for(K, 64), 128, 0, c->stream>>>(K, params, feat, out);
  return launched(c, "mlp_infer");
}

int fmm_mlp_grad(fmm_ctx *c, const float *params, const float *feat, const float *label, int64_t B, float *grad,
                 float *loss) {
  if (!c || !params || !feat || !label || !grad || B < 1) return FMM_EINVAL;
  const int nblk = static_cast<int>((B + 63) / 64);
  AMFMM_TRY(ensure<float>(c, c->sel_part, static_cast<size_t>(nblk) * kNWeights + nblk + 8));
  float *part = ptr<float>(c->sel_part);
  float *lpart = part + static_cast<size_t>(nblk) * kNWeights;
  const size_t shm = sizeof(TrainSmem);
  // per function and device, so set on every launch (a host-side call)
  AMFMM_CUDA(c, cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(shm)));
  k_mlp_grad<<<nblk, 128, shm, c->stream>>>(B, params, feat, label, part, lpart);
  AMFMM_TRY(launched(c, "mlp_grad"));
  k_grad_reduce<<<grid_for(kNWeights, 256), 256, 0, c->stream>>>(nblk, part, lpart, B, grad, loss);
  return launched(c, "grad_reduce");
}

int fmm_mlp_adam(fmm_ctx *c, float *params, float *m, float *v, const float *grad, float lr, int step) {
  if (!c || !params || !m || !v || !grad || step < 1) return FMM_EINVAL;
  k_adam<<<grid_for(kNWeights, 256), 256, 0, c->stream>>>(params, m, v, grad, lr, 0.9f, 0.999f, 1e-8f, step);
  return launched(c, "adam");
}

// Adam on minibatches drawn in the order of one seeded permutation of the
// samples (wrapping around), one device step per minibatch.
int fmm_selector_train(fmm_ctx *c, float *params, float *adam, const float *X, const float *y, int64_t n, int batch,
                       int steps, float lr, unsigned long long seed, float *loss_out) {
  if (!c || !params || !adam || !X || !y || n < 1 || batch < 1 || steps < 0) return FMM_EINVAL;
  std::vector<int64_t> perm(static_cast<size_t>(n));
  for (int64_t i = 0; i < n; ++i) perm[static_cast<size_t>(i)] = i;
  std::mt19937_64 rng(seed);
  for (int64_t i = n - 1; i > 0; --i) {
    std::uniform_int_distribution<int64_t> d(0, i);
    std::swap(perm[static_cast<size_t>(i)], perm[static_cast<size_t>(d(rng))]);
  }
  AMFMM_TRY(ensure<int64_t>(c, c->sel_perm, static_cast<size_t>(n)));
  AMFMM_CUDA(c, cudaMemcpyAsync(c->sel_perm.p, perm.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, c->stream));
  AMFMM_TRY(ensure<float>(c, c->sel_xb, static_cast<size_t>(batch) * kF));
  AMFMM_TRY(ensure<float>(c, c->sel_yb, static_cast<size_t>(batch)));
  AMFMM_TRY(ensure<float>(c, c->sel_grad, static_cast<size_t>(kNWeights) + 1 + static_cast<size_t>(steps)));
  float *grad = ptr<float>(c->sel_grad);
  float *losses = grad + kNWeights + 1;
  for (int s = 0; s < steps; ++s) {
    k_gather_batch<<<grid_for(batch, 256), 256, 0, c->stream>>>(batch, ptr<int64_t>(c->sel_perm),
                                                                static_cast<int64_t>(s) * batch, n, X, y,
                                                                ptr<float>(c->sel_xb), ptr<float>(c->sel_yb));
    AMFMM_TRY(launched(c, "gather_batch"));
    AMFMM_TRY(fmm_mlp_grad(c, params, ptr<float>(c->sel_xb), ptr<float>(c->sel_yb), batch, grad, losses + s));
    AMFMM_TRY(fmm_mlp_adam(c, params, adam, adam + kNWeights, grad, lr, s + 1));
  }
  if (loss_out && steps > 0)
    AMFMM_CUDA(c, cudaMemcpyAsync(loss_out, losses, sizeof(float) * steps, cudaMemcpyDeviceToHost, c->stream));
  AMFMM_CUDA(c, cudaStreamSynchronize(c->stream));
  return FMM_OK;
}

}  // extern "C"
