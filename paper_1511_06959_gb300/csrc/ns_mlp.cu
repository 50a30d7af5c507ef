// Learned adjoint-viscosity closure: per-cell features, BF16 tensor-core inference and
// a BF16 training step with an FP32 Adam master copy.
//
// The stabilised adjoint of section "Energy analysis" adds div(lambda sigma_1 grad w_hat)
// with a hand-tuned constant lambda (its automatic estimation is left open in the
// conclusion).  Here lambda(x) = dx^2 softplus(MLP(f(x))) per cell, so that
//   nu(x) = kappa dx^2 sigma_1(x) softplus(MLP(f(x)))
// with a global factor kappa.  Network: 14 -> 64 -> 64 -> 1, GELU, softplus; weights
// BF16, accumulation FP32, hidden activations rounded to BF16 between the two tensor-core
// layers, the last layer an FP32 dot product.
//
// Features f (14 per cell, stored padded to 16 floats): v = S(q_bar)(q - q_bar) / c_bar
// (symmetrised variables about the box-mean primitive state, section "Symmetrization")
// and the 9 central-difference entries of grad u times L / c_bar (L = 1).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "ns_common.cuh"
#include "ns_kernels.h"
#include "ns_mlp.h"

namespace ns {

namespace {

constexpr int RB = 256;
constexpr int RGM = 296;

// a state value as float: the FP64 state rounded (d2f), or the float mirror as it is
// (the mirror holds exactly d2f of the state, so both give the same bits)
__device__ __forceinline__ float ldf(const double* p, size_t o) { return d2f(p[o]); }
__device__ __forceinline__ float ldf(const float* p, size_t o) { return p[o]; }

// ------------------------------------------------------------------------------------
// box means of (rho, u1, u2, u3, p): FP32 per cell, FP64 sums, deterministic
// ------------------------------------------------------------------------------------
template <class TIN>
__global__ void __launch_bounds__(RB) k_box_means(GridDesc g, float gamma, const TIN* __restrict__ w,
                                                  double* partial) {
  __shared__ double sh[5][RB];
  const int b = blockIdx.y;
  const size_t box = (size_t)b * 5 * g.cells;
  double acc[5] = {0, 0, 0, 0, 0};
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < g.cells; i += (long long)gridDim.x * RB) {
    const float r = ldf(w, box + i);
    const float ir = 1.0f / r;
    const float u0 = ldf(w, box + g.cells + i) * ir, u1 = ldf(w, box + 2 * g.cells + i) * ir,
                u2 = ldf(w, box + 3 * g.cells + i) * ir;
    const float p = (gamma - 1.0f) * (ldf(w, box + 4 * g.cells + i) - 0.5f * r * (u0 * u0 + u1 * u1 + u2 * u2));
    acc[0] += f2d(r);
    acc[1] += f2d(u0);
    acc[2] += f2d(u1);
    acc[3] += f2d(u2);
    acc[4] += f2d(p);
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int s = RB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 5) partial[((size_t)b * 5 + threadIdx.x) * gridDim.x + blockIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(RB) k_box_means_final(int nblk, double inv_cells, const double* partial,
                                                        double* qbar) {
  __shared__ double sh[RB];
  const int b = blockIdx.x / 5, q = blockIdx.x % 5;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += RB) s += partial[((size_t)b * 5 + q) * nblk + i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = RB / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) qbar[b * 5 + q] = sh[0] * inv_cells;
}

// ------------------------------------------------------------------------------------
// features
// ------------------------------------------------------------------------------------
template <class TIN>
__global__ void k_features(GridDesc g, Coef<float> c, const TIN* __restrict__ w, const double* qbar,
                           float* __restrict__ feat) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.cells * g.batch) return;
  const long long b = i / g.cells, r = i - b * g.cells;
  const int x = (int)(r % g.nx), y = (int)((r / g.nx) % g.ny), z = (int)(r / g.plane);
  const size_t box = (size_t)b * 5 * g.cells;
  const float gam = c.gamma, gm1 = c.gm1;
  auto vel = [&](int xx, int yy, int zz, float* u) {
    const size_t o = box + (size_t)wrap(zz, g.nz) * g.plane + (size_t)wrap(yy, g.ny) * g.nx + wrap(xx, g.nx);
    const float ir = 1.0f / ldf(w, o);
    u[0] = ldf(w, o + g.cells) * ir;
    u[1] = ldf(w, o + 2 * g.cells) * ir;
    u[2] = ldf(w, o + 3 * g.cells) * ir;
  };
  const size_t o = box + r;
  const float rho = ldf(w, o);
  float u[3];
  vel(x, y, z, u);
  const float p = gm1 * (ldf(w, o + 4 * g.cells) - 0.5f * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  const float rb = (float)qbar[b * 5 + 0], pb = (float)qbar[b * 5 + 4];
  const float cb = sqrtf(gam * pb / rb);
  const float icb = 1.0f / cb;
  float f[16];
  f[0] = cb / (sqrtf(gam) * rb) * (rho - rb) * icb;
#pragma unroll
  for (int k = 0; k < 3; ++k) f[1 + k] = (u[k] - (float)qbar[b * 5 + 1 + k]) * icb;
  f[4] = (-cb / (rb * sqrtf(gam * gm1)) * (rho - rb) + sqrtf(gam / gm1) / (rb * cb) * (p - pb)) * icb;
  float um[3], up[3];
  const int dd[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    vel(x - dd[j][0], y - dd[j][1], z - dd[j][2], um);
    vel(x + dd[j][0], y + dd[j][1], z + dd[j][2], up);
#pragma unroll
    for (int k = 0; k < 3; ++k) f[5 + 3 * k + j] = (up[k] - um[k]) * c.hidx[j] * icb;
  }
  f[14] = 0.0f;
  f[15] = 0.0f;
  float4* out = reinterpret_cast<float4*>(feat + (size_t)i * 16);
#pragma unroll
  for (int q = 0; q < 4; ++q) out[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
}

// ------------------------------------------------------------------------------------
// activations
// ------------------------------------------------------------------------------------
// erf by the rational approximation of Abramowitz & Stegun, formula 7.1.26
// (|error| <= 1.5e-7, below the BF16 resolution of the activations it feeds):
// erf(x) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-x^2), t = 1 / (1 + p x), x >= 0
__device__ __forceinline__ float erf_as(float x) {
  const float ax = fabsf(x);
  const float t = __fdividef(1.0f, fmaf(0.3275911f, ax, 1.0f));
  float q = fmaf(1.061405429f, t, -1.453152027f);
  q = fmaf(q, t, 1.421413741f);
  q = fmaf(q, t, -0.284496736f);
  q = fmaf(q, t, 0.254829592f);
  const float y = fmaf(-q * t, __expf(-ax * ax), 1.0f);
  return copysignf(y, x);
}
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erf_as(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erf_as(z * 0.70710678118654752f)) + z * __expf(-0.5f * z * z) * 0.39894228040143268f;
}
__device__ __forceinline__ float softplus(float y) { return fmaxf(y, 0.0f) + log1pf(expf(-fabsf(y))); }
__device__ __forceinline__ float sigmoid(float y) { return 1.0f / (1.0f + expf(-y)); }
__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&v);
}

// D = A (16x16 bf16, row) * B (16x8 bf16, col) + C, FP32 accumulate
__device__ __forceinline__ void mma_bf16(float d[4], const unsigned a[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ------------------------------------------------------------------------------------
// tensor-core inference: one warp per 16-cell tile; the weights are staged once per CTA
// in shared memory (rows padded so that the B-fragment reads of a warp hit distinct
// banks) and read as B fragments per mma, which keeps the registers, and so the number
// of resident warps that hide the GELU latency, at three CTAs of 256 threads per SM
// ------------------------------------------------------------------------------------
constexpr int W1S = 12;   // padded row stride (32-bit words) of W1t: 16 bf16 = 8 words
constexpr int W2S = 36;   // padded row stride of W2t: 64 bf16 = 32 words

__global__ void __launch_bounds__(256, 3) k_mlp_infer(long long n, MlpView net, const float* __restrict__ feat,
                                                      const float* __restrict__ sigma1, float scale, float limit_nu,
                                                      float* __restrict__ nu, unsigned* err, bool cap) {
  __shared__ unsigned sW1[NH * W1S];
  __shared__ unsigned sW2[NH * W2S];
  __shared__ float sb1[NH], sb2[NH], sw3[NH];
  {
    const unsigned* w1 = reinterpret_cast<const unsigned*>(net.W1t);
    const unsigned* w2 = reinterpret_cast<const unsigned*>(net.W2t);
    for (int i = threadIdx.x; i < NH * 8; i += blockDim.x) sW1[(i >> 3) * W1S + (i & 7)] = w1[i];
    for (int i = threadIdx.x; i < NH * 32; i += blockDim.x) sW2[(i >> 5) * W2S + (i & 31)] = w2[i];
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
      sb1[i] = net.b1[i];
      sb2[i] = net.b2[i];
      sw3[i] = net.w3q[i];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int gq = lane >> 2, tq = lane & 3;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const float b3 = net.b3[0];
  const long long ntiles = (n + 15) / 16;
  for (long long tile = warp; tile < ntiles; tile += nwarps) {
    const long long r0 = tile * 16 + gq, r1 = r0 + 8;
    auto fv = [&](long long r, int k) -> float { return r < n ? feat[(size_t)r * 16 + k] : 0.0f; };
    unsigned a[4];
    a[0] = pack_bf16(fv(r0, 2 * tq), fv(r0, 2 * tq + 1));
    a[1] = pack_bf16(fv(r1, 2 * tq), fv(r1, 2 * tq + 1));
    a[2] = pack_bf16(fv(r0, 2 * tq + 8), fv(r0, 2 * tq + 9));
    a[3] = pack_bf16(fv(r1, 2 * tq + 8), fv(r1, 2 * tq + 9));
    float h1[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int row = (8 * j + gq) * W1S + tq;
      h1[j][0] = h1[j][1] = h1[j][2] = h1[j][3] = 0.0f;
      mma_bf16(h1[j], a, sW1[row], sW1[row + 4]);
      const float c0 = sb1[8 * j + 2 * tq], c1 = sb1[8 * j + 2 * tq + 1];
      h1[j][0] = gelu(h1[j][0] + c0);
      h1[j][1] = gelu(h1[j][1] + c1);
      h1[j][2] = gelu(h1[j][2] + c0);
      h1[j][3] = gelu(h1[j][3] + c1);
    }
    unsigned a2[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      a2[kk][0] = pack_bf16(h1[2 * kk][0], h1[2 * kk][1]);
      a2[kk][1] = pack_bf16(h1[2 * kk][2], h1[2 * kk][3]);
      a2[kk][2] = pack_bf16(h1[2 * kk + 1][0], h1[2 * kk + 1][1]);
      a2[kk][3] = pack_bf16(h1[2 * kk + 1][2], h1[2 * kk + 1][3]);
    }
    float y0 = 0.0f, y1 = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      const int row = (8 * j + gq) * W2S + tq;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) mma_bf16(z, a2[kk], sW2[row + 8 * kk], sW2[row + 8 * kk + 4]);
      const float c0 = sb2[8 * j + 2 * tq], c1 = sb2[8 * j + 2 * tq + 1];
      const float v0 = sw3[8 * j + 2 * tq], v1 = sw3[8 * j + 2 * tq + 1];
      y0 += gelu(z[0] + c0) * v0 + gelu(z[1] + c1) * v1;
      y1 += gelu(z[2] + c0) * v0 + gelu(z[3] + c1) * v1;
    }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
    if (tq == 0) {
      if (r0 < n) nu[r0] = nu_checked(scale * sigma1[r0] * softplus(y0 + b3), limit_nu, cap, err);
      if (r1 < n) nu[r1] = nu_checked(scale * sigma1[r1] * softplus(y1 + b3), limit_nu, cap, err);
    }
  }
}

// ------------------------------------------------------------------------------------
// training: forward + backward of one minibatch chunk of TS samples per CTA, with the
// quantisation points of the inference path; per-CTA gradient partials, then a fixed-
// order reduction and an FP32 Adam update that also rewrites the inference copies.
// Every matrix product (the two layers, the backward through layer 2 and the two
// weight gradients) runs on the tensor cores as BF16 m16n8k16 products with FP32
// accumulation; their operands are the BF16 values of the inference path (inputs,
// weights, hidden activations) and, in the backward pass, the BF16-rounded gradients
// dZ2 and dZ1 of the pre-activations (the bias gradients sum the FP32 ones).
// ------------------------------------------------------------------------------------
constexpr int TS = 64;       // samples per CTA
constexpr int TT = 256;      // threads per CTA (8 warps)
constexpr int LD = NH + 1;   // padded row of the per-sample activations

struct TrainSmem {
  float W1[NF][NH];   // bf16-rounded master weights as float, rows 14, 15 zero
  float W2[NH][LD];
  float b1[NH], b2[NH], w3[NH];
  float X[TS][NF];
  float Z1[TS][LD];
  float H1[TS][LD];   // bf16(gelu(Z1))
  float Z2[TS][LD];
  float D2[TS][LD];   // dZ2
  float D1[TS][LD];   // dZ1
  float dy[TS];
  float b3;
};

// acc += A (rows m0..m0+15, K columns) * B (K rows, columns n0..n0+7) on the tensor
// cores, one warp; A(m, k) = As[m ars + k acs], B(k, n) = Bs[k brs + n bcs] are floats
// in shared memory rounded to BF16 as they are packed into the fragments (the m16n8k16
// layouts: A rows gq and gq + 8, columns 2tq.. of each 16-wide k slice; B columns gq,
// rows 2tq..; the accumulator rows gq, gq + 8 and columns 2tq, 2tq + 1).
__device__ __forceinline__ void mma_tile(const float* As, int ars, int acs, const float* Bs, int brs, int bcs,
                                         int m0, int n0, int K, float acc[4]) {
  const int lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int ka = k0 + 2 * tq;
    const float* r0 = As + (m0 + gq) * ars;
    const float* r1 = As + (m0 + gq + 8) * ars;
    unsigned a[4];
    a[0] = pack_bf16(r0[ka * acs], r0[(ka + 1) * acs]);
    a[1] = pack_bf16(r1[ka * acs], r1[(ka + 1) * acs]);
    a[2] = pack_bf16(r0[(ka + 8) * acs], r0[(ka + 9) * acs]);
    a[3] = pack_bf16(r1[(ka + 8) * acs], r1[(ka + 9) * acs]);
    const float* cb = Bs + (n0 + gq) * bcs;
    const unsigned b0 = pack_bf16(cb[ka * brs], cb[(ka + 1) * brs]);
    const unsigned b1 = pack_bf16(cb[(ka + 8) * brs], cb[(ka + 9) * brs]);
    mma_bf16(acc, a, b0, b1);
  }
}

// the (m, n) accumulator element of fragment slot q (0..3) of this lane
__device__ __forceinline__ void acc_at(int m0, int n0, int q, int& m, int& n) {
  const int lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  m = m0 + gq + (q >= 2 ? 8 : 0);
  n = n0 + 2 * tq + (q & 1);
}

__global__ void __launch_bounds__(TT) k_mlp_train_partial(MlpView net, const float* __restrict__ feat,
                                                          const float* __restrict__ target,
                                                          const int* __restrict__ idx, int n,
                                                          float* __restrict__ partial, float* loss_partial) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smraw);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const float* P = net.master;
  for (int q = tid; q < NF * NH; q += TT) {
    const int k = q / NH, j = q % NH;
    S.W1[k][j] = k < NIN ? bfr(P[OFF_W1 + k * NH + j]) : 0.0f;
  }
  for (int q = tid; q < NH * NH; q += TT) S.W2[q / NH][q % NH] = bfr(P[OFF_W2 + q]);   // [k][j]
  for (int q = tid; q < NH; q += TT) {
    S.b1[q] = P[OFF_B1 + q];
    S.b2[q] = P[OFF_B2 + q];
    S.w3[q] = bfr(P[OFF_W3 + q]);
  }
  if (tid == 0) S.b3 = P[OFF_B3];
  const int s0 = blockIdx.x * TS;
  for (int q = tid; q < TS * NF; q += TT) {
    const int s = q / NF, k = q % NF;
    const int gs = s0 + s;
    S.X[s][k] = (gs < n && k < NIN) ? bfr(feat[(size_t)idx[gs] * 16 + k]) : 0.0f;
  }
  __syncthreads();
  // layer 1: Z1 = X W1 + b1 (64 x 16 by 16 x 64), H1 = bf16(gelu(Z1))
  for (int t = warp; t < (TS / 16) * (NH / 8); t += TT / 32) {
    const int m0 = (t / (NH / 8)) * 16, n0 = (t % (NH / 8)) * 8;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    mma_tile(&S.X[0][0], NF, 1, &S.W1[0][0], NH, 1, m0, n0, NF, acc);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int m, nn;
      acc_at(m0, n0, q, m, nn);
      const float z = acc[q] + S.b1[nn];
      S.Z1[m][nn] = z;
      S.H1[m][nn] = bfr(gelu(z));
    }
  }
  __syncthreads();
  // layer 2: Z2 = H1 W2 + b2 (64 x 64 by 64 x 64)
  for (int t = warp; t < (TS / 16) * (NH / 8); t += TT / 32) {
    const int m0 = (t / (NH / 8)) * 16, n0 = (t % (NH / 8)) * 8;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    mma_tile(&S.H1[0][0], LD, 1, &S.W2[0][0], LD, 1, m0, n0, NH, acc);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int m, nn;
      acc_at(m0, n0, q, m, nn);
      S.Z2[m][nn] = acc[q] + S.b2[nn];
    }
  }
  __syncthreads();
  // output, loss and dL/dy
  if (tid < TS) {
    const int s = tid, gs = s0 + s;
    float y = S.b3;
    for (int k = 0; k < NH; ++k) y += gelu(S.Z2[s][k]) * S.w3[k];
    float d = 0.0f, l = 0.0f;
    if (gs < n) {
      const float r = softplus(y) - target[idx[gs]];
      l = r * r;
      d = 2.0f * r / (float)n * sigmoid(y);
    }
    S.dy[s] = d;
    loss_partial[(size_t)blockIdx.x * TS + s] = l;
  }
  __syncthreads();
  // dZ2 = dy w3 gelu'(Z2)
  for (int q = tid; q < TS * NH; q += TT) {
    const int s = q / NH, j = q % NH;
    S.D2[s][j] = S.dy[s] * S.w3[j] * gelu_grad(S.Z2[s][j]);
  }
  __syncthreads();
  // dZ1 = (bf16(dZ2) W2^T) gelu'(Z1): A(s, j) = D2[s][j], B(j, k) = W2[k][j]
  for (int t = warp; t < (TS / 16) * (NH / 8); t += TT / 32) {
    const int m0 = (t / (NH / 8)) * 16, n0 = (t % (NH / 8)) * 8;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    mma_tile(&S.D2[0][0], LD, 1, &S.W2[0][0], 1, LD, m0, n0, NH, acc);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int m, kk;
      acc_at(m0, n0, q, m, kk);
      S.D1[m][kk] = acc[q] * gelu_grad(S.Z1[m][kk]);
    }
  }
  __syncthreads();
  // weight gradients of this CTA, in parameter order:
  //   dW2[k][j] = sum_s H1[s][k] bf16(dZ2[s][j]),  dW1[k][j] = sum_s X[s][k] bf16(dZ1[s][j])
  float* G = partial + (size_t)blockIdx.x * NPAR;
  for (int t = warp; t < (NH / 16) * (NH / 8); t += TT / 32) {
    const int m0 = (t / (NH / 8)) * 16, n0 = (t % (NH / 8)) * 8;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    mma_tile(&S.H1[0][0], 1, LD, &S.D2[0][0], LD, 1, m0, n0, TS, acc);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int k, j;
      acc_at(m0, n0, q, k, j);
      G[OFF_W2 + k * NH + j] = acc[q];
    }
  }
  if (warp < NH / 8) {
    const int n0 = warp * 8;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    mma_tile(&S.X[0][0], 1, NF, &S.D1[0][0], LD, 1, 0, n0, TS, acc);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int k, j;
      acc_at(0, n0, q, k, j);
      if (k < NIN) G[OFF_W1 + k * NH + j] = acc[q];
    }
  }
  for (int j = tid; j < NH; j += TT) {
    float a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    for (int s = 0; s < TS; ++s) {
      a1 += S.D1[s][j];
      a2 += S.D2[s][j];
      a3 += gelu(S.Z2[s][j]) * S.dy[s];
    }
    G[OFF_B1 + j] = a1;
    G[OFF_B2 + j] = a2;
    G[OFF_W3 + j] = a3;
  }
  if (tid == 0) {
    float a = 0.0f;
    for (int s = 0; s < TS; ++s) a += S.dy[s];
    G[OFF_B3] = a;
  }
}

__global__ void k_mlp_adam(int nblk, MlpView net, const float* __restrict__ partial, int step, float lr,
                           float beta1, float beta2, float eps) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= NPAR) return;
  float g = 0.0f;
  for (int b = 0; b < nblk; ++b) g += partial[(size_t)b * NPAR + q];
  float m = net.m[q] = beta1 * net.m[q] + (1.0f - beta1) * g;
  float v = net.v[q] = beta2 * net.v[q] + (1.0f - beta2) * g * g;
  const float mh = m / (1.0f - powf(beta1, (float)step));
  const float vh = v / (1.0f - powf(beta2, (float)step));
  net.master[q] -= lr * mh / (sqrtf(vh) + eps);
}

// inference copies of the master parameters: transposed BF16 weights, FP32 biases,
// BF16-rounded output weights
__global__ void k_mlp_publish(MlpView net) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const float* P = net.master;
  if (q < NH * 16) {
    const int nn = q / 16, k = q % 16;
    net.W1t[nn * 16 + k] = __float2bfloat16_rn(k < NIN ? P[OFF_W1 + k * NH + nn] : 0.0f);
  }
  if (q < NH * NH) {
    const int nn = q / NH, k = q % NH;
    net.W2t[nn * NH + k] = __float2bfloat16_rn(P[OFF_W2 + k * NH + nn]);
  }
  if (q < NH) {
    net.b1[q] = P[OFF_B1 + q];
    net.b2[q] = P[OFF_B2 + q];
    net.w3q[q] = bfr(P[OFF_W3 + q]);
  }
  if (q == 0) net.b3[0] = P[OFF_B3];
}

__global__ void k_mlp_reset(MlpView net, const float* __restrict__ params) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= NPAR) return;
  net.master[q] = params[q];
  net.m[q] = 0.0f;
  net.v[q] = 0.0f;
}

// mean over the n real samples of the per-sample losses (padding samples hold 0)
__global__ void k_loss_sum(int nslots, int n, const float* __restrict__ lp, float* loss) {
  __shared__ float sh[256];
  float s = 0.0f;
  for (int i = threadIdx.x; i < nslots; i += 256) s += lp[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = sh[0] / (float)n;
}

__global__ void k_label_target(long long n, const float* __restrict__ acc, const float* __restrict__ sig,
                               float dx2, float tmax, float* __restrict__ t) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float v = acc[i] / (dx2 * sig[i] + 1e-30f);
  t[i] = v < tmax ? v : tmax;
}

}  // namespace

cudaError_t launch_label_target(long long n, const float* acc, const float* sig, double dx2, double tmax,
                                float* t, cudaStream_t st) {
  k_label_target<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, acc, sig, (float)dx2, (float)tmax, t);
  count_launch();
  return cudaGetLastError();
}

MlpView mlp_view(void* blob) {
  char* p = (char*)blob;
  MlpView v;
  v.master = (float*)(p + MLP_OFF_MASTER);
  v.m = (float*)(p + MLP_OFF_M);
  v.v = (float*)(p + MLP_OFF_V);
  v.W1t = (__nv_bfloat16*)(p + MLP_OFF_W1T);
  v.W2t = (__nv_bfloat16*)(p + MLP_OFF_W2T);
  v.b1 = (float*)(p + MLP_OFF_VEC);
  v.b2 = v.b1 + NH;
  v.w3q = v.b2 + NH;
  v.b3 = v.w3q + NH;
  return v;
}

template <class TIN>
cudaError_t launch_box_means(const GridDesc& g, double gamma, const TIN* w, double* qbar, double* scratch,
                             cudaStream_t st) {
  k_box_means<TIN><<<dim3(RGM, g.batch), RB, 0, st>>>(g, (float)gamma, w, scratch);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_box_means_final<<<g.batch * 5, RB, 0, st>>>(RGM, 1.0 / (double)g.cells, scratch, qbar);
  count_launch();
  return cudaGetLastError();
}

size_t box_means_scratch_doubles(const GridDesc& g) { return (size_t)5 * RGM * g.batch; }

template <class TIN>
cudaError_t launch_features(const GridDesc& g, const Coef<float>& c, const TIN* w, const double* qbar,
                            float* feat, cudaStream_t st) {
  const long long n = g.cells * g.batch;
  k_features<TIN><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, c, w, qbar, feat);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_box_means<double>(const GridDesc&, double, const double*, double*, double*, cudaStream_t);
template cudaError_t launch_box_means<float>(const GridDesc&, double, const float*, double*, double*, cudaStream_t);
template cudaError_t launch_features<double>(const GridDesc&, const Coef<float>&, const double*, const double*,
                                             float*, cudaStream_t);
template cudaError_t launch_features<float>(const GridDesc&, const Coef<float>&, const float*, const double*,
                                            float*, cudaStream_t);

cudaError_t launch_mlp_infer(long long n, void* blob, const float* feat, const float* sigma1, double scale,
                             double limit_nu, float* nu, unsigned* err, cudaStream_t st, bool cap) {
  const long long tiles = (n + 15) / 16;
  long long blocks = (tiles + 7) / 8;
  if (blocks > 3 * 152) blocks = 3 * 152;   // one wave at three resident CTAs per SM
  if (blocks < 1) blocks = 1;
  k_mlp_infer<<<(unsigned)blocks, 256, 0, st>>>(n, mlp_view(blob), feat, sigma1, (float)scale, (float)limit_nu,
                                                nu, err, cap);
  count_launch();
  return cudaGetLastError();
}

size_t mlp_train_scratch_floats(int n) {
  const int nblk = (n + TS - 1) / TS;
  return (size_t)nblk * NPAR + (size_t)nblk * TS + 16;
}

cudaError_t launch_mlp_train_step(void* blob, const float* feat, const float* target, const int* idx, int n,
                                  int step, double lr, float* scratch, float* loss, cudaStream_t st) {
  const int nblk = (n + TS - 1) / TS;
  MlpView v = mlp_view(blob);
  float* partial = scratch;
  float* lp = scratch + (size_t)nblk * NPAR;
  const size_t smem = sizeof(TrainSmem);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_train_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_mlp_train_partial<<<nblk, TT, smem, st>>>(v, feat, target, idx, n, partial, lp);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (loss) {
    k_loss_sum<<<1, 256, 0, st>>>(nblk * TS, n, lp, loss);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_mlp_adam<<<(NPAR + 255) / 256, 256, 0, st>>>(nblk, v, partial, step, (float)lr, 0.9f, 0.999f, 1e-8f);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_mlp_publish<<<(NH * NH + 255) / 256, 256, 0, st>>>(v);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_mlp_set(void* blob, const float* params, cudaStream_t st) {
  MlpView v = mlp_view(blob);
  k_mlp_reset<<<(NPAR + 255) / 256, 256, 0, st>>>(v, params);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mlp_publish<<<(NH * NH + 255) / 256, 256, 0, st>>>(v);
  count_launch();
  return cudaGetLastError();
}

}  // namespace ns
