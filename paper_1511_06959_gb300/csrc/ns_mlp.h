// Internal layout of the learned-closure network.
//
// Parameter order of the FP32 master array (NPAR floats): W1[14][64] (input-major),
// b1[64], W2[64][64] (input-major), b2[64], w3[64], b3.  A network blob holds the
// master parameters, the two Adam moments and the inference copies (transposed BF16
// weight matrices, FP32 biases, BF16-rounded output weights), each region 256-byte
// aligned.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

#include "ns_common.cuh"

namespace ns {

constexpr int NIN = 14, NH = 64, NF = 16;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + NIN * NH;
constexpr int OFF_W2 = OFF_B1 + NH;
constexpr int OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH;
constexpr int OFF_B3 = OFF_W3 + NH;
constexpr int NPAR = OFF_B3 + 1;

constexpr size_t mlp_align(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t MLP_OFF_MASTER = 0;
constexpr size_t MLP_OFF_M = mlp_align(NPAR * 4);
constexpr size_t MLP_OFF_V = MLP_OFF_M + mlp_align(NPAR * 4);
constexpr size_t MLP_OFF_W1T = MLP_OFF_V + mlp_align(NPAR * 4);
constexpr size_t MLP_OFF_W2T = MLP_OFF_W1T + mlp_align(NH * 16 * 2);
constexpr size_t MLP_OFF_VEC = MLP_OFF_W2T + mlp_align(NH * NH * 2);
constexpr size_t MLP_BYTES = MLP_OFF_VEC + mlp_align((3 * NH + 1) * 4);

struct MlpView {
  float* master;
  float* m;
  float* v;
  __nv_bfloat16* W1t;   // [64][16]: W1t[n][k] = bf16(W1[k][n]), k = 14, 15 zero
  __nv_bfloat16* W2t;   // [64][64]: W2t[n][k] = bf16(W2[k][n])
  float* b1;
  float* b2;
  float* w3q;
  float* b3;
};

MlpView mlp_view(void* blob);
template <class TIN>
cudaError_t launch_box_means(const GridDesc& g, double gamma, const TIN* w, double* qbar, double* scratch,
                             cudaStream_t st);
size_t box_means_scratch_doubles(const GridDesc& g);
template <class TIN>
cudaError_t launch_features(const GridDesc& g, const Coef<float>& c, const TIN* w, const double* qbar,
                            float* feat, cudaStream_t st);
cudaError_t launch_mlp_infer(long long n, void* blob, const float* feat, const float* sigma1, double scale,
                             double limit_nu, float* nu, unsigned* err, cudaStream_t st, bool cap = false);
size_t mlp_train_scratch_floats(int n);
cudaError_t launch_mlp_train_step(void* blob, const float* feat, const float* target, const int* idx, int n,
                                  int step, double lr, float* scratch, float* loss, cudaStream_t st);
cudaError_t launch_mlp_set(void* blob, const float* params, cudaStream_t st);
cudaError_t launch_label_target(long long n, const float* acc, const float* sig, double dx2, double tmax,
                                float* t, cudaStream_t st);

}  // namespace ns
