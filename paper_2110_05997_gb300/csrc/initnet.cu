// Learned initialiser: a multilayer perceptron that maps a compressed core
// (zero-padded to 16 x 16 x 16, divided by its norm) and the rank (one-hot,
// R <= 8) to initial factor matrices for dGN on that core (up to 16 x 8 per
// mode).  The thesis initialises dGN from random factors or from the
// compressed core itself (Sec. 4.1.2); this network is an extra initial
// guess, trained on cores and CPDs produced by the method, with the MLSVD
// start kept as fallback by the solver.
//
//   x (4104, padded to 4160) -> h1 = relu(W1 x + b1) (512)
//                            -> h2 = relu(W2 h1 + b2) (512)
//                            -> y  = W3 h2 + b3 (384 = 3 modes x 8 terms x 16 rows)
//
// Parameters, one FP32 vector: W1 (512 x 4160, row-major) | b1 | W2 (512 x 512)
// | b2 | W3 (384 x 512) | b3.  All products run on the BF16 tensor-core GEMM
// (k_gemm_tc); the loss gradient, bias gradients and Adam are small kernels
// here.  Losses: masked mean squared error against given factors,
// L = sum mask (y - t)^2 / sum mask, or the reconstruction error of the input
// core by the proposed factors (no targets needed).
#include <math.h>
#include <stdint.h>

#include "kernels.h"

namespace cpdk {
namespace {

constexpr int kIn = CPD_INITNET_IN, kInPad = CPD_INITNET_IN_PAD, kH = CPD_INITNET_HIDDEN, kOut = CPD_INITNET_OUT;
constexpr size_t oW1 = 0, ob1 = oW1 + (size_t)kH * kInPad, oW2 = ob1 + kH, ob2 = oW2 + (size_t)kH * kH,
                 oW3 = ob2 + kH, ob3 = oW3 + (size_t)kOut * kH, kParams = ob3 + kOut;

struct Act {                    // activations and backward buffers in the workspace (floats)
  float *h1, *h2, *y, *dy, *dh2, *dh1;
  double* red;
};

size_t act_floats(int B) { return (size_t)B * (2 * kH + 2 * kOut + 2 * kH) + 64; }

Act carve_act(void* ws, int B) {
  float* p = static_cast<float*>(ws);
  Act a{};
  a.red = reinterpret_cast<double*>(p); p += 64;
  a.h1 = p; p += (size_t)B * kH;
  a.h2 = p; p += (size_t)B * kH;
  a.y = p; p += (size_t)B * kOut;
  a.dy = p; p += (size_t)B * kOut;
  a.dh2 = p; p += (size_t)B * kH;
  a.dh1 = p; p += (size_t)B * kH;
  return a;
}

GemmArgs gemm(const float* A, long long sam, long long sak, const float* B, long long sbn, long long sbk, float* D,
              long long ldd, int M, int N, int K) {
  GemmArgs g{};
  g.A = A; g.sam = sam; g.sak = sak; g.B = B; g.sbn = sbn; g.sbk = sbk; g.D = D; g.ldd = ldd;
  g.M = M; g.N = N; g.K = K;
  return g;
}

cudaError_t forward(const float* P, const float* X, int B, const Act& a, float* y, cudaStream_t st) {
  GemmArgs g = gemm(X, kInPad, 1, P + oW1, kInPad, 1, a.h1, kH, B, kH, kIn);
  g.bias = P + ob1; g.relu = 1;
  cudaError_t e = launch_gemm_tc(g, st);
  if (e != cudaSuccess) return e;
  g = gemm(a.h1, kH, 1, P + oW2, kH, 1, a.h2, kH, B, kH, kH);
  g.bias = P + ob2; g.relu = 1;
  if ((e = launch_gemm_tc(g, st)) != cudaSuccess) return e;
  g = gemm(a.h2, kH, 1, P + oW3, kH, 1, y, kOut, B, kOut, kH);
  g.bias = P + ob3;
  return launch_gemm_tc(g, st);
}

// dy = 2 mask (y - t) / sum(mask); red[0] = sum mask (y - t)^2, red[1] = sum mask
__global__ void k_mask_sum(const float* __restrict__ mask, long long n, double* red) {
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += mask[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(red + 1, s);
}

__global__ void k_loss_grad(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ mask,
                            long long n, const double* msum, float* dy, double* red) {
  const double denom = msum[1] > 0.0 ? msum[1] : 1.0;
  const float scale = (float)(2.0 / denom);
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = (y[i] - t[i]) * mask[i];
    dy[i] = scale * d;
    s += (double)d * (double)d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(red, s / denom);
}

// Reconstruction loss of the normalised cores in X by the proposed factors
// in Y (the CP objective on each core, Sec. 3.1):
//   L = (1/B) sum_b ||S_b - sum_r a_r (x) b_r (x) c_r||^2,
// and dL/dy = -(2/B) [E_(l) (Khatri-Rao of the other two factors)] under the
// mask (the CP gradient, Sec. 3.1).  One CTA per sample: the 16^3 core and
// then its residual E in shared memory, one thread per output entry.
__global__ void __launch_bounds__(256) k_recon_grad(const float* __restrict__ X, const float* __restrict__ Y,
                                                    const float* __restrict__ mask, int B, float* dy, double* red) {
  __shared__ float E[4096];
  __shared__ float W[3][16][8];
  __shared__ float part[8];
  const int b = blockIdx.x, tid = threadIdx.x;
  const float* x = X + (size_t)b * kInPad;
  const float* y = Y + (size_t)b * kOut;
  const float* m = mask + (size_t)b * kOut;
  for (int e = tid; e < 4096; e += blockDim.x) E[e] = x[e];
  for (int e = tid; e < kOut; e += blockDim.x) {
    const int l = e >> 7, r = (e >> 4) & 7, i = e & 15;
    W[l][i][r] = y[e] * m[e];
  }
  __syncthreads();
  float sq = 0.f;
  for (int e = tid; e < 4096; e += blockDim.x) {
    const int i = e & 15, j = (e >> 4) & 15, k = e >> 8;
    float v = E[e];
#pragma unroll
    for (int r = 0; r < 8; ++r) v = fmaf(-W[0][i][r] * W[1][j][r], W[2][k][r], v);
    E[e] = v;
    sq = fmaf(v, v, sq);
  }
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((tid & 31) == 0) part[tid >> 5] = sq;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    atomicAdd(red, (double)t / B);
  }
  const float scale = -2.f / (float)B;
  for (int e = tid; e < kOut; e += blockDim.x) {
    const int l = e >> 7, r = (e >> 4) & 7, i = e & 15;
    float acc = 0.f;
    if (m[e] != 0.f) {
      if (l == 0) {
        for (int q = 0; q < 256; ++q) { const int j = q & 15, k = q >> 4; acc = fmaf(E[i + 16 * j + 256 * k], W[1][j][r] * W[2][k][r], acc); }
      } else if (l == 1) {
        for (int q = 0; q < 256; ++q) { const int i0 = q & 15, k = q >> 4; acc = fmaf(E[i0 + 16 * i + 256 * k], W[0][i0][r] * W[2][k][r], acc); }
      } else {
        for (int q = 0; q < 256; ++q) { const int i0 = q & 15, j = q >> 4; acc = fmaf(E[i0 + 16 * j + 256 * i], W[0][i0][r] * W[1][j][r], acc); }
      }
    }
    dy[(size_t)b * kOut + e] = scale * acc * m[e];
  }
}

// db[n] = sum_b d[b, n] for a row-major B x N matrix: one thread per column
__global__ void k_colsum(const float* __restrict__ d, int B, int N, float* db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += d[(size_t)b * N + n];
  db[n] = s;
}

__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi; v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

size_t initnet_param_count() { return kParams; }
size_t initnet_act_bytes(int B) { return act_floats(B) * sizeof(float); }

cudaError_t initnet_forward(const float* P, const float* X, int B, void* ws, float* y, cudaStream_t st) {
  const Act a = carve_act(ws, B);
  return forward(P, X, B, a, y, st);
}

cudaError_t initnet_grad(const float* P, const float* X, const float* t, const float* mask, int B, void* ws,
                         float* G, double* loss_out, cudaStream_t st) {
  const Act a = carve_act(ws, B);
  cudaError_t e = forward(P, X, B, a, a.y, st);
  if (e != cudaSuccess) return e;
  const long long ny = (long long)B * kOut;
  if ((e = cudaMemsetAsync(a.red, 0, 2 * sizeof(double), st)) != cudaSuccess) return e;
  if (t != nullptr) {                       // masked mean squared error against t
    k_mask_sum<<<64, 256, 0, st>>>(mask, ny, a.red);
    k_loss_grad<<<64, 256, 0, st>>>(a.y, t, mask, ny, a.red, a.dy, a.red);
    count_launch(2);
  } else {                                  // reconstruction error of the input cores
    k_recon_grad<<<B, 256, 0, st>>>(X, a.y, mask, B, a.dy, a.red);
    count_launch();
  }
  // layer 3
  GemmArgs g = gemm(a.dy, 1, kOut, a.h2, 1, kH, G + oW3, kH, kOut, kH, B);
  if ((e = launch_gemm_tc(g, st)) != cudaSuccess) return e;
  k_colsum<<<(kOut + 127) / 128, 128, 0, st>>>(a.dy, B, kOut, G + ob3);
  count_launch();
  g = gemm(a.dy, kOut, 1, P + oW3, 1, kH, a.dh2, kH, B, kH, kOut);
  g.mask = a.h2; g.ldm = kH;
  if ((e = launch_gemm_tc(g, st)) != cudaSuccess) return e;
  // layer 2
  g = gemm(a.dh2, 1, kH, a.h1, 1, kH, G + oW2, kH, kH, kH, B);
  if ((e = launch_gemm_tc(g, st)) != cudaSuccess) return e;
  k_colsum<<<(kH + 127) / 128, 128, 0, st>>>(a.dh2, B, kH, G + ob2);
  count_launch();
  g = gemm(a.dh2, kH, 1, P + oW2, 1, kH, a.dh1, kH, B, kH, kH);
  g.mask = a.h1; g.ldm = kH;
  if ((e = launch_gemm_tc(g, st)) != cudaSuccess) return e;
  // layer 1 (the padding columns of X are zero, so their gradient is zero)
  g = gemm(a.dh1, 1, kH, X, 1, kInPad, G + oW1, kInPad, kH, kInPad, B);
  if ((e = launch_gemm_tc(g, st)) != cudaSuccess) return e;
  k_colsum<<<(kH + 127) / 128, 128, 0, st>>>(a.dh1, B, kH, G + ob1);
  count_launch();
  if (loss_out) {
    if ((e = cudaMemcpyAsync(loss_out, a.red, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t initnet_adam(float* P, float* m, float* v, const float* G, int step, double lr, double b1, double b2,
                         double eps, cudaStream_t st) {
  const float c1 = (float)(1.0 - pow(b1, step)), c2 = (float)(1.0 - pow(b2, step));
  k_adam<<<4 * 152, 256, 0, st>>>(P, m, v, G, (long long)kParams, (float)lr, (float)b1, (float)b2, (float)eps, c1, c2);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cpdk

using namespace cpdk;

extern "C" {

size_t cpd_initnet_param_count(void) { return initnet_param_count(); }

size_t cpd_initnet_workspace_size(int B) { return B < 1 ? 0 : initnet_act_bytes(B); }

int cpd_initnet_forward(const float* params, const float* X, int B, float* Y, void* workspace, size_t ws_bytes,
                        void* stream) {
  if (B < 1 || !params || !X || !Y || !workspace) return CPD_ERR_INVALID_ARG;
  if (ws_bytes < initnet_act_bytes(B)) return CPD_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ProfScope ps(st, "initnet_forward");
  return initnet_forward(params, X, B, workspace, Y, st) == cudaSuccess ? CPD_OK : CPD_ERR_CUDA;
}

int cpd_initnet_grad(const float* params, const float* X, const float* target, const float* mask, int B,
                     float* grad, double* loss_dev, void* workspace, size_t ws_bytes, void* stream) {
  if (B < 1 || !params || !X || !mask || !grad || !workspace) return CPD_ERR_INVALID_ARG;
  if (ws_bytes < initnet_act_bytes(B)) return CPD_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ProfScope ps(st, "initnet_grad");
  return initnet_grad(params, X, target, mask, B, workspace, grad, loss_dev, st) == cudaSuccess ? CPD_OK
                                                                                                  : CPD_ERR_CUDA;
}

int cpd_initnet_adam(float* params, float* m, float* v, const float* grad, int step, double lr, double beta1,
                     double beta2, double eps, void* stream) {
  if (!params || !m || !v || !grad || step < 1 || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) ||
      !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
    return CPD_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return initnet_adam(params, m, v, grad, step, lr, beta1, beta2, eps, st) == cudaSuccess ? CPD_OK : CPD_ERR_CUDA;
}

int cpd_gemm_bf16(int M, int N, int K, const float* A, int64_t sam, int64_t sak, const float* B, int64_t sbn,
                  int64_t sbk, float* D, int64_t ldd, const float* bias, int relu, const float* mask, int64_t ldm,
                  int accumulate, void* stream) {
  if (M < 0 || N < 0 || K < 0 || (M > 0 && N > 0 && (!D || (K > 0 && (!A || !B))))) return CPD_ERR_INVALID_ARG;
  GemmArgs g{};
  g.A = A; g.sam = sam; g.sak = sak; g.B = B; g.sbn = sbn; g.sbk = sbk; g.D = D; g.ldd = ldd;
  g.bias = bias; g.relu = relu; g.mask = mask; g.ldm = ldm; g.accumulate = accumulate;
  g.M = M; g.N = N; g.K = K;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ProfScope ps(st, "gemm_bf16_tc");
  return launch_gemm_tc(g, st) == cudaSuccess ? CPD_OK : CPD_ERR_CUDA;
}

}  // extern "C"
