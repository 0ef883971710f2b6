// Slice-level selector network on the device: a two-hidden-layer tanh MLP in FP32 with its own
// forward, backward (chain rule written out per layer) and Adam kernels.
//   H1 = tanh(X W1 + b1), H2 = tanh(H1 W2 + b2), Y = H2 W3 + b3,
//   loss = sum(M (Y - T)^2) / max(1, sum M).
// It maps statistics of an emulated product's operands to log10 of its relative error at every
// slice level; oz_heff_select_levels turns those predictions into per-block levels.  Every
// reduction runs in a fixed order (one thread per output, sequential over the batch), so training
// is bitwise reproducible for a given seed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ozdmrg.h"
#include "oz_internal.cuh"

namespace {

#define ML_CU(call)                                                                 \
  do {                                                                              \
    cudaError_t _e = (call);                                                        \
    if (_e != cudaSuccess)                                                          \
      return oz::api_fail(_e == cudaErrorMemoryAllocation ? OZ_ENOMEM : OZ_ECUDA,   \
                          std::string(#call) + ": " + cudaGetErrorString(_e));      \
  } while (0)

constexpr int T1 = 256;

inline unsigned cdivu(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Z = X W + b (X: B x nin, W: nin x nout), H = tanh(Z) when act, else H = Z.
__global__ void dense_fwd_kernel(const float* __restrict__ X, int B, int nin, const float* __restrict__ W,
                                 const float* __restrict__ b, int nout, int act, float* __restrict__ H) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)B * nout) return;
  const int r = (int)(idx / nout), j = (int)(idx % nout);
  float z = b[j];
  for (int i = 0; i < nin; ++i) z = fmaf(X[(long long)r * nin + i], W[i * nout + j], z);
  H[idx] = act ? tanhf(z) : z;
}

// dY = 2 M (Y - T) / den, per-row partial of M (Y - T)^2 into part[r].
__global__ void loss_grad_kernel(const float* __restrict__ Y, const float* __restrict__ T,
                                 const float* __restrict__ M, int B, int nout, const float* __restrict__ den,
                                 float* __restrict__ dY, float* __restrict__ part) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= B) return;
  float s = 0.0f;
  const float d = *den;
  for (int j = 0; j < nout; ++j) {
    const long long k = (long long)r * nout + j;
    const float e = Y[k] - T[k];
    s = fmaf(M[k] * e, e, s);
    dY[k] = 2.0f * M[k] * e / d;
  }
  part[r] = s;
}

// sum of v[0..n) in a fixed order (one block), optionally clamped below by 1.
__global__ void sum_kernel(const float* __restrict__ v, long long n, int clamp1, float* __restrict__ out) {
  __shared__ float sh[T1];
  float s = 0.0f;
  for (long long i = threadIdx.x; i < n; i += T1) s += v[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = T1 / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = clamp1 ? fmaxf(1.0f, sh[0]) : sh[0];
}

// dW = Xin^T dZ (nin x nout), db = column sums of dZ.
__global__ void dense_bwd_w_kernel(const float* __restrict__ Xin, int B, int nin, const float* __restrict__ dZ,
                                   int nout, float* __restrict__ dW, float* __restrict__ db) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nin * nout) {
    const int i = idx / nout, j = idx % nout;
    float s = 0.0f;
    for (int r = 0; r < B; ++r) s = fmaf(Xin[(long long)r * nin + i], dZ[(long long)r * nout + j], s);
    dW[idx] = s;
  } else if (idx < nin * nout + nout) {
    const int j = idx - nin * nout;
    float s = 0.0f;
    for (int r = 0; r < B; ++r) s += dZ[(long long)r * nout + j];
    db[j] = s;
  }
}

// dZin = (dZ W^T) * (1 - Hin^2)  (tanh'), Hin: B x nin.
__global__ void dense_bwd_x_kernel(const float* __restrict__ dZ, int B, int nout, const float* __restrict__ W,
                                   int nin, const float* __restrict__ Hin, float* __restrict__ dZin) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)B * nin) return;
  const int r = (int)(idx / nin), i = (int)(idx % nin);
  float s = 0.0f;
  for (int j = 0; j < nout; ++j) s = fmaf(dZ[(long long)r * nout + j], W[i * nout + j], s);
  const float h = Hin[idx];
  dZin[idx] = s * (1.0f - h * h);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  m[i] = b1 * m[i] + (1.0f - b1) * g[i];
  v[i] = b2 * v[i] + (1.0f - b2) * g[i] * g[i];
  const float mh = m[i] / c1, vh = v[i] / c2;
  p[i] -= lr * mh / (sqrtf(vh) + eps);
}

// rows idx[0..B) of src (n x w) into dst (B x w)
__global__ void gather_rows_kernel(const float* __restrict__ src, int w, const int* __restrict__ idx, int B,
                                   float* __restrict__ dst) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (long long)B * w) return;
  const int r = (int)(k / w), c = (int)(k % w);
  dst[k] = src[(long long)idx[r] * w + c];
}

unsigned long long splitmix64_host(unsigned long long z) {
  // SplitMix64 (Steele, Lea and Flood, OOPSLA 2014)
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

struct oz_mlp_s {
  int nin = 0, nh = 0, nout = 0, count = 0, cap = 0, t = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  // batch scratch (cap rows)
  float *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *dY = nullptr, *dZ2 = nullptr, *dZ1 = nullptr, *part = nullptr;
  float *den = nullptr, *lossv = nullptr;
  float *Xb = nullptr, *Tb = nullptr, *Mb = nullptr;
  int* idx = nullptr;
  float* W1() { return p; }
  float* b1() { return p + nin * nh; }
  float* W2() { return b1() + nh; }
  float* b2() { return W2() + nh * nh; }
  float* W3() { return b2() + nh; }
  float* b3() { return W3() + nh * nout; }
  int reserve(int B) {
    if (B <= cap) return OZ_OK;
    for (float* q : {H1, H2, Y, dY, dZ2, dZ1, part, Xb, Tb, Mb}) cudaFree(q);
    cudaFree(idx);
    cap = std::max(B, 256);
    ML_CU(cudaMalloc(&H1, (size_t)cap * nh * 4));
    ML_CU(cudaMalloc(&H2, (size_t)cap * nh * 4));
    ML_CU(cudaMalloc(&Y, (size_t)cap * nout * 4));
    ML_CU(cudaMalloc(&dY, (size_t)cap * nout * 4));
    ML_CU(cudaMalloc(&dZ2, (size_t)cap * nh * 4));
    ML_CU(cudaMalloc(&dZ1, (size_t)cap * nh * 4));
    ML_CU(cudaMalloc(&part, (size_t)cap * 4));
    ML_CU(cudaMalloc(&Xb, (size_t)cap * nin * 4));
    ML_CU(cudaMalloc(&Tb, (size_t)cap * nout * 4));
    ML_CU(cudaMalloc(&Mb, (size_t)cap * nout * 4));
    ML_CU(cudaMalloc(&idx, (size_t)cap * 4));
    return OZ_OK;
  }
  int forward(const float* X, int B, float* Yout, cudaStream_t st) {
    dense_fwd_kernel<<<cdivu((long long)B * nh, T1), T1, 0, st>>>(X, B, nin, W1(), b1(), nh, 1, H1);
    dense_fwd_kernel<<<cdivu((long long)B * nh, T1), T1, 0, st>>>(H1, B, nh, W2(), b2(), nh, 1, H2);
    dense_fwd_kernel<<<cdivu((long long)B * nout, T1), T1, 0, st>>>(H2, B, nh, W3(), b3(), nout, 0, Yout);
    ML_CU(cudaGetLastError());
    return OZ_OK;
  }
  // gradients of the loss over B rows into g; loss into lossv[0]
  int backward(const float* X, const float* T, const float* M, int B, cudaStream_t st) {
    if (int rc = forward(X, B, Y, st)) return rc;
    sum_kernel<<<1, T1, 0, st>>>(M, (long long)B * nout, 1, den);
    loss_grad_kernel<<<cdivu(B, T1), T1, 0, st>>>(Y, T, M, B, nout, den, dY, part);
    sum_kernel<<<1, T1, 0, st>>>(part, B, 0, lossv);
    float* gW1 = g;
    float* gb1 = g + nin * nh;
    float* gW2 = gb1 + nh;
    float* gb2 = gW2 + nh * nh;
    float* gW3 = gb2 + nh;
    float* gb3 = gW3 + nh * nout;
    dense_bwd_w_kernel<<<cdivu(nh * nout + nout, T1), T1, 0, st>>>(H2, B, nh, dY, nout, gW3, gb3);
    dense_bwd_x_kernel<<<cdivu((long long)B * nh, T1), T1, 0, st>>>(dY, B, nout, W3(), nh, H2, dZ2);
    dense_bwd_w_kernel<<<cdivu(nh * nh + nh, T1), T1, 0, st>>>(H1, B, nh, dZ2, nh, gW2, gb2);
    dense_bwd_x_kernel<<<cdivu((long long)B * nh, T1), T1, 0, st>>>(dZ2, B, nh, W2(), nh, H1, dZ1);
    dense_bwd_w_kernel<<<cdivu(nin * nh + nh, T1), T1, 0, st>>>(X, B, nin, dZ1, nh, gW1, gb1);
    ML_CU(cudaGetLastError());
    return OZ_OK;
  }
};

extern "C" int oz_mlp_create(int nin, int nhidden, int nout, unsigned long long seed, oz_mlp** out) {
  if (!out) return oz::api_fail(OZ_EINVAL, "out is null");
  *out = nullptr;
  if (nin < 1 || nhidden < 1 || nout < 1 || nin > 4096 || nhidden > 4096 || nout > 4096)
    return oz::api_fail(OZ_EINVAL, "layer sizes must be in 1..4096");
  oz_mlp* n = new oz_mlp_s();
  n->nin = nin;
  n->nh = nhidden;
  n->nout = nout;
  n->count = nin * nhidden + nhidden + nhidden * nhidden + nhidden + nhidden * nout + nout;
  // Xavier-uniform weights from a counter-based generator, zero biases
  std::vector<float> h(n->count, 0.0f);
  auto fill = [&](int off, int fi, int fo) {
    const double a = std::sqrt(6.0 / (fi + fo));
    for (int k = 0; k < fi * fo; ++k) {
      const unsigned long long r = splitmix64_host(seed ^ splitmix64_host((unsigned long long)(off + k)));
      h[off + k] = (float)(a * (2.0 * ((double)(r >> 11) * 0x1.0p-53) - 1.0));
    }
  };
  fill(0, nin, nhidden);
  fill(nin * nhidden + nhidden, nhidden, nhidden);
  fill(nin * nhidden + nhidden + nhidden * nhidden + nhidden, nhidden, nout);
  cudaError_t e = cudaMalloc(&n->p, (size_t)n->count * 4 * 4 + 64);
  if (e != cudaSuccess) {
    delete n;
    return oz::api_fail(OZ_ENOMEM, "oz_mlp_create cudaMalloc");
  }
  n->g = n->p + n->count;
  n->m = n->g + n->count;
  n->v = n->m + n->count;
  n->den = n->v + n->count;
  n->lossv = n->den + 4;
  cudaMemcpy(n->p, h.data(), (size_t)n->count * 4, cudaMemcpyHostToDevice);
  cudaMemset(n->m, 0, (size_t)n->count * 8);
  *out = n;
  return OZ_OK;
}

extern "C" int oz_mlp_destroy(oz_mlp* n) {
  if (!n) return OZ_OK;
  cudaDeviceSynchronize();
  for (float* q : {n->H1, n->H2, n->Y, n->dY, n->dZ2, n->dZ1, n->part, n->Xb, n->Tb, n->Mb}) cudaFree(q);
  cudaFree(n->idx);
  cudaFree(n->p);
  delete n;
  return OZ_OK;
}

extern "C" int oz_mlp_param_count(const oz_mlp* n) { return n ? n->count : 0; }
extern "C" int oz_mlp_nin(const oz_mlp* n) { return n ? n->nin : 0; }
extern "C" int oz_mlp_nout(const oz_mlp* n) { return n ? n->nout : 0; }

extern "C" int oz_mlp_get_params(const oz_mlp* n, float* host) {
  if (!n || !host) return oz::api_fail(OZ_EINVAL, "null argument");
  ML_CU(cudaMemcpy(host, n->p, (size_t)n->count * 4, cudaMemcpyDeviceToHost));
  return OZ_OK;
}

extern "C" int oz_mlp_set_params(oz_mlp* n, const float* host) {
  if (!n || !host) return oz::api_fail(OZ_EINVAL, "null argument");
  ML_CU(cudaMemcpy(n->p, host, (size_t)n->count * 4, cudaMemcpyHostToDevice));
  return OZ_OK;
}

extern "C" int oz_mlp_forward(oz_mlp* n, const float* d_X, int rows, float* d_Y, oz_stream_t stream) {
  if (!n || !d_X || !d_Y) return oz::api_fail(OZ_EINVAL, "null argument");
  if (rows < 0) return oz::api_fail(OZ_EINVAL, "rows must be >= 0");
  if (rows == 0) return OZ_OK;
  if (int rc = n->reserve(rows)) return rc;
  return n->forward(d_X, rows, d_Y, (cudaStream_t)stream);
}

extern "C" int oz_mlp_gradient(oz_mlp* n, const float* d_X, const float* d_T, const float* d_M, int rows, float* loss,
                               float* host_grad, oz_stream_t stream) {
  if (!n || !d_X || !d_T || !d_M || !loss) return oz::api_fail(OZ_EINVAL, "null argument");
  if (rows < 1) return oz::api_fail(OZ_EINVAL, "rows must be positive");
  cudaStream_t st = (cudaStream_t)stream;
  if (int rc = n->reserve(rows)) return rc;
  if (int rc = n->backward(d_X, d_T, d_M, rows, st)) return rc;
  ML_CU(cudaMemcpyAsync(loss, n->lossv, 4, cudaMemcpyDeviceToHost, st));
  float den = 1.0f;
  ML_CU(cudaMemcpyAsync(&den, n->den, 4, cudaMemcpyDeviceToHost, st));
  if (host_grad) ML_CU(cudaMemcpyAsync(host_grad, n->g, (size_t)n->count * 4, cudaMemcpyDeviceToHost, st));
  ML_CU(cudaStreamSynchronize(st));
  *loss /= den;
  return OZ_OK;
}

extern "C" int oz_mlp_train(oz_mlp* n, const float* d_X, const float* d_T, const float* d_M, int rows, int epochs,
                            int batch, float lr, unsigned long long seed, float* final_loss, oz_stream_t stream) {
  if (!n || !d_X || !d_T || !d_M) return oz::api_fail(OZ_EINVAL, "null argument");
  if (rows < 1 || epochs < 0 || batch < 1 || !(lr > 0.0f)) return oz::api_fail(OZ_EINVAL, "bad training arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const int B = std::min(batch, rows);
  if (int rc = n->reserve(B)) return rc;
  std::vector<int> perm(rows);
  for (int i = 0; i < rows; ++i) perm[i] = i;
  unsigned long long ctr = seed;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = rows - 1; i > 0; --i) {  // Fisher-Yates with a counter-based generator
      const unsigned long long r = splitmix64_host(++ctr);
      std::swap(perm[i], perm[(int)(r % (unsigned long long)(i + 1))]);
    }
    for (int b0 = 0; b0 + B <= rows; b0 += B) {
      ML_CU(cudaMemcpyAsync(n->idx, perm.data() + b0, (size_t)B * 4, cudaMemcpyHostToDevice, st));
      gather_rows_kernel<<<cdivu((long long)B * n->nin, T1), T1, 0, st>>>(d_X, n->nin, n->idx, B, n->Xb);
      gather_rows_kernel<<<cdivu((long long)B * n->nout, T1), T1, 0, st>>>(d_T, n->nout, n->idx, B, n->Tb);
      gather_rows_kernel<<<cdivu((long long)B * n->nout, T1), T1, 0, st>>>(d_M, n->nout, n->idx, B, n->Mb);
      if (int rc = n->backward(n->Xb, n->Tb, n->Mb, B, st)) return rc;
      n->t += 1;
      const float c1 = 1.0f - powf(0.9f, (float)n->t), c2 = 1.0f - powf(0.999f, (float)n->t);
      adam_kernel<<<cdivu(n->count, T1), T1, 0, st>>>(n->p, n->g, n->m, n->v, n->count, lr, c1, c2);
      ML_CU(cudaGetLastError());
      // the index buffer is rewritten by the next batch: wait for this one
      ML_CU(cudaStreamSynchronize(st));
    }
  }
  if (final_loss) {
    // loss over the whole set (in chunks of the batch capacity, weighted by mask counts)
    double num = 0.0, den = 0.0;
    for (int b0 = 0; b0 < rows; b0 += B) {
      const int nb = std::min(B, rows - b0);
      float l = 0.0f;
      if (int rc = oz_mlp_gradient(n, d_X + (long long)b0 * n->nin, d_T + (long long)b0 * n->nout,
                                   d_M + (long long)b0 * n->nout, nb, &l, nullptr, stream))
        return rc;
      float d = 1.0f;
      ML_CU(cudaMemcpy(&d, n->den, 4, cudaMemcpyDeviceToHost));
      num += (double)l * d;
      den += d;
    }
    *final_loss = (float)(num / std::max(1.0, den));
  }
  return OZ_OK;
}
