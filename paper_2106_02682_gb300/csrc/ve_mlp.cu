// ve_mlp.cu -- the multilayer perceptron of the learned warm start: forward, backward and Adam
// kernels (float32) behind the ve_mlp_* entry points of include/ve.h.
//
// Network: a_0 = x; a_l = tanh(W_l a_{l-1} + b_l) for the hidden layers; y = W_L a_{L-1} + b_L.
// Loss: mean over samples and outputs of (y - t)^2 / 2.  Parameters are stored layer by layer,
// W_l (rows = outputs, row-major) then b_l.  Batches are small (tens to hundreds of samples,
// widths of hundreds), so one tiled float32 GEMM kernel serves every product.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/ve.h"

namespace {

constexpr int TILE = 16;

// C[M x N] = op(A) op(B) (+ bias[n]) (tanh if act), with op(A) M x K, op(B) K x N.
// A is row-major with leading dimension lda; transA reads A^T.  Same for B.
__global__ void k_gemm(int M, int N, int K, const float* __restrict__ A, int lda, int transA,
                       const float* __restrict__ B, int ldb, int transB, float* C, int ldc,
                       const float* __restrict__ bias, int act, float beta) {
  __shared__ float As[TILE][TILE + 1];
  __shared__ float Bs[TILE][TILE + 1];
  const int row = blockIdx.y * TILE + threadIdx.y;
  const int col = blockIdx.x * TILE + threadIdx.x;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += TILE) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    float a = 0.f, b = 0.f;
    if (row < M && ka < K) a = transA ? A[(long)ka * lda + row] : A[(long)row * lda + ka];
    if (kb < K && col < N) b = transB ? B[(long)col * ldb + kb] : B[(long)kb * ldb + col];
    As[threadIdx.y][threadIdx.x] = a;
    Bs[threadIdx.y][threadIdx.x] = b;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TILE; ++k) acc = fmaf(As[threadIdx.y][k], Bs[k][threadIdx.x], acc);
    __syncthreads();
  }
  if (row < M && col < N) {
    if (bias) acc += bias[col];
    if (act) acc = tanhf(acc);
    float* c = C + (long)row * ldc + col;
    *c = beta != 0.f ? beta * (*c) + acc : acc;
  }
}

// d = (y - t) * scale.  One CTA of 256 threads also forms sum (y - t)^2 into loss[0] in a fixed
// order (thread-strided partial sums, then a tree), so the reported loss is reproducible bit for
// bit; the gradient itself never depended on an order of atomics.
__global__ void k_out_grad(int n, const float* y, const float* t, float* d, float scale,
                           float* loss) {
  __shared__ float red[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float r = y[i] - t[i];
    d[i] = r * scale;
    s += r * r;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[0] = red[0];
}

// dz = da * (1 - a^2)  (tanh derivative, in place on da)
__global__ void k_tanh_back(int n, const float* a, float* da) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    da[i] *= 1.f - a[i] * a[i];
}

// db[j] = sum_r dz[r, j]
__global__ void k_colsum(int rows, int cols, const float* dz, float* db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += dz[(long)r * cols + j];
  db[j] = s;
}

__global__ void k_adam(int n, float* p, const float* g, float* m, float* v, float lr, float b1,
                       float b2, float c1, float c2, float eps) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

struct ve_mlp {
  int n_in = 0, n_hidden = 0, n_layers = 0, n_out = 0;
  std::vector<int> din, dout;     // per layer (hidden layers then the output layer)
  std::vector<size_t> woff, boff; // parameter offsets
  size_t np = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // device
  long adam_t = 0;
  // batch buffers (device), sized for `cap` samples
  int cap = 0;
  float *x = nullptr, *t = nullptr, *loss = nullptr;
  std::vector<float*> act;  // activations a_0 .. a_L (a_L = output)
  float *d0 = nullptr, *d1 = nullptr;  // gradient ping-pong buffers
  cudaStream_t s = nullptr;
};

namespace {

void mlp_free_batch(ve_mlp* m) {
  for (size_t l = 1; l < m->act.size(); ++l)  // act[0] is m->x, freed below
    if (m->act[l]) cudaFree(m->act[l]);
  m->act.clear();
  if (m->x) cudaFree(m->x);
  if (m->t) cudaFree(m->t);
  if (m->d0) cudaFree(m->d0);
  if (m->d1) cudaFree(m->d1);
  m->x = m->t = m->d0 = m->d1 = nullptr;
  m->cap = 0;
}

int mlp_reserve(ve_mlp* m, int n) {
  if (n <= m->cap) return VE_OK;
  mlp_free_batch(m);
  const int L = m->n_layers + 1;
  int widest = m->n_in;
  for (int l = 0; l < L; ++l) widest = m->dout[l] > widest ? m->dout[l] : widest;
  if (cudaMalloc(&m->x, sizeof(float) * n * m->n_in) != cudaSuccess) return VE_ENOMEM;
  if (cudaMalloc(&m->t, sizeof(float) * n * m->n_out) != cudaSuccess) return VE_ENOMEM;
  if (cudaMalloc(&m->d0, sizeof(float) * n * widest) != cudaSuccess) return VE_ENOMEM;
  if (cudaMalloc(&m->d1, sizeof(float) * n * widest) != cudaSuccess) return VE_ENOMEM;
  m->act.assign(L + 1, nullptr);
  m->act[0] = m->x;
  for (int l = 0; l < L; ++l)
    if (cudaMalloc(&m->act[l + 1], sizeof(float) * n * m->dout[l]) != cudaSuccess) return VE_ENOMEM;
  m->cap = n;
  return VE_OK;
}

cudaError_t gemm(cudaStream_t s, int M, int N, int K, const float* A, int lda, int tA,
                 const float* B, int ldb, int tB, float* C, int ldc, const float* bias, int act,
                 float beta = 0.f) {
  dim3 blk(TILE, TILE), grd((N + TILE - 1) / TILE, (M + TILE - 1) / TILE);
  k_gemm<<<grd, blk, 0, s>>>(M, N, K, A, lda, tA, B, ldb, tB, C, ldc, bias, act, beta);
  return cudaGetLastError();
}

cudaError_t forward(ve_mlp* m, int n) {
  const int L = m->n_layers + 1;
  for (int l = 0; l < L; ++l) {
    // a_{l+1} = act(a_l W_l^T + b_l): (n x din) (din x dout)
    cudaError_t e = gemm(m->s, n, m->dout[l], m->din[l], m->act[l], m->din[l], 0, m->p + m->woff[l],
                         m->din[l], 1, m->act[l + 1], m->dout[l], m->p + m->boff[l], l < L - 1 ? 1 : 0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Gradient of the loss into m->g; loss sum of squares into m->loss[0].
cudaError_t backward(ve_mlp* m, int n) {
  const int L = m->n_layers + 1;
  cudaError_t e = cudaMemsetAsync(m->loss, 0, sizeof(float), m->s);
  if (e != cudaSuccess) return e;
  const int no = n * m->n_out;
  const float scale = 1.f / (float)no;
  k_out_grad<<<1, 256, 0, m->s>>>(no, m->act[L], m->t, m->d0, scale, m->loss);
  float* dz = m->d0;
  float* other = m->d1;
  for (int l = L - 1; l >= 0; --l) {
    // dW_l = dz^T a_l : (dout x n)(n x din);  db_l = colsum(dz)
    e = gemm(m->s, m->dout[l], m->din[l], n, dz, m->dout[l], 1, m->act[l], m->din[l], 0,
             m->g + m->woff[l], m->din[l], nullptr, 0);
    if (e != cudaSuccess) return e;
    k_colsum<<<(m->dout[l] + 255) / 256, 256, 0, m->s>>>(n, m->dout[l], dz, m->g + m->boff[l]);
    if (l == 0) break;
    // da_l = dz W_l : (n x dout)(dout x din); then dz_l = da_l (1 - a_l^2)
    e = gemm(m->s, n, m->din[l], m->dout[l], dz, m->dout[l], 0, m->p + m->woff[l], m->din[l], 0,
             other, m->din[l], nullptr, 0);
    if (e != cudaSuccess) return e;
    const int cnt = n * m->din[l];
    k_tanh_back<<<(cnt + 255) / 256, 256, 0, m->s>>>(cnt, m->act[l], other);
    float* tmp = dz;
    dz = other;
    other = tmp;
  }
  return cudaGetLastError();
}

// splitmix64: deterministic initial weights, uniform in +-sqrt(6 / (din + dout)) (Glorot)
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int ve_mlp_create(int n_in, int n_hidden, int n_layers, int n_out, unsigned long long seed,
                  ve_mlp** out) {
  if (!out || n_in < 1 || n_hidden < 1 || n_layers < 1 || n_out < 1) return VE_EINVAL;
  *out = nullptr;
  ve_mlp* m = new (std::nothrow) ve_mlp();
  if (!m) return VE_ENOMEM;
  m->n_in = n_in;
  m->n_hidden = n_hidden;
  m->n_layers = n_layers;
  m->n_out = n_out;
  const int L = n_layers + 1;
  size_t off = 0;
  for (int l = 0; l < L; ++l) {
    const int di = l == 0 ? n_in : n_hidden, dd = l == L - 1 ? n_out : n_hidden;
    m->din.push_back(di);
    m->dout.push_back(dd);
    m->woff.push_back(off);
    off += (size_t)di * dd;
    m->boff.push_back(off);
    off += dd;
  }
  m->np = off;
  std::vector<float> h(off, 0.f);
  uint64_t st = seed;
  for (int l = 0; l < L; ++l) {
    const float lim = sqrtf(6.f / (float)(m->din[l] + m->dout[l]));
    for (size_t i = 0; i < (size_t)m->din[l] * m->dout[l]; ++i) {
      const double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
      h[m->woff[l] + i] = (float)((2.0 * u - 1.0) * lim);
    }
  }
  if (cudaStreamCreateWithFlags(&m->s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&m->p, sizeof(float) * off) != cudaSuccess ||
      cudaMalloc(&m->g, sizeof(float) * off) != cudaSuccess ||
      cudaMalloc(&m->m, sizeof(float) * off) != cudaSuccess ||
      cudaMalloc(&m->v, sizeof(float) * off) != cudaSuccess ||
      cudaMalloc(&m->loss, sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    ve_mlp_destroy(m);
    return VE_ENOMEM;
  }
  if (cudaMemcpy(m->p, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->m, 0, sizeof(float) * off) != cudaSuccess ||
      cudaMemset(m->v, 0, sizeof(float) * off) != cudaSuccess) {
    ve_mlp_destroy(m);
    return VE_ECUDA;
  }
  *out = m;
  return VE_OK;
}

void ve_mlp_destroy(ve_mlp* m) {
  if (!m) return;
  if (m->s) cudaStreamSynchronize(m->s);
  mlp_free_batch(m);
  if (m->p) cudaFree(m->p);
  if (m->g) cudaFree(m->g);
  if (m->m) cudaFree(m->m);
  if (m->v) cudaFree(m->v);
  if (m->loss) cudaFree(m->loss);
  if (m->s) cudaStreamDestroy(m->s);
  delete m;
}

size_t ve_mlp_num_params(const ve_mlp* m) { return m ? m->np : 0; }

int ve_mlp_get_params(ve_mlp* m, float* host, size_t count) {
  if (!m || !host || count != m->np) return VE_EINVAL;
  if (cudaMemcpyAsync(host, m->p, sizeof(float) * count, cudaMemcpyDeviceToHost, m->s) != cudaSuccess ||
      cudaStreamSynchronize(m->s) != cudaSuccess)
    return VE_ECUDA;
  return VE_OK;
}

int ve_mlp_set_params(ve_mlp* m, const float* host, size_t count) {
  if (!m || !host || count != m->np) return VE_EINVAL;
  if (cudaMemcpyAsync(m->p, host, sizeof(float) * count, cudaMemcpyHostToDevice, m->s) != cudaSuccess ||
      cudaMemsetAsync(m->m, 0, sizeof(float) * count, m->s) != cudaSuccess ||
      cudaMemsetAsync(m->v, 0, sizeof(float) * count, m->s) != cudaSuccess ||
      cudaStreamSynchronize(m->s) != cudaSuccess)
    return VE_ECUDA;
  m->adam_t = 0;
  return VE_OK;
}

int ve_mlp_loss_grad(ve_mlp* m, const float* x, const float* t, int n, float* loss, float* grad) {
  cudaGetLastError();  // report only errors raised by this call
  if (!m || !x || !t || n < 1) return VE_EINVAL;
  int r = mlp_reserve(m, n);
  if (r != VE_OK) return r;
  if (cudaMemcpyAsync(m->x, x, sizeof(float) * n * m->n_in, cudaMemcpyHostToDevice, m->s) != cudaSuccess ||
      cudaMemcpyAsync(m->t, t, sizeof(float) * n * m->n_out, cudaMemcpyHostToDevice, m->s) != cudaSuccess ||
      forward(m, n) != cudaSuccess || backward(m, n) != cudaSuccess)
    return VE_ECUDA;
  float sq = 0.f;
  if (cudaMemcpyAsync(&sq, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->s) != cudaSuccess) return VE_ECUDA;
  if (grad && cudaMemcpyAsync(grad, m->g, sizeof(float) * m->np, cudaMemcpyDeviceToHost, m->s) != cudaSuccess)
    return VE_ECUDA;
  if (cudaStreamSynchronize(m->s) != cudaSuccess) return VE_ECUDA;
  if (loss) *loss = 0.5f * sq / (float)(n * m->n_out);
  return VE_OK;
}

int ve_mlp_train(ve_mlp* m, const float* x, const float* t, int n, int steps, float lr,
                 float* loss_out) {
  cudaGetLastError();  // report only errors raised by this call
  if (!m || !x || !t || n < 1 || steps < 0 || !(lr > 0.f)) return VE_EINVAL;
  int r = mlp_reserve(m, n);
  if (r != VE_OK) return r;
  if (cudaMemcpyAsync(m->x, x, sizeof(float) * n * m->n_in, cudaMemcpyHostToDevice, m->s) != cudaSuccess ||
      cudaMemcpyAsync(m->t, t, sizeof(float) * n * m->n_out, cudaMemcpyHostToDevice, m->s) != cudaSuccess)
    return VE_ECUDA;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int np = (int)m->np;
  for (int it = 0; it < steps; ++it) {
    if (forward(m, n) != cudaSuccess || backward(m, n) != cudaSuccess) return VE_ECUDA;
    ++m->adam_t;
    const float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
    k_adam<<<(np + 255) / 256 < 1024 ? (np + 255) / 256 : 1024, 256, 0, m->s>>>(np, m->p, m->g, m->m, m->v,
                                                                             lr, b1, b2, c1, c2, eps);
    if (cudaGetLastError() != cudaSuccess) return VE_ECUDA;
  }
  if (loss_out) {
    if (forward(m, n) != cudaSuccess || backward(m, n) != cudaSuccess) return VE_ECUDA;
    float sq = 0.f;
    if (cudaMemcpyAsync(&sq, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->s) != cudaSuccess ||
        cudaStreamSynchronize(m->s) != cudaSuccess)
      return VE_ECUDA;
    *loss_out = 0.5f * sq / (float)(n * m->n_out);
  } else if (cudaStreamSynchronize(m->s) != cudaSuccess) {
    return VE_ECUDA;
  }
  return VE_OK;
}

int ve_mlp_predict(ve_mlp* m, const float* x, int n, float* y) {
  cudaGetLastError();  // report only errors raised by this call
  if (!m || !x || !y || n < 1) return VE_EINVAL;
  int r = mlp_reserve(m, n);
  if (r != VE_OK) return r;
  const int L = m->n_layers + 1;
  if (cudaMemcpyAsync(m->x, x, sizeof(float) * n * m->n_in, cudaMemcpyHostToDevice, m->s) != cudaSuccess ||
      forward(m, n) != cudaSuccess ||
      cudaMemcpyAsync(y, m->act[L], sizeof(float) * n * m->n_out, cudaMemcpyDeviceToHost, m->s) != cudaSuccess ||
      cudaStreamSynchronize(m->s) != cudaSuccess)
    return VE_ECUDA;
  return VE_OK;
}

}  // extern "C"
