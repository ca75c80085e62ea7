// ve_dense.cu -- PSD projection of ONE dense real symmetric n x n matrix on the whole GPU: the
// X step of Algorithm 5 (Khoo & Lindsey, arXiv:2106.02682, Sec. 3.2), X <- Pi_{>=0}(X - eps G),
// whose (N D) x (N D) matrix has no block structure to batch over.
//
// Method: cyclic Jacobi in the circle ordering with the matrix kept implicitly as
// A = V^T Y V, through the eigenvector estimates V (row i of Vt = column v_i) and W = Y V
// (row i of Wt = w_i).  The 2 x 2 block of a pair (p, q) is
//     a_pp = v_p.w_p,   a_qq = v_q.w_q,   a_pq = (v_p.w_q + v_q.w_p) / 2,
// dot products over the pair's own two columns, so the n/2 rotations of a round are
// independent: CTA k forms the block of pair k, computes its rotation J (sym_schur2) and
// applies it to its two columns of V and of W (W J = Y (V J)).  A round needs no grid-wide
// synchronisation; the kernel boundary orders the rounds.  The n - 1 rounds of a sweep and the
// sweep's convergence test are captured as one CUDA graph.
//
// Per round: 4 n^2 words read and written (L2-resident for n <= 1024) and 6 n^2 float64
// instructions (10 n^2 flops: per pair 4 dot products and 4 rotated vectors of length n); a sweep
// is (n - 1) rounds.  The FP64 pipe bounds it: the GPU's whole FP64 rate applies only
// because every round spreads over n/2 CTAs.
//
// Warm start: V from the previous call on the same workspace (consecutive ADMM sweeps project
// nearby matrices), W = Y V by one GEMM.  Stopping: after a sweep whose rotated blocks satisfy
// 2 sum a_pq^2 <= (n u)^2 ||Y||_F^2 (the rule of the batched eigensolvers).  Then
// lambda_i = v_i.w_i and X = V diag(max(lambda, 0)) V^T by a GEMM.
// Early stop (allow_dk): once a sweep's rotations were small (2 sum a_pq^2 <= 1e-6 ||Y||_F^2,
// so quadratic convergence has left A = V^T Y V within ~1e-6 ||Y|| / gap of diagonal), A is
// formed by one GEMM and its off-diagonal part E checked: ||E||_F^2 <= (n u)^2 ||A||_F^2 means converged
// without the confirming sweep; ||E||_F^4 <= (n u)^2 ||A||_F^2 d^2 and ||E||_F <= d / 4, d the
// distance of diag(A) from zero, means the first-order expansion f(A) = f(Lambda) + L o E
// (Daleckii-Krein, f = max(., 0), L the divided differences) is as accurate as the exact rule,
// and X = V (f(Lambda) + L o E) V^T by two GEMMs replaces the remaining sweeps.  The input is used as
// (Y + Y^T) / 2: a_pq averages both orders and v_i.w_i = v_i^T Y v_i.
#include <cstdint>

#include "ve_device.cuh"
#include "ve_dense.h"

namespace ve {

namespace {

constexpr int RT = 128;  // threads of a round CTA
// A sweep whose rotations summed below this fraction of ||Y||_F^2 triggers the explicit check
// (one GEMM and one reduction: cheap against a sweep of n - 1 round launches, so it is tried as
// soon as one more sweep could leave A within ~1e-12 of diagonal; measured on the 20-site
// fermion rings, 1e-6 instead of 1e-10 took the float64 sweeps per X step from 3.55 to 3.1).
constexpr double kDkTrigger = 1e-6;

template <int EPT>
__global__ void __launch_bounds__(RT) k_dense_round(double* __restrict__ Vt, double* __restrict__ Wt,
                                                    double* __restrict__ slot, int n, int r) {
  __shared__ double red[RT / 32][4];
  __shared__ double rot[2];
  int p, q;
  rr_pair(n, r, blockIdx.x, p, q);
  double* vp = Vt + (size_t)p * n;
  double* vq = Vt + (size_t)q * n;
  double* wp = Wt + (size_t)p * n;
  double* wq = Wt + (size_t)q * n;
  double xvp[EPT], xvq[EPT], xwp[EPT], xwq[EPT];
  double s_pp = 0.0, s_qq = 0.0, s_pq = 0.0, s_qp = 0.0;
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int a = threadIdx.x + RT * e;
    if (a < n) {
      xvp[e] = vp[a];
      xvq[e] = vq[a];
      xwp[e] = wp[a];
      xwq[e] = wq[a];
      s_pp = fma(xvp[e], xwp[e], s_pp);
      s_qq = fma(xvq[e], xwq[e], s_qq);
      s_pq = fma(xvp[e], xwq[e], s_pq);
      s_qp = fma(xvq[e], xwp[e], s_qp);
    }
  }
  // Transposing butterfly: the four warp sums in 6 shuffles and 6 float64 adds a thread (not
  // 20 of each).  Across 16 a lane keeps two of the values and hands over the other two, across
  // 8 it keeps one, then three plain levels; lane L ends with the total of value
  // 2 bit4(L) + bit3(L) of (s_pp, s_qq, s_pq, s_qp).
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool hi = (lane & 16) != 0, mid = (lane & 8) != 0;
  double k0 = hi ? s_pq : s_pp, k1 = hi ? s_qp : s_qq;
  const double g0 = hi ? s_pp : s_pq, g1 = hi ? s_qq : s_qp;
  k0 += __shfl_xor_sync(0xffffffffu, g0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, g1, 16);
  double v = mid ? k1 : k0;
  v += __shfl_xor_sync(0xffffffffu, mid ? k0 : k1, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  if ((lane & 7) == 0) red[w][lane >> 3] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double app = 0.0, aqq = 0.0, bpq = 0.0, bqp = 0.0;
#pragma unroll
    for (int k = 0; k < RT / 32; ++k) {
      app += red[k][0];
      aqq += red[k][1];
      bpq += red[k][2];
      bqp += red[k][3];
    }
    const double apq = 0.5 * (bpq + bqp);
    slot[blockIdx.x] += apq * apq;
    double c, s, t;
    sym_schur2<double>(app, aqq, apq, c, s, t);
    rot[0] = c;
    rot[1] = s;
  }
  __syncthreads();
  const double c = rot[0], s = rot[1];
  if (s == 0.0) return;  // a_pq = 0: J = I
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int a = threadIdx.x + RT * e;
    if (a < n) {
      vp[a] = c * xvp[e] - s * xvq[e];
      vq[a] = s * xvp[e] + c * xvq[e];
      wp[a] = c * xwp[e] - s * xwq[e];
      wq[a] = s * xwp[e] + c * xwq[e];
    }
  }
}

// Sum of the sweep's a_pq^2 in a fixed order, the convergence flag, and the slots cleared.
__global__ void __launch_bounds__(256) k_dense_sweep_end(double* slot, int H, DenseCtl* ctl, int n) {
  __shared__ double red[8];
  double v = 0.0;
  for (int k = threadIdx.x; k < H; k += 256) {
    v += slot[k];
    slot[k] = 0.0;
  }
  v = gsum<256>(v, red);
  if (threadIdx.x == 0) {
    const double tol = (double)n * JacobiTol<double>::u;
    ctl->off2 = 2.0 * v;
    ctl->converged = (2.0 * v <= tol * tol * ctl->nrm2) ? 1 : 0;
    ctl->sweeps += 1;
  }
}

// The explicit early-stop test on A = V^T Y V (B[i][j] = v_i.w_j, symmetrised).
__global__ void __launch_bounds__(1024) k_dense_dk_check(const double* B, int n, DenseCtl* ctl) {
  __shared__ double red[32];
  double off = 0.0, d = INFINITY;
  const size_t nn = (size_t)n * n;
  for (size_t e = threadIdx.x; e < nn; e += 1024) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (i < j) {
      const double a = 0.5 * (B[e] + B[(size_t)j * n + i]);
      off = fma(2.0 * a, a, off);
    } else if (i == j) {
      d = nan_min(d, fabs(B[e]));
    }
  }
  off = gsum<1024>(off, red);
  d = gmin<1024>(d, red);
  if (threadIdx.x == 0) {
    const double tol = (double)n * JacobiTol<double>::u;
    const double rel2 = tol * tol * ctl->nrm2;
    int dk = 0;
    if (off <= rel2) dk = 1;
    else if (off * off <= rel2 * d * d && 16.0 * off <= d * d) dk = 2;
    ctl->dk = dk;
  }
}

// M = f(Lambda) + L o E from A (B, symmetrised) into M; lam receives the diagonal.
__global__ void k_dense_dk_matrix(const double* B, double* M, double* lam, int n) {
  const size_t nn = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const double li = B[(size_t)i * n + i];
    if (i == j) {
      M[e] = li > 0.0 ? li : 0.0;
      lam[i] = li;
    } else {
      const double a = 0.5 * (B[e] + B[(size_t)j * n + i]);
      M[e] = a * dk_weight<double>(li, B[(size_t)j * n + j]);
    }
  }
}

// ||Y||_F^2 (fixed order), and the control block reset for a new projection.
__global__ void __launch_bounds__(1024) k_dense_begin(const double* Y, int n, double* slot, DenseCtl* ctl) {
  __shared__ double red[32];
  double v = 0.0;
  const size_t nn = (size_t)n * n;
  for (size_t e = threadIdx.x; e < nn; e += 1024) v = fma(Y[e], Y[e], v);
  v = gsum<1024>(v, red);
  for (int k = threadIdx.x; k < n / 2; k += 1024) slot[k] = 0.0;
  if (threadIdx.x == 0) {
    ctl->nrm2 = v;
    ctl->off2 = 0.0;
    ctl->converged = 0;
    ctl->sweeps = 0;
    ctl->dk = 0;
  }
}

__global__ void k_dense_identity(double* Vt, int n) {
  const size_t nn = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x)
    Vt[e] = (e / n == e % n) ? 1.0 : 0.0;
}

// lambda_i = v_i.w_i (a warp per i, fixed order); lmin = min_i lambda_i when requested.
__global__ void __launch_bounds__(256) k_dense_rayleigh(const double* Vt, const double* Wt, double* lam, int n) {
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  const double* v = Vt + (size_t)i * n;
  const double* w = Wt + (size_t)i * n;
  double s = 0.0;
  for (int a = lane; a < n; a += 32) s = fma(v[a], w[a], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) lam[i] = s;
}

__global__ void __launch_bounds__(256) k_dense_min(const double* lam, int n, DenseCtl* ctl) {
  __shared__ double red[8];
  double v = INFINITY;
  for (int k = threadIdx.x; k < n; k += 256) v = nan_min(v, lam[k]);
  v = gmin<256>(v, red);
  if (threadIdx.x == 0) ctl->lmin = v;
}

// A certified lmin from the explicit A = V^T Y V = diag + E (B[i][j] = v_i.w_j, symmetrised):
// by Weyl's inequality every eigenvalue of A lies within ||E||_2 <= ||E||_F of the sorted
// diagonal, so lmin(Y) >= min_i a_ii - ||E||_F whether or not the sweeps converged.  A NaN
// passes through to ctl->lmin.
__global__ void __launch_bounds__(1024) k_dense_weyl_min(const double* B, int n, DenseCtl* ctl) {
  __shared__ double red[32];
  double off = 0.0, d = INFINITY;
  const size_t nn = (size_t)n * n;
  for (size_t e = threadIdx.x; e < nn; e += 1024) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (i < j) {
      const double a = 0.5 * (B[e] + B[(size_t)j * n + i]);
      off = fma(2.0 * a, a, off);
    } else if (i == j) {
      d = nan_min(d, B[e]);
    }
  }
  off = gsum<1024>(off, red);
  d = gmin<1024>(d, red);
  if (threadIdx.x == 0) ctl->lmin = d - sqrt(off);
}

// C (M x N) = op(A) diag(s) op(B), op(A)(i,k) = TA ? A[k][i] : A[i][k], op(B)(k,j) = TB ? B[j][k] :
// B[k][j], s_k = max(scale[k], 0) (scale null: 1).  BS x BS tiles, 64 threads with
// (BS/8) x (BS/8) outputs each; float64 FMAs bound it (the part's float64 rate is ~2 FMA per SM
// clock), so the simple shared-memory tiling suffices, and products too small to give every SM a
// 32 x 32 tile take 16 x 16 tiles (n = 160: 100 CTAs instead of 25).  Every output sums its K
// terms in the same order whatever the tile, so the results do not depend on it.
template <bool TA, bool TB, int BS>
__global__ void __launch_bounds__(64) k_gemm(int M, int N, int K, const double* __restrict__ A, int lda,
                                             const double* __restrict__ B, int ldb, double* __restrict__ C,
                                             int ldc, const double* __restrict__ scale) {
  constexpr int BM = BS, BN = BS, BK = 16, TT = BS / 8;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  double acc[TT][TT];
#pragma unroll
  for (int u = 0; u < TT; ++u)
#pragma unroll
    for (int v = 0; v < TT; ++v) acc[u][v] = 0.0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int l = threadIdx.x; l < BM * BK; l += 64) {
      int ii, kk;
      if (TA) {
        ii = l % BM;
        kk = l / BM;
      } else {
        kk = l % BK;
        ii = l / BK;
      }
      const int gi = i0 + ii, gk = k0 + kk;
      double x = 0.0;
      if (gi < M && gk < K) {
        x = TA ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk];
        if (scale) x *= fmax(scale[gk], 0.0);
      }
      As[kk][ii] = x;
    }
    for (int l = threadIdx.x; l < BN * BK; l += 64) {
      int jj, kk;
      if (TB) {
        kk = l % BK;
        jj = l / BK;
      } else {
        jj = l % BN;
        kk = l / BN;
      }
      const int gj = j0 + jj, gk = k0 + kk;
      double x = 0.0;
      if (gj < N && gk < K) x = TB ? B[(size_t)gj * ldb + gk] : B[(size_t)gk * ldb + gj];
      Bs[kk][jj] = x;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[TT], b[TT];
#pragma unroll
      for (int u = 0; u < TT; ++u) a[u] = As[kk][ty * TT + u];
#pragma unroll
      for (int v = 0; v < TT; ++v) b[v] = Bs[kk][tx * TT + v];
#pragma unroll
      for (int u = 0; u < TT; ++u)
#pragma unroll
        for (int v = 0; v < TT; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < TT; ++u) {
    const int gi = i0 + ty * TT + u;
    if (gi >= M) continue;
#pragma unroll
    for (int v = 0; v < TT; ++v) {
      const int gj = j0 + tx * TT + v;
      if (gj < N) C[(size_t)gi * ldc + gj] = acc[u][v];
    }
  }
}

template <bool TA, bool TB>
cudaError_t gemm(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                 int ldc, const double* scale, cudaStream_t s) {
  if ((long)((M + 31) / 32) * ((N + 31) / 32) < 152) {
    const dim3 grid((unsigned)((N + 15) / 16), (unsigned)((M + 15) / 16));
    k_gemm<TA, TB, 16><<<grid, 64, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, scale);
  } else {
    const dim3 grid((unsigned)((N + 31) / 32), (unsigned)((M + 31) / 32));
    k_gemm<TA, TB, 32><<<grid, 64, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, scale);
  }
  return cudaGetLastError();
}

cudaError_t launch_round(DenseWs& w, int r, cudaStream_t s) {
  const unsigned grid = (unsigned)(w.n / 2);
  const int ept = (w.n + RT - 1) / RT;
  if (ept <= 1) k_dense_round<1><<<grid, RT, 0, s>>>(w.Vt, w.Wt, w.slot, w.n, r);
  else if (ept <= 2) k_dense_round<2><<<grid, RT, 0, s>>>(w.Vt, w.Wt, w.slot, w.n, r);
  else if (ept <= 4) k_dense_round<4><<<grid, RT, 0, s>>>(w.Vt, w.Wt, w.slot, w.n, r);
  else k_dense_round<8><<<grid, RT, 0, s>>>(w.Vt, w.Wt, w.slot, w.n, r);
  return cudaGetLastError();
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t dense_ws_bytes(int n) {
  if (n < 2 || n > DENSE_MAX_N || (n & 1)) return 0;
  const size_t nn = (size_t)n * n * sizeof(double);
  return 3 * al256(nn) + al256(n * sizeof(double)) + al256((n / 2) * sizeof(double)) +
         al256(sizeof(DenseCtl));
}

int dense_ws_init(DenseWs& w, int n, void* mem, size_t bytes) {
  const size_t need = dense_ws_bytes(n);
  if (need == 0 || !mem || bytes < need || ((uintptr_t)mem & 255)) return -1;
  unsigned char* p = (unsigned char*)mem;
  const size_t nn = (size_t)n * n * sizeof(double);
  w = DenseWs();
  w.n = n;
  w.Vt = (double*)p;
  p += al256(nn);
  w.Wt = (double*)p;
  p += al256(nn);
  w.Bt = (double*)p;
  p += al256(nn);
  w.lam = (double*)p;
  p += al256(n * sizeof(double));
  w.slot = (double*)p;
  p += al256((n / 2) * sizeof(double));
  w.ctl = (DenseCtl*)p;
  return 0;
}

void dense_ws_release(DenseWs& w) {
  if (w.g0) cudaEventDestroy(w.g0);
  if (w.g1) cudaEventDestroy(w.g1);
  w.g0 = w.g1 = nullptr;
  if (w.exec) cudaGraphExecDestroy(w.exec);
  if (w.graph) cudaGraphDestroy(w.graph);
  if (w.hctl) cudaFreeHost(w.hctl);
  w.exec = nullptr;
  w.graph = nullptr;
  w.hctl = nullptr;
}

namespace {

// The n - 1 rounds of one sweep and its convergence test, as a graph (built on first use).
cudaError_t sweep_graph(DenseWs& w, cudaStream_t s) {
  if (w.exec) return cudaSuccess;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int r = 0; r < w.n - 1 && e == cudaSuccess; ++r) e = launch_round(w, r, cs);
    if (e == cudaSuccess) {
      k_dense_sweep_end<<<1, 256, 0, cs>>>(w.slot, w.n / 2, w.ctl, w.n);
      e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) {
      e = cudaGraphInstantiate(&w.exec, g, 0);
      w.graph = g;
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  cudaStreamDestroy(cs);
  (void)s;
  return e;
}

}  // namespace

cudaError_t dense_eig(DenseWs& w, const double* Y, int mode, cudaStream_t s) {
  const int n = w.n;
  cudaError_t e;
  w.dk_mode = 0;
  if (!w.hctl) {
    e = cudaMallocHost((void**)&w.hctl, sizeof(DenseCtl));
    if (e != cudaSuccess) return e;
  }
  e = sweep_graph(w, s);
  if (e != cudaSuccess) return e;
  k_dense_begin<<<1, 1024, 0, s>>>(Y, n, w.slot, w.ctl);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  w.launches += 1;
  if (mode == DENSE_COLD) {
    k_dense_identity<<<256, 256, 0, s>>>(w.Vt, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    w.launches += 1;
  }
  // W = Y V, i.e. Wt = Vt Y^T
  e = gemm<false, true>(n, n, n, w.Vt, n, Y, n, w.Wt, n, nullptr, s);
  if (e != cudaSuccess) return e;
  w.launches += 1;
  if (w.prof && !w.g0) {
    if ((e = cudaEventCreate(&w.g0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&w.g1)) != cudaSuccess) return e;
  }
  int sweeps = 0;
  for (; sweeps < JacobiTol<double>::max_sweeps; ++sweeps) {
    if (w.prof && (e = cudaEventRecord(w.g0, s)) != cudaSuccess) return e;
    if ((e = cudaGraphLaunch(w.exec, s)) != cudaSuccess) return e;
    if (w.prof && (e = cudaEventRecord(w.g1, s)) != cudaSuccess) return e;
    w.launches += n;
    if ((e = cudaMemcpyAsync(w.hctl, w.ctl, sizeof(DenseCtl), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (w.prof) {
      float ms = 0.f;
      if ((e = cudaEventElapsedTime(&ms, w.g0, w.g1)) != cudaSuccess) return e;
      w.graph_ms += ms;
      w.graph_rounds += n - 1;
    }
    if (w.hctl->converged) {
      ++sweeps;
      break;
    }
    if (w.allow_dk && w.hctl->off2 <= kDkTrigger * w.hctl->nrm2) {
      // A = V^T (Y V): B[i][j] = v_i.w_j
      if ((e = gemm<false, true>(n, n, n, w.Vt, n, w.Wt, n, w.Bt, n, nullptr, s)) != cudaSuccess) return e;
      k_dense_dk_check<<<1, 1024, 0, s>>>(w.Bt, n, w.ctl);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      w.launches += 2;
      if ((e = cudaMemcpyAsync(w.hctl, w.ctl, sizeof(DenseCtl), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
      if (w.hctl->dk) {
        w.dk_mode = w.hctl->dk;
        ++w.dk_stops;
        ++sweeps;
        break;
      }
    }
  }
  w.last_sweeps = sweeps;
  w.total_sweeps += sweeps;
  k_dense_rayleigh<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(w.Vt, w.Wt, w.lam, n);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  w.launches += 1;
  return cudaSuccess;
}

cudaError_t dense_reconstruct(DenseWs& w, double* X, cudaStream_t s) {
  const int n = w.n;
  if (w.dk_mode == 2) {
    // X = V M V^T = Vt^T (M Vt), M = f(Lambda) + L o E built in Wt (free after the check)
    k_dense_dk_matrix<<<256, 256, 0, s>>>(w.Bt, w.Wt, w.lam, n);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = gemm<false, false>(n, n, n, w.Wt, n, w.Vt, n, w.Bt, n, nullptr, s);
    if (e == cudaSuccess) e = gemm<true, false>(n, n, n, w.Vt, n, w.Bt, n, X, n, nullptr, s);
    w.launches += 3;
    return e;
  }
  // X = V diag(max(lambda, 0)) V^T = Vt^T diag(.) Vt
  const cudaError_t e = gemm<true, false>(n, n, n, w.Vt, n, w.Vt, n, X, n, w.lam, s);
  w.launches += 1;
  return e;
}

cudaError_t dense_lmin(DenseWs& w, cudaStream_t s) {
  k_dense_min<<<1, 256, 0, s>>>(w.lam, w.n, w.ctl);
  w.launches += 1;
  return cudaGetLastError();
}

cudaError_t dense_lmin_certified(DenseWs& w, cudaStream_t s) {
  const int n = w.n;
  cudaError_t e = gemm<false, true>(n, n, n, w.Vt, n, w.Wt, n, w.Bt, n, nullptr, s);
  if (e != cudaSuccess) return e;
  k_dense_weyl_min<<<1, 1024, 0, s>>>(w.Bt, n, w.ctl);
  w.launches += 2;
  return cudaGetLastError();
}

}  // namespace ve
