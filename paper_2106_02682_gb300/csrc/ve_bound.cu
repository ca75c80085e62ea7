// ve_bound.cu -- certified lower bound of the current state and the standalone batched PSD
// projections.
//
// Bound (weak duality of Eq. (partialDual) of Khoo & Lindsey, arXiv:2106.02682, with the
// Lagrangian of Eq. (lagrangian)): for PSD X and any multipliers, with the pair (a, b), a < b,
// offset delta = b - a, given Lambda1_delta on its first and Lambda1_{-delta} on its second
// factor,
//   F[X] >= N lmin(K_0) + sum_delta c(delta) lmin(K_delta),
//   K_delta = H'_{0,delta} + Lambda1_delta (x) I + I (x) Lambda1_{-delta},
//   K_0     = H'_0 - sum_delta Lambda1_delta.
// This file computes lmin(K_delta) for every delta and lmin(K_0) in float64 (values-only
// Jacobi); the host adds the weights c(delta) and the correction for a slightly indefinite X.
// Each lmin is the smallest diagonal entry of the rotated matrix minus the Frobenius norm of its
// remaining off-diagonal part, a lower bound by Weyl's inequality whether or not the Jacobi
// sweeps converged; minima pass a NaN on (nan_min), so a non-finite state cannot certify.
#include "ve_device.cuh"
#include "ve_internal.h"

namespace ve {

namespace {

template <int D>
struct BShape {
  static constexpr int m = ClusterDim<D>::m;
  static constexpr int NT = GroupShape<D>::NT, LD = GroupShape<D>::LD;
  static constexpr int GPC = GroupShape<D>::GPC;
  static constexpr size_t MAT = ((sizeof(double) * D * LD + 15) / 16) * 16;
  static constexpr size_t bytes = MAT + sizeof(double) * D * D + sizeof(double) * (D + 32);
};

template <int D>
__global__ void __launch_bounds__(BShape<D>::NT * BShape<D>::GPC, GroupShape<D>::MINB) k_bound_pairs(const BoundArgs a) {
  constexpr int m = BShape<D>::m, NT = BShape<D>::NT, LD = BShape<D>::LD, GPC = BShape<D>::GPC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = threadIdx.x / NT, tid = threadIdx.x % NT;
  unsigned char* base = GroupShape<D>::GLOBAL ? a.gws + (size_t)blockIdx.x * BShape<D>::bytes
                                              : smem_raw + (size_t)g * BShape<D>::bytes;
  double* A = reinterpret_cast<double*>(base);
  double* Xs = reinterpret_cast<double*>(base + BShape<D>::MAT);
  double* cs = Xs + D * D;
  double* red = cs + D;
  for (long p = (long)blockIdx.x * GPC + g; p < a.P; p += (long)gridDim.x * GPC) {
    const long dl = p + 1;
    const double* Xb = a.X + dl * D * D;
    const int hs = a.hslot[dl];
    const double* Hb = hs >= 0 ? a.hb + (long)hs * D * D : nullptr;
    const double* l1 = a.lam1 + p * m * m;
    const double* l1n = a.lam1 + (long)(a.neg[dl] - 1) * m * m;
    for (int e = tid; e < D * D; e += NT) Xs[e] = Xb[e];
    gsync<NT>();
    for (int e = tid; e < D * D; e += NT) {
      const int i = e / D, j = e % D;
      const int pa = i / m, pb = i % m, pc = j / m, pd = j % m;
      double k = Hb ? Hb[e] : 0.0;
      k -= Xs[(pa * m + pc) * D + (pd * m + pb)] + Xs[(pc * m + pa) * D + (pb * m + pd)];
      if (pb == pd) k += l1[pa * m + pc];
      if (pa == pc) k += l1n[pb * m + pd];
      A[i * LD + j] = k;
    }
    gsync<NT>();
    for (int e = tid; e < D * D; e += NT) {
      const int i = e / D, j = e % D;
      if (i < j) {
        const double v = 0.5 * (A[i * LD + j] + A[j * LD + i]);
        A[i * LD + j] = v;
        A[j * LD + i] = v;
      }
    }
    gsync<NT>();
    double off = 0.0;
    jacobi_sym<double, D, LD, NT, false>(A, nullptr, cs, red, tid, nullptr, &off);
    double w = INFINITY;
    for (int k = tid; k < D; k += NT) w = nan_min(w, A[k * LD + k]);
    w = gmin<NT>(w, red);
    // Weyl: the rotated matrix is diag + E, so lmin >= min diag - ||E||_2 >= min diag - ||E||_F
    if (tid == 0) a.lmin_pairs[p] = w - sqrt(off);
    gsync<NT>();
  }
}

template <int m>
__global__ void __launch_bounds__(256) k_bound_k0(const BoundArgs a) {
  constexpr int mm = m * m, LD = m + 1;
  __shared__ double S[256];
  __shared__ double A[m * LD];
  __shared__ double cs[2 * m + 2];
  __shared__ double red[8];
  const int t = threadIdx.x, D = a.D;
  const int chunks = 256 / mm;
  if (t < chunks * mm) {
    const int idx = t % mm, c = t / mm;
    const long per = (a.P + chunks - 1) / chunks;
    const long lo = c * per, hi = min((long)a.P, lo + per);
    double s = 0.0;
    for (long p = lo; p < hi; ++p) s += a.lam1[p * mm + idx];
    S[t] = s;
  }
  __syncthreads();
  if (t < mm) {
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += S[c * mm + t];
    const int b = t / m, d = t % m;
    double hx = 0.0;
    for (int x = 0; x < m; ++x) hx += a.X[(x * m + b) * D + (x * m + d)];
    A[b * LD + d] = a.H0[t] - hx - s;
  }
  __syncthreads();
  if (t < 32) {
    for (int e = t; e < mm; e += 32) {
      const int i = e / m, j = e % m;
      if (i < j) {
        const double v = 0.5 * (A[i * LD + j] + A[j * LD + i]);
        A[i * LD + j] = v;
        A[j * LD + i] = v;
      }
    }
    __syncwarp();
    double off = 0.0;
    jacobi_sym<double, m, LD, 32, false>(A, nullptr, cs, red, t, nullptr, &off);
    double w = INFINITY;
    for (int k = t; k < m; k += 32) w = nan_min(w, A[k * LD + k]);
    w = gmin<32>(w, red);
    if (t == 0) a.lmin0[0] = w - sqrt(off);  // Weyl, as in k_bound_pairs
  }
}

// ---------------------------------------------------------------- standalone projections
// n <= 64: the matrices are staged in shared memory; n = 256, 512: in a per-CTA slice of a
// caller workspace (one CTA of 512 threads per SM), as the D = 256 solver kernels do.
template <int n, typename T>
struct PShape {
  static constexpr int NT = GroupShape<n>::NT, LD = GroupShape<n>::LD;
  static constexpr bool G = GroupShape<n>::GLOBAL;
  static constexpr int GPC = (NT == 32) ? 4 : 1;
  static constexpr size_t MAT = ((sizeof(T) * n * LD + 15) / 16) * 16;
  static constexpr size_t bytes = ((4 * MAT + sizeof(T) * (3 * n + 16) + 255) / 256) * 256;
};

template <int n, typename T>
__global__ void __launch_bounds__(PShape<n, T>::NT * PShape<n, T>::GPC)
    k_proj_sym(const double* in, double* out, long count, unsigned char* gws) {
  constexpr int NT = PShape<n, T>::NT, LD = PShape<n, T>::LD, GPC = PShape<n, T>::GPC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = threadIdx.x / NT, tid = threadIdx.x % NT;
  unsigned char* base = PShape<n, T>::G ? gws + (size_t)blockIdx.x * PShape<n, T>::bytes
                                        : smem_raw + (size_t)g * PShape<n, T>::bytes;
  T* A = reinterpret_cast<T*>(base);
  T* V = reinterpret_cast<T*>(base + PShape<n, T>::MAT);
  T* cs = reinterpret_cast<T*>(base + 4 * PShape<n, T>::MAT);
  T* W = cs + 2 * n;
  T* red = W + n;
  for (long b = (long)blockIdx.x * GPC + g; b < count; b += (long)gridDim.x * GPC) {
    const double* M = in + b * n * n;
    for (int e = tid; e < n * n; e += NT) {
      const int i = e / n, j = e % n;
      if (i <= j) {
        const T v = (T)(0.5 * (M[i * n + j] + M[j * n + i]));
        A[i * LD + j] = v;
        A[j * LD + i] = v;
      }
    }
    gsync<NT>();
    jacobi_sym<T, n, LD, NT, true>(A, V, cs, red, tid);
    for (int k = tid; k < n; k += NT) {
      const T w = A[k * LD + k];
      W[k] = w > T(0) ? w : T(0);
    }
    gsync<NT>();
    double* O = out + b * n * n;
    if constexpr (PShape<n, T>::G) {
      // V^T into A's storage, then the output row by row with the lanes along j, so that
      // V^T[k][j] is read contiguously and V^T[k][i] is the same for the whole warp
      for (int e = tid; e < n * n; e += NT) A[(e % n) * LD + e / n] = V[(e / n) * LD + e % n];
      gsync<NT>();
      for (int e = tid; e < n * n; e += NT) {
        const int i = e / n, j = e % n;
        T s = T(0);
        for (int k = 0; k < n; ++k) s += W[k] * A[k * LD + i] * A[k * LD + j];
        O[e] = (double)s;
      }
    } else {
      for (int e = tid; e < n * n; e += NT) {
        const int i = e / n, j = e % n;
        T s = T(0);
        for (int k = 0; k < n; ++k) s += W[k] * V[i * LD + k] * V[j * LD + k];
        O[e] = (double)s;
      }
    }
    gsync<NT>();
  }
}

template <int n, typename T>
__global__ void __launch_bounds__(PShape<n, T>::NT * PShape<n, T>::GPC)
    k_proj_herm(const double* in, double* out, long count, unsigned char* gws) {
  constexpr int NT = PShape<n, T>::NT, LD = PShape<n, T>::LD, GPC = PShape<n, T>::GPC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = threadIdx.x / NT, tid = threadIdx.x % NT;
  unsigned char* base = PShape<n, T>::G ? gws + (size_t)blockIdx.x * PShape<n, T>::bytes
                                        : smem_raw + (size_t)g * PShape<n, T>::bytes;
  T* Ar = reinterpret_cast<T*>(base);
  T* Ai = reinterpret_cast<T*>(base + PShape<n, T>::MAT);
  T* Vr = reinterpret_cast<T*>(base + 2 * PShape<n, T>::MAT);
  T* Vi = reinterpret_cast<T*>(base + 3 * PShape<n, T>::MAT);
  T* cs = reinterpret_cast<T*>(base + 4 * PShape<n, T>::MAT);
  T* W = cs + 2 * n;
  T* red = W + n;
  for (long b = (long)blockIdx.x * GPC + g; b < count; b += (long)gridDim.x * GPC) {
    const double* M = in + b * n * n * 2;
    for (int e = tid; e < n * n; e += NT) {
      const int i = e / n, j = e % n;
      if (i < j) {
        const T r = (T)(0.5 * (M[2 * (i * n + j)] + M[2 * (j * n + i)]));
        const T im = (T)(0.5 * (M[2 * (i * n + j) + 1] - M[2 * (j * n + i) + 1]));
        Ar[i * LD + j] = r;
        Ai[i * LD + j] = im;
        Ar[j * LD + i] = r;
        Ai[j * LD + i] = -im;
      } else if (i == j) {
        Ar[i * LD + i] = (T)M[2 * (i * n + i)];
        Ai[i * LD + i] = T(0);
      }
    }
    gsync<NT>();
    jacobi_herm<T, n, LD, NT, true>(Ar, Ai, Vr, Vi, cs, red, tid);
    for (int k = tid; k < n; k += NT) {
      const T w = Ar[k * LD + k];
      W[k] = w > T(0) ? w : T(0);
    }
    gsync<NT>();
    double* O = out + b * n * n * 2;
    // n > 64: V^T into (Ar, Ai) first (see k_proj_sym), so the lanes read along rows
    if constexpr (PShape<n, T>::G) {
      for (int e = tid; e < n * n; e += NT) {
        Ar[(e % n) * LD + e / n] = Vr[(e / n) * LD + e % n];
        Ai[(e % n) * LD + e / n] = Vi[(e / n) * LD + e % n];
      }
      gsync<NT>();
    }
    for (int e = tid; e < n * n; e += NT) {
      const int i = e / n, j = e % n;
      T yr = T(0), yi = T(0);
      for (int k = 0; k < n; ++k) {
        const T w = W[k];
        T air, aii, ajr, aji;
        if constexpr (PShape<n, T>::G) {
          air = Ar[k * LD + i];
          aii = Ai[k * LD + i];
          ajr = Ar[k * LD + j];
          aji = Ai[k * LD + j];
        } else {
          air = Vr[i * LD + k];
          aii = Vi[i * LD + k];
          ajr = Vr[j * LD + k];
          aji = Vi[j * LD + k];
        }
        yr += w * (air * ajr + aii * aji);
        yi += w * (aii * ajr - air * aji);
      }
      O[2 * e] = (double)yr;
      O[2 * e + 1] = (double)yi;
    }
    gsync<NT>();
  }
}


template <int D>
cudaError_t launch_bound_t(const BoundArgs& a, cudaStream_t s) {
  constexpr int NT = BShape<D>::NT, GPC = BShape<D>::GPC, m = BShape<D>::m;
  constexpr bool G = GroupShape<D>::GLOBAL;
  const size_t smem = G ? 0 : BShape<D>::bytes * GPC;
  cudaError_t e = cudaSuccess;
  if (!G) {
    static unsigned long long mask = 0;
    e = smem_once(k_bound_pairs<D>, smem, mask);
    if (e != cudaSuccess) return e;
  } else if (!a.gws) {
    return cudaErrorInvalidValue;
  }
  long blocks = (a.P + GPC - 1) / GPC;
  if (G && blocks > big_grid()) blocks = big_grid();
  k_bound_pairs<D><<<(unsigned)blocks, NT * GPC, smem, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_bound_k0<m><<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <int n, typename T>
cudaError_t launch_proj_sym_t(const double* in, double* out, long count, unsigned char* gws,
                              cudaStream_t s) {
  using S = PShape<n, T>;
  long blocks = (count + S::GPC - 1) / S::GPC;
  if (blocks > 65535L * 8) blocks = 65535L * 8;
  if constexpr (S::G) {
    if (!gws) return cudaErrorInvalidValue;
    if (blocks > big_grid()) blocks = big_grid();
    k_proj_sym<n, T><<<(unsigned)blocks, S::NT, 0, s>>>(in, out, count, gws);
  } else {
    const size_t smem = S::bytes * S::GPC;
    static unsigned long long mask = 0;
    cudaError_t e = smem_once(k_proj_sym<n, T>, smem, mask);
    if (e != cudaSuccess) return e;
    k_proj_sym<n, T><<<(unsigned)blocks, S::NT * S::GPC, smem, s>>>(in, out, count, nullptr);
  }
  return cudaGetLastError();
}

template <int n, typename T>
cudaError_t launch_proj_herm_t(const double* in, double* out, long count, unsigned char* gws,
                               cudaStream_t s) {
  using S = PShape<n, T>;
  long blocks = (count + S::GPC - 1) / S::GPC;
  if (blocks > 65535L * 8) blocks = 65535L * 8;
  if constexpr (S::G) {
    if (!gws) return cudaErrorInvalidValue;
    if (blocks > big_grid()) blocks = big_grid();
    k_proj_herm<n, T><<<(unsigned)blocks, S::NT, 0, s>>>(in, out, count, gws);
  } else {
    const size_t smem = S::bytes * S::GPC;
    static unsigned long long mask = 0;
    cudaError_t e = smem_once(k_proj_herm<n, T>, smem, mask);
    if (e != cudaSuccess) return e;
    k_proj_herm<n, T><<<(unsigned)blocks, S::NT * S::GPC, smem, s>>>(in, out, count, nullptr);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bound(const BoundArgs& a, cudaStream_t s) {
  switch (a.D) {
    case 4: return launch_bound_t<4>(a, s);
    case 16: return launch_bound_t<16>(a, s);
    case 64: return launch_bound_t<64>(a, s);
    case 256: return launch_bound_t<256>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

size_t bound_ws_bytes(int D) { return D == 256 ? BShape<256>::bytes * (size_t)big_grid() : 0; }

template <int n>
cudaError_t proj_sym_n(const double* in, double* out, long count, int arith, unsigned char* gws,
                       cudaStream_t s) {
  switch (arith) {
    case ARITH_FP64: return launch_proj_sym_t<n, double>(in, out, count, gws, s);
    case ARITH_FP32: return launch_proj_sym_t<n, float>(in, out, count, gws, s);
    case ARITH_DF64: return launch_proj_sym_t<n, df64>(in, out, count, gws, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int n>
cudaError_t proj_herm_n(const double* in, double* out, long count, int arith, unsigned char* gws,
                        cudaStream_t s) {
  switch (arith) {
    case ARITH_FP64: return launch_proj_herm_t<n, double>(in, out, count, gws, s);
    case ARITH_FP32: return launch_proj_herm_t<n, float>(in, out, count, gws, s);
    case ARITH_DF64: return launch_proj_herm_t<n, df64>(in, out, count, gws, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_proj_sym(const double* in, double* out, int n, long count, int arith,
                            cudaStream_t s, unsigned char* gws) {
  if (count == 0) return cudaSuccess;
  switch (n) {
    case 2: return proj_sym_n<2>(in, out, count, arith, nullptr, s);
    case 4: return proj_sym_n<4>(in, out, count, arith, nullptr, s);
    case 8: return proj_sym_n<8>(in, out, count, arith, nullptr, s);
    case 16: return proj_sym_n<16>(in, out, count, arith, nullptr, s);
    case 64: return proj_sym_n<64>(in, out, count, arith, nullptr, s);
    case 256: return proj_sym_n<256>(in, out, count, arith, gws, s);
    case 512: return proj_sym_n<512>(in, out, count, arith, gws, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_proj_herm(const double* in, double* out, int n, long count, int arith,
                             cudaStream_t s, unsigned char* gws) {
  if (count == 0) return cudaSuccess;
  switch (n) {
    case 4: return proj_herm_n<4>(in, out, count, arith, nullptr, s);
    case 16: return proj_herm_n<16>(in, out, count, arith, nullptr, s);
    case 64: return proj_herm_n<64>(in, out, count, arith, nullptr, s);
    case 256: return proj_herm_n<256>(in, out, count, arith, gws, s);
    default: return cudaErrorInvalidValue;
  }
}

size_t proj_ws_bytes(int n, bool herm, int arith) {
  size_t per = 0;
  if (herm) {
    if (n != 256) return 0;
    per = arith == ARITH_FP32 ? PShape<256, float>::bytes : PShape<256, double>::bytes;
  } else if (n == 256) {
    per = arith == ARITH_FP32 ? PShape<256, float>::bytes : PShape<256, double>::bytes;
  } else if (n == 512) {
    per = arith == ARITH_FP32 ? PShape<512, float>::bytes : PShape<512, double>::bytes;
  } else {
    return 0;
  }
  return per * (size_t)big_grid();
}

}  // namespace ve
