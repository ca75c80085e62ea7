// ve_general.cu -- Algorithm 5 (Khoo & Lindsey, arXiv:2106.02682, Sec. 3.2 "practical scheme")
// for a spin-1/2 Hamiltonian WITHOUT translation invariance: random fields, long-range or
// inhomogeneous couplings.  Every cluster i has its own H_i and rho_i, every pair i < j its own
// H_ij, rho~_ij, Lambda_ij, Lambda1_ij, Lambda2_ij, and X is one dense (N D) x (N D) matrix.
//
// One sweep on the GPU:
//   k5_pair    one thread group per pair: H'_ij (Eq. (effHam)), the closed-form rho_ij
//              (Eq. (rhoijUpdate)), rho~_ij = Pi(rho_ij - Lambda_ij / mu) by the warm-started
//              Jacobi of the Algorithm-6 pair pass (Eq. (rhoijTildeUpdate)), the Lambda update,
//              A1 rho, A2 rho, and the off-diagonal blocks of Y = X - eps G (G_ij and G_ji =
//              G_ij^T, Sec. 2.2);
//   k5_rho     one CTA per cluster: Eq. (rhoiUpdate) over the pairs on either side with the
//              trace shift, and the diagonal block Y_ii = X_ii - eps G_00[rho_i];
//   k5_dual    Lambda1 / Lambda2 updates with the new rho_i;
//   k5_status  energy per spin, Eq. (feasErr), residual (fixed-order sums);
//   X = Pi(Y)  the whole-GPU dense eigensolver of ve_dense.cu (warm-started).
// The X step takes the sign X - eps G: the ascent direction of the dual function, the only
// sign whose fixed point meets the optimality conditions (the paper prints X + eps G).
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/ve.h"
#include "ve_dense.h"
#include "ve_device.cuh"
#include "ve_internal.h"

namespace ve {
namespace {

struct GenStatus {
  long long iter;
  double energy, feas, d_energy, residual, e_prev;
};

struct GenArgs {
  int N, m, D, n, L;
  long K;
  double mu, nu, eps;
  double* rho;          // N m^2
  double* rt;           // K D^2  rho~
  double* lam;          // K D^2  Lambda
  double* lam1;         // K m^2
  double* lam2;         // K m^2
  const double* X;      // n x n
  double* Y;            // n x n  X - eps G
  const double* Hi;     // N m^2
  const double* Hij;    // K D^2
  const int* pi;        // K: first cluster of pair p
  const int* pj;        // K: second cluster
  double* a1;           // K m^2  A1 rho_ij
  double* a2;           // K m^2  A2 rho_ij
  double* part;         // K * 3: |rho - rho~|^2, Tr[H_ij rho_ij], Lambda1/2 feasibility terms
  double* parti;        // N: Tr[H_i rho_i]
  double* vstore;       // K D^2: eigenvectors of the last pair projections
  int warm;
  int fermionic;        // parity signs on the off-diagonal blocks of G and in H' (Eq. (sdpFerm))
  GenStatus* st;
};

// Parity sign of entry (a, b), (c, d) of an off-diagonal block of the fermionic global matrix:
// in the pair's Jordan-Wigner ordering a second-cluster operator E_cd that changes the fermion
// parity carries the first cluster's parity string P, and E_ab^dagger P = (-1)^p(a) E_ba; so the
// sign is odd when p(a) (p(c) + p(d)) is odd, p the parity of a cluster basis state's bits.
__device__ __forceinline__ bool parity_odd(int a, int c, int d) {
  return ((__popc(a) & (__popc(c) ^ __popc(d))) & 1) != 0;
}

// Index of the pair (i, j), i < j, in lexicographic order.
__host__ __device__ __forceinline__ long pair_index(int N, int i, int j) {
  return (long)i * N - (long)i * (i + 1) / 2 + (j - i - 1);
}

template <int D>
struct GenSmem {
  static constexpr int m = ClusterDim<D>::m, LD = GroupShape<D>::LD;
  static constexpr size_t al(size_t x) { return ((x + 15) / 16) * 16; }
  static constexpr size_t R = 0;                                     // D*D  rhs, then rho
  static constexpr size_t Xs = R + al(sizeof(double) * D * D);       // D*D  X_ij
  static constexpr size_t A = Xs + al(sizeof(double) * D * D);       // D*LD
  static constexpr size_t V = A + al(sizeof(double) * D * LD);
  static constexpr size_t WT = V + al(sizeof(double) * D * LD);
  static constexpr size_t CS = WT + al(sizeof(double) * D * LD);     // D
  static constexpr size_t W = CS + al(sizeof(double) * D);           // D
  static constexpr size_t TR = W + al(sizeof(double) * D);           // 2 m^2
  static constexpr size_t RED = TR + al(sizeof(double) * (2 * m * m + 2));
  static constexpr size_t bytes = RED + al(sizeof(double) * 32);
};

template <int D>
__global__ void __launch_bounds__(GroupShape<D>::NT, GroupShape<D>::MINB) k5_pair(const GenArgs a) {
  using T = double;
  constexpr int m = ClusterDim<D>::m, NT = GroupShape<D>::NT, LD = GroupShape<D>::LD;
  using S = GenSmem<D>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  T* R = reinterpret_cast<T*>(smem_raw + S::R);
  T* Xs = reinterpret_cast<T*>(smem_raw + S::Xs);
  T* A = reinterpret_cast<T*>(smem_raw + S::A);
  T* V = reinterpret_cast<T*>(smem_raw + S::V);
  T* Wt = reinterpret_cast<T*>(smem_raw + S::WT);
  T* cs = reinterpret_cast<T*>(smem_raw + S::CS);
  T* W = reinterpret_cast<T*>(smem_raw + S::W);
  T* t1 = reinterpret_cast<T*>(smem_raw + S::TR);
  T* t2 = t1 + m * m;
  T* red = reinterpret_cast<T*>(smem_raw + S::RED);

  const T mu = a.mu, nu = a.nu, eps = a.eps;
  const T alpha = nu * m;
  const T c0 = T(1) / mu, c1 = T(1) / (mu + alpha), c2 = T(1) / (mu + T(2) * alpha);
  const T imu = T(1) / mu;
  const size_t n = (size_t)a.n;

  for (long p = blockIdx.x; p < a.K; p += gridDim.x) {
    const int ci = a.pi[p], cj = a.pj[p];
    const double* rhoi = a.rho + (size_t)ci * m * m;
    const double* rhoj = a.rho + (size_t)cj * m * m;
    const double* rt = a.rt + p * D * D;
    const double* lam = a.lam + p * D * D;
    const double* l1 = a.lam1 + p * m * m;
    const double* l2 = a.lam2 + p * m * m;
    const double* Hb = a.Hij + p * D * D;
    const double* Xb = a.X + (size_t)ci * D * n + (size_t)cj * D;

    for (int e = tid; e < D * D; e += NT) Xs[e] = Xb[(size_t)(e / D) * n + (e % D)];
    gsync<NT>();
    // right-hand side of Eq. (rhoijUpdate) with H'_ij of Eq. (effHam)
    for (int e = tid; e < D * D; e += NT) {
      const int i = e / D, j = e % D;
      const int pa = i / m, pb = i % m, pc = j / m, pd = j % m;
      // (R^* X)_{(a,b),(c,d)} = X_{(a,c),(d,b)} and its transpose X_{(c,a),(b,d)} (with the
      // parity signs of those X entries for fermions)
      T x1 = Xs[(pa * m + pc) * D + (pd * m + pb)], x2 = Xs[(pc * m + pa) * D + (pb * m + pd)];
      if (a.fermionic) {
        if (parity_odd(pa, pd, pb)) x1 = -x1;
        if (parity_odd(pc, pb, pd)) x2 = -x2;
      }
      const T hp = Hb[e] - x1 - x2;
      T y = mu * rt[e] + lam[e] - hp;
      if (pb == pd) y += nu * rhoi[pa * m + pc] - l1[pa * m + pc];
      if (pa == pc) y += nu * rhoj[pb * m + pd] - l2[pb * m + pd];
      R[e] = y;
    }
    gsync<NT>();
    for (int idx = tid; idx < m * m; idx += NT) {
      const int x = idx / m, z = idx % m;
      T s1 = T(0), s2 = T(0);
      for (int k = 0; k < m; ++k) {
        s1 += R[(x * m + k) * D + (z * m + k)];
        s2 += R[(k * m + x) * D + (k * m + z)];
      }
      t1[idx] = s1;
      t2[idx] = s2;
    }
    gsync<NT>();
    T tr = T(0);
    for (int k = 0; k < m; ++k) tr += t1[k * m + k];
    // rho = (mu + nu A1^*A1 + nu A2^*A2)^{-1} rhs on the commuting projectors P1, P2, Q
    for (int e = tid; e < D * D; e += NT) {
      const int i = e / D, j = e % D;
      const int pa = i / m, pb = i % m, pc = j / m, pd = j % m;
      const T y = R[e];
      const T P1 = (pb == pd) ? t1[pa * m + pc] / m : T(0);
      const T P2 = (pa == pc) ? t2[pb * m + pd] / m : T(0);
      const T Q = (i == j) ? tr / D : T(0);
      R[e] = (y - P1 - P2 + Q) * c0 + (P1 + P2 - T(2) * Q) * c1 + Q * c2;
    }
    gsync<NT>();
    T* vs = a.vstore + p * D * D;
    bool dk = false;
    if (a.warm) {
      for (int e = tid; e < D * D; e += NT) V[(e / D) * LD + (e % D)] = vs[e];
    }
    // C = rho - Lambda / mu, symmetrised, into A
    for (int t = tid; t < D * (D + 1) / 2; t += NT) {
      int i, j;
      tri_index(D, t, i, j);
      const T v = T(0.5) * (R[i * D + j] + R[j * D + i]) - T(0.5) * (lam[i * D + j] + lam[j * D + i]) * imu;
      A[i * LD + j] = v;
      A[j * LD + i] = v;
    }
    gsync<NT>();
    if (a.warm) {
      // A <- V^T C V with the previous eigenvectors
      for (int e = tid; e < D * D; e += NT) {
        const int i = e / D, j = e % D;
        T acc = T(0);
#pragma unroll 4
        for (int k = 0; k < D; ++k) acc += A[i * LD + k] * V[k * LD + j];
        Wt[i * LD + j] = acc;
      }
      gsync<NT>();
      for (int t = tid; t < D * (D + 1) / 2; t += NT) {
        int i, j;
        tri_index(D, t, i, j);
        T acc = T(0);
#pragma unroll 4
        for (int k = 0; k < D; ++k) acc += V[k * LD + i] * Wt[k * LD + j];
        A[i * LD + j] = acc;
        A[j * LD + i] = acc;
      }
      gsync<NT>();
      jacobi_sym<T, D, LD, NT, true, false, true>(A, V, cs, red, tid, &dk);
    } else {
      jacobi_sym<T, D, LD, NT, true, true, true>(A, V, cs, red, tid, &dk);
    }
    for (int e = tid; e < D * D; e += NT) vs[e] = V[(e / D) * LD + (e % D)];
    if (dk) {
      // first-order (Daleckii-Krein) reconstruction V M V^T, M = f(Lambda) + L o E
      dk_matrix_sym<T, D, LD, NT>(A, cs, tid);
      for (int e = tid; e < D * D; e += NT) {
        const int i = e / D, j = e % D;
        T acc = T(0);
#pragma unroll 4
        for (int k = 0; k < D; ++k) acc += V[i * LD + k] * A[k * LD + j];
        Wt[i * LD + j] = acc;
      }
      gsync<NT>();
      for (int t = tid; t < D * (D + 1) / 2; t += NT) {
        int i, j;
        tri_index(D, t, i, j);
        T s = T(0);
#pragma unroll 4
        for (int k = 0; k < D; ++k) s += Wt[i * LD + k] * V[j * LD + k];
        A[i * LD + j] = s;
        A[j * LD + i] = s;
      }
    } else {
      for (int k = tid; k < D; k += NT) {
        const T w = A[k * LD + k];
        W[k] = w > T(0) ? w : T(0);
      }
      gsync<NT>();
      for (int t = tid; t < D * (D + 1) / 2; t += NT) {
        int i, j;
        tri_index(D, t, i, j);
        T s = T(0);
#pragma unroll 4
        for (int k = 0; k < D; ++k) s += W[k] * V[i * LD + k] * V[j * LD + k];
        A[i * LD + j] = s;
        A[j * LD + i] = s;
      }
    }
    gsync<NT>();
    T rr = T(0), en = T(0);
    double* rtw = a.rt + p * D * D;
    double* lamw = a.lam + p * D * D;
    double* Yij = a.Y + (size_t)ci * D * n + (size_t)cj * D;
    double* Yji = a.Y + (size_t)cj * D * n + (size_t)ci * D;
    for (int e = tid; e < D * D; e += NT) {
      const int i = e / D, j = e % D;
      const int pa = i / m, pb = i % m, pc = j / m, pd = j % m;
      const T rho = R[e];
      const T rtn = A[i * LD + j];
      lamw[e] = lam[e] + mu * (rtn - rho);
      rtw[e] = rtn;
      // Y_ij = X_ij - eps G_ij[rho], G entry (a,b),(c,d) = rho_{(a,d),(b,c)} (times the parity
      // sign for fermions); Y_ji = Y_ij^T
      T g = R[(pa * m + pd) * D + (pb * m + pc)];
      if (a.fermionic && parity_odd(pa, pc, pd)) g = -g;
      const double y = Xs[e] - eps * g;
      Yij[(size_t)i * n + j] = y;
      Yji[(size_t)j * n + i] = y;
      rr += (rho - rtn) * (rho - rtn);
      en += Hb[e] * R[j * D + i];
    }
    for (int idx = tid; idx < m * m; idx += NT) {
      const int x = idx / m, z = idx % m;
      T s1 = T(0), s2 = T(0);
      for (int k = 0; k < m; ++k) {
        s1 += R[(x * m + k) * D + (z * m + k)];
        s2 += R[(k * m + x) * D + (k * m + z)];
      }
      a.a1[p * m * m + idx] = s1;
      a.a2[p * m * m + idx] = s2;
    }
    rr = gsum<NT>(rr, red);
    en = gsum<NT>(en, red);
    if (tid == 0) {
      a.part[p * 3 + 0] = rr;
      a.part[p * 3 + 1] = en;
    }
    gsync<NT>();
  }
}

// Eq. (rhoiUpdate) for cluster blockIdx.x: rho_i' = (sum_{j>i} (nu A1 rho_ij + Lambda1_ij) +
// sum_{j<i} (nu A2 rho_ji + Lambda2_ji) - H'_i) / (nu (N - 1)), then the trace shift; the
// diagonal block Y_ii = X_ii - eps G_00[rho_i] and Tr[H_i rho_i].
template <int m>
__global__ void __launch_bounds__(64) k5_rho(const GenArgs a) {
  constexpr int MM = m * m, D = MM;
  __shared__ double r[MM], rn[MM];
  __shared__ double zs;
  const int i = blockIdx.x, t = threadIdx.x, N = a.N;
  const size_t n = (size_t)a.n;
  const double* Xii = a.X + (size_t)i * D * n + (size_t)i * D;
  if (t < MM) {
    const int b = t / m, d = t % m;
    // H'_i = H_i - G_00^*(X_ii), G_00^*(X)_{bd} = sum_a X_{(a,b),(a,d)}
    double g = 0.0;
    for (int x = 0; x < m; ++x) g += Xii[(size_t)(x * m + b) * n + (x * m + d)];
    double acc = -(a.Hi[(size_t)i * MM + t] - g);
    for (int j = 0; j < N; ++j) {
      if (j > i) {
        const long p = pair_index(N, i, j);
        acc += a.nu * a.a1[p * MM + t] + a.lam1[p * MM + t];
      } else if (j < i) {
        const long p = pair_index(N, j, i);
        acc += a.nu * a.a2[p * MM + t] + a.lam2[p * MM + t];
      }
    }
    r[t] = acc / (a.nu * (N - 1));
  }
  __syncthreads();
  if (t == 0) {
    double tr = 0.0;
    for (int k = 0; k < m; ++k) tr += r[k * m + k];
    zs = (1.0 - tr) / m;
  }
  __syncthreads();
  if (t < MM) {
    const double v = r[t] + ((t / m == t % m) ? zs : 0.0);
    rn[t] = v;
    a.rho[(size_t)i * MM + t] = v;
  }
  __syncthreads();
  double* Yii = a.Y + (size_t)i * D * n + (size_t)i * D;
  for (int e = t; e < D * D; e += 64) {
    const int ii = e / D, jj = e % D;
    const int pa = ii / m, pb = ii % m, pc = jj / m, pd = jj % m;
    double x = Xii[(size_t)ii * n + jj];
    // G_00[rho]_{(a,b),(c,d)} = delta_ac rho_{d,b}
    if (pa == pc) x -= a.eps * rn[pd * m + pb];
    Yii[(size_t)ii * n + jj] = x;
  }
  if (t == 0) {
    double en = 0.0;
    for (int b = 0; b < m; ++b)
      for (int d = 0; d < m; ++d) en += a.Hi[(size_t)i * MM + b * m + d] * rn[d * m + b];
    a.parti[i] = en;
  }
}

// Lambda1 / Lambda2 updates (a warp per pair) and their terms of Eq. (feasErr).
template <int m>
__global__ void __launch_bounds__(256) k5_dual(const GenArgs a) {
  constexpr int MM = m * m;
  const long p = (long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= a.K) return;
  const int ci = a.pi[p], cj = a.pj[p];
  double f = 0.0;
  for (int e = lane; e < MM; e += 32) {
    const double d1 = a.a1[p * MM + e] - a.rho[(size_t)ci * MM + e];
    const double d2 = a.a2[p * MM + e] - a.rho[(size_t)cj * MM + e];
    a.lam1[p * MM + e] += a.nu * d1;
    a.lam2[p * MM + e] += a.nu * d2;
    f += d1 * d1 + d2 * d2;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if (lane == 0) a.part[p * 3 + 2] = f;
}

__global__ void __launch_bounds__(256) k5_status(const GenArgs a) {
  __shared__ double red[8];
  double rr = 0.0, en = 0.0, ff = 0.0, ei = 0.0;
  for (long p = threadIdx.x; p < a.K; p += 256) {
    rr += a.part[p * 3 + 0];
    en += a.part[p * 3 + 1];
    ff += a.part[p * 3 + 2];
  }
  for (int i = threadIdx.x; i < a.N; i += 256) ei += a.parti[i];
  rr = gsum<256>(rr, red);
  en = gsum<256>(en, red);
  ff = gsum<256>(ff, red);
  ei = gsum<256>(ei, red);
  if (threadIdx.x == 0) {
    GenStatus* st = a.st;
    const double E = (ei + en) / ((double)a.N * a.L);
    const double feas = sqrt((rr + ff) / (double)a.K);
    const double dE = isfinite(st->e_prev) ? fabs(E - st->e_prev) : INFINITY;
    st->energy = E;
    st->feas = feas;
    st->d_energy = dE;
    st->residual = fmax(feas, dE);
    st->e_prev = E;
    st->iter += 1;
  }
}

// ---------------------------------------------------------------- certified bound
// lmin of K_ij = H'_ij + A1^* Lambda1_ij + A2^* Lambda2_ij (a group per pair, symmetrised).
template <int D>
__global__ void __launch_bounds__(GroupShape<D>::NT, GroupShape<D>::MINB) k5_bound_pair(const GenArgs a,
                                                                                      double* lmin) {
  constexpr int m = ClusterDim<D>::m, NT = GroupShape<D>::NT, LD = GroupShape<D>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Xs = reinterpret_cast<double*>(smem_raw);
  double* A = Xs + D * D;
  double* cs = A + D * LD;
  double* red = cs + D;
  const int tid = threadIdx.x;
  const size_t n = (size_t)a.n;
  for (long p = blockIdx.x; p < a.K; p += gridDim.x) {
    const int ci = a.pi[p], cj = a.pj[p];
    const double* Xb = a.X + (size_t)ci * D * n + (size_t)cj * D;
    const double* Hb = a.Hij + p * D * D;
    const double* l1 = a.lam1 + p * m * m;
    const double* l2 = a.lam2 + p * m * m;
    for (int e = tid; e < D * D; e += NT) Xs[e] = Xb[(size_t)(e / D) * n + (e % D)];
    gsync<NT>();
    for (int e = tid; e < D * D; e += NT) {
      const int i = e / D, j = e % D;
      const int pa = i / m, pb = i % m, pc = j / m, pd = j % m;
      double x1 = Xs[(pa * m + pc) * D + (pd * m + pb)], x2 = Xs[(pc * m + pa) * D + (pb * m + pd)];
      if (a.fermionic) {
        if (parity_odd(pa, pd, pb)) x1 = -x1;
        if (parity_odd(pc, pb, pd)) x2 = -x2;
      }
      double k = Hb[e] - x1 - x2;
      if (pb == pd) k += l1[pa * m + pc];
      if (pa == pc) k += l2[pb * m + pd];
      A[i * LD + j] = k;
    }
    gsync<NT>();
    for (int t = tid; t < D * (D + 1) / 2; t += NT) {
      int i, j;
      tri_index(D, t, i, j);
      const double v = 0.5 * (A[i * LD + j] + A[j * LD + i]);
      A[i * LD + j] = v;
      A[j * LD + i] = v;
    }
    gsync<NT>();
    double off = 0.0;
    jacobi_sym<double, D, LD, NT, false>(A, nullptr, cs, red, tid, nullptr, &off);
    double v = INFINITY;
    for (int k = tid; k < D; k += NT) v = nan_min(v, A[k * LD + k]);
    v = gmin<NT>(v, red);
    // Weyl: lmin >= min diag - ||E||_F for the rotated diag + E; a NaN passes through
    if (tid == 0) lmin[p] = v - sqrt(off);
    gsync<NT>();
  }
}

// lmin of K_i = H'_i - sum_{j>i} Lambda1_ij - sum_{j<i} Lambda2_ji (a warp per cluster).
template <int m>
__global__ void __launch_bounds__(32) k5_bound_cluster(const GenArgs a, double* lmin) {
  constexpr int MM = m * m, D = MM, LD = m + 1;
  __shared__ double A[m * LD];
  __shared__ double cs[m < 2 ? 2 : m];
  __shared__ double red[2];
  const int i = blockIdx.x, t = threadIdx.x, N = a.N;
  const size_t n = (size_t)a.n;
  const double* Xii = a.X + (size_t)i * D * n + (size_t)i * D;
  for (int e = t; e < MM; e += 32) {
    const int b = e / m, d = e % m;
    double g = 0.0;
    for (int x = 0; x < m; ++x) g += Xii[(size_t)(x * m + b) * n + (x * m + d)];
    double k = a.Hi[(size_t)i * MM + e] - g;
    for (int j = 0; j < N; ++j) {
      if (j > i) k -= a.lam1[pair_index(N, i, j) * MM + e];
      else if (j < i) k -= a.lam2[pair_index(N, j, i) * MM + e];
    }
    A[b * LD + d] = k;
  }
  __syncwarp();
  for (int e = t; e < MM; e += 32) {
    const int b = e / m, d = e % m;
    if (b < d) {
      const double v = 0.5 * (A[b * LD + d] + A[d * LD + b]);
      A[b * LD + d] = v;
      A[d * LD + b] = v;
    }
  }
  __syncwarp();
  double off = 0.0;
  jacobi_sym<double, m, LD, 32, false>(A, nullptr, cs, red, t, nullptr, &off);
  double v = INFINITY;
  for (int k = t; k < m; k += 32) v = nan_min(v, A[k * LD + k]);
  v = gmin<32>(v, red);
  if (t == 0) lmin[i] = v - sqrt(off);  // Weyl, as in k5_bound_pair
}

template <int D>
cudaError_t launch_pair5(const GenArgs& a, cudaStream_t s) {
  const size_t smem = GenSmem<D>::bytes;
  static unsigned long long mask = 0;
  cudaError_t e = smem_once(k5_pair<D>, smem, mask);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k5_pair<D>, GroupShape<D>::NT, smem);
  long grid = (long)(sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  if (grid > a.K) grid = a.K;
  k5_pair<D><<<(unsigned)grid, GroupShape<D>::NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_bound_pair5(const GenArgs& a, double* lmin, cudaStream_t s) {
  constexpr int LD = GroupShape<D>::LD;
  const size_t smem = sizeof(double) * (D * D + D * LD + D + 32);
  static unsigned long long mask = 0;
  cudaError_t e = smem_once(k5_bound_pair<D>, smem, mask);
  if (e != cudaSuccess) return e;
  long grid = a.K < 4096 ? a.K : 4096;
  k5_bound_pair<D><<<(unsigned)grid, GroupShape<D>::NT, smem, s>>>(a, lmin);
  return cudaGetLastError();
}

template <int m>
cudaError_t launch_small5(const GenArgs& a, int which, double* lmin, cudaStream_t s) {
  switch (which) {
    case 0: k5_rho<m><<<(unsigned)a.N, 64, 0, s>>>(a); break;
    case 1: k5_dual<m><<<(unsigned)((a.K + 7) / 8), 256, 0, s>>>(a); break;
    default: k5_bound_cluster<m><<<(unsigned)a.N, 32, 0, s>>>(a, lmin); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_small(const GenArgs& a, int which, double* lmin, cudaStream_t s) {
  switch (a.m) {
    case 2: return launch_small5<2>(a, which, lmin, s);
    case 4: return launch_small5<4>(a, which, lmin, s);
    case 8: return launch_small5<8>(a, which, lmin, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gpair(const GenArgs& a, cudaStream_t s) {
  switch (a.D) {
    case 4: return launch_pair5<4>(a, s);
    case 16: return launch_pair5<16>(a, s);
    case 64: return launch_pair5<64>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gbound_pair(const GenArgs& a, double* lmin, cudaStream_t s) {
  switch (a.D) {
    case 4: return launch_bound_pair5<4>(a, lmin, s);
    case 16: return launch_bound_pair5<16>(a, lmin, s);
    case 64: return launch_bound_pair5<64>(a, lmin, s);
    default: return cudaErrorInvalidValue;
  }
}

// Add the k-spin operator op (2^k x 2^k, factor q on spin pos[q]) into out (2^nb x 2^nb) over nb
// spins, spin 0 the most significant Kronecker factor.
void embed(const double* op, int k, const int* pos, int nb, double* out) {
  const int dim = 1 << nb, kd = 1 << k;
  for (int col = 0; col < dim; ++col) {
    int sc = 0;
    for (int q = 0; q < k; ++q) sc = (sc << 1) | ((col >> (nb - 1 - pos[q])) & 1);
    for (int sr = 0; sr < kd; ++sr) {
      const double amp = op[sr * kd + sc];
      if (amp == 0.0) continue;
      int row = col;
      for (int q = 0; q < k; ++q) {
        const int sh = nb - 1 - pos[q];
        row = (row & ~(1 << sh)) | (((sr >> (k - 1 - q)) & 1) << sh);
      }
      out[(size_t)row * dim + col] += amp;
    }
  }
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace ve

using namespace ve;

struct ve_general {
  int N = 0, L = 0, m = 0, D = 0, n = 0;
  long K = 0;
  ve_options opt;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  void* dev = nullptr;
  size_t state_count = 0;  // doubles
  double *state = nullptr, *rho = nullptr, *rt = nullptr, *lam = nullptr, *lam1 = nullptr,
         *lam2 = nullptr, *X = nullptr;
  double *Hi = nullptr, *Hij = nullptr, *a1 = nullptr, *a2 = nullptr, *part = nullptr,
         *parti = nullptr, *Y = nullptr, *vstore = nullptr, *lmin_p = nullptr, *lmin_c = nullptr;
  int *pi = nullptr, *pj = nullptr;
  GenStatus *dst = nullptr, *hst = nullptr;
  DenseWs dws, bws;  // X-step eigensolver; the bound's eigensolve of X
  bool pair_warm = false;
  int fermionic = 0;
  long projections = 0;
  // profiling: 0 pair pass, 1 cluster + dual + status, 2 dense eigensolve, 3 reconstruction
  bool prof = false;
  cudaEvent_t ev[VE_GENERAL_NSTAGE + 1] = {};
  double prof_ms[VE_GENERAL_NSTAGE] = {};
  long prof_launch[VE_GENERAL_NSTAGE] = {};
  long prof_sweeps = 0, prof_solves = 0, prof_dk = 0;
};

namespace {

#define VG_CU(call)                         \
  do {                                      \
    cudaError_t _e = (call);                \
    if (_e != cudaSuccess) return VE_ECUDA; \
  } while (0)

struct Guard {
  int prev = -1;
  explicit Guard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != d) cudaSetDevice(d);
  }
  ~Guard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Every refresh-th projection restarts the X eigensolve from V = I, so that rounding in the
// rotated eigenvectors cannot accumulate over a long run.
constexpr long kRefresh = 256;

GenArgs gen_args(ve_general* h) {
  GenArgs a;
  a.N = h->N;
  a.m = h->m;
  a.D = h->D;
  a.n = h->n;
  a.L = h->L;
  a.K = h->K;
  a.mu = h->opt.mu;
  a.nu = h->opt.nu;
  a.eps = h->opt.eps;
  a.rho = h->rho;
  a.rt = h->rt;
  a.lam = h->lam;
  a.lam1 = h->lam1;
  a.lam2 = h->lam2;
  a.X = h->X;
  a.Y = h->Y;
  a.Hi = h->Hi;
  a.Hij = h->Hij;
  a.pi = h->pi;
  a.pj = h->pj;
  a.a1 = h->a1;
  a.a2 = h->a2;
  a.part = h->part;
  a.parti = h->parti;
  a.vstore = h->vstore;
  a.warm = h->pair_warm ? 1 : 0;
  a.fermionic = h->fermionic;
  a.st = h->dst;
  return a;
}

void stage_mark(ve_general* h, int k) {
  if (h->prof) cudaEventRecord(h->ev[k], h->stream);
}

int sweep(ve_general* h) {
  const cudaStream_t s = h->stream;
  GenArgs a = gen_args(h);
  stage_mark(h, 0);
  VG_CU(launch_gpair(a, s));
  stage_mark(h, 1);
  VG_CU(launch_small(a, 0, nullptr, s));
  VG_CU(launch_small(a, 1, nullptr, s));
  k5_status<<<1, 256, 0, s>>>(a);
  VG_CU(cudaGetLastError());
  h->pair_warm = true;
  stage_mark(h, 2);
  const long l0 = h->dws.launches;
  const int mode = (h->projections % kRefresh == 0) ? DENSE_COLD : DENSE_WARM;
  VG_CU(dense_eig(h->dws, h->Y, mode, s));
  const long l1 = h->dws.launches;
  stage_mark(h, 3);
  VG_CU(dense_reconstruct(h->dws, h->X, s));
  stage_mark(h, 4);
  ++h->projections;
  if (h->prof) {
    VG_CU(cudaEventSynchronize(h->ev[4]));
    for (int k = 0; k < VE_GENERAL_NSTAGE; ++k) {
      float ms = 0.f;
      VG_CU(cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1]));
      h->prof_ms[k] += ms;
    }
    h->prof_launch[0] += 1;
    h->prof_launch[1] += 3;
    h->prof_launch[2] += l1 - l0;
    h->prof_launch[3] += 1;
    h->prof_sweeps += h->dws.last_sweeps;
    h->prof_solves += 1;
    h->prof_dk += h->dws.dk_mode == 2 ? 1 : 0;
  }
  return VE_OK;
}

int read_status(ve_general* h, ve_status* out) {
  VG_CU(cudaMemcpyAsync(h->hst, h->dst, sizeof(GenStatus), cudaMemcpyDeviceToHost, h->stream));
  VG_CU(cudaStreamSynchronize(h->stream));
  ve_status s;
  s.iter = (long)h->hst->iter;
  s.energy_per_spin = h->hst->energy;
  s.feas_err = h->hst->feas;
  s.d_energy = h->hst->d_energy;
  s.residual = h->hst->residual;
  if (out) *out = s;
  if (h->hst->iter > 0 && (!isfinite(s.energy_per_spin) || !isfinite(s.feas_err))) return VE_ENONFINITE;
  return VE_OK;
}

void init_state_host(ve_general* h, std::vector<double>& v) {
  const int N = h->N, m = h->m, D = h->D, n = h->n;
  const long K = h->K;
  v.assign(h->state_count, 0.0);
  double* p = v.data();
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < m; ++k) p[(size_t)i * m * m + k * m + k] = 1.0 / m;
  p += (size_t)N * m * m;
  for (long q = 0; q < K; ++q)
    for (int k = 0; k < D; ++k) p[(size_t)q * D * D + k * D + k] = 1.0 / D;
  p += (size_t)K * D * D;  // rho~
  p += (size_t)K * D * D;  // Lambda
  p += (size_t)K * m * m * 2;
  for (int k = 0; k < n; ++k) p[(size_t)k * n + k] = 1.0;
}

void reset_status(ve_general* h) {
  GenStatus g;
  g.iter = 0;
  g.energy = g.feas = g.d_energy = g.residual = NAN;
  g.e_prev = NAN;
  *h->hst = g;
}

int check_shape(int N, int L) {
  if (L < 1 || N < 2) return VE_EINVAL;
  if (L > 3) return VE_EUNSUPPORTED;
  if ((long)N * (1 << (2 * L)) > DENSE_MAX_N) return VE_EUNSUPPORTED;
  return VE_OK;
}

int check_options(const ve_options* opt, ve_options& o) {
  ve_default_options(&o);
  if (opt) o = *opt;
  if (!(o.mu > 0) || !(o.nu > 0) || !(o.eps > 0) || o.check_every < 1) return VE_EINVAL;
  if (o.precision != VE_PREC_FP64) return VE_EUNSUPPORTED;
  return VE_OK;
}

// Jordan-Wigner images on nb sites in a fixed order (position 0 the most significant bit of a
// basis index, a site's bit set when it is occupied): a_p^dagger = Z ... Z sigma^- at position p,
// Z = diag(1, -1) on every earlier position.  Terms are added into out (2^nb x 2^nb).
int parity_before(int x, int nb, int p) {
  const int before = ((1 << nb) - 1) & ~((1 << (nb - p)) - 1);  // positions 0 .. p-1
  return __builtin_popcount((unsigned)(x & before)) & 1;
}

// t (a_p^dagger a_q + a_q^dagger a_p), p != q: each product applied to every basis state.
void jw_add_hop(double* out, int nb, int p, int q, double t) {
  const int dim = 1 << nb;
  for (int dir = 0; dir < 2; ++dir) {
    const int pc = dir ? q : p, pa = dir ? p : q;  // created, annihilated position
    const int bc = 1 << (nb - 1 - pc), ba = 1 << (nb - 1 - pa);
    for (int x = 0; x < dim; ++x) {
      if (!(x & ba) || (x & bc)) continue;
      const int y = x & ~ba;  // after a_pa: sign of the occupied positions before pa in x
      const int z = y | bc;   // after a_pc^dagger: those before pc in y
      const int odd = parity_before(x, nb, pa) ^ parity_before(y, nb, pc);
      out[(size_t)z * dim + x] += odd ? -t : t;
    }
  }
}

// v (n_p - 1/2)(n_q - 1/2): diagonal.
void jw_add_density(double* out, int nb, int p, int q, double v) {
  const int dim = 1 << nb;
  for (int x = 0; x < dim; ++x) {
    const double np = ((x >> (nb - 1 - p)) & 1) - 0.5, nq = ((x >> (nb - 1 - q)) & 1) - 0.5;
    out[(size_t)x * dim + x] += v * np * nq;
  }
}

int create_from_blocks(int N, int L, std::vector<double>& Hi, std::vector<double>& Hij, int fermionic,
                       const ve_options& o, ve_general** out);
void spin_blocks(const ve_terms* t, int L, std::vector<double>& Hi, std::vector<double>& Hij);
int check_spin_terms(const ve_terms* t, int L);

}  // namespace

extern "C" {

int ve_general_create(const ve_terms* t, int cluster_spins, const ve_options* opt, ve_general** out) {
  if (!out) return VE_EINVAL;
  *out = nullptr;
  const int L = cluster_spins;
  int rc = check_spin_terms(t, L);
  if (rc != VE_OK) return rc;
  ve_options o;
  if ((rc = check_options(opt, o)) != VE_OK) return rc;
  std::vector<double> Hi, Hij;
  spin_blocks(t, L, Hi, Hij);
  return create_from_blocks(t->nspins / L, L, Hi, Hij, 0, o, out);
}

}  // extern "C"

namespace {

// Cluster blocks of spin terms (Sec. 2.1 pairwise form): a term inside cluster c goes to H_c, a
// term between clusters c < c' to H_cc' with cluster c the first factor.
void spin_blocks(const ve_terms* t, int L, std::vector<double>& Hi, std::vector<double>& Hij) {
  const int N = t->nspins / L, m = 1 << L, D = m * m;
  const long K = (long)N * (N - 1) / 2;
  Hi.assign((size_t)N * m * m, 0.0);
  Hij.assign((size_t)K * D * D, 0.0);
  for (int sp = 0; sp < t->nspins; ++sp) {
    if (!t->onsite) break;
    const int pos = sp % L;
    embed(t->onsite + 4 * sp, 1, &pos, L, Hi.data() + (size_t)(sp / L) * m * m);
  }
  for (int b = 0; b < t->nbond; ++b) {
    const int s0 = t->bond_sites[2 * b], s1 = t->bond_sites[2 * b + 1];
    const int c0 = s0 / L, c1 = s1 / L;
    const double* B = t->bond_ops + 16 * b;
    if (c0 == c1) {
      const int pos[2] = {s0 % L, s1 % L};
      embed(B, 2, pos, L, Hi.data() + (size_t)c0 * m * m);
    } else if (c0 < c1) {
      const int pos[2] = {s0 % L, L + s1 % L};
      embed(B, 2, pos, 2 * L, Hij.data() + (size_t)pair_index(N, c0, c1) * D * D);
    } else {
      const int pos[2] = {L + s0 % L, s1 % L};
      embed(B, 2, pos, 2 * L, Hij.data() + (size_t)pair_index(N, c1, c0) * D * D);
    }
  }
}

// Eq. (sdpFerm): H_c is the Jordan-Wigner image of the terms inside cluster c in the cluster's
// site order; H_cc' (c < c') that of the terms between the two clusters, c's sites first.
void fermion_blocks(const ve_fermion_terms* t, int L, std::vector<double>& Hi, std::vector<double>& Hij) {
  const int N = t->nsites / L, m = 1 << L, D = m * m;
  const long K = (long)N * (N - 1) / 2;
  Hi.assign((size_t)N * m * m, 0.0);
  Hij.assign((size_t)K * D * D, 0.0);
  for (int k = 0; k < t->nhop + t->npair; ++k) {
    const bool hop = k < t->nhop;
    const int* st = hop ? t->hop_sites + 2 * k : t->pair_sites + 2 * (k - t->nhop);
    const double c = hop ? t->hop_t[k] : t->pair_v[k - t->nhop];
    const int s0 = st[0], s1 = st[1], c0 = s0 / L, c1 = s1 / L;
    double* blk;
    int nb, p0, p1;
    if (c0 == c1) {
      blk = Hi.data() + (size_t)c0 * m * m;
      nb = L;
      p0 = s0 % L;
      p1 = s1 % L;
    } else {
      const int g = c0 < c1 ? c0 : c1, d = c0 < c1 ? c1 : c0;
      blk = Hij.data() + (size_t)pair_index(N, g, d) * D * D;
      nb = 2 * L;
      p0 = (c0 == g ? 0 : L) + s0 % L;
      p1 = (c1 == g ? 0 : L) + s1 % L;
    }
    if (hop) {
      jw_add_hop(blk, nb, p0, p1, c);
    } else {
      jw_add_density(blk, nb, p0, p1, c);
    }
  }
}

int check_fermion_terms(const ve_fermion_terms* t, int L) {
  if (!t || L < 1 || t->nsites < 2 * L || t->nsites % L != 0 || t->nhop < 0 || t->npair < 0)
    return VE_EINVAL;
  if ((t->nhop > 0 && (!t->hop_sites || !t->hop_t)) || (t->npair > 0 && (!t->pair_sites || !t->pair_v)))
    return VE_EINVAL;
  const int rc = check_shape(t->nsites / L, L);
  if (rc != VE_OK) return rc;
  for (int k = 0; k < t->nhop + t->npair; ++k) {
    const int* st = k < t->nhop ? t->hop_sites + 2 * k : t->pair_sites + 2 * (k - t->nhop);
    if (st[0] < 0 || st[1] < 0 || st[0] >= t->nsites || st[1] >= t->nsites || st[0] == st[1])
      return VE_EINVAL;
  }
  return VE_OK;
}

int check_spin_terms(const ve_terms* t, int L) {
  if (!t || L < 1 || t->nspins < 2 * L || t->nspins % L != 0 || t->nbond < 0) return VE_EINVAL;
  if (t->nbond > 0 && (!t->bond_sites || !t->bond_ops)) return VE_EINVAL;
  const int rc = check_shape(t->nspins / L, L);
  if (rc != VE_OK) return rc;
  for (int b = 0; b < t->nbond; ++b) {
    const int s0 = t->bond_sites[2 * b], s1 = t->bond_sites[2 * b + 1];
    if (s0 < 0 || s1 < 0 || s0 >= t->nspins || s1 >= t->nspins || s0 == s1) return VE_EINVAL;
  }
  return VE_OK;
}

}  // namespace

extern "C" {

int ve_spin_blocks(const ve_terms* terms, int cluster_spins, double* Hi, double* Hij) {
  if (!Hi || !Hij) return VE_EINVAL;
  const int rc = check_spin_terms(terms, cluster_spins);
  if (rc != VE_OK) return rc;
  std::vector<double> a, b;
  spin_blocks(terms, cluster_spins, a, b);
  memcpy(Hi, a.data(), a.size() * sizeof(double));
  memcpy(Hij, b.data(), b.size() * sizeof(double));
  return VE_OK;
}

int ve_fermion_blocks(const ve_fermion_terms* terms, int cluster_sites, double* Hi, double* Hij) {
  if (!Hi || !Hij) return VE_EINVAL;
  const int rc = check_fermion_terms(terms, cluster_sites);
  if (rc != VE_OK) return rc;
  std::vector<double> a, b;
  fermion_blocks(terms, cluster_sites, a, b);
  memcpy(Hi, a.data(), a.size() * sizeof(double));
  memcpy(Hij, b.data(), b.size() * sizeof(double));
  return VE_OK;
}

int ve_general_create_fermions(const ve_fermion_terms* t, int cluster_sites, const ve_options* opt,
                               ve_general** out) {
  if (!out) return VE_EINVAL;
  *out = nullptr;
  int rc = check_fermion_terms(t, cluster_sites);
  if (rc != VE_OK) return rc;
  ve_options o;
  if ((rc = check_options(opt, o)) != VE_OK) return rc;
  std::vector<double> Hi, Hij;
  fermion_blocks(t, cluster_sites, Hi, Hij);
  return create_from_blocks(t->nsites / cluster_sites, cluster_sites, Hi, Hij, 1, o, out);
}

}  // extern "C"

namespace {

int create_from_blocks(int N, int L, std::vector<double>& Hi, std::vector<double>& Hij, int fermionic,
                       const ve_options& o, ve_general** out) {
  const int m = 1 << L, D = m * m;
  const long n = (long)N * D;
  const long K = (long)N * (N - 1) / 2;
  std::vector<int> pi(K), pj(K);
  for (int i = 0, p = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j, ++p) {
      pi[p] = i;
      pj[p] = j;
    }

  ve_general* h = new (std::nothrow) ve_general();
  if (!h) return VE_ENOMEM;
  h->N = N;
  h->L = L;
  h->m = m;
  h->D = D;
  h->n = (int)n;
  h->K = K;
  h->opt = o;
  h->fermionic = fermionic;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return VE_ECUDA;
  }
  h->state_count = (size_t)N * m * m + (size_t)K * (2 * D * D + 2 * m * m) + (size_t)n * n;
  const size_t nd = (size_t)n * n;
  const size_t dense = dense_ws_bytes((int)n);
  size_t bytes = al256(h->state_count * 8) + al256(Hi.size() * 8) + al256(Hij.size() * 8) +
                 2 * al256((size_t)K * m * m * 8) + al256((size_t)K * 3 * 8) + al256((size_t)N * 8) +
                 al256(nd * 8) + al256((size_t)K * D * D * 8) + al256((size_t)K * 8) + al256((size_t)N * 8) +
                 2 * al256((size_t)K * 4) + al256(sizeof(GenStatus)) + 2 * dense;
  if (cudaMalloc(&h->dev, bytes) != cudaSuccess) {
    delete h;
    return VE_ENOMEM;
  }
  unsigned char* p = (unsigned char*)h->dev;
  auto take = [&](size_t b) {
    unsigned char* q = p;
    p += al256(b);
    return q;
  };
  h->state = (double*)take(h->state_count * 8);
  h->rho = h->state;
  h->rt = h->rho + (size_t)N * m * m;
  h->lam = h->rt + (size_t)K * D * D;
  h->lam1 = h->lam + (size_t)K * D * D;
  h->lam2 = h->lam1 + (size_t)K * m * m;
  h->X = h->lam2 + (size_t)K * m * m;
  h->Hi = (double*)take(Hi.size() * 8);
  h->Hij = (double*)take(Hij.size() * 8);
  h->a1 = (double*)take((size_t)K * m * m * 8);
  h->a2 = (double*)take((size_t)K * m * m * 8);
  h->part = (double*)take((size_t)K * 3 * 8);
  h->parti = (double*)take((size_t)N * 8);
  h->Y = (double*)take(nd * 8);
  h->vstore = (double*)take((size_t)K * D * D * 8);
  h->lmin_p = (double*)take((size_t)K * 8);
  h->lmin_c = (double*)take((size_t)N * 8);
  h->pi = (int*)take((size_t)K * 4);
  h->pj = (int*)take((size_t)K * 4);
  h->dst = (GenStatus*)take(sizeof(GenStatus));
  void* dmem = take(dense);
  void* bmem = take(dense);
  int rc = VE_OK;
  if (dense_ws_init(h->dws, (int)n, dmem, dense) != 0 || dense_ws_init(h->bws, (int)n, bmem, dense) != 0)
    rc = VE_EINVAL;
  // the X step may end with the first-order correction; the bound's eigensolve of X stays exact
  h->dws.allow_dk = true;
  if (rc == VE_OK) {
    if (o.stream) {
      h->stream = (cudaStream_t)o.stream;
    } else if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) == cudaSuccess) {
      h->own_stream = true;
    } else {
      rc = VE_ECUDA;
    }
  }
  if (rc == VE_OK && cudaMallocHost((void**)&h->hst, sizeof(GenStatus)) != cudaSuccess) rc = VE_ENOMEM;
  if (rc == VE_OK) {
    std::vector<double> init;
    init_state_host(h, init);
    reset_status(h);
    const cudaStream_t s = h->stream;
    if (cudaMemcpyAsync(h->state, init.data(), init.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->Hi, Hi.data(), Hi.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->Hij, Hij.data(), Hij.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->pi, pi.data(), (size_t)K * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->pj, pj.data(), (size_t)K * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(h->Y, 0, nd * 8, s) != cudaSuccess ||
        cudaMemcpyAsync(h->dst, h->hst, sizeof(GenStatus), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = VE_ECUDA;
  }
  for (int k = 0; rc == VE_OK && k <= VE_GENERAL_NSTAGE; ++k)
    if (cudaEventCreate(&h->ev[k]) != cudaSuccess) rc = VE_ECUDA;
  if (rc != VE_OK) {
    ve_general_destroy(h);
    return rc;
  }
  *out = h;
  return VE_OK;
}

}  // namespace

extern "C" {

void ve_general_destroy(ve_general* h) {
  if (!h) return;
  Guard g(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  dense_ws_release(h->dws);
  dense_ws_release(h->bws);
  for (int k = 0; k <= VE_GENERAL_NSTAGE; ++k)
    if (h->ev[k]) cudaEventDestroy(h->ev[k]);
  if (h->hst) cudaFreeHost(h->hst);
  if (h->dev) cudaFree(h->dev);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int ve_general_dims(const ve_general* h, int* N, int* m, int* D, long* K) {
  if (!h) return VE_EINVAL;
  if (N) *N = h->N;
  if (m) *m = h->m;
  if (D) *D = h->D;
  if (K) *K = h->K;
  return VE_OK;
}

int ve_general_iterate(ve_general* h, long max_iter, double tol, ve_status* out) {
  if (!h || max_iter < 0) return VE_EINVAL;
  Guard g(h->device);
  ve_status s;
  if (max_iter == 0) {
    const int r = read_status(h, &s);
    if (out) *out = s;
    return r;
  }
  long done = 0;
  int rc = VE_NOT_CONVERGED;
  while (done < max_iter) {
    const long chunk = h->opt.check_every < max_iter - done ? (long)h->opt.check_every : max_iter - done;
    for (long k = 0; k < chunk; ++k) {
      const int r = sweep(h);
      if (r != VE_OK) return r;
    }
    done += chunk;
    const int r = read_status(h, &s);
    if (r == VE_ENONFINITE) {
      if (out) *out = s;
      return r;
    }
    if (r != VE_OK) return r;
    if (tol > 0 && s.residual <= tol) {
      rc = VE_OK;
      break;
    }
  }
  if (out) *out = s;
  return tol <= 0 ? VE_OK : rc;
}

int ve_general_get_status(ve_general* h, ve_status* out) {
  if (!h || !out) return VE_EINVAL;
  Guard g(h->device);
  return read_status(h, out);
}

int ve_general_bound(ve_general* h, ve_cert* out) {
  if (!h || !out) return VE_EINVAL;
  Guard g(h->device);
  const cudaStream_t s = h->stream;
  GenArgs a = gen_args(h);
  VG_CU(launch_gbound_pair(a, h->lmin_p, s));
  VG_CU(launch_small(a, 2, h->lmin_c, s));
  // lmin(X): the eigensolve starts from the X step's eigenvectors (those of Y, which X shares)
  const size_t nd = (size_t)h->n * h->n * sizeof(double);
  VG_CU(cudaMemcpyAsync(h->bws.Vt, h->dws.Vt, nd, cudaMemcpyDeviceToDevice, s));
  VG_CU(dense_eig(h->bws, h->X, h->projections > 0 ? DENSE_WARM : DENSE_COLD, s));
  VG_CU(dense_lmin_certified(h->bws, s));
  std::vector<double> lp((size_t)h->K), lc((size_t)h->N);
  DenseCtl ctl;
  VG_CU(cudaMemcpyAsync(lp.data(), h->lmin_p, lp.size() * 8, cudaMemcpyDeviceToHost, s));
  VG_CU(cudaMemcpyAsync(lc.data(), h->lmin_c, lc.size() * 8, cudaMemcpyDeviceToHost, s));
  VG_CU(cudaMemcpyAsync(&ctl, h->bws.ctl, sizeof(DenseCtl), cudaMemcpyDeviceToHost, s));
  ve_status st;
  const int r = read_status(h, &st);  // synchronises
  if (r != VE_OK) return r;  // a non-finite iterate certifies nothing
  double raw = 0.0;
  for (double v : lc) raw += v;
  for (double v : lp) raw += v;
  const double xmin = ctl.lmin;
  // every minimum passes a NaN on, and an Inf stays in the sum: one check covers them all
  if (!std::isfinite(raw) || !std::isfinite(xmin)) return VE_ENONFINITE;
  const double corr = (double)h->N * h->m * (xmin < 0 ? -xmin : 0.0);
  out->raw_bound = raw;
  out->x_min_eig = xmin;
  out->x_neg_correction = corr;
  out->bound_per_spin = (raw - corr) / ((double)h->N * h->L);
  out->primal_per_spin = st.energy_per_spin;
  return VE_OK;
}

size_t ve_general_state_size(const ve_general* h) { return h ? h->state_count * sizeof(double) : 0; }

int ve_general_get_state(ve_general* h, double* host, size_t bytes) {
  if (!h || !host || bytes != h->state_count * sizeof(double)) return VE_EINVAL;
  Guard g(h->device);
  VG_CU(cudaMemcpyAsync(host, h->state, bytes, cudaMemcpyDeviceToHost, h->stream));
  VG_CU(cudaStreamSynchronize(h->stream));
  return VE_OK;
}

int ve_general_set_state(ve_general* h, const double* host, size_t bytes) {
  if (!h || !host || bytes != h->state_count * sizeof(double)) return VE_EINVAL;
  Guard g(h->device);
  VG_CU(cudaMemcpyAsync(h->state, host, bytes, cudaMemcpyHostToDevice, h->stream));
  VG_CU(cudaMemcpyAsync(h->hst, h->dst, sizeof(GenStatus), cudaMemcpyDeviceToHost, h->stream));
  VG_CU(cudaStreamSynchronize(h->stream));
  h->hst->e_prev = NAN;
  VG_CU(cudaMemcpyAsync(h->dst, h->hst, sizeof(GenStatus), cudaMemcpyHostToDevice, h->stream));
  VG_CU(cudaStreamSynchronize(h->stream));
  return VE_OK;
}

int ve_general_profile(ve_general* h, int enable) {
  if (!h) return VE_EINVAL;
  h->prof = enable != 0;
  h->dws.prof = h->prof;
  h->dws.graph_ms = 0.0;
  h->dws.graph_rounds = 0;
  for (int k = 0; k < VE_GENERAL_NSTAGE; ++k) {
    h->prof_ms[k] = 0.0;
    h->prof_launch[k] = 0;
  }
  h->prof_sweeps = h->prof_solves = h->prof_dk = 0;
  return VE_OK;
}

int ve_general_profile_read(ve_general* h, double* ms, long* launches, double* jacobi_sweeps) {
  if (!h) return VE_EINVAL;
  for (int k = 0; k < VE_GENERAL_NSTAGE; ++k) {
    if (ms) ms[k] = h->prof_ms[k];
    if (launches) launches[k] = h->prof_launch[k];
  }
  if (jacobi_sweeps) *jacobi_sweeps = h->prof_solves ? (double)h->prof_sweeps / h->prof_solves : 0.0;
  return VE_OK;
}

int ve_general_profile_rounds(ve_general* h, double* ms, long* rounds, long* first_order) {
  if (!h) return VE_EINVAL;
  if (ms) *ms = h->dws.graph_ms;
  if (rounds) *rounds = h->dws.graph_rounds;
  if (first_order) *first_order = h->prof_dk;
  return VE_OK;
}

// ---- standalone dense projection
size_t ve_project_psd_dense_workspace_size(int n) { return dense_ws_bytes(n); }

int ve_project_psd_dense(const double* in, double* out, int n, int flags, void* workspace,
                         size_t workspace_bytes, void* stream, int* sweeps) {
  if (!in || !out || dense_ws_bytes(n) == 0 || (flags & ~(VE_DENSE_WARM | VE_DENSE_FIRST_ORDER)))
    return VE_EINVAL;
  DenseWs w;
  if (dense_ws_init(w, n, workspace, workspace_bytes) != 0) return VE_EINVAL;
  w.allow_dk = (flags & VE_DENSE_FIRST_ORDER) != 0;
  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = dense_eig(w, in, (flags & VE_DENSE_WARM) ? DENSE_WARM : DENSE_COLD, s);
  if (e == cudaSuccess) e = dense_reconstruct(w, out, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (sweeps) *sweeps = w.last_sweeps + (w.dk_mode == 2 ? 1000 : 0);
  dense_ws_release(w);
  return e == cudaSuccess ? VE_OK : VE_ECUDA;
}

}  // extern "C"
