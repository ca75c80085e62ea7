// ve_sweep.cu -- the pair pass and the small reductions of one sweep of Algorithm 6
// (Khoo & Lindsey, arXiv:2106.02682, Sec. 3.3).
//
// k_pair     : one thread group per pair offset delta != 0.  Fuses the effective pair
//              Hamiltonian (Eq. (effHam)), the closed-form pair update (Eq. (rhoijUpdate)),
//              the PSD projection (Eq. (rhoijTildeUpdate)), the Lambda update, the X' = X - eps G
//              step for the block (Algorithm 6), the partial traces A1 rho, A2 rho and the
//              per-delta terms of Eq. (feasErr) and of the energy.
//              The offsets delta and -delta describe the same pairs of clusters seen from
//              either end, and the update commutes with exchanging the two clusters (S): from a
//              state with rho~_{-delta} = S rho~_delta S, Lambda likewise, Lambda1_{-delta} =
//              Lambda2_delta and X_{0,-delta} = X_{0,delta}^T, the -delta results are the swap
//              images of the delta ones.  So one group updates the canonical member of each
//              pair {delta, -delta} and writes the images for the other: half the eigensolves.
// k_rho0     : rho_0 update (Eq. (rhoiUpdate), translation-invariant form) with the trace
//              shift, and X'_00 = X_00 - eps G_00[rho_0]: every CTA sums a chunk of offsets, the
//              last CTA to finish adds the chunk sums and updates rho_0.
// k_dual12   : Lambda1/Lambda2 updates (they need the new rho_0) and their feasibility terms.
// k_status   : energy per spin, Eq. (feasErr), |energy change|, residual (CTA sums, then
//              the last CTA).
// All reductions run in a fixed order, so a sweep is bitwise reproducible.
#include "ve_device.cuh"
#include "ve_internal.h"

namespace ve {

namespace {

template <int D>
struct PairShape {
  static constexpr int m = ClusterDim<D>::m;
  static constexpr int NT = GroupShape<D>::NT;
  static constexpr int LD = GroupShape<D>::LD;
  static constexpr int GPC = GroupShape<D>::GPC;  // groups per CTA
};

template <int D, typename T>
struct PairSmem {
  static constexpr int m = PairShape<D>::m, LD = PairShape<D>::LD;
  static constexpr size_t al(size_t x) { return ((x + 15) / 16) * 16; }
  // per group, in bytes; every array 16-byte aligned
  static constexpr size_t R = 0;                                   // T D*D  (rhs, then rho)
  static constexpr size_t Xs = R + al(sizeof(T) * D * D);          // T D*D  (X_{0,delta})
  static constexpr size_t A = Xs + al(sizeof(T) * D * D);          // T D*LD
  static constexpr size_t V = A + al(sizeof(T) * D * LD);
  static constexpr size_t WT = V + al(sizeof(T) * D * LD);         // T D*LD
  static constexpr size_t CS = WT + al(sizeof(T) * D * LD);        // T D
  static constexpr size_t W = CS + al(sizeof(T) * D);              // T D
  static constexpr size_t TR = W + al(sizeof(T) * D);              // T 2*m*m + 2
  static constexpr size_t RED = TR + al(sizeof(T) * (2 * m * m + 2));
  static constexpr size_t bytes = RED + al(sizeof(T) * 32);
};

// Arithmetic in T (double, or float in the mixed-precision sweep); the state stays float64.
template <int D, typename T>
__global__ void __launch_bounds__(PairShape<D>::NT * PairShape<D>::GPC, GroupShape<D>::MINB)
    k_pair(const PairArgs a) {
  constexpr int m = PairShape<D>::m, NT = PairShape<D>::NT, LD = PairShape<D>::LD;
  constexpr int GPC = PairShape<D>::GPC;
  // register-tiled warp products (rgemm16) in float32 only: they compute whole 16 x 16 results
  // where the loops below compute triangles, and float64 / double-float issue is the bound there
  constexpr bool TILE16 = D == 16 && NT == 32 && std::is_same<T, float>::value;
  using S = PairSmem<D, T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = threadIdx.x / NT, tid = threadIdx.x % NT;
  unsigned char* base = GroupShape<D>::GLOBAL ? a.gws + (size_t)blockIdx.x * S::bytes
                                              : smem_raw + (size_t)g * S::bytes;
  T* R = reinterpret_cast<T*>(base + S::R);
  T* Xs = reinterpret_cast<T*>(base + S::Xs);
  T* A = reinterpret_cast<T*>(base + S::A);
  T* V = reinterpret_cast<T*>(base + S::V);
  T* Wt = reinterpret_cast<T*>(base + S::WT);
  T* cs = reinterpret_cast<T*>(base + S::CS);
  T* W = reinterpret_cast<T*>(base + S::W);
  T* t1 = reinterpret_cast<T*>(base + S::TR);
  T* t2 = t1 + m * m;
  T* red = reinterpret_cast<T*>(base + S::RED);

  const T mu = (T)a.mu, nu = (T)a.nu, eps = (T)a.eps;
  const T alpha = nu * m;
  const T c0 = T(1) / mu, c1 = T(1) / (mu + alpha), c2 = T(1) / (mu + T(2) * alpha);
  const T imu = T(1) / mu;

  for (long it = (long)blockIdx.x * GPC + g; it < a.Pc; it += (long)gridDim.x * GPC) {
    const long p = a.pidx ? a.pidx[it] : it;
    const long pm = a.pidx ? a.pmir[it] : -1;  // pair index of -delta, or -1
    const long dl = p + 1;  // linear cluster offset delta
    const double* rt = a.rt + p * D * D;
    const double* lam = a.lam + p * D * D;
    const double* l1 = a.lam1 + p * m * m;
    const double* l2 = a.lam2 + p * m * m;
    double* Xb = a.X + dl * D * D;
    const int hs = a.hslot[dl];
    const double* Hb = hs >= 0 ? a.hb + (long)hs * D * D : nullptr;

    for (int e = tid; e < D * D; e += NT) Xs[e] = (T)Xb[e];
    if (pm >= 0) {
      // the multipliers of -delta as images of these, before the rho_0 reduction reads them
      for (int idx = tid; idx < m * m; idx += NT) {
        a.lam1[pm * m * m + idx] = l2[idx];
        a.lam2[pm * m * m + idx] = l1[idx];
      }
    }
    gsync<NT>();
    // right-hand side of Eq. (rhoijUpdate) with H' of Eq. (effHam)
    for (int e = tid; e < D * D; e += NT) {
      const int i = e / D, j = e % D;
      const int pa = i / m, pb = i % m, pc = j / m, pd = j % m;
      const T h = Hb ? (T)Hb[e] : T(0);
      // (R^* X)_{(a,b),(c,d)} = X_{(a,c),(d,b)} and its transpose X_{(c,a),(b,d)}
      const T hp = h - Xs[(pa * m + pc) * D + (pd * m + pb)] - Xs[(pc * m + pa) * D + (pb * m + pd)];
      T y = mu * (T)rt[e] + (T)lam[e] - hp;
      if (pb == pd) y += nu * (T)a.rho0[pa * m + pc] - (T)l1[pa * m + pc];
      if (pa == pc) y += nu * (T)a.rho0[pb * m + pd] - (T)l2[pb * m + pd];
      R[e] = y;
    }
    gsync<NT>();
    // partial traces of the right-hand side
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
    // rho = (mu + nu A1^*A1 + nu A2^*A2)^{-1} rhs, closed form on the projectors P1, P2, Q
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
    T* vs = reinterpret_cast<T*>(a.vstore) + p * D * D;
    int nsw = 0;
    bool dk = false;  // the eigensolve stopped early: reconstruct with the first-order correction
    if (a.warm) {
      for (int e = tid; e < D * D; e += NT) V[(e / D) * LD + (e % D)] = vs[e];
      gsync<NT>();
      if (ns_due<T>(a.iter) && TILE16) {
        // as below, register-tiled warp products
        T acc[2][4];
        rgemm16<T, true, false>(V, LD, V, LD, acc, tid);
        const int r0 = 2 * (tid >> 2), c0 = 4 * (tid & 3);
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[x][u] = ((r0 + x == c0 + u) ? T(1.5) : T(0)) - T(0.5) * acc[x][u];
        store16(Wt, LD, acc, tid);
        __syncwarp();
        rgemm16<T, false, false>(V, LD, Wt, LD, acc, tid);
        __syncwarp();
        store16(V, LD, acc, tid);
        __syncwarp();
      } else if (ns_due<T>(a.iter)) {
        // rotations erode V's orthogonality over many sweeps; one Newton-Schulz step
        // V <- V (3 I - V^T V) / 2 squares the error before V is used (A and Wt as scratch)
        for (int e = tid; e < D * D; e += NT) {
          const int i = e / D, j = e % D;
          T acc = T(0);
          for (int k = 0; k < D; ++k) acc += V[k * LD + i] * V[k * LD + j];
          Wt[i * LD + j] = ((i == j) ? T(1.5) : T(0)) - T(0.5) * acc;
        }
        gsync<NT>();
        for (int e = tid; e < D * D; e += NT) {
          const int i = e / D, j = e % D;
          T acc = T(0);
          for (int k = 0; k < D; ++k) acc += V[i * LD + k] * Wt[k * LD + j];
          A[i * LD + j] = acc;
        }
        gsync<NT>();
        for (int e = tid; e < D * D; e += NT) V[(e / D) * LD + (e % D)] = A[(e / D) * LD + (e % D)];
        gsync<NT>();
      }
    }
    // C = rho - Lambda / mu, symmetrised, into A
    for (int t = tid; t < D * (D + 1) / 2; t += NT) {
      int i, j;
      tri_index(D, t, i, j);
      const T v = T(0.5) * (R[i * D + j] + R[j * D + i]) -
                  T(0.5) * ((T)lam[i * D + j] + (T)lam[j * D + i]) * imu;
      A[i * LD + j] = v;
      A[j * LD + i] = v;
    }
    gsync<NT>();
    if (a.warm && TILE16) {
      // A <- V^T C V with register-tiled warp products (upper triangle mirrored)
      T acc[2][4];
      rgemm16<T, false, false>(A, LD, V, LD, acc, tid);
      store16(Wt, LD, acc, tid);
      __syncwarp();
      rgemm16<T, true, false>(V, LD, Wt, LD, acc, tid);
      store16(A, LD, acc, tid);
      mirror16<T>(A, nullptr, LD, tid);
      nsw = jacobi_sym<T, D, LD, NT, true, false, true>(A, V, cs, red, tid, &dk);
    } else if (a.warm) {
      // start from the previous eigenvectors: A <- V^T C V
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
      nsw = jacobi_sym<T, D, LD, NT, true, false, true>(A, V, cs, red, tid, &dk);
    } else {
      nsw = jacobi_sym<T, D, LD, NT, true, true, true>(A, V, cs, red, tid, &dk);
    }
    if (a.stats && tid == 0) {
      atomicAdd(a.stats, (unsigned long long)nsw);
      atomicAdd(a.stats + 1, 1ull);
      if (dk) atomicAdd(a.stats + 2, 1ull);
    }
    for (int e = tid; e < D * D; e += NT) vs[e] = V[(e / D) * LD + (e % D)];
    if (TILE16) {
      // rho~ = V M V^T (M = f(Lambda) + L o E after a first-order stop, else diag(max(l, 0)))
      // with register-tiled warp products; the upper triangle is mirrored
      T acc[2][4];
      if (dk) {
        dk_matrix_sym<T, D, LD, NT>(A, cs, tid);
        rgemm16<T, false, false>(V, LD, A, LD, acc, tid);
        store16(Wt, LD, acc, tid);
        __syncwarp();
        rgemm16<T, false, true>(Wt, LD, V, LD, acc, tid);
      } else {
        for (int k = tid; k < D; k += NT) {
          const T w = A[k * LD + k];
          W[k] = w > T(0) ? w : T(0);
        }
        __syncwarp();
        rgemm16<T, false, true>(V, LD, V, LD, acc, tid, W);
      }
      __syncwarp();
      store16(A, LD, acc, tid);
      mirror16<T>(A, nullptr, LD, tid);
    } else if (dk) {
      // rho~ = V M V^T with M = f(Lambda) + L o E (dk_stop): Wt = V M, then Wt V^T
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
      // rho~ = V diag(max(w, 0)) V^T
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
    // swap images for -delta: rho~ and Lambda conjugated by S, X' transposed
    double* rtm = pm >= 0 ? a.rt + pm * D * D : nullptr;
    double* lamm = pm >= 0 ? a.lam + pm * D * D : nullptr;
    double* Xm = pm >= 0 ? a.X + (pm + 1) * D * D : nullptr;
    for (int e = tid; e < D * D; e += NT) {
      const int i = e / D, j = e % D;
      const int pa = i / m, pb = i % m, pc = j / m, pd = j % m;
      const T rho = R[e];
      const T rtn = A[i * LD + j];
      const T h = Hb ? (T)Hb[e] : T(0);
      const double lamn = (double)((T)lam[e] + mu * (rtn - rho));
      // X'_{0,delta} = X_{0,delta} - eps G_{0,delta}[rho], G entry (a,b),(c,d) = rho_{(a,d),(b,c)}
      const double xn = (double)(Xs[e] - eps * R[(pa * m + pd) * D + (pb * m + pc)]);
      lamw[e] = lamn;
      rtw[e] = (double)rtn;
      Xb[e] = xn;
      if (pm >= 0) {
        const int es = (pb * m + pa) * D + (pd * m + pc);
        lamm[es] = lamn;
        rtm[es] = (double)rtn;
        Xm[j * D + i] = xn;
      }
      rr += (rho - rtn) * (rho - rtn);
      en += h * R[j * D + i];
    }
    for (int idx = tid; idx < m * m; idx += NT) {
      const int x = idx / m, z = idx % m;
      T s1 = T(0), s2 = T(0);
      for (int k = 0; k < m; ++k) {
        s1 += R[(x * m + k) * D + (z * m + k)];
        s2 += R[(k * m + x) * D + (k * m + z)];
      }
      a.a1r[p * m * m + idx] = (double)s1;
      a.a2r[p * m * m + idx] = (double)s2;
      if (pm >= 0) {
        a.a1r[pm * m * m + idx] = (double)s2;
        a.a2r[pm * m * m + idx] = (double)s1;
      }
    }
    rr = gsum<NT>(rr, red);
    en = gsum<NT>(en, red);
    if (tid == 0) {
      a.part[p * 2 + 0] = (double)rr;
      a.part[p * 2 + 1] = (double)en;
      if (pm >= 0) {
        a.part[pm * 2 + 0] = (double)rr;
        a.part[pm * 2 + 1] = (double)en;
      }
    }
    gsync<NT>();
  }
}

// ---- D = 256 in float32 with the projection on the tensor cores (ve_tcproj.cu): the pair
// pass splits around one batched projection.  k_pair256_pre forms rho (Eq. (rhoijUpdate)) into
// rbuf and C = rho - Lambda / mu (symmetrised) into the projection's split input; after
// tc_project256, k_pair256_post does what k_pair does after its eigensolve.  Arithmetic in
// float32, as k_pair<256, float>.
constexpr int P256_NT = 512;

__device__ __forceinline__ float tf32_part(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__global__ void __launch_bounds__(P256_NT) k_pair256_pre(const PairArgs a, float* __restrict__ Cout) {
  constexpr int D = 256, m = 16, NT = P256_NT, PL = D * D;
  __shared__ float t1[m * m], t2[m * m];
  __shared__ float rho0[m * m];
  const int tid = threadIdx.x;
  const float mu = (float)a.mu, nu = (float)a.nu;
  const float alpha = nu * m;
  const float c0 = 1.f / mu, c1 = 1.f / (mu + alpha), c2 = 1.f / (mu + 2.f * alpha);
  const float imu = 1.f / mu;
  for (int k = tid; k < m * m; k += NT) rho0[k] = (float)a.rho0[k];
  for (long it = blockIdx.x; it < a.Pc; it += gridDim.x) {
    const long p = a.pidx ? a.pidx[it] : it;
    const long pm = a.pidx ? a.pmir[it] : -1;
    const long dl = p + 1;
    const double* rt = a.rt + p * PL;
    const double* lam = a.lam + p * PL;
    const double* l1 = a.lam1 + p * m * m;
    const double* l2 = a.lam2 + p * m * m;
    const double* Xb = a.X + dl * PL;
    const int hs = a.hslot[dl];
    const double* Hb = hs >= 0 ? a.hb + (long)hs * PL : nullptr;
    float* R = a.rbuf + it * PL;
    if (pm >= 0) {
      for (int idx = tid; idx < m * m; idx += NT) {
        a.lam1[pm * m * m + idx] = l2[idx];
        a.lam2[pm * m * m + idx] = l1[idx];
      }
    }
    __syncthreads();
    // right-hand side of Eq. (rhoijUpdate) with H' of Eq. (effHam)
    for (int e = tid; e < PL; e += NT) {
      const int i = e / D, j = e % D;
      const int pa = i / m, pb = i % m, pc = j / m, pd = j % m;
      const float h = Hb ? (float)Hb[e] : 0.f;
      const float hp = h - (float)Xb[(pa * m + pc) * D + (pd * m + pb)] - (float)Xb[(pc * m + pa) * D + (pb * m + pd)];
      float y = mu * (float)rt[e] + (float)lam[e] - hp;
      if (pb == pd) y += nu * rho0[pa * m + pc] - (float)l1[pa * m + pc];
      if (pa == pc) y += nu * rho0[pb * m + pd] - (float)l2[pb * m + pd];
      R[e] = y;
    }
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += NT) {
      const int x = idx / m, z = idx % m;
      float s1 = 0.f, s2 = 0.f;
      for (int k = 0; k < m; ++k) {
        s1 += R[(x * m + k) * D + (z * m + k)];
        s2 += R[(k * m + x) * D + (k * m + z)];
      }
      t1[idx] = s1;
      t2[idx] = s2;
    }
    __syncthreads();
    float tr = 0.f;
    for (int k = 0; k < m; ++k) tr += t1[k * m + k];
    for (int e = tid; e < PL; e += NT) {
      const int i = e / D, j = e % D;
      const int pa = i / m, pb = i % m, pc = j / m, pd = j % m;
      const float y = R[e];
      const float P1 = (pb == pd) ? t1[pa * m + pc] / m : 0.f;
      const float P2 = (pa == pc) ? t2[pb * m + pd] / m : 0.f;
      const float Q = (i == j) ? tr / D : 0.f;
      R[e] = (y - P1 - P2 + Q) * c0 + (P1 + P2 - 2.f * Q) * c1 + Q * c2;
    }
    __syncthreads();
    // C = rho - Lambda / mu, symmetrised, split into the KC4 input of the projection
    float* C = Cout + it * 2 * PL;
    for (int q = tid; q < PL / 4; q += NT) {
      const int r = q % D, k0 = (q / D) * 4;
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = k0 + u;
        v[u] = 0.5f * (R[r * D + j] + R[j * D + r]) - 0.5f * ((float)lam[r * D + j] + (float)lam[j * D + r]) * imu;
      }
      float4 hi, lo;
      hi = make_float4(tf32_part(v[0]), tf32_part(v[1]), tf32_part(v[2]), tf32_part(v[3]));
      lo = make_float4(v[0] - hi.x, v[1] - hi.y, v[2] - hi.z, v[3] - hi.w);
      *reinterpret_cast<float4*>(C + 4 * q) = hi;
      *reinterpret_cast<float4*>(C + PL + 4 * q) = lo;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(P256_NT) k_pair256_post(const PairArgs a, const float* __restrict__ Y) {
  constexpr int D = 256, m = 16, NT = P256_NT, PL = D * D;
  __shared__ float red[NT / 32];
  const int tid = threadIdx.x;
  const float mu = (float)a.mu, eps = (float)a.eps;
  for (long it = blockIdx.x; it < a.Pc; it += gridDim.x) {
    const long p = a.pidx ? a.pidx[it] : it;
    const long pm = a.pidx ? a.pmir[it] : -1;
    const long dl = p + 1;
    const float* R = a.rbuf + it * PL;
    const float* y = Y + it * 2 * PL;
    double* Xb = a.X + dl * PL;
    const int hs = a.hslot[dl];
    const double* Hb = hs >= 0 ? a.hb + (long)hs * PL : nullptr;
    double* rtw = a.rt + p * PL;
    double* lamw = a.lam + p * PL;
    double* rtm = pm >= 0 ? a.rt + pm * PL : nullptr;
    double* lamm = pm >= 0 ? a.lam + pm * PL : nullptr;
    double* Xm = pm >= 0 ? a.X + (pm + 1) * PL : nullptr;
    float rr = 0.f, en = 0.f;
    // X' reads X_{0,delta} before this item overwrites it: each thread rewrites only entries
    // it has read (e), and the transposed image goes to another block (-delta)
    for (int e = tid; e < PL; e += NT) {
      const int i = e / D, j = e % D;
      const int pa = i / m, pb = i % m, pc = j / m, pd = j % m;
      const float rho = R[e];
      const int o = ((j >> 2) * D + i) * 4 + (j & 3);
      const float rtn = y[o] + y[PL + o];
      const float h = Hb ? (float)Hb[e] : 0.f;
      const double lamn = (double)((float)a.lam[p * PL + e] + mu * (rtn - rho));
      const double xn = (double)((float)Xb[e] - eps * R[(pa * m + pd) * D + (pb * m + pc)]);
      lamw[e] = lamn;
      rtw[e] = (double)rtn;
      Xb[e] = xn;
      if (pm >= 0) {
        const int es = (pb * m + pa) * D + (pd * m + pc);
        lamm[es] = lamn;
        rtm[es] = (double)rtn;
        Xm[j * D + i] = xn;
      }
      rr += (rho - rtn) * (rho - rtn);
      en += h * R[j * D + i];
    }
    for (int idx = tid; idx < m * m; idx += NT) {
      const int x = idx / m, z = idx % m;
      float s1 = 0.f, s2 = 0.f;
      for (int k = 0; k < m; ++k) {
        s1 += R[(x * m + k) * D + (z * m + k)];
        s2 += R[(k * m + x) * D + (k * m + z)];
      }
      a.a1r[p * m * m + idx] = (double)s1;
      a.a2r[p * m * m + idx] = (double)s2;
      if (pm >= 0) {
        a.a1r[pm * m * m + idx] = (double)s2;
        a.a2r[pm * m * m + idx] = (double)s1;
      }
    }
    rr = gsum<NT>(rr, red);
    en = gsum<NT>(en, red);
    if (tid == 0) {
      a.part[p * 2 + 0] = (double)rr;
      a.part[p * 2 + 1] = (double)en;
      if (pm >= 0) {
        a.part[pm * 2 + 0] = (double)rr;
        a.part[pm * 2 + 1] = (double)en;
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_pair_tc(const PairArgs& a, cudaStream_t s) {
  TcProjWs& w = *a.tcw;
  const int grid = (int)(a.Pc < 2 * big_grid() ? a.Pc : 2 * big_grid());
  k_pair256_pre<<<grid, P256_NT, 0, s>>>(a, w.C);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = tc_project256(w, a.Pc, a.warm != 0, a.stats, s)) != cudaSuccess) return e;
  k_pair256_post<<<grid, P256_NT, 0, s>>>(a, w.Wt);
  return cudaGetLastError();
}

template <int D, typename T>
cudaError_t launch_pair_t(const PairArgs& a, cudaStream_t s) {
  constexpr int NT = PairShape<D>::NT, GPC = PairShape<D>::GPC;
  constexpr bool G = GroupShape<D>::GLOBAL;
  const size_t smem = G ? 0 : PairSmem<D, T>::bytes * GPC;
  cudaError_t e = cudaSuccess;
  if (!G) {
    static unsigned long long mask = 0;
    e = smem_once(k_pair<D, T>, smem, mask);
    if (e != cudaSuccess) return e;
  }
  long blocks = (a.Pc + GPC - 1) / GPC;
  const long res = G ? (long)big_grid() : resident_grid((const void*)k_pair<D, T>, NT * GPC, smem);
  if (blocks > res) blocks = res;
  if (blocks < 1) blocks = 1;
  k_pair<D, T><<<(unsigned)blocks, NT * GPC, smem, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- rho_0 and X'_00
// RHO0_CHUNKS CTAs each sum a contiguous range of offsets delta of nu A1[rho_{0,delta}] +
// Lambda1_{0,delta} (m*m entries); the last CTA to finish (a counter in the status block) adds
// the chunk sums in order.  Both orders are fixed, so the result is reproducible bit for bit.
constexpr int RHO0_CHUNKS = 128;

__global__ void __launch_bounds__(256) k_rho0(const SmallArgs a, double* partial) {
  const int mm = a.m * a.m;
  const long per = (a.P + RHO0_CHUNKS - 1) / RHO0_CHUNKS;
  const long lo = blockIdx.x * per, hi = min((long)a.P, lo + per);
  // threads: (entry, sub-range) with 256 / mm sub-ranges per chunk
  const int subs = 256 / mm;
  __shared__ double S[256];
  const int t = threadIdx.x;
  double acc = 0.0;
  if (t < subs * mm) {
    const int idx = t % mm, c = t / mm;
    for (long p = lo + c; p < hi; p += subs) acc += a.nu * a.a1r[p * mm + idx] + a.lam1[p * mm + idx];
  }
  S[t] = acc;
  __syncthreads();
  if (t < mm) {
    double s = 0.0;
    for (int c = 0; c < subs; ++c) s += S[c * mm + t];
    partial[blockIdx.x * mm + t] = s;
  }
  __threadfence();
  __shared__ bool last;
  __syncthreads();
  if (t == 0) last = atomicAdd(&a.st->done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last CTA: rho_0 from the chunk sums (read past L1: other CTAs wrote them), each entry
  // summed by subs threads over interleaved chunks, then in order over the threads
  {
    double acc2 = 0.0;
    if (t < subs * mm) {
      const int idx = t % mm, c0 = t / mm;
      for (int c = c0; c < RHO0_CHUNKS; c += subs) acc2 += __ldcg(partial + c * mm + idx);
    }
    S[t] = acc2;
  }
  __syncthreads();
  __shared__ double rp[256];
  __shared__ double red[8];
  const int m = a.m, D = a.D;
  if (t < mm) {
    double s = 0.0;
    for (int c = 0; c < subs; ++c) s += S[c * mm + t];
    // H'_0 = H_0 - sum_a X_{(a,b),(a,d)}  (Eq. (effHam) with matrix units)
    const int b = t / m, d = t % m;
    double hx = 0.0;
    for (int x = 0; x < m; ++x) hx += a.X[(x * m + b) * D + (x * m + d)];
    const double h0p = a.H0[t] - hx;
    rp[t] = (s - h0p) / (a.nu * (a.N - 1));
  }
  __syncthreads();
  double tr = 0.0;
  for (int k = 0; k < m; ++k) tr += rp[k * m + k];
  const double z = (1.0 - tr) / m;
  __syncthreads();
  if (t < mm) {
    const int b = t / m, d = t % m;
    rp[t] = rp[t] + (b == d ? z : 0.0);
  }
  __syncthreads();
  if (t < mm) a.rho0[t] = rp[t];
  // X'_00 = X_00 - eps G_00[rho_0], G_00 entry (a,b),(c,d) = delta_ac rho0_{d,b}
  for (int e = t; e < D * D; e += 256) {
    const int i = e / D, j = e % D;
    const int pa = i / m, pb = i % m, pc = j / m, pd = j % m;
    if (pa == pc) a.X[e] -= a.eps * rp[pd * m + pb];
  }
  // Tr[H_0 rho_0]
  double h = 0.0;
  if (t < mm) h = a.H0[t] * rp[(t % m) * m + (t / m)];
  h = gsum<256>(h, red);
  if (t == 0) {
    a.st->h0rho0 = h;
    a.st->done = 0u;  // ready for the next sweep
  }
}

// ---------------------------------------------------------------- Lambda1, Lambda2
// One warp per pair offset.  With ties (see k_pair) the canonical member of {delta, -delta}
// also writes the other's multipliers, Lambda1_{-delta} = Lambda2_delta and Lambda2_{-delta} =
// Lambda1_delta, so the two stay exact swap images.
__global__ void k_dual12(const SmallArgs a) {
  const int lane = threadIdx.x & 31;
  const long w = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int mm = a.m * a.m;
  if (w >= a.P) return;
  const long tie = a.ptie ? a.ptie[w] : -1;
  if (tie == -2) return;  // uniform over the warp
  double s = 0.0;
  for (int idx = lane; idx < mm; idx += 32) {
    const double r0 = a.rho0[idx];
    const double d1 = a.a1r[w * mm + idx] - r0;
    const double d2 = a.a2r[w * mm + idx] - r0;
    const double n1 = a.lam1[w * mm + idx] + a.nu * d1;
    const double n2 = a.lam2[w * mm + idx] + a.nu * d2;
    a.lam1[w * mm + idx] = n1;
    a.lam2[w * mm + idx] = n2;
    if (tie >= 0) {
      a.lam1[tie * mm + idx] = n2;
      a.lam2[tie * mm + idx] = n1;
    }
    s += d1 * d1 + d2 * d2;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    a.part2[w] = s;
    if (tie >= 0) a.part2[tie] = s;
  }
}

// ---------------------------------------------------------------- status
// STATUS_CTAS CTAs each sum a contiguous range of offsets (float64 adds are spread over as many
// SMs); the last CTA to finish adds the CTA sums in order and writes the status block.
constexpr int STATUS_CTAS = 32;

__global__ void __launch_bounds__(256) k_status(const SmallArgs a, double* partial) {
  __shared__ double red[8];
  const long per = (a.P + STATUS_CTAS - 1) / STATUS_CTAS;
  const long lo = blockIdx.x * per, hi = min((long)a.P, lo + per);
  double rr = 0.0, en = 0.0, ff = 0.0;
  for (long p = lo + threadIdx.x; p < hi; p += 256) {
    rr += a.part[p * 2 + 0];
    en += a.part[p * 2 + 1];
    ff += a.part2[p];
  }
  rr = gsum<256>(rr, red);
  en = gsum<256>(en, red);
  ff = gsum<256>(ff, red);
  if (threadIdx.x == 0) {
    partial[blockIdx.x * 3 + 0] = rr;
    partial[blockIdx.x * 3 + 1] = en;
    partial[blockIdx.x * 3 + 2] = ff;
  }
  __threadfence();
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&a.st->done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int t = threadIdx.x;
  rr = t < STATUS_CTAS ? __ldcg(partial + t * 3 + 0) : 0.0;
  en = t < STATUS_CTAS ? __ldcg(partial + t * 3 + 1) : 0.0;
  ff = t < STATUS_CTAS ? __ldcg(partial + t * 3 + 2) : 0.0;
  rr = gsum<256>(rr, red);
  en = gsum<256>(en, red);
  ff = gsum<256>(ff, red);
  if (t == 0) {
    DevStatus* st = a.st;
    st->done = 0u;
    const double E = (st->h0rho0 + 0.5 * en) / a.L;
    const double feas = sqrt((rr + ff) / a.P);
    const double dE = isfinite(st->e_prev) ? fabs(E - st->e_prev) : INFINITY;
    st->energy = E;
    st->feas = feas;
    st->d_energy = dE;
    st->residual = fmax(feas, dE);
    st->e_prev = E;
    st->iter += 1;
  }
}

}  // namespace

int resident_grid(const void* kernel, int threads, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  if (sms < 1) sms = 1;
  if (per < 1) per = 1;
  return sms * per;
}

template <int D>
cudaError_t launch_pair_d(const PairArgs& a, int arith, cudaStream_t s) {
  switch (arith) {
    case ARITH_FP64: return launch_pair_t<D, double>(a, s);
    case ARITH_FP32: return launch_pair_t<D, float>(a, s);
    case ARITH_DF64: return launch_pair_t<D, df64>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pair(const PairArgs& a, int arith, cudaStream_t s) {
  if (a.D == 256 && arith == ARITH_FP32 && a.tcw && a.rbuf) return launch_pair_tc(a, s);
  switch (a.D) {
    case 4: return launch_pair_d<4>(a, arith, s);
    case 16: return launch_pair_d<16>(a, arith, s);
    case 64: return launch_pair_d<64>(a, arith, s);
    case 256: return launch_pair_d<256>(a, arith, s);
    default: return cudaErrorInvalidValue;
  }
}

size_t pair_ws_bytes(int D) {
  if (D != 256) return 0;
  size_t a = PairSmem<256, double>::bytes;
  if (PairSmem<256, df64>::bytes > a) a = PairSmem<256, df64>::bytes;
  return a * (size_t)big_grid();
}

int big_grid() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

cudaError_t launch_rho0(const SmallArgs& a, cudaStream_t s) {
  k_rho0<<<RHO0_CHUNKS, 256, 0, s>>>(a, a.rho0_partial);
  return cudaGetLastError();
}

cudaError_t launch_dual12(const SmallArgs& a, cudaStream_t s) {
  const long threads = (long)a.P * 32;
  const unsigned blocks = (unsigned)((threads + 255) / 256);
  k_dual12<<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_status(const SmallArgs& a, cudaStream_t s) {
  k_status<<<STATUS_CTAS, 256, 0, s>>>(a, a.rho0_partial);
  return cudaGetLastError();
}

}  // namespace ve
