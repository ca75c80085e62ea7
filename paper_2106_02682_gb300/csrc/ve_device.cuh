// ve_device.cuh -- device building blocks shared by the solver kernels: thread-group
// synchronisation and reductions, and parallel cyclic Jacobi eigensolvers (real symmetric
// and complex Hermitian) working on a matrix staged in shared memory.
//
// A "group" is NT threads that own one matrix: one warp (NT = 32) for n <= 16, the whole CTA
// (NT = 256) for n = 64.  The Jacobi sweep uses the round-robin (circle) ordering: n - 1
// rounds per sweep, n/2 disjoint index pairs per round, so all rotations of a round commute
// and the two-sided update splits into independent 2x2 blocks (one per pair of pairs).
// Eigenvalues end on the diagonal of A, eigenvectors in the columns of V.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ve {

template <int NT>
__device__ __forceinline__ void gsync() {
  if constexpr (NT == 32) {
    __syncwarp();
  } else {
    __syncthreads();
  }
}

// Sum over the group, identical result (same order) in every thread.  `red` is shared scratch
// of NT/32 entries, used only when NT > 32.
template <int NT, typename T>
__device__ __forceinline__ T gsum(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if constexpr (NT == 32) {
    return v;
  } else {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T s = T(0);
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) s += red[i];
    __syncthreads();
    return s;
  }
}

template <int NT, typename T>
__device__ __forceinline__ T gmin(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  if constexpr (NT == 32) {
    return v;
  } else {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T s = red[0];
#pragma unroll
    for (int i = 1; i < NT / 32; ++i) s = fmin(s, red[i]);
    __syncthreads();
    return s;
  }
}

// Pair k of round r of the circle ordering of n (even) indices, returned with p < q.
__device__ __forceinline__ void rr_pair(int n, int r, int k, int& p, int& q) {
  int a, b;
  if (k == 0) {
    a = n - 1;
    b = r;
  } else {
    a = (r + k) % (n - 1);
    b = (r - k + n - 1) % (n - 1);
  }
  p = a < b ? a : b;
  q = a < b ? b : a;
}

template <typename T>
struct JacobiTol;
template <>
struct JacobiTol<double> {
  static constexpr double rel2 = 1e-30;  // stop when off(A)^2 <= rel2 ||A||_F^2
  static constexpr double big = 1e150;   // |tau| above which t = 1/(2 tau)
  static constexpr int max_sweeps = 24;
};
template <>
struct JacobiTol<float> {
  static constexpr float rel2 = 1e-13f;
  static constexpr float big = 1e18f;
  static constexpr int max_sweeps = 14;
};

// Rotation (c, s) that annihilates the (p,q) entry of [[app, apq], [apq, aqq]] with
// J = [[c, s], [-s, c]] (Golub & Van Loan, symmetric 2x2 Schur decomposition).
template <typename T>
__device__ __forceinline__ void sym_schur2(T app, T aqq, T apq, T& c, T& s) {
  if (apq == T(0)) {
    c = T(1);
    s = T(0);
    return;
  }
  const T tau = (aqq - app) / (T(2) * apq);
  const T at = fabs(tau);
  T t;
  if (at > JacobiTol<T>::big) {
    t = T(0.5) / tau;
  } else {
    t = copysign(T(1), tau) / (at + sqrt(T(1) + tau * tau));
  }
  c = T(1) / sqrt(T(1) + t * t);
  s = t * c;
}

// Real symmetric Jacobi on A (n x n, leading dimension LD) in shared memory.  If VEC, V (same
// layout) receives the eigenvectors.  cs: shared scratch of n entries; red: NT/32 entries.
template <typename T, int n, int LD, int NT, bool VEC>
__device__ void jacobi_sym(T* A, T* V, T* cs, T* red, int tid) {
  constexpr int H = n / 2;
  T nrm = T(0);
  for (int e = tid; e < n * n; e += NT) {
    const T a = A[(e / n) * LD + (e % n)];
    nrm += a * a;
  }
  nrm = gsum<NT>(nrm, red);
  if constexpr (VEC) {
    for (int e = tid; e < n * n; e += NT) V[(e / n) * LD + (e % n)] = (e / n == e % n) ? T(1) : T(0);
  }
  gsync<NT>();
  for (int sweep = 0; sweep < JacobiTol<T>::max_sweeps; ++sweep) {
    T off = T(0);
    for (int e = tid; e < n * n; e += NT) {
      const int i = e / n, j = e % n;
      if (i != j) {
        const T a = A[i * LD + j];
        off += a * a;
      }
    }
    off = gsum<NT>(off, red);
    if (off <= JacobiTol<T>::rel2 * nrm) break;
    for (int r = 0; r < n - 1; ++r) {
      for (int k = tid; k < H; k += NT) {
        int p, q;
        rr_pair(n, r, k, p, q);
        T c, s;
        sym_schur2<T>(A[p * LD + p], A[q * LD + q], A[p * LD + q], c, s);
        cs[k] = c;
        cs[H + k] = s;
      }
      gsync<NT>();
      for (int b = tid; b < H * H; b += NT) {
        const int k1 = b / H, k2 = b % H;
        int p1, q1, p2, q2;
        rr_pair(n, r, k1, p1, q1);
        rr_pair(n, r, k2, p2, q2);
        const T c1 = cs[k1], s1 = cs[H + k1], c2 = cs[k2], s2 = cs[H + k2];
        const T m11 = A[p1 * LD + p2], m12 = A[p1 * LD + q2];
        const T m21 = A[q1 * LD + p2], m22 = A[q1 * LD + q2];
        const T x11 = c2 * m11 - s2 * m12, x12 = s2 * m11 + c2 * m12;
        const T x21 = c2 * m21 - s2 * m22, x22 = s2 * m21 + c2 * m22;
        A[p1 * LD + p2] = c1 * x11 - s1 * x21;
        A[q1 * LD + q2] = s1 * x12 + c1 * x22;
        if (k1 == k2) {
          A[p1 * LD + q2] = T(0);
          A[q1 * LD + p2] = T(0);
        } else {
          A[p1 * LD + q2] = c1 * x12 - s1 * x22;
          A[q1 * LD + p2] = s1 * x11 + c1 * x21;
        }
      }
      if constexpr (VEC) {
        for (int t = tid; t < n * H; t += NT) {
          const int i = t / H, k = t % H;
          int p, q;
          rr_pair(n, r, k, p, q);
          const T c = cs[k], s = cs[H + k];
          const T vp = V[i * LD + p], vq = V[i * LD + q];
          V[i * LD + p] = c * vp - s * vq;
          V[i * LD + q] = s * vp + c * vq;
        }
      }
      gsync<NT>();
    }
  }
}

// Complex Hermitian Jacobi on (Ar, Ai).  For the pair (p, q) with a_pq = |b| e^{i phi} the
// unitary U = diag(1, w) J, w = e^{-i phi}, J the real rotation of [[a_pp, |b|], [|b|, a_qq]],
// diagonalises the 2x2 block; A <- U^H A U, V <- V U.  cs: shared scratch of 2n entries.
template <typename T, int n, int LD, int NT, bool VEC>
__device__ void jacobi_herm(T* Ar, T* Ai, T* Vr, T* Vi, T* cs, T* red, int tid) {
  constexpr int H = n / 2;
  T nrm = T(0);
  for (int e = tid; e < n * n; e += NT) {
    const int o = (e / n) * LD + (e % n);
    nrm += Ar[o] * Ar[o] + Ai[o] * Ai[o];
  }
  nrm = gsum<NT>(nrm, red);
  if constexpr (VEC) {
    for (int e = tid; e < n * n; e += NT) {
      const int o = (e / n) * LD + (e % n);
      Vr[o] = (e / n == e % n) ? T(1) : T(0);
      Vi[o] = T(0);
    }
  }
  gsync<NT>();
  for (int sweep = 0; sweep < JacobiTol<T>::max_sweeps; ++sweep) {
    T off = T(0);
    for (int e = tid; e < n * n; e += NT) {
      const int i = e / n, j = e % n;
      if (i != j) {
        const int o = i * LD + j;
        off += Ar[o] * Ar[o] + Ai[o] * Ai[o];
      }
    }
    off = gsum<NT>(off, red);
    if (off <= JacobiTol<T>::rel2 * nrm) break;
    for (int r = 0; r < n - 1; ++r) {
      for (int k = tid; k < H; k += NT) {
        int p, q;
        rr_pair(n, r, k, p, q);
        const T br = Ar[p * LD + q], bi = Ai[p * LD + q];
        const T mag = hypot(br, bi);
        T c, s, wr = T(1), wi = T(0);
        sym_schur2<T>(Ar[p * LD + p], Ar[q * LD + q], mag, c, s);
        if (mag > T(0)) {
          wr = br / mag;
          wi = -bi / mag;
        }
        cs[k] = c;
        cs[H + k] = s;
        cs[2 * H + k] = wr;
        cs[3 * H + k] = wi;
      }
      gsync<NT>();
      for (int b = tid; b < H * H; b += NT) {
        const int k1 = b / H, k2 = b % H;
        int p1, q1, p2, q2;
        rr_pair(n, r, k1, p1, q1);
        rr_pair(n, r, k2, p2, q2);
        const T c1 = cs[k1], s1 = cs[H + k1], w1r = cs[2 * H + k1], w1i = cs[3 * H + k1];
        const T c2 = cs[k2], s2 = cs[H + k2], w2r = cs[2 * H + k2], w2i = cs[3 * H + k2];
        const T m11r = Ar[p1 * LD + p2], m11i = Ai[p1 * LD + p2];
        const T m12r = Ar[p1 * LD + q2], m12i = Ai[p1 * LD + q2];
        const T m21r = Ar[q1 * LD + p2], m21i = Ai[q1 * LD + p2];
        const T m22r = Ar[q1 * LD + q2], m22i = Ai[q1 * LD + q2];
        // X = M U2: col p = c2 m_p - s2 w2 m_q ; col q = s2 m_p + c2 w2 m_q
        const T sw2r = s2 * w2r, sw2i = s2 * w2i, cw2r = c2 * w2r, cw2i = c2 * w2i;
        const T x11r = c2 * m11r - (sw2r * m12r - sw2i * m12i);
        const T x11i = c2 * m11i - (sw2r * m12i + sw2i * m12r);
        const T x12r = s2 * m11r + (cw2r * m12r - cw2i * m12i);
        const T x12i = s2 * m11i + (cw2r * m12i + cw2i * m12r);
        const T x21r = c2 * m21r - (sw2r * m22r - sw2i * m22i);
        const T x21i = c2 * m21i - (sw2r * m22i + sw2i * m22r);
        const T x22r = s2 * m21r + (cw2r * m22r - cw2i * m22i);
        const T x22i = s2 * m21i + (cw2r * m22i + cw2i * m22r);
        // Y = U1^H X: row p = c1 x_p - s1 conj(w1) x_q ; row q = s1 x_p + c1 conj(w1) x_q
        const T sw1r = s1 * w1r, sw1i = -s1 * w1i, cw1r = c1 * w1r, cw1i = -c1 * w1i;
        const T y11r = c1 * x11r - (sw1r * x21r - sw1i * x21i);
        const T y11i = c1 * x11i - (sw1r * x21i + sw1i * x21r);
        const T y22r = s1 * x12r + (cw1r * x22r - cw1i * x22i);
        const T y22i = s1 * x12i + (cw1r * x22i + cw1i * x22r);
        if (k1 == k2) {
          Ar[p1 * LD + p2] = y11r;
          Ai[p1 * LD + p2] = T(0);
          Ar[q1 * LD + q2] = y22r;
          Ai[q1 * LD + q2] = T(0);
          Ar[p1 * LD + q2] = T(0);
          Ai[p1 * LD + q2] = T(0);
          Ar[q1 * LD + p2] = T(0);
          Ai[q1 * LD + p2] = T(0);
        } else {
          const T y12r = c1 * x12r - (sw1r * x22r - sw1i * x22i);
          const T y12i = c1 * x12i - (sw1r * x22i + sw1i * x22r);
          const T y21r = s1 * x11r + (cw1r * x21r - cw1i * x21i);
          const T y21i = s1 * x11i + (cw1r * x21i + cw1i * x21r);
          Ar[p1 * LD + p2] = y11r;
          Ai[p1 * LD + p2] = y11i;
          Ar[q1 * LD + q2] = y22r;
          Ai[q1 * LD + q2] = y22i;
          Ar[p1 * LD + q2] = y12r;
          Ai[p1 * LD + q2] = y12i;
          Ar[q1 * LD + p2] = y21r;
          Ai[q1 * LD + p2] = y21i;
        }
      }
      if constexpr (VEC) {
        for (int t = tid; t < n * H; t += NT) {
          const int i = t / H, k = t % H;
          int p, q;
          rr_pair(n, r, k, p, q);
          const T c = cs[k], s = cs[H + k], wr = cs[2 * H + k], wi = cs[3 * H + k];
          const T vpr = Vr[i * LD + p], vpi = Vi[i * LD + p];
          const T vqr = Vr[i * LD + q], vqi = Vi[i * LD + q];
          // v_p' = c v_p - s w v_q ; v_q' = s v_p + c w v_q
          const T wvr = wr * vqr - wi * vqi, wvi = wr * vqi + wi * vqr;
          Vr[i * LD + p] = c * vpr - s * wvr;
          Vi[i * LD + p] = c * vpi - s * wvi;
          Vr[i * LD + q] = s * vpr + c * wvr;
          Vi[i * LD + q] = s * vpi + c * wvi;
        }
      }
      gsync<NT>();
    }
  }
}

// Threads per group and leading dimension used for an n x n matrix.
template <int n>
struct GroupShape {
  static constexpr int NT = (n <= 16) ? 32 : 256;
  static constexpr int LD = n + 1;
};

}  // namespace ve
