// ve_device.cuh -- device building blocks shared by the solver kernels: thread-group
// synchronisation and reductions, and parallel cyclic Jacobi eigensolvers (real symmetric
// and complex Hermitian) working on a matrix staged in shared memory.
//
// A "group" is NT threads that own one matrix: one warp (NT = 32) for n <= 16, the whole CTA
// (NT = 256) for n = 64.  The Jacobi sweep uses the round-robin (circle) ordering: n - 1
// rounds per sweep, n/2 disjoint index pairs per round, so all rotations of a round commute
// and the two-sided update splits into independent 2x2 blocks (one per pair of pairs).  A
// pair's own block becomes diagonal in closed form; of the other blocks only those above the
// diagonal are transformed, their mirror images are stored as (conjugate) transposes, so A
// stays exactly symmetric and a round costs half the flops of the full two-sided update.
// Eigenvalues end on the diagonal of A, eigenvectors in the columns of V.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "ve_df64.cuh"

namespace ve {

template <typename T>
__device__ __forceinline__ T shfl_xor(T v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}

template <int NT>
__device__ __forceinline__ void gsync() {
  if constexpr (NT == 32) {
    __syncwarp();
  } else {
    __syncthreads();
  }
}

// Sum over the group, identical result (same order) in every thread.  `red` is shared scratch
// of NT/32 entries, used only when NT > 32.  The warp sums are combined by warp 0 alone and
// broadcast: float64 issue is scarce, so no other warp repeats that work.
template <int NT, typename T>
__device__ __forceinline__ T gsum(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
  if constexpr (NT == 32) {
    return v;
  } else {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
      T s = lane < NT / 32 ? red[lane] : T(0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += shfl_xor(s, o);
      __syncwarp();
      if (lane == 0) red[0] = s;
    }
    __syncthreads();
    const T s = red[0];
    __syncthreads();
    return s;
  }
}

// min(a, b) that passes a NaN of either argument on (fmin drops it): a reduction that feeds a
// certificate must not turn a non-finite input into a finite minimum.
__device__ __forceinline__ double nan_min(double a, double b) { return (a < b || a != a) ? a : b; }
__device__ __forceinline__ float nan_min(float a, float b) { return (a < b || a != a) ? a : b; }
__device__ __forceinline__ df64 nan_min(df64 a, df64 b) {
  return (a < b || a.hi != a.hi) ? a : b;
}

template <int NT, typename T>
__device__ __forceinline__ T gmin(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nan_min(v, shfl_xor(v, o));
  if constexpr (NT == 32) {
    return v;
  } else {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
      T s = red[lane < NT / 32 ? lane : 0];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s = nan_min(s, shfl_xor(s, o));
      __syncwarp();
      if (lane == 0) red[0] = s;
    }
    __syncthreads();
    const T s = red[0];
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

// Entry t of the upper triangle (i <= j) of an n x n matrix in row-major order, so a group
// can share out the n (n + 1) / 2 entries of a symmetric result without idle lanes.  Row
// r = n - 1 - i from the bottom holds entries r (r + 1) / 2 ... of the reversed count u.
__device__ __forceinline__ void tri_index(int n, int t, int& i, int& j) {
  const int u = n * (n + 1) / 2 - 1 - t;
  int r = (int)((sqrtf(8.f * (float)u + 1.f) - 1.f) * 0.5f);
  if ((r + 1) * (r + 2) / 2 <= u) ++r;
  if (r * (r + 1) / 2 > u) --r;
  i = n - 1 - r;
  j = n - 1 - (u - r * (r + 1) / 2);
}

template <typename T>
struct JacobiTol;
// A sweep loop stops when off(A)^2 <= (n u)^2 ||A||_F^2, u the unit roundoff of the arithmetic:
// the projection's error is at most off(A), and n u ||A|| is the rounding level of the n-term
// sums of the reconstruction V diag V^T itself.  A fixed threshold would sit below the rounding
// floor of the off-diagonal (~sqrt(n) u ||A||) for large n.
template <>
struct JacobiTol<double> {
  static constexpr double u = 1.1102230246251565e-16;  // 2^-53
  static constexpr double big = 1e150;                 // |tau| above which t = 1/(2 tau)
  static constexpr int max_sweeps = 24;
};
template <>
struct JacobiTol<float> {
  static constexpr double u = 5.9604644775390625e-08;  // 2^-24
  static constexpr float big = 1e18f;
  static constexpr int max_sweeps = 14;
};
template <>
struct JacobiTol<df64> {
  static constexpr double u = 3.552713678800501e-15;   // 2^-48
  static constexpr double big = 1e18;
  static constexpr int max_sweeps = 24;
};
template <typename T, int n>
struct JacobiStop {
  static constexpr double rel2 = (n * JacobiTol<T>::u) * (n * JacobiTol<T>::u);
};

// Rotation (c, s) that annihilates the (p,q) entry of [[app, apq], [apq, aqq]] with
// J = [[c, s], [-s, c]] (Golub & Van Loan, symmetric 2x2 Schur decomposition): the tangent t is
// the root of smallest magnitude of b t^2 + d t - b = 0 (d = aqq - app, b = apq), i.e.
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), tau = d / (2 b), and c = 1 / sqrt(1 + t^2), s = t c.
//
// float: evaluated directly.  double: the float64 divide and square root are long multi-
// instruction sequences on a part with a narrow float64 pipe, so (d, b) are scaled by a power of
// two into [1, 2), t is seeded in float32 and refined by two float64 Newton steps on the
// quadratic (each squares the relative error: 1e-7 -> 1e-14 -> 1e-16; the derivative
// 2 b t + d never falls below max(|d|, 2|b|) >= 1 near the root), and c by two Newton steps of
// the reciprocal square root seeded in float32.  c^2 + s^2 = 1 to float64 rounding, which is
// what keeps the accumulated eigenvectors orthogonal.
//
// The tangent is returned too: the rotated diagonal is app - t apq, aqq + t apq (the root
// condition turns c^2 app - 2 c s apq + s^2 aqq into app - t apq).
template <typename T>
__device__ __forceinline__ void sym_schur2(T app, T aqq, T apq, T& c, T& s, T& t);

template <>
__device__ __forceinline__ void sym_schur2<float>(float app, float aqq, float apq, float& c, float& s,
                                                  float& t) {
  if (apq == 0.f) {
    c = 1.f;
    s = 0.f;
    t = 0.f;
    return;
  }
  const float tau = (aqq - app) / (2.f * apq);
  const float at = fabsf(tau);
  t = (at > JacobiTol<float>::big) ? 0.5f / tau : copysignf(1.f, tau) / (at + sqrtf(1.f + tau * tau));
  const float u = fmaf(t, t, 1.f);  // in [1, 2]
  float y = rsqrtf(u);
  y = y * fmaf(-0.5f * u, y * y, 1.5f);  // one Newton step: c^2 + s^2 = 1 to float rounding
  c = y;
  s = t * y;
}

// 2^-e for the float64 exponent e of x (x finite, nonzero): scales x into [1, 2).  The
// reciprocal 2^e is returned in *inv when requested.
__device__ __forceinline__ double pow2_inverse_scale(double x, double* inv = nullptr) {
  int ex = (__double2hiint(x) >> 20) & 0x7ff;
  ex = ex < 1 ? 1 : (ex > 2045 ? 2045 : ex);
  if (inv) *inv = __hiloint2double(ex << 20, 0);
  return __hiloint2double((2046 - ex) << 20, 0);
}

template <>
__device__ __forceinline__ void sym_schur2<double>(double app, double aqq, double apq, double& c,
                                                   double& s, double& t) {
  if (apq == 0.0) {
    c = 1.0;
    s = 0.0;
    t = 0.0;
    return;
  }
  const double d0 = aqq - app;
  const double sc = pow2_inverse_scale(fmax(fabs(d0), fabs(apq)));
  const double d = d0 * sc, b = apq * sc;  // exact; max(|d|, |b|) in [1, 2)
  const float df = (float)d, bf = (float)b;
  float tf = 0.f;
  if (bf != 0.f) {
    const float tau = df / (2.f * bf);
    const float at = fabsf(tau);
    tf = (at > 1e18f) ? 0.5f / tau : copysignf(1.f, tau) / (at + sqrtf(1.f + tau * tau));
  }
  t = (double)tf;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double g = fma(fma(b, t, d), t, -b);
    const double gp = fma(2.0 * b, t, d);
    t = fma(-g, (double)__frcp_rn((float)gp), t);
  }
  const double u = fma(t, t, 1.0);  // in [1, 2]
  const double hu = -0.5 * u;
  double y = (double)rsqrtf((float)u);
  y = y * fma(hu, y * y, 1.5);
  y = y * fma(hu, y * y, 1.5);
  c = y;
  s = t * y;
}

// |b| and the unit phase w = conj(b) / |b| of b = (br, bi), b != 0, without a float64 divide or
// square root (power-of-two scaling, float32 seed, two float64 Newton steps of rsqrt).
template <typename T>
__device__ __forceinline__ void unit_phase(T br, T bi, T& mag, T& wr, T& wi);

template <>
__device__ __forceinline__ void unit_phase<float>(float br, float bi, float& mag, float& wr, float& wi) {
  // scale into [1, 2) by a power of two first: squares of tiny entries would underflow
  int ex = (__float_as_int(fmaxf(fabsf(br), fabsf(bi))) >> 23) & 0xff;
  ex = ex < 1 ? 1 : (ex > 253 ? 253 : ex);
  const float sc = __int_as_float((254 - ex) << 23), isc = __int_as_float(ex << 23);
  const float xr = br * sc, xi = bi * sc;
  const float q = fmaf(xr, xr, xi * xi);
  float y = rsqrtf(q);
  y = y * fmaf(-0.5f * q, y * y, 1.5f);
  wr = xr * y;
  wi = -xi * y;
  mag = (q * y) * isc;
}

template <>
__device__ __forceinline__ void unit_phase<double>(double br, double bi, double& mag, double& wr,
                                                   double& wi) {
  double isc;
  const double sc = pow2_inverse_scale(fmax(fabs(br), fabs(bi)), &isc);
  const double xr = br * sc, xi = bi * sc;
  const double q = fma(xr, xr, xi * xi);  // in [1, 8)
  const double hq = -0.5 * q;
  double y = (double)rsqrtf((float)q);
  y = y * fma(hq, y * y, 1.5);
  y = y * fma(hq, y * y, 1.5);
  wr = xr * y;
  wi = -xi * y;
  mag = (q * y) * isc;  // times a power of two: exact
}

// df64: the float64 recipe above in double-float words -- power-of-two scaling, float32 seed,
// two df64 Newton steps for t and for 1/sqrt(1 + t^2).
__device__ __forceinline__ float pow2_inverse_scale_f(float x, float* inv = nullptr) {
  int ex = (__float_as_int(x) >> 23) & 0xff;
  ex = ex < 1 ? 1 : (ex > 253 ? 253 : ex);
  if (inv) *inv = __int_as_float(ex << 23);
  return __int_as_float((254 - ex) << 23);
}

template <>
__device__ __forceinline__ void sym_schur2<df64>(df64 app, df64 aqq, df64 apq, df64& c, df64& s,
                                                 df64& t) {
  if (apq.hi == 0.f) {
    c = df64(1.f);
    s = df64(0.f);
    t = df64(0.f);
    return;
  }
  const df64 d0 = aqq - app;
  const float sc = pow2_inverse_scale_f(fmaxf(fabsf(d0.hi), fabsf(apq.hi)));
  const df64 d = ldexp_df(d0, sc), b = ldexp_df(apq, sc);
  float tf = 0.f;
  if (b.hi != 0.f) {
    const float tau = d.hi / (2.f * b.hi);
    const float at = fabsf(tau);
    tf = (at > 1e18f) ? 0.5f / tau : copysignf(1.f, tau) / (at + sqrtf(1.f + tau * tau));
  }
  t = df64(tf);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const df64 g = (b * t + d) * t - b;
    const df64 gp = (b + b) * t + d;
    t = t - g * df64(__frcp_rn(gp.hi));
  }
  const df64 u = t * t + df64(1.f);
  const df64 hu = u * df64(-0.5f);
  df64 y(rsqrtf(u.hi));
  y = y * (hu * y * y + df64(1.5f));
  y = y * (hu * y * y + df64(1.5f));
  c = y;
  s = t * y;
}

template <>
__device__ __forceinline__ void unit_phase<df64>(df64 br, df64 bi, df64& mag, df64& wr, df64& wi) {
  float isc;
  const float sc = pow2_inverse_scale_f(fmaxf(fabsf(br.hi), fabsf(bi.hi)), &isc);
  const df64 xr = ldexp_df(br, sc), xi = ldexp_df(bi, sc);
  const df64 q = xr * xr + xi * xi;
  const df64 hq = q * df64(-0.5f);
  df64 y(rsqrtf(q.hi));
  y = y * (hq * y * y + df64(1.5f));
  y = y * (hq * y * y + df64(1.5f));
  wr = xr * y;
  wi = -(xi * y);
  mag = ldexp_df(q * y, isc);
}

// Early stop with a first-order correction (Daleckii-Krein).  With A = Lambda + E (Lambda its
// diagonal) and f(x) = max(x, 0), f(A) = f(Lambda) + L o E + R, L_ij the divided difference
// (f(l_i) - f(l_j)) / (l_i - l_j) (1 between two non-negative diagonal entries, 0 between two
// negative ones, l_+ / (l_+ - l_-) across zero).  While the spectrum of Lambda + t E stays clear
// of zero, f is linear on either side of it and the remainder is of second order, governed by
// the distance d of the diagonal from zero: ||R||_F <= c ||E||_F^2 / d (c well below 1 over
// random 16 x 16 tests).  The sweeps may stop once ||E||_F^2 <= n u ||A||_F d -- as accurate as
// the exact stopping rule -- provided also ||E||_F <= d / 4, so that no eigenvalue can reach
// zero.  `off` and `nrm` are the squared Frobenius norms of E and A; the test is uniform over
// the group.
template <typename T, int n, int LD, int NT>
__device__ bool dk_stop(const T* A, T off, T nrm, T* red, int tid) {
  T d = T(1e30f);
  for (int k = tid; k < n; k += NT) d = nan_min(d, fabs(A[k * LD + k]));
  d = gmin<NT>(d, red);
  return off * off <= T(JacobiStop<T, n>::rel2) * nrm * d * d && T(16) * off <= d * d;
}

// 1 / x for x > 0 without a float64 divide: power-of-two scaling, float32 seed, two Newton steps.
template <typename T>
__device__ __forceinline__ T recip_pos(T x) {
  return T(1) / x;
}
template <>
__device__ __forceinline__ double recip_pos<double>(double x) {
  const double sc = pow2_inverse_scale(x);
  const double xs = x * sc;  // in [1, 2)
  double r = (double)__frcp_rn((float)xs);
  r = r * fma(-xs, r, 2.0);
  r = r * fma(-xs, r, 2.0);
  return r * sc;
}

// The weight L_ij of dk_stop for the diagonal entries l_i, l_j.
template <typename T>
__device__ __forceinline__ T dk_weight(T li, T lj) {
  const bool pi = li >= T(0), pj = lj >= T(0);
  if (pi && pj) return T(1);
  if (!pi && !pj) return T(0);
  const T lp = pi ? li : lj, lm = pi ? lj : li;  // lp >= 0 > lm
  return lp * recip_pos<T>(lp - lm);
}

// M = f(Lambda) + L o E in place of A after an early stop (the eigenvalue estimates go to lam,
// n entries); the projection is then V M V^T (V M V^H).
template <typename T, int n, int LD, int NT>
__device__ void dk_matrix_sym(T* A, T* lam, int tid) {
  for (int k = tid; k < n; k += NT) lam[k] = A[k * LD + k];
  gsync<NT>();
  for (int e = tid; e < n * n; e += NT) {
    const int i = e / n, j = e % n;
    const T li = lam[i];
    A[i * LD + j] = (i == j) ? (li > T(0) ? li : T(0)) : A[i * LD + j] * dk_weight<T>(li, lam[j]);
  }
  gsync<NT>();
}

template <typename T, int n, int LD, int NT>
__device__ void dk_matrix_herm(T* Ar, T* Ai, T* lam, int tid) {
  for (int k = tid; k < n; k += NT) lam[k] = Ar[k * LD + k];
  gsync<NT>();
  for (int e = tid; e < n * n; e += NT) {
    const int i = e / n, j = e % n;
    const T li = lam[i];
    if (i == j) {
      Ar[i * LD + i] = li > T(0) ? li : T(0);
      Ai[i * LD + i] = T(0);
    } else {
      const T w = dk_weight<T>(li, lam[j]);
      Ar[i * LD + j] = Ar[i * LD + j] * w;
      Ai[i * LD + j] = Ai[i * LD + j] * w;
    }
  }
  gsync<NT>();
}

// Real symmetric Jacobi on A (n x n, leading dimension LD) in shared memory.  If VEC, V (same
// layout) receives the eigenvectors.  cs: shared scratch of n entries; red: NT/32 entries.
// Returns the number of sweeps performed.
// With DK the sweeps may also stop early under dk_stop; *dk then tells the caller to
// reconstruct with the first-order correction (dk_matrix) instead of diag(max(l, 0)).
// nrm_min (squared Frobenius norm) raises the scale of the stopping test, for a principal block
// whose accuracy is judged against the whole matrix it belongs to; max_sw caps the sweeps (an
// inexact solve, for the sub-problems of a block method that a later solve completes).
template <typename T, int n, int LD, int NT, bool VEC, bool INIT_V = true, bool DK = false>
__device__ int jacobi_sym(T* A, T* V, T* cs, T* red, int tid, bool* dk = nullptr,
                          T* off_out = nullptr, T nrm_min = T(0),
                          int max_sw = JacobiTol<T>::max_sweeps) {
  static_assert(n == 2 || n % 4 == 0, "the block ordering pairs n / 2 indices");
  constexpr int H = n / 2;
  // blocks (GB) and eigenvector rows (GV) a thread loads before it stores any: a matrix staged
  // in global memory (n > 64) needs several loads in flight per thread; every block and row of a
  // round is disjoint from the others, so the reordering changes no result (GV = 8 measured
  // fastest for real matrices, 2 for complex ones, whose rows hold twice the words)
  constexpr int GB = n > 64 ? 2 : 1, GV = n > 64 ? 8 : 1;
  // a matrix in global memory in float32 / double-float words takes the row-block form of the
  // two-sided update (see below); float64 keeps the symmetric form, its pipe is the bound
  constexpr bool ROWS = n > 64 && !std::is_same<T, double>::value;
  T nrm = T(0);
  for (int e = tid; e < n * n; e += NT) {
    const T a = A[(e / n) * LD + (e % n)];
    nrm += a * a;
  }
  nrm = gsum<NT>(nrm, red);
  if (nrm < nrm_min) nrm = nrm_min;  // a block of a larger matrix: stop at that matrix's scale
  if constexpr (VEC && INIT_V) {
    for (int e = tid; e < n * n; e += NT) V[(e / n) * LD + (e % n)] = (e / n == e % n) ? T(1) : T(0);
  }
  gsync<NT>();
  if constexpr (DK) *dk = false;
  T off_last = T(0);
  int sweep = 0;
  for (; sweep < max_sw; ++sweep) {
    T off = T(0);
    for (int e = tid; e < n * n; e += NT) {
      const int i = e / n, j = e % n;
      if (i != j) {
        const T a = A[i * LD + j];
        off += a * a;
      }
    }
    off = gsum<NT>(off, red);
    off_last = off;
    if (off <= T(JacobiStop<T, n>::rel2) * nrm) break;
    if constexpr (DK) {
      if (dk_stop<T, n, LD, NT>(A, off, nrm, red, tid)) {
        *dk = true;
        break;
      }
    }
    for (int r = 0; r < n - 1; ++r) {
      // the rotation of each pair, and the pair's own 2x2 block made diagonal
      for (int k = tid; k < H; k += NT) {
        int p, q;
        rr_pair(n, r, k, p, q);
        const T app = A[p * LD + p], aqq = A[q * LD + q], apq = A[p * LD + q];
        T c, s, t;
        sym_schur2<T>(app, aqq, apq, c, s, t);
        cs[k] = c;
        cs[H + k] = s;
        A[p * LD + p] = app - t * apq;
        A[q * LD + q] = aqq + t * apq;
        A[p * LD + q] = T(0);
        A[q * LD + p] = T(0);
      }
      gsync<NT>();
      if constexpr (H >= 2 && !ROWS) {
        // the blocks (k1, k2), k1 < k2 -- enumerated as the pairs of a circle ordering of the
        // H pair indices -- and their transposes (k2, k1)
        constexpr int NB = H * (H - 1) / 2;
        for (int b0 = tid; b0 < NB; b0 += GB * NT) {
          int k1[GB], k2[GB], p1[GB], q1[GB], p2[GB], q2[GB];
          T m11[GB], m12[GB], m21[GB], m22[GB];
#pragma unroll
          for (int g = 0; g < GB; ++g) {
            const int b = b0 + g * NT;
            if (b < NB) {
              rr_pair(H, b / (H / 2), b % (H / 2), k1[g], k2[g]);
              rr_pair(n, r, k1[g], p1[g], q1[g]);
              rr_pair(n, r, k2[g], p2[g], q2[g]);
              m11[g] = A[p1[g] * LD + p2[g]];
              m12[g] = A[p1[g] * LD + q2[g]];
              m21[g] = A[q1[g] * LD + p2[g]];
              m22[g] = A[q1[g] * LD + q2[g]];
            }
          }
#pragma unroll
          for (int g = 0; g < GB; ++g) {
            if (b0 + g * NT < NB) {
              const T c1 = cs[k1[g]], s1 = cs[H + k1[g]], c2 = cs[k2[g]], s2 = cs[H + k2[g]];
              const T x11 = c2 * m11[g] - s2 * m12[g], x12 = s2 * m11[g] + c2 * m12[g];
              const T x21 = c2 * m21[g] - s2 * m22[g], x22 = s2 * m21[g] + c2 * m22[g];
              const T y11 = c1 * x11 - s1 * x21, y12 = c1 * x12 - s1 * x22;
              const T y21 = s1 * x11 + c1 * x21, y22 = s1 * x12 + c1 * x22;
              A[p1[g] * LD + p2[g]] = y11;
              A[p2[g] * LD + p1[g]] = y11;
              A[p1[g] * LD + q2[g]] = y12;
              A[q2[g] * LD + p1[g]] = y12;
              A[q1[g] * LD + p2[g]] = y21;
              A[p2[g] * LD + q1[g]] = y21;
              A[q1[g] * LD + q2[g]] = y22;
              A[q2[g] * LD + q1[g]] = y22;
            }
          }
        }
      } else if constexpr (H >= 2) {
        // row-block form: warp w takes the row blocks k1 = w, w + NW, ... and its lanes the
        // column blocks k2, so the four entries of a block lie in two rows the warp reads and
        // writes contiguously; every block k1 != k2 is transformed and none mirrored (twice the
        // arithmetic of the symmetric form for a fraction of its scattered L2 sectors)
        constexpr int NW = NT / 32;
        const int w = tid >> 5, lane = tid & 31;
        for (int k1 = w; k1 < H; k1 += NW) {
          int p1, q1;
          rr_pair(n, r, k1, p1, q1);
          const T c1 = cs[k1], s1 = cs[H + k1];
          for (int k0 = 0; k0 < H; k0 += 32 * GB) {
            int k2[GB], p2[GB], q2[GB];
            T m11[GB], m12[GB], m21[GB], m22[GB];
#pragma unroll
            for (int g = 0; g < GB; ++g) {
              k2[g] = k0 + lane + 32 * g;
              if (k2[g] < H && k2[g] != k1) {
                rr_pair(n, r, k2[g], p2[g], q2[g]);
                m11[g] = A[p1 * LD + p2[g]];
                m12[g] = A[p1 * LD + q2[g]];
                m21[g] = A[q1 * LD + p2[g]];
                m22[g] = A[q1 * LD + q2[g]];
              }
            }
#pragma unroll
            for (int g = 0; g < GB; ++g) {
              if (k2[g] < H && k2[g] != k1) {
                const T c2 = cs[k2[g]], s2 = cs[H + k2[g]];
                const T x11 = c2 * m11[g] - s2 * m12[g], x12 = s2 * m11[g] + c2 * m12[g];
                const T x21 = c2 * m21[g] - s2 * m22[g], x22 = s2 * m21[g] + c2 * m22[g];
                A[p1 * LD + p2[g]] = c1 * x11 - s1 * x21;
                A[p1 * LD + q2[g]] = c1 * x12 - s1 * x22;
                A[q1 * LD + p2[g]] = s1 * x11 + c1 * x21;
                A[q1 * LD + q2[g]] = s1 * x12 + c1 * x22;
              }
            }
          }
        }
      }
      if constexpr (VEC) {
        for (int t0 = tid; t0 < n * H; t0 += GV * NT) {
          int ix[GV], kk[GV], pp[GV], qq[GV];
          T vp[GV], vq[GV];
#pragma unroll
          for (int g = 0; g < GV; ++g) {
            const int t = t0 + g * NT;
            if (t < n * H) {
              ix[g] = t / H;
              kk[g] = t % H;
              rr_pair(n, r, kk[g], pp[g], qq[g]);
              vp[g] = V[ix[g] * LD + pp[g]];
              vq[g] = V[ix[g] * LD + qq[g]];
            }
          }
#pragma unroll
          for (int g = 0; g < GV; ++g) {
            if (t0 + g * NT < n * H) {
              const T c = cs[kk[g]], s = cs[H + kk[g]];
              V[ix[g] * LD + pp[g]] = c * vp[g] - s * vq[g];
              V[ix[g] * LD + qq[g]] = s * vp[g] + c * vq[g];
            }
          }
        }
      }
      gsync<NT>();
    }
  }
  if (off_out) {
    if (sweep == max_sw) {  // the last sweep ran after the last test
      T off = T(0);
      for (int e = tid; e < n * n; e += NT) {
        const int i = e / n, j = e % n;
        if (i != j) off += A[i * LD + j] * A[i * LD + j];
      }
      off_last = gsum<NT>(off, red);
    }
    *off_out = off_last;
  }
  return sweep;
}

// Complex Hermitian Jacobi on (Ar, Ai).  For the pair (p, q) with a_pq = |b| e^{i phi} the
// unitary U = diag(1, w) J, w = e^{-i phi}, J the real rotation of [[a_pp, |b|], [|b|, a_qq]],
// diagonalises the 2x2 block; A <- U^H A U, V <- V U.  cs: shared scratch of 2n entries.
// Returns the number of sweeps performed.
template <typename T, int n, int LD, int NT, bool VEC, bool INIT_V = true, bool DK = false>
__device__ int jacobi_herm(T* Ar, T* Ai, T* Vr, T* Vi, T* cs, T* red, int tid, bool* dk = nullptr,
                           T* off_out = nullptr, T nrm_min = T(0),
                           int max_sw = JacobiTol<T>::max_sweeps) {
  static_assert(n % 4 == 0, "the block ordering pairs n / 2 indices");
  constexpr int H = n / 2;
  constexpr int GB = n > 64 ? 2 : 1, GV = n > 64 ? 2 : 1;  // as in jacobi_sym (measured)
  constexpr bool ROWS = n > 64 && !std::is_same<T, double>::value;
  T nrm = T(0);
  for (int e = tid; e < n * n; e += NT) {
    const int o = (e / n) * LD + (e % n);
    nrm += Ar[o] * Ar[o] + Ai[o] * Ai[o];
  }
  nrm = gsum<NT>(nrm, red);
  if (nrm < nrm_min) nrm = nrm_min;  // a block of a larger matrix: stop at that matrix's scale
  if constexpr (VEC && INIT_V) {
    for (int e = tid; e < n * n; e += NT) {
      const int o = (e / n) * LD + (e % n);
      Vr[o] = (e / n == e % n) ? T(1) : T(0);
      Vi[o] = T(0);
    }
  }
  gsync<NT>();
  if constexpr (DK) *dk = false;
  T off_last = T(0);
  int sweep = 0;
  for (; sweep < max_sw; ++sweep) {
    T off = T(0);
    for (int e = tid; e < n * n; e += NT) {
      const int i = e / n, j = e % n;
      if (i != j) {
        const int o = i * LD + j;
        off += Ar[o] * Ar[o] + Ai[o] * Ai[o];
      }
    }
    off = gsum<NT>(off, red);
    off_last = off;
    if (off <= T(JacobiStop<T, n>::rel2) * nrm) break;
    if constexpr (DK) {
      if (dk_stop<T, n, LD, NT>(Ar, off, nrm, red, tid)) {
        *dk = true;
        break;
      }
    }
    for (int r = 0; r < n - 1; ++r) {
      // the rotation of each pair, and the pair's own 2x2 block made (real) diagonal
      for (int k = tid; k < H; k += NT) {
        int p, q;
        rr_pair(n, r, k, p, q);
        const T app = Ar[p * LD + p], aqq = Ar[q * LD + q];
        const T br = Ar[p * LD + q], bi = Ai[p * LD + q];
        T c, s, t, mag = T(0), wr = T(1), wi = T(0);
        if (br != T(0) || bi != T(0)) unit_phase<T>(br, bi, mag, wr, wi);
        sym_schur2<T>(app, aqq, mag, c, s, t);
        cs[k] = c;
        cs[H + k] = s;
        cs[2 * H + k] = wr;
        cs[3 * H + k] = wi;
        Ar[p * LD + p] = app - t * mag;
        Ar[q * LD + q] = aqq + t * mag;
        Ai[p * LD + p] = T(0);
        Ai[q * LD + q] = T(0);
        Ar[p * LD + q] = T(0);
        Ai[p * LD + q] = T(0);
        Ar[q * LD + p] = T(0);
        Ai[q * LD + p] = T(0);
      }
      gsync<NT>();
      if constexpr (!ROWS) {
      // the blocks (k1, k2), k1 < k2 (pairs of a circle ordering of the H pair indices), and
      // their conjugate transposes (k2, k1)
      constexpr int NB = H * (H - 1) / 2;
      for (int b0 = tid; b0 < NB; b0 += GB * NT) {
        int k1[GB], k2[GB], p1[GB], q1[GB], p2[GB], q2[GB];
        T m11r[GB], m11i[GB], m12r[GB], m12i[GB], m21r[GB], m21i[GB], m22r[GB], m22i[GB];
#pragma unroll
        for (int g = 0; g < GB; ++g) {
          const int b = b0 + g * NT;
          if (b < NB) {
            rr_pair(H, b / (H / 2), b % (H / 2), k1[g], k2[g]);
            rr_pair(n, r, k1[g], p1[g], q1[g]);
            rr_pair(n, r, k2[g], p2[g], q2[g]);
            m11r[g] = Ar[p1[g] * LD + p2[g]];
            m11i[g] = Ai[p1[g] * LD + p2[g]];
            m12r[g] = Ar[p1[g] * LD + q2[g]];
            m12i[g] = Ai[p1[g] * LD + q2[g]];
            m21r[g] = Ar[q1[g] * LD + p2[g]];
            m21i[g] = Ai[q1[g] * LD + p2[g]];
            m22r[g] = Ar[q1[g] * LD + q2[g]];
            m22i[g] = Ai[q1[g] * LD + q2[g]];
          }
        }
#pragma unroll
        for (int g = 0; g < GB; ++g) {
          if (b0 + g * NT >= NB) continue;
          const int a1 = k1[g], a2 = k2[g];
          const T c1 = cs[a1], s1 = cs[H + a1], w1r = cs[2 * H + a1], w1i = cs[3 * H + a1];
          const T c2 = cs[a2], s2 = cs[H + a2], w2r = cs[2 * H + a2], w2i = cs[3 * H + a2];
          // X = M U2: col p = c2 m_p - s2 w2 m_q ; col q = s2 m_p + c2 w2 m_q
          const T sw2r = s2 * w2r, sw2i = s2 * w2i, cw2r = c2 * w2r, cw2i = c2 * w2i;
          const T x11r = c2 * m11r[g] - (sw2r * m12r[g] - sw2i * m12i[g]);
          const T x11i = c2 * m11i[g] - (sw2r * m12i[g] + sw2i * m12r[g]);
          const T x12r = s2 * m11r[g] + (cw2r * m12r[g] - cw2i * m12i[g]);
          const T x12i = s2 * m11i[g] + (cw2r * m12i[g] + cw2i * m12r[g]);
          const T x21r = c2 * m21r[g] - (sw2r * m22r[g] - sw2i * m22i[g]);
          const T x21i = c2 * m21i[g] - (sw2r * m22i[g] + sw2i * m22r[g]);
          const T x22r = s2 * m21r[g] + (cw2r * m22r[g] - cw2i * m22i[g]);
          const T x22i = s2 * m21i[g] + (cw2r * m22i[g] + cw2i * m22r[g]);
          // Y = U1^H X: row p = c1 x_p - s1 conj(w1) x_q ; row q = s1 x_p + c1 conj(w1) x_q
          const T sw1r = s1 * w1r, sw1i = -s1 * w1i, cw1r = c1 * w1r, cw1i = -c1 * w1i;
          const T y11r = c1 * x11r - (sw1r * x21r - sw1i * x21i);
          const T y11i = c1 * x11i - (sw1r * x21i + sw1i * x21r);
          const T y22r = s1 * x12r + (cw1r * x22r - cw1i * x22i);
          const T y22i = s1 * x12i + (cw1r * x22i + cw1i * x22r);
          const T y12r = c1 * x12r - (sw1r * x22r - sw1i * x22i);
          const T y12i = c1 * x12i - (sw1r * x22i + sw1i * x22r);
          const T y21r = s1 * x11r + (cw1r * x21r - cw1i * x21i);
          const T y21i = s1 * x11i + (cw1r * x21i + cw1i * x21r);
          const int P1 = p1[g], Q1 = q1[g], P2 = p2[g], Q2 = q2[g];
          Ar[P1 * LD + P2] = y11r;
          Ai[P1 * LD + P2] = y11i;
          Ar[P2 * LD + P1] = y11r;
          Ai[P2 * LD + P1] = -y11i;
          Ar[Q1 * LD + Q2] = y22r;
          Ai[Q1 * LD + Q2] = y22i;
          Ar[Q2 * LD + Q1] = y22r;
          Ai[Q2 * LD + Q1] = -y22i;
          Ar[P1 * LD + Q2] = y12r;
          Ai[P1 * LD + Q2] = y12i;
          Ar[Q2 * LD + P1] = y12r;
          Ai[Q2 * LD + P1] = -y12i;
          Ar[Q1 * LD + P2] = y21r;
          Ai[Q1 * LD + P2] = y21i;
          Ar[P2 * LD + Q1] = y21r;
          Ai[P2 * LD + Q1] = -y21i;
        }
      }
      } else {
        // row-block form, as in jacobi_sym
        constexpr int NW = NT / 32;
        const int w = tid >> 5, lane = tid & 31;
        for (int k1 = w; k1 < H; k1 += NW) {
          int p1, q1;
          rr_pair(n, r, k1, p1, q1);
          const T c1 = cs[k1], s1 = cs[H + k1], w1r = cs[2 * H + k1], w1i = cs[3 * H + k1];
          const T sw1r = s1 * w1r, sw1i = -s1 * w1i, cw1r = c1 * w1r, cw1i = -c1 * w1i;
          for (int k0 = 0; k0 < H; k0 += 32 * GB) {
            int k2[GB], p2[GB], q2[GB];
            T m11r[GB], m11i[GB], m12r[GB], m12i[GB], m21r[GB], m21i[GB], m22r[GB], m22i[GB];
#pragma unroll
            for (int g = 0; g < GB; ++g) {
              k2[g] = k0 + lane + 32 * g;
              if (k2[g] < H && k2[g] != k1) {
                rr_pair(n, r, k2[g], p2[g], q2[g]);
                m11r[g] = Ar[p1 * LD + p2[g]];
                m11i[g] = Ai[p1 * LD + p2[g]];
                m12r[g] = Ar[p1 * LD + q2[g]];
                m12i[g] = Ai[p1 * LD + q2[g]];
                m21r[g] = Ar[q1 * LD + p2[g]];
                m21i[g] = Ai[q1 * LD + p2[g]];
                m22r[g] = Ar[q1 * LD + q2[g]];
                m22i[g] = Ai[q1 * LD + q2[g]];
              }
            }
#pragma unroll
            for (int g = 0; g < GB; ++g) {
              if (k2[g] >= H || k2[g] == k1) continue;
              const int a2 = k2[g];
              const T c2 = cs[a2], s2 = cs[H + a2], w2r = cs[2 * H + a2], w2i = cs[3 * H + a2];
              // X = M U2, then Y = U1^H X (as in the symmetric form)
              const T sw2r = s2 * w2r, sw2i = s2 * w2i, cw2r = c2 * w2r, cw2i = c2 * w2i;
              const T x11r = c2 * m11r[g] - (sw2r * m12r[g] - sw2i * m12i[g]);
              const T x11i = c2 * m11i[g] - (sw2r * m12i[g] + sw2i * m12r[g]);
              const T x12r = s2 * m11r[g] + (cw2r * m12r[g] - cw2i * m12i[g]);
              const T x12i = s2 * m11i[g] + (cw2r * m12i[g] + cw2i * m12r[g]);
              const T x21r = c2 * m21r[g] - (sw2r * m22r[g] - sw2i * m22i[g]);
              const T x21i = c2 * m21i[g] - (sw2r * m22i[g] + sw2i * m22r[g]);
              const T x22r = s2 * m21r[g] + (cw2r * m22r[g] - cw2i * m22i[g]);
              const T x22i = s2 * m21i[g] + (cw2r * m22i[g] + cw2i * m22r[g]);
              const int P2 = p2[g], Q2 = q2[g];
              Ar[p1 * LD + P2] = c1 * x11r - (sw1r * x21r - sw1i * x21i);
              Ai[p1 * LD + P2] = c1 * x11i - (sw1r * x21i + sw1i * x21r);
              Ar[q1 * LD + Q2] = s1 * x12r + (cw1r * x22r - cw1i * x22i);
              Ai[q1 * LD + Q2] = s1 * x12i + (cw1r * x22i + cw1i * x22r);
              Ar[p1 * LD + Q2] = c1 * x12r - (sw1r * x22r - sw1i * x22i);
              Ai[p1 * LD + Q2] = c1 * x12i - (sw1r * x22i + sw1i * x22r);
              Ar[q1 * LD + P2] = s1 * x11r + (cw1r * x21r - cw1i * x21i);
              Ai[q1 * LD + P2] = s1 * x11i + (cw1r * x21i + cw1i * x21r);
            }
          }
        }
      }
      if constexpr (VEC) {
        for (int t0 = tid; t0 < n * H; t0 += GV * NT) {
          int ix[GV], kk[GV], pp[GV], qq[GV];
          T vpr[GV], vpi[GV], vqr[GV], vqi[GV];
#pragma unroll
          for (int g = 0; g < GV; ++g) {
            const int t = t0 + g * NT;
            if (t < n * H) {
              ix[g] = t / H;
              kk[g] = t % H;
              rr_pair(n, r, kk[g], pp[g], qq[g]);
              vpr[g] = Vr[ix[g] * LD + pp[g]];
              vpi[g] = Vi[ix[g] * LD + pp[g]];
              vqr[g] = Vr[ix[g] * LD + qq[g]];
              vqi[g] = Vi[ix[g] * LD + qq[g]];
            }
          }
#pragma unroll
          for (int g = 0; g < GV; ++g) {
            if (t0 + g * NT >= n * H) continue;
            const int k = kk[g];
            const T c = cs[k], s = cs[H + k], wr = cs[2 * H + k], wi = cs[3 * H + k];
            // v_p' = c v_p - s w v_q ; v_q' = s v_p + c w v_q
            const T wvr = wr * vqr[g] - wi * vqi[g], wvi = wr * vqi[g] + wi * vqr[g];
            const int op = ix[g] * LD + pp[g], oq = ix[g] * LD + qq[g];
            Vr[op] = c * vpr[g] - s * wvr;
            Vi[op] = c * vpi[g] - s * wvi;
            Vr[oq] = s * vpr[g] + c * wvr;
            Vi[oq] = s * vpi[g] + c * wvi;
          }
        }
      }
      gsync<NT>();
    }
  }
  if (off_out) {
    if (sweep == max_sw) {  // the last sweep ran after the last test
      T off = T(0);
      for (int e = tid; e < n * n; e += NT) {
        const int i = e / n, j = e % n;
        if (i != j) {
          const int o = i * LD + j;
          off += Ar[o] * Ar[o] + Ai[o] * Ai[o];
        }
      }
      off_last = gsum<NT>(off, red);
    }
    *off_out = off_last;
  }
  return sweep;
}

// ---------------------------------------------------------------- 16 x 16 warp products
// One warp computes a 16 x 16 product with lane l owning the 2 x 4 output tile at rows
// 2 (l / 4), 2 (l / 4) + 1 and columns 4 (l % 4) .. + 3: eight independent accumulator chains
// and six shared-memory reads per eight multiply-adds (a lane computing single outputs needs two
// reads per multiply-add and has one chain).  TA / TB take the operand transposed (element
// (i, k) of op(A) is A[k][i]); CA / CB conjugate it (complex forms).  The caller stores the
// accumulators after a __syncwarp when the output aliases an operand.
template <typename T, bool TA, bool TB>
__device__ __forceinline__ void rgemm16(const T* A, int lda, const T* B, int ldb, T (&acc)[2][4],
                                        int lane, const T* scale = nullptr) {
  const int r0 = 2 * (lane >> 2), c0 = 4 * (lane & 3);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[a][u] = T(0);
#pragma unroll 4
  for (int k = 0; k < 16; ++k) {
    T a0 = TA ? A[k * lda + r0] : A[r0 * lda + k];
    T a1 = TA ? A[k * lda + r0 + 1] : A[(r0 + 1) * lda + k];
    if (scale) {  // op(A) diag(scale)
      a0 = a0 * scale[k];
      a1 = a1 * scale[k];
    }
    T b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) b[u] = TB ? B[(c0 + u) * ldb + k] : B[k * ldb + c0 + u];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc[0][u] += a0 * b[u];
      acc[1][u] += a1 * b[u];
    }
  }
}

template <typename T, bool TA, bool CA, bool TB, bool CB>
__device__ __forceinline__ void cgemm16(const T* Ar, const T* Ai, int lda, const T* Br, const T* Bi,
                                        int ldb, T (&cr)[2][4], T (&ci)[2][4], int lane,
                                        const T* scale = nullptr) {
  const int r0 = 2 * (lane >> 2), c0 = 4 * (lane & 3);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      cr[a][u] = T(0);
      ci[a][u] = T(0);
    }
#pragma unroll 2
  for (int k = 0; k < 16; ++k) {
    T xr[2], xi[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int o = TA ? k * lda + r0 + a : (r0 + a) * lda + k;
      xr[a] = Ar[o];
      xi[a] = CA ? -Ai[o] : Ai[o];
      if (scale) {  // op(A) diag(scale), scale real
        xr[a] = xr[a] * scale[k];
        xi[a] = xi[a] * scale[k];
      }
    }
    T yr[4], yi[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int o = TB ? (c0 + u) * ldb + k : k * ldb + c0 + u;
      yr[u] = Br[o];
      yi[u] = CB ? -Bi[o] : Bi[o];
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cr[a][u] += xr[a] * yr[u] - xi[a] * yi[u];
        ci[a][u] += xr[a] * yi[u] + xi[a] * yr[u];
      }
  }
}

// Make a 16 x 16 matrix exactly symmetric (Hermitian when Ai is given) from its upper triangle.
template <typename T>
__device__ __forceinline__ void mirror16(T* Ar, T* Ai, int ld, int lane) {
  __syncwarp();
  for (int e = lane; e < 256; e += 32) {
    const int i = e >> 4, j = e & 15;
    if (i > j) {
      Ar[i * ld + j] = Ar[j * ld + i];
      if (Ai) Ai[i * ld + j] = -Ai[j * ld + i];
    } else if (i == j && Ai) {
      Ai[i * ld + i] = T(0);
    }
  }
  __syncwarp();
}

// Store a 2 x 4 lane tile of a 16 x 16 result (row-major, leading dimension ld).
template <typename T>
__device__ __forceinline__ void store16(T* C, int ld, const T (&acc)[2][4], int lane) {
  const int r0 = 2 * (lane >> 2), c0 = 4 * (lane & 3);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int u = 0; u < 4; ++u) C[(r0 + a) * ld + c0 + u] = acc[a][u];
}

// Threads per group, leading dimension and staging of an n x n matrix.  n <= 16: one warp;
// n = 64: one CTA of 256 threads; n = 256: one CTA of 512 threads whose matrices are staged in a
// per-CTA slice of a global workspace (1 MB per float64 matrix and its eigenvectors does not fit
// in shared memory), one CTA per SM so that the slices stay L2-resident where they fit.
template <int n>
struct GroupShape {
  static constexpr int NT = (n <= 16) ? 32 : (n <= 64 ? 256 : 512);
  static constexpr int LD = n + 1;
  static constexpr bool GLOBAL = n > 64;
  // One group per CTA: a batch of a few thousand warp-sized groups then spreads over the SMs
  // to within one group (four-warp CTAs left a quarter of the SMs a whole CTA short).
  static constexpr int GPC = 1;
  // resident CTAs per SM the register budget must allow: at most 128 registers a thread
  static constexpr int MINB = (NT == 32) ? 16 : (NT == 256 ? 2 : 1);
};

// m = sqrt(D) for the pair dimension D = m^2 of a cluster of dimension m.
template <int D>
struct ClusterDim {
  static constexpr int m = (D == 4) ? 2 : (D == 16) ? 4 : (D == 64) ? 8 : 16;
};

}  // namespace ve
