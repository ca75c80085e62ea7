// ve_fft.cu -- the global X step of Algorithm 6 (Khoo & Lindsey, arXiv:2106.02682, Sec. 3.3):
// block DFT of X's first block row over the cluster offsets, per-wavevector PSD projection of
// the Hermitian blocks, inverse DFT.
//
// Layout.  The first block row is N slots (cluster offsets, row-major) of D*D reals.  Because
// every entry sequence over delta is real, two entries share one complex sequence:
// z_t[e] = X_t[e] + i X_t[e + E], E = D*D/2.  After the forward transform the true blocks are
// recovered per wavevector from z[k] and conj(z[-k]); the inverse transform of
// Y_k[e] + i Y_k[e + E] returns both real entry sequences at once.
//
// Transform.  Each pass is a length-n DFT (n <= 64) along one axis of the slot array viewed as
// [A][n][B], done in shared memory by one CTA per (line, chunk of entries): radix-2 in place
// when n is a power of two, the direct sum otherwise.  A 1-D lattice with N > 64 clusters uses
// the four-step split N = N1 * N2 with a twiddle between the two passes; the spectrum is then
// stored digit-reversed (slot c*N2 + e holds k = c + N1*e), which the projection handles through
// the partner map k -> -k.  A 2-D lattice takes one pass per axis.  Forward sign e^{-i}, no
// scaling; the projection kernel applies 1/N.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <mutex>
#include <string>

#include "../../include/ve.h"
#include "ve_device.cuh"
#include "ve_internal.h"

namespace ve {

namespace {

template <typename R>
struct C2;
template <>
struct C2<double> {
  using type = double2;
  static __device__ __forceinline__ double2 make(double x, double y) { return make_double2(x, y); }
};
template <>
struct C2<float> {
  using type = float2;
  static __device__ __forceinline__ float2 make(float x, float y) { return make_float2(x, y); }
};

// Spectrum word of each per-matrix arithmetic: float32 work reads a float32 spectrum; float64
// and double-float work read the float64 one.
template <typename T>
struct SpecOf {
  using R = T;
};
template <>
struct SpecOf<df64> {
  using R = double;
};

template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

__device__ __forceinline__ int bitrev(int j, int logn) { return (int)(__brev((unsigned)j) >> (32 - logn)); }

// tf32 part of a float32 value (the significand bits a tf32 tensor-core operand keeps).
__device__ __forceinline__ float tc_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

constexpr int FFT_EC = 32;        // largest number of entries per CTA
constexpr int FFT_THREADS = 256;

// One pass in precision R (double or float): the spectrum buffers hold C2<R>::type; the real
// first block row (xin / xout) is always float64.  Twiddles are float64 tables, rounded to R.
template <typename R>
__global__ void __launch_bounds__(FFT_THREADS)
    k_fft_pass(const double* __restrict__ xin, const typename C2<R>::type* __restrict__ cin,
               typename C2<R>::type* cout, double* xout, const FftPass ps, const int dir,
               const int E, const double2* __restrict__ tw, const int EC) {
  using V = typename C2<R>::type;
  extern __shared__ __align__(16) unsigned char sraw[];
  V* sbuf = reinterpret_cast<V*>(sraw);
  const int line = blockIdx.x;
  const int la = line / ps.B, lb = line % ps.B;
  const int e0 = blockIdx.y * EC;
  const int ec = min(EC, E - e0);
  const int n = ps.n;
  const bool pow2 = (n & (n - 1)) == 0;
  const int logn = 31 - __clz(n);
  for (int idx = threadIdx.x; idx < n * EC; idx += FFT_THREADS) {
    const int j = idx / EC, e = idx % EC;
    if (e >= ec) continue;
    const long slot = ((long)la * n + j) * ps.B + lb;
    V v;
    if (xin) {
      v.x = (R)xin[slot * 2 * E + e0 + e];
      v.y = (R)xin[slot * 2 * E + E + e0 + e];
    } else {
      v = cin[slot * E + e0 + e];
    }
    const int jj = (pow2 && n > 1) ? bitrev(j, logn) : j;
    sbuf[jj * EC + e] = v;
  }
  __syncthreads();
  const double2* Wn = tw + ps.w_off;  // exp(-2 pi i t / n)
  const V* res = sbuf;
  const R sg = dir > 0 ? R(-1) : R(1);
  if (pow2) {
    for (int half = 1; half < n; half <<= 1) {
      const int stride = n / (2 * half);
      for (int idx = threadIdx.x; idx < (n / 2) * EC; idx += FFT_THREADS) {
        const int e = idx % EC, bf = idx / EC;
        const int grp = bf / half, j = bf % half;
        const int i0 = grp * 2 * half + j, i1 = i0 + half;
        const double2 wd = Wn[j * stride];
        const V w = C2<R>::make((R)wd.x, sg * (R)wd.y);
        const V u = sbuf[i0 * EC + e];
        const V t = cmul(w, sbuf[i1 * EC + e]);
        sbuf[i0 * EC + e] = C2<R>::make(u.x + t.x, u.y + t.y);
        sbuf[i1 * EC + e] = C2<R>::make(u.x - t.x, u.y - t.y);
      }
      __syncthreads();
    }
  } else {
    V* obuf = sbuf + n * EC;
    for (int idx = threadIdx.x; idx < n * EC; idx += FFT_THREADS) {
      const int k = idx / EC, e = idx % EC;
      V acc = C2<R>::make(R(0), R(0));
      for (int j = 0; j < n; ++j) {
        const double2 wd = Wn[(j * k) % n];
        const V t = cmul(C2<R>::make((R)wd.x, sg * (R)wd.y), sbuf[j * EC + e]);
        acc.x += t.x;
        acc.y += t.y;
      }
      obuf[idx] = acc;
    }
    __syncthreads();
    res = obuf;
  }
  for (int idx = threadIdx.x; idx < n * EC; idx += FFT_THREADS) {
    const int k = idx / EC, e = idx % EC;
    if (e >= ec) continue;
    V v = res[idx];
    if (ps.tw_mode) {
      const int other = (ps.tw_mode == 1) ? lb : la;
      const double2 wd = tw[ps.tw_off + (int)(((long)k * other) % ps.twN)];
      v = cmul(v, C2<R>::make((R)wd.x, sg * (R)wd.y));
    }
    const long slot = ((long)la * n + k) * ps.B + lb;
    if (xout) {
      xout[slot * 2 * E + e0 + e] = (double)v.x;
      xout[slot * 2 * E + E + e0 + e] = (double)v.y;
    } else {
      cout[slot * E + e0 + e] = v;
    }
  }
}

__global__ void k_fft_tables(double2* tw, const FftPlan p) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < p.ntw; t += gridDim.x * blockDim.x) {
    int tab = 0;
    while (tab + 1 < p.ntab && t >= p.tab_off[tab + 1]) ++tab;
    const int n = p.tab_n[tab], j = t - p.tab_off[tab];
    double s, c;
    sincospi(2.0 * (double)j / (double)n, &s, &c);
    tw[t] = make_double2(c, -s);
  }
}

// Slot of -k for the spectrum slot s (see the layout notes at the top of the file).
__device__ __forceinline__ int partner_slot(const FftPlan& p, int s) {
  if (p.dim == 2) {
    const int k0 = s / p.M1, k1 = s % p.M1;
    return ((p.M0 - k0) % p.M0) * p.M1 + (p.M1 - k1) % p.M1;
  }
  if (p.npass == 1) return (p.N - s) % p.N;
  const int c = s / p.N2, e = s % p.N2;
  const int k = c + p.N1 * e;
  const int kk = (p.N - k) % p.N;
  return (kk % p.N1) * p.N2 + kk / p.N1;
}

template <int D, typename T>
struct XSmem {
  static constexpr int LD = GroupShape<D>::LD;
  static constexpr size_t MAT = ((sizeof(T) * D * LD + 15) / 16) * 16;
  static constexpr size_t bytes = 6 * MAT + ((sizeof(T) * 2 * D + 15) / 16) * 16 +
                                  ((sizeof(T) * D + 15) / 16) * 16 + 32 * sizeof(T);
};

// Unpack block C_k (unnormalised) of slot s from the packed spectrum into (Ar, Ai), Hermitised.
template <int D, int NT, int LD, typename T, typename V>
__device__ void unpack_block(const V* spec, int s, int s2, int E, T* Ar, T* Ai, int tid) {
  using R = decltype(V{}.x);
  for (int f = tid; f < D * D; f += NT) {
    const int e = f < E ? f : f - E;
    const V z = spec[(long)s * E + e];
    const V zz = spec[(long)s2 * E + e];  // conj taken below
    R cr, ci;
    if (f < E) {  // (z + conj(zz)) / 2
      cr = R(0.5) * (z.x + zz.x);
      ci = R(0.5) * (z.y - zz.y);
    } else {      // (z - conj(zz)) / (2i)
      const R dr = z.x - zz.x, di = z.y + zz.y;
      cr = R(0.5) * di;
      ci = R(-0.5) * dr;
    }
    Ar[(f / D) * LD + (f % D)] = (T)cr;
    Ai[(f / D) * LD + (f % D)] = (T)ci;
  }
  gsync<NT>();
  for (int f = tid; f < D * D; f += NT) {
    const int i = f / D, j = f % D;
    if (i < j) {
      const T r = T(0.5) * (Ar[i * LD + j] + Ar[j * LD + i]);
      const T im = T(0.5) * (Ai[i * LD + j] - Ai[j * LD + i]);
      Ar[i * LD + j] = r;
      Ai[i * LD + j] = im;
      Ar[j * LD + i] = r;
      Ai[j * LD + i] = -im;
    } else if (i == j) {
      Ai[i * LD + i] = T(0);
    }
  }
  gsync<NT>();
}

template <int D, typename T>
__global__ void __launch_bounds__(GroupShape<D>::NT * GroupShape<D>::GPC, GroupShape<D>::MINB)
    k_xproj(typename C2<typename SpecOf<T>::R>::type* spec, const int* __restrict__ canon, const int ncanon,
            const FftPlan p, const double invN, T* vstore, const int warm,
            unsigned long long* stats, unsigned char* gws, const long long* iter) {
  constexpr int NT = GroupShape<D>::NT, LD = GroupShape<D>::LD;
  constexpr int GPC = GroupShape<D>::GPC;
  // register-tiled warp products (cgemm16) in float32 only: they compute whole 16 x 16 results
  // where the loops below compute triangles, and float64 / double-float issue is the bound there
  constexpr bool TILE16 = D == 16 && NT == 32 && std::is_same<T, float>::value;
  using S = XSmem<D, T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = threadIdx.x / NT, tid = threadIdx.x % NT;
  unsigned char* base = GroupShape<D>::GLOBAL ? gws + (size_t)blockIdx.x * S::bytes
                                              : smem_raw + (size_t)g * S::bytes;
  T* Ar = reinterpret_cast<T*>(base);
  T* Ai = reinterpret_cast<T*>(base + S::MAT);
  T* Vr = reinterpret_cast<T*>(base + 2 * S::MAT);
  T* Vi = reinterpret_cast<T*>(base + 3 * S::MAT);
  T* Wr = reinterpret_cast<T*>(base + 4 * S::MAT);
  T* Wi = reinterpret_cast<T*>(base + 5 * S::MAT);
  T* cs = reinterpret_cast<T*>(base + 6 * S::MAT);
  T* W = cs + 2 * D;
  T* red = W + D;
  const int E = p.E;
  for (int j = blockIdx.x * GPC + g; j < ncanon; j += gridDim.x * GPC) {
    const int s = canon[j];
    const int s2 = partner_slot(p, s);
    T* vr = vstore ? vstore + (long)s * 2 * D * D : nullptr;
    T* vi = vr ? vr + D * D : nullptr;
    int nsw = 0;
    bool dk = false;  // the eigensolve stopped early: reconstruct with the first-order correction
    if (warm && vr) {
      for (int e = tid; e < D * D; e += NT) {
        Vr[(e / D) * LD + (e % D)] = vr[e];
        Vi[(e / D) * LD + (e % D)] = vi[e];
      }
      gsync<NT>();
      if (ns_due<T>(iter) && TILE16) {
        // as below, register-tiled warp products
        T gr[2][4], gi[2][4];
        cgemm16<T, true, true, false, false>(Vr, Vi, LD, Vr, Vi, LD, gr, gi, tid);
        const int r0 = 2 * (tid >> 2), c0 = 4 * (tid & 3);
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            gr[x][u] = ((r0 + x == c0 + u) ? T(1.5) : T(0)) - T(0.5) * gr[x][u];
            gi[x][u] = -T(0.5) * gi[x][u];
          }
        store16(Wr, LD, gr, tid);
        store16(Wi, LD, gi, tid);
        __syncwarp();
        cgemm16<T, false, false, false, false>(Vr, Vi, LD, Wr, Wi, LD, gr, gi, tid);
        __syncwarp();
        store16(Vr, LD, gr, tid);
        store16(Vi, LD, gi, tid);
        __syncwarp();
      } else if (ns_due<T>(iter)) {
        // one Newton-Schulz step V <- V (3 I - V^H V) / 2 against the rounding drift of the
        // stored eigenvectors (Wr/Wi hold the Gram correction, Ar/Ai the new V)
        for (int e = tid; e < D * D; e += NT) {
          const int i = e / D, jj = e % D;
          T gr = T(0), gi = T(0);
          for (int k = 0; k < D; ++k) {
            const T ar = Vr[k * LD + i], ai = -Vi[k * LD + i];
            const T br = Vr[k * LD + jj], bi = Vi[k * LD + jj];
            gr += ar * br - ai * bi;
            gi += ar * bi + ai * br;
          }
          Wr[i * LD + jj] = ((i == jj) ? T(1.5) : T(0)) - T(0.5) * gr;
          Wi[i * LD + jj] = -T(0.5) * gi;
        }
        gsync<NT>();
        for (int e = tid; e < D * D; e += NT) {
          const int i = e / D, jj = e % D;
          T xr = T(0), xi = T(0);
          for (int k = 0; k < D; ++k) {
            const T ar = Vr[i * LD + k], ai = Vi[i * LD + k];
            const T br = Wr[k * LD + jj], bi = Wi[k * LD + jj];
            xr += ar * br - ai * bi;
            xi += ar * bi + ai * br;
          }
          Ar[i * LD + jj] = xr;
          Ai[i * LD + jj] = xi;
        }
        gsync<NT>();
        for (int e = tid; e < D * D; e += NT) {
          Vr[(e / D) * LD + (e % D)] = Ar[(e / D) * LD + (e % D)];
          Vi[(e / D) * LD + (e % D)] = Ai[(e / D) * LD + (e % D)];
        }
        gsync<NT>();
      }
    }
    unpack_block<D, NT, LD, T>(spec, s, s2, E, Ar, Ai, tid);
    if (warm && vr && TILE16) {
      // A <- V^H C V with register-tiled warp products (upper triangle mirrored)
      T xr[2][4], xi[2][4];
      cgemm16<T, false, false, false, false>(Ar, Ai, LD, Vr, Vi, LD, xr, xi, tid);
      store16(Wr, LD, xr, tid);
      store16(Wi, LD, xi, tid);
      __syncwarp();
      cgemm16<T, true, true, false, false>(Vr, Vi, LD, Wr, Wi, LD, xr, xi, tid);
      store16(Ar, LD, xr, tid);
      store16(Ai, LD, xi, tid);
      mirror16<T>(Ar, Ai, LD, tid);
      nsw = jacobi_herm<T, D, LD, NT, true, false, true>(Ar, Ai, Vr, Vi, cs, red, tid, &dk);
    } else if (warm && vr) {
      // start from the previous eigenvectors: A <- V^H C V
      for (int e = tid; e < D * D; e += NT) {  // W = C V
        const int i = e / D, jj = e % D;
        T xr = T(0), xi = T(0);
        for (int k = 0; k < D; ++k) {
          const T ar = Ar[i * LD + k], ai = Ai[i * LD + k];
          const T br = Vr[k * LD + jj], bi = Vi[k * LD + jj];
          xr += ar * br - ai * bi;
          xi += ar * bi + ai * br;
        }
        Wr[i * LD + jj] = xr;
        Wi[i * LD + jj] = xi;
      }
      gsync<NT>();
      for (int t = tid; t < D * (D + 1) / 2; t += NT) {  // A = V^H W, Hermitian
        int i, jj;
        tri_index(D, t, i, jj);
        T xr = T(0), xi = T(0);
        for (int k = 0; k < D; ++k) {
          const T ar = Vr[k * LD + i], ai = -Vi[k * LD + i];
          const T br = Wr[k * LD + jj], bi = Wi[k * LD + jj];
          xr += ar * br - ai * bi;
          xi += ar * bi + ai * br;
        }
        Ar[i * LD + jj] = xr;
        Ar[jj * LD + i] = xr;
        Ai[i * LD + jj] = (i == jj) ? T(0) : xi;
        Ai[jj * LD + i] = (i == jj) ? T(0) : -xi;
      }
      gsync<NT>();
      nsw = jacobi_herm<T, D, LD, NT, true, false, true>(Ar, Ai, Vr, Vi, cs, red, tid, &dk);
    } else {
      nsw = jacobi_herm<T, D, LD, NT, true, true, true>(Ar, Ai, Vr, Vi, cs, red, tid, &dk);
    }
    if (stats && tid == 0) {
      atomicAdd(stats, (unsigned long long)nsw);
      atomicAdd(stats + 1, 1ull);
      if (dk) atomicAdd(stats + 2, 1ull);
    }
    if (vr) {
      for (int e = tid; e < D * D; e += NT) {
        vr[e] = Vr[(e / D) * LD + (e % D)];
        vi[e] = Vi[(e / D) * LD + (e % D)];
      }
    }
    if (TILE16) {
      // Y = V M V^H (M = f(Lambda) + L o E after a first-order stop, else diag(max(l, 0)))
      // with register-tiled warp products; the upper triangle is mirrored
      T yr[2][4], yi[2][4];
      if (dk) {
        dk_matrix_herm<T, D, LD, NT>(Ar, Ai, cs, tid);
        cgemm16<T, false, false, false, false>(Vr, Vi, LD, Ar, Ai, LD, yr, yi, tid);
        store16(Wr, LD, yr, tid);
        store16(Wi, LD, yi, tid);
        __syncwarp();
        cgemm16<T, false, false, true, true>(Wr, Wi, LD, Vr, Vi, LD, yr, yi, tid);
      } else {
        for (int k = tid; k < D; k += NT) {
          const T w = Ar[k * LD + k];
          W[k] = w > T(0) ? w : T(0);
        }
        __syncwarp();
        cgemm16<T, false, false, true, true>(Vr, Vi, LD, Vr, Vi, LD, yr, yi, tid, W);
      }
      __syncwarp();
      store16(Ar, LD, yr, tid);
      store16(Ai, LD, yi, tid);
      mirror16<T>(Ar, Ai, LD, tid);
    } else if (dk) {
      // Y = V M V^H with M = f(Lambda) + L o E (dk_stop): W = V M, then W V^H
      dk_matrix_herm<T, D, LD, NT>(Ar, Ai, cs, tid);
      for (int e = tid; e < D * D; e += NT) {
        const int i = e / D, jj = e % D;
        T xr = T(0), xi = T(0);
        for (int k = 0; k < D; ++k) {
          const T vr_ = Vr[i * LD + k], vi_ = Vi[i * LD + k];
          const T mr = Ar[k * LD + jj], mi = Ai[k * LD + jj];
          xr += vr_ * mr - vi_ * mi;
          xi += vr_ * mi + vi_ * mr;
        }
        Wr[i * LD + jj] = xr;
        Wi[i * LD + jj] = xi;
      }
      gsync<NT>();
      for (int t = tid; t < D * (D + 1) / 2; t += NT) {
        int i, jj;
        tri_index(D, t, i, jj);
        T yr = T(0), yi = T(0);
        for (int k = 0; k < D; ++k) {  // sum_k W_ik conj(V_jk)
          const T wr_ = Wr[i * LD + k], wi_ = Wi[i * LD + k];
          const T ajr = Vr[jj * LD + k], aji = Vi[jj * LD + k];
          yr += wr_ * ajr + wi_ * aji;
          yi += wi_ * ajr - wr_ * aji;
        }
        Ar[i * LD + jj] = yr;
        Ai[i * LD + jj] = (i == jj) ? T(0) : yi;
        Ar[jj * LD + i] = yr;
        Ai[jj * LD + i] = (i == jj) ? T(0) : -yi;
      }
    } else {
      for (int k = tid; k < D; k += NT) {
        const T w = Ar[k * LD + k];
        W[k] = w > T(0) ? w : T(0);
      }
      gsync<NT>();
      // Y = V diag(max(w,0)) V^H, written back into (Ar, Ai)
      for (int t = tid; t < D * (D + 1) / 2; t += NT) {
        int i, jj;
        tri_index(D, t, i, jj);
        T yr = T(0), yi = T(0);
        for (int k = 0; k < D; ++k) {
          const T w = W[k];
          const T air = Vr[i * LD + k], aii = Vi[i * LD + k];
          const T ajr = Vr[jj * LD + k], aji = Vi[jj * LD + k];
          yr += w * (air * ajr + aii * aji);
          yi += w * (aii * ajr - air * aji);
        }
        Ar[i * LD + jj] = yr;
        Ai[i * LD + jj] = yi;
        Ar[jj * LD + i] = yr;
        Ai[jj * LD + i] = -yi;
      }
    }
    gsync<NT>();
    // pack Y_k (and Y_{-k} = conj Y_k) back, scaled by 1/N
    using R = typename SpecOf<T>::R;
    const T sc = (T)invN;
    for (int e = tid; e < E; e += NT) {
      const int f1 = e, f2 = e + E;
      const T y1r = Ar[(f1 / D) * LD + f1 % D] * sc;
      const T y1i = Ai[(f1 / D) * LD + f1 % D] * sc;
      const T y2r = Ar[(f2 / D) * LD + f2 % D] * sc;
      const T y2i = Ai[(f2 / D) * LD + f2 % D] * sc;
      spec[(long)s * E + e] = C2<R>::make((R)(y1r - y2i), (R)(y1i + y2r));
      if (s2 != s) spec[(long)s2 * E + e] = C2<R>::make((R)(y1r + y2i), (R)(y2r - y1i));
    }
    gsync<NT>();
  }
}

// One CTA: canonical slots in increasing order (block-wide scan over chunks of 256 slots).
__global__ void __launch_bounds__(256) k_canon_list(const FftPlan p, int* canon) {
  __shared__ int scan[256];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < p.N; c0 += 256) {
    const int s = c0 + threadIdx.x;
    const int flag = (s < p.N && s <= partner_slot(p, s)) ? 1 : 0;
    scan[threadIdx.x] = flag;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
      const int v = threadIdx.x >= o ? scan[threadIdx.x - o] : 0;
      __syncthreads();
      scan[threadIdx.x] += v;
      __syncthreads();
    }
    if (flag) canon[base + scan[threadIdx.x] - 1] = s;
    __syncthreads();
    if (threadIdx.x == 255) base += scan[255];
    __syncthreads();
  }
}

template <int D>
__global__ void __launch_bounds__(GroupShape<D>::NT * GroupShape<D>::GPC, GroupShape<D>::MINB)
    k_xeig(const double2* spec, const int* __restrict__ canon, const int ncanon, const FftPlan p,
           double* lmin, unsigned char* gws) {
  constexpr int NT = GroupShape<D>::NT, LD = GroupShape<D>::LD;
  constexpr int GPC = GroupShape<D>::GPC;
  using S = XSmem<D, double>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = threadIdx.x / NT, tid = threadIdx.x % NT;
  unsigned char* base = GroupShape<D>::GLOBAL ? gws + (size_t)blockIdx.x * S::bytes
                                              : smem_raw + (size_t)g * S::bytes;
  double* Ar = reinterpret_cast<double*>(base);
  double* Ai = reinterpret_cast<double*>(base + S::MAT);
  double* cs = reinterpret_cast<double*>(base + 4 * S::MAT);
  double* red = cs + 3 * D;
  for (int j = blockIdx.x * GPC + g; j < ncanon; j += gridDim.x * GPC) {
    const int s = canon[j];
    const int s2 = partner_slot(p, s);
    unpack_block<D, NT, LD, double>(spec, s, s2, p.E, Ar, Ai, tid);
    double off = 0.0;
    jacobi_herm<double, D, LD, NT, false>(Ar, Ai, nullptr, nullptr, cs, red, tid, nullptr, &off);
    double w = INFINITY;
    for (int k = tid; k < D; k += NT) w = nan_min(w, Ar[k * LD + k]);
    w = gmin<NT>(w, red);
    // Weyl: lmin >= min diag - ||E||_F for the rotated diag + E; a NaN passes through
    if (tid == 0) lmin[j] = w - sqrt(off);
    gsync<NT>();
  }
}


template <int D, typename T>
cudaError_t launch_xproj_t(const FftPlan& p, double2* spec, const int* canon, void* vstore,
                           int warm, cudaStream_t s, unsigned long long* stats,
                           unsigned char* gws, const long long* iter) {
  constexpr int NT = GroupShape<D>::NT, GPC = GroupShape<D>::GPC;
  constexpr bool G = GroupShape<D>::GLOBAL;
  const size_t smem = G ? 0 : XSmem<D, T>::bytes * GPC;
  if (!G) {
    static unsigned long long mask = 0;
    cudaError_t e = smem_once(k_xproj<D, T>, smem, mask);
    if (e != cudaSuccess) return e;
  } else if (!gws) {
    return cudaErrorInvalidValue;
  }
  const int nc = fft_ncanon(p);
  long blocks = (nc + GPC - 1) / GPC;
  const long res = G ? (long)big_grid() : resident_grid((const void*)k_xproj<D, T>, NT * GPC, smem);
  if (blocks > res) blocks = res;
  k_xproj<D, T><<<(unsigned)blocks, NT * GPC, smem, s>>>(
      reinterpret_cast<typename C2<typename SpecOf<T>::R>::type*>(spec), canon, nc, p, 1.0 / p.N,
      reinterpret_cast<T*>(vstore), warm, stats, gws, iter);
  return cudaGetLastError();
}

template <int D>
cudaError_t launch_xeig_t(const FftPlan& p, const double2* spec, const int* canon, double* lmin,
                          cudaStream_t s, unsigned char* gws) {
  constexpr int NT = GroupShape<D>::NT, GPC = GroupShape<D>::GPC;
  constexpr bool G = GroupShape<D>::GLOBAL;
  const size_t smem = G ? 0 : XSmem<D, double>::bytes * GPC;
  if (!G) {
    static unsigned long long mask = 0;
    cudaError_t e = smem_once(k_xeig<D>, smem, mask);
    if (e != cudaSuccess) return e;
  } else if (!gws) {
    return cudaErrorInvalidValue;
  }
  const int nc = fft_ncanon(p);
  long blocks = (nc + GPC - 1) / GPC;
  const long res = G ? (long)big_grid() : resident_grid((const void*)k_xeig<D>, NT * GPC, smem);
  if (blocks > res) blocks = res;
  k_xeig<D><<<(unsigned)blocks, NT * GPC, smem, s>>>(spec, canon, nc, p, lmin, gws);
  return cudaGetLastError();
}

template <typename R>
cudaError_t run_pass_t(const FftPlan& p, const FftPass& ps, int dir, const double* xin,
                       const void* cin, void* cout, double* xout, const double2* tw,
                       cudaStream_t s) {
  using V = typename C2<R>::type;
  const bool pow2 = (ps.n & (ps.n - 1)) == 0;
  // narrower entry chunks when the pass has few lines, so that the grid fills the GPU
  const long lines = (long)ps.A * ps.B;
  int ec = ps.ec[sizeof(R) == 4 ? 1 : 0];
  if (ec <= 0) {
    ec = FFT_EC;
    while (ec > 8 && lines * ((p.E + ec - 1) / ec) < 304) ec /= 2;
  }
  const size_t smem = sizeof(V) * ps.n * ec * (pow2 ? 1 : 2);
  static unsigned long long mask = 0;
  cudaError_t e = smem_once(k_fft_pass<R>, 2 * sizeof(V) * 64 * FFT_EC, mask);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)lines, (unsigned)((p.E + ec - 1) / ec));
  k_fft_pass<R><<<grid, FFT_THREADS, smem, s>>>(xin, reinterpret_cast<const V*>(cin),
                                                reinterpret_cast<V*>(cout), xout, ps, dir, p.E, tw,
                                                ec);
  return cudaGetLastError();
}

cudaError_t run_pass(const FftPlan& p, const FftPass& ps, int dir, const double* xin,
                     const void* cin, void* cout, double* xout, const double2* tw, bool fp32,
                     cudaStream_t s) {
  return fp32 ? run_pass_t<float>(p, ps, dir, xin, cin, cout, xout, tw, s)
              : run_pass_t<double>(p, ps, dir, xin, cin, cout, xout, tw, s);
}

int smallest_factor_pair(int N, int& N1, int& N2) {
  // N = N1 * N2 with N1 >= N2, both <= 64, preferring the most balanced split (N2 = 1 when
  // N <= 64 is prime)
  int best = -1;
  for (int a = 1; a <= 64; ++a) {
    if (N % a) continue;
    const int b = N / a;
    if (b > 64 || a < b) continue;
    if (best < 0 || a < best) best = a;
  }
  if (best < 0) return -1;
  N1 = best;
  N2 = N / best;
  return 0;
}

}  // namespace

int fft_plan_build(FftPlan& p, int dim, const int M[2], int D) {
  p = FftPlan{};
  p.dim = dim;
  p.D = D;
  p.E = D * D / 2;
  if (dim == 1) {
    p.M0 = M[0];
    p.M1 = 1;
    p.N = M[0];
    if (p.N < 2) return VE_EINVAL;
    int f1 = 0, f2 = 0;
    const bool pow2 = (p.N & (p.N - 1)) == 0;
    const bool split = p.N > 64 || (!pow2 && smallest_factor_pair(p.N, f1, f2) == 0 && f2 > 1);
    if (!split) {
      p.npass = 1;
      p.N1 = p.N;
      p.N2 = 1;
      p.ntab = 1;
      p.tab_n[0] = p.N;
      p.tab_off[0] = 0;
      p.ntw = p.N;
      p.fwd[0] = FftPass{1, p.N, 1, 0, 1, 0, 0};
      p.inv[0] = p.fwd[0];
    } else {
      int N1, N2;
      if (p.N > 4096 || smallest_factor_pair(p.N, N1, N2) || N2 < 2) return VE_EUNSUPPORTED;
      p.npass = 2;
      p.N1 = N1;
      p.N2 = N2;
      p.ntab = 3;
      p.tab_n[0] = N1;
      p.tab_n[1] = N2;
      p.tab_n[2] = p.N;
      p.tab_off[0] = 0;
      p.tab_off[1] = N1;
      p.tab_off[2] = N1 + N2;
      p.ntw = N1 + N2 + p.N;
      // forward: along a (length N1, lines b), twiddle w_N^(c b); then along b (length N2, lines c)
      p.fwd[0] = FftPass{1, N1, N2, 1, p.N, p.tab_off[0], p.tab_off[2]};
      p.fwd[1] = FftPass{N1, N2, 1, 0, 1, p.tab_off[1], 0};
      // inverse: along e (length N2, lines c) with twiddle w_N^(-b c); then along c (lines b)
      p.inv[0] = FftPass{N1, N2, 1, 2, p.N, p.tab_off[1], p.tab_off[2]};
      p.inv[1] = FftPass{1, N1, N2, 0, 1, p.tab_off[0], 0};
    }
  } else if (dim == 2) {
    p.M0 = M[0];
    p.M1 = M[1];
    p.N = M[0] * M[1];
    if (p.M0 < 1 || p.M1 < 1 || p.N < 2) return VE_EINVAL;
    if (p.M0 > 64 || p.M1 > 64) return VE_EUNSUPPORTED;
    p.npass = 2;
    p.N1 = p.M0;
    p.N2 = p.M1;
    p.ntab = 2;
    p.tab_n[0] = p.M0;
    p.tab_n[1] = p.M1;
    p.tab_off[0] = 0;
    p.tab_off[1] = p.M0;
    p.ntw = p.M0 + p.M1;
    p.fwd[0] = FftPass{1, p.M0, p.M1, 0, 1, p.tab_off[0], 0};
    p.fwd[1] = FftPass{p.M0, p.M1, 1, 0, 1, p.tab_off[1], 0};
    p.inv[0] = p.fwd[1];
    p.inv[1] = p.fwd[0];
  } else {
    return VE_EINVAL;
  }
  if (D != 4 && D != 16 && D != 64 && D != 256) return VE_EUNSUPPORTED;
  return 0;
}

cudaError_t launch_fft_tables(const FftPlan& p, double2* tw, cudaStream_t s) {
  k_fft_tables<<<(p.ntw + 255) / 256, 256, 0, s>>>(tw, p);
  return cudaGetLastError();
}

namespace {

std::mutex g_tune_mu;
std::map<std::string, std::string> g_tune;  // key -> "ec ec ec ec" (fwd0 fwd1 inv0 inv1)
bool g_tune_loaded = false;

std::string tune_key(const FftPlan& p, bool fp32) {
  int dev = 0, sms = 0, ma = 0, mi = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&ma, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&mi, cudaDevAttrComputeCapabilityMinor, dev);
  char k[128];
  snprintf(k, sizeof(k), "cc%d%d_sm%d_dim%d_M%dx%d_D%d_%s", ma, mi, sms, p.dim, p.M0, p.M1, p.D,
           fp32 ? "f32" : "f64");
  return k;
}

void tune_load_file() {
  g_tune_loaded = true;
  const char* path = getenv("VE_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char key[128];
  int a, b, c, d;
  while (fscanf(f, "%127s %d %d %d %d", key, &a, &b, &c, &d) == 5) {
    char v[64];
    snprintf(v, sizeof(v), "%d %d %d %d", a, b, c, d);
    g_tune[key] = v;
  }
  fclose(f);
}

void tune_store_file(const std::string& key, const std::string& val) {
  const char* path = getenv("VE_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %s\n", key.c_str(), val.c_str());
  fclose(f);
}

// Mean time of `reps` launches of one pass with entries-per-CTA ec (ms), or < 0 on error.
float time_pass(const FftPlan& p, FftPass ps, int slot, int ec, int dir, const double* xin,
                const void* cin, void* cout, double* xout, const double2* tw, bool fp32,
                cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  ps.ec[slot] = ec;
  const int reps = 5;
  if (run_pass(p, ps, dir, xin, cin, cout, xout, tw, fp32, s) != cudaSuccess) return -1.f;
  if (cudaEventRecord(e0, s) != cudaSuccess) return -1.f;
  for (int r = 0; r < reps; ++r)
    if (run_pass(p, ps, dir, xin, cin, cout, xout, tw, fp32, s) != cudaSuccess) return -1.f;
  if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
    return -1.f;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms / reps;
}

}  // namespace

cudaError_t fft_tune(FftPlan& p, const double* x, double2* bufA, double2* bufB, const double2* tw,
                     bool fp32, cudaStream_t s) {
  const int slot = fp32 ? 1 : 0;
  const std::string key = tune_key(p, fp32);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!g_tune_loaded) tune_load_file();
    const auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      int v[4];
      if (sscanf(it->second.c_str(), "%d %d %d %d", &v[0], &v[1], &v[2], &v[3]) == 4) {
        p.fwd[0].ec[slot] = v[0];
        p.fwd[1].ec[slot] = v[1];
        p.inv[0].ec[slot] = v[2];
        p.inv[1].ec[slot] = v[3];
        return cudaSuccess;
      }
    }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cudaGetLastError();
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cudaGetLastError();
  }
  // scratch block-row output for the last inverse pass: a spectrum buffer holds N D^2 doubles
  double* xscratch = reinterpret_cast<double*>(bufA);
  // the passes in use: forward then inverse (one each for a one-pass transform)
  FftPass* passes[4] = {&p.fwd[0], &p.fwd[1], &p.inv[0], &p.inv[1]};
  if (p.npass == 1) passes[1] = &p.inv[0];
  const int n = p.npass == 1 ? 2 : 4;
  cudaError_t err = cudaSuccess;
  for (int i = 0; i < n && err == cudaSuccess; ++i) {
    // (forward 0: x -> bufA; forward 1: bufA -> bufB; inverse 0: the spectrum -> the other
    // buffer; inverse 1: that buffer -> scratch block row)
    const bool fwd = p.npass == 1 ? i == 0 : i < 2;
    const int k = p.npass == 1 ? 0 : (i % 2);
    const double* xin = nullptr;
    const void* cin = nullptr;
    void* cout = nullptr;
    double* xout = nullptr;
    if (fwd && k == 0) { xin = x; cout = bufA; }
    else if (fwd) { cin = bufA; cout = bufB; }
    else if (p.npass == 1) { cin = bufB; xout = xscratch; }
    else if (k == 0) { cin = bufA; cout = bufB; }
    else { cin = bufB; xout = xscratch; }
    int best = 0;
    float best_ms = 0.f;
    for (int ec = 8; ec <= FFT_EC; ec *= 2) {
      const float ms = time_pass(p, *passes[i], slot, ec, fwd ? -1 : +1, xin, cin, cout, xout, tw,
                                 fp32, s, e0, e1);
      if (ms < 0.f) {
        err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaErrorUnknown;
        break;
      }
      if (best == 0 || ms < best_ms) {
        best = ec;
        best_ms = ms;
      }
    }
    passes[i]->ec[slot] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return err;
  char v[64];
  snprintf(v, sizeof(v), "%d %d %d %d", p.fwd[0].ec[slot], p.fwd[1].ec[slot], p.inv[0].ec[slot],
           p.inv[1].ec[slot]);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_tune.find(key) == g_tune.end()) {
    g_tune[key] = v;
    tune_store_file(key, v);
  }
  return cudaSuccess;
}

cudaError_t fft_forward(const FftPlan& p, const double* x, double2* bufA, double2* bufB,
                        const double2* tw, double2** spec, bool fp32, cudaStream_t s) {
  cudaError_t e = run_pass(p, p.fwd[0], -1, x, nullptr, bufA, nullptr, tw, fp32, s);
  if (e != cudaSuccess) return e;
  if (p.npass == 1) {
    *spec = bufA;
    return cudaSuccess;
  }
  e = run_pass(p, p.fwd[1], -1, nullptr, bufA, bufB, nullptr, tw, fp32, s);
  *spec = bufB;
  return e;
}

cudaError_t fft_inverse(const FftPlan& p, double2* spec, double2* bufA, double2* bufB, double* x,
                        const double2* tw, bool fp32, cudaStream_t s) {
  if (p.npass == 1) return run_pass(p, p.inv[0], +1, nullptr, spec, nullptr, x, tw, fp32, s);
  double2* other = (spec == bufA) ? bufB : bufA;
  cudaError_t e = run_pass(p, p.inv[0], +1, nullptr, spec, other, nullptr, tw, fp32, s);
  if (e != cudaSuccess) return e;
  return run_pass(p, p.inv[1], +1, nullptr, other, nullptr, x, tw, fp32, s);
}

// ---- D = 256 in float32: the projection itself runs in ve_tcproj.cu (tensor-core products);
// these kernels move the canonical blocks between the float32 spectrum and its split KC4 input
// and output buffers.
__device__ __forceinline__ float2 x256_entry(const float2* spec, int s, int s2, int E, int f) {
  if (f < E) {  // (z + conj(zz)) / 2
    const float2 z = spec[(long)s * E + f], zz = spec[(long)s2 * E + f];
    return make_float2(0.5f * (z.x + zz.x), 0.5f * (z.y - zz.y));
  }
  const float2 z = spec[(long)s * E + f - E], zz = spec[(long)s2 * E + f - E];  // (z - conj(zz)) / 2i
  return make_float2(0.5f * (z.y + zz.y), -0.5f * (z.x - zz.x));
}

__global__ void __launch_bounds__(256) k_x256_unpack(const float2* __restrict__ spec, const int* __restrict__ canon,
                                                     int ncanon, const FftPlan p, float* __restrict__ C) {
  constexpr int D = 256, PL = D * D;
  const long total = (long)ncanon * (PL / 4);
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
    const int j = (int)(q / (PL / 4)), c4 = (int)(q % (PL / 4));
    const int r = c4 % D, k0 = (c4 / D) * 4;
    const int s = canon[j], s2 = partner_slot(p, s);
    float re[4], im[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + u;
      const float2 a = x256_entry(spec, s, s2, p.E, r * D + k);
      const float2 b = x256_entry(spec, s, s2, p.E, k * D + r);
      re[u] = r == k ? a.x : 0.5f * (a.x + b.x);  // Hermitised as in unpack_block
      im[u] = r == k ? 0.f : 0.5f * (a.y - b.y);
    }
    float* out = C + (size_t)j * 4 * PL + 4 * (size_t)c4;
    float4 h, l;
    h = make_float4(tc_hi(re[0]), tc_hi(re[1]), tc_hi(re[2]), tc_hi(re[3]));
    l = make_float4(re[0] - h.x, re[1] - h.y, re[2] - h.z, re[3] - h.w);
    *reinterpret_cast<float4*>(out) = h;
    *reinterpret_cast<float4*>(out + PL) = l;
    h = make_float4(tc_hi(im[0]), tc_hi(im[1]), tc_hi(im[2]), tc_hi(im[3]));
    l = make_float4(im[0] - h.x, im[1] - h.y, im[2] - h.z, im[3] - h.w);
    *reinterpret_cast<float4*>(out + 2 * PL) = h;
    *reinterpret_cast<float4*>(out + 3 * PL) = l;
  }
}

// Y_k (split KC4, Hermitian) back into the spectrum, scaled by 1/N, with Y_{-k} = conj Y_k.
__global__ void __launch_bounds__(256) k_x256_pack(const float* __restrict__ Y, const int* __restrict__ canon,
                                                   int ncanon, const FftPlan p, float sc, float2* __restrict__ spec) {
  constexpr int D = 256, PL = D * D;
  const int E = p.E;
  const long total = (long)ncanon * E;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
    const int j = (int)(q / E), e = (int)(q % E);
    const int s = canon[j], s2 = partner_slot(p, s);
    const float* y = Y + (size_t)j * 4 * PL;
    const int i1 = e / D, k1 = e % D, i2 = (e + E) / D, k2 = (e + E) % D;
    const int o1 = ((k1 >> 2) * D + i1) * 4 + (k1 & 3), o2 = ((k2 >> 2) * D + i2) * 4 + (k2 & 3);
    const float y1r = (y[o1] + y[PL + o1]) * sc, y1i = (y[2 * PL + o1] + y[3 * PL + o1]) * sc;
    const float y2r = (y[o2] + y[PL + o2]) * sc, y2i = (y[2 * PL + o2] + y[3 * PL + o2]) * sc;
    spec[(long)s * E + e] = make_float2(y1r - y2i, y1i + y2r);
    if (s2 != s) spec[(long)s2 * E + e] = make_float2(y1r + y2i, y2r - y1i);
  }
}

template <int D>
cudaError_t launch_xproj_d(const FftPlan& p, double2* spec, const int* canon, int arith,
                           void* vstore, int warm, cudaStream_t s, unsigned long long* stats,
                           unsigned char* gws, const long long* iter) {
  switch (arith) {
    case ARITH_FP64: return launch_xproj_t<D, double>(p, spec, canon, vstore, warm, s, stats, gws, iter);
    case ARITH_FP32: return launch_xproj_t<D, float>(p, spec, canon, vstore, warm, s, stats, gws, iter);
    case ARITH_DF64: return launch_xproj_t<D, df64>(p, spec, canon, vstore, warm, s, stats, gws, iter);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_xproj(const FftPlan& p, double2* spec, const int* canon, int arith,
                         void* vstore, int warm, cudaStream_t s, unsigned long long* stats,
                         unsigned char* gws, const long long* iter) {
  switch (p.D) {
    case 4: return launch_xproj_d<4>(p, spec, canon, arith, vstore, warm, s, stats, gws, iter);
    case 16: return launch_xproj_d<16>(p, spec, canon, arith, vstore, warm, s, stats, gws, iter);
    case 64: return launch_xproj_d<64>(p, spec, canon, arith, vstore, warm, s, stats, gws, iter);
    case 256: return launch_xproj_d<256>(p, spec, canon, arith, vstore, warm, s, stats, gws, iter);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_xproj_tc(const FftPlan& p, double2* spec, const int* canon, TcProjWs& w, int warm,
                            cudaStream_t s, unsigned long long* stats) {
  if (p.D != 256 || !w.cplx) return cudaErrorInvalidValue;
  const int nc = fft_ncanon(p);
  float2* sp = reinterpret_cast<float2*>(spec);
  const int grid = 4 * big_grid();
  k_x256_unpack<<<grid, 256, 0, s>>>(sp, canon, nc, p, w.C);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = tc_project256(w, nc, warm != 0, stats, s)) != cudaSuccess) return e;
  k_x256_pack<<<grid, 256, 0, s>>>(w.Wt, canon, nc, p, (float)(1.0 / p.N), sp);
  return cudaGetLastError();
}

cudaError_t launch_xeig(const FftPlan& p, const double2* spec, const int* canon, double* lmin,
                        cudaStream_t s, unsigned char* gws) {
  switch (p.D) {
    case 4: return launch_xeig_t<4>(p, spec, canon, lmin, s, gws);
    case 16: return launch_xeig_t<16>(p, spec, canon, lmin, s, gws);
    case 64: return launch_xeig_t<64>(p, spec, canon, lmin, s, gws);
    case 256: return launch_xeig_t<256>(p, spec, canon, lmin, s, gws);
    default: return cudaErrorInvalidValue;
  }
}

size_t xproj_ws_bytes(int D) {
  if (D != 256) return 0;
  size_t a = XSmem<256, double>::bytes;
  if (XSmem<256, df64>::bytes > a) a = XSmem<256, df64>::bytes;
  return a * (size_t)big_grid();
}

cudaError_t launch_canon_list(const FftPlan& p, int* canon, cudaStream_t s) {
  k_canon_list<<<1, 256, 0, s>>>(p, canon);
  return cudaGetLastError();
}

int fft_ncanon(const FftPlan& p) {
  // k and -k pair up; the self-conjugate wavevectors (2k = 0 on every axis) stand alone
  int selfc = 1;
  if (p.dim == 1) {
    selfc = (p.N % 2 == 0) ? 2 : 1;
  } else {
    selfc = ((p.M0 % 2 == 0) ? 2 : 1) * ((p.M1 % 2 == 0) ? 2 : 1);
  }
  return (p.N - selfc) / 2 + selfc;
}

}  // namespace ve
