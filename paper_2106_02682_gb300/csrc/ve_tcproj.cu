// ve_tcproj.cu -- batched float32 PSD projection of 256 x 256 matrices, Pi_{>=0}(C) = V max(L, 0)
// V^H, with its GEMM-shaped work on the tensor cores (ve_tcgemm.cu).  It serves the float32
// phase of the 4-spin-cluster solver: the pair projections of Eq. (rhoijTildeUpdate) (real
// symmetric) and the per-wavevector projections of Algorithm 6 (complex Hermitian), Khoo &
// Lindsey, arXiv:2106.02682.
//
// Per matrix, starting from the eigenvectors V kept from the previous sweep (V = I cold):
//   1. T = (3 I - V^H V) / 2          Newton-Schulz step against float32 drift of V
//   2. V1 = V T
//   3. W = C V1,  A = V1^H W           A is diagonal up to the change since the last sweep
//   4. block-Jacobi sweeps on A whose rotations are applied by tensor-core products (below),
//      then scalar Jacobi (SIMT, one CTA per matrix) from Q = I with the first-order stop: it leaves
//      M = diag(max(l, 0)), or M = f(L) + L o E when the off-diagonal part E is small enough
//      (Daleckii-Krein, see dk_stop in ve_device.cuh), and the rotations Q
//   5. V2 = V1 Q (kept for the next sweep),  Y = V2 M V2^H
// Steps 1-3 and 5 are seven batched tensor-core products; only step 4 runs on the SIMT pipes.
// Matrices are held "split" (hi = tf32 part, lo = remainder) in the KC4 layout of ve_tcgemm.cu,
// except the block-Jacobi operands A, W^T and V1, which the rotation products read and write
// whole every round: those are plain float32 planes (re; re, im) in the same layout, split on
// load inside the rotation kernel -- half the bytes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ve_device.cuh"
#include "ve_internal.h"
#include "ve_tc.cuh"

namespace ve {

namespace {

constexpr int kN = 256, kPl = kN * kN, kLD = kN + 1, kNT = 512;

__device__ __forceinline__ void split4(const float* v, float4& hi, float4& lo) {
  hi = make_float4(tc::tf32_hi(v[0]), tc::tf32_hi(v[1]), tc::tf32_hi(v[2]), tc::tf32_hi(v[3]));
  lo = make_float4(v[0] - hi.x, v[1] - hi.y, v[2] - hi.z, v[3] - hi.w);
}

// Identity in split form (the cold start V = I) for `count` matrices of `npl` planes.
__global__ void k_tc_identity(float* V, float* Vt, long count, int npl) {
  const long total = count * npl * (long)(kPl / 4);
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
    const long mat = q / (npl * (kPl / 4));
    const int rem = (int)(q % (npl * (kPl / 4)));
    const int pl = rem / (kPl / 4), c4 = rem % (kPl / 4);  // c4 = chunk * 256 + row
    const int r = c4 % kN, k0 = (c4 / kN) * 4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pl == 0) {
      v.x = (r == k0) ? 1.f : 0.f;
      v.y = (r == k0 + 1) ? 1.f : 0.f;
      v.z = (r == k0 + 2) ? 1.f : 0.f;
      v.w = (r == k0 + 3) ? 1.f : 0.f;
    }
    const size_t off = ((size_t)mat * npl + pl) * kPl + (size_t)c4 * 4;
    *reinterpret_cast<float4*>(V + off) = v;
    *reinterpret_cast<float4*>(Vt + off) = v;
  }
}

template <bool CPLX>
struct JShape {
  static constexpr size_t MAT = ((sizeof(float) * kN * kLD + 255) / 256) * 256;
  static constexpr int NMAT = CPLX ? 4 : 2;
  static constexpr size_t bytes = NMAT * MAT + 4096;
};

// Step 4: one CTA of 512 threads per matrix, the matrix and its rotations staged in a per-CTA
// slice of a global workspace (L2-resident).  In: A (plain, KC4).  Out: M (split, KC4) and Q^T.
template <bool CPLX>
__global__ void __launch_bounds__(kNT, 1)
    k_tc_jacobi(const float* __restrict__ Ain, float* __restrict__ Mout, float* __restrict__ Qt, long count,
                unsigned char* ws, unsigned long long* stats) {
  using S = JShape<CPLX>;
  constexpr int NPL = CPLX ? 4 : 2, NPX = CPLX ? 2 : 1;
  unsigned char* base = ws + (size_t)blockIdx.x * S::bytes;
  float* Ar = reinterpret_cast<float*>(base);
  float* Vr = reinterpret_cast<float*>(base + S::MAT);
  float* Ai = CPLX ? reinterpret_cast<float*>(base + 2 * S::MAT) : nullptr;
  float* Vi = CPLX ? reinterpret_cast<float*>(base + 3 * S::MAT) : nullptr;
  float* cs = reinterpret_cast<float*>(base + S::NMAT * S::MAT);
  float* red = cs + 2 * kN;
  const int tid = threadIdx.x;
  for (long b = blockIdx.x; b < count; b += gridDim.x) {
    const float* A = Ain + (size_t)b * NPX * kPl;
    // load (plain planes; one float4 chunk of a row per thread and step: coalesced)
    for (int q = tid; q < kPl / 4; q += kNT) {
      const int r = q % kN, k0 = (q / kN) * 4;
      const float4 h = *reinterpret_cast<const float4*>(A + 4 * q);
      float* row = Ar + r * kLD + k0;
      row[0] = h.x;
      row[1] = h.y;
      row[2] = h.z;
      row[3] = h.w;
      if constexpr (CPLX) {
        const float4 h2 = *reinterpret_cast<const float4*>(A + kPl + 4 * q);
        float* ri = Ai + r * kLD + k0;
        ri[0] = h2.x;
        ri[1] = h2.y;
        ri[2] = h2.z;
        ri[3] = h2.w;
      }
    }
    __syncthreads();
    // (A + A^H) / 2: the product V^H C V is Hermitian only to rounding
    for (int t = tid; t < kN * (kN + 1) / 2; t += kNT) {
      int i, j;
      tri_index(kN, t, i, j);
      if (i == j) {
        if constexpr (CPLX) Ai[i * kLD + i] = 0.f;
        continue;
      }
      const float r = 0.5f * (Ar[i * kLD + j] + Ar[j * kLD + i]);
      Ar[i * kLD + j] = r;
      Ar[j * kLD + i] = r;
      if constexpr (CPLX) {
        const float im = 0.5f * (Ai[i * kLD + j] - Ai[j * kLD + i]);
        Ai[i * kLD + j] = im;
        Ai[j * kLD + i] = -im;
      }
    }
    __syncthreads();
    bool dk = false;
    int nsw;
    if constexpr (CPLX)
      nsw = jacobi_herm<float, kN, kLD, kNT, true, true, true>(Ar, Ai, Vr, Vi, cs, red, tid, &dk);
    else
      nsw = jacobi_sym<float, kN, kLD, kNT, true, true, true>(Ar, Vr, cs, red, tid, &dk);
    if (stats && tid == 0) {
      atomicAdd(stats, (unsigned long long)nsw);
      atomicAdd(stats + 1, 1ull);
      if (dk) atomicAdd(stats + 2, 1ull);
    }
    // M: f(L) + L o E after a first-order stop, else diag(max(l, 0))
    if (dk) {
      if constexpr (CPLX)
        dk_matrix_herm<float, kN, kLD, kNT>(Ar, Ai, cs, tid);
      else
        dk_matrix_sym<float, kN, kLD, kNT>(Ar, cs, tid);
    } else {
      for (int e = tid; e < kPl; e += kNT) {
        const int i = e / kN, j = e % kN;
        const float a = Ar[i * kLD + j];
        Ar[i * kLD + j] = (i == j) ? (a > 0.f ? a : 0.f) : 0.f;
        if constexpr (CPLX) Ai[i * kLD + j] = 0.f;
      }
      __syncthreads();
    }
    float* M = Mout + (size_t)b * NPL * kPl;
    float* Q = Qt + (size_t)b * NPL * kPl;
    for (int q = tid; q < kPl / 4; q += kNT) {
      const int r = q % kN, k0 = (q / kN) * 4;
      float v[4];
      float4 hi, lo;
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = Ar[r * kLD + k0 + u];
      split4(v, hi, lo);
      *reinterpret_cast<float4*>(M + 4 * q) = hi;
      *reinterpret_cast<float4*>(M + kPl + 4 * q) = lo;
      // Q^T[r][k] = Q[k][r]: the rotations accumulated in V
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = Vr[(k0 + u) * kLD + r];
      split4(v, hi, lo);
      *reinterpret_cast<float4*>(Q + 4 * q) = hi;
      *reinterpret_cast<float4*>(Q + kPl + 4 * q) = lo;
      if constexpr (CPLX) {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = Ai[r * kLD + k0 + u];
        split4(v, hi, lo);
        *reinterpret_cast<float4*>(M + 2 * kPl + 4 * q) = hi;
        *reinterpret_cast<float4*>(M + 3 * kPl + 4 * q) = lo;
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = Vi[(k0 + u) * kLD + r];
        split4(v, hi, lo);
        *reinterpret_cast<float4*>(Q + 2 * kPl + 4 * q) = hi;
        *reinterpret_cast<float4*>(Q + 3 * kPl + 4 * q) = lo;
      }
    }
    __syncthreads();
  }
}

// ---- block Jacobi: the 256 indices form TC_BJ_NB = 16 blocks of TC_BJ_BS = 16; a round pairs
// the blocks by the circle ordering (15 rounds a sweep, 8 disjoint pairs a round).  For each pair
// (I, J) the 32 x 32 principal block A[I u J, I u J] is diagonalised exactly by one warp in shared
// memory (k_bj_sub), its eigenvectors U placed in the round's rotation R (R[I u J, I u J] = U,
// zero elsewhere), and A <- R^H A R, V <- V R are three tensor-core products that touch only
// R's nonzero blocks (tc_rot256), which are stored compactly (one 32 x 32 block per pair).  A sweep of rounds annihilates every off-diagonal
// block once; like scalar Jacobi it converges quadratically.
constexpr int kBS = TC_BJ_BS, kNB = TC_BJ_NB, kSub = 2 * kBS, kSLD = kSub + 1, kSubWarps = 4;
constexpr int kRc = kN * kSub;  // floats of one plane of a compact rotation (256 rows x 32 K)

template <bool CPLX>
struct SubShape {
  static constexpr int NMAT = CPLX ? 4 : 2;
  static constexpr size_t per_warp = sizeof(float) * (NMAT * kSub * kSLD + 2 * kSub + 32);
  static constexpr size_t bytes = per_warp * kSubWarps;
};

__device__ __forceinline__ int kc4i(int r, int k) { return ((k >> 2) * kN + r) * 4 + (k & 3); }

// ||A_b||_F^2 of every matrix (npx plain planes), one CTA per matrix, fixed summation order.
__global__ void __launch_bounds__(256) k_fro2(const float* __restrict__ A, int npx, float* __restrict__ out) {
  __shared__ float red[8];
  const float* a = A + (size_t)blockIdx.x * npx * kPl;
  float s = 0.f;
  for (int pl = 0; pl < npx; ++pl)
    for (int e = threadIdx.x; e < kPl; e += 256) {
      const float v = a[pl * kPl + e];
      s = fmaf(v, v, s);
    }
  s = gsum<256>(s, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// fro2[b] = ||A_b||_F^2: a pair block stops at the accuracy the whole matrix needs.  The scalar
// test off^2 <= (n u)^2 ||A||^2 over 120 block pairs of a sweep holds for the matrix when every
// block meets off^2 <= (256 u)^2 ||A||^2 / 120, i.e. the block test (32 u)^2 nrm with
// nrm >= (256 / 32)^2 / 120 ||A||^2 ~ 0.5 ||A||^2.
template <bool CPLX>
__global__ void __launch_bounds__(32 * kSubWarps)
    k_bj_sub(const float* __restrict__ A, float* __restrict__ Rt, long count, int round,
             const float* __restrict__ fro2, int max_inner) {
  constexpr int NPL = CPLX ? 4 : 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* Sr = reinterpret_cast<float*>(smem_raw + w * SubShape<CPLX>::per_warp);
  float* Ur = Sr + kSub * kSLD;
  float* Si = CPLX ? Ur + kSub * kSLD : nullptr;
  float* Ui = CPLX ? Si + kSub * kSLD : nullptr;
  float* cs = Sr + SubShape<CPLX>::NMAT * kSub * kSLD;
  float* red = cs + 2 * kSub;
  const long items = count * (kNB / 2);
  for (long item = (long)blockIdx.x * kSubWarps + w; item < items; item += (long)gridDim.x * kSubWarps) {
    const long b = item / (kNB / 2);
    const int k = (int)(item % (kNB / 2));
    int bp, bq;
    rr_pair(kNB, round, k, bp, bq);
    auto g = [&](int t) { return t < kBS ? bp * kBS + t : bq * kBS + (t - kBS); };
    const float* a = A + (size_t)b * (NPL / 2) * kPl;  // plain: re (, im)
    for (int e = lane; e < kSub * kSub; e += 32) {
      const int i = e / kSub, j = e % kSub;
      const int o = kc4i(g(i), g(j));
      Sr[i * kSLD + j] = a[o];
      if constexpr (CPLX) Si[i * kSLD + j] = a[kPl + o];
    }
    __syncwarp();
    // (S + S^H) / 2
    for (int e = lane; e < kSub * kSub; e += 32) {
      const int i = e / kSub, j = e % kSub;
      if (i < j) {
        const float v = 0.5f * (Sr[i * kSLD + j] + Sr[j * kSLD + i]);
        Sr[i * kSLD + j] = v;
        Sr[j * kSLD + i] = v;
        if constexpr (CPLX) {
          const float x = 0.5f * (Si[i * kSLD + j] - Si[j * kSLD + i]);
          Si[i * kSLD + j] = x;
          Si[j * kSLD + i] = -x;
        }
      } else if (i == j) {
        if constexpr (CPLX) Si[i * kSLD + i] = 0.f;
      }
    }
    __syncwarp();
    const float floor2 = 0.5f * fro2[b];
    if constexpr (CPLX)
      jacobi_herm<float, kSub, kSLD, 32, true>(Sr, Si, Ur, Ui, cs, red, lane, nullptr, nullptr, floor2,
                                               max_inner);
    else
      jacobi_sym<float, kSub, kSLD, 32, true>(Sr, Ur, cs, red, lane, nullptr, nullptr, floor2, max_inner);
    // The round's rotation, compact: per matrix NPL split planes of 256 rows x 32 K (KC4), row
    // 32 k + c and K index a holding U[a][c] (pair-local indices, block bp then block bq): the
    // rotation products read each pair's 32 x 32 block as one box.  A lane writes one 4-index
    // chunk of one row as a float4.
    float* rc = Rt + (size_t)b * NPL * kRc;
    for (int e = lane; e < kSub * (kSub / 4); e += 32) {
      const int c = e / (kSub / 4), ch = e % (kSub / 4);  // row 32 k + c, K chunk 4 ch .. + 3
      float ur[4], ui[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ur[u] = Ur[(4 * ch + u) * kSLD + c];
        if constexpr (CPLX) ui[u] = Ui[(4 * ch + u) * kSLD + c];
      }
      const int o = (ch * kN + kSub * k + c) * 4;
      float4 hi, lo;
      split4(ur, hi, lo);
      *reinterpret_cast<float4*>(rc + o) = hi;
      *reinterpret_cast<float4*>(rc + kRc + o) = lo;
      if constexpr (CPLX) {
        split4(ui, hi, lo);
        *reinterpret_cast<float4*>(rc + 2 * kRc + o) = hi;
        *reinterpret_cast<float4*>(rc + 3 * kRc + o) = lo;
      }
    }
    __syncwarp();
  }
}

// Plain -> split: every float32 of `count` matrices of npx plain planes (KC4) becomes its hi / lo
// pair in 2 npx planes.
__global__ void k_tc_split(const float* __restrict__ in, float* __restrict__ out, long count, int npx) {
  const long total = count * npx * (long)(kPl / 4);
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
    const long mp = q / (kPl / 4);  // matrix * npx + plane
    const int c = (int)(q % (kPl / 4));
    const float4 v = reinterpret_cast<const float4*>(in)[q];
    float hv[4] = {v.x, v.y, v.z, v.w};
    float4 hi, lo;
    split4(hv, hi, lo);
    const long mat = mp / npx, pl = mp % npx;
    float* o = out + ((size_t)mat * 2 * npx + 2 * pl) * kPl + (size_t)c * 4;
    *reinterpret_cast<float4*>(o) = hi;
    *reinterpret_cast<float4*>(o + kPl) = lo;
  }
}

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

size_t tc_proj_ws_bytes(long cap, int cplx) {
  const size_t mat = (size_t)(cplx ? 4 : 2) * kPl * sizeof(float);
  const size_t jws = (cplx ? JShape<true>::bytes : JShape<false>::bytes) * (size_t)big_grid();
  return 9 * al256(mat * (size_t)cap) + al256(jws) + 256;
}

int tc_proj_ws_init(TcProjWs& w, long cap, int cplx, void* mem, size_t bytes) {
  if (cap <= 0 || !mem || bytes < tc_proj_ws_bytes(cap, cplx) || ((uintptr_t)mem & 255)) return -1;
  w = TcProjWs();
  w.cap = cap;
  w.cplx = cplx;
  const size_t mat = al256((size_t)(cplx ? 4 : 2) * kPl * sizeof(float) * (size_t)cap);
  unsigned char* p = (unsigned char*)mem;
  float** bufs[9] = {&w.V, &w.Vt, &w.C, &w.T, &w.V1, &w.V1t, &w.Wt, &w.M, &w.Qt};
  for (auto b : bufs) {
    *b = (float*)p;
    p += mat;
  }
  w.jws = p;
  p += al256((cplx ? JShape<true>::bytes : JShape<false>::bytes) * (size_t)big_grid());
  w.err = (int*)p;
  return 0;
}

cudaError_t tc_project256(TcProjWs& w, long count, bool warm, unsigned long long* stats, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (count > w.cap) return cudaErrorInvalidValue;
  const int npl = w.cplx ? 4 : 2;
  cudaError_t e;
  if (!warm) {
    const long q = count * npl * (long)(kPl / 4);
    const int grid = (int)((q + 255) / 256 < 4096 ? (q + 255) / 256 : 4096);
    k_tc_identity<<<grid, 256, 0, s>>>(w.V, w.Vt, count, npl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  auto gemm = [&](const float* x, int cx, const float* y, int cy, float alpha, float beta, float* on,
                  float* ot, int plain_n = 0) {
    TcGemm g;
    g.x = x;
    g.y = y;
    g.batch = count;
    g.cplx = w.cplx;
    g.conj_x = cx;
    g.conj_y = cy;
    g.alpha = alpha;
    g.beta = beta;
    g.out_n = on;
    g.out_t = ot;
    g.plain_n = plain_n;
    g.err = w.err;
    return tc_gemm256(g, s);
  };
  // The block-Jacobi operands A, W^T (as B = A R) and V1 are kept plain (float32 planes, half the
  // bytes of the split form): the rotation products read and write them whole every round.
  // 1. T = 1.5 I - 0.5 V^H V   (V^H V)_ij = sum_k conj(Vt_ik) Vt_jk
  if ((e = gemm(w.Vt, 1, w.Vt, 0, -0.5f, 1.5f, w.T, nullptr)) != cudaSuccess) return e;
  // 2. V1 = V T (plain) and V1^T (split): the right factor enters as T^T = conj(T)
  if ((e = gemm(w.V, 0, w.T, 1, 1.f, 0.f, w.V1, w.V1t, 1)) != cudaSuccess) return e;
  // 3. W = C V1 (kept as W^T), then A = V1^H W into T's storage (plain)
  if ((e = gemm(w.C, 0, w.V1t, 0, 1.f, 0.f, nullptr, w.Wt)) != cudaSuccess) return e;
  float* A = w.T;
  if ((e = gemm(w.V1t, 1, w.Wt, 0, 1.f, 0.f, A, nullptr, 1)) != cudaSuccess) return e;
  // block-Jacobi sweeps: the compact rotations in Qt's storage, A R kept transposed in Wt
  {
    const size_t smem = w.cplx ? SubShape<true>::bytes : SubShape<false>::bytes;
    static bool attr[2] = {false, false};
    if (!attr[w.cplx]) {
      e = w.cplx ? cudaFuncSetAttribute(k_bj_sub<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                 : cudaFuncSetAttribute(k_bj_sub<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr[w.cplx] = true;
    }
    const long items = count * (kNB / 2);
    const long ctas = (items + kSubWarps - 1) / kSubWarps;
    const int sgrid = (int)(ctas < 8L * big_grid() ? ctas : 8L * big_grid());
    float* fro2 = reinterpret_cast<float*>(w.M);  // M is free until the polish
    k_fro2<<<(unsigned)count, 256, 0, s>>>(A, w.cplx ? 2 : 1, fro2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Two block sweeps, each sub-problem one Jacobi sweep (an inexact block solve: the polish
    // below completes the eigensolve to the full tolerance).  Measured in steady state on the
    // 4-spin-cluster chain and the 2-D lattice: one block sweep leaves the scalar polish 1.2
    // sweeps per wavevector block (far dearer than a second block sweep), a third block sweep
    // costs more than the polish it saves, and sub-problems solved to convergence instead of one
    // sweep cost 3-4 % more time for the same polish work.
    const int inner = w.bj_inner > 0 ? w.bj_inner : JacobiTol<float>::max_sweeps;
    for (int sw = 0; sw < w.bj_sweeps; ++sw) {
      for (int r = 0; r < kNB - 1; ++r) {
        if (w.cplx)
          k_bj_sub<true><<<sgrid, 32 * kSubWarps, smem, s>>>(A, w.Qt, count, r, fro2, inner);
        else
          k_bj_sub<false><<<sgrid, 32 * kSubWarps, smem, s>>>(A, w.Qt, count, r, fro2, inner);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // B = A R (kept transposed in Wt); A <- R^H B written as (B^H R)^H; V1 <- V1 R.  All
        // three multiply by the block rotation R on the right (tc_rot256: its nonzero blocks
        // only), plain in and plain out.
        auto rot = [&](const float* x, int cx, float* on, float* ot, int co) {
          TcGemm g;
          g.x = x;
          g.y = w.Qt;
          g.batch = count;
          g.cplx = w.cplx;
          g.conj_x = cx;
          g.out_n = on;
          g.out_t = ot;
          g.plain_n = 1;
          g.plain_t = 1;
          g.conj_out = co;
          g.round = r;
          g.err = w.err;
          return tc_rot256(g, s);
        };
        if ((e = rot(A, 0, nullptr, w.Wt, 0)) != cudaSuccess) return e;
        if ((e = rot(w.Wt, 1, nullptr, A, 1)) != cudaSuccess) return e;
        // (V1^T is not read again in this projection: the steps after the sweeps use V1)
        if ((e = rot(w.V1, 0, w.V1, nullptr, 0)) != cudaSuccess) return e;
      }
    }
  }
  // 4. Jacobi from Q = I with the first-order stop: M and Q^T
  const int grid = (int)(count < big_grid() ? count : big_grid());
  if (w.cplx)
    k_tc_jacobi<true><<<grid, kNT, 0, s>>>(A, w.M, w.Qt, count, w.jws, stats);
  else
    k_tc_jacobi<false><<<grid, kNT, 0, s>>>(A, w.M, w.Qt, count, w.jws, stats);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // 5. V2 = V1 Q (the stored eigenvectors; V1 split into V1t's storage first), Z = V2 M into C,
  // Y = Z V2^H into Wt
  {
    const long q = count * (npl / 2) * (long)(kPl / 4);
    const int g2 = (int)((q + 255) / 256 < 8192 ? (q + 255) / 256 : 8192);
    k_tc_split<<<g2, 256, 0, s>>>(w.V1, w.V1t, count, npl / 2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = gemm(w.V1t, 0, w.Qt, 0, 1.f, 0.f, w.V, w.Vt)) != cudaSuccess) return e;
  if ((e = gemm(w.V, 0, w.M, 1, 1.f, 0.f, w.C, nullptr)) != cudaSuccess) return e;
  return gemm(w.C, 0, w.V, 1, 1.f, 0.f, w.Wt, nullptr);
}

}  // namespace ve
