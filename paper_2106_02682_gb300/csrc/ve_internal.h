// ve_internal.h -- declarations shared by the solver's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace ve {

// Arithmetic of the per-matrix work (pair pass, projections): native float64, float32, or
// double-float words (48-bit significand) on the float32 pipe (ve_df64.cuh).
enum Arith { ARITH_FP64 = 0, ARITH_FP32 = 1, ARITH_DF64 = 2 };

// Raise a kernel's dynamic shared-memory limit once per device (outside any stream capture:
// the first sweep of a handle runs uncaptured).
template <typename K>
inline cudaError_t smem_once(K kernel, size_t bytes, unsigned long long& mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (mask & bit) return cudaSuccess;
  e = cudaFuncSetAttribute((const void*)kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes);
  if (e == cudaSuccess) mask |= bit;
  return e;
}

// ------------------------------------------------------------------ sweep kernels
// Warm-started eigensolves rotate the eigenvectors kept from the previous sweep, and rounding
// erodes their orthogonality a little every sweep; a drifted V makes V^T C V a non-similarity
// and the projection inexact by as much.  A Newton-Schulz step V <- V (3 I - V^T V) / 2 squares
// the drift: every sweep in float32, every NS_EVERY-th sweep in float64 and double-float words
// (measured with a step every sweep: the float64 state after 300 sweeps agrees with the oracle to
// ~3e-13 instead of ~1e-10 at D = 64, 256; the drift between steps grows linearly, so a step every
// 16 sweeps keeps it far below the 1e-10 target at 1/16 of the cost).
constexpr int NS_EVERY = 16;
template <typename T>
__device__ __forceinline__ bool ns_due(const long long* iter) {
  if (sizeof(T) == 4) return true;
  return iter && (*iter % NS_EVERY) == 0;
}
struct PairArgs {
  int N, P, m, D;
  double mu, nu, eps;
  const double* rho0;   // m*m
  double* rt;           // P*D*D   rho~ (read, then overwritten)
  double* lam;          // P*D*D   Lambda
  double* lam1;         // P*m*m   (read; the images of tied offsets are written)
  double* lam2;         // P*m*m
  double* X;            // N*D*D   X_{0,delta}; blocks 1..N-1 become X' in the pair pass
  const double* hb;     // nonzero pair Hamiltonian blocks, D*D each
  const int* hslot;     // per linear delta: index into hb or -1
  double* a1r;          // P*m*m   A1[rho_{0,delta}]
  double* a2r;          // P*m*m   A2[rho_{0,delta}]
  double* part;         // P*2     ||rho - rho~||^2, Tr[H rho]
  void* vstore;         // P*D*D eigenvectors of the last projection (float or double)
  int warm;             // 1: start each Jacobi from V^T C V with the stored V
  // sweeps done so far (device); the stored V is re-orthogonalised when it is a multiple of
  // NS_EVERY (float64 / double-float; float32 every sweep).  null: never in those arithmetics
  const long long* iter = nullptr;
  // null, or [0] += Jacobi sweeps, [1] += matrices, [2] += first-order stops (profiling)
  unsigned long long* stats;
  unsigned char* gws;   // D = 256: per-CTA staging workspace (pair_ws_bytes), else unused
  // Offsets delta and -delta carry swap images of each other; the pass runs over Pc items, item
  // i updating pair index pidx[i] (delta - 1) and writing the image into pmir[i] (-1: -delta =
  // delta).  pidx == nullptr: Pc = P items, item i = pair index i, no images.
  int Pc;
  const int* pidx;
  const int* pmir;
  // D = 256 in float32 with the projection on the tensor cores (null: the k_pair kernel):
  // tcw holds the projection workspace for Pc matrices, rbuf Pc * D * D floats of rho
  struct TcProjWs* tcw = nullptr;
  float* rbuf = nullptr;
};

struct DevStatus {
  long long iter;
  double energy, feas, d_energy, residual;
  double e_prev;
  double h0rho0;  // Tr[H_0 rho_0] of the current sweep
  unsigned int done;  // CTAs of the running multi-CTA reduction finished (0 between kernels)
  unsigned int pad;
};

struct SmallArgs {
  int N, P, m, D, L;
  double mu, nu, eps;
  double* rho0;
  double* lam1;
  double* lam2;
  double* X;
  const double* H0;
  const double* a1r;
  const double* a2r;
  const double* part;
  double* part2;  // P: ||A1 rho - rho0||^2 + ||A2 rho - rho0||^2
  // P: for the canonical member of {delta, -delta} the pair index of the other, -1 when
  // -delta = delta, -2 for the member whose Lambda1, Lambda2 its partner writes; or nullptr
  const int* ptie;
  DevStatus* st;
  double* rho0_partial;  // 128 * m*m chunk sums of the rho_0 reduction, then the status sums
};

// Number of CTAs that keep every SM busy for a kernel with the given block shape.
int resident_grid(const void* kernel, int threads, size_t smem);
// D = 256 kernels run one CTA per SM with their matrices in a global workspace; these give the
// grid and the workspace bytes each kernel family needs (0 for D <= 64).
int big_grid();
size_t pair_ws_bytes(int D);
size_t xproj_ws_bytes(int D);
size_t bound_ws_bytes(int D);

// D in {4, 16, 64, 256}; arith is an Arith.
cudaError_t launch_pair(const PairArgs& a, int arith, cudaStream_t s);
// rho_0 update: two launches (chunk sums over delta, then one CTA), fixed reduction order.
cudaError_t launch_rho0(const SmallArgs& a, cudaStream_t s);
cudaError_t launch_dual12(const SmallArgs& a, cudaStream_t s);
cudaError_t launch_status(const SmallArgs& a, cudaStream_t s);

// ------------------------------------------------------------------ block DFT over delta
// The first block row is viewed as a row-major array [A][n][B] of slots (delta, or wavevector
// after the forward passes), each slot holding E = D*D/2 complex values: entry e of slot t is
// X_t[e] + i X_t[e + E] (two real block entries packed in one complex sequence).
struct FftPass {
  int A, n, B;
  int tw_mode;  // 0: none; 1: times w_twN^(dir*k*b); 2: times w_twN^(dir*k*a)  (k = output index)
  int twN;
  int w_off;    // offset of the length-n table exp(-2 pi i j / n) in the twiddle buffer
  int tw_off;   // offset of the length-twN table
  int ec[2];    // entries per CTA chosen by fft_tune (float64, float32 passes); 0: heuristic
};

struct FftPlan {
  int dim, M0, M1, N, N1, N2, E, D, npass;
  FftPass fwd[2], inv[2];
  int ntab;
  int tab_n[3], tab_off[3];
  int ntw;  // total twiddle entries
};

// Returns 0, or VE_EUNSUPPORTED / VE_EINVAL codes.
int fft_plan_build(FftPlan& p, int dim, const int M[2], int D);
cudaError_t launch_fft_tables(const FftPlan& p, double2* tw, cudaStream_t s);
// Forward: real first block row x (N*D*D) -> spectrum (returned pointer is bufA or bufB).
// fp32: the spectrum is float2 (the buffers are reinterpreted) and the passes run in float32.
cudaError_t fft_forward(const FftPlan& p, const double* x, double2* bufA, double2* bufB,
                        const double2* tw, double2** spec, bool fp32, cudaStream_t s);
// Autotuning of the passes' entries per CTA (8, 16 or 32; the result of a pass does not depend
// on it): each candidate is timed on the caller's data -- x is only read, block-row outputs go to
// bufA -- and the fastest kept in the plan.  Choices are cached per device, lattice, D and
// precision for the process, and in the file named by VE_TUNE_CACHE when that is set.
// Not to be called during stream capture.
cudaError_t fft_tune(FftPlan& p, const double* x, double2* bufA, double2* bufB, const double2* tw,
                     bool fp32, cudaStream_t s);
// Inverse: spectrum (in `spec`, which is bufA or bufB) -> real first block row x.
cudaError_t fft_inverse(const FftPlan& p, double2* spec, double2* bufA, double2* bufB, double* x,
                        const double2* tw, bool fp32, cudaStream_t s);
// List of the canonical spectrum slots (s <= slot of -k), ncanon of them, in increasing order.
cudaError_t launch_canon_list(const FftPlan& p, int* canon, cudaStream_t s);
int fft_ncanon(const FftPlan& p);
// Per-wavevector projection in place on the spectrum, scaled by 1/N; fp32 = float2 spectrum and
// float32 eigensolve.  vstore (N * 2 * D*D of float or double, or null): eigenvectors kept per
// slot; warm = 1 starts from them.
cudaError_t launch_xproj(const FftPlan& p, double2* spec, const int* canon, int arith,
                         void* vstore, int warm, cudaStream_t s,
                         unsigned long long* stats = nullptr, unsigned char* gws = nullptr,
                         const long long* iter = nullptr);
// D = 256 in float32 (float2 spectrum): the same projection with its products on the tensor
// cores (tc_project256); the eigenvectors persist in w between calls.
struct TcProjWs;
cudaError_t launch_xproj_tc(const FftPlan& p, double2* spec, const int* canon, TcProjWs& w, int warm,
                            cudaStream_t s, unsigned long long* stats = nullptr);
// lmin[slot] = smallest eigenvalue of the (unnormalised) block C_k, +inf for non-canonical slots.
cudaError_t launch_xeig(const FftPlan& p, const double2* spec, const int* canon, double* lmin,
                       cudaStream_t s, unsigned char* gws = nullptr);

// ------------------------------------------------------------------ tensor-core products
// Batched 256 x 256 x 256 products D_b = alpha x_b y_b^T + beta I on the tcgen05 tensor cores
// (ve_tcgemm.cu): x and y are split float32 matrices in the KC4 layout -- per matrix 2 planes
// (hi, lo) when real, 4 (re hi, re lo, im hi, im lo) when complex, each 256 x 256 with element
// (r, k) at ((k / 4) * 256 + r) * 4 + k % 4 -- and x_b y_b^T contracts the k index of both.
// conj_x / conj_y conjugate a complex operand.  The result goes to out_n (D, KC4, split) and/or
// out_t (D^T); every pointer 16-byte aligned.  *err is set to 1 when a wait of the kernel gave up.
struct TcGemm {
  const float* x = nullptr;
  const float* y = nullptr;
  long batch = 0;
  int cplx = 0, conj_x = 0, conj_y = 0;
  float alpha = 1.f, beta = 0.f;
  float* out_n = nullptr;
  float* out_t = nullptr;
  int* err = nullptr;
  int round = 0;     // tc_rot256: the block-Jacobi round
  int conj_out = 0;  // conjugate the result before writing it
  // "plain" outputs: out_n / out_t written as float32 planes (re; re, im when complex) in the KC4
  // layout, half the bytes of the split form; tc_rot256 always takes its x operand plain
  int plain_n = 0, plain_t = 0;
  // failure-detection test only (ve_selftest_bounded_wait): the loads are never issued, so the
  // kernel's bounded waits run out and it must report *err = 1 and return
  int withhold_loads = 0;
};
cudaError_t tc_gemm256(const TcGemm& g, cudaStream_t s);
// Block Jacobi on 256 x 256 matrices: TC_BJ_NB blocks of TC_BJ_BS indices, paired by the circle
// ordering (rr_pair(TC_BJ_NB, round, k)), TC_BJ_NB - 1 rounds a sweep.
constexpr int TC_BJ_BS = 16, TC_BJ_NB = 256 / TC_BJ_BS;
// x_b R_b for a block rotation R of round g.round, R nonzero only on each pair's 2 TC_BJ_BS square
// block.  g.y holds R compactly (split): per matrix NPL planes of 256 rows x 2 TC_BJ_BS columns in
// the KC4 layout, row 2 TC_BJ_BS j + c and column a holding R[I_j[a]][I_j[c]] for pair j's index
// list I_j (its block p, then block q); each output column block accumulates over its pair's
// indices: 2 TC_BJ_BS / 256 of the products of tc_gemm256.  g.x is
// plain (split inside the kernel: the rotations move their whole operand for 1/8 of a product's
// MMAs, so its bytes are the cost).
cudaError_t tc_rot256(const TcGemm& g, cudaStream_t s);

// Batched float32 PSD projection of 256 x 256 matrices with the products on the tensor cores
// (ve_tcproj.cu).  One workspace serves up to `cap` matrices of one kind (real or complex); V and
// Vt keep the eigenvectors between calls (warm = true starts from them, false from V = I).  The
// caller writes the inputs C (split, KC4, symmetric / Hermitian) into w.C; the projections come
// back in w.Wt (split, KC4).  stats as in PairArgs.
struct TcProjWs {
  long cap = 0;
  int cplx = 0;
  float *V = nullptr, *Vt = nullptr, *C = nullptr, *T = nullptr, *V1 = nullptr, *V1t = nullptr,
        *Wt = nullptr, *M = nullptr, *Qt = nullptr;
  unsigned char* jws = nullptr;  // Jacobi staging, one slice per CTA
  int* err = nullptr;            // device word: 1 after a tensor-core kernel gave up waiting
  int bj_sweeps = 2;             // block-Jacobi sweeps per projection
  int bj_inner = 1;              // Jacobi sweeps per block sub-problem (0: to convergence)
};
size_t tc_proj_ws_bytes(long cap, int cplx);
int tc_proj_ws_init(TcProjWs& w, long cap, int cplx, void* mem, size_t bytes);
cudaError_t tc_project256(TcProjWs& w, long count, bool warm, unsigned long long* stats, cudaStream_t s);

// ------------------------------------------------------------------ bound
struct BoundArgs {
  int N, P, m, D;
  const double* X;
  const double* lam1;
  const double* hb;
  const int* hslot;
  const int* neg;       // linear index of -delta
  const double* H0;
  double* lmin_pairs;   // P
  double* lmin0;        // 1
  unsigned char* gws;   // D = 256: per-CTA staging workspace (bound_ws_bytes)
};
cudaError_t launch_bound(const BoundArgs& a, cudaStream_t s);

// ------------------------------------------------------------------ standalone projections
// Standalone batched projections; n = 256, 512 (Hermitian: 256) stage each matrix in a
// per-CTA slice of gws (proj_ws_bytes), smaller n ignore it.
cudaError_t launch_proj_sym(const double* in, double* out, int n, long count, int arith,
                            cudaStream_t s, unsigned char* gws = nullptr);
cudaError_t launch_proj_herm(const double* in, double* out, int n, long count, int arith,
                             cudaStream_t s, unsigned char* gws = nullptr);
size_t proj_ws_bytes(int n, bool herm, int arith);

}  // namespace ve
