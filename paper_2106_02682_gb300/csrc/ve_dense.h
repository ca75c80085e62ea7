// ve_dense.h -- the whole-GPU dense symmetric eigensolver of ve_dense.cu (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace ve {

constexpr int DENSE_MAX_N = 1024;  // a round CTA holds 8 entries of each of its 4 columns a thread

struct DenseCtl {
  double nrm2;   // ||Y||_F^2
  double off2;   // 2 sum a_pq^2 over the last sweep's rotations
  double lmin;   // smallest lambda_i (dense_lmin)
  int converged; // the last sweep met the stopping rule
  int sweeps;    // sweeps of the current eigensolve
  int dk;        // explicit check: 0 go on, 1 converged, 2 first-order reconstruction suffices
  int pad;
};

// Device workspace of one n x n eigensolve (carved from caller memory by dense_ws_init); Vt
// survives between calls and is the warm start.
struct DenseWs {
  int n = 0;
  double* Vt = nullptr;     // n x n: row i = eigenvector estimate v_i
  double* Wt = nullptr;     // n x n: row i = w_i = Y v_i
  double* lam = nullptr;    // n: lambda_i = v_i.w_i after dense_eig
  double* slot = nullptr;   // n/2: per-CTA sum of a_pq^2 over a sweep
  double* Bt = nullptr;     // n x n: A = V^T Y V formed explicitly for the early-stop check
  DenseCtl* ctl = nullptr;  // device
  DenseCtl* hctl = nullptr; // pinned host copy (allocated on first use)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool allow_dk = false;    // take the first-order (Daleckii-Krein) early stop
  int dk_mode = 0;          // how the last eigensolve stopped (DenseCtl::dk)
  long dk_stops = 0;        // eigensolves ended by the explicit check
  int last_sweeps = 0;
  long total_sweeps = 0;
  long launches = 0;        // kernels launched (graph rounds counted one by one)
  // profiling: CUDA events around every sweep graph (created on first use when prof is set)
  bool prof = false;
  cudaEvent_t g0 = nullptr, g1 = nullptr;
  double graph_ms = 0.0;    // device time of the profiled sweep graphs
  long graph_rounds = 0;    // round launches in them
};

enum { DENSE_COLD = 0, DENSE_WARM = 1 };

// Bytes of the workspace for n (even, 2 <= n <= DENSE_MAX_N), else 0.
size_t dense_ws_bytes(int n);
// Carve `mem` (256-byte aligned, >= dense_ws_bytes(n)) into w; 0 or -1.
int dense_ws_init(DenseWs& w, int n, void* mem, size_t bytes);
// Free the graph and the pinned block (not the workspace memory).
void dense_ws_release(DenseWs& w);
// Eigen-decompose (Y + Y^T)/2 (device, n x n row-major): Vt, lam.  mode DENSE_COLD starts from
// V = I, DENSE_WARM from the Vt left by the previous call.  Synchronises `s` once per sweep (the
// stopping test is read on the host).  Not to be called during stream capture.
cudaError_t dense_eig(DenseWs& w, const double* Y, int mode, cudaStream_t s);
// X = V diag(max(lambda, 0)) V^T after dense_eig, or V (f(Lambda) + L o E) V^T when the
// eigensolve took the first-order stop (X may alias the Y given to dense_eig).
cudaError_t dense_reconstruct(DenseWs& w, double* X, cudaStream_t s);
// ctl->lmin = min_i lambda_i after dense_eig.
cudaError_t dense_lmin(DenseWs& w, cudaStream_t s);
// ctl->lmin = min_i a_ii - ||offdiag(A)||_F for A = V^T Y V formed from Vt and Wt after
// dense_eig: a lower bound on lmin(Y) by Weyl's inequality (one GEMM into Bt).
cudaError_t dense_lmin_certified(DenseWs& w, cudaStream_t s);

}  // namespace ve
