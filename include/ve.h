/*
 * ve.h -- C ABI of the GB300 solver for the variational-embedding semidefinite relaxation of
 * Khoo & Lindsey, "Scalable semidefinite programming approach to variational embedding for
 * quantum many-body problems" (arXiv:2106.02682).
 *
 * The solver runs the translation-invariant ADMM / projected dual-gradient ascent of the
 * paper's Algorithm 6 (Sec. 3.3) on one GPU and returns a certified lower bound on the
 * ground-state energy of a periodic spin-1/2 lattice.  One sweep is:
 *   effective Hamiltonians from X (Eq. (effHam)); closed-form pair update (Eq. (rhoijUpdate));
 *   PSD projection of every pair marginal (Eq. (rhoijTildeUpdate)); one-cluster marginal
 *   update (Eq. (rhoiUpdate)); dual updates (Algorithm 4); X' = X - eps G; block DFT of X's
 *   first block row; PSD projection of every wavevector block; inverse DFT.
 *
 * Conventions shared by every entry point:
 *   - Return value: VE_OK (0), VE_NOT_CONVERGED (1) or a negative VE_E* code.  No entry point
 *     aborts or prints; ve_error_string() names a code.
 *   - Pointers documented "host" are read or written during the call only; the caller keeps
 *     ownership.  Pointers documented "device" must be CUDA device (or managed) memory on the
 *     current device, valid until the work issued on the given stream has completed.
 *   - Matrices are row-major, float64.  Complex matrices are interleaved (re, im) float64.
 *   - Cluster marginals are m x m (m = 2^L, L spins per cluster); pair marginals and X blocks
 *     are D x D, D = m^2, with the pair basis index a*m + b (cluster 0 = first tensor factor).
 *   - Cluster offsets delta are numbered row-major over the cluster lattice; pair arrays hold
 *     delta = 1 .. N-1 (N = number of clusters), X holds delta = 0 .. N-1.
 *   - Energies are per spin.
 *   - A handle is used by one host thread at a time (thread-compatible, not thread-safe).
 */
#ifndef VE_H
#define VE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VE_OK 0
#define VE_NOT_CONVERGED 1
#define VE_EINVAL (-1)       /* bad argument, shape or size                               */
#define VE_ENOMEM (-2)       /* device or host allocation failed                          */
#define VE_ECUDA (-3)        /* a CUDA call failed                                        */
#define VE_ENONFINITE (-4)   /* the iteration produced a NaN or Inf                       */
#define VE_EUNSUPPORTED (-5) /* valid but not implemented here (e.g. cluster size)        */
#define VE_ETIMEOUT (-6)     /* a bounded wait inside a kernel gave up; the result is invalid */

#define VE_PREC_FP64 0  /* every step in float64                                          */
#define VE_PREC_MIXED 1 /* float32 arithmetic in the pair pass, the block DFT and both PSD
                           projections, float64 state and reductions; ve_iterate finishes in
                           VE_PREC_DF64 arithmetic                                         */
#define VE_PREC_DF64 2  /* the pair pass and both PSD projections in double-float words (an
                           unevaluated sum of two float32 numbers: 48-bit significand, ~2^-48
                           rounding against float64's 2^-53) on the float32 pipe, everything
                           else in float64                                                    */

#define VE_MAX_BONDS 4

/* Periodic lattice: dim = 1 or 2, extent[p] spins along axis p (extent[1] ignored if dim 1). */
typedef struct {
  int dim;
  int extent[2];
} ve_lattice;

/* Rectangular cluster of extent[0] x extent[1] spins (Sec. 2.3); must tile the lattice. */
typedef struct {
  int extent[2];
} ve_cluster;

/* Translation-invariant real spin-1/2 Hamiltonian (Sec. 2.1):
 *   H = sum_s onsite(s) + sum_s sum_b bond_b(s, s + bond_offset[b]).
 * onsite: 2x2 real symmetric; bond[b]: 4x4 real symmetric acting on (s, s + offset) with s the
 * first tensor factor; the spin basis is (sigma^z = +1, sigma^z = -1). */
typedef struct {
  double onsite[4];
  int nbond;
  int bond_offset[VE_MAX_BONDS][2];
  double bond[VE_MAX_BONDS][16];
} ve_hamiltonian;

/* Algorithm parameters.  Defaults (ve_default_options) are those of Sec. 4: mu = nu = 10,
 * eps = 2, VE_PREC_FP64, check_every = 10, stream = NULL (the handle creates its own). */
typedef struct {
  double mu, nu, eps;
  int precision;   /* VE_PREC_FP64, VE_PREC_MIXED or VE_PREC_DF64 */
  int check_every; /* sweeps between residual read-backs in ve_iterate, >= 1 */
  void* stream;    /* cudaStream_t for all of the handle's work, or NULL */
} ve_options;

/* Convergence measures after the last sweep (Sec. 4): energy per spin of the closed-form pair
 * marginals with the bare Hamiltonian, feasibility error Eq. (feasErr), |energy change| between
 * the last two sweeps, residual = max(feas_err, d_energy). */
typedef struct {
  long iter;
  double energy_per_spin, feas_err, d_energy, residual;
} ve_status;

/* Certified lower bound (weak duality of Eq. (partialDual) with the Lagrangian of Eq.
 * (lagrangian)): raw_bound (whole lattice) = N lmin(K_0) + sum_delta c(delta) lmin(K_delta);
 * x_min_eig = smallest eigenvalue of the block-circulant X; x_neg_correction = N m max(0,
 * -x_min_eig); bound_per_spin = (raw_bound - x_neg_correction) / spins.  primal_per_spin is
 * the energy of the last sweep. */
typedef struct {
  double bound_per_spin, raw_bound, x_min_eig, x_neg_correction, primal_per_spin;
} ve_cert;

typedef struct ve_handle ve_handle;

/* Fill *opt with the defaults above. */
void ve_default_options(ve_options* opt);

/* Transverse-field Ising site terms, Eq. (TFI): onsite -h sigma^x, bond -J sigma^z sigma^z along
 * each lattice axis.  Returns VE_EINVAL for dim not 1 or 2 or out == NULL. */
int ve_ham_tfim(int dim, double J, double h, ve_hamiltonian* out);

/* XXZ site terms J (sigma^x sigma^x + sigma^y sigma^y + delta sigma^z sigma^z) along each axis;
 * delta = 1 is the antiferromagnetic Heisenberg model, Eq. (AFH). */
int ve_ham_xxz(int dim, double J, double delta, ve_hamiltonian* out);

/* Build the cluster blocks H_0, H_{0,delta} (Sec. 2.3, 3.3), allocate the device state and
 * initialise it as in Sec. 4 (Lambda = 0, rho_0 = I/m, rho~ = I/D, X = I).
 * Supported: L = spins per cluster in {1, 2, 3, 4} (D = 4, 16, 64, 256); clusters per axis
 * M_p >= 1 with N >= 2; 1-D lattices with N <= 64, or N <= 4096 factoring as N1*N2 with
 * N1, N2 <= 64; 2-D lattices with M_p <= 64.  With L = 4 the eigensolves stage their 256 x 256
 * matrices in a device workspace of ~3.2 MB per SM.
 * opt may be NULL (defaults).  On success *out owns all device memory until ve_destroy.
 * The first sweep of each precision times the block DFT's launch shapes on the handle's data
 * (results do not depend on the choice) and keeps the fastest; choices are cached per device,
 * lattice, D and precision for the process, and in the text file named by the environment
 * variable VE_TUNE_CACHE (read once, appended to) when it is set.
 * Errors: VE_EINVAL (bad shape, cluster does not tile the lattice, N < 2, bad options),
 * VE_EUNSUPPORTED (sizes outside the list above), VE_ENOMEM, VE_ECUDA. */
int ve_create(const ve_lattice* lattice, const ve_cluster* cluster, const ve_hamiltonian* ham,
              const ve_options* opt, ve_handle** out);

/* Run sweeps of Algorithm 6 until max_iter sweeps or, when tol > 0, until the residual is
 * <= tol at a read-back (every check_every sweeps).  In VE_PREC_MIXED the sweeps use float32
 * projections until the residual reaches tol (or stops falling: no 1 % gain over 100
 * read-backs, counted across calls), then continue in VE_PREC_DF64 arithmetic until the
 * residual is <= tol again; with tol <= 0 they stay in float32.  ve_set_state returns a handle
 * to the float32 phase.
 * Writes the last status to *out (may be NULL).  Returns VE_OK if converged (or tol <= 0 and
 * max_iter sweeps ran), VE_NOT_CONVERGED, VE_ENONFINITE, VE_EINVAL, VE_ECUDA.  Synchronous. */
int ve_iterate(ve_handle* h, long max_iter, double tol, ve_status* out);

/* Certified lower bound of the current state, all in float64 on the GPU (eigenvalues by
 * Jacobi).  Synchronous.  Errors: VE_EINVAL, VE_ECUDA. */
int ve_bound(ve_handle* h, ve_cert* out);

/* Release everything the handle owns.  NULL-safe. */
void ve_destroy(ve_handle* h);

/* Sizes of the instance: clusters N, cluster dimension m, pair dimension D (any may be NULL). */
int ve_dims(const ve_handle* h, int* N, int* m, int* D);

/* Packed state: rho_0 (m^2), rho~ (P D^2), Lambda (P D^2), Lambda1 (P m^2), Lambda2 (P m^2),
 * X (N D^2), P = N - 1, float64, each block row-major.  ve_state_size gives the byte count;
 * get/set copy through `host` (host memory, bytes must equal that size; VE_EINVAL otherwise).
 * ve_set_state clears the stored previous energy, so the next d_energy is +inf.  The
 * eigenvectors of the last projections are not part of the state; the handle keeps them as the
 * starting point of the next sweep's eigensolves (any orthogonal start converges), so a state
 * read and set back on the same handle continues bit for bit, and on a fresh handle to rounding.
 *
 * Opposite offsets delta and -delta describe the same pairs of clusters seen from either end,
 * and a sweep commutes with exchanging the two clusters of a pair.  A sweep therefore updates,
 * of each pair {delta, -delta} (delta != -delta), only the member with the smaller linear index
 * and writes the other as its swap image: rho~ and Lambda conjugated by the factor exchange,
 * Lambda1 and Lambda2 exchanged, X' transposed.  Every state the solver produces from
 * ve_create's initial state has this symmetry (X up to rounding); a state set here without it
 * takes it from those members in its first sweep.  An offset with -delta = delta is updated on
 * its own; the X step needs its X' block symmetric (the wavevector blocks Hermitian), which
 * holds when that offset's rho~, Lambda are swap-symmetric and its Lambda1 = Lambda2, as in
 * every state the solver produces. */
size_t ve_state_size(const ve_handle* h);
int ve_get_state(ve_handle* h, double* host, size_t bytes);
int ve_set_state(ve_handle* h, const double* host, size_t bytes);

/* Last status of the handle without running a sweep. */
int ve_get_status(ve_handle* h, ve_status* out);

/* Per-stage timing.  ve_profile(h, 1) clears the accumulators and makes every following sweep
 * run uncaptured with CUDA events (on the handle's stream) around each of its VE_NSTAGE stages:
 * 0 pair pass, 1 rho_0 update, 2 Lambda1/Lambda2 update, 3 status, 4 forward block DFT,
 * 5 per-wavevector projection, 6 inverse block DFT.  ve_profile(h, 0) returns to graph replay.
 * ve_profile_read writes accumulated milliseconds and kernel launches per stage (arrays of
 * VE_NSTAGE, host).  Errors: VE_EINVAL, VE_ECUDA. */
#define VE_NSTAGE 7
int ve_profile(ve_handle* h, int enable);
int ve_profile_read(ve_handle* h, double* ms, long* launches);
/* Mean Jacobi sweeps per eigensolve over the profiled sweeps: pair projections (*pair) and
 * wavevector projections (*wavevector); 0 if none ran.  Errors: VE_EINVAL, VE_ECUDA. */
int ve_profile_sweeps(ve_handle* h, double* pair, double* wavevector);
/* How many eigensolves of the profiled sweeps ended with the first-order (Daleckii-Krein)
 * reconstruction instead of a converged Jacobi sweep -- the early stop of the projections of
 * Eq. (rhoijTildeUpdate) and of Algorithm 6's per-wavevector step.  pair[0] / wavevector[0]
 * receive those counts, pair[1] / wavevector[1] the eigensolves (two longs each, host).
 * Errors: VE_EINVAL, VE_ECUDA. */
int ve_profile_first_order(ve_handle* h, long* pair, long* wavevector);

/* Name of a status code (static string). */
const char* ve_error_string(int code);

/* ---- batches of independent instances ----------------------------------------------------
 * n independent instances (any mix of lattices, cluster sizes, Hamiltonians) advanced together:
 * each sweep of the batch is one CUDA graph launch whose branches are the sweeps of the
 * instances, so small instances that would leave most of the GPU idle run concurrently.  Every
 * instance keeps its own state, convergence test and precision phase and stops when it
 * converges; its iterates are identical to those of a single handle run with the same calls.
 * opt applies to every instance (opt->stream must be NULL: each instance gets a stream).
 * ve_batch_iterate writes n statuses to `out` (host, may be NULL) and returns VE_OK when every
 * instance converged (or tol <= 0), else VE_NOT_CONVERGED / VE_ENONFINITE / VE_ECUDA.
 * ve_batch_handle gives instance i for ve_get_state / ve_set_state / ve_bound (owned by the
 * batch; do not destroy it, and do not call ve_iterate or ve_profile on it). */
typedef struct ve_batch ve_batch;
int ve_create_batch(int n, const ve_lattice* lattices, const ve_cluster* clusters,
                    const ve_hamiltonian* hams, const ve_options* opt, ve_batch** out);
int ve_batch_size(const ve_batch* b);
ve_handle* ve_batch_handle(ve_batch* b, int i);
int ve_batch_iterate(ve_batch* b, long max_iter, double tol, ve_status* out);
int ve_batch_bound(ve_batch* b, ve_cert* out);
void ve_batch_destroy(ve_batch* b);

/* Project the handle's X onto the PSD cone in place (block DFT, per-wavevector projection in
 * float64, inverse DFT -- the last three steps of Algorithm 6 without the G term).  Used after
 * ve_set_state with a predicted state: the certified bound needs X >= 0 and then holds whatever
 * the prediction was.  Synchronous.  Errors: VE_EINVAL, VE_ECUDA. */
int ve_project_state_x(ve_handle* h);

/* ---- learned warm start ------------------------------------------------------------------
 * The paper has no learned component.  This is a float32 multilayer perceptron
 *   a_0 = x, a_l = tanh(W_l a_{l-1} + b_l) (n_layers hidden layers of width n_hidden),
 *   y = W_out a_{n_layers} + b_out,
 * trained on the GPU by full-batch Adam (beta 0.9 / 0.999) on loss = mean over samples and
 * outputs of (y - t)^2 / 2, with hand-written forward, backward and update kernels.  It maps
 * model parameters to a compressed warm-start state (see paper_2106_02682_gb300/warmstart.py).
 * Parameters are stored layer by layer: W (outputs x inputs, row-major) then b; initial weights
 * are Glorot-uniform from `seed`, biases zero.  x (n x n_in), t (n x n_out), y (n x n_out) and
 * grad (num_params) are host arrays, row-major.  All calls are synchronous.
 * Errors: VE_EINVAL (sizes, NULL), VE_ENOMEM, VE_ECUDA. */
typedef struct ve_mlp ve_mlp;
int ve_mlp_create(int n_in, int n_hidden, int n_layers, int n_out, unsigned long long seed,
                  ve_mlp** out);
void ve_mlp_destroy(ve_mlp* m);
size_t ve_mlp_num_params(const ve_mlp* m);
int ve_mlp_get_params(ve_mlp* m, float* host, size_t count);
int ve_mlp_set_params(ve_mlp* m, const float* host, size_t count);  /* also resets Adam */
int ve_mlp_loss_grad(ve_mlp* m, const float* x, const float* t, int n, float* loss, float* grad);
int ve_mlp_train(ve_mlp* m, const float* x, const float* t, int n, int steps, float lr,
                 float* loss_out);
int ve_mlp_predict(ve_mlp* m, const float* x, int n, float* y);

/* ---- batched building blocks on caller device memory ------------------------------------ */

/* Pi_{>=0} (Sec. 3, the Frobenius-nearest PSD matrix, Eq. (rhoijTildeUpdate)) of `count` real
 * symmetric n x n matrices: in, out = device pointers to count*n*n float64 (in == out allowed).
 * n in {2, 4, 8, 16, 64}; precision VE_PREC_FP64, VE_PREC_MIXED (float32 eigensolve) or
 * VE_PREC_DF64 (double-float eigensolve).  The
 * input is symmetrised as (A + A^T)/2.  Asynchronous on `stream` (cudaStream_t or NULL).
 * Errors: VE_EINVAL (n, count < 0, precision), VE_ECUDA (launch failure). */
int ve_project_psd_sym(const double* in, double* out, int n, long count, int precision,
                       void* stream);

/* Same for complex Hermitian n x n matrices (Algorithm 6, the per-wavevector projection),
 * interleaved complex: count*n*n*2 float64 each; n in {4, 16, 64}. */
int ve_project_psd_herm(const double* in, double* out, int n, long count, int precision,
                        void* stream);

/* The same projections for larger matrices: real symmetric n in {256, 512}, complex Hermitian
 * n = 256 (the per-wavevector blocks of 2 x 2 clusters, Algorithm 6).  Each matrix is staged
 * in a per-SM slice of `workspace` (device memory owned by the caller, 256-byte aligned, at
 * least ve_project_psd_large_workspace_size(n, hermitian, precision) bytes -- that size is
 * for the current device); one CTA per SM runs a cyclic Jacobi eigensolve from V = I.
 * Layout as above (in == out allowed).  Calls sharing a workspace must not overlap on the GPU.
 * ve_project_psd_large_workspace_size returns 0 for an unsupported n or precision.
 * Errors: VE_EINVAL (n, count < 0, precision, workspace missing, small or misaligned),
 * VE_ECUDA. */
size_t ve_project_psd_large_workspace_size(int n, int hermitian, int precision);
int ve_project_psd_sym_large(const double* in, double* out, int n, long count, int precision,
                             void* workspace, size_t workspace_bytes, void* stream);
int ve_project_psd_herm_large(const double* in, double* out, int n, long count, int precision,
                              void* workspace, size_t workspace_bytes, void* stream);

/* The global X step of Algorithm 6 on a first block row, without the G term: given X'_{0,delta}
 * (N blocks D x D, device, N = M0*M1 clusters of a dim-1 or dim-2 cluster lattice with M[p]
 * clusters per axis), write X_{0,delta} = (1/N) sum_k e^{+i 2 pi delta.k/M} Pi_{>=0}(C_k),
 * C_k = sum_delta e^{-i 2 pi delta.k/M} X'_{0,delta}.  The input must satisfy
 * X'_{0,-delta} = X'_{0,delta}^T (then every C_k is Hermitian); it may alias the output.
 * workspace: device buffer of at least ve_circulant_workspace_size(...) bytes, 256-byte
 * aligned.  D in {4, 16, 64}.  Asynchronous on `stream`.  Errors: VE_EINVAL (sizes, NULL,
 * small workspace), VE_EUNSUPPORTED (lattice not factorable as for ve_create, or D = 256,
 * which only a handle serves), VE_ECUDA.  ve_circulant_workspace_size returns 0 for unsupported
 * shapes. */
size_t ve_circulant_workspace_size(int dim, const int M[2], int D);
int ve_circulant_project(const double* x_in, double* x_out, int dim, const int M[2], int D,
                         int precision, void* workspace, size_t workspace_bytes, void* stream);

/* ---- X step without allocation ----------------------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that may not allocate
 * device memory themselves: a plugin whose host framework owns every device allocation and
 * hands it only input and output buffers, or a latency-critical loop in which cudaMalloc's
 * implicit synchronisation and unpredictable latency are not allowed.
 *
 * ve_circulant_project_noalloc computes exactly what ve_circulant_project computes (same
 * arguments, same kernels) but takes its scratch from a fixed array of
 * VE_NOALLOC_SCRATCH_BYTES bytes compiled into this library (a file-scope __device__ array;
 * every GPU that loads the library holds it until the process exits).  It calls no cudaMalloc,
 * cudaFree or allocating library routine.  Limit: the call needs
 * ve_circulant_workspace_size(dim, M, D) <= VE_NOALLOC_SCRATCH_BYTES, which admits every
 * first block row with N * D * D <= 2^20 float64 entries (e.g. 4096 clusters with D = 16);
 * larger requests return VE_EINVAL before any GPU work.
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress), so the address stays right after cudaDeviceReset.  The first call
 *     on a device may load the library's device code there: make it before any stream capture.
 *   - All calls on a device share the one array and leave their data in it.  Calls whose GPU
 *     work overlaps (other streams, or other host threads, without ordering between them) race
 *     on it and produce wrong results; order them on one stream or with events.
 * Errors: VE_EINVAL (NULL pointers, bad sizes, request above the limit), VE_EUNSUPPORTED (as
 * for ve_circulant_project), VE_ECUDA. */
#define VE_NOALLOC_SCRATCH_BYTES ((size_t)(16u << 20) + (size_t)(256u << 10))
int ve_circulant_project_noalloc(const double* x_in, double* x_out, int dim, const int M[2], int D,
                                 int precision, void* stream);

/* ---- failure detection (the paper has no counterpart) ----------------------------------
 * Every wait inside the tensor-core kernels (mbarrier phases of the TMA ring and of the tensor-
 * memory accumulators) gives up after ~2 s of clock, sets an error word, drains the copies and
 * products it issued, frees its tensor memory and returns; ve_iterate then reports VE_ETIMEOUT.
 * ve_selftest_bounded_wait exercises that path on the current device without a fault: it runs
 * one 256 x 256 tensor-core product whose loads are deliberately never issued, so its waits run
 * out, then the same product normally.  Returns VE_OK when the first reported its timeout and
 * the second ran clean on the same context; *seconds receives the first call's device time.
 * Errors: VE_EINVAL, VE_ENOMEM, VE_ECUDA, VE_ETIMEOUT (a timeout went unreported, or a clean
 * product reported one).  Takes ~2 s. */
int ve_selftest_bounded_wait(double* seconds);

/* ---- general Hamiltonians: Algorithm 5 (Sec. 3.2, "practical scheme") -------------------
 * No translation invariance: random fields, inhomogeneous or long-range couplings.  Every
 * cluster i has its own H_i and rho_i, every pair i < j its own H_ij, rho~_ij, Lambda_ij,
 * Lambda1_ij, Lambda2_ij, and X is one dense (N D) x (N D) matrix whose projection X <-
 * Pi_{>=0}(X - eps G) runs as one eigensolve spread over the whole GPU (cyclic Jacobi in the
 * circle ordering, one launch per round, warm-started from the previous sweep's eigenvectors).
 * The X step takes the ascent sign X - eps G, as ve_create's solver does.
 *
 * The Hamiltonian is a list of terms on nspins spins:
 *   H = sum_s onsite[s] + sum_b B_b acting on spins (bond_sites[2b], bond_sites[2b+1]),
 * onsite[s]: 2x2 real symmetric (row-major, 4 doubles each; onsite NULL = none); B_b: 4x4 real
 * symmetric (16 doubles each) with the first listed spin as its first tensor factor; spin basis
 * (sigma^z = +1, sigma^z = -1).  Clusters are runs of cluster_spins consecutive spins: cluster c
 * holds spins c L .. c L + L - 1 (L = cluster_spins, N = nspins / L clusters, m = 2^L, D = m^2).
 * A term inside one cluster belongs to its H_i, a term between clusters i < j to H_ij (cluster i
 * the first factor).  Pairs are numbered i < j in lexicographic order, K = N (N - 1) / 2. */
typedef struct {
  int nspins;
  const double* onsite;
  int nbond;
  const int* bond_sites;
  const double* bond_ops;
} ve_terms;

/* Spinless fermions (the paper's fermionic section, Eq. (spinlessFerm) and its long-range form):
 *   H = sum_k hop_t[k] (a_i^dagger a_j + a_j^dagger a_i), (i, j) = hop_sites[2k], hop_sites[2k+1]
 *     + sum_k pair_v[k] (n_i - 1/2)(n_j - 1/2),         (i, j) = pair_sites[2k], pair_sites[2k+1]
 * on nsites sites (i != j in every term).  Clusters are runs of cluster_sites consecutive sites,
 * as for spins.  ve_general_create_fermions builds the blocks of Eq. (sdpFerm): each cluster's
 * terms under the Jordan-Wigner transformation in the cluster's site order, each pair's terms
 * under the one in the pair's order (the first cluster's sites first); a site's basis is
 * (empty, occupied), a^dagger acting as [[0, 0], [1, 0]] after a sigma^z string over the earlier
 * sites.  The global matrix then carries parity signs on its off-diagonal blocks: with the
 * complete collection of matrix units, entry (a, b), (c, d) of G_ij is multiplied by
 * (-1)^(p(a) (p(c) + p(d))), p the parity of a cluster state's occupation bits (an operator of
 * the second cluster that changes the parity carries the first cluster's parity string), and
 * H'_ij takes the adjoint of that signed map.  Everything else is ve_general's solver. */
typedef struct {
  int nsites;
  int nhop;
  const int* hop_sites;
  const double* hop_t;
  int npair;
  const int* pair_sites;
  const double* pair_v;
} ve_fermion_terms;

typedef struct ve_general ve_general;

/* Build the cluster blocks (copied; the caller keeps the terms) and the initial state of Sec. 4
 * (rho_i = I/m, rho~_ij = I/D, multipliers 0, X = I).  Supported: L in {1, 2, 3}, N >= 2,
 * N D <= 1024, precision VE_PREC_FP64.  opt may be NULL (defaults of ve_default_options).
 * Errors: VE_EINVAL (sizes, spins out of range, a bond on one spin, bad options),
 * VE_EUNSUPPORTED (L > 3, N D > 1024, other precisions), VE_ENOMEM, VE_ECUDA. */
int ve_general_create(const ve_terms* terms, int cluster_spins, const ve_options* opt,
                      ve_general** out);
/* The same for spinless fermions (sizes and errors as ve_general_create, with sites for spins);
 * every other ve_general_* call applies to the handle unchanged. */
int ve_general_create_fermions(const ve_fermion_terms* terms, int cluster_sites,
                               const ve_options* opt, ve_general** out);
/* The cluster blocks those two calls build, written to host memory without touching a GPU:
 * Hi (N m^2) and Hij (K D^2, pairs i < j in lexicographic order), row-major.  Errors as for
 * the create calls (the options are not checked). */
int ve_spin_blocks(const ve_terms* terms, int cluster_spins, double* Hi, double* Hij);
int ve_fermion_blocks(const ve_fermion_terms* terms, int cluster_sites, double* Hi, double* Hij);
void ve_general_destroy(ve_general* h);  /* NULL-safe */
int ve_general_dims(const ve_general* h, int* N, int* m, int* D, long* K);

/* Sweeps of Algorithm 5 until max_iter sweeps or, when tol > 0, until the residual is <= tol
 * at a read-back (every check_every sweeps).  Convergence measures: energy per spin
 * (sum_i Tr[H_i rho_i] + sum_{i<j} Tr[H_ij rho_ij]) / nspins with the closed-form pair
 * marginals, Eq. (feasErr) as sqrt(sum_{i<j} (|A1 rho_ij - rho_i|^2 + |A2 rho_ij - rho_j|^2 +
 * |rho_ij - rho~_ij|^2) / K), |energy change|, residual = max of the last two.  Synchronous
 * (the X step's eigensolve reads its stopping test on the host once per Jacobi sweep).  The X
 * step starts from the previous sweep's eigenvectors (from V = I on the first sweep and every
 * 256th), and ends either by the exact stopping rule or, once A = V^T Y V is nearly diagonal,
 * with the first-order reconstruction of VE_DENSE_FIRST_ORDER (below), equally accurate.
 * Returns as ve_iterate. */
int ve_general_iterate(ve_general* h, long max_iter, double tol, ve_status* out);
int ve_general_get_status(ve_general* h, ve_status* out);

/* Certified lower bound of the current state (weak duality with the ADMM's own multipliers):
 * raw_bound = sum_i lmin(K_i) + sum_{i<j} lmin(K_ij), K_ij = H'_ij + A1^* Lambda1_ij +
 * A2^* Lambda2_ij, K_i = H'_i - sum_{j>i} Lambda1_ij - sum_{j<i} Lambda2_ji; x_min_eig =
 * lmin(X); x_neg_correction = N m max(0, -x_min_eig); bound_per_spin = (raw_bound -
 * x_neg_correction) / nspins.  All in float64 on the GPU.  Synchronous. */
int ve_general_bound(ve_general* h, ve_cert* out);

/* Packed state: rho_i (N m^2), rho~ (K D^2), Lambda (K D^2), Lambda1 (K m^2), Lambda2 (K m^2),
 * X (N D x N D), float64, each block row-major; bytes must equal ve_general_state_size.
 * ve_general_set_state clears the stored previous energy.  Eigenvectors of the last
 * projections stay with the handle as the next eigensolves' start. */
size_t ve_general_state_size(const ve_general* h);
int ve_general_get_state(ve_general* h, double* host, size_t bytes);
int ve_general_set_state(ve_general* h, const double* host, size_t bytes);

/* Per-stage timing with CUDA events around every following sweep: 0 pair pass, 1 cluster
 * marginals + Lambda1/Lambda2 + status, 2 dense eigensolve of the X step (W = Y V, Jacobi
 * sweeps, Rayleigh quotients), 3 reconstruction X = V diag(max(lambda, 0)) V^T.
 * ve_general_profile(h, 1) clears the accumulators; profile_read gives milliseconds and kernel
 * launches per stage (arrays of VE_GENERAL_NSTAGE) and the mean Jacobi sweeps per X step. */
#define VE_GENERAL_NSTAGE 4
int ve_general_profile(ve_general* h, int enable);
int ve_general_profile_read(ve_general* h, double* ms, long* launches, double* jacobi_sweeps);
/* Device time of the profiled X-step Jacobi sweeps alone (CUDA events around each sweep's graph
 * of n - 1 round launches and its convergence test), the round launches they held, and the X
 * steps that ended with the first-order reconstruction (VE_DENSE_FIRST_ORDER below). */
int ve_general_profile_rounds(ve_general* h, double* ms, long* rounds, long* first_order);

/* Pi_{>=0} of ONE real symmetric n x n matrix (device, row-major; used as (A + A^T)/2) by the
 * whole-GPU eigensolver of the general solver's X step.  n even, 2 <= n <= 1024.  out may alias
 * in.  workspace: device memory of ve_project_psd_dense_workspace_size(n) bytes (0 for an
 * unsupported n), 256-byte aligned, owned by the caller; it keeps the eigenvectors.
 * flags: VE_DENSE_WARM starts from the eigenvectors left by the previous call on the same
 * workspace and n (else from V = I).  VE_DENSE_FIRST_ORDER lets the sweeps stop early: once a
 * sweep's rotations were small, A = V^T Y V is formed by one GEMM, and when its off-diagonal part
 * E satisfies ||E||_F^4 <= (n u)^2 ||A||_F^2 d^2 and ||E||_F <= d/4 (d = distance of diag(A) from
 * zero, u = 2^-53) the result is V (f(Lambda) + L o E) V^T, f = max(., 0), L the divided
 * differences of f (Daleckii-Krein): as accurate as running the sweeps to the exact rule (the
 * general solver's X step always does this).  Every Jacobi round is one launch over n/2 CTAs;
 * the n - 1 rounds of a sweep are one CUDA graph.  *sweeps (may be NULL) receives the Jacobi
 * sweeps taken, plus 1000 if the first-order reconstruction was used.  Synchronises `stream`
 * (once per Jacobi sweep).  Each call captures and instantiates the graph of a sweep's n - 1
 * round launches anew (milliseconds for n = 512); a ve_general handle keeps its graph.
 * Errors: VE_EINVAL (NULL, n, workspace, flags), VE_ECUDA. */
#define VE_DENSE_WARM 1
#define VE_DENSE_FIRST_ORDER 2
size_t ve_project_psd_dense_workspace_size(int n);
int ve_project_psd_dense(const double* in, double* out, int n, int flags, void* workspace,
                         size_t workspace_bytes, void* stream, int* sweeps);

#ifdef __cplusplus
}
#endif

#endif /* VE_H */
