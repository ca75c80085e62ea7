// ve_api.cu -- host side of the C ABI declared in include/ve.h: cluster-model construction,
// device state, sweep orchestration (CUDA graphs), certified bound assembly, and the
// standalone batched entry points.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <stdint.h>
#include <string.h>

#include <map>
#include <vector>

#include "../../include/ve.h"
#include "ve_internal.h"

using namespace ve;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Embed a one-site operator h (2x2) on spin i / a two-site operator B (4x4) on spins (i, j) --
// B's first factor on spin i -- into the 2^K-dimensional space of K spins (spin 0 = first
// Kronecker factor).  Accumulates into out (row-major 2^K x 2^K).
void embed1(const double* h, int i, int K, double* out) {
  const int dim = 1 << K, sh = K - 1 - i;
  for (int col = 0; col < dim; ++col) {
    const int sc = (col >> sh) & 1;
    for (int sr = 0; sr < 2; ++sr) {
      const double amp = h[sr * 2 + sc];
      if (amp == 0.0) continue;
      const int row = (col & ~(1 << sh)) | (sr << sh);
      out[(size_t)row * dim + col] += amp;
    }
  }
}

void embed2(const double* B, int i, int j, int K, double* out) {
  const int dim = 1 << K, si = K - 1 - i, sj = K - 1 - j;
  for (int col = 0; col < dim; ++col) {
    const int sc = (((col >> si) & 1) << 1) | ((col >> sj) & 1);
    for (int sr = 0; sr < 4; ++sr) {
      const double amp = B[sr * 4 + sc];
      if (amp == 0.0) continue;
      int row = col & ~(1 << si) & ~(1 << sj);
      row |= ((sr >> 1) & 1) << si;
      row |= (sr & 1) << sj;
      out[(size_t)row * dim + col] += amp;
    }
  }
}

struct Model {
  int dim, e0, e1, c0, c1, M0, M1, N, L, m, D;
  std::vector<double> H0;                       // m*m
  std::map<int, std::vector<double>> pair;      // linear delta -> D*D
  std::vector<int> neg;                         // N
  std::vector<long long> count;                 // N, c(delta)
};

// Cluster blocks of a translation-invariant lattice (Sec. 2.3 / 3.3 of the paper): every term
// starting on a spin of cluster 0 is placed in H_0 (both ends in cluster 0) or in the pair
// block of the cluster it reaches, and its translate -- the same term seen from the other
// cluster -- in the pair block of the opposite offset with the factors swapped.
int build_model(const ve_lattice* lat, const ve_cluster* clu, const ve_hamiltonian* ham, Model& md) {
  if (!lat || !clu || !ham) return VE_EINVAL;
  md.dim = lat->dim;
  if (md.dim != 1 && md.dim != 2) return VE_EINVAL;
  md.e0 = lat->extent[0];
  md.e1 = md.dim == 2 ? lat->extent[1] : 1;
  md.c0 = clu->extent[0];
  md.c1 = md.dim == 2 ? clu->extent[1] : 1;
  if (md.e0 < 1 || md.e1 < 1 || md.c0 < 1 || md.c1 < 1) return VE_EINVAL;
  if (md.e0 % md.c0 || md.e1 % md.c1) return VE_EINVAL;
  md.M0 = md.e0 / md.c0;
  md.M1 = md.e1 / md.c1;
  md.N = md.M0 * md.M1;
  md.L = md.c0 * md.c1;
  if (md.N < 2) return VE_EINVAL;
  if (md.L < 1 || md.L > 4) return VE_EUNSUPPORTED;
  if (ham->nbond < 0 || ham->nbond > VE_MAX_BONDS) return VE_EINVAL;
  md.m = 1 << md.L;
  md.D = md.m * md.m;
  const int L = md.L, D = md.D;
  md.H0.assign((size_t)md.m * md.m, 0.0);
  md.pair.clear();
  auto lin = [&](int X, int Y) { return X * md.M1 + Y; };
  auto negl = [&](int dl) {
    const int X = dl / md.M1, Y = dl % md.M1;
    return lin((md.M0 - X) % md.M0, (md.M1 - Y) % md.M1);
  };
  for (int x = 0; x < md.c0; ++x) {
    for (int y = 0; y < md.c1; ++y) {
      const int u = x * md.c1 + y;
      embed1(ham->onsite, u, L, md.H0.data());
      for (int b = 0; b < ham->nbond; ++b) {
        const int ox = ham->bond_offset[b][0], oy = md.dim == 2 ? ham->bond_offset[b][1] : 0;
        const int tx = ((x + ox) % md.e0 + md.e0) % md.e0;
        const int ty = ((y + oy) % md.e1 + md.e1) % md.e1;
        const int tX = tx / md.c0, tY = ty / md.c1;
        const int ut = (tx % md.c0) * md.c1 + (ty % md.c1);
        const double* B = ham->bond[b];
        if (tX == 0 && tY == 0) {
          if (ut == u) return VE_EINVAL;  // a bond from a spin to itself
          embed2(B, u, ut, L, md.H0.data());
        } else {
          const int dl = lin(tX, tY), nd = negl(dl);
          auto& blk = md.pair[dl];
          if (blk.empty()) blk.assign((size_t)D * D, 0.0);
          embed2(B, u, L + ut, 2 * L, blk.data());
          auto& nblk = md.pair[nd];
          if (nblk.empty()) nblk.assign((size_t)D * D, 0.0);
          embed2(B, L + u, ut, 2 * L, nblk.data());
        }
      }
    }
  }
  md.neg.resize(md.N);
  for (int dl = 0; dl < md.N; ++dl) md.neg[dl] = negl(dl);
  // c(delta) = #{a : l(a) < l(a + delta)}, l = row-major linear index
  md.count.assign(md.N, 0);
  for (int dl = 1; dl < md.N; ++dl) {
    const int dX = dl / md.M1, dY = dl % md.M1;
    long long c = 0;
    for (int a = 0; a < md.N; ++a) {
      const int aX = a / md.M1, aY = a % md.M1;
      if (lin((aX + dX) % md.M0, (aY + dY) % md.M1) > a) ++c;
    }
    md.count[dl] = c;
  }
  return VE_OK;
}

// True when H_{0,-delta} = S H_{0,delta} S for every offset, S the exchange of the two
// clusters' factors.  build_model places every bond in both blocks this way, so this holds up
// to the order in which bond terms were added; it is what lets a sweep update one member of
// each pair {delta, -delta} and write the other as its swap image.
bool model_swap_symmetric(const Model& md) {
  const int m = md.m, D = md.D;
  double scale = 0.0;
  for (const auto& kv : md.pair)
    for (double x : kv.second) scale = fmax(scale, fabs(x));
  for (const auto& kv : md.pair) {
    const auto it = md.pair.find(md.neg[kv.first]);
    for (int e = 0; e < D * D; ++e) {
      const int i = e / D, j = e % D;
      const int pa = i / m, pb = i % m, pc = j / m, pd = j % m;
      const double img = it == md.pair.end() ? 0.0 : it->second[(size_t)(pb * m + pa) * D + (pd * m + pc)];
      if (fabs(kv.second[e] - img) > 1e-13 * (1.0 + scale)) return false;
    }
  }
  return true;
}

}  // namespace

struct ve_handle {
  Model md;
  ve_options opt;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  FftPlan plan;
  int P = 0;
  // device memory
  void* dev = nullptr;  // one allocation, carved below
  size_t state_bytes = 0;
  double *state = nullptr, *rho0 = nullptr, *rt = nullptr, *lam = nullptr, *lam1 = nullptr,
         *lam2 = nullptr, *X = nullptr;
  double* rho0_partial = nullptr;
  double *a1r = nullptr, *a2r = nullptr, *part = nullptr, *part2 = nullptr, *hb = nullptr,
         *H0 = nullptr, *lmin_pairs = nullptr, *lmin_k = nullptr, *lmin0 = nullptr;
  int *hslot = nullptr, *neg = nullptr, *canon = nullptr;
  int ncanon = 0;
  // pair offsets tied to their opposite (k_pair, k_dual12): Pc work items
  int Pc = 0;
  int *pidx = nullptr, *pmir = nullptr, *ptie = nullptr;
  double2 *specA = nullptr, *specB = nullptr, *tw = nullptr;
  // eigenvectors of the last projections, per arithmetic (an Arith: float64, float32, df64)
  void* vpair[3] = {nullptr, nullptr, nullptr};
  void* vk[3] = {nullptr, nullptr, nullptr};
  bool vvalid[3] = {false, false, false};
  DevStatus* dst = nullptr;
  DevStatus* hst = nullptr;  // pinned
  cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
  cudaGraph_t graph[3] = {nullptr, nullptr, nullptr};
  bool fp64_phase = false;  // MIXED: switched to the double-float refinement phase
  bool fft_tuned[2] = {false, false};  // DFT passes autotuned (float64, float32 spectrum)
  double mx_best = INFINITY;  // MIXED float32 phase: best residual and read-backs without a
  int mx_stall = 0;           // 1 % gain, kept across ve_iterate calls
  // per-stage profiling
  bool prof = false;
  cudaEvent_t ev[VE_NSTAGE + 1] = {};
  double prof_ms[VE_NSTAGE] = {};
  // device: pair sweeps, pair matrices, pair first-order stops, then the same for wavevectors
  unsigned long long* jstats = nullptr;
  unsigned char* gws = nullptr;          // D = 256: staging workspace of the eigensolver kernels
  // D = 256 in mixed precision: the float32 per-wavevector projections with their products on
  // the tensor cores (ve_tcproj.cu); a separate allocation, made only for such handles
  void* tcmem = nullptr;
  TcProjWs tcx;         // the wavevector projections (complex, ncanon matrices)
  TcProjWs tcp;         // the pair projections (real, Pc matrices)
  float* rbuf = nullptr;  // rho of the pair pass, Pc * D * D floats
  long prof_launch[VE_NSTAGE] = {};
  int stage_launches[VE_NSTAGE] = {};
};

namespace {

#define VE_CU(call)                       \
  do {                                    \
    cudaError_t _e = (call);              \
    if (_e != cudaSuccess) return VE_ECUDA; \
  } while (0)

PairArgs pair_args(ve_handle* h) {
  PairArgs a;
  a.iter = &h->dst->iter;
  a.N = h->md.N;
  a.P = h->P;
  a.m = h->md.m;
  a.D = h->md.D;
  a.mu = h->opt.mu;
  a.nu = h->opt.nu;
  a.eps = h->opt.eps;
  a.rho0 = h->rho0;
  a.rt = h->rt;
  a.lam = h->lam;
  a.lam1 = h->lam1;
  a.lam2 = h->lam2;
  a.X = h->X;
  a.hb = h->hb;
  a.hslot = h->hslot;
  a.a1r = h->a1r;
  a.a2r = h->a2r;
  a.part = h->part;
  a.vstore = nullptr;
  a.warm = 0;
  a.Pc = h->Pc;
  a.pidx = h->pidx;
  a.pmir = h->pmir;
  return a;
}

SmallArgs small_args(ve_handle* h) {
  SmallArgs a;
  a.N = h->md.N;
  a.P = h->P;
  a.m = h->md.m;
  a.D = h->md.D;
  a.L = h->md.L;
  a.mu = h->opt.mu;
  a.nu = h->opt.nu;
  a.eps = h->opt.eps;
  a.rho0 = h->rho0;
  a.lam1 = h->lam1;
  a.lam2 = h->lam2;
  a.X = h->X;
  a.H0 = h->H0;
  a.a1r = h->a1r;
  a.a2r = h->a2r;
  a.part = h->part;
  a.part2 = h->part2;
  a.st = h->dst;
  a.rho0_partial = h->rho0_partial;
  a.ptie = h->ptie;
  return a;
}

// One sweep of Algorithm 6, all on h->stream (with stage events when profiling).
cudaError_t issue_sweep(ve_handle* h, int arith, bool warm) {
  cudaStream_t s = h->stream;
  const int v = arith;
  const bool fp32 = arith == ARITH_FP32;
  PairArgs pa = pair_args(h);
  pa.vstore = h->vpair[v];
  pa.warm = warm ? 1 : 0;
  pa.stats = h->prof ? h->jstats : nullptr;
  pa.gws = h->gws;
  if (fp32 && h->tcmem) {
    pa.tcw = &h->tcp;
    pa.rbuf = h->rbuf;
  }
  const SmallArgs sa = small_args(h);
  cudaError_t e;
  if (!warm && !h->fft_tuned[fp32 ? 1 : 0]) {
    // a cold sweep runs uncaptured: time the DFT passes' launch shapes once (fft_tune)
    if ((e = fft_tune(h->plan, h->X, h->specA, h->specB, h->tw, fp32, s)) != cudaSuccess) return e;
    h->fft_tuned[fp32 ? 1 : 0] = true;
  }
  auto mark = [&](int i) { return h->prof ? cudaEventRecord(h->ev[i], s) : cudaSuccess; };
  if ((e = mark(0)) != cudaSuccess) return e;
  if ((e = launch_pair(pa, arith, s)) != cudaSuccess) return e;
  if ((e = mark(1)) != cudaSuccess) return e;
  if ((e = launch_rho0(sa, s)) != cudaSuccess) return e;
  if ((e = mark(2)) != cudaSuccess) return e;
  if ((e = launch_dual12(sa, s)) != cudaSuccess) return e;
  if ((e = mark(3)) != cudaSuccess) return e;
  if ((e = launch_status(sa, s)) != cudaSuccess) return e;
  if ((e = mark(4)) != cudaSuccess) return e;
  double2* spec = nullptr;
  if ((e = fft_forward(h->plan, h->X, h->specA, h->specB, h->tw, &spec, fp32, s)) != cudaSuccess)
    return e;
  if ((e = mark(5)) != cudaSuccess) return e;
  if (fp32 && h->tcmem) {
    if ((e = launch_xproj_tc(h->plan, spec, h->canon, h->tcx, warm ? 1 : 0, s,
                             h->prof ? h->jstats + 3 : nullptr)) != cudaSuccess)
      return e;
  } else if ((e = launch_xproj(h->plan, spec, h->canon, arith, h->vk[v], warm ? 1 : 0, s,
                              h->prof ? h->jstats + 3 : nullptr, h->gws, &h->dst->iter)) != cudaSuccess) {
    return e;
  }
  if ((e = mark(6)) != cudaSuccess) return e;
  if ((e = fft_inverse(h->plan, spec, h->specA, h->specB, h->X, h->tw, fp32, s)) != cudaSuccess)
    return e;
  return mark(7);
}

// Add the stage times of the last profiled sweep (its events have completed).
int accumulate_profile(ve_handle* h) {
  for (int i = 0; i < VE_NSTAGE; ++i) {
    float ms = 0.f;
    VE_CU(cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]));
    h->prof_ms[i] += ms;
    h->prof_launch[i] += h->stage_launches[i];
  }
  return VE_OK;
}

// Run `count` sweeps.  The first sweep of a precision on a handle runs directly and cold
// (Jacobi from V = I; it also sets kernel attributes outside any capture); the others replay a
// captured one-sweep graph that starts every Jacobi from the eigenvectors stored by the
// previous sweep of that precision (kept across ve_set_state).
int read_status(ve_handle* h, ve_status* out);

int run_sweeps(ve_handle* h, long count, int arith) {
  const int v = arith;
  if (count <= 0) return VE_OK;
  if (h->prof) {
    for (long i = 0; i < count; ++i) {
      VE_CU(issue_sweep(h, arith, h->vvalid[v]));
      h->vvalid[v] = true;
      VE_CU(cudaStreamSynchronize(h->stream));
      const int r = accumulate_profile(h);
      if (r != VE_OK) return r;
    }
    return VE_OK;
  }
  if (!h->vvalid[v]) {
    VE_CU(issue_sweep(h, arith, false));
    h->vvalid[v] = true;
    --count;
  }
  if (count <= 0) return VE_OK;
  if (!h->exec[v]) {
    VE_CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = issue_sweep(h, arith, true);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return VE_ECUDA;
    }
    h->graph[v] = g;
    VE_CU(cudaGraphInstantiate(&h->exec[v], g, 0));
  }
  for (long i = 0; i < count; ++i) VE_CU(cudaGraphLaunch(h->exec[v], h->stream));
  return VE_OK;
}

int read_status(ve_handle* h, ve_status* out) {
  VE_CU(cudaMemcpyAsync(h->hst, h->dst, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
  int tc_err = 0;
  if (h->tcmem) VE_CU(cudaMemcpyAsync(&tc_err, h->tcx.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  VE_CU(cudaStreamSynchronize(h->stream));
  if (tc_err) return VE_ETIMEOUT;  // a tensor-core kernel gave up waiting: the sweep is invalid
  if (out) {
    out->iter = (long)h->hst->iter;
    out->energy_per_spin = h->hst->energy;
    out->feas_err = h->hst->feas;
    out->d_energy = h->hst->d_energy;
    out->residual = h->hst->residual;
  }
  return VE_OK;
}

int precision_arith(int precision) {
  return precision == VE_PREC_MIXED ? ARITH_FP32 : precision == VE_PREC_DF64 ? ARITH_DF64 : ARITH_FP64;
}

// Entry points that launch work start from a clean error state: a failed runtime call made
// earlier by the caller (not a device fault, which stays sticky) must not be reported as this
// call's launch failure.
class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    cudaGetLastError();
    cudaGetDevice(&old_);
    if (old_ != dev) cudaSetDevice(dev);
    dev_ = dev;
  }
  ~DeviceGuard() {
    if (old_ != dev_) cudaSetDevice(old_);
  }

 private:
  int old_ = 0, dev_ = 0;
};

}  // namespace

extern "C" {

const char* ve_error_string(int code) {
  switch (code) {
    case VE_OK: return "ok";
    case VE_NOT_CONVERGED: return "not converged";
    case VE_EINVAL: return "invalid argument";
    case VE_ENOMEM: return "out of memory";
    case VE_ECUDA: return "CUDA error";
    case VE_ENONFINITE: return "non-finite value in the iteration";
    case VE_EUNSUPPORTED: return "unsupported size";
    case VE_ETIMEOUT: return "a device-side wait timed out";
    default: return "unknown status";
  }
}

void ve_default_options(ve_options* opt) {
  if (!opt) return;
  opt->mu = 10.0;
  opt->nu = 10.0;
  opt->eps = 2.0;
  opt->precision = VE_PREC_FP64;
  opt->check_every = 10;
  opt->stream = nullptr;
}

int ve_ham_tfim(int dim, double J, double h, ve_hamiltonian* out) {
  if (!out || (dim != 1 && dim != 2)) return VE_EINVAL;
  memset(out, 0, sizeof(*out));
  out->onsite[1] = -h;
  out->onsite[2] = -h;
  out->nbond = dim;
  for (int b = 0; b < dim; ++b) {
    out->bond_offset[b][0] = (b == 0);
    out->bond_offset[b][1] = (b == 1);
    out->bond[b][0] = -J;
    out->bond[b][5] = J;
    out->bond[b][10] = J;
    out->bond[b][15] = -J;
  }
  return VE_OK;
}

int ve_ham_xxz(int dim, double J, double delta, ve_hamiltonian* out) {
  if (!out || (dim != 1 && dim != 2)) return VE_EINVAL;
  memset(out, 0, sizeof(*out));
  out->nbond = dim;
  for (int b = 0; b < dim; ++b) {
    out->bond_offset[b][0] = (b == 0);
    out->bond_offset[b][1] = (b == 1);
    // s^x s^x + s^y s^y = 2 (|01><10| + |10><01|); s^z s^z = diag(1, -1, -1, 1)
    out->bond[b][0] = J * delta;
    out->bond[b][5] = -J * delta;
    out->bond[b][10] = -J * delta;
    out->bond[b][15] = J * delta;
    out->bond[b][6] = 2.0 * J;
    out->bond[b][9] = 2.0 * J;
  }
  return VE_OK;
}

int ve_create(const ve_lattice* lattice, const ve_cluster* cluster, const ve_hamiltonian* ham,
              const ve_options* opt, ve_handle** out) {
  if (!out) return VE_EINVAL;
  *out = nullptr;
  ve_handle* h = new (std::nothrow) ve_handle();
  if (!h) return VE_ENOMEM;
  cudaGetLastError();  // report only errors raised by this call
  int rc = build_model(lattice, cluster, ham, h->md);
  if (rc != VE_OK) {
    delete h;
    return rc;
  }
  if (opt) {
    h->opt = *opt;
  } else {
    ve_default_options(&h->opt);
  }
  if (!(h->opt.mu > 0) || !(h->opt.nu > 0) || !(h->opt.eps > 0) || h->opt.check_every < 1 ||
      (h->opt.precision != VE_PREC_FP64 && h->opt.precision != VE_PREC_MIXED &&
       h->opt.precision != VE_PREC_DF64)) {
    delete h;
    return VE_EINVAL;
  }
  const int Ms[2] = {h->md.M0, h->md.M1};
  rc = fft_plan_build(h->plan, h->md.dim, Ms, h->md.D);
  if (rc != 0) {
    delete h;
    return rc;
  }
  cudaGetDevice(&h->device);
  const Model& md = h->md;
  const int N = md.N, m = md.m, D = md.D, P = N - 1;
  h->P = P;
  const size_t mm = (size_t)m * m, DD = (size_t)D * D;
  h->state_bytes = sizeof(double) * (mm + 2 * P * DD + 2 * P * mm + N * DD);
  const int nb = (int)md.pair.size();
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const size_t o_state = take(h->state_bytes);
  const size_t o_a1r = take(sizeof(double) * P * mm);
  const size_t o_a2r = take(sizeof(double) * P * mm);
  const size_t o_part = take(sizeof(double) * 2 * P);
  const size_t o_part2 = take(sizeof(double) * P);
  const size_t o_r0p = take(sizeof(double) * 128 * mm);
  const size_t o_hb = take(sizeof(double) * (nb > 0 ? nb : 1) * DD);
  const size_t o_H0 = take(sizeof(double) * mm);
  const size_t o_lp = take(sizeof(double) * P);
  const size_t o_lk = take(sizeof(double) * N);
  const size_t o_l0 = take(sizeof(double));
  const size_t o_hslot = take(sizeof(int) * N);
  const size_t o_neg = take(sizeof(int) * N);
  const size_t o_canon = take(sizeof(int) * N);
  const size_t o_pidx = take(sizeof(int) * P);
  const size_t o_pmir = take(sizeof(int) * P);
  const size_t o_ptie = take(sizeof(int) * P);
  const size_t o_vp64 = take(sizeof(double) * P * DD);
  const size_t o_vp32 = take(sizeof(float) * P * DD);
  const size_t o_vk64 = take(sizeof(double) * 2 * N * DD);
  const size_t o_vk32 = take(sizeof(float) * 2 * N * DD);
  const size_t o_vpdf = take(sizeof(double) * P * DD);
  const size_t o_vkdf = take(sizeof(double) * 2 * N * DD);
  const size_t o_sa = take(sizeof(double2) * N * h->plan.E);
  const size_t o_sb = take(sizeof(double2) * N * h->plan.E);
  const size_t o_tw = take(sizeof(double2) * h->plan.ntw);
  const size_t o_st = take(sizeof(DevStatus));
  const size_t o_js = take(sizeof(unsigned long long) * 6);
  size_t gws_bytes = pair_ws_bytes(D);
  if (xproj_ws_bytes(D) > gws_bytes) gws_bytes = xproj_ws_bytes(D);
  if (bound_ws_bytes(D) > gws_bytes) gws_bytes = bound_ws_bytes(D);
  const size_t o_gws = take(gws_bytes > 0 ? gws_bytes : 1);
  if (cudaMalloc(&h->dev, off) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return VE_ENOMEM;
  }
  if (cudaMallocHost((void**)&h->hst, sizeof(DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(h->dev);
    delete h;
    return VE_ENOMEM;
  }
  char* base = (char*)h->dev;
  h->state = (double*)(base + o_state);
  h->rho0 = h->state;
  h->rt = h->rho0 + mm;
  h->lam = h->rt + P * DD;
  h->lam1 = h->lam + P * DD;
  h->lam2 = h->lam1 + P * mm;
  h->X = h->lam2 + P * mm;
  h->a1r = (double*)(base + o_a1r);
  h->a2r = (double*)(base + o_a2r);
  h->part = (double*)(base + o_part);
  h->part2 = (double*)(base + o_part2);
  h->rho0_partial = (double*)(base + o_r0p);
  h->hb = (double*)(base + o_hb);
  h->H0 = (double*)(base + o_H0);
  h->lmin_pairs = (double*)(base + o_lp);
  h->lmin_k = (double*)(base + o_lk);
  h->lmin0 = (double*)(base + o_l0);
  h->hslot = (int*)(base + o_hslot);
  h->neg = (int*)(base + o_neg);
  h->canon = (int*)(base + o_canon);
  h->pidx = (int*)(base + o_pidx);
  h->pmir = (int*)(base + o_pmir);
  h->ptie = (int*)(base + o_ptie);
  h->ncanon = fft_ncanon(h->plan);
  h->vpair[0] = base + o_vp64;
  h->vpair[1] = base + o_vp32;
  h->vk[0] = base + o_vk64;
  h->vk[1] = base + o_vk32;
  h->vpair[2] = base + o_vpdf;
  h->vk[2] = base + o_vkdf;
  h->specA = (double2*)(base + o_sa);
  h->specB = (double2*)(base + o_sb);
  h->tw = (double2*)(base + o_tw);
  h->dst = (DevStatus*)(base + o_st);
  h->jstats = (unsigned long long*)(base + o_js);
  h->gws = gws_bytes > 0 ? (unsigned char*)(base + o_gws) : nullptr;
  if (D == 256 && h->opt.precision == VE_PREC_MIXED) {
    // the pair work items are known only below; P bounds their number
    const long nc = fft_ncanon(h->plan);
    const size_t tx = tc_proj_ws_bytes(nc, 1), tp = tc_proj_ws_bytes(P, 0);
    const size_t tr = (size_t)P * DD * sizeof(float);
    if (cudaMalloc(&h->tcmem, tx + tp + tr) != cudaSuccess) {
      cudaGetLastError();
      h->tcmem = nullptr;
      ve_destroy(h);
      return VE_ENOMEM;
    }
    unsigned char* tb = (unsigned char*)h->tcmem;
    if (tc_proj_ws_init(h->tcx, nc, 1, tb, tx) != 0 || tc_proj_ws_init(h->tcp, P, 0, tb + tx, tp) != 0 ||
        cudaMemset(h->tcx.err, 0, sizeof(int)) != cudaSuccess) {
      ve_destroy(h);
      return VE_ECUDA;
    }
    h->tcp.err = h->tcx.err;  // one error word for both
    h->rbuf = (float*)(tb + tx + tp);
  }
  if (h->opt.stream) {
    h->stream = (cudaStream_t)h->opt.stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      ve_destroy(h);
      return VE_ECUDA;
    }
    h->own_stream = true;
  }
  // host staging: initial state (Sec. 4), Hamiltonian blocks, index tables
  std::vector<double> st(h->state_bytes / sizeof(double), 0.0);
  for (int i = 0; i < m; ++i) st[(size_t)i * m + i] = 1.0 / m;
  for (int p = 0; p < P; ++p)
    for (int i = 0; i < D; ++i) st[mm + (size_t)p * DD + (size_t)i * D + i] = 1.0 / D;
  const size_t xo = mm + 2 * P * DD + 2 * P * mm;
  for (int i = 0; i < D; ++i) st[xo + (size_t)i * D + i] = 1.0;
  std::vector<double> hb((size_t)(nb > 0 ? nb : 1) * DD, 0.0);
  std::vector<int> hslot(N, -1);
  int k = 0;
  for (auto& kv : md.pair) {
    hslot[kv.first] = k;
    memcpy(hb.data() + (size_t)k * DD, kv.second.data(), sizeof(double) * DD);
    ++k;
  }
  // work items of the pair pass: the canonical (smaller linear index) member of each pair of
  // opposite offsets, with the other as its image; every offset on its own if H is not tied
  std::vector<int> pidx, pmir, ptie(P, -2);
  const bool tied = model_swap_symmetric(md);
  for (int dl = 1; dl < N; ++dl) {
    const int nd = md.neg[dl];
    if (tied && nd < dl) continue;
    const int img = (!tied || nd == dl) ? -1 : nd - 1;
    pidx.push_back(dl - 1);
    pmir.push_back(img);
    ptie[dl - 1] = img;
  }
  h->Pc = (int)pidx.size();
  DevStatus ds;
  memset(&ds, 0, sizeof(ds));
  ds.e_prev = NAN;
  ds.energy = NAN;
  ds.feas = NAN;
  ds.d_energy = INFINITY;
  ds.residual = INFINITY;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->state, st.data(), h->state_bytes, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->hb, hb.data(), sizeof(double) * hb.size(), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->H0, md.H0.data(), sizeof(double) * mm, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->hslot, hslot.data(), sizeof(int) * N, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->neg, md.neg.data(), sizeof(int) * N, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->pidx, pidx.data(), sizeof(int) * h->Pc, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->pmir, pmir.data(), sizeof(int) * h->Pc, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->ptie, ptie.data(), sizeof(int) * P, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->dst, &ds, sizeof(ds), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = launch_fft_tables(h->plan, h->tw, h->stream);
  if (e == cudaSuccess) e = launch_canon_list(h->plan, h->canon, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    ve_destroy(h);
    return VE_ECUDA;
  }
  *h->hst = ds;
  const int launches[VE_NSTAGE] = {1, 1, 1, 1, h->plan.npass, 1, h->plan.npass};
  for (int i = 0; i < VE_NSTAGE; ++i) h->stage_launches[i] = launches[i];
  *out = h;
  return VE_OK;
}

void ve_destroy(ve_handle* h) {
  if (!h) return;
  DeviceGuard g(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (int v = 0; v < 3; ++v) {
    if (h->exec[v]) cudaGraphExecDestroy(h->exec[v]);
    if (h->graph[v]) cudaGraphDestroy(h->graph[v]);
  }
  for (int i = 0; i <= VE_NSTAGE; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  if (h->hst) cudaFreeHost(h->hst);
  if (h->dev) cudaFree(h->dev);
  if (h->tcmem) cudaFree(h->tcmem);
  delete h;
}

int ve_dims(const ve_handle* h, int* N, int* m, int* D) {
  if (!h) return VE_EINVAL;
  if (N) *N = h->md.N;
  if (m) *m = h->md.m;
  if (D) *D = h->md.D;
  return VE_OK;
}

size_t ve_state_size(const ve_handle* h) { return h ? h->state_bytes : 0; }

int ve_get_state(ve_handle* h, double* host, size_t bytes) {
  if (!h || !host || bytes != h->state_bytes) return VE_EINVAL;
  DeviceGuard g(h->device);
  VE_CU(cudaMemcpyAsync(host, h->state, bytes, cudaMemcpyDeviceToHost, h->stream));
  VE_CU(cudaStreamSynchronize(h->stream));
  return VE_OK;
}

int ve_set_state(ve_handle* h, const double* host, size_t bytes) {
  if (!h || !host || bytes != h->state_bytes) return VE_EINVAL;
  DeviceGuard g(h->device);
  VE_CU(cudaStreamSynchronize(h->stream));
  const int r = read_status(h, nullptr);
  if (r != VE_OK) return r;
  h->hst->e_prev = NAN;
  h->hst->d_energy = INFINITY;
  h->hst->residual = INFINITY;
  VE_CU(cudaMemcpyAsync(h->state, host, bytes, cudaMemcpyHostToDevice, h->stream));
  VE_CU(cudaMemcpyAsync(h->dst, h->hst, sizeof(DevStatus), cudaMemcpyHostToDevice, h->stream));
  VE_CU(cudaStreamSynchronize(h->stream));
  h->fp64_phase = false;
  h->mx_best = INFINITY;
  h->mx_stall = 0;
  // the stored eigenvectors stay: any orthogonal start is valid for the Jacobi eigensolves, and
  // those of the last sweep are the right one when the state set is near the handle's own
  return VE_OK;
}

int ve_profile(ve_handle* h, int enable) {
  if (!h) return VE_EINVAL;
  DeviceGuard g(h->device);
  if (enable) {
    for (int i = 0; i <= VE_NSTAGE; ++i)
      if (!h->ev[i]) VE_CU(cudaEventCreate(&h->ev[i]));
    for (int i = 0; i < VE_NSTAGE; ++i) {
      h->prof_ms[i] = 0.0;
      h->prof_launch[i] = 0;
    }
    VE_CU(cudaMemsetAsync(h->jstats, 0, sizeof(unsigned long long) * 6, h->stream));
    VE_CU(cudaStreamSynchronize(h->stream));
  }
  h->prof = enable != 0;
  return VE_OK;
}

int ve_profile_sweeps(ve_handle* h, double* pair, double* wavevector) {
  if (!h || !pair || !wavevector) return VE_EINVAL;
  DeviceGuard g(h->device);
  unsigned long long c[6] = {0, 0, 0, 0, 0, 0};
  VE_CU(cudaMemcpyAsync(c, h->jstats, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
  VE_CU(cudaStreamSynchronize(h->stream));
  *pair = c[1] ? (double)c[0] / (double)c[1] : 0.0;
  *wavevector = c[4] ? (double)c[3] / (double)c[4] : 0.0;
  return VE_OK;
}

int ve_profile_first_order(ve_handle* h, long* pair, long* wavevector) {
  if (!h || !pair || !wavevector) return VE_EINVAL;
  DeviceGuard g(h->device);
  unsigned long long c[6] = {0, 0, 0, 0, 0, 0};
  VE_CU(cudaMemcpyAsync(c, h->jstats, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
  VE_CU(cudaStreamSynchronize(h->stream));
  pair[0] = (long)c[2];
  pair[1] = (long)c[1];
  wavevector[0] = (long)c[5];
  wavevector[1] = (long)c[4];
  return VE_OK;
}

int ve_profile_read(ve_handle* h, double* ms, long* launches) {
  if (!h || !ms || !launches) return VE_EINVAL;
  for (int i = 0; i < VE_NSTAGE; ++i) {
    ms[i] = h->prof_ms[i];
    launches[i] = h->prof_launch[i];
  }
  return VE_OK;
}

int ve_get_status(ve_handle* h, ve_status* out) {
  if (!h || !out) return VE_EINVAL;
  DeviceGuard g(h->device);
  return read_status(h, out);
}

// Arithmetic of the next sweeps of a handle.
int handle_arith(const ve_handle* h) {
  switch (h->opt.precision) {
    case VE_PREC_DF64: return ARITH_DF64;
    case VE_PREC_MIXED: return h->fp64_phase ? ARITH_DF64 : ARITH_FP32;
    default: return ARITH_FP64;
  }
}

// Stopping rule shared by ve_iterate and ve_batch_iterate: in VE_PREC_MIXED, float32 sweeps
// until the residual meets tol or has not fallen by 1 % over 100 read-backs (the float32
// rounding floor), then float64 sweeps until the residual meets tol.
struct IterCtl {
  bool finished = false;
  int rc = VE_NOT_CONVERGED;
};

void ctl_update(ve_handle* h, IterCtl& c, const ve_status& s, double tol) {
  if (!isfinite(s.energy_per_spin) || !isfinite(s.feas_err)) {
    c.finished = true;
    c.rc = VE_ENONFINITE;
    return;
  }
  if (tol <= 0) return;
  const bool fp32 = h->opt.precision == VE_PREC_MIXED && !h->fp64_phase;
  if (fp32) {
    if (s.residual < 0.99 * h->mx_best) {
      h->mx_best = s.residual;
      h->mx_stall = 0;
    } else {
      ++h->mx_stall;
    }
    if (s.residual <= tol || h->mx_stall >= 100) h->fp64_phase = true;
  } else if (s.residual <= tol) {
    c.finished = true;
    c.rc = VE_OK;
  }
}

int ve_iterate(ve_handle* h, long max_iter, double tol, ve_status* out) {
  if (!h || max_iter < 0) return VE_EINVAL;
  DeviceGuard g(h->device);
  ve_status s;
  IterCtl c;
  long done = 0;
  if (max_iter == 0) {
    int r = read_status(h, &s);
    if (out) *out = s;
    return r != VE_OK ? r : VE_OK;
  }
  while (done < max_iter && !c.finished) {
    const long chunk = (long)h->opt.check_every < max_iter - done ? (long)h->opt.check_every : max_iter - done;
    int r = run_sweeps(h, chunk, handle_arith(h));
    if (r != VE_OK) return r;
    r = read_status(h, &s);
    if (r != VE_OK) return r;
    done += chunk;
    ctl_update(h, c, s, tol);
  }
  if (out) *out = s;
  if (c.rc == VE_ENONFINITE) return VE_ENONFINITE;
  if (tol <= 0) return VE_OK;
  return c.rc;
}

int ve_bound(ve_handle* h, ve_cert* out) {
  if (!h || !out) return VE_EINVAL;
  DeviceGuard g(h->device);
  const Model& md = h->md;
  const int N = md.N, P = h->P;
  double2* spec = nullptr;
  VE_CU(fft_forward(h->plan, h->X, h->specA, h->specB, h->tw, &spec, false, h->stream));
  VE_CU(launch_xeig(h->plan, spec, h->canon, h->lmin_k, h->stream, h->gws));
  BoundArgs b;
  b.N = N;
  b.P = P;
  b.m = md.m;
  b.D = md.D;
  b.X = h->X;
  b.lam1 = h->lam1;
  b.hb = h->hb;
  b.hslot = h->hslot;
  b.neg = h->neg;
  b.H0 = h->H0;
  b.lmin_pairs = h->lmin_pairs;
  b.lmin0 = h->lmin0;
  b.gws = h->gws;
  VE_CU(launch_bound(b, h->stream));
  std::vector<double> lp(P), lk(h->ncanon);
  double l0 = 0;
  VE_CU(cudaMemcpyAsync(lp.data(), h->lmin_pairs, sizeof(double) * P, cudaMemcpyDeviceToHost, h->stream));
  VE_CU(cudaMemcpyAsync(lk.data(), h->lmin_k, sizeof(double) * h->ncanon, cudaMemcpyDeviceToHost,
                        h->stream));
  VE_CU(cudaMemcpyAsync(&l0, h->lmin0, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  ve_status s;
  int r = read_status(h, &s);  // synchronises the stream
  if (r != VE_OK) return r;
  double raw = (double)N * l0;
  for (int p = 0; p < P; ++p) raw += (double)md.count[p + 1] * lp[p];
  double xmin = INFINITY;
  bool finite = std::isfinite(raw);  // a NaN or Inf in any pair or cluster term reaches raw
  for (int k = 0; k < h->ncanon; ++k) {
    finite = finite && std::isfinite(lk[k]);
    xmin = lk[k] < xmin ? lk[k] : xmin;
  }
  if (!finite) return VE_ENONFINITE;  // a non-finite state certifies nothing
  const double corr = (double)N * md.m * (xmin < 0 ? -xmin : 0.0);
  const double spins = (double)N * md.L;
  out->raw_bound = raw;
  out->x_min_eig = xmin;
  out->x_neg_correction = corr;
  out->bound_per_spin = (raw - corr) / spins;
  out->primal_per_spin = s.energy_per_spin;
  return VE_OK;
}

int ve_project_state_x(ve_handle* h) {
  if (!h) return VE_EINVAL;
  DeviceGuard g(h->device);
  double2* spec = nullptr;
  VE_CU(fft_forward(h->plan, h->X, h->specA, h->specB, h->tw, &spec, false, h->stream));
  VE_CU(launch_xproj(h->plan, spec, h->canon, ARITH_FP64, nullptr, 0, h->stream, nullptr, h->gws));
  VE_CU(fft_inverse(h->plan, spec, h->specA, h->specB, h->X, h->tw, false, h->stream));
  VE_CU(cudaStreamSynchronize(h->stream));
  return VE_OK;
}

int ve_project_psd_sym(const double* in, double* out, int n, long count, int precision,
                       void* stream) {
  cudaGetLastError();  // report only errors raised by this call
  if (!in || !out || count < 0) return VE_EINVAL;
  if (n != 2 && n != 4 && n != 8 && n != 16 && n != 64) return VE_EINVAL;
  if (precision != VE_PREC_FP64 && precision != VE_PREC_MIXED && precision != VE_PREC_DF64)
    return VE_EINVAL;
  VE_CU(launch_proj_sym(in, out, n, count, precision_arith(precision), (cudaStream_t)stream));
  return VE_OK;
}

int ve_project_psd_herm(const double* in, double* out, int n, long count, int precision,
                        void* stream) {
  cudaGetLastError();  // report only errors raised by this call
  if (!in || !out || count < 0) return VE_EINVAL;
  if (n != 4 && n != 16 && n != 64) return VE_EINVAL;
  if (precision != VE_PREC_FP64 && precision != VE_PREC_MIXED && precision != VE_PREC_DF64)
    return VE_EINVAL;
  VE_CU(launch_proj_herm(in, out, n, count, precision_arith(precision), (cudaStream_t)stream));
  return VE_OK;
}

size_t ve_project_psd_large_workspace_size(int n, int hermitian, int precision) {
  if (precision != VE_PREC_FP64 && precision != VE_PREC_MIXED && precision != VE_PREC_DF64)
    return 0;
  return proj_ws_bytes(n, hermitian != 0, precision_arith(precision));
}

static int project_large(const double* in, double* out, int n, long count, int precision,
                         void* workspace, size_t workspace_bytes, void* stream, bool herm) {
  cudaGetLastError();  // report only errors raised by this call
  if (!in || !out || !workspace || count < 0) return VE_EINVAL;
  const size_t need = ve_project_psd_large_workspace_size(n, herm ? 1 : 0, precision);
  if (need == 0 || workspace_bytes < need || ((uintptr_t)workspace) % kAlign) return VE_EINVAL;
  const int arith = precision_arith(precision);
  unsigned char* ws = (unsigned char*)workspace;
  if (herm) {
    VE_CU(launch_proj_herm(in, out, n, count, arith, (cudaStream_t)stream, ws));
  } else {
    VE_CU(launch_proj_sym(in, out, n, count, arith, (cudaStream_t)stream, ws));
  }
  return VE_OK;
}

int ve_project_psd_sym_large(const double* in, double* out, int n, long count, int precision,
                             void* workspace, size_t workspace_bytes, void* stream) {
  return project_large(in, out, n, count, precision, workspace, workspace_bytes, stream, false);
}

int ve_project_psd_herm_large(const double* in, double* out, int n, long count, int precision,
                              void* workspace, size_t workspace_bytes, void* stream) {
  return project_large(in, out, n, count, precision, workspace, workspace_bytes, stream, true);
}

size_t ve_circulant_workspace_size(int dim, const int M[2], int D) {
  if (!M || D == 256) return 0;
  FftPlan p;
  if (fft_plan_build(p, dim, M, D) != 0) return 0;
  return align_up(sizeof(double2) * (size_t)p.N * p.E) * 2 + align_up(sizeof(double2) * p.ntw) +
         align_up(sizeof(int) * (size_t)p.N);
}

int ve_circulant_project(const double* x_in, double* x_out, int dim, const int M[2], int D,
                         int precision, void* workspace, size_t workspace_bytes, void* stream) {
  cudaGetLastError();  // report only errors raised by this call
  if (!x_in || !x_out || !M || !workspace) return VE_EINVAL;
  if (precision != VE_PREC_FP64 && precision != VE_PREC_MIXED && precision != VE_PREC_DF64)
    return VE_EINVAL;
  if (((uintptr_t)workspace) % kAlign) return VE_EINVAL;
  if (D == 256) return VE_EUNSUPPORTED;
  FftPlan p;
  const int rc = fft_plan_build(p, dim, M, D);
  if (rc != 0) return rc;
  const size_t sb = align_up(sizeof(double2) * (size_t)p.N * p.E);
  const size_t stw = align_up(sizeof(double2) * p.ntw);
  if (workspace_bytes < 2 * sb + stw + align_up(sizeof(int) * (size_t)p.N)) return VE_EINVAL;
  char* w = (char*)workspace;
  double2* A = (double2*)w;
  double2* B = (double2*)(w + sb);
  double2* tw = (double2*)(w + 2 * sb);
  int* canon = (int*)(w + 2 * sb + stw);
  cudaStream_t s = (cudaStream_t)stream;
  VE_CU(launch_fft_tables(p, tw, s));
  VE_CU(launch_canon_list(p, canon, s));
  double2* spec = nullptr;
  const bool fp32 = precision == VE_PREC_MIXED;
  VE_CU(fft_forward(p, x_in, A, B, tw, &spec, fp32, s));
  VE_CU(launch_xproj(p, spec, canon, precision_arith(precision), nullptr, 0, s));
  VE_CU(fft_inverse(p, spec, A, B, x_out, tw, fp32, s));
  return VE_OK;
}


// ------------------------------------------------------------------------- batches
}  // extern "C"

struct ve_batch {
  int n = 0;
  int device = 0;
  std::vector<ve_handle*> h;
  cudaStream_t main = nullptr;
  DevStatus* dst = nullptr;  // device, n entries (the instances' status words)
  DevStatus* hst = nullptr;  // pinned mirror
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> key;  // per instance: -1 idle, else the Arith of its branch
};

namespace {

void batch_drop_graph(ve_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->key.clear();
}

// One graph whose branches are one sweep of every instance with key >= 0 (fork on the main
// stream, one branch per instance stream, join back).
int batch_capture(ve_batch* b, const std::vector<int>& key) {
  batch_drop_graph(b);
  VE_CU(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaEventRecord(b->fork, b->main);
  for (int i = 0; i < b->n && e == cudaSuccess; ++i) {
    if (key[i] < 0) continue;
    ve_handle* h = b->h[i];
    e = cudaStreamWaitEvent(h->stream, b->fork, 0);
    if (e == cudaSuccess) e = issue_sweep(h, key[i], true);
    if (e == cudaSuccess) e = cudaEventRecord(b->join[i], h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->main, b->join[i], 0);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->main, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return VE_ECUDA;
  }
  b->graph = g;
  VE_CU(cudaGraphInstantiate(&b->exec, g, 0));
  b->key = key;
  return VE_OK;
}

}  // namespace

extern "C" {

int ve_create_batch(int n, const ve_lattice* lattices, const ve_cluster* clusters,
                    const ve_hamiltonian* hams, const ve_options* opt, ve_batch** out) {
  if (!out || n < 1 || !lattices || !clusters || !hams) return VE_EINVAL;
  *out = nullptr;
  if (opt && opt->stream) return VE_EINVAL;  // every instance runs on a stream of its own
  ve_batch* b = new (std::nothrow) ve_batch();
  if (!b) return VE_ENOMEM;
  cudaGetDevice(&b->device);
  b->n = n;
  b->h.assign(n, nullptr);
  b->join.assign(n, nullptr);
  for (int i = 0; i < n; ++i) {
    const int rc = ve_create(&lattices[i], &clusters[i], &hams[i], opt, &b->h[i]);
    if (rc != VE_OK) {
      ve_batch_destroy(b);
      return rc;
    }
  }
  if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc((void**)&b->dst, sizeof(DevStatus) * n) != cudaSuccess ||
      cudaMallocHost((void**)&b->hst, sizeof(DevStatus) * n) != cudaSuccess) {
    cudaGetLastError();
    ve_batch_destroy(b);
    return VE_ENOMEM;
  }
  for (int i = 0; i < n; ++i) {
    if (cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess) {
      ve_batch_destroy(b);
      return VE_ECUDA;
    }
    // the instance's status word moves into the batch array, so one copy reads them all
    ve_handle* h = b->h[i];
    b->hst[i] = *h->hst;
    h->dst = b->dst + i;
  }
  if (cudaMemcpy(b->dst, b->hst, sizeof(DevStatus) * n, cudaMemcpyHostToDevice) != cudaSuccess) {
    ve_batch_destroy(b);
    return VE_ECUDA;
  }
  *out = b;
  return VE_OK;
}

int ve_batch_size(const ve_batch* b) { return b ? b->n : 0; }

ve_handle* ve_batch_handle(ve_batch* b, int i) {
  if (!b || i < 0 || i >= b->n) return nullptr;
  return b->h[i];
}

int ve_batch_iterate(ve_batch* b, long max_iter, double tol, ve_status* out) {
  if (!b || max_iter < 0) return VE_EINVAL;
  DeviceGuard g(b->device);
  const int n = b->n;
  std::vector<IterCtl> ctl(n);
  std::vector<ve_status> st(n);
  long done = 0;
  int check = b->h[0]->opt.check_every;
  for (int i = 1; i < n; ++i) check = b->h[i]->opt.check_every < check ? b->h[i]->opt.check_every : check;
  while (done < max_iter) {
    const long chunk = (long)check < max_iter - done ? (long)check : max_iter - done;
    std::vector<int> key(n, -1);
    bool any = false, cold = false;
    for (int i = 0; i < n; ++i) {
      if (ctl[i].finished) continue;
      ve_handle* h = b->h[i];
      if (h->prof) return VE_EINVAL;  // per-stage profiling is per handle, not in a batch
      key[i] = handle_arith(h);
      any = true;
      if (!h->vvalid[key[i]]) cold = true;
    }
    if (!any) break;
    long launches = chunk;
    if (cold) {
      // some instance starts a precision phase: its first sweep runs directly and cold (as in
      // run_sweeps), and every other active instance takes one direct warm sweep beside it so
      // that all advance by exactly `chunk` sweeps; the main stream then waits for them all
      for (int i = 0; i < n; ++i) {
        if (key[i] < 0) continue;
        ve_handle* h = b->h[i];
        const int v = key[i];
        VE_CU(issue_sweep(h, v, h->vvalid[v]));
        h->vvalid[v] = true;
        VE_CU(cudaEventRecord(b->join[i], h->stream));
        VE_CU(cudaStreamWaitEvent(b->main, b->join[i], 0));
      }
      --launches;
    }
    if (launches > 0 && (!b->exec || key != b->key)) {
      const int r = batch_capture(b, key);
      if (r != VE_OK) return r;
    }
    for (long c = 0; c < launches; ++c) VE_CU(cudaGraphLaunch(b->exec, b->main));
    VE_CU(cudaMemcpyAsync(b->hst, b->dst, sizeof(DevStatus) * n, cudaMemcpyDeviceToHost, b->main));
    VE_CU(cudaStreamSynchronize(b->main));
    done += chunk;
    for (int i = 0; i < n; ++i) {
      if (ctl[i].finished) continue;
      ve_handle* h = b->h[i];
      *h->hst = b->hst[i];
      st[i].iter = (long)b->hst[i].iter;
      st[i].energy_per_spin = b->hst[i].energy;
      st[i].feas_err = b->hst[i].feas;
      st[i].d_energy = b->hst[i].d_energy;
      st[i].residual = b->hst[i].residual;
      ctl_update(h, ctl[i], st[i], tol);
    }
  }
  int rc = VE_OK;
  for (int i = 0; i < n; ++i) {
    if (out) {
      const int r = read_status(b->h[i], &out[i]);
      if (r != VE_OK) return r;
    }
    if (ctl[i].rc == VE_ENONFINITE) rc = VE_ENONFINITE;
    else if (tol > 0 && ctl[i].rc != VE_OK && rc == VE_OK) rc = VE_NOT_CONVERGED;
  }
  return rc;
}

int ve_batch_bound(ve_batch* b, ve_cert* out) {
  if (!b || !out) return VE_EINVAL;
  for (int i = 0; i < b->n; ++i) {
    const int r = ve_bound(b->h[i], &out[i]);
    if (r != VE_OK) return r;
  }
  return VE_OK;
}

void ve_batch_destroy(ve_batch* b) {
  if (!b) return;
  DeviceGuard g(b->device);
  if (b->main) cudaStreamSynchronize(b->main);
  batch_drop_graph(b);
  for (int i = 0; i < (int)b->h.size(); ++i) {
    if (b->h[i]) {
      // give the instance back a status word of its own before it is released
      b->h[i]->dst = nullptr;
      ve_destroy(b->h[i]);
    }
    if (i < (int)b->join.size() && b->join[i]) cudaEventDestroy(b->join[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->main) cudaStreamDestroy(b->main);
  if (b->dst) cudaFree(b->dst);
  if (b->hst) cudaFreeHost(b->hst);
  delete b;
}

}  // extern "C"
