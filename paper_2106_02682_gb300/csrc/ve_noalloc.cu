// ve_noalloc.cu -- ve_circulant_project_noalloc: the X step (block DFT, per-wavevector PSD
// projection, inverse DFT) with its scratch in a fixed file-scope device array instead of
// caller-provided or freshly allocated memory.  See include/ve.h for the contract.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ve.h"
#include "ve_internal.h"

using namespace ve;

namespace {

// The scratch array.  In host code `g_scratch` names only a host-side stand-in for the symbol;
// its device address must come from cudaGetSymbolAddress on the device that runs the kernels.
static __device__ __align__(256) unsigned char g_scratch[VE_NOALLOC_SCRATCH_BYTES];

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Device address of g_scratch on the current device, looked up on every call: the lookup is a
// host-side query, and an address kept from an earlier call would go stale if the device's
// primary context were torn down (cudaDeviceReset) and the module loaded again elsewhere.
int scratch_address(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return VE_ECUDA;
  *out = p;
  return VE_OK;
}

}  // namespace

extern "C" int ve_circulant_project_noalloc(const double* x_in, double* x_out, int dim,
                                            const int M[2], int D, int precision, void* stream) {
  if (!x_in || !x_out || !M) return VE_EINVAL;
  if (precision != VE_PREC_FP64 && precision != VE_PREC_MIXED && precision != VE_PREC_DF64)
    return VE_EINVAL;
  if (D == 256) return VE_EUNSUPPORTED;
  cudaGetLastError();  // report only errors raised by this call
  FftPlan p;
  const int rc = fft_plan_build(p, dim, M, D);
  if (rc != 0) return rc;
  const size_t sb = align_up(sizeof(double2) * (size_t)p.N * p.E);
  const size_t stw = align_up(sizeof(double2) * p.ntw);
  const size_t need = 2 * sb + stw + align_up(sizeof(int) * (size_t)p.N);
  if (need > VE_NOALLOC_SCRATCH_BYTES) return VE_EINVAL;
  void* scratch = nullptr;
  const int r = scratch_address(&scratch);
  if (r != VE_OK) return r;
  char* w = (char*)scratch;
  double2* A = (double2*)w;
  double2* B = (double2*)(w + sb);
  double2* tw = (double2*)(w + 2 * sb);
  int* canon = (int*)(w + 2 * sb + stw);
  cudaStream_t s = (cudaStream_t)stream;
  // nothing in the scratch has to start at zero: the tables, the wavevector list and both
  // spectra are fully rewritten by this call before they are read
  if (launch_fft_tables(p, tw, s) != cudaSuccess) return VE_ECUDA;
  if (launch_canon_list(p, canon, s) != cudaSuccess) return VE_ECUDA;
  double2* spec = nullptr;
  const bool fp32 = precision == VE_PREC_MIXED;
  if (fft_forward(p, x_in, A, B, tw, &spec, fp32, s) != cudaSuccess) return VE_ECUDA;
  const int arith = fp32 ? ARITH_FP32 : precision == VE_PREC_DF64 ? ARITH_DF64 : ARITH_FP64;
  if (launch_xproj(p, spec, canon, arith, nullptr, 0, s) != cudaSuccess) return VE_ECUDA;
  if (fft_inverse(p, spec, A, B, x_out, tw, fp32, s) != cudaSuccess) return VE_ECUDA;
  return VE_OK;
}
