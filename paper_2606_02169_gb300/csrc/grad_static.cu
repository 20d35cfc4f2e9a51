// Coupling gradients without any device allocation.
//
// hm_apply_adjoint grows a per-plan scratch buffer with cudaMalloc for the
// per-CTA partial sums of the coupling gradients. Some callers cannot let a
// library allocate: code that runs while a stream is being captured into a
// CUDA graph (cudaMalloc is not a stream operation and is not allowed
// there), and processes whose device memory belongs to another allocator
// (a framework's caching pool or a fixed serving budget). For them this file
// keeps the partials in a fixed, file-scope device array instead.
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>

#include "hm_internal.h"

namespace hm {

int check_vec_args(const Plan* p, const void* x, const void* y, long long nvec, hm_dtype dt);
int grad_grid(const Plan* p);
size_t grad_smem(const Plan* p);
int launch_term_grad(const Plan* p, const void* gy, const void* x, double* gcoef, long long nvec, hm_dtype dt,
                     double* partial, int grid, cudaStream_t s);

// 1 MiB of partial sums: grid * nterms <= 131072. Every GPU that loads the
// library holds this array until the process exits.
constexpr long long kStaticPartials = 131072;
static __device__ __align__(256) double g_static_partials[kStaticPartials];

// Device address of g_static_partials per device. In host code the symbol
// names a host-side stand-in, so the address is looked up once per device
// with that device current.
static std::mutex g_static_mu;
static std::map<int, double*> g_static_addr;

static int static_partials(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> g(g_static_mu);
  auto it = g_static_addr.find(dev);
  if (it == g_static_addr.end()) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static partials)");
    it = g_static_addr.emplace(dev, (double*)ptr).first;
  }
  *out = it->second;
  return HM_OK;
}

}  // namespace hm

extern "C" int hm_coupling_gradients_static(hm_handle h, const void* gy, const void* x, double* gcoef,
                                            int64_t nvec, hm_dtype dtype, void* stream) {
  using namespace hm;
  if (dtype == HM_C128 || dtype == HM_C64) {  // real H: the (re, im) parts are 2 * nvec real columns
    dtype = dtype == HM_C128 ? HM_F64 : HM_F32;
    if (nvec > 0 && nvec < (1LL << 40)) nvec *= 2;
  }
  Plan* p = reinterpret_cast<Plan*>(h);
  if (!p || p->magic != 0x484d504cU || p->is_batch) {
    set_error("invalid handle");
    return HM_ERR_INVALID_ARG;
  }
  if (p->sector) {
    set_error("hm_coupling_gradients_static is not available for sector plans (hm_create_sector)");
    return HM_ERR_UNSUPPORTED;
  }
  if (p->im || !p->grad_ok) {
    set_error("coupling gradients are not available for a complex H or a term with imaginary elements");
    return HM_ERR_UNSUPPORTED;
  }
  if (!gy || !x || !gcoef || nvec < 1 || (dtype != HM_F64 && dtype != HM_F32)) {
    set_error("gy, x and gcoef must be device pointers, nvec >= 1, dtype HM_F64 or HM_F32");
    return HM_ERR_INVALID_ARG;
  }
  // the same vector checks as hm_apply_adjoint: element alignment, the nvec
  // cap and the int64 bound on D * nvec; gy and x may be the same vector
  int rc = check_vec_args(p, gy, x, nvec, dtype);
  if (rc == HM_ERR_ALIAS) rc = HM_OK;
  if (rc) return rc;
  if ((uintptr_t)gcoef % sizeof(double)) {
    set_error("gcoef must be aligned to 8 bytes");
    return HM_ERR_INVALID_ARG;
  }
  // the plan's tables and the scratch address are per device: the call must
  // run with the plan's device current
  int cur = -1;
  cudaError_t ce = cudaGetDevice(&cur);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
  if (cur != p->device) {
    set_error("hm_coupling_gradients_static: device " + std::to_string(cur) + " is current but the plan lives on device " +
              std::to_string(p->device));
    return HM_ERR_INVALID_ARG;
  }
  const long long nterms = (long long)p->terms.size();
  if (nterms == 0) return HM_OK;
  if (nterms > kStaticPartials) {
    set_error("hm_coupling_gradients_static: " + std::to_string(nterms) +
              " terms exceed its fixed scratch of 131072 partial sums");
    return HM_ERR_TOO_LARGE;
  }
  if (grad_smem(p) > 200 * 1024) {
    set_error("too many terms for the gradient reduction (limit 3200)");
    return HM_ERR_UNSUPPORTED;
  }
  double* partial = nullptr;
  rc = static_partials(&partial);
  if (rc) return rc;
  // each CTA writes all nterms of its row before the reduction reads them,
  // so nothing in the shared array has to be cleared between calls
  const int grid = (int)std::min<long long>(grad_grid(p), kStaticPartials / nterms);
  return launch_term_grad(p, gy, x, gcoef, nvec, dtype, partial, grid, (cudaStream_t)stream);
}
