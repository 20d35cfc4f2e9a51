// Host entry points of the apply path: dtype dispatch, device properties and
// the batched launch. The kernels live in apply_kernel.cuh and are
// instantiated per arithmetic policy in apply_f32.cu / apply_df64.cu /
// apply_f64.cu.
#include <algorithm>
#include <vector>

#include "device_common.cuh"

namespace hm {

template <int AR>
cudaError_t launch_apply_t(const KPlan& k, const void* x, void* y, long long nvec, cudaStream_t st, int ctas);
template <int AR>
cudaError_t launch_batch_t(const KPlan* dplans, const std::vector<const Plan*>& members, const void* const* xs,
                           void* const* ys, long long nvec, cudaStream_t st);

static int g_nsm = 0;
int num_sms() {
  if (g_nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_nsm, cudaDevAttrMultiProcessorCount, dev);
    if (g_nsm <= 0) g_nsm = 1;
  }
  return g_nsm;
}

cudaError_t apply_kplan(const KPlan& k, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s,
                        int ctas, bool native_f64) {
  if (dt == HM_F32) return launch_apply_t<AR_F32>(k, x, y, nvec, s, ctas);
  if (native_f64) return launch_apply_t<AR_F64>(k, x, y, nvec, s, ctas);
  return launch_apply_t<AR_DF64>(k, x, y, nvec, s, ctas);
}

int launch_apply(const Plan* p, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s,
                 int ctas_override) {
  cudaError_t e = apply_kplan(p->k, x, y, nvec, dt, s, ctas_override, false);
  if (e != cudaSuccess) return cuda_fail(e, "apply launch");
  return HM_OK;
}

int batch_setup(Plan* b) {
  const size_t n = b->members.size();
  std::vector<KPlan> ks(n);
  b->member_gen.assign(n, 0);
  for (size_t i = 0; i < n; ++i) {
    ks[i] = b->members[i]->k;
    b->member_gen[i] = b->members[i]->gen;
  }
  if (!b->batch_dev) {
    cudaError_t e = cudaMalloc(&b->batch_dev, sizeof(KPlan) * n);
    if (e != cudaSuccess) {
      b->batch_dev = nullptr;
      return cuda_fail(e, "batch plan table");
    }
  }
  cudaError_t e = cudaMemcpy(b->batch_dev, ks.data(), sizeof(KPlan) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "batch plan upload");
  return HM_OK;
}

int launch_batch(Plan* b, const void* const* xs, void* const* ys, long long nvec, hm_dtype dt, cudaStream_t s) {
  bool stale = false;
  for (size_t i = 0; i < b->members.size(); ++i) stale |= (b->members[i]->gen != b->member_gen[i]);
  if (stale) {  // a member was re-planned (hm_set_coefficients): refresh its tables
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs != cudaStreamCaptureStatusNone) {
      set_error("a batch member changed since the batch was built; refresh outside stream capture");
      return HM_ERR_INVALID_ARG;
    }
    int rc = batch_setup(b);
    if (rc) return rc;
  }
  std::vector<const Plan*> mem(b->members.begin(), b->members.end());
  cudaError_t e = (dt == HM_F32) ? launch_batch_t<AR_F32>((const KPlan*)b->batch_dev, mem, xs, ys, nvec, s)
                                 : launch_batch_t<AR_DF64>((const KPlan*)b->batch_dev, mem, xs, ys, nvec, s);
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  return HM_OK;
}

}  // namespace hm
