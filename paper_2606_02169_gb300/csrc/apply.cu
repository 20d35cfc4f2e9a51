// Host entry points of the apply path: dtype dispatch, the FP64 split pass,
// device properties and the batched launch. The kernels live in
// apply_kernel.cuh and are instantiated per arithmetic policy in
// apply_f32.cu / apply_df64.cu / apply_f64.cu.
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <vector>

#include "apply_kernel.cuh"

namespace hm {

template <int AR>
cudaError_t launch_apply_t(const KPlan& k, const void* x, void* y, long long nvec, cudaStream_t st, TuneCfg cfg);
template <int AR>
cudaError_t launch_batch_t(const std::vector<const Plan*>& members, const void* const* xs, void* const* ys,
                           long long nvec, cudaStream_t st);
template <int AR>
cudaError_t launch_tile_t(const KTile& k, const void* x, void* y, cudaStream_t st, TuneCfg cfg);

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

// FP64 input split into (hi, lo) float pairs: 16-byte loads and stores when
// x is 16-byte aligned (the output buffer always is)
__global__ void __launch_bounds__(256) k_split_f64(const double* __restrict__ x, float2* __restrict__ xs, long long n) {
  const long long n2 = n >> 1;
  const double2* __restrict__ x2 = reinterpret_cast<const double2*>(x);
  float4* __restrict__ xs4 = reinterpret_cast<float4*>(xs);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
    const double2 v = __ldcs(x2 + i);
    const float2 a = split_f64(v.x), b = split_f64(v.y);
    xs4[i] = make_float4(a.x, a.y, b.x, b.y);
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) xs[n - 1] = split_f64(x[n - 1]);
}

// element-wise variant for an x that is only 8-byte aligned
__global__ void __launch_bounds__(256) k_split_f64_scalar(const double* __restrict__ x, float2* __restrict__ xs, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    xs[i] = split_f64(__ldcs(x + i));
}

// FP64 inputs are split into float pairs in per-call scratch from one
// library pool per device whose release threshold keeps its memory: calls of
// one plan on different streams get separate buffers, and inside a stream
// capture the allocation and release become the graph's own memory nodes.
constexpr int kMaxDevices = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[kMaxDevices] = {};

static cudaError_t scratch_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps pp = {};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = dev;
    cudaMemPool_t m = nullptr;
    e = cudaMemPoolCreate(&m, &pp);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(m, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(m);
      return e;
    }
    g_pool[dev] = m;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

int scratch_alloc(Scratch& b, size_t bytes, cudaStream_t s) {
  cudaMemPool_t m = nullptr;
  cudaError_t e = scratch_pool(&m);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&b.ptr, std::max<size_t>(bytes, 16), m, s);
  if (e != cudaSuccess) {
    b.ptr = nullptr;
    return cuda_fail(e, "FP64 split scratch");
  }
  b.s = s;
  return HM_OK;
}

// hand the pools' unused memory back (allocations still queued keep theirs)
void scratch_trim() {
  std::lock_guard<std::mutex> g(g_pool_mu);
  for (cudaMemPool_t m : g_pool)
    if (m) cudaMemPoolTrimTo(m, 0);
}

cudaError_t split_into(const void* x, void* xs, long long n, cudaStream_t s) {
  const long long grid = std::max<long long>(1, std::min<long long>((n / 2 + 255) / 256, (long long)num_sms() * 8));
  if (((uintptr_t)x % 16) == 0 && ((uintptr_t)xs % 16) == 0)
    k_split_f64<<<(unsigned)grid, 256, 0, s>>>((const double*)x, (float2*)xs, n);
  else
    k_split_f64_scalar<<<(unsigned)grid, 256, 0, s>>>((const double*)x, (float2*)xs, n);
  return cudaGetLastError();
}

int split_vector(const void* x, long long n, cudaStream_t s, Scratch& b, const float2** out) {
  int rc = scratch_alloc(b, (size_t)n * sizeof(float2), s);
  if (rc) return rc;
  cudaError_t e = split_into(x, b.ptr, n, s);
  if (e != cudaSuccess) return cuda_fail(e, "FP64 split launch");
  *out = (const float2*)b.ptr;
  return HM_OK;
}

// y = H x (or H^T x) on stream s. Kernel: cfg.kern = 2 the tile kernel (an
// autotuner candidate; on the benchmark workloads it executes about twice the
// general kernel's instructions per state), otherwise the general kernel.
int apply_on(Plan* p, bool transpose, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s,
             TuneCfg cfg, bool native_f64) {
  if (p->sector) return launch_sector(p, x, y, nvec, dt, s);  // the Lanczos driver on a sector plan
  const KPlan& k = transpose ? p->kt : p->k;
  const KTile* tk = cfg.kern == 2 ? get_tile(p, nvec, transpose, s) : nullptr;
  if (cfg.kern == 2 && !tk && cfg.strict) {
    set_error("this plan has no tile form for that nvec (or its tables cannot be built during stream capture)");
    return HM_ERR_UNSUPPORTED;
  }
  // a tuned tile choice whose tables are unavailable (e.g. first use inside a
  // stream capture) runs the general kernel with its default shape
  TuneCfg gcfg = cfg;
  if (cfg.kern == 2) gcfg = TuneCfg{};
  cudaError_t e;
  const void* xin = x;
  Scratch xsb;
  if (dt == HM_F64 && !native_f64) {
    const float2* xs = nullptr;
    int rc = split_vector(x, p->D * nvec, s, xsb, &xs);
    if (rc) return rc;
    xin = xs;
  }
  e = cudaErrorInvalidConfiguration;
  if (tk) {
    if (dt == HM_F32) e = launch_tile_t<AR_F32>(*tk, xin, y, s, cfg);
    else if (native_f64) e = launch_tile_t<AR_F64>(*tk, xin, y, s, cfg);
    else e = launch_tile_t<AR_DF64>(*tk, xin, y, s, cfg);
    if (e == cudaErrorInvalidConfiguration && cfg.strict) {
      set_error("tile kernel needs more shared memory than a CTA has");
      return HM_ERR_UNSUPPORTED;
    }
  }
  if (e == cudaErrorInvalidConfiguration) {
    if (dt == HM_F32) e = launch_apply_t<AR_F32>(k, xin, y, nvec, s, gcfg);
    else if (native_f64) e = launch_apply_t<AR_F64>(k, xin, y, nvec, s, gcfg);
    else e = launch_apply_t<AR_DF64>(k, xin, y, nvec, s, gcfg);
  }
  if (e != cudaSuccess) return cuda_fail(e, "apply launch");
  return HM_OK;
}

// y_re -= sg t_im, y_im += sg t_re on (re, im) pairs: y = H_re x + sg i H_im x
// from y = H_re x and t = H_im x
template <class T>
__global__ void k_cmix(T* __restrict__ y, const T* __restrict__ t, T sg, long long npairs) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npairs;
       i += (long long)gridDim.x * blockDim.x) {
    const T tr = t[2 * i], ti = t[2 * i + 1];
    y[2 * i] = y[2 * i] - sg * ti;
    y[2 * i + 1] = y[2 * i + 1] + sg * tr;
  }
}

// Complex H = H_re + i H_im: two real applies on the 2 * nvec (re, im)
// columns, then one combining pass. The adjoint H^dagger = H_re^T - i H_im^T.
int apply_complex(Plan* p, bool adjoint, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s) {
  const long long nc = 2 * nvec;
  int rc = apply_on(p, adjoint, x, y, nc, dt, s, tuned_cfg(p, dt, nc), false);
  if (rc) return rc;
  Scratch tb;
  const long long n = vec_states(p) * nc;
  rc = scratch_alloc(tb, (size_t)n * (dt == HM_F32 ? 4 : 8), s);
  if (rc) return rc;
  rc = apply_on(p->im, adjoint, x, tb.ptr, nc, dt, s, tuned_cfg(p->im, dt, nc), false);
  if (rc) return rc;
  const long long np = n / 2;
  const int grid = (int)std::max<long long>(1, std::min<long long>((np + 255) / 256, (long long)num_sms() * 8));
  if (dt == HM_F32)
    k_cmix<float><<<grid, 256, 0, s>>>((float*)y, (const float*)tb.ptr, adjoint ? -1.0f : 1.0f, np);
  else
    k_cmix<double><<<grid, 256, 0, s>>>((double*)y, (const double*)tb.ptr, adjoint ? -1.0 : 1.0, np);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "complex combine");
  return HM_OK;
}

int launch_apply(Plan* p, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s, TuneCfg cfg) {
  return apply_on(p, false, x, y, nvec, dt, s, cfg, false);
}

// Nothing to upload: each launch carries the members' current plans in its
// kernel parameters.
int batch_setup(Plan* b) {
  (void)b;
  return HM_OK;
}

// Instances with enough work to fill the GPU on their own (at least two
// chunk items per resident CTA) run as plain launches of the single-plan
// kernel, whose plan fields are constant-bank operands at fixed offsets; the
// rest share one persistent work-queue launch, which replaces their
// under-filled launches.
static bool fills_gpu(const Plan* p, long long nvec) {
  const long long items = p->nblk * (((long long)p->B * nvec + 2047) / 2048);
  return items >= 2LL * 4 * num_sms();
}

int launch_batch(Plan* b, const void* const* xs, void* const* ys, long long nvec, hm_dtype dt, cudaStream_t s) {
  std::vector<const Plan*> mem;
  std::vector<const void*> sx;
  std::vector<void*> sy;
  // FP64: the queue members' inputs are split into one scratch allocation
  Scratch xsb;
  std::vector<size_t> at(b->members.size(), 0);
  if (dt == HM_F64) {
    size_t total = 0;
    for (size_t i = 0; i < b->members.size(); ++i) {
      const Plan* p = b->members[i];
      if (fills_gpu(p, nvec)) continue;
      at[i] = total;
      total += ((size_t)(p->D * nvec) * sizeof(float2) + 255) & ~size_t(255);
    }
    if (total) {
      int rc = scratch_alloc(xsb, total, s);
      if (rc) return rc;
    }
  }
  for (size_t i = 0; i < b->members.size(); ++i) {
    Plan* p = b->members[i];
    if (fills_gpu(p, nvec)) {
      int rc = apply_on(p, false, xs[i], ys[i], nvec, dt, s, tuned_cfg(p, dt, nvec), false);
      if (rc) return rc;
      continue;
    }
    mem.push_back(p);
    sy.push_back(ys[i]);
    if (dt == HM_F32) {
      sx.push_back(xs[i]);
    } else {
      void* buf = (char*)xsb.ptr + at[i];
      cudaError_t e = split_into(xs[i], buf, p->D * nvec, s);
      if (e != cudaSuccess) return cuda_fail(e, "batch split");
      sx.push_back(buf);
    }
  }
  if (mem.empty()) return HM_OK;
  cudaError_t e = dt == HM_F32 ? launch_batch_t<AR_F32>(mem, sx.data(), sy.data(), nvec, s)
                               : launch_batch_t<AR_DF64>(mem, sx.data(), sy.data(), nvec, s);
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  return HM_OK;
}

}  // namespace hm
