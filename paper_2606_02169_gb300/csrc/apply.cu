// Host entry points of the apply path: dtype dispatch, the FP64 split pass,
// device properties and the batched launch. The kernels live in
// apply_kernel.cuh and are instantiated per arithmetic policy and variant in
// the apply_*.cu units (apply_launch.cuh).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "apply_kernel.cuh"

namespace hm {

template <int AR>
cudaError_t launch_apply_cx_t(const KPlan& kr, const KPlan& ki, const void* x, void* y, long long nvec,
                              cudaStream_t st, int ctas, KGate gate, bool conj, bool cap);

template <int AR, bool VI>
cudaError_t launch_apply_t(const KPlan& k, const void* x, void* y, long long nvec, cudaStream_t st, TuneCfg cfg);
template <int AR>
cudaError_t launch_batch_t(const std::vector<const Plan*>& members, const void* const* xs, void* const* ys,
                           long long nvec, cudaStream_t st);
template <int AR>
cudaError_t launch_tile_t(const KTile& k, const void* x, void* y, cudaStream_t st, TuneCfg cfg);
template <int AR>
cudaError_t launch_stream_t(const KPlan& k, const void* x, void* y, long long nvec, cudaStream_t st, TuneCfg cfg);
template <int AR, bool VI>
cudaError_t launch_apply_pf_t(const KPlan& k, const void* x, void* y, long long nvec, cudaStream_t st, TuneCfg cfg);

// The general kernel (PF: prefetching) with the per-thread group factor
// where the launch asks for it and the plan's groups allow it (FP32 and
// double-float scalar policies).
template <int AR, bool PF>
static cudaError_t general_t(const KPlan& k, const void* x, void* y, long long nvec, cudaStream_t s,
                             const TuneCfg& c) {
  if constexpr (AR == AR_F32 || AR == AR_DF64) {
    if (c.vinv && groups_invariant(k, nvec))
      return PF ? launch_apply_pf_t<AR, true>(k, x, y, nvec, s, c) : launch_apply_t<AR, true>(k, x, y, nvec, s, c);
  }
  return PF ? launch_apply_pf_t<AR, false>(k, x, y, nvec, s, c) : launch_apply_t<AR, false>(k, x, y, nvec, s, c);
}

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
// x is 16-byte aligned (the output buffer always is). With range != NULL an
// element outside the double-float window sets *range.
// |v| outside [lo, hi) with v != 0 (lo, hi the bit patterns of the positive
// window ends: for non-negative doubles the bit patterns order like the
// values, and Inf and NaN patterns lie above every finite hi)
__device__ __forceinline__ bool outside_df_window(double v, unsigned long long lo, unsigned long long hi) {
  const unsigned long long a = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
  return a != 0ull && (a < lo || a >= hi);
}

__global__ void __launch_bounds__(256) k_split_f64(const double* __restrict__ x, float2* __restrict__ xs, long long n,
                                                   int* range, unsigned long long wlo, unsigned long long whi) {
  const long long n2 = n >> 1;
  const double2* __restrict__ x2 = reinterpret_cast<const double2*>(x);
  float4* __restrict__ xs4 = reinterpret_cast<float4*>(xs);
  bool bad = false;
  const long long st = (long long)gridDim.x * blockDim.x;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i + 3 * st < n2; i += 4 * st) {  // four 16-byte loads in flight per thread
    double2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = __ldcs(x2 + i + u * st);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 a = split_f64(v[u].x), b = split_f64(v[u].y);
      bad |= outside_df_window(v[u].x, wlo, whi) | outside_df_window(v[u].y, wlo, whi);
      xs4[i + u * st] = make_float4(a.x, a.y, b.x, b.y);
    }
  }
  for (; i < n2; i += st) {
    const double2 v = __ldcs(x2 + i);
    const float2 a = split_f64(v.x), b = split_f64(v.y);
    bad |= outside_df_window(v.x, wlo, whi) | outside_df_window(v.y, wlo, whi);
    xs4[i] = make_float4(a.x, a.y, b.x, b.y);
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    xs[n - 1] = split_f64(x[n - 1]);
    bad |= outside_df_window(x[n - 1], wlo, whi);
  }
  if (range && bad) atomicOr(range, 1);
}

// element-wise variant for an x that is only 8-byte aligned
__global__ void __launch_bounds__(256) k_split_f64_scalar(const double* __restrict__ x, float2* __restrict__ xs,
                                                          long long n, int* range, unsigned long long wlo,
                                                          unsigned long long whi) {
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = __ldcs(x + i);
    xs[i] = split_f64(v);
    bad |= outside_df_window(v, wlo, whi);
  }
  if (range && bad) atomicOr(range, 1);
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

static unsigned long long dbits(double v) {
  unsigned long long u;
  std::memcpy(&u, &v, 8);
  return u;
}

cudaError_t split_into(const void* x, void* xs, long long n, cudaStream_t s, int* range, double xlo, double xhi) {
  const long long grid = std::max<long long>(1, std::min<long long>((n / 2 + 255) / 256, (long long)num_sms() * 8));
  const unsigned long long wlo = dbits(xlo), whi = dbits(xhi);
  if (((uintptr_t)x % 16) == 0 && ((uintptr_t)xs % 16) == 0)
    k_split_f64<<<(unsigned)grid, 256, 0, s>>>((const double*)x, (float2*)xs, n, range, wlo, whi);
  else
    k_split_f64_scalar<<<(unsigned)grid, 256, 0, s>>>((const double*)x, (float2*)xs, n, range, wlo, whi);
  return cudaGetLastError();
}

cudaError_t split_into(const void* x, void* xs, long long n, cudaStream_t s) {
  return split_into(x, xs, n, s, nullptr, 0.0, 0.0);
}

int split_vector(const void* x, long long n, cudaStream_t s, Scratch& b, const float2** out, const int** range,
                 double xlo, double xhi) {
  const size_t pairs = ((size_t)n * sizeof(float2) + 255) & ~size_t(255);
  int rc = scratch_alloc(b, pairs + (range ? 256 : 0), s);
  if (rc) return rc;
  int* flag = nullptr;
  if (range) {
    flag = (int*)((char*)b.ptr + pairs);
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "FP64 range flag");
    *range = flag;
  }
  cudaError_t e = split_into(x, b.ptr, n, s, flag, xlo, xhi);
  if (e != cudaSuccess) return cuda_fail(e, "FP64 split launch");
  *out = (const float2*)b.ptr;
  return HM_OK;
}

static bool aligned(const void* p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

// The general kernel with the widest policy the call allows: 4 or 2
// right-hand sides of one state per element when nvec is a multiple and the
// vectors are aligned to the wider loads (bit-identical to the scalar
// policy), else one element per thread.
static cudaError_t launch_general(const KPlan& k, const void* x, void* y, long long nvec, hm_dtype dt, bool native,
                                  cudaStream_t s, const TuneCfg& c) {
  if (dt == HM_F32) {
    if (!c.scalar && nvec % 4 == 0 && aligned(x, 16) && aligned(y, 16))
      return launch_apply_t<AR_F32V4, false>(k, x, y, nvec / 4, s, c);
    if (!c.scalar && nvec % 2 == 0 && aligned(x, 8) && aligned(y, 8))
      return launch_apply_t<AR_F32V2, false>(k, x, y, nvec / 2, s, c);
    return general_t<AR_F32, false>(k, x, y, nvec, s, c);
  }
  if (native) return launch_apply_t<AR_F64, false>(k, x, y, nvec, s, c);
  if (!c.scalar && nvec % 2 == 0 && aligned(x, 16) && aligned(y, 16))
    return launch_apply_t<AR_DF64V2, false>(k, x, y, nvec / 2, s, c);
  return general_t<AR_DF64, false>(k, x, y, nvec, s, c);
}

// Page-locked host memory (reached by kernels over the CPU-GPU link)?
bool host_resident(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// dst = src, n 4-byte words, one pass (src may be pinned host memory); V4:
// src and dst 16-byte aligned, 16-byte accesses for all but the tail
template <bool V4>
__global__ void k_copy_words(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, long long n) {
  const long long n4 = V4 ? n / 4 : 0;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  if constexpr (V4) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (long long i = t0; i < n4; i += st) d4[i] = s4[i];
  }
  for (long long i = 4 * n4 + t0; i < n; i += st) dst[i] = src[i];
}

// y = H x (or H^T x) on stream s. Kernels: cfg.kern = 0 or 1 the general
// kernel (on the plan's low block, or with cfg.small on the small one), 2 the
// tile kernel, 3 the staged kernel (autotuner candidates). A strict request
// (hm_apply_ex) never falls back to another kernel.
int apply_on(Plan* p, bool transpose, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s,
             TuneCfg cfg, bool native_f64) {
  if (p->sector) return launch_sector(p, x, y, nvec, dt, s);  // the Lanczos driver on a sector plan
  // vectors in pinned host memory: FP64 x is read once by the split pass
  // below; FP32 x is first copied once into device scratch (the kernels read
  // each element once per hop); y is written once by the kernel. The split
  // into two passes (whose second pass reads y back) is not used for host y.
  Scratch xstage;
  if (dt == HM_F32 && host_resident(x)) {
    const long long n = vec_states(p) * nvec;
    int rc = scratch_alloc(xstage, (size_t)n * 4, s);
    if (rc) return rc;
    const long long grid = std::max<long long>(1, std::min<long long>((n / 4 + 255) / 256, (long long)num_sms() * 8));
    if (((uintptr_t)x % 16) == 0)
      k_copy_words<true><<<(unsigned)grid, 256, 0, s>>>((const uint32_t*)x, (uint32_t*)xstage.ptr, n);
    else
      k_copy_words<false><<<(unsigned)grid, 256, 0, s>>>((const uint32_t*)x, (uint32_t*)xstage.ptr, n);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return cuda_fail(e0, "host x staging");
    x = xstage.ptr;
  }
  if (cfg.split && host_resident(y)) {
    if (cfg.strict) {
      set_error("the top-site split reads y back: not for y in host memory");
      return HM_ERR_UNSUPPORTED;
    }
    cfg.split = 0;
  }
  const KPlan& k = transpose ? p->kt : p->k;
  const StreamSet* ss = cfg.kern == 3 ? get_stream(p, nvec, s) : nullptr;
  // the general kernel on the small low block (the staged kernel's tables)
  const bool want_small = (cfg.kern == 0 || cfg.kern == 1) && cfg.small;
  const StreamSet* small = want_small ? get_stream(p, nvec, s) : nullptr;
  if (want_small && !small && cfg.strict) {
    set_error("this plan has no small-block tables for that nvec");
    return HM_ERR_UNSUPPORTED;
  }
  const KPlan& kg = small ? (transpose ? small->kt : small->k) : k;
  if (small && !small->df_ok && dt == HM_F64 && !cfg.presplit) native_f64 = true;
  if (cfg.kern == 3 && !ss && cfg.strict) {
    set_error("this plan has no staged form for that nvec (a site above the slot size, or tables that cannot be "
              "built during stream capture)");
    return HM_ERR_UNSUPPORTED;
  }
  // top-site split (general kernel on the plan's own low block)
  const SplitSet* sp = nullptr;
  if (cfg.split && (cfg.kern == 0 || cfg.kern == 1) && !small && !native_f64) {
    const int T = cfg.split_T ? cfg.split_T : split_top_sites(p, nvec, dt == HM_F32 ? 4 : 8);
    sp = T > 0 ? get_split(p, T, s) : nullptr;
    if (sp && dt == HM_F64 && !cfg.presplit && !sp->df_ok) sp = nullptr;
  }
  if (cfg.split && !sp && cfg.strict) {
    set_error("this plan has no top-site split for that request (no term moves a leading site's digit, a "
              "pass without terms, a leading site inside the low block, native FP64, or a stream capture)");
    return HM_ERR_UNSUPPORTED;
  }
  const KTile* tk = cfg.kern == 2 ? get_tile(p, nvec, transpose, s) : nullptr;
  if (cfg.kern == 2 && !tk && cfg.strict) {
    set_error("this plan has no tile form for that nvec (or its tables cannot be built during stream capture)");
    return HM_ERR_UNSUPPORTED;
  }
  // a tuned choice whose tables are unavailable (e.g. first use inside a
  // stream capture) runs the general kernel with its default shape
  TuneCfg gcfg = cfg;
  if (cfg.kern == 2 || cfg.kern == 3) gcfg = TuneCfg{};
  cudaError_t e;
  const void* xin = x;
  Scratch xsb;
  // FP64 storage: double-float arithmetic on the split x, unless a
  // coefficient lies outside its window (native FP64 throughout) or an input
  // element does (the split flags it on the device; the double-float launch
  // then stands down and a native FP64 launch of the same apply runs)
  if (dt == HM_F64 && !native_f64 && !cfg.presplit && (!p->df_ok || (ss && !ss->df_ok))) native_f64 = true;
  const int* range = nullptr;
  if (dt == HM_F64 && !native_f64 && !cfg.presplit) {
    // the input window of the tables this call uses (the narrower of the two)
    double xlo = p->df_xlo, xhi = p->df_xhi;
    for (const StreamSet* t : {ss, small})
      if (t) {
        xlo = std::max(xlo, t->df_xlo);
        xhi = std::min(xhi, t->df_xhi);
      }
    if (sp) {
      xlo = std::max(xlo, sp->df_xlo);
      xhi = std::min(xhi, sp->df_xhi);
    }
    const float2* xs = nullptr;
    int rc = split_vector(x, vec_states(p) * nvec, s, xsb, &xs, &range, xlo, xhi);
    if (rc) return rc;
    xin = xs;
    cfg.gate = gcfg.gate = range;
    cfg.gate_run = gcfg.gate_run = 0;
  }
  e = cudaErrorInvalidConfiguration;
  if (ss) {
    const KPlan& ks = transpose ? ss->kt : ss->k;
    if (dt == HM_F32) e = launch_stream_t<AR_F32>(ks, xin, y, nvec, s, cfg);
    else if (native_f64) e = launch_stream_t<AR_F64>(ks, xin, y, nvec, s, cfg);
    else e = launch_stream_t<AR_DF64>(ks, xin, y, nvec, s, cfg);
    if (e == cudaErrorInvalidConfiguration && cfg.kern == 3 && cfg.strict) {
      set_error("staged kernel needs more shared memory than a CTA has");
      return HM_ERR_UNSUPPORTED;
    }
    if (e == cudaErrorInvalidConfiguration) gcfg = TuneCfg{};
  }
  if (tk) {
    if (dt == HM_F32) e = launch_tile_t<AR_F32>(*tk, xin, y, s, cfg);
    else if (native_f64) e = launch_tile_t<AR_F64>(*tk, xin, y, s, cfg);
    else e = launch_tile_t<AR_DF64>(*tk, xin, y, s, cfg);
    if (e == cudaErrorInvalidConfiguration && cfg.strict) {
      set_error("tile kernel needs more shared memory than a CTA has");
      return HM_ERR_UNSUPPORTED;
    }
  }
  // the general kernel's plan: the whole operator, or pass A of the split
  const KPlan& kA = sp ? (transpose ? sp->kat : sp->ka) : kg;
  if (e == cudaErrorInvalidConfiguration && gcfg.pf) {
    if (dt == HM_F32) e = general_t<AR_F32, true>(kA, xin, y, nvec, s, gcfg);
    else if (native_f64) e = launch_apply_pf_t<AR_F64, false>(kA, xin, y, nvec, s, gcfg);
    else e = general_t<AR_DF64, true>(kA, xin, y, nvec, s, gcfg);
    if (e == cudaErrorInvalidConfiguration && cfg.strict) {
      set_error("prefetching general kernel needs more shared memory than a CTA has");
      return HM_ERR_UNSUPPORTED;
    }
  }
  if (e == cudaErrorInvalidConfiguration) e = launch_general(kA, xin, y, nvec, dt, native_f64, s, gcfg);
  if (e == cudaSuccess && sp) {
    // pass B adds the top-site hops to y; default launch shape, same gate
    TuneCfg bc{};
    bc.gate = gcfg.gate;
    bc.gate_run = gcfg.gate_run;
    bc.scalar = gcfg.scalar;
    e = launch_general(transpose ? sp->kbt : sp->kb, xin, y, nvec, dt, native_f64, s, bc);
  }
  if (e != cudaSuccess) return cuda_fail(e, "apply launch");
  if (range) {  // native FP64 fallback, runs only when the split flagged x
    TuneCfg fb{};
    fb.gate = range;
    fb.gate_run = 1;
    e = cudaErrorInvalidConfiguration;
    if (ss) e = launch_stream_t<AR_F64>(transpose ? ss->kt : ss->k, x, y, nvec, s, fb);
    if (e == cudaErrorInvalidConfiguration) e = launch_apply_t<AR_F64, false>(k, x, y, nvec, s, fb);
    if (e != cudaSuccess) return cuda_fail(e, "apply launch (FP64 fallback)");
  }
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

// One pass over both real operators (apply_cx.cuh): FP32 storage on float
// (re, im) pairs; FP64 storage in double-float on the split x, with the
// native FP64 pass gated on the split's range flag (as in apply_on), or
// native FP64 throughout. 1: the call does not allow it (vectors not aligned
// to one complex element, FP32 x in host memory, lists beyond shared memory).
static int apply_complex_fused(Plan* p, bool adjoint, const void* x, void* y, long long nvec, hm_dtype dt,
                               cudaStream_t s, bool native, int ctas, bool cap) {
  const KPlan& kr = adjoint ? p->kt : p->k;
  const KPlan& ki = adjoint ? p->im->kt : p->im->k;
  const uintptr_t el = dt == HM_F32 ? 8 : 16;
  if (!aligned(x, el) || !aligned(y, el) || (dt == HM_F32 && host_resident(x))) return 1;
  if (!cx_compatible(kr, ki) || cx_lists_bytes<AR_DF64V2>(kr) + cx_lists_bytes<AR_DF64V2>(ki) > 227 * 1024) return 1;
  cudaError_t e;
  if (dt == HM_F32) {
    e = launch_apply_cx_t<AR_F32V2>(kr, ki, x, y, nvec, s, ctas, KGate{nullptr, 0}, adjoint, cap);
  } else if (native || !p->df_ok || !p->im->df_ok) {
    e = launch_apply_cx_t<AR_F64V2>(kr, ki, x, y, nvec, s, ctas, KGate{nullptr, 0}, adjoint, cap);
  } else {
    Scratch xsb;
    const float2* xs = nullptr;
    const int* range = nullptr;
    int rc = split_vector(x, vec_states(p) * nvec * 2, s, xsb, &xs, &range, std::max(p->df_xlo, p->im->df_xlo),
                          std::min(p->df_xhi, p->im->df_xhi));
    if (rc) return rc;
    e = launch_apply_cx_t<AR_DF64V2>(kr, ki, xs, y, nvec, s, ctas, KGate{range, 0}, adjoint, cap);
    if (e == cudaSuccess)  // native FP64 pass, runs only when the split flagged x
      e = launch_apply_cx_t<AR_F64V2>(kr, ki, x, y, nvec, s, ctas, KGate{range, 1}, adjoint, cap);
    if (e == cudaErrorInvalidConfiguration) return cuda_fail(e, "complex apply launch");
  }
  if (e == cudaErrorInvalidConfiguration) {
    cudaGetLastError();
    return 1;
  }
  if (e != cudaSuccess) return cuda_fail(e, "complex apply launch");
  return HM_OK;
}

// Complex H = H_re + i H_im. The adjoint H^dagger = H_re^T - i H_im^T. The
// two-pass form: two real applies on the 2 * nvec (re, im) columns, then
// one combining pass. Untuned plans take the two-pass form: measured on the
// Dzyaloshinskii-Moriya ring (N = 26) it is as fast as the one-pass kernel
// for complex128 and faster for complex64.
constexpr int kCxDefaultForm = 2;

int apply_complex(Plan* p, bool adjoint, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s,
                  int mode, bool native, int ctas, bool cap) {
  const long long nc = 2 * nvec;
  int form = 2;
  if (mode == 0) {
    const auto it = p->cx_form.find({(int)dt, nvec});
    form = it == p->cx_form.end() ? kCxDefaultForm : it->second;
  } else if (mode == 2) {
    form = cap ? 1 : 0;
  }
  if (form != 2) {
    const int rc = apply_complex_fused(p, adjoint, x, y, nvec, dt, s, native, ctas, form == 1);
    if (rc != 1) return rc;
    if (mode == 2) {
      set_error("the one-pass complex kernel needs x and y aligned to one complex element, FP32 x in device "
                "memory, and both operators' block lists within shared memory");
      return HM_ERR_UNSUPPORTED;
    }
  }
  TuneCfg c0 = tuned_cfg(p, dt, nc), c1 = tuned_cfg(p->im, dt, nc);
  if (mode == 1) {  // an explicit two-pass request: the general kernel's default launch
    c0 = c1 = TuneCfg{};
    c0.ctas = c1.ctas = ctas;
  }
  int rc = apply_on(p, adjoint, x, y, nc, dt, s, c0, native);
  if (rc) return rc;
  Scratch tb;
  const long long n = vec_states(p) * nc;
  rc = scratch_alloc(tb, (size_t)n * (dt == HM_F32 ? 4 : 8), s);
  if (rc) return rc;
  rc = apply_on(p->im, adjoint, x, tb.ptr, nc, dt, s, c1, native);
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
      // the launch hm_apply makes for this member: its tuned choice, or the
      // general kernel's default (the block code the persistent queue shares)
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
  // the widest policy every queued member's vectors allow (bit-identical)
  bool a16 = true, a8 = true;
  for (size_t i = 0; i < mem.size(); ++i) {
    a16 = a16 && aligned(sx[i], 16) && aligned(sy[i], 16);
    a8 = a8 && aligned(sx[i], 8) && aligned(sy[i], 8);
  }
  cudaError_t e;
  if (dt == HM_F32) {
    if (nvec % 4 == 0 && a16) e = launch_batch_t<AR_F32V4>(mem, sx.data(), sy.data(), nvec / 4, s);
    else if (nvec % 2 == 0 && a8) e = launch_batch_t<AR_F32V2>(mem, sx.data(), sy.data(), nvec / 2, s);
    else e = launch_batch_t<AR_F32>(mem, sx.data(), sy.data(), nvec, s);
  } else {
    if (nvec % 2 == 0 && a16) e = launch_batch_t<AR_DF64V2>(mem, sx.data(), sy.data(), nvec / 2, s);
    else e = launch_batch_t<AR_DF64>(mem, sx.data(), sy.data(), nvec, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "batch launch");
  return HM_OK;
}

}  // namespace hm
