// extern "C" boundary of the hm library: argument validation, error codes and
// dispatch to the plan builder and kernels. No torch types cross this line.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <string>

#include "hm_internal.h"

namespace hm {

static thread_local std::string g_err;

void set_error(const std::string& s) { g_err = s; }

int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return (e == cudaErrorMemoryAllocation) ? HM_ERR_OOM : HM_ERR_CUDA;
}

static Plan* as_plan(hm_handle h) {
  Plan* p = reinterpret_cast<Plan*>(h);
  if (!p || p->magic != 0x484d504cU) return nullptr;
  return p;
}


constexpr int kKrylovMax = 128;  // Krylov dimension limit of hm_evolve

static size_t esize(hm_dtype dt) { return dt == HM_F32 ? 4 : 8; }

// Complex storage: every plan holds a real operator (an imaginary matrix
// element is rejected when the plan is built), so the real and imaginary
// parts of a complex vector are applied independently -- nvec complex
// right-hand sides are 2 * nvec interleaved real ones on the same memory.
static void real_view(hm_dtype& dt, long long& nvec) {
  if (dt != HM_C128 && dt != HM_C64) return;
  dt = dt == HM_C128 ? HM_F64 : HM_F32;
  if (nvec > 0 && nvec < (1LL << 40)) nvec *= 2;
}

static bool overlap(const void* a, const void* b, size_t bytes) {
  auto pa = (uintptr_t)a, pb = (uintptr_t)b;
  return pa < pb + bytes && pb < pa + bytes;
}

int check_vec_args(const Plan* p, const void* x, const void* y, long long nvec, hm_dtype dt) {
  if (!p) { set_error("invalid handle"); return HM_ERR_INVALID_ARG; }
  if (p->is_batch) { set_error("batch handle given to a single-plan call"); return HM_ERR_INVALID_ARG; }
  if (dt != HM_F64 && dt != HM_F32) { set_error("dtype must be HM_F64 or HM_F32"); return HM_ERR_INVALID_ARG; }
  if (nvec < 1) { set_error("nvec must be >= 1"); return HM_ERR_INVALID_ARG; }
  if (nvec > (1 << 19)) { set_error("nvec above 2^19 (a low block of B*nvec elements must stay below 2^31)"); return HM_ERR_UNSUPPORTED; }
  if (!x || !y) { set_error("null vector pointer"); return HM_ERR_INVALID_ARG; }
  if (((uintptr_t)x % esize(dt)) || ((uintptr_t)y % esize(dt))) {
    set_error("vector pointers must be aligned to the element size");
    return HM_ERR_INVALID_ARG;
  }
  if ((double)vec_states(p) * (double)nvec > 9.0e18) { set_error("D * nvec overflows int64"); return HM_ERR_OVERFLOW; }
  // device memory, managed memory or page-locked host memory registered with
  // CUDA (kernels reach it through the unified address space); plain
  // pageable host memory is not accepted
  for (const void* v : {x, y}) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, v) != cudaSuccess || a.type == cudaMemoryTypeUnregistered) {
      cudaGetLastError();
      set_error("vectors must be device memory or page-locked (pinned) host memory");
      return HM_ERR_INVALID_ARG;
    }
  }
  if (overlap(x, y, (size_t)(vec_states(p) * nvec) * esize(dt))) {
    set_error("x and y overlap (the pull form needs x read-only while y is written)");
    return HM_ERR_ALIAS;
  }
  return HM_OK;
}

static std::mutex g_tune_mu;
static std::map<std::string, TuneCfg> g_tune_cache;

static std::string tune_signature(const Plan* p, hm_dtype dt, long long nvec) {
  std::string s = std::to_string((int)dt) + "/" + std::to_string(nvec) + "/";
  for (auto& st : p->sites) s += std::to_string(st.dim) + ",";
  s += "/" + std::to_string(p->k.n_hh) + "," + std::to_string(p->k.n_grp) + "," + std::to_string(p->k.n_mem) + "," + std::to_string(p->k.ell_w);
  return s;
}

TuneCfg tuned_cfg(Plan* p, hm_dtype dt, long long nvec) {
  auto it = p->tuned.find({(int)dt, nvec});
  if (it != p->tuned.end()) return it->second;
  std::lock_guard<std::mutex> g(g_tune_mu);
  if (g_tune_cache.empty()) return TuneCfg{};
  auto jt = g_tune_cache.find(tune_signature(p, dt, nvec));
  if (jt == g_tune_cache.end()) return TuneCfg{};
  p->tuned[{(int)dt, nvec}] = jt->second;
  return jt->second;
}

}  // namespace hm

using namespace hm;

extern "C" {

// The companion plan of a complex H (its imaginary part), rebuilt from the
// current terms; dropped when the term list is real.
static void destroy_plan(Plan* p);
static int build_companion(Plan* p) {
  if (!p->complex_h) {
    if (p->im) destroy_plan(p->im);
    p->im = nullptr;
    return HM_OK;
  }
  if (!p->im) {
    p->im = new Plan();
    p->im->N = p->N;
    p->im->sites = p->sites;
    p->im->device = p->device;
    p->im->part = 1;
  }
  p->im->terms = p->terms;
  return build_plan(p->im);
}

static int needs_complex_storage() {
  set_error("the term list has imaginary matrix elements (e.g. a lone Sy): use HM_C128 or HM_C64 storage");
  return HM_ERR_COMPLEX_REQUIRED;
}

int hm_create(const hm_site* sites, int32_t nsites, const hm_term* terms, int32_t nterms,
              hm_handle* out) {
  if (!out) { set_error("out is NULL"); return HM_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!sites || nsites < 1 || nterms < 0 || (nterms > 0 && !terms)) {
    set_error("sites/terms arrays invalid");
    return HM_ERR_INVALID_ARG;
  }
  if (nsites > kMaxSites) { set_error("nsites must be in [1, 64]"); return HM_ERR_INVALID_ARG; }
  Plan* p = new Plan();
  p->N = nsites;
  p->sites.assign(sites, sites + nsites);
  p->terms.assign(terms, terms + nterms);
  cudaGetDevice(&p->device);
  int rc = plan_check(p);
  if (rc == HM_OK) rc = build_plan(p);
  if (rc == HM_OK) rc = build_companion(p);
  if (rc != HM_OK) {
    destroy_plan(p);
    return rc;
  }
  *out = reinterpret_cast<hm_handle>(p);
  return HM_OK;
}

int hm_create_sector(const hm_site* sites, int32_t nsites, const hm_term* terms, int32_t nterms,
                     int64_t digit_total, hm_handle* out) {
  if (!out) { set_error("out is NULL"); return HM_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!sites || nsites < 1 || nterms < 0 || (nterms > 0 && !terms)) {
    set_error("sites/terms arrays invalid");
    return HM_ERR_INVALID_ARG;
  }
  if (nsites > kMaxSites) { set_error("nsites must be in [1, 64]"); return HM_ERR_INVALID_ARG; }
  Plan* p = new Plan();
  p->N = nsites;
  p->sites.assign(sites, sites + nsites);
  p->terms.assign(terms, terms + nterms);
  p->sector = true;
  p->sec_total = digit_total;
  cudaGetDevice(&p->device);
  int rc = plan_check(p);
  if (rc == HM_OK) rc = build_plan(p);   // builds the sector tables too
  if (rc == HM_OK && p->complex_h) {
    set_error("complex term lists (imaginary matrix elements) are not available for sector plans");
    rc = HM_ERR_UNSUPPORTED;
  }
  if (rc != HM_OK) {
    free_plan_device(p);
    free_sector(p);
    delete p;
    return rc;
  }
  *out = reinterpret_cast<hm_handle>(p);
  return HM_OK;
}

static int no_sector(const Plan* p, const char* what) {
  if (p && p->sector) {
    set_error(std::string(what) + " is not available for sector plans (hm_create_sector)");
    return HM_ERR_UNSUPPORTED;
  }
  return HM_OK;
}

int hm_set_coefficients(hm_handle h, const double* coefs) {
  Plan* p = as_plan(h);
  if (!p || p->is_batch || !coefs) { set_error("invalid handle or coefficients"); return HM_ERR_INVALID_ARG; }
  for (size_t t = 0; t < p->terms.size(); ++t)
    if (!std::isfinite(coefs[t])) { set_error("non-finite coefficient"); return HM_ERR_INVALID_ARG; }
  cudaError_t e = cudaDeviceSynchronize();  // no apply of the old tables may still run
  if (e != cudaSuccess) return cuda_fail(e, "set_coefficients sync");
  std::vector<hm_term> old = p->terms;
  for (size_t t = 0; t < p->terms.size(); ++t) p->terms[t].coef = coefs[t];
  int rc = build_plan(p);
  if (rc == HM_OK) rc = build_companion(p);
  if (rc != HM_OK) {
    p->terms = old;
    int rc2 = build_plan(p);
    if (rc2 == HM_OK) rc2 = build_companion(p);
    (void)rc2;
  }
  return rc;
}

int64_t hm_dim(hm_handle h) {
  Plan* p = as_plan(h);
  if (!p) return HM_ERR_INVALID_ARG;
  return vec_states(p);
}

int32_t hm_num_terms(hm_handle h) {
  Plan* p = as_plan(h);
  if (!p) return HM_ERR_INVALID_ARG;
  return (int32_t)p->terms.size();
}

int hm_apply(hm_handle h, const void* x, void* y, int64_t nvec_in, hm_dtype dtype, void* stream) {
  Plan* p = as_plan(h);
  const bool cx = dtype == HM_C128 || dtype == HM_C64;
  long long nvec = nvec_in;
  real_view(dtype, nvec);
  int rc = check_vec_args(p, x, y, nvec, dtype);
  if (rc) return rc;
  if (p->im) return cx ? apply_complex(p, false, x, y, nvec / 2, dtype, (cudaStream_t)stream) : needs_complex_storage();
  if (p->sector) return launch_sector(p, x, y, nvec, dtype, (cudaStream_t)stream);
  return launch_apply(p, x, y, nvec, dtype, (cudaStream_t)stream, tuned_cfg(p, dtype, nvec));
}

int hm_apply_ex(hm_handle h, const void* x, void* y, int64_t nvec_in, hm_dtype dtype, int32_t flags,
                int32_t ctas, void* stream) {
  Plan* p = as_plan(h);
  const bool cx = dtype == HM_C128 || dtype == HM_C64;
  long long nvec = nvec_in;
  real_view(dtype, nvec);
  int rc = check_vec_args(p, x, y, nvec, dtype);
  if (rc) return rc;
  if (p->im) {  // complex H: bits 0 (native FP64), 1 (H^dagger), 2 (register cap), 4 (no effect), 13 (two passes)
    if (flags & ~(1 | 2 | 4 | 16 | 8192)) {
      set_error("hm_apply_ex on a complex H takes flag bits 0, 1, 2, 4 and 13 only");
      return HM_ERR_UNSUPPORTED;
    }
    if ((flags & 4) && (flags & 8192)) {
      set_error("flag bit 2 (the register-capped one-pass kernel) does not combine with bit 13 (two passes)");
      return HM_ERR_INVALID_ARG;
    }
    if (!cx) return needs_complex_storage();
    return apply_complex(p, (flags & 2) != 0, x, y, nvec / 2, dtype, (cudaStream_t)stream, (flags & 8192) ? 1 : 2,
                         (flags & 1) != 0, ctas > 0 ? ctas : 0, (flags & 4) != 0);
  }
  if (p->sector) {  // sector plans: bit 4 selects the per-row kernel, nothing else applies
    if (flags & ~16) {
      set_error("hm_apply_ex on a sector plan takes flag bit 4 (the per-row kernel) only");
      return HM_ERR_UNSUPPORTED;
    }
    return launch_sector(p, x, y, nvec, dtype, (cudaStream_t)stream, (flags & 16) != 0);
  }
  TuneCfg cfg;
  cfg.ctas = ctas > 0 ? ctas : 0;
  cfg.mb = (flags >> 2) & 1;
  cfg.s = (flags >> 8) & 15;
  const bool tile = (flags & 8) != 0, general = (flags & 16) != 0;
  if (tile && general) {
    set_error("flags ask for both kernels");
    return HM_ERR_INVALID_ARG;
  }
  const bool staged = (flags & 32) != 0;
  if (staged && (tile || general)) {
    set_error("flags ask for more than one kernel");
    return HM_ERR_INVALID_ARG;
  }
  cfg.kern = tile ? 2 : (general ? 1 : (staged ? 3 : 0));
  cfg.presplit = (flags >> 6) & 1;
  cfg.small = (flags >> 7) & 1;
  cfg.pf = (flags >> 12) & 1;
  cfg.scalar = (flags >> 13) & 1;
  cfg.split = (flags >> 14) & 1;
  cfg.vinv = (flags >> 15) & 1;
  cfg.split_T = (flags >> 16) & 15;
  if ((cfg.small || cfg.pf || cfg.scalar || cfg.split || cfg.vinv) && (tile || staged)) {
    set_error("flag bits 7, 12, 13, 14 and 15 (small low block, prefetching, one right-hand side per element, "
              "top-site split, one group factor per thread) apply to the general kernel only");
    return HM_ERR_INVALID_ARG;
  }
  if (cfg.split_T && !cfg.split) {
    set_error("flag bits 16..19 (leading sites of a split) need bit 14");
    return HM_ERR_INVALID_ARG;
  }
  if (cfg.split && (cfg.small || (flags & 1))) {
    set_error("the top-site split runs on the plan's own low block with the double-float or FP32 arithmetic");
    return HM_ERR_INVALID_ARG;
  }
  if (cfg.pf && cfg.s && cfg.s != 4 && cfg.s != 6 && cfg.s != 8) {
    set_error("the prefetching general kernel takes 4, 6 or 8 elements per thread");
    return HM_ERR_INVALID_ARG;
  }
  if (cfg.presplit && (dtype != HM_F64 || (flags & 1))) {
    set_error("flag bit 6 (pre-split input) needs HM_F64 storage and the double-float arithmetic");
    return HM_ERR_INVALID_ARG;
  }
  cfg.strict = 1;
  if (tile && cfg.s && cfg.s != 1 && cfg.s != 2 && cfg.s != 4) {
    set_error("tile kernel rows per iteration must be 0 (default), 1, 2 or 4");
    return HM_ERR_INVALID_ARG;
  }
  if (staged && cfg.s) {
    set_error("the staged kernel takes no elements-per-thread setting");
    return HM_ERR_INVALID_ARG;
  }
  if (!tile && cfg.s && cfg.s != 2 && cfg.s != 3 && cfg.s != 4 && cfg.s != 6 && cfg.s != 8) {
    set_error("elements per thread must be 0 (default), 2, 3, 4, 6 or 8");
    return HM_ERR_INVALID_ARG;
  }
  if (!tile && cfg.s) cfg.kern = 1;  // an element count names the general kernel
  if (cfg.kern == 0) cfg.kern = 1;    // no kernel bit: the general kernel
  return apply_on(p, (flags & 2) != 0, x, y, nvec, dtype, (cudaStream_t)stream, cfg, (flags & 1) != 0);
}

int hm_apply_adjoint(hm_handle h, const void* gy, const void* x, void* gx, double* gcoef,
                     int64_t nvec_in, hm_dtype dtype, void* stream) {
  Plan* p = as_plan(h);
  const bool cx = dtype == HM_C128 || dtype == HM_C64;
  long long nvec = nvec_in;
  real_view(dtype, nvec);
  if (!p) { set_error("invalid handle"); return HM_ERR_INVALID_ARG; }
  if (p->sector) {  // sector plan: gx = H^T gy = H gy for a symmetric term list
    if (gcoef || !p->hermitian) {
      set_error("sector plans provide gx only, and only for a symmetric term list");
      return HM_ERR_UNSUPPORTED;
    }
    if (!gx) return HM_OK;
    int rc = check_vec_args(p, gy, gx, nvec, dtype);
    if (rc) return rc;
    return launch_sector(p, gy, gx, nvec, dtype, (cudaStream_t)stream);
  }
  if (p->im) {  // complex H: gx = H^dagger gy only
    if (gcoef) {
      set_error("coupling gradients are not available for a complex H");
      return HM_ERR_UNSUPPORTED;
    }
    if (!gx) return HM_OK;
    if (!cx) return needs_complex_storage();
    int rc = check_vec_args(p, gy, gx, nvec, dtype);
    if (rc) return rc;
    return apply_complex(p, true, gy, gx, nvec / 2, dtype, (cudaStream_t)stream);
  }
  if (!gx && !gcoef) return HM_OK;
  if (gx) {
    int rc = check_vec_args(p, gy, gx, nvec, dtype);
    if (rc) return rc;
  }
  if (gcoef && !p->grad_ok) {
    set_error("a term of this list has imaginary matrix elements: its coupling gradient is undefined");
    return HM_ERR_UNSUPPORTED;
  }
  if (gcoef) {
    int rc = check_vec_args(p, gy, x ? x : gy, nvec, dtype);
    if (rc == HM_ERR_ALIAS) rc = HM_OK;  // gy and x may be the same vector
    if (rc) return rc;
    if (!x) { set_error("x is required for coupling gradients"); return HM_ERR_INVALID_ARG; }
  }
  return launch_adjoint(p, gy, x, gx, gcoef, nvec, dtype, (cudaStream_t)stream);
}

int hm_lanczos(hm_handle h, const void* v0, int32_t steps, hm_dtype dtype, int32_t flags,
               double* alpha, double* beta, int32_t* steps_done, void* psi0_out, double* e0,
               void* stream) {
  Plan* p = as_plan(h);
  if (!p || p->is_batch || !v0 || steps < 1 || !alpha || !beta || !steps_done || !e0) {
    set_error("invalid Lanczos arguments");
    return HM_ERR_INVALID_ARG;
  }
  long long nvec = 1;
  real_view(dtype, nvec);
  if (dtype != HM_F64 && dtype != HM_F32) { set_error("bad dtype"); return HM_ERR_INVALID_ARG; }
  if (p->im && nvec != 2) return needs_complex_storage();
  if (!p->hermitian_c) {
    set_error("Lanczos needs a self-adjoint term list");
    return HM_ERR_NOT_HERMITIAN;
  }
  int sd = 0;
  int rc = run_lanczos(p, v0, steps, dtype, nvec, flags, alpha, beta, &sd, psi0_out, e0, (cudaStream_t)stream);
  *steps_done = sd;
  return rc;
}

int hm_batch_create(const hm_handle* hs, int32_t n, hm_handle* batch_out) {
  if (!batch_out || !hs || n < 1) { set_error("invalid batch arguments"); return HM_ERR_INVALID_ARG; }
  *batch_out = nullptr;
  Plan* b = new Plan();
  b->is_batch = true;
  for (int i = 0; i < n; ++i) {
    Plan* p = as_plan(hs[i]);
    if (!p || p->is_batch || p->sector || p->im) {
      delete b;
      set_error("batch member " + std::to_string(i) + " is not a full-basis plan handle");
      return HM_ERR_INVALID_ARG;
    }
    b->members.push_back(p);
  }
  int rc = batch_setup(b);
  if (rc) {
    delete b;
    return rc;
  }
  *batch_out = reinterpret_cast<hm_handle>(b);
  return HM_OK;
}

int hm_batch_apply(hm_handle batch, const void* const* xs, void* const* ys, int64_t nvec_in,
                   hm_dtype dtype, void* stream) {
  Plan* b = as_plan(batch);
  long long nvec = nvec_in;
  real_view(dtype, nvec);
  if (!b || !b->is_batch || !xs || !ys || nvec < 1) {
    set_error("invalid batch apply arguments");
    return HM_ERR_INVALID_ARG;
  }
  if (dtype != HM_F64 && dtype != HM_F32) { set_error("bad dtype"); return HM_ERR_INVALID_ARG; }
  for (size_t i = 0; i < b->members.size(); ++i) {
    if (b->members[i]->im) {  // a coefficient update made the member complex
      set_error("batch member " + std::to_string(i) + " has imaginary matrix elements; batches hold real plans");
      return HM_ERR_UNSUPPORTED;
    }
    int rc = check_vec_args(b->members[i], xs[i], ys[i], nvec, dtype);
    if (rc) {
      set_error("batch member " + std::to_string(i) + ": " + std::string(hm_last_error()));
      return rc;
    }
  }
  return launch_batch(b, xs, ys, nvec, dtype, (cudaStream_t)stream);
}

static void destroy_plan(Plan* p) {
  if (p->im) destroy_plan(p->im);
  p->im = nullptr;
  free_plan_device(p);
  free_tiles(p);
  free_streams(p);
  free_splits(p);
  free_sector(p);
  if (p->scratch) cudaFree(p->scratch);
  p->magic = 0;
  delete p;
}

int hm_destroy(hm_handle h) {
  Plan* p = as_plan(h);
  if (!p) { set_error("invalid handle"); return HM_ERR_INVALID_ARG; }
  cudaDeviceSynchronize();
  destroy_plan(p);
  scratch_trim();
  return HM_OK;
}

// Autotuner: time the apply variants on scratch vectors -- the general
// kernel's elements per thread S in {2, 3, 4, 6, 8} x register cap (default,
// or one more resident CTA per SM) and the tile kernel's rows per iteration
// {1, 2, 4}, each at its occupancy-sized persistent grid, then the grid
// ladder (1..16 CTAs per SM) for the best of those -- and keep the fastest
// per (dtype, nvec), also in a process-wide cache keyed by the site
// dimensions and channel counts. Each candidate: one untimed launch, then the
// minimum of three event-timed launches.
static int tune_plan(Plan* p, long long nvec, hm_dtype dtype, void* stream);
static int tune_complex(Plan* p, long long ncx, hm_dtype dtype, void* stream);

int hm_tune(hm_handle h, int64_t nvec_in, hm_dtype dtype, void* stream) {
  Plan* p = as_plan(h);
  long long nvec = nvec_in;
  real_view(dtype, nvec);
  if (!p || p->is_batch || nvec < 1 || (dtype != HM_F64 && dtype != HM_F32)) {
    set_error("invalid tune arguments");
    return HM_ERR_INVALID_ARG;
  }
  if (int rc = no_sector(p, "hm_tune")) return rc;
  int rc = tune_plan(p, nvec, dtype, stream);
  // complex H: both real parts are applied to the 2 * nvec columns; then
  // the one-pass complex kernel against the two tuned passes
  if (rc == HM_OK && p->im) rc = tune_plan(p->im, nvec, dtype, stream);
  if (rc == HM_OK && p->im && nvec % 2 == 0) rc = tune_complex(p, nvec / 2, dtype, stream);
  return rc;
}

// Complex H on ncx complex right-hand sides: time the two separately tuned
// real passes with their combine, the one-pass kernel and its
// register-capped variant (one untimed call, then the minimum of three),
// and keep the fastest for apply_complex.
static int tune_complex(Plan* p, long long ncx, hm_dtype dtype, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)p->D * 2 * ncx * esize(dtype);
  void *x = nullptr, *y = nullptr;
  cudaError_t e = cudaMalloc(&x, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "tune scratch x");
  e = cudaMalloc(&y, bytes);
  if (e != cudaSuccess) { cudaFree(x); return cuda_fail(e, "tune scratch y"); }
  cudaMemsetAsync(x, 0, bytes, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = HM_OK;
  auto time_mode = [&](int mode, bool cap) {
    float tmin = 1e30f;
    for (int rep = 0; rep < 4 && rc == HM_OK; ++rep) {
      cudaEventRecord(e0, s);
      rc = apply_complex(p, false, x, y, ncx, dtype, s, mode, false, 0, cap);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = HM_ERR_CUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tmin = std::min(tmin, ms);
    }
    return tmin;
  };
  int form = 2;
  float tbest = time_mode(3, false);
  for (int f = 0; f < 2 && rc == HM_OK; ++f) {
    const float t = time_mode(2, f == 1);
    if (rc == HM_ERR_UNSUPPORTED) {  // the one-pass kernel does not fit this plan or these vectors
      rc = HM_OK;
      break;
    }
    if (t < tbest) {
      tbest = t;
      form = f;
    }
  }
  if (rc == HM_OK) p->cx_form[{(int)dtype, ncx}] = form;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  return rc;
}

// Time the launch variants of one real plan for (nvec, dtype) and store the best.
static int tune_plan(Plan* p, long long nvec, hm_dtype dtype, void* stream) {
  const std::string sig = tune_signature(p, dtype, nvec);
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune_cache.find(sig);
    if (it != g_tune_cache.end()) {
      p->tuned[{(int)dtype, (long long)nvec}] = it->second;
      return HM_OK;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)p->D * nvec * esize(dtype);
  void *x = nullptr, *y = nullptr;
  cudaError_t e = cudaMalloc(&x, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "tune scratch x");
  e = cudaMalloc(&y, bytes);
  if (e != cudaSuccess) { cudaFree(x); return cuda_fail(e, "tune scratch y"); }
  cudaMemsetAsync(x, 0, bytes, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = HM_OK;
  auto time_cfg = [&](TuneCfg c) {
    float tmin = 1e30f;
    for (int rep = 0; rep < 4 && rc == HM_OK; ++rep) {
      cudaEventRecord(e0, s);
      rc = launch_apply(p, x, y, nvec, dtype, s, c);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = HM_ERR_CUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tmin = std::min(tmin, ms);
    }
    return tmin;
  };
  TuneCfg best{};
  best.kern = 1;
  float tbest = time_cfg(best);
  for (int sh : {4, 6, 8}) {
    for (int mb = 0; mb < 2 && rc == HM_OK; ++mb) {
      TuneCfg c;
      c.kern = 1;
      c.pf = 1;
      c.s = sh;
      c.mb = mb;
      c.strict = 1;
      const float t = time_cfg(c);
      if (rc == HM_ERR_UNSUPPORTED) { rc = HM_OK; continue; }
      if (t < tbest) { tbest = t; best = c; }
    }
  }
  if (rc == HM_OK && get_stream(p, nvec, s)) {
    for (int sh : {0, 2, 4}) {
      for (int mb = 0; mb < 2 && rc == HM_OK; ++mb) {
        TuneCfg c;
        c.kern = 1;
        c.small = 1;
        c.s = sh;
        c.mb = mb;
        c.strict = 1;
        const float t = time_cfg(c);
        if (t < tbest) { tbest = t; best = c; }
      }
    }
  }
  if (rc == HM_OK && get_stream(p, nvec, s)) {
    TuneCfg c;
    c.kern = 3;
    c.strict = 1;  // time the staged kernel itself, never a fallback
    const float t = time_cfg(c);
    if (rc == HM_ERR_UNSUPPORTED) rc = HM_OK;
    else if (t < tbest) { tbest = t; best = c; }
  }
  for (int sh : {2, 3, 4, 6, 8}) {
    for (int mb = 0; mb < 2 && rc == HM_OK; ++mb) {
      TuneCfg c;
      c.kern = 1;
      c.s = sh;
      c.mb = mb;
      const float t = time_cfg(c);
      if (t < tbest) { tbest = t; best = c; }
    }
  }
  // the best general-kernel shape with one group factor per thread (a no-op
  // where the plan's groups do not allow it)
  if (rc == HM_OK && best.kern == 1) {
    TuneCfg c = best;
    c.vinv = 1;
    const float t = time_cfg(c);
    if (t < tbest) { tbest = t; best = c; }
  }
  // the best general-kernel shape again as a top-site split, where the
  // vectors are large enough for one
  const int T0 = split_top_sites(p, nvec, esize(dtype));
  if (rc == HM_OK && best.kern == 1 && !best.small && T0 > 0) {
    const TuneCfg base = best;
    for (int T : {T0 - 1, T0, T0 + 1}) {  // the best T sits near the 32 MiB rule
      if (T < 1 || T >= p->N || rc != HM_OK) continue;
      TuneCfg c = base;
      c.split = 1;
      c.split_T = T;
      c.strict = 1;
      const float t = time_cfg(c);
      if (rc == HM_ERR_UNSUPPORTED) rc = HM_OK;
      else if (t < tbest) { tbest = t; best = c; }
    }
  }
  // nvec even: the calls above ran 2 or 4 right-hand sides per lane; one per
  // lane (bit-identical) is a candidate too
  if (nvec % 2 == 0) {
    for (int sh : {4, 6, 8}) {
      for (int mb = 0; mb < 2 && rc == HM_OK; ++mb) {
        TuneCfg c;
        c.kern = 1;
        c.s = sh;
        c.mb = mb;
        c.scalar = 1;
        const float t = time_cfg(c);
        if (t < tbest) { tbest = t; best = c; }
      }
    }
  }
  if (rc == HM_OK && get_tile(p, nvec, false, s)) {
    for (int rs : {1, 2, 4}) {
      if (rc != HM_OK) break;
      TuneCfg c;
      c.kern = 2;
      c.s = rs;
      c.strict = 1;  // time the tile kernel itself, never a fallback
      const float t = time_cfg(c);
      if (rc == HM_ERR_UNSUPPORTED) {  // tile kernel cannot launch for this plan
        rc = HM_OK;
        break;
      }
      if (t < tbest) { tbest = t; best = c; }
    }
  }
  const int sms = num_sms();
  for (int per : {1, 2, 4, 8, 16}) {
    if (rc != HM_OK) break;
    TuneCfg c = best;
    c.ctas = sms * per;
    const float t = time_cfg(c);
    if (t < tbest) { tbest = t; best = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(y);
  if (rc != HM_OK) return rc;
  best.strict = 0;  // a stored choice may fall back (see apply_on)
  p->tuned[{(int)dtype, (long long)nvec}] = best;
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune_cache[sig] = best;
  return HM_OK;
}

/* Device status word; see include/hm.h. */
int hm_device_status(int32_t* status, int32_t clear) {
  if (!status) {
    set_error("status must not be NULL");
    return HM_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "device status sync");
  int v = 0;
  for (auto f : {stream_status_f32, stream_status_df64, stream_status_f64}) {
    int w = 0;
    int rc = f(&w, clear != 0);
    if (rc) return rc;
    v |= w;
  }
  *status = v;
  return HM_OK;
}

/* Launch choice hm_tune stored for (nvec, dtype); see include/hm.h. */
int hm_tuned_config(hm_handle h, int64_t nvec_in, hm_dtype dtype, int32_t* out) {
  Plan* p = as_plan(h);
  const bool cx = dtype == HM_C128 || dtype == HM_C64;
  long long nvec = nvec_in;
  real_view(dtype, nvec);
  if (!p || p->is_batch || !out) {
    set_error("invalid arguments");
    return HM_ERR_INVALID_ARG;
  }
  const TuneCfg c = tuned_cfg(p, dtype, nvec);
  out[0] = c.ctas;
  out[1] = c.s;
  out[2] = c.mb | (c.small << 1) | (c.pf << 2) | (c.scalar << 3) | (c.split << 4) | (c.vinv << 5) |
           (c.split_T << 8);
  if (cx && p->im) {  // complex H: the choice between one pass and two tuned passes
    const auto it = p->cx_form.find({(int)dtype, nvec / 2});
    const int form = it == p->cx_form.end() ? -1 : it->second;
    if (form == 0 || form == 1) out[2] |= 1 << 6;
    if (form == 1) out[2] |= 1 << 7;
  }
  out[3] = c.kern;
  return HM_OK;
}

/* Time evolution y = exp(-i t H) x; see include/hm.h. */
int hm_evolve(hm_handle h, const void* x, void* y, double t, int32_t m, int32_t nsub, int32_t flags,
              hm_dtype dtype, double* err, void* stream) {
  Plan* p = as_plan(h);
  if (dtype != HM_C128 && dtype != HM_C64) {
    set_error("hm_evolve needs complex storage (HM_C128 or HM_C64)");
    return HM_ERR_INVALID_ARG;
  }
  if (m < 1 || m > kKrylovMax || nsub < 1 || !std::isfinite(t) || (flags & ~3)) {
    set_error("hm_evolve needs 1 <= m <= 128, nsub >= 1, a finite t and flags in bits 0..1");
    return HM_ERR_INVALID_ARG;
  }
  long long nvec = 1;
  real_view(dtype, nvec);
  int rc = check_vec_args(p, x, y, nvec, dtype);
  if (rc) return rc;
  if (!p->hermitian_c) {
    set_error("time evolution needs a self-adjoint term list");
    return HM_ERR_NOT_HERMITIAN;
  }
  return run_evolve(p, x, y, t, m, nsub, flags, dtype, err, (cudaStream_t)stream);
}

/* Host-only Krylov propagator coefficients; see include/hm.h. */
int hm_krylov_coefficients(const double* alpha, const double* beta, int32_t m, double tau, double nu, double* c) {
  if (!alpha || !c || m < 1 || m > kKrylovMax || (m > 1 && !beta) || !std::isfinite(tau) || !std::isfinite(nu)) {
    set_error("invalid Krylov coefficient arguments");
    return HM_ERR_INVALID_ARG;
  }
  std::vector<double> a(alpha, alpha + m), b;
  if (m > 1) b.assign(beta, beta + m - 1);
  for (double v : a) if (!std::isfinite(v)) { set_error("non-finite alpha"); return HM_ERR_INVALID_ARG; }
  for (double v : b) if (!std::isfinite(v)) { set_error("non-finite beta"); return HM_ERR_INVALID_ARG; }
  std::vector<double> cc;
  krylov_coeffs(a, b, tau, nu, cc);
  std::copy(cc.begin(), cc.end(), c);
  return HM_OK;
}

const char* hm_strerror(int code) {
  switch (code) {
    case HM_OK: return "ok";
    case HM_ERR_INVALID_ARG: return "invalid argument";
    case HM_ERR_OVERFLOW: return "dimension overflow (D >= 2^62)";
    case HM_ERR_ALIAS: return "x and y overlap";
    case HM_ERR_COMPLEX_REQUIRED: return "complex matrix elements with a real dtype";
    case HM_ERR_NOT_HERMITIAN: return "term list is not self-adjoint";
    case HM_ERR_CUDA: return "CUDA error";
    case HM_ERR_OOM: return "out of device memory";
    case HM_ERR_TIMEOUT: return "bounded device wait timed out";
    case HM_ERR_UNSUPPORTED: return "unsupported shape";
    case HM_ERR_TOO_LARGE: return "size above the fixed maximum";
    case HM_LANCZOS_BREAKDOWN: return "Lanczos breakdown (Krylov space exhausted)";
    default: return "unknown error";
  }
}

const char* hm_last_error(void) { return g_err.c_str(); }

}  // extern "C"
