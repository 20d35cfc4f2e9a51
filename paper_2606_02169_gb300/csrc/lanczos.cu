// Device Lanczos ground state and time evolution (Sec. I, Sec. VIII: Krylov
// methods consume only y = H x; Sec. VII: exact propagation).
//   w = H v_k;  alpha_k = <v_k, w>;  w -= alpha_k v_k + beta_{k-1} v_{k-1};
//   [optional second Gram-Schmidt pass against v_k, v_{k-1}];
//   beta_k = ||w||;  v_{k+1} = w / beta_k.
// Dot products and norms accumulate to FP64 accuracy (even for FP32 storage)
// and are reduced in a fixed order (per-block partials, then one block), so a rerun
// from the same v0 reproduces every Krylov vector bit for bit. The ground
// state Ritz vector is assembled in that rerun, so the Krylov basis is never
// stored. Scalars live on the device between kernels: the step loop has no
// host round trip. The tridiagonal eigenproblem is solved on the host in
// FP64 (Sturm-sequence bisection for the lowest eigenvalue, then inverse
// iteration with a partially pivoted tridiagonal solve for its vector).
// Time evolution y = exp(-i t H) x is the short-iterative Lanczos propagator
// (Park and Light, 1986): per step tau, u <- |u| V_m exp(-i tau T_m) e_1,
// with exp(-i tau T_m) from a Jacobi eigendecomposition of T_m on the host
// and the Krylov basis V_m stored on the device or rebuilt by a second pass.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_common.cuh"

namespace hm {


constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

// Arithmetic of the vector kernels. GB300 executes FP64 FMA at about 1/70 of
// the FP32 rate, which would make these memory-bound kernels FP64-bound, so
//   * dot products accumulate a double-float sum of exact (FP32 data) or
//     Dekker (FP64 data, split as read) products on the FP32 pipe, reduced in
//     a fixed order (lanes, warps, blocks), then rounded once to FP64;
//   * updates of FP32 vectors run in double-float and round once to FP32;
//   * updates of FP64 vectors stay native FP64.
template <class T>
__device__ __forceinline__ double tod(T v);
template <>
__device__ __forceinline__ double tod<float>(float v) { return f2d_exact(v); }
template <>
__device__ __forceinline__ double tod<double>(double v) { return v; }

__device__ __forceinline__ float2 pair_of(float v) { return make_float2(v, 0.0f); }
__device__ __forceinline__ float2 pair_of(double v) { return split_f64(v); }

// acc += a * b
__device__ __forceinline__ void dot_acc(DF& acc, float a, float b) {
  const float p = __fmul_rn(a, b);
  df_add(acc, make_float2(p, __fmaf_rn(a, b, -p)));   // exact product
}
__device__ __forceinline__ void dot_acc(DF& acc, double a, double b) {
  const float2 x = split_f64(a), y = split_f64(b);
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, e);
  e = __fmaf_rn(x.y, y.x, e);
  df_add(acc, make_float2(p, e));
}

// Fixed-order CTA sum of a double-float value; the FP64 result is valid in
// thread 0.
__device__ __forceinline__ double block_sum(DF v, float2* sh) {
  for (int o = 16; o > 0; o >>= 1)
    df_add(v, make_float2(__shfl_xor_sync(0xffffffffu, v.s, o), __shfl_xor_sync(0xffffffffu, v.c, o)));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = make_float2(v.s, v.c);
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    DF t{0.f, 0.f};
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) df_add(t, sh[i]);
    s = df_to_double(t);
  }
  __syncthreads();
  return s;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  __syncthreads();
  return s;  // valid in thread 0
}

// x0 + c1 * x1 + c2 * x2 rounded to T (c as double-float pairs, x1, x2 FP32)
__device__ __forceinline__ float lin3(float x0, float2 c1, float x1, float2 c2, float x2) {
  DF r{x0, 0.0f};
  df_fma(r, c1, x1, 0.0f);
  df_fma(r, c2, x2, 0.0f);
  return __fadd_rn(r.s, r.c);
}

// partial[b] = sum over the block's grid-stride share of a[i]*b[i]
template <class T>
__global__ void __launch_bounds__(kRedThreads) k_dot(const T* __restrict__ a, const T* __restrict__ b,
                                                     long long n, double* __restrict__ partial) {
  __shared__ float2 sh[32];
  DF s{0.f, 0.f};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dot_acc(s, a[i], b[i]);
  const double t = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// out[0] = sum partial (fixed order); if sqrt_it, out = sqrt(out)
__global__ void k_finish(const double* __restrict__ partial, int n, double* __restrict__ out, int sqrt_it) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] = sqrt_it ? sqrt(s) : s;
}

// w -= a[0] * v + (bprev ? bprev[0] : 0) * vp, fused with the block partials
// of dot products of the updated w: nd = 1: <w, w>; nd = 2: <v, w> and
// <vp, w> (partial[b] and partial[gridDim.x + b]). Same grid and thread
// mapping as k_dot, so the sums keep a fixed order.
template <class T>
__global__ void __launch_bounds__(kRedThreads) k_axpy2_dot(T* __restrict__ w, const T* __restrict__ v,
                                                            const T* __restrict__ vp, const double* __restrict__ a,
                                                            const double* __restrict__ bprev, long long n, int nd,
                                                            double* __restrict__ partial) {
  __shared__ float2 sh[32];
  const double al = a[0];
  const double be = bprev ? bprev[0] : 0.0;
  const float2 mal = pair_of(-al), mbe = pair_of(-be);
  DF s0{0.f, 0.f}, s1{0.f, 0.f};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T vi = v[i];
    const T pi = vp ? vp[i] : T(0);
    T wt;
    if constexpr (sizeof(T) == 4) {
      wt = lin3(w[i], mal, vi, mbe, pi);
    } else {
      double r = fma(-al, vi, w[i]);
      if (vp) r = fma(-be, pi, r);
      wt = r;
    }
    w[i] = wt;
    if (nd == 1) {
      dot_acc(s0, wt, wt);
    } else {
      dot_acc(s0, vi, wt);
      dot_acc(s1, pi, wt);
    }
  }
  const double t0 = block_sum(s0, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t0;
  if (nd == 2) {
    const double t1 = block_sum(s1, sh);
    if (threadIdx.x == 0) partial[gridDim.x + blockIdx.x] = t1;
  }
}

// dst = src * c (c a double-float pair for FP32 data)
template <class T>
__device__ __forceinline__ T scale_one(T x, double c, float2 cp) {
  if constexpr (sizeof(T) == 4) {
    const float p = __fmul_rn(cp.x, x);
    float e = __fmaf_rn(cp.x, x, -p);
    e = __fmaf_rn(cp.y, x, e);
    return __fadd_rn(p, e);
  } else {
    return x * c;
  }
}

// v = w / b[0] (zero vector if b[0] is below tol: breakdown)
template <class T>
__global__ void k_scale(T* __restrict__ v, const T* __restrict__ w, const double* __restrict__ b,
                        double tol, long long n) {
  const double bb = b[0];
  const double inv = (bb > tol) ? 1.0 / bb : 0.0;
  const float2 ip = pair_of(inv);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = scale_one(w[i], inv, ip);
}

// psi += coef * v
template <class T>
__global__ void k_axpy(T* __restrict__ psi, const T* __restrict__ v, double coef, long long n) {
  const float2 cp = pair_of(coef), zero = make_float2(0.f, 0.f);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if constexpr (sizeof(T) == 4) psi[i] = lin3(psi[i], cp, v[i], zero, 0.0f);
    else psi[i] = fma(coef, v[i], psi[i]);
  }
}

template <class T>
__global__ void k_copy_scaled(T* __restrict__ dst, const T* __restrict__ src, double scale, long long n) {
  const float2 sp = pair_of(scale);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = scale_one(src[i], scale, sp);
}

// ---------------------------------------------------------------------------
// host tridiagonal eigensolver
// ---------------------------------------------------------------------------
static int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double lam) {
  int cnt = 0;
  double q = 1.0;
  for (size_t i = 0; i < a.size(); ++i) {
    const double bb = (i == 0) ? 0.0 : b[i - 1] * b[i - 1];
    q = (a[i] - lam) - ((i == 0) ? 0.0 : bb / q);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

static double lowest_eigenvalue(const std::vector<double>& a, const std::vector<double>& b) {
  double lo = 1e300, hi = -1e300;
  for (size_t i = 0; i < a.size(); ++i) {  // Gershgorin interval
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < a.size() ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (sturm_count(a, b, mid) >= 1) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Solve (T - lam I) u = rhs with Gaussian elimination and partial pivoting on
// the tridiagonal band (one extra superdiagonal appears from row swaps).
static void tri_solve(const std::vector<double>& a, const std::vector<double>& b, double lam,
                      std::vector<double>& u) {
  const int n = (int)a.size();
  std::vector<double> d(n), du(n, 0.0), du2(n, 0.0), dl(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = a[i] - lam;
  for (int i = 0; i + 1 < n; ++i) { du[i] = b[i]; dl[i] = b[i]; }
  std::vector<double> r = u;
  for (int i = 0; i + 1 < n; ++i) {
    if (std::fabs(d[i]) >= std::fabs(dl[i])) {
      double piv = (d[i] == 0.0) ? 1e-300 : d[i];
      double f = dl[i] / piv;
      d[i + 1] -= f * du[i];
      if (i + 2 < n) du[i + 1] -= f * du2[i];
      r[i + 1] -= f * r[i];
    } else {
      double f = d[i] / dl[i];
      // swap rows i and i+1
      double t0 = d[i], t1 = du[i];
      d[i] = dl[i];
      du[i] = d[i + 1];
      du2[i] = (i + 2 < n) ? du[i + 1] : 0.0;
      d[i + 1] = t1 - f * du[i];
      if (i + 2 < n) du[i + 1] = -f * du2[i];
      (void)t0;
      std::swap(r[i], r[i + 1]);
      r[i + 1] -= f * r[i];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = r[i];
    if (i + 1 < n) s -= du[i] * r[i + 1];
    if (i + 2 < n) s -= du2[i] * r[i + 2];
    double piv = (d[i] == 0.0) ? 1e-300 : d[i];
    r[i] = s / piv;
  }
  u.swap(r);
}

static std::vector<double> lowest_eigvec(const std::vector<double>& a, const std::vector<double>& b,
                                         double lam) {
  const int n = (int)a.size();
  std::vector<double> u(n, 1.0);
  double scale = 1.0;
  for (size_t i = 0; i < a.size(); ++i) scale = std::max(scale, std::fabs(a[i]));
  const double shift = lam - 1e-13 * scale;
  for (int it = 0; it < 4; ++it) {
    tri_solve(a, b, shift, u);
    double nrm = 0.0;
    for (double v : u) nrm += v * v;
    nrm = std::sqrt(nrm);
    for (double& v : u) v /= nrm;
  }
  return u;
}

// ---------------------------------------------------------------------------
// the recurrence
// ---------------------------------------------------------------------------

// Work vectors, device scalars and launch shapes of one Lanczos recurrence on
// vectors of n = states * nvec elements (nvec = 2: the real and imaginary
// parts of a complex vector, interleaved). For a self-adjoint H, alpha =
// <v, H v> and beta = |w| are real, and the real dot products of the pairs
// are the real parts of the complex ones, so the recurrence on the pairs is
// the complex recurrence (for a complex H the apply is the complex one).
template <class T>
struct Recurrence {
  Plan* p = nullptr;
  hm_dtype dt = HM_F64;
  long long nvec = 1, n = 0;
  int flags = 0, vb = 1, rb = 1;
  cudaStream_t s = nullptr;
  T* V = nullptr;
  T *vk = nullptr, *vp = nullptr, *w = nullptr;
  double* dsc = nullptr;  // [2 rb partials][alpha steps][beta steps][tmp 8]
  double *part = nullptr, *dal = nullptr, *dbe = nullptr, *tmp = nullptr;

  int init(Plan* p_, hm_dtype dt_, long long nvec_, int flags_, int steps, cudaStream_t s_) {
    p = p_;
    dt = dt_;
    nvec = nvec_;
    flags = flags_;
    s = s_;
    n = vec_states(p) * nvec;
    vb = (int)std::min<long long>((n + 255) / 256, (long long)num_sms() * 8);
    rb = (int)std::min<long long>((n + kRedThreads - 1) / kRedThreads, kRedBlocks);
    cudaError_t e = cudaMalloc(&V, sizeof(T) * n * 3);
    if (e != cudaSuccess) {
      V = nullptr;
      return cuda_fail(e, "Lanczos work vectors");
    }
    e = cudaMalloc(&dsc, sizeof(double) * (2 * (size_t)rb + 2 * (size_t)steps + 8));
    if (e != cudaSuccess) {
      dsc = nullptr;
      return cuda_fail(e, "Lanczos scalars");
    }
    vk = V;
    vp = V + n;
    w = V + 2 * n;
    part = dsc;
    dal = dsc + 2 * rb;
    dbe = dal + steps;
    tmp = dbe + steps;
    return HM_OK;
  }
  ~Recurrence() {
    if (s || V || dsc) cudaStreamSynchronize(s);
    if (V) cudaFree(V);
    if (dsc) cudaFree(dsc);
  }

  void dot(const T* a, const T* b, double* out, int sq) {
    k_dot<T><<<rb, kRedThreads, 0, s>>>(a, b, n, part);
    k_finish<<<1, 256, 0, s>>>(part, rb, out, sq);
  }

  // One pass of m steps from v0 (tmp[0] = |v0|, v_0 = v0 / |v0|);
  // at_step(k, v_k) is queued before the apply of step k. beta of the last
  // step is formed too when last_beta (the residual norm of the m-step space).
  // With a basis (m vectors of n), v_k is written straight into basis + k n
  // (the same values as in the work vectors).
  template <class F>
  int run(const T* v0, int m, bool last_beta, F&& at_step, T* basis = nullptr) {
    if (basis) {
      vk = basis;
      vp = nullptr;
    } else {
      vk = V;
      vp = V + n;
    }
    dot(v0, v0, tmp, 1);
    k_scale<T><<<vb, 256, 0, s>>>(vk, v0, tmp, 0.0, n);
    if (!basis) cudaMemsetAsync(vp, 0, sizeof(T) * n, s);
    for (int k = 0; k < m; ++k) {
      int arc = at_step(k, (const T*)vk);
      if (arc) return arc;
      arc = p->im ? apply_complex(p, false, vk, w, nvec / 2, dt, s)  // complex H: nvec = 2
                  : apply_on(p, false, vk, w, nvec, dt, s, tuned_cfg(p, dt, nvec), false);
      if (arc) return arc;
      dot(vk, w, dal + k, 0);
      const T* vpk = k > 0 ? vp : nullptr;
      const bool last = k == m - 1;
      if (flags & 1) {
        // w -= alpha v_k + beta v_{k-1}, with <v_k, w> and <v_{k-1}, w> of the
        // result for the second Gram-Schmidt pass
        k_axpy2_dot<T><<<rb, kRedThreads, 0, s>>>(w, vk, vpk, dal + k, k > 0 ? dbe + k - 1 : nullptr, n, 2, part);
        k_finish<<<1, 256, 0, s>>>(part, rb, tmp + 1, 0);
        k_finish<<<1, 256, 0, s>>>(part + rb, rb, tmp + 2, 0);
        // second pass, fused with beta_k = ||w||
        k_axpy2_dot<T><<<rb, kRedThreads, 0, s>>>(w, vk, vpk, tmp + 1, k > 0 ? tmp + 2 : nullptr, n, 1, part);
      } else {
        k_axpy2_dot<T><<<rb, kRedThreads, 0, s>>>(w, vk, vpk, dal + k, k > 0 ? dbe + k - 1 : nullptr, n, 1, part);
      }
      if (last && !last_beta) break;
      k_finish<<<1, 256, 0, s>>>(part, rb, dbe + k, 1);
      if (last) break;
      if (basis) {                                            // v_{k-1} <- v_k
        vp = vk;
        vk = basis + (size_t)(k + 1) * n;
      } else {
        std::swap(vp, vk);
      }
      k_scale<T><<<vb, 256, 0, s>>>(vk, w, dbe + k, 0.0, n);  // v_{k+1} = w / beta_k
    }
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return cuda_fail(le, "Lanczos kernels");
    return HM_OK;
  }

  // alpha[0..m), beta[0..nb) and |v0| to the host
  int scalars(int m, int nb, std::vector<double>& ha, std::vector<double>& hb, double* nu) {
    ha.assign(m, 0.0);
    hb.assign(std::max(nb, 0), 0.0);
    cudaError_t e = cudaMemcpyAsync(ha.data(), dal, sizeof(double) * m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && nb > 0)
      e = cudaMemcpyAsync(hb.data(), dbe, sizeof(double) * nb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && nu) e = cudaMemcpyAsync(nu, tmp, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "Lanczos scalars to host");
    return HM_OK;
  }
};

// ---------------------------------------------------------------------------
// ground state
// ---------------------------------------------------------------------------
template <class T>
static int lanczos_t(Plan* p, const T* v0, int steps, hm_dtype dt, long long nvec, int flags, double* alpha,
                     double* beta, int* steps_done, T* psi0, double* e0, cudaStream_t s) {
  Recurrence<T> R;
  int rc = R.init(p, dt, nvec, flags, steps, s);
  if (rc) return rc;
  const long long n = R.n;
  auto none = [](int, const T*) -> int { return HM_OK; };
  rc = R.run(v0, steps, false, none);
  if (rc) return rc;
  std::vector<double> ha, hb;
  rc = R.scalars(steps, steps - 1, ha, hb, nullptr);
  if (rc) return rc;
  hb.push_back(0.0);
  double amax = 0.0;
  for (double v : ha) amax = std::max(amax, std::fabs(v));
  int m = steps;
  for (int k = 0; k + 1 < steps; ++k)
    if (!(hb[k] > 1e-14 * std::max(1.0, amax))) {  // breakdown (also catches NaN)
      m = k + 1;
      rc = HM_LANCZOS_BREAKDOWN;
      break;
    }
  std::vector<double> a(ha.begin(), ha.begin() + m), b(hb.begin(), hb.begin() + std::max(0, m - 1));
  for (int k = 0; k < steps; ++k) {
    alpha[k] = k < m ? ha[k] : 0.0;
    beta[k] = k + 1 < m ? hb[k] : 0.0;
  }
  *steps_done = m;
  *e0 = lowest_eigenvalue(a, b);
  if (psi0) {
    // the Ritz vector, assembled in a second pass of the same recurrence
    std::vector<double> u = lowest_eigvec(a, b, *e0);
    cudaMemsetAsync(psi0, 0, sizeof(T) * n, s);
    int rc2 = R.run(v0, m, false, [&](int k, const T* vk) -> int {
      k_axpy<T><<<R.vb, 256, 0, s>>>(psi0, vk, u[k], n);
      return HM_OK;
    });
    if (rc2 != HM_OK) return rc2;
    R.dot(psi0, psi0, R.tmp + 3, 1);
    double nrm = 0.0;
    cudaError_t e = cudaMemcpyAsync(&nrm, R.tmp + 3, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && nrm > 0.0) {
      k_copy_scaled<T><<<R.vb, 256, 0, s>>>(psi0, psi0, 1.0 / nrm, n);
      e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "Ritz vector");
  }
  return rc;
}

int run_lanczos(Plan* p, const void* v0, int steps, hm_dtype dt, long long nvec, int flags, double* alpha,
                double* beta, int* steps_done, void* psi0, double* e0, cudaStream_t s) {
  if (dt == HM_F32)
    return lanczos_t<float>(p, (const float*)v0, steps, dt, nvec, flags, alpha, beta, steps_done, (float*)psi0,
                            e0, s);
  return lanczos_t<double>(p, (const double*)v0, steps, dt, nvec, flags, alpha, beta, steps_done,
                           (double*)psi0, e0, s);
}

// ---------------------------------------------------------------------------
// time evolution
// ---------------------------------------------------------------------------

// y += (cr + i ci) v on interleaved (re, im) pairs
template <class T>
__global__ void k_caxpy(T* __restrict__ y, const T* __restrict__ v, double cr, double ci, long long npairs) {
  const float2 pr = pair_of(cr), pi = pair_of(ci), mpi = pair_of(-ci);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npairs;
       i += (long long)gridDim.x * blockDim.x) {
    const T vr = v[2 * i], vi = v[2 * i + 1];
    if constexpr (sizeof(T) == 4) {
      y[2 * i] = lin3(y[2 * i], pr, vr, mpi, vi);
      y[2 * i + 1] = lin3(y[2 * i + 1], pr, vi, pi, vr);
    } else {
      y[2 * i] = fma(cr, vr, fma(-ci, vi, y[2 * i]));
      y[2 * i + 1] = fma(cr, vi, fma(ci, vr, y[2 * i + 1]));
    }
  }
}

// y = sum_k (c_re[k] + i c_im[k]) v_k over a stored basis (v_k at B + k n),
// in one pass: per element the same operations in the same order as me
// k_caxpy launches from y = 0, so the result is bit for bit theirs (the
// rebuilt-basis path runs those launches)
constexpr int kCombineMax = 128;  // the Krylov dimension limit of hm_evolve

struct CombineCoefs {
  double c[2 * kCombineMax];
  int me;
};

// (re, im) pair i of a vector in the library's basis allocation (aligned)
__device__ __forceinline__ void ld_pair(const float* v, long long i, float& r, float& m) {
  const float2 p = __ldcs(reinterpret_cast<const float2*>(v) + i);
  r = p.x;
  m = p.y;
}
__device__ __forceinline__ void ld_pair(const double* v, long long i, double& r, double& m) {
  const double2 p = __ldcs(reinterpret_cast<const double2*>(v) + i);
  r = p.x;
  m = p.y;
}

// Each thread owns kCombinePairs pairs a block's width apart and walks the
// basis once for all of them (that many independent 8- or 16-byte loads in
// flight per vector).
constexpr int kCombinePairs = 4;

template <class T>
__device__ __forceinline__ void caxpy_one(T& yr, T& yi, double cr, double ci, T vr, T vi) {
  if constexpr (sizeof(T) == 4) {
    const float2 pr = pair_of(cr), pi = pair_of(ci), mpi = pair_of(-ci);
    yr = lin3(yr, pr, vr, mpi, vi);
    yi = lin3(yi, pr, vi, pi, vr);
  } else {
    yr = fma(cr, vr, fma(-ci, vi, yr));
    yi = fma(cr, vi, fma(ci, vr, yi));
  }
}

template <class T>
__global__ void k_ccombine(T* __restrict__ y, const T* __restrict__ B, long long n, const CombineCoefs cc) {
  constexpr int P = kCombinePairs;
  const long long npairs = n / 2;
  const long long span = (long long)blockDim.x * P;
  for (long long base = blockIdx.x * span + threadIdx.x; base < npairs; base += (long long)gridDim.x * span) {
    T yr[P], yi[P];
#pragma unroll
    for (int j = 0; j < P; ++j) yr[j] = yi[j] = T(0);
    for (int k = 0; k < cc.me; ++k) {
      const double cr = cc.c[2 * k], ci = cc.c[2 * k + 1];
      const T* __restrict__ v = B + (size_t)k * n;
      T vr[P], vi[P];
#pragma unroll
      for (int j = 0; j < P; ++j)
        if (base + j * blockDim.x < npairs) ld_pair(v, base + j * blockDim.x, vr[j], vi[j]);
#pragma unroll
      for (int j = 0; j < P; ++j)
        if (base + j * blockDim.x < npairs) caxpy_one(yr[j], yi[j], cr, ci, vr[j], vi[j]);
    }
#pragma unroll
    for (int j = 0; j < P; ++j) {
      const long long i = base + j * blockDim.x;
      if (i < npairs) {
        y[2 * i] = yr[j];
        y[2 * i + 1] = yi[j];
      }
    }
  }
}

// Eigendecomposition of the real symmetric tridiagonal T (diagonal a,
// off-diagonal b) by the cyclic Jacobi method: rotations in the (p, q)
// plane with tan t the smaller root of t^2 + 2 t theta - 1 = 0, theta =
// (T_qq - T_pp) / (2 T_pq), until the off-diagonal mass is negligible.
// lam[j] and column j of Q (row-major, Q[k * m + j]) are the eigenpairs.
static void jacobi_eig(const std::vector<double>& a, const std::vector<double>& b, std::vector<double>& lam,
                       std::vector<double>& Q) {
  const int m = (int)a.size();
  std::vector<double> A((size_t)m * m, 0.0);
  Q.assign((size_t)m * m, 0.0);
  double fro = 0.0;
  for (int i = 0; i < m; ++i) {
    A[(size_t)i * m + i] = a[i];
    Q[(size_t)i * m + i] = 1.0;
    fro += a[i] * a[i];
    if (i + 1 < m) {
      A[(size_t)i * m + i + 1] = A[(size_t)(i + 1) * m + i] = b[i];
      fro += 2 * b[i] * b[i];
    }
  }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) off += A[(size_t)p * m + q] * A[(size_t)p * m + q];
    if (off <= 1e-34 * fro || off == 0.0) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[(size_t)p * m + q];
        if (apq == 0.0) continue;
        const double theta = (A[(size_t)q * m + q] - A[(size_t)p * m + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < m; ++k) {  // columns p, q
          const double akp = A[(size_t)k * m + p], akq = A[(size_t)k * m + q];
          A[(size_t)k * m + p] = c * akp - sn * akq;
          A[(size_t)k * m + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q
          const double apk = A[(size_t)p * m + k], aqk = A[(size_t)q * m + k];
          A[(size_t)p * m + k] = c * apk - sn * aqk;
          A[(size_t)q * m + k] = sn * apk + c * aqk;
        }
        A[(size_t)p * m + q] = A[(size_t)q * m + p] = 0.0;
        for (int k = 0; k < m; ++k) {
          const double qkp = Q[(size_t)k * m + p], qkq = Q[(size_t)k * m + q];
          Q[(size_t)k * m + p] = c * qkp - sn * qkq;
          Q[(size_t)k * m + q] = sn * qkp + c * qkq;
        }
      }
  }
  lam.resize(m);
  for (int i = 0; i < m; ++i) lam[i] = A[(size_t)i * m + i];
}

// c[k] = nu [exp(-i tau T) e_1]_k as (re, im) pairs, T = tridiag(b, a, b)
void krylov_coeffs(const std::vector<double>& a, const std::vector<double>& b, double tau, double nu,
                   std::vector<double>& c) {
  const int m = (int)a.size();
  std::vector<double> lam, Q;
  jacobi_eig(a, b, lam, Q);
  c.assign(2 * (size_t)m, 0.0);
  for (int j = 0; j < m; ++j) {
    const double fr = std::cos(tau * lam[j]) * Q[j], fi = -std::sin(tau * lam[j]) * Q[j];  // Q[0 * m + j]
    for (int k = 0; k < m; ++k) {
      c[2 * k] += nu * Q[(size_t)k * m + j] * fr;
      c[2 * k + 1] += nu * Q[(size_t)k * m + j] * fi;
    }
  }
}

template <class T>
static int evolve_t(Plan* p, const T* x, T* y, double t, int m, int nsub, int flags, hm_dtype dt, double* err,
                    cudaStream_t s) {
  Recurrence<T> R;
  int rc = R.init(p, dt, 2, flags, m, s);
  if (rc) return rc;
  const long long n = R.n;
  T* B = nullptr;  // the Krylov basis, when stored
  T* scratch = nullptr;
  if (!(flags & 2)) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && (size_t)m * n * sizeof(T) <= fr / 2 &&
        cudaMalloc(&B, (size_t)m * n * sizeof(T)) != cudaSuccess) {
      B = nullptr;
      cudaGetLastError();  // fall back to the second pass
    }
  }
  if (nsub > 1) {
    cudaError_t e = cudaMalloc(&scratch, (size_t)n * sizeof(T));
    if (e != cudaSuccess) {
      if (B) cudaFree(B);
      return cuda_fail(e, "evolution scratch vector");
    }
  }
  const double tau = t / nsub;
  double esum = 0.0;
  const T* u = x;
  for (int j = 0; j < nsub && rc == HM_OK; ++j) {
    T* out = ((nsub - 1 - j) % 2 == 0) ? y : scratch;
    rc = R.run(u, m, true, [](int, const T*) -> int { return HM_OK; }, B);  // v_k stored in B
    if (rc) break;
    std::vector<double> ha, hb;
    double nu = 0.0;
    rc = R.scalars(m, m, ha, hb, &nu);
    if (rc) break;
    double amax = 0.0;
    for (double v : ha)
      if (std::isfinite(v)) amax = std::max(amax, std::fabs(v));
    int me = m;
    for (int k = 0; k + 1 < m; ++k)
      if (!(hb[k] > 1e-14 * std::max(1.0, amax))) {  // invariant Krylov space: exact
        me = k + 1;
        break;
      }
    bool finite = std::isfinite(nu) && (me < m || std::isfinite(hb[m - 1]));
    for (int k = 0; k < me; ++k) finite = finite && std::isfinite(ha[k]);
    if (!finite) {
      set_error("non-finite value in the Krylov recurrence (x or H holds NaN or Inf)");
      rc = HM_ERR_INVALID_ARG;
      break;
    }
    std::vector<double> a(ha.begin(), ha.begin() + me), b(hb.begin(), hb.begin() + (me - 1)), c;
    krylov_coeffs(a, b, tau, nu, c);
    if (me == m) esum += hb[m - 1] * std::hypot(c[2 * (m - 1)], c[2 * (m - 1) + 1]);
    if (B && me <= kCombineMax) {
      CombineCoefs cc{};
      for (int k = 0; k < 2 * me; ++k) cc.c[k] = c[k];
      cc.me = me;
      k_ccombine<T><<<R.vb, 256, 0, s>>>(out, B, n, cc);
    } else if (B) {
      cudaMemsetAsync(out, 0, sizeof(T) * n, s);
      for (int k = 0; k < me; ++k)
        k_caxpy<T><<<R.vb, 256, 0, s>>>(out, B + (size_t)k * n, c[2 * k], c[2 * k + 1], n / 2);
    } else {  // second pass of the same recurrence: the same v_k, bit for bit
      cudaMemsetAsync(out, 0, sizeof(T) * n, s);
      rc = R.run(u, me, false, [&](int k, const T* vk) -> int {
        k_caxpy<T><<<R.vb, 256, 0, s>>>(out, vk, c[2 * k], c[2 * k + 1], n / 2);
        return HM_OK;
      });
    }
    cudaError_t le = cudaGetLastError();
    if (rc == HM_OK && le != cudaSuccess) rc = cuda_fail(le, "evolution kernels");
    u = out;
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (rc == HM_OK && e != cudaSuccess) rc = cuda_fail(e, "evolution");
  if (B) cudaFree(B);
  if (scratch) cudaFree(scratch);
  if (err) *err = esum;
  return rc;
}

int run_evolve(Plan* p, const void* x, void* y, double t, int m, int nsub, int flags, hm_dtype dt, double* err,
               cudaStream_t s) {
  if (dt == HM_F32)
    return evolve_t<float>(p, (const float*)x, (float*)y, t, m, nsub, flags, dt, err, s);
  return evolve_t<double>(p, (const double*)x, (double*)y, t, m, nsub, flags, dt, err, s);
}

}  // namespace hm
