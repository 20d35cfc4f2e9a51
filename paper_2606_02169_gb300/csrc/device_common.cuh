// Device helpers shared by the hm kernels.
//
// Arithmetic policies:
//   AR_F32  : FP32 storage, FP32 accumulation.
//   AR_DF64 : FP64 storage, accumulation in an unevaluated sum of two floats
//             ("double-float", Dekker 1971; TwoSum of Knuth TAOCP vol. 2,
//             4.2.2). GB300 executes FP64 FMA at ~1/70 of the FP32 rate and
//             its f64<->f32 conversions run on the same slow pipe, so doubles
//             are split into float pairs and rebuilt with integer bit
//             operations only. Relative accuracy ~2^-46 per product.
//   AR_F64  : FP64 storage, native FP64 accumulation (reference variant).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hm_internal.h"

namespace hm {

enum { AR_F32 = 0, AR_DF64 = 1, AR_F64 = 2 };

struct DF {  // unevaluated sum s + c
  float s, c;
};

// Split a double into hi (truncated to 24 significant bits) and lo (the next
// 23 bits, truncated) using integer operations only. Exact range handling:
// |x| < 2^-126 -> (0, 0); |x| < 2^-80 -> lo = 0; |x| >= 2^128 -> inf/nan.
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
  const unsigned E = (h >> 20) & 0x7FFu;
  const unsigned sign = h & 0x80000000u;
  const unsigned mant = ((h & 0xFFFFFu) << 3) | (l >> 29);
  const unsigned hb = sign | ((E - 896u) << 23) | mant;
  const float ft = __fsub_rn(__uint_as_float(0x4B000000u | ((l >> 6) & 0x7FFFFFu)), 8388608.0f);
  const float scale = __uint_as_float(sign | ((E - 942u) << 23));
  const bool hnorm = (E >= 897u) & (E <= 1150u);
  const bool lnorm = (E >= 943u) & (E <= 1150u);
  const unsigned special = (E > 1150u) ? (sign | 0x7F800000u | ((E == 2047u && ((h & 0xFFFFFu) | l)) ? 0x400000u : 0u))
                                       : sign;
  hi = __uint_as_float(hnorm ? hb : special);
  lo = lnorm ? __fmul_rn(ft, scale) : 0.0f;
}

// Exact float -> double by bit manipulation (denormal floats flush to 0).
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned sign = u & 0x80000000u;
  unsigned hi = sign | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
  unsigned lo = u << 29;
  if (e == 0u) { hi = sign; lo = 0u; }
  if (e == 255u) { hi = sign | 0x7FF00000u | ((u & 0x7FFFFFu) ? 0x80000u : 0u); lo = 0u; }
  return __hiloint2double((int)hi, (int)lo);
}

// a += k * (xh + xl), k = (k.x + k.y). Product error from FMA; sum error from
// TwoSum. The rn intrinsics keep the compiler from contracting or
// reassociating the error-free transformations.
__device__ __forceinline__ void df_fma(DF& a, float2 k, float xh, float xl) {
  const float p = __fmul_rn(k.x, xh);
  float pe = __fmaf_rn(k.x, xh, -p);
  pe = __fmaf_rn(k.x, xl, pe);
  pe = __fmaf_rn(k.y, xh, pe);
  const float t = __fadd_rn(a.s, p);
  const float bp = __fsub_rn(t, a.s);
  const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  a.s = t;
  a.c = __fadd_rn(a.c, __fadd_rn(e, pe));
}

// a += k (double-float add of a coefficient)
__device__ __forceinline__ void df_add(DF& a, float2 k) {
  const float t = __fadd_rn(a.s, k.x);
  const float bp = __fsub_rn(t, a.s);
  const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(k.x, bp));
  a.s = t;
  a.c = __fadd_rn(a.c, __fadd_rn(e, k.y));
}

// renormalise so that |c| <= ulp(s)/2
__device__ __forceinline__ float2 df_norm(DF a) {
  const float t = __fadd_rn(a.s, a.c);
  const float bp = __fsub_rn(t, a.s);
  const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(a.c, bp));
  return make_float2(t, e);
}

__device__ __forceinline__ double df_to_double(DF a) {
  return f2d_exact(a.s) + f2d_exact(a.c);  // one FP64 add per output element
}

// ---------------------------------------------------------------------------
// Arithmetic policies
// ---------------------------------------------------------------------------
template <int AR> struct Ar;

template <> struct Ar<AR_F32> {
  using T = float;     // storage
  using C = float;     // coefficient
  using Acc = float;   // accumulator
  using X = float;     // prepared input value
  using Dsum = float;  // diagonal sum
  __device__ static const C* tab(const KPlan& P) { return P.tab_f; }
  __device__ static const C* diag(const KPlan& P) { return P.diag_f; }
  __device__ static const C* ell(const KPlan& P) { return P.ell_f; }
  __device__ static const C* ttab(const KPlan& P) { return P.ttab_f; }
  __device__ static C czero() { return 0.0f; }
  __device__ static bool nz(C c) { return c != 0.0f; }
  __device__ static X prep(T v) { return v; }
  __device__ static Acc azero() { return 0.0f; }
  __device__ static void fma(Acc& a, C c, X x) { a = __fmaf_rn(c, x, a); }
  __device__ static Dsum dzero() { return 0.0f; }
  __device__ static void dadd(Dsum& d, C c) { d = __fadd_rn(d, c); }
  __device__ static Acc dmul(Dsum d, X x) { return __fmul_rn(d, x); }
  __device__ static void dmadd(Dsum& d, C v, Dsum u) { d = __fmaf_rn(v, u, d); }
  __device__ static void acc_mul(Acc& a, C v, Acc g) { a = __fmaf_rn(v, g, a); }
  __device__ static T out(Acc a) { return a; }
  __device__ static double to_double(X x) { return (double)x; }
};

template <> struct Ar<AR_F64> {
  using T = double;
  using C = double;
  using Acc = double;
  using X = double;
  using Dsum = double;
  __device__ static const C* tab(const KPlan& P) { return P.tab_d; }
  __device__ static const C* diag(const KPlan& P) { return P.diag_d; }
  __device__ static const C* ell(const KPlan& P) { return P.ell_d; }
  __device__ static const C* ttab(const KPlan& P) { return P.ttab_d; }
  __device__ static C czero() { return 0.0; }
  __device__ static bool nz(C c) { return c != 0.0; }
  __device__ static X prep(T v) { return v; }
  __device__ static Acc azero() { return 0.0; }
  __device__ static void fma(Acc& a, C c, X x) { a = __fma_rn(c, x, a); }
  __device__ static Dsum dzero() { return 0.0; }
  __device__ static void dadd(Dsum& d, C c) { d = __dadd_rn(d, c); }
  __device__ static Acc dmul(Dsum d, X x) { return __dmul_rn(d, x); }
  __device__ static void dmadd(Dsum& d, C v, Dsum u) { d = __fma_rn(v, u, d); }
  __device__ static void acc_mul(Acc& a, C v, Acc g) { a = __fma_rn(v, g, a); }
  __device__ static T out(Acc a) { return a; }
  __device__ static double to_double(X x) { return x; }
};

template <> struct Ar<AR_DF64> {
  using T = double;
  using C = float2;
  using Acc = DF;
  using X = float2;
  using Dsum = DF;
  __device__ static const C* tab(const KPlan& P) { return P.tab_df; }
  __device__ static const C* diag(const KPlan& P) { return P.diag_df; }
  __device__ static const C* ell(const KPlan& P) { return P.ell_df; }
  __device__ static const C* ttab(const KPlan& P) { return P.ttab_df; }
  __device__ static C czero() { return make_float2(0.f, 0.f); }
  __device__ static bool nz(C c) { return c.x != 0.0f; }
  __device__ static X prep(T v) {
    float h, l;
    split_f64(v, h, l);
    return make_float2(h, l);
  }
  __device__ static Acc azero() { return DF{0.f, 0.f}; }
  __device__ static void fma(Acc& a, C c, X x) { df_fma(a, c, x.x, x.y); }
  __device__ static Dsum dzero() { return DF{0.f, 0.f}; }
  __device__ static void dadd(Dsum& d, C c) { df_add(d, c); }
  __device__ static Acc dmul(Dsum d, X x) {
    DF a{0.f, 0.f};
    df_fma(a, df_norm(d), x.x, x.y);
    return a;
  }
  __device__ static void dmadd(Dsum& d, C v, Dsum u) {
    const float2 n = df_norm(u);
    df_fma(d, v, n.x, n.y);
  }
  __device__ static void acc_mul(Acc& a, C v, Acc g) {
    const float2 n = df_norm(g);
    df_fma(a, v, n.x, n.y);
  }
  __device__ static T out(Acc a) { return df_to_double(a); }
  __device__ static double to_double(X x) { return f2d_exact(x.x) + f2d_exact(x.y); }
};

// ---------------------------------------------------------------------------
// Vector loads/stores of NV consecutive values (alignment checked on the host)
// ---------------------------------------------------------------------------
template <class T, int NV>
__device__ __forceinline__ void ldv(const T* __restrict__ p, T (&v)[NV]) {
  constexpr int bytes = NV * (int)sizeof(T);
  if constexpr (bytes % 16 == 0) {
#pragma unroll
    for (int u = 0; u < NV; u += 16 / (int)sizeof(T)) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(p + u));
      const T* t = reinterpret_cast<const T*>(&q);
#pragma unroll
      for (int w = 0; w < 16 / (int)sizeof(T); ++w) v[u + w] = t[w];
    }
  } else if constexpr (bytes == 8 && sizeof(T) == 4) {
    const float2 q = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = q.x;
    v[1] = q.y;
  } else {
#pragma unroll
    for (int u = 0; u < NV; ++u) v[u] = __ldg(p + u);
  }
}

template <class T, int NV>
__device__ __forceinline__ void stv(T* __restrict__ p, const T (&v)[NV]) {
  constexpr int bytes = NV * (int)sizeof(T);
  if constexpr (bytes % 16 == 0) {
#pragma unroll
    for (int u = 0; u < NV; u += 16 / (int)sizeof(T)) {
      uint4 q;
      T* t = reinterpret_cast<T*>(&q);
#pragma unroll
      for (int w = 0; w < 16 / (int)sizeof(T); ++w) t[w] = v[u + w];
      *reinterpret_cast<uint4*>(p + u) = q;
    }
  } else {
#pragma unroll
    for (int u = 0; u < NV; ++u) p[u] = v[u];
  }
}

// digit of a high (tile-uniform) site, held by lane (site % 32) in nh0/nh1
__device__ __forceinline__ int high_digit(int site, int nh0, int nh1) {
  return __shfl_sync(0xffffffffu, site < 32 ? nh0 : nh1, site & 31);
}

__device__ __forceinline__ int low_digit(uint32_t pk, int bit, int wid) {
  return (int)((pk >> bit) & ((1u << wid) - 1u));
}

// Digits of the high (tile-uniform) sites of low block hb, n = floor(hb / M'_k)
// mod d_k with M'_k = M_k / B (Eq. decode on the high part). Lane l gets site
// l in nh0 and site l+32 in nh1; plain 64-bit division, once per tile.
__device__ __forceinline__ void high_digits(const KPlan& P, long long hb, int& nh0, int& nh1) {
  const int lane = threadIdx.x & 31;
  nh0 = (lane < P.nhigh) ? (int)((hb / P.sites[lane].mh) % P.sites[lane].d) : 0;
  nh1 = (lane + 32 < P.nhigh) ? (int)((hb / P.sites[lane + 32].mh) % P.sites[lane + 32].d) : 0;
}

}  // namespace hm
