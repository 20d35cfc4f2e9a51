// Device helpers shared by the hm kernels.
//
// Arithmetic policies:
//   AR_F32  : FP32 storage, FP32 accumulation.
//   AR_DF64 : FP64 storage. GB300 executes FP64 FMA at ~1/70 of the FP32 rate
//             and its f64<->f32 conversions run on the same slow pipe, so each
//             double is split once per apply into a pair of floats (integer
//             bit operations only; a separate pass) and the kernel accumulates
//             an unevaluated sum of two floats ("double-float": Dekker 1971;
//             TwoSum of Knuth, TAOCP vol. 2, 4.2.2). Relative accuracy about
//             2^-46 per product; the result is rebuilt as a double with one
//             FP64 add.
//   AR_F64  : FP64 storage, native FP64 accumulation (reference variant).
//   AR_F32V2, AR_F32V4, AR_DF64V2: the AR_F32 / AR_DF64 arithmetic on 2 or 4
//             consecutive right-hand sides of one state per kernel element
//             (8- or 16-byte loads and stores; decode, table lookups and
//             coefficients once per state instead of once per right-hand
//             side). Each right-hand side takes exactly the scalar policy's
//             operations in the same order, so results are bit-identical.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hm_internal.h"

namespace hm {

enum { AR_F32 = 0, AR_DF64 = 1, AR_F64 = 2, AR_F32V2 = 3, AR_F32V4 = 4, AR_DF64V2 = 5, AR_F64V2 = 6 };

// Launch gate: a kernel runs iff flag == NULL or (*flag != 0) == run. A
// double-float apply (run = 0) and its native FP64 fallback (run = 1) are
// queued together; the split pass sets *flag when an input is outside the
// double-float window, so exactly one of them does the work.
struct KGate {
  const int* flag;
  int run;
};

__device__ __forceinline__ bool gate_closed(const KGate g) {
  return g.flag != nullptr && ((__ldcg(g.flag) != 0) != (g.run != 0));
}

struct DF {  // unevaluated sum s + c
  float s, c;
};

// Split a double into hi (truncated to 24 significant bits) and lo (the next
// 23 bits, truncated): x = hi + lo + r with |r| < 2^-46 |x|. Integer
// operations only. Fast path for 2^-80 <= |x| < 2^128; the rare remainder
// (zero, tiny, huge, inf, nan) takes a slower exact-range branch:
// |x| < 2^-126 -> (0, 0); |x| < 2^-80 -> lo = 0; |x| >= 2^128 -> inf/nan.
__device__ __forceinline__ float2 split_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h = (unsigned)(b >> 32), l = (unsigned)b;
  const unsigned sign = h & 0x80000000u;
  // funnel shift: bits 31..23 hold the low 9 bits of the double exponent E;
  // E - 896 is the float exponent, and E mod 512 = (E - 896 + 384) mod 512
  const unsigned t = __funnelshift_l(l, h, 3) - 0xC0000000u;
  const unsigned hb = (t & 0x7FFFFFFFu) | sign;
  const float ft = __fsub_rn(__uint_as_float(0x4B000000u | ((l >> 6) & 0x7FFFFFu)), 8388608.0f);
  const unsigned scale = (hb & 0xFF800000u) - (46u << 23);
  float hi = __uint_as_float(hb);
  float lo = __fmul_rn(ft, __uint_as_float(scale));
  const unsigned ax = h & 0x7FFFFFFFu;
  if (ax - (943u << 20) >= ((1151u - 943u) << 20)) {  // outside [2^-80, 2^128)
    const unsigned E = ax >> 20;
    if (E >= 897u && E <= 1150u) {
      lo = 0.0f;                          // hi is exact, lo would be subnormal
    } else if (E < 897u) {
      hi = __uint_as_float(sign);
      lo = 0.0f;
    } else {
      hi = __uint_as_float(sign | 0x7F800000u | ((E == 2047u && ((h & 0xFFFFFu) | l)) ? 0x400000u : 0u));
      lo = 0.0f;
    }
  }
  return make_float2(hi, lo);
}

// Exact float -> double by bit manipulation (denormal floats flush to 0).
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7FFFFFFFu;
  unsigned hi = (u & 0x80000000u) | ((a >> 3) + (896u << 20));
  unsigned lo = u << 29;
  if (a - 0x00800000u >= 0x7F000000u) {  // zero, subnormal, inf or nan
    const unsigned e = a >> 23;
    hi = (u & 0x80000000u) | (e == 255u ? (0x7FF00000u | ((a & 0x7FFFFFu) ? 0x80000u : 0u)) : 0u);
    lo = 0u;
  }
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
// Arithmetic policies. TX: input storage as the kernel reads it; TY: output
// storage; C: coefficient; E: packed ELL entry {delta, coefficient}.
// ---------------------------------------------------------------------------
template <int AR> struct Ar;

template <> struct Ar<AR_F32> {
  using TX = float;
  using TY = float;
  using C = float;
  using Acc = float;
  using Dsum = float;
  using E = int2;
  __device__ static const C* tab(const KPlan& P) { return P.tab_f; }
  __device__ static const C* diag(const KPlan& P) { return P.diag_f; }
  __device__ static const E* ell(const KPlan& P) { return (const E*)P.ell_pf; }
  __device__ static int ell_delta(E e) { return e.x; }
  __device__ static C ell_coef(E e) { return __int_as_float(e.y); }
  __device__ static bool nz(C c) { return c != 0.0f; }
  __device__ static Acc azero() { return 0.0f; }
  __device__ static void fma(Acc& a, C c, TX x) { a = __fmaf_rn(c, x, a); }
  __device__ static Dsum dzero() { return 0.0f; }
  __device__ static void dadd(Dsum& d, C c) { d = __fadd_rn(d, c); }
  __device__ static Acc dmul(Dsum d, TX x) { return __fmul_rn(d, x); }
  __device__ static void dmadd(Dsum& d, C v, Dsum u) { d = __fmaf_rn(v, u, d); }
  __device__ static void acc_mul(Acc& a, C v, Acc g) { a = __fmaf_rn(v, g, a); }
  __device__ static TY out(Acc a) { return a; }
  __device__ static TY add_out(TY a, TY b) { return __fadd_rn(a, b); }
  __device__ static C cmul(C a, C b) { return __fmul_rn(a, b); }
};

template <> struct Ar<AR_F64> {
  using TX = double;
  using TY = double;
  using C = double;
  using Acc = double;
  using Dsum = double;
  using E = int4;
  __device__ static const C* tab(const KPlan& P) { return P.tab_d; }
  __device__ static const C* diag(const KPlan& P) { return P.diag_d; }
  __device__ static const E* ell(const KPlan& P) { return (const E*)P.ell_pd; }
  __device__ static int ell_delta(E e) { return e.x; }
  __device__ static C ell_coef(E e) { return __hiloint2double(e.w, e.z); }
  __device__ static bool nz(C c) { return c != 0.0; }
  __device__ static Acc azero() { return 0.0; }
  __device__ static void fma(Acc& a, C c, TX x) { a = __fma_rn(c, x, a); }
  __device__ static Dsum dzero() { return 0.0; }
  __device__ static void dadd(Dsum& d, C c) { d = __dadd_rn(d, c); }
  __device__ static Acc dmul(Dsum d, TX x) { return __dmul_rn(d, x); }
  __device__ static void dmadd(Dsum& d, C v, Dsum u) { d = __fma_rn(v, u, d); }
  __device__ static void acc_mul(Acc& a, C v, Acc g) { a = __fma_rn(v, g, a); }
  __device__ static TY out(Acc a) { return a; }
  __device__ static TY add_out(TY a, TY b) { return __dadd_rn(a, b); }
  __device__ static C cmul(C a, C b) { return __dmul_rn(a, b); }
};

template <> struct Ar<AR_DF64> {
  using TX = float2;  // pre-split (hi, lo) input
  using TY = double;
  using C = float2;
  using Acc = DF;
  using Dsum = DF;
  using E = int4;
  __device__ static const C* tab(const KPlan& P) { return P.tab_df; }
  __device__ static const C* diag(const KPlan& P) { return P.diag_df; }
  __device__ static const E* ell(const KPlan& P) { return (const E*)P.ell_pdf; }
  __device__ static int ell_delta(E e) { return e.x; }
  __device__ static C ell_coef(E e) { return make_float2(__int_as_float(e.z), __int_as_float(e.w)); }
  __device__ static bool nz(C c) { return c.x != 0.0f; }
  __device__ static Acc azero() { return DF{0.f, 0.f}; }
  __device__ static void fma(Acc& a, C c, TX x) { df_fma(a, c, x.x, x.y); }
  __device__ static Dsum dzero() { return DF{0.f, 0.f}; }
  __device__ static void dadd(Dsum& d, C c) { df_add(d, c); }
  __device__ static Acc dmul(Dsum d, TX x) {
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
  __device__ static TY out(Acc a) { return df_to_double(a); }
  __device__ static TY add_out(TY a, TY b) { return __dadd_rn(a, b); }
  // product of two coefficients as a normalised float pair (Dekker product
  // with the cross terms, then a fast two-sum): relative error ~2^-46
  __device__ static C cmul(C a, C b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float t = __fadd_rn(p, e);
    return make_float2(t, __fsub_rn(e, __fsub_rn(t, p)));
  }
};

// Vector policies: TX/TY/Acc hold W right-hand sides of one state; the
// coefficient, diagonal-sum and ELL types stay the scalar policy's.
template <> struct Ar<AR_F32V2> : Ar<AR_F32> {
  using TX = float2;
  using TY = float2;
  using Acc = float2;
  __device__ static Acc azero() { return make_float2(0.f, 0.f); }
  __device__ static void fma(Acc& a, C c, TX x) {
    a.x = __fmaf_rn(c, x.x, a.x);
    a.y = __fmaf_rn(c, x.y, a.y);
  }
  __device__ static Acc dmul(Dsum d, TX x) { return make_float2(__fmul_rn(d, x.x), __fmul_rn(d, x.y)); }
  __device__ static void acc_mul(Acc& a, C v, Acc g) {
    a.x = __fmaf_rn(v, g.x, a.x);
    a.y = __fmaf_rn(v, g.y, a.y);
  }
  __device__ static TY out(Acc a) { return a; }
  __device__ static TY add_out(TY a, TY b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
};

template <> struct Ar<AR_F32V4> : Ar<AR_F32> {
  using TX = float4;
  using TY = float4;
  using Acc = float4;
  __device__ static Acc azero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ static void fma(Acc& a, C c, TX x) {
    a.x = __fmaf_rn(c, x.x, a.x);
    a.y = __fmaf_rn(c, x.y, a.y);
    a.z = __fmaf_rn(c, x.z, a.z);
    a.w = __fmaf_rn(c, x.w, a.w);
  }
  __device__ static Acc dmul(Dsum d, TX x) {
    return make_float4(__fmul_rn(d, x.x), __fmul_rn(d, x.y), __fmul_rn(d, x.z), __fmul_rn(d, x.w));
  }
  __device__ static void acc_mul(Acc& a, C v, Acc g) {
    a.x = __fmaf_rn(v, g.x, a.x);
    a.y = __fmaf_rn(v, g.y, a.y);
    a.z = __fmaf_rn(v, g.z, a.z);
    a.w = __fmaf_rn(v, g.w, a.w);
  }
  __device__ static TY out(Acc a) { return a; }
  __device__ static TY add_out(TY a, TY b) {
    return make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
  }
};

struct DF2 {  // two right-hand sides' double-float accumulators
  DF a, b;
};

template <> struct Ar<AR_DF64V2> : Ar<AR_DF64> {
  using TX = float4;  // (hi, lo) of two consecutive right-hand sides
  using TY = double2;
  using Acc = DF2;
  __device__ static Acc azero() { return DF2{DF{0.f, 0.f}, DF{0.f, 0.f}}; }
  __device__ static void fma(Acc& a, C c, TX x) {
    df_fma(a.a, c, x.x, x.y);
    df_fma(a.b, c, x.z, x.w);
  }
  __device__ static Acc dmul(Dsum d, TX x) {
    const float2 n = df_norm(d);
    DF2 r = azero();
    df_fma(r.a, n, x.x, x.y);
    df_fma(r.b, n, x.z, x.w);
    return r;
  }
  __device__ static void acc_mul(Acc& a, C v, Acc g) {
    const float2 na = df_norm(g.a);
    df_fma(a.a, v, na.x, na.y);
    const float2 nb = df_norm(g.b);
    df_fma(a.b, v, nb.x, nb.y);
  }
  __device__ static TY out(Acc a) { return make_double2(df_to_double(a.a), df_to_double(a.b)); }
  __device__ static TY add_out(TY a, TY b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
};

template <> struct Ar<AR_F64V2> : Ar<AR_F64> {
  using TX = double2;  // two consecutive right-hand sides (or the (re, im) of one complex value)
  using TY = double2;
  using Acc = double2;
  __device__ static Acc azero() { return make_double2(0.0, 0.0); }
  __device__ static void fma(Acc& a, C c, TX x) {
    a.x = __fma_rn(c, x.x, a.x);
    a.y = __fma_rn(c, x.y, a.y);
  }
  __device__ static Acc dmul(Dsum d, TX x) { return make_double2(__dmul_rn(d, x.x), __dmul_rn(d, x.y)); }
  __device__ static void acc_mul(Acc& a, C v, Acc g) {
    a.x = __fma_rn(v, g.x, a.x);
    a.y = __fma_rn(v, g.y, a.y);
  }
  __device__ static TY out(Acc a) { return a; }
  __device__ static TY add_out(TY a, TY b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
};

// y = r + i t for the rounded (re, im) values r = H_re x and t = H_im x of
// one element, or r - i t (conj: the adjoint's H_re^T - i H_im^T)
__device__ __forceinline__ float2 cx_comb(float2 r, float2 t, bool conj) {
  return conj ? make_float2(__fadd_rn(r.x, t.y), __fsub_rn(r.y, t.x))
              : make_float2(__fsub_rn(r.x, t.y), __fadd_rn(r.y, t.x));
}
__device__ __forceinline__ double2 cx_comb(double2 r, double2 t, bool conj) {
  return conj ? make_double2(__dadd_rn(r.x, t.y), __dsub_rn(r.y, t.x))
              : make_double2(__dsub_rn(r.x, t.y), __dadd_rn(r.y, t.x));
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
