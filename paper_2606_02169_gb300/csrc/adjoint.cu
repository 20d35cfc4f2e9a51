// Reverse mode of y = H(c) x:
//   gx = H^T gy  -- the apply kernel run on the transposed channel set (for a
//                   self-adjoint real H the same tables);
//   g_t = sum_F gy_F (O_t x)_F -- per-term coupling gradients. O_t is term t
//                   with unit coefficient; its channels follow the same source
//                   reconstruction as the forward map (Sec. IV.B steps 1-5).
// g_t is accumulated per lane as a double-float sum on the FP32 pipe (GB300
// runs FP64 FMA at about 1/70 of the FP32 rate): FP64 inputs are split into
// (hi, lo) float pairs as they are read, the product gy * x is formed from the
// exact product of the hi parts (Dekker) plus the cross terms, and the
// coefficient product and the sum use the error-free transformations of
// device_common.cuh (about 2^-46 relative overall). Lanes are reduced per
// warp by shuffles in a fixed order, per CTA through shared memory in FP64 in
// warp order, and across CTAs by a second kernel in CTA order: a fixed-order
// reduction, bit-reproducible for a fixed grid.
#include <algorithm>

#include "device_common.cuh"

namespace hm {

// input element as a (hi, lo) float pair
__device__ __forceinline__ float2 as_pair(float v) { return make_float2(v, 0.0f); }
__device__ __forceinline__ float2 as_pair(double v) { return split_f64(v); }
__device__ __forceinline__ float2 as_pair(float2 v) { return v; }  // already split

// product of two float pairs without the lo*lo term: (s, c) with s + c equal
// to a * b to about 2^-46 relative
__device__ __forceinline__ float2 pair_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return make_float2(p, e);
}

constexpr int kGradWarps = 8;
constexpr int kGradV = 8;

template <class T>
__global__ void __launch_bounds__(256)
k_term_grad(const KPlan P, const T* __restrict__ gy, const T* __restrict__ x, long long nvec,
            double* __restrict__ partial) {
  extern __shared__ double sm[];  // [kGradWarps][nterms]
  const int nterms = P.nterms;
  for (int i = threadIdx.x; i < kGradWarps * nterms; i += blockDim.x) sm[i] = 0.0;
  __syncthreads();
  constexpr int V = kGradV;
  constexpr int WT = 32 * V;
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const long long tpb = (P.B + WT - 1) / WT;
  const long long ntiles = P.nblk * tpb;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  double* mysm = sm + wid * nterms;
  long long prev_hb = -1;
  int nh0 = 0, nh1 = 0;
  for (long long wt = gw; wt < ntiles; wt += nw) {
    const long long hb = wt / tpb;
    const int lo0 = (int)(wt - hb * tpb) * WT;
    if (hb != prev_hb) {
      prev_hb = hb;
      high_digits(P, hb, nh0, nh1);
    }
    int lo[V];
    bool ok[V];
    long long kk[V];
    uint32_t pk[V];
    float2 g1[V];  // gy of the row (nvec == 1)
    float2 d0[V];  // sum_v gy x of the row itself: shared by every diagonal channel
#pragma unroll
    for (int v = 0; v < V; ++v) {
      lo[v] = lo0 + lane + 32 * v;
      ok[v] = lo[v] < P.B;
      if (!ok[v]) lo[v] = 0;
      kk[v] = hb * P.B + lo[v];
      pk[v] = __ldg(P.ptab + lo[v]);
      g1[v] = (nvec == 1 && ok[v]) ? as_pair(gy[kk[v]]) : make_float2(0.f, 0.f);
      d0[v] = make_float2(0.f, 0.f);
      if (ok[v]) {
        if (nvec == 1) {
          d0[v] = pair_mul(g1[v], as_pair(x[kk[v]]));
        } else {
          DF sd{0.f, 0.f};
          for (long long u = 0; u < nvec; ++u) df_add(sd, pair_mul(as_pair(gy[kk[v] * nvec + u]), as_pair(x[kk[v] * nvec + u])));
          d0[v] = df_norm(sd);
        }
      }
    }
    int cur = -1;
    DF acc{0.f, 0.f};
    for (int c = 0; c <= P.nterm_ch; ++c) {
      const bool last = (c == P.nterm_ch);
      KTermChan ch;
      if (!last) ch = P.tch[c];
      if (last || ch.term != cur) {
        if (cur >= 0) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float2 w = make_float2(__shfl_xor_sync(0xffffffffu, acc.s, o),
                                         __shfl_xor_sync(0xffffffffu, acc.c, o));
            df_add(acc, w);
          }
          if (lane == 0) mysm[cur] += df_to_double(acc);
        }
        if (last) break;
        cur = ch.term;
        acc = DF{0.f, 0.f};
      }
      const KSite si = P.sites[ch.si];
      const bool single = ch.sj == 255;
      KSite sj{};
      if (!single) sj = P.sites[ch.sj];
      const int hi_i = si.is_low ? 0 : high_digit(ch.si, nh0, nh1);
      const int hi_j = (single || sj.is_low) ? 0 : high_digit(ch.sj, nh0, nh1);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int ni = si.is_low ? low_digit(pk[v], si.lbit, si.lwid) : hi_i;
        const int nj = single ? 0 : (sj.is_low ? low_digit(pk[v], sj.lbit, sj.lwid) : hi_j);
        const float2 cf = P.ttab_df[ch.tab + ni * ch.dj + nj];
        if (ok[v] && cf.x != 0.0f) {
          if (ch.off == 0) {
            df_fma(acc, cf, d0[v].x, d0[v].y);
          } else if (nvec == 1) {
            const float2 t = pair_mul(g1[v], as_pair(x[kk[v] + ch.off]));
            df_fma(acc, cf, t.x, t.y);
          } else {
            const T* g = gy + kk[v] * nvec;
            const T* xs = x + (kk[v] + ch.off) * nvec;
            DF s{0.f, 0.f};
            for (long long u = 0; u < nvec; ++u) df_add(s, pair_mul(as_pair(g[u]), as_pair(xs[u])));
            const float2 n = df_norm(s);
            df_fma(acc, cf, n.x, n.y);
          }
        }
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nterms; t += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < kGradWarps; ++w) s += sm[w * nterms + t];
    partial[(long long)blockIdx.x * nterms + t] = s;
  }
}

__global__ void k_reduce_partials(const double* __restrict__ partial, int nblocks, int nterms,
                                  double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nterms) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[(long long)b * nterms + t];
  out[t] = s;
}

int grad_grid(const Plan* p) {
  const long long tpb = (p->B + 32 * kGradV - 1) / (32 * kGradV);
  const long long need = (p->nblk * tpb + kGradWarps - 1) / kGradWarps;
  return (int)std::max<long long>(1, std::min<long long>(need, (long long)num_sms() * 4));
}

size_t grad_smem(const Plan* p) { return (size_t)kGradWarps * std::max<size_t>(1, p->terms.size()) * 8; }

// Term gradients into gcoef using `partial` (grid*nterms doubles) as scratch.
// gy and x already split into float pairs (FP64 data)
static int launch_term_grad_split(const Plan* p, const float2* gy, const float2* x, double* gcoef, long long nvec,
                                  double* partial, int grid, cudaStream_t s) {
  const int nterms = (int)p->terms.size();
  if (nterms == 0) return HM_OK;
  const size_t smem = grad_smem(p);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_term_grad<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_term_grad<float2><<<grid, 256, smem, s>>>(p->k, gy, x, nvec, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "term gradient launch");
  k_reduce_partials<<<(nterms + 255) / 256, 256, 0, s>>>(partial, grid, nterms, gcoef);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "gradient reduction launch");
  return HM_OK;
}

int launch_term_grad(const Plan* p, const void* gy, const void* x, double* gcoef, long long nvec,
                     hm_dtype dt, double* partial, int grid, cudaStream_t s) {
  const int nterms = (int)p->terms.size();
  if (nterms == 0) return HM_OK;
  const size_t smem = grad_smem(p);
  cudaError_t e;
  if (dt == HM_F32) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_term_grad<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_term_grad<float><<<grid, 256, smem, s>>>(p->k, (const float*)gy, (const float*)x, nvec, partial);
  } else {
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_term_grad<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_term_grad<double><<<grid, 256, smem, s>>>(p->k, (const double*)gy, (const double*)x, nvec, partial);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "term gradient launch");
  k_reduce_partials<<<(nterms + 255) / 256, 256, 0, s>>>(partial, grid, nterms, gcoef);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "gradient reduction launch");
  return HM_OK;
}

int launch_adjoint(Plan* p, const void* gy, const void* x, void* gx, double* gcoef, long long nvec,
                   hm_dtype dt, cudaStream_t s) {
  if (gx) {
    int rc = apply_on(p, true, gy, gx, nvec, dt, s, tuned_cfg(p, dt, nvec), false);
    if (rc) return rc;
  }
  if (!gcoef) return HM_OK;
  const int nterms = (int)p->terms.size();
  if (grad_smem(p) > 200 * 1024) {
    set_error("too many terms for the gradient reduction (limit 3200)");
    return HM_ERR_UNSUPPORTED;
  }
  const int grid = grad_grid(p);
  const size_t need = (size_t)grid * std::max(1, nterms) * sizeof(double);
  if (p->scratch_bytes < need) {
    // stream-ordered growth: earlier users of the old buffer finish first
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "scratch sync");
    if (p->scratch) cudaFree(p->scratch);
    p->scratch = nullptr;
    p->scratch_bytes = 0;
    e = cudaMalloc(&p->scratch, need);
    if (e != cudaSuccess) {
      p->scratch = nullptr;
      return cuda_fail(e, "gradient scratch allocation");
    }
    p->scratch_bytes = need;
  }
  if (dt == HM_F64) {  // split gy and x once instead of at every gather
    const float2 *gs = nullptr, *xs = nullptr;
    Scratch gsb, xsb;
    int rc = split_vector(gy, p->D * nvec, s, gsb, &gs);
    if (rc == HM_OK) rc = split_vector(x, p->D * nvec, s, xsb, &xs);
    if (rc) return rc;
    return launch_term_grad_split(p, gs, xs, gcoef, nvec, (double*)p->scratch, grid, s);
  }
  return launch_term_grad(p, gy, x, gcoef, nvec, dt, (double*)p->scratch, grid, s);
}

}  // namespace hm
