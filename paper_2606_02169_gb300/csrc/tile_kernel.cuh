// y = H x in the leaf-tiled form (pull form, Sec. II: every output element is
// written by exactly one thread; no atomics). See KTile for the decomposition
// k = (b R + r) F + f. A CTA of F*nvec threads (rounded up to a warp) walks a
// contiguous range of rows; thread t always owns leaf element t, so
//   * its leaf diagonal, leaf factors v_g and leaf-only hops are read from
//     shared memory once per CTA (no per-state table traffic);
//   * every other coefficient is uniform across the CTA for a row: members on
//     high digits are evaluated once per block, members with a mid digit once
//     per row, and both are compacted to the admissible ones (Sec. IV.B
//     steps 2-4), so an inadmissible hop costs nothing.
// All gathers of a row are independent loads: their addresses need no table
// lookup, only the uniform offset and the thread's element index.
#pragma once

#include "device_common.cuh"

namespace hm {

// Byte offsets of each thread's element index are formed as 32-bit unsigned
// products: the tile form requires D * nvec < 2^31 (checked when the tables
// are built).

template <int AR>
__device__ __forceinline__ typename Ar<AR>::C to_coef(double v);
template <>
__device__ __forceinline__ float to_coef<AR_F32>(double v) { return __double2float_rn(v); }
template <>
__device__ __forceinline__ double to_coef<AR_F64>(double v) { return v; }
template <>
__device__ __forceinline__ float2 to_coef<AR_DF64>(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

template <int AR>
__device__ __forceinline__ typename Ar<AR>::Dsum to_dsum(double v);
template <>
__device__ __forceinline__ float to_dsum<AR_F32>(double v) { return __double2float_rn(v); }
template <>
__device__ __forceinline__ double to_dsum<AR_F64>(double v) { return v; }
template <>
__device__ __forceinline__ DF to_dsum<AR_DF64>(double v) {
  const float hi = __double2float_rn(v);
  return DF{hi, __double2float_rn(v - (double)hi)};
}

template <int AR> struct TilePtr;
template <> struct TilePtr<AR_F32> {
  __device__ static const float* dF(const KTile& k) { return k.dF_f; }
  __device__ static const float* v(const KTile& k) { return k.v_f; }
  __device__ static const float* fs(const KTile& k) { return k.fs_f; }
};
template <> struct TilePtr<AR_DF64> {
  __device__ static const float2* dF(const KTile& k) { return k.dF_df; }
  __device__ static const float2* v(const KTile& k) { return k.v_df; }
  __device__ static const float2* fs(const KTile& k) { return k.fs_df; }
};
template <> struct TilePtr<AR_F64> {
  __device__ static const double* dF(const KTile& k) { return k.dF_d; }
  __device__ static const double* v(const KTile& k) { return k.v_d; }
  __device__ static const double* fs(const KTile& k) { return k.fs_d; }
};

constexpr int kTileRowsMax = 64;  // rows evaluated at once (R <= 64 by construction)

// Shared-memory carve of the tile kernel.
template <int AR>
struct TileSm {
  using C = typename Ar<AR>::C;
  using Dsum = typename Ar<AR>::Dsum;
  C* dF;          // [F]
  C* v;           // [(G-1) F]
  int* fix;       // [(G-1) F]
  int* fs_n;      // [F]
  int* fs_off;    // [fs_w F]
  C* fs;          // [fs_w F]
  int* hd;        // [64] high digits of the current block
  long long* boff;  // [n_bmem] block-uniform members, compacted per group
  C* bu;            // [n_bmem]
  int* bn;          // [G] active members of each group
  double* bdiag;    // [G] sum of the group's diagonal members
  long long* roff;  // [rows * n_rmem] row members, compacted per (row, group)
  C* ru;            // [rows * n_rmem]
  int* rn;          // [rows * G]
  Dsum* rdiag;      // [rows * G] block + row diagonal sums
  int* gdiag;       // [G] group has diagonal members
  unsigned char* rdig;  // [R * nmid] mid digits of each row of a block
};

// rows = R (<= 64); the mid-digit table holds R * nmid bytes, nmid <= 6 (R <= 64)
template <int AR>
__host__ __device__ inline size_t tile_smem_bytes(int F, int G, int fs_w, int n_bmem, int n_rmem, int rows) {
  using C = typename Ar<AR>::C;
  using Dsum = typename Ar<AR>::Dsum;
  auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
  return al(F * sizeof(C)) + al((size_t)(G - 1) * F * sizeof(C)) + al((size_t)(G - 1) * F * 4) + al(F * 4) +
         al((size_t)fs_w * F * 4) + al((size_t)fs_w * F * sizeof(C)) + al(64 * 4) + al(n_bmem * 8) +
         al(n_bmem * sizeof(C)) + al(G * 4) + al(G * 8) + al((size_t)rows * n_rmem * 8) +
         al((size_t)rows * n_rmem * sizeof(C)) + al((size_t)rows * G * 4) + al((size_t)rows * G * sizeof(Dsum)) +
         al(G * 4) + al((size_t)rows * 8);
}

template <int AR>
__device__ inline TileSm<AR> tile_carve(unsigned char* sm, const KTile& k, int rows) {
  using C = typename Ar<AR>::C;
  using Dsum = typename Ar<AR>::Dsum;
  auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
  const int F = k.F, G = k.G;
  TileSm<AR> S;
  size_t o = 0;
  S.dF = (C*)(sm + o);      o += al(F * sizeof(C));
  S.v = (C*)(sm + o);       o += al((size_t)(G - 1) * F * sizeof(C));
  S.fix = (int*)(sm + o);   o += al((size_t)(G - 1) * F * 4);
  S.fs_n = (int*)(sm + o);  o += al(F * 4);
  S.fs_off = (int*)(sm + o); o += al((size_t)k.fs_w * F * 4);
  S.fs = (C*)(sm + o);      o += al((size_t)k.fs_w * F * sizeof(C));
  S.hd = (int*)(sm + o);    o += al(64 * 4);
  S.boff = (long long*)(sm + o); o += al(k.n_bmem * 8);
  S.bu = (C*)(sm + o);      o += al(k.n_bmem * sizeof(C));
  S.bn = (int*)(sm + o);    o += al(G * 4);
  S.bdiag = (double*)(sm + o); o += al(G * 8);
  S.roff = (long long*)(sm + o); o += al((size_t)rows * k.n_rmem * 8);
  S.ru = (C*)(sm + o);      o += al((size_t)rows * k.n_rmem * sizeof(C));
  S.rn = (int*)(sm + o);    o += al((size_t)rows * G * 4);
  S.rdiag = (Dsum*)(sm + o); o += al((size_t)rows * G * sizeof(Dsum));
  S.gdiag = (int*)(sm + o); o += al(G * 4);
  S.rdig = (unsigned char*)(sm + o);
  return S;
}

// member coefficient at the given digits (target-digit table, zero if inadmissible)
__device__ __forceinline__ double member_u(const KTile& k, const KTMem& m, int na, int nb) {
  return __ldg(k.tab + m.tab + na * m.db + nb);
}

// digit of non-leaf site s for row r of the current block (high digits in
// hd, mid digits tabulated per row)
__device__ __forceinline__ int row_digit(const KTile& k, const int* hd, const unsigned char* rdig, int s, int r) {
  return s < k.nhigh ? hd[s] : (int)rdig[r * k.nmid + (s - k.nhigh)];
}

// Block-uniform part: high digits, then members on high sites only, compacted
// per group (one warp per group; fixed-order sums of diagonal members).
template <int AR>
__device__ void tile_eval_block(const KTile& k, const TileSm<AR>& S, long long blk) {
  for (int s = threadIdx.x; s < k.nhigh; s += blockDim.x) {
    const KTileSite st = k.sites[s];
    S.hd[s] = (int)((blk / st.stride) % st.d);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int g = warp; g < k.G; g += nwarp) {
    const int m0 = __ldg(k.bgrp + g), m1 = __ldg(k.bgrp + g + 1);
    int count = 0;
    double dsum = 0.0;
    for (int base = m0; base < m1; base += 32) {
      const int j = base + lane;
      double u = 0.0;
      bool dg = false;
      KTMem m{};
      if (j < m1) {
        m = k.bmem[j];
        u = member_u(k, m, S.hd[m.sa], m.sb == 255 ? 0 : S.hd[m.sb]);
        dg = m.diag;
      }
      if (dg) dsum += u;
      const bool act = j < m1 && !dg && u != 0.0;
      const unsigned msk = __ballot_sync(0xffffffffu, act);
      if (act) {
        const int pos = m0 + count + __popc(msk & ((1u << lane) - 1u));
        S.boff[pos] = m.off;
        S.bu[pos] = to_coef<AR>(u);
      }
      count += __popc(msk);
    }
    for (int o = 16; o > 0; o >>= 1) dsum = __dadd_rn(dsum, __shfl_xor_sync(0xffffffffu, dsum, o));
    if (lane == 0) {
      S.bn[g] = count;
      S.bdiag[g] = dsum;
    }
  }
  __syncthreads();
}

// Row part for rows r0 .. r0+nr-1 of the current block: members with a mid
// digit, compacted per (row, group) by one thread per pair in member order;
// diagonal sums include the block part.
template <int AR>
__device__ void tile_eval_rows(const KTile& k, const TileSm<AR>& S, int r0, int nr) {
  const int nrm = k.n_rmem, G = k.G;
  for (int p = threadIdx.x; p < nr * G; p += blockDim.x) {
    const int rr = p / G, g = p - rr * G;
    const int r = r0 + rr;
    const int m0 = __ldg(k.rgrp + g), m1 = __ldg(k.rgrp + g + 1);
    int count = 0;
    double dsum = 0.0;
    for (int j = m0; j < m1; ++j) {
      const KTMem m = k.rmem[j];
      const double u = member_u(k, m, row_digit(k, S.hd, S.rdig, m.sa, r),
                                m.sb == 255 ? 0 : row_digit(k, S.hd, S.rdig, m.sb, r));
      if (m.diag) {
        dsum += u;
      } else if (u != 0.0) {
        S.roff[rr * nrm + m0 + count] = m.off;
        S.ru[rr * nrm + m0 + count] = to_coef<AR>(u);
        ++count;
      }
    }
    S.rn[rr * G + g] = count;
    S.rdiag[rr * G + g] = to_dsum<AR>(__dadd_rn(S.bdiag[g], dsum));
  }
  __syncthreads();
}

// RS consecutive rows starting at row `rb` of block blk (rr0 = rb - r0 of
// the evaluated range); rows at or beyond nrows are skipped.
template <int AR, int RS>
__device__ __forceinline__ void tile_rows(const KTile& k, const TileSm<AR>& S, const typename Ar<AR>::TX* __restrict__ x,
                                          typename Ar<AR>::TY* __restrict__ y, long long blk, int rb, int rr0,
                                          int nrows, int t, int f, unsigned rowE) {
  using A = Ar<AR>;
  using TX = typename A::TX;
  using C = typename A::C;
  using Acc = typename A::Acc;
  using Dsum = typename A::Dsum;
  const int G = k.G, F = k.F;
  unsigned kk[RS];
  bool ok[RS];
#pragma unroll
  for (int s = 0; s < RS; ++s) {
    ok[s] = rr0 + s < nrows;
    kk[s] = (unsigned)(blk * k.R + rb + s) * rowE + (unsigned)t;
  }
  Acc acc[RS];
  // ---- diagonal: block/row part + leaf part + cross (leaf factor x uniform) ----
  {
    const C dF = S.dF[f];
    Dsum ds[RS];
#pragma unroll
    for (int s = 0; s < RS; ++s) {
      ds[s] = A::dzero();
      if (ok[s]) {
        ds[s] = S.rdiag[(rr0 + s) * G];
        A::dadd(ds[s], dF);
      }
    }
    for (int g = 1; g < G; ++g) {
      if (!S.gdiag[g]) continue;
      const C v = S.v[(g - 1) * F + f];
#pragma unroll
      for (int s = 0; s < RS; ++s)
        if (ok[s]) A::dmadd(ds[s], v, S.rdiag[(rr0 + s) * G + g]);
    }
#pragma unroll
    for (int s = 0; s < RS; ++s) acc[s] = A::dmul(ds[s], ok[s] ? __ldg(x + kk[s]) : TX{});
  }
  // ---- group 0 (leaf factor 1): block members, then row members ----
  {
    const int n = S.bn[0];
    const long long* __restrict__ bo = S.boff;
    const C* __restrict__ bu = S.bu;
#pragma unroll 2
    for (int j = 0; j < n; ++j) {
      const C u = bu[j];
      const TX* __restrict__ q = x + bo[j];
#pragma unroll
      for (int s = 0; s < RS; ++s)
        if (ok[s]) A::fma(acc[s], u, __ldg(q + kk[s]));
    }
#pragma unroll
    for (int s = 0; s < RS; ++s) {
      if (!ok[s]) continue;
      const int base = (rr0 + s) * k.n_rmem;
      const int nr = S.rn[(rr0 + s) * G];
      for (int j = 0; j < nr; ++j) {
        const TX* __restrict__ q = x + S.roff[base + j];
        A::fma(acc[s], S.ru[base + j], __ldg(q + kk[s]));
      }
    }
  }
  // ---- groups with a leaf factor ----
  for (int g = 1; g < G; ++g) {
    const int nb = S.bn[g];
    int nrs[RS];
    int any = nb;
#pragma unroll
    for (int s = 0; s < RS; ++s) {
      nrs[s] = ok[s] ? S.rn[(rr0 + s) * G + g] : 0;
      any |= nrs[s];
    }
    if (!any) continue;
    const C v = S.v[(g - 1) * F + f];
    // v = 0: gather the in-range element with the leaf shift undone (times 0)
    const TX* __restrict__ xg = x + S.fix[(g - 1) * F + f];
    Acc ag[RS];
#pragma unroll
    for (int s = 0; s < RS; ++s) ag[s] = A::azero();
    const int mb = __ldg(k.bgrp + g);
    for (int j = 0; j < nb; ++j) {
      const C u = S.bu[mb + j];
      const TX* __restrict__ q = xg + S.boff[mb + j];
#pragma unroll
      for (int s = 0; s < RS; ++s)
        if (ok[s]) A::fma(ag[s], u, __ldg(q + kk[s]));
    }
    const int mr = __ldg(k.rgrp + g);
#pragma unroll
    for (int s = 0; s < RS; ++s) {
      const int base = (rr0 + s) * k.n_rmem + mr;
      for (int j = 0; j < nrs[s]; ++j) {
        const TX* __restrict__ q = xg + S.roff[base + j];
        A::fma(ag[s], S.ru[base + j], __ldg(q + kk[s]));
      }
    }
#pragma unroll
    for (int s = 0; s < RS; ++s) A::acc_mul(acc[s], v, ag[s]);
  }
  // ---- leaf-only hops (per-thread list) ----
  {
    const int n = S.fs_n[f];
    for (int w = 0; w < n; ++w) {
      const int o = S.fs_off[w * F + f];
      const C c = S.fs[w * F + f];
      const TX* __restrict__ q = x + o;
#pragma unroll
      for (int s = 0; s < RS; ++s)
        if (ok[s]) A::fma(acc[s], c, __ldg(q + kk[s]));
    }
  }
  typename A::TY* __restrict__ yy = y;
#pragma unroll
  for (int s = 0; s < RS; ++s)
    if (ok[s]) yy[kk[s]] = A::out(acc[s]);
}

template <int AR> struct TileMinBlocks { static constexpr int v = 1; };
template <> struct TileMinBlocks<AR_F32> { static constexpr int v = 2; };

// CTA c walks rows [c*T, (c+1)*T) of the nblk*R rows (T = rows_per_cta).
template <int AR, int RS>
__global__ void __launch_bounds__(512, TileMinBlocks<AR>::v)
k_tile(const KTile k, const typename Ar<AR>::TX* __restrict__ x, typename Ar<AR>::TY* __restrict__ y,
       long long rows_per_cta, KGate gate) {
  if (gate_closed(gate)) return;
  using C = typename Ar<AR>::C;
  extern __shared__ __align__(16) unsigned char sm[];
  const int rows_cap = k.R < kTileRowsMax ? k.R : kTileRowsMax;
  const TileSm<AR> S = tile_carve<AR>(sm, k, rows_cap);
  const int F = k.F;
  // per-CTA copy of the leaf tables
  {
    const C* dF = TilePtr<AR>::dF(k);
    const C* v = TilePtr<AR>::v(k);
    const C* fs = TilePtr<AR>::fs(k);
    for (int i = threadIdx.x; i < F; i += blockDim.x) {
      S.dF[i] = dF[i];
      S.fs_n[i] = k.fs_n[i];
    }
    for (int i = threadIdx.x; i < (k.G - 1) * F; i += blockDim.x) {
      S.v[i] = v[i];
      S.fix[i] = k.fix[i];
    }
    for (int i = threadIdx.x; i < k.fs_w * F; i += blockDim.x) {
      S.fs[i] = fs[i];
      S.fs_off[i] = k.fs_off[i];
    }
    for (int i = threadIdx.x; i < k.R * k.nmid; i += blockDim.x) {
      const int r = i / k.nmid, s = k.nhigh + (i - r * k.nmid);
      const KTileSite st = k.sites[s];
      S.rdig[i] = (unsigned char)((r / (int)st.stride) % st.d);
    }
    // groups with diagonal members (on high or mid sites)
    for (int g = threadIdx.x; g < k.G; g += blockDim.x) {
      int has = 0;
      for (int j = k.bgrp[g]; j < k.bgrp[g + 1]; ++j) has |= k.bmem[j].diag;
      for (int j = k.rgrp[g]; j < k.rgrp[g + 1]; ++j) has |= k.rmem[j].diag;
      S.gdiag[g] = has;
    }
  }
  __syncthreads();
  const unsigned rowE = (unsigned)(F * k.nvec);
  const int t = threadIdx.x;
  const bool active = t < (int)rowE;
  const int f = active ? t / k.nvec : 0;
  const long long total = k.nblk * k.R;
  long long row = (long long)blockIdx.x * rows_per_cta;
  const long long end = row + rows_per_cta < total ? row + rows_per_cta : total;
  long long cur = -1;
  while (row < end) {
    const long long blk = row / k.R;
    const int r0 = (int)(row - blk * k.R);
    long long left = end - row;
    int nr = k.R - r0;
    if (nr > rows_cap) nr = rows_cap;
    if (nr > left) nr = (int)left;
    if (blk != cur) {
      tile_eval_block<AR>(k, S, blk);
      cur = blk;
    }
    tile_eval_rows<AR>(k, S, r0, nr);
    if (active)
      for (int rr = 0; rr < nr; rr += RS) tile_rows<AR, RS>(k, S, x, y, blk, r0 + rr, rr, nr, t, f, rowE);
    __syncthreads();
    row += nr;
  }
}

}  // namespace hm

namespace hm {

template <int AR, int RS>
static cudaError_t tile_launch(const KTile& k, const void* x, void* y, cudaStream_t st, int ctas, KGate gate) {
  using TX = typename Ar<AR>::TX;
  using TY = typename Ar<AR>::TY;
  const int rows_cap = k.R < kTileRowsMax ? k.R : kTileRowsMax;
  const size_t smem = tile_smem_bytes<AR>(k.F, k.G, k.fs_w, k.n_bmem, k.n_rmem, rows_cap);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  static size_t attr_set = 0;
  if (smem > 48 * 1024 && smem > attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tile<AR, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = smem;
  }
  long long grid = ctas;
  if (grid <= 0) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tile<AR, RS>, k.nt, smem);
    grid = (long long)num_sms() * (occ > 0 ? occ : 1);
  }
  const long long total = k.nblk * k.R;
  if (grid > total) grid = total;
  if (grid < 1) grid = 1;
  const long long per = (total + grid - 1) / grid;
  grid = (total + per - 1) / per;
  k_tile<AR, RS><<<(unsigned)grid, k.nt, smem, st>>>(k, (const TX*)x, (TY*)y, per, gate);
  return cudaGetLastError();
}

// rows per iteration: 0 = default, else 1, 2 or 4
template <int AR>
cudaError_t launch_tile_t(const KTile& k, const void* x, void* y, cudaStream_t st, TuneCfg cfg) {
  const int rs = cfg.s ? cfg.s : (AR == AR_F32 ? 4 : 2);
  switch (rs) {
    case 1: return tile_launch<AR, 1>(k, x, y, st, cfg.ctas, KGate{cfg.gate, cfg.gate_run});
    case 4: return tile_launch<AR, 4>(k, x, y, st, cfg.ctas, KGate{cfg.gate, cfg.gate_run});
    default: return tile_launch<AR, 2>(k, x, y, st, cfg.ctas, KGate{cfg.gate, cfg.gate_run});
  }
}

}  // namespace hm
