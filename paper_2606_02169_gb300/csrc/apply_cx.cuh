// Complex H = H_re + i H_im (Sec. IV.A: complex ladder couplings, here the
// imaginary matrix elements of Sy factors) applied in one pass: the general
// kernel's per-element sums of both real operators on the same (re, im)
// element, y = H_re x + i H_im x combined in registers.
//
// The two plans are built on the same sites, so they share the low block,
// its packed digits and the high/low split; per low block the CTA evaluates
// both plans' block-uniform lists into shared memory, and per element a
// thread decodes the state once, gathers x for H_re's hops and for H_im's
// hops (each (re, im) pair one 8- or 16-byte load), rounds both sums and
// writes y once. Each sum takes the operations of the real kernel on the
// (re, im) columns, and the combination is the one rounding the separate
// passes' combine takes, so the result is bit-identical to applying the two
// real operators separately and combining them.
#pragma once

#include <algorithm>

#include "apply_launch.cuh"

namespace hm {

template <int AR, int S, bool FULL, bool NV1>
__device__ __forceinline__ void cx_chunk(const KPlan& Pr, const Lists<AR>& Lr, const KPlan& Pi, const Lists<AR>& Li,
                                         const typename Ar<AR>::TX* __restrict__ x,
                                         typename Ar<AR>::TY* __restrict__ y, int nvec_rt, NvDiv nvdiv,
                                         long long blk, int e_start, bool conj) {
  using A = Ar<AR>;
  const int nvec = NV1 ? 1 : nvec_rt;
  const int belems = Pr.B * nvec;
  const long long ebase = blk * (long long)belems;
  const int e0 = e_start + (int)threadIdx.x;
  bool ok[S];
  int lo[S];
  uint32_t pk[S];
  chunk_states<S, FULL, NV1>(Pr, belems, e0, nvdiv, ok, lo, pk);
  const typename A::TX* __restrict__ xb = x + ebase + e0;
  typename A::Acc ar[S], ai[S];
  chunk_sum<AR, S, FULL, NV1>(Pr, Lr, x, nvec, e0, xb, ok, lo, pk, ar, nullptr);
  chunk_sum<AR, S, FULL, NV1>(Pi, Li, x, nvec, e0, xb, ok, lo, pk, ai, nullptr);
  typename A::TY* __restrict__ yb = y + ebase + e0;
#pragma unroll
  for (int s = 0; s < S; ++s)
    if (FULL || ok[s]) st_y(yb + s * kNT, cx_comb(A::out(ar[s]), A::out(ai[s]), conj));
}

template <int AR, int S, bool NV1>
__device__ __forceinline__ void cx_item(const KPlan& Pr, const Lists<AR>& Lr, const KPlan& Pi, const Lists<AR>& Li,
                                        const typename Ar<AR>::TX* x, typename Ar<AR>::TY* y, int nvec, NvDiv nvdiv,
                                        long long blk, const ChunkPlan& cp, int c, bool conj) {
  if (c < cp.nS) {
    cx_chunk<AR, S, true, NV1>(Pr, Lr, Pi, Li, x, y, nvec, nvdiv, blk, c * kNT * S, conj);
  } else if (c < cp.nS + cp.n1) {
    cx_chunk<AR, 1, true, NV1>(Pr, Lr, Pi, Li, x, y, nvec, nvdiv, blk, cp.nS * kNT * S + (c - cp.nS) * kNT, conj);
  } else {
    cx_chunk<AR, 1, false, NV1>(Pr, Lr, Pi, Li, x, y, nvec, nvdiv, blk, cp.nS * kNT * S + cp.n1 * kNT, conj);
  }
}

// x, y: nvec complex right-hand sides per state, each element one (re, im)
// pair (AR: a two-wide policy). Work is distributed as in k_apply: whole low
// blocks per CTA when there are enough of them, else (block, chunk) items.
// MB: resident CTAs per SM the register allocation must allow (2, or 3 for
// the register-capped variant).
template <int AR, int S, bool NV1, int MB>
__global__ void __launch_bounds__(kNT, MB)
k_apply_cx(const KPlan Pr, const KPlan Pi, const typename Ar<AR>::TX* __restrict__ x,
           typename Ar<AR>::TY* __restrict__ y, int nvec, NvDiv nvdiv, KGate gate, int conj) {
  if (gate_closed(gate)) return;
  extern __shared__ __align__(16) unsigned char sm[];
  const Lists<AR> Lr = carve<AR>(sm, Pr.n_hh_diag + Pr.n_hh, Pr.n_mem, Pr.n_grp_diag + Pr.n_grp, Pr.n_grp_diag);
  const Lists<AR> Li = carve<AR>(sm + cx_lists_bytes<AR>(Pr), Pi.n_hh_diag + Pi.n_hh, Pi.n_mem,
                                 Pi.n_grp_diag + Pi.n_grp, Pi.n_grp_diag);
  load_descriptors<AR>(Pr, Lr);
  load_descriptors<AR>(Pi, Li);
  const bool cj = conj != 0;
  const ChunkPlan cp = chunk_plan(Pr.B * nvec, S);
  const int nchunks = cp.count();
  const long long nblk = Pr.nblk;
  long long cur = -1;
  const long long inflight = (long long)Pr.B * nvec * sizeof(typename Ar<AR>::TX) * gridDim.x;
  long long full = 0;
  if (nblk >= 2LL * gridDim.x && inflight <= kInflightMax) {
    full = (nblk / gridDim.x) * gridDim.x;
    if (2 * (nblk - full) >= gridDim.x) full = nblk;
    for (long long blk = blockIdx.x; blk < full; blk += gridDim.x) {
      eval_block<AR>(Pr, Lr, blk, nvec);
      eval_block<AR>(Pi, Li, blk, nvec);
      for (int c = 0; c < nchunks; ++c) cx_item<AR, S, NV1>(Pr, Lr, Pi, Li, x, y, nvec, nvdiv, blk, cp, c, cj);
      __syncthreads();
    }
  }
  const long long rest = (nblk - full) * nchunks;
  for (long long w = blockIdx.x; w < rest; w += gridDim.x) {
    const long long blk = full + w / nchunks;
    if (blk != cur) {
      cur = blk;
      eval_block<AR>(Pr, Lr, blk, nvec);
      eval_block<AR>(Pi, Li, blk, nvec);
    }
    cx_item<AR, S, NV1>(Pr, Lr, Pi, Li, x, y, nvec, nvdiv, blk, cp, (int)(w - (blk - full) * nchunks), cj);
    __syncthreads();
  }
}

template <int AR, int S, bool NV1, int MB>
static cudaError_t launch_cx_nv(const KPlan& kr, const KPlan& ki, const void* x, void* y, long long nvec,
                                int nchunks, cudaStream_t st, int ctas, KGate gate, bool conj) {
  using TX = typename Ar<AR>::TX;
  using TY = typename Ar<AR>::TY;
  auto kern = k_apply_cx<AR, S, NV1, MB>;
  const size_t smem = cx_lists_bytes<AR>(kr) + cx_lists_bytes<AR>(ki);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  static size_t attr_set = 0;
  if (smem > 48 * 1024 && smem > attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = smem;
  }
  long long grid = ctas;
  if (grid <= 0) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kNT, smem);
    grid = (long long)num_sms() * std::max(1, occ);
  }
  grid = std::max<long long>(1, std::min(grid, kr.nblk * nchunks));
  kern<<<(unsigned)grid, kNT, smem, st>>>(kr, ki, (const TX*)x, (TY*)y, (int)nvec, make_nvdiv(nvec), gate,
                                          conj ? 1 : 0);
  return cudaGetLastError();
}

template <int AR, int S, int MB>
static cudaError_t launch_cx_shape(const KPlan& kr, const KPlan& ki, const void* x, void* y, long long nvec,
                                   cudaStream_t st, int ctas, KGate gate, bool conj) {
  const int nc = chunk_plan((int)(kr.B * nvec), S).count();
  if (nvec == 1) return launch_cx_nv<AR, S, true, MB>(kr, ki, x, y, nvec, nc, st, ctas, gate, conj);
  return launch_cx_nv<AR, S, false, MB>(kr, ki, x, y, nvec, nc, st, ctas, gate, conj);
}

// kr, ki: the real and imaginary operators' tables (both of H, or both of
// H^T for the adjoint with conj); cudaErrorInvalidConfiguration when the two
// plans do not share their block structure or their lists exceed shared
// memory. Elements per thread: 2 for 16-byte elements, 2 or 3 for 8-byte
// ones (more spill at the two-CTA register limit: each element carries two
// accumulators); the register-capped variant (cap) takes 2.
template <int AR>
cudaError_t launch_apply_cx_t(const KPlan& kr, const KPlan& ki, const void* x, void* y, long long nvec,
                              cudaStream_t st, int ctas, KGate gate, bool conj, bool cap) {
  if (!cx_compatible(kr, ki)) return cudaErrorInvalidConfiguration;
  if (cap) return launch_cx_shape<AR, 2, 3>(kr, ki, x, y, nvec, st, ctas, gate, conj);
  if constexpr (sizeof(typename Ar<AR>::TX) < 16) {
    if (pick_shape((long long)kr.B * nvec, 3).s == 3)
      return launch_cx_shape<AR, 3, 2>(kr, ki, x, y, nvec, st, ctas, gate, conj);
  }
  return launch_cx_shape<AR, 2, 2>(kr, ki, x, y, nvec, st, ctas, gate, conj);
}

}  // namespace hm
