// Host-side launch logic for the apply kernels (templated on the arithmetic
// policy; instantiated once per policy in apply_<policy>.cu).
#pragma once

#include <algorithm>
#include <vector>

#include "apply_kernel.cuh"

namespace hm {

struct Shape {
  int s, nchunks;
};

// Elements per thread of the main chunks of a block of `belems` elements:
// the most work in full S-chunks (more loads in flight per thread), the
// remainder in single-element chunks (see chunk_plan).
inline Shape pick_shape(long long belems, int smax = 8) {
  Shape best{2, chunk_plan((int)belems, 2).count()};
  double bs = 0.0;
  for (int s : {8, 6, 4, 3, 2}) {
    if (s > smax) continue;
    const ChunkPlan cp = chunk_plan((int)belems, s);
    const double frac = (double)cp.nS * kNT * s / (double)belems;   // share in S-chunks
    const double score = frac * (1.0 + 0.02 * s);
    if (score > bs + 1e-12) {
      bs = score;
      best = {s, cp.count()};
    }
  }
  return best;
}

inline NvDiv make_nvdiv(long long nvec) {
  NvDiv d{0u, 0};
  if ((nvec & (nvec - 1)) == 0) {
    while ((1LL << d.shift) < nvec) ++d.shift;
    return d;
  }
  // round-up magic for dividends below 2^31: s = floor(log2 n),
  // m = ceil(2^(32+s) / n) < 2^32 (n not a power of two), e/n = umulhi(e, m) >> s
  int l = 0;
  while ((2LL << l) <= nvec) ++l;
  d.magic = (unsigned)(((1ULL << (32 + l)) + (unsigned long long)nvec - 1) / (unsigned long long)nvec);
  d.shift = l;
  return d;
}

int num_sms();

template <int AR, int S, bool NV1, int MBV, int PF, bool VI>
static cudaError_t launch_nv(const KPlan& k, const void* x, void* y, long long nvec, int nchunks, cudaStream_t st,
                             int ctas, KGate gate) {
  using TX = typename Ar<AR>::TX;
  using TY = typename Ar<AR>::TY;
  auto kern = k_apply<AR, S, NV1, MBV, PF, VI>;
  size_t smem = lists_bytes<AR>(k.n_hh_diag + k.n_hh, k.n_mem, k.n_grp_diag + k.n_grp, k.n_grp_diag);
  if (PF > 0) smem = ((smem + 15) & ~size_t(15)) + pf_bytes<AR, S, PF>();
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
  const long long items = k.nblk * nchunks;
  grid = std::max<long long>(1, std::min(grid, items));
  kern<<<(unsigned)grid, kNT, smem, st>>>(k, (const TX*)x, (TY*)y, (int)nvec, make_nvdiv(nvec), gate);
  return cudaGetLastError();
}

// 16-byte elements (4 FP32 or 2 double-float right-hand sides per lane):
// at most 4 of them per thread (more would spill their accumulators).
template <int AR>
constexpr bool wide_elem() {
  return sizeof(typename Ar<AR>::TX) == 16;
}

template <int AR, int S, int PF, bool VI>
static cudaError_t launch_shape(const KPlan& k, const void* x, void* y, long long nvec, int nchunks,
                                cudaStream_t st, TuneCfg cfg) {
  const KGate g{cfg.gate, cfg.gate_run};
  if constexpr (AR != AR_F64) {
    if (cfg.mb) {
      if (nvec == 1) return launch_nv<AR, S, true, 1, PF, VI>(k, x, y, nvec, nchunks, st, cfg.ctas, g);
      return launch_nv<AR, S, false, 1, PF, VI>(k, x, y, nvec, nchunks, st, cfg.ctas, g);
    }
  }
  if (nvec == 1) return launch_nv<AR, S, true, 0, PF, VI>(k, x, y, nvec, nchunks, st, cfg.ctas, g);
  return launch_nv<AR, S, false, 0, PF, VI>(k, x, y, nvec, nchunks, st, cfg.ctas, g);
}


// Elements-per-thread values the kernels are instantiated for.
constexpr int kShapes[] = {2, 3, 4, 6, 8};

template <int AR, bool VI>
cudaError_t launch_apply_t(const KPlan& k, const void* x, void* y, long long nvec, cudaStream_t st, TuneCfg cfg) {
  Shape sh = pick_shape((long long)k.B * nvec);
  if (cfg.s) sh = {cfg.s, chunk_plan((int)(k.B * nvec), cfg.s).count()};
  if constexpr (wide_elem<AR>()) {
    if (!cfg.s) sh = pick_shape((long long)k.B * nvec, 4);
    const int s = std::min(sh.s, 4);
    const int nc = chunk_plan((int)(k.B * nvec), s).count();
    switch (s) {
      case 4: return launch_shape<AR, 4, 0, VI>(k, x, y, nvec, nc, st, cfg);
      case 3: return launch_shape<AR, 3, 0, VI>(k, x, y, nvec, nc, st, cfg);
      default: return launch_shape<AR, 2, 0, VI>(k, x, y, nvec, nc, st, cfg);
    }
  } else {
    switch (sh.s) {
      case 8: return launch_shape<AR, 8, 0, VI>(k, x, y, nvec, sh.nchunks, st, cfg);
      case 6: return launch_shape<AR, 6, 0, VI>(k, x, y, nvec, sh.nchunks, st, cfg);
      case 4: return launch_shape<AR, 4, 0, VI>(k, x, y, nvec, sh.nchunks, st, cfg);
      case 3: return launch_shape<AR, 3, 0, VI>(k, x, y, nvec, sh.nchunks, st, cfg);
      default: return launch_shape<AR, 2, 0, VI>(k, x, y, nvec, sh.nchunks, st, cfg);
    }
  }
}

// The prefetching variant (PF = 4 stages), for 4, 6 or 8 elements per
// thread (default: the shape pick_shape chooses, rounded to those).
template <int AR, bool VI>
cudaError_t launch_apply_pf_t(const KPlan& k, const void* x, void* y, long long nvec, cudaStream_t st, TuneCfg cfg) {
  Shape sh = pick_shape((long long)k.B * nvec);
  int s = cfg.s ? cfg.s : sh.s;
  s = s >= 8 ? 8 : (s >= 6 ? 6 : 4);
  const int nchunks = chunk_plan((int)(k.B * nvec), s).count();
  switch (s) {
    case 8: return launch_shape<AR, 8, 4, VI>(k, x, y, nvec, nchunks, st, cfg);
    case 6: return launch_shape<AR, 6, 4, VI>(k, x, y, nvec, nchunks, st, cfg);
    default: return launch_shape<AR, 4, 4, VI>(k, x, y, nvec, nchunks, st, cfg);
  }
}

template <int AR, int S, bool NV1>
static cudaError_t batch_nv(const std::vector<const Plan*>& members, const void* const* xs, void* const* ys,
                            long long nvec, cudaStream_t st) {
  size_t smem = 0;
  for (const Plan* p : members) {
    const KPlan& k = p->k;
    smem = std::max(smem, lists_bytes<AR>(k.n_hh_diag + k.n_hh, k.n_mem, k.n_grp_diag + k.n_grp, k.n_grp_diag));
  }
  static size_t attr_set = 0;
  if (smem > 48 * 1024 && smem > attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_batch<AR, S, NV1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = smem;
  }
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<AR, S, NV1>, kNT, smem);
  const int n = (int)members.size();
  const long long grid0 = (long long)num_sms() * std::max(1, occ);
  for (int c0 = 0; c0 < n; c0 += kBatchMax) {
    BatchArgs A{};
    A.n = std::min(kBatchMax, n - c0);
    // whole blocks per item when there are many and the blocks in flight fit
    // in L2 with room to spare (as in k_apply), else (block, chunk) items
    long long blocks = 0, bmax = 0;
    for (int i = 0; i < A.n; ++i) {
      blocks += members[c0 + i]->nblk;
      bmax = std::max<long long>(bmax, members[c0 + i]->B);
    }
    A.by_block = blocks >= 2 * grid0 && bmax * nvec * (long long)sizeof(typename Ar<AR>::TX) * grid0 <= kInflightMax;
    A.start[0] = 0;
    for (int i = 0; i < A.n; ++i) {
      const Plan* m = members[c0 + i];
      const long long items = A.by_block ? m->nblk : m->nblk * chunk_plan((int)(m->B * nvec), S).count();
      A.start[i + 1] = A.start[i] + items;
      A.x[i] = xs[c0 + i];
      A.y[i] = ys[c0 + i];
      A.plans[i] = m->k;
    }
    const long long grid = std::max<long long>(1, std::min(grid0, A.start[A.n]));
    k_batch<AR, S, NV1><<<(unsigned)grid, kNT, smem, st>>>(A, (int)nvec, make_nvdiv(nvec));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <int AR, int S>
static cudaError_t batch_shape(const std::vector<const Plan*>& members, const void* const* xs, void* const* ys,
                               long long nvec, cudaStream_t st) {
  if (nvec == 1) return batch_nv<AR, S, true>(members, xs, ys, nvec, st);
  return batch_nv<AR, S, false>(members, xs, ys, nvec, st);
}

// One elements-per-thread count for the whole batch, chosen on the median block size.
template <int AR>
cudaError_t launch_batch_t(const std::vector<const Plan*>& members, const void* const* xs, void* const* ys,
                           long long nvec, cudaStream_t st) {
  std::vector<long long> be;
  for (const Plan* p : members) be.push_back((long long)p->B * nvec);
  std::nth_element(be.begin(), be.begin() + be.size() / 2, be.end());
  const Shape sh = pick_shape(be[be.size() / 2], wide_elem<AR>() ? 4 : 8);
  if constexpr (wide_elem<AR>()) {
    switch (sh.s) {
      case 4: return batch_shape<AR, 4>(members, xs, ys, nvec, st);
      case 3: return batch_shape<AR, 3>(members, xs, ys, nvec, st);
      default: return batch_shape<AR, 2>(members, xs, ys, nvec, st);
    }
  } else {
    switch (sh.s) {
      case 8: return batch_shape<AR, 8>(members, xs, ys, nvec, st);
      case 6: return batch_shape<AR, 6>(members, xs, ys, nvec, st);
      case 4: return batch_shape<AR, 4>(members, xs, ys, nvec, st);
      case 3: return batch_shape<AR, 3>(members, xs, ys, nvec, st);
      default: return batch_shape<AR, 2>(members, xs, ys, nvec, st);
    }
  }
}

}  // namespace hm
