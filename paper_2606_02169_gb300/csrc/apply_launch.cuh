// Host-side launch logic for the apply kernels (templated on the arithmetic
// policy; instantiated once per policy in apply_<policy>.cu).
#pragma once

#include <algorithm>
#include <vector>

#include "apply_kernel.cuh"

namespace hm {

struct Shape {
  int nt, s, nchunks;
};

// Threads per CTA and elements per thread for a block of `belems` elements:
// the least padding (ragged last chunk), preferring more elements per thread
// (memory-level parallelism) and at least 256 threads.
inline Shape pick_shape(long long belems) {
  Shape best{256, 1, 1};
  double bs = 1e30;
  for (int nt : {512, 256, 128})
    for (int s : {8, 4, 2, 1}) {
      const long long chunk = (long long)nt * s;
      const long long nch = (belems + chunk - 1) / chunk;
      const double waste = (double)(nch * chunk) / (double)belems - 1.0;
      const double score = waste + (s == 1 ? 0.05 : s == 2 ? 0.02 : 0.0) + (nt == 128 ? 0.02 : 0.0);
      if (score < bs - 1e-12) {
        bs = score;
        best = {nt, s, (int)nch};
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

template <int AR, int NT, int S>
static cudaError_t launch_shape(const KPlan& k, const void* x, void* y, long long nvec, int nchunks,
                                cudaStream_t st, int ctas) {
  using T = typename Ar<AR>::T;
  const size_t smem = lists_bytes<AR>(k.n_hh_diag + k.n_hh, k.n_mem, k.n_grp_diag + k.n_grp, k.n_grp_diag);
  static size_t attr_set = 0;
  if (smem > 48 * 1024 && smem > attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_apply<AR, NT, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = smem;
  }
  long long grid = ctas;
  if (grid <= 0) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_apply<AR, NT, S>, NT, smem);
    grid = (long long)num_sms() * std::max(1, occ);
  }
  const long long items = k.nblk * nchunks;
  grid = std::max<long long>(1, std::min(grid, items));
  k_apply<AR, NT, S><<<(unsigned)grid, NT, smem, st>>>(k, (const T*)x, (T*)y, nvec, make_nvdiv(nvec), nchunks);
  return cudaGetLastError();
}

template <int AR>
cudaError_t launch_apply_t(const KPlan& k, const void* x, void* y, long long nvec, cudaStream_t st, int ctas) {
  const Shape sh = pick_shape((long long)k.B * nvec);
#define HM_CASE(NT_, S_) \
  if (sh.nt == NT_ && sh.s == S_) return launch_shape<AR, NT_, S_>(k, x, y, nvec, sh.nchunks, st, ctas);
  HM_CASE(512, 8) HM_CASE(512, 4) HM_CASE(512, 2) HM_CASE(512, 1)
  HM_CASE(256, 8) HM_CASE(256, 4) HM_CASE(256, 2) HM_CASE(256, 1)
  HM_CASE(128, 8) HM_CASE(128, 4) HM_CASE(128, 2) HM_CASE(128, 1)
#undef HM_CASE
  return cudaErrorInvalidConfiguration;
}

template <int AR, int NT, int S>
static cudaError_t batch_shape(const KPlan* dplans, const std::vector<const Plan*>& members,
                               const void* const* xs, void* const* ys, long long nvec, cudaStream_t st) {
  size_t lists = 0;
  for (const Plan* p : members) {
    const KPlan& k = p->k;
    lists = std::max(lists, lists_bytes<AR>(k.n_hh_diag + k.n_hh, k.n_mem, k.n_grp_diag + k.n_grp, k.n_grp_diag));
  }
  const size_t off = (sizeof(KPlan) + 15) & ~size_t(15);
  const size_t smem = off + lists;
  static size_t attr_set = 0;
  if (smem > 48 * 1024 && smem > attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_batch<AR, NT, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = smem;
  }
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<AR, NT, S>, NT, smem);
  const int n = (int)members.size();
  for (int c0 = 0; c0 < n; c0 += kBatchMax) {
    BatchArgs A{};
    A.n = std::min(kBatchMax, n - c0);
    A.blk_start[0] = 0;
    for (int i = 0; i < A.n; ++i) {
      A.blk_start[i + 1] = A.blk_start[i] + members[c0 + i]->nblk;
      A.x[i] = xs[c0 + i];
      A.y[i] = ys[c0 + i];
    }
    long long grid = (long long)num_sms() * std::max(1, occ);
    grid = std::max<long long>(1, std::min(grid, A.blk_start[A.n]));
    k_batch<AR, NT, S><<<(unsigned)grid, NT, smem, st>>>(dplans + c0, A, nvec, make_nvdiv(nvec), off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One (NT, S) for the whole batch, chosen on the median block size.
template <int AR>
cudaError_t launch_batch_t(const KPlan* dplans, const std::vector<const Plan*>& members, const void* const* xs,
                           void* const* ys, long long nvec, cudaStream_t st) {
  std::vector<long long> be;
  for (const Plan* p : members) be.push_back((long long)p->B * nvec);
  std::nth_element(be.begin(), be.begin() + be.size() / 2, be.end());
  const Shape sh = pick_shape(be[be.size() / 2]);
#define HM_CASE(NT_, S_) \
  if (sh.nt == NT_ && sh.s == S_) return batch_shape<AR, NT_, S_>(dplans, members, xs, ys, nvec, st);
  HM_CASE(512, 8) HM_CASE(512, 4) HM_CASE(512, 2) HM_CASE(512, 1)
  HM_CASE(256, 8) HM_CASE(256, 4) HM_CASE(256, 2) HM_CASE(256, 1)
  HM_CASE(128, 8) HM_CASE(128, 4) HM_CASE(128, 2) HM_CASE(128, 1)
#undef HM_CASE
  return cudaErrorInvalidConfiguration;
}

}  // namespace hm
