// Host launch of the staged apply kernel (stream_kernel.cuh), instantiated
// once per arithmetic policy by the translation unit that includes it
// (stream_f32.cu, stream_df64.cu, stream_f64.cu), and the status word its
// bounded waits report to.
#pragma once

#include <algorithm>

#include "apply_launch.cuh"
#include "stream_kernel.cuh"

namespace hm {

// Consumer warps per CTA: 8 for double-float and native FP64 arithmetic,
// 4 for FP32 (the faster of 4 and 8 on the chain and spin-boson workloads).
template <int AR>
constexpr int stream_nc() {
  return AR == AR_F32 ? 4 : 8;
}

template <int AR, int S, bool NV1>
static cudaError_t stream_nv(const KPlan& k, const void* x, void* y, long long nvec, cudaStream_t st, int ctas,
                             KGate gate) {
  using TX = typename Ar<AR>::TX;
  using TY = typename Ar<AR>::TY;
  constexpr int NC = stream_nc<AR>();
  auto kern = k_stream<AR, S, NC, NV1>;
  const size_t smem = stream_layout<AR>(k).total;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  static size_t attr_set = 0;
  if (smem > 48 * 1024 && smem > attr_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = smem;
  }
  const int nt = 32 * (NC + 2);
  long long grid = ctas;
  if (grid <= 0) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nt, smem);
    grid = (long long)num_sms() * std::max(1, occ);
  }
  grid = std::max<long long>(1, std::min(grid, k.nblk));
  kern<<<(unsigned)grid, nt, smem, st>>>(k, (const TX*)x, (TY*)y, (int)nvec, make_nvdiv(nvec), gate);
  return cudaGetLastError();
}

template <int AR>
cudaError_t launch_stream_t(const KPlan& k, const void* x, void* y, long long nvec, cudaStream_t st, TuneCfg cfg) {
  const long long E = (long long)k.B * nvec;
  if (E > kStreamElems) return cudaErrorInvalidConfiguration;
  constexpr int NC = stream_nc<AR>();
  const long long per = (E + 32 * NC - 1) / (32 * NC);  // elements per consumer thread
  const bool nv1 = nvec == 1;
  const KGate g{cfg.gate, cfg.gate_run};
  if (per <= 1) return nv1 ? stream_nv<AR, 1, true>(k, x, y, nvec, st, cfg.ctas, g)
                           : stream_nv<AR, 1, false>(k, x, y, nvec, st, cfg.ctas, g);
  if (per <= 2) return nv1 ? stream_nv<AR, 2, true>(k, x, y, nvec, st, cfg.ctas, g)
                           : stream_nv<AR, 2, false>(k, x, y, nvec, st, cfg.ctas, g);
  if (per <= 4) return nv1 ? stream_nv<AR, 4, true>(k, x, y, nvec, st, cfg.ctas, g)
                           : stream_nv<AR, 4, false>(k, x, y, nvec, st, cfg.ctas, g);
  return nv1 ? stream_nv<AR, 8, true>(k, x, y, nvec, st, cfg.ctas, g)
             : stream_nv<AR, 8, false>(k, x, y, nvec, st, cfg.ctas, g);
}

// Read (and optionally clear) this translation unit's status word on the
// current device.
static int stream_status(int* out, bool clear) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_hm_status, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "device status read");
  if (clear && v) {
    const int z = 0;
    e = cudaMemcpyToSymbol(g_hm_status, &z, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "device status clear");
  }
  *out = v;
  return HM_OK;
}

}  // namespace hm
