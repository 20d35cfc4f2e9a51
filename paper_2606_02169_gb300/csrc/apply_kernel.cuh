// y = H x, target-driven (pull) form (Sec. II): every output element y_F is
// produced by exactly one thread from gathered inputs x_{F+offset}; x is
// read-only, so there is no synchronisation on y and no atomics.
//
// Index space: the trailing sites form a low block of B <= 4096 states whose
// digits are tabulated once per plan (packed words, no division per state);
// the leading ("high") sites are uniform across a block. A CTA owns whole low
// blocks. Per block, its threads evaluate in parallel, into shared memory:
//   * the high digits (Eq. decode on the block index);
//   * every channel on high digits only (Sec. IV.B steps 2-4: admissibility
//     and coefficient are uniform over the block);
//   * the high factor u of every factorised high/low channel.
// Per element the thread then does one load and one FMA per active uniform
// hop, a low-digit lookup per factorised group, and reads the channels inside
// the low block (the same small operator for every block) from an ELL table.
// Thread t owns elements t, t+NT, ..., t+(S-1)NT of each chunk, so each hop
// is S independent coalesced loads with immediate offsets.
#pragma once

#include "device_common.cuh"

namespace hm {

template <int AR>
struct Lists {  // per-block uniform values (shared memory)
  using C = typename Ar<AR>::C;
  using Dsum = typename Ar<AR>::Dsum;
  int* hd;              // [64] high digits
  C* hh_c;              // [n_hh_diag + n_hh] coefficient of each high channel
  long long* hh_src;    // [n_hh_diag + n_hh] element index of its source block
  C* mem_u;             // [n_mem]
  int* grp_v;           // [n_grp_diag + n_grp] v row base
  Dsum* grp_U;          // [n_grp_diag] sum of member u (diagonal groups)
  Dsum* du;             // [1] sum of high diagonal channels
};

template <int AR>
__host__ __device__ inline size_t lists_bytes(int n_hh, int n_mem, int n_grp, int n_grpd) {
  using C = typename Ar<AR>::C;
  using Dsum = typename Ar<AR>::Dsum;
  auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
  return al(64 * 4) + al(n_hh * sizeof(C)) + al(n_hh * 8) + al(n_mem * sizeof(C)) + al(n_grp * 4) +
         al(n_grpd * sizeof(Dsum)) + al(sizeof(Dsum));
}

template <int AR>
__device__ inline Lists<AR> carve(unsigned char* sm, int n_hh, int n_mem, int n_grp, int n_grpd) {
  using C = typename Ar<AR>::C;
  using Dsum = typename Ar<AR>::Dsum;
  auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
  Lists<AR> L;
  size_t o = 0;
  L.hd = (int*)(sm + o);
  o += al(64 * 4);
  L.hh_c = (C*)(sm + o);
  o += al(n_hh * sizeof(C));
  L.hh_src = (long long*)(sm + o);
  o += al(n_hh * 8);
  L.mem_u = (C*)(sm + o);
  o += al(n_mem * sizeof(C));
  L.grp_v = (int*)(sm + o);
  o += al(n_grp * 4);
  L.grp_U = (Dsum*)(sm + o);
  o += al(n_grpd * sizeof(Dsum));
  L.du = (Dsum*)(sm + o);
  return L;
}

// Evaluate the uniform values of low block `blk`. Must be called by all
// threads of the CTA; ends with a barrier.
template <int AR>
__device__ __forceinline__ void eval_block(const KPlan& P, const Lists<AR>& L, long long blk, long long nvec) {
  using A = Ar<AR>;
  using C = typename A::C;
  using Dsum = typename A::Dsum;
  const C* __restrict__ tab = A::tab(P);
  const int nt = blockDim.x;
  for (int t = threadIdx.x; t < P.nhigh; t += nt) L.hd[t] = (int)((blk / P.sites[t].mh) % P.sites[t].d);
  __syncthreads();
  const int nhh = P.n_hh_diag + P.n_hh;
  for (int c = threadIdx.x; c < nhh; c += nt) {
    const KChan ch = P.ch[c];
    const int ni = L.hd[ch.si];
    const int nj = (ch.kind & CK_SINGLE) ? 0 : L.hd[ch.sj];
    L.hh_c[c] = tab[ch.tab + ni * ch.dj + nj];
    L.hh_src[c] = (blk * P.B + ch.off) * nvec;
  }
  for (int m = threadIdx.x; m < P.n_mem; m += nt) {
    const KMember mb = P.mem[m];
    L.mem_u[m] = tab[mb.utab + L.hd[mb.usite]];
  }
  const int ng = P.n_grp_diag + P.n_grp;
  for (int g = threadIdx.x; g < ng; g += nt) {
    const KGroup gr = P.grp[g];
    L.grp_v[g] = gr.vtab + (gr.vstride ? L.hd[gr.vsite] * gr.vstride : 0);
  }
  __syncthreads();
  // fixed-order sums (deterministic)
  if (threadIdx.x == 0) {
    Dsum d = A::dzero();
    for (int c = 0; c < P.n_hh_diag; ++c) A::dadd(d, L.hh_c[c]);
    L.du[0] = d;
  }
  for (int g = threadIdx.x; g < P.n_grp_diag; g += nt) {
    const KGroup gr = P.grp[g];
    Dsum d = A::dzero();
    for (int m = gr.m0; m < gr.m1; ++m) A::dadd(d, L.mem_u[m]);
    L.grp_U[g] = d;
  }
  __syncthreads();
}

// element -> state index within the block (nvec > 1 interleaves values)
struct NvDiv {
  unsigned magic;  // 0: power of two, use shift only
  int shift;
  __device__ __forceinline__ int operator()(int e) const {
    return magic ? (int)(__umulhi((unsigned)e, magic) >> shift) : (e >> shift);
  }
};

// One chunk of NT*S elements of low block blk (uniforms already in L).
template <int AR, int NT, int S>
__device__ __forceinline__ void apply_chunk(const KPlan& P, const Lists<AR>& L,
                                            const typename Ar<AR>::T* __restrict__ x,
                                            typename Ar<AR>::T* __restrict__ y, long long nvec,
                                            NvDiv nvdiv, long long blk, int chunk) {
  using A = Ar<AR>;
  using T = typename A::T;
  using C = typename A::C;
  using Acc = typename A::Acc;
  using Dsum = typename A::Dsum;
  const C* __restrict__ tab = A::tab(P);
  const int belems = (int)(P.B * nvec);
  const long long ebase = blk * (long long)belems;
  const int e0 = chunk * (NT * S) + (int)threadIdx.x;
  const T* __restrict__ xb = x + ebase + e0;  // own element s at xb[s*NT]

  bool ok[S];
  int lo[S];
  uint32_t pk[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int e = e0 + s * NT;
    ok[s] = e < belems;
    lo[s] = ok[s] ? nvdiv(e) : 0;
    pk[s] = __ldg(P.ptab + lo[s]);
  }

  Acc acc[S];
  // ---- diagonal (Sec. IV.A diag rule, Sec. IV.B zz collapse, App. B/C) ----
  {
    const C* __restrict__ dtab = A::diag(P);
    Dsum ds[S];
    const Dsum du = L.du[0];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      ds[s] = du;
      A::dadd(ds[s], dtab[lo[s]]);
    }
    for (int g = 0; g < P.n_grp_diag; ++g) {
      const KGroup gr = P.grp[g];
      const Dsum U = L.grp_U[g];
      const int vb = L.grp_v[g];
#pragma unroll
      for (int s = 0; s < S; ++s) A::dmadd(ds[s], tab[vb + low_digit(pk[s], gr.lbit, gr.lwid)], U);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const T xv = ok[s] ? xb[s * NT] : T(0);
      acc[s] = A::dmul(ds[s], A::prep(xv));
    }
  }
  // ---- hops with block-uniform coefficients (high digits only) ----
  const int nhh = P.n_hh_diag + P.n_hh;
  for (int c = P.n_hh_diag; c < nhh; ++c) {
    const C cf = L.hh_c[c];
    if (!A::nz(cf)) continue;  // a source digit leaves its range (Sec. IV.B step 3)
    const T* __restrict__ src = x + L.hh_src[c] + e0;
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (ok[s]) A::fma(acc[s], cf, A::prep(__ldg(src + s * NT)));
  }
  // ---- factorised high/low hops, grouped by their low factor ----
  for (int g = P.n_grp_diag; g < P.n_grp_diag + P.n_grp; ++g) {
    const KGroup gr = P.grp[g];
    const int vb = L.grp_v[g];
    C v[S];
    bool pr[S];
    Acc ag[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      v[s] = tab[vb + low_digit(pk[s], gr.lbit, gr.lwid)];
      pr[s] = ok[s] && A::nz(v[s]);
      ag[s] = A::azero();
    }
    for (int m = gr.m0; m < gr.m1; ++m) {
      const C u = L.mem_u[m];
      if (!A::nz(u)) continue;
      const T* __restrict__ src = xb + P.mem[m].off * nvec;
#pragma unroll
      for (int s = 0; s < S; ++s)
        if (pr[s]) A::fma(ag[s], u, A::prep(__ldg(src + s * NT)));
    }
#pragma unroll
    for (int s = 0; s < S; ++s) A::acc_mul(acc[s], v[s], ag[s]);
  }
  // ---- hops inside the low block (ELL over the low index) ----
  {
    const C* __restrict__ etab = A::ell(P);
    for (int w = 0; w < P.ell_w; ++w) {
      const long long rb = (long long)w * P.B;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const C cf = etab[rb + lo[s]];
        const int dl = __ldg(P.ell_delta + rb + lo[s]);
        if (ok[s] && A::nz(cf)) A::fma(acc[s], cf, A::prep(__ldg(xb + s * NT + (long long)dl * nvec)));
      }
    }
  }
  // ---- store: one write per output element ----
  T* __restrict__ yb = y + ebase + e0;
#pragma unroll
  for (int s = 0; s < S; ++s)
    if (ok[s]) yb[s * NT] = A::out(acc[s]);
}

template <int AR, int NT, int S>
__global__ void __launch_bounds__(NT)
k_apply(const KPlan P, const typename Ar<AR>::T* __restrict__ x, typename Ar<AR>::T* __restrict__ y,
        long long nvec, NvDiv nvdiv, int nchunks) {
  extern __shared__ __align__(16) unsigned char sm[];
  const Lists<AR> L = carve<AR>(sm, P.n_hh_diag + P.n_hh, P.n_mem, P.n_grp_diag + P.n_grp, P.n_grp_diag);
  const long long nitems = P.nblk * nchunks;
  long long cur = -1;
  // blocks outer when there are enough of them, else (block, chunk) items
  const bool by_block = P.nblk >= 2LL * gridDim.x;
  if (by_block) {
    for (long long blk = blockIdx.x; blk < P.nblk; blk += gridDim.x) {
      eval_block<AR>(P, L, blk, nvec);
      for (int c = 0; c < nchunks; ++c) apply_chunk<AR, NT, S>(P, L, x, y, nvec, nvdiv, blk, c);
      __syncthreads();
    }
  } else {
    for (long long w = blockIdx.x; w < nitems; w += gridDim.x) {
      const long long blk = w / nchunks;
      if (blk != cur) {
        cur = blk;
        eval_block<AR>(P, L, blk, nvec);
      }
      apply_chunk<AR, NT, S>(P, L, x, y, nvec, nvdiv, blk, (int)(w - blk * nchunks));
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Batched apply: many plans of uneven size in one persistent launch. Work
// items (instance, low block) are numbered by a prefix sum over instances;
// CTAs stride over that single index space, so instances of 6561 and of 4.8M
// states are cut into the same unit of work.
// ---------------------------------------------------------------------------
constexpr int kBatchMax = 256;
struct BatchArgs {
  int n, pad;
  long long blk_start[kBatchMax + 1];
  const void* x[kBatchMax];
  void* y[kBatchMax];
};

template <int AR, int NT, int S>
__global__ void __launch_bounds__(NT)
k_batch(const KPlan* __restrict__ plans, const BatchArgs A, long long nvec, NvDiv nvdiv, size_t lists_off) {
  extern __shared__ __align__(16) unsigned char sm[];
  KPlan& P = *reinterpret_cast<KPlan*>(sm);
  using T = typename Ar<AR>::T;
  const long long total = A.blk_start[A.n];
  int inst = -1;
  Lists<AR> L{};
  for (long long w = blockIdx.x; w < total; w += gridDim.x) {
    int ni = inst < 0 ? 0 : inst;
    while (A.blk_start[ni + 1] <= w) ++ni;
    if (ni != inst) {
      __syncthreads();
      if (threadIdx.x == 0) P = plans[ni];
      __syncthreads();
      inst = ni;
      L = carve<AR>(sm + lists_off, P.n_hh_diag + P.n_hh, P.n_mem, P.n_grp_diag + P.n_grp, P.n_grp_diag);
    }
    const long long blk = w - A.blk_start[inst];
    eval_block<AR>(P, L, blk, nvec);
    const int nchunks = (int)((P.B * nvec + NT * S - 1) / (NT * S));
    for (int c = 0; c < nchunks; ++c)
      apply_chunk<AR, NT, S>(P, L, (const T*)A.x[inst], (T*)A.y[inst], nvec, nvdiv, blk, c);
    __syncthreads();
  }
}

}  // namespace hm
