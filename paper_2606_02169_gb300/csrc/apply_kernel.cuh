// y = H x, target-driven (pull) form (Sec. II): every output element y_F is
// produced by exactly one thread from gathered inputs x_{F+offset}; x is
// read-only, so there is no synchronisation on y and no atomics.
//
// Index space: the trailing sites form a low block of B <= 8192 states whose
// digits are tabulated once per plan (packed words, no division per state);
// the leading ("high") sites are uniform across a block. A CTA owns whole low
// blocks. Per block, its threads evaluate in parallel, into shared memory:
//   * the high digits (Eq. decode on the block index);
//   * every channel on high digits only (Sec. IV.B steps 2-4: admissibility
//     and coefficient are uniform over the block);
//   * the high factor u of every factorised high/low channel, and whether
//     the member's source range of this block lies inside the vector.
// Per element the thread then does one load and one FMA per active uniform
// hop, a low-digit lookup per factorised group, and one packed ELL entry per
// hop inside the low block (the same small operator for every block).
// Thread t owns elements t, t+NT, ..., t+(S-1)NT of a chunk, so each hop is S
// independent coalesced loads with immediate offsets.
#pragma once

#include "device_common.cuh"

namespace hm {

constexpr int kNT = 256;  // threads per CTA of the apply kernels

// y is written once and not read again by the kernel: streaming stores
// (evict-first), so that L2 keeps x for the hops of neighbouring blocks.
template <class T>
__device__ __forceinline__ void st_y(T* p, T v) {
  __stcs(p, v);
}

// Per-thread asynchronous copies (cp.async) of one element from global to
// shared memory, for the prefetching variant of the general kernel: each
// thread copies, and later reads, only its own slots, so completion is
// tracked per thread (commit / wait_group) with no barrier between threads.
template <class TX>
__device__ __forceinline__ void cp_async_elem(TX* dst, const TX* src) {
  static_assert(sizeof(TX) == 4 || sizeof(TX) == 8 || sizeof(TX) == 16, "element size");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(TX) == 16)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
  else if constexpr (sizeof(TX) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// acc[s] += sum_{j < n} c[j] * src_j[s * kNT] with src_j = base + off[j],
// the gathers issued PF items ahead through PF per-thread shared-memory
// stages (slot (stage, s) of this thread at pf[(stage * S + s) * kNT]).
// mask[s] = false skips element s (its copy and its FMA).
// SCALE: the coefficients are vs * c[j] (formed per item, A::cmul).
template <int AR, int S, int PF, bool SCALE = false>
__device__ __forceinline__ void pf_sum(typename Ar<AR>::Acc (&acc)[S], const typename Ar<AR>::C* c,
                                       const long long* off, int n, const typename Ar<AR>::TX* base,
                                       const bool (&mask)[S], typename Ar<AR>::TX* pf,
                                       typename Ar<AR>::C vs = typename Ar<AR>::C{}) {
  using A = Ar<AR>;
  using TX = typename A::TX;
  static_assert((PF & (PF - 1)) == 0, "PF a power of two");
#pragma unroll
  for (int j = 0; j < PF; ++j) {
    if (j < n) {
      const TX* src = base + off[j];
#pragma unroll
      for (int s = 0; s < S; ++s)
        if (mask[s]) cp_async_elem(pf + (j * S + s) * kNT, src + s * kNT);
    }
    cp_async_commit();
  }
  for (int j = 0; j < n; ++j) {
    cp_async_wait<PF - 1>();
    const int st = j & (PF - 1);
    const typename A::C cj = SCALE ? A::cmul(vs, c[j]) : c[j];
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (mask[s]) A::fma(acc[s], cj, pf[(st * S + s) * kNT]);
    if (j + PF < n) {
      const TX* src = base + off[j + PF];
#pragma unroll
      for (int s = 0; s < S; ++s)
        if (mask[s]) cp_async_elem(pf + (st * S + s) * kNT, src + s * kNT);
    }
    cp_async_commit();
  }
}
// bytes of x the CTAs may hold in whole-block work at once (L2 is 129 MB)
constexpr long long kInflightMax = 48LL << 20;

template <int AR>
struct Lists {  // per-block uniform values (shared memory)
  using C = typename Ar<AR>::C;
  using Dsum = typename Ar<AR>::Dsum;
  int* hd;              // [64] high digits
  C* hh_c;              // [n_hh_diag + n_hh] coefficient of each high channel
  long long* hh_src;    // [n_hh_diag + n_hh] element index of its source block
  int* n_act;           // [1] number of active off-diagonal high channels
  C* act_c;             // [n_hh] their coefficients, in channel order
  long long* act_src;   // [n_hh] their source-block element index
  C* mem_u;             // [n_mem] high factor u of each group member
  long long* mem_src;   // [n_mem] element offset of each member's source
  int* mem_ok;          // [n_mem] source range of this block inside the vector
  C* gact_u;            // [n_mem] active members of each group, compacted in place
  long long* gact_src;  //        within the group's member range [m0, m0 + gact_n)
  int* gact_n;          // [n_grp_diag + n_grp] number of active members
  int* gact_ok;         // [n_grp_diag + n_grp] every active source range inside the vector
  int* grp_v;           // [n_grp_diag + n_grp] v row base
  Dsum* grp_U;          // [n_grp_diag] sum of member u (diagonal groups)
  Dsum* du;             // [1] sum of high diagonal channels
  KChan* dch;           // plan descriptors, copied once per CTA
  KMember* dmem;
  KGroup* dgrp;
};

template <int AR>
__host__ __device__ inline size_t lists_bytes(int n_hh, int n_mem, int n_grp, int n_grpd) {
  using C = typename Ar<AR>::C;
  using Dsum = typename Ar<AR>::Dsum;
  auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
  return al(64 * 4) + 2 * al(n_hh * sizeof(C)) + 2 * al(n_hh * 8) + al(16) + 2 * al(n_mem * sizeof(C)) +
         2 * al(n_mem * 8) + al(n_mem * 4) + 3 * al(n_grp * 4) + al(n_grpd * sizeof(Dsum)) + al(sizeof(Dsum)) +
         al(n_hh * sizeof(KChan)) + al(n_mem * sizeof(KMember)) + al(n_grp * sizeof(KGroup));
}

// shared memory of one plan's lists in the complex kernel (16-byte aligned
// so that the second plan's lists follow)
template <int AR>
__host__ __device__ inline size_t cx_lists_bytes(const KPlan& k) {
  return (lists_bytes<AR>(k.n_hh_diag + k.n_hh, k.n_mem, k.n_grp_diag + k.n_grp, k.n_grp_diag) + 15) & ~size_t(15);
}

// two plans on the same sites (the real and imaginary parts of a complex H)
// share their low block, packed low digits and high/low split
inline bool cx_compatible(const KPlan& a, const KPlan& b) {
  return a.B == b.B && a.nblk == b.nblk && a.nhigh == b.nhigh && a.D == b.D;
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
  L.n_act = (int*)(sm + o);
  o += al(16);
  L.act_c = (C*)(sm + o);
  o += al(n_hh * sizeof(C));
  L.act_src = (long long*)(sm + o);
  o += al(n_hh * 8);
  L.mem_u = (C*)(sm + o);
  o += al(n_mem * sizeof(C));
  L.mem_src = (long long*)(sm + o);
  o += al(n_mem * 8);
  L.mem_ok = (int*)(sm + o);
  o += al(n_mem * 4);
  L.gact_u = (C*)(sm + o);
  o += al(n_mem * sizeof(C));
  L.gact_src = (long long*)(sm + o);
  o += al(n_mem * 8);
  L.gact_n = (int*)(sm + o);
  o += al(n_grp * 4);
  L.gact_ok = (int*)(sm + o);
  o += al(n_grp * 4);
  L.grp_v = (int*)(sm + o);
  o += al(n_grp * 4);
  L.grp_U = (Dsum*)(sm + o);
  o += al(n_grpd * sizeof(Dsum));
  L.du = (Dsum*)(sm + o);
  o += al(sizeof(Dsum));
  L.dch = (KChan*)(sm + o);
  o += al(n_hh * sizeof(KChan));
  L.dmem = (KMember*)(sm + o);
  o += al(n_mem * sizeof(KMember));
  L.dgrp = (KGroup*)(sm + o);
  return L;
}

// Copy the plan's channel, member and group descriptors into shared memory
// (once per CTA; ends with a barrier).
template <int AR>
__device__ __forceinline__ void load_descriptors(const KPlan& P, const Lists<AR>& L) {
  for (int c = threadIdx.x; c < P.n_hh_diag + P.n_hh; c += blockDim.x) L.dch[c] = P.ch[c];
  for (int m = threadIdx.x; m < P.n_mem; m += blockDim.x) L.dmem[m] = P.mem[m];
  for (int g = threadIdx.x; g < P.n_grp_diag + P.n_grp; g += blockDim.x) L.dgrp[g] = P.grp[g];
  __syncthreads();
}

// Warp-wide sums in a fixed order (deterministic).
__device__ __forceinline__ float wsum(float v) {
  for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ DF wsum(DF v) {
  for (int o = 16; o > 0; o >>= 1) {
    const float2 w = make_float2(__shfl_xor_sync(0xffffffffu, v.s, o), __shfl_xor_sync(0xffffffffu, v.c, o));
    df_add(v, w);
  }
  return v;
}

// Evaluate the uniform values of low block `blk` (descriptors already in
// shared memory). Called by all threads of the CTA (8 warps); ends with a
// barrier.
template <int AR>
__device__ __forceinline__ void eval_block(const KPlan& P, const Lists<AR>& L, long long blk, int nvec) {
  using A = Ar<AR>;
  using C = typename A::C;
  using Dsum = typename A::Dsum;
  const C* __restrict__ tab = A::tab(P);
  const int nt = blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = nt >> 5;
  for (int t = threadIdx.x; t < P.nhigh; t += nt) L.hd[t] = (int)((blk / P.sites[t].mh) % P.sites[t].d);
  __syncthreads();
  const int nhh = P.n_hh_diag + P.n_hh;
  for (int c = threadIdx.x; c < nhh; c += nt) {
    const KChan ch = L.dch[c];
    const int ni = L.hd[ch.si];
    const int nj = (ch.kind & CK_SINGLE) ? 0 : L.hd[ch.sj];
    L.hh_c[c] = tab[ch.tab + ni * ch.dj + nj];
    L.hh_src[c] = (blk * P.B + ch.off) * (long long)nvec;
  }
  const long long b0 = blk * P.B;
  for (int m = threadIdx.x; m < P.n_mem; m += nt) {
    const KMember mb = L.dmem[m];
    L.mem_u[m] = tab[mb.utab + L.hd[mb.usite]];
    L.mem_src[m] = mb.off * (long long)nvec;
    L.mem_ok[m] = (b0 + mb.off >= 0) && (b0 + mb.off + P.B <= P.D);
  }
  const int ng = P.n_grp_diag + P.n_grp;
  for (int g = threadIdx.x; g < ng; g += nt) {
    const KGroup gr = L.dgrp[g];
    L.grp_v[g] = gr.vtab + (gr.vstride ? L.hd[gr.vsite] * gr.vstride : 0);
  }
  __syncthreads();
  // warp-parallel reductions and order-preserving compactions
  if (warp == 0) {
    Dsum d = A::dzero();
    for (int c = lane; c < P.n_hh_diag; c += 32) A::dadd(d, L.hh_c[c]);
    d = wsum(d);
    if (lane == 0) L.du[0] = d;
  } else if (warp == 1) {
    int count = 0;
    for (int base = P.n_hh_diag; base < nhh; base += 32) {
      const int c = base + lane;
      const bool act = c < nhh && A::nz(L.hh_c[c]);
      const unsigned msk = __ballot_sync(0xffffffffu, act);
      if (act) {
        const int pos = count + __popc(msk & ((1u << lane) - 1u));
        L.act_c[pos] = L.hh_c[c];
        L.act_src[pos] = L.hh_src[c];
      }
      count += __popc(msk);
    }
    if (lane == 0) L.n_act[0] = count;
  } else {
    for (int g = warp - 2; g < ng; g += nwarp - 2) {
      const KGroup gr = L.dgrp[g];
      if (g < P.n_grp_diag) {
        Dsum d = A::dzero();
        for (int m = gr.m0 + lane; m < gr.m1; m += 32) A::dadd(d, L.mem_u[m]);
        d = wsum(d);
        if (lane == 0) L.grp_U[g] = d;
      } else {
        int count = 0, bad = 0;
        for (int base = gr.m0; base < gr.m1; base += 32) {
          const int m = base + lane;
          const bool act = m < gr.m1 && A::nz(L.mem_u[m]);
          const unsigned msk = __ballot_sync(0xffffffffu, act);
          bad |= __any_sync(0xffffffffu, act && !L.mem_ok[m]);
          if (act) {
            const int pos = gr.m0 + count + __popc(msk & ((1u << lane) - 1u));
            L.gact_u[pos] = L.mem_u[m];
            L.gact_src[pos] = L.mem_src[m];
          }
          count += __popc(msk);
        }
        if (lane == 0) {
          L.gact_n[g] = count;
          L.gact_ok[g] = !bad;
        }
      }
    }
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

// The thread's elements e0 + s NT of a chunk of low block blk: whether each
// lies inside the block, its state within the block and that state's packed
// low digits (the same for every plan on these sites).
template <int S, bool FULL, bool NV1>
__device__ __forceinline__ void chunk_states(const KPlan& P, int belems, int e0, NvDiv nvdiv, bool (&ok)[S],
                                             int (&lo)[S], uint32_t (&pk)[S]) {
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int e = e0 + s * kNT;
    ok[s] = FULL || e < belems;
    lo[s] = ok[s] ? (NV1 ? e : nvdiv(e)) : 0;
    pk[s] = __ldg(P.ptab + lo[s]);
  }
}

// acc[s] = (H x) of the thread's element s of a chunk (uniforms of the block
// already in L; xb = x + the element's index for s = 0). FULL: every element
// of the chunk lies inside the block, so no per-element bounds predicates
// are needed. NV1: nvec == 1. VINV: the low digit of every factorised group
// is the same for the thread's S elements (its period M_k d_k divides their
// stride), so each group has one v per thread and member coefficients v u
// are formed once.
template <int AR, int S, bool FULL, bool NV1, int PF = 0, bool VINV = false>
__device__ __forceinline__ void chunk_sum(const KPlan& P, const Lists<AR>& L,
                                          const typename Ar<AR>::TX* __restrict__ x, int nvec_rt, int e0,
                                          const typename Ar<AR>::TX* __restrict__ xb, const bool (&ok)[S],
                                          const int (&lo)[S], const uint32_t (&pk)[S],
                                          typename Ar<AR>::Acc (&acc)[S], typename Ar<AR>::TX* pfbuf) {
  using A = Ar<AR>;
  using TX = typename A::TX;
  using C = typename A::C;
  using Acc = typename A::Acc;
  using Dsum = typename A::Dsum;
  using E = typename A::E;
  constexpr int NT = kNT;
  const int nvec = NV1 ? 1 : nvec_rt;
  const C* __restrict__ tab = A::tab(P);
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
      const KGroup gr = L.dgrp[g];
      const Dsum U = L.grp_U[g];
      const int vb = L.grp_v[g];
#pragma unroll
      for (int s = 0; s < S; ++s) A::dmadd(ds[s], tab[vb + low_digit(pk[s], gr.lbit, gr.lwid)], U);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      TX xv;
      if (FULL || ok[s]) xv = __ldg(xb + s * NT);
      else xv = TX{};
      acc[s] = A::dmul(ds[s], xv);
    }
  }
  // ---- hops with block-uniform coefficients (high digits only); the list
  //      holds only channels whose source digits are in range (Sec. IV.B step 3) ----
  const int nact = L.n_act[0];
  TX* pf = pfbuf ? pfbuf + threadIdx.x : nullptr;
  if constexpr (PF > 0) {
    // source offsets relative to the block start: act_src - ebase
    pf_sum<AR, S, PF>(acc, L.act_c, L.act_src, nact, x + e0, ok, pf);
  } else {
#pragma unroll(S >= 6 ? 2 : 4)
  for (int c = 0; c < nact; ++c) {
    const C cf = L.act_c[c];
    const TX* __restrict__ src = x + L.act_src[c] + e0;
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (FULL || ok[s]) A::fma(acc[s], cf, __ldg(src + s * NT));
  }
  }
  // ---- factorised high/low hops, grouped by their low factor ----
  for (int g = P.n_grp_diag; g < P.n_grp_diag + P.n_grp; ++g) {
    const KGroup gr = L.dgrp[g];
    const int vb = L.grp_v[g];
    if constexpr (VINV) {
      const C v0 = tab[vb + low_digit(pk[0], gr.lbit, gr.lwid)];
      if (!A::nz(v0)) continue;  // inadmissible low digit for all S elements
      const int na = L.gact_n[g];
      const C* __restrict__ gu = L.gact_u + gr.m0;
      const long long* __restrict__ gs = L.gact_src + gr.m0;
      if constexpr (PF > 0) {
        pf_sum<AR, S, PF, true>(acc, gu, gs, na, xb, ok, pf, v0);
      } else {
#pragma unroll(S >= 6 ? 2 : 4)
        for (int j = 0; j < na; ++j) {
          const C c = A::cmul(v0, gu[j]);
          const TX* __restrict__ src = xb + gs[j];
#pragma unroll
          for (int s = 0; s < S; ++s)
            if (FULL || ok[s]) A::fma(acc[s], c, __ldg(src + s * NT));
        }
      }
      continue;
    }
    C v[S];
    Acc ag[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      v[s] = tab[vb + low_digit(pk[s], gr.lbit, gr.lwid)];
      ag[s] = A::azero();
    }
    const int na = L.gact_n[g];
    const C* __restrict__ gu = L.gact_u + gr.m0;
    const long long* __restrict__ gs = L.gact_src + gr.m0;
    if (PF > 0 && L.gact_ok[g]) {
      pf_sum<AR, S, (PF > 0 ? PF : 1)>(ag, gu, gs, na, xb, ok, pf);
    } else if (PF > 0) {
      bool m[S];
#pragma unroll
      for (int s = 0; s < S; ++s) m[s] = (FULL || ok[s]) && A::nz(v[s]);
      pf_sum<AR, S, (PF > 0 ? PF : 1)>(ag, gu, gs, na, xb, m, pf);
    } else if (L.gact_ok[g]) {
      // every active member's addresses lie inside x: an inadmissible low
      // digit (v = 0) gathers a finite in-range value scaled by exactly zero
#pragma unroll(S >= 6 ? 2 : 4)
      for (int j = 0; j < na; ++j) {
        const C u = gu[j];
        const TX* __restrict__ src = xb + gs[j];
#pragma unroll
        for (int s = 0; s < S; ++s)
          if (FULL || ok[s]) A::fma(ag[s], u, __ldg(src + s * NT));
      }
    } else {
      for (int j = 0; j < na; ++j) {
        const C u = gu[j];
        const TX* __restrict__ src = xb + gs[j];
#pragma unroll
        for (int s = 0; s < S; ++s)
          if ((FULL || ok[s]) && A::nz(v[s])) A::fma(ag[s], u, __ldg(src + s * NT));
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) A::acc_mul(acc[s], v[s], ag[s]);
  }
  // ---- hops inside the low block: packed ELL {delta, coef}, zero padding ----
  {
    const E* __restrict__ et = A::ell(P);
#pragma unroll(S >= 6 ? 2 : 4)
    for (int w = 0; w < P.ell_w; ++w) {
      const E* __restrict__ er = et + (long long)w * P.B;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const E en = __ldg(er + lo[s]);
        if (FULL || ok[s])
          A::fma(acc[s], A::ell_coef(en), __ldg(xb + (s * NT + A::ell_delta(en) * nvec)));
      }
    }
  }
}

// One chunk of NT*S elements starting at element `e_start` of low block blk
// (uniforms already in L): the sums of chunk_sum, stored.
template <int AR, int S, bool FULL, bool NV1, int PF = 0, bool VINV = false>
__device__ __forceinline__ void apply_chunk(const KPlan& P, const Lists<AR>& L,
                                            const typename Ar<AR>::TX* __restrict__ x,
                                            typename Ar<AR>::TY* __restrict__ y, int nvec_rt, NvDiv nvdiv,
                                            long long blk, int e_start, typename Ar<AR>::TX* pfbuf = nullptr) {
  using A = Ar<AR>;
  using TY = typename A::TY;
  constexpr int NT = kNT;
  const int nvec = NV1 ? 1 : nvec_rt;
  const int belems = P.B * nvec;
  const long long ebase = blk * (long long)belems;
  const int e0 = e_start + (int)threadIdx.x;
  bool ok[S];
  int lo[S];
  uint32_t pk[S];
  chunk_states<S, FULL, NV1>(P, belems, e0, nvdiv, ok, lo, pk);
  typename A::Acc acc[S];
  chunk_sum<AR, S, FULL, NV1, PF, VINV>(P, L, x, nvec, e0, x + ebase + e0, ok, lo, pk, acc, pfbuf);
  // ---- store: one write per output element (the second pass of a
  //      top-site split adds its rounded sum to the first pass's value) ----
  TY* __restrict__ yb = y + ebase + e0;
  if (P.accum) {
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (FULL || ok[s]) st_y(yb + s * NT, A::add_out(yb[s * NT], A::out(acc[s])));
  } else {
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (FULL || ok[s]) st_y(yb + s * NT, A::out(acc[s]));
  }
}

// Low block visited at position q of a launch: q itself, or, for the second
// pass of a top-site split, the block whose leading tperm_T digits are
// q mod R (R their combinations) and whose other high digits are q / R.
__device__ __forceinline__ long long visit_block(const KPlan& P, long long q) {
  if (P.tperm_T <= 0) return q;
  const long long Mt = P.sites[P.tperm_T - 1].mh;  // blocks per top-digit combination
  const long long R = P.nblk / Mt;
  return (q % R) * Mt + q / R;
}

// A block of belems elements is cut into nS chunks of NT*S elements, then n1
// chunks of NT elements, then (if needed) one partial NT-chunk, so all but
// the last chunk run without per-element predicates.
struct ChunkPlan {
  int nS, n1, tail;  // tail: 1 if a partial chunk follows
  __host__ __device__ int count() const { return nS + n1 + tail; }
};

__host__ __device__ inline ChunkPlan chunk_plan(int belems, int S) {
  ChunkPlan c;
  c.nS = belems / (kNT * S);
  const int rem = belems - c.nS * kNT * S;
  c.n1 = rem / kNT;
  c.tail = (rem - c.n1 * kNT) > 0;
  return c;
}

template <int AR, int S, bool NV1, int PF = 0, bool VINV = false>
__device__ __forceinline__ void apply_item(const KPlan& P, const Lists<AR>& L, const typename Ar<AR>::TX* x,
                                           typename Ar<AR>::TY* y, int nvec, NvDiv nvdiv, long long blk,
                                           const ChunkPlan& cp, int c, typename Ar<AR>::TX* pfbuf = nullptr) {
  if (c < cp.nS) {
    apply_chunk<AR, S, true, NV1, PF, VINV>(P, L, x, y, nvec, nvdiv, blk, c * kNT * S, pfbuf);
  } else if (c < cp.nS + cp.n1) {
    apply_chunk<AR, 1, true, NV1, 0, VINV>(P, L, x, y, nvec, nvdiv, blk, cp.nS * kNT * S + (c - cp.nS) * kNT);
  } else {
    apply_chunk<AR, 1, false, NV1, 0, VINV>(P, L, x, y, nvec, nvdiv, blk, cp.nS * kNT * S + cp.n1 * kNT);
  }
}

// Every factorised group's low digit is the same for a thread's elements
// t, t + NT, ...: the digit's period (KPlan::vperiod, in states) divides the
// stride NT / nvec states (the elements interleave nvec right-hand sides).
inline bool groups_invariant(const KPlan& k, long long nvec) {
  if (k.vperiod <= 0 || kNT % nvec != 0) return false;
  return (kNT / nvec) % k.vperiod == 0;
}

// Resident CTAs per SM the register allocation must allow: default (MBV = 0)
// or one more (MBV = 1, fewer registers per thread); the autotuner picks.
template <int AR, int MBV> struct MinBlocks { static constexpr int v = 2 + MBV; };
template <int MBV> struct MinBlocks<AR_F32, MBV> { static constexpr int v = 4 + MBV; };
template <int MBV> struct MinBlocks<AR_F32V2, MBV> { static constexpr int v = 2 + MBV; };

// bytes of the per-thread prefetch stages of the PF variant, placed after
// the block lists
template <int AR, int S, int PF>
__host__ __device__ constexpr size_t pf_bytes() {
  return (size_t)PF * S * kNT * sizeof(typename Ar<AR>::TX);
}

// PF = 0: gathers as plain loads; PF > 0: each thread prefetches its gathers
// of the full-size chunks PF items ahead with cp.async (pf_sum)
template <int AR, int S, bool NV1, int MBV, int PF = 0, bool VINV = false>
__global__ void __launch_bounds__(kNT, MinBlocks<AR, MBV>::v)
k_apply(const KPlan P, const typename Ar<AR>::TX* __restrict__ x, typename Ar<AR>::TY* __restrict__ y,
        int nvec, NvDiv nvdiv, KGate gate) {
  if (gate_closed(gate)) return;
  extern __shared__ __align__(16) unsigned char sm[];
  const Lists<AR> L = carve<AR>(sm, P.n_hh_diag + P.n_hh, P.n_mem, P.n_grp_diag + P.n_grp, P.n_grp_diag);
  typename Ar<AR>::TX* pfbuf = nullptr;
  if constexpr (PF > 0)
    pfbuf = (typename Ar<AR>::TX*)(sm + ((lists_bytes<AR>(P.n_hh_diag + P.n_hh, P.n_mem, P.n_grp_diag + P.n_grp,
                                                          P.n_grp_diag) + 15) & ~size_t(15)));
  load_descriptors<AR>(P, L);
  const ChunkPlan cp = chunk_plan(P.B * nvec, S);
  const int nchunks = cp.count();
  const long long nitems = P.nblk * nchunks;
  long long cur = -1;
  // whole blocks per CTA when there are enough of them and the blocks in
  // flight fit in L2 with room to spare; else (block, chunk) items, so that
  // the CTAs share a few blocks at a time
  const long long inflight = (long long)P.B * nvec * sizeof(typename Ar<AR>::TX) * gridDim.x;
  if (P.nblk >= 2LL * gridDim.x && inflight <= kInflightMax) {
    // full rounds of whole blocks; the blocks of a last round that would
    // leave most CTAs idle are cut into (block, chunk) items so that every
    // CTA shares that round
    long long full = (P.nblk / gridDim.x) * gridDim.x;
    if (2 * (P.nblk - full) >= gridDim.x) full = P.nblk;
    for (long long q = blockIdx.x; q < full; q += gridDim.x) {
      const long long blk = visit_block(P, q);
      eval_block<AR>(P, L, blk, nvec);
      for (int c = 0; c < nchunks; ++c) apply_item<AR, S, NV1, PF, VINV>(P, L, x, y, nvec, nvdiv, blk, cp, c, pfbuf);
      __syncthreads();
    }
    const long long rest = (P.nblk - full) * nchunks;
    for (long long w = blockIdx.x; w < rest; w += gridDim.x) {
      const long long q = full + w / nchunks;
      const long long blk = visit_block(P, q);
      if (blk != cur) {
        cur = blk;
        eval_block<AR>(P, L, blk, nvec);
      }
      apply_item<AR, S, NV1, PF, VINV>(P, L, x, y, nvec, nvdiv, blk, cp, (int)(w - (q - full) * nchunks), pfbuf);
      __syncthreads();
    }
  } else {
    for (long long w = blockIdx.x; w < nitems; w += gridDim.x) {
      const long long q = w / nchunks;
      const long long blk = visit_block(P, q);
      if (blk != cur) {
        cur = blk;
        eval_block<AR>(P, L, blk, nvec);
      }
      apply_item<AR, S, NV1, PF, VINV>(P, L, x, y, nvec, nvdiv, blk, cp, (int)(w - q * nchunks), pfbuf);
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Batched apply: many plans of uneven size in one persistent launch. Work
// items (instance, block) or (instance, block, chunk) are numbered by a
// prefix sum over instances; CTAs stride over that single index space. The
// batch's plans travel inside the kernel parameters (__grid_constant__, at
// most 32 KB), so, like k_apply's single plan, they are read from the
// constant bank; larger batches take several launches.
// ---------------------------------------------------------------------------
constexpr int kBatchMax = 128;
struct BatchArgs {
  int n, by_block;                 // by_block: items are whole blocks, else (block, chunk)
  long long start[kBatchMax + 1];  // prefix sum of items over instances
  const void* x[kBatchMax];
  void* y[kBatchMax];
  KPlan plans[kBatchMax];
};
static_assert(sizeof(BatchArgs) + 64 <= 32764, "kernel parameter limit");

template <int AR, int S, bool NV1>
__global__ void __launch_bounds__(kNT, MinBlocks<AR, 0>::v)
k_batch(const __grid_constant__ BatchArgs A, int nvec, NvDiv nvdiv) {
  extern __shared__ __align__(16) unsigned char sm[];
  using TX = typename Ar<AR>::TX;
  using TY = typename Ar<AR>::TY;
  const long long total = A.start[A.n];
  int inst = -1;
  long long cur = -1;
  Lists<AR> L{};
  ChunkPlan cp{};
  int nchunks = 1;
  for (long long w = blockIdx.x; w < total; w += gridDim.x) {
    int ni = inst < 0 ? 0 : inst;
    while (A.start[ni + 1] <= w) ++ni;
    const KPlan& P = A.plans[ni];
    if (ni != inst) {
      __syncthreads();
      inst = ni;
      cur = -1;
      L = carve<AR>(sm, P.n_hh_diag + P.n_hh, P.n_mem, P.n_grp_diag + P.n_grp, P.n_grp_diag);
      load_descriptors<AR>(P, L);
      cp = chunk_plan(P.B * nvec, S);
      nchunks = cp.count();
    }
    const long long local = w - A.start[inst];
    const TX* xi = (const TX*)A.x[inst];
    TY* yi = (TY*)A.y[inst];
    if (A.by_block) {
      eval_block<AR>(P, L, local, nvec);
      for (int c = 0; c < nchunks; ++c) apply_item<AR, S, NV1>(P, L, xi, yi, nvec, nvdiv, local, cp, c);
    } else {
      const long long blk = local / nchunks;
      if (blk != cur) {
        cur = blk;
        eval_block<AR>(P, L, blk, nvec);
      }
      apply_item<AR, S, NV1>(P, L, xi, yi, nvec, nvdiv, blk, cp, (int)(local - blk * nchunks));
    }
    __syncthreads();
  }
}

// FP64 input split into (hi, lo) float pairs, once per apply (range and the
// window bit patterns wlo, whi: see split_vector)
__global__ void k_split_f64(const double* __restrict__ x, float2* __restrict__ xs, long long n, int* range,
                            unsigned long long wlo, unsigned long long whi);

}  // namespace hm
