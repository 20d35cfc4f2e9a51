// y = H x, target-driven (pull) form of Sec. II with every gather served from
// shared memory: the "staged" apply kernel.
//
// The index space is cut into blocks of B states (the trailing, "low" sites;
// B * nvec <= kStreamElems elements). Within a block the leading ("high")
// digits are uniform, so every channel that touches a high site reads one
// contiguous range of x: the block shifted by the channel's source offset
// (Sec. IV.B Eq. sourceoffset). A CTA is warp-specialised:
//
//   * warp 0 (evaluator) computes, per block and up to two blocks ahead,
//     the high digits, the coefficient of every high channel and the high
//     factor of every factorised high/low channel, keeps the admissible ones
//     (Sec. IV.B steps 2-4: a zero coefficient is an inadmissible source
//     digit) and writes them to a block descriptor (three in flight);
//   * warp 1 (copier) streams each block's own x and every admissible hop's
//     source range into shared memory with 1-D bulk copies (cp.async.bulk)
//     through a ring of slots guarded by mbarriers, so copies never wait for
//     a descriptor to be computed;
//   * warps 2..NC+1 (consumers) own S elements each (stride 32 * NC, so every
//     shared-memory access of a warp is one contiguous run) and apply
//       y_F = (diagonal) x_F + sum_low hops c(F) x_{F+d}         [own block]
//           + sum_uniform hops c x_{F+off}                        [ring]
//           + sum_groups v_g(F) sum_members u_m x_{F+off_m}       [ring]
//     then write y_F once (no atomics).
//
// The copier runs up to kSRing ranges ahead of the consumers, so the copies
// of later ranges are in flight while they compute: the kernel's memory
// parallelism comes from the bulk copies, not from thread count.
// Every mbarrier wait is bounded (tma.cuh); a wait that gives up sets
// g_hm_status and the CTA stops after draining its own copies.
#pragma once

#include "apply_kernel.cuh"
#include "tma.cuh"

namespace hm {

#ifndef HM_SRING
#define HM_SRING 4
#endif
constexpr int kSRing = HM_SRING;  // ring slots per CTA
constexpr int kSDesc = 3;         // block descriptors in flight

// device status word (per device and per translation unit that includes this
// header): bit 0 = a bounded wait of the staged kernel gave up
static __device__ int g_hm_status = 0;

template <int AR>
struct StreamDesc {  // per-block uniform values written by the producer warp
  using C = typename Ar<AR>::C;
  using Dsum = typename Ar<AR>::Dsum;
  Dsum* du;       // [1] sum of the high diagonal channels
  Dsum* gU;       // [n_grp_diag] sum of member u of each diagonal group
  int* gv;        // [n_grp_diag + n_grp] v row base of each group
  int* gcnt;      // [n_grp] admissible members of each off-diagonal group
  int* gok;       // [n_grp] 1: every admissible member range lies inside x
  int* nuni;      // [1] admissible uniform (high-high) hops
  C* rc;          // [nr] coefficient of each range, in consumption order
  int* rshift;    // [nr] first element of the range inside its slot
  long long* rsrc;  // [nr] element index of the range start (producer side)
};

template <int AR>
__host__ __device__ inline size_t stream_desc_bytes(int n_hh, int n_mem, int n_grp, int n_grpd) {
  using C = typename Ar<AR>::C;
  using Dsum = typename Ar<AR>::Dsum;
  auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
  const int nr = n_hh + n_mem;
  return al(sizeof(Dsum)) + al(n_grpd * sizeof(Dsum)) + al((n_grp + n_grpd) * 4) + 2 * al(n_grp * 4) + al(16) +
         al(nr * sizeof(C)) + al(nr * 4) + al(nr * 8);
}

template <int AR>
__device__ inline StreamDesc<AR> stream_desc_carve(unsigned char* sm, int n_hh, int n_mem, int n_grp, int n_grpd) {
  using C = typename Ar<AR>::C;
  using Dsum = typename Ar<AR>::Dsum;
  auto al = [](size_t b) { return (b + 15) & ~size_t(15); };
  const int nr = n_hh + n_mem;
  StreamDesc<AR> D;
  size_t o = 0;
  D.du = (Dsum*)(sm + o);     o += al(sizeof(Dsum));
  D.gU = (Dsum*)(sm + o);     o += al(n_grpd * sizeof(Dsum));
  D.gv = (int*)(sm + o);      o += al((n_grp + n_grpd) * 4);
  D.gcnt = (int*)(sm + o);    o += al(n_grp * 4);
  D.gok = (int*)(sm + o);     o += al(n_grp * 4);
  D.nuni = (int*)(sm + o);    o += al(16);
  D.rc = (C*)(sm + o);        o += al(nr * sizeof(C));
  D.rshift = (int*)(sm + o);  o += al(nr * 4);
  D.rsrc = (long long*)(sm + o);
  return D;
}

// bytes of one slot: a block of x plus up to 16 bytes of alignment slack on
// each side, rounded to 128
template <int AR>
__host__ __device__ constexpr size_t stream_slot_bytes() {
  return ((size_t)kStreamElems * sizeof(typename Ar<AR>::TX) + 32 + 127) & ~size_t(127);
}

struct StreamLayout {  // byte offsets inside dynamic shared memory
  size_t bars, own, ring, desc, grp, hd, total, desc_bytes;
};

template <int AR>
__host__ __device__ inline StreamLayout stream_layout(const KPlan& P) {
  StreamLayout L;
  const size_t sb = stream_slot_bytes<AR>();
  L.bars = 0;                                      // 2 * kSRing + 4 + 2 * kSDesc barriers
  L.own = 256;
  L.ring = L.own + 2 * sb;
  L.desc = L.ring + kSRing * sb;
  L.desc_bytes = (stream_desc_bytes<AR>(P.n_hh, P.n_mem, P.n_grp, P.n_grp_diag) + 127) & ~size_t(127);
  L.grp = L.desc + kSDesc * L.desc_bytes;
  L.hd = L.grp + (((size_t)(P.n_grp_diag + P.n_grp) * sizeof(KGroup) + 15) & ~size_t(15));
  L.total = L.hd + 64 * 4;
  return L;
}

// Producer side of one range: bring x[src, src + E) (element indices into x
// of n elements) into `slot` and arrive on `full` expecting the bulk bytes.
// Element src + j lands at slot element shift + j, shift = (address of src
// mod 16) / element size. When the range widened to 16-byte boundaries stays
// inside x (every range but those touching the ends of x), that widened
// range is one bulk copy. Otherwise the aligned interior of the part inside x
// is bulk-copied and its unaligned head and tail (< 16 bytes each) are
// copied with plain loads; elements outside x are left untouched (the
// consumers read them only behind an admissibility test). One thread.
template <class TX>
__device__ __forceinline__ void stage_range(const TX* __restrict__ x, long long n, long long src, int E,
                                            unsigned char* slot, uint64_t* full) {
  constexpr long long es = sizeof(TX);
  const uintptr_t xb = (uintptr_t)x, xe = (uintptr_t)(x + n);
  const uintptr_t g0 = ((uintptr_t)(x + src)) & ~(uintptr_t)15;  // slot byte 0 (may lie before x)
  const uintptr_t g1 = ((uintptr_t)(x + src + E) + 15) & ~(uintptr_t)15;
  if (src >= 0 && src + E <= n && g0 >= xb && g1 <= xe) {
    mbar_arrive_expect_tx(full, (unsigned)(g1 - g0));
    bulk_g2s(slot, (const void*)g0, (unsigned)(g1 - g0), full);
    return;
  }
  const long long lo = src < 0 ? 0 : src;
  const long long hi = (src + E > n) ? n : src + E;
  if (hi > lo) {
    const uintptr_t b0 = (uintptr_t)(x + lo), b1 = (uintptr_t)(x + hi);
    const uintptr_t a0 = (b0 + 15) & ~(uintptr_t)15, a1 = b1 & ~(uintptr_t)15;
    if (a1 > a0) {
      for (uintptr_t b = b0; b < a0; b += es) *(TX*)(slot + (b - g0)) = __ldg((const TX*)b);
      for (uintptr_t b = a1; b < b1; b += es) *(TX*)(slot + (b - g0)) = __ldg((const TX*)b);
      fence_proxy_async();
      mbar_arrive_expect_tx(full, (unsigned)(a1 - a0));
      bulk_g2s(slot + (a0 - g0), (const void*)a0, (unsigned)(a1 - a0), full);
      return;
    }
    for (uintptr_t b = b0; b < b1; b += es) *(TX*)(slot + (b - g0)) = __ldg((const TX*)b);
  }
  mbar_arrive(full);
}

template <class TX>
__device__ __forceinline__ int range_shift(const TX* x, long long src) {
  return (int)((((uintptr_t)(x + src)) & 15) / sizeof(TX));
}

// Producer: uniform values of block blk into descriptor D (whole warp).
template <int AR>
__device__ __forceinline__ void stream_eval(const KPlan& P, const StreamDesc<AR>& D, const KGroup* grp, int* hd,
                                            const typename Ar<AR>::TX* x, long long blk, int nvec) {
  using A = Ar<AR>;
  using C = typename A::C;
  using Dsum = typename A::Dsum;
  const C* __restrict__ tab = A::tab(P);
  const int lane = threadIdx.x & 31;
  const long long E = (long long)P.B * nvec;
  const long long e0 = blk * E;
  const long long n = P.D * nvec;
  for (int t = lane; t < P.nhigh; t += 32) hd[t] = (int)((blk / P.sites[t].mh) % P.sites[t].d);
  __syncwarp();
  // diagonal high channels: fixed-order warp sum
  {
    Dsum d = A::dzero();
    for (int c = lane; c < P.n_hh_diag; c += 32) {
      const KChan ch = P.ch[c];
      const int nj = (ch.kind & CK_SINGLE) ? 0 : hd[ch.sj];
      A::dadd(d, tab[ch.tab + hd[ch.si] * ch.dj + nj]);
    }
    d = wsum(d);
    if (lane == 0) D.du[0] = d;
  }
  // admissible off-diagonal high channels, in channel order
  int nr = 0;
  for (int base = P.n_hh_diag; base < P.n_hh_diag + P.n_hh; base += 32) {
    const int c = base + lane;
    C cf{};
    long long src = 0;
    bool act = false;
    if (c < P.n_hh_diag + P.n_hh) {
      const KChan ch = P.ch[c];
      const int nj = (ch.kind & CK_SINGLE) ? 0 : hd[ch.sj];
      cf = tab[ch.tab + hd[ch.si] * ch.dj + nj];
      act = A::nz(cf);
      src = e0 + ch.off * nvec;
    }
    const unsigned msk = __ballot_sync(0xffffffffu, act);
    if (act) {
      const int pos = nr + __popc(msk & ((1u << lane) - 1u));
      D.rc[pos] = cf;
      D.rsrc[pos] = src;
      D.rshift[pos] = range_shift(x, src);
    }
    nr += __popc(msk);
  }
  if (lane == 0) D.nuni[0] = nr;
  // groups: v row base; diagonal groups sum their u, off-diagonal groups keep
  // their admissible members in member order
  const int ng = P.n_grp_diag + P.n_grp;
  for (int g = lane; g < ng; g += 32) {
    const KGroup gr = grp[g];
    D.gv[g] = gr.vtab + (gr.vstride ? hd[gr.vsite] * gr.vstride : 0);
  }
  for (int g = 0; g < P.n_grp_diag; ++g) {
    const KGroup gr = grp[g];
    Dsum d = A::dzero();
    for (int m = gr.m0 + lane; m < gr.m1; m += 32) {
      const KMember mb = P.mem[m];
      A::dadd(d, tab[mb.utab + hd[mb.usite]]);
    }
    d = wsum(d);
    if (lane == 0) D.gU[g] = d;
  }
  for (int g = P.n_grp_diag; g < ng; ++g) {
    const KGroup gr = grp[g];
    int cnt = 0;
    bool bad = false;
    for (int base = gr.m0; base < gr.m1; base += 32) {
      const int m = base + lane;
      C u{};
      bool act = false, ok = true;
      long long src = 0;
      if (m < gr.m1) {
        const KMember mb = P.mem[m];
        u = tab[mb.utab + hd[mb.usite]];
        act = A::nz(u);
        src = e0 + mb.off * nvec;
        ok = (src >= 0) && (src + E <= n);
      }
      const unsigned msk = __ballot_sync(0xffffffffu, act);
      bad |= __any_sync(0xffffffffu, act && !ok);
      if (act) {
        const int pos = nr + cnt + __popc(msk & ((1u << lane) - 1u));
        D.rc[pos] = u;
        D.rsrc[pos] = src;
        D.rshift[pos] = range_shift(x, src);
      }
      cnt += __popc(msk);
    }
    if (lane == 0) {
      D.gcnt[g - P.n_grp_diag] = cnt;
      D.gok[g - P.n_grp_diag] = !bad;
    }
    nr += cnt;
  }
  __syncwarp();
}

template <int AR, int NC>
struct StreamMinBlocks { static constexpr int v = 3; };
template <int NC>
struct StreamMinBlocks<AR_F32, NC> { static constexpr int v = 4; };

// S: elements per consumer thread (NC warps of consumers; S * 32 * NC >=
// B * nvec). NV1: nvec == 1.
template <int AR, int S, int NC, bool NV1>
__global__ void __launch_bounds__(32 * (NC + 2), StreamMinBlocks<AR, NC>::v)
k_stream(const KPlan P, const typename Ar<AR>::TX* __restrict__ x, typename Ar<AR>::TY* __restrict__ y, int nvec,
         NvDiv nvdiv, KGate gate) {
  if (gate_closed(gate)) return;
  using A = Ar<AR>;
  using TX = typename A::TX;
  using TY = typename A::TY;
  using C = typename A::C;
  using Acc = typename A::Acc;
  using Dsum = typename A::Dsum;
  using E_t = typename A::E;
  extern __shared__ __align__(128) unsigned char sm[];
  const StreamLayout Lo = stream_layout<AR>(P);
  constexpr size_t SB = stream_slot_bytes<AR>();
  uint64_t* bar = (uint64_t*)(sm + Lo.bars);
  uint64_t* full = bar;                       // [kSRing]
  uint64_t* empty = bar + kSRing;             // [kSRing]
  uint64_t* own_full = bar + 2 * kSRing;      // [2]
  uint64_t* own_empty = own_full + 2;         // [2]
  uint64_t* desc_full = own_full + 4;         // [kSDesc]
  uint64_t* desc_empty = desc_full + kSDesc;  // [kSDesc]
  unsigned char* own = sm + Lo.own;
  unsigned char* ring = sm + Lo.ring;
  KGroup* grp = (KGroup*)(sm + Lo.grp);
  int* hd = (int*)(sm + Lo.hd);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ng = P.n_grp_diag + P.n_grp;
  const int nvec_c = NV1 ? 1 : nvec;
  const int E = P.B * nvec_c;
  const long long nx = P.D * nvec_c;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kSRing; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, NC);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(own_full + i, 1);
      mbar_init(own_empty + i, NC);
    }
    for (int i = 0; i < kSDesc; ++i) {
      mbar_init(desc_full + i, 1);
      mbar_init(desc_empty + i, NC + 1);  // consumers and the copier read it
    }
    mbar_fence_init();
  }
  for (int g = threadIdx.x; g < ng; g += blockDim.x) grp[g] = P.grp[g];
  __syncthreads();

  bool failed = false;
  if (warp == 0) {
    // ------------------------------ evaluator -----------------------------
    int it = 0;
    for (long long blk = blockIdx.x; blk < P.nblk; blk += gridDim.x, ++it) {
      const int d = it % kSDesc;
      const unsigned use = (unsigned)(it / kSDesc);
      if (it >= kSDesc && !__all_sync(0xffffffffu, mbar_wait(desc_empty + d, (use - 1) & 1))) { failed = true; break; }
      const StreamDesc<AR> D = stream_desc_carve<AR>(sm + Lo.desc + d * Lo.desc_bytes, P.n_hh, P.n_mem, P.n_grp,
                                                     P.n_grp_diag);
      stream_eval<AR>(P, D, grp, hd, x, blk, nvec_c);
      if (lane == 0) mbar_arrive(desc_full + d);
    }
    if (failed && lane == 0) atomicOr(&g_hm_status, 1);
    return;
  }
  if (warp == 1) {
    // ------------------------------- copier -------------------------------
    long long k = 0;  // ranges issued so far (ring slot k % kSRing)
    int it = 0;
    int own_last[2] = {-1, -1};  // last block iteration staged into own[b]
    for (long long blk = blockIdx.x; blk < P.nblk; blk += gridDim.x, ++it) {
      const int d = it % kSDesc;
      const int b = it & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(desc_full + d, (unsigned)(it / kSDesc) & 1))) { failed = true; break; }
      const StreamDesc<AR> D = stream_desc_carve<AR>(sm + Lo.desc + d * Lo.desc_bytes, P.n_hh, P.n_mem, P.n_grp,
                                                     P.n_grp_diag);
      // the block's own x
      if (it >= 2 && !__all_sync(0xffffffffu, mbar_wait(own_empty + b, (unsigned)((it >> 1) - 1) & 1))) {
        failed = true;
        break;
      }
      if (lane == 0) stage_range<TX>(x, nx, blk * E, E, own + b * SB, own_full + b);
      own_last[b] = it;
      // every admissible hop's source range, in consumption order
      int nr = D.nuni[0];
      for (int g = 0; g < P.n_grp; ++g) nr += D.gcnt[g];
      for (int r = 0; r < nr; ++r, ++k) {
        const int slot = (int)(k % kSRing);
        const unsigned u = (unsigned)(k / kSRing);
        if (k >= kSRing && !__all_sync(0xffffffffu, mbar_wait(empty + slot, (u - 1) & 1))) { failed = true; break; }
        if (lane == 0) stage_range<TX>(x, nx, D.rsrc[r], E, ring + slot * SB, full + slot);
      }
      if (failed) break;
      __syncwarp();
      if (lane == 0) mbar_arrive(desc_empty + d);  // done with this descriptor
    }
    if (failed && lane == 0) {
      atomicOr(&g_hm_status, 1);
      // drain (bounded) the copies this CTA issued: the last use of each
      // ring slot and of each own buffer
      for (int i = 0; i < kSRing; ++i)
        if (k > i) {
          const long long kl = i + ((k - 1 - i) / kSRing) * kSRing;
          mbar_wait(full + i, (unsigned)(kl / kSRing) & 1);
        }
      for (int i = 0; i < 2; ++i)
        if (own_last[i] >= 0) mbar_wait(own_full + i, (unsigned)(own_last[i] >> 1) & 1);
    }
    return;
  }
  // ------------------------------ consumers -------------------------------
  const int c = threadIdx.x - 64;  // consumer thread index
  constexpr int NCT = 32 * NC;
  const C* __restrict__ tab = A::tab(P);
  const C* __restrict__ dtab = A::diag(P);
  const E_t* __restrict__ ell = A::ell(P);
  int es[S], lo[S];
  bool ok[S];
  uint32_t pk[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    es[s] = c + s * NCT;
    ok[s] = es[s] < E;
    lo[s] = ok[s] ? (NV1 ? es[s] : nvdiv(es[s])) : 0;
    pk[s] = __ldg(P.ptab + lo[s]);
  }
  long long k = 0;
  int it = 0;
  for (long long blk = blockIdx.x; blk < P.nblk; blk += gridDim.x, ++it) {
    const int d = it % kSDesc;
    const int b = it & 1;
    if (!__all_sync(0xffffffffu, mbar_wait(desc_full + d, (unsigned)(it / kSDesc) & 1))) { failed = true; break; }
    const StreamDesc<AR> D =
        stream_desc_carve<AR>(sm + Lo.desc + d * Lo.desc_bytes, P.n_hh, P.n_mem, P.n_grp, P.n_grp_diag);
    if (!__all_sync(0xffffffffu, mbar_wait(own_full + b, (unsigned)(it >> 1) & 1))) { failed = true; break; }
    const TX* __restrict__ xo = (const TX*)(own + b * SB) + range_shift(x, blk * (long long)E);
    Acc acc[S];
    // ---- diagonal: block-uniform sum + low table + factorised diagonal groups ----
    {
      Dsum ds[S];
      const Dsum du = D.du[0];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        ds[s] = du;
        A::dadd(ds[s], dtab[lo[s]]);
      }
      for (int g = 0; g < P.n_grp_diag; ++g) {
        const KGroup gr = grp[g];
        const Dsum U = D.gU[g];
        const int vb = D.gv[g];
#pragma unroll
        for (int s = 0; s < S; ++s) A::dmadd(ds[s], tab[vb + low_digit(pk[s], gr.lbit, gr.lwid)], U);
      }
#pragma unroll
      for (int s = 0; s < S; ++s) acc[s] = A::dmul(ds[s], ok[s] ? xo[es[s]] : TX{});
    }
    // ---- hops inside the low block: packed ELL over the own block ----
#pragma unroll 2
    for (int w = 0; w < P.ell_w; ++w) {
      const E_t* __restrict__ er = ell + (long long)w * P.B;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        if (!ok[s]) continue;
        const E_t en = __ldg(er + lo[s]);
        A::fma(acc[s], A::ell_coef(en), xo[es[s] + A::ell_delta(en) * nvec_c]);
      }
    }
    // ---- uniform hops (high digits only): one ring range each ----
    const int nuni = D.nuni[0];
    for (int r = 0; r < nuni; ++r, ++k) {
      const int slot = (int)(k % kSRing);
      if (!__all_sync(0xffffffffu, mbar_wait(full + slot, (unsigned)(k / kSRing) & 1))) { failed = true; break; }
      const TX* __restrict__ xs = (const TX*)(ring + slot * SB) + D.rshift[r];
      const C cf = D.rc[r];
#pragma unroll
      for (int s = 0; s < S; ++s)
        if (ok[s]) A::fma(acc[s], cf, xs[es[s]]);
      __syncwarp();
      if (lane == 0) mbar_arrive(empty + slot);
    }
    if (failed) break;
    // ---- factorised high/low hops, one ring range per admissible member ----
    int r = nuni;
    for (int g = 0; g < P.n_grp && !failed; ++g) {
      const KGroup gr = grp[P.n_grp_diag + g];
      const int vb = D.gv[P.n_grp_diag + g];
      C v[S];
      Acc ag[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        v[s] = tab[vb + low_digit(pk[s], gr.lbit, gr.lwid)];
        ag[s] = A::azero();
      }
      const int cnt = D.gcnt[g];
      const bool gok = D.gok[g] != 0;
      for (int j = 0; j < cnt; ++j, ++r, ++k) {
        const int slot = (int)(k % kSRing);
        if (!__all_sync(0xffffffffu, mbar_wait(full + slot, (unsigned)(k / kSRing) & 1))) { failed = true; break; }
        const TX* __restrict__ xs = (const TX*)(ring + slot * SB) + D.rshift[r];
        const C u = D.rc[r];
        if (gok) {
          // every address of the range lies inside x: an inadmissible low
          // digit (v = 0) gathers a finite value that is scaled by zero
#pragma unroll
          for (int s = 0; s < S; ++s)
            if (ok[s]) A::fma(ag[s], u, xs[es[s]]);
        } else {
#pragma unroll
          for (int s = 0; s < S; ++s)
            if (ok[s] && A::nz(v[s])) A::fma(ag[s], u, xs[es[s]]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + slot);
      }
#pragma unroll
      for (int s = 0; s < S; ++s) A::acc_mul(acc[s], v[s], ag[s]);
    }
    if (failed) break;
    // ---- store: one write per output element, streamed past L2 ----
    TY* __restrict__ yb = y + blk * (long long)E;
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (ok[s]) __stcs(yb + es[s], A::out(acc[s]));
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(own_empty + b);
      mbar_arrive(desc_empty + d);
    }
  }
  if (failed && lane == 0) atomicOr(&g_hm_status, 1);
}

}  // namespace hm
