// Block-structured form of the fixed digit-sum sector apply (Sec. VI case 2,
// App. D), the sector counterpart of the full-basis kernel's low block.
//
// The sites split into a prefix (the leading h sites) and a suffix (the
// trailing ones, at most kSBMax suffix tuples). In the packed order
// (ascending full index) the retained states with a given prefix tuple p of
// digit sum P form one contiguous block: the suffix tuples of sum t = K - P in
// ascending order, so a state is (block p, rank r within the suffix sector t).
// Everything that depends on the suffix only is tabulated once per plan,
// indexed by the suffix tuple's position g = off[t] + r (at most kSBMax
// entries): its packed digits, the suffix-only diagonal, the suffix-only
// moves as {rank delta, coefficient} (the suffix sum is conserved, so source
// and target share the sector) and, for every move that couples a prefix
// site with a suffix site, the rank of the source suffix tuple in its sector
// t' = t - q (q the suffix digit's move). Per block the prefix digits are
// decoded once; prefix-only channels are block-uniform (diagonal sum, and
// moves whose source is the same rank in block p' with an offset
// start[p'] - start[p]); coupled channels keep their prefix digit's factor
// and source block fixed for the block. Per state: one packed-digit read,
// the tables above and one gather per admissible move -- no unranking, no
// per-state rank arithmetic. Arithmetic as in the per-row sector kernel
// (FP32, or double-float on the FP32 pipe for FP64 storage).
#include <algorithm>
#include <cstring>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "device_common.cuh"

namespace hm {

constexpr long long kSBMax = 16384;        // suffix tuples (per-suffix tables)
constexpr long long kSBBlocksMax = 1 << 22; // prefix tuples (block starts)
constexpr int kSBNT = 256;
constexpr int kSBChMax = 256;               // channels of one plan in shared memory
// states per thread and pass with one right-hand side: the faster of 2, 4
// and 8 on the N = 30 chain's M = 0 sector (FP32 4: 3.1 ms; double-float 2:
// 6.4 ms)
template <int AR>
constexpr int sb_states_per_thread() {
  return AR == AR_F32 ? 4 : 2;
}

template <int AR> struct SBAr;
template <> struct SBAr<AR_F32> {
  using TX = float;
  using TY = float;
  using C = float;
  using Acc = float;
  __device__ static const C* tab(const KSecBlk& S) { return S.tab_f; }
  __device__ static const C* dS(const KSecBlk& S) { return S.dS_f; }
  __device__ static const C* ell(const KSecBlk& S) { return S.ell_f; }
  __device__ static bool nz(C c) { return c != 0.0f; }
  __device__ static Acc zero() { return 0.0f; }
  __device__ static void add(Acc& a, C c) { a = __fadd_rn(a, c); }
  __device__ static void fma(Acc& a, C c, TX x) { a = __fmaf_rn(c, x, a); }
  __device__ static C norm(Acc a) { return a; }
  __device__ static TY out(Acc hop, Acc d, TX xo) { return __fmaf_rn(d, xo, hop); }
};
template <> struct SBAr<AR_DF64> {
  using TX = float2;
  using TY = double;
  using C = float2;
  using Acc = DF;
  __device__ static const C* tab(const KSecBlk& S) { return S.tab_df; }
  __device__ static const C* dS(const KSecBlk& S) { return S.dS_df; }
  __device__ static const C* ell(const KSecBlk& S) { return S.ell_df; }
  __device__ static bool nz(C c) { return c.x != 0.0f; }
  __device__ static Acc zero() { return DF{0.f, 0.f}; }
  __device__ static void add(Acc& a, C c) { df_add(a, c); }
  __device__ static void fma(Acc& a, C c, TX x) { df_fma(a, c, x.x, x.y); }
  __device__ static C norm(Acc a) { return df_norm(a); }
  __device__ static TY out(Acc hop, Acc d, TX xo) {
    df_fma(hop, df_norm(d), xo.x, xo.y);
    return df_to_double(hop);
  }
};

__device__ __forceinline__ int sb_digit(uint32_t pk, int bit, int wid) { return (int)((pk >> bit) & ((1u << wid) - 1u)); }

// NV: right-hand sides, fixed (1: SE states per thread and pass) or up to 8
// per pass chosen at run time (0: one state per thread and pass)
template <int AR, int NV, int SE = sb_states_per_thread<AR>()>
__global__ void __launch_bounds__(kSBNT) k_sector_blk(const KSecBlk S, const typename SBAr<AR>::TX* __restrict__ x,
                                                      typename SBAr<AR>::TY* __restrict__ y, int nvec) {
  using P = SBAr<AR>;
  using C = typename P::C;
  using TX = typename P::TX;
  __shared__ int dig[64];
  __shared__ KSBChan chs[kSBChMax];
  __shared__ C du_s;
  __shared__ int nact;
  __shared__ C act_c[kSBChMax];
  __shared__ long long act_off[kSBChMax];
  __shared__ int mrow[kSBChMax];    // coupled channels: table index = mrow + mmul * n_suffix
  __shared__ int mmul[kSBChMax];
  __shared__ long long msrc[kSBChMax];  // coupled moves: start of the source block (-1: none)
  const C* __restrict__ tab = P::tab(S);
  for (int c = threadIdx.x; c < S.nch; c += kSBNT) chs[c] = S.ch[c];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long ib = blockIdx.x; ib < S.nvb; ib += gridDim.x) {
    const long long b = S.vb[ib];
    for (int k = threadIdx.x; k < S.h; k += kSBNT) dig[k] = (int)((b / S.mp[k]) % S.pdim[k]);
    __syncthreads();
    const long long sb = S.start[b];
    if (warp == 0) {
      // prefix diagonal sum, in channel order (deterministic)
      if (lane == 0) {
        typename P::Acc d = P::zero();
        for (int c = 0; c < S.n0; ++c) {
          const KSBChan ch = chs[c];
          P::add(d, tab[ch.tab + dig[ch.si] * ch.dj + (ch.sj >= 0 ? dig[ch.sj] : 0)]);
        }
        du_s = P::norm(d);
      }
    } else if (warp == 1) {
      // admissible prefix moves, compacted in channel order
      int count = 0;
      for (int base = S.n0; base < S.n1; base += 32) {
        const int c = base + lane;
        C cf{};
        bool act = false;
        if (c < S.n1) {
          const KSBChan ch = chs[c];
          cf = tab[ch.tab + dig[ch.si] * ch.dj + dig[ch.sj]];
          act = P::nz(cf);
        }
        const unsigned msk = __ballot_sync(0xffffffffu, act);
        if (act) {
          const int pos = count + __popc(msk & ((1u << lane) - 1u));
          act_c[pos] = cf;
          act_off[pos] = S.start[b - chs[c].dblk] - sb;
        }
        count += __popc(msk);
      }
      if (lane == 0) nact = count;
    } else {
      // coupled channels: prefix factor row and source block
      for (int c = S.n1 + (int)threadIdx.x - 64; c < S.nch; c += kSBNT - 64) {
        const KSBChan ch = chs[c];
        const int np = dig[ch.pfx ? ch.sj : ch.si];
        mrow[c] = ch.pfx ? ch.tab + np : ch.tab + np * ch.dj;
        mmul[c] = ch.pfx ? ch.dj : 1;
        long long src = -1;
        if (ch.kind == SB_MMOVE) {
          const int ps = ch.pfx ? ch.sj : ch.si;
          const int ns = np - ch.qp;
          if (ns >= 0 && ns < S.pdim[ps]) src = S.start[b - ch.dblk];
        }
        msrc[c] = src;
      }
    }
    __syncthreads();
    int P0 = 0;
    for (int k = 0; k < S.h; ++k) P0 += dig[k];
    const int t = S.K - P0;
    const int g0 = S.off[t], len = S.off[t + 1] - g0;
    const C du = du_s;
    const int na = nact;
    if constexpr (NV == 1) {
      // SE states per thread and pass, every gather of a pass independent
      // (padding ELL entries are {0, 0}: an in-range read scaled by zero)
      for (int r0 = 0; r0 < len; r0 += kSBNT * SE) {
        int gs[SE];
        bool ok[SE];
        uint32_t pk[SE];
        typename P::Acc d[SE], acc[SE];
        long long F[SE];
#pragma unroll
        for (int e = 0; e < SE; ++e) {
          const int r = r0 + (int)threadIdx.x + e * kSBNT;
          ok[e] = r < len;
          gs[e] = g0 + (ok[e] ? r : 0);
          F[e] = sb + (ok[e] ? r : 0);
          pk[e] = __ldg(S.sdig + gs[e]);
          d[e] = P::zero();
          P::add(d[e], du);
          P::add(d[e], __ldg(P::dS(S) + gs[e]));
          acc[e] = P::zero();
        }
        for (int c = S.n1; c < S.n2; ++c) {
          const KSBChan& ch = chs[c];
#pragma unroll
          for (int e = 0; e < SE; ++e) P::add(d[e], tab[mrow[c] + mmul[c] * sb_digit(pk[e], ch.lbit, ch.lwid)]);
        }
#pragma unroll 2
        for (int j = 0; j < na; ++j) {
          const C cf = act_c[j];
          const long long o = act_off[j];
#pragma unroll
          for (int e = 0; e < SE; ++e) P::fma(acc[e], cf, __ldg(x + F[e] + o));
        }
#pragma unroll 2
        for (int w = 0; w < S.w; ++w) {
#pragma unroll
          for (int e = 0; e < SE; ++e) {
            const long long i = (long long)w * S.G + gs[e];
            P::fma(acc[e], __ldg(P::ell(S) + i), __ldg(x + F[e] + __ldg(S.ell_r + i)));
          }
        }
        for (int c = S.n2; c < S.nch; ++c) {
          const KSBChan& ch = chs[c];
          if (msrc[c] < 0) continue;
#pragma unroll
          for (int e = 0; e < SE; ++e) {
            const C cf = tab[mrow[c] + mmul[c] * sb_digit(pk[e], ch.lbit, ch.lwid)];
            if (P::nz(cf)) P::fma(acc[e], cf, __ldg(x + msrc[c] + __ldg(S.xr + (long long)ch.xr * S.G + gs[e])));
          }
        }
#pragma unroll
        for (int e = 0; e < SE; ++e)
          if (ok[e]) y[F[e]] = P::out(acc[e], d[e], __ldg(x + F[e]));
      }
    } else {
      for (int r = threadIdx.x; r < len; r += kSBNT) {
        const int g = g0 + r;
        const uint32_t pk = __ldg(S.sdig + g);
        typename P::Acc d = P::zero();
        P::add(d, du);
        P::add(d, __ldg(P::dS(S) + g));
        for (int c = S.n1; c < S.n2; ++c) {
          const KSBChan& ch = chs[c];
          P::add(d, tab[mrow[c] + mmul[c] * sb_digit(pk, ch.lbit, ch.lwid)]);
        }
        const long long F = sb + r;
        for (int v0 = 0; v0 < nvec; v0 += 8) {
          const int nv = min(8, nvec - v0);
          auto at = [&](long long row) { return row * nvec + v0; };
          typename P::Acc acc[8];
          for (int v = 0; v < nv; ++v) acc[v] = P::zero();
          for (int j = 0; j < na; ++j) {
            const C cf = act_c[j];
            const TX* xs = x + at(F + act_off[j]);
            for (int v = 0; v < nv; ++v) P::fma(acc[v], cf, xs[v]);
          }
          for (int w = 0; w < S.w; ++w) {
            const C cf = __ldg(P::ell(S) + (long long)w * S.G + g);
            if (!P::nz(cf)) continue;
            const TX* xs = x + at(F + __ldg(S.ell_r + (long long)w * S.G + g));
            for (int v = 0; v < nv; ++v) P::fma(acc[v], cf, xs[v]);
          }
          for (int c = S.n2; c < S.nch; ++c) {
            const KSBChan& ch = chs[c];
            if (msrc[c] < 0) continue;
            const C cf = tab[mrow[c] + mmul[c] * sb_digit(pk, ch.lbit, ch.lwid)];
            if (!P::nz(cf)) continue;
            const TX* xs = x + at(msrc[c] + __ldg(S.xr + (long long)ch.xr * S.G + g));
            for (int v = 0; v < nv; ++v) P::fma(acc[v], cf, xs[v]);
          }
          const TX* xo = x + at(F);
          typename P::TY* ys = y + at(F);
          for (int v = 0; v < nv; ++v) ys[v] = P::out(acc[v], d, xo[v]);
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host: tables of the block form (none when the plan does not fit them)
// ---------------------------------------------------------------------------

// Host tables of the block form for digit total K (ok = false when the plan
// does not fit it: then the per-row kernel serves). No device calls.
struct SBHost {
  bool ok = false;
  int h = 0, w = 0, G = 0, n0 = 0, n1 = 0, n2 = 0;
  long long K = 0;
  std::vector<long long> start, mp;
  std::vector<int> vb, pdim, off, ell_r, xr_flat;
  std::vector<uint32_t> sdig;
  std::vector<KSBChan> ch;
  std::vector<double> tab, dS, ell_d;
};

static int derive_sector_blk(const Plan* p, long long K, SBHost& o) {
  o = SBHost{};
  o.K = K;
  const int N = p->N;
  long long maxsum = 0;
  for (auto& st : p->sites) maxsum += st.dim - 1;
  if (K < 0 || K > maxsum) {
    set_error("digit total outside [0, sum_k (d_k - 1)]: the sector is empty");
    return HM_ERR_INVALID_ARG;
  }
  for (const Channel& c : p->chH) {  // the sector's terms conserve the digit sum
    bool nz = false;
    for (auto& z : c.T) nz = nz || z != std::complex<double>(0, 0);
    if (nz && c.qi + (c.j >= 0 ? c.qj : 0) != 0) {
      set_error("the term list does not conserve the sector's digit sum");
      return HM_ERR_UNSUPPORTED;
    }
  }
  // suffix: trailing sites with at most kSBMax tuples
  int h = N;
  long long Bs = 1;
  while (h > 0 && Bs * p->sites[h - 1].dim <= kSBMax) {
    Bs *= p->sites[h - 1].dim;
    --h;
  }
  long long nblk = 1;
  for (int k = 0; k < h; ++k) {
    nblk *= p->sites[k].dim;
    if (nblk > kSBBlocksMax) return HM_OK;  // no block form: the per-row kernel serves
  }
  if (h > 64 || K > 255) return HM_OK;
  // packed suffix digits and multipliers
  std::vector<long long> Ms(N, 1), mp(std::max(h, 1), 1);
  for (int k = N - 2; k >= h; --k) Ms[k] = Ms[k + 1] * p->sites[k + 1].dim;
  for (int k = h - 2; k >= 0; --k) mp[k] = mp[k + 1] * p->sites[k + 1].dim;
  std::vector<int> lbit(N, 0), lwid(N, 0);
  int bits = 0;
  for (int k = N - 1; k >= h; --k) {
    int w = 0;
    while ((1 << w) < p->sites[k].dim) ++w;
    lbit[k] = bits;
    lwid[k] = std::max(w, 1);
    bits += lwid[k];
  }
  if (bits > 32) return HM_OK;
  // suffix tuples by sum, ascending full index within a sum
  const int K1 = (int)K + 1;
  std::vector<int> cnt(K1 + 1, 0), tsum(Bs), rank(Bs, -1);
  std::vector<std::vector<int>> sdg(Bs, std::vector<int>(N, 0));
  for (long long i = 0; i < Bs; ++i) {
    int s = 0;
    for (int k = h; k < N; ++k) {
      sdg[i][k] = (int)((i / Ms[k]) % p->sites[k].dim);
      s += sdg[i][k];
    }
    tsum[i] = s;
    if (s <= K) rank[i] = cnt[s]++;
  }
  std::vector<int> off(K1 + 1, 0);
  for (int t = 0; t < K1; ++t) off[t + 1] = off[t] + cnt[t];
  const int G = off[K1];
  std::vector<int> gof(Bs, -1);
  std::vector<uint32_t> sdig(G, 0);
  for (long long i = 0; i < Bs; ++i) {
    if (rank[i] < 0) continue;
    const int g = off[tsum[i]] + rank[i];
    gof[i] = g;
    uint32_t w = 0;
    for (int k = h; k < N; ++k) w |= (uint32_t)sdg[i][k] << lbit[k];
    sdig[g] = w;
  }
  std::vector<long long> sidx(G);
  for (long long i = 0; i < Bs; ++i)
    if (gof[i] >= 0) sidx[gof[i]] = i;
  // blocks
  std::vector<long long> start(nblk, 0);
  std::vector<int> vb;
  long long run = 0;
  for (long long b = 0; b < nblk; ++b) {
    int P = 0;
    for (int k = 0; k < h; ++k) P += (int)((b / mp[k]) % p->sites[k].dim);
    start[b] = run;
    const long long t = K - P;
    if (t >= 0 && t <= K && cnt[t] > 0) {
      vb.push_back((int)b);
      run += cnt[t];
    }
  }
  // channels
  std::vector<KSBChan> ch;
  std::vector<double> tab;
  std::vector<double> dS(G, p->constant);
  std::vector<std::vector<std::pair<int, double>>> ell(G);
  std::vector<std::vector<int>> xr;
  std::map<std::pair<int, int>, int> xr_id;
  for (const Channel& c : p->chH) {
    bool nz = false;
    for (auto& z : c.T) nz = nz || z != std::complex<double>(0, 0);
    if (!nz) continue;
    const int si = c.i, sj = c.j;
    const int qi = c.qi, qj = sj >= 0 ? c.qj : 0;
    const bool diag = qi == 0 && qj == 0;
    const bool pi = si < h, pj = sj >= 0 && sj < h;
    const bool single = sj < 0;
    auto T = [&](int ni, int nj) { return c.T[(size_t)ni * c.dj + nj].real(); };
    if ((single && !pi) || (!single && !pi && !pj)) {  // suffix only
      for (int g = 0; g < G; ++g) {
        const std::vector<int>& s = sdg[sidx[g]];
        const int ni = s[si], nj = single ? 0 : s[sj];
        const double v = T(ni, nj);
        if (v == 0.0) continue;
        if (diag) {
          dS[g] += v;
        } else {
          const long long i2 = sidx[g] - (long long)qi * Ms[si] - (long long)qj * Ms[sj];
          ell[g].push_back({gof[i2] - g, v});   // same suffix sum: same sector
        }
      }
      continue;
    }
    KSBChan k{};
    k.tab = (int)tab.size();
    k.dj = c.dj;
    k.si = si;
    k.sj = sj;
    for (auto& z : c.T) tab.push_back(z.real());
    if (single || (pi && pj)) {  // prefix only
      k.kind = diag ? SB_PDIAG : SB_PMOVE;
      if (!diag) k.dblk = (long long)qi * mp[si] + (long long)qj * mp[sj];
    } else {                     // one prefix site, one suffix site
      k.pfx = pi ? 0 : 1;
      const int l = pi ? sj : si;
      const int ql = pi ? qj : qi;
      k.lbit = lbit[l];
      k.lwid = lwid[l];
      k.kind = diag ? SB_MDIAG : SB_MMOVE;
      if (!diag) {
        const int ps = pi ? si : sj;
        k.qp = pi ? qi : qj;
        k.dblk = (long long)k.qp * mp[ps];
        auto key = std::make_pair(l, ql);
        auto it = xr_id.find(key);
        if (it == xr_id.end()) {
          std::vector<int> tb(G, -1);
          for (int g = 0; g < G; ++g) {
            const std::vector<int>& s = sdg[sidx[g]];
            const int ns = s[l] - ql;
            if (ns < 0 || ns >= p->sites[l].dim) continue;
            const long long i2 = sidx[g] - (long long)ql * Ms[l];
            const int t2 = tsum[i2];
            if (t2 > K || gof[i2] < 0) continue;
            tb[g] = gof[i2] - off[t2];
          }
          it = xr_id.emplace(key, (int)xr.size()).first;
          xr.push_back(std::move(tb));
        }
        k.xr = it->second;
      }
    }
    ch.push_back(k);
  }
  if ((int)ch.size() > kSBChMax) return HM_OK;
  // kind order: prefix diagonal, prefix moves, coupled diagonal, coupled moves
  std::stable_sort(ch.begin(), ch.end(), [](const KSBChan& a, const KSBChan& b) {
    auto rank = [](int k) { return k == SB_PDIAG ? 0 : k == SB_PMOVE ? 1 : k == SB_MDIAG ? 2 : 3; };
    return rank(a.kind) < rank(b.kind);
  });
  int nk[4] = {0, 0, 0, 0};
  for (auto& c : ch) ++nk[c.kind == SB_PDIAG ? 0 : c.kind == SB_PMOVE ? 1 : c.kind == SB_MDIAG ? 2 : 3];
  int w = 0;
  for (auto& e : ell) w = std::max(w, (int)e.size());
  std::vector<int> ell_r((size_t)w * G, 0);
  std::vector<double> ell_d((size_t)w * G, 0.0);
  for (int g = 0; g < G; ++g)
    for (size_t e = 0; e < ell[g].size(); ++e) {
      ell_r[e * G + g] = ell[g][e].first;
      ell_d[e * G + g] = ell[g][e].second;
    }
  for (auto& v : xr) o.xr_flat.insert(o.xr_flat.end(), v.begin(), v.end());
  o.pdim.assign(std::max(h, 1), 1);
  for (int k = 0; k < h; ++k) o.pdim[k] = p->sites[k].dim;
  o.ok = true;
  o.h = h;
  o.w = w;
  o.G = G;
  o.n0 = nk[0];
  o.n1 = nk[0] + nk[1];
  o.n2 = nk[0] + nk[1] + nk[2];
  o.start = std::move(start);
  o.mp = std::move(mp);
  o.vb = std::move(vb);
  o.off = std::move(off);
  o.sdig = std::move(sdig);
  o.ch = std::move(ch);
  o.tab = std::move(tab);
  o.dS = std::move(dS);
  o.ell_r = std::move(ell_r);
  o.ell_d = std::move(ell_d);
  return HM_OK;
}

int build_sector_blk(Plan* p) {
  free_sector_blk(p);
  SBHost o;
  int rc = derive_sector_blk(p, p->sec_total, o);
  if (rc || !o.ok) return rc;
  long long cover = 0;
  for (size_t i = 0; i < o.vb.size(); ++i) {
    int P = 0;
    for (int k = 0; k < o.h; ++k) P += (int)((o.vb[i] / o.mp[k]) % o.pdim[k]);
    cover += o.off[o.K - P + 1] - o.off[o.K - P];
  }
  if (cover != p->Dsec) {
    set_error("internal: sector block form does not cover the sector");
    return HM_ERR_CUDA;
  }
  auto split = [](const std::vector<double>& v, std::vector<float2>& df, std::vector<float>& f) {
    for (double a : v) {
      const float hi = (float)a;
      df.push_back(make_float2(hi, (float)(a - (double)hi)));
      f.push_back(hi);
    }
  };
  std::vector<float2> tab_df, dS_df, ell_df;
  std::vector<float> tab_f, dS_f, ell_f;
  split(o.tab, tab_df, tab_f);
  split(o.dS, dS_df, dS_f);
  split(o.ell_d, ell_df, ell_f);
  struct Sec { const void* src; size_t bytes; size_t off; };
  std::vector<Sec> secs;
  size_t cur = 0;
  auto add = [&](const void* src, size_t bytes) {
    cur = (cur + 255) & ~size_t(255);
    secs.push_back({src, bytes, cur});
    const size_t o = cur;
    cur += std::max<size_t>(bytes, 1);
    return o;
  };
  const size_t o_start = add(o.start.data(), o.start.size() * 8);
  const size_t o_vb = add(o.vb.data(), o.vb.size() * 4);
  const size_t o_mp = add(o.mp.data(), o.mp.size() * 8);
  const size_t o_pd = add(o.pdim.data(), o.pdim.size() * 4);
  const size_t o_off = add(o.off.data(), o.off.size() * 4);
  const size_t o_sdig = add(o.sdig.data(), o.sdig.size() * 4);
  const size_t o_ch = add(o.ch.data(), o.ch.size() * sizeof(KSBChan));
  const size_t o_td = add(o.tab.data(), o.tab.size() * 8);
  const size_t o_tdf = add(tab_df.data(), tab_df.size() * 8);
  const size_t o_tf = add(tab_f.data(), tab_f.size() * 4);
  const size_t o_sd = add(o.dS.data(), o.dS.size() * 8);
  const size_t o_sdf = add(dS_df.data(), dS_df.size() * 8);
  const size_t o_sf = add(dS_f.data(), dS_f.size() * 4);
  const size_t o_er = add(o.ell_r.data(), o.ell_r.size() * 4);
  const size_t o_ed = add(o.ell_d.data(), o.ell_d.size() * 8);
  const size_t o_edf = add(ell_df.data(), ell_df.size() * 8);
  const size_t o_ef = add(ell_f.data(), ell_f.size() * 4);
  const size_t o_xr = add(o.xr_flat.data(), o.xr_flat.size() * 4);
  const size_t total = (cur + 255) & ~size_t(255);
  std::vector<unsigned char> host(total, 0);
  for (auto& sc : secs)
    if (sc.bytes) std::memcpy(host.data() + sc.off, sc.src, sc.bytes);
  cudaError_t e = cudaMalloc(&p->secb_dev, total);
  if (e != cudaSuccess) {
    p->secb_dev = nullptr;
    cudaGetLastError();
    return HM_OK;  // no room: the per-row kernel serves
  }
  e = cudaMemcpy(p->secb_dev, host.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "sector block table upload");
  const unsigned char* b = (const unsigned char*)p->secb_dev;
  KSecBlk& S = p->ksb;
  S = KSecBlk{};
  S.nvb = (long long)o.vb.size();
  S.h = o.h;
  S.K = (int)o.K;
  S.nch = (int)o.ch.size();
  S.n0 = o.n0;
  S.n1 = o.n1;
  S.n2 = o.n2;
  S.w = o.w;
  S.G = o.G;
  S.start = (const long long*)(b + o_start);
  S.vb = (const int*)(b + o_vb);
  S.mp = (const long long*)(b + o_mp);
  S.pdim = (const int*)(b + o_pd);
  S.off = (const int*)(b + o_off);
  S.sdig = (const uint32_t*)(b + o_sdig);
  S.ch = (const KSBChan*)(b + o_ch);
  S.tab_d = (const double*)(b + o_td);
  S.tab_df = (const float2*)(b + o_tdf);
  S.tab_f = (const float*)(b + o_tf);
  S.dS_d = (const double*)(b + o_sd);
  S.dS_df = (const float2*)(b + o_sdf);
  S.dS_f = (const float*)(b + o_sf);
  S.ell_r = (const int*)(b + o_er);
  S.ell_d = (const double*)(b + o_ed);
  S.ell_df = (const float2*)(b + o_edf);
  S.ell_f = (const float*)(b + o_ef);
  S.xr = (const int*)(b + o_xr);
  p->secb_ok = true;
  return HM_OK;
}

// The host tables of the block form with digit total K as JSON text
// ("ok": false when the plan does not fit the block form).
std::string export_sector_blk_json(const Plan* p, long long K, int* rc) {
  SBHost o;
  *rc = derive_sector_blk(p, K, o);
  if (*rc) return std::string();
  std::string s = std::string("{\"ok\":") + (o.ok ? "true" : "false");
  auto num = [&](double v) {
    char b[40];
    snprintf(b, sizeof(b), "%.17g", v);
    s += b;
  };
  auto arr = [&](const char* name, size_t n, auto f) {
    s += ",\"";
    s += name;
    s += "\":[";
    for (size_t i = 0; i < n; ++i) {
      if (i) s += ",";
      f(i);
    }
    s += "]";
  };
  s += ",\"h\":" + std::to_string(o.h) + ",\"K\":" + std::to_string(o.K) + ",\"w\":" + std::to_string(o.w) +
       ",\"G\":" + std::to_string(o.G) + ",\"n0\":" + std::to_string(o.n0) + ",\"n1\":" + std::to_string(o.n1) +
       ",\"n2\":" + std::to_string(o.n2);
  arr("start", o.start.size(), [&](size_t i) { s += std::to_string(o.start[i]); });
  arr("vb", o.vb.size(), [&](size_t i) { s += std::to_string(o.vb[i]); });
  arr("mp", o.mp.size(), [&](size_t i) { s += std::to_string(o.mp[i]); });
  arr("pdim", o.pdim.size(), [&](size_t i) { s += std::to_string(o.pdim[i]); });
  arr("off", o.off.size(), [&](size_t i) { s += std::to_string(o.off[i]); });
  arr("sdig", o.sdig.size(), [&](size_t i) { s += std::to_string(o.sdig[i]); });
  arr("ch", o.ch.size(), [&](size_t i) {
    const KSBChan& c = o.ch[i];
    s += "[" + std::to_string(c.kind) + "," + std::to_string(c.tab) + "," + std::to_string(c.dj) + "," +
         std::to_string(c.si) + "," + std::to_string(c.sj) + "," + std::to_string(c.pfx) + "," + std::to_string(c.qp) +
         "," + std::to_string(c.xr) + "," + std::to_string(c.dblk) + "," + std::to_string(c.lbit) + "," +
         std::to_string(c.lwid) + "]";
  });
  arr("tab", o.tab.size(), [&](size_t i) { num(o.tab[i]); });
  arr("dS", o.dS.size(), [&](size_t i) { num(o.dS[i]); });
  arr("ell_r", o.ell_r.size(), [&](size_t i) { s += std::to_string(o.ell_r[i]); });
  arr("ell", o.ell_d.size(), [&](size_t i) { num(o.ell_d[i]); });
  arr("xr", o.xr_flat.size(), [&](size_t i) { s += std::to_string(o.xr_flat[i]); });
  s += "}";
  return s;
}

void free_sector_blk(Plan* p) {
  if (p->secb_dev) cudaFree(p->secb_dev);
  p->secb_dev = nullptr;
  p->secb_ok = false;
}

template <int AR>
static cudaError_t sector_blk_t(const Plan* p, const void* x, void* y, long long nvec, cudaStream_t s) {
  using P = SBAr<AR>;
  const KSecBlk& S = p->ksb;
  const long long grid = std::max<long long>(1, std::min<long long>(S.nvb, (long long)num_sms() * 8));
  if (nvec == 1)
    k_sector_blk<AR, 1><<<(unsigned)grid, kSBNT, 0, s>>>(S, (const typename P::TX*)x, (typename P::TY*)y, 1);
  else
    k_sector_blk<AR, 0><<<(unsigned)grid, kSBNT, 0, s>>>(S, (const typename P::TX*)x, (typename P::TY*)y,
                                                         (int)nvec);
  return cudaGetLastError();
}

// x already split into float pairs for FP64 storage
cudaError_t launch_sector_blk(const Plan* p, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s) {
  return dt == HM_F32 ? sector_blk_t<AR_F32>(p, x, y, nvec, s) : sector_blk_t<AR_DF64>(p, x, y, nvec, s);
}

}  // namespace hm
