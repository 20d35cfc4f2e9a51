// y = H x inside a fixed digit-sum sector (Sec. VI case 2; App. D): the
// retained states are the digit tuples with sum_k n_k = K (a fixed total
// magnetization for spins, a fixed excitation number for spin-boson models),
// stored packed in ascending full-index order. Pull form (Sec. II): one
// thread per packed target row F:
//   1. unpack F to its digits by combinatorial unranking (count tables);
//   2. for every channel, the target-digit coefficient table gives the
//      matrix element, zero for an inadmissible source digit (Sec. IV.B);
//   3. the source's packed index is the lookup of Sec. VI, done as a rank
//      update: a move on sites i < j changes only the rank terms of sites
//      i..j (KSector), so the lookup costs O(j - i + 1) table reads and
//      cannot fail for a channel that conserves the digit sum; for adjacent
//      sites the update depends on (digits total left before i, n_i, n_j)
//      alone and is tabulated when the plan is built (one read);
//   4. y_F accumulates coefficient * x[source] (App. D step 4).
// Arithmetic as in the full-basis kernel (FP32, or double-float for FP64
// storage). Channels that do not conserve the digit sum are rejected when the plan is
// built (their sources lie outside the sector, so the projected operator
// would silently drop them).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "device_common.cuh"

namespace hm {

constexpr int kSecNT = 256;
constexpr size_t kSecTablesMax = 96 * 1024;  // tables staged in shared memory up to this size
constexpr size_t kSecDeltaMax = 48 * 1024;   // rank-delta tables of adjacent-site moves up to this size
constexpr size_t kSecLongMax = 32 * 1024;    // long-move tables up to this size

// Table pointers of one launch (shared-memory copies, or the global tables).
template <class C, class DT>
struct SecTabs {
  const int* d;
  const long long* cnt;
  const long long* A;
  const int* Aoff;
  const KSecChan* ch;
  const C* tab;
  const DT* dl;
  const DT* lt;
};

__host__ __device__ inline size_t sec_align(size_t b) { return (b + 15) & ~size_t(15); }

// bytes of the staged tables (host and device agree on the layout); nA = 0
// when no channel reads the rank tables
__host__ __device__ inline size_t sec_tables_bytes(int N, int K, long long nA, int nch, long long ntab, size_t csize,
                                                   long long ndl, long long nlt, size_t dsize) {
  return sec_align((size_t)N * 4) + sec_align((size_t)(N + 1) * (K + 1) * 8) + sec_align((size_t)nA * 8) +
         sec_align((size_t)N * 4) + sec_align((size_t)nch * sizeof(KSecChan)) + sec_align((size_t)ntab * csize) +
         sec_align((size_t)ndl * dsize) + sec_align((size_t)nlt * dsize);
}

// Arithmetic of the sector kernel, as in the full-basis kernel: FP32 storage
// in FP32; FP64 storage as double-float sums on the FP32 pipe of the input
// split once into float pairs (GB300 runs FP64 at ~1/70 of the FP32 rate).
template <int AR> struct SecAr;
template <> struct SecAr<AR_F32> {
  using TX = float;
  using TY = float;
  using C = float;
  using Acc = float;
  __device__ static const C* tab(const KSector& S) { return S.tab_f; }
  __device__ static bool nz(C c) { return c != 0.0f; }
  __device__ static Acc zero() { return 0.0f; }
  __device__ static void add(Acc& a, C c) { a = __fadd_rn(a, c); }
  __device__ static void fma(Acc& a, C c, TX x) { a = __fmaf_rn(c, x, a); }
  __device__ static TY out(Acc hop, Acc d, TX xo) { return __fmaf_rn(d, xo, hop); }
};
template <> struct SecAr<AR_DF64> {
  using TX = float2;
  using TY = double;
  using C = float2;
  using Acc = DF;
  __device__ static const C* tab(const KSector& S) { return S.tab_df; }
  __device__ static bool nz(C c) { return c.x != 0.0f; }
  __device__ static Acc zero() { return DF{0.f, 0.f}; }
  __device__ static void add(Acc& a, C c) { df_add(a, c); }
  __device__ static void fma(Acc& a, C c, TX x) { df_fma(a, c, x.x, x.y); }
  __device__ static TY out(Acc hop, Acc d, TX xo) {
    df_fma(hop, df_norm(d), xo.x, xo.y);
    return df_to_double(hop);
  }
};

// Per thread and site, the target's digit and the digit total left before
// that site, packed in 16 bits (both are at most K <= 255).
__device__ __forceinline__ int sec_digit(unsigned w) { return (int)(w & 0xffu); }
__device__ __forceinline__ int sec_rem(unsigned w) { return (int)(w >> 8); }

// The kernel body over one set of table pointers (shared-memory copies when
// STAGED, so every table read is a 32-bit-addressed shared load).
// NV: right-hand sides per pass, fixed (1) or up to 8 chosen at run time (0).
template <int AR, class DT, int NV>
__device__ __forceinline__ void sector_rows(const KSector& S, const SecTabs<typename SecAr<AR>::C, DT>& G,
                                            unsigned short* dr, const typename SecAr<AR>::TX* __restrict__ x,
                                            typename SecAr<AR>::TY* __restrict__ y, int nvec) {
  using P = SecAr<AR>;
  using C = typename P::C;
  using TX = typename P::TX;
  const int N = S.N, K1 = S.K + 1, nch = S.nch, ndiag = S.ndiag;
  const int t = threadIdx.x;
  // row index of a state (32-bit when the sector has fewer than 2^31 states)
  auto at = [&](DT row, int v0) -> size_t {
    const size_t r = sizeof(DT) == 4 ? (size_t)(unsigned)row : (size_t)row;
    return NV == 1 ? r : r * (size_t)nvec + v0;
  };
  auto Aat = [&](int k, int tt, int n) { return G.A[G.Aoff[k] + tt * (G.d[k] + 1) + n]; };
  for (long long F = blockIdx.x * (long long)kSecNT + t; F < S.Dsec; F += (long long)gridDim.x * kSecNT) {
    // 1. unrank: digit m at site k is the first whose block of states
    // (cnt_{k+1}[left - m] of them) holds the remaining rank r; the last
    // admissible digit needs no test. Every count met on the way is at most
    // Dsec, so DT (32-bit below 2^31 states) holds it.
    DT r = (DT)F;
    int left = S.K;
    for (int k = 0; k < N; ++k) {
      const long long* c = G.cnt + (k + 1) * K1;
      const int dk = G.d[k];
      int m = 0;
      while (m + 1 < dk && left - m >= 0) {
        const DT cm = (DT)c[left - m];
        if (r < cm) break;
        r -= cm;
        ++m;
      }
      dr[k * kSecNT + t] = (unsigned short)(m | (left << 8));
      left -= m;
    }
    // 2.-4. channels, up to 8 right-hand sides per pass: first the diagonal
    // ones (their coefficients are summed and multiply x_F once), then the
    // moves
    const DT Fd = (DT)F;
    for (int v0 = 0; v0 < nvec; v0 += (NV ? NV : 8)) {
      const int nv = NV ? NV : min(8, nvec - v0);
      typename P::Acc acc[8];
      for (int v = 0; v < nv; ++v) acc[v] = P::zero();
      typename P::Acc dsum = P::zero();
      for (int c = 0; c < ndiag; ++c) {
        const KSecChan ch = G.ch[c];
        const int ni = sec_digit(dr[ch.si * kSecNT + t]);
        const int nj = ch.sj >= 0 ? sec_digit(dr[ch.sj * kSecNT + t]) : 0;
        P::add(dsum, G.tab[ch.tab + ni * ch.dj + nj]);
      }
      for (int c = ndiag; c < nch; ++c) {
        const KSecChan ch = G.ch[c];
        const unsigned wi = dr[ch.si * kSecNT + t];
        const int ni = sec_digit(wi);
        const int nj = sec_digit(dr[ch.sj * kSecNT + t]);   // moves span two sites
        const int ci = ni * ch.dj + nj;
        const C cf = G.tab[ch.tab + ci];
        if (!P::nz(cf)) continue;
        // rank terms of sites si..sj, target and source (sj > si)
        DT dlt;
        if (ch.dtab >= 0) {  // adjacent sites: one table entry
          dlt = G.dl[ch.dtab + sec_rem(wi) * ch.rstride + ci];
        } else if (ch.dtab <= -2) {  // long move: one entry per site si..sj
          const DT* T = G.lt + (-2 - ch.dtab);
          dlt = 0;
          for (int k = ch.si; k <= ch.sj; ++k) {
            const unsigned wk = dr[k * kSecNT + t];
            dlt += T[((k - ch.si) * K1 + sec_rem(wk)) * ch.rstride + sec_digit(wk)];
          }
        } else {
          const int i = ch.si, j = ch.sj, q = ch.q;
          const int ri = sec_rem(wi);
          long long d = Aat(i, ri, ni - q) - Aat(i, ri, ni);
          for (int k = i + 1; k < j; ++k) {
            const unsigned wk = dr[k * kSecNT + t];
            const int rk = sec_rem(wk), nk = sec_digit(wk);
            d += Aat(k, rk + q, nk) - Aat(k, rk, nk);
          }
          const int rj = sec_rem(dr[j * kSecNT + t]);
          d += Aat(j, rj + q, nj + q) - Aat(j, rj, nj);
          dlt = (DT)d;
        }
        const TX* xs = x + at(Fd + dlt, v0);
        for (int v = 0; v < nv; ++v) P::fma(acc[v], cf, xs[v]);
      }
      const TX* xo = x + at(Fd, v0);
      typename P::TY* ys = y + at(Fd, v0);
      for (int v = 0; v < nv; ++v) ys[v] = P::out(acc[v], dsum, xo[v]);
    }
  }
}

template <int AR, class DT, int NV, bool STAGED>
__global__ void __launch_bounds__(kSecNT) k_sector(const KSector S, const typename SecAr<AR>::TX* __restrict__ x,
                                                   typename SecAr<AR>::TY* __restrict__ y, int nvec, long long nA,
                                                   long long ntab, long long ndl, long long nlt) {
  using P = SecAr<AR>;
  using C = typename P::C;
  extern __shared__ __align__(16) unsigned char ssm[];
  const int N = S.N, K1 = S.K + 1;
  if constexpr (STAGED) {  // copy the tables once per CTA
    size_t o = 0;
    int* d = (int*)(ssm + o);               o += sec_align((size_t)N * 4);
    long long* cnt = (long long*)(ssm + o); o += sec_align((size_t)(N + 1) * K1 * 8);
    long long* A = (long long*)(ssm + o);   o += sec_align((size_t)nA * 8);
    int* Aoff = (int*)(ssm + o);            o += sec_align((size_t)N * 4);
    KSecChan* ch = (KSecChan*)(ssm + o);    o += sec_align((size_t)S.nch * sizeof(KSecChan));
    C* tab = (C*)(ssm + o);                 o += sec_align((size_t)ntab * sizeof(C));
    DT* dl = (DT*)(ssm + o);                o += sec_align((size_t)ndl * sizeof(DT));
    DT* lt = (DT*)(ssm + o);                o += sec_align((size_t)nlt * sizeof(DT));
    for (int i = threadIdx.x; i < N; i += kSecNT) { d[i] = S.d[i]; Aoff[i] = S.Aoff[i]; }
    for (int i = threadIdx.x; i < (N + 1) * K1; i += kSecNT) cnt[i] = S.cnt[i];
    for (long long i = threadIdx.x; i < nA; i += kSecNT) A[i] = S.A[i];
    for (int i = threadIdx.x; i < S.nch; i += kSecNT) ch[i] = S.ch[i];
    for (long long i = threadIdx.x; i < ntab; i += kSecNT) tab[i] = P::tab(S)[i];
    for (long long i = threadIdx.x; i < ndl; i += kSecNT) dl[i] = ((const DT*)S.dl)[i];
    for (long long i = threadIdx.x; i < nlt; i += kSecNT) lt[i] = ((const DT*)S.lt)[i];
    __syncthreads();
    // nA = 0: no channel reads the rank tables
    const SecTabs<C, DT> G{d, cnt, A, Aoff, ch, tab, dl, lt};
    sector_rows<AR, DT, NV>(S, G, (unsigned short*)(ssm + o), x, y, nvec);
  } else {
    const SecTabs<C, DT> G{S.d, S.cnt, S.A, S.Aoff, S.ch, P::tab(S), (const DT*)S.dl, (const DT*)S.lt};
    sector_rows<AR, DT, NV>(S, G, (unsigned short*)ssm, x, y, nvec);
  }
}

void free_sector(Plan* p) {
  if (p->sec_dev) cudaFree(p->sec_dev);
  p->sec_dev = nullptr;
  p->ksec = KSector{};
  free_sector_blk(p);
}

// Host half of a sector plan: counts, rank tables, channels, rank-delta
// tables (also the plan export's source, so it touches no GPU).
struct SecHost {
  long long Dsec = 0;
  int K = 0, ndiag = 0;
  bool wide = false, needA = false;
  std::vector<int> dims, Aoff;
  std::vector<long long> cnt, A, dl, lt;
  std::vector<KSecChan> ch;
  std::vector<double> tab;
};

static int derive_sector(const Plan* p, long long Kl, SecHost& out) {
  const int N = p->N;
  long long maxsum = 0;
  for (auto& st : p->sites) maxsum += st.dim - 1;
  if (Kl < 0 || Kl > maxsum) {
    set_error("digit total outside [0, sum_k (d_k - 1)]: the sector is empty");
    return HM_ERR_INVALID_ARG;
  }
  if (Kl > 255) {
    set_error("sector digit totals above 255 are not supported");
    return HM_ERR_UNSUPPORTED;
  }
  const int K = (int)Kl, K1 = K + 1;
  // counts, with an overflow guard (Dsec < 2^62)
  std::vector<long long> cnt((size_t)(N + 1) * K1, 0);
  cnt[(size_t)N * K1 + 0] = 1;
  const long long lim = (1LL << 62);
  for (int k = N - 1; k >= 0; --k)
    for (int t = 0; t <= K; ++t) {
      long long s = 0;
      for (int m = 0; m < p->sites[k].dim && m <= t; ++m) {
        s += cnt[(size_t)(k + 1) * K1 + t - m];
        if (s >= lim) {
          set_error("sector dimension must be below 2^62");
          return HM_ERR_OVERFLOW;
        }
      }
      cnt[(size_t)k * K1 + t] = s;
    }
  const long long Dsec = cnt[K];
  std::vector<int>& dims = out.dims;
  std::vector<int>& Aoff = out.Aoff;
  std::vector<long long>& A = out.A;
  dims.assign(N, 0);
  Aoff.assign(N, 0);
  A.clear();
  for (int k = 0; k < N; ++k) {
    // a digit above K cannot occur in the sector: the rank tables stop at K + 1
    dims[k] = std::min(p->sites[k].dim, K + 1);
    Aoff[k] = (int)A.size();
    for (int t = 0; t <= K; ++t)
      for (int n = 0; n <= dims[k]; ++n) {
        long long s = 0;
        for (int m = 0; m < n; ++m)
          if (t - m >= 0) s += cnt[(size_t)(k + 1) * K1 + t - m];
        A.push_back(s);
      }
  }
  // channels: every merged channel must conserve the digit sum
  struct HC {
    int si, sj, qi, qj, dj;
    std::vector<double> T;  // [n_i * dj + n_j], target digits
  };
  std::vector<HC> hc;
  for (const Channel& c : p->chH) {
    bool nz = false;
    for (auto& z : c.T) nz = nz || z != std::complex<double>(0, 0);
    if (!nz) continue;
    if (c.qi + (c.j >= 0 ? c.qj : 0) != 0) {
      set_error("the term list does not conserve the sector's digit sum (a channel moves it by " +
                std::to_string(c.qi + (c.j >= 0 ? c.qj : 0)) + ")");
      return HM_ERR_UNSUPPORTED;
    }
    HC h{c.i, c.j >= 0 ? c.j : -1, c.qi, c.j >= 0 ? c.qj : 0, c.dj, {}};
    for (auto& z : c.T) h.T.push_back(z.real());
    hc.push_back(std::move(h));
  }
  if (p->constant != 0.0)  // identity terms: a diagonal channel on site 0
    hc.push_back(HC{0, -1, 0, 0, 1, std::vector<double>(p->sites[0].dim, p->constant)});
  // Diagonal channels only add to the row's diagonal element: a single-site
  // one is folded into a two-site diagonal table on its site, and the rest
  // are paired into two-site tables (fewer channels per row, same sums).
  auto is_diag = [](const HC& h) { return h.qi == 0 && h.qj == 0; };
  std::vector<bool> gone(hc.size(), false);
  for (size_t a = 0; a < hc.size(); ++a) {
    if (!is_diag(hc[a]) || hc[a].sj >= 0) continue;
    for (size_t b = 0; b < hc.size(); ++b) {
      HC& t = hc[b];
      if (b == a || gone[b] || !is_diag(t) || t.sj < 0 || (t.si != hc[a].si && t.sj != hc[a].si)) continue;
      const int di = (int)t.T.size() / t.dj;
      for (int ni = 0; ni < di; ++ni)
        for (int nj = 0; nj < t.dj; ++nj) t.T[(size_t)ni * t.dj + nj] += hc[a].T[t.si == hc[a].si ? ni : nj];
      gone[a] = true;
      break;
    }
  }
  int lone = -1;
  for (size_t a = 0; a < hc.size(); ++a) {
    if (gone[a] || !is_diag(hc[a]) || hc[a].sj >= 0) continue;
    if (lone < 0 || hc[lone].si == hc[a].si) {
      if (lone >= 0) {  // same site: sum the tables
        for (size_t n = 0; n < hc[a].T.size(); ++n) hc[lone].T[n] += hc[a].T[n];
        gone[a] = true;
      } else {
        lone = (int)a;
      }
      continue;
    }
    HC& u = hc[lone];
    const HC& w = hc[a];
    const int si = std::min(u.si, w.si), sj = std::max(u.si, w.si);
    const std::vector<double>& Ti = u.si == si ? u.T : w.T;
    const std::vector<double>& Tj = u.si == si ? w.T : u.T;
    HC m{si, sj, 0, 0, (int)Tj.size(), {}};
    for (size_t ni = 0; ni < Ti.size(); ++ni)
      for (size_t nj = 0; nj < Tj.size(); ++nj) m.T.push_back(Ti[ni] + Tj[nj]);
    u = std::move(m);
    gone[a] = true;
    lone = -1;
  }
  // rank-delta tables of moves on adjacent sites, within a shared-memory budget
  const bool wide = Dsec > 0x7fffffffLL;
  const size_t dsize = wide ? 8 : 4;
  auto Ah = [&](int k, int t, int n) {
    long long s = 0;
    for (int m = 0; m < n && m <= t; ++m) s += cnt[(size_t)(k + 1) * K1 + t - m];
    return s;
  };
  std::vector<KSecChan>& ch = out.ch;
  std::vector<double>& tab = out.tab;
  std::vector<long long>& dl = out.dl;
  std::vector<long long>& lt = out.lt;
  ch.clear();
  tab.clear();
  dl.clear();
  lt.clear();
  bool needA = false;
  // diagonal channels first (the kernel sums them in a loop of their own)
  std::vector<size_t> order;
  for (int pass = 0; pass < 2; ++pass)
    for (size_t a = 0; a < hc.size(); ++a)
      if (!gone[a] && (is_diag(hc[a]) == (pass == 0))) order.push_back(a);
  int ndiag = 0;
  for (size_t a : order) {
    const HC& h = hc[a];
    if (is_diag(h)) ++ndiag;
    const int di = (int)h.T.size() / h.dj;
    KSecChan k{};
    k.tab = (int)tab.size();
    k.dtab = -1;
    k.dj = h.dj;
    k.rstride = di * h.dj;
    k.si = h.si;
    k.sj = h.sj;
    k.q = h.qi;
    k.diag = is_diag(h) ? 1 : 0;
    for (double v : h.T) tab.push_back(v);
    if (!k.diag) {
      const size_t n = (size_t)K1 * k.rstride;
      if (h.sj == h.si + 1 && (dl.size() + n) * dsize <= kSecDeltaMax) {
        k.dtab = (int)dl.size();
        const int i = h.si, j = h.sj, q = h.qi;
        for (int ri = 0; ri <= K; ++ri)
          for (int ni = 0; ni < di; ++ni)
            for (int nj = 0; nj < h.dj; ++nj) {
              // target digits (ni, nj), source (ni - q, nj + q); totals left
              // before j: ri - ni (target), ri - ni + q (source)
              const int si = ni - q, sj = nj + q, rj = ri - ni;
              long long v = 0;
              if (ni <= ri && nj <= rj && si >= 0 && si < di && sj >= 0 && sj < h.dj && rj + q >= 0 && rj + q <= K)
                v = Ah(i, ri, si) - Ah(i, ri, ni) + Ah(j, rj + q, sj) - Ah(j, rj, nj);
              dl.push_back(v);
            }
      } else if (h.sj > h.si + 1) {
        // long move: per-site entries over sites i..j
        const int i = h.si, j = h.sj, q = h.qi;
        int dm = 1;
        for (int kk = i; kk <= j; ++kk) dm = std::max(dm, dims[kk]);
        const size_t nl = (size_t)(j - i + 1) * K1 * dm;
        if ((lt.size() + nl) * dsize > kSecLongMax) {
          needA = true;
        } else {
          k.dtab = -2 - (int)lt.size();
          k.rstride = dm;
          const size_t off = lt.size();
          lt.resize(off + nl, 0);
          for (int kk = i; kk <= j; ++kk) {
            const int dfull = p->sites[kk].dim;
            for (int r = 0; r <= K; ++r)
              for (int n = 0; n < dims[kk]; ++n) {
                long long v = 0;
                if (kk == i) {           // target digit n, source n - q
                  if (n - q >= 0 && n - q < dfull) v = Ah(kk, r, n - q) - Ah(kk, r, n);
                } else if (kk < j) {     // digit kept, total left shifted by q
                  if (r + q >= 0 && r + q <= K) v = Ah(kk, r + q, n) - Ah(kk, r, n);
                } else {                 // target digit n, source n + q
                  if (r + q >= 0 && r + q <= K && n + q >= 0 && n + q < dfull)
                    v = Ah(kk, r + q, n + q) - Ah(kk, r, n);
                }
                lt[off + ((size_t)(kk - i) * K1 + r) * dm + n] = v;
              }
          }
        }
      } else {
        needA = true;
      }
    }
    ch.push_back(k);
  }
  out.Dsec = Dsec;
  out.ndiag = ndiag;
  out.K = K;
  out.wide = wide;
  out.needA = needA;
  out.cnt = std::move(cnt);
  return HM_OK;
}

int build_sector(Plan* p) {
  SecHost h;
  int rc = derive_sector(p, p->sec_total, h);
  if (rc) return rc;
  const int N = p->N;
  std::vector<float> tabf;
  std::vector<float2> tabdf;
  for (double v : h.tab) {
    const float hi = (float)v;
    tabf.push_back(hi);
    tabdf.push_back(make_float2(hi, (float)(v - (double)hi)));
  }
  std::vector<int32_t> dl32, lt32;
  if (!h.wide) {
    for (long long v : h.dl) dl32.push_back((int32_t)v);
    for (long long v : h.lt) lt32.push_back((int32_t)v);
  }
  // upload
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
  const size_t o_d = add(h.dims.data(), h.dims.size() * 4);
  const size_t o_cnt = add(h.cnt.data(), h.cnt.size() * 8);
  const size_t o_A = add(h.A.data(), h.A.size() * 8);
  const size_t o_Aoff = add(h.Aoff.data(), h.Aoff.size() * 4);
  const size_t o_ch = add(h.ch.data(), h.ch.size() * sizeof(KSecChan));
  const size_t o_tab = add(h.tab.data(), h.tab.size() * 8);
  const size_t o_tabf = add(tabf.data(), tabf.size() * 4);
  const size_t o_tabdf = add(tabdf.data(), tabdf.size() * 8);
  const size_t o_dl = h.wide ? add(h.dl.data(), h.dl.size() * 8) : add(dl32.data(), dl32.size() * 4);
  const size_t o_lt = h.wide ? add(h.lt.data(), h.lt.size() * 8) : add(lt32.data(), lt32.size() * 4);
  const size_t total = (cur + 255) & ~size_t(255);
  std::vector<unsigned char> host(total, 0);
  for (auto& sc : secs)
    if (sc.bytes) std::memcpy(host.data() + sc.off, sc.src, sc.bytes);
  free_sector(p);
  cudaError_t e = cudaMalloc(&p->sec_dev, total);
  if (e != cudaSuccess) {
    p->sec_dev = nullptr;
    return cuda_fail(e, "sector tables");
  }
  e = cudaMemcpy(p->sec_dev, host.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "sector table upload");
  const unsigned char* b = (const unsigned char*)p->sec_dev;
  KSector& S = p->ksec;
  S.Dsec = h.Dsec;
  S.N = N;
  S.K = h.K;
  S.nch = (int)h.ch.size();
  S.ndiag = h.ndiag;
  S.d = (const int*)(b + o_d);
  S.cnt = (const long long*)(b + o_cnt);
  S.A = (const long long*)(b + o_A);
  S.Aoff = (const int*)(b + o_Aoff);
  S.ch = (const KSecChan*)(b + o_ch);
  S.tab_d = (const double*)(b + o_tab);
  S.tab_f = (const float*)(b + o_tabf);
  S.tab_df = (const float2*)(b + o_tabdf);
  S.dl = b + o_dl;
  S.lt = b + o_lt;
  S.nlt = (long long)h.lt.size();
  S.wide = h.wide ? 1 : 0;
  p->Dsec = h.Dsec;
  p->sec_nA = (long long)h.A.size();
  p->sec_ntab = (long long)h.tab.size();
  p->sec_ndl = (long long)h.dl.size();
  p->sec_needA = h.needA;
  return build_sector_blk(p);
}

// The host tables of the sector plan with digit total Kl as JSON text.
std::string export_sector_json(const Plan* p, long long Kl, int* rc) {
  SecHost h;
  *rc = derive_sector(p, Kl, h);
  if (*rc) return std::string();
  std::string o = "{\"Dsec\":" + std::to_string(h.Dsec) + ",\"K\":" + std::to_string(h.K) +
                  ",\"wide\":" + (h.wide ? "true" : "false") + ",\"needA\":" + (h.needA ? "true" : "false");
  auto arr = [&](const char* name, size_t n, auto f) {
    o += ",\"";
    o += name;
    o += "\":[";
    for (size_t i = 0; i < n; ++i) {
      if (i) o += ",";
      f(i);
    }
    o += "]";
  };
  auto num = [&](double v) {
    char b[40];
    snprintf(b, sizeof(b), "%.17g", v);
    o += b;
  };
  arr("d", h.dims.size(), [&](size_t i) { o += std::to_string(h.dims[i]); });
  arr("Aoff", h.Aoff.size(), [&](size_t i) { o += std::to_string(h.Aoff[i]); });
  arr("cnt", h.cnt.size(), [&](size_t i) { o += std::to_string(h.cnt[i]); });
  arr("A", h.A.size(), [&](size_t i) { o += std::to_string(h.A[i]); });
  arr("dl", h.dl.size(), [&](size_t i) { o += std::to_string(h.dl[i]); });
  arr("lt", h.lt.size(), [&](size_t i) { o += std::to_string(h.lt[i]); });
  arr("tab", h.tab.size(), [&](size_t i) { num(h.tab[i]); });
  arr("ch", h.ch.size(), [&](size_t i) {
    const KSecChan& k = h.ch[i];
    o += "[" + std::to_string(k.tab) + "," + std::to_string(k.dtab) + "," + std::to_string(k.rstride) + "," +
         std::to_string(k.dj) + "," + std::to_string(k.si) + "," + std::to_string(k.sj) + "," +
         std::to_string(k.q) + "," + std::to_string(k.sj >= 0 ? -k.q : 0) + "," + std::to_string(k.diag) + "]";
  });
  o += "}";
  return o;
}

template <int AR, class DT>
static cudaError_t sector_launch(Plan* p, const void* x, void* y, long long nvec, cudaStream_t s) {
  using P = SecAr<AR>;
  const KSector& S = p->ksec;
  const long long nA = p->sec_needA ? p->sec_nA : 0;
  const size_t tabs = sec_tables_bytes(S.N, S.K, nA, S.nch, p->sec_ntab, sizeof(typename P::C), p->sec_ndl,
                                      S.nlt, sizeof(DT));
  const int staged = tabs <= kSecTablesMax;
  const size_t smem = (staged ? tabs : 0) + (size_t)S.N * kSecNT * sizeof(unsigned short);
  auto kern = staged ? (nvec == 1 ? k_sector<AR, DT, 1, true> : k_sector<AR, DT, 0, true>)
                     : (nvec == 1 ? k_sector<AR, DT, 1, false> : k_sector<AR, DT, 0, false>);
  if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const long long need = (S.Dsec + kSecNT - 1) / kSecNT;
  const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)num_sms() * 8));
  kern<<<grid, kSecNT, smem, s>>>(S, (const typename P::TX*)x, (typename P::TY*)y, (int)nvec, nA, p->sec_ntab,
                                  p->sec_ndl, S.nlt);
  return cudaGetLastError();
}

template <int AR>
static cudaError_t sector_launch(Plan* p, const void* x, void* y, long long nvec, cudaStream_t s) {
  return p->ksec.wide ? sector_launch<AR, long long>(p, x, y, nvec, s) : sector_launch<AR, int>(p, x, y, nvec, s);
}

// The block form where the plan has it (rows = false), else the per-row kernel.
int launch_sector(Plan* p, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s, bool rows) {
  const bool blk = p->secb_ok && !rows;
  cudaError_t e;
  if (dt == HM_F32) {
    e = blk ? launch_sector_blk(p, x, y, nvec, dt, s) : sector_launch<AR_F32>(p, x, y, nvec, s);
  } else {  // FP64: split into float pairs first
    const float2* xs = nullptr;
    Scratch xsb;
    int rc = split_vector(x, p->Dsec * nvec, s, xsb, &xs);
    if (rc) return rc;
    e = blk ? launch_sector_blk(p, xs, y, nvec, dt, s) : sector_launch<AR_DF64>(p, xs, y, nvec, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "sector apply launch");
  return HM_OK;
}

}  // namespace hm
