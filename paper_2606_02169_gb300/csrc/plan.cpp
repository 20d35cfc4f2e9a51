// Plan builder: site list + term list -> the O(N + |terms| + B) tables the
// apply kernels read. Host code, runs once per Hamiltonian (and again on
// hm_set_coefficients). This is the "Setup" phase that the matrix-free form
// keeps small (Sec. V, Table I; operator memory O(N + |P|), Sec. V.A).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "hm_internal.h"

namespace hm {

using cplx = std::complex<double>;

// Local d x d matrix of a named operator in ascending local index n = m + s
// (Sec. II notation guide; App. C for bosons). mat[nt * d + ns].
static bool local_matrix(int kind, int d, int op, std::vector<cplx>& mat) {
  mat.assign((size_t)d * d, cplx(0, 0));
  auto at = [&](int nt, int ns) -> cplx& { return mat[(size_t)nt * d + ns]; };
  if (op == HM_ID) {
    for (int n = 0; n < d; ++n) at(n, n) = 1.0;
    return true;
  }
  if (kind == HM_SPIN) {
    const double s = 0.5 * (d - 1);
    std::vector<cplx> sp((size_t)d * d, 0.0), sm((size_t)d * d, 0.0);
    // <m+1| S+ |m> = sqrt(s(s+1) - m(m+1))   (Sec. IV.A raising rule)
    for (int n = 0; n + 1 < d; ++n) {
      double m = n - s;
      double v = std::sqrt(s * (s + 1.0) - m * (m + 1.0));
      sp[(size_t)(n + 1) * d + n] = v;
      sm[(size_t)n * d + (n + 1)] = v;  // S- = (S+)^T
    }
    auto mul = [&](const std::vector<cplx>& a, const std::vector<cplx>& b) {
      std::vector<cplx> c((size_t)d * d, 0.0);
      for (int r = 0; r < d; ++r)
        for (int q = 0; q < d; ++q)
          for (int cidx = 0; cidx < d; ++cidx) c[(size_t)r * d + cidx] += a[(size_t)r * d + q] * b[(size_t)q * d + cidx];
      return c;
    };
    switch (op) {
      case HM_SZ:
        for (int n = 0; n < d; ++n) at(n, n) = n - s;
        return true;
      case HM_SZ2:
        for (int n = 0; n < d; ++n) at(n, n) = (n - s) * (n - s);
        return true;
      case HM_SP: mat = sp; return true;
      case HM_SM: mat = sm; return true;
      case HM_SP2: mat = mul(sp, sp); return true;   // App. B: q = +2
      case HM_SM2: mat = mul(sm, sm); return true;   // App. B: q = -2
      case HM_SX:  // (S+ + S-)/2  (Sec. IV.A, h_+ = (h_x - i h_y)/2)
        for (size_t e = 0; e < mat.size(); ++e) mat[e] = 0.5 * (sp[e] + sm[e]);
        return true;
      case HM_SY:  // (S+ - S-)/(2i)
        for (size_t e = 0; e < mat.size(); ++e) mat[e] = (sp[e] - sm[e]) / cplx(0.0, 2.0);
        return true;
      default: return false;
    }
  }
  if (kind == HM_BOSON) {
    switch (op) {
      case HM_N:
        for (int n = 0; n < d; ++n) at(n, n) = (double)n;
        return true;
      case HM_ADAG:  // a^dag |n> = sqrt(n+1) |n+1>   (App. C)
        for (int n = 0; n + 1 < d; ++n) at(n + 1, n) = std::sqrt((double)n + 1.0);
        return true;
      case HM_A:     // a |n> = sqrt(n) |n-1>
        for (int n = 1; n < d; ++n) at(n - 1, n) = std::sqrt((double)n);
        return true;
      default: return false;
    }
  }
  return false;
}

// Diagonals of a local matrix: q -> vector over TARGET digit nt of mat[nt][nt-q]
// (zero where nt-q is outside [0, d-1]).
static std::map<int, std::vector<cplx>> diagonals(const std::vector<cplx>& mat, int d) {
  std::map<int, std::vector<cplx>> out;
  for (int nt = 0; nt < d; ++nt)
    for (int ns = 0; ns < d; ++ns) {
      cplx v = mat[(size_t)nt * d + ns];
      if (v == cplx(0, 0)) continue;
      int q = nt - ns;
      auto& vec = out[q];
      if (vec.empty()) vec.assign(d, 0.0);
      vec[nt] += v;
    }
  return out;
}

// Sums of several term contributions that cancel mathematically (0.2 - 0.2
// after rounding, S+S+ parts of SxSx and SySy) leave roundoff residues of a
// few ulps of the largest contribution. They are set to exactly zero: the
// matrix element is zero, and a residue of ~1e-17 would otherwise count as a
// coefficient of that size.
constexpr double kCancelTol = 16.0 * 2.220446049250313e-16;

static inline double clean_sum(double v, double maxabs) {
  return std::fabs(v) <= kCancelTol * maxabs ? 0.0 : v;
}

static int ilog2ceil(int d) {
  int w = 0;
  while ((1 << w) < d) ++w;
  return std::max(w, 1);
}

struct Derived {
  std::vector<Channel> ch;        // merged channels of H
  std::vector<std::vector<double>> chmax;  // largest contribution summed into each entry
  std::vector<Channel> tch;       // per-term channels (unit coefficient)
  std::vector<int> tch_term;
  cplx constant = 0.0;            // identity terms
};

// Expand terms into channels: each local operator splits into fixed-shift
// diagonals (App. B generic shift q); a two-site product of shifts (qi, qj)
// has the source offset -(qi M_i + qj M_j) (Sec. IV.B Eq. sourceoffset).
static int expand(const Plan* p, const std::vector<double>& coefs, Derived& out) {
  std::map<std::tuple<int, int, int, int>, size_t> index;
  for (size_t t = 0; t < p->terms.size(); ++t) {
    const hm_term& tm = p->terms[t];
    int i = tm.site_i, j = tm.site_j, oi = tm.op_i, oj = tm.op_j;
    if (j >= 0 && oj == HM_ID) j = -1;
    if (oi == HM_ID && j >= 0) { i = j; oi = oj; j = -1; }
    if (j >= 0 && j < i) { std::swap(i, j); std::swap(oi, oj); }
    double c = coefs[t];
    std::vector<cplx> A, Bm;
    if (!local_matrix(p->sites[i].kind, p->sites[i].dim, oi, A)) return HM_ERR_INVALID_ARG;
    int di = p->sites[i].dim, dj = 1;
    std::map<int, std::vector<cplx>> dA = diagonals(A, di), dB;
    if (j >= 0) {
      if (!local_matrix(p->sites[j].kind, p->sites[j].dim, oj, Bm)) return HM_ERR_INVALID_ARG;
      dj = p->sites[j].dim;
      dB = diagonals(Bm, dj);
    } else {
      dB[0] = std::vector<cplx>(1, 1.0);
    }
    if (j < 0 && oi == HM_ID) {  // pure constant
      out.constant += c;
      // per-term channel: identity on site i (diag, value 1)
    }
    for (auto& a : dA)
      for (auto& b : dB) {
        Channel unit;
        unit.i = i; unit.j = j; unit.qi = a.first; unit.qj = (j >= 0) ? b.first : 0;
        unit.di = di; unit.dj = dj;
        unit.T.assign((size_t)di * dj, 0.0);
        for (int ni = 0; ni < di; ++ni)
          for (int nj = 0; nj < dj; ++nj) unit.T[(size_t)ni * dj + nj] = a.second[ni] * b.second[nj];
        // per-term (unit coefficient) copy for gradients
        out.tch.push_back(unit);
        out.tch_term.push_back((int)t);
        if (j < 0 && oi == HM_ID) continue;  // constants live in out.constant
        auto key = std::make_tuple(unit.i, unit.qi, unit.j, unit.qj);
        auto it = index.find(key);
        std::vector<cplx> fa = a.second, fb = (j >= 0) ? b.second : std::vector<cplx>(1, 1.0);
        for (auto& v : fa) v *= c;
        if (it == index.end()) {
          index[key] = out.ch.size();
          Channel m = unit;
          for (auto& v : m.T) v *= c;
          m.parts.push_back({fa, fb});
          out.ch.push_back(m);
          out.chmax.emplace_back(m.T.size());
          for (size_t e = 0; e < m.T.size(); ++e) out.chmax.back()[e] = std::abs(m.T[e]);
        } else {
          Channel& m = out.ch[it->second];
          for (size_t e = 0; e < m.T.size(); ++e) {
            m.T[e] += c * unit.T[e];
            out.chmax[it->second][e] = std::max(out.chmax[it->second][e], std::abs(c * unit.T[e]));
          }
          m.parts.push_back({fa, fb});
        }
      }
  }
  for (size_t c = 0; c < out.ch.size(); ++c)
    for (size_t e = 0; e < out.ch[c].T.size(); ++e) {
      const cplx v = out.ch[c].T[e];
      out.ch[c].T[e] = cplx(clean_sum(v.real(), out.chmax[c][e]), clean_sum(v.imag(), out.chmax[c][e]));
    }
  return HM_OK;
}

// Real-storage check: every merged matrix element must be real.
static bool all_real(const Derived& d) {
  double mx = 0.0;
  for (auto& c : d.ch)
    for (auto& v : c.T) mx = std::max(mx, std::abs(v));
  for (auto& c : d.ch)
    for (auto& v : c.T)
      if (std::abs(v.imag()) > 1e-13 * (1.0 + mx)) return false;
  return std::abs(d.constant.imag()) <= 1e-13 * (1.0 + mx);
}

// Transpose of one channel: target I, source F = I - off; H^T[I][F] = H[F][I]
// = T[digits(F)], digits(F) = digits(I) + q.
static Channel transpose_channel(const Channel& c) {
  Channel t = c;
  t.qi = -c.qi;
  t.qj = -c.qj;
  std::fill(t.T.begin(), t.T.end(), 0.0);
  for (int ni = 0; ni < c.di; ++ni)
    for (int nj = 0; nj < c.dj; ++nj) {
      int si = ni + c.qi, sj = (c.j >= 0) ? nj + c.qj : nj;
      if (si < 0 || si >= c.di || sj < 0 || sj >= c.dj) continue;
      t.T[(size_t)ni * c.dj + nj] = c.T[(size_t)si * c.dj + sj];
    }
  // factor pairs: a'(n) = a(n + q) on the shifted range, zero elsewhere
  auto shift = [](const std::vector<cplx>& f, int q) {
    std::vector<cplx> g(f.size(), 0.0);
    for (int n = 0; n < (int)f.size(); ++n)
      if (n + q >= 0 && n + q < (int)f.size()) g[n] = f[n + q];
    return g;
  };
  for (auto& pr : t.parts) {
    pr.first = shift(pr.first, c.qi);
    pr.second = (c.j >= 0) ? shift(pr.second, c.qj) : pr.second;
  }
  return t;
}

static bool is_symmetric(const std::vector<Channel>& ch) {
  std::map<std::tuple<int, int, int, int>, const Channel*> idx;
  double mx = 0.0;
  for (auto& c : ch) {
    idx[std::make_tuple(c.i, c.qi, c.j, c.qj)] = &c;
    for (auto& v : c.T) mx = std::max(mx, std::abs(v));
  }
  for (auto& c : ch) {
    Channel t = transpose_channel(c);
    auto it = idx.find(std::make_tuple(t.i, t.qi, t.j, t.qj));
    bool zero_t = std::all_of(t.T.begin(), t.T.end(), [](cplx v) { return v == cplx(0, 0); });
    if (it == idx.end()) {
      if (!zero_t) return false;
      continue;
    }
    for (size_t e = 0; e < t.T.size(); ++e)
      if (std::abs(t.T[e] - it->second->T[e]) > 1e-12 * (1.0 + mx)) return false;
  }
  return true;
}

// H^dagger = H: every channel's transpose equals the complex conjugate of
// the channel with the transposed shifts.
static bool is_self_adjoint(const std::vector<Channel>& ch) {
  std::map<std::tuple<int, int, int, int>, const Channel*> idx;
  double mx = 0.0;
  for (auto& c : ch) {
    idx[std::make_tuple(c.i, c.qi, c.j, c.qj)] = &c;
    for (auto& v : c.T) mx = std::max(mx, std::abs(v));
  }
  for (auto& c : ch) {
    Channel t = transpose_channel(c);
    auto it = idx.find(std::make_tuple(t.i, t.qi, t.j, t.qj));
    bool zero_t = std::all_of(t.T.begin(), t.T.end(), [](cplx v) { return v == cplx(0, 0); });
    if (it == idx.end()) {
      if (!zero_t) return false;
      continue;
    }
    for (size_t e = 0; e < t.T.size(); ++e)
      if (std::abs(t.T[e] - std::conj(it->second->T[e])) > 1e-12 * (1.0 + mx)) return false;
  }
  return true;
}

// A complex H = H_re + i H_im is held as two real operators on the same
// channel structure: keep the real (part 0) or imaginary (part 1) part of
// every table, and split each contributing product a (x) b so that the
// factor lists still sum to the kept table:
//   Re(a (x) b) = Re a (x) Re b - Im a (x) Im b,
//   Im(a (x) b) = Re a (x) Im b + Im a (x) Re b.
// Channels whose kept part vanishes are dropped.
static void keep_part(std::vector<Channel>& ch, int part) {
  auto re = [](const std::vector<cplx>& v, double sg) {
    std::vector<cplx> r(v.size());
    for (size_t i = 0; i < v.size(); ++i) r[i] = sg * v[i].real();
    return r;
  };
  auto im = [](const std::vector<cplx>& v) {
    std::vector<cplx> r(v.size());
    for (size_t i = 0; i < v.size(); ++i) r[i] = v[i].imag();
    return r;
  };
  auto zero = [](const std::vector<cplx>& v) {
    return std::all_of(v.begin(), v.end(), [](cplx z) { return z == cplx(0, 0); });
  };
  std::vector<Channel> out;
  for (Channel c : ch) {
    for (auto& v : c.T) v = part ? cplx(v.imag(), 0.0) : cplx(v.real(), 0.0);
    if (zero(c.T)) continue;
    std::vector<std::pair<std::vector<cplx>, std::vector<cplx>>> np;
    for (auto& pr : c.parts) {
      std::pair<std::vector<cplx>, std::vector<cplx>> u, w;
      if (part == 0) {
        u = {re(pr.first, 1.0), re(pr.second, 1.0)};
        w = {re(im(pr.first), -1.0), im(pr.second)};
      } else {
        u = {re(pr.first, 1.0), im(pr.second)};
        w = {im(pr.first), re(pr.second, 1.0)};
      }
      for (auto* q : {&u, &w})
        if (!zero(q->first) && !zero(q->second)) np.push_back(*q);
    }
    c.parts = np;
    out.push_back(std::move(c));
  }
  ch.swap(out);
}

// Device-table assembly for one operator (H or H^T) under the plan's split.
struct HostTables {
  std::vector<KChan> kch;       // [HH diag | HH off-diagonal]
  std::vector<KGroup> grp;      // [diag groups | off-diagonal groups]
  std::vector<KMember> mem;
  std::vector<double> tab;      // coefficient pool
  std::vector<double> diag;     // [B]
  std::vector<int> ell_delta;   // [w*B]
  std::vector<double> ell;      // [w*B]
  int n_hh_diag = 0, n_hh = 0, n_grp_diag = 0, n_grp = 0, ell_w = 0;
  long long vperiod = 0;        // see KPlan::vperiod
};

struct HostPlanData {
  double cmin = 0.0, cmax = 0.0;   // smallest / largest nonzero |coefficient| of the pools
  std::vector<KSite> ks;
  std::vector<uint32_t> ptab;
  HostTables Hf, Ht;
  std::vector<KTermChan> tk;
  std::vector<double> ttab;
  int nhigh = 0;
};

static bool same_bits(const std::vector<cplx>& a, const std::vector<cplx>& b) {
  return a.size() == b.size() && std::memcmp(a.data(), b.data(), a.size() * sizeof(cplx)) == 0;
}

static void build_tables(const Plan* p, const std::vector<Channel>& chans, cplx constant,
                         const std::vector<uint32_t>& ptab, const std::vector<KSite>& ks,
                         HostTables& H) {
  const int nhigh = p->N - p->nlow;
  const int B = p->B;
  auto high = [&](int s) { return s >= 0 && s < nhigh; };
  auto push_tab = [&](const std::vector<double>& v) {
    int base = (int)H.tab.size();
    H.tab.insert(H.tab.end(), v.begin(), v.end());
    return base;
  };
  std::vector<KChan> hh_diag, hh;
  H.diag.assign(B, constant.real());
  std::vector<double> diagmax(B, std::fabs(constant.real()));
  auto low_digit = [&](int lo, int site) -> int {
    return (int)((ptab[lo] >> ks[site].lbit) & ((1u << ks[site].lwid) - 1u));
  };
  std::vector<std::vector<std::pair<int, double>>> ell_rows(B);

  // mixed channels, collected per (diag?, low site, low factor) group
  struct Mixed {
    int lsite, hsite;
    bool diag;
    long long off;
    bool factored;
    std::vector<cplx> u, v;        // factored: T[n_h][n_l] = u[n_h] v[n_l]
    std::vector<double> rows;      // not factored: [d_h][d_l] table
  };
  std::vector<Mixed> mixed;

  for (const Channel& c : chans) {
    bool all_zero = std::all_of(c.T.begin(), c.T.end(), [](cplx v) { return v == cplx(0, 0); });
    if (all_zero) continue;
    const bool diag = (c.qi == 0 && c.qj == 0);
    const bool ih = high(c.i), jh = (c.j < 0) ? true : high(c.j);
    const bool il = !high(c.i), jl = (c.j < 0) ? true : !high(c.j);
    long long off = -((long long)c.qi * p->M[c.i] + (c.j >= 0 ? (long long)c.qj * p->M[c.j] : 0LL));
    if (il && jl) {  // entirely inside the low block: ELL / low diagonal
      for (int lo = 0; lo < B; ++lo) {
        int ni = low_digit(lo, c.i);
        int nj = (c.j >= 0) ? low_digit(lo, c.j) : 0;
        double v = c.T[(size_t)ni * c.dj + nj].real();
        if (v == 0.0) continue;
        if (diag) {
          H.diag[lo] += v;
          diagmax[lo] = std::max(diagmax[lo], std::fabs(v));
        }
        else ell_rows[lo].push_back({(int)off, v});
      }
      continue;
    }
    if (ih && jh) {  // tile-uniform coefficient
      KChan k{};
      k.off = off;
      std::vector<double> t;
      for (auto& v : c.T) t.push_back(v.real());
      k.tab = push_tab(t);
      k.dj = c.dj;
      k.kind = (diag ? CK_DIAG : 0) | (c.j < 0 ? CK_SINGLE : 0);
      k.si = (uint8_t)c.i;
      k.sj = (uint8_t)(c.j >= 0 ? c.j : 255);
      (diag ? hh_diag : hh).push_back(k);
      continue;
    }
    // one high, one low site. Low sites are the trailing ones, so with i < j
    // the low site is always j: the coefficient sits on the high factor.
    Mixed m;
    const bool low_is_i = !ih;
    m.lsite = low_is_i ? c.i : c.j;
    m.hsite = low_is_i ? c.j : c.i;
    m.diag = diag;
    m.off = off;
    // factorisation from the contributing products: exact when every product
    // carries the same low-site factor (bitwise)
    const auto& lowf0 = low_is_i ? c.parts[0].first : c.parts[0].second;
    bool fac = true;
    for (auto& pr : c.parts) fac = fac && same_bits(low_is_i ? pr.first : pr.second, lowf0);
    m.factored = fac;
    const int dh = p->sites[m.hsite].dim, dl = p->sites[m.lsite].dim;
    if (fac) {
      // the low factor of a single product is a raw local diagonal; the
      // coefficient sits on the high factor
      m.v = lowf0;
      m.u.assign(dh, 0.0);
      std::vector<double> ucontrib(dh, 0.0);
      for (auto& pr : c.parts) {
        const auto& hf = low_is_i ? pr.second : pr.first;
        for (int n = 0; n < dh; ++n) {
          m.u[n] += hf[n];
          ucontrib[n] = std::max(ucontrib[n], std::abs(hf[n]));
        }
      }
      for (int n = 0; n < dh; ++n)
        m.u[n] = cplx(clean_sum(m.u[n].real(), ucontrib[n]), clean_sum(m.u[n].imag(), ucontrib[n]));
      if (low_is_i) m.factored = false;  // unreachable for suffix low blocks; keep the table path
      // u and v may each be imaginary with a real product (SySy): move the
      // phase of v onto u so that both are real, else use the table path
      cplx ph = 0.0;
      for (auto& z : m.v)
        if (z != cplx(0, 0)) { ph = z / std::abs(z); break; }
      if (ph == cplx(0, 0)) m.factored = false;
      double vmax = 0.0, umax = 0.0, vim = 0.0, uim = 0.0;
      for (auto& z : m.v) { z /= (ph == cplx(0, 0) ? cplx(1, 0) : ph); vmax = std::max(vmax, std::abs(z)); vim = std::max(vim, std::abs(z.imag())); }
      for (auto& z : m.u) { z *= ph; umax = std::max(umax, std::abs(z)); uim = std::max(uim, std::abs(z.imag())); }
      if (vim > 1e-14 * vmax || uim > 1e-14 * umax) m.factored = false;
    }
    if (!m.factored) {
      m.rows.assign((size_t)dh * dl, 0.0);
      for (int nh = 0; nh < dh; ++nh)
        for (int nl = 0; nl < dl; ++nl) {
          size_t idx = low_is_i ? (size_t)nl * c.dj + nh : (size_t)nh * c.dj + nl;
          m.rows[(size_t)nh * dl + nl] = c.T[idx].real();
        }
    }
    mixed.push_back(std::move(m));
  }
  for (int lo = 0; lo < B; ++lo) H.diag[lo] = clean_sum(H.diag[lo], diagmax[lo]);

  // ---- groups ----
  std::vector<KGroup> gd, go;
  std::vector<std::vector<KMember>> gmem_d, gmem_o;
  auto add_group = [&](bool diag, const Mixed& m) {
    auto& G = diag ? gd : go;
    auto& GM = diag ? gmem_d : gmem_o;
    if (!diag) {  // period of the low digit the group's v reads
      const long long per = p->M[m.lsite] * p->sites[m.lsite].dim;
      long long a = H.vperiod ? H.vperiod : 1, b = per;
      while (b) { const long long t = a % b; a = b; b = t; }
      const long long l = (H.vperiod ? H.vperiod : 1) / a * per;
      H.vperiod = l > (1LL << 40) ? (1LL << 40) : l;
    }
    const int dh = p->sites[m.hsite].dim;
    KMember mb{};
    mb.off = diag ? 0 : m.off;
    mb.usite = (uint8_t)m.hsite;
    if (m.factored) {
      std::vector<double> vr, ur;
      for (auto& z : m.v) vr.push_back(z.real());
      for (auto& z : m.u) ur.push_back(z.real());
      // find a group with the same low site and identical v
      for (size_t g = 0; g < G.size(); ++g) {
        if (G[g].vstride != 0 || G[g].lbit != ks[m.lsite].lbit || G[g].lwid != ks[m.lsite].lwid) continue;
        const double* gv = H.tab.data() + G[g].vtab;
        if ((int)vr.size() == (int)p->sites[m.lsite].dim && std::memcmp(gv, vr.data(), vr.size() * 8) == 0) {
          mb.utab = push_tab(ur);
          GM[g].push_back(mb);
          return;
        }
      }
      KGroup k{};
      k.vtab = push_tab(vr);
      k.vstride = 0;
      k.vsite = 255;
      k.lbit = ks[m.lsite].lbit;
      k.lwid = ks[m.lsite].lwid;
      mb.utab = push_tab(ur);
      G.push_back(k);
      GM.push_back({mb});
    } else {
      KGroup k{};
      k.vtab = push_tab(m.rows);
      k.vstride = p->sites[m.lsite].dim;
      k.vsite = (uint8_t)m.hsite;
      k.lbit = ks[m.lsite].lbit;
      k.lwid = ks[m.lsite].lwid;
      mb.utab = push_tab(std::vector<double>(dh, 1.0));
      G.push_back(k);
      GM.push_back({mb});
    }
  };
  for (auto& m : mixed) add_group(m.diag, m);
  for (int pass = 0; pass < 2; ++pass) {
    auto& G = pass == 0 ? gd : go;
    auto& GM = pass == 0 ? gmem_d : gmem_o;
    for (size_t g = 0; g < G.size(); ++g) {
      G[g].m0 = (int)H.mem.size();
      H.mem.insert(H.mem.end(), GM[g].begin(), GM[g].end());
      G[g].m1 = (int)H.mem.size();
      H.grp.push_back(G[g]);
    }
  }
  H.n_grp_diag = (int)gd.size();
  H.n_grp = (int)go.size();

  // ---- ELL: merge equal offsets, pad to a common width ----
  int w = 0;
  for (auto& r : ell_rows) {
    std::sort(r.begin(), r.end(), [](auto& a, auto& b) { return a.first < b.first; });
    std::vector<std::pair<int, double>> mm;
    std::vector<double> mx;
    for (auto& e : r) {
      if (!mm.empty() && mm.back().first == e.first) {
        mm.back().second += e.second;
        mx.back() = std::max(mx.back(), std::fabs(e.second));
      } else {
        mm.push_back(e);
        mx.push_back(std::fabs(e.second));
      }
    }
    r.clear();
    for (size_t k = 0; k < mm.size(); ++k)
      if (clean_sum(mm[k].second, mx[k]) != 0.0) r.push_back(mm[k]);
    w = std::max(w, (int)r.size());
  }
  H.ell_w = w;
  H.ell_delta.assign((size_t)w * B, 0);
  H.ell.assign((size_t)w * B, 0.0);
  for (int lo = 0; lo < B; ++lo)
    for (size_t e = 0; e < ell_rows[lo].size(); ++e) {
      H.ell_delta[e * B + lo] = ell_rows[lo][e].first;
      H.ell[e * B + lo] = ell_rows[lo][e].second;
    }
  H.n_hh_diag = (int)hh_diag.size();
  H.n_hh = (int)hh.size();
  H.kch = hh_diag;
  H.kch.insert(H.kch.end(), hh.begin(), hh.end());
}

static float2 split_df(double v) {
  float hi = (float)v;
  float lo = (float)(v - (double)hi);
  return make_float2(hi, lo);
}

void free_plan_device(Plan* p) {
  if (p->dev) cudaFree(p->dev);
  p->dev = nullptr;
  p->dev_bytes = 0;
}

int plan_check(const Plan* p) {
  if (p->N < 1 || p->N > kMaxSites) {
    set_error("nsites must be in [1, 64]");
    return HM_ERR_INVALID_ARG;
  }
  for (int s = 0; s < p->N; ++s) {
    const hm_site& st = p->sites[s];
    if (st.kind != HM_SPIN && st.kind != HM_BOSON) {
      set_error("site " + std::to_string(s) + ": unknown kind");
      return HM_ERR_INVALID_ARG;
    }
    if (st.dim < 2) {
      set_error("site " + std::to_string(s) + ": dim must be >= 2");
      return HM_ERR_INVALID_ARG;
    }
    if (st.dim > kMaxDim) {
      set_error("site " + std::to_string(s) + ": dim above 65536");
      return HM_ERR_UNSUPPORTED;
    }
  }
  for (size_t t = 0; t < p->terms.size(); ++t) {
    const hm_term& tm = p->terms[t];
    std::string where = "term " + std::to_string(t) + ": ";
    if (tm.site_i < 0 || tm.site_i >= p->N || tm.site_j < -1 || tm.site_j >= p->N) {
      set_error(where + "site index out of range");
      return HM_ERR_INVALID_ARG;
    }
    if (tm.site_i == tm.site_j) {
      set_error(where + "site_i == site_j (write same-site products as Sz2/Sp2/Sm2)");
      return HM_ERR_INVALID_ARG;
    }
    if (!std::isfinite(tm.coef)) {
      set_error(where + "non-finite coefficient");
      return HM_ERR_INVALID_ARG;
    }
    std::vector<cplx> tmp;
    if (!local_matrix(p->sites[tm.site_i].kind, p->sites[tm.site_i].dim, tm.op_i, tmp) ||
        (tm.site_j >= 0 && !local_matrix(p->sites[tm.site_j].kind, p->sites[tm.site_j].dim, tm.op_j, tmp))) {
      set_error(where + "operator not defined on that site kind");
      return HM_ERR_INVALID_ARG;
    }
  }
  return HM_OK;
}

// Host half of the plan build: every table the kernels read, for H and (when
// H is not symmetric) H^T. No device calls.
int derive_plan(Plan* p, HostPlanData& out, long long cap) {
  std::vector<KSite>& ks = out.ks;
  std::vector<uint32_t>& ptab = out.ptab;
  HostTables& Hf = out.Hf;
  HostTables& Ht = out.Ht;
  std::vector<KTermChan>& tk = out.tk;
  std::vector<double>& ttab = out.ttab;
  // multipliers M_k = prod_{l>k} d_l (Sec. III), D = prod d_k (Sec. I Eq. 1)
  p->M.assign(p->N, 1);
  long long m = 1;
  for (int k = p->N - 1; k >= 0; --k) {
    p->M[k] = m;
    if (m > kMaxD / p->sites[k].dim) {
      set_error("D = prod d_k must be below 2^62");
      return HM_ERR_OVERFLOW;
    }
    m *= p->sites[k].dim;
  }
  p->D = m;

  // split: trailing sites whose product stays <= cap form the low block
  // (digits tabulated per low index); the rest are tile-uniform.
  int nlow = 0;
  long long B = 1;
  for (int k = p->N - 1; k >= 0; --k) {
    if (B * p->sites[k].dim > cap && nlow > 0) break;
    B *= p->sites[k].dim;
    ++nlow;
    if (B > cap) break;  // a single large site
  }
  p->nlow = nlow;
  p->B = (int)B;
  p->nblk = p->D / B;
  const int nhigh = p->N - nlow;

  ks.assign(p->N, KSite{});
  int bit = 0;
  for (int k = p->N - 1; k >= 0; --k) {
    ks[k].M = p->M[k];
    ks[k].d = p->sites[k].dim;
    if (k >= nhigh) {
      ks[k].is_low = 1;
      ks[k].lbit = (uint8_t)bit;
      ks[k].lwid = (uint8_t)ilog2ceil(p->sites[k].dim);
      bit += ks[k].lwid;
      ks[k].mh = 0;
    } else {
      ks[k].mh = p->M[k] / B;
    }
  }
  if (bit > 32) {
    set_error("low block needs more than 32 digit bits");
    return HM_ERR_UNSUPPORTED;
  }
  ptab.assign(B, 0);
  for (int lo = 0; lo < B; ++lo) {
    uint32_t w = 0;
    for (int k = nhigh; k < p->N; ++k) {
      uint32_t n = (uint32_t)((lo / p->M[k]) % p->sites[k].dim);  // Eq. decode on the low part
      w |= n << ks[k].lbit;
    }
    ptab[lo] = w;
  }

  std::vector<double> coefs(p->terms.size());
  for (size_t t = 0; t < p->terms.size(); ++t) coefs[t] = p->terms[t].coef;
  Derived dv;
  int rc = expand(p, coefs, dv);
  if (rc) {
    set_error("operator expansion failed");
    return rc;
  }
  p->grad_ok = true;
  p->complex_h = !all_real(dv);
  if (p->complex_h) {  // imaginary matrix elements (Sy factors): keep one part
    p->hermitian_c = is_self_adjoint(dv.ch);
    keep_part(dv.ch, p->part);
    dv.tch.clear();    // coupling gradients are not provided for complex H
    dv.tch_term.clear();
    p->grad_ok = false;
  } else if (p->part == 1) {
    dv.ch.clear();     // the imaginary part of a real H
  }
  if (p->part == 1) dv.constant = 0.0;  // coefficients are real: constants are real
  p->hermitian = is_symmetric(dv.ch);
  if (!p->complex_h) p->hermitian_c = p->hermitian;

  build_tables(p, dv.ch, dv.constant, ptab, ks, Hf);
  std::vector<Channel> tr;
  if (!p->hermitian) {
    for (auto& c : dv.ch) tr.push_back(transpose_channel(c));
    build_tables(p, tr, dv.constant, ptab, ks, Ht);
  }
  p->chH = dv.ch;
  p->chT = tr;
  p->constant = dv.constant.real();

  // per-term channels (adjoint gradients): full-digit lookups, unit coefficients
  for (size_t c = 0; c < dv.tch.size(); ++c) {
    const Channel& ch = dv.tch[c];
    bool all_zero = std::all_of(ch.T.begin(), ch.T.end(), [](cplx v) { return v == cplx(0, 0); });
    if (all_zero) continue;
    KTermChan k{};
    k.off = -((long long)ch.qi * p->M[ch.i] + (ch.j >= 0 ? (long long)ch.qj * p->M[ch.j] : 0LL));
    k.tab = (int)ttab.size();
    k.dj = ch.dj;
    k.term = dv.tch_term[c];
    k.si = (uint8_t)ch.i;
    k.sj = (uint8_t)(ch.j >= 0 ? ch.j : 255);
    // A term of a real H may itself be imaginary (a Sy term whose
    // coefficient is zero, or two that cancel): its operator O_t has no real
    // gradient, so the plan then offers no coupling gradients at all.
    bool term_real = true;
    for (auto& v : ch.T) {
      term_real = term_real && std::abs(v.imag()) <= 1e-13 * (1.0 + std::abs(v));
      ttab.push_back(v.real());
    }
    if (!term_real) {
      p->grad_ok = false;
      tk.clear();
      ttab.clear();
      break;
    }
    tk.push_back(k);
  }
  out.nhigh = nhigh;
  // coefficient range of the pools: it fixes the input window of the
  // double-float arithmetic (df_window)
  double cmin = HUGE_VAL, cmax = 0.0;
  auto see = [&](double v) {
    const double a = std::fabs(v);
    if (a == 0.0) return;
    cmin = std::min(cmin, a);
    cmax = std::max(cmax, a);
  };
  for (const HostTables* H : {&Hf, &Ht}) {
    for (double v : H->tab) see(v);
    for (double v : H->diag) see(v);
    for (double v : H->ell) see(v);
  }
  out.cmin = cmax > 0.0 ? cmin : 0.0;
  out.cmax = cmax;
  return HM_OK;
}

// Input window of the double-float arithmetic for a coefficient range
// [cmin, cmax]: every product c x then lies in [2^-100, 2^120), so its
// rounding error and the split's low parts are normal floats (relative
// accuracy ~2^-46) and sums of a few hundred products stay finite; x itself
// must split into normal floats ([2^-100, 2^126)). Empty window (lo >= hi):
// native FP64 only.
void df_window(double cmin, double cmax, double* lo, double* hi) {
  double l = std::ldexp(1.0, -100), h = std::ldexp(1.0, 126);
  if (cmax > 0.0) {
    l = std::max(l, std::ldexp(1.0, -100) / cmin);
    h = std::min(h, std::ldexp(1.0, 120) / cmax);
  }
  *lo = l;
  *hi = h;
}

// Upload the tables of `hd` (derived for p's split) into one fresh device
// allocation and fill the kernel plans of H and H^T with pointers into it.
static int upload_tables(const Plan* p, const HostPlanData& hd, void** dev_out, size_t* bytes_out, KPlan* kh,
                         KPlan* kth) {
  const std::vector<KSite>& ks = hd.ks;
  const std::vector<uint32_t>& ptab = hd.ptab;
  const HostTables& Hf = hd.Hf;
  const HostTables& Ht = hd.Ht;
  const std::vector<KTermChan>& tk = hd.tk;
  const std::vector<double>& ttab = hd.ttab;
  const int nhigh = hd.nhigh;
  // ---- device layout: one allocation, 256-byte aligned sections ----
  struct Sec { const void* src; size_t bytes; size_t off; };
  std::vector<Sec> secs;
  size_t cur = 0;
  auto add = [&](const void* src, size_t bytes) -> size_t {
    cur = (cur + 255) & ~size_t(255);
    secs.push_back({src, bytes, cur});
    size_t o = cur;
    cur += std::max<size_t>(bytes, 1);
    return o;
  };
  std::vector<float2> tabdf[2], diagdf[2];
  std::vector<float> tabf[2], diagf[2];
  const HostTables* HT[2] = {&Hf, p->hermitian ? &Hf : &Ht};
  for (int s = 0; s < 2; ++s) {
    const HostTables& H = *HT[s];
    for (double v : H.tab) { tabdf[s].push_back(split_df(v)); tabf[s].push_back((float)v); }
    for (double v : H.diag) { diagdf[s].push_back(split_df(v)); diagf[s].push_back((float)v); }
  }
  // packed ELL entries {delta, coefficient}; padding is {0, 0} (own element, zero weight)
  std::vector<int32_t> ellpf[2], ellpdf[2], ellpd[2];
  for (int s = 0; s < 2; ++s) {
    const HostTables& H = *HT[s];
    for (size_t e = 0; e < H.ell.size(); ++e) {
      const double v = H.ell[e];
      const float f = (float)v;
      const float2 df = split_df(v);
      int32_t fb, hb, lb, w[2];
      std::memcpy(&fb, &f, 4);
      std::memcpy(&hb, &df.x, 4);
      std::memcpy(&lb, &df.y, 4);
      std::memcpy(w, &v, 8);
      ellpf[s].insert(ellpf[s].end(), {H.ell_delta[e], fb});
      ellpdf[s].insert(ellpdf[s].end(), {H.ell_delta[e], 0, hb, lb});
      ellpd[s].insert(ellpd[s].end(), {H.ell_delta[e], 0, w[0], w[1]});
    }
  }
  std::vector<float2> ttabdf;
  std::vector<float> ttabf;
  for (double v : ttab) { ttabdf.push_back(split_df(v)); ttabf.push_back((float)v); }

  size_t o_sites = add(ks.data(), ks.size() * sizeof(KSite));
  size_t o_ptab = add(ptab.data(), ptab.size() * 4);
  size_t o_tch = add(tk.data(), tk.size() * sizeof(KTermChan));
  size_t o_ttd = add(ttab.data(), ttab.size() * 8);
  size_t o_ttdf = add(ttabdf.data(), ttabdf.size() * 8);
  size_t o_ttf = add(ttabf.data(), ttabf.size() * 4);
  size_t o[2][14];
  int nsets = p->hermitian ? 1 : 2;
  for (int s = 0; s < nsets; ++s) {
    const HostTables& H = *HT[s];
    o[s][0] = add(H.kch.data(), H.kch.size() * sizeof(KChan));
    o[s][1] = add(ellpf[s].data(), ellpf[s].size() * 4);
    o[s][2] = add(H.tab.data(), H.tab.size() * 8);
    o[s][3] = add(tabdf[s].data(), tabdf[s].size() * 8);
    o[s][4] = add(tabf[s].data(), tabf[s].size() * 4);
    o[s][5] = add(H.diag.data(), H.diag.size() * 8);
    o[s][6] = add(diagdf[s].data(), diagdf[s].size() * 8);
    o[s][7] = add(diagf[s].data(), diagf[s].size() * 4);
    o[s][8] = add(ellpdf[s].data(), ellpdf[s].size() * 4);
    o[s][9] = add(ellpd[s].data(), ellpd[s].size() * 4);
    o[s][11] = add(H.grp.data(), H.grp.size() * sizeof(KGroup));
    o[s][12] = add(H.mem.data(), H.mem.size() * sizeof(KMember));
  }
  size_t total = (cur + 255) & ~size_t(255);

  std::vector<unsigned char> host(total, 0);
  for (auto& sc : secs)
    if (sc.bytes) std::memcpy(host.data() + sc.off, sc.src, sc.bytes);

  void* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, total);
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc of plan tables failed: ") + cudaGetErrorString(e));
    return HM_ERR_OOM;
  }
  e = cudaMemcpy(dev, host.data(), total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return cuda_fail(e, "plan upload");
  }
  *dev_out = dev;
  *bytes_out = total;

  auto P = [&](size_t off) { return (const char*)dev + off; };
  auto fill = [&](KPlan& k, int s) {
    const HostTables& H = *HT[s];
    int ss = p->hermitian ? 0 : s;
    k = KPlan{};
    k.D = p->D;
    k.nblk = p->nblk;
    k.B = p->B;
    k.nsites = p->N;
    k.nhigh = nhigh;
    k.n_hh_diag = H.n_hh_diag;
    k.n_hh = H.n_hh;
    k.n_grp_diag = H.n_grp_diag;
    k.n_grp = H.n_grp;
    k.n_mem = (int)H.mem.size();
    k.ell_w = H.ell_w;
    k.vperiod = H.vperiod;
    k.nterm_ch = (int)tk.size();
    k.nterms = (int)p->terms.size();
    k.sites = (const KSite*)P(o_sites);
    k.ch = (const KChan*)P(o[ss][0]);
    k.ptab = (const uint32_t*)P(o_ptab);
    k.ell_pf = (const int2*)P(o[ss][1]);
    k.tab_d = (const double*)P(o[ss][2]);
    k.tab_df = (const float2*)P(o[ss][3]);
    k.tab_f = (const float*)P(o[ss][4]);
    k.diag_d = (const double*)P(o[ss][5]);
    k.diag_df = (const float2*)P(o[ss][6]);
    k.diag_f = (const float*)P(o[ss][7]);
    k.ell_pdf = (const int4*)P(o[ss][8]);
    k.ell_pd = (const int4*)P(o[ss][9]);
    k.grp = (const KGroup*)P(o[ss][11]);
    k.mem = (const KMember*)P(o[ss][12]);
    k.tch = (const KTermChan*)P(o_tch);
    k.ttab_d = (const double*)P(o_ttd);
    k.ttab_df = (const float2*)P(o_ttdf);
    k.ttab_f = (const float*)P(o_ttf);
  };
  fill(*kh, 0);
  fill(*kth, 1);
  return HM_OK;
}

int build_plan(Plan* p) {
  HostPlanData hd;
  int rc = derive_plan(p, hd, kLowBlockMax);
  if (rc) return rc;
  free_plan_device(p);
  free_tiles(p);
  free_streams(p);
  free_splits(p);
  df_window(hd.cmin, hd.cmax, &p->df_xlo, &p->df_xhi);
  p->df_ok = p->df_xlo < p->df_xhi;
  rc = upload_tables(p, hd, &p->dev, &p->dev_bytes, &p->k, &p->kt);
  if (rc) {
    p->dev = nullptr;
    p->dev_bytes = 0;
    return rc;
  }
  ++p->gen;
  if (p->sector) return build_sector(p);
  return HM_OK;
}

// Tables of the staged kernel for nvec right-hand sides: the same operator
// with a low block of at most kStreamElems / nvec states, so that one block
// of x fits one shared-memory slot. Built on first use, cached per nvec.
const StreamSet* get_stream(Plan* p, long long nvec, cudaStream_t s, bool* deferred) {
  if (deferred) *deferred = false;
  auto it = p->streams.find(nvec);
  if (it != p->streams.end()) return it->second.ok ? &it->second : nullptr;
  if (p->sector || nvec < 1 || nvec > kStreamElems) return nullptr;
  // uploading needs synchronous allocation: not inside a stream capture
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    if (deferred) *deferred = true;
    return nullptr;
  }
  Plan t;
  t.N = p->N;
  t.sites = p->sites;
  t.terms = p->terms;
  t.part = p->part;
  t.device = p->device;
  HostPlanData hd;
  StreamSet ss;
  const long long cap = kStreamElems / nvec;
  if (derive_plan(&t, hd, cap) != HM_OK || (long long)t.B * nvec > kStreamElems) {
    p->streams[nvec] = ss;  // no staged form (a single site above the slot size)
    return nullptr;
  }
  if (upload_tables(&t, hd, &ss.dev, &ss.bytes, &ss.k, &ss.kt) != HM_OK) {
    cudaGetLastError();
    if (deferred) *deferred = true;
    return nullptr;  // not cached: a later call may find memory
  }
  ss.ok = true;
  df_window(hd.cmin, hd.cmax, &ss.df_xlo, &ss.df_xhi);
  ss.df_ok = ss.df_xlo < ss.df_xhi;
  p->streams[nvec] = ss;
  return &p->streams[nvec];
}

void free_streams(Plan* p) {
  for (auto& kv : p->streams)
    if (kv.second.dev) cudaFree(kv.second.dev);
  p->streams.clear();
}

// ---------------------------------------------------------------------------
// Top-site split. A hop along site k reads x at distance M_k; when M_k times
// the bytes per state exceeds what L2 keeps of x behind the blocks in flight,
// every such source is read from DRAM a second time. The split applies the
// terms with an off-diagonal operator (a nonzero digit move, Sec. IV.A) on
// one of the leading T sites in a second pass that visits the low blocks with
// those T digits varying fastest: the blocks a top-site hop connects are then
// in flight together and x is read from DRAM about once per pass.
// ---------------------------------------------------------------------------

constexpr long long kSplitBytes = 32LL << 20;  // hop distance beyond which L2 misses
constexpr long long kSplitCombos = 512;        // top-digit combinations visited together

static bool moves_digit(int op) {
  return op == HM_SX || op == HM_SY || op == HM_SP || op == HM_SM || op == HM_SP2 || op == HM_SM2 ||
         op == HM_A || op == HM_ADAG;
}

int split_top_sites(const Plan* p, long long nvec, size_t es) {
  if (p->sector || p->N < 2) return 0;
  int T = 0;
  long long R = 1;
  while (T < p->N - 1 && (long long)p->M[T] * nvec * (long long)es >= kSplitBytes &&
         R * p->sites[T].dim <= kSplitCombos) {
    R *= p->sites[T].dim;
    ++T;
  }
  return T;
}

const SplitSet* get_split(Plan* p, int T, cudaStream_t s) {
  auto it = p->splits.find(T);
  if (it != p->splits.end()) return it->second.ok ? &it->second : nullptr;
  if (p->sector || T < 1 || T >= p->N) return nullptr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return nullptr;  // uploading needs synchronous allocation
  }
  SplitSet sp;
  Plan ta, tb;
  for (Plan* t : {&ta, &tb}) {
    t->N = p->N;
    t->sites = p->sites;
    t->part = p->part;
    t->device = p->device;
  }
  for (const hm_term& tm : p->terms) {
    const bool top = (tm.site_i < T && moves_digit(tm.op_i)) || (tm.site_j >= 0 && tm.site_j < T && moves_digit(tm.op_j));
    (top ? tb : ta).terms.push_back(tm);
  }
  if (ta.terms.empty() || tb.terms.empty()) {
    p->splits[T] = sp;  // nothing to split
    return nullptr;
  }
  HostPlanData ha, hb;
  if (derive_plan(&ta, ha, kLowBlockMax) != HM_OK || derive_plan(&tb, hb, kLowBlockMax) != HM_OK ||
      (long long)(tb.N - tb.nlow) < T) {
    cudaGetLastError();
    p->splits[T] = sp;  // the top sites must be high sites of the second pass
    return nullptr;
  }
  size_t bytes = 0;
  if (upload_tables(&ta, ha, &sp.dev_a, &bytes, &sp.ka, &sp.kat) != HM_OK) {
    cudaGetLastError();
    return nullptr;  // not cached: a later call may find memory
  }
  if (upload_tables(&tb, hb, &sp.dev_b, &bytes, &sp.kb, &sp.kbt) != HM_OK) {
    cudaGetLastError();
    cudaFree(sp.dev_a);
    return nullptr;
  }
  for (KPlan* k : {&sp.kb, &sp.kbt}) {
    k->tperm_T = T;
    k->accum = 1;
  }
  double la, ua, lb, ub;
  df_window(ha.cmin, ha.cmax, &la, &ua);
  df_window(hb.cmin, hb.cmax, &lb, &ub);
  sp.df_xlo = std::max(la, lb);
  sp.df_xhi = std::min(ua, ub);
  sp.df_ok = sp.df_xlo < sp.df_xhi;
  sp.ok = true;
  p->splits[T] = sp;
  return &p->splits[T];
}

void free_splits(Plan* p) {
  for (auto& kv : p->splits) {
    if (kv.second.dev_a) cudaFree(kv.second.dev_a);
    if (kv.second.dev_b) cudaFree(kv.second.dev_b);
  }
  p->splits.clear();
}

}  // namespace hm

// ---------------------------------------------------------------------------
// Host-only diagnostic export of the plan tables (JSON text)
// ---------------------------------------------------------------------------
namespace hm {

static void jnum(std::string& o, double v) {
  char b[40];
  snprintf(b, sizeof(b), "%.17g", v);
  o += b;
}
template <class V, class F>
static void jarr(std::string& o, const char* name, const V& v, F f) {
  o += "\"";
  o += name;
  o += "\":[";
  for (size_t i = 0; i < v.size(); ++i) {
    if (i) o += ",";
    f(v[i]);
  }
  o += "],";
}

int export_plan(Plan* p, int which, std::string& o) {
  HostPlanData hd;
  int rc = derive_plan(p, hd, kLowBlockMax);
  if (rc) return rc;
  if ((which & 4) && p->complex_h) {
    set_error("complex term lists (imaginary matrix elements) are not available for sector plans");
    return HM_ERR_UNSUPPORTED;
  }
  if ((which & 4) && (which & 16)) {  // block-form sector tables for the digit total which >> 8
    o = export_sector_blk_json(p, which >> 8, &rc);
    return rc;
  }
  if (which & 4) {  // sector tables for the digit total which >> 8
    o = export_sector_json(p, which >> 8, &rc);
    return rc;
  }
  if (which & 2) {  // tile tables for nvec = which >> 8 (at least 1)
    const bool tr = (which & 1) && !p->hermitian;
    const long long nvec = std::max(1, which >> 8);
    o = export_tile_json(p, tr ? p->chT : p->chH, p->constant, nvec, &rc);
    return rc;
  }
  const HostTables& H = ((which & 1) && !p->hermitian) ? hd.Ht : hd.Hf;
  auto I = [&](long long v) { o += std::to_string(v); };
  o = "{";
  o += "\"D\":" + std::to_string(p->D) + ",\"B\":" + std::to_string(p->B) + ",\"nblk\":" + std::to_string(p->nblk) +
       ",\"nhigh\":" + std::to_string(hd.nhigh) + ",\"hermitian\":" + (p->hermitian ? "true" : "false") +
       ",\"n_hh_diag\":" + std::to_string(H.n_hh_diag) + ",\"n_grp_diag\":" + std::to_string(H.n_grp_diag) +
       ",\"ell_w\":" + std::to_string(H.ell_w) + ",";
  jarr(o, "sites", hd.ks, [&](const KSite& k) {
    o += "[" + std::to_string(k.M) + "," + std::to_string(k.mh) + "," + std::to_string(k.d) + "," +
         std::to_string(k.lbit) + "," + std::to_string(k.lwid) + "," + std::to_string(k.is_low) + "]";
  });
  jarr(o, "ptab", hd.ptab, [&](uint32_t v) { I(v); });
  jarr(o, "ch", H.kch, [&](const KChan& k) {
    o += "[" + std::to_string(k.off) + "," + std::to_string(k.tab) + "," + std::to_string(k.dj) + "," +
         std::to_string(k.si) + "," + std::to_string(k.sj) + "," + std::to_string(k.kind) + "]";
  });
  jarr(o, "grp", H.grp, [&](const KGroup& g) {
    o += "[" + std::to_string(g.vtab) + "," + std::to_string(g.vstride) + "," + std::to_string(g.m0) + "," +
         std::to_string(g.m1) + "," + std::to_string(g.vsite) + "," + std::to_string(g.lbit) + "," +
         std::to_string(g.lwid) + "]";
  });
  jarr(o, "mem", H.mem, [&](const KMember& m) {
    o += "[" + std::to_string(m.off) + "," + std::to_string(m.utab) + "," + std::to_string(m.usite) + "]";
  });
  jarr(o, "tab", H.tab, [&](double v) { jnum(o, v); });
  jarr(o, "diag", H.diag, [&](double v) { jnum(o, v); });
  jarr(o, "ell_delta", H.ell_delta, [&](int v) { I(v); });
  jarr(o, "ell", H.ell, [&](double v) { jnum(o, v); });
  o.back() = '}';
  return HM_OK;
}

}  // namespace hm

extern "C" int hm_plan_export(const hm_site* sites, int32_t nsites, const hm_term* terms, int32_t nterms,
                              int32_t which, char* buf, int64_t bufsize, int64_t* len) {
  using namespace hm;
  if (!sites || nsites < 1 || nsites > kMaxSites || nterms < 0 || (nterms > 0 && !terms) || !len) {
    set_error("invalid export arguments");
    return HM_ERR_INVALID_ARG;
  }
  Plan p;
  p.N = nsites;
  p.sites.assign(sites, sites + nsites);
  p.terms.assign(terms, terms + nterms);
  p.part = (which >> 3) & 1;  // bit 3: the imaginary part of a complex H
  int rc = plan_check(&p);
  if (rc) return rc;
  std::string o;
  rc = export_plan(&p, which, o);
  if (rc) return rc;
  *len = (int64_t)o.size() + 1;
  if (buf && bufsize >= *len) std::memcpy(buf, o.c_str(), o.size() + 1);
  return HM_OK;
}
