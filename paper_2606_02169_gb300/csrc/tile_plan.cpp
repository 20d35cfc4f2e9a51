// Host side of the leaf-tiled apply: split the sites into high | mid | leaf
// levels and turn the merged channel list (the same fixed-shift channels as
// the general plan: local diagonals of each operator, Sec. IV.B / App. B,
// source offset -(q_i M_i + q_j M_j), Eq. sourceoffset) into
//   * members: channels without a leaf site, with their target-digit
//     coefficient table (zero = inadmissible, Sec. IV.B step 3);
//   * groups: channels with one leaf and one non-leaf site, written as
//     v(n_leaf) * u(n_other) per contributing product and grouped by v;
//   * leaf tables: per leaf state f, the diagonal from leaf-only channels and
//     the list of leaf-only hops (offset, coefficient).
// Built per (nvec, H or H^T) on first use and uploaded as one allocation.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "hm_internal.h"

namespace hm {

using cplx = std::complex<double>;

struct HostTile {
  KTile k{};
  std::vector<KTileSite> sites;
  std::vector<KTMem> bmem, rmem;
  std::vector<int> bgrp, rgrp;
  std::vector<double> tab;
  std::vector<double> dF, v, fs;
  std::vector<int> fix, fs_n, fs_off;
};

static int round_warp(long long n) { return (int)((n + 31) / 32 * 32); }

constexpr int kTileMaxThreads = 512;
constexpr int kTileMaxRows = 64;

// Leaf: the trailing sites whose product F gives F * nvec threads in
// [32, 512] with the least idle lanes (a warp-multiple is best), preferring
// at most 256 threads. Mid: the next sites while R = prod d stays <= 64.
static bool choose_split(const Plan* p, long long nvec, int& nleaf, long long& F, int& nmid, long long& R) {
  const int N = p->N;
  nleaf = -1;
  double best = -1.0;
  long long f = 1;
  for (int L = 1; L <= N; ++L) {
    f *= p->sites[N - L].dim;
    if (f * nvec > kTileMaxThreads) break;
    if (f * nvec < 32 && L < N) continue;
    const double eff = (double)(f * nvec) / round_warp(f * nvec);
    const double score = eff + (f * nvec <= 256 ? 0.05 : 0.0) + 1e-7 * (double)(f * nvec);
    if (score > best) {
      best = score;
      nleaf = L;
      F = f;
    }
  }
  if (nleaf < 0) return false;
  R = 1;
  nmid = 0;
  for (int k = N - nleaf - 1; k >= 0; --k) {
    if (R * p->sites[k].dim > kTileMaxRows) break;
    R *= p->sites[k].dim;
    ++nmid;
  }
  return true;
}

// A product's two factors as real vectors: the phase of the leaf factor is
// moved onto the other one (SySy products have two imaginary factors).
static bool real_pair(const std::vector<cplx>& other, const std::vector<cplx>& leaf, std::vector<double>& u,
                      std::vector<double>& v) {
  cplx ph = 0.0;
  for (auto& z : leaf)
    if (z != cplx(0, 0)) {
      ph = z / std::abs(z);
      break;
    }
  if (ph == cplx(0, 0)) return false;
  double umax = 0.0, vmax = 0.0, uim = 0.0, vim = 0.0;
  u.clear();
  v.clear();
  for (auto& z : leaf) {
    const cplx w = z / ph;
    v.push_back(w.real());
    vmax = std::max(vmax, std::abs(w));
    vim = std::max(vim, std::abs(w.imag()));
  }
  for (auto& z : other) {
    const cplx w = z * ph;
    u.push_back(w.real());
    umax = std::max(umax, std::abs(w));
    uim = std::max(uim, std::abs(w.imag()));
  }
  if (!(vim <= 1e-14 * vmax && uim <= 1e-14 * umax)) return false;
  // scale v to max |v| = 1 (the scale moves onto u), so that products whose
  // leaf factors differ only by a constant share one group
  double vm = 0.0;
  for (double z : v) vm = std::max(vm, std::abs(z));
  for (double& z : v) z /= vm;
  for (double& z : u) z *= vm;
  return true;
}

int derive_tile(const Plan* p, const std::vector<Channel>& ch, double constant, long long nvec, HostTile& H) {
  int nleaf = 0, nmid = 0;
  long long F = 1, R = 1;
  if (nvec < 1 || p->D * nvec >= (1LL << 31) || !choose_split(p, nvec, nleaf, F, nmid, R)) return HM_ERR_UNSUPPORTED;
  const int N = p->N;
  const int nhigh = N - nleaf - nmid;
  const int first_leaf = N - nleaf;
  auto level = [&](int s) { return s < nhigh ? 0 : (s < first_leaf ? 1 : 2); };  // 0 high, 1 mid, 2 leaf
  KTile& k = H.k;
  k.D = p->D;
  k.F = (int)F;
  k.R = (int)R;
  k.nblk = p->D / (F * R);
  k.nvec = (int)nvec;
  k.nt = round_warp(F * nvec);
  k.nhigh = nhigh;
  k.nmid = nmid;
  H.sites.assign(nhigh + nmid, KTileSite{});
  for (int s = 0; s < nhigh + nmid; ++s) {
    H.sites[s].d = p->sites[s].dim;
    H.sites[s].stride = (s < nhigh) ? p->M[s] / (F * R) : p->M[s] / F;
  }
  auto leaf_digit = [&](long long f, int s) { return (int)((f / p->M[s]) % p->sites[s].dim); };

  H.dF.assign(F, constant);
  std::vector<std::map<long long, double>> slots(F);

  struct Group {
    int site, q;
    std::vector<double> v;
    std::map<std::pair<int, long long>, std::vector<double>> mem;  // (other site, offset) -> u table
  };
  std::vector<Group> groups;
  std::vector<KTMem> m0;  // group-0 members
  auto push_tab = [&](const std::vector<double>& t) {
    const int base = (int)H.tab.size();
    H.tab.insert(H.tab.end(), t.begin(), t.end());
    return base;
  };

  for (const Channel& c : ch) {
    if (std::all_of(c.T.begin(), c.T.end(), [](cplx z) { return z == cplx(0, 0); })) continue;
    const long long off = -((long long)c.qi * p->M[c.i] + (c.j >= 0 ? (long long)c.qj * p->M[c.j] : 0LL));
    const int li = level(c.i), lj = (c.j >= 0) ? level(c.j) : -1;
    const bool leaf_i = li == 2, leaf_j = lj == 2;
    if (!leaf_i && !leaf_j) {  // member of group 0: the merged table as it is
      KTMem m{};
      m.off = off * nvec;
      std::vector<double> t;
      for (auto& z : c.T) t.push_back(z.real());
      m.tab = push_tab(t);
      m.db = c.dj;
      m.sa = (uint8_t)c.i;
      m.sb = (uint8_t)(c.j >= 0 ? c.j : 255);
      m.grp = 0;
      m.diag = off == 0;
      m0.push_back(m);
      continue;
    }
    if (leaf_i && (c.j < 0 || leaf_j)) {  // leaf-only: per-leaf-state diagonal or hop
      for (long long f = 0; f < F; ++f) {
        const int ni = leaf_digit(f, c.i);
        const int nj = (c.j >= 0) ? leaf_digit(f, c.j) : 0;
        const double v = c.T[(size_t)ni * c.dj + nj].real();
        if (v == 0.0) continue;
        if (off == 0) H.dF[f] += v;
        else slots[f][off * nvec] += v;
      }
      continue;
    }
    // one leaf site: sites are ordered i < j and the leaf sites trail, so the
    // leaf site is j and the other site i carries u
    if (leaf_i || !leaf_j) return HM_ERR_UNSUPPORTED;
    for (auto& pr : c.parts) {
      std::vector<double> u, v;
      if (!real_pair(pr.first, pr.second, u, v)) return HM_ERR_UNSUPPORTED;
      bool nz = false;
      for (double z : u) nz = nz || z != 0.0;
      if (!nz) continue;
      // same leaf site and shift, and the same (unit-scaled) leaf factor up
      // to rounding: one group (its first v stands for all)
      int g = -1;
      for (size_t q = 0; q < groups.size() && g < 0; ++q) {
        if (groups[q].site != c.j || groups[q].q != c.qj || groups[q].v.size() != v.size()) continue;
        bool same = true;
        for (size_t n = 0; n < v.size() && same; ++n) same = std::abs(groups[q].v[n] - v[n]) <= 1e-15;
        if (same) g = (int)q;
      }
      if (g < 0) {
        groups.push_back(Group{c.j, c.qj, v, {}});
        g = (int)groups.size() - 1;
      }
      auto& t = groups[g].mem[{c.i, off}];
      if (t.empty()) t.assign(u.size(), 0.0);
      for (size_t n = 0; n < u.size(); ++n) t[n] += u[n];
    }
  }
  if (groups.size() + 1 > 255) return HM_ERR_UNSUPPORTED;
  k.G = (int)groups.size() + 1;

  // members: group 0, then each group's; split by level (mid site or not)
  std::vector<KTMem> all = m0;
  for (size_t g = 0; g < groups.size(); ++g)
    for (auto& kv : groups[g].mem) {
      KTMem m{};
      m.off = kv.first.second * nvec;
      m.tab = push_tab(kv.second);
      m.db = 1;
      m.sa = (uint8_t)kv.first.first;
      m.sb = 255;
      m.grp = (uint8_t)(g + 1);
      m.diag = kv.first.second == 0;
      all.push_back(m);
    }
  H.bgrp.assign(k.G + 1, 0);
  H.rgrp.assign(k.G + 1, 0);
  for (int g = 0; g < k.G; ++g) {
    H.bgrp[g] = (int)H.bmem.size();
    H.rgrp[g] = (int)H.rmem.size();
    for (auto& m : all) {
      if (m.grp != g) continue;
      const bool mid = level(m.sa) == 1 || (m.sb != 255 && level(m.sb) == 1);
      (mid ? H.rmem : H.bmem).push_back(m);
    }
  }
  H.bgrp[k.G] = (int)H.bmem.size();
  H.rgrp[k.G] = (int)H.rmem.size();
  k.n_bmem = (int)H.bmem.size();
  k.n_rmem = (int)H.rmem.size();

  // leaf factors and redirections of each group
  H.v.assign((size_t)(k.G - 1) * F, 0.0);
  H.fix.assign((size_t)(k.G - 1) * F, 0);
  for (size_t g = 0; g < groups.size(); ++g) {
    const Group& gr = groups[g];
    for (long long f = 0; f < F; ++f) {
      const double v = gr.v[leaf_digit(f, gr.site)];
      H.v[g * F + f] = v;
      // v = 0: undo the leaf part of the shift so the gather stays in range
      H.fix[g * F + f] = (v == 0.0) ? (int)((long long)gr.q * p->M[gr.site] * nvec) : 0;
    }
  }
  // leaf slots, [w][f]
  int w = 0;
  for (auto& sl : slots) {
    int n = 0;
    for (auto& e : sl)
      if (e.second != 0.0) ++n;
    w = std::max(w, n);
  }
  k.fs_w = w;
  H.fs_n.assign(F, 0);
  H.fs_off.assign((size_t)std::max(w, 1) * F, 0);
  H.fs.assign((size_t)std::max(w, 1) * F, 0.0);
  for (long long f = 0; f < F; ++f) {
    int n = 0;
    for (auto& e : slots[f]) {
      if (e.second == 0.0) continue;
      H.fs_off[(size_t)n * F + f] = (int)e.first;
      H.fs[(size_t)n * F + f] = e.second;
      ++n;
    }
    H.fs_n[f] = n;
  }
  return HM_OK;
}

static float2 split_pair(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

const KTile* get_tile(Plan* p, long long nvec, bool transpose, cudaStream_t s) {
  const bool tr = transpose && !p->hermitian;
  auto key = std::make_pair(nvec, tr ? 1 : 0);
  auto it = p->tiles.find(key);
  if (it != p->tiles.end()) return it->second.ok ? &it->second.k : nullptr;
  // uploading needs synchronous allocation: not inside a stream capture
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
  Plan::TileSet ts;
  HostTile H;
  if (derive_tile(p, tr ? p->chT : p->chH, p->constant, nvec, H) != HM_OK) {
    p->tiles[key] = ts;
    return nullptr;
  }
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
  std::vector<float2> dFdf, vdf, fsdf;
  std::vector<float> dFf, vf, fsf;
  for (double z : H.dF) { dFdf.push_back(split_pair(z)); dFf.push_back((float)z); }
  for (double z : H.v) { vdf.push_back(split_pair(z)); vf.push_back((float)z); }
  for (double z : H.fs) { fsdf.push_back(split_pair(z)); fsf.push_back((float)z); }
  const size_t o_sites = add(H.sites.data(), H.sites.size() * sizeof(KTileSite));
  const size_t o_bmem = add(H.bmem.data(), H.bmem.size() * sizeof(KTMem));
  const size_t o_rmem = add(H.rmem.data(), H.rmem.size() * sizeof(KTMem));
  const size_t o_bgrp = add(H.bgrp.data(), H.bgrp.size() * 4);
  const size_t o_rgrp = add(H.rgrp.data(), H.rgrp.size() * 4);
  const size_t o_tab = add(H.tab.data(), H.tab.size() * 8);
  const size_t o_dFd = add(H.dF.data(), H.dF.size() * 8);
  const size_t o_dFdf = add(dFdf.data(), dFdf.size() * 8);
  const size_t o_dFf = add(dFf.data(), dFf.size() * 4);
  const size_t o_vd = add(H.v.data(), H.v.size() * 8);
  const size_t o_vdf = add(vdf.data(), vdf.size() * 8);
  const size_t o_vf = add(vf.data(), vf.size() * 4);
  const size_t o_fix = add(H.fix.data(), H.fix.size() * 4);
  const size_t o_fsn = add(H.fs_n.data(), H.fs_n.size() * 4);
  const size_t o_fso = add(H.fs_off.data(), H.fs_off.size() * 4);
  const size_t o_fsd = add(H.fs.data(), H.fs.size() * 8);
  const size_t o_fsdf = add(fsdf.data(), fsdf.size() * 8);
  const size_t o_fsf = add(fsf.data(), fsf.size() * 4);
  const size_t total = (cur + 255) & ~size_t(255);
  std::vector<unsigned char> host(total, 0);
  for (auto& sc : secs)
    if (sc.bytes) std::memcpy(host.data() + sc.off, sc.src, sc.bytes);
  void* dev = nullptr;
  if (cudaMalloc(&dev, total) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;  // not cached: a later call may find memory
  }
  if (cudaMemcpy(dev, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(dev);
    cudaGetLastError();
    return nullptr;
  }
  unsigned char* b = (unsigned char*)dev;
  KTile k = H.k;
  k.sites = (const KTileSite*)(b + o_sites);
  k.bmem = (const KTMem*)(b + o_bmem);
  k.rmem = (const KTMem*)(b + o_rmem);
  k.bgrp = (const int*)(b + o_bgrp);
  k.rgrp = (const int*)(b + o_rgrp);
  k.tab = (const double*)(b + o_tab);
  k.dF_d = (const double*)(b + o_dFd);
  k.dF_df = (const float2*)(b + o_dFdf);
  k.dF_f = (const float*)(b + o_dFf);
  k.v_d = (const double*)(b + o_vd);
  k.v_df = (const float2*)(b + o_vdf);
  k.v_f = (const float*)(b + o_vf);
  k.fix = (const int*)(b + o_fix);
  k.fs_n = (const int*)(b + o_fsn);
  k.fs_off = (const int*)(b + o_fso);
  k.fs_d = (const double*)(b + o_fsd);
  k.fs_df = (const float2*)(b + o_fsdf);
  k.fs_f = (const float*)(b + o_fsf);
  ts.ok = true;
  ts.k = k;
  ts.dev = dev;
  p->tiles[key] = ts;
  return &p->tiles[key].k;
}

void free_tiles(Plan* p) {
  for (auto& kv : p->tiles)
    if (kv.second.dev) cudaFree(kv.second.dev);
  p->tiles.clear();
}

// JSON text of the tile tables (diagnostic export; host only).
std::string export_tile_json(const Plan* p, const std::vector<Channel>& ch, double constant, long long nvec,
                             int* rc) {
  HostTile H;
  *rc = derive_tile(p, ch, constant, nvec, H);
  if (*rc != HM_OK) return std::string();
  std::string o;
  char buf[64];
  auto num = [&](double v) {
    std::snprintf(buf, sizeof buf, "%.17g", v);
    o += buf;
  };
  auto ival = [&](long long v) { o += std::to_string(v); };
  auto darr = [&](const char* name, const std::vector<double>& a) {
    o += "\"";
    o += name;
    o += "\":[";
    for (size_t i = 0; i < a.size(); ++i) {
      if (i) o += ",";
      num(a[i]);
    }
    o += "],";
  };
  auto iarr = [&](const char* name, const std::vector<int>& a) {
    o += "\"";
    o += name;
    o += "\":[";
    for (size_t i = 0; i < a.size(); ++i) {
      if (i) o += ",";
      ival(a[i]);
    }
    o += "],";
  };
  auto marr = [&](const char* name, const std::vector<KTMem>& a) {
    o += "\"";
    o += name;
    o += "\":[";
    for (size_t i = 0; i < a.size(); ++i) {
      if (i) o += ",";
      o += "[";
      ival(a[i].off); o += ",";
      ival(a[i].tab); o += ",";
      ival(a[i].db); o += ",";
      ival(a[i].sa); o += ",";
      ival(a[i].sb == 255 ? -1 : a[i].sb); o += ",";
      ival(a[i].grp); o += ",";
      ival(a[i].diag);
      o += "]";
    }
    o += "],";
  };
  const KTile& k = H.k;
  o += "{";
  o += "\"D\":"; ival(k.D); o += ",";
  o += "\"nblk\":"; ival(k.nblk); o += ",";
  o += "\"F\":"; ival(k.F); o += ",";
  o += "\"R\":"; ival(k.R); o += ",";
  o += "\"nvec\":"; ival(k.nvec); o += ",";
  o += "\"nt\":"; ival(k.nt); o += ",";
  o += "\"nhigh\":"; ival(k.nhigh); o += ",";
  o += "\"nmid\":"; ival(k.nmid); o += ",";
  o += "\"G\":"; ival(k.G); o += ",";
  o += "\"fs_w\":"; ival(k.fs_w); o += ",";
  o += "\"sites\":[";
  for (size_t s = 0; s < H.sites.size(); ++s) {
    if (s) o += ",";
    o += "[";
    ival(H.sites[s].stride);
    o += ",";
    ival(H.sites[s].d);
    o += "]";
  }
  o += "],";
  marr("bmem", H.bmem);
  marr("rmem", H.rmem);
  iarr("bgrp", H.bgrp);
  iarr("rgrp", H.rgrp);
  darr("tab", H.tab);
  darr("dF", H.dF);
  darr("v", H.v);
  iarr("fix", H.fix);
  iarr("fs_n", H.fs_n);
  iarr("fs_off", H.fs_off);
  darr("fs", H.fs);
  o += "\"ok\":1}";
  return o;
}

}  // namespace hm
