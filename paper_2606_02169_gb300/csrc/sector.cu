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
//      cannot fail for a channel that conserves the digit sum;
//   4. y_F accumulates coefficient * x[source] (App. D step 4).
// Arithmetic as in the full-basis kernel (FP32, or double-float for FP64
// storage). Channels that do not conserve the digit sum are rejected when the plan is
// built (their sources lie outside the sector, so the projected operator
// would silently drop them).
#include <algorithm>
#include <cstring>
#include <vector>

#include "device_common.cuh"

namespace hm {

constexpr int kSecNT = 256;
constexpr size_t kSecTablesMax = 96 * 1024;  // tables staged in shared memory up to this size

// Table pointers of one launch (shared-memory copies, or the global tables).
template <class C>
struct SecTabs {
  const int* d;
  const long long* cnt;
  const long long* A;
  const int* Aoff;
  const KSecChan* ch;
  const C* tab;
};

__host__ __device__ inline size_t sec_align(size_t b) { return (b + 15) & ~size_t(15); }

// bytes of the staged tables (host and device agree on the layout)
__host__ __device__ inline size_t sec_tables_bytes(int N, int K, long long nA, int nch, long long ntab, size_t csize) {
  return sec_align((size_t)N * 4) + sec_align((size_t)(N + 1) * (K + 1) * 8) + sec_align((size_t)nA * 8) +
         sec_align((size_t)N * 4) + sec_align((size_t)nch * sizeof(KSecChan)) + sec_align((size_t)ntab * csize);
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

template <int AR>
__global__ void __launch_bounds__(kSecNT) k_sector(const KSector S, const typename SecAr<AR>::TX* __restrict__ x,
                                                   typename SecAr<AR>::TY* __restrict__ y, int nvec, long long nA,
                                                   long long ntab, int staged) {
  using P = SecAr<AR>;
  using C = typename P::C;
  using TX = typename P::TX;
  extern __shared__ __align__(16) unsigned char ssm[];
  const int N = S.N, K1 = S.K + 1;
  SecTabs<C> G{S.d, S.cnt, S.A, S.Aoff, S.ch, P::tab(S)};
  size_t o = 0;
  if (staged) {  // copy the tables once per CTA
    int* d = (int*)(ssm + o);            o += sec_align((size_t)N * 4);
    long long* cnt = (long long*)(ssm + o); o += sec_align((size_t)(N + 1) * K1 * 8);
    long long* A = (long long*)(ssm + o);   o += sec_align((size_t)nA * 8);
    int* Aoff = (int*)(ssm + o);          o += sec_align((size_t)N * 4);
    KSecChan* ch = (KSecChan*)(ssm + o);  o += sec_align((size_t)S.nch * sizeof(KSecChan));
    C* tab = (C*)(ssm + o);               o += sec_align((size_t)ntab * sizeof(C));
    for (int i = threadIdx.x; i < N; i += blockDim.x) { d[i] = S.d[i]; Aoff[i] = S.Aoff[i]; }
    for (int i = threadIdx.x; i < (N + 1) * K1; i += blockDim.x) cnt[i] = S.cnt[i];
    for (long long i = threadIdx.x; i < nA; i += blockDim.x) A[i] = S.A[i];
    for (int i = threadIdx.x; i < S.nch; i += blockDim.x) ch[i] = S.ch[i];
    for (long long i = threadIdx.x; i < ntab; i += blockDim.x) tab[i] = P::tab(S)[i];
    G = SecTabs<C>{d, cnt, A, Aoff, ch, tab};
    __syncthreads();
  }
  // per-thread digits and remaining totals (before each site)
  unsigned char* dig = ssm + o;                    // [N][blockDim]
  unsigned char* rem = dig + N * blockDim.x;       // [N][blockDim]
  const int t = threadIdx.x;
  auto Aat = [&](int k, int tt, int n) { return G.A[G.Aoff[k] + tt * (G.d[k] + 1) + n]; };
  for (long long F = blockIdx.x * (long long)blockDim.x + t; F < S.Dsec; F += (long long)gridDim.x * blockDim.x) {
    // 1. unrank
    long long r = F;
    int left = S.K;
    for (int k = 0; k < N; ++k) {
      const long long* c = G.cnt + (k + 1) * K1;
      int m = 0;
      while (true) {
        const long long cm = (left - m >= 0) ? c[left - m] : 0LL;
        if (r < cm) break;
        r -= cm;
        ++m;
      }
      dig[k * blockDim.x + t] = (unsigned char)m;
      rem[k * blockDim.x + t] = (unsigned char)left;
      left -= m;
    }
    // 2.-4. channels, up to 8 right-hand sides per pass; the diagonal
    // channels' coefficients are summed first and multiply x_F once
    for (int v0 = 0; v0 < nvec; v0 += 8) {
      const int nv = min(8, nvec - v0);
      typename P::Acc acc[8];
      for (int v = 0; v < nv; ++v) acc[v] = P::zero();
      typename P::Acc dsum = P::zero();
      for (int c = 0; c < S.nch; ++c) {
        const KSecChan ch = G.ch[c];
        const int ni = dig[ch.si * blockDim.x + t];
        const int nj = ch.sj >= 0 ? dig[ch.sj * blockDim.x + t] : 0;
        const C cf = G.tab[ch.tab + ni * ch.dj + nj];
        if (!P::nz(cf)) continue;
        if (ch.qi == 0 && ch.qj == 0) {
          P::add(dsum, cf);
          continue;
        }
        // rank terms of sites si..sj, target and source (sj > si)
        const int i = ch.si, j = ch.sj, q = ch.qi;
        const int ri = rem[i * blockDim.x + t];
        long long dlt = Aat(i, ri, ni - q) - Aat(i, ri, ni);
        for (int k = i + 1; k < j; ++k) {
          const int rk = rem[k * blockDim.x + t], nk = dig[k * blockDim.x + t];
          dlt += Aat(k, rk + q, nk) - Aat(k, rk, nk);
        }
        const int rj = rem[j * blockDim.x + t];
        dlt += Aat(j, rj + q, nj - ch.qj) - Aat(j, rj, nj);
        const TX* xs = x + (F + dlt) * nvec + v0;
        for (int v = 0; v < nv; ++v) P::fma(acc[v], cf, xs[v]);
      }
      const TX* xo = x + F * nvec + v0;
      typename P::TY* ys = y + F * nvec + v0;
      for (int v = 0; v < nv; ++v) ys[v] = P::out(acc[v], dsum, xo[v]);
    }
  }
}

void free_sector(Plan* p) {
  if (p->sec_dev) cudaFree(p->sec_dev);
  p->sec_dev = nullptr;
  p->ksec = KSector{};
}

int build_sector(Plan* p) {
  const int N = p->N;
  const long long Kl = p->sec_total;
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
  std::vector<int> dims(N), Aoff(N);
  std::vector<long long> A;
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
  std::vector<KSecChan> ch;
  std::vector<double> tab;
  std::vector<float> tabf;
  std::vector<float2> tabdf;
  auto split2 = [](double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
  };
  double cst = p->constant;
  for (const Channel& c : p->chH) {
    bool nz = false;
    for (auto& z : c.T) nz = nz || z != std::complex<double>(0, 0);
    if (!nz) continue;
    if (c.qi + (c.j >= 0 ? c.qj : 0) != 0) {
      set_error("the term list does not conserve the sector's digit sum (a channel moves it by " +
                std::to_string(c.qi + (c.j >= 0 ? c.qj : 0)) + ")");
      return HM_ERR_UNSUPPORTED;
    }
    KSecChan k{};
    k.tab = (int)tab.size();
    k.dj = c.dj;
    k.si = (int16_t)c.i;
    k.sj = (int16_t)(c.j >= 0 ? c.j : -1);
    k.qi = (int8_t)c.qi;
    k.qj = (int8_t)(c.j >= 0 ? c.qj : 0);
    for (auto& z : c.T) {
      tab.push_back(z.real());
      tabf.push_back((float)z.real());
      tabdf.push_back(split2(z.real()));
    }
    ch.push_back(k);
  }
  if (cst != 0.0) {  // identity terms: a diagonal channel on site 0 with value cst
    KSecChan k{};
    k.tab = (int)tab.size();
    k.dj = 1;
    k.si = 0;
    k.sj = -1;
    for (int n = 0; n < p->sites[0].dim; ++n) {
      tab.push_back(cst);
      tabf.push_back((float)cst);
      tabdf.push_back(split2(cst));
    }
    ch.push_back(k);
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
  const size_t o_d = add(dims.data(), dims.size() * 4);
  const size_t o_cnt = add(cnt.data(), cnt.size() * 8);
  const size_t o_A = add(A.data(), A.size() * 8);
  const size_t o_Aoff = add(Aoff.data(), Aoff.size() * 4);
  const size_t o_ch = add(ch.data(), ch.size() * sizeof(KSecChan));
  const size_t o_tab = add(tab.data(), tab.size() * 8);
  const size_t o_tabf = add(tabf.data(), tabf.size() * 4);
  const size_t o_tabdf = add(tabdf.data(), tabdf.size() * 8);
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
  S.Dsec = Dsec;
  S.N = N;
  S.K = K;
  S.nch = (int)ch.size();
  S.d = (const int*)(b + o_d);
  S.cnt = (const long long*)(b + o_cnt);
  S.A = (const long long*)(b + o_A);
  S.Aoff = (const int*)(b + o_Aoff);
  S.ch = (const KSecChan*)(b + o_ch);
  S.tab_d = (const double*)(b + o_tab);
  S.tab_f = (const float*)(b + o_tabf);
  S.tab_df = (const float2*)(b + o_tabdf);
  p->Dsec = Dsec;
  p->sec_nA = (long long)A.size();
  p->sec_ntab = (long long)tab.size();
  return HM_OK;
}

template <int AR>
static cudaError_t sector_launch(Plan* p, const void* x, void* y, long long nvec, cudaStream_t s) {
  using P = SecAr<AR>;
  const KSector& S = p->ksec;
  const size_t tabs = sec_tables_bytes(S.N, S.K, p->sec_nA, S.nch, p->sec_ntab, sizeof(typename P::C));
  const int staged = tabs <= kSecTablesMax;
  const size_t smem = (staged ? tabs : 0) + (size_t)2 * S.N * kSecNT;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_sector<AR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const long long need = (S.Dsec + kSecNT - 1) / kSecNT;
  const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)num_sms() * 8));
  k_sector<AR><<<grid, kSecNT, smem, s>>>(S, (const typename P::TX*)x, (typename P::TY*)y, (int)nvec, p->sec_nA,
                                          p->sec_ntab, staged);
  return cudaGetLastError();
}

int launch_sector(Plan* p, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s) {
  cudaError_t e;
  if (dt == HM_F32) {
    e = sector_launch<AR_F32>(p, x, y, nvec, s);
  } else {  // FP64: split into float pairs first
    const float2* xs = nullptr;
    Scratch xsb;
    int rc = split_vector(x, p->Dsec * nvec, s, xsb, &xs);
    if (rc) return rc;
    e = sector_launch<AR_DF64>(p, xs, y, nvec, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "sector apply launch");
  return HM_OK;
}

}  // namespace hm
