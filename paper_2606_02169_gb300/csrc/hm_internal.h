// Internal structures of the hm library (host plan + the POD block the
// kernels receive by value). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <map>
#include <set>
#include <cstdint>
#include <string>
#include <vector>

#include "hm.h"
#include "sector_types.h"

namespace hm {

constexpr int kMaxSites = 64;
constexpr int kLowBlockMax = 8192;  // low-digit block size bound (tables are O(B))
// elements (states x nvec) of one block of the staged kernel: one block of x
// fills one shared-memory slot (8 KB in FP64 storage)
constexpr int kStreamElems = 1024;
constexpr int kMaxDim = 65536;      // largest local dimension accepted
constexpr long long kMaxD = (1LL << 62) - 1;

// Channel kinds for the per-tile channel list (high/low split of the digits).
enum : uint8_t { CK_DIAG = 1, CK_SINGLE = 8 };

// Channel on tile-uniform ("high") digits only: coefficient tab[n_i * dj + n_j]
// indexed by TARGET digits, exactly zero where a source digit would leave
// [0, d-1], so a zero coefficient doubles as the admissibility test of
// Sec. IV.B. Its source offset is a multiple of the low-block size B.
struct KChan {
  long long off;   // source index = target index + off  (Eq. sourceoffset)
  int tab;         // base of this channel's table in the coefficient pool
  int dj;          // row length of the table (1 for single-site channels)
  uint8_t si, sj;  // sites (sj = 255: single-site)
  uint8_t kind;    // CK_* flags
  uint8_t pad[5];
};
static_assert(sizeof(KChan) == 24, "KChan layout");

// Channels on one high site h and one low site l whose coefficient factorises
// as u(n_h) * v(n_l) are grouped by their low factor v:
//   y_F += v(n_l(F)) * sum_{members m} u_m(n_h(F)) x_{F + off_m}
// so a hop costs one load and one FMA. v(n_l) = 0 marks an inadmissible low
// source digit, u_m(n_h) = 0 an inadmissible high one. A channel that does not
// factorise forms a group of its own whose v row is selected per block by the
// high digit (vstride > 0) and whose member has u = 1.
struct KGroup {
  int vtab;       // v table base in the pool
  int vstride;    // 0: fixed v; else v row = vtab + n_vsite * vstride
  int m0, m1;     // member range
  uint8_t vsite;  // high site selecting the v row (255: none)
  uint8_t lbit, lwid;  // low digit field
  uint8_t pad;
};
static_assert(sizeof(KGroup) == 20, "KGroup layout");

struct KMember {
  long long off;  // source offset (0 for diagonal groups)
  int utab;       // u table base, indexed by the digit of usite
  uint8_t usite;
  uint8_t pad[3];
};
static_assert(sizeof(KMember) == 16, "KMember layout");

// Per-term channel used by the adjoint/gradient pass: like KChan, but every
// site is resolved per lane (full digits), so it works for any split.
struct KTermChan {
  long long off;
  int tab;      // base in the per-term coefficient pool
  int dj;
  int term;     // term index t
  uint8_t si, sj;  // sites (sj = 255 for single-site)
  uint8_t pad[2];
};
static_assert(sizeof(KTermChan) == 24, "KTermChan layout");

struct KSite {
  long long mh;   // high sites: multiplier relative to the low block, M_k / B
  long long M;    // global multiplier M_k
  int d;
  uint8_t lbit, lwid, is_low, pad;
};

// Everything a kernel needs, passed by value (device pointers inside).
struct KPlan {
  long long D;      // dimension
  long long nblk;   // D / B
  int B;            // low-block size
  int nsites, nhigh;
  int n_hh_diag, n_hh;         // KChan list: [diag | off-diagonal]
  int n_grp_diag, n_grp;       // KGroup list: [diag | off-diagonal]
  int n_mem;                   // KMember list (all groups)
  int ell_w;                   // width of the low-block ELL table
  int nterm_ch;                // per-term channels (adjoint)
  int nterms;
  // second pass of a top-site split (general kernel only): tperm_T > 0
  // visits the low blocks with the digits of the leading tperm_T sites
  // varying fastest, so that the blocks a top-site hop connects are in
  // flight together; accum = 1 adds the result to y instead of storing it
  int tperm_T;
  int accum;
  // least common multiple, over the off-diagonal groups, of M_k d_k of the
  // group's low site k (the period of its digit in states; 0: no group)
  long long vperiod;
  const KSite* sites;     // [nsites]
  const KChan* ch;
  const KGroup* grp;
  const KMember* mem;
  const uint32_t* ptab;   // [B] packed low digits of each low index
  const int2* ell_pf;     // [ell_w * B] packed {delta, coef} (w-major), FP32
  const int4* ell_pdf;    // {delta, 0, coef.hi, coef.lo}, double-float
  const int4* ell_pd;     // {delta, 0, double coef}, native FP64
  const double* tab_d;    // coefficient pool (HH tables, u and v tables)
  const float2* tab_df;
  const float* tab_f;
  const double* diag_d;   // [B] diagonal from low-only channels (+ constants)
  const float2* diag_df;
  const float* diag_f;
  const KTermChan* tch;   // [nterm_ch]
  const double* ttab_d;   // per-term tables
  const float2* ttab_df;
  const float* ttab_f;
};

// ---------------------------------------------------------------------------
// Leaf-tiled form of the same operator (the "tile" kernel). The sites split
// into high | mid | leaf levels (most to least significant). A state index is
// k = (b * R + r) * F + f with block b (high digits), row r (mid digits) and
// leaf index f (leaf digits); with nvec right-hand sides the element index is
// k * nvec + v and a row holds F * nvec consecutive elements. One thread owns
// one leaf element f*nvec+v for all rows, so everything that depends on the
// leaf digits only is a per-thread constant, read once per CTA:
//   * the leaf part of the diagonal, dF(f);
//   * the hops between leaf sites ("leaf slots": offset, coefficient);
//   * the leaf factor v_g(f) of every group g >= 1 (below).
// Every other channel is a "member" whose coefficient u depends on high and
// mid digits only, so it is uniform across the CTA for a given (b, r):
//   y_k += sum_{g} v_g(f) * sum_{members m of g} u_m(b, r) x_{k + off_m}
// with v_0 = 1. Group g >= 1 collects the channels with one leaf site whose
// leaf factor (local diagonal of the leaf operator, Sec. IV.B) is v_g; their
// other site carries u. Zero factors are inadmissible digits (Sec. IV.B step
// 3): a zero u drops the member for the whole row; a zero v_g(f) redirects the
// thread's gathers of that group to an in-range element (fix_g) that is then
// scaled by exactly zero.
// ---------------------------------------------------------------------------
struct KTileSite {
  long long stride;  // high: in blocks; mid: in rows
  int d;
  int pad;
};

struct KTMem {
  long long off;   // element offset of the source (0 for diagonal members)
  int tab;         // coefficient table base: tab[n_a * db + n_b] over TARGET digits
  int db;          // row length (1: single-site table)
  uint8_t sa, sb;  // sites (index into KTile::sites; sb = 255: none)
  uint8_t grp;     // group (0: leaf factor 1)
  uint8_t diag;    // source offset 0
};
static_assert(sizeof(KTMem) == 24, "KTMem layout");

struct KTile {
  long long D;          // states
  long long nblk;       // blocks of R rows x F leaf states
  int F, R;             // leaf states per row, rows per block
  int nvec;             // right-hand sides the element offsets were built for
  int nt;               // threads per CTA: F * nvec rounded up to a warp
  int nhigh, nmid;      // sites [0, nhigh) high, [nhigh, nhigh + nmid) mid
  int G;                // groups including group 0
  int n_bmem, n_rmem;   // members on high sites only | with a mid site
  int fs_w;             // leaf-slot width (max over f)
  const KTileSite* sites;   // [nhigh + nmid]
  const KTMem* bmem;        // [n_bmem] sorted by group
  const KTMem* rmem;        // [n_rmem] sorted by group
  const int* bgrp;          // [G + 1] member ranges of bmem per group
  const int* rgrp;          // [G + 1] member ranges of rmem per group
  const double* tab;        // member coefficient tables
  // per-leaf-state tables (F entries each), one copy per arithmetic
  const double* dF_d; const float2* dF_df; const float* dF_f;
  const double* v_d;  const float2* v_df;  const float* v_f;   // [(G-1) * F]
  const int* fix;           // [(G-1) * F] element offset added when v = 0
  const int* fs_n;          // [F] leaf slots of each leaf state
  const int* fs_off;        // [fs_w * F] element offsets
  const double* fs_d; const float2* fs_df; const float* fs_f;  // [fs_w * F]
};

// Kernel tables of the staged apply kernel for one nvec (H and H^T), in a
// device allocation of their own.
// Top-site split of one plan (general kernel): pass A holds every term
// without an off-diagonal operator on the leading T sites (it writes y),
// pass B the others (it adds to y, visiting blocks top-digits-fastest).
// Built on first use per T.
struct SplitSet {
  bool ok = false;
  bool df_ok = true;                   // both passes' double-float windows are non-empty
  double df_xlo = 0.0, df_xhi = 0.0;   // their intersection
  KPlan ka{}, kat{}, kb{}, kbt{};      // pass A / pass B, H and H^T
  void* dev_a = nullptr;
  void* dev_b = nullptr;
};

struct StreamSet {
  bool ok = false;
  bool df_ok = true;   // the double-float input window is not empty
  double df_xlo = 0.0, df_xhi = 0.0;  // that window (see df_window)
  KPlan k{}, kt{};
  void* dev = nullptr;
  size_t bytes = 0;
};

// Launch choice of the apply kernel; 0 = library default for each field.
struct TuneCfg {
  int ctas = 0;  // persistent grid size
  int s = 0;     // elements per thread (rows of a chunk)
  int mb = 0;    // 1: register cap for one more resident CTA per SM
  int kern = 0;  // 0: library choice, 1: general kernel, 2: tile kernel, 3: staged kernel
  int strict = 0;  // 1: an explicit request (hm_apply_ex) -- no fallback
  // launch gate (device word): the kernel runs iff (*gate != 0) == gate_run;
  // NULL = always. Pairs a double-float launch with its native FP64 fallback.
  const int* gate = nullptr;
  int gate_run = 0;
  int presplit = 0;  // 1: FP64 input already holds float pairs (diagnostic timing)
  // general kernel: 0 = the plan's low block (B <= 8192 states), 1 = the
  // small low block of the staged tables (B * nvec <= 1024), whose per-plan
  // tables (ELL, diagonal, packed digits) stay in L1
  int small = 0;
  int pf = 0;  // general kernel: 1 = prefetch its gathers with cp.async (4 stages)
  // general kernel: 1 = one right-hand side per element even when nvec and
  // the vectors' alignment allow the 2- or 4-wide policies
  int scalar = 0;
  // general kernel: 1 = top-site split into two passes (SplitSet), with
  // split_T leading sites (0 = chosen from the vector size, split_top_sites)
  int split = 0;
  int split_T = 0;
  // general kernel: 1 = one v and member coefficients v u per thread where
  // every factorised group's low digit is the same for the thread's elements
  // (groups_invariant); rounds differently from 0
  int vinv = 0;
};

struct Channel {            // host-side merged channel
  int i = -1, j = -1;       // j = -1: single-site
  int qi = 0, qj = 0;       // n_target = n_source + q
  int di = 1, dj = 1;
  std::vector<std::complex<double>> T;  // [di*dj], target-digit indexed
  // the contributing products: T = sum_p a_p (x) b_p (coefficient folded into a)
  std::vector<std::pair<std::vector<std::complex<double>>, std::vector<std::complex<double>>>> parts;
};

struct Plan {
  uint32_t magic = 0x484d504cU;
  int device = 0;
  std::vector<hm_site> sites;
  std::vector<hm_term> terms;
  int N = 0;
  long long D = 0;
  std::vector<long long> M;
  bool hermitian = false;

  // split
  int nlow = 0, B = 1;
  long long nblk = 1;

  KPlan k{};    // H
  KPlan kt{};   // H^T (shares k's tables when H is symmetric)
  bool df_ok = true;  // the double-float input window is not empty
  double df_xlo = 0.0, df_xhi = 0.0;  // that window (see df_window)
  void* dev = nullptr;        // one device allocation holding every table
  size_t dev_bytes = 0;

  // scratch for the adjoint reduction (grown on demand)
  void* scratch = nullptr;
  size_t scratch_bytes = 0;

  // complex H = H_re + i H_im (imaginary matrix elements from Sy factors):
  // this plan holds H_re (part 0), `im` the companion plan holding H_im
  // (part 1); both are real operators on the kernels above
  int part = 0;
  bool complex_h = false;     // the term list has imaginary matrix elements
  bool hermitian_c = false;   // H^dagger = H for the complex operator
  Plan* im = nullptr;
  bool grad_ok = true;        // every term's operator is real (coupling gradients defined)

  // fixed digit-sum sector (hm_create_sector): vectors hold the Dsec
  // retained states instead of all D
  bool sector = false;
  long long sec_total = 0;
  long long Dsec = 0;
  KSector ksec{};
  void* sec_dev = nullptr;
  // block form of the sector apply (sector_blk.cu), when the plan fits it
  KSecBlk ksb{};
  void* secb_dev = nullptr;
  bool secb_ok = false;
  long long sec_nA = 0, sec_ntab = 0;   // rank-table and coefficient-pool lengths
  long long sec_ndl = 0;                // rank-delta pool length
  bool sec_needA = true;                // some channel updates ranks from the rank tables

  // merged channels of H and H^T (H^T empty when H is symmetric) and the
  // identity part, kept for building tile tables per nvec
  std::vector<Channel> chH, chT;
  double constant = 0.0;
  // tile tables per (nvec, transpose); device memory owned here. A plan whose
  // shape has no tile form records that with ok = false.
  struct TileSet {
    bool ok = false;
    KTile k{};
    void* dev = nullptr;
  };
  std::map<std::pair<long long, int>, TileSet> tiles;

  // staged-kernel (and small-block) tables per nvec, built on first use
  std::map<long long, StreamSet> streams;
  // top-site splits per number of top sites T, built on first use
  std::map<int, SplitSet> splits;

  // autotuned launch choice per (dtype, nvec); absent = default
  std::map<std::pair<int, long long>, TuneCfg> tuned;
  // complex H: the form the autotuner measured fastest per (dtype, nvec):
  // 0 the one-pass complex kernel, 1 its register-capped variant, 2 two
  // tuned real passes and the combine
  std::map<std::pair<int, long long>, int> cx_form;

  // batch handle
  bool is_batch = false;
  std::vector<Plan*> members;
  unsigned long long gen = 0;   // bumped by every (re)build of the tables
};

// plan.cpp
int build_plan(Plan* p);            // (re)derive tables from sites/terms and upload
void free_plan_device(Plan* p);
// staged-kernel tables for nvec (NULL: no staged form, or not buildable now,
// e.g. during stream capture; then *deferred = true)
const StreamSet* get_stream(Plan* p, long long nvec, cudaStream_t s, bool* deferred = nullptr);
void free_streams(Plan* p);
// top-site split with T leading sites (NULL: no split form for T, or not
// buildable now, e.g. during stream capture)
const SplitSet* get_split(Plan* p, int T, cudaStream_t s);
void free_splits(Plan* p);
// number of leading sites whose hops a split moves to its second pass for
// vectors of es-byte elements and nvec right-hand sides (0: no split)
int split_top_sites(const Plan* p, long long nvec, size_t es);

// sector.cu
int build_sector(Plan* p);   // sector tables from p->chH (after build_plan's host half)
void free_sector(Plan* p);
std::string export_sector_json(const Plan* p, long long digit_total, int* rc);
int launch_sector(Plan* p, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s,
                  bool rows = false);
// sector_blk.cu: block-form tables (none when the plan does not fit them)
// and its launch on x already split into float pairs for FP64 storage
int build_sector_blk(Plan* p);
std::string export_sector_blk_json(const Plan* p, long long digit_total, int* rc);
void free_sector_blk(Plan* p);
cudaError_t launch_sector_blk(const Plan* p, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s);
// length of the plan's vectors in states: D, or Dsec for a sector plan
inline long long vec_states(const Plan* p) { return p->sector ? p->Dsec : p->D; }

// tile_plan.cpp
struct HostTile;
int derive_tile(const Plan* p, const std::vector<Channel>& ch, double constant, long long nvec, HostTile& out);
// tile tables for (nvec, transpose), built and uploaded on first use; NULL
// when the plan has no tile form (or cannot be built right now, e.g. during
// stream capture)
const KTile* get_tile(Plan* p, long long nvec, bool transpose, cudaStream_t s);
void free_tiles(Plan* p);
std::string export_tile_json(const Plan* p, const std::vector<Channel>& ch, double constant, long long nvec,
                             int* rc);
int plan_check(const Plan* p);

// error text (capi.cpp)
void set_error(const std::string& s);
int cuda_fail(cudaError_t e, const char* what);

// kernels (apply.cu / adjoint.cu / lanczos.cu / batch.cu)
int launch_apply(Plan* p, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s, TuneCfg cfg);
int apply_on(Plan* p, bool transpose, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s,
             TuneCfg cfg, bool native_f64);
TuneCfg tuned_cfg(Plan* p, hm_dtype dt, long long nvec);
// Stream-ordered device scratch from a library-owned pool that keeps its
// memory between calls; released on the same stream when the owner goes out
// of scope (after the launches that read it were queued).
struct Scratch {
  void* ptr = nullptr;
  cudaStream_t s = nullptr;
  Scratch() = default;
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  ~Scratch() {
    if (ptr) cudaFreeAsync(ptr, s);
  }
};
int scratch_alloc(Scratch& b, size_t bytes, cudaStream_t s);
void scratch_trim();
// n FP64 values split into float pairs in fresh scratch `b`. With range !=
// NULL the split also zeroes and then sets *range (a word in the same
// scratch) when some element is outside [xlo, xhi) (zero excepted; a
// subnormal, Inf or NaN is always outside).
int split_vector(const void* x, long long n, cudaStream_t s, Scratch& b, const float2** out,
                 const int** range = nullptr, double xlo = 0.0, double xhi = 0.0);
// input window [lo, hi) of the double-float arithmetic for a plan whose
// nonzero coefficients span [cmin, cmax] (plan.cpp)
void df_window(double cmin, double cmax, double* lo, double* hi);
// y = H x (or H^dagger x when adjoint) for nvec complex right-hand sides of a
// complex plan, dt the real type of the (re, im) pairs
// Complex H (this plan H_re, p->im H_im) on nvec complex right-hand sides
// (dt the real dtype of their parts). mode 0: the form hm_tune chose (else
// kCxDefaultForm), two passes where the one-pass kernel is not available;
// 1: two passes of the general kernel's default launch; 2: the one-pass
// kernel (cap: its register-capped variant) or HM_ERR_UNSUPPORTED; 3: two
// passes with each part's tuned launch. native: FP64 arithmetic throughout.
int apply_complex(Plan* p, bool adjoint, const void* x, void* y, long long nvec, hm_dtype dt, cudaStream_t s,
                  int mode = 0, bool native = false, int ctas = 0, bool cap = false);
int launch_adjoint(Plan* p, const void* gy, const void* x, void* gx, double* gcoef,
                   long long nvec, hm_dtype dt, cudaStream_t s);
// Lanczos on vectors of vec_states * nvec elements of the real dtype dt
// (nvec = 2 for a complex vector of a real H)
int run_lanczos(Plan* p, const void* v0, int steps, hm_dtype dt, long long nvec, int flags, double* alpha,
                double* beta, int* steps_done, void* psi0, double* e0, cudaStream_t s);
// y = exp(-i t H) x for one complex vector stored as interleaved pairs of dt
int run_evolve(Plan* p, const void* x, void* y, double t, int m, int nsub, int flags, hm_dtype dt, double* err,
               cudaStream_t s);
// c[k] = nu [exp(-i tau T) e_1]_k, (re, im) pairs, T = tridiag(b, a, b)
void krylov_coeffs(const std::vector<double>& a, const std::vector<double>& b, double tau, double nu,
                   std::vector<double>& c);
int batch_setup(Plan* b);
int launch_batch(Plan* b, const void* const* xs, void* const* ys, long long nvec, hm_dtype dt,
                 cudaStream_t s);
int num_sms();
// status words of the staged kernel's translation units on the current device
int stream_status_f32(int* out, bool clear);
int stream_status_df64(int* out, bool clear);
int stream_status_f64(int* out, bool clear);

}  // namespace hm
