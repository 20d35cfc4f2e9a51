// Device tables of a fixed digit-sum sector plan (hm_create_sector).
#pragma once

#include <vector_types.h>

#include <cstdint>

namespace hm {

// ---------------------------------------------------------------------------
// Fixed digit-sum sector (Sec. VI case 2, App. D): retained states are the
// digit tuples with sum_k n_k = K, packed in ascending full-index order. The
// packed index of a tuple is its combinatorial rank
//   rank(n) = sum_k A_k[K - P_k][n_k],   P_k = n_0 + ... + n_{k-1},
//   A_k[t][n] = sum_{m<n} cnt_{k+1}[t - m],
// with cnt_k[t] the number of digit tuples of sites k..N-1 summing to t.
// A hop that changes sites i < j by -q_i, -q_j (q_i + q_j = 0) changes only
// the terms of sites i..j, so the source rank is the target's plus O(j-i+1)
// table differences: the lookup of Sec. VI without a search.
// ---------------------------------------------------------------------------
struct alignas(16) KSecChan {
  int tab;         // coefficient table base, entry [n_i * dj + n_j] (target digits)
  int dtab;        // rank-delta table base for a move on adjacent sites,
                   // entry [rem_i * rstride + n_i * dj + n_j]; -2 - off: long
                   // move, per-site entries at off in the long-move pool;
                   // -1: rank update from the rank tables
  int rstride;     // d_i * dj (long move: the per-site digit stride)
  int dj;          // d_j (1 for a single-site channel)
  int si, sj;      // sites (sj = -1: single-site)
  int q;           // n_target - n_source on site si (the opposite on sj)
  int diag;        // q = 0 on both sites
};
static_assert(sizeof(KSecChan) == 32, "KSecChan layout");

struct KSector {
  long long Dsec;          // retained states
  int N, K;                // sites, digit total
  int nch;                 // channels (all conserve the digit sum)
  int ndiag;               // the first ndiag channels are diagonal
  int wide;                // rank deltas stored as int64 (else int32)
  const int* d;            // [N] local dimensions capped at K + 1 (rank-table strides)
  const long long* cnt;    // [(N + 1) * (K + 1)] cnt_k[t] at k * (K + 1) + t
  const long long* A;      // rank tables, site k at Aoff[k]: [t * (d_k + 1) + n]
  const int* Aoff;         // [N]
  const KSecChan* ch;      // [nch]
  const double* tab_d;     // coefficient pool
  const float* tab_f;
  const float2* tab_df;    // as float pairs (double-float arithmetic)
  const void* dl;          // rank-delta pool (int32 or int64 entries)
  // moves spanning non-adjacent sites ("long" moves): the rank change is a
  // sum over sites si..sj of per-site entries, for the channel with
  // dtab = -2 - off at lt[off + ((k - si) * (K + 1) + rem_k) * rstride + n_k]
  const void* lt;          // long-move pool (int32 or int64 entries)
  long long nlt;           // its length
};

enum { SB_PDIAG = 0, SB_MDIAG = 1, SB_PMOVE = 2, SB_MMOVE = 3 };

struct KSBChan {
  int kind;
  int tab;         // coefficient table base, entry [n_si * dj + n_sj] (target digits)
  int dj;
  int si, sj;      // sites (sj = -1: single-site)
  int pfx;         // SB_M*: 0 if si is the prefix site, 1 if sj is
  int qp;          // SB_PMOVE: unused; SB_MMOVE: move of the prefix digit (source = target - qp)
  int xr;          // SB_MMOVE: index of its source-rank table
  long long dblk;  // moves: source block = block - dblk
  int lbit, lwid;  // SB_M*: packed-digit field of the suffix site
};

// Block form (sector_blk.cu): prefix blocks of contiguous packed states,
// per-suffix tables. Channels in kind order: [0, n0) SB_PDIAG, [n0, n1)
// SB_PMOVE, [n1, n2) SB_MDIAG, [n2, nch) SB_MMOVE.
struct KSecBlk {
  long long nvb;           // blocks with retained states
  int h, K, nch, w, G;
  int n0, n1, n2;
  const long long* start;  // [prefix tuples] packed index of the block's first state
  const int* vb;           // [nvb] those blocks, ascending
  const long long* mp;     // [h] prefix multipliers (block units)
  const int* pdim;         // [h] prefix site dimensions
  const int* off;          // [K + 2] suffix-sector offsets (positions g)
  const uint32_t* sdig;    // [G] packed suffix digits
  const KSBChan* ch;       // [nch]
  const double* tab_d;
  const float2* tab_df;
  const float* tab_f;
  const double* dS_d;      // [G] suffix-only diagonal (+ constant)
  const float2* dS_df;
  const float* dS_f;
  const int* ell_r;        // [w * G] source rank - target rank (same sector)
  const double* ell_d;     // [w * G] coefficients
  const float2* ell_df;
  const float* ell_f;
  const int* xr;           // [nxr * G] source ranks of coupled moves
};

}  // namespace hm
