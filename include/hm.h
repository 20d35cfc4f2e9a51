/*
 * hm.h -- C ABI of the GB300 matrix-free spin / truncated-boson Hamiltonian
 * library (y = H x on the full tensor-product basis, mixed-radix indexed).
 *
 * Operation (from "Spin Hamiltonian as Matrix-Free Linear Map"):
 *   sites k = 0..N-1 with local dimension d_k (spin: d = 2s+1, Sec. I Eq. 1;
 *   truncated boson: d = n_max+1, App. C). Basis index
 *     I = sum_k n_k M_k,  M_k = prod_{l>k} d_l           (Sec. III Eq. encode)
 *   site 0 is the MOST significant digit; local digit n = m + s, so n = 0 is
 *   m = -s (Sec. II notation guide). Bosons: n = occupation.
 *   H = sum_t coef_t op_i(t)(site i) op_j(t)(site j)    (Sec. IV Eq. pairham,
 *   App. B higher powers, App. C spin-boson terms), applied target-driven:
 *     y_F = <F|H|x> = sum over channels of coef * Lambda * Lambda * x_{F+offset}
 *   (Sec. II, Sec. IV.B Eq. sourceoffset, App. A).
 *
 * Vectors: caller-owned DEVICE pointers (hm_apply also takes page-locked
 * host memory, see there), state-major interleaved: element v
 * of state k is at [k*nvec + v]. Real storage (HM_F64 / HM_F32) or complex
 * storage (HM_C128 / HM_C64: each element an interleaved (re, im) pair, the
 * layout of C99 double/float _Complex). For a real H the real and imaginary
 * parts of a complex vector are applied independently: a complex call with
 * nvec right-hand sides is the real call with 2*nvec interleaved right-hand
 * sides on the same memory (same kernels, same results); hm_apply,
 * hm_apply_ex, hm_apply_adjoint, hm_coupling_gradients_static,
 * hm_batch_apply, hm_tune, hm_tuned_config and hm_lanczos accept complex
 * dtypes, hm_evolve requires one. A term list with imaginary matrix
 * elements (Sy factors: a lone Sy, Sx Sy, ...) gives a complex H = H_re +
 * i H_im, held as two real operators on the same sites: y = H_re x +
 * i H_im x runs as two real applies of the 2*nvec columns and one
 * combining pass, or, where hm_tune measured it faster, as one pass in
 * which a thread forms both operators' sums for each (re, im) element and
 * combines them in registers (one read of the state's digits, one write of
 * y; it needs x and y aligned to one complex element, 8 or 16 bytes,
 * HM_C64 x in device memory and both operators' block lists within shared
 * memory, else the two passes run). With the general kernel in both real
 * passes the two forms give the same bits. Such
 * plans need complex storage (real dtypes give HM_ERR_COMPLEX_REQUIRED)
 * and support hm_apply, hm_apply_ex (flag bits 0, 1, 4 and 13, see
 * there), hm_apply_adjoint (gx = H^dagger gy only), hm_lanczos, hm_evolve,
 * hm_tune, hm_set_coefficients; coupling gradients, batches and sectors
 * return HM_ERR_UNSUPPORTED.
 * Every call is asynchronous on the given CUDA stream (NULL = legacy default
 * stream) unless stated otherwise. Plans are library-owned. Applies of one
 * plan (hm_apply, hm_batch_apply) may run on several streams at once: the
 * FP64 input split takes per-call scratch (see hm_apply), and hm_lanczos
 * allocates its own vectors. Adjoint passes share a plan-owned reduction
 * buffer, so adjoint calls of one plan must not overlap on the GPU.
 * hm_set_coefficients must not overlap any call of the same plan.
 *
 * Errors: every int-returning call returns HM_OK (0) or a negative HM_ERR_*;
 * hm_strerror() names a code and hm_last_error() returns a thread-local text
 * with details of the most recent failure on the calling thread.
 */
#ifndef HM_H
#define HM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hm_plan* hm_handle;

/* site kinds */
enum { HM_SPIN = 0, HM_BOSON = 1 };

typedef struct {
    int32_t kind;  /* HM_SPIN or HM_BOSON */
    int32_t dim;   /* spin: 2s+1 >= 2; boson: n_max+1 >= 2 */
} hm_site;

/* local operators (Sec. IV.A, App. B, App. C) */
enum {
    HM_ID = 0,   /* identity                                          */
    HM_SZ = 1,   /* S_z                                  (q = 0)       */
    HM_SX = 2,   /* S_x = (S+ + S-)/2   (Sec. IV.A h_+- split)          */
    HM_SY = 3,   /* S_y = (S+ - S-)/(2i); imaginary alone: needs pairing */
    HM_SP = 4,   /* S_+                                  (q = +1)      */
    HM_SM = 5,   /* S_-                                  (q = -1)      */
    HM_SZ2 = 6,  /* S_z^2                                (App. B q = 0)*/
    HM_SP2 = 7,  /* S_+^2                                (App. B q = +2)*/
    HM_SM2 = 8,  /* S_-^2                                (App. B q = -2)*/
    HM_N = 9,    /* boson a^dagger a                     (App. C)      */
    HM_A = 10,   /* boson a                              (q = -1)      */
    HM_ADAG = 11 /* boson a^dagger                       (q = +1)      */
};

/* One term: coef * op_i(site_i) * op_j(site_j); site_j = -1 for a
 * single-site term (op_j ignored). site_i != site_j. Duplicates add. */
typedef struct {
    int32_t site_i, op_i, site_j, op_j;
    double coef;
} hm_term;

typedef enum { HM_F64 = 0, HM_F32 = 1, HM_C128 = 2, HM_C64 = 3 } hm_dtype;

/* return codes */
enum {
    HM_OK = 0,
    HM_ERR_INVALID_ARG = -1,      /* bad site/op kind, i == j, null pointer, nvec < 1 */
    HM_ERR_OVERFLOW = -2,         /* D >= 2^62                                      */
    HM_ERR_ALIAS = -3,            /* x and y overlap                                */
    HM_ERR_COMPLEX_REQUIRED = -4, /* real storage asked of a complex H              */
    HM_ERR_NOT_HERMITIAN = -5,    /* Lanczos on a non-self-adjoint term list        */
    HM_ERR_CUDA = -6,             /* CUDA runtime error (text in hm_last_error)      */
    HM_ERR_OOM = -7,              /* device allocation failed                       */
    HM_ERR_TIMEOUT = -8,          /* a bounded device wait gave up                  */
    HM_ERR_UNSUPPORTED = -9,      /* shape outside the implemented limits           */
    HM_ERR_TOO_LARGE = -10,       /* size above a documented fixed maximum          */
    HM_LANCZOS_BREAKDOWN = 1      /* warning: Krylov space exhausted early          */
};

/* Build a plan (host call; allocates the plan's small device tables on the
 * current device and synchronises). sites[nsites], terms[nterms] are read and
 * copied. Limits: 1 <= nsites <= 64, D = prod d_k < 2^62, each d_k <= 65536.
 * Cost O(N + |terms|) plus O(B) tables for the low-digit block (B <= 8192).
 * A term list with imaginary matrix elements builds a complex plan (two real
 * operators, see Vectors above). */
int hm_create(const hm_site* sites, int32_t nsites, const hm_term* terms, int32_t nterms,
              hm_handle* out);

/* Plan restricted to a globally constrained sector (Sec. VI case 2, App. D):
 * the retained basis is every digit tuple with sum_k n_k = digit_total (for
 * spins the fixed magnetization M = digit_total - sum_k s_k; for spin-boson
 * models the excitation number), packed in ascending full-basis order, and
 * vectors hold those hm_dim(h) retained states (state-major, nvec values
 * each). A source's packed index is found by combinatorial ranking, updated
 * per hop from the target's (no search). Every term must conserve the digit
 * sum (else HM_ERR_UNSUPPORTED); digit_total outside [0, sum_k (d_k - 1)]
 * gives HM_ERR_INVALID_ARG, above 255 HM_ERR_UNSUPPORTED. hm_apply,
 * hm_set_coefficients, hm_lanczos, hm_evolve, hm_dim, hm_num_terms and
 * hm_destroy accept sector plans (arithmetic as in hm_apply);
 * hm_apply_adjoint gives gx = H^T gy = H gy for a symmetric term list (no
 * gcoef); hm_apply_ex, hm_coupling_gradients_static, hm_tune, batches and
 * complex term lists return HM_ERR_UNSUPPORTED. */
int hm_create_sector(const hm_site* sites, int32_t nsites, const hm_term* terms, int32_t nterms,
                     int64_t digit_total, hm_handle* out);

/* Replace all term coefficients (host array of nterms doubles) without
 * re-planning (Sec. VII: repeatedly rebuilt Hamiltonians). Synchronous. The
 * new list must not make any matrix element imaginary; channels whose
 * coefficient was exactly zero at create time stay present. */
int hm_set_coefficients(hm_handle h, const double* coefs);

/* D = prod d_k (Sec. I Eq. 1), or a negative code for a NULL handle. */
int64_t hm_dim(hm_handle h);
int32_t hm_num_terms(hm_handle h);

/* y = H x for nvec right-hand sides (x, y: D*nvec elements of dtype in
 * device memory or in page-locked host memory registered with CUDA --
 * cudaHostAlloc / cudaHostRegister -- which the kernels reach over the
 * CPU-GPU link: FP64 x is read once by the split pass, FP32 x is copied once
 * into device scratch, y is written once; plain pageable host memory gives
 * HM_ERR_INVALID_ARG; x read-only, y fully overwritten; x and y must not
 * overlap). Each output
 * element is owned by exactly one GPU lane (pull form, Sec. II): no atomics,
 * bit-reproducible run to run. HM_F64 first splits x into D*nvec float
 * pairs of stream-ordered scratch from a library memory pool per device,
 * released on the same stream after the apply; the pool keeps freed memory
 * for later calls (hm_destroy hands the unused part back). Inside a stream
 * capture the scratch becomes the graph's own allocation.
 * FP64 arithmetic: by default a double-float sum on the FP32 pipe (error-free
 * products and sums, ~2^-46 relative per product), valid while every
 * product of a nonzero input and a nonzero coefficient (merged table entry,
 * magnitudes in [cmin, cmax]) stays in [2^-100, 2^120): the plan's input
 * window is |x| in [max(2^-100, 2^-100/cmin), min(2^126, 2^120/cmax)), plus
 * x = 0. The split pass checks x on the device: if any element is outside
 * (or subnormal, Inf, NaN) the double-float launch stands down and a second
 * launch queued behind it computes the same call in native FP64, so results
 * keep FP64's range for every input; a plan whose window is empty always
 * computes in native FP64. Merged coefficients whose terms cancel to within
 * 16 ulps of the largest contribution are exactly zero.
 * nvec a multiple of 4 (FP32) or 2 (FP32, FP64 double-float) with x and y
 * aligned to 4 or 2 elements: each lane of the general kernel handles that
 * many consecutive right-hand sides of one state (wider loads, one decode
 * and one coefficient per state); results are bit-identical to one
 * right-hand side per lane.
 * Kernel: the general kernel (block-uniform hops as coalesced gathers, hops
 * inside the low block from a per-plan table) unless hm_tune chose another
 * launch: a variant of the general kernel (elements per thread, register
 * cap, prefetching, one group factor per lane, the top-site split into two
 * passes, one right-hand side per lane), the general kernel on a small low
 * block, the leaf-tiled kernel, or the staged kernel (each hop's source
 * range streamed into shared memory by bulk asynchronous copies; its
 * bounded waits report to hm_device_status). The small-block, split, tile
 * and staged forms build extra tables on their first call for each nvec
 * (or split size), which hm_tune makes; a first call inside a stream capture
 * runs the general kernel's default instead. */
int hm_apply(hm_handle h, const void* x, void* y, int64_t nvec, hm_dtype dtype, void* stream);

/* Diagnostic variant of hm_apply (it ignores hm_tune's choice). flags
 * bit 0: native FP64 arithmetic for HM_F64 (default: FP64 values split into
 * FP32 pairs, accumulated as a double-float sum with error-free
 * transformations; ~2^-46 relative); bit 1: apply H^T instead of H; bit 2:
 * register-capped general kernel (one more resident CTA per SM); bit 3: the
 * leaf-tiled kernel (HM_ERR_UNSUPPORTED if the plan has no tile form for
 * this nvec); bit 4: the general kernel; bit 5: the staged kernel
 * (HM_ERR_UNSUPPORTED if the plan has no staged form for this nvec); bits
 * 8..11: rows per iteration of the tile kernel (1, 2, 4) or elements per
 * thread of the general kernel (2, 3, 4, 6, 8), 0 = default, anything else
 * HM_ERR_INVALID_ARG. At most one of bits 3, 4, 5; without them the general
 * kernel runs. Bit 6 (timing diagnostic, HM_F64 without bit 0): x already
 * holds each value as a float pair (hi, lo) with hi + lo equal to the double
 * within 2^-46 relative; the split pass and its range check are skipped and
 * only the double-float apply kernel runs. Bit 7 (general kernel only): use
 * the small low block (B * nvec <= 1024 states, the staged kernel's split)
 * whose per-plan tables stay in L1. Bit 12 (general kernel only): prefetch
 * each thread's gathers four hops ahead with per-thread asynchronous copies
 * into shared memory (elements per thread 4, 6 or 8). Bit 13 (general
 * kernel only): one right-hand side per lane even where hm_apply would
 * process 2 or 4 per lane (bit-identical either way). Bit 14 (general
 * kernel, not with bits 0 or 7): top-site split -- the terms with an
 * off-diagonal operator on one of the leading T sites run as a second pass
 * that adds to y and visits the low blocks with those T digits varying
 * fastest, so that each pass reads x from DRAM about once; T = bits
 * 16..19, or 0 for every leading site whose hop distance M_k * nvec * element
 * size is at least 32 MiB (at most 512 digit combinations).
 * HM_ERR_UNSUPPORTED when the plan has no such split (no term moves a
 * leading digit, a pass would be empty, or a leading site lies in the low
 * block). Results differ from the one-pass kernel by rounding only (each
 * pass rounds once). Bit 15 (general kernel): where every factorised
 * high/low group's low digit is the same for all elements a lane handles
 * (its period M_k d_k divides their stride), one group factor v per lane
 * and member coefficients v*u formed once per lane instead of
 * v * sum(u x) per element (fewer registers and operations; rounds
 * differently, within the same tolerance); ignored elsewhere. ctas > 0
 * forces the persistent grid size (0 = library default).
 * A complex H (complex storage only) takes bits 0, 1 (H^dagger = H_re^T -
 * i H_im^T), 2, 4 (no effect) and 13; other bits give HM_ERR_UNSUPPORTED.
 * Without bit 13 the one-pass complex kernel runs, with bit 2 its
 * register-capped variant (three resident CTAs per SM) (HM_ERR_UNSUPPORTED
 * where it is not available, see Vectors above); with bit 13, two real
 * applies of the general kernel's default launch and the combining pass.
 * All three give the same bits.
 * Same ownership and error rules as hm_apply. */
int hm_apply_ex(hm_handle h, const void* x, void* y, int64_t nvec, hm_dtype dtype, int32_t flags,
                int32_t ctas, void* stream);

/* Adjoint / gradient pass (reverse mode of y = H(c) x):
 *   gx[k*nvec+v] = (H^T gy)                     if gx != NULL (overwritten)
 *   gcoef[t]     = sum_v <gy_v| O_t |x_v>        if gcoef != NULL (device,
 *                  nterms doubles, overwritten), O_t = op_i op_j without coef.
 * gy, x: device vectors of dtype. gcoef is always FP64, reduced
 * deterministically (fixed-order two-pass reduction, no atomics). For
 * complex dtypes gcoef[t] = Re sum_v <gy_v| O_t |x_v> (the real and
 * imaginary parts as separate real columns), the gradient of a real loss
 * L(y) with gy = dL/dRe(y) + i dL/dIm(y), coefficients being real. Uses
 * plan-owned scratch of O(nterms * grid) doubles, grown on demand (so the
 * first call of a size should come before any stream capture) and, for
 * HM_F64, per-call pool scratch as in hm_apply for gy and x split once.
 * Calls on the same plan must not overlap on the GPU. gcoef gives
 * HM_ERR_UNSUPPORTED when a term's own operator has imaginary elements
 * (its real gradient is undefined), e.g. a Sy term with zero coefficient. */
int hm_apply_adjoint(hm_handle h, const void* gy, const void* x, void* gx, double* gcoef,
                     int64_t nvec, hm_dtype dtype, void* stream);

/* Coupling gradients gcoef[t] = sum_v <gy_v| O_t |x_v> -- what
 * hm_apply_adjoint returns with gx = NULL -- without allocating device memory.
 * The paper has no counterpart: this serves callers that cannot let the
 * library call cudaMalloc, such as code running while a stream is captured
 * into a CUDA graph, or a process whose device memory is owned by another
 * allocator (a framework's caching pool, a fixed serving budget).
 * The per-CTA partial sums live in one file-scope device array of 131072
 * doubles (1 MiB) that every GPU loading the library holds until the process
 * exits; the grid is capped so that grid * nterms <= 131072. A term list
 * longer than 131072 returns HM_ERR_TOO_LARGE; one longer than 3200 returns
 * HM_ERR_UNSUPPORTED (shared-memory limit of the reduction). The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current: make it before any stream capture. Every call
 * shares the array, so calls that overlap on the GPU race; each call writes
 * every partial it reads, so nothing is cleared between calls. gy, x: device
 * vectors of dtype, aligned to the element size (gy == x allowed); gcoef:
 * device, nterms doubles, 8-byte aligned, overwritten. The plan's device
 * must be current (else HM_ERR_INVALID_ARG); the vector checks of
 * hm_apply_adjoint apply (nvec <= 2^19, D * nvec within int64). */
int hm_coupling_gradients_static(hm_handle h, const void* gy, const void* x, double* gcoef,
                                 int64_t nvec, hm_dtype dtype, void* stream);

/* Status word of the current device's kernels (no counterpart in the paper).
 * Synchronises the device, then *status = the bits set since the last clear:
 * bit 0 = a bounded wait inside the staged apply kernel gave up (the CTA left
 * its blocks unwritten; results of that call are invalid). clear != 0 resets
 * the word. */
int hm_device_status(int32_t* status, int32_t clear);

/* Lanczos ground state (Sec. I: Krylov solvers need only y = H x).
 * v0: device start vector (D elements of dtype, need not be normalised).
 * Runs up to `steps` steps; alpha/beta (host, >= steps doubles) receive the
 * tridiagonal matrix (FP64 dot products even for HM_F32 storage), *steps_done
 * the number of alpha values, *e0 the lowest Ritz value (FP64 host
 * tridiagonal eigensolver). If psi0_out (device, D elements) is not NULL the
 * recurrence is re-run from v0 to assemble the normalised Ritz vector without
 * storing the Krylov basis. Synchronous on `stream`. flags: bit 0 = local
 * reorthogonalisation against v_{k-1} and v_k (default off = plain
 * three-term recurrence). Returns HM_LANCZOS_BREAKDOWN (> 0) when beta_k
 * falls below 1e-14 |alpha|max before `steps`. Allocates 3 (4 with psi0)
 * work vectors per call. A complex v0 (HM_C128 / HM_C64) runs the same
 * recurrence with the Hermitian inner product (alpha and beta stay real). */
int hm_lanczos(hm_handle h, const void* v0, int32_t steps, hm_dtype dtype, int32_t flags,
               double* alpha, double* beta, int32_t* steps_done, void* psi0_out, double* e0,
               void* stream);

/* Time evolution y = exp(-i t H) x (hbar = 1) of one complex vector (Sec. VII:
 * exact propagation under time-dependent or repeatedly rebuilt couplings;
 * Sec. VIII: Krylov methods need only y = H x). Short-iterative Lanczos
 * propagator (Park and Light, 1986): t is split into nsub equal steps tau;
 * each builds an m-step Lanczos basis V_m (T_m = V_m^H H V_m tridiagonal,
 * real) from the current vector u and sets u <- |u| V_m exp(-i tau T_m) e_1,
 * the small exponential from a Jacobi eigendecomposition on the host.
 * x, y: device, hm_dim(h) complex values of dtype HM_C128 or HM_C64 (x
 * read-only, y overwritten, no overlap). 1 <= m <= 128, nsub >= 1, t
 * finite (negative t runs backwards). flags bit 0: local
 * reorthogonalisation as in hm_lanczos; bit 1: rebuild the basis in a second
 * pass of the recurrence instead of storing it (by default the m basis
 * vectors are stored when they fit in half the free device memory; both ways
 * give the same y bit for bit). err (host, nullable): sum over the steps of
 * the a-posteriori estimate beta_m |[ |u| exp(-i tau T_m) e_1 ]_m| of the
 * Krylov error (Saad 1992). A step whose Krylov space closes (beta_k below
 * 1e-14 |alpha|max) ends early and exactly. HM_ERR_NOT_HERMITIAN for a
 * term list that is not self-adjoint; HM_ERR_INVALID_ARG for NaN or Inf in
 * the recurrence. Allocates 3 work vectors (+1 if nsub > 1, + m if stored).
 * Synchronous on stream. Works on sector plans (vectors of hm_dim states). */
int hm_evolve(hm_handle h, const void* x, void* y, double t, int32_t m, int32_t nsub, int32_t flags,
              hm_dtype dtype, double* err, void* stream);

/* Host only (no GPU): the coefficients hm_evolve combines a Krylov basis
 * with (the propagation step of the Sec. VII use case, short-iterative
 * Lanczos), c[k] = nu [exp(-i tau T) e_1]_k for k < m as (re, im) pairs in
 * c[2m] (caller-owned host array), T the real symmetric tridiagonal matrix
 * with diagonal alpha[m] and off-diagonal beta[m-1] (host arrays; beta may
 * be NULL for m = 1). 1 <= m <= 128; non-finite input gives
 * HM_ERR_INVALID_ARG. Synchronous, thread-safe. */
int hm_krylov_coefficients(const double* alpha, const double* beta, int32_t m, double tau, double nu,
                           double* c);

/* Batched apply over many plans of uneven size: one persistent launch per
 * 128 instances walks an (instance, block[, chunk]) work list; an instance
 * with enough work to fill the GPU by itself gets the launch hm_apply would
 * make for it instead (its hm_tune choice, else the general kernel's
 * default). A queued member's y, and an untuned member's y, equals
 * hm_apply_ex with the general kernel (flag bit 4) on it, bit for bit; a
 * tuned member that fills the GPU gets hm_apply's y. hs[n] stay owned by the caller
 * and must outlive the batch; each call reads the members' tables as they
 * are then (a CUDA graph captured before an hm_set_coefficients on a member
 * must be captured again). xs[b], ys[b]: device pointers (arrays of n
 * pointers, host memory). All instances share nvec and dtype. */
int hm_batch_create(const hm_handle* hs, int32_t n, hm_handle* batch_out);
int hm_batch_apply(hm_handle batch, const void* const* xs, void* const* ys, int64_t nvec,
                   hm_dtype dtype, void* stream);

/* Autotuner (no counterpart in the paper; a launch-shape search): time the apply
 * variants for (nvec, dtype) on scratch vectors it allocates and frees -- the
 * general kernel (elements per thread x register cap, with and without
 * prefetching, on the plan's low block and on the small one), the staged
 * kernel and the tile kernel (rows per iteration), then the persistent grid
 * size for the best -- and
 * cache the fastest in the plan, and in a process-wide cache keyed by the
 * site dimensions and channel counts, for hm_apply, hm_apply_adjoint (gx) and
 * hm_lanczos. Synchronous. The variants of one kernel compute the same y bit
 * for bit; the kernels sum in different orders (all within the FP64 /
 * FP32 tolerances). For a complex H (complex dtype) it tunes both real
 * operators on the 2*nvec columns, then times the two tuned real passes
 * with their combine against the one-pass complex kernel and its
 * register-capped variant and keeps the fastest for that (nvec, dtype). */
int hm_tune(hm_handle h, int64_t nvec, hm_dtype dtype, void* stream);

/* The launch choice hm_tune stored for (nvec, dtype): out[0] = grid size,
 * out[1] = elements per thread (general) or rows per iteration (tile),
 * out[2] = bit 0 register-cap variant, bit 1 small low block, bit 2
 * prefetching, bit 3 one right-hand side per lane, bit 4 top-site split,
 * bit 5 one group factor per lane, bits 8..11 the split's number of
 * leading sites (general kernel), bit 6 (complex H asked with a complex
 * dtype) the one-pass complex kernel instead of two tuned real passes,
 * bit 7 its register-capped variant; the other fields describe H_re's
 * tuned launch,
 * out[3] = kernel (1 general, 2 tile, 3 staged) (int32_t[4], host; 0 each =
 * library default). No counterpart in the paper (a diagnostic). */
int hm_tuned_config(hm_handle h, int64_t nvec, hm_dtype dtype, int32_t* out);

/* Diagnostic, host only: run the host half of hm_create (validation,
 * operator expansion, channel merging, high/low split, tables) without
 * touching the GPU, and write the resulting tables as JSON text. which
 * bit 0: H^T instead of H; bit 1: the tile kernel's tables for
 * nvec = which >> 8 (at least 1; HM_ERR_UNSUPPORTED if there is no tile
 * form); bit 2: the tables of hm_create_sector for digit_total =
 * which >> 8 (same error codes as hm_create_sector), with bit 4 those of
 * its block form ("ok": false when the plan has none); else the general
 * kernel's. bit 3: the imaginary part H_im of a complex H (else H_re, or
 * the whole real H). On success *len = bytes needed including
 * the terminating NUL; the text is written only if buf != NULL and
 * bufsize >= *len. Same error codes as hm_create. */
int hm_plan_export(const hm_site* sites, int32_t nsites, const hm_term* terms, int32_t nterms,
                   int32_t which, char* buf, int64_t bufsize, int64_t* len);

int hm_destroy(hm_handle h);
const char* hm_strerror(int code);
const char* hm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HM_H */
