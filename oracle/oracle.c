/*
 * CPU ORACLE -- test infrastructure only.
 *
 * A deliberately plain CPU evaluation of y = H x for the mixed spin /
 * truncated-boson Hamiltonians of "Spin Hamiltonian as Matrix-Free Linear
 * Map". Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may call it. It shares no code, header, table or constant with the CUDA
 * library.
 *
 * What it computes, row by row. The output element of basis index F is the
 * matrix row <F|H| contracted with x. The row's local digits come from the
 * mixed-radix place values M_k (Sec. III, Eq. decode). Each named local
 * operator is written as a short sum of matrix elements that move the digit
 * by a fixed amount q: 0 for Sz, Sz^2, N; +1/-1 for the spin ladders and the
 * boson creation/annihilation operators; +2/-2 for the squared ladders.
 * Sx and Sy are the ladder combinations of Sec. IV.A. The squared ladders
 * and Sz^2 are App. B; a, a^dagger and N are App. C. A term that pairs two
 * sites contributes only when both source digits stay inside their ranges.
 * Its source index differs from F by the two moves times their place
 * values (Sec. IV.B, Eq. sourceoffset). Its weight is the coefficient times
 * the two local matrix elements, evaluated at the source projection
 * (App. A ladder factors Lambda, App. B squared-ladder factors). Each row is
 * written once.
 *
 * Arithmetic is complex double throughout; indices are int64 with plain
 * division (no magic numbers, no tiling, no reordering). Rows may be spread
 * over OpenMP threads; each row's sum is taken in term order.
 */
#include <complex.h>
#define I_COMPLEX_UNIT _Complex_I
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* site kinds */
#define ORC_SPIN 0
#define ORC_BOSON 1

/* operator names, in the order the Python side passes them */
enum {
    ORC_I = 0, ORC_SZ, ORC_SX, ORC_SY, ORC_SP, ORC_SM, ORC_SZ2, ORC_SP2, ORC_SM2,
    ORC_N, ORC_A, ORC_ADAG
};

/* monomial kinds: which local matrix element formula to evaluate on n_src */
enum { MK_ONE = 0, MK_SZ, MK_SZ2, MK_SP, MK_SM, MK_SP2, MK_SM2, MK_BN, MK_BA, MK_BADAG };

typedef struct {
    int q;               /* n_target = n_source + q */
    double complex w;    /* weight of this monomial inside the named op */
    int kind;
} mono;

/* Lambda(alpha; s, m) of App. A */
static double lam_plus(double s, double m) { return sqrt(s * (s + 1.0) - m * (m + 1.0)); }
static double lam_minus(double s, double m) { return sqrt(s * (s + 1.0) - m * (m - 1.0)); }

/* Matrix element <n_src + q| monomial |n_src> on a site of dimension d. */
static double mono_coef(int kind, int d, int64_t nsrc)
{
    double s = 0.5 * (double)(d - 1);      /* spin: d = 2s+1 (Sec. I Eq. 1) */
    double m = (double)nsrc - s;           /* m = n - s (Sec. III)          */
    switch (kind) {
    case MK_ONE: return 1.0;
    case MK_SZ: return m;                                     /* Lambda(z) = m     */
    case MK_SZ2: return m * m;                                /* App. B, q = 0     */
    case MK_SP: return lam_plus(s, m);                        /* Sec. IV.A S+ rule */
    case MK_SM: return lam_minus(s, m);                       /* Sec. IV.A S- rule */
    case MK_SP2: return lam_plus(s, m + 1.0) * lam_plus(s, m);   /* App. B C^(2)_+ */
    case MK_SM2: return lam_minus(s, m - 1.0) * lam_minus(s, m); /* App. B C^(2)_- */
    case MK_BN: return (double)nsrc;                          /* a^dagger a        */
    case MK_BA: return sqrt((double)nsrc);                    /* App. C: a |n> = sqrt(n) |n-1>   */
    case MK_BADAG: return sqrt((double)nsrc + 1.0);           /* App. C: a^dag |n> = sqrt(n+1) |n+1> */
    }
    return 0.0;
}

/* Expand a named local operator into monomials; returns count, or -1 if the
 * operator does not exist on this site kind. */
static int expand_op(int op, int site_kind, mono out[2])
{
    if (op == ORC_I) { out[0] = (mono){0, 1.0, MK_ONE}; return 1; }
    if (site_kind == ORC_SPIN) {
        switch (op) {
        case ORC_SZ: out[0] = (mono){0, 1.0, MK_SZ}; return 1;
        case ORC_SZ2: out[0] = (mono){0, 1.0, MK_SZ2}; return 1;
        case ORC_SP: out[0] = (mono){+1, 1.0, MK_SP}; return 1;
        case ORC_SM: out[0] = (mono){-1, 1.0, MK_SM}; return 1;
        case ORC_SP2: out[0] = (mono){+2, 1.0, MK_SP2}; return 1;
        case ORC_SM2: out[0] = (mono){-2, 1.0, MK_SM2}; return 1;
        case ORC_SX:  /* Sx = (S+ + S-)/2 */
            out[0] = (mono){+1, 0.5, MK_SP};
            out[1] = (mono){-1, 0.5, MK_SM};
            return 2;
        case ORC_SY:  /* Sy = (S+ - S-)/(2i) = -i/2 S+ + i/2 S- */
            out[0] = (mono){+1, -0.5 * I, MK_SP};
            out[1] = (mono){-1, +0.5 * I, MK_SM};
            return 2;
        }
        return -1;
    }
    switch (op) {
    case ORC_N: out[0] = (mono){0, 1.0, MK_BN}; return 1;
    case ORC_A: out[0] = (mono){-1, 1.0, MK_BA}; return 1;
    case ORC_ADAG: out[0] = (mono){+1, 1.0, MK_BADAG}; return 1;
    }
    return -1;
}

/* D and multipliers M_k = prod_{l>k} d_l, M_{N-1} = 1 (Sec. III). Returns D or -1. */
int64_t oracle_multipliers(int nsites, const int* dims, int64_t* mult)
{
    int64_t m = 1;
    for (int k = nsites - 1; k >= 0; --k) {
        if (dims[k] < 1) return -1;
        mult[k] = m;
        if (m > INT64_MAX / dims[k]) return -1;
        m *= dims[k];
    }
    return m;
}

/* Eq. (decode): n_k = floor(I / M_k) mod d_k */
void oracle_decode(int nsites, const int* dims, int64_t index, int* digits)
{
    int64_t mult[128];
    oracle_multipliers(nsites, dims, mult);
    for (int k = 0; k < nsites; ++k) digits[k] = (int)((index / mult[k]) % dims[k]);
}

/* Eq. (encode): I = sum_k n_k M_k */
int64_t oracle_encode(int nsites, const int* dims, const int* digits)
{
    int64_t mult[128];
    oracle_multipliers(nsites, dims, mult);
    int64_t idx = 0;
    for (int k = 0; k < nsites; ++k) idx += (int64_t)digits[k] * mult[k];
    return idx;
}

typedef struct {
    int nsites;
    const int* kinds;
    const int* dims;
    int64_t mult[128];
    int64_t D;
    int nterms;
    const int* ti; const int* oi; const int* tj; const int* oj;
    const double* cre; const double* cim;
} problem;

/* Input vectors too large to hold on the host are synthesised on the fly:
 * x_i = (splitmix64 output number i+1 from state seed) >> 11, times 2^-53,
 * minus 1/2 (i = 0, 1, ...), splitmix64 being the
 * published finaliser of Steele, Lea and Flood (OOPSLA 2014): add the golden
 * gamma 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds and a final
 * xor-shift. With f32 != 0 the value is rounded to float (an FP32-storage
 * vector). The test inputs module implements the same generator. */
typedef struct {
    const double* re;  /* NULL: synthesised from seed */
    const double* im;
    uint64_t seed;
    int f32;
} xsource;

static double hashed_x(uint64_t seed, int64_t idx, int f32)
{
    uint64_t z = seed + (uint64_t)idx * 0x9E3779B97F4A7C15ULL + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    double v = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    return f32 ? (double)(float)v : v;
}

static double complex x_at(const xsource* X, int64_t idx)
{
    if (!X->re) return hashed_x(X->seed, idx, X->f32);
    return X->re[idx] + I_COMPLEX_UNIT * (X->im ? X->im[idx] : 0.0);
}

/* One target row: y_F = <F|H|x> (Sec. II). */
static double complex row_value_x(const problem* P, int64_t F, const xsource* X)
{
    int n[128];
    for (int k = 0; k < P->nsites; ++k) n[k] = (int)((F / P->mult[k]) % P->dims[k]);
    double complex acc = 0.0;
    for (int t = 0; t < P->nterms; ++t) {
        int i = P->ti[t], j = P->tj[t];
        mono mi[2], mj[2];
        int ci = expand_op(P->oi[t], P->kinds[i], mi);
        int cj = 1;
        if (j >= 0) cj = expand_op(P->oj[t], P->kinds[j], mj);
        else mj[0] = (mono){0, 1.0, MK_ONE};
        double complex coef = P->cre[t] + I * (P->cim ? P->cim[t] : 0.0);
        for (int a = 0; a < ci; ++a) {
            int64_t si = (int64_t)n[i] - mi[a].q;
            if (si < 0 || si > P->dims[i] - 1) continue;
            for (int b = 0; b < cj; ++b) {
                int64_t src = F - (int64_t)mi[a].q * P->mult[i];
                double cb = 1.0;
                if (j >= 0) {
                    int64_t sj = (int64_t)n[j] - mj[b].q;
                    if (sj < 0 || sj > P->dims[j] - 1) continue;
                    src -= (int64_t)mj[b].q * P->mult[j];
                    cb = mono_coef(mj[b].kind, P->dims[j], sj);
                }
                double ca = mono_coef(mi[a].kind, P->dims[i], si);
                acc += coef * mi[a].w * mj[b].w * ca * cb * x_at(X, src);
            }
        }
    }
    return acc;
}

/* x given as real and imaginary parts (xim may be NULL for a real vector) */
static double complex row_value(const problem* P, int64_t F, const double* xre, const double* xim)
{
    xsource X = {xre, xim, 0, 0};
    return row_value_x(P, F, &X);
}

static int setup(problem* P, int nsites, const int* kinds, const int* dims, int nterms,
                 const int* ti, const int* oi, const int* tj, const int* oj,
                 const double* cre, const double* cim)
{
    if (nsites < 1 || nsites > 128) return -1;
    P->nsites = nsites; P->kinds = kinds; P->dims = dims;
    P->D = oracle_multipliers(nsites, dims, P->mult);
    if (P->D < 0) return -2;
    P->nterms = nterms; P->ti = ti; P->oi = oi; P->tj = tj; P->oj = oj;
    P->cre = cre; P->cim = cim;
    for (int t = 0; t < nterms; ++t) {
        mono tmp[2];
        if (ti[t] < 0 || ti[t] >= nsites || tj[t] >= nsites || tj[t] == ti[t]) return -3;
        if (expand_op(oi[t], kinds[ti[t]], tmp) < 0) return -4;
        if (tj[t] >= 0 && expand_op(oj[t], kinds[tj[t]], tmp) < 0) return -4;
    }
    return 0;
}

/* y[F - row_begin] for F in [row_begin, row_end). Returns 0 or a negative code. */
int oracle_apply(int nsites, const int* kinds, const int* dims, int nterms,
                 const int* ti, const int* oi, const int* tj, const int* oj,
                 const double* cre, const double* cim,
                 const double* xre, const double* xim,
                 double* yre, double* yim, int64_t row_begin, int64_t row_end, int nthreads)
{
    problem P;
    int rc = setup(&P, nsites, kinds, dims, nterms, ti, oi, tj, oj, cre, cim);
    if (rc) return rc;
    if (row_begin < 0 || row_end > P.D || row_begin > row_end) return -5;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t F = row_begin; F < row_end; ++F) {
        double complex v = row_value(&P, F, xre, xim);
        yre[F - row_begin] = creal(v);
        if (yim) yim[F - row_begin] = cimag(v);
    }
    return 0;
}

/* y for an explicit list of rows (sampled-row checks on large D). */
int oracle_rows(int nsites, const int* kinds, const int* dims, int nterms,
                const int* ti, const int* oi, const int* tj, const int* oj,
                const double* cre, const double* cim,
                const double* xre, const double* xim,
                const int64_t* rows, int64_t nrows, double* yre, double* yim, int nthreads)
{
    problem P;
    int rc = setup(&P, nsites, kinds, dims, nterms, ti, oi, tj, oj, cre, cim);
    if (rc) return rc;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= P.D) return -5;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t r = 0; r < nrows; ++r) {
        double complex v = row_value(&P, rows[r], xre, xim);
        yre[r] = creal(v);
        if (yim) yim[r] = cimag(v);
    }
    return 0;
}

/* y for an explicit list of rows with x synthesised from seed (above). */
int oracle_rows_hashed(int nsites, const int* kinds, const int* dims, int nterms,
                       const int* ti, const int* oi, const int* tj, const int* oj,
                       const double* cre, const double* cim, uint64_t seed, int f32,
                       const int64_t* rows, int64_t nrows, double* yre, double* yim, int nthreads)
{
    problem P;
    int rc = setup(&P, nsites, kinds, dims, nterms, ti, oi, tj, oj, cre, cim);
    if (rc) return rc;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= P.D) return -5;
    xsource X = {NULL, NULL, seed, f32};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int64_t r = 0; r < nrows; ++r) {
        double complex v = row_value_x(&P, rows[r], &X);
        yre[r] = creal(v);
        if (yim) yim[r] = cimag(v);
    }
    return 0;
}

/* x_I of the synthesised vector for an explicit list of indices (so that the
 * tests can pin this generator against the inputs module's). */
void oracle_hashed_values(uint64_t seed, int f32, const int64_t* idx, int64_t n, double* out)
{
    for (int64_t k = 0; k < n; ++k) out[k] = hashed_x(seed, idx[k], f32);
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
