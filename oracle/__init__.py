"""CPU oracle for y = H x -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never does, and this
package never imports the library: the two share no code.

Contents
  * ``apply`` / ``rows``  -- plain C restatement of the target-driven matvec
    (App. A, extended by App. B powers and App. C bosons); see oracle.c.
  * ``dense``             -- explicit Kronecker-product assembly of H for tiny
    systems (Sec. I: the operator the matrix-free map must equal), built from
    textbook local spin/boson matrices with site 0 as the leftmost factor
    (Sec. III Eq. encode: site 1 is the most significant digit).
  * ``lanczos``           -- plain FP64 Lanczos with full reorthogonalisation
    (Sec. I: Krylov solvers need only y = H x).
  * ``term_gradients``    -- <gy| O_t |x> per term, by applying one-term
    Hamiltonians (with gy = x = psi, the Hellmann-Feynman gradient
    <psi|O_t|psi>).
  * ``evolve``            -- y = exp(-i t H) x (Sec. VII: exact propagation
    under time-dependent or repeatedly rebuilt couplings), the definition
    written out through a dense eigendecomposition of H (tiny systems).
  * ``sector_*``          -- the globally constrained sector of Sec. VI case 2
    (local digits summing to a fixed total; App. D): enumeration of the
    retained states, combinatorial rank / unrank, the projected apply
    P H P^T x, and a row-wise restatement of the case-2 steps (unpack target,
    undo the local move, look the source up, accumulate).

Parity pins live in tests/test_oracle_*.py (closed forms, invariants, brute
force); every oracle function there is pinned to something other than itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SPIN_KIND, BOSON_KIND = 0, 1
OP_CODES = {"I": 0, "Sz": 1, "Sx": 2, "Sy": 3, "Sp": 4, "Sm": 5, "Sz2": 6, "Sp2": 7,
            "Sm2": 8, "N": 9, "a": 10, "adag": 11}


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2 -fopenmp) into oracle/_build/liboracle.so."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i32p = ctypes.POINTER(ctypes.c_int)
            f64p = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            common = [ctypes.c_int, i32p, i32p, ctypes.c_int, i32p, i32p, i32p, i32p, f64p, f64p,
                      f64p, f64p]
            lib.oracle_apply.argtypes = common + [f64p, f64p, ctypes.c_int64, ctypes.c_int64,
                                                  ctypes.c_int]
            lib.oracle_apply.restype = ctypes.c_int
            lib.oracle_rows.argtypes = common + [i64p, ctypes.c_int64, f64p, f64p, ctypes.c_int]
            lib.oracle_rows.restype = ctypes.c_int
            lib.oracle_decode.argtypes = [ctypes.c_int, i32p, ctypes.c_int64, i32p]
            lib.oracle_encode.argtypes = [ctypes.c_int, i32p, i32p]
            lib.oracle_encode.restype = ctypes.c_int64
            lib.oracle_multipliers.argtypes = [ctypes.c_int, i32p, i64p]
            lib.oracle_multipliers.restype = ctypes.c_int64
            lib.oracle_max_threads.restype = ctypes.c_int
            prob = common[:10]
            lib.oracle_rows_hashed.argtypes = prob + [ctypes.c_uint64, ctypes.c_int, i64p, ctypes.c_int64, f64p,
                                                      f64p, ctypes.c_int]
            lib.oracle_rows_hashed.restype = ctypes.c_int
            lib.oracle_hashed_values.argtypes = [ctypes.c_uint64, ctypes.c_int, i64p, ctypes.c_int64, f64p]
            lib.oracle_hashed_values.restype = None
            _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


class _Packed:
    """Term list packed into C arrays."""

    def __init__(self, sites, terms, coefs=None):
        self.kinds = np.array([SPIN_KIND if k == "spin" else BOSON_KIND for k, _ in sites],
                              dtype=np.int32)
        self.dims = np.array([d for _, d in sites], dtype=np.int32)
        self.ti = np.array([t[0] for t in terms], dtype=np.int32)
        self.oi = np.array([OP_CODES[t[1]] for t in terms], dtype=np.int32)
        self.tj = np.array([t[2] for t in terms], dtype=np.int32)
        self.oj = np.array([OP_CODES[t[3]] for t in terms], dtype=np.int32)
        c = np.array([t[4] for t in terms] if coefs is None else coefs, dtype=np.complex128)
        self.cre = np.ascontiguousarray(c.real)
        self.cim = np.ascontiguousarray(c.imag)
        self.n = len(sites)
        self.nt = len(terms)

    def args(self):
        i32 = ctypes.c_int
        return [self.n, _ptr(self.kinds, i32), _ptr(self.dims, i32), self.nt, _ptr(self.ti, i32),
                _ptr(self.oi, i32), _ptr(self.tj, i32), _ptr(self.oj, i32),
                _ptr(self.cre, ctypes.c_double), _ptr(self.cim, ctypes.c_double)]


def _split(x):
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return (np.ascontiguousarray(x.real, dtype=np.float64),
                np.ascontiguousarray(x.imag, dtype=np.float64))
    return np.ascontiguousarray(x, dtype=np.float64), None


def dimension(sites) -> int:
    """D = prod d_i (Sec. I Eq. 1), as a Python int."""
    D = 1
    for _, d in sites:
        D *= int(d)
    return D


def multipliers(dims):
    """M_k = prod_{l>k} d_l (Sec. III), from the C oracle."""
    lib = _load()
    d = np.asarray(dims, dtype=np.int32)
    m = np.zeros(len(d), dtype=np.int64)
    D = lib.oracle_multipliers(len(d), _ptr(d, ctypes.c_int), _ptr(m, ctypes.c_int64))
    return m, int(D)


def decode(dims, index):
    lib = _load()
    d = np.asarray(dims, dtype=np.int32)
    out = np.zeros(len(d), dtype=np.int32)
    lib.oracle_decode(len(d), _ptr(d, ctypes.c_int), int(index), _ptr(out, ctypes.c_int))
    return out


def encode(dims, digits):
    lib = _load()
    d = np.asarray(dims, dtype=np.int32)
    n = np.asarray(digits, dtype=np.int32)
    return int(lib.oracle_encode(len(d), _ptr(d, ctypes.c_int), _ptr(n, ctypes.c_int)))


def apply(sites, terms, x, coefs=None, row_begin=0, row_end=None, nthreads=0, nvec=1):
    """y = H x for rows [row_begin, row_end) (all rows by default).

    x: length D*nvec (state-major, x[k*nvec + v]) real or complex. Returns a
    complex128 array of (row_end-row_begin)*nvec values, same layout."""
    lib = _load()
    P = _Packed(sites, terms, coefs)
    D = dimension(sites)
    row_end = D if row_end is None else row_end
    x = np.asarray(x)
    out = np.zeros((row_end - row_begin, nvec), dtype=np.complex128)
    xs = x.reshape(D, nvec)
    for v in range(nvec):
        xre, xim = _split(xs[:, v])
        yre = np.zeros(row_end - row_begin)
        yim = np.zeros(row_end - row_begin)
        rc = lib.oracle_apply(*P.args(), _ptr(xre, ctypes.c_double), _ptr(xim, ctypes.c_double),
                              _ptr(yre, ctypes.c_double), _ptr(yim, ctypes.c_double),
                              int(row_begin), int(row_end), int(nthreads))
        if rc != 0:
            raise ValueError(f"oracle_apply rejected the problem (code {rc})")
        out[:, v] = yre + 1j * yim
    return out.reshape(-1)


def rows(sites, terms, x, row_idx, coefs=None, nthreads=0):
    """y_F for an explicit list of target rows F (sampled-row checks); x real
    or complex, length D (nvec = 1)."""
    lib = _load()
    P = _Packed(sites, terms, coefs)
    r = np.ascontiguousarray(row_idx, dtype=np.int64)
    xre, xim = _split(x)
    yre = np.zeros(len(r))
    yim = np.zeros(len(r))
    rc = lib.oracle_rows(*P.args(), _ptr(xre, ctypes.c_double), _ptr(xim, ctypes.c_double),
                         _ptr(r, ctypes.c_int64), len(r), _ptr(yre, ctypes.c_double),
                         _ptr(yim, ctypes.c_double), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_rows rejected the problem (code {rc})")
    return yre + 1j * yim


def rows_hashed(sites, terms, seed, row_idx, f32=False, coefs=None, nthreads=0):
    """y_F for an explicit list of target rows F with x synthesised on the
    fly from a counter-based generator (splitmix64, see oracle.c): for
    vectors too large to hold on the host. f32: x rounded to float (FP32
    storage)."""
    lib = _load()
    P = _Packed(sites, terms, coefs)
    r = np.ascontiguousarray(row_idx, dtype=np.int64)
    yre = np.zeros(len(r))
    yim = np.zeros(len(r))
    rc = lib.oracle_rows_hashed(*P.args()[:10], ctypes.c_uint64(int(seed) & (2 ** 64 - 1)), 1 if f32 else 0,
                                _ptr(r, ctypes.c_int64), len(r), _ptr(yre, ctypes.c_double),
                                _ptr(yim, ctypes.c_double), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_rows_hashed rejected the problem (code {rc})")
    return yre + 1j * yim


def hashed_values(seed, idx, f32=False):
    """The oracle's synthesised x at the given indices."""
    lib = _load()
    r = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.zeros(len(r))
    lib.oracle_hashed_values(ctypes.c_uint64(int(seed) & (2 ** 64 - 1)), 1 if f32 else 0, _ptr(r, ctypes.c_int64),
                             len(r), _ptr(out, ctypes.c_double))
    return out


def max_threads() -> int:
    return int(_load().oracle_max_threads())


# ----------------------------------------------------------------------------
# Dense Kronecker assembly (tiny D)
# ----------------------------------------------------------------------------

def local_matrix(kind, d, op):
    """Textbook local matrices in ascending local index n = m + s (Sec. III
    notation guide: n = 0 is m = -s; App. C: n = boson occupation).

    Spin: Sz = diag(m); <m+1|S+|m> = sqrt(s(s+1) - m(m+1)); S- = (S+)^T;
    Sx = (S+ + S-)/2; Sy = (S+ - S-)/(2i); squares as matrix products.
    Boson: <n+1|a^dag|n> = sqrt(n+1); a = (a^dag)^T; N = a^dag a."""
    if op == "I":
        return np.eye(d, dtype=np.complex128)
    if kind == "spin":
        s = (d - 1) / 2.0
        m = np.arange(d) - s
        sz = np.diag(m).astype(np.complex128)
        sp = np.zeros((d, d), dtype=np.complex128)
        for n in range(d - 1):
            sp[n + 1, n] = np.sqrt(s * (s + 1) - m[n] * (m[n] + 1))
        sm = sp.T.copy()
        table = {"Sz": sz, "Sp": sp, "Sm": sm, "Sx": (sp + sm) / 2, "Sy": (sp - sm) / 2j,
                 "Sz2": sz @ sz, "Sp2": sp @ sp, "Sm2": sm @ sm}
    else:
        ad = np.zeros((d, d), dtype=np.complex128)
        for n in range(d - 1):
            ad[n + 1, n] = np.sqrt(n + 1)
        a = ad.T.copy()
        table = {"adag": ad, "a": a, "N": ad @ a}
    if op not in table:
        raise ValueError(f"operator {op} is not defined on a {kind} site")
    return table[op]


def dense(sites, terms, coefs=None, sparse=False):
    """H = sum_t coef_t (I x ... x A_i x ... x B_j x ... x I), site 0 leftmost."""
    n = len(sites)
    D = dimension(sites)
    if sparse:
        import scipy.sparse as sp
        H = sp.csr_matrix((D, D), dtype=np.complex128)
        # format="csr" keeps scipy on its COO path (nnz(A) * nnz(B) entries);
        # its default BSR path stores dense blocks including explicit zeros
        kron = lambda a, b: sp.kron(a, b, format="csr")
        eye = lambda d: sp.identity(d, dtype=np.complex128, format="csr")
    else:
        if D > 1 << 13:
            raise ValueError("dense assembly is for tiny systems (D <= 8192)")
        H = np.zeros((D, D), dtype=np.complex128)
        kron, eye = np.kron, (lambda d: np.eye(d, dtype=np.complex128))
    cs = [t[4] for t in terms] if coefs is None else list(coefs)
    for t, (i, oi, j, oj, _) in enumerate(terms):
        factors = [eye(d) for _, d in sites]
        factors[i] = local_matrix(sites[i][0], sites[i][1], oi)
        if j >= 0:
            factors[j] = local_matrix(sites[j][0], sites[j][1], oj)
        if sparse:
            factors = [sp.csr_matrix(f) for f in factors]
        M = factors[0]
        for f in factors[1:]:
            M = kron(M, f)
        H = H + cs[t] * M
    return H


# ----------------------------------------------------------------------------
# Lanczos and gradients on top of the row-wise oracle
# ----------------------------------------------------------------------------

def lanczos(sites, terms, v0, steps, coefs=None, nthreads=0):
    """Plain FP64 Lanczos with full reorthogonalisation. Returns
    (alpha, beta, E0, psi0) where psi0 is the Ritz vector of the lowest Ritz
    value; the tridiagonal eigenproblem is solved with numpy.linalg.eigh."""
    v = np.asarray(v0, dtype=np.float64)
    v = v / np.linalg.norm(v)
    V = [v]
    alpha, beta = [], []
    for k in range(steps):
        w = apply(sites, terms, V[-1], coefs=coefs, nthreads=nthreads).real
        a = float(np.dot(V[-1], w))
        w = w - a * V[-1] - (beta[-1] * V[-2] if k > 0 else 0.0)
        for u in V:                        # full reorthogonalisation
            w = w - np.dot(u, w) * u
        b = float(np.linalg.norm(w))
        alpha.append(a)
        if k == steps - 1 or b < 1e-14:
            break
        beta.append(b)
        V.append(w / b)
    m = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:m - 1], 1) + np.diag(beta[:m - 1], -1)
    evals, evecs = np.linalg.eigh(T)
    psi = np.zeros_like(v)
    for k in range(m):
        psi += evecs[k, 0] * V[k]
    return np.array(alpha), np.array(beta[:m - 1]), float(evals[0]), psi


def term_gradients(sites, terms, gy, x, nthreads=0):
    """g_t = <gy| O_t |x> for every term t, O_t = op_i op_j without its
    coefficient: the derivative of <gy|H|x> with respect to coef_t."""
    g = np.zeros(len(terms), dtype=np.complex128)
    gy = np.asarray(gy)
    for t, term in enumerate(terms):
        one = [(term[0], term[1], term[2], term[3], 1.0)]
        Ox = apply(sites, one, x, nthreads=nthreads)
        g[t] = np.vdot(gy, Ox)
    return g


# ---------------------------------------------------------------------------
# Globally constrained sector (Sec. VI case 2, App. D): the retained states
# are those whose local digits sum to a fixed total K (for spins the fixed
# magnetization sum_i m_i = K - sum_i s_i; for the Jaynes-Cummings /
# Tavis-Cummings models the excitation number). Packed storage index = the
# state's position among the retained states in ascending full-basis order.
# ---------------------------------------------------------------------------

def sector_basis(sites, total):
    """Full-basis indices of the retained states, ascending (by enumeration of
    every digit tuple; small D only)."""
    s = np.zeros(1, dtype=np.int64)
    for _, d in sites:   # site 0 outermost: flat index = sum_k n_k M_k (Sec. III)
        s = (s[:, None] + np.arange(int(d), dtype=np.int64)[None, :]).reshape(-1)
    return np.nonzero(s == int(total))[0]


def sector_counts(dims, total):
    """cnt[k][r] = number of digit tuples of sites k..N-1 whose sum is r."""
    N = len(dims)
    cnt = [[0] * (total + 1) for _ in range(N + 1)]
    cnt[N][0] = 1
    for k in range(N - 1, -1, -1):
        for r in range(total + 1):
            cnt[k][r] = sum(cnt[k + 1][r - m] for m in range(min(int(dims[k]) - 1, r) + 1))
    return cnt


def sector_dimension(sites, total):
    dims = [int(d) for _, d in sites]
    return sector_counts(dims, total)[0][total] if total >= 0 else 0


def sector_rank(dims, total, digits, cnt=None):
    """Packed index of a digit tuple: the number of retained tuples that
    precede it in lexicographic (= full-index) order, counted site by site
    (combinatorial ranking); -1 if the tuple is not in the sector."""
    cnt = cnt or sector_counts(dims, total)
    rank, rem = 0, total
    for k, n in enumerate(digits):
        n = int(n)
        if n < 0 or n >= dims[k]:
            return -1
        for m in range(n):
            if rem - m >= 0:
                rank += cnt[k + 1][rem - m]
        rem -= n
        if rem < 0:
            return -1
    return rank if rem == 0 else -1


def sector_unrank(dims, total, r, cnt=None):
    """Digit tuple of packed index r (inverse of sector_rank)."""
    cnt = cnt or sector_counts(dims, total)
    digits, rem = [], total
    for k in range(len(dims)):
        m = 0
        while True:
            c = cnt[k + 1][rem - m] if rem - m >= 0 else 0
            if r < c:
                break
            r -= c
            m += 1
        digits.append(m)
        rem -= m
    return digits


def sector_apply(sites, terms, total, x, nvec=1, coefs=None):
    """y = P H P^T x on the packed sector vector (P selects the retained rows
    of the full basis): the full-basis oracle applied to x embedded with zeros
    outside the sector, restricted back to the sector. Equal to the action of
    H inside the sector when H conserves the digit sum."""
    basis = sector_basis(sites, total)
    D = dimension(sites)
    x = np.asarray(x).reshape(basis.size, nvec)
    xf = np.zeros((D, nvec), dtype=np.result_type(x.dtype, np.float64))
    xf[basis] = x
    y = apply(sites, terms, xf.reshape(-1), coefs=coefs, nvec=nvec).reshape(D, nvec)
    return y[basis].reshape(-1)


def sector_rows(sites, terms, total, x, rows, nvec=1, seed=None, f32=False):
    """y_F for packed target rows F, following the case-2 steps of Sec. VI /
    App. D one by one: unpack the target's digits, undo each term's local move
    (every source digit pair with a nonzero local matrix element), look the
    source up in the sector (a failed lookup contributes nothing), accumulate
    coefficient x x[source]. Row by row in Python: a few thousand rows.
    With seed given (x = None, nvec = 1), x[source] is the synthesised value
    of the counter-based generator (hashed_values), for sectors too large to
    hold x on the host."""
    if seed is not None:
        class _Synth:
            def __getitem__(self, I):
                return hashed_values(seed, [I], f32)[0]
        x = None
        xs = _Synth()
    dims = [int(d) for _, d in sites]
    cnt = sector_counts(dims, total)
    mats = {}

    def mat(site, op):
        key = (site, op)
        if key not in mats:
            kind, d = sites[site]
            mats[key] = local_matrix(kind, d, op)
        return mats[key]
    if seed is None:
        xs = np.asarray(x).reshape(-1, nvec)
    out = np.zeros((len(rows), nvec), dtype=np.complex128)
    for o, F in enumerate(rows):
        tgt = sector_unrank(dims, total, int(F), cnt)
        for (i, oi, j, oj, c) in terms:
            A = mat(i, oi)
            if j < 0 or oj in ("I", 0):
                B, j = None, -1
            else:
                B = mat(j, oj)
            for si in range(dims[i]):
                a = A[tgt[i], si]
                if a == 0:
                    continue
                js = [None] if B is None else range(dims[j])
                for sj in js:
                    b = 1.0 if sj is None else B[tgt[j], sj]
                    if b == 0:
                        continue
                    src = list(tgt)
                    src[i] = si
                    if sj is not None:
                        src[j] = sj
                    I = sector_rank(dims, total, src, cnt)
                    if I >= 0:
                        out[o] += c * a * b * xs[I]
    return out.reshape(-1)


# ----------------------------------------------------------------------------
# Time evolution (Sec. VII use case: exact propagation)
# ----------------------------------------------------------------------------

def evolve(sites, terms, x, t, coefs=None, sector_total=None):
    """y = exp(-i t H) x (hbar = 1) for a Hermitian term list: H from the
    Kronecker assembly (restricted to the sector's retained states when
    sector_total is given), H = V diag(lam) V^H by numpy.linalg.eigh, then
    y = V diag(exp(-i t lam)) V^H x. Tiny systems only (D <= 8192)."""
    H = dense(sites, terms, coefs=coefs)
    if sector_total is not None:
        b = sector_basis(sites, sector_total)
        H = H[np.ix_(b, b)]
    lam, V = np.linalg.eigh(H)
    x = np.asarray(x, dtype=np.complex128)
    return V @ (np.exp(-1j * t * lam) * (V.conj().T @ x))
