"""Python front end of the hm C ABI. Argument marshalling only: every step of
the Hamiltonian action runs in the CUDA library; torch supplies device memory
and streams."""
from __future__ import annotations

import ctypes

import torch

from . import _capi as C


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


_CODES = {torch.float64: C.HM_F64, torch.float32: C.HM_F32, torch.complex128: C.HM_C128,
          torch.complex64: C.HM_C64}


def _dtype_code(t) -> int:
    """Library dtype of a tensor (or of a torch dtype)."""
    dt = t if isinstance(t, torch.dtype) else t.dtype
    if dt not in _CODES:
        raise TypeError(f"vectors must be float64, float32, complex128 or complex64, got {dt}")
    return _CODES[dt]


def _check_vec(t: torch.Tensor, name: str, host_ok: bool = False):
    if not t.is_cuda and not (host_ok and t.device.type == "cpu" and t.is_pinned()):
        raise ValueError(f"{name} must be a CUDA tensor" + (" or a pinned CPU tensor" if host_ok else ""))
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _site_kind(k):
    if k in ("spin", C.HM_SPIN):
        return C.HM_SPIN
    if k in ("boson", C.HM_BOSON):
        return C.HM_BOSON
    raise ValueError(f"unknown site kind {k!r}")


def _op(o):
    return C.OPS[o] if isinstance(o, str) else int(o)


class Hamiltonian:
    """H = sum_t coef_t op_i(t) op_j(t) on sites [(kind, dim), ...].

    terms: iterable of (i, op_i, j, op_j, coef), j = -1 for single-site terms;
    op names as in include/hm.h ("Sz", "Sx", "Sy", "Sp", "Sm", "Sz2", "Sp2",
    "Sm2", "N", "a", "adag", "I"). Vectors are float64 / float32 or
    complex128 / complex64 tensors; a term list with imaginary matrix elements
    (Sy factors) needs complex vectors."""

    def __init__(self, sites, terms, sector_total=None):
        """sector_total: None for the full product basis, else the fixed sum of
        the local digits n_k = m_k + s_k (a fixed-magnetization or
        excitation-number sector, hm_create_sector); D is then the number of
        retained states and vectors hold only those."""
        self._lib = C.load()
        torch.cuda.init()
        self.sites = [(_site_kind(k), int(d)) for k, d in sites]
        self.terms = [(int(i), _op(oi), int(j), _op(oj), float(c)) for i, oi, j, oj, c in terms]
        cs = (C.hm_site * len(self.sites))(*[C.hm_site(k, d) for k, d in self.sites])
        ts = (C.hm_term * max(1, len(self.terms)))(*[C.hm_term(i, oi, j, oj, c) for i, oi, j, oj, c in self.terms])
        h = ctypes.c_void_p()
        self.sector_total = sector_total
        if sector_total is None:
            C.check(self._lib.hm_create(cs, len(self.sites), ts, len(self.terms), ctypes.byref(h)), "hm_create")
        else:
            C.check(self._lib.hm_create_sector(cs, len(self.sites), ts, len(self.terms), int(sector_total),
                                               ctypes.byref(h)), "hm_create_sector")
        self._h = h
        self.D = int(self._lib.hm_dim(h))
        self.nterms = len(self.terms)
        self.coefs = [t[4] for t in self.terms]

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.hm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- coefficients ------------------------------------------------------
    def set_coefficients(self, coefs):
        c = [float(v) for v in (coefs.detach().cpu().tolist() if torch.is_tensor(coefs) else coefs)]
        if len(c) != self.nterms:
            raise ValueError(f"expected {self.nterms} coefficients, got {len(c)}")
        arr = (ctypes.c_double * max(1, self.nterms))(*c)
        C.check(self._lib.hm_set_coefficients(self._h, arr), "hm_set_coefficients")
        self.coefs = c
        self._coef_ref = None   # the autograd wrappers compare against this

    # -- y = H x -------------------------------------------------------------
    def _nvec(self, x):
        if x.numel() % self.D:
            raise ValueError(f"vector length {x.numel()} is not a multiple of D={self.D}")
        return x.numel() // self.D

    def apply(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """y = H x for x of D*nvec elements (state-major, x[k*nvec + v]).
        x and out may be CUDA tensors or pinned CPU tensors (the library then
        reads x and writes y over the CPU-GPU link inside the call)."""
        _check_vec(x, "x", host_ok=True)
        if out is None:
            y = torch.empty_like(x) if x.is_cuda else torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        else:
            y = out
        _check_vec(y, "out", host_ok=True)
        C.check(self._lib.hm_apply(self._h, x.data_ptr(), y.data_ptr(), self._nvec(x), _dtype_code(x),
                                   _stream(stream)), "hm_apply")
        return y

    def apply_ex(self, x, out=None, native_f64=False, transpose=False, ctas=0, s=0, mb=False, kernel=None,
                 stream=None, presplit=False, small=False, prefetch=False, scalar=False, split=False,
                 split_sites=0, vinv=False):
        """hm_apply with an explicit launch choice. kernel: None or "general"
        (the general kernel), "tile" or "staged"; on a sector plan None (the
        block form where the plan has it) or "rows" (the per-row kernel). s: rows per iteration of the
        tile kernel (1, 2, 4) or elements per thread of the general one (2, 3,
        4, 6, 8); 0 = default. mb: register-capped general kernel. ctas: grid
        size. small: the general kernel on the small low block (tables in L1).
        prefetch: the general kernel with its gathers prefetched by cp.async.
        scalar: one right-hand side per lane (no 2- or 4-wide policy).
        split: top-site split into two passes; split_sites: its number of
        leading sites (0 = chosen from the vector size). vinv: one group
        factor per lane where the plan allows it.
        A complex H takes native_f64, transpose (H^dagger), mb (the register-capped one-pass kernel) and
        scalar (two real passes instead of the one-pass complex kernel).
        presplit (timing diagnostic): x is a float32 tensor of 2 * D *
        nvec (hi, lo) pairs of FP64 values and out a float64 tensor; only the
        double-float apply kernel runs."""
        _check_vec(x, "x")
        kf = {None: 0, "tile": 8, "general": 16, "rows": 16, "staged": 32}[kernel]
        flags = (1 if native_f64 else 0) | (2 if transpose else 0) | (4 if mb else 0) | kf | (int(s) << 8)
        flags |= (128 if small else 0) | (4096 if prefetch else 0) | (8192 if scalar else 0)
        flags |= (1 << 14 if split else 0) | (1 << 15 if vinv else 0) | (int(split_sites) << 16)
        if presplit:
            if x.dtype != torch.float32 or out is None or out.dtype != torch.float64 or x.numel() != 2 * out.numel():
                raise ValueError("presplit needs float32 pairs x (2 * D * nvec) and a float64 out")
            _check_vec(out, "out")
            C.check(self._lib.hm_apply_ex(self._h, x.data_ptr(), out.data_ptr(), self._nvec(out), C.HM_F64,
                                          flags | 64, int(ctas), _stream(stream)), "hm_apply_ex")
            return out
        y = torch.empty_like(x) if out is None else out
        C.check(self._lib.hm_apply_ex(self._h, x.data_ptr(), y.data_ptr(), self._nvec(x), _dtype_code(x),
                                      flags, int(ctas), _stream(stream)), "hm_apply_ex")
        return y

    def adjoint(self, gy, x=None, want_gx=True, want_gcoef=True, gx=None, gcoef=None, stream=None):
        """gx = H^T gy and gcoef[t] = sum_v <gy_v|O_t|x_v> (float64, device)."""
        _check_vec(gy, "gy")
        if want_gx and gx is None:
            gx = torch.empty_like(gy)
        if want_gcoef and gcoef is None:
            gcoef = torch.empty(max(1, self.nterms), dtype=torch.float64, device=gy.device)
        if want_gcoef:
            if x is None:
                raise ValueError("x is needed for coupling gradients")
            _check_vec(x, "x")
        C.check(self._lib.hm_apply_adjoint(
            self._h, gy.data_ptr(), x.data_ptr() if x is not None else None,
            gx.data_ptr() if want_gx else None, gcoef.data_ptr() if want_gcoef else None,
            self._nvec(gy), _dtype_code(gy), _stream(stream)), "hm_apply_adjoint")
        return (gx if want_gx else None), (gcoef[: self.nterms] if want_gcoef else None)

    def lanczos(self, v0: torch.Tensor, steps: int, reorth: bool = False, ritz_vector: bool = False,
                stream=None):
        """Ground state by device Lanczos; returns dict(e0, alpha, beta, steps, psi0, breakdown)."""
        _check_vec(v0, "v0")
        if v0.numel() != self.D:
            raise ValueError("v0 must have D elements")
        a = (ctypes.c_double * steps)()
        b = (ctypes.c_double * steps)()
        done = ctypes.c_int32(0)
        e0 = ctypes.c_double(0.0)
        psi = torch.empty_like(v0) if ritz_vector else None
        rc = self._lib.hm_lanczos(self._h, v0.data_ptr(), steps, _dtype_code(v0), 1 if reorth else 0, a, b,
                                  ctypes.byref(done), psi.data_ptr() if psi is not None else None,
                                  ctypes.byref(e0), _stream(stream))
        C.check(rc, "hm_lanczos")
        m = done.value
        return {"e0": e0.value, "alpha": list(a)[:m], "beta": list(b)[: max(0, m - 1)], "steps": m,
                "psi0": psi, "breakdown": rc == C.HM_LANCZOS_BREAKDOWN}

    def evolve(self, x: torch.Tensor, t: float, m: int = 30, substeps: int = 1, reorth: bool = False,
               recompute: bool = False, out: torch.Tensor | None = None, stream=None):
        """y = exp(-i t H) x for a complex128/complex64 vector of D elements
        (short-iterative Lanczos, m Krylov vectors per substep). Returns
        (y, error estimate)."""
        _check_vec(x, "x")
        if not x.is_complex() or x.numel() != self.D:
            raise ValueError("x must be a complex vector of D elements")
        y = torch.empty_like(x) if out is None else out
        _check_vec(y, "out")
        err = ctypes.c_double(0.0)
        flags = (1 if reorth else 0) | (2 if recompute else 0)
        C.check(self._lib.hm_evolve(self._h, x.data_ptr(), y.data_ptr(), float(t), int(m), int(substeps), flags,
                                    _dtype_code(x), ctypes.byref(err), _stream(stream)), "hm_evolve")
        return y, err.value

    def tune(self, nvec: int = 1, dtype=torch.float64, stream=None):
        """Autotune the apply launch for (nvec, dtype); returns the stored choice."""
        code = _dtype_code(dtype)
        C.check(self._lib.hm_tune(self._h, int(nvec), code, _stream(stream)), "hm_tune")
        return self.tuned_config(nvec, dtype)

    def tuned_config(self, nvec: int = 1, dtype=torch.float64):
        """dict(ctas, s, mb, small, prefetch, scalar, split, vinv, split_sites, kernel, one_pass, one_pass_capped)
        of the stored launch choice (0 = library default; kernel 1 = general, 2 = tile, 3 = staged; one_pass: a
        complex H asked with a complex dtype runs the one-pass complex kernel, one_pass_capped its register-capped
        variant, instead of two tuned real passes)."""
        code = _dtype_code(dtype)
        out = (ctypes.c_int32 * 4)()
        C.check(self._lib.hm_tuned_config(self._h, int(nvec), code, out), "hm_tuned_config")
        return {"ctas": out[0], "s": out[1], "mb": out[2] & 1, "small": (out[2] >> 1) & 1,
                "prefetch": (out[2] >> 2) & 1, "scalar": (out[2] >> 3) & 1, "split": (out[2] >> 4) & 1,
                "vinv": (out[2] >> 5) & 1, "split_sites": (out[2] >> 8) & 15, "kernel": out[3],
                "one_pass": (out[2] >> 6) & 1, "one_pass_capped": (out[2] >> 7) & 1}


class Batch:
    """Many Hamiltonians applied in one persistent launch (uneven sizes)."""

    def __init__(self, hams):
        self._lib = C.load()
        self.hams = list(hams)
        arr = (ctypes.c_void_p * len(self.hams))(*[h.handle.value for h in self.hams])
        b = ctypes.c_void_p()
        C.check(self._lib.hm_batch_create(arr, len(self.hams), ctypes.byref(b)), "hm_batch_create")
        self._b = b

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            self._lib.hm_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, xs, ys=None, stream=None):
        if len(xs) != len(self.hams):
            raise ValueError("one x per Hamiltonian")
        ys = [torch.empty_like(x) for x in xs] if ys is None else ys
        for x, y in zip(xs, ys):
            _check_vec(x, "x")
            _check_vec(y, "y")
        nvec = xs[0].numel() // self.hams[0].D
        xp = (ctypes.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
        yp = (ctypes.c_void_p * len(ys))(*[y.data_ptr() for y in ys])
        C.check(self._lib.hm_batch_apply(self._b, xp, yp, nvec, _dtype_code(xs[0]), _stream(stream)),
                "hm_batch_apply")
        return ys
