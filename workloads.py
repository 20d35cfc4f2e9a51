"""Seeded synthetic workloads: site lists, term lists and vectors.

This module only *describes* models and draws random numbers. It holds none of
the Hamiltonian-action arithmetic: no digit decoding, no index offsets, no
ladder factors. Both the CPU oracle (``oracle/``) and the CUDA library read the
same descriptions and interpret the operator names independently.

A model is
  sites : list of (kind, dim), kind in {"spin", "boson"};
          spin dim = 2s+1, boson dim = n_max+1 (Sec. I Eq. 1, App. C)
  terms : list of (i, op_i, j, op_j, coef); j = -1 marks a single-site term.
          Each term adds coef * op_i(site i) * op_j(site j).
Operator names:
  spin : "I", "Sz", "Sx", "Sy", "Sp", "Sm", "Sz2", "Sp2", "Sm2"
  boson: "I", "N" (= a^dagger a), "a", "adag"

Random parameters are drawn with ``numpy.random.default_rng(seed)`` in the
order stated in each generator's docstring.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SPIN = "spin"
BOSON = "boson"
SPIN_OPS = ("I", "Sz", "Sx", "Sy", "Sp", "Sm", "Sz2", "Sp2", "Sm2")
BOSON_OPS = ("I", "N", "a", "adag")


@dataclass
class Model:
    name: str
    sites: list
    terms: list
    # free-form, e.g. which term indices carry which physical coupling
    meta: dict = field(default_factory=dict)

    @property
    def dims(self):
        return [d for _, d in self.sites]


def spin_dim(s2: int) -> int:
    """Local dimension for spin s = s2/2 (Sec. I Eq. 1: d = 2s+1)."""
    return s2 + 1


def heisenberg_bond(i, j, J):
    """J S_i.S_j written as J (SxSx + SySy + SzSz)."""
    return [(i, "Sx", j, "Sx", J), (i, "Sy", j, "Sy", J), (i, "Sz", j, "Sz", J)]


def xxz_bond(i, j, jxy, jz):
    """Jxy (SxSx + SySy) + Jz SzSz."""
    return [(i, "Sx", j, "Sx", jxy), (i, "Sy", j, "Sy", jxy), (i, "Sz", j, "Sz", jz)]


# ----------------------------------------------------------------------------
# The five workload shapes
# ----------------------------------------------------------------------------

def heisenberg_ring(n=12, J=1.0) -> Model:
    """Spin-1/2 Heisenberg ring, periodic bonds (i, i+1 mod n), H = J sum S_i.S_{i+1}.
    n=12 gives D=4096."""
    sites = [(SPIN, 2)] * n
    terms = []
    for i in range(n):
        terms += heisenberg_bond(i, (i + 1) % n, J)
    return Model(f"heisenberg_ring_n{n}", sites, terms)


def ferrimagnet_chain(n=20, J=1.0, hz=0.1, seed=2) -> Model:
    """Mixed-spin open chain alternating s=1/2 (even sites) and s=1 (odd sites).
    Nearest-neighbour Heisenberg J, uniform field hz Sz on every site, and a
    single-ion anisotropy D_i (Sz_i)^2 with D_i ~ U[-0.5, 0.5] drawn in site
    order on the spin-1 sites (rng seed `seed`). n=20 gives D = 2^10 3^10."""
    rng = np.random.default_rng(seed)
    sites = [(SPIN, 2) if i % 2 == 0 else (SPIN, 3) for i in range(n)]
    terms = []
    for i in range(n - 1):
        terms += heisenberg_bond(i, i + 1, J)
    for i in range(n):
        terms.append((i, "Sz", -1, "I", hz))
    for i in range(1, n, 2):
        terms.append((i, "Sz2", -1, "I", float(rng.uniform(-0.5, 0.5))))
    return Model(f"ferrimagnet_chain_n{n}", sites, terms)


def xxz_spin1_chain(n, jxy=1.0, jz=1.5, seed=1000) -> Model:
    """Random-field spin-1 XXZ open chain: Jxy, Jz on bonds (i, i+1) and
    h_i Sz_i with h_i ~ U[-2, 2] (rng seed `seed`, drawn in site order)."""
    rng = np.random.default_rng(seed)
    sites = [(SPIN, 3)] * n
    terms = []
    for i in range(n - 1):
        terms += xxz_bond(i, i + 1, jxy, jz)
    h = rng.uniform(-2.0, 2.0, size=n)
    for i in range(n):
        terms.append((i, "Sz", -1, "I", float(h[i])))
    return Model(f"xxz_spin1_n{n}_s{seed}", sites, terms)


def disorder_ensemble(count=256, nmin=8, nmax=14, base_seed=1000):
    """Ensemble of random-field spin-1 XXZ chains. Instance b draws its length
    N_b = nmin + rng.integers(0, nmax-nmin+1) and its fields from
    default_rng(base_seed + b)."""
    models = []
    for b in range(count):
        rng = np.random.default_rng(base_seed + b)
        n = int(nmin + rng.integers(0, nmax - nmin + 1))
        models.append(xxz_spin1_chain(n, seed=base_seed + b))
    return models


def square_lattice_xxz(rows=4, cols=5, seed=4) -> Model:
    """Open rows x cols spin-1/2 lattice, site = r*cols + c. Bonds: all
    horizontal (row-major), then all vertical (row-major). Bond b carries
    J_b ~ U[0.5, 1.5] and Delta_b ~ U[0.8, 1.2]; then fields h_i ~ U[-0.5, 0.5].
    Draw order: J (all bonds), Delta (all bonds), h (all sites).
    H = sum_b J_b (SxSx + SySy + Delta_b SzSz) + sum_i h_i Sz_i.
    meta maps each physical parameter to its term indices:
      meta["J"][b]     -> (t_xx, t_yy, t_zz)   coef(t_zz) = J_b * Delta_b
      meta["h"][i]     -> t_z
    """
    rng = np.random.default_rng(seed)
    bonds = []
    for r in range(rows):
        for c in range(cols - 1):
            bonds.append((r * cols + c, r * cols + c + 1))
    for r in range(rows - 1):
        for c in range(cols):
            bonds.append((r * cols + c, (r + 1) * cols + c))
    nb = len(bonds)
    J = rng.uniform(0.5, 1.5, size=nb)
    Delta = rng.uniform(0.8, 1.2, size=nb)
    n = rows * cols
    h = rng.uniform(-0.5, 0.5, size=n)
    sites = [(SPIN, 2)] * n
    terms = []
    meta = {"J": [], "h": [], "Jv": J.tolist(), "Deltav": Delta.tolist(), "hv": h.tolist(),
            "bonds": bonds}
    for b, (i, j) in enumerate(bonds):
        t0 = len(terms)
        terms += [(i, "Sx", j, "Sx", float(J[b])), (i, "Sy", j, "Sy", float(J[b])),
                  (i, "Sz", j, "Sz", float(J[b] * Delta[b]))]
        meta["J"].append((t0, t0 + 1, t0 + 2))
    for i in range(n):
        meta["h"].append(len(terms))
        terms.append((i, "Sz", -1, "I", float(h[i])))
    return Model(f"square_xxz_{rows}x{cols}", sites, terms, meta)


def tavis_cummings(nspins=24, nlevels=64, omega=1.0, omega0=1.0, seed=7,
                   boson_first=False) -> Model:
    """Tavis-Cummings: nspins spin-1/2 sites plus one boson mode truncated to
    nlevels levels (App. C): H = omega N + omega0 sum Sz_i
    + sum_i g_i (adag Sm_i + a Sp_i), g_i ~ U[0.05, 0.15] (seed, site order).
    The boson is the last site unless boson_first."""
    rng = np.random.default_rng(seed)
    g = rng.uniform(0.05, 0.15, size=nspins)
    spins = list(range(1, nspins + 1)) if boson_first else list(range(nspins))
    b = 0 if boson_first else nspins
    sites = [None] * (nspins + 1)
    sites[b] = (BOSON, nlevels)
    for s in spins:
        sites[s] = (SPIN, 2)
    terms = [(b, "N", -1, "I", omega)]
    for k, s in enumerate(spins):
        terms.append((s, "Sz", -1, "I", omega0))
    for k, s in enumerate(spins):
        terms.append((b, "adag", s, "Sm", float(g[k])))
        terms.append((b, "a", s, "Sp", float(g[k])))
    return Model(f"tavis_cummings_n{nspins}_l{nlevels}", sites, terms, {"g": g.tolist(), "boson": b})


def paper_c1_chain() -> Model:
    """Uniform spin-1 periodic chain, N=15, XXZ Jxy=Jz=1, staggered field
    +0.2 on site 0, alternating (Sec. V testbed 1; D = 3^15)."""
    n = 15
    sites = [(SPIN, 3)] * n
    terms = []
    for i in range(n):
        terms += xxz_bond(i, (i + 1) % n, 1.0, 1.0)
    for i in range(n):
        terms.append((i, "Sz", -1, "I", 0.2 if i % 2 == 0 else -0.2))
    return Model("paper_c1_spin1_pbc_n15", sites, terms)


def paper_c2_chain() -> Model:
    """Mixed-spin periodic chain (1/2)^6 (1)^6 (3/2)^6, XXZ Jxy=Jz=1, staggered
    field +-0.2 (Sec. V testbed 2; D = 24^6)."""
    dims = [2] * 6 + [3] * 6 + [4] * 6
    n = len(dims)
    sites = [(SPIN, d) for d in dims]
    terms = []
    for i in range(n):
        terms += xxz_bond(i, (i + 1) % n, 1.0, 1.0)
    for i in range(n):
        terms.append((i, "Sz", -1, "I", 0.2 if i % 2 == 0 else -0.2))
    return Model("paper_c2_mixed_pbc_n18", sites, terms)


# ----------------------------------------------------------------------------
# Random models for parity tests: every operator kind, odd dimensions
# ----------------------------------------------------------------------------

def random_model(dims, kinds=None, nterms=24, seed=0, real=True, hermitian=False) -> Model:
    """Random term list on the given local dims. With real=True only products
    whose matrices are real are drawn (Sy appears only as SySy). With
    hermitian=True each off-diagonal product is added together with its
    adjoint partner at the same coefficient."""
    rng = np.random.default_rng(seed)
    n = len(dims)
    kinds = kinds or [SPIN] * n
    sites = list(zip(kinds, dims))
    spin_real = ["Sz", "Sx", "Sp", "Sm", "Sz2", "Sp2", "Sm2", "I"]
    boson_ops = ["N", "a", "adag", "I"]
    adj = {"Sp": "Sm", "Sm": "Sp", "Sp2": "Sm2", "Sm2": "Sp2", "a": "adag", "adag": "a"}
    terms = []
    while len(terms) < nterms:
        i = int(rng.integers(0, n))
        two = n > 1 and rng.random() < 0.7
        j = int(rng.integers(0, n - 1)) if two else -1
        if two and j >= i:
            j += 1
        pool_i = boson_ops if kinds[i] == BOSON else spin_real
        oi = pool_i[int(rng.integers(0, len(pool_i)))]
        if two:
            pool_j = boson_ops if kinds[j] == BOSON else spin_real
            oj = pool_j[int(rng.integers(0, len(pool_j)))]
        else:
            oj = "I"
        if kinds[i] == SPIN and two and kinds[j] == SPIN and rng.random() < 0.15:
            oi, oj = "Sy", "Sy"
        c = float(rng.normal())
        terms.append((i, oi, j, oj, c))
        if hermitian:
            ai, aj = adj.get(oi, oi), adj.get(oj, oj)
            if (ai, aj) != (oi, oj):
                terms.append((i, ai, j, aj, c))
    return Model(f"random_{'_'.join(map(str, dims))}_s{seed}", sites, terms)


def vector(D: int, seed: int, nvec: int = 1, normalize=True, dtype=np.float64):
    """x ~ N(0,1) with default_rng(seed), shape (D, nvec) flattened state-major
    (x[k*nvec + v]); each column normalised to unit 2-norm if requested."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((D, nvec))
    if normalize:
        x /= np.linalg.norm(x, axis=0, keepdims=True)
    return np.ascontiguousarray(x.reshape(-1)).astype(dtype)


def torch_vector(D: int, seed: int, nvec: int = 1, device="cuda", dtype=None, normalize=True):
    """Large-D variant drawn on the device with torch's Philox generator
    (seeded); used where a host draw of ~1e9 numbers would dominate."""
    import torch
    dtype = dtype or torch.float64
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    x = torch.randn((D, nvec), generator=g, device=device, dtype=torch.float32).to(dtype)
    if normalize:
        x /= torch.linalg.vector_norm(x.double(), dim=0, keepdim=True).to(dtype)
    return x.reshape(-1).contiguous()


# ---------------------------------------------------------------------------
# Counter-based input vectors for sizes whose x cannot be held on the host:
# x_i = (splitmix64 output number i+1 from state `seed`) >> 11, times 2^-53,
# minus 1/2. splitmix64 is the published generator of Steele, Lea and Flood
# (OOPSLA 2014). The oracle implements the same definition in C on its own.
# ---------------------------------------------------------------------------
_SM_GAMMA = 0x9E3779B97F4A7C15
_SM_M1 = 0xBF58476D1CE4E5B9
_SM_M2 = 0x94D049BB133111EB


def hashed_values(seed, idx, f32=False):
    """numpy: the synthesised x at the given indices (float64; rounded to
    float first when f32)."""
    i = np.asarray(idx, dtype=np.int64).astype(np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed % 2 ** 64) + (i + np.uint64(1)) * np.uint64(_SM_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_SM_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_SM_M2)
        z = z ^ (z >> np.uint64(31))
    v = (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 - 0.5
    return v.astype(np.float32).astype(np.float64) if f32 else v


def _signed64(u):
    return u - 2 ** 64 if u >= 2 ** 63 else u


def torch_hashed_vector(D, seed, dtype=None, device="cuda", chunk=1 << 26):
    """torch: the synthesised x of length D built on the device in chunks
    (int64 arithmetic wraps like uint64; shifts are made logical by masks)."""
    import torch
    dtype = dtype or torch.float64
    out = torch.empty(D, dtype=dtype, device=device)
    g, m1, m2 = (torch.tensor(_signed64(c), dtype=torch.int64, device=device) for c in (_SM_GAMMA, _SM_M1, _SM_M2))
    sd = torch.tensor(_signed64(seed % 2 ** 64), dtype=torch.int64, device=device)

    def shr(z, k):
        return (z >> k) & ((1 << (64 - k)) - 1)

    for a in range(0, D, chunk):
        b = min(D, a + chunk)
        z = sd + (torch.arange(a, b, dtype=torch.int64, device=device) + 1) * g
        z = (z ^ shr(z, 30)) * m1
        z = (z ^ shr(z, 27)) * m2
        z = z ^ shr(z, 31)
        v = shr(z, 11).to(torch.float64) * 2.0 ** -53 - 0.5
        out[a:b] = v.to(dtype)
        del z, v
    return out
