"""CPU emulation of the apply kernel's algorithm on the exported plan tables.

It follows the per-block steps of the CUDA kernel (high digits, block-uniform
channels, factorised groups, ELL inside the low block) in numpy, so the
host-side plan builder can be checked against the oracle without a GPU. It
is test infrastructure: the oracle never uses it, and it never uses the
oracle."""
import numpy as np


def emulate(P, x):
    D, B, nblk, nhigh = P["D"], P["B"], P["nblk"], P["nhigh"]
    sites = P["sites"]  # [M, mh, d, lbit, lwid, is_low]
    tab = np.asarray(P["tab"], dtype=np.float64)
    ptab = np.asarray(P["ptab"], dtype=np.int64)
    diag = np.asarray(P["diag"], dtype=np.float64)
    ell_w = P["ell_w"]
    ell_d = np.asarray(P["ell_delta"], dtype=np.int64).reshape(max(ell_w, 0), B) if ell_w else None
    ell_c = np.asarray(P["ell"], dtype=np.float64).reshape(max(ell_w, 0), B) if ell_w else None
    ch, grp, mem = P["ch"], P["grp"], P["mem"]
    nhd, ngd = P["n_hh_diag"], P["n_grp_diag"]
    lo = np.arange(B)
    x = np.asarray(x, dtype=np.float64)
    y = np.zeros(D)

    def low_digit(bit, wid):
        return (ptab >> bit) & ((1 << wid) - 1)

    for blk in range(nblk):
        hd = [(blk // sites[t][1]) % sites[t][2] for t in range(nhigh)]
        hh_c = []
        for off, tb, dj, si, sj, kind in ch:
            nj = 0 if (kind & 8) else hd[sj]
            hh_c.append(tab[tb + hd[si] * dj + nj])
        mem_u = [tab[ut + hd[us]] for _, ut, us in mem]
        grp_v = [vt + (hd[vs] * vst if vst else 0) for vt, vst, _, _, vs, _, _ in grp]
        base = blk * B
        ds = np.full(B, sum(hh_c[:nhd])) + diag
        for g in range(ngd):
            vt, vst, m0, m1, vs, lb, lw = grp[g]
            U = sum(mem_u[m0:m1])
            ds = ds + tab[grp_v[g] + low_digit(lb, lw)] * U
        acc = ds * x[base + lo]
        for c in range(nhd, len(ch)):
            if hh_c[c] == 0.0:
                continue
            acc = acc + hh_c[c] * x[base + ch[c][0] + lo]
        for g in range(ngd, len(grp)):
            vt, vst, m0, m1, vs, lb, lw = grp[g]
            v = tab[grp_v[g] + low_digit(lb, lw)]
            pr = v != 0.0
            ag = np.zeros(B)
            for m in range(m0, m1):
                u = mem_u[m]
                if u == 0.0:
                    continue
                src = base + lo[pr] + mem[m][0]
                assert src.min(initial=0) >= 0 and src.max(initial=0) < D, "group member reads out of range"
                ag[pr] += u * x[src]
            acc = acc + v * ag
        for w in range(ell_w):
            cf = ell_c[w]
            nz = cf != 0.0
            src = base + lo[nz] + ell_d[w][nz]
            assert src.min(initial=0) >= 0 and src.max(initial=0) < D, "ELL reads out of range"
            acc[nz] += cf[nz] * x[src]
        y[base:base + B] = acc
    return y
