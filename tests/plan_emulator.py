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


def emulate_tile(T, x):
    """The tile kernel's algorithm on its exported tables (hm_plan_export with
    the tile bit): blocks of R rows of F leaf states, per-row uniform members
    compacted by group, per-leaf-state diagonal, leaf factors and leaf hops.
    x: D*nvec values, state-major. Asserts that every gather is in range."""
    F, R, nblk, nvec = T["F"], T["R"], T["nblk"], T["nvec"]
    nhigh, G = T["nhigh"], T["G"]
    sites = T["sites"]
    tab = np.asarray(T["tab"], dtype=np.float64)
    mems = T["bmem"] + T["rmem"]
    dF = np.asarray(T["dF"], dtype=np.float64)
    v = np.asarray(T["v"], dtype=np.float64).reshape(G - 1, F) if G > 1 else np.zeros((0, F))
    fix = np.asarray(T["fix"], dtype=np.int64).reshape(G - 1, F) if G > 1 else np.zeros((0, F), np.int64)
    fs_w = T["fs_w"]
    fs_n = np.asarray(T["fs_n"], dtype=np.int64)
    fs_off = np.asarray(T["fs_off"], dtype=np.int64).reshape(-1, F)
    fs = np.asarray(T["fs"], dtype=np.float64).reshape(-1, F)
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    rowE = F * nvec
    t = np.arange(rowE)
    f = t // nvec
    y = np.zeros(n)

    def gather(idx):
        assert idx.min(initial=0) >= 0 and idx.max(initial=0) < n, "gather out of range"
        return x[idx]

    for blk in range(nblk):
        hd = [(blk // sites[s][0]) % sites[s][1] for s in range(nhigh)]
        for r in range(R):
            def digit(s):
                return hd[s] if s < nhigh else (r // sites[s][0]) % sites[s][1]
            k = (blk * R + r) * rowE + t
            lists = [[] for _ in range(G)]
            ud = np.zeros(G)
            for off, tb, db, sa, sb, g, dg in mems:
                u = tab[tb + digit(sa) * db + (digit(sb) if sb >= 0 else 0)]
                if dg:
                    ud[g] += u
                elif u != 0.0:
                    lists[g].append((off, u))
            xs = gather(k)
            acc = (ud[0] + dF[f]) * xs
            for g in range(1, G):
                acc = acc + v[g - 1][f] * (ud[g] * xs)
            for off, u in lists[0]:
                acc = acc + u * gather(k + off)
            for g in range(1, G):
                kk = k + fix[g - 1][f]
                ag = np.zeros(rowE)
                for off, u in lists[g]:
                    ag = ag + u * gather(kk + off)
                acc = acc + v[g - 1][f] * ag
            for w in range(fs_w):
                msk = w < fs_n[f]
                if not msk.any():
                    continue
                acc[msk] = acc[msk] + fs[w][f[msk]] * gather(k[msk] + fs_off[w][f[msk]])
            y[k] = acc
    return y


def emulate_sector(S, x, nvec=1):
    """The sector kernel's steps on exported sector tables (hm_plan_export
    bit 2), over all packed rows at once: unranking by the count tables, the
    coefficient of every channel from the target digits, the source row from
    the adjacent-site rank-delta table or the rank-table update over sites
    si..sj, and the diagonal channels summed before they multiply x_F."""
    Dsec, K = S["Dsec"], S["K"]
    K1 = K + 1
    d = S["d"]
    N = len(d)
    Aoff = S["Aoff"]
    cnt = np.asarray(S["cnt"], dtype=np.int64).reshape(N + 1, K1)
    A = np.asarray(S["A"], dtype=np.int64)
    dl = np.asarray(S["dl"], dtype=np.int64)
    lt = np.asarray(S["lt"], dtype=np.int64)
    tab = np.asarray(S["tab"], dtype=np.float64)
    F = np.arange(Dsec, dtype=np.int64)
    r = F.copy()
    left = np.full(Dsec, K, dtype=np.int64)
    dig = np.zeros((N, Dsec), dtype=np.int64)
    rem = np.zeros((N, Dsec), dtype=np.int64)
    for k in range(N):
        c = cnt[k + 1]
        m = np.zeros(Dsec, dtype=np.int64)
        active = np.ones(Dsec, dtype=bool)
        while active.any():
            idx = left - m
            cm = np.where(idx >= 0, c[np.clip(idx, 0, K)], 0)
            adv = active & (r >= cm)
            r[adv] -= cm[adv]
            m[adv] += 1
            active = adv
        dig[k], rem[k] = m, left
        left = left - m

    def Aat(k, t, n):
        return A[Aoff[k] + t * (d[k] + 1) + n]

    X = np.asarray(x, dtype=np.float64).reshape(Dsec, nvec)
    acc = np.zeros((Dsec, nvec))
    dsum = np.zeros(Dsec)
    for tb, dtab, rstride, dj, si, sj, qi, qj, diag in S["ch"]:
        ni = dig[si]
        nj = dig[sj] if sj >= 0 else np.zeros(Dsec, dtype=np.int64)
        ci = ni * dj + nj
        cf = tab[tb + ci]
        if diag:
            dsum += cf
            continue
        rows = np.flatnonzero(cf != 0)
        ni, nj, ci = ni[rows], nj[rows], ci[rows]
        if dtab >= 0:
            dlt = dl[dtab + rem[si][rows] * rstride + ci]
        elif dtab <= -2:                    # long move: per-site entries summed over si..sj
            off = -2 - dtab
            dlt = np.zeros(rows.size, dtype=np.int64)
            for k in range(si, sj + 1):
                dlt = dlt + lt[off + ((k - si) * K1 + rem[k][rows]) * rstride + dig[k][rows]]
        else:
            q = qi
            ri = rem[si][rows]
            dlt = Aat(si, ri, ni - q) - Aat(si, ri, ni)
            for k in range(si + 1, sj):
                rk, nk = rem[k][rows], dig[k][rows]
                dlt = dlt + Aat(k, rk + q, nk) - Aat(k, rk, nk)
            rj = rem[sj][rows]
            dlt = dlt + Aat(sj, rj + q, nj - qj) - Aat(sj, rj, nj)
        acc[rows] += cf[rows, None] * X[rows + dlt]
    return (acc + dsum[:, None] * X).reshape(-1)


def emulate_sector_blk(P, x, nvec=1):
    """The block-form sector kernel's steps on its exported tables (numpy,
    one prefix block at a time): prefix digits of the block, its suffix
    sector t = K - P, block-uniform prefix diagonal and moves, per-suffix
    diagonal and in-sector moves, coupled channels through the prefix
    digit's table row and the source-rank tables."""
    h, K, G, w = P["h"], P["K"], P["G"], P["w"]
    n0, n1, n2 = P["n0"], P["n1"], P["n2"]
    start = np.asarray(P["start"], dtype=np.int64)
    mp, pdim, off = P["mp"], P["pdim"], P["off"]
    sdig = np.asarray(P["sdig"], dtype=np.int64)
    tab = np.asarray(P["tab"], dtype=np.float64)
    dS = np.asarray(P["dS"], dtype=np.float64)
    ell_r = np.asarray(P["ell_r"], dtype=np.int64).reshape(w, G) if w else np.zeros((0, G), np.int64)
    ell = np.asarray(P["ell"], dtype=np.float64).reshape(w, G) if w else np.zeros((0, G))
    xr = np.asarray(P["xr"], dtype=np.int64).reshape(-1, G) if P["xr"] else np.zeros((0, G), np.int64)
    ch = [dict(zip(("kind", "tab", "dj", "si", "sj", "pfx", "qp", "xr", "dblk", "lbit", "lwid"), c)) for c in P["ch"]]
    X = np.asarray(x, dtype=np.float64).reshape(-1, nvec)
    Y = np.zeros_like(X)
    for b in P["vb"]:
        dig = [(b // mp[k]) % pdim[k] for k in range(h)]
        t = K - sum(dig)
        g = np.arange(off[t], off[t + 1])
        F = start[b] + np.arange(g.size)
        pk = sdig[g]
        digit = lambda c: (pk >> c["lbit"]) & ((1 << c["lwid"]) - 1)
        d = dS[g].copy()
        for c in ch[:n0]:
            d += tab[c["tab"] + dig[c["si"]] * c["dj"] + (dig[c["sj"]] if c["sj"] >= 0 else 0)]
        rows = {}
        for i, c in enumerate(ch[n1:], start=n1):
            npf = dig[c["sj"] if c["pfx"] else c["si"]]
            rows[i] = (c["tab"] + npf, c["dj"]) if c["pfx"] else (c["tab"] + npf * c["dj"], 1)
        for i in range(n1, n2):
            base, mul = rows[i]
            d += tab[base + mul * digit(ch[i])]
        acc = d[:, None] * X[F]
        for c in ch[n0:n1]:
            cf = tab[c["tab"] + dig[c["si"]] * c["dj"] + dig[c["sj"]]]
            if cf != 0.0:
                acc += cf * X[F + (start[b - c["dblk"]] - start[b])]
        for e in range(w):
            acc += ell[e, g][:, None] * X[F + ell_r[e, g]]
        for i in range(n2, len(ch)):
            c = ch[i]
            ps = c["sj"] if c["pfx"] else c["si"]
            if not 0 <= dig[ps] - c["qp"] < pdim[ps]:
                continue
            base, mul = rows[i]
            cf = tab[base + mul * digit(c)]
            nz = cf != 0.0
            src = start[b - c["dblk"]] + xr[c["xr"], g[nz]]
            acc[nz] += cf[nz, None] * X[src]
        Y[F] = acc
    return Y.reshape(-1)
