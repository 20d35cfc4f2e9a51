"""The multi-rank path on CPU: instances of an ensemble are sharded across
ranks with no data-path collective (world_size 2, gloo). Each rank applies
its own members (here with the oracle, the CPU stand-in for the GPU apply);
rank 0 gathers the results and checks them against one process doing all
of them, and checks the timing reductions the benchmark uses."""
import os
import socket

import numpy as np
import pytest

from paper_2606_02169_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_every_instance_once():
    rng = np.random.default_rng(0)
    for ws in (1, 2, 3, 8):
        costs = [float(3 ** int(n)) for n in rng.integers(3, 9, size=37)]
        parts = shard.partition(costs, ws)
        assert len(parts) == ws
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        # greedy bound: the heaviest rank exceeds the mean by at most one instance
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= sum(costs) / ws + max(costs) + 1e-9
        for r in range(ws):
            assert shard.owned(costs, r, ws) == parts[r]


def test_partition_is_balanced_on_the_disorder_ensemble_shape():
    import workloads as W
    # chain lengths of the 256-chain spin-1 ensemble (seeded exactly as the
    # ensemble generator draws them), cost = D_b x 16 right-hand sides
    sizes = []
    for b in range(256):
        rng = np.random.default_rng(1000 + b)
        n = int(8 + rng.integers(0, 7))
        sizes.append(3 ** n * 16)
    models = W.disorder_ensemble(4, 8, 14, 1000)
    assert [3 ** len(m.sites) * 16 for m in models] == sizes[:4]
    for ws in (2, 4, 8):
        parts = shard.partition(sizes, ws)
        assert shard.imbalance(sizes, parts) < 1.05


def test_partition_rejects_bad_arguments():
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)
    with pytest.raises(ValueError):
        shard.partition([-1.0], 2)
    with pytest.raises(ValueError):
        shard.owned([1.0, 2.0], 2, 2)


def test_reductions_without_a_process_group():
    assert shard.max_over_ranks(3.5) == 3.5
    assert shard.sum_over_ranks(2.0) == 2.0


def _worker(rank, world, port, out_dir):
    import torch.distributed as td

    import oracle
    import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        models = W.disorder_ensemble(10, 3, 6, 500)
        nvec = 2
        costs = [oracle.dimension(m.sites) * nvec for m in models]
        mine = shard.owned(costs, rank, world)
        res = {}
        for b in mine:
            m = models[b]
            D = oracle.dimension(m.sites)
            x = W.vector(D, 700 + b, nvec=nvec)
            res[b] = oracle.apply(m.sites, m.terms, x, nvec=nvec).real
        gathered = [None] * world
        td.all_gather_object(gathered, res)
        tmax = shard.max_over_ranks(float(rank + 1))
        tsum = shard.sum_over_ranks(float(sum(costs[b] for b in mine)))
        if rank == 0:
            merged = {}
            for part in gathered:
                assert not (set(part) & set(merged)), "an instance was applied on two ranks"
                merged.update(part)
            assert sorted(merged) == list(range(len(models)))
            for b, m in enumerate(models):
                D = oracle.dimension(m.sites)
                x = W.vector(D, 700 + b, nvec=nvec)
                ref = oracle.apply(m.sites, m.terms, x, nvec=nvec).real
                assert np.array_equal(merged[b], ref)
            assert tmax == float(world)
            assert tsum == float(sum(costs))
            with open(os.path.join(out_dir, "ok"), "w") as f:
                f.write("ok")
        td.barrier()
    finally:
        td.destroy_process_group()


def test_sharded_ensemble_on_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    assert (tmp_path / "ok").read_text() == "ok"


def test_slice_plans_cover_the_index_range_and_agree_between_ranks():
    import workloads as W
    for m in (W.ferrimagnet_chain(8), W.tavis_cummings(4, 8, seed=3), W.random_model([3, 2, 4, 2, 3], None, 20, 1)):
        D = int(np.prod([d for _, d in m.sites]))
        for world in (1, 2, 3, 4, 5):
            plans = [shard.slice_plan(m.sites, m.terms, world, r) for r in range(world)]
            assert plans[0].bounds[0] == 0 and plans[0].bounds[-1] == D
            assert all(p.bounds == plans[0].bounds for p in plans)
            assert all(b % plans[0].unit == 0 for b in plans[0].bounds)
            offs = shard.source_offsets(m.sites, m.terms)
            for p in plans:
                assert p.halo_lo <= p.lo and p.hi <= p.halo_hi
                assert p.halo_lo == max(0, p.lo + min(offs)) and p.halo_hi == min(D, p.hi + max(offs))
                for r, (a, b) in p.recv.items():      # what one rank receives the other sends
                    assert plans[r].send[p.rank] == (a, b)
                    assert p.bounds[r] <= a < b <= p.bounds[r + 1]


def _slice_worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as td

    import oracle
    import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ok = []
        for b, m in enumerate((W.ferrimagnet_chain(8), W.random_model([3, 2, 4, 2, 3, 2], None, 24, 3),
                               W.tavis_cummings(5, 6, seed=2))):
            D = oracle.dimension(m.sites)
            plan = shard.slice_plan(m.sites, m.terms, world, rank)
            x = W.vector(D, 900 + b)
            ext = shard.exchange_halo(plan, torch.from_numpy(x[plan.lo:plan.hi].copy()))
            assert np.array_equal(ext.numpy(), x[plan.halo_lo:plan.halo_hi])

            def apply_local(e, m=m, plan=plan, D=D):
                xf = np.zeros(D)
                xf[plan.halo_lo:plan.halo_hi] = e.numpy()    # nothing outside the halo is ever read
                return torch.from_numpy(oracle.apply(m.sites, m.terms, xf, row_begin=plan.lo, row_end=plan.hi).real)

            y_local = apply_local(ext).numpy()
            parts = [None] * world
            td.all_gather_object(parts, (plan.lo, plan.hi, y_local))
            if rank == 0:
                y = np.concatenate([p[2] for p in sorted(parts, key=lambda p: p[0])])
                ok.append(np.array_equal(y, oracle.apply(m.sites, m.terms, x).real))
            if b == 0:   # sharded Lanczos: two scalars summed over ranks per step
                v0 = W.vector(D, 31)
                a, bt, e0 = shard.sharded_lanczos(apply_local, plan, torch.from_numpy(v0[plan.lo:plan.hi].copy()),
                                                  160)
                if rank == 0:
                    w = np.linalg.eigvalsh(oracle.dense(m.sites, m.terms).real)
                    ok.append(abs(e0 - w[0]) < 1e-9 * abs(w[0]))
                    a1, b1, _, _ = oracle.lanczos(m.sites, m.terms, v0, 6)
                    ok.append(np.allclose(a[:6], a1[:6], rtol=1e-12) and np.allclose(bt[:5], b1[:5], rtol=1e-12))
        if rank == 0:
            assert all(ok), ok
            with open(os.path.join(out_dir, "ok"), "w") as f:
                f.write("ok")
        td.barrier()
    finally:
        td.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_single_hamiltonian_on_gloo_ranks(tmp_path, world):
    """One Hamiltonian cut into row slices over `world` gloo ranks: the halo
    exchange delivers exactly the x each rank's rows read, the merged rows
    equal the single-process oracle bit for bit, and the sharded Lanczos
    reaches the dense ground-state energy."""
    import torch.multiprocessing as mp
    mp.start_processes(_slice_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    assert (tmp_path / "ok").read_text() == "ok"
