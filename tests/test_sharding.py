"""Radial-shell sharding on CPU: the slab partition, the exclusive prefix over ranks
(gloo process groups of 2 and 3 ranks) and the decomposition of the recurrences it
relies on, checked on the oracle's own sums."""
import os
import socket
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2602_02507_gb300.sharding import outer_from_totals, slab_of  # noqa: E402


def test_slabs_cover_the_shells_in_order():
    for n_r, world in ((10, 3), (2048, 8), (5, 5), (7, 2)):
        spans = [slab_of(n_r, r, world) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == n_r
        assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
        sizes = [b - a for a, b in spans]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        slab_of(3, 0, 4)


def test_outer_sums_are_the_exclusive_prefix_and_suffix():
    rng = np.random.default_rng(3)
    T = torch.from_numpy(rng.standard_normal((4, 2, 9)))
    for rank in range(4):
        out = outer_from_totals(T, rank)
        np.testing.assert_allclose(out[0].numpy(), T[:rank, 0].sum(0).numpy() if rank else 0.0, rtol=1e-15, atol=0)
        np.testing.assert_allclose(out[1].numpy(), T[rank + 1:, 1].sum(0).numpy() if rank < 3 else 0.0,
                                   rtol=1e-15, atol=0)


def test_slab_recurrences_plus_outer_sums_equal_the_whole_mesh():
    """The oracle's edge moments of a whole mesh equal, on every slab, the slab's own
    recurrences started from the other slabs' totals (the algebra mp_slab_potential uses)."""
    from oracle import oracle as O
    from paper_2602_02507_gb300 import workloads as W
    w = W.random_small((9, 6, 8), 4, seed=5, r0=0.0, r1=1.0, uneven=True)
    m = w.mesh
    tab = O.build_tables(m.r, m.theta, m.phi, m.L)
    ref = O.solve(tab, w.rho, m.G)
    A, WR, WI = ref["A"], tab.WR, tab.WI
    lq = np.repeat(np.arange(m.L + 1), 2 * np.arange(m.L + 1) + 1)
    wR = WR[lq].T * A                       # [n_r][K_L] terms of the regular recurrence
    wI = np.where(np.isfinite(WI), WI, 0.0)[lq].T * A
    world = 3
    spans = [slab_of(9, r, world) for r in range(world)]
    totals = torch.from_numpy(np.stack([np.stack([wR[a:b].sum(0), wI[a:b].sum(0)]) for a, b in spans]))
    for rank, (a, b) in enumerate(spans):
        outer = outer_from_totals(totals, rank).numpy()
        MR = outer[0] + np.concatenate([np.zeros((1, wR.shape[1])), np.cumsum(wR[a:b], axis=0)])
        MI = outer[1] + np.concatenate([np.cumsum(wI[a:b][::-1], axis=0)[::-1], np.zeros((1, wI.shape[1]))])
        scale = np.abs(ref["MR"]).max() + np.abs(ref["MI"][1:]).max()
        np.testing.assert_allclose(MR, ref["MR"][a:b + 1], rtol=0, atol=1e-13 * scale)
        # edge 0 of the origin shell excludes its divergent own term (l >= 2) in the oracle
        lo = 1 if a == 0 else 0
        np.testing.assert_allclose(MI[lo:], ref["MI"][a + lo:b + 1], rtol=0, atol=1e-13 * scale)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2602_02507_gb300.sharding import exchange_slab_totals
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        totals = torch.from_numpy(np.random.default_rng(100 + rank).standard_normal((2, 25)))
        outer = exchange_slab_totals(totals)
        np.save(os.path.join(out_dir, f"outer{rank}.npy"), outer.numpy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_over_gloo_ranks(tmp_path, world):
    import torch.multiprocessing as mp
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    T = np.stack([np.random.default_rng(100 + r).standard_normal((2, 25)) for r in range(world)])
    for rank in range(world):
        got = np.load(tmp_path / f"outer{rank}.npy")
        want = np.stack([T[:rank, 0].sum(0) if rank else np.zeros(25),
                         T[rank + 1:, 1].sum(0) if rank < world - 1 else np.zeros(25)])
        np.testing.assert_allclose(got, want, rtol=1e-15, atol=1e-15)
