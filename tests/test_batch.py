"""Batched path: 24 problems of mixed sizes (8 each at 64^3, 128^3 and 192^3,
K = 2N, M = 2N, azimuth counts from {90, 180, 360} and polar counts from
{64, 128}) run as one CUDA-graph replay, tiles chosen by the autotuner.

Per item the graph result equals the plan's direct forward/adjoint (same
kernels); every item's forward matches the FP64 oracle on sampled lines, and
every item's adjoint matches it element by element on line data supported on
a few lines, in the variants the autotuner chose; the adjoint also passes the
dot-product identity for every item.
"""
import numpy as np
import pytest

from oracle import nufft3d_oracle as O
from paper_1605_05231_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _items(works):
    return [dict(n=w.n, dirs=w.directions(), m=w.m, k=w.k, j=w.j, table_oversamp=w.table_oversamp) for w in works]


def _rel(a, b):
    import torch

    return float(torch.linalg.norm((a - b).to(torch.complex128)) / torch.linalg.norm(b.to(torch.complex128)))


@pytest.fixture(scope="module")
def batch_run(cuda_lib, tmp_path_factory):
    import torch

    from paper_1605_05231_gb300 import autotune

    works = I.batched_workloads()
    assert len(works) == 24 and sorted({w.n for w in works}) == [64, 128, 192]
    b = cuda_lib.Batch(_items(works))
    cache = str(tmp_path_factory.mktemp("tune") / "tune.json")
    chosen = autotune.tune_batch(b, candidates=((3, 3, 512, 8), (3, 2, 1024, 8), (2, 2, 1024, 8)),
                                 reps=1, cache=cache)
    assert len(chosen) == len({autotune.signature(p) for p in b.items})
    vols = [torch.from_numpy(w.volume(np.float32)).cuda() for w in works]
    lines = [torch.empty((p.n_dirs, p.m), dtype=torch.complex64, device="cuda") for p in b.items]
    outs = [torch.empty_like(v) for v in vols]
    b.forward_adjoint(vols, lines, outs)
    first = [o.clone() for o in outs]
    b.forward_adjoint(vols, lines, outs)  # graph replay
    torch.cuda.synchronize()
    yield b, works, vols, lines, outs, first
    b.close()


def test_batch_replay_matches_direct_path(cuda_lib, batch_run):
    import torch

    b, works, vols, lines, outs, first = batch_run
    for p, v, l, o, f in zip(b.items, vols, lines, outs, first):
        assert p.sync_status() == 0
        ref_l = p.forward(v)
        ref_o = p.adjoint(ref_l)
        assert _rel(l, ref_l) < 1e-6
        assert _rel(o, ref_o) < 1e-6
        assert _rel(f, ref_o) < 1e-6


def test_batch_items_forward_match_oracle(cuda_lib, batch_run):
    """Every item's graph-replayed forward against the FP64 oracle on 16
    sampled lines of that item."""
    b, works, vols, lines, outs, first = batch_run
    worst = 0.0
    for i, w in enumerate(works):
        dirs = w.directions()
        sel = np.sort(np.random.default_rng(1000 + i).choice(dirs.shape[0], 16, replace=False))
        op = O.OraclePlan(w.n, w.k, w.j, w.table_oversamp, dirs, w.m)
        ref = O.nufft_forward(vols[i].cpu().numpy().astype(np.float64), op, lines=sel)
        err = O.rel_l2(lines[i].cpu().numpy()[sel], ref)
        worst = max(worst, err)
        assert err < TOL, (i, w.n, err)
    print(f"batch forward, worst per-item rel-L2 vs FP64 oracle: {worst:.3e}")


def test_batch_items_adjoint_match_oracle(cuda_lib, batch_run):
    """Every item's adjoint, element by element, in the kernel variants the
    autotuner chose for the graph: line data that vanish outside 16 random lines
    go through the item's plan, whose adjoint then equals the oracle's adjoint
    of a plan of only those lines."""
    import torch

    b, works, vols, lines, outs, first = batch_run
    worst = 0.0
    for i, (w, p) in enumerate(zip(works, b.items)):
        dirs = w.directions()
        sel = np.sort(np.random.default_rng(2000 + i).choice(dirs.shape[0], 16, replace=False))
        ys = I.random_lines(sel.size, w.m, 100 + i).astype(np.complex64)
        y = np.zeros((dirs.shape[0], w.m), dtype=np.complex64)
        y[sel] = ys
        a = p.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
        assert p.sync_status() == 0
        op = O.OraclePlan(w.n, w.k, w.j, w.table_oversamp, dirs[sel], w.m)
        err = O.rel_l2(a, O.nufft_adjoint(ys.astype(np.complex128), op))
        worst = max(worst, err)
        assert err < TOL, (i, w.n, err)
    print(f"batch adjoint, worst per-item rel-L2 vs FP64 oracle: {worst:.3e}")


def test_batch_items_adjoint_dot_product(cuda_lib, batch_run):
    import torch

    b, works, vols, lines, outs, first = batch_run
    for i, p in enumerate(b.items):
        y = torch.from_numpy(I.random_lines(p.n_dirs, p.m, 100 + i).astype(np.complex64)).cuda()
        Ax = lines[i].to(torch.complex128)
        Ahy = p.adjoint(y).to(torch.float64)
        lhs = torch.sum(torch.conj(y.to(torch.complex128)) * Ax).real
        rhs = torch.sum(Ahy * vols[i].to(torch.float64))
        rel = abs(float(lhs - rhs)) / float(torch.linalg.norm(Ax) * torch.linalg.norm(y.to(torch.complex128)))
        assert rel < 1e-6, (i, rel)


def test_batch_recaptures_on_new_buffers(cuda_lib):
    import torch

    works = I.batched_workloads()[:3]
    b = cuda_lib.Batch(_items(works))
    vols = [torch.from_numpy(w.volume(np.float32)).cuda() for w in works]
    lines = [torch.empty((p.n_dirs, p.m), dtype=torch.complex64, device="cuda") for p in b.items]
    outs = [torch.empty_like(v) for v in vols]
    b.forward_adjoint(vols, lines, outs)
    outs2 = [torch.empty_like(v) for v in vols]
    b.forward_adjoint(vols, lines, outs2)
    torch.cuda.synchronize()
    for o, o2 in zip(outs, outs2):
        assert _rel(o2, o) < 1e-6
    b.close()


@pytest.fixture(scope="module")
def grouped_run(cuda_lib):
    """Nine items (three each at 64^3, 128^3, 192^3) with exact coefficients
    and grouping switched on: the default kernels, so the items of each size
    form one group whose gather and spread are single launches over all three
    plans."""
    import torch

    works = [w for w in I.batched_workloads() if w.n == 64][:3] + \
            [w for w in I.batched_workloads() if w.n == 128][:3] + \
            [w for w in I.batched_workloads() if w.n == 192][:3]
    items = [dict(n=w.n, dirs=w.directions(), m=w.m, k=w.k, j=w.j, exact_coeffs=True) for w in works]
    b = cuda_lib.Batch(items)
    b.set_grouping(True)
    assert all((p.info()["gather_variant"], p.info()["spread_variant"]) == (10, 7) for p in b.items)
    vols = [torch.from_numpy(w.volume(np.float32)).cuda() for w in works]
    lines = [torch.empty((p.n_dirs, p.m), dtype=torch.complex64, device="cuda") for p in b.items]
    outs = [torch.empty_like(v) for v in vols]
    b.forward_adjoint(vols, lines, outs)
    b.forward_adjoint(vols, lines, outs)  # replay
    torch.cuda.synchronize()
    yield b, works, vols, lines, outs
    b.close()


def test_grouped_batch_matches_direct_path_and_ungrouped(cuda_lib, grouped_run):
    import torch

    b, works, vols, lines, outs = grouped_run
    for p, v, l, o in zip(b.items, vols, lines, outs):
        assert p.sync_status() == 0
        ref_l = p.forward(v)
        ref_o = p.adjoint(ref_l)
        assert _rel(l, ref_l) < 1e-6
        assert _rel(o, ref_o) < 1e-6
    b.set_grouping(False)
    lines2 = [torch.empty_like(l) for l in lines]
    outs2 = [torch.empty_like(o) for o in outs]
    b.forward_adjoint(vols, lines2, outs2)
    torch.cuda.synchronize()
    for l, o, l2, o2 in zip(lines, outs, lines2, outs2):
        assert _rel(l2, l) < 1e-6 and _rel(o2, o) < 1e-6
    b.set_grouping(True)


def test_grouped_batch_items_match_oracle(cuda_lib, grouped_run):
    """One item of each size: the grouped forward on 8 sampled lines, and the
    adjoint of the grouped graph's own forward output checked through the
    dot-product identity, against the FP64 oracle's exact-coefficient variant."""
    import torch

    b, works, vols, lines, outs = grouped_run
    for i in (0, 3, 6):
        w = works[i]
        dirs = w.directions()
        sel = np.sort(np.random.default_rng(3000 + i).choice(dirs.shape[0], 8, replace=False))
        op = O.OraclePlan(w.n, w.k, w.j, 0, dirs, w.m)
        ref = O.nufft_forward(vols[i].cpu().numpy().astype(np.float64), op, lines=sel)
        assert O.rel_l2(lines[i].cpu().numpy()[sel], ref) < TOL, i
        # <A x, A x> = <x, A^H A x>: the graph's adjoint of its own forward
        Ax = lines[i].to(torch.complex128)
        lhs = float(torch.sum(torch.abs(Ax) ** 2))
        rhs = float(torch.sum(outs[i].to(torch.float64) * vols[i].to(torch.float64)))
        assert abs(lhs - rhs) / lhs < 1e-6, (i, lhs, rhs)
