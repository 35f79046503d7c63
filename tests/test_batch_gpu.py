"""Batched coupling: many uneven FP32 instances in one persistent launch per
phase.

* Every field of every instance is bit-identical to cg_step of that
  instance alone (its own grids handle, same buffers), for any
  decomposition (digit width, items per thread, grid size), eagerly and
  as a replayed CUDA graph.  The FP64 conservation sums are merged from
  per-block partials whose per-thread FP32 accumulations depend on the
  decomposition: they agree within the FP32 path tolerance of their scale.
* One instance against the FP64 oracle within the FP32 path tolerance.
* The Euler advance, the autotuner (and its cache) and argument checks.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import TOL_FP32, assert_close, assert_close_interp, to_dev, to_np

pytestmark = pytest.mark.gpu

FIELDS = ("eps_bulk", "u_bulk", "var_bulk", "S_bulk", "force", "S_fine", "eps_fine")


def small_batch():
    """Seven instances: fine edges 16..48, ratios 2/4/8, 1 to ~60,000
    particles (one tile, ragged tiles); five take the digit sort (one and
    two passes), two the per-cell sort, in one batch (one by one, cg_step
    picks the sort by its own rule: the fields must agree either way)."""
    specs = [(16, 2, 1, 0.01), (32, 4, 5000, 0.01), (48, 8, 61_000, 0.004), (32, 2, 40_000, 0.006),
             (16, 4, 4097, 0.02), (48, 4, 12_345, 0.003), (40, 8, 30_000, 0.005)]
    ws = [synth.batch_instance(5, k, e, r, n, d) for k, (e, r, n, d) in enumerate(specs)]
    for k in (3, 5):
        ws[k].desc["sort_digits"] = 1   # CG_SORT_CELLS
    return ws


def make_batch(cg, ws, eps_fine=(True,), var=(True,)):
    import torch
    inst, tensors = [], []
    for k, w in enumerate(ws):
        g = cg.Grids(w.desc)
        out = g.alloc_outputs(w.n, var=var[k % len(var)], eps_fine=eps_fine[k % len(eps_fine)])
        g.close()
        pos = to_dev(w.pos_d)
        vel = to_dev(w.vel)
        uf = to_dev(w.u_fine.reshape(3, -1))
        inst.append((w.desc, pos, vel, uf, out))
        tensors.append((pos, vel, uf, out))
    return cg.Batch(inst), tensors


def snapshot(tensors):
    import torch
    torch.cuda.synchronize()
    return [{k: (to_np(v) if v is not None else None) for k, v in out.items()} for _, _, _, out in tensors]


def assert_same(a, b, sums_tol=TOL_FP32):
    for i, (x, y) in enumerate(zip(a, b)):
        for k in FIELDS:
            if x.get(k) is None:
                continue
            assert np.array_equal(x[k], y[k]), (i, k)
        s, t = x["sums"], y["sums"]
        # volumes relative to sum V_p, forces and sources to sum |F|
        scale = np.array([abs(t[0])] * 2 + [abs(t[11])] * 14)
        assert np.all(np.abs(s - t) <= sums_tol * scale), (i, s, t)


def one_by_one(b, n, dt=0.0):
    for i in range(n):
        b.step_one(i, dt)


def test_batched_equals_one_by_one_and_oracle(cuda_lib):
    ws = small_batch()
    b, tens = make_batch(cuda_lib, ws, eps_fine=(True, False), var=(True, True, False))
    b.step()
    rc, flags, counts = b.sync_status()
    assert rc == 0 and counts[0] == 0 and counts[1] == 0
    got = snapshot(tens)
    one_by_one(b, len(ws))
    want = snapshot(tens)
    assert_same(got, want)
    # instance 3 against the FP64 oracle
    w = ws[3]
    ref = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine)
    for k in ("eps_bulk", "var_bulk"):
        assert_close(k, got[3][k], ref[k], TOL_FP32)
    for k in ("u_bulk", "S_bulk", "force"):
        assert_close(k, got[3][k], ref[k], TOL_FP32, vec=True)
    # the projection interpolates S_B of either sign: its FP32 rounding is
    # relative to the interpolant of |S_B|, which the oracle projects too
    ref_abs = oracle.project(w.desc, np.abs(ref["S_bulk"]))
    assert_close_interp("S_fine", got[3]["S_fine"], ref["S_fine"], ref_abs, TOL_FP32)
    # the single-particle instance: its cell alone holds the particle
    assert np.count_nonzero(got[0]["eps_bulk"] < 1.0) == 1
    # both sorts in one batch: the digit sort's 5 launches beside the per-cell
    # sort's 2 (key and scan shared), 19 in all
    assert b.launches_per_step() <= 19
    b.close()


@pytest.mark.parametrize("cfg", [dict(digit_bits=8), dict(digit_bits=9, drag_items=4, avg_items=2),
                                 dict(seg_chunks=4, grid_mult=2), dict(drag_items=8, seg_chunks=2, grid_mult=4)])
def test_decomposition_does_not_change_results(cuda_lib, cfg):
    ws = small_batch()
    b, tens = make_batch(cuda_lib, ws)
    b.step()
    base = snapshot(tens)
    b.set_config(**cfg)
    assert all(b.config()[k] == v for k, v in cfg.items())
    b.step()
    assert_same(snapshot(tens), base)
    b.close()


def test_graph_replay_equals_eager(cuda_lib):
    ws = small_batch()
    b, tens = make_batch(cuda_lib, ws)
    b.step()
    base = snapshot(tens)
    b.use_graph(True)
    l0 = b.launch_count()
    for _ in range(3):
        b.step()
    assert b.launch_count() - l0 == 3 * b.launches_per_step()
    assert_same(snapshot(tens), base, sums_tol=0.0)
    b.step_each()          # the one-by-one sequence as a graph
    b.step_each()
    assert_same(snapshot(tens), base)
    assert b.sync_status()[0] == 0
    b.close()


def test_euler_advance_batched_equals_one_by_one(cuda_lib):
    ws = small_batch()
    dt = 1e-3
    b1, t1 = make_batch(cuda_lib, ws)
    b1.step(dt)
    b1.step(dt)
    b2, t2 = make_batch(cuda_lib, ws)
    one_by_one(b2, len(ws), dt)
    one_by_one(b2, len(ws), dt)
    import torch
    torch.cuda.synchronize()
    for (p1, v1, _, _), (p2, v2, _, _) in zip(t1, t2):
        assert torch.equal(p1, p2) and torch.equal(v1, v2)
    assert_same(snapshot(t1), snapshot(t2))
    b1.close()
    b2.close()


def test_autotuner_picks_a_valid_config_and_caches_it(cuda_lib, tmp_path):
    ws = small_batch()
    b, tens = make_batch(cuda_lib, ws)
    b.step()
    base = snapshot(tens)
    cache = tmp_path / "tune.txt"
    cfg, ms = b.tune(reps=3, cache_path=cache)
    assert ms > 0 and 8 <= cfg["digit_bits"] <= 11
    assert cache.read_text().count("\n") == 1
    cfg2, ms2 = b.tune(reps=3, cache_path=cache)
    assert cfg2 == cfg and ms2 == -1.0
    b.step()
    assert_same(snapshot(tens), base)
    b.close()


def test_bad_items_are_rejected(cuda_lib):
    import torch
    cg = cuda_lib
    w = synth.batch_instance(0, 0, 16, 4, 100, 0.01)
    g = cg.Grids(w.desc)
    out = g.alloc_outputs(w.n)
    g.close()
    pos, vel, uf = to_dev(w.pos_d), to_dev(w.vel), to_dev(w.u_fine.reshape(3, -1))
    for bad in (dict(fp64=True), dict(ratio=3, fine_n=(18, 18, 18))):
        d = dict(w.desc)
        d.update(bad)
        with pytest.raises(cg.CgError):
            cg.Batch([(d, pos, vel, uf, out)])
    o2 = dict(out)
    o2["cell"] = torch.empty(w.n, dtype=torch.int32, device="cuda")
    with pytest.raises(cg.CgError):
        cg.Batch([(w.desc, pos, vel, uf, o2)])
    with pytest.raises(cg.CgError):
        cg.Batch([(w.desc, pos[:0], vel[:0], uf, out)])
