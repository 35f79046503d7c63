"""Incremental rebinning (the per-step particle-cell connectivity rebuild,
Sec. 2.2) started from the handle's previous binning, and the sorted step
that keeps the particles in cell order.

Every binning must equal the stable order by (cell, index) bit for bit,
whatever the particles did since the previous one: a few moved (the
incremental path), most moved or one cell received many (the device's
fallback to the per-cell sort), or the caller handed in another particle
set of the same count.  The reference is the oracle's binning of the same
positions, and a handle that sorts from scratch (a digit-sort descriptor)."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import TOL_FP32, assert_close, assert_close_slip, inputs, to_dev, to_np

pytestmark = pytest.mark.gpu

BINS = ("cell", "perm", "cell_start")


def _scratch_bins(cg, desc, pos):
    """Bins of pos from a handle that always sorts from scratch."""
    import torch
    d = dict(desc)
    d["sort_digits"] = 8
    g = cg.Grids(d)
    n = pos.shape[0]
    cell = torch.empty(n, dtype=torch.int32, device="cuda")
    perm = torch.empty_like(cell)
    cs = torch.empty(g.n_bulk + 1, dtype=torch.int32, device="cuda")
    g.cg_bin_particles(pos, cell, perm, cs)
    torch.cuda.synchronize()
    g.close()
    return {"cell": cell, "perm": perm, "cell_start": cs}


def _assert_bins_equal(got, ref, what):
    import torch
    for k in BINS:
        assert torch.equal(got[k], ref[k]), f"{what}: {k} differs"


def _assert_oracle_bins(w, pos, got, what):
    cell, perm, cs, _ = oracle.bin(w.desc, to_np(pos))
    assert np.array_equal(to_np(got["cell"]), cell), f"{what}: cells differ from the oracle"
    assert np.array_equal(to_np(got["perm"]), perm), f"{what}: permutation differs from the oracle"
    assert np.array_equal(to_np(got["cell_start"]), cs), f"{what}: cell starts differ from the oracle"


@pytest.mark.parametrize("fp64", [False, True])
def test_moving_steps_rebin_exactly_in_caller_order(cuda_lib, fp64):
    """12 advanced steps of the small clustered bed through cg_step (the
    particles keep the caller's order): each step's bins equal the oracle's
    for the positions it was given, and its fields equal those of a fresh
    handle's step on the same state bit for bit."""
    import torch
    cg = cuda_lib
    w = synth.small_clustered_bed(seed=11, fp64=fp64)
    g = cg.Grids(w.desc)
    pos, vel, uf = inputs(w)
    out = g.alloc_outputs(w.n, eps_fine=True, bins=True)
    for step in range(12):
        before = (pos.clone(), vel.clone())
        g.cg_step(pos, vel, uf, out, dt=w.dt)
        torch.cuda.synchronize()
        if step in (0, 1, 5, 11):
            _assert_oracle_bins(w, before[0], out, f"step {step}")
        if step in (1, 11):
            f = cg.Grids(w.desc)
            p2, v2 = before[0].clone(), before[1].clone()
            o2 = f.alloc_outputs(w.n, eps_fine=True, bins=True)
            f.cg_step(p2, v2, uf, o2, dt=w.dt)
            torch.cuda.synchronize()
            for k in ("cell", "perm", "cell_start", "eps_bulk", "u_bulk", "var_bulk", "force", "S_bulk", "S_fine",
                      "eps_fine"):
                assert torch.equal(out[k], o2[k]), (step, k)
            assert torch.equal(pos, p2) and torch.equal(vel, v2)
            f.close()
    assert g.cg_sync_status()[0] == 0
    g.close()


def test_sorted_steps_keep_cell_order_and_match_cg_step(cuda_lib):
    """12 sorted steps (double-buffered particle arrays): the output arrays
    hold the advanced particles in the step's bin order, exactly the
    records cg_step advances, gathered by the step's permutation; the bins
    of every step equal the oracle's; fields and forces equal cg_step's."""
    import torch
    cg = cuda_lib
    w = synth.small_clustered_bed(seed=12)
    g = cg.Grids(w.desc)
    pos, vel, uf = inputs(w)
    # particle ids ride in vel.w, which the step carries unchanged
    vel[:, 3] = torch.arange(w.n, device="cuda", dtype=torch.int32).view(torch.float32)
    bufs = [(pos, vel), (torch.empty_like(pos), torch.empty_like(vel))]
    out = g.alloc_outputs(w.n, eps_fine=True, bins=True)
    f = cg.Grids(w.desc)
    o2 = f.alloc_outputs(w.n, eps_fine=True, bins=True)
    for step in range(12):
        (pi, vi), (po, vo) = bufs[step % 2], bufs[(step + 1) % 2]
        ref_pos, ref_vel = pi.clone(), vi.clone()
        g.cg_step_sorted(pi, vi, po, vo, uf, out, dt=w.dt)
        f.cg_step(ref_pos, ref_vel, uf, o2, dt=w.dt)     # advances ref_* in place, caller order
        torch.cuda.synchronize()
        perm = out["perm"].long()
        assert torch.equal(po, ref_pos[perm]) and torch.equal(vo, ref_vel[perm]), step
        for k in ("cell", "perm", "cell_start", "eps_bulk", "u_bulk", "force", "S_bulk", "S_fine", "eps_fine"):
            assert torch.equal(out[k], o2[k]), (step, k)
        if step in (0, 1, 11):
            _assert_oracle_bins(w, pi, out, f"sorted step {step}")
        if step >= 1:
            # in cell order from the first step on: the binning nearly keeps
            # runs of consecutive particles together
            pm = out["perm"]
            breaks = (pm[1:] != pm[:-1] + 1).float().mean().item()
            assert breaks < 0.2, (step, breaks)
    ids = bufs[0][1][:, 3].view(torch.int32)
    assert torch.equal(torch.sort(ids.long())[0], torch.arange(w.n, device="cuda"))
    # the entry points on the sorted step's binning: a drag in the caller's
    # order gives the step's forces and reaction again
    pi, vi = bufs[1]     # the last step's input
    F2 = torch.empty_like(out["force"])
    S2 = torch.empty_like(out["S_bulk"])
    g.cg_drag(pi, vi, out["eps_bulk"], out["u_bulk"], F2, S2)
    torch.cuda.synchronize()
    assert torch.equal(F2, out["force"]) and torch.equal(S2, out["S_bulk"])
    assert g.cg_sync_status()[0] == 0
    g.close()
    f.close()


def test_stencil_window_gives_the_gather_bits(cuda_lib):
    """Six sorted steps of the small clustered bed with the drag's stencil
    windows staged in shared memory (CG_STENCIL_WINDOW) against the global
    gather: the same bins, fields, forces and advanced particles, bit for
    bit.  The first step's input is in generation order, so most warps'
    boxes are too large and take the gather path inside the windowed
    kernel; the later inputs are in cell order and use the windows."""
    import torch
    cg = cuda_lib
    w = synth.small_clustered_bed(seed=13)
    runs = []
    for stencil in (cg.CG_STENCIL_GATHER, cg.CG_STENCIL_WINDOW):
        d = dict(w.desc)
        d["stencil"] = stencil
        g = cg.Grids(d)
        pos, vel, uf = inputs(w)
        bufs = [(pos, vel), (torch.empty_like(pos), torch.empty_like(vel))]
        out = g.alloc_outputs(w.n, eps_fine=True, bins=True)
        steps = []
        for step in range(6):
            (pi, vi), (po, vo) = bufs[step % 2], bufs[(step + 1) % 2]
            g.cg_step_sorted(pi, vi, po, vo, uf, out, dt=w.dt)
            torch.cuda.synchronize()
            steps.append({k: v.clone() for k, v in out.items() if v is not None} | {"pos": po.clone(), "vel": vo.clone()})
        assert g.cg_sync_status()[0] == 0
        g.close()
        runs.append(steps)
    for step, (a, b) in enumerate(zip(*runs)):
        for k in a:
            assert torch.equal(a[k], b[k]), (step, k)


@pytest.mark.parametrize("sorted_step", [False, True])
def test_no_movers_with_new_diameters(cuda_lib, sorted_step):
    """Steps whose particles keep their cells (no advance) while their
    diameters change, then two particles of one cell swap places in the
    caller's arrays: the rebinning finds no mover and keeps the bins (its
    scans left out), and the porosity and forces follow the new diameters
    and the swap.  Then 64 particles take the positions of others (movers
    after steps without any: the scans run again) and a last step has no
    mover again.  Bins, fields and forces equal a fresh handle's on the
    same input, bit for bit, at every step."""
    import torch
    cg = cuda_lib
    w = synth.small_clustered_bed(seed=17)
    g = cg.Grids(w.desc)
    pos, vel, uf = inputs(w)
    out = g.alloc_outputs(w.n, eps_fine=True, bins=True)
    bufs = [(pos, vel), (torch.empty_like(pos), torch.empty_like(vel))]
    par = 0
    rng = np.random.default_rng(3)
    for step in range(7):
        pi, vi = bufs[par]
        if step in (2, 3):   # new diameters, same positions
            scale = torch.from_numpy(rng.uniform(0.8, 1.2, w.n).astype(np.float32)).cuda()
            pi[:, 3] *= scale
        if step == 4:   # two particles of one cell swap places in the caller's arrays
            cs = out["cell_start"].cpu().numpy()
            s0 = int(cs[np.nonzero(np.diff(cs) >= 2)[0][0]])   # first slot of a cell holding two or more
            # the input's indices: the last binning's slots (sorted step) or its perm (caller order)
            a, b = (s0, s0 + 1) if sorted_step else (int(out["perm"][s0]), int(out["perm"][s0 + 1]))
            for arr in (pi, vi):
                t = arr[a].clone()
                arr[a] = arr[b]
                arr[b] = t
        if step == 5:   # 64 particles move onto the positions of others (diameters kept)
            dst = torch.from_numpy(rng.choice(w.n, 64, replace=False)).cuda()
            src = torch.from_numpy(rng.choice(w.n, 64, replace=False)).cuda()
            pi[dst, :3] = pi[src, :3]
        ref_in = (pi.clone(), vi.clone())
        if sorted_step:
            po, vo = bufs[par ^ 1]
            g.cg_step_sorted(pi, vi, po, vo, uf, out, dt=0.0)
            par ^= 1
        else:
            g.cg_step(pi, vi, uf, out, dt=0.0)
        f = cg.Grids(w.desc)
        o2 = f.alloc_outputs(w.n, eps_fine=True, bins=True)
        f.cg_step(ref_in[0], ref_in[1], uf, o2, dt=0.0)
        torch.cuda.synchronize()
        for k in ("cell", "perm", "cell_start", "eps_bulk", "u_bulk", "force", "S_bulk", "S_fine", "eps_fine"):
            assert torch.equal(out[k], o2[k]), (step, k)
        f.close()
    assert g.cg_sync_status()[0] == 0
    g.close()


def test_fallback_when_most_particles_changed(cuda_lib):
    """The same handle bins three unrelated particle sets of one count (every
    particle a mover: the device falls back to the per-cell sort) and then
    the first set again: every binning equals a from-scratch sort."""
    import torch
    cg = cuda_lib
    ws = [synth.small_clustered_bed(seed=s) for s in (21, 22, 23)]
    ws.append(ws[0])
    g = cg.Grids(ws[0].desc)
    n = ws[0].n
    for k, w in enumerate(ws):
        pos = to_dev(w.pos_d)
        got = {"cell": torch.empty(n, dtype=torch.int32, device="cuda"),
               "perm": torch.empty(n, dtype=torch.int32, device="cuda"),
               "cell_start": torch.empty(g.n_bulk + 1, dtype=torch.int32, device="cuda")}
        g.cg_bin_particles(pos, got["cell"], got["perm"], got["cell_start"])
        torch.cuda.synchronize()
        _assert_bins_equal(got, _scratch_bins(cg, w.desc, pos), f"set {k}")
    g.close()


@pytest.mark.parametrize("fp64", [False, True])
def test_movers_into_crowded_cells_and_the_arrival_limit(cuda_lib, fp64):
    """Particles of one cell, a crowded one (3,000 particles) and the rest
    spread out; between binnings 1% move at random, then 200 move into the
    crowded cell (under the per-cell arrival limit), then 600 (over it: the
    fallback), then a few move out of it.  Each binning equals the oracle's."""
    import torch
    cg = cuda_lib
    w = synth.tiny(seed=31, n=20_000, fine=32, ratio=4, fp64=fp64)
    rng = np.random.default_rng(5)
    pos = w.pos_d.copy()
    pos[:3000, :3] = 0.3 + 0.05 * rng.random((3000, 3))      # one bulk cell of 1/8
    g = cg.Grids(w.desc)
    cell = torch.empty(w.n, dtype=torch.int32, device="cuda")
    perm = torch.empty_like(cell)
    cs = torch.empty(g.n_bulk + 1, dtype=torch.int32, device="cuda")
    stages = []
    p = pos.copy()
    stages.append(p.copy())
    m = rng.random(w.n) < 0.01
    p[m, :3] = rng.random((m.sum(), 3))
    stages.append(p.copy())
    for count in (200, 600):
        idx = rng.choice(np.arange(3000, w.n), size=count, replace=False)
        p[idx, :3] = 0.3 + 0.05 * rng.random((count, 3))
        stages.append(p.copy())
    p[:50, :3] = rng.random((50, 3))
    stages.append(p.copy())
    for k, st in enumerate(stages):
        d = to_dev(st)
        g.cg_bin_particles(d, cell, perm, cs)
        torch.cuda.synchronize()
        _assert_oracle_bins(w, d, {"cell": cell, "perm": perm, "cell_start": cs}, f"stage {k}")
    g.close()


def test_full_clustered_bed_sorted_steps_bit_exact(cuda_lib):
    """The 32M-particle clustered bed, 12 sorted steps with the Euler
    advance: every step's bins equal a from-scratch sort of the same
    positions (and the oracle's at the first, second and last step); the
    last step's fields match the oracle within the FP32 tolerance."""
    import torch
    cg = cuda_lib
    w = synth.clustered_bed(seed=0)
    g = cg.Grids(w.desc)
    pos, vel, uf = inputs(w)
    bufs = [(pos, vel), (torch.empty_like(pos), torch.empty_like(vel))]
    out = g.alloc_outputs(w.n, eps_fine=True, bins=True)
    for step in range(12):
        (pi, vi), (po, vo) = bufs[step % 2], bufs[(step + 1) % 2]
        state = (pi.clone(), vi.clone()) if step == 11 else None
        g.cg_step_sorted(pi, vi, po, vo, uf, out, dt=w.dt)
        torch.cuda.synchronize()
        _assert_bins_equal(out, _scratch_bins(cg, w.desc, pi), f"step {step}")
        if step in (0, 1, 11):
            _assert_oracle_bins(w, pi, out, f"step {step}")
    p11, v11 = to_np(state[0]), to_np(state[1])
    ref = oracle.step(w.desc, p11, v11, w.u_fine, dt=w.dt)
    # after 11 steps the particles move with the fluid: the force is judged
    # against the terms of its slip (FP32 rounding of u_f cancels in u_f - u_p)
    _, slip = oracle.particle_state(w.desc, p11, v11, ref["eps_bulk"], ref["u_bulk"])
    report = {}
    assert_close_slip("force", to_np(out["force"]), ref["force"], slip, v11[:, :3], TOL_FP32, report)
    assert_close("S_bulk", to_np(out["S_bulk"]), ref["S_bulk"], TOL_FP32, vec=True)
    print("clustered bed after 11 sorted steps:", report)
    perm = to_np(out["perm"])
    got_pos = to_np(bufs[0][0]).astype(np.float64)
    assert np.max(np.abs(got_pos[:, :3] - ref["pos_d"][perm, :3])) <= 2e-6
    rc, flags, counts = g.cg_sync_status()
    assert rc == 0
    g.close()


def test_sorted_step_argument_checks(cuda_lib):
    import torch
    cg = cuda_lib
    w = synth.tiny(seed=1, n=1000, fp64=False)
    g = cg.Grids(w.desc)
    pos, vel, uf = inputs(w)
    out = g.alloc_outputs(w.n)
    with pytest.raises(cg.CgError) as e:
        g.cg_step_sorted(pos, vel, pos, torch.empty_like(vel), uf, out)     # output over the input
    assert e.value.code == 1
    big = torch.empty(2 * w.n, 4, device="cuda")
    with pytest.raises(cg.CgError) as e:
        g.cg_step_sorted(pos, vel, big[:w.n], big[w.n // 2:w.n // 2 + w.n], uf, out)   # outputs overlap
    assert e.value.code == 1
    g.close()
