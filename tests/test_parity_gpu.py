"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bins and permutations must match bit for bit; FP64 fields within 1e-12 and
FP32 fields within 2e-6 relative (per cell / per particle, denominator
max(|ref|, 1e-3 max|ref|), vectors by Euclidean norm).  Sizes span several
4096-particle sort tiles with ragged tails, one- and two-pass sorts, and
the benchmark's full packed-bed workload."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import (TOL_FP32, TOL_FP64, assert_close, assert_close_interp, inputs, to_dev, to_np,
                         switch_exclusions, switch_mask)

pytestmark = pytest.mark.gpu


def run_step(cg, w, dt=0.0, eps_fine=True):
    import torch
    g = cg.Grids(w.desc)
    pos, vel, uf = inputs(w)
    out = g.alloc_outputs(w.n, eps_fine=eps_fine, bins=True)
    g.cg_step(pos, vel, uf, out, dt=dt)
    rc, flags, counts = g.cg_sync_status()
    torch.cuda.synchronize()
    host = {k: to_np(v) for k, v in out.items()}
    host["pos_d"], host["vel"] = to_np(pos), to_np(vel)
    host["rc"], host["flags"], host["counts"] = rc, flags, counts
    g.close()
    return host


def compare_step(w, got, ref, tol, mask=None, report=None):
    """Bins bit for bit, then every field within tol.  mask ([n] bool,
    nullable) drops the particles within rounding of a correlation switch
    (FP32 and FP64 may take different branches there): their forces, the
    reaction of the bulk cells holding them and the fine cells whose
    stencil reads those bulk cells; everything else is compared.  report
    (nullable dict) receives the number of excluded particles and cells and
    the widened-denominator statistics of the interpolated fields."""
    assert np.array_equal(got["cell"], ref["cell"]), "cells differ"
    assert np.array_equal(got["cell_start"], ref["cell_start"]), "cell starts differ"
    assert np.array_equal(got["perm"], ref["perm"]), "permutation differs"
    errs = {}
    errs["eps_bulk"] = assert_close("eps_bulk", got["eps_bulk"], ref["eps_bulk"], tol)
    errs["u_bulk"] = assert_close("u_bulk", got["u_bulk"], ref["u_bulk"], tol, vec=True)
    errs["var_bulk"] = assert_close("var_bulk", got["var_bulk"], ref["var_bulk"], tol)
    errs["force"] = assert_close("force", got["force"], ref["force"], tol, vec=True, mask=mask)
    bulk_ok = fine_ok = None
    if mask is not None and not mask.all():
        bulk_ok, fine_ok = switch_exclusions(w, ref, mask)
    if report is not None:
        report["excluded"] = {"particles": 0 if mask is None else int((~mask).sum()),
                              "bulk_cells": 0 if bulk_ok is None else int((~bulk_ok).sum()),
                              "fine_cells": 0 if fine_ok is None else int((~fine_ok).sum())}
    # the projections interpolate bulk values of either sign (sources; the
    # porosity, negative where spheres overlap): their rounding is relative
    # to the interpolant of the absolute bulk values, projected by the oracle
    errs["S_bulk"] = assert_close("S_bulk", got["S_bulk"], ref["S_bulk"], tol, vec=True, mask=bulk_ok)
    S_abs = oracle.project(w.desc, np.abs(ref["S_bulk"]))
    errs["S_fine"] = assert_close_interp("S_fine", got["S_fine"], ref["S_fine"], S_abs, tol, mask=fine_ok,
                                         report=report)
    if got.get("eps_fine") is not None and ref.get("eps_fine") is not None:
        e_abs = oracle.project(w.desc, np.abs(ref["eps_bulk"]))
        errs["eps_fine"] = assert_close_interp("eps_fine", got["eps_fine"], ref["eps_fine"], e_abs, tol,
                                               report=report)
    return errs


def _without_particles(sums, force, keep, mass_u=None):
    """The step's sums with the drag of the particles outside keep taken
    out: sum F loses their forces, sum S_B V_B and sum S_f V_f (each equal to
    -sum F by action-reaction and conservative projection) lose their
    reactions, sum |F| loses their magnitudes, and the momentum after the
    advance loses their m u (mass_u, [3][n], when given)."""
    s = np.array(sums, np.float64)
    if keep is None or keep.all():
        return s
    F = np.asarray(force, np.float64)[:, ~keep]
    fx = F.sum(axis=1)
    s[2:5] -= fx
    s[5:8] += fx
    s[8:11] += fx
    s[11] -= np.sqrt((F ** 2).sum(axis=0)).sum()
    if mass_u is not None:
        s[12:15] -= np.asarray(mass_u, np.float64)[:, ~keep].sum(axis=1)
    return s


def compare_sums(got, ref, tol, mask=None, w=None):
    """The device's FP64 conservation sums against the oracle's (with the
    particles outside mask taken out of both, see _without_particles)."""
    mu_got = mu_ref = None
    if mask is not None and not mask.all() and w is not None and "vel" in got:
        d = w.pos_d[:, 3].astype(np.float64)
        m = w.desc["rho_p"] * np.pi * d ** 3 / 6.0
        mu_got = m * np.asarray(got["vel"], np.float64)[:, :3].T
        mu_ref = m * np.asarray(ref["vel"], np.float64)[:, :3].T
    s = _without_particles(got["sums"], got["force"], mask, mu_got)
    r = _without_particles(ref["sums"], ref["force"], mask, mu_ref)
    vol = abs(r[0])
    fs = r[11]
    assert abs(s[0] - r[0]) <= tol * vol and abs(s[1] - r[1]) <= tol * vol
    for k in list(range(2, 11)) + [11]:
        assert abs(s[k] - r[k]) <= tol * fs + 1e-300, (k, s[k], r[k])
    # conservation on the device sums themselves
    assert np.all(np.abs(s[2:5] + s[5:8]) <= 10 * tol * fs)
    assert np.all(np.abs(s[5:8] - s[8:11]) <= 10 * tol * fs)
    assert s[15] == r[15]


# ------------------------------------------------------------------ FP64
def test_tiny_fp64_step(cuda_lib):
    w = synth.tiny(seed=0)
    ref = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, want_eps_fine=True)
    got = run_step(cuda_lib, w)
    assert got["rc"] == 0 and got["counts"] == [0, 0, 0, 0, 0]
    compare_step(w, got, ref, TOL_FP64)
    compare_sums(got, ref, 1e-12)


def test_tiny_fp64_individual_entry_points(cuda_lib):
    import torch
    w = synth.tiny(seed=3, n=25_000)
    d = w.desc
    g = cuda_lib.Grids(d)
    pos, vel, uf = inputs(w)
    n = w.n
    cell = torch.empty(n, dtype=torch.int32, device="cuda")
    perm = torch.empty_like(cell)
    cs = torch.empty(g.n_bulk + 1, dtype=torch.int32, device="cuda")
    g.cg_bin_particles(pos, cell, perm, cs)
    rc_cell, rc_perm, rc_cs, _ = oracle.bin(d, w.pos_d)
    assert np.array_equal(to_np(cell), rc_cell)
    assert np.array_equal(to_np(perm), rc_perm)
    assert np.array_equal(to_np(cs), rc_cs)
    eps = torch.empty(g.n_bulk, dtype=torch.float64, device="cuda")
    g.cg_deposit(cuda_lib.CG_DEP_VOLUME, n, pos, eps)
    r_eps, _ = oracle.deposit_volume(d, w.pos_d, rc_cs, rc_perm)
    assert_close("eps", to_np(eps), r_eps, TOL_FP64)
    ub = torch.empty(3, g.n_bulk, dtype=torch.float64, device="cuda")
    var = torch.empty(g.n_bulk, dtype=torch.float64, device="cuda")
    g.cg_average_fine_to_bulk(uf, ub, var)
    r_ub, r_var = oracle.average(d, w.u_fine)
    assert_close("u_bulk", to_np(ub), r_ub, TOL_FP64, vec=True)
    assert_close("var", to_np(var), r_var, TOL_FP64)
    # drag from the oracle's own bulk fields (isolates the drag step)
    F = torch.empty(3, n, dtype=torch.float64, device="cuda")
    S = torch.empty(3, g.n_bulk, dtype=torch.float64, device="cuda")
    g.cg_drag(pos, vel, to_dev(r_eps), to_dev(r_ub), F, S)
    r_F, _ = oracle.drag(d, w.pos_d, w.vel, r_eps, r_ub)
    assert_close("force", to_np(F), r_F, TOL_FP64, vec=True)
    r_S = oracle.deposit_momentum(d, r_F, rc_cs, rc_perm)
    assert_close("S_bulk(fused)", to_np(S), r_S, TOL_FP64, vec=True)
    # momentum deposit from caller-order forces
    S2 = torch.empty_like(S)
    g.cg_deposit(cuda_lib.CG_DEP_MOMENTUM, n, to_dev(r_F), S2)
    assert_close("S_bulk(deposit)", to_np(S2), r_S, TOL_FP64, vec=True)
    # projection of the oracle's bulk source
    Sf = torch.empty(3, g.n_fine, dtype=torch.float64, device="cuda")
    g.cg_project_bulk_to_fine(to_dev(r_S), Sf)
    assert_close("S_fine", to_np(Sf), oracle.project(d, r_S), TOL_FP64, vec=True)
    rc, flags, counts = g.cg_sync_status()
    assert rc == 0
    g.close()


@pytest.mark.parametrize("r", [2, 3, 8])
def test_ratios_fp64(cuda_lib, r):
    nb = 6 if r != 8 else 4
    w = synth.tiny(seed=r, n=7_777, fine=nb * r, ratio=r)
    ref = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, want_eps_fine=True)
    got = run_step(cuda_lib, w)
    compare_step(w, got, ref, TOL_FP64)
    compare_sums(got, ref, 1e-12)


def test_cell_value_interp_fp64(cuda_lib):
    w = synth.tiny(seed=5, n=9_000)
    w.desc["interp"] = synth.INTERP_CELL
    ref = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, want_eps_fine=True)
    got = run_step(cuda_lib, w)
    compare_step(w, got, ref, TOL_FP64)


# ------------------------------------------------------------------ FP32
def test_tiny_fp32_step(cuda_lib):
    w = synth.tiny(seed=1, n=50_000, fp64=False)
    ref = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, want_eps_fine=True)
    got = run_step(cuda_lib, w)
    compare_step(w, got, ref, TOL_FP32)
    compare_sums(got, ref, TOL_FP32)


def test_small_packed_bed_fp32(cuda_lib):
    """The packed-bed recipe at 1/64 of its cells (Ergun / Wen-Yu): every
    field and the sums, with only the particles at the correlation switch
    and the cells that depend on them left out."""
    w = synth.small_packed_bed(seed=0)
    ref = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, want_eps_fine=True)
    got = run_step(cuda_lib, w)
    mask = switch_mask(w, ref)
    report = {}
    errs = compare_step(w, got, ref, TOL_FP32, mask=mask, report=report)
    compare_sums(got, ref, TOL_FP32, mask=mask, w=w)
    assert {"S_bulk", "S_fine", "eps_fine"} <= set(errs)
    print("small_packed_bed max rel errors:", {k: f"{v:.2e}" for k, v in errs.items()}, report)


def test_small_clustered_bed_fp32_with_euler(cuda_lib):
    """One step with the Euler advance; parity of the advanced state is
    checked from the shared initial state (trajectories are not compared
    over many steps)."""
    w = synth.small_clustered_bed(seed=0)
    ref = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, dt=w.dt, want_eps_fine=True)
    got = run_step(cuda_lib, w, dt=w.dt)
    compare_step(w, got, ref, TOL_FP32)
    compare_sums(got, ref, 5 * TOL_FP32)
    _euler_checks(w, got, ref)


def test_packed_bed_full_size_fp32(cuda_lib):
    """The benchmark's workload (4M particles, fine 256x256x512) at full size,
    in the launch configuration the benchmark times."""
    w = synth.packed_bed(seed=0)
    ref = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, want_eps_fine=True)
    got = run_step(cuda_lib, w)
    mask = switch_mask(w, ref)
    report = {}
    errs = compare_step(w, got, ref, TOL_FP32, mask=mask, report=report)
    compare_sums(got, ref, TOL_FP32, mask=mask, w=w)
    assert {"S_bulk", "S_fine", "eps_fine"} <= set(errs)
    # the exclusion stays local: a few particles, their cells and stencils
    ex = report["excluded"]
    assert ex["particles"] < 1e-4 * w.n and ex["fine_cells"] <= 64 * ex["bulk_cells"] * 8
    print("packed_bed max rel errors:", {k: f"{v:.2e}" for k, v in errs.items()}, report)


def _euler_checks(w, got, ref):
    # u_new = u + dt (F/m + g): drag and gravity cancel for some particles, so
    # the bound is relative to the magnitude of the terms, not of the result
    d = w.pos_d[:, 3].astype(np.float64)
    m = w.desc["rho_p"] * np.pi * d ** 3 / 6.0
    scale_u = np.abs(w.vel[:, :3]).sum(axis=1) + w.dt * (np.linalg.norm(ref["force"], axis=0) / m + 9.81)
    du = np.linalg.norm(got["vel"][:, :3].astype(np.float64) - ref["vel"][:, :3], axis=1)
    assert np.max(du / scale_u) <= TOL_FP32, np.max(du / scale_u)
    scale_x = np.abs(w.pos_d[:, :3].astype(np.float64)).max(axis=1) + w.dt * np.linalg.norm(ref["vel"][:, :3], axis=1)
    dx = np.abs(got["pos_d"][:, :3].astype(np.float64) - ref["pos_d"][:, :3]).max(axis=1)
    assert np.max(dx / scale_x) <= TOL_FP32, np.max(dx / scale_x)
    assert np.array_equal(got["pos_d"][:, 3], w.pos_d[:, 3])


def test_clustered_bed_full_size_fp32_with_euler(cuda_lib):
    """The 32M-particle clustered bed (fine 512x512x256, ratio 4, Di Felice,
    gravity, dt 1e-4) at full size: one step with the Euler advance from
    the shared initial state, every field and particle against the oracle."""
    w = synth.clustered_bed(seed=0)
    ref = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, dt=w.dt, want_eps_fine=True)
    got = run_step(cuda_lib, w, dt=w.dt)
    errs = compare_step(w, got, ref, TOL_FP32)
    compare_sums(got, ref, 5 * TOL_FP32)
    _euler_checks(w, got, ref)
    print("clustered_bed max rel errors:", {k: f"{v:.2e}" for k, v in errs.items()},
          "clamped porosities:", got["counts"][2])


def test_clustered_bed_100_steps_conservation_drift(cuda_lib):
    """100 coupled steps of the clustered bed (fluid frozen, particles
    advanced).  After every step the device's FP64 conservation sums must
    close: sum F_p + sum S_B V_B = 0, sum S_B V_B = sum S_f V_f and
    sum V_p = sum (1 - eps_B) V_B, each to FP32 round-off of the summed
    terms; the per-step residuals are printed (the drift report)."""
    import torch
    w = synth.clustered_bed(seed=0)
    g = cuda_lib.Grids(w.desc)
    pos, vel, uf = inputs(w)
    out = g.alloc_outputs(w.n, eps_fine=True)
    res = []
    for _ in range(w.steps):
        g.cg_step(pos, vel, uf, out, dt=w.dt)
        s = out["sums"].cpu().numpy()
        res.append((np.abs(s[2:5] + s[5:8]).max() / s[11], np.abs(s[5:8] - s[8:11]).max() / s[11],
                    abs(s[0] - s[1]) / s[0]))
    rc, flags, counts = g.cg_sync_status()
    g.close()
    res = np.array(res)
    print("per-step residuals (action-reaction, projection, volume): max", res.max(axis=0),
          "last", res[-1], "first", res[0])
    assert rc == 0 and counts[0] == 0 and counts[1] == 0
    assert np.all(res[:, 0] <= 10 * TOL_FP32) and np.all(res[:, 1] <= 10 * TOL_FP32)
    assert np.all(res[:, 2] <= TOL_FP32)
    assert torch.isfinite(pos).all()


@pytest.mark.parametrize("digits", [1, 6, 7, 9, 11])
def test_sort_digit_width_does_not_change_bins(cuda_lib, digits):
    """The per-cell sort (1) and one, two or three passes of any digit width
    give the same stable order (and so the same fields) as the oracle."""
    import torch
    w = synth.small_clustered_bed(seed=6)
    ref_cell, ref_perm, ref_cs, _ = oracle.bin(w.desc, w.pos_d)
    d = dict(w.desc)
    d["sort_digits"] = digits
    g = cuda_lib.Grids(d)
    pos = to_dev(w.pos_d)
    cell = torch.empty(w.n, dtype=torch.int32, device="cuda")
    perm = torch.empty(w.n, dtype=torch.int32, device="cuda")
    cs = torch.empty(g.n_bulk + 1, dtype=torch.int32, device="cuda")
    g.cg_bin_particles(pos, cell, perm, cs)
    assert np.array_equal(to_np(cell), ref_cell)
    assert np.array_equal(to_np(perm), ref_perm)
    assert np.array_equal(to_np(cs), ref_cs)
    g.close()


@pytest.mark.parametrize("fp64", [False, True])
def test_cells_of_every_sort_size_class(cuda_lib, fp64):
    """Cells holding 1 to 9,000 particles in shuffled order: every size class
    of the default per-cell sort (one element, the warp sorts of 32, 64, 128
    and 256, the CTA sort of larger cells with one to three 4096-id chunks)
    and both sides of each boundary give the oracle's stable order, as does
    the digit sort."""
    import torch
    w = synth.tiny(seed=4, n=1, fine=64, ratio=4, fp64=fp64)
    rng = np.random.default_rng(11)
    sizes = [1, 2, 3, 31, 32, 33, 63, 64, 65, 127, 128, 129, 255, 256, 257, 1000, 4095, 4096, 4097, 9000]
    cells = rng.choice(16 ** 3, size=len(sizes), replace=False)
    H = 1.0 / 16
    parts = []
    for c, m in zip(cells, sizes):
        ijk = np.array([c % 16, (c // 16) % 16, c // 256], dtype=np.float64)
        parts.append((ijk + 0.05 + 0.9 * rng.random((m, 3))) * H)
    parts.append(rng.random((5000, 3)))
    xyz = np.concatenate(parts)[rng.permutation(sum(sizes) + 5000)]
    pos = np.empty((len(xyz), 4), dtype=w.pos_d.dtype)
    pos[:, :3] = xyz
    pos[:, 3] = 0.002
    ref_cell, ref_perm, ref_cs, _ = oracle.bin(w.desc, pos)
    counts = np.diff(ref_cs)
    assert all(counts[c] >= m for c, m in zip(cells, sizes))
    for digits in (cuda_lib.CG_SORT_CELLS, 8):
        d = dict(w.desc)
        d["sort_digits"] = digits
        g = cuda_lib.Grids(d)
        p = to_dev(pos)
        cell = torch.empty(len(pos), dtype=torch.int32, device="cuda")
        perm = torch.empty(len(pos), dtype=torch.int32, device="cuda")
        cs = torch.empty(g.n_bulk + 1, dtype=torch.int32, device="cuda")
        g.cg_bin_particles(p, cell, perm, cs)
        assert np.array_equal(to_np(cell), ref_cell), digits
        assert np.array_equal(to_np(cs), ref_cs), digits
        assert np.array_equal(to_np(perm), ref_perm), digits
        g.close()


def test_both_sorts_agree_at_full_clustered_size(cuda_lib):
    """32M particles in random order: the per-cell sort (beyond the size it
    is picked for automatically) gives the digit sort's bins, and the
    automatic choice the same again."""
    import torch
    w = synth.clustered_bed(seed=1)
    pos = to_dev(w.pos_d)
    got = []
    for digits in (cuda_lib.CG_SORT_CELLS, 8, cuda_lib.CG_SORT_AUTO):
        d = dict(w.desc)
        d["sort_digits"] = digits
        g = cuda_lib.Grids(d)
        cell = torch.empty(w.n, dtype=torch.int32, device="cuda")
        perm = torch.empty(w.n, dtype=torch.int32, device="cuda")
        cs = torch.empty(g.n_bulk + 1, dtype=torch.int32, device="cuda")
        g.cg_bin_particles(pos, cell, perm, cs)
        torch.cuda.synchronize()
        got.append((cell, perm, cs))
        g.close()
    for other in got[1:]:
        for a, b in zip(got[0], other):
            assert torch.equal(a, b)
    # the order is a permutation sorted by cell, ids ascending within a cell
    cell, perm, cs = got[0]
    ks = cell[perm.long()]
    assert bool((ks[1:] >= ks[:-1]).all())
    same = ks[1:] == ks[:-1]
    assert bool((perm[1:][same] > perm[:-1][same]).all())
    assert int(cs[-1]) == w.n


def test_repeat_is_bit_identical(cuda_lib):
    w = synth.small_clustered_bed(seed=1)
    a = run_step(cuda_lib, w)
    b = run_step(cuda_lib, w)
    for k in ["cell", "perm", "cell_start", "eps_bulk", "u_bulk", "var_bulk", "force", "S_bulk", "S_fine",
              "sums"]:
        assert np.array_equal(a[k], b[k], equal_nan=True), k


def test_host_entry_matches_device_entry(cuda_lib):
    import torch
    w = synth.small_packed_bed(seed=2)
    dev = run_step(cuda_lib, w, eps_fine=False)
    g = cuda_lib.Grids(w.desc)
    out = {k: (v.cpu().pin_memory() if v is not None else None)
           for k, v in g.alloc_outputs(w.n, bins=True).items()}
    pos = torch.from_numpy(w.pos_d.copy()).pin_memory()
    vel = torch.from_numpy(w.vel.copy()).pin_memory()
    uf = torch.from_numpy(np.ascontiguousarray(w.u_fine.reshape(3, -1))).pin_memory()
    g.cg_step_host(pos, vel, uf, out)
    for k in ["cell", "perm", "cell_start", "eps_bulk", "u_bulk", "force", "S_bulk", "S_fine", "sums"]:
        assert np.array_equal(out[k].numpy(), dev[k]), k
    g.close()


def test_pipelined_host_steps_match_device_steps(cuda_lib):
    """Three enqueued host steps on different inputs (so the two staging sets
    alternate and one is reused), then one wait: each step's outputs equal
    cg_step on the device of the same inputs."""
    import torch
    ws = [synth.small_clustered_bed(seed=s) for s in (3, 4, 5)]
    refs = [run_step(cuda_lib, w, eps_fine=True) for w in ws]
    g = cuda_lib.Grids(ws[0].desc)
    hosts = []
    for w in ws:
        out = {k: (v.cpu().pin_memory() if v is not None else None)
               for k, v in g.alloc_outputs(w.n, eps_fine=True, bins=True).items()}
        pos = torch.from_numpy(w.pos_d.copy()).pin_memory()
        vel = torch.from_numpy(w.vel.copy()).pin_memory()
        uf = torch.from_numpy(np.ascontiguousarray(w.u_fine.reshape(3, -1))).pin_memory()
        hosts.append((pos, vel, uf, out))
    for pos, vel, uf, out in hosts:
        g.cg_step_host_async(pos, vel, uf, out)
    g.cg_step_host_wait()
    for (pos, vel, uf, out), ref in zip(hosts, refs):
        for k in ["cell", "perm", "cell_start", "eps_bulk", "u_bulk", "var_bulk", "force", "S_bulk", "S_fine",
                  "eps_fine", "sums"]:
            assert np.array_equal(out[k].numpy(), ref[k], equal_nan=True), k
    assert g.cg_sync_status()[0] == 0
    g.close()


def test_advancing_host_steps_enqueued_back_to_back(cuda_lib):
    """Four advancing steps (dt > 0) enqueued on one pair of host particle
    arrays without waiting in between: each step reads the particles the
    step before advanced, so the final particles and the last step's outputs
    equal four blocking host steps, bit for bit."""
    import torch
    w = synth.small_clustered_bed(seed=6)
    dt = 1e-4
    g = cuda_lib.Grids(w.desc)
    runs = []
    for pipelined in (False, True):
        out = {k: (v.cpu().pin_memory() if v is not None else None)
               for k, v in g.alloc_outputs(w.n, eps_fine=True, bins=True).items()}
        pos = torch.from_numpy(w.pos_d.copy()).pin_memory()
        vel = torch.from_numpy(w.vel.copy()).pin_memory()
        uf = torch.from_numpy(np.ascontiguousarray(w.u_fine.reshape(3, -1))).pin_memory()
        for _ in range(4):
            if pipelined:
                g.cg_step_host_async(pos, vel, uf, out, dt=dt)
            else:
                g.cg_step_host(pos, vel, uf, out, dt=dt)
        g.cg_step_host_wait()
        runs.append((pos.numpy().copy(), vel.numpy().copy(), {k: v.numpy().copy() for k, v in out.items()
                                                              if v is not None}))
    (p0, v0, o0), (p1, v1, o1) = runs
    assert not np.array_equal(p0, w.pos_d)   # the particles did move
    assert np.array_equal(p0, p1) and np.array_equal(v0, v1)
    for k in o0:
        assert np.array_equal(o0[k], o1[k], equal_nan=True), k
    assert g.cg_sync_status()[0] == 0
    g.close()


# ------------------------------------------------------------- edge cases
def test_edge_empty_particle_set(cuda_lib):
    w = synth.tiny(seed=0, n=0)
    ref = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, want_eps_fine=True)
    got = run_step(cuda_lib, w)
    assert np.all(got["cell_start"] == 0)
    assert np.all(got["eps_bulk"] == 1.0)
    assert np.all(got["S_bulk"] == 0.0) and np.all(got["S_fine"] == 0.0)
    assert_close("u_bulk", got["u_bulk"], ref["u_bulk"], TOL_FP64, vec=True)
    assert got["sums"][0] == 0.0 and got["sums"][2] == 0.0


@pytest.mark.parametrize("sort", [0, 1])
def test_edge_faces_outside_and_one_crowded_cell(cuda_lib, sort):
    """Particles exactly on bulk faces and on the upper domain faces, some
    outside (clamped and counted), and 30,000 in a single cell (one long
    segment across many sort tiles), with the automatic sort (the digit sort
    at this density) and with the per-cell sort (the cell goes to its
    large-cell digit passes)."""
    w = synth.tiny(seed=9, n=40_000, fine=32, ratio=4, fp64=False)
    w.desc["sort_digits"] = sort
    rng = np.random.default_rng(0)
    pos = w.pos_d
    H = 1.0 / 8
    k = 5000
    pos[:k, :3] = rng.integers(0, 9, (k, 3)) * H             # exactly on faces, incl. x = 1
    pos[k:k + 100, 0] = -0.01                                 # outside below
    pos[k + 100:k + 200, 2] = 1.02                            # outside above
    pos[10_000:40_000, :3] = 0.3 + 0.01 * rng.random((30_000, 3))
    ref = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, want_eps_fine=True)
    got = run_step(cuda_lib, w)
    assert got["counts"][0] == ref["outside"] == 200
    assert got["flags"] & 1
    # the crowded cell is over-packed: porosity ~ -7 there, clamped for the
    # drag.  The projected porosity then crosses zero next to it, where the
    # float rounding of |eps| ~ 7 exceeds a relative bound; it is checked
    # against the field's magnitude instead.
    eps_f_got, eps_f_ref = got.pop("eps_fine"), ref.pop("eps_fine")
    compare_step(w, got, ref, TOL_FP32)
    assert np.max(np.abs(eps_f_got - eps_f_ref)) <= TOL_FP32 * np.max(np.abs(eps_f_ref))
    assert got["counts"][2] == int(ref["sums"][15])


def test_edge_nonfinite_positions_are_reported(cuda_lib):
    import torch
    w = synth.tiny(seed=2, n=5_000, fp64=False)
    w.pos_d[17, 0] = np.nan
    w.pos_d[99, 2] = np.inf
    g = cuda_lib.Grids(w.desc)
    pos, vel, uf = inputs(w)
    cell = torch.empty(w.n, dtype=torch.int32, device="cuda")
    g.cg_bin_particles(pos, cell)
    rc, flags, counts = g.cg_sync_status()
    assert rc == 7 and flags & 2 and counts[1] == 2
    ref_cell, _, _, _ = oracle.bin(w.desc, w.pos_d)
    assert np.array_equal(to_np(cell), ref_cell)
    rc, flags, counts = g.cg_sync_status()    # read-and-clear
    assert rc == 0 and flags == 0
    g.close()


def test_edge_minimal_grid_and_two_particles(cuda_lib):
    desc = synth.make_desc((0.25, -1.0, 3.0), (0.5, 2.0, 1.0), (2, 4, 6), 1, fp64=True, law=1)
    pos = np.array([[0.3, -0.5, 3.2, 0.01], [0.74, 0.99, 3.99, 0.02]])
    vel = np.array([[0.1, 0.0, -0.1, 0.0], [0.0, 0.2, 0.0, 0.0]])
    u = np.random.default_rng(1).normal(size=(3, 6, 4, 2))
    w = synth.Workload("minimal", desc, pos, vel, u)
    ref = oracle.step(desc, pos, vel, u, want_eps_fine=True)
    got = run_step(cuda_lib, w)
    compare_step(w, got, ref, TOL_FP64)


def test_not_binned_and_bad_args(cuda_lib):
    import torch
    w = synth.tiny(seed=0, n=100)
    g = cuda_lib.Grids(w.desc)
    pos, vel, uf = inputs(w)
    eps = torch.empty(g.n_bulk, dtype=torch.float64, device="cuda")
    with pytest.raises(cuda_lib.CgError) as e:
        g.cg_deposit(cuda_lib.CG_DEP_VOLUME, w.n, pos, eps)
    assert e.value.code == 4
    L = cuda_lib.lib()
    # misaligned particle array
    assert L.cg_bin_particles(g.h, 10, pos.data_ptr() + 4, None, None, None) == 1
    g.close()
    # sort choices other than automatic, per-cell and digit widths 6..11
    for bad in (-1, 2, 5, 12):
        d = dict(w.desc)
        d["sort_digits"] = bad
        with pytest.raises(cuda_lib.CgError):
            cuda_lib.Grids(d)


@pytest.mark.parametrize("fp64", [False, True])
def test_reorder_particles_into_cell_order(cuda_lib, fp64):
    """cg_reorder_particles gathers the records into the binned order;
    rebinning them gives the identity permutation, and a step on the
    reordered particles gives bit-identical bulk and fine fields (each cell
    sums the same particles in the same order) and the same forces,
    permuted."""
    import torch
    cg = cuda_lib
    w = synth.tiny(seed=8, n=20_000) if fp64 else synth.small_clustered_bed(seed=8)
    d = dict(w.desc)
    d["sort_digits"] = cg.CG_SORT_CELLS
    g = cg.Grids(d)
    pos, vel, uf = inputs(w)
    out = g.alloc_outputs(w.n, eps_fine=True, bins=True)
    g.cg_step(pos, vel, uf, out)
    pos2, vel2 = torch.empty_like(pos), torch.empty_like(vel)
    g.cg_reorder_particles(pos, vel, pos2, vel2)
    perm = out["perm"].long()
    torch.cuda.synchronize()
    assert torch.equal(pos2, pos[perm]) and torch.equal(vel2, vel[perm])
    out2 = g.alloc_outputs(w.n, eps_fine=True, bins=True)
    g.cg_step(pos2, vel2, uf, out2)
    torch.cuda.synchronize()
    assert torch.equal(out2["perm"], torch.arange(w.n, device="cuda", dtype=torch.int32))
    assert torch.equal(out2["cell_start"], out["cell_start"])
    for k in ("eps_bulk", "u_bulk", "var_bulk", "S_bulk", "S_fine", "eps_fine"):
        assert torch.equal(out2[k], out[k]), k
    assert torch.equal(out2["force"], out["force"][:, perm])
    # a different particle count has no binning; overlapping outputs are refused
    with pytest.raises(cg.CgError) as e:
        g.cg_reorder_particles(pos[:-1], None, pos2[:-1], None)
    assert e.value.code == 4
    with pytest.raises(cg.CgError):
        g.cg_reorder_particles(pos2, None, pos2, None)
    g.close()


def test_allocation_failures_are_reported_and_recovered(cuda_lib):
    """Host-side fault injection (no device fault): each allocation of
    cg_create_grids fails in turn with CG_ERR_OOM and leaves no handle; a
    device step and a host-buffer step whose buffers cannot be allocated
    fail with CG_ERR_OOM, and the same handle then steps exactly as a
    fresh one."""
    import ctypes as C
    import torch
    cg = cuda_lib
    L = cg.lib()
    w = synth.tiny(seed=4)          # 10,000 particles: more than a new handle's particle scratch
    ref = run_step(cg, w, eps_fine=False)
    keys = ("cell", "perm", "cell_start", "eps_bulk", "u_bulk", "var_bulk", "force", "S_bulk", "S_fine", "sums")
    try:
        k = 0
        while True:
            assert L.cg_debug_fail_alloc_after(k) == 0
            h = C.c_void_p()
            rc = L.cg_create_grids(C.byref(cg.make_desc(w.desc)), None, C.byref(h))
            if rc == 0:                 # k allocations were all it needed: the injection is still armed
                assert L.cg_debug_fail_alloc_after(-1) == 0
                L.cg_destroy_grids(h)
                break
            assert rc == 3 and not h.value, (k, rc)
            k += 1
            assert k < 100
        assert k >= 6               # the bulk buffers and the particle scratch
        # device entry: the particle scratch grows for 10,000 particles and fails
        g = cg.Grids(w.desc)
        pos, vel, uf = inputs(w)
        out = g.alloc_outputs(w.n, bins=True)
        assert L.cg_debug_fail_alloc_after(0) == 0
        with pytest.raises(cg.CgError) as e:
            g.cg_step(pos, vel, uf, out)
        assert e.value.code == 3
        g.cg_step(pos, vel, uf, out)   # the injection switched itself off
        assert g.cg_sync_status()[0] == 0
        torch.cuda.synchronize()
        for key in keys:
            assert np.array_equal(to_np(out[key]), ref[key]), key
        g.close()
        # host entry: its first staging buffer fails, then (after the 13
        # staging buffers these outputs need) its particle scratch
        g = cg.Grids(w.desc)
        hout = {key: (v.cpu().pin_memory() if v is not None else None)
                for key, v in g.alloc_outputs(w.n, bins=True).items()}
        hpos = torch.from_numpy(w.pos_d.copy()).pin_memory()
        hvel = torch.from_numpy(w.vel.copy()).pin_memory()
        huf = torch.from_numpy(np.ascontiguousarray(w.u_fine.reshape(3, -1))).pin_memory()
        for fail_at in (0, 13):
            assert L.cg_debug_fail_alloc_after(fail_at) == 0
            with pytest.raises(cg.CgError) as e:
                g.cg_step_host(hpos, hvel, huf, hout)
            assert e.value.code == 3, fail_at
        g.cg_step_host(hpos, hvel, huf, hout)
        for key in keys:
            assert np.array_equal(hout[key].numpy(), ref[key]), key
        g.close()
    finally:
        L.cg_debug_fail_alloc_after(-1)
