"""Semi-implicit exchange coefficients (Eq. UFP: F_fpi treated
semi-implicitly) on the GPU against the FP64 oracle: A = sum beta_p / V_B and
b = sum beta_p u_p / V_B per bulk cell, and their projection onto the fine
grid, within the path tolerance; requesting them changes no other output."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import TOL_FP32, TOL_FP64, assert_close, assert_close_interp, inputs, switch_mask, to_np

pytestmark = pytest.mark.gpu


def run(cg, w, dt=0.0, implicit=True, fine=True):
    import torch
    g = cg.Grids(w.desc)
    pos, vel, uf = inputs(w)
    out = g.alloc_outputs(w.n, eps_fine=True, bins=True, implicit=implicit, implicit_fine=implicit and fine)
    g.cg_step(pos, vel, uf, out, dt=dt)
    rc, _, _ = g.cg_sync_status()
    torch.cuda.synchronize()
    host = {k: to_np(v) for k, v in out.items()}
    host["rc"] = rc
    g.close()
    return host


def check(w, got, tol, dt=0.0):
    ref = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, dt=0.0)
    A, b = oracle.implicit(w.desc, w.pos_d, w.vel, ref["eps_bulk"], ref["u_bulk"], ref["cell_start"], ref["perm"])
    # cells holding a particle within rounding of a correlation switch may
    # legitimately take the other branch in FP32
    keep = switch_mask(w, ref)
    bad = np.zeros(A.size, bool)
    bad[ref["cell"][~keep]] = True
    cm = ~bad
    assert_close("A", got["implicit_bulk"][0], A, tol, mask=cm)
    assert_close("b", got["implicit_bulk"][1:], b, tol, vec=True, mask=cm)
    if got.get("implicit_fine") is not None and cm.all():
        coef = np.vstack([A[None, :], b])
        ref_f = oracle.project(w.desc, coef)
        ref_abs = oracle.project(w.desc, np.abs(coef))
        assert_close_interp("A_f", got["implicit_fine"][0], ref_f[0], ref_abs[0], tol)
        assert_close_interp("b_f", got["implicit_fine"][1:], ref_f[1:], ref_abs[1:], tol)
    return A, b


def test_fp64_tiny_coefficients_and_projection(cuda_lib):
    w = synth.tiny(seed=12, n=6000)
    got = run(cuda_lib, w)
    assert got["rc"] == 0
    check(w, got, TOL_FP64)


@pytest.mark.parametrize("name", ["small_packed_bed", "small_clustered_bed"])
def test_fp32_beds(cuda_lib, name):
    w = getattr(synth, name)(seed=4)
    got = run(cuda_lib, w)
    A, b = check(w, got, TOL_FP32)
    assert np.count_nonzero(A) > 0


def test_euler_uses_velocity_before_the_advance(cuda_lib):
    w = synth.small_clustered_bed(seed=5)
    got = run(cuda_lib, w, dt=w.dt, fine=False)
    check(w, got, TOL_FP32)


def test_requesting_them_changes_nothing_else(cuda_lib):
    w = synth.small_packed_bed(seed=6)
    a = run(cuda_lib, w)
    b = run(cuda_lib, w, implicit=False)
    for k in ("eps_bulk", "u_bulk", "var_bulk", "S_bulk", "force", "S_fine", "eps_fine", "perm", "cell_start"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["sums"], b["sums"])


def test_invalid_requests(cuda_lib):
    import torch
    cg = cuda_lib
    w = synth.tiny(seed=1, n=200, fp64=False)
    g = cg.Grids(w.desc)
    pos, vel, uf = inputs(w)
    out = g.alloc_outputs(w.n, implicit_fine=True)
    out2 = dict(out)
    out2["implicit_bulk"] = None
    with pytest.raises(cg.CgError):
        g.cg_step(pos, vel, uf, out2)
    m = cg.Mlp(np.zeros(cg.MLP_NPARAM, np.float32), np.zeros(cg.MLP_NFEAT, np.float32),
               np.ones(cg.MLP_NFEAT, np.float32))
    with pytest.raises(cg.CgError):
        g.cg_step_learned(pos, vel, uf, out, m, age=0)
    with pytest.raises(cg.CgError):
        cg.Batch([(w.desc, pos, vel, uf, out)])
    torch.cuda.synchronize()
    m.close()
    g.close()
