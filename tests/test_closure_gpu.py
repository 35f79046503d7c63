"""The learned drag closure on the coupling grids, against the FP64 oracle.

* cg_mlp_features: closure inputs and targets at every particle from a
  stale and a fresh bulk record.  FP64 grids: each float32 output within
  two float roundings of the oracle's FP64 value.  FP32 grids: the path
  tolerance of its inputs, widened for the porosity gradient and the
  target, which are differences and ratios of drag forces (tolerances in
  the test bodies).
* cg_drag with a closure (FP32 only): in-range rows F = (1 + age r) F_stale
  with r the oracle network (bf16 mode) on the oracle's features; out-of-range
  rows the plain drag with the fresh fluid velocity.  The feature box is
  chosen so that a good share of rows falls back.  Rows whose scaled
  features sit within rounding of the box edge may take either branch and
  are checked against both.
* cg_step_learned: at age 0 it is cg_step bit for bit; at age >= 1 the
  stale record is left unchanged, the reaction and projection conserve the
  learned forces, and the fallback count is the number of rows outside the
  box.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import mlp as om
from parity_util import TOL_FP32, assert_close, inputs, rel_err, to_dev, to_np

pytestmark = pytest.mark.gpu


def _records(w):
    """Oracle porosity, stale record (from the workload's field) and fresh
    record (from the evolved field)."""
    u1 = synth.evolved_field(w, seed=3)
    ref = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine)
    ub1, _ = oracle.average(w.desc, u1, want_var=False)
    return ref, u1, ub1


def _features_on_gpu(cg, w, ref, ub1):
    import torch
    g = cg.Grids(w.desc)
    pos, vel, _ = inputs(w)
    dt = pos.dtype
    feat = torch.empty(w.n, 8, device="cuda", dtype=torch.float32)
    target = torch.empty(w.n, device="cuda", dtype=torch.float32)
    g.cg_mlp_features(pos, vel, to_dev(ref["eps_bulk"]), to_dev(ref["u_bulk"]).to(dt),
                      to_dev(ref["var_bulk"]).to(dt), to_dev(ub1).to(dt), feat, target)
    rc, _, _ = g.cg_sync_status()
    assert rc == 0
    out = to_np(feat), to_np(target)
    g.close()
    return out


def test_features_fp64_grids(cuda_lib):
    w = synth.tiny(seed=5, n=9_000)       # ragged: 9000 = 35 * 256 + 40
    ref, _, ub1 = _records(w)
    f, t = _features_on_gpu(cuda_lib, w, ref, ub1)
    fo, to, _ = oracle.mlp_features(w.desc, w.pos_d, w.vel, ref["eps_bulk"], ref["u_bulk"], ref["var_bulk"], ub1)
    # FP64 arithmetic, one rounding to float32 on each side of the compare
    tol = 2.0 ** -23
    for k in range(7):
        assert_close(f"feature {k}", f[:, k], fo[:, k], tol)
    assert np.all(f[:, 7] == 0.0)
    assert_close("target", t, to, tol)
    assert np.abs(to - 1.0).max() > 1e-3      # the stale and fresh records differ


def test_features_fp32_grids(cuda_lib):
    w = synth.small_packed_bed(seed=1)
    ref, _, ub1 = _records(w)
    f, t = _features_on_gpu(cuda_lib, w, ref, ub1)
    fo, to, _ = oracle.mlp_features(w.desc, w.pos_d, w.vel, ref["eps_bulk"], ref["u_bulk"], ref["var_bulk"], ub1)
    for k in (0, 1, 2, 6):
        assert_close(f"feature {k}", f[:, k], fo[:, k], TOL_FP32)
    # the gradient is a difference of bulk porosities, each rounded to FP32
    # (2^-24 |eps|), divided by H, then interpolated: absolute error within
    # 8 roundings of max |eps| over H, plus the path tolerance of the value
    eps_max = float(np.abs(ref["eps_bulk"]).max())
    H = min(w.desc["extent"][a] / w.desc["fine_n"][a] * w.desc["ratio"] for a in range(3))
    bound = 8 * 2.0 ** -24 * eps_max / H + TOL_FP32 * np.abs(fo[:, 3:6])
    err = np.abs(f[:, 3:6] - fo[:, 3:6])
    print("grad eps max err / bound", (err / bound).max())
    assert np.all(err <= bound)
    # the target is a ratio of two drags, each within the path tolerance
    assert_close("target", t, to, 4 * TOL_FP32)


# ---------------------------------------------------------------- learned drag
def _closure(cg, fo, seed=0, q=(0.03, 0.97), act="gelu"):
    """A random closure with a feature box from quantiles of the oracle's
    features (so that a good share of rows falls outside)."""
    lo = np.quantile(fo[:, :7], q[0], axis=0).astype(np.float32)
    hi = np.quantile(fo[:, :7], q[1], axis=0).astype(np.float32)
    hi = np.where(hi > lo, hi, lo + np.float32(1e-3) * np.maximum(np.abs(lo), 1)).astype(np.float32)
    p = om.init_params(hidden=64, seed=seed)
    rng = np.random.default_rng(seed + 1)
    p["b1"] = rng.normal(size=64) * 0.1
    p["b2"] = rng.normal(size=64) * 0.1
    m = cg.Mlp(cg.mlp_pack(p), lo, hi, activation=act)
    return m, cg.mlp_unpack(cg.mlp_pack(p)), lo, hi


def _expected_learned(w, ref, ub1, p, lo, hi, age=1, act="gelu"):
    """Oracle learned forces, the in-range decision, and the rows whose
    decision sits within rounding of the box edge."""
    fo, _, Fs = oracle.mlp_features(w.desc, w.pos_d, w.vel, ref["eps_bulk"], ref["u_bulk"], ref["var_bulk"], ub1)
    f32 = fo[:, :7].astype(np.float32)
    inv = (np.float32(1.0) / (hi - lo)).astype(np.float32)
    xs = ((f32 - lo) * inv).astype(np.float32)
    inside = np.all((xs >= 0) & (xs <= 1), axis=1)
    edge = np.any((np.abs(xs) < 1e-4) | (np.abs(xs - 1) < 1e-4), axis=1)
    X = np.zeros((w.n, om.K0))
    X[:, :7] = xs
    r, _ = om.forward(p, X, bf16_inputs=True, act=act)
    F_fresh, _ = oracle.drag(w.desc, w.pos_d, w.vel, ref["eps_bulk"], ub1)
    return (1.0 + age * r) * Fs, F_fresh, inside, edge, Fs


def _learned_drag(cg, w, ref, ub1, u1, m, age):
    import torch
    g = cg.Grids(w.desc)
    pos, vel, _ = inputs(w)
    var = to_dev(ref["var_bulk"]).float()
    uf1 = to_dev(u1.reshape(3, -1)).float()
    m.bind(var, uf1, age)
    F = torch.empty(3, w.n, device="cuda", dtype=torch.float32)
    g.cg_drag(pos, vel, to_dev(ref["eps_bulk"]), to_dev(ref["u_bulk"]).float(), F, mlp=m)
    rc, flags, counts = g.cg_sync_status()
    assert rc == 0 and m.sync_status()[0] == 0
    out = to_np(F), counts
    g.close()
    return out


@pytest.mark.parametrize("act", ["gelu", "relu"])
@pytest.mark.parametrize("make", [synth.small_clustered_bed, synth.small_packed_bed])
def test_learned_drag_matches_oracle(cuda_lib, make, act):
    w = make(seed=2)
    ref, u1, ub1 = _records(w)
    fo, _, _ = oracle.mlp_features(w.desc, w.pos_d, w.vel, ref["eps_bulk"], ref["u_bulk"], ref["var_bulk"], ub1)
    m, p, lo, hi = _closure(cuda_lib, fo, act=act)
    age = 2
    F, counts = _learned_drag(cuda_lib, w, ref, ub1, u1, m, age)
    F_c, F_fresh, inside, edge, Fs = _expected_learned(w, ref, ub1, p, lo, hi, age, act)
    sure = ~edge
    print("rows", w.n, "in range", inside.sum(), "edge", edge.sum(), "fallbacks", counts[4])
    assert 0.1 * w.n < (~inside).sum() < 0.9 * w.n
    # learned rows: r within 5e-3 (bf16 operands, FP32 accumulation and
    # GELU, one-ulp bf16 re-rounding of inputs and activations), times the
    # age, on top of the FP32 drag
    scale = np.sqrt((Fs ** 2).sum(axis=0))
    floor = 1e-3 * scale.max()
    err_c = np.sqrt(((F - F_c) ** 2).sum(axis=0)) / np.maximum(scale, floor)
    a = inside & sure
    print("learned rows max err", err_c[a].max(), "median", np.median(err_c[a]))
    assert err_c[a].max() < age * 5e-3 + 4 * TOL_FP32 and np.median(err_c[a]) < age * 2e-4
    # fallback rows: plain drag with the fresh velocity, averaged by the
    # kernel with plain FP32 sums of r^3 = 64 values
    b = ~inside & sure
    mx, _ = rel_err(F[:, b], F_fresh[:, b], vec=True)
    print("fallback rows max err", mx)
    assert mx < 1e-5
    # edge rows: either branch
    for i in np.nonzero(edge)[0]:
        e1 = np.linalg.norm(F[:, i] - F_c[:, i]) / max(np.linalg.norm(Fs[:, i]), floor)
        e2 = np.linalg.norm(F[:, i] - F_fresh[:, i]) / max(np.linalg.norm(F_fresh[:, i]), floor)
        assert min(e1, e2) < age * 5e-3 + 1e-5
    assert abs(counts[4] - int((~inside).sum())) <= int(edge.sum())
    m.close()


def test_learned_drag_argument_checks(cuda_lib):
    import torch
    w = synth.tiny(seed=0, n=1000, fp64=False)
    g = cuda_lib.Grids(w.desc)
    pos, vel, uf = inputs(w)
    p = om.init_params(hidden=64, seed=0)
    m = cuda_lib.Mlp(cuda_lib.mlp_pack(p), np.zeros(7, np.float32), np.ones(7, np.float32))
    eps = torch.ones(g.n_bulk, device="cuda", dtype=torch.float64)
    ub = torch.zeros(3, g.n_bulk, device="cuda")
    F = torch.empty(3, w.n, device="cuda")
    with pytest.raises(cuda_lib.CgError):       # nothing bound yet
        g.cg_drag(pos, vel, eps, ub, F, mlp=m)
    g.close()
    w64 = synth.tiny(seed=0, n=1000, fp64=True)
    g64 = cuda_lib.Grids(w64.desc)
    pos64, vel64, uf64 = inputs(w64)
    m.bind(torch.zeros(g64.n_bulk, device="cuda"), uf64.float())
    with pytest.raises(cuda_lib.CgError):       # FP64 grids have no learned path
        g64.cg_drag(pos64, vel64, eps, ub.double(), torch.empty(3, w64.n, device="cuda", dtype=torch.float64),
                    mlp=m)
    g64.close()
    m.close()


# ---------------------------------------------------------------- learned step
def test_learned_step(cuda_lib):
    import torch
    cg = cuda_lib
    w = synth.small_clustered_bed(seed=4)
    ref, u1, ub1 = _records(w)
    fo, _, _ = oracle.mlp_features(w.desc, w.pos_d, w.vel, ref["eps_bulk"], ref["u_bulk"], ref["var_bulk"], ub1)
    m, p, lo, hi = _closure(cg, fo, seed=7)
    g = cg.Grids(w.desc)
    pos, vel, uf0 = inputs(w)
    uf1 = to_dev(u1.reshape(3, -1)).float()

    # age 0 (a refresh): identical to cg_step
    o_ref = g.alloc_outputs(w.n, eps_fine=True)
    g.cg_step(pos, vel, uf0, o_ref)
    o = g.alloc_outputs(w.n, eps_fine=True)
    g.cg_step_learned(pos, vel, uf0, o, m, age=0)
    torch.cuda.synchronize()
    for k in ("eps_bulk", "u_bulk", "var_bulk", "S_bulk", "force", "S_fine", "eps_fine"):
        assert torch.equal(o[k], o_ref[k]), k
    assert g.cg_sync_status()[2][4] == 0

    # age 3, fresh fine field: stale record kept, learned forces
    ub_keep, var_keep = o["u_bulk"].clone(), o["var_bulk"].clone()
    g.cg_step_learned(pos, vel, uf1, o, m, age=3)
    rc, _, counts = g.cg_sync_status()
    assert rc == 0
    assert torch.equal(o["u_bulk"], ub_keep) and torch.equal(o["var_bulk"], var_keep)
    assert torch.equal(o["eps_bulk"], o_ref["eps_bulk"])
    # the same forces as the learned drag entry on the same record
    m.bind(o["var_bulk"], uf1, 3)
    F = torch.empty_like(o["force"])
    g.cg_drag(pos, vel, o["eps_bulk"], o["u_bulk"], F, mlp=m)
    torch.cuda.synchronize()
    assert torch.equal(F, o["force"])
    _, _, inside, edge, _ = _expected_learned(w, ref, ub1, p, lo, hi, 3)
    assert abs(counts[4] - int((~inside).sum())) <= int(edge.sum())
    # reaction and projection conserve the learned forces
    s = to_np(o["sums"])
    Fsum = to_np(o["force"]).astype(np.float64).sum(axis=1)
    absF = np.sqrt((to_np(o["force"]).astype(np.float64) ** 2).sum(axis=0)).sum()
    assert np.all(np.abs(Fsum + s[5:8]) <= 1e-5 * absF)
    assert np.all(np.abs(s[5:8] - s[8:11]) <= 1e-5 * absF)
    assert np.all(np.isnan(s[[0, 2, 3, 4, 11, 12, 13, 14, 15]]))
    g.close()
    m.close()
