"""The binding's checks of the tensors whose pointers cross the ABI, on the
CPU: the output layout it enforces is the one alloc_outputs builds, and a
host tensor handed to a device entry (which a kernel would dereference), a
wrong dtype, a wrong element count or a strided view is refused before any
call into the library."""
import types

import pytest
import torch

import paper_1807_11834_gb300 as cg


def _outputs(dtype, n=50, nb=64, nf=512, **kw):
    fake = types.SimpleNamespace(n_bulk=nb, n_fine=nf, dtype=dtype)
    return cg.Grids.alloc_outputs(fake, n, device="cpu", **kw), (n, nb, nf)


def test_layout_covers_every_step_output():
    assert set(cg.STEP_OUT_LAYOUT) == {name for name, _ in cg.StepOut._fields_}


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_alloc_outputs_satisfy_the_checks(dtype):
    for kw in (dict(), dict(var=False), dict(eps_fine=True, bins=True), dict(implicit=True),
               dict(eps_fine=True, bins=True, implicit_fine=True)):
        out, (n, nb, nf) = _outputs(dtype, **kw)
        cg.check_step_outputs(out, n, nb, nf, dtype, on_device=False)
    out, (n, nb, nf) = _outputs(dtype, n=0, bins=True)
    cg.check_step_outputs(out, 0, nb, nf, dtype, on_device=False)


def test_wrong_outputs_are_refused():
    dtype = torch.float32
    out, (n, nb, nf) = _outputs(dtype, eps_fine=True, bins=True)
    with pytest.raises(ValueError, match="CUDA"):
        cg.check_step_outputs(out, n, nb, nf, dtype, on_device=True)     # host memory to a device entry
    cases = {
        "eps_bulk": torch.empty(nb, dtype=torch.float32),                # porosity is always double
        "force": torch.empty(3, n + 1, dtype=dtype),                     # another particle count
        "S_fine": torch.empty(3, 2 * nf, dtype=dtype)[:, ::2],           # strided view
        "cell_start": torch.empty(nb, dtype=torch.int32),                # one short
        "perm": torch.empty(n, dtype=torch.int64),
        "u_bulk": torch.empty(3, nb, dtype=torch.float64),               # the other precision
    }
    for name, bad in cases.items():
        o = dict(out)
        o[name] = bad
        with pytest.raises(ValueError, match=name):
            cg.check_step_outputs(o, n, nb, nf, dtype, on_device=False)
    # None fields are the library's to judge (it refuses bad combinations itself)
    o = dict(out)
    o["var_bulk"] = o["eps_fine"] = o["cell"] = None
    cg.check_step_outputs(o, n, nb, nf, dtype, on_device=False)


def test_check_tensor():
    t = torch.zeros(4, 3)
    assert cg.check_tensor(t, 12, torch.float32, False, "t") is t
    with pytest.raises(ValueError):
        cg.check_tensor(t, 12, torch.float32, True, "t")
    with pytest.raises(ValueError):
        cg.check_tensor(t.t(), 12, torch.float32, False, "t")
    with pytest.raises(ValueError):
        cg.check_tensor(t, 11, torch.float32, False, "t")


def test_batch_refuses_host_tensors_before_any_library_call():
    import synth
    w = synth.batch_instance(0, 0, 16, 4, 100, 0.01)
    out, _ = _outputs(torch.float32, n=w.n, nb=(16 // 4) ** 3, nf=16 ** 3)
    pos, vel = torch.from_numpy(w.pos_d), torch.from_numpy(w.vel)
    uf = torch.from_numpy(w.u_fine.reshape(3, -1).copy())
    with pytest.raises(ValueError, match="CUDA"):
        cg.Batch([(w.desc, pos, vel, uf, out)])


def test_closure_entries_check_their_tensors_first():
    fake = types.SimpleNamespace(h=None)
    feats = torch.zeros(10, 8)
    with pytest.raises(ValueError, match="features"):
        cg.Mlp.forward(fake, feats, torch.zeros(10))                 # host memory
    with pytest.raises(ValueError, match="features"):
        cg.Mlp.train_step(fake, torch.zeros(10, 7), torch.zeros(10), 1e-3)
    with pytest.raises(ValueError, match="var_stale"):
        cg.Mlp.bind(fake, torch.zeros(5, dtype=torch.float64), None)


def test_static_binning_checks_its_tensors_first():
    """cg_bin_particles_static's wrapper refuses a host tensor, a particle
    array of the other precision and a short cell_start before its pointers
    reach the library (a kernel would otherwise read or write out of
    bounds)."""
    import synth
    w = synth.tiny(seed=0, n=64, fp64=False)
    nb = (w.desc["fine_n"][0] // w.desc["ratio"]) ** 3
    pos = torch.from_numpy(w.pos_d)
    perm = torch.empty(w.n, dtype=torch.int32)
    cs = torch.empty(nb + 1, dtype=torch.int32)
    with pytest.raises(ValueError, match="pos_d"):
        cg.cg_bin_particles_static(w.desc, pos, perm, cs)                      # host memory
    with pytest.raises(ValueError, match="pos_d"):
        cg.cg_bin_particles_static(w.desc, pos.double(), perm, cs)             # FP64 under an FP32 descriptor
    d64 = dict(w.desc, fp64=True)
    with pytest.raises(ValueError, match="pos_d"):
        cg.cg_bin_particles_static(d64, pos, perm, cs)                         # FP32 under an FP64 descriptor
