"""Maps between non-nested uniform grids on the GPU against the FP64 oracle
(volume-weighted fine -> bulk average, conservative bulk -> fine
projection): FP64 within 1e-12, FP32 within 2e-6; conservation of sum S V;
argument checks."""
import numpy as np
import pytest

import oracle
from parity_util import TOL_FP32, TOL_FP64, assert_close, assert_close_interp, to_dev, to_np

pytestmark = pytest.mark.gpu

# a bulk grid and an offset fine grid with a non-integer spacing ratio
# (2.7 to 3.3 fine cells per bulk cell) reaching past the bulk grid
BULK = ((0.0, 0.0, 0.0), (1.0, 0.8, 1.2), (12, 9, 14))
FINE = ((-0.013, -0.021, -0.007), (1.031, 0.845, 1.219), (37, 29, 41))


def nb(g):
    return int(np.prod(g[2]))


@pytest.mark.parametrize("fp64", [True, False])
def test_average_and_projection_match_oracle(cuda_lib, fp64):
    import torch
    cg = cuda_lib
    tol = TOL_FP64 if fp64 else TOL_FP32
    dt = np.float64 if fp64 else np.float32
    rng = np.random.default_rng(7)
    u = (0.5 + 0.1 * rng.standard_normal((3, nb(FINE)))).astype(dt)
    S = rng.standard_normal((4, nb(BULK))).astype(dt)
    m = cg.Map(BULK, FINE, fp64=fp64)
    ub = torch.empty(3, nb(BULK), dtype=m.dtype, device="cuda")
    sf = torch.empty(4, nb(FINE), dtype=m.dtype, device="cuda")
    m.average(to_dev(u), ub)
    m.project(to_dev(S), sf)
    torch.cuda.synchronize()
    ref_u = oracle.map_average(BULK, FINE, u)
    ref_s = oracle.map_project(BULK, FINE, S)
    assert_close("u_B", to_np(ub), ref_u, tol, vec=True)
    ref_abs = oracle.map_project(BULK, FINE, np.abs(S.astype(np.float64)))
    assert_close_interp("S_f", to_np(sf), ref_s, ref_abs, tol)
    # conservation on the device result (the fine grid covers the bulk one)
    VB = np.prod(np.asarray(BULK[1]) / np.asarray(BULK[2]))
    Vf = np.prod(np.asarray(FINE[1]) / np.asarray(FINE[2]))
    tot_b = S.astype(np.float64).sum(axis=1) * VB
    tot_f = to_np(sf).astype(np.float64).sum(axis=1) * Vf
    scale = np.abs(S).astype(np.float64).sum(axis=1) * VB
    assert np.all(np.abs(tot_f - tot_b) <= (1e-12 if fp64 else 1e-5) * scale)
    m.close()


def test_one_component_and_large_fine_cells(cuda_lib):
    # fine cells larger than the bulk cells: several bulk cells per fine cell
    import torch
    cg = cuda_lib
    bulk = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (20, 16, 12))
    fine = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (7, 5, 9))
    rng = np.random.default_rng(8)
    u = rng.standard_normal(nb(fine))
    S = rng.standard_normal(nb(bulk))
    m = cg.Map(bulk, fine, fp64=True)
    ub = torch.empty(nb(bulk), dtype=torch.float64, device="cuda")
    sf = torch.empty(nb(fine), dtype=torch.float64, device="cuda")
    m.average(to_dev(u), ub)
    m.project(to_dev(S), sf)
    torch.cuda.synchronize()
    assert_close("u_B", to_np(ub), oracle.map_average(bulk, fine, u), TOL_FP64)
    assert_close("S_f", to_np(sf), oracle.map_project(bulk, fine, S), TOL_FP64)
    m.close()


def test_argument_checks(cuda_lib):
    import torch
    cg = cuda_lib
    with pytest.raises(cg.CgError):
        cg.Map(((0, 0, 0), (1, 1, 1), (4, 4, 0)), FINE)
    with pytest.raises(cg.CgError):
        cg.Map(((0, 0, 0), (1, -1, 1), (4, 4, 4)), FINE)
    m = cg.Map(BULK, FINE)
    L = cg.lib()
    a = torch.zeros(9, nb(FINE), device="cuda")
    b = torch.zeros(9, nb(BULK), device="cuda")
    assert L.cg_map_average(m.h, 9, a.data_ptr(), b.data_ptr()) == 1
    assert L.cg_map_average(m.h, 0, a.data_ptr(), b.data_ptr()) == 1
    assert L.cg_map_project(m.h, 2, b.data_ptr() + 2, a.data_ptr()) == 1
    m.close()
