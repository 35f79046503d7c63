"""Pins of the oracle's maps between non-nested uniform grids (the
grid-to-grid maps computed once per simulation, Sec. 2.3):
u_B = sum_f V(B & f) u_f / sum_f V(B & f) and S_f = sum_B V(B & f) S_B / V_f.

Each pin checks something the formula does not restate: the weights against
an exact rational intersection on tiny grids, the reduction to the plain
mean and to cell injection for nested grids, conservation of sum S V, the
adjoint identity between the two maps, and constants kept constant."""
from fractions import Fraction as Fr
import itertools

import numpy as np
import pytest

import oracle

BULK = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (3, 2, 2))
FINE = ((-0.125, 0.0625, 0.0), (1.25, 1.0, 1.5), (7, 5, 4))


def exact_average(bulk, fine, u):
    """Rational-arithmetic intersection volumes (coordinates are dyadic
    numbers, cell bounds exact fractions)."""
    def bounds(g, a, i):
        x0, L, n = Fr(g[0][a]), Fr(g[1][a]), g[2][a]
        return x0 + i * L / n, x0 + (i + 1) * L / n
    nb, nf = bulk[2], fine[2]
    out = np.zeros(int(np.prod(nb)))
    for B in itertools.product(*[range(n) for n in nb]):
        cb = B[0] + nb[0] * (B[1] + nb[1] * B[2])
        W, acc = Fr(0), Fr(0)
        for f in itertools.product(*[range(n) for n in nf]):
            v = Fr(1)
            for a in range(3):
                b0, b1 = bounds(bulk, a, B[a])
                f0, f1 = bounds(fine, a, f[a])
                v *= max(Fr(0), min(b1, f1) - max(b0, f0))
            if v:
                cf = f[0] + nf[0] * (f[1] + nf[1] * f[2])
                W += v
                acc += v * Fr(float(u[cf]))
        out[cb] = float(acc / W) if W else 0.0
    return out


def test_average_matches_exact_rational_intersections():
    rng = np.random.default_rng(0)
    u = rng.normal(size=int(np.prod(FINE[2])))
    got = oracle.map_average(BULK, FINE, u)
    want = exact_average(BULK, FINE, u)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_nested_grids_reduce_to_mean_and_injection():
    desc = dict(origin=(0.0, 0.0, 0.0), extent=(1.0, 2.0, 1.0), fine_n=(8, 12, 6), ratio=2, law=0, interp=0,
                rho_f=1000.0, mu_f=1e-3, rho_p=2500.0, eps_switch=0.8, eps_min=0.1, prec=1)
    bulk = ((0.0, 0.0, 0.0), (1.0, 2.0, 1.0), (4, 6, 3))
    fine = ((0.0, 0.0, 0.0), (1.0, 2.0, 1.0), (8, 12, 6))
    rng = np.random.default_rng(1)
    u = rng.normal(size=(3, 8 * 12 * 6))
    mean, _ = oracle.average(desc, u)
    got = oracle.map_average(bulk, fine, u)
    assert np.max(np.abs(got - mean)) <= 1e-14
    S = rng.normal(size=(2, 4 * 6 * 3))
    Sf = oracle.map_project(bulk, fine, S)
    i, j, k = np.meshgrid(np.arange(8), np.arange(12), np.arange(6), indexing="ij")
    cb = (i // 2 + 4 * (j // 2 + 6 * (k // 2)))
    cf = i + 8 * (j + 12 * k)
    # each fine cell lies in one bulk cell: S_f = S_B up to the rounding of
    # the cell-bound differences against V_f
    assert np.max(np.abs(Sf[:, cf.ravel()] - S[:, cb.ravel()])) <= 1e-14 * np.max(np.abs(S))


def test_projection_conserves_and_maps_are_adjoint():
    bulk = ((0.0, 0.0, 0.0), (1.0, 1.0, 2.0), (5, 4, 7))
    fine = ((-0.01, -0.02, -0.03), (1.05, 1.03, 2.1), (13, 11, 19))   # covers the bulk grid
    rng = np.random.default_rng(2)
    S = rng.normal(size=(3, 5 * 4 * 7))
    Sf = oracle.map_project(bulk, fine, S)
    VB = 1.0 / 5 * 1.0 / 4 * 2.0 / 7
    Vf = 1.05 / 13 * 1.03 / 11 * 2.1 / 19
    tot_b = S.sum(axis=1) * VB
    tot_f = Sf.sum(axis=1) * Vf
    assert np.allclose(tot_f, tot_b, rtol=1e-12, atol=1e-12 * np.abs(S).sum() * VB)
    # sum_f V_f u_f S_f = sum_B S_B W_B u_B with W_B the covered volume (V_B here)
    u = rng.normal(size=13 * 11 * 19)
    ub = oracle.map_average(bulk, fine, u)
    lhs = (Vf * u[None, :] * Sf).sum(axis=1)
    rhs = (VB * ub[None, :] * S).sum(axis=1)
    assert np.allclose(lhs, rhs, rtol=1e-11, atol=1e-12)


def test_constants_stay_constant_and_uncovered_cells_are_zero():
    u = np.full(int(np.prod(FINE[2])), 3.25)
    got = oracle.map_average(BULK, FINE, u)
    assert np.max(np.abs(got - 3.25)) <= 4e-15
    # a bulk grid reaching beyond the fine one: cells with no overlap read 0
    bulk = ((0.0, 0.0, 0.0), (2.0, 1.0, 1.0), (4, 1, 1))
    fine = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (3, 3, 3))
    got = oracle.map_average(bulk, fine, np.ones(27))
    assert np.allclose(got[:2], 1.0) and np.all(got[2:] == 0.0)


def test_random_geometries_conserve_and_stay_adjoint():
    """Any pair of box grids where the fine one covers the bulk one:
    conservation of sum S V, the adjoint identity, constants kept."""
    hypothesis = pytest.importorskip("hypothesis")
    st = hypothesis.strategies

    @hypothesis.settings(max_examples=40, deadline=None)
    @hypothesis.given(st.lists(st.integers(1, 6), min_size=3, max_size=3),
                      st.lists(st.integers(1, 9), min_size=3, max_size=3),
                      st.lists(st.floats(0.0, 0.3), min_size=6, max_size=6),
                      st.integers(0, 2 ** 31 - 1))
    def check(nb, nf, pad, seed):
        L = np.array([1.0, 0.7, 1.3])
        bulk = ((0.0, 0.0, 0.0), tuple(L), tuple(nb))
        lo = -np.array(pad[:3]) * L
        hi = L * (1.0 + np.array(pad[3:]))
        fine = (tuple(lo), tuple(hi - lo), tuple(nf))
        rng = np.random.default_rng(seed)
        S = rng.normal(size=int(np.prod(nb)))
        u = rng.normal(size=int(np.prod(nf)))
        Sf = oracle.map_project(bulk, fine, S)
        ub = oracle.map_average(bulk, fine, u)
        VB = np.prod(L / np.array(nb))
        Vf = np.prod((hi - lo) / np.array(nf))
        scale = np.abs(S).sum() * VB + 1e-300
        assert abs(Sf.sum() * Vf - S.sum() * VB) <= 1e-12 * scale
        assert abs((Vf * u * Sf).sum() - (VB * ub * S).sum()) <= 1e-11 * (np.abs(u).max() * scale)
        assert np.allclose(oracle.map_average(bulk, fine, np.full(u.size, 2.5)), 2.5, rtol=0, atol=1e-14)

    check()
