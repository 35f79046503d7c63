"""Pins of the oracle's grid operations: binning, porosity, fine->bulk
averaging, trilinear gather and bulk->fine projection.

Each pin comes from something other than the oracle's own formula: brute
force on tiny grids written independently here, closed forms, or
conservation invariants.  Grids use dyadic spacings so that the brute-force
geometry is exact in double precision.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def desc_small(nf=(8, 12, 16), r=4, origin=(-0.5, 0.25, 1.0), extent=(1.0, 1.5, 2.0), **kw):
    # bulk (2, 3, 4) with H = 0.5 on every axis: all faces exactly representable
    d = synth.make_desc(origin, extent, nf, r, fp64=True, law=kw.pop("law", 0), **kw)
    return d


def nb_of(desc):
    return tuple(v // desc["ratio"] for v in desc["fine_n"])


def brute_cell(desc, x):
    """Cell by testing every box [x0 + i H, x0 + (i+1) H) (last box closed)."""
    nb = nb_of(desc)
    idx = []
    for a in range(3):
        H = desc["extent"][a] / nb[a]
        lo = desc["origin"][a]
        found = None
        for i in range(nb[a]):
            a0 = lo + i * H
            a1 = lo + (i + 1) * H
            if a0 <= x[a] < a1 or (i == nb[a] - 1 and x[a] == a1):
                found = i
        if found is None:  # outside: nearest cell
            found = 0 if x[a] < lo else nb[a] - 1
        idx.append(found)
    return idx[0] + nb[0] * (idx[1] + nb[1] * idx[2])


# --------------------------------------------------------------------------
# B1: bin index and stable sort (Sec. 2.2: per-step particle/cell connectivity)
# --------------------------------------------------------------------------
def test_bin_brute_force_and_faces():
    desc = desc_small()
    rng = np.random.default_rng(7)
    nb = nb_of(desc)
    x0 = np.array(desc["origin"])
    L = np.array(desc["extent"])
    pts = [x0 + rng.random(3) * L for _ in range(300)]
    H = L / np.array(nb)
    # exactly on interior faces, on the lower faces and on the upper domain faces
    for i in range(nb[0] + 1):
        for j in range(nb[1] + 1):
            for k in range(nb[2] + 1):
                pts.append(x0 + np.array([i, j, k]) * H)
    for p in pts:
        c, out = oracle.bin_cell(desc, p)
        assert c == brute_cell(desc, p)
        assert not out


def test_bin_linear_index_is_x_fastest():
    desc = desc_small()
    nb = nb_of(desc)
    x0 = np.array(desc["origin"])
    H = np.array(desc["extent"]) / np.array(nb)
    centre = lambda i, j, k: x0 + (np.array([i, j, k]) + 0.5) * H
    assert oracle.bin_cell(desc, centre(1, 0, 0))[0] == 1
    assert oracle.bin_cell(desc, centre(0, 1, 0))[0] == nb[0]
    assert oracle.bin_cell(desc, centre(0, 0, 1))[0] == nb[0] * nb[1]
    assert oracle.bin_cell(desc, centre(1, 2, 3))[0] == 1 + nb[0] * (2 + nb[1] * 3)


def test_bin_outside_is_clamped_and_counted():
    desc = desc_small()
    x0 = np.array(desc["origin"])
    L = np.array(desc["extent"])
    nb = nb_of(desc)
    below = x0 - 0.01
    above = x0 + L + 0.01
    assert oracle.bin_cell(desc, below) == (0, True)
    assert oracle.bin_cell(desc, above) == (nb[0] * nb[1] * nb[2] - 1, True)
    assert oracle.bin_cell(desc, [np.nan, 0.5, 1.5])[1]
    pos = np.zeros((3, 4))
    pos[0, :3] = below
    pos[1, :3] = above
    pos[2, :3] = x0 + L / 2
    cell, perm, cs, nout = oracle.bin(desc, pos)
    assert nout == 2


def test_bin_is_stable_sort():
    desc = desc_small()
    rng = np.random.default_rng(3)
    n = 5000
    x0 = np.array(desc["origin"])
    L = np.array(desc["extent"])
    pos = np.zeros((n, 4))
    pos[:, :3] = x0 + rng.random((n, 3)) * L
    # snap some to faces so ties and faces both appear
    pos[::7, 0] = x0[0] + 0.5
    cell, perm, cs, nout = oracle.bin(desc, pos)
    assert nout == 0
    want_cell = np.array([brute_cell(desc, p[:3]) for p in pos])
    assert np.array_equal(cell, want_cell)
    assert np.array_equal(perm, np.argsort(want_cell, kind="stable"))
    nbulk = np.prod(nb_of(desc))
    counts = np.bincount(want_cell, minlength=nbulk)
    assert cs[0] == 0 and cs[-1] == n
    assert np.array_equal(np.diff(cs), counts)


# --------------------------------------------------------------------------
# D0: porosity (Table 1: sum V_p / V_cell; Sec. 2.4: eps = fluid / cell volume)
# --------------------------------------------------------------------------
def test_porosity_conserves_volume_and_empty_cells():
    w = synth.tiny(seed=1, n=3000)
    desc = w.desc
    cell, perm, cs, _ = oracle.bin(desc, w.pos_d)
    eps, phi = oracle.deposit_volume(desc, w.pos_d, cs, perm)
    nb = nb_of(desc)
    VB = np.prod(np.array(desc["extent"]) / np.array(nb))
    # sphere volume as 4/3 pi r^3
    vp = 4.0 / 3.0 * math.pi * (w.pos_d[:, 3] / 2.0) ** 3
    assert math.isclose(np.sum((1.0 - eps) * VB), math.fsum(vp), rel_tol=1e-13)
    assert np.allclose(eps, 1.0 - phi, rtol=0, atol=1e-15)
    # remove every particle of cell 5: that cell must be exactly 1
    keep = cell != 5
    pos2 = w.pos_d[keep]
    c2, p2, cs2, _ = oracle.bin(desc, pos2)
    e2, _ = oracle.deposit_volume(desc, pos2, cs2, p2)
    assert e2[5] == 1.0


def test_porosity_single_particle():
    desc = desc_small()
    nb = nb_of(desc)
    VB = 0.5 ** 3
    d = 0.3
    pos = np.array([[-0.5 + 0.7, 0.25 + 1.1, 1.0 + 0.2, d]])
    cell, perm, cs, _ = oracle.bin(desc, pos)
    eps, phi = oracle.deposit_volume(desc, pos, cs, perm)
    c = brute_cell(desc, pos[0, :3])
    want = 4.0 / 3.0 * math.pi * (d / 2) ** 3 / VB
    assert math.isclose(phi[c], want, rel_tol=1e-15)
    others = np.delete(eps, c)
    assert np.all(others == 1.0)


def test_porosity_hand_worked_golden():
    """tests/golden/porosity_2x2x2.txt: two spheres in a 2^3 bulk grid."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "porosity_2x2x2.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    desc = synth.make_desc((0, 0, 0), (1, 1, 1), (4, 4, 4), 2, fp64=True, law=0)
    pos = np.array([[float(v) for v in r[1:5]] for r in rows if r[0] == "particle"])
    want = {int(r[1]): float(r[2]) for r in rows if r[0] == "phi"}
    cell, perm, cs, _ = oracle.bin(desc, pos)
    eps, phi = oracle.deposit_volume(desc, pos, cs, perm)
    for c in range(8):
        assert math.isclose(phi[c], want.get(c, 0.0), rel_tol=1e-15, abs_tol=0)


# --------------------------------------------------------------------------
# A: fine -> bulk averaging (Fig. 1, fine-to-coarse arrow)
# --------------------------------------------------------------------------
def test_average_brute_force_reshape_mean():
    desc = desc_small()
    nf = desc["fine_n"]
    r = desc["ratio"]
    rng = np.random.default_rng(11)
    u = rng.normal(size=(3, nf[2], nf[1], nf[0]))
    ub, var = oracle.average(desc, u)
    nb = nb_of(desc)
    blocks = u.reshape(3, nb[2], r, nb[1], r, nb[0], r)
    mean = blocks.mean(axis=(2, 4, 6))
    assert np.allclose(ub.reshape(3, nb[2], nb[1], nb[0]), mean, rtol=1e-14, atol=1e-15)
    dev = blocks - mean[:, :, None, :, None, :, None]
    v = (dev ** 2).sum(axis=0).mean(axis=(1, 3, 5))
    assert np.allclose(var.reshape(nb[2], nb[1], nb[0]), v, rtol=1e-13, atol=1e-15)


def test_average_linear_field_closed_forms():
    desc = desc_small()
    nf = desc["fine_n"]
    r = desc["ratio"]
    nb = nb_of(desc)
    h = np.array(desc["extent"]) / np.array(nf)
    H = h * r
    cx, cy, cz = synth.fine_centres(desc["origin"], desc["extent"], nf)
    Z, Y, X = np.meshgrid(cz, cy, cx, indexing="ij")
    b = np.array([[0.5, -1.0, 2.0], [1.5, 0.25, -0.75], [0.0, 0.0, 3.0]])
    a0 = np.array([1.0, -2.0, 0.5])
    u = np.stack([a0[c] + b[c, 0] * X + b[c, 1] * Y + b[c, 2] * Z for c in range(3)])
    ub, var = oracle.average(desc, u)
    # mean of a linear field over the symmetric r^3 points = value at the bulk centre
    bx = desc["origin"][0] + (np.arange(nb[0]) + 0.5) * H[0]
    by = desc["origin"][1] + (np.arange(nb[1]) + 0.5) * H[1]
    bz = desc["origin"][2] + (np.arange(nb[2]) + 0.5) * H[2]
    BZ, BY, BX = np.meshgrid(bz, by, bx, indexing="ij")
    for c in range(3):
        want = a0[c] + b[c, 0] * BX + b[c, 1] * BY + b[c, 2] * BZ
        assert np.allclose(ub[c].reshape(want.shape), want, rtol=1e-13, atol=1e-13)
    # variance of r equispaced points with spacing h is h^2 (r^2 - 1) / 12 per axis
    want_var = sum(b[c, a] ** 2 * h[a] ** 2 * (r * r - 1) / 12.0 for c in range(3) for a in range(3))
    assert np.allclose(var, want_var, rtol=1e-12)
    # constant field: exact mean, zero variance
    uc = np.full_like(u, 0.3)
    ubc, varc = oracle.average(desc, uc)
    assert np.all(ubc == 0.3) and np.all(varc == 0.0)


def test_average_conserves_volume_integral():
    desc = desc_small()
    nf = desc["fine_n"]
    rng = np.random.default_rng(5)
    u = rng.normal(size=(3, nf[2], nf[1], nf[0]))
    ub, _ = oracle.average(desc, u, want_var=False)
    r = desc["ratio"]
    # V_B = r^3 V_f
    assert np.allclose(ub.sum(axis=1) * r ** 3, u.reshape(3, -1).sum(axis=1), rtol=1e-13)


# --------------------------------------------------------------------------
# I: interpolation (cell value or local interpolant, Sec. 1)
# --------------------------------------------------------------------------
def hat_interp(desc, bulk, x):
    """Independent formulation: clamp the lattice coordinate to the hull of
    the bulk-cell centres, then sum hat functions max(0, 1 - |xi - j|)."""
    nb = nb_of(desc)
    H = np.array(desc["extent"]) / np.array(nb)
    xi = (np.asarray(x) - np.array(desc["origin"])) / H - 0.5
    xi = np.clip(xi, 0.0, np.array(nb) - 1.0)
    wx = [np.maximum(0.0, 1.0 - np.abs(xi[a] - np.arange(nb[a]))) for a in range(3)]
    B = np.asarray(bulk).reshape(nb[2], nb[1], nb[0])
    return np.einsum("k,j,i,kji->", wx[2], wx[1], wx[0], B)


def test_gather_matches_hat_functions():
    desc = desc_small()
    nb = nb_of(desc)
    rng = np.random.default_rng(2)
    bulk = rng.normal(size=int(np.prod(nb)))
    x0 = np.array(desc["origin"])
    L = np.array(desc["extent"])
    for _ in range(400):
        x = x0 + rng.random(3) * L
        assert math.isclose(oracle.gather(desc, bulk, x)[0], hat_interp(desc, bulk, x),
                            rel_tol=1e-13, abs_tol=1e-14)


def test_gather_reproduces_constant_linear_and_centres():
    desc = desc_small()
    nb = nb_of(desc)
    H = np.array(desc["extent"]) / np.array(nb)
    x0 = np.array(desc["origin"])
    L = np.array(desc["extent"])
    b = np.array([0.7, -1.3, 0.4])
    cen = [x0[a] + (np.arange(nb[a]) + 0.5) * H[a] for a in range(3)]
    BZ, BY, BX = np.meshgrid(cen[2], cen[1], cen[0], indexing="ij")
    lin = (2.0 + b[0] * BX + b[1] * BY + b[2] * BZ).ravel()
    const = np.full(int(np.prod(nb)), -0.25)
    rng = np.random.default_rng(9)
    for _ in range(300):
        x = x0 + rng.random(3) * L
        assert oracle.gather(desc, const, x)[0] == pytest.approx(-0.25, abs=1e-15)
        xin = x0 + H / 2 + rng.random(3) * (L - H)          # inside the centre hull
        assert oracle.gather(desc, lin, xin)[0] == pytest.approx(2.0 + b @ xin, rel=1e-13, abs=1e-13)
        g = oracle.gather_grad(desc, lin, xin)
        assert np.allclose(g, b, rtol=1e-12, atol=1e-12)
    for k in range(nb[2]):
        for j in range(nb[1]):
            for i in range(nb[0]):
                c = i + nb[0] * (j + nb[1] * k)
                xc = [cen[0][i], cen[1][j], cen[2][k]]
                assert oracle.gather(desc, lin, xc)[0] == pytest.approx(lin[c], rel=1e-14, abs=1e-14)
    # outer half cell: constant extrapolation -> zero gradient along that axis
    xo = np.array([x0[0] + 0.1 * H[0], x0[1] + 1.3 * H[1], x0[2] + 1.7 * H[2]])
    g = oracle.gather_grad(desc, lin, xo)
    assert g[0] == 0.0 and g[1] == pytest.approx(b[1]) and g[2] == pytest.approx(b[2])


def test_gather_gradient_matches_finite_difference():
    desc = desc_small()
    nb = nb_of(desc)
    rng = np.random.default_rng(12)
    bulk = rng.normal(size=int(np.prod(nb)))
    H = np.array(desc["extent"]) / np.array(nb)
    x0 = np.array(desc["origin"])
    for _ in range(100):
        # a point strictly inside a centre-to-centre cell, away from its faces
        cell = np.array([rng.integers(0, nb[a] - 1) for a in range(3)])
        frac = 0.2 + 0.6 * rng.random(3)
        x = x0 + (cell + 0.5 + frac) * H
        g = oracle.gather_grad(desc, bulk, x)
        for a in range(3):
            e = np.zeros(3)
            e[a] = 1e-4 * H[a]
            fd = (oracle.gather(desc, bulk, x + e)[0] - oracle.gather(desc, bulk, x - e)[0]) / (2 * e[a])
            assert fd == pytest.approx(g[a], rel=1e-6, abs=1e-8)


def test_cell_interp_is_cell_value():
    desc = desc_small(interp=synth.INTERP_CELL)
    nb = nb_of(desc)
    rng = np.random.default_rng(4)
    bulk = rng.normal(size=int(np.prod(nb)))
    x0 = np.array(desc["origin"])
    L = np.array(desc["extent"])
    for _ in range(100):
        x = x0 + rng.random(3) * L
        assert oracle.gather(desc, bulk, x)[0] == bulk[brute_cell(desc, x)]


# --------------------------------------------------------------------------
# P: bulk -> fine projection (Fig. 1, coarse-to-fine arrow)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("r", [2, 3, 4, 8])
def test_projection_brute_force_and_conservation(r):
    nb = (2, 3, 4)
    nf = tuple(v * r for v in nb)
    desc = synth.make_desc((-0.5, 0.25, 1.0), (1.0, 1.5, 2.0), nf, r, fp64=True, law=0)
    rng = np.random.default_rng(r)
    bulk = rng.normal(size=(2, int(np.prod(nb))))
    fine = oracle.project(desc, bulk)
    cx, cy, cz = synth.fine_centres(desc["origin"], desc["extent"], nf)
    f = 0
    for k in range(nf[2]):
        for j in range(nf[1]):
            for i in range(nf[0]):
                x = (cx[i], cy[j], cz[k])
                for comp in range(2):
                    assert math.isclose(fine[comp, f], hat_interp(desc, bulk[comp], x),
                                        rel_tol=1e-13, abs_tol=1e-14)
                f += 1
    # sum_f S_f V_f = sum_B S_B V_B with V_B = r^3 V_f
    assert np.allclose(fine.sum(axis=1), bulk.sum(axis=1) * r ** 3, rtol=1e-12, atol=1e-12)


def test_projection_constant_and_linear_interior():
    desc = desc_small()
    nb = nb_of(desc)
    nf = desc["fine_n"]
    H = np.array(desc["extent"]) / np.array(nb)
    x0 = np.array(desc["origin"])
    cen = [x0[a] + (np.arange(nb[a]) + 0.5) * H[a] for a in range(3)]
    BZ, BY, BX = np.meshgrid(cen[2], cen[1], cen[0], indexing="ij")
    b = np.array([0.3, 0.9, -0.6])
    lin = (1.0 + b[0] * BX + b[1] * BY + b[2] * BZ).ravel()
    fine = oracle.project(desc, lin).reshape(nf[2], nf[1], nf[0])
    cx, cy, cz = synth.fine_centres(desc["origin"], desc["extent"], nf)
    for k in range(nf[2]):
        for j in range(nf[1]):
            for i in range(nf[0]):
                x = np.array([cx[i], cy[j], cz[k]])
                if np.all(x >= x0 + H / 2) and np.all(x <= x0 + np.array(desc["extent"]) - H / 2):
                    assert fine[k, j, i] == pytest.approx(1.0 + b @ x, rel=1e-13)
    const = oracle.project(desc, np.full(int(np.prod(nb)), 2.5))
    assert np.all(np.abs(const - 2.5) < 1e-15)


def test_threaded_build_is_bit_identical():
    """The OpenMP build of the oracle (its loops over independent particles,
    cells and fine cells on every host core) gives the single-thread
    build's step bit for bit, Euler advance included."""
    import os
    import oracle
    import synth
    w = synth.small_clustered_bed(seed=2)
    a = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, dt=w.dt, want_eps_fine=True)
    b = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, dt=w.dt, want_eps_fine=True, threads=True)
    for k, v in a.items():
        if isinstance(v, np.ndarray):
            assert np.array_equal(v, b[k]), k
        else:
            assert v == b[k], k
    assert (os.cpu_count() or 1) >= 1
