"""Pins of the oracle's drag laws, momentum deposit, Euler advance and
whole-step invariants.

The paper fixes only the form F_drag = beta (u_f - u_p) (Eq. DragLaw) and
leaves beta to a cited correlation; the correlations are readings (Di Felice;
Ergun / Wen-Yu in Gidaspow's form).  Every pin below is a textbook limit or
an independent textbook form, not the oracle's expression retyped:
Stokes drag, Dallavalle's single-sphere law and its Stokes limit,
Schiller-Naumann and Newton drag, Ergun's packed-bed pressure-drop equation
written in superficial velocity, the peak of Di Felice's exponent, and
conservation of momentum between particles and the bulk source.
"""
import math

import numpy as np
import pytest

import oracle
import synth

RHO, MU = 1000.0, 1.0e-3


def desc_law(law, **kw):
    return synth.make_desc((0, 0, 0), (1, 1, 1), (8, 8, 8), 2, fp64=True, law=law, **kw)


def force(desc, eps, d, s):
    beta, cl = oracle.drag_beta(desc, eps, d, s)
    return beta * np.asarray(s, dtype=float), cl


def slip_for_re(re, eps, d, with_eps=True):
    return re * MU / (RHO * (eps if with_eps else 1.0) * d)


# ---------------------------------------------------------------- Di Felice
def test_difelice_zero_slip_is_zero_force():
    desc = desc_law(0)
    F, _ = force(desc, 0.6, 0.003, [0.0, 0.0, 0.0])
    assert np.all(F == 0.0)


def test_difelice_stokes_limit_dallavalle():
    """Re -> 0: C_D0 -> 4.8^2 / Re, so F -> 2.88 pi mu d s eps^(1 - 3.7)."""
    desc = desc_law(0)
    d = 0.002
    for eps in (1.0, 0.7, 0.45):
        s = np.array([1e-13, -2e-13, 0.5e-13])
        F, _ = force(desc, eps, d, s)
        want = 2.88 * math.pi * MU * d * eps ** (1.0 - 3.7) * s
        assert np.allclose(F, want, rtol=5e-5)


def test_difelice_single_sphere_dallavalle():
    """eps = 1: F = 1/2 C_D rho (pi d^2/4) |s| s with C_D = (0.63 + 4.8 / sqrt(Re))^2."""
    desc = desc_law(0)
    d = 0.004
    for re in (0.1, 1.0, 10.0, 100.0, 1000.0):
        sm = slip_for_re(re, 1.0, d)
        s = sm * np.array([0.6, 0.0, 0.8])
        F, _ = force(desc, 1.0, d, s)
        cd = (0.63 + 4.8 / math.sqrt(re)) ** 2
        want = 0.5 * cd * RHO * (math.pi * d * d / 4.0) * sm * s
        assert np.allclose(F, want, rtol=1e-12)
    # Newton-like limit of the Dallavalle law: C_D -> 0.63^2
    sm = slip_for_re(1e12, 1.0, d)
    F, _ = force(desc, 1.0, d, [sm, 0, 0])
    cd = F[0] / (0.5 * RHO * math.pi * d * d / 4.0 * sm * sm)
    assert cd == pytest.approx(0.63 ** 2, rel=1e-4)


def test_difelice_exponent_peak_is_3_05():
    """At Re = 10^1.5 the exponent chi = 3.7 - 0.65 = 3.05.  With Re held
    fixed (slip scaled by 1/eps), F(eps)/F(1) = eps^(2 - chi) eps^(-2)."""
    desc = desc_law(0)
    d = 0.003
    re = 10.0 ** 1.5
    F1, _ = force(desc, 1.0, d, [slip_for_re(re, 1.0, d), 0, 0])
    for eps in (0.3, 0.5, 0.8):
        Fe, _ = force(desc, eps, d, [slip_for_re(re, eps, d), 0, 0])
        chi = -math.log(Fe[0] / F1[0]) / math.log(eps)
        assert chi == pytest.approx(3.05, abs=1e-12)
    # away from the peak chi is larger, approaching 3.7 at both ends
    for re2, lo in ((1e-6, 3.69), (1e7, 3.69)):
        F1, _ = force(desc, 1.0, d, [slip_for_re(re2, 1.0, d), 0, 0])
        Fe, _ = force(desc, 0.5, d, [slip_for_re(re2, 0.5, d), 0, 0])
        chi = -math.log(Fe[0] / F1[0]) / math.log(0.5)
        assert lo < chi <= 3.7 + 1e-12


def test_difelice_odd_and_parallel():
    desc = desc_law(0)
    s = np.array([0.03, -0.02, 0.05])
    Fp, _ = force(desc, 0.55, 0.002, s)
    Fm, _ = force(desc, 0.55, 0.002, -s)
    assert np.allclose(Fm, -Fp, rtol=0, atol=0)
    assert np.allclose(np.cross(Fp, s), 0.0, atol=1e-20)
    assert np.dot(Fp, s) > 0


# ------------------------------------------------------------ Ergun / Wen-Yu
def test_wenyu_stokes_limit():
    """eps = 1, Re -> 0: F = 3 pi mu d s exactly (Stokes)."""
    desc = desc_law(1)
    d = 0.004
    s = np.array([1e-12, 2e-12, -1e-12])
    F, _ = force(desc, 1.0, d, s)
    assert np.allclose(F, 3.0 * math.pi * MU * d * s, rtol=1e-6)


def test_wenyu_single_sphere_schiller_naumann_and_newton():
    desc = desc_law(1)
    d = 0.004
    A = math.pi * d * d / 4.0
    for re in (0.5, 5.0, 50.0, 500.0, 999.0):
        sm = slip_for_re(re, 1.0, d, with_eps=False)
        F, _ = force(desc, 1.0, d, [0, 0, sm])
        cd = 24.0 / re * (1.0 + 0.15 * re ** 0.687)
        assert F[2] == pytest.approx(0.5 * cd * RHO * A * sm * sm, rel=1e-12)
    for re in (1000.0, 5000.0):
        sm = slip_for_re(re, 1.0, d, with_eps=False)
        F, _ = force(desc, 1.0, d, [0, 0, sm])
        assert F[2] == pytest.approx(0.5 * 0.44 * RHO * A * sm * sm, rel=1e-12)


def test_wenyu_is_interstitial_single_sphere_times_eps_power():
    """In a suspension (eps >= switch) Wen-Yu is the single-sphere drag at the
    interstitial Reynolds number eps Re, times eps^(1 - 2.65)."""
    desc = desc_law(1)
    d = 0.003
    A = math.pi * d * d / 4.0
    for eps in (0.8, 0.9, 0.97):
        for sm in (1e-3, 0.05, 1.0):
            F, _ = force(desc, eps, d, [sm, 0, 0])
            rei = eps * RHO * d * sm / MU
            cd = 24.0 / rei * (1.0 + 0.15 * rei ** 0.687) if rei < 1000 else 0.44
            want = 0.5 * cd * RHO * A * sm * sm * eps ** (1.0 - 2.65)
            assert F[0] == pytest.approx(want, rel=1e-12)


def test_ergun_matches_packed_bed_pressure_drop():
    """Ergun's equation for a packed bed in superficial velocity U = eps |s|:
    dP/L = 150 mu (1-eps)^2 U / (eps^3 d^2) + 1.75 (1-eps) rho U^2 / (eps^3 d).
    The fluid force balance eps dP/L = n F with n = (1-eps)/V_p particles per
    unit volume must hold for the per-particle force."""
    desc = desc_law(1)
    d = 0.004
    vp = 4.0 / 3.0 * math.pi * (d / 2) ** 3
    for eps in (0.35, 0.45, 0.6, 0.79):
        for sm in (1e-4, 0.01, 0.5, 2.0):
            F, _ = force(desc, eps, d, [0, sm, 0])
            U = eps * sm
            dpdl = (150.0 * MU * (1 - eps) ** 2 * U / (eps ** 3 * d * d)
                    + 1.75 * (1 - eps) * RHO * U * U / (eps ** 3 * d))
            n = (1 - eps) / vp
            assert n * F[1] == pytest.approx(eps * dpdl, rel=1e-12)


def test_switch_tie_and_clamp():
    desc = desc_law(1, eps_switch=0.8, eps_min=0.1)
    d = 0.004
    s = [0.0, 0.0, 0.3]
    # exactly at the switch porosity the dilute (Wen-Yu) branch is taken
    Fw, _ = force(desc, 0.8, d, s)
    rei = 0.8 * RHO * d * 0.3 / MU
    cd = 24.0 / rei * (1.0 + 0.15 * rei ** 0.687) if rei < 1000 else 0.44
    want = 0.5 * cd * RHO * math.pi * d * d / 4 * 0.3 * 0.3 * 0.8 ** (1 - 2.65)
    assert Fw[2] == pytest.approx(want, rel=1e-12)
    # porosity below eps_min acts as eps_min and is reported
    Fa, cla = force(desc, 0.05, d, s)
    Fb, clb = force(desc, 0.1, d, s)
    assert cla and not clb and np.array_equal(Fa, Fb)


# ----------------------------------------------------- drag at the particles
def test_drag_uniform_fields_and_zero_slip():
    desc = desc_law(0)
    nb = 4 ** 3
    eps_b = np.full(nb, 0.7)
    ub = np.zeros((3, nb))
    ub[0] = 0.2
    ub[2] = -0.1
    rng = np.random.default_rng(1)
    n = 50
    pos = np.zeros((n, 4))
    pos[:, :3] = rng.random((n, 3))
    pos[:, 3] = 0.002
    vel = np.zeros((n, 4))
    vel[:, 0] = 0.2
    vel[:, 2] = -0.1
    F, _ = oracle.drag(desc, pos, vel, eps_b, ub)
    # the interpolated constant carries one rounding: slip is at most a few ulps
    beta, _ = oracle.drag_beta(desc, 0.7, 0.002, [1e-16, 0, 0])
    assert np.all(np.abs(F) <= beta * 1e-16)
    vel[:, 0] = 0.0
    F, _ = oracle.drag(desc, pos, vel, eps_b, ub)
    want, _ = force(desc, 0.7, 0.002, [0.2, 0.0, 0.0])
    assert np.allclose(F[:, 0], want, rtol=1e-14)


# ------------------------------------------------ momentum deposit (Eq. UFP)
def test_momentum_deposit_brute_force_and_conservation():
    w = synth.tiny(seed=2, n=4000)
    desc = w.desc
    cell, perm, cs, _ = oracle.bin(desc, w.pos_d)
    rng = np.random.default_rng(0)
    F = rng.normal(size=(3, w.n))
    S = oracle.deposit_momentum(desc, F, cs, perm)
    nb = [v // desc["ratio"] for v in desc["fine_n"]]
    VB = np.prod(np.array(desc["extent"]) / np.array(nb))
    want = np.zeros_like(S)
    for c in range(3):
        np.add.at(want[c], cell, F[c])
    want *= -1.0 / VB
    assert np.allclose(S, want, rtol=1e-12, atol=1e-12)
    tot = F.sum(axis=1) + S.sum(axis=1) * VB
    assert np.all(np.abs(tot) <= 1e-12 * np.abs(F).sum(axis=1))


# ------------------------------------------------ Euler (Eq. DEM_EQUATIONS)
def test_euler_gravity_closed_form_velocity_first():
    """With F = 0 and gravity g, velocity-first Euler gives
    u_n = g n dt and x_n = x_0 + g dt^2 n (n + 1) / 2."""
    desc = synth.make_desc((0, 0, 0), (1, 1, 1), (8, 8, 8), 2, fp64=True, law=0,
                           gravity=(0.0, 0.0, -9.81))
    pos = np.array([[0.5, 0.5, 0.9, 0.002]])
    vel = np.zeros((1, 4))
    F = np.zeros((3, 1))
    dt = 1e-3
    nsteps = 20
    for _ in range(nsteps):
        pos, vel = oracle.euler(desc, pos, vel, F, dt)
    assert vel[0, 2] == pytest.approx(-9.81 * nsteps * dt, rel=1e-12)
    assert pos[0, 2] == pytest.approx(0.9 - 9.81 * dt * dt * nsteps * (nsteps + 1) / 2, rel=1e-12)


def test_euler_specular_walls():
    desc = synth.make_desc((0, 0, 0), (1, 1, 1), (8, 8, 8), 2, fp64=True, law=0)
    pos = np.array([[0.999, 0.001, 0.5, 0.002]])
    vel = np.array([[2.0, -3.0, 0.0, 0.0]])
    pos2, vel2 = oracle.euler(desc, pos, vel, np.zeros((3, 1)), 1e-3)
    assert pos2[0, 0] == pytest.approx(2.0 - 1.001) and vel2[0, 0] == -2.0
    assert pos2[0, 1] == pytest.approx(0.002) and vel2[0, 1] == 3.0


def test_euler_stokes_relaxation_single_particle():
    """One particle at rest in a uniform flow, eps = 1, no gravity, Stokes
    regime: the discrete velocity relaxes as u_f (1 - (1 - dt/tau)^n) with
    tau = m / (3 pi mu d), and stays within O(dt/tau) of u_f (1 - exp(-t/tau))."""
    desc = synth.make_desc((0, 0, 0), (1, 1, 1), (8, 8, 8), 2, fp64=True, law=1)
    d = 1e-5
    m = 2500.0 * math.pi * d ** 3 / 6.0
    tau = m / (3 * math.pi * MU * d)
    dt = tau / 50
    nb = 4 ** 3
    eps_b = np.ones(nb)
    ub = np.zeros((3, nb))
    ub[0] = 1e-7   # Re = 1e-6: the 0.15 Re^0.687 correction is 1e-5
    pos = np.array([[0.5, 0.5, 0.5, d]])
    vel = np.zeros((1, 4))
    for k in range(1, 101):
        F, _ = oracle.drag(desc, pos, vel, eps_b, ub)
        pos, vel = oracle.euler(desc, pos, vel, F, dt)
        disc = 1e-7 * (1 - (1 - dt / tau) ** k)
        cont = 1e-7 * (1 - math.exp(-k * dt / tau))
        assert vel[0, 0] == pytest.approx(disc, rel=1e-4)
        assert abs(vel[0, 0] - cont) < 1e-7 * dt / tau


# ------------------------------------------------------ whole-step invariants
@pytest.mark.parametrize("make", [synth.tiny, synth.small_packed_bed])
def test_step_conservation_invariants(make):
    w = make()
    o = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, want_eps_fine=True)
    s = o["sums"]
    assert s[1] == pytest.approx(s[0], rel=1e-13)
    scale = s[11]
    assert np.all(np.abs(s[2:5] + s[5:8]) <= 1e-12 * scale)
    assert np.all(np.abs(s[5:8] - s[8:11]) <= 1e-12 * scale)
    assert o["outside"] == 0
    assert np.all(o["eps_fine"] <= 1.0 + 1e-15)


def test_one_particle_sweep_is_continuous_across_bulk_faces():
    """Continuity across cell boundaries (the paper's one-particle check,
    Sec. 3.1, made a sweep): a particle moved along a line through fixed bulk
    fields crosses interior bulk faces and the outer half cells; the
    interpolated porosity and fluid velocity, and with them the Di Felice
    drag, change continuously.  Halving the step halves the largest change
    between neighbouring positions; a jump at a face would not shrink.  The
    particle's own deposit moves wholly from one cell to the next at each
    face (NGP), and its total stays V_p."""
    desc = synth.make_desc((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (8, 8, 8), 2, fp64=True, law=0)
    rng = np.random.default_rng(5)
    bg = np.zeros((400, 4))
    bg[:, :3] = rng.random((400, 3))
    bg[:, 3] = 0.04
    _, perm, cs, _ = oracle.bin(desc, bg)
    eps, _ = oracle.deposit_volume(desc, bg, cs, perm)
    u_fine = rng.normal(0.0, 0.2, (3, 8, 8, 8))
    u_bulk, _ = oracle.average(desc, u_fine)

    def largest_change(m, d):
        pos = np.zeros((m, 4))
        pos[:, 0], pos[:, 1], pos[:, 2], pos[:, 3] = np.linspace(0.01, 0.99, m), 0.37, 0.61, 0.01
        vel = np.zeros((m, 4))
        vel[:, :3] = [0.05, -0.02, 0.01]
        F, _ = oracle.drag(d, pos, vel, eps, u_bulk)
        return np.max(np.linalg.norm(np.diff(F, axis=1), axis=0))

    j1, j2 = largest_change(1001, desc), largest_change(2001, desc)
    assert j1 > 0 and j2 <= 0.6 * j1, (j1, j2)
    # the criterion sees a jump: the cell-value gather (Sec. 1's other option)
    # is discontinuous at the faces, and there halving the step changes nothing
    cell = dict(desc, interp=1)
    assert largest_change(2001, cell) >= 0.9 * largest_change(1001, cell)
    # the moving particle's own deposit: one cell at a time, all of V_p
    vp = math.pi * 0.01 ** 3 / 6.0
    H = 0.25
    for x in (0.2499999, 0.25, 0.2500001, 0.7499999, 0.75):
        p = np.array([[x, 0.37, 0.61, 0.01]])
        _, pm, c, _ = oracle.bin(desc, p)
        e, _ = oracle.deposit_volume(desc, p, c, pm)
        phi = 1.0 - e
        assert np.count_nonzero(phi) == 1 and phi.sum() * H ** 3 == pytest.approx(vp, rel=1e-12)
        assert int(np.argmax(phi)) % 4 == int(math.floor(x / H))


def test_step_is_invariant_under_particle_renumbering():
    """The paper finds the coupled results identical whatever the
    decomposition (Sec. 3.1); here, whatever the particle numbering: a step
    on the particles in another order gives each particle the same cell and
    force, each cell the same particles, and the same fields, to the
    rounding of the compensated per-cell sums taken in another order."""
    w = synth.small_packed_bed(seed=3, fp64=True)
    a = oracle.step(w.desc, w.pos_d, w.vel, w.u_fine, dt=1e-4, want_eps_fine=True)
    p = np.random.default_rng(11).permutation(w.n)
    b = oracle.step(w.desc, w.pos_d[p], w.vel[p], w.u_fine, dt=1e-4, want_eps_fine=True)
    assert np.array_equal(b["cell"], a["cell"][p])
    assert np.array_equal(b["cell_start"], a["cell_start"])
    for c in np.random.default_rng(12).choice(len(a["cell_start"]) - 1, 200, replace=False):
        s0, s1 = a["cell_start"][c], a["cell_start"][c + 1]
        assert sorted(a["perm"][s0:s1]) == sorted(p[b["perm"][s0:s1]]), c
    assert np.all(np.diff(b["perm"][b["cell_start"][5]:b["cell_start"][6]]) > 0)   # still stable
    for k in ("eps_bulk", "u_bulk", "var_bulk", "S_bulk", "S_fine", "eps_fine"):
        x, y = a[k], b[k]
        assert np.allclose(y, x, rtol=1e-13, atol=1e-13 * np.max(np.abs(x))), k
    F = a["force"]
    assert np.allclose(b["force"], F[:, p], rtol=1e-12, atol=1e-13 * np.max(np.abs(F)))
    assert np.allclose(b["pos_d"], a["pos_d"][p], rtol=0, atol=1e-15)
    assert np.allclose(b["vel"], a["vel"][p], rtol=1e-12, atol=1e-15)
