"""Pins of the oracle's semi-implicit exchange coefficients (Eq. UFP: the
fluid-particle force F_fpi, the fluid-side reaction to F_drag, is treated
semi-implicitly): A_B = sum beta_p / V_B and b_B = sum beta_p u_p / V_B, so
the fluid solver takes F_fpi = -A u_f + b.

The pins tie the coefficients to quantities computed another way, not to
their own formula: in a uniform fluid field the explicit bulk source of the
momentum deposit must equal -(A u_f - b) cell by cell; the volume-weighted
sum of A must equal the sum of the per-particle drag factors obtained one
particle at a time; one particle gives A = beta / V_B in its own cell only;
particles at rest give b = 0 exactly, and b scales with the particle
velocity when the drag factor does not change (Stokes regime, Di Felice
at vanishing Reynolds number is not linear, so Ergun's viscous term is used).
"""
import numpy as np

import oracle
import synth


def setup(law=0, n=3000, seed=3, vel_scale=0.05):
    w = synth.tiny(seed=seed, n=n, fine=16, ratio=2)
    d = dict(w.desc)
    d["law"] = law
    cell, perm, cs, _ = oracle.bin(d, w.pos_d)
    eps, _ = oracle.deposit_volume(d, w.pos_d, cs, perm)
    nf, nb = oracle.dims(d)
    nbulk = nb[0] * nb[1] * nb[2]
    vel = w.vel.copy()
    vel[:, :3] *= vel_scale / 0.05
    return d, w.pos_d, vel, eps, cs, perm, nbulk


def uniform_u(nbulk, u=(0.3, -0.2, 0.5)):
    return np.tile(np.asarray(u, dtype=float)[:, None], (1, nbulk))


def test_uniform_field_source_equals_implicit_split():
    for law in (0, 1):
        d, pos, vel, eps, cs, perm, nbulk = setup(law=law)
        u = uniform_u(nbulk)
        A, b = oracle.implicit(d, pos, vel, eps, u, cs, perm)
        F, _ = oracle.drag(d, pos, vel, eps, u)
        S = oracle.deposit_momentum(d, F, cs, perm)
        split = -(A[None, :] * u - b)
        scale = np.max(np.abs(S)) + 1e-300
        assert np.max(np.abs(S - split)) <= 1e-12 * scale, law
        assert np.count_nonzero(A) > nbulk // 2


def test_volume_weighted_sum_equals_particle_factors():
    d, pos, vel, eps, cs, perm, nbulk = setup(law=1, n=600)
    u = uniform_u(nbulk, (0.1, 0.0, 0.4))
    A, b = oracle.implicit(d, pos, vel, eps, u, cs, perm)
    VB = np.prod(np.asarray(d["extent"]) / (np.asarray(d["fine_n"]) // d["ratio"]))
    betas = []
    for p in range(pos.shape[0]):
        x = pos[p, :3].astype(float)
        e = oracle.gather(d, eps, x)[0]
        uf = oracle.gather(d, u, x)
        beta, _ = oracle.drag_beta(d, e, float(pos[p, 3]), uf - vel[p, :3])
        betas.append(beta)
    betas = np.asarray(betas)
    assert abs(np.sum(A) * VB - betas.sum()) <= 1e-12 * betas.sum()
    bsum = (betas[:, None] * vel[:, :3]).sum(axis=0)
    assert np.allclose(b.sum(axis=1) * VB, bsum, rtol=1e-12, atol=1e-12 * np.abs(bsum).max())


def test_one_particle_and_particles_at_rest():
    d, pos, vel, eps, cs, perm, nbulk = setup(law=0, n=1)
    u = uniform_u(nbulk)
    A, b = oracle.implicit(d, pos, vel, eps, u, cs, perm)
    c = oracle.bin(d, pos)[0][0]
    VB = np.prod(np.asarray(d["extent"]) / (np.asarray(d["fine_n"]) // d["ratio"]))
    e = oracle.gather(d, eps, pos[0, :3].astype(float))[0]
    beta, _ = oracle.drag_beta(d, e, float(pos[0, 3]), u[:, 0] - vel[0, :3])
    assert np.count_nonzero(A) == 1 and A[c] == beta / VB
    assert np.allclose(b[:, c], A[c] * vel[0, :3], rtol=1e-15)
    d, pos, vel, eps, cs, perm, nbulk = setup(law=1, n=500)
    vel[:, :3] = 0.0
    A, b = oracle.implicit(d, pos, vel, eps, uniform_u(nbulk), cs, perm)
    assert np.all(b == 0.0) and np.all(A >= 0.0)


def test_b_is_linear_in_particle_velocity_in_the_viscous_regime():
    # Ergun's viscous term dominates at vanishing slip (here its inertial term
    # is ~1e-8 of it): beta barely depends on |s|, so b follows u_p linearly
    # while A stays put.
    d, pos, vel, eps, cs, perm, nbulk = setup(law=1, n=800, vel_scale=1e-14)
    d = dict(d)
    d["eps_switch"] = 1.0          # Ergun everywhere
    u = uniform_u(nbulk, (0.0, 0.0, 0.0))
    A1, b1 = oracle.implicit(d, pos, vel, eps, u, cs, perm)
    v2 = vel.copy()
    v2[:, :3] *= 2.0
    A2, b2 = oracle.implicit(d, pos, v2, eps, u, cs, perm)
    assert np.allclose(A2, A1, rtol=1e-6)
    assert np.allclose(b2, 2.0 * b1, rtol=1e-6, atol=1e-6 * np.abs(b1).max())


def test_uniform_field_identity_over_random_cases():
    """The uniform-field identity for random particle sets, laws, fluid
    velocities and particle speeds (property-based)."""
    import pytest
    hypothesis = pytest.importorskip("hypothesis")
    st = hypothesis.strategies

    @hypothesis.settings(max_examples=25, deadline=None)
    @hypothesis.given(st.integers(0, 2), st.integers(1, 800), st.sampled_from([0, 1]),
                      st.floats(1e-6, 2.0), st.lists(st.floats(-1.0, 1.0), min_size=3, max_size=3))
    def check(seed, n, law, vscale, uf):
        d, pos, vel, eps, cs, perm, nbulk = setup(law=law, n=n, seed=seed, vel_scale=vscale)
        u = uniform_u(nbulk, uf)
        A, b = oracle.implicit(d, pos, vel, eps, u, cs, perm)
        F, _ = oracle.drag(d, pos, vel, eps, u)
        S = oracle.deposit_momentum(d, F, cs, perm)
        split = -(A[None, :] * u - b)
        scale = np.max(np.abs(S)) + np.max(np.abs(b)) + 1e-300
        assert np.max(np.abs(S - split)) <= 1e-11 * scale
        assert np.all(A >= 0.0)

    check()
