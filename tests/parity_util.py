"""Helpers shared by the GPU parity tests: the error metric and tensor
marshalling.  The metric is the per-cell / per-particle relative error
with the denominator max(|ref|, 1e-3 max|ref|) per field; vector fields
([3][n] arrays) use the Euclidean norm per cell or particle."""
import numpy as np

TOL_FP64 = 1e-12
TOL_FP32 = 2e-6


def rel_err(got, ref, vec=False, mask=None):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if vec:
        num = np.sqrt(((got - ref) ** 2).sum(axis=0))
        den = np.sqrt((ref ** 2).sum(axis=0))
    else:
        num = np.abs(got - ref)
        den = np.abs(ref)
    if mask is not None:
        num, den = num[mask], den[mask]
    if den.size == 0:
        return 0.0, 0.0
    floor = 1e-3 * den.max()
    r = num / np.maximum(den, max(floor, 1e-300))
    return float(r.max()), float(np.quantile(r, 0.9999))


def assert_close(name, got, ref, tol, vec=False, mask=None):
    mx, q = rel_err(got, ref, vec=vec, mask=mask)
    assert mx <= tol, f"{name}: max rel err {mx:.3e} (p99.99 {q:.3e}) > {tol:.1e}"
    return mx


def interp_errors(got, ref, ref_abs, mask=None):
    """Per-cell errors of an interpolated field ([3][m] or [m]) under the two
    denominators: (plain, widened).  plain is the metric of rel_err
    (max(|ref|, 1e-3 max|ref|)); widened also takes |interpolant of the
    absolute corner values| (ref_abs).  Euclidean norms per cell; mask
    (nullable, [m] bool) keeps the cells compared."""
    got = np.atleast_2d(np.asarray(got, np.float64))
    ref = np.atleast_2d(np.asarray(ref, np.float64))
    ref_abs = np.atleast_2d(np.asarray(ref_abs, np.float64))
    if mask is not None:
        got, ref, ref_abs = got[:, mask], ref[:, mask], ref_abs[:, mask]
    if ref.shape[1] == 0:
        return np.zeros(0), np.zeros(0)
    num = np.sqrt(((got - ref) ** 2).sum(axis=0))
    den_ref = np.sqrt((ref ** 2).sum(axis=0))
    den_w = np.maximum(den_ref, np.sqrt((ref_abs ** 2).sum(axis=0)))
    plain = num / np.maximum(den_ref, max(1e-3 * den_ref.max(), 1e-300))
    widened = num / np.maximum(den_w, max(1e-3 * den_w.max(), 1e-300))
    return plain, widened


def assert_close_interp(name, got, ref, ref_abs, tol, mask=None, report=None):
    """Interpolated field ([3][m] or [m]): the error of each cell within tol
    of max(|ref|, |interpolant of the absolute corner values| (ref_abs),
    1e-3 max|ref|), Euclidean norms per cell.  An FP32 lerp between values
    of opposite sign rounds relative to the corner magnitudes, not to the
    (possibly near-zero) result.  report (nullable dict) receives both
    metrics' maxima and the number of cells that pass only under the
    widened denominator, so that the widening is seen not to hide error."""
    plain, widened = interp_errors(got, ref, ref_abs, mask)
    if plain.size == 0:
        return 0.0
    if report is not None:
        report[name] = {"max_widened": float(widened.max()), "max_plain": float(plain.max()),
                        "cells_only_widened": int(((plain > tol) & (widened <= tol)).sum()),
                        "cells": int(plain.size)}
    assert widened.max() <= tol, f"{name}: max rel err {widened.max():.3e} > {tol:.1e}"
    return float(widened.max())


def assert_close_slip(name, got, ref, slip, u_p, tol, report=None):
    """Drag forces ([3][n]) of particles that move: F = beta s with the slip
    s = u_f - u_p, and where u_p is close to u_f the subtraction cancels, so
    an FP32 rounding of the interpolated u_f is relative to |u_f| + |u_p|,
    not to |s|.  The error of each particle is taken within tol of
    max(|F|, |F| (|s| + 2 |u_p|) / |s|, 1e-3 max|F|) (|s| + 2 |u_p| bounds
    |u_f| + |u_p|); report (nullable dict) gets the maxima of this metric and
    of the plain one, and the particles that pass only under this one."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    num = np.sqrt(((got - ref) ** 2).sum(axis=0))
    fm = np.sqrt((ref ** 2).sum(axis=0))
    slip = np.asarray(slip, np.float64)
    up = np.sqrt((np.asarray(u_p, np.float64) ** 2).sum(axis=1))
    amp = np.where(slip > 0, (slip + 2 * up) / np.maximum(slip, 1e-300), 1.0)
    floor = max(1e-3 * fm.max(), 1e-300)
    plain = num / np.maximum(fm, floor)
    terms = num / np.maximum(fm * amp, floor)
    if report is not None:
        report[name] = {"max_terms": float(terms.max()), "max_plain": float(plain.max()),
                        "particles_only_terms": int(((plain > tol) & (terms <= tol)).sum())}
    assert terms.max() <= tol, f"{name}: max rel err {terms.max():.3e} > {tol:.1e}"
    return float(terms.max())


def to_dev(a, dev="cuda:0"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def to_np(t):
    return None if t is None else t.detach().cpu().numpy()


def inputs(w, dev="cuda:0"):
    """pos_d, vel, u_fine (flattened [3][n_f]) as device tensors."""
    return to_dev(w.pos_d, dev), to_dev(w.vel, dev), to_dev(w.u_fine.reshape(3, -1), dev)


def switch_exclusions(w, ref, mask):
    """The cells whose values depend on a particle excluded by mask (near a
    correlation switch): bulk cells holding one (their reaction sums its
    force) and fine cells whose projection stencil reads such a bulk cell
    (the oracle's projection of the cells' indicator is non-zero there).
    Returns (bulk cells kept, fine cells kept) as bool arrays."""
    import oracle
    nb = np.asarray(ref["eps_bulk"]).shape[0]
    bad = np.zeros(nb, bool)
    bad[np.asarray(ref["cell"])[~mask]] = True
    fine_bad = oracle.project(w.desc, bad.astype(np.float64)) > 0
    return ~bad, ~fine_bad


def switch_mask(w, ref):
    """Particles away from the correlation branch points (FP32 vs FP64 may
    legitimately take different branches within rounding of the switch)."""
    import oracle
    desc = w.desc
    if desc["law"] != 1:
        return np.ones(w.n, bool)
    eps_p, slip = oracle.particle_state(desc, w.pos_d, w.vel, ref["eps_bulk"], ref["u_bulk"])
    eps_c = np.maximum(eps_p, desc["eps_min"])
    ere = eps_c * desc["rho_f"] * w.pos_d[:, 3].astype(np.float64) * slip / desc["mu_f"]
    near = (np.abs(eps_c - desc["eps_switch"]) < 1e-5) | (np.abs(ere - 1000.0) < 1e-2)
    return ~near
