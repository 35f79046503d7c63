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


def assert_close_interp(name, got, ref, ref_abs, tol):
    """Interpolated field ([3][m] or [m]): the error of each cell within tol
    of max(|ref|, |interpolant of the absolute corner values| (ref_abs),
    1e-3 max|ref|), Euclidean norms per cell.  An FP32 lerp between values
    of opposite sign rounds relative to the corner magnitudes, not to the
    (possibly near-zero) result."""
    got = np.atleast_2d(np.asarray(got, np.float64))
    ref = np.atleast_2d(np.asarray(ref, np.float64))
    ref_abs = np.atleast_2d(np.asarray(ref_abs, np.float64))
    num = np.sqrt(((got - ref) ** 2).sum(axis=0))
    den = np.maximum(np.sqrt((ref ** 2).sum(axis=0)), np.sqrt((ref_abs ** 2).sum(axis=0)))
    den = np.maximum(den, max(1e-3 * den.max(), 1e-300))
    r = num / den
    assert r.max() <= tol, f"{name}: max rel err {r.max():.3e} > {tol:.1e}"
    return float(r.max())


def to_dev(a, dev="cuda:0"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def to_np(t):
    return None if t is None else t.detach().cpu().numpy()


def inputs(w, dev="cuda:0"):
    """pos_d, vel, u_fine (flattened [3][n_f]) as device tensors."""
    return to_dev(w.pos_d, dev), to_dev(w.vel, dev), to_dev(w.u_fine.reshape(3, -1), dev)


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
