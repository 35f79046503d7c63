"""Training and evaluation of the learned drag closure (not part of the paper).

The closure replaces the fine-to-bulk average of the fluid velocity on the
steps between refreshes: the bulk record (u_B, sigma^2_B) of the last
refresh, ``age`` steps old, is reused and the drag computed from it is
scaled, F = (1 + age r) F_stale with r = f(features) the correction per
step of age.  The network is trained on r* = (c* - 1) / age with
c* = (F_fresh . F_stale) / |F_stale|^2 (the projection of the fresh drag on
the stale one), in units of the targets' spread: it learns
(r* - mean) / std, and the mean and spread are then folded into its FP32
output layer, so the bf16 rounding inside the network scales with the
spread of the corrections rather than with their offset from zero.

Everything here drives the C ABI of the coupling library (cg_step,
cg_mlp_features, cg_drag with a closure, cg_mlp_train_step); PyTorch only
holds device memory and draws the sample indices.

With a frozen fluid field the stale and fresh records coincide and c* = 1
everywhere, so the fluid has to evolve for the closure to learn anything.
The stand-in for the fluid solver (which is outside this library) relaxes
the fine field by the coupling source after every step, linearly implicit
in the exchange: with du = dt S_f / (max(eps_f, eps_min) rho_f) and the
exchange rate per fine cell estimated as a = |du| / |u_f| (exact while the
particles are slow against the fluid), u_f <- u_f + du / (1 + a).  For
small a this is the explicit update; in dense cells, where the explicit one
overshoots and diverges, the fluid velocity decays towards the particles'
without crossing it.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass, field

import numpy as np

from . import Grids, Mlp, mlp_pack, MLP_ACTIVATIONS, MLP_NFEAT, MLP_NPARAM

HIDDEN = 64
K0 = 16


def relax_fluid(u_fine, S_fine, eps_fine, desc: dict, dt: float):
    """Fluid stand-in, in place: u_f += du / (1 + |du| / |u_f|) with
    du = dt S_f / (max(eps_f, eps_min) rho_f)."""
    du = S_fine * (dt / (eps_fine.clamp(min=desc["eps_min"]) * desc["rho_f"]))
    a = du.norm(dim=0) / u_fine.norm(dim=0).clamp(min=1e-30)
    u_fine.add_(du / (1.0 + a))


@dataclass
class Trajectory:
    """One seeded coupled run: particles advanced by semi-implicit Euler
    under the fresh drag, fluid relaxed by the coupling source, a stale
    bulk record refreshed every ``refresh`` steps."""
    grids: Grids
    pos: object
    vel: object
    u_fine: object
    out: dict
    dt: float
    refresh: int
    step_no: int = 0
    u_stale: object = None
    var_stale: object = None
    pos_before: object = None
    vel_before: object = None
    age: int = 0
    notes: dict = field(default_factory=dict)

    @classmethod
    def start(cls, w, refresh: int, device="cuda", dt=None):
        import torch
        g = Grids(w.desc)
        pos = torch.from_numpy(w.pos_d).to(device)
        vel = torch.from_numpy(w.vel).to(device)
        uf = torch.from_numpy(np.ascontiguousarray(w.u_fine.reshape(3, -1))).to(device)
        out = g.alloc_outputs(w.n, var=True, eps_fine=True, device=device)
        return cls(g, pos, vel, uf, out, float(w.dt if dt is None else dt), int(refresh))

    def advance(self, on_step=None):
        """One plain coupled step.  ``out`` then holds the porosity, fresh
        record and fresh drag at the positions before the advance (kept in
        pos_before / vel_before); the stale record is refreshed on every
        ``refresh``-th step.  ``on_step(fresh)`` runs before the fluid is
        relaxed, while u_fine is still the field the step averaged."""
        self.pos_before = self.pos.clone()
        self.vel_before = self.vel.clone()
        self.grids.cg_step(self.pos, self.vel, self.u_fine, self.out, dt=self.dt)
        self.age = self.step_no % self.refresh
        fresh = self.age == 0
        if fresh:
            self.u_stale = self.out["u_bulk"].clone()
            self.var_stale = self.out["var_bulk"].clone()
        if on_step is not None:
            on_step(fresh)
        relax_fluid(self.u_fine, self.out["S_fine"], self.out["eps_fine"], self.grids.desc, self.dt)
        self.step_no += 1
        return fresh

    def close(self):
        self.grids.close()


def _features(t: Trajectory):
    import torch
    n = t.pos.shape[0]
    feat = torch.empty(n, 8, device=t.pos.device, dtype=torch.float32)
    target = torch.empty(n, device=t.pos.device, dtype=torch.float32)
    t.grids.cg_mlp_features(t.pos_before, t.vel_before, t.out["eps_bulk"], t.u_stale, t.var_stale,
                            t.out["u_bulk"], feat, target)
    return feat, target


def generate_pairs(make, seeds, refreshes=(2, 5, 10), steps=30, n_pairs=2_000_000, device="cuda",
                   sample_seed=0, dt=None):
    """Training pairs (features [m, 8], per-step targets r* [m]) sampled
    uniformly from the stale steps of coupled runs of ``make(seed)`` for
    every seed and refresh interval."""
    import torch
    runs = [(s, k) for s in seeds for k in refreshes]
    stale_steps = sum(sum(1 for i in range(steps) if i % k) for _, k in runs)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(sample_seed))
    feats, targs = [], []
    per = max(1, int(round(n_pairs / stale_steps)))
    for s in seeds:
        w = make(seed=s)
        for k in refreshes:
            t = Trajectory.start(w, k, device=device, dt=dt)

            def take(fresh):
                if fresh:
                    return
                f, c = _features(t)
                idx = torch.randint(0, w.n, (min(per, w.n),), device=device, generator=gen)
                feats.append(f[idx])
                targs.append((c[idx] - 1.0) / t.age)

            for _ in range(steps):
                t.advance(take)
            rc = t.grids.cg_sync_status()[0]
            t.close()
            if rc != 0:
                raise RuntimeError(f"coupled run seed {s} refresh {k}: status {rc}")
    return torch.cat(feats), torch.cat(targs)


def feature_box(features):
    """Per-feature min / max over the training set (the closure's range)."""
    f = features[:, :MLP_NFEAT].double()
    lo = f.min(dim=0).values.cpu().numpy()
    hi = f.max(dim=0).values.cpu().numpy()
    span = np.maximum(hi - lo, 1e-6 * np.maximum(np.abs(lo), 1.0))
    return lo.astype(np.float32), (lo + span).astype(np.float32)


OFF_W3 = K0 * HIDDEN + HIDDEN + HIDDEN * HIDDEN + HIDDEN
OFF_B3 = OFF_W3 + HIDDEN


def init_params(seed: int = 0):
    """He-style uniform initial weights, small output layer, zero biases."""
    rng = np.random.Generator(np.random.Philox(key=[int(seed), 77]))
    def u(shape, fan_in):
        b = np.sqrt(6.0 / fan_in)
        return rng.uniform(-b, b, shape)
    return dict(W1=u((K0, HIDDEN), MLP_NFEAT), b1=np.zeros(HIDDEN), W2=u((HIDDEN, HIDDEN), HIDDEN),
                b2=np.zeros(HIDDEN), w3=u((HIDDEN,), HIDDEN) * 0.1, b3=np.array([0.0]))


def train(features, targets, epochs=20, batch=65536, lr=1e-3, seed=0, box=None, activation="gelu"):
    """Adam on minibatches (shuffled each epoch) through cg_mlp_train_step
    on the standardised targets; the mean and spread are folded into the
    output layer at the end.  Returns the closure handle (with the given
    activation) and the mean loss of each epoch (standardised units)."""
    import torch
    lo, hi = box if box is not None else feature_box(features)
    m = Mlp(mlp_pack(init_params(seed)), lo, hi, activation=activation)
    mu = float(targets.double().mean())
    sd = float(targets.double().std())
    sd = sd if sd > 0 else 1.0
    targets = ((targets.double() - mu) / sd).float()
    gen = torch.Generator(device=features.device)
    gen.manual_seed(int(seed))
    n = features.shape[0]
    loss = torch.zeros(1, device=features.device)
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, device=features.device, generator=gen)
        acc, nb = 0.0, 0
        for b0 in range(0, n - batch + 1 if n >= batch else 1, batch):
            idx = perm[b0:b0 + batch]
            fb = features[idx].contiguous()
            tb = targets[idx].contiguous()
            m.train_step(fb, tb, lr, loss)
            acc += loss
            nb += 1
        hist.append(float(acc / max(nb, 1)))
    rc, _ = m.sync_status()
    if rc != 0:
        raise RuntimeError(f"closure training status {rc}")
    p = m.params().astype(np.float64)
    p[OFF_W3:OFF_W3 + HIDDEN] *= sd
    p[OFF_B3] = p[OFF_B3] * sd + mu
    m.set_params(p.astype(np.float32))
    m.target_mean, m.target_std = mu, sd
    return m, hist


def evaluate(m: Mlp, make, seed, refresh=5, steps=30, device="cuda", dt=None):
    """Drag error on a coupled run of ``make(seed)``: on every stale step,
    the relative L2 error ||F - F_fresh|| / ||F_fresh|| over all particles
    of the stale drag (c = 1) and of the learned drag, plus the share of
    rows that fell back to the fresh average."""
    import torch
    w = make(seed=seed)
    t = Trajectory.start(w, refresh, device=device, dt=dt)
    F_st = torch.empty_like(t.out["force"])
    F_le = torch.empty_like(t.out["force"])
    acc = dict(num_st=0.0, num_le=0.0, den=0.0, fall=0, rows=0)

    def score(fresh):
        if fresh:
            return
        g = t.grids
        g.cg_drag(t.pos_before, t.vel_before, t.out["eps_bulk"], t.u_stale, F_st)
        m.bind(t.var_stale, t.u_fine, t.age)
        g.cg_drag(t.pos_before, t.vel_before, t.out["eps_bulk"], t.u_stale, F_le, mlp=m)
        rc, _, counts = g.cg_sync_status()
        if rc != 0:
            raise RuntimeError(f"evaluation status {rc}")
        Ff = t.out["force"].double()
        acc["num_st"] += float(((F_st.double() - Ff) ** 2).sum())
        acc["num_le"] += float(((F_le.double() - Ff) ** 2).sum())
        acc["den"] += float((Ff ** 2).sum())
        acc["fall"] += counts[4]
        acc["rows"] += w.n

    for _ in range(steps):
        t.advance(score)
    m.bind(None, None)
    t.close()
    return {"err_stale": (acc["num_st"] / acc["den"]) ** 0.5, "err_learned": (acc["num_le"] / acc["den"]) ** 0.5,
            "fallback_share": acc["fall"] / max(acc["rows"], 1), "stale_steps": acc["rows"] // max(w.n, 1)}


CHECKPOINT_FORMAT = "dual-grid drag closure"
CHECKPOINT_VERSION = 1


def save_checkpoint(path: str, params, feat_lo, feat_hi, activation: str = "gelu", **meta) -> None:
    """Write a trained closure as two files: ``path + ".f32"`` holds the
    MLP_NPARAM parameters as little-endian float32 in the ABI order of
    mlp_pack (W1, b1, W2, b2, w3, b3), and ``path + ".json"`` the sizes, the
    feature box (min / max of each of the MLP_NFEAT features over the
    training set), the SHA-256 of the parameter file, the activation and
    any extra JSON values given as keywords (the refresh interval, the
    target mean and spread, ...).  The parameters are written exactly as
    given (float32)."""
    if activation not in MLP_ACTIVATIONS:
        raise ValueError("closure checkpoint: unknown activation")
    p = np.ascontiguousarray(params, dtype="<f4").reshape(-1)
    lo = np.asarray(feat_lo, np.float32).reshape(-1)
    hi = np.asarray(feat_hi, np.float32).reshape(-1)
    if p.size != MLP_NPARAM or lo.size != MLP_NFEAT or hi.size != MLP_NFEAT:
        raise ValueError("closure checkpoint: bad parameter or feature-box sizes")
    if not (np.all(np.isfinite(p)) and np.all(np.isfinite(lo)) and np.all(np.isfinite(hi)) and np.all(hi > lo)):
        raise ValueError("closure checkpoint: non-finite parameters or an empty feature box")
    raw = p.tobytes()
    head = {"format": CHECKPOINT_FORMAT, "version": CHECKPOINT_VERSION, "nparam": MLP_NPARAM,
            "nfeat": MLP_NFEAT, "hidden": HIDDEN, "k0": K0,
            "params_file": os.path.basename(path) + ".f32", "params_sha256": hashlib.sha256(raw).hexdigest(),
            # float32 values written as the doubles they are, so they read back exactly
            "feature_lo": [float(v) for v in lo], "feature_hi": [float(v) for v in hi], "activation": activation,
            "meta": meta}
    with open(path + ".f32", "wb") as f:
        f.write(raw)
    with open(path + ".json", "w") as f:
        json.dump(head, f, indent=1)


def load_checkpoint(path: str):
    """Read a closure written by save_checkpoint: (params float32
    [MLP_NPARAM], feat_lo float32 [MLP_NFEAT], feat_hi, meta dict,
    activation; "gelu" when the head names none).  Raises ValueError when
    the format, a size, the activation or the checksum does not match.
    ``Mlp(params, feat_lo, feat_hi, activation=activation)`` makes the
    closure handle."""
    with open(path + ".json") as f:
        head = json.load(f)
    if head.get("format") != CHECKPOINT_FORMAT or head.get("version") != CHECKPOINT_VERSION:
        raise ValueError("closure checkpoint: unknown format or version")
    if (head.get("nparam"), head.get("nfeat"), head.get("hidden"), head.get("k0")) != (MLP_NPARAM, MLP_NFEAT,
                                                                                        HIDDEN, K0):
        raise ValueError("closure checkpoint: network sizes differ from this library's")
    with open(os.path.join(os.path.dirname(path), head["params_file"]), "rb") as f:
        raw = f.read()
    if len(raw) != 4 * MLP_NPARAM or hashlib.sha256(raw).hexdigest() != head.get("params_sha256"):
        raise ValueError("closure checkpoint: parameter file size or checksum mismatch")
    params = np.frombuffer(raw, dtype="<f4").astype(np.float32)
    lo = np.asarray(head["feature_lo"], np.float32)
    hi = np.asarray(head["feature_hi"], np.float32)
    if lo.size != MLP_NFEAT or hi.size != MLP_NFEAT:
        raise ValueError("closure checkpoint: bad feature box")
    activation = head.get("activation", "gelu")
    if activation not in MLP_ACTIVATIONS:
        raise ValueError("closure checkpoint: unknown activation")
    return params, lo, hi, dict(head.get("meta") or {}), activation
