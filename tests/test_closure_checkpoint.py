"""The trained closure's checkpoint (parameters as raw float32 beside a JSON
head with the feature box and a checksum) reads back bit for bit and
refuses files that do not match."""
import json

import numpy as np
import pytest

from paper_1807_11834_gb300 import MLP_NFEAT, MLP_NPARAM, mlp_pack, mlp_unpack
from paper_1807_11834_gb300 import closure


def _closure(seed=3):
    rng = np.random.default_rng(seed)
    p = rng.normal(size=MLP_NPARAM).astype(np.float32)
    lo = rng.uniform(-2, 0, MLP_NFEAT).astype(np.float32)
    hi = lo + rng.uniform(0.1, 3, MLP_NFEAT).astype(np.float32)
    return p, lo, hi


def test_round_trip_is_bit_exact(tmp_path):
    p, lo, hi = _closure()
    base = str(tmp_path / "closure")
    closure.save_checkpoint(base, p, lo, hi, refresh=10, target_mean=0.01, target_std=0.2)
    q, lo2, hi2, meta = closure.load_checkpoint(base)
    assert q.dtype == np.float32 and q.tobytes() == p.tobytes()
    assert lo2.tobytes() == lo.tobytes() and hi2.tobytes() == hi.tobytes()
    assert meta == {"refresh": 10, "target_mean": 0.01, "target_std": 0.2}
    # the ABI order: unpacking the read-back parameters gives the packed blocks
    blocks = mlp_unpack(q)
    assert np.array_equal(mlp_pack(blocks), q.astype(np.float64))
    head = json.load(open(base + ".json"))
    assert head["nparam"] == MLP_NPARAM and head["params_file"] == "closure.f32"
    assert (tmp_path / "closure.f32").stat().st_size == 4 * MLP_NPARAM


def test_mismatches_are_refused(tmp_path):
    p, lo, hi = _closure()
    base = str(tmp_path / "c")
    with pytest.raises(ValueError):
        closure.save_checkpoint(base, p[:-1], lo, hi)
    with pytest.raises(ValueError):
        closure.save_checkpoint(base, p, hi, lo)          # empty feature box
    bad = p.copy()
    bad[5] = np.nan
    with pytest.raises(ValueError):
        closure.save_checkpoint(base, bad, lo, hi)
    closure.save_checkpoint(base, p, lo, hi)
    raw = bytearray(open(base + ".f32", "rb").read())
    raw[100] ^= 1                                          # one flipped bit
    open(base + ".f32", "wb").write(bytes(raw))
    with pytest.raises(ValueError):
        closure.load_checkpoint(base)
    closure.save_checkpoint(base, p, lo, hi)
    head = json.load(open(base + ".json"))
    head["hidden"] = 32
    json.dump(head, open(base + ".json", "w"))
    with pytest.raises(ValueError):
        closure.load_checkpoint(base)
