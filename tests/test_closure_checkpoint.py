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


# ---------------------------------------------- the C ABI's checkpoint calls
def test_c_abi_writes_what_python_reads_bit_exact(tmp_path):
    """cg_mlp_checkpoint_write (C: FIPS 180-4 SHA-256, its own JSON) gives
    files that the Python reader (hashlib, json) takes back bit for bit,
    with the caller's meta object."""
    import paper_1807_11834_gb300 as cg
    p, lo, hi = _closure(7)
    base = str(tmp_path / "c_written")
    cg.checkpoint_write(base, p, lo, hi, meta={"refresh": 5, "note": "a \"quoted\" word"})
    q, lo2, hi2, meta = closure.load_checkpoint(base)
    assert q.tobytes() == p.tobytes() and lo2.tobytes() == lo.tobytes() and hi2.tobytes() == hi.tobytes()
    assert meta == {"refresh": 5, "note": "a \"quoted\" word"}
    import hashlib
    raw = open(base + ".f32", "rb").read()
    assert json.load(open(base + ".json"))["params_sha256"] == hashlib.sha256(raw).hexdigest()


def test_c_abi_reads_what_python_writes_bit_exact(tmp_path):
    import paper_1807_11834_gb300 as cg
    p, lo, hi = _closure(8)
    base = str(tmp_path / "py_written")
    closure.save_checkpoint(base, p, lo, hi, refresh=20, target_mean=0.0)
    q, lo2, hi2 = cg.checkpoint_read(base)
    assert q.tobytes() == p.tobytes() and lo2.tobytes() == lo.tobytes() and hi2.tobytes() == hi.tobytes()


def test_c_abi_refuses_what_does_not_match(tmp_path):
    """CG_ERR_INVALID_ARG for a flipped bit, other network sizes, another
    format version, a missing file, a non-finite parameter, an empty
    feature box, a directory in the parameter file's name and a meta text
    that is not a JSON object."""
    import paper_1807_11834_gb300 as cg
    p, lo, hi = _closure(9)
    base = str(tmp_path / "c")

    def refused(fn, *a, **k):
        with pytest.raises(cg.CgError) as e:
            fn(*a, **k)
        assert e.value.code == 1

    cg.checkpoint_write(base, p, lo, hi)
    raw = bytearray(open(base + ".f32", "rb").read())
    raw[7] ^= 4
    open(base + ".f32", "wb").write(bytes(raw))
    refused(cg.checkpoint_read, base)
    for key, val in (("hidden", 32), ("version", 2), ("nparam", 5312), ("params_file", "../c.f32")):
        cg.checkpoint_write(base, p, lo, hi)
        head = json.load(open(base + ".json"))
        head[key] = val
        json.dump(head, open(base + ".json", "w"))
        refused(cg.checkpoint_read, base)
    refused(cg.checkpoint_read, str(tmp_path / "absent"))
    bad = p.copy()
    bad[0] = np.inf
    refused(cg.checkpoint_write, base, bad, lo, hi)
    refused(cg.checkpoint_write, base, p, hi, lo)
    L = cg.lib()
    for meta in (b"[1, 2]", b"{\"a\": }", b"{} {}"):
        assert L.cg_mlp_checkpoint_write(str(tmp_path / "m").encode(), p.ctypes.data, lo.ctypes.data,
                                         hi.ctypes.data, meta) == 1
