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
    q, lo2, hi2, meta, act = closure.load_checkpoint(base)
    assert q.dtype == np.float32 and q.tobytes() == p.tobytes()
    assert lo2.tobytes() == lo.tobytes() and hi2.tobytes() == hi.tobytes()
    assert meta == {"refresh": 10, "target_mean": 0.01, "target_std": 0.2} and act == "gelu"
    closure.save_checkpoint(base, p, lo, hi, activation="relu")
    assert closure.load_checkpoint(base)[4] == "relu"
    # a head without the activation key (an older file) reads as GELU
    head = json.load(open(base + ".json"))
    del head["activation"]
    json.dump(head, open(base + ".json", "w"))
    assert closure.load_checkpoint(base)[4] == "gelu"
    closure.save_checkpoint(base, p, lo, hi, refresh=10, target_mean=0.01, target_std=0.2)
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
    with pytest.raises(ValueError):
        closure.save_checkpoint(base, p, lo, hi, activation="tanh")
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
    cg.checkpoint_write(base, p, lo, hi, meta={"refresh": 5, "note": "a \"quoted\" word"}, activation="relu")
    q, lo2, hi2, meta, act = closure.load_checkpoint(base)
    assert q.tobytes() == p.tobytes() and lo2.tobytes() == lo.tobytes() and hi2.tobytes() == hi.tobytes()
    assert meta == {"refresh": 5, "note": "a \"quoted\" word"} and act == "relu"
    import hashlib
    raw = open(base + ".f32", "rb").read()
    assert json.load(open(base + ".json"))["params_sha256"] == hashlib.sha256(raw).hexdigest()


def test_c_abi_reads_what_python_writes_bit_exact(tmp_path):
    import paper_1807_11834_gb300 as cg
    p, lo, hi = _closure(8)
    base = str(tmp_path / "py_written")
    closure.save_checkpoint(base, p, lo, hi, refresh=20, target_mean=0.0)
    q, lo2, hi2, act = cg.checkpoint_read(base)
    assert q.tobytes() == p.tobytes() and lo2.tobytes() == lo.tobytes() and hi2.tobytes() == hi.tobytes()
    assert act == "gelu"
    closure.save_checkpoint(base, p, lo, hi, activation="relu")
    assert cg.checkpoint_read(base)[3] == "relu"


def test_c_abi_refuses_what_does_not_match(tmp_path):
    """CG_ERR_INVALID_ARG for a flipped bit, other network sizes, another
    format version, an unknown activation, a missing file, a non-finite
    parameter, an empty feature box, a directory in the parameter file's
    name and a meta text that is not a JSON object."""
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
    for key, val in (("hidden", 32), ("version", 2), ("nparam", 5312), ("params_file", "../c.f32"),
                     ("activation", "tanh")):
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
                                         hi.ctypes.data, 0, meta) == 1
    assert L.cg_mlp_checkpoint_write(str(tmp_path / "m").encode(), p.ctypes.data, lo.ctypes.data,
                                     hi.ctypes.data, 2, b"{}") == 1       # no activation 2


def test_bias_split_into_three_bf16_terms_is_exact():
    """The tensor-core kernels carry each FP32 bias into the products as
    three BF16 terms h = bf16(b), m = bf16(b - h), l = b - h - m (the
    remainders formed in FP32): l is itself a BF16 value and h + m + l
    equals b exactly, for normal values across the exponent range, ties of
    the first rounding, and zero."""
    from oracle.mlp import bf16
    rng = np.random.default_rng(11)
    b = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.uniform(-30, 30, 20000),
                        (1.0 + rng.integers(0, 2 ** 23, 2000) * 2.0 ** -23) * 2.0 ** rng.integers(-100, 100, 2000),
                        [0.0, 1.0, -1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -23, 3.0 * 2 ** -9, -(2 - 2 ** -23)]])
    b = b.astype(np.float32)
    h = bf16(b).astype(np.float32)
    r = b - h                                   # FP32, exact
    m = bf16(r).astype(np.float32)
    lo = r - m                                  # FP32, exact
    assert np.array_equal(bf16(lo), lo.astype(np.float64))
    assert np.array_equal(h.astype(np.float64) + m.astype(np.float64) + lo.astype(np.float64), b.astype(np.float64))
