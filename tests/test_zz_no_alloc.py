"""The binning entry point that allocates nothing.

Some callers must not allocate device memory: code that runs while another
component is capturing a CUDA graph, or plug-ins that may only use the
memory their host application hands them.  cg_bin_particles_static serves
them with scratch held in a fixed device array inside the library.  This
test calls it through the C ABI twice in a row (the array keeps the
previous call's contents) and checks that its cells, permutation and cell
starts match those of the handle-based cg_bin_particles bit for bit, as all
binning results in this suite must.  It sits in a file of its own that
pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _bins_handle(cg, w):
    import torch
    g = cg.Grids(w.desc)
    pos = torch.from_numpy(w.pos_d).cuda()
    cell = torch.empty(w.n, dtype=torch.int32, device="cuda")
    perm = torch.empty_like(cell)
    cs = torch.empty(g.n_bulk + 1, dtype=torch.int32, device="cuda")
    g.cg_bin_particles(pos, cell, perm, cs)
    torch.cuda.synchronize()
    out = (cell.cpu().numpy(), perm.cpu().numpy(), cs.cpu().numpy())
    g.close()
    return out


def _bins_static(cg, w):
    import torch
    L = cg.lib()
    d = cg.make_desc(w.desc)
    nb = int(np.prod([v // w.desc["ratio"] for v in w.desc["fine_n"]]))
    pos = torch.from_numpy(w.pos_d).cuda()
    cell = torch.full((w.n,), -7, dtype=torch.int32, device="cuda")
    perm = torch.full((w.n,), -7, dtype=torch.int32, device="cuda")
    cs = torch.full((nb + 1,), -7, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.cg_bin_particles_static(C.byref(d), w.n, C.c_void_p(pos.data_ptr()), C.c_void_p(cell.data_ptr()),
                                   C.c_void_p(perm.data_ptr()), C.c_void_p(cs.data_ptr()), stream)
    assert rc == 0, cg.STATUS_NAMES.get(rc, rc)
    torch.cuda.synchronize()
    return cell.cpu().numpy(), perm.cpu().numpy(), cs.cpu().numpy()


def _with_sort(w, sort_digits):
    w.desc["sort_digits"] = sort_digits
    return w


@pytest.mark.parametrize("make", [
    lambda: synth.small_packed_bed(seed=3),            # FP32, 62,500 particles, two sort passes
    lambda: synth.tiny(seed=4, n=20_000),              # FP64, one sort pass
    lambda: _with_sort(synth.small_packed_bed(seed=5), 1),     # the per-cell sort, asked for
    lambda: _with_sort(synth.small_packed_bed(seed=6), 6),     # three digit passes (both intermediates)
    lambda: _with_sort(synth.small_packed_bed(seed=7), 11),    # two passes of the widest digit
    # the largest call the scratch holds: 262,144 particles, one pass of 11-bit
    # digits over 12^3 cells, so the tile histograms fill their whole region
    lambda: _with_sort(synth.tiny(seed=8, n=262_144, fine=48, fp64=False), 11),
], ids=["packed_bed_fp32", "tiny_fp64", "per_cell_sort", "three_digit_passes", "widest_digits",
        "largest_call"])
def test_static_binning_matches_handle_binning_on_two_calls(cuda_lib, make):
    w = make()
    ref = _bins_handle(cuda_lib, w)
    for _ in range(2):
        got = _bins_static(cuda_lib, w)
        for name, a, b in zip(("cell", "perm", "cell_start"), got, ref):
            assert np.array_equal(a, b), name


def test_static_binning_of_no_particles(cuda_lib):
    """n = 0: every cell starts at 0, after a call that left the scratch full."""
    import torch
    _bins_static(cuda_lib, synth.tiny(seed=9, n=5_000))
    L = cuda_lib.lib()
    w = synth.tiny(seed=0, n=1)
    d = cuda_lib.make_desc(w.desc)
    nb = (w.desc["fine_n"][0] // w.desc["ratio"]) ** 3
    pos = torch.from_numpy(w.pos_d).cuda()
    perm = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    cs = torch.full((nb + 1,), -7, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.cg_bin_particles_static(C.byref(d), 0, C.c_void_p(pos.data_ptr()), None, C.c_void_p(perm.data_ptr()),
                                   C.c_void_p(cs.data_ptr()), stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert bool((cs == 0).all())
    assert int(perm[0]) == -7          # nothing written for no particles


def test_static_binning_rejects_sizes_beyond_its_scratch(cuda_lib):
    import torch
    L = cuda_lib.lib()
    w = synth.tiny(seed=0, n=16)
    d = cuda_lib.make_desc(w.desc)
    buf = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = L.cg_bin_particles_static(C.byref(d), 262_145, C.c_void_p(buf.data_ptr()), None,
                                   C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr()), None)
    assert rc == 5   # CG_ERR_OUT_OF_RANGE, checked before any work is enqueued
