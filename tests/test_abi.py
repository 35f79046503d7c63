"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/cg.h declares; the binding's signatures cover them."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(cg_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libcg():
    from paper_1807_11834_gb300 import _build_lib
    path = _build_lib.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = declared_functions()
    for must in ["cg_create_grids", "cg_bin_particles", "cg_deposit", "cg_average_fine_to_bulk",
                 "cg_drag", "cg_project_bulk_to_fine", "cg_step"]:
        assert must in names


def test_library_exports_every_declared_symbol(libcg):
    missing = [n for n in declared_functions() if not hasattr(libcg, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    import paper_1807_11834_gb300 as cg
    assert set(declared_functions()) <= set(cg._SIGS)


def test_status_strings_without_gpu(libcg):
    libcg.cg_status_string.restype = ctypes.c_char_p
    assert libcg.cg_status_string(0) == b"ok"
    assert libcg.cg_status_string(4).startswith(b"particles not binned")


def test_struct_layout_matches_header():
    import paper_1807_11834_gb300 as cg
    # cg_grid_desc: 6 doubles, 3+1+4 int32 + reserved, 5 doubles, 3 doubles
    assert ctypes.sizeof(cg.GridDesc) == 6 * 8 + 10 * 4 + 5 * 8 + 3 * 8   # 9 int32 and 4 bytes of padding
    assert ctypes.sizeof(cg.StepOut) == 13 * 8
    assert ctypes.sizeof(cg.Particles) == 24
    # cg_batch_item: desc, particles, u_fine pointer, step outputs; cg_batch_config: 5 int32
    assert ctypes.sizeof(cg.BatchItem) == ctypes.sizeof(cg.GridDesc) + 24 + 8 + 13 * 8
    assert ctypes.sizeof(cg.BatchConfig) == 5 * 4


def test_struct_layout_matches_the_c_compiler(tmp_path):
    """sizeof / offsetof of the ABI structs as gcc lays them out from cg.h."""
    import shutil
    import subprocess
    import paper_1807_11834_gb300 as cg
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "cg.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(cg_grid_desc), '
                   'sizeof(cg_particles), sizeof(cg_step_out), sizeof(cg_batch_item), '
                   'offsetof(cg_batch_item, u_fine), offsetof(cg_batch_item, out), sizeof(cg_batch_config));'
                   'printf("%zu %zu\\n", sizeof(cg_box_grid), offsetof(cg_box_grid, prec));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(cg.GridDesc), ctypes.sizeof(cg.Particles), ctypes.sizeof(cg.StepOut),
            ctypes.sizeof(cg.BatchItem), cg.BatchItem.u_fine.offset, cg.BatchItem.out.offset,
            ctypes.sizeof(cg.BatchConfig), ctypes.sizeof(cg.BoxGrid), cg.BoxGrid.prec.offset]
    assert got == want


def test_invalid_arguments_rejected_before_any_gpu_work(libcg):
    import paper_1807_11834_gb300 as cg
    L = cg.lib()
    h = ctypes.c_void_p()
    d = cg.make_desc(dict(origin=(0, 0, 0), extent=(1, 1, 1), fine_n=(32, 32, 30), ratio=4, fp64=False,
                          law=0, eps_switch=0.8, eps_min=0.1, rho_f=1000.0, mu_f=1e-3, rho_p=2500.0))
    # fine_n not divisible by the ratio
    assert L.cg_create_grids(ctypes.byref(d), None, ctypes.byref(h)) == 1
    d.fine_n[2] = 32
    d.eps_switch = 1.5
    assert L.cg_create_grids(ctypes.byref(d), None, ctypes.byref(h)) == 1
    d.eps_switch = 0.8
    d.fine_n[0] = 4   # one bulk cell along x
    assert L.cg_create_grids(ctypes.byref(d), None, ctypes.byref(h)) == 1
    assert L.cg_create_grids(None, None, ctypes.byref(h)) == 1
    assert L.cg_bin_particles(None, 0, None, None, None, None) == 1


def test_argument_checks_answer_before_any_device_work():
    """Descriptors and grids the ABI rejects come back CG_ERR_INVALID_ARG
    (1) synchronously, before the library touches a device, so these run
    without a GPU: unknown sort and stencil choices, non-nested ratios, a bulk axis of
    one cell, and degenerate or mixed-precision map grids."""
    import paper_1807_11834_gb300 as cg
    import synth
    L = cg.lib()
    base = synth.tiny(seed=0, n=1).desc
    for bad in (dict(sort_digits=2), dict(sort_digits=12), dict(sort_digits=-1), dict(stencil=2), dict(stencil=-1),
                dict(ratio=3),
                dict(fine_n=(8, 8, 4), ratio=4), dict(extent=(1.0, 0.0, 1.0))):
        d = dict(base)
        d.update(bad)
        h = ctypes.c_void_p()
        assert L.cg_create_grids(ctypes.byref(cg.make_desc(d)), None, ctypes.byref(h)) == 1, bad
        assert not h.value
    ok = ((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (4, 4, 4))

    def box(o, e, n, prec=0):
        g = cg.BoxGrid()
        g.origin[:] = o
        g.extent[:] = e
        g.n[:] = n
        g.prec = prec
        return g
    for b, f in ((box(*ok), box((0, 0, 0), (1, 1, 1), (4, 0, 4))),
                 (box((0, 0, 0), (1, -1, 1), (4, 4, 4)), box(*ok)),
                 (box(*ok, prec=1), box(*ok, prec=0)),
                 (box(*ok, prec=3), box(*ok, prec=3)),
                 (box((0, 0, float("nan")), (1, 1, 1), (4, 4, 4)), box(*ok))):
        h = ctypes.c_void_p()
        assert L.cg_map_create(ctypes.byref(b), ctypes.byref(f), None, ctypes.byref(h)) == 1
        assert not h.value
    assert L.cg_map_average(None, 1, None, None) == 1
    assert L.cg_destroy_grids(None) == 0 and L.cg_map_destroy(None) == 0
    # the allocation fault injection is host-side: set, switched off, refused below -1
    assert L.cg_debug_fail_alloc_after(-2) == 1
    assert L.cg_debug_fail_alloc_after(3) == 0 and L.cg_debug_fail_alloc_after(-1) == 0


def test_constants_match_the_header(tmp_path):
    """Every constant the binding hard-codes equals the header's, as the C
    compiler sees it."""
    import shutil
    import subprocess
    import paper_1807_11834_gb300 as cg
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    names = ["CG_OK", "CG_ERR_INVALID_ARG", "CG_ERR_CUDA", "CG_ERR_OOM", "CG_ERR_NOT_BINNED", "CG_ERR_OUT_OF_RANGE",
             "CG_ERR_TIMEOUT", "CG_ERR_NONFINITE", "CG_FP32", "CG_FP64", "CG_DRAG_DI_FELICE", "CG_DRAG_ERGUN_WEN_YU",
             "CG_INTERP_TRILINEAR", "CG_INTERP_CELL", "CG_DEP_VOLUME", "CG_DEP_MOMENTUM", "CG_FLAG_OUTSIDE",
             "CG_FLAG_NONFINITE", "CG_FLAG_EPS_CLAMPED", "CG_FLAG_TIMEOUT", "CG_SORT_AUTO", "CG_SORT_CELLS",
             "CG_SORT_CELLS_AUTO_MAX", "CG_SORT_CELLS_AUTO_DENSITY", "CG_NCOUNTS", "CG_NSUMS", "CG_MLP_NPARAM",
             "CG_MLP_NFEAT"]
    src = tmp_path / "k.c"
    src.write_text('#include <stdio.h>\n#include "cg.h"\nint main(void){\n'
                   + "".join(f'printf("%lld\\n", (long long)({n}));\n' for n in names) + "return 0;}\n")
    exe = tmp_path / "k"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    py = {n: getattr(cg, n) for n in names if hasattr(cg, n)}
    py["CG_MLP_NPARAM"], py["CG_MLP_NFEAT"] = cg.MLP_NPARAM, cg.MLP_NFEAT
    for k in ("CG_ERR_INVALID_ARG", "CG_ERR_CUDA", "CG_ERR_OOM", "CG_ERR_NOT_BINNED", "CG_ERR_OUT_OF_RANGE",
              "CG_ERR_TIMEOUT", "CG_ERR_NONFINITE"):
        py[k] = {v: c for c, v in cg.STATUS_NAMES.items()}[k]
    assert {n: v for n, v in zip(names, got)} == {n: py[n] for n in names}


def test_grid_sizes_whose_product_overflows_are_refused():
    """Cell counts are checked while their product grows: fine_n of
    2^21 x 2^21 x 2^22 (ratio 1) would wrap a 64-bit product to 0; both the
    handle and the allocation-free binning refuse it (CG_ERR_OUT_OF_RANGE)
    before any device work, as they refuse a grid just over 2^22 bulk
    cells."""
    import paper_1807_11834_gb300 as cg
    import synth
    L = cg.lib()
    base = synth.tiny(seed=0, n=1).desc
    for fine_n, ratio in (((1 << 21, 1 << 21, 1 << 22), 1), ((1 << 30, 1 << 30, 4), 2),
                          ((4096, 2050, 4), 2)):
        d = dict(base, fine_n=fine_n, ratio=ratio)
        h = ctypes.c_void_p()
        assert L.cg_create_grids(ctypes.byref(cg.make_desc(d)), None, ctypes.byref(h)) == 5, fine_n
        assert not h.value
        buf = ctypes.c_int32 * 4
        perm, cs = buf(), buf()
        assert L.cg_bin_particles_static(ctypes.byref(cg.make_desc(d)), 0, None, None, perm, cs, None) == 5, fine_n
