"""The C-ABI library builds, loads and exports every entry point of include/fgbd.h.

These run without a GPU: only symbol lookup and host-side argument checks that
return before any CUDA call are exercised.
"""
import ctypes
import os
import re

import pytest

from paper_2401_09721_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fgbd.h")


@pytest.fixture(scope="module")
def so():
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(fgbd_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_four_steps():
    names = declared_functions()
    for step in ("fgbd_build_graph", "fgbd_estimate_noise", "fgbd_select_filter", "fgbd_denoise"):
        assert step in names


def test_every_declared_symbol_is_exported(so):
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_every_entry_point():
    from paper_2401_09721_gb300 import fgbd
    assert sorted(fgbd._SIGS) == declared_functions()


def test_only_the_abi_is_exported():
    import subprocess
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("nm unavailable")
    syms = [line.split()[-1] for line in out.stdout.splitlines() if line.strip()]
    assert syms and all(s.startswith("fgbd_") for s in syms), syms


def test_host_side_checks_without_gpu(so):
    from paper_2401_09721_gb300 import fgbd
    lib = fgbd.lib()
    assert lib.fgbd_abi_version() == fgbd.ABI_VERSION == 3
    p = fgbd.Params()
    assert lib.fgbd_params_default(ctypes.byref(p)) == 0
    assert (p.bits, p.window, p.fslr_factor, p.q_max) == (10, 1, 2.0, 64)
    assert lib.fgbd_params_default(None) == 1
    out = ctypes.c_void_p()
    assert lib.fgbd_ctx_create(0, None, ctypes.byref(out)) == 1            # capacity < 1
    assert lib.fgbd_ctx_create(1 << 30, None, ctypes.byref(out)) == 1      # capacity too large
    bad = fgbd.Params()
    lib.fgbd_params_default(ctypes.byref(bad))
    bad.bits = 11
    assert lib.fgbd_ctx_create(100, ctypes.byref(bad), ctypes.byref(out)) == 1
    bad.bits, bad.q_max = 10, 257
    assert lib.fgbd_ctx_create(100, ctypes.byref(bad), ctypes.byref(out)) == 1
    bad.q_max, bad.variant = 64, 128                                        # no such ablation switch
    assert lib.fgbd_ctx_create(100, ctypes.byref(bad), ctypes.byref(out)) == 1
    bad.variant = fgbd.VARIANT_SIGMA_NODE | fgbd.VARIANT_SIGMA_PAIR         # two readings of one quantity
    assert lib.fgbd_ctx_create(100, ctypes.byref(bad), ctypes.byref(out)) == 1
    bad.variant, bad.reserved[0] = 0, 1                                     # reserved must stay zero
    assert lib.fgbd_ctx_create(100, ctypes.byref(bad), ctypes.byref(out)) == 1
    bad.reserved[0], bad.flags = 0, 2                                       # no such execution flag
    assert lib.fgbd_ctx_create(100, ctypes.byref(bad), ctypes.byref(out)) == 1
    bad.flags, bad.window = 0, 0                                            # window < 1
    assert lib.fgbd_ctx_create(100, ctypes.byref(bad), ctypes.byref(out)) == 1
    bad.window = fgbd.MAX_WINDOW + 1                                        # wider than built
    assert lib.fgbd_ctx_create(100, ctypes.byref(bad), ctypes.byref(out)) == 7
    bad.window, bad.variant = 2, fgbd.VARIANT_UNSORTED_PATCH                # link order defined at w = 1 only
    assert lib.fgbd_ctx_create(100, ctypes.byref(bad), ctypes.byref(out)) == 7
    for v in (fgbd.VARIANT_SIGMA_PAIR, fgbd.VARIANT_POOLED_PATCH):           # built for window 1 only
        bad.variant = v
        assert lib.fgbd_ctx_create(100, ctypes.byref(bad), ctypes.byref(out)) == 7
    assert (fgbd.MAX_WINDOW, fgbd.PATCH_DIM_MAX) == (3, 57)
    assert p.flags == 0 and fgbd.FLAG_FUSED_SELECT == 1
    assert p.variant == 0 and fgbd.VARIANT_NO_FSLR == 1 and fgbd.VARIANT_UNSORTED_PATCH == 2
    assert fgbd.VARIANT_SAME_LINE == 4
    assert lib.fgbd_ctx_create(100, None, None) == 1
    assert lib.fgbd_build_graph(None, None, 0, None) == 1
    assert lib.fgbd_sync(None, None) == 1
    assert lib.fgbd_status_str(0) == b"FGBD_OK"
    assert lib.fgbd_status_str(5).startswith(b"FGBD_ETIMEOUT")
    assert lib.fgbd_debug_set_wait_limit(None, 0) == 1
    assert lib.fgbd_debug_moments(None, None, None, None) == 1
    # the graph handle: argument checks before any CUDA call
    g = ctypes.c_void_p()
    assert lib.fgbd_graph_export(None, ctypes.byref(g), None) == 1
    assert lib.fgbd_graph_csr(None, None, None, None, None, None, None) == 1
    lib.fgbd_graph_free(None)                                               # NULL is ignored
    shape = fgbd.BatchShape()
    assert lib.fgbd_get_batch_shape(0, 1000000, ctypes.byref(shape)) == 0   # the defaults, no GPU needed
    assert (shape.seg_frames, shape.scatter_threads, shape.filter_threads, shape.filter_blocks_per_sm) == (0, 512, 512, 2)
    assert lib.fgbd_get_batch_shape(0, 20000, ctypes.byref(shape)) == 0     # small frames: segmented by default
    assert shape.seg_frames == 16
    assert lib.fgbd_get_batch_shape(0, -1, ctypes.byref(shape)) == 1
    shape.scatter_threads = 300
    assert lib.fgbd_set_batch_shape(0, 1000, ctypes.byref(shape)) == 1      # not a built shape
    assert lib.fgbd_tune_batch(None, None, None, None, None, None, None, 1, None, None) == 1
    assert lib.fgbd_estimate_noise(None, None, 0, None, None, None) == 1
    assert lib.fgbd_select_filter(None, None, 0, None, None, None, None) == 1


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes structures have the size and field offsets that a C compiler
    gives the header's structs (a field added on one side only fails here)."""
    import shutil
    import subprocess
    from paper_2401_09721_gb300 import fgbd
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"fgbd_params": fgbd.Params, "fgbd_stats": fgbd.Stats, "fgbd_batch_shape": fgbd.BatchShape}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "fgbd.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
