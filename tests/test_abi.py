"""The C-ABI library builds, loads and exports every symbol its header
declares (no GPU calls)."""
import ctypes
import os
import re

from paper_2208_10008_gb300 import build_ext, rtbvh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(rt_\w+)\s*\(", src, re.M))
    return names


def test_library_exports_every_declared_symbol():
    path = build_ext.build()
    lib = ctypes.CDLL(path)
    names = declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(rtbvh.EXPORTS) == names


def test_version_and_error_string_without_gpu():
    lib = rtbvh.lib()
    assert lib.rt_version() >= 100
    assert isinstance(lib.rt_last_error(), bytes)


def test_null_arguments_rejected_without_gpu():
    lib = rtbvh.lib()
    assert lib.rt_scene_destroy(None) == -1
    assert lib.rt_bvh_build(None, None, None) == -1
    assert lib.rt_trace_closest(None, None, 0, None, None, None) == -1
    out = ctypes.c_void_p()
    assert lib.rt_scene_upload(None, -5, 0, None, ctypes.byref(out)) == -1
    assert b"n_tri" in lib.rt_last_error()


def test_ray_count_without_gpu():
    lib = rtbvh.lib()
    assert lib.rt_ray_count(0, 4096) == 4096
    assert [lib.rt_ray_count(1, L) for L in (0, 1, 8)] == [12, 42, 655362]
    assert lib.rt_ray_count(1, 13) == -1 and lib.rt_ray_count(7, 1) == -1 and lib.rt_ray_count(0, -1) == -1


def test_new_entry_points_reject_null_without_gpu():
    lib = rtbvh.lib()
    assert lib.rt_scene_set_split_events(None, None, None) == -1
    assert lib.rt_autotune(None, None, None, 0, 1.0, None, None) == -1
    assert b"NULL" in lib.rt_last_error()
    assert lib.rt_session_release(None, 1) == -1
    assert b"NULL" in lib.rt_last_error()


def test_debug_hooks_validate_without_gpu():
    lib = rtbvh.lib()
    assert lib.rt_debug_inject(99, 1) == -1
    assert lib.rt_debug_inject(rtbvh.RT_DEBUG_SPIN_LIMIT, -5) == -1
    for hook in (rtbvh.RT_DEBUG_SPIN_LIMIT, rtbvh.RT_DEBUG_PHANTOM_TASK, rtbvh.RT_DEBUG_PHANTOM_ITEM,
                 rtbvh.RT_DEBUG_FAIL_ALLOC):
        assert lib.rt_debug_inject(hook, 0) == 0


def test_reception_entry_points_validate_without_gpu():
    import ctypes
    lib = rtbvh.lib()
    rx = (ctypes.c_float * 6)(0, 0, 0, 1, 1, 1)
    h = ctypes.c_void_p()
    assert lib.rt_rxset_create(None, 2, 1.0, ctypes.byref(h)) == -1
    assert lib.rt_rxset_create(rx, 0, 1.0, ctypes.byref(h)) == -1
    assert lib.rt_rxset_create(rx, (1 << 26) + 1, 1.0, ctypes.byref(h)) == -1   # checked before rx is read
    assert b"2^26" in lib.rt_last_error()
    assert lib.rt_rxset_create(rx, 2, 0.0, ctypes.byref(h)) == -1
    assert lib.rt_rxset_create(rx, 2, float("inf"), ctypes.byref(h)) == -1
    bad = (ctypes.c_float * 3)(0, float("nan"), 0)
    assert lib.rt_rxset_create(bad, 1, 1.0, ctypes.byref(h)) == -1
    assert b"non-finite" in lib.rt_last_error()
    assert lib.rt_rxset_destroy(None) == -1
    p = rtbvh.ReceiveParams(0.01, 500.0, 16, 0, None)
    assert lib.rt_receive(None, None, None, 0, None, ctypes.byref(p), None, None, None) == -1
    assert b"NULL" in lib.rt_last_error()


def test_ctypes_mirrors_match_the_header_structs():
    # a binding struct that is shorter or longer than the library's makes the
    # library read or write past it: every mirror must have the C size
    import ctypes
    lib = rtbvh.lib()
    sizes = (ctypes.c_int64 * 12)()
    assert lib.rt_abi_struct_sizes(sizes, 12) == 12
    mirrors = [32, 16, rtbvh.BuildParams, rtbvh.TraceParams, rtbvh.BvhInfo, rtbvh.TuneResult, 16,
               rtbvh.ReceiveParams, rtbvh.BatchDesc, rtbvh.BatchStats, rtbvh.Request, rtbvh.SessionStats]
    for i, m in enumerate(mirrors):
        want = m if isinstance(m, int) else ctypes.sizeof(m)
        assert sizes[i] == want, (i, m, sizes[i], want)


def test_build_params_marshalling_without_gpu():
    p = rtbvh.build_params(alpha=0.7, source=(1.0, 2.0, 3.0), max_leaf=6, bins=8, dist_norm=1, range=250.0)
    assert abs(p.alpha - 0.7) < 1e-7 and list(p.source) == [1.0, 2.0, 3.0]
    assert (p.max_leaf, p.bins, p.width, p.dist_norm) == (6, 8, 4, 1) and p.range == 250.0
    assert rtbvh.build_params().range == 0.0


def test_host_trace_binding_rejects_malformed_buffers_without_gpu():
    """The host-buffer binding checks shapes and types before any library call
    (a short hit buffer would otherwise be overrun on the host)."""
    import numpy as np
    import pytest
    import torch
    bad = [
        (np.zeros((4, 9), np.float32), None),                     # not [n, 8]
        (np.zeros(32, np.float32), None),                         # flat
        (np.zeros((4, 8), np.float32), np.zeros((3, 4), np.float32)),   # hits too short
        (np.zeros((4, 8), np.float32), np.zeros((4, 4), np.float64)),   # wrong dtype
        (np.zeros((4, 8), np.float32), np.zeros((4, 8), np.float32)[:, ::2]),  # strided
        (torch.zeros(4, 9), None),
        (torch.zeros(4, 8, dtype=torch.float64), None),
        (torch.zeros(4, 8), torch.zeros(3, 4)),
        (torch.zeros(4, 8), torch.zeros(4, 4, dtype=torch.int32)),
        (torch.zeros(4, 8), np.zeros((4, 4), np.float32)),        # mixed kinds
    ]
    for rays, hits in bad:
        with pytest.raises(TypeError):
            rtbvh.rt_trace_closest_host(None, rays, hits)


def test_header_is_plain_c_and_a_c_program_links_without_gpu(tmp_path):
    """The boundary is a C ABI: the header compiles as pedantic C99 and a C
    program links against the library and calls it (no GPU calls)."""
    import shutil
    import subprocess
    import pytest
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not found")
    inc = os.path.join(ROOT, "include")
    hdr = os.path.join(inc, "rtbvh.h")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", "c", hdr],
                   check=True)
    lib_path = build_ext.build()
    src = tmp_path / "main.c"
    src.write_text(
        '#include "rtbvh.h"\n'
        "int main(void) {\n"
        "  rt_ray r = {0};\n"
        "  (void)r;\n"
        "  if (rt_version() < 100) return 1;\n"
        "  if (rt_ray_count(RT_RAYS_ICOSPHERE, 8) != 655362) return 2;\n"
        "  if (rt_scene_destroy(0) != RT_EINVAL || rt_last_error()[0] == 0) return 3;\n"
        "  return 0;\n"
        "}\n")
    exe = tmp_path / "main"
    libdir = os.path.dirname(lib_path)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", inc, str(src), "-L", libdir, "-lrtbvh",
                    "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    assert subprocess.run([str(exe)]).returncode == 0
