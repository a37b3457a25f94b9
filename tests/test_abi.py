"""The C ABI library builds, loads and exports every symbol include/mrfmap.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mrfmap.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(mrf_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2006_03512_gb300 as m
    m.build()
    return m.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mrf_create", "mrf_add_frame", "mrf_infer", "mrf_marginals", "mrf_stats", "mrf_last_error",
                     "mrf_destroy", "mrf_ray_messages", "mrf_voxel_reduce"]:
        assert required in names


def test_header_is_plain_c(tmp_path):
    """The boundary is a C ABI: the header compiles as strict C99 (no C++ types) and as C++."""
    import shutil
    import subprocess
    src = tmp_path / "use.c"
    src.write_text('#include "mrfmap.h"\nint main(void) { mrf_options o; mrf_default_options(&o); '
                   'return o.precision; }\n')
    for cc, lang, std in [("gcc", "c", "-std=c99"), ("g++", "c++", "-std=c++17")]:
        if shutil.which(cc) is None:
            pytest.skip(f"no {cc}")
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", lang,
                            "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_library_exports_every_declared_symbol(lib):
    import paper_2006_03512_gb300 as m
    names = declared_functions()
    for n in names:
        assert hasattr(lib, n), f"{n} not exported"
        assert n in m.SIGNATURES, f"{n} has no binding signature"
    assert set(m.SIGNATURES) == set(names)


def test_library_is_built_for_sm103a():
    import paper_2006_03512_gb300 as m
    from paper_2006_03512_gb300 import builder as b
    assert "arch=compute_103a,code=sm_103a" in " ".join(b.ARCH)
    assert os.path.exists(m.LIB_PATH)


def test_null_and_range_arguments_fail_cleanly(lib):
    # argument checks happen before any CUDA call
    lib.mrf_create.restype = ctypes.c_int
    assert lib.mrf_create(None, None, ctypes.c_float(0.5), None, None) == -1
    import paper_2006_03512_gb300 as m
    h = ctypes.c_void_p()
    g = m._Grid(0, 4, 4, 0.1, (ctypes.c_float * 3)(0, 0, 0))
    assert lib.mrf_create(ctypes.byref(h), ctypes.byref(g), ctypes.c_float(0.5), None, None) == m.MRF_EINVAL
    g = m._Grid(4, 4, 4, 0.1, (ctypes.c_float * 3)(0, 0, 0))
    assert lib.mrf_create(ctypes.byref(h), ctypes.byref(g), ctypes.c_float(1.5), None, None) == m.MRF_EINVAL
    g = m._Grid(4096, 4096, 4096, 0.1, (ctypes.c_float * 3)(0, 0, 0))
    assert lib.mrf_create(ctypes.byref(h), ctypes.byref(g), ctypes.c_float(0.5), None, None) == m.MRF_ERANGE
    assert lib.mrf_launch_count(None) == 0
    assert lib.mrf_ray_messages(None, 0, 0, None, None, None, None, ctypes.c_float(0), 0, ctypes.c_float(0), None, 0,
                                None) == m.MRF_EINVAL


def test_workspace_queries(lib):
    assert lib.mrf_ray_messages_workspace(10, 1000, 50) >= 8
    assert lib.mrf_ray_messages_workspace(10, 1000, 100000) == 0  # ray longer than the kernel supports
    assert lib.mrf_voxel_reduce_workspace(10 ** 6) >= 4 * (10 ** 6 // 4096)


def test_product_path_has_no_fallback(monkeypatch, tmp_path):
    import paper_2006_03512_gb300 as m
    monkeypatch.setattr(m, "_lib", None)
    monkeypatch.setattr(m, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        m.lib()


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2006_03512_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dp, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
