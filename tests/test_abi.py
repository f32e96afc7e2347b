"""Host-side checks of the C ABI library (no GPU work): it loads, exports every
symbol include/nvd.h declares, and its pure host functions behave."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nvd.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2310_11222_gb300 import build
    build.build()
    import paper_2310_11222_gb300 as nvd
    return nvd.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(nvd_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["nvd_graph_create", "nvd_graph_destroy", "nvd_graph_info", "nvd_ge_distance",
                 "nvd_ge_distance_batched", "nvd_ge_grad", "nvd_status_string", "nvd_laplacian_apply",
                 "nvd_effective_resistance", "nvd_graph_set_weights", "nvd_dot_f32"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings_and_version(lib):
    assert lib.nvd_status_string(0) == b"NVD_OK"
    assert lib.nvd_status_string(2) == b"NVD_ERR_NOT_SYMMETRIC"
    assert lib.nvd_status_string(123) == b"NVD_ERR_UNKNOWN"
    assert b"sm_103a" in lib.nvd_version()


def test_default_opts(lib):
    import paper_2310_11222_gb300 as nvd
    o = nvd.SolveOpts()
    lib.nvd_solve_opts_default(ctypes.byref(o))
    assert o.mode == 0 and o.rtol == 1e-10 and o.max_iter == 10000 and o.kt == 0
    assert ctypes.sizeof(nvd.SolveOpts) == 40 and ctypes.sizeof(nvd.SolveStats) == 24


def test_invalid_arguments_rejected_before_device_work(lib):
    h = ctypes.c_void_p(None)
    # n = 0, NULL rowptr, bad dtype: all rejected on the host
    assert lib.nvd_graph_create(ctypes.byref(h), 0, 0, None, None, None, 1, 0, None) == 1
    assert h.value is None
    assert lib.nvd_graph_create(None, 3, 0, None, None, None, 1, 0, None) == 1
    assert lib.nvd_graph_create(ctypes.byref(h), 3, 0, None, None, None, 7, 0, None) == 1
    assert b"invalid" in lib.nvd_last_error()
    assert lib.nvd_ge_distance(None, 1, None, None, 1, None, None, None, None, None) == 1
    assert lib.nvd_ge_grad(None, 1, None, 1, None, None, None, None, None) == 1
    assert lib.nvd_graph_tune(None, 0, 1, 0, None, None) == 1
    assert lib.nvd_effective_resistance(None, 1, None, None, None, None, None, None) == 1
    assert lib.nvd_resistance_matrix(None, 1, None, None, None, None, None) == 1
    assert lib.nvd_network_variance(None, 1, None, None, None, None, None) == 1
    assert lib.nvd_ge_distance_warm(None, 1, None, None, 1, None, None, None, None, None, None) == 1
    assert lib.nvd_graph_set_tuning(None, 0, None) == 1
    assert lib.nvd_dot_f32(None, None, -1, None, None) == 1
    assert lib.nvd_graph_destroy(None) == 0
    assert lib.nvd_profile_read(3, None, None, None) == 1


def test_package_fails_loudly_without_library(monkeypatch):
    import paper_2310_11222_gb300 as nvd
    monkeypatch.setattr(nvd, "_LIB_PATH", "/nonexistent/libnvd.so")
    monkeypatch.setattr(nvd, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        nvd.load_library()


def test_plain_c_program_uses_the_library(lib, tmp_path):
    """The boundary is a C ABI: a C99 program that includes only include/nvd.h links
    against libnvd.so and calls its host-only entry points."""
    import shutil
    import subprocess
    import paper_2310_11222_gb300 as nvd
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_nvd.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "nvd.h"
int main(void) {
    nvd_solve_opts o;
    nvd_solve_opts_default(&o);
    if (o.mode != NVD_MODE_FP64 || o.max_iter != 10000) return 2;
    if (strcmp(nvd_status_string(0), "NVD_OK") != 0) return 3;
    /* a path 0-1-2-3 eliminates down to one node, with no device work */
    int64_t rp[5] = {0, 1, 3, 5, 6};
    int32_t ci[6] = {1, 0, 2, 1, 3, 2};
    double w[6] = {1, 1, 2, 2, 4, 4};
    int64_t kept = -1;
    int32_t rounds = -1;
    if (nvd_eliminate_host(4, rp, ci, w, &kept, NULL, NULL, NULL, NULL, &rounds) != NVD_OK) return 4;
    if (kept != 1) return 5;
    if (nvd_ge_distance(NULL, 1, NULL, NULL, NVD_F64, NULL, NULL, NULL, NULL, NULL) != NVD_ERR_INVALID_ARG) return 6;
    printf("%s\n", nvd_version());
    return 0;
}
''')
    exe = tmp_path / "use_nvd"
    libdir = os.path.dirname(nvd.library_path())
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                           "-L", libdir, "-lnvd", "-Wl,-rpath," + libdir, "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert "sm_103a" in out.stdout
