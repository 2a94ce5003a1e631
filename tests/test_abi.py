"""The C ABI: the library builds for sm_103a, loads, and exports every
function include/mrrr.h declares (CPU only: no compute call needs a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1205_2107_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mrrr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mrrr_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_declares_the_abi():
    names = declared_functions()
    assert names == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_built_for_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(build.LIB)


def test_options_defaults(lib):
    o = _lib.Options()
    assert lib.mrrr_options_default(ctypes.byref(o)) == 0
    assert o.gap_tol == 1e-4  # floor; blocks of order m use max(gap_tol, 1/m)
    assert o.classify_rtol == 2.0 ** -20
    assert o.max_depth == 64 and o.threads_per_block % 32 == 0
    assert o.singleton_rq == 1 and o.vector_precision == 1
    assert o.prebisect_rtol == 2.0 ** -17
    assert lib.mrrr_options_default(None) == _lib.ERR_ARG


@pytest.mark.parametrize("field,value", [
    ("multisection_width", 3), ("multisection_width", 64), ("root_side", 3),
    ("vector_precision", 3), ("singleton_rq", 5), ("singleton_rq", -2),
    ("gap_tol", 1.5), ("gap_tol", float("inf")), ("classify_rtol", 0.5),
    ("cluster_rtol", 0.25), ("cluster_rtol", float("inf")), ("prebisect_rtol", 0.5),
    ("prebisect_rtol", float("inf")), ("root_perturb", float("inf")),
    ("width_scale", float("inf")), ("threads_per_block", 48),
])
def test_plan_create_rejects_options_out_of_range(lib, field, value):
    # the checks come before the first CUDA call, so they run without a GPU
    o = _lib.Options()
    assert lib.mrrr_options_default(ctypes.byref(o)) == 0
    setattr(o, field, value)
    plan = ctypes.c_void_p(0x1234)
    assert lib.mrrr_plan_create(ctypes.byref(plan), ctypes.byref(o)) == _lib.ERR_ARG
    assert plan.value is None  # NULL on failure


def test_status_strings(lib):
    for code in range(9):
        s = lib.mrrr_status_string(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert lib.mrrr_version() >= 100


def test_null_plan_is_rejected(lib):
    sz = ctypes.c_size_t()
    assert lib.mrrr_workspace_size(None, 1, 10, 10, 10, ctypes.byref(sz)) == _lib.ERR_ARG
    assert lib.mrrr_stein(None, 10, None, None, 1, 10, None, None, 10, None, 0, None) == _lib.ERR_ARG
    assert lib.mrrr_plan_destroy(None) == _lib.ERR_ARG
    assert lib.mrrr_plan_create(None, None) == _lib.ERR_ARG


def test_every_entry_rejects_a_null_plan_before_any_device_work(lib):
    """Host-side argument checks return before any CUDA call, so they run
    here without a GPU."""
    ERR = _lib.ERR_ARG
    sz = ctypes.c_size_t()
    assert lib.mrrr_stein_batched(None, 1, None, None, None, None, None, None, None, None, None, 1, 1, 1, None, 0,
                                  None) == ERR
    assert lib.mrrr_autotune_batched(None, 1, None, None, None, None, None, None, None, None, None, 1, 1, 1, None, 0,
                                     None, None) == ERR
    assert lib.mrrr_backward(None, 1, None, None, None, None, None, 0.0, 1, 1, None, None, None, 0, None) == ERR
    assert lib.mrrr_backward_workspace_size(None, 1, 1, ctypes.byref(sz)) == ERR
    assert lib.mrrr_get_status(None, None, None) == ERR
    assert lib.mrrr_set_timing(None, 1) == ERR
    assert lib.mrrr_get_profile(None, None) == ERR


def test_static_entry_checks_its_arguments_first(lib):
    """mrrr_eigenvalues_static: 0 <= n <= MRRR_STATIC_MAX_N, 1 <= il <= iu <=
    n and non-null pointers, all checked before the scratch is touched."""
    text = open(os.path.join(ROOT, "include", "mrrr.h")).read()
    nmax = int(re.search(r"#define MRRR_STATIC_MAX_N (\d+)", text).group(1))
    buf = (ctypes.c_double * 8)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert lib.mrrr_eigenvalues_static(0, None, None, 1, 0, None, None) == _lib.OK  # n = 0: no-op
    assert lib.mrrr_eigenvalues_static(-1, p, p, 1, 1, p, None) == _lib.ERR_ARG
    assert lib.mrrr_eigenvalues_static(nmax + 1, p, p, 1, 1, p, None) == _lib.ERR_ARG
    assert lib.mrrr_eigenvalues_static(5, None, p, 1, 5, p, None) == _lib.ERR_ARG
    assert lib.mrrr_eigenvalues_static(5, p, None, 1, 5, p, None) == _lib.ERR_ARG
    assert lib.mrrr_eigenvalues_static(5, p, p, 1, 5, None, None) == _lib.ERR_ARG
    assert lib.mrrr_eigenvalues_static(5, p, p, 0, 3, p, None) == _lib.ERR_ARG
    assert lib.mrrr_eigenvalues_static(5, p, p, 4, 3, p, None) == _lib.ERR_ARG
    assert lib.mrrr_eigenvalues_static(5, p, p, 2, 6, p, None) == _lib.ERR_ARG


def test_probe_checks_its_arguments_first(lib):
    """mrrr_probe_peak rejects an unknown kind or a NULL rate before any
    device call (kinds 0..6)."""
    rate = ctypes.c_double(-1.0)
    assert lib.mrrr_probe_peak(7, ctypes.byref(rate)) == _lib.ERR_ARG
    assert lib.mrrr_probe_peak(-1, ctypes.byref(rate)) == _lib.ERR_ARG
    assert lib.mrrr_probe_peak(0, None) == _lib.ERR_ARG


C_CLIENT = r"""
#include <stdio.h>
#include <string.h>
#include "mrrr.h"

int main(void) {
  mrrr_options o;
  if (mrrr_options_default(&o) != MRRR_OK) return 1;
  if (o.gap_tol != 1e-4 || o.max_depth != 64) return 2;
  if (mrrr_options_default(NULL) != MRRR_ERR_ARG) return 3;
  if (strcmp(mrrr_status_string(MRRR_ERR_QUEUE), mrrr_status_string(MRRR_OK)) == 0) return 4;
  size_t bytes = 0;
  if (mrrr_workspace_size(NULL, 1, 10, 10, 10, &bytes) != MRRR_ERR_ARG) return 5;
  if (mrrr_stein(NULL, 10, NULL, NULL, 1, 10, NULL, NULL, 10, NULL, 0, NULL) != MRRR_ERR_ARG) return 6;
  printf("version %d\n", mrrr_version());
  return 0;
}
"""


def test_plain_c_client_links_and_runs(lib, tmp_path):
    """The header is a C ABI: a C99 program includes it, links libmrrr.so
    and calls the entry points that need no GPU."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(build.LIB)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe), "-L", libdir, "-l:" + os.path.basename(build.LIB), "-Wl,-rpath," + libdir],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert out.stdout.strip() == f"version {lib.mrrr_version()}"


LAYOUT_CLIENT = r"""
#include <stddef.h>
#include <stdio.h>
#include "mrrr.h"

#define F(T, m) printf(#T "." #m " %zu\n", offsetof(T, m))
int main(void) {
  printf("mrrr_options %zu\nmrrr_info %zu\nmrrr_tuning %zu\nmrrr_profile %zu\n", sizeof(mrrr_options),
         sizeof(mrrr_info), sizeof(mrrr_tuning), sizeof(mrrr_profile));
  F(mrrr_options, width_scale); F(mrrr_options, prebisect_rtol); F(mrrr_options, multisection_width);
  F(mrrr_options, vector_precision); F(mrrr_options, singleton_rq); F(mrrr_options, reserved_);
  F(mrrr_info, diag); F(mrrr_info, sturm_counts); F(mrrr_info, warp_passes);
  F(mrrr_tuning, best_ms); F(mrrr_tuning, singleton_rq);
  return 0;
}
"""


def test_ctypes_structs_match_the_header(lib, tmp_path):
    """The ctypes mirrors of the ABI structs have the header's sizes and
    field offsets (a C compiler lays the header out; ctypes must agree, or
    options and counters would be read from the wrong bytes)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_CLIENT)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                              timeout=60).stdout.strip().splitlines())
    mirrors = {"mrrr_options": _lib.Options, "mrrr_info": _lib.Info, "mrrr_tuning": _lib.Tuning,
               "mrrr_profile": _lib.Profile}
    for name, cls in mirrors.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
    for key, value in got.items():
        if "." in key:
            struct, field = key.split(".")
            assert int(value) == getattr(mirrors[struct], field).offset, key
