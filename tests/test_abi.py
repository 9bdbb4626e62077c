"""The C-ABI library builds, loads and exports every entry point that
include/shdom_gb300.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "shdom_gb300.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(shd_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def built():
    from paper_1507_05141_gb300 import build
    return build.build()


def test_header_declares_the_step(built):
    names = _declared()
    for must in ["shd_create", "shd_destroy", "shd_set_grid", "shd_set_angles", "shd_set_groups",
                 "shd_set_fields", "shd_set_scattering", "shd_step", "shd_get_moments", "shd_get_state",
                 "shd_solve_static"]:
        assert must in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(built):
    from paper_1507_05141_gb300 import native
    assert set(_declared()) <= set(native.exported_symbols())


def test_library_is_built_for_sm103a(built):
    import subprocess
    out = subprocess.run(["cuobjdump", "--list-elf", built], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_no_cpu_fallback_without_library(monkeypatch, tmp_path):
    """The binding refuses to run when the CUDA library is missing."""
    from paper_1507_05141_gb300 import build, native
    monkeypatch.setattr(build, "lib_path", lambda: str(tmp_path / "missing.so"))
    monkeypatch.setattr(native, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        native.lib()


def test_launch_count_is_host_side(built):
    """The launch counter needs no GPU: it only reads a host counter."""
    from paper_1507_05141_gb300 import native
    a = native.launch_count()
    b = native.launch_count()
    assert 0 <= a <= b
