"""The CUDA library builds, loads without a GPU and exports every entry point
declared in include/*.h; the binding declares each of them (CPU only)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(fcm_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1601_00072_gb300 import _build
    return _build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("fcm_create", "fcm_destroy", "fcm_run"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_declares_every_symbol(libpath):
    from paper_1601_00072_gb300 import _lib
    lib = _lib.load()
    bound = {name for name, _, _ in _lib.SIGNATURES}
    assert declared_functions() <= bound, sorted(declared_functions() - bound)
    for name in bound:
        assert hasattr(lib, name)


def test_status_strings_without_gpu(libpath):
    from paper_1601_00072_gb300 import _lib
    lib = _lib.load()
    assert lib.fcm_status_string(0) == b"FCM_OK"
    assert lib.fcm_status_string(-4) == b"FCM_ERR_BAD_INPUT"
    assert lib.fcm_version().count(b".") == 2


def test_create_fails_cleanly_without_gpu(libpath):
    import ctypes

    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1601_00072_gb300 import _lib
    h = ctypes.c_void_p()
    assert _lib.load().fcm_create(ctypes.byref(h), 0, None) == _lib.FCM_ERR_CUDA
    assert not h.value


def test_kernels_are_sm103a(libpath):
    """The library carries device code for sm_103a (checked from the build
    flags the library was linked with, not by disassembling it)."""
    from paper_1601_00072_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in _build.ARCH


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built CUDA library the binding raises; nothing falls back
    to a CPU path."""
    from paper_1601_00072_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "library_path", lambda: str(tmp_path / "libfcm_gb300.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load()


def test_bounds_variant_is_a_separate_build():
    """FCM_DEBUG_BOUNDS=1 selects the bounds-guarded variant: its own build
    folder and -DFCM_DEBUG_BOUNDS on every translation unit."""
    import subprocess
    import sys
    code = ("from paper_1601_00072_gb300 import _build, _lib; "
            "print(_build.LIB); print(_lib.library_path()); print('-DFCM_DEBUG_BOUNDS=1' in _build.FLAGS)")
    for val, folder, flag in (("1", "_build_bounds", "True"), ("0", "_build", "False")):
        env = dict(os.environ, FCM_DEBUG_BOUNDS=val)
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True,
                             cwd=ROOT).stdout.split()
        assert out[0] == out[1] and os.path.basename(os.path.dirname(out[0])) == folder and out[2] == flag
