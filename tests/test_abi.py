"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lhv.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lhv_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1201_5430_gb300 import build as b
    from paper_1201_5430_gb300 import _lib
    b.build()
    return ctypes.CDLL(_lib.LIB_PATH)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("lhv_create", "lhv_build_tree", "lhv_evaluate_velocity_stretching", "lhv_step", "lhv_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    from paper_1201_5430_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(_declared())


def test_status_strings_without_gpu(lib):
    lib.lhv_status_string.restype = ctypes.c_char_p
    assert lib.lhv_status_string(0) == b"ok"
    assert lib.lhv_status_string(-5) == b"non-finite input"


def test_create_rejects_bad_config_without_gpu(lib):
    from paper_1201_5430_gb300 import _lib
    L = _lib.load()
    h = ctypes.c_void_p()
    for kw in (dict(p=0), dict(p=25), dict(leaf_max=0), dict(core_a=-1.0), dict(precision=7), dict(eps=0.0)):
        cfg = dict(p=8, leaf_max=64, core_a=0.01, eps=1e-6, precision=0, terms=3, max_level=0)
        cfg.update(kw)
        assert L.lhv_create(ctypes.byref(_lib.Config(**cfg)), None, ctypes.byref(h)) == -1


def test_binding_structs_match_the_header(tmp_path):
    """ctypes mirrors of lhv_config / lhv_stats have the C sizes and field offsets
    (a short struct on the Python side would let lhv_get_stats write past it)."""
    import shutil
    import subprocess
    from paper_1201_5430_gb300 import _lib
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    fields = [f[0] for f in _lib.Stats._fields_]
    src = tmp_path / "sz.c"
    body = "\n".join(f'    printf("{f} %zu\\n", offsetof(lhv_stats, {f}));' for f in fields)
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"lhv.h\"\nint main(void) {\n"
                   f"    printf(\"sizeof %zu\\n\", sizeof(lhv_stats));\n"
                   f"    printf(\"config %zu\\n\", sizeof(lhv_config));\n{body}\n    return 0;\n}}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    assert int(out["sizeof"]) == ctypes.sizeof(_lib.Stats)
    assert int(out["config"]) == ctypes.sizeof(_lib.Config)
    for f in fields:
        assert int(out[f]) == getattr(_lib.Stats, f).offset, f
