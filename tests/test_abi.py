"""The C-ABI library builds for sm_103a and exports every entry point the public header
declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bmf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bmf_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_1703_00734_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("bmf_init", "bmf_sweep", "bmf_stage", "bmf_predict", "bmf_destroy",
              "bmf_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads(libpath):
    from paper_1703_00734_gb300 import bmf
    L = bmf.load(libpath)
    assert L.bmf_last_error(None) is not None or True


def test_missing_library_fails_loudly(tmp_path):
    from paper_1703_00734_gb300 import bmf
    with pytest.raises(RuntimeError):
        bmf._lib = None
        try:
            bmf.load(str(tmp_path / "nope.so"))
        finally:
            bmf._lib = None


def header_enums():
    """name -> value of every `BMF_NAME = value` enumerator in the public header."""
    src = open(os.path.join(ROOT, "include", "bmf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return {k: int(v) for k, v in re.findall(r"\b(BMF_[A-Z0-9_]+)\s*=\s*(\d+)", src)}


def test_binding_constants_match_the_header():
    from paper_1703_00734_gb300 import bmf
    enums = header_enums()
    for name in ("BMF_FP64", "BMF_FP32", "BMF_BF16", "BMF_TF32"):
        assert getattr(bmf, name) == enums[name], name
    assert bmf.PRECISION == {"fp64": enums["BMF_FP64"], "fp32": enums["BMF_FP32"],
                             "bf16": enums["BMF_BF16"], "tf32": enums["BMF_TF32"]}
    assert (bmf.FACTOR_X, bmf.FACTOR_W) == (enums["BMF_FACTOR_X"], enums["BMF_FACTOR_W"])
