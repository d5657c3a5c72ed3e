"""The boundary from plain C: tests/c_abi_pp.c includes only bmf.h, builds with gcc as strict
C99, links against libbmf.so and runs posterior propagation on a 2 x 2 grid (Algorithm 1,
Eq. 14).  On a GPU its aggregated means and predictions must equal, bit for bit, those of the
Python binding on the same data (both call the same library with the same device-generator
seed, and every kernel reduces in a fixed order)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1703_00734_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi_pp.c")

K, I, J, SWEEPS, BURNIN, SEED = 5, 2, 2, 9, 2, 7


def _cuda_libdir():
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
              "/usr/local/cuda/targets/x86_64-linux/lib"):
        if os.path.isdir(d):
            return d
    return None


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_1703_00734_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path_factory.mktemp("cabi") / "c_abi_pp")
    cmd = ["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-O2",
           "-I", os.path.join(ROOT, "include"), SRC, "-o", exe,
           "-L", libdir, "-lbmf", "-Wl,-rpath," + libdir]
    cu = _cuda_libdir()
    if cu:
        cmd.append("-Wl,-rpath-link," + cu)
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def _workload():
    return synth.make_workload(None, N=260, D=180, M=7000, pattern="zipf", K=K, sigma=0.5,
                               tau=4.0, seed=11, s_row=1.1, s_col=1.1)


def _write_input(path, d):
    with open(path, "wb") as f:
        hdr = [d["N"], d["D"], len(d["row"]), len(d["test_row"]), K, I, J, SWEEPS, BURNIN, SEED]
        f.write(np.asarray(hdr, dtype="<i8").tobytes())
        f.write(np.asarray([d["tau"]], dtype="<f8").tobytes())
        for key, dt in (("row", "<i4"), ("col", "<i4"), ("val", "<f8"), ("X0", "<f8"),
                        ("W0", "<f8"), ("test_row", "<i4"), ("test_col", "<i4"),
                        ("test_val", "<f8")):
            f.write(np.ascontiguousarray(d[key], dtype=dt).tobytes())


def test_c_client_builds_as_strict_c99(client):
    assert os.access(client, os.X_OK)


def test_header_compiles_as_cxx(tmp_path):
    """bmf.h is also usable from C++ (extern "C" linkage, no C-only constructs)."""
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    src = tmp_path / "use.cpp"
    src.write_text('#include "bmf.h"\nint main() { bmf_config c{}; c.K = 4; '
                   'return bmf_last_error(nullptr) == nullptr && c.K != 4; }\n')
    r = subprocess.run(["g++", "-std=c++11", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.gpu
def test_c_client_matches_python_binding(client, tmp_path):
    from paper_1703_00734_gb300 import bmf
    d = _workload()
    inp, out = tmp_path / "in.bin", tmp_path / "out.bin"
    _write_input(inp, d)
    r = subprocess.run([client, str(inp), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c abi ok" in r.stdout
    raw = out.read_bytes()
    n_corr = int(np.frombuffer(raw[:8], dtype="<i8")[0])
    body = np.frombuffer(raw[8:], dtype="<f8")
    N, D, T = d["N"], d["D"], len(d["test_row"])
    rmse_c = body[0]
    Xc = body[1:1 + N * K].reshape(N, K)
    Wc = body[1 + N * K:1 + (N + D) * K].reshape(D, K)
    yc = body[1 + (N + D) * K:]
    assert yc.shape == (T,)

    m = bmf.BMF(N, D, d["row"], d["col"], d["val"], K, d["tau"], "fp64", I=I, J=J,
                X0=d["X0"], W0=d["W0"], test=(d["test_row"], d["test_col"], d["test_val"]),
                burnin=BURNIN, seed=SEED)
    for s in (1, 2, 3):
        m.stage(s, SWEEPS)
    Xm, Wm, nc = m.posterior_means()
    yhat, rmse = m.predict(d["test_row"], d["test_col"], d["test_val"])
    m.close()
    np.testing.assert_array_equal(Xc, Xm)
    np.testing.assert_array_equal(Wc, Wm)
    np.testing.assert_array_equal(yc, yhat)
    assert n_corr == nc and rmse_c == rmse
    # the propagated model predicts held-out entries far better than the training mean
    base = np.sqrt(np.mean((d["test_val"] - d["val"].mean()) ** 2))
    assert np.isfinite(rmse) and rmse < 0.8 * base
