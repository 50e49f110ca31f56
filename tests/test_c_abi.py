"""The C ABI called from a C program (tests/c_abi/abi_smoke.c), compiled with
the system C compiler against include/kldi.h and the in-tree libkldi.so."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PKG = os.path.join(ROOT, "paper_2605_10363_gb300")

Z = np.array([8, 1, 1], np.int32)
XYZ = np.array([[0.0, 0.0, 0.0], [1.43, 1.11, 0.0], [-1.43, 1.11, 0.0]])


def _run(tmp_path, *args):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    if not os.path.exists(os.path.join(PKG, "libkldi.so")):
        pytest.skip("libkldi.so is not built")
    exe = str(tmp_path / "abi_smoke")
    subprocess.run([cc, "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(HERE, "c_abi", "abi_smoke.c"), "-L", PKG, "-lkldi", f"-Wl,-rpath,{PKG}", "-lm",
                    "-o", exe], check=True)
    r = subprocess.run([exe, str(tmp_path / "water.grid"), *args], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    out = {}
    for line in r.stdout.splitlines():
        key, *vals = line.split()
        out[key] = vals if key != "exc" else out.get("exc", []) + [vals]
    assert "ok" in out
    return out


def test_c_program_host_calls(tmp_path):
    from oracle import reorder as orr
    from paper_2605_10363_gb300 import kldi
    out = _run(tmp_path)
    g = kldi.make_grid(Z, XYZ, 40, [6])
    assert [int(v) for v in out["grid"]] == [g.npoints, g.nreal, g.nblocks]
    assert out["reload"] == ["same", str(kldi.EIO)]
    assert out["mismatch"] == [str(kldi.EINVAL)]
    for v in out["gauss"]:            # a Gaussian of integral pi^(3/2) on each atom
        assert abs(float(v) - math.pi ** 1.5) <= 1e-2
    S = np.eye(7)
    S[0, 1] = S[1, 0] = 0.3
    S[5, 6] = S[6, 5] = 0.2
    assert [int(v) for v in out["order"]] == orr.order_shells(S, [1, 1, 3, 1, 1]).tolist()


@pytest.mark.gpu
def test_c_program_energy(tmp_path):
    from paper_2605_10363_gb300 import kldi
    out = _run(tmp_path, "--gpu")
    rows = {int(r[0]): (float(r[1]), float(r[2]), float(r[3])) for r in out["exc"]}
    e64, asym64, v00 = rows[kldi.PREC["fp64"]]
    e6, asym6, _ = rows[kldi.PREC["bf16x6"]]
    assert asym64 == 0.0 and asym6 == 0.0
    assert abs(e6 - e64) <= 1e-6
    # the same system through the Python binding
    g = kldi.make_grid(Z, XYZ, 40, [6])
    plan = kldi.screen(g, Z, XYZ, [0, 0, 0, 1, 2], [0, 0, 1, 0, 0], [1] * 5, [5.0, 0.5, 0.8, 1.0, 1.0], [1.0] * 5,
                       1e-12, 1e-12, prec="fp64", xc="lda_x")
    D = 0.4 * np.eye(7)
    D[0, 1] = D[1, 0] = 0.1
    V = np.zeros((7, 7))
    E = np.zeros(1)
    kldi.exc(plan, "lda_x", D, V, E)
    assert abs(E[0] - e64) <= 1e-12 * abs(e64) and abs(V[0, 0] - v00) <= 1e-12 * abs(v00)
