"""Write the stored expected values of the full-size water-cluster workload
(33 waters, PBE-form GGA, t_b = t_d = 1e-10) by calling only the CPU oracle.

Output: tests/golden/water33_pbe.json with the screened and dense E_xc, the
trace tr(D V), a seeded sample of V elements, and rho / grad rho on a seeded
sample of grid blocks.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import basis as ob  # noqa: E402
from oracle import exc as oe  # noqa: E402
from oracle import grid as og  # noqa: E402


def main():
    t0 = time.time()
    s = synth.make_system(2)
    g = og.build_grid(s.Z, s.xyz, s.grid)
    sh = ob.build_shells(s.xyz, s.basis)
    print(f"grid {g.npoints} points in {time.time() - t0:.0f} s", flush=True)
    scr = oe.evaluate(s, g, sh, screened=True)
    print(f"screened E {scr.E:.12f} ({time.time() - t0:.0f} s)", flush=True)
    den = oe.evaluate(s, g, sh, screened=False, want_v=False)
    print(f"dense E {den.E:.12f} ({time.time() - t0:.0f} s)", flush=True)
    rng = np.random.default_rng(7)
    n = s.nbf
    idx = rng.integers(0, n, size=(400, 2))
    blocks = sorted(rng.choice(g.nblocks, size=24, replace=False).tolist())
    pts = np.concatenate([np.arange(b * 128, (b + 1) * 128) for b in blocks])
    out = {
        "workload": "33 waters, PBE-form GGA, 825 functions, t_b = t_d = 1e-10",
        "nbf": n, "npoints": int(g.npoints), "nblocks": int(g.nblocks),
        "E_screened": scr.E, "E_dense": den.E,
        "trace_DV": float(np.sum(s.D * scr.V)),
        "V_samples": [[int(a), int(b), float(scr.V[a, b])] for a, b in idx],
        "V_diag_max": float(np.abs(np.diag(scr.V)).max()),
        "rho_blocks": blocks,
        "rho": scr.rho[pts].tolist(),
        "grad": scr.grad[pts].tolist(),
    }
    path = os.path.join(ROOT, "tests", "golden", "water33_pbe.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(f"wrote {path} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
