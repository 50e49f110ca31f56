"""Write the stored expected values of the water-cluster workloads (PBE-form
GGA, t_b = t_d = 1e-10) by calling only the CPU oracle.

Output: tests/golden/water<N>_pbe.json with the screened E_xc (and the dense
one for the 33-water workload), the trace tr(D V), a seeded sample of V
elements, and rho / grad rho on a seeded sample of grid blocks.  The oracle
runs on the host's cores: a process pool (spawn) fills the Becke weights in
chunks of points and evaluates ranges of grid blocks; the partial E_xc and
V of the ranges are summed in range order.  Run from the repository root:
    python tests/golden/make_golden.py            # 33 waters (1.15M points)
    python tests/golden/make_golden.py 100        # 100 waters (3.5M points, screened only)
"""
import json
import multiprocessing as mp
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

_W = {}


def _init(nwaters, points=None, weights=None):
    sys.path.insert(0, ROOT)
    s = synth.make_system(2, nwaters=nwaters)
    _W["s"] = s
    _W["sh"] = ob.build_shells(s.xyz, s.basis)
    if points is not None:
        g = og.build_grid(s.Z, s.xyz, s.grid, weight_blocks=[])
        g.weights[:] = weights
        _W["g"] = g


def _weights(args):
    pts, owner = args
    return og.becke_weights(pts, owner, _W["s"].xyz)


def _evaluate(args):
    blocks, screened, want_v = args
    r = oe.evaluate(_W["s"], _W["g"], _W["sh"], screened=screened, blocks=blocks, want_v=want_v)
    sl = slice(blocks[0] * 128, (blocks[-1] + 1) * 128)
    return r.E, (r.V if want_v else None), r.rho[sl], r.grad[sl]


def main(nwaters: int = 33, nproc: int = 0):
    t0 = time.time()
    nproc = nproc or os.cpu_count() or 1
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"      # one BLAS thread per worker process
    s = synth.make_system(2, nwaters=nwaters)
    g = og.build_grid(s.Z, s.xyz, s.grid, weight_blocks=[])
    ctx = mp.get_context("spawn")
    chunk = 20000
    jobs = [(g.points[i:min(i + chunk, g.nreal)], g.atom_of[i:min(i + chunk, g.nreal)])
            for i in range(0, g.nreal, chunk)]
    with ctx.Pool(nproc, initializer=_init, initargs=(nwaters,)) as pool:
        ws = pool.map(_weights, jobs)
    g.weights[:g.nreal] = g.raw_w[:g.nreal] * np.concatenate(ws)
    print(f"grid {g.npoints} points in {time.time() - t0:.0f} s", flush=True)
    span = -(-g.nblocks // (4 * nproc))
    ranges = [list(range(b, min(b + span, g.nblocks))) for b in range(0, g.nblocks, span)]
    rho = np.zeros(g.npoints)
    grad = np.zeros((g.npoints, 3))
    with ctx.Pool(nproc, initializer=_init, initargs=(nwaters, g.points, g.weights)) as pool:
        E = 0.0
        V = np.zeros((s.nbf, s.nbf))
        for blocks, (e, v, r, gr) in zip(ranges, pool.imap(_evaluate, [(b, True, True) for b in ranges])):
            E += e
            V += v
            sl = slice(blocks[0] * 128, (blocks[-1] + 1) * 128)
            rho[sl] = r
            grad[sl] = gr
        print(f"screened E {E:.12f} ({time.time() - t0:.0f} s)", flush=True)
        E_dense = None
        if nwaters == 33:
            E_dense = sum(e for e, _, _, _ in pool.imap(_evaluate, [(b, False, False) for b in ranges]))
            print(f"dense E {E_dense:.12f} ({time.time() - t0:.0f} s)", flush=True)
    rng = np.random.default_rng(7)
    n = s.nbf
    idx = rng.integers(0, n, size=(400, 2))
    blocks = sorted(rng.choice(g.nblocks, size=24, replace=False).tolist())
    pts = np.concatenate([np.arange(b * 128, (b + 1) * 128) for b in blocks])
    out = {
        "workload": f"{nwaters} waters, PBE-form GGA, {s.nbf} functions, t_b = t_d = 1e-10",
        "nbf": n, "npoints": int(g.npoints), "nblocks": int(g.nblocks),
        "E_screened": E, "E_dense": E_dense,
        "trace_DV": float(np.sum(s.D * V)),
        "V_samples": [[int(a), int(b), float(V[a, b])] for a, b in idx],
        "V_diag_max": float(np.abs(np.diag(V)).max()),
        "V_absmax": float(np.abs(V).max()),
        "rho_blocks": blocks,
        "rho": rho[pts].tolist(),
        "grad": grad[pts].tolist(),
    }
    path = os.path.join(ROOT, "tests", "golden", f"water{nwaters}_pbe.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(f"wrote {path} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 33)
