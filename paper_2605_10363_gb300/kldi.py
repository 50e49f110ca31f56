"""Thin ctypes binding of libkldi (include/kldi.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  The functions carry the C names without the
``kldi_`` prefix.  Arrays may be numpy arrays (host) or torch tensors (host or
CUDA); the library detects device pointers itself.  Importing this module
raises if the library has not been built -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkldi.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, EIO = 0, -1, -2, -3, -4, -5, -6
XC = {"lda_x": 1, "pbe": 2, "mlp": 3}
PREC = {"fp64": 0, "bf16x3": 1, "tf32x3": 2, "bf16x6": 3, "bf16x10": 4}
STAGES = ("dprep", "phi", "rho", "xc", "x", "v", "finish")
NSTAGES = len(STAGES)


class KldiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"kldi status {status}: {msg}")
        self.status = status


class Molecule(C.Structure):
    _fields_ = [("natm", C.c_int), ("Z", C.POINTER(C.c_int32)), ("xyz", C.POINTER(C.c_double))]


class Basis(C.Structure):
    _fields_ = [("nshell", C.c_int), ("atom", C.POINTER(C.c_int32)), ("l", C.POINTER(C.c_int32)),
                ("nprim", C.POINTER(C.c_int32)), ("exps", C.POINTER(C.c_double)),
                ("coefs", C.POINTER(C.c_double))]


class GridSpec(C.Structure):
    _fields_ = [("nrad", C.c_int), ("nregions", C.c_int), ("ntheta", C.POINTER(C.c_int32)), ("block", C.c_int)]


class Options(C.Structure):
    _fields_ = [("t_b", C.c_double), ("t_d", C.c_double), ("rho_min", C.c_double), ("prec", C.c_int),
                ("xc", C.c_int), ("stream", C.c_void_p), ("shell_order", C.c_void_p)]


class TrainOptions(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr0", C.c_double), ("lr1", C.c_double),
                ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double), ("rho_min", C.c_double),
                ("stream", C.c_void_p)]


MLP_NPARAMS = 4482


class Tuning(C.Structure):
    _fields_ = [("v_seg", C.c_int), ("rho_ntile", C.c_int), ("v_align", C.c_int)]


class PlanStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("nbf", "nbasis_blocks", "npoints", "nblocks", "retained",
                                          "pair_slots", "vtile_work", "workspace_bytes")]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libkldi.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i64p = C.c_void_p, C.POINTER(C.c_int64)
    sig = {
        "kldi_make_grid": (C.c_int, [C.POINTER(Molecule), C.POINTER(GridSpec), C.POINTER(vp)]),
        "kldi_order_shells": (C.c_int, [C.c_int, vp, vp, vp]),
        "kldi_grid_info": (C.c_int, [vp, i64p, i64p, i64p]),
        "kldi_grid_export": (C.c_int, [vp, vp, vp, vp]),
        "kldi_grid_save": (C.c_int, [vp, C.c_char_p]),
        "kldi_grid_load": (C.c_int, [C.c_char_p, C.POINTER(vp)]),
        "kldi_screen": (C.c_int, [vp, C.POINTER(Molecule), C.POINTER(Basis), C.POINTER(Options), C.POINTER(vp)]),
        "kldi_plan_info": (C.c_int, [vp, C.POINTER(PlanStats)]),
        "kldi_plan_export_lists": (C.c_int, [vp, vp, vp, vp]),
        "kldi_density": (C.c_int, [vp, vp, vp, vp]),
        "kldi_vxc": (C.c_int, [vp, C.c_int, vp, vp, vp, vp]),
        "kldi_exc": (C.c_int, [vp, C.c_int, vp, vp, vp]),
        "kldi_exc_batched": (C.c_int, [C.POINTER(vp), C.c_int, C.c_int, C.POINTER(vp), C.POINTER(vp), vp]),
        "kldi_exc_grad": (C.c_int, [vp, C.c_int, vp, vp, vp]),
        "kldi_plan_set_precision": (C.c_int, [vp, C.c_int]),
        "kldi_plan_set_wait_limit": (C.c_int, [vp, C.c_uint64]),
        "kldi_plan_set_withhold": (C.c_int, [vp, C.c_int64]),
        "kldi_selftest_wait": (C.c_int, [C.c_uint64, C.c_int, vp]),
        "kldi_plan_profile": (C.c_int, [vp, C.c_int]),
        "kldi_plan_stage_times": (C.c_int, [vp, vp, vp]),
        "kldi_exc_energy_noalloc": (C.c_int, [C.c_int, C.c_int64, vp, vp, vp, C.c_double, vp, vp]),
        "kldi_mlp_create": (C.c_int, [vp, vp, C.POINTER(vp)]),
        "kldi_mlp_get_params": (C.c_int, [vp, vp]),
        "kldi_mlp_get_state": (C.c_int, [vp, vp, i64p]),
        "kldi_mlp_set_state": (C.c_int, [vp, vp, C.c_int64]),
        "kldi_mlp_loss_grad": (C.c_int, [vp, vp, vp, C.c_int64, C.c_double, vp, vp]),
        "kldi_mlp_adam_step": (C.c_int, [vp, vp, C.c_double, C.c_double, C.c_double, C.c_double]),
        "kldi_mlp_train": (C.c_int, [vp, vp, vp, C.c_int64, C.POINTER(TrainOptions), vp]),
        "kldi_mlp_eval": (C.c_int, [vp, vp, vp, C.c_int64, C.c_double, vp, vp, vp, vp]),
        "kldi_plan_set_mlp": (C.c_int, [vp, vp]),
        "kldi_mlp_free": (None, [vp]),
        "kldi_workspace_create": (C.c_int, [C.c_int64, C.POINTER(vp)]),
        "kldi_workspace_free": (None, [vp]),
        "kldi_plan_set_workspace": (C.c_int, [vp, vp]),
        "kldi_plan_set_tuning": (C.c_int, [vp, C.POINTER(Tuning)]),
        "kldi_plan_set_block_range": (C.c_int, [vp, C.c_int64, C.c_int64]),
        "kldi_plan_get_tuning": (C.c_int, [vp, C.POINTER(Tuning)]),
        "kldi_plan_autotune": (C.c_int, [vp, C.c_int, vp, C.c_int, C.POINTER(Tuning), C.POINTER(C.c_double)]),
        "kldi_batch_create": (C.c_int, [C.POINTER(vp), C.c_int, C.c_int, C.POINTER(vp), C.POINTER(vp), vp, vp,
                                        C.POINTER(vp)]),
        "kldi_batch_launch": (C.c_int, [vp]),
        "kldi_batch_sync": (C.c_int, [vp]),
        "kldi_batch_free": (None, [vp]),
        "kldi_plan_free": (None, [vp]),
        "kldi_grid_free": (None, [vp]),
        "kldi_last_error": (C.c_char_p, []),
        "kldi_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


def _check(status):
    if status != OK:
        raise KldiError(status, LIB.kldi_last_error().decode())


def _ptr(a):
    """Address of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    raise TypeError(type(a))


class Grid:
    """Owning handle of a kldi_grid."""

    def __init__(self, handle):
        self.h = C.c_void_p(handle)
        n, r, b = C.c_int64(), C.c_int64(), C.c_int64()
        _check(LIB.kldi_grid_info(self.h, C.byref(n), C.byref(r), C.byref(b)))
        self.npoints, self.nreal, self.nblocks = n.value, r.value, b.value

    def export(self):
        xyz = np.empty((self.npoints, 3))
        w = np.empty(self.npoints)
        atom = np.empty(self.npoints, np.int32)
        _check(LIB.kldi_grid_export(self.h, _ptr(xyz), _ptr(w), _ptr(atom)))
        return xyz, w, atom

    def save(self, path):
        """Write the grid to a file (kldi_grid_save); load_grid reads it back."""
        _check(LIB.kldi_grid_save(self.h, os.fsencode(path)))

    def __del__(self):
        if getattr(self, "h", None) is not None and self.h.value:
            LIB.kldi_grid_free(self.h)
            self.h = None


def _molecule(Z, xyz):
    Z = np.ascontiguousarray(Z, np.int32)
    xyz = np.ascontiguousarray(xyz, np.float64)
    m = Molecule(len(Z), Z.ctypes.data_as(C.POINTER(C.c_int32)), xyz.ctypes.data_as(C.POINTER(C.c_double)))
    return m, (Z, xyz)


def order_shells(S, nfn):
    """Shell order by overlap signatures (kldi_order_shells): S the nbf x nbf
    overlap matrix, nfn the functions per shell; returns perm (position k holds
    old shell perm[k])."""
    S = np.ascontiguousarray(S, np.float64)
    nfn = np.ascontiguousarray(nfn, np.int32)
    if S.shape != (int(nfn.sum()), int(nfn.sum())):
        raise ValueError("S must be nbf x nbf with nbf = sum(nfn)")
    perm = np.zeros(nfn.size, np.int32)
    _check(LIB.kldi_order_shells(int(nfn.size), _ptr(nfn), _ptr(S), _ptr(perm)))
    return perm


def make_grid(Z, xyz, nrad, ntheta, block=128) -> Grid:
    m, keep = _molecule(Z, xyz)
    nt = np.ascontiguousarray(ntheta, np.int32)
    spec = GridSpec(int(nrad), len(nt), nt.ctypes.data_as(C.POINTER(C.c_int32)), int(block))
    h = C.c_void_p()
    _check(LIB.kldi_make_grid(C.byref(m), C.byref(spec), C.byref(h)))
    return Grid(h.value)


def load_mlp(path) -> "Mlp":
    """A learned functional from a checkpoint written by Mlp.save."""
    with np.load(path) as z:
        if set(z.files) != {"state", "step", "box"}:
            raise ValueError(f"{path}: not a learned-functional checkpoint")
        state = np.asarray(z["state"], np.float32)
        step = int(z["step"])
        box = np.asarray(z["box"], np.float64)
    if state.shape != (3 * MLP_NPARAMS,) or box.shape != (4,) or step < 0:
        raise ValueError(f"{path}: not a learned-functional checkpoint")
    net = Mlp(state[:MLP_NPARAMS], box)
    net.set_state(state, step)
    return net


def load_grid(path) -> Grid:
    """A grid saved by Grid.save (kldi_grid_load)."""
    h = C.c_void_p()
    _check(LIB.kldi_grid_load(os.fsencode(path), C.byref(h)))
    return Grid(h.value)


class Plan:
    """Owning handle of a kldi_plan (the grid is kept alive with it)."""

    def __init__(self, handle, grid, keep):
        self.h = C.c_void_p(handle)
        self.grid = grid
        self._keep = keep
        s = PlanStats()
        _check(LIB.kldi_plan_info(self.h, C.byref(s)))
        self.stats = {n: getattr(s, n) for n, _ in PlanStats._fields_}
        self.nbf = self.stats["nbf"]
        self.npoints = self.stats["npoints"]

    def lists(self):
        nblk = self.stats["nblocks"]
        nt = self.stats["retained"]
        ptr = np.empty(nblk + 1, np.int32)
        idx = np.empty(nt, np.int32)
        b = np.empty(nt)
        _check(LIB.kldi_plan_export_lists(self.h, _ptr(ptr), _ptr(idx), _ptr(b)))
        return ptr, idx, b

    def profile(self, enable=True):
        _check(LIB.kldi_plan_profile(self.h, int(enable)))

    def stage_times(self):
        """(ms[7], launches[7]) per stage since profile(True)."""
        ms = np.zeros(NSTAGES)
        n = np.zeros(NSTAGES, np.int64)
        _check(LIB.kldi_plan_stage_times(self.h, _ptr(ms), _ptr(n)))
        return ms, n

    def set_workspace(self, ws):
        _check(LIB.kldi_plan_set_workspace(self.h, ws.h if ws is not None else None))
        self._ws = ws               # the workspace must outlive its use by the plan

    def set_block_range(self, g0, g1):
        """Evaluate only grid blocks [g0, g1) (partial E_xc and V)."""
        _check(LIB.kldi_plan_set_block_range(self.h, int(g0), int(g1)))

    def set_tuning(self, v_seg=0, rho_ntile=0, v_align=0):
        t = Tuning(int(v_seg), int(rho_ntile), int(v_align))
        _check(LIB.kldi_plan_set_tuning(self.h, C.byref(t)))

    def tuning(self):
        t = Tuning()
        _check(LIB.kldi_plan_get_tuning(self.h, C.byref(t)))
        return {"v_seg": t.v_seg, "rho_ntile": t.rho_ntile, "v_align": t.v_align}

    def autotune(self, xc, D, reps=3):
        """Tune on a device density matrix; returns (tuning, ms per call)."""
        t = Tuning()
        ms = C.c_double()
        _check(LIB.kldi_plan_autotune(self.h, XC[xc] if isinstance(xc, str) else int(xc), _ptr(D), int(reps),
                                      C.byref(t), C.byref(ms)))
        return {"v_seg": t.v_seg, "rho_ntile": t.rho_ntile, "v_align": t.v_align}, ms.value

    def set_precision(self, prec):
        _check(LIB.kldi_plan_set_precision(self.h, PREC[prec] if isinstance(prec, str) else int(prec)))

    def set_wait_limit(self, ns):
        """Bounded device waits give up after ns nanoseconds (0: the default 2 s)."""
        _check(LIB.kldi_plan_set_wait_limit(self.h, int(ns)))

    def set_withhold(self, item):
        """Test hook: the V product withholds work item `item` (-1: off)."""
        _check(LIB.kldi_plan_set_withhold(self.h, int(item)))

    def __del__(self):
        if getattr(self, "h", None) is not None and self.h.value:
            LIB.kldi_plan_free(self.h)
            self.h = None


def screen(grid: Grid, Z, xyz, shells_atom, shells_l, shells_nprim, exps, coefs, t_b, t_d,
           rho_min=1e-14, prec="bf16x3", xc="pbe", stream=0, shell_order=None) -> Plan:
    m, keepm = _molecule(Z, xyz)
    arrs = [np.ascontiguousarray(a, np.int32) for a in (shells_atom, shells_l, shells_nprim)]
    ex = np.ascontiguousarray(exps, np.float64)
    co = np.ascontiguousarray(coefs, np.float64)
    b = Basis(len(arrs[0]), *[a.ctypes.data_as(C.POINTER(C.c_int32)) for a in arrs],
              ex.ctypes.data_as(C.POINTER(C.c_double)), co.ctypes.data_as(C.POINTER(C.c_double)))
    order = None if shell_order is None else np.ascontiguousarray(shell_order, np.int32)
    opt = Options(float(t_b), float(t_d), float(rho_min), PREC[prec] if isinstance(prec, str) else int(prec),
                  XC[xc] if isinstance(xc, str) else int(xc), C.c_void_p(int(stream)),
                  C.c_void_p(None if order is None else order.ctypes.data))
    h = C.c_void_p()
    _check(LIB.kldi_screen(grid.h, C.byref(m), C.byref(b), C.byref(opt), C.byref(h)))
    return Plan(h.value, grid, (keepm, arrs, ex, co))


def density(plan: Plan, D, rho, grad=None):
    _check(LIB.kldi_density(plan.h, _ptr(D), _ptr(rho), _ptr(grad)))


def vxc(plan: Plan, xc, rho, grad, V, Exc):
    _check(LIB.kldi_vxc(plan.h, XC[xc] if isinstance(xc, str) else int(xc), _ptr(rho), _ptr(grad), _ptr(V),
                        _ptr(Exc)))


def exc(plan: Plan, xc, D, V, Exc):
    _check(LIB.kldi_exc(plan.h, XC[xc] if isinstance(xc, str) else int(xc), _ptr(D), _ptr(V), _ptr(Exc)))


def exc_grad(plan: Plan, xc, D, G, Exc):
    """Nuclear gradient G[natm, 3] of E_xc on the fixed grid (FP64 plans)."""
    _check(LIB.kldi_exc_grad(plan.h, XC[xc] if isinstance(xc, str) else int(xc), _ptr(D), _ptr(G), _ptr(Exc)))


def exc_batched(plans, xc, Ds, Vs, Exc):
    n = len(plans)
    ph = (C.c_void_p * n)(*[p.h.value for p in plans])
    dh = (C.c_void_p * n)(*[_ptr(d) for d in Ds])
    vh = (C.c_void_p * n)(*[_ptr(v) for v in Vs])
    _check(LIB.kldi_exc_batched(ph, n, XC[xc] if isinstance(xc, str) else int(xc), dh, vh, _ptr(Exc)))


def exc_energy_noalloc(xc, npoints, rho, grad, w, Exc, rho_min=1e-14, stream=0):
    """E_xc of a device-resident density with no allocation (kldi_exc_energy_noalloc)."""
    _check(LIB.kldi_exc_energy_noalloc(XC[xc] if isinstance(xc, str) else int(xc), int(npoints), _ptr(rho),
                                       _ptr(grad), _ptr(w), float(rho_min), _ptr(Exc), C.c_void_p(int(stream))))


class Workspace:
    """Shared device arena for the per-tile buffers of several plans."""

    def __init__(self, nbytes):
        h = C.c_void_p()
        _check(LIB.kldi_workspace_create(int(nbytes), C.byref(h)))
        self.h = h
        self.nbytes = int(nbytes)

    def __del__(self):
        if getattr(self, "h", None) is not None and self.h.value:
            LIB.kldi_workspace_free(self.h)
            self.h = None


class Batch:
    """All frames' evaluations captured into one CUDA graph (device arrays)."""

    def __init__(self, plans, xc, Ds, Vs, Exc, stream=0):
        n = len(plans)
        self._keep = (list(plans), list(Ds), list(Vs), Exc)
        ph = (C.c_void_p * n)(*[p.h.value for p in plans])
        dh = (C.c_void_p * n)(*[_ptr(d) for d in Ds])
        vh = (C.c_void_p * n)(*[_ptr(v) for v in Vs])
        h = C.c_void_p()
        _check(LIB.kldi_batch_create(ph, n, XC[xc] if isinstance(xc, str) else int(xc), dh, vh, _ptr(Exc),
                                     C.c_void_p(int(stream)), C.byref(h)))
        self.h = h

    def launch(self):
        _check(LIB.kldi_batch_launch(self.h))

    def sync(self):
        _check(LIB.kldi_batch_sync(self.h))

    def __del__(self):
        if getattr(self, "h", None) is not None and self.h.value:
            LIB.kldi_batch_free(self.h)
            self.h = None


class Mlp:
    """Owning handle of a kldi_mlp (the learned functional)."""

    def __init__(self, params, box):
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == MLP_NPARAMS
        self.box = np.ascontiguousarray(box, np.float64)
        h = C.c_void_p()
        _check(LIB.kldi_mlp_create(_ptr(p), _ptr(self.box), C.byref(h)))
        self.h = h

    def params(self):
        out = np.empty(MLP_NPARAMS, np.float32)
        _check(LIB.kldi_mlp_get_params(self.h, _ptr(out)))
        return out

    def state(self):
        """Training checkpoint: (parameters, Adam moments m and v stacked, step)."""
        out = np.empty(3 * MLP_NPARAMS, np.float32)
        step = C.c_int64()
        _check(LIB.kldi_mlp_get_state(self.h, _ptr(out), C.byref(step)))
        return out, int(step.value)

    def set_state(self, state, step):
        s = np.ascontiguousarray(state, np.float32)
        assert s.size == 3 * MLP_NPARAMS
        _check(LIB.kldi_mlp_set_state(self.h, _ptr(s), int(step)))

    def save(self, path):
        """Training checkpoint file (.npz): parameters, Adam moments, step
        counter and training box; load_mlp restores a network whose training
        continues bit for bit."""
        state, step = self.state()
        np.savez(path, state=state, step=np.int64(step), box=self.box)

    def loss_grad(self, rho, sigma, rho_min=1e-14):
        rho = np.ascontiguousarray(rho, np.float64) if isinstance(rho, np.ndarray) else rho
        sigma = np.ascontiguousarray(sigma, np.float64) if isinstance(sigma, np.ndarray) else sigma
        g = np.empty(MLP_NPARAMS, np.float32)
        loss = np.empty(1, np.float32)
        _check(LIB.kldi_mlp_loss_grad(self.h, _ptr(rho), _ptr(sigma), int(len(rho)), float(rho_min), _ptr(g),
                                      _ptr(loss)))
        return float(loss[0]), g

    def adam_step(self, grad, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        g = np.ascontiguousarray(grad, np.float32) if isinstance(grad, np.ndarray) else grad
        _check(LIB.kldi_mlp_adam_step(self.h, _ptr(g), float(lr), float(beta1), float(beta2), float(eps)))

    def train(self, rho, sigma, epochs, batch=8192, lr0=3e-3, lr1=3e-5, beta1=0.9, beta2=0.999, eps=1e-8,
              rho_min=1e-14, stream=0):
        """GPU training; returns the mean batch loss of each epoch."""
        rho = np.ascontiguousarray(rho, np.float64) if isinstance(rho, np.ndarray) else rho
        sigma = np.ascontiguousarray(sigma, np.float64) if isinstance(sigma, np.ndarray) else sigma
        opt = TrainOptions(int(epochs), int(batch), float(lr0), float(lr1), float(beta1), float(beta2), float(eps),
                           float(rho_min), C.c_void_p(int(stream)))
        hist = np.zeros(int(epochs), np.float32)
        _check(LIB.kldi_mlp_train(self.h, _ptr(rho), _ptr(sigma), int(len(rho)), C.byref(opt), _ptr(hist)))
        return hist

    def eval(self, rho, sigma, rho_min=1e-14):
        """(f, v_rho, v_sigma, used) at the points (host arrays)."""
        rho = np.ascontiguousarray(rho, np.float64)
        sigma = np.ascontiguousarray(sigma, np.float64)
        n = rho.size
        f, vr, vs = np.empty(n), np.empty(n), np.empty(n)
        used = np.empty(n, np.int32)
        _check(LIB.kldi_mlp_eval(self.h, _ptr(rho), _ptr(sigma), n, float(rho_min), _ptr(f), _ptr(vr), _ptr(vs),
                                 _ptr(used)))
        return f, vr, vs, used.astype(bool)

    def __del__(self):
        if getattr(self, "h", None) is not None and self.h.value:
            LIB.kldi_mlp_free(self.h)
            self.h = None


def plan_set_mlp(plan: Plan, mlp):
    _check(LIB.kldi_plan_set_mlp(plan.h, mlp.h if mlp is not None else None))
    plan._mlp = mlp            # keep the network alive as long as the plan uses it


def selftest_wait(limit_ns, arrive, stream=0):
    """One CTA waits limit_ns on an mbarrier; raises KldiError(ETIMEOUT) when
    nothing arrives (arrive=False)."""
    _check(LIB.kldi_selftest_wait(int(limit_ns), int(bool(arrive)), C.c_void_p(stream)))


def version() -> str:
    return LIB.kldi_version().decode()


# ----------------------------------------------------------------------------
# convenience: build grid + plan for a ``synth.System``
def plan_for_system(system, prec="bf16x3", xc=None, stream=0, rho_min=1e-14, shell_order=None, grid=None):
    """Grid (built here unless a Grid, e.g. from load_grid, is given) and plan
    of a synthetic system."""
    g = grid if grid is not None else make_grid(system.Z, system.xyz, system.grid.nrad, system.grid.ntheta,
                                                system.grid.block)
    b = system.basis
    return screen(g, system.Z, system.xyz, b.atom, b.l, b.nprim, b.exps, b.coefs, system.t_b, system.t_d,
                  rho_min=rho_min, prec=prec, xc=xc or system.xc, stream=stream, shell_order=shell_order)
