"""Python binding of libtreepm: the TreePM gravitational force on active
particles (Weinberger, Springel & Pakmor, "The AREPO public code release",
Sec. 3) on a GB300 GPU.

This module only marshals arguments: every step of the force path runs in the
CUDA kernels of ``libtreepm.so`` behind the C ABI of ``include/treepm.h``.
PyTorch supplies device memory and the current stream.  The names follow the
C functions: ``build_tree``, ``pm_long_range``, ``compute_forces``,
``release``, ``tree_info``, ``tree_export``, ``pm_export``.

There is no CPU fallback: if the library is missing or cannot be loaded,
importing this module raises ``ImportError``.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import _build

__all__ = ["Context", "System", "Plan", "BuildParams", "ForceParams", "StepParams", "TreePMError", "lib_path",
           "CRIT_BH", "CRIT_RELATIVE", "BATCH_PRESORTED", "GRAD_FD4", "GRAD_IK"]

CRIT_BH = 0
CRIT_RELATIVE = 1
GRAD_FD4 = 0  # TPM_GRAD_FD4
GRAD_IK = 1   # TPM_GRAD_IK
NOALLOC_MAX_ACTIVE = 1 << 18  # TPM_NOALLOC_MAX_ACTIVE

_STATUS = {0: "TPM_OK", -1: "TPM_EINVAL", -2: "TPM_EBUDGET", -3: "TPM_ENOSYS_HANDLE", -4: "TPM_ECUDA",
           -5: "TPM_ETIMEDOUT", -6: "TPM_ENAN"}


class TreePMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class _BuildParams(C.Structure):
    _fields_ = [("G", C.c_double), ("h", C.c_double), ("periodic", C.c_int32), ("box", C.c_double),
                ("shift", C.c_double * 3), ("leaf_bucket", C.c_int32)]


class _ForceParams(C.Structure):
    _fields_ = [("crit", C.c_int32), ("theta", C.c_double), ("alpha", C.c_double), ("box_guard", C.c_int32),
                ("treepm", C.c_int32), ("pm_n", C.c_int32), ("asmth", C.c_double), ("rcut", C.c_double),
                ("pm_grad", C.c_int32), ("plain_fp32", C.c_int32)]


class _StepParams(C.Structure):
    _fields_ = [("dt_tick", C.c_double), ("nbins", C.c_int32), ("c_grav", C.c_double), ("eps", C.c_double)]


def lib_path() -> str:
    return _build.LIB


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError("libtreepm.so is not built (%s); run __graft_entry__.build() or "
                          "python -m paper_1909_04667_gb300._build" % path)
    try:
        lib = C.CDLL(path)
    except OSError as e:
        raise ImportError("cannot load %s: %s" % (path, e)) from e
    i32, i64, vp, sz = C.c_int, C.c_int64, C.c_void_p, C.c_size_t
    sig = {
        "tpm_version": (i32, []),
        "tpm_last_error": (C.c_char_p, []),
        "tpm_create": (i32, [C.POINTER(vp), i32, sz]),
        "tpm_destroy": (i32, [vp]),
        "tpm_memory": (i32, [vp, C.POINTER(sz), C.POINTER(sz)]),
        "tpm_build_tree": (i32, [vp, vp, vp, i64, C.POINTER(_BuildParams), vp, C.POINTER(C.c_uint64)]),
        "tpm_build_tree_soft": (i32, [vp, vp, vp, vp, i64, C.POINTER(_BuildParams), vp, C.POINTER(C.c_uint64)]),
        "tpm_pm_long_range": (i32, [vp, C.c_uint64, C.POINTER(_ForceParams), vp]),
        "tpm_compute_forces": (i32, [vp, C.c_uint64, vp, i64, vp, C.POINTER(_ForceParams), vp, vp, vp, vp]),
        "tpm_release": (i32, [vp, C.c_uint64]),
        "tpm_sync_status": (i32, [vp, C.c_uint64, vp]),
        "tpm_tree_info": (i32, [vp, C.c_uint64, C.POINTER(i64), C.POINTER(i64), vp, vp]),
        "tpm_tree_export": (i32, [vp, C.c_uint64] + [vp] * 10),
        "tpm_pm_export": (i32, [vp, C.c_uint64, vp, i64]),
        "tpm_launch_counts": (i32, [C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
        "tpm_compute_forces_noalloc": (i32, [vp, C.c_uint64, vp, i64, vp, C.POINTER(_ForceParams), vp, vp, vp,
                                             vp]),
        "tpm_plan_create": (i32, [vp, i64, i64, C.POINTER(vp)]),
        "tpm_plan_destroy": (i32, [vp, vp]),
        "tpm_plan_set_group_size": (i32, [vp, i32]),
        "tpm_plan_group_size": (i32, [vp]),
        "tpm_plan_set_stack_depth": (i32, [vp, i32]),
        "tpm_diagnostics": (i32, [vp, C.c_uint64, vp, vp, vp, vp, vp]),
        "tpm_plan_stack_depth": (i32, [vp]),
        "tpm_compute_forces_batch": (i32, [vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, C.c_uint32, vp]),
        "tpm_plan_sync_status": (i32, [vp, vp, vp]),
        "tpm_plan_autotune": (i32, [vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, C.c_uint32, i32, vp,
                                    C.POINTER(i32), C.POINTER(C.c_float)]),
        "tpm_drift": (i32, [vp, vp, vp, i64, C.c_double, C.c_int32, C.c_double, vp]),
        "tpm_active_set": (i32, [vp, vp, vp, i64, i64, C.c_int32, vp, vp, C.POINTER(i64), vp]),
        "tpm_kick": (i32, [vp, vp, i64, i64, vp, vp, vp, vp, i64, C.POINTER(_StepParams), C.c_int32, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def _check(status: int):
    if status != 0:
        raise TreePMError(status, _lib.tpm_last_error().decode(errors="replace"))


def _ptr(x):
    """Address of a torch tensor (host or device) or numpy array; None -> NULL."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(x))


def _stream(stream, device):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch

    return torch.cuda.current_stream(device).cuda_stream


@dataclass
class BuildParams:
    G: float = 1.0
    h: float = 0.01
    periodic: bool = False
    box: float = 1.0
    shift: tuple = (0.0, 0.0, 0.0)
    leaf_bucket: int = 8

    def _c(self):
        return _BuildParams(self.G, self.h, int(self.periodic), self.box, (C.c_double * 3)(*self.shift),
                            int(self.leaf_bucket))


@dataclass
class ForceParams:
    crit: int = CRIT_BH
    theta: float = 0.7
    alpha: float = 0.0025
    box_guard: bool = True
    treepm: bool = False
    pm_n: int = 256
    asmth: float = 1.25
    rcut: float = 4.5
    pm_grad: int = 0  # GRAD_FD4 or GRAD_IK (periodic systems)
    plain_fp32: bool = False  # the plain FP32 comparison arm (open boundaries)

    def _c(self):
        return _ForceParams(int(self.crit), self.theta, self.alpha, int(self.box_guard), int(self.treepm),
                            int(self.pm_n), self.asmth, self.rcut, int(self.pm_grad), int(self.plain_fp32))


@dataclass
class StepParams:
    """Time-bin hierarchy and step criterion (``tpm_step_params``)."""
    dt_tick: float = 1e-3
    nbins: int = 8
    c_grav: float = 0.025
    eps: float = 0.01 / 2.8

    def _c(self):
        return _StepParams(self.dt_tick, int(self.nbins), self.c_grav, self.eps)


def drift(ctx: "Context", pos, vel, dt: float, periodic: bool = False, box: float = 1.0, stream=None):
    """``tpm_drift``: pos += vel dt in place (n x 3 FP64 device tensors)."""
    _check(_lib.tpm_drift(ctx._h, _ptr(pos), _ptr(vel), int(pos.shape[0]), float(dt), int(periodic), float(box),
                          _stream(stream, ctx.device)))


def active_set(ctx: "Context", bins, tick: int, nbins: int, ids, amag=None, a_old=None, stream=None) -> int:
    """``tpm_active_set``: indices of the particles due at ``tick`` into ``ids``
    (and their previous |a| into ``a_old``); returns how many."""
    n = C.c_int64(0)
    _check(_lib.tpm_active_set(ctx._h, _ptr(bins), _ptr(amag), int(bins.shape[0]), int(tick), int(nbins), _ptr(ids),
                               _ptr(a_old), C.byref(n), _stream(stream, ctx.device)))
    return n.value


def kick(ctx: "Context", ids, n_active: int, acc, vel, bins, amag, tick: int, sp: StepParams, first: bool = False,
         stream=None):
    """``tpm_kick``: closing half kick, new bin, opening half kick for the
    particles ``ids[:n_active]`` with accelerations ``acc`` (ids order)."""
    cp = sp._c()
    _check(_lib.tpm_kick(ctx._h, _ptr(ids), int(n_active), int(vel.shape[0]), _ptr(acc), _ptr(vel), _ptr(bins),
                         _ptr(amag), int(tick), C.byref(cp), int(first), _stream(stream, ctx.device)))


BATCH_PRESORTED = 1


class Plan:
    """Scratch for batched evaluations (``tpm_plan_create``): many requests,
    on one or several resident systems, in one persistent walk launch.  A
    batched call allocates nothing and can be captured in a CUDA graph."""

    def __init__(self, ctx: "Context", max_ids: int, max_requests: int):
        h = C.c_void_p()
        _check(_lib.tpm_plan_create(ctx._h, int(max_ids), int(max_requests), C.byref(h)))
        self.ctx, self._h, self.max_ids, self.max_requests = ctx, h, int(max_ids), int(max_requests)
        self._keep = None

    def close(self):
        if getattr(self, "_h", None):
            _lib.tpm_plan_destroy(self.ctx._h, self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def group_size(self) -> int:
        return int(_lib.tpm_plan_group_size(self._h))

    @group_size.setter
    def group_size(self, g: int):
        _check(_lib.tpm_plan_set_group_size(self._h, int(g)))

    @property
    def stack_depth(self) -> int:
        """``tpm_plan_stack_depth``: the batched walk's candidate-stack capacity."""
        return int(_lib.tpm_plan_stack_depth(self._h))

    @stack_depth.setter
    def stack_depth(self, d: int):
        _check(_lib.tpm_plan_set_stack_depth(self._h, int(d)))

    def _args(self, systems, offsets, params):
        n_req = len(systems)
        sys_arr = (C.c_uint64 * n_req)(*[s.handle for s in systems])
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        if len(off) != n_req + 1:
            raise ValueError("offsets must have len(systems) + 1 entries")
        if isinstance(params, ForceParams):
            params = [params] * n_req
        par = (_ForceParams * n_req)(*[p._c() for p in params])
        self._keep = (sys_arr, off, par)  # the call copies them; keep them alive through it
        return n_req, sys_arr, off, par

    def compute_forces_batch(self, systems, offsets, params, ids, acc, a_old=None, pot=None, n_int=None,
                             presorted: bool = False, stream=None):
        """``tpm_compute_forces_batch``: request r covers ids[offsets[r]:offsets[r+1]]
        of ``systems[r]`` with ``params[r]`` (or one ForceParams for all).
        ids, a_old, acc, pot, n_int are device tensors indexed by position."""
        n_req, sys_arr, off, par = self._args(systems, offsets, params)
        _check(_lib.tpm_compute_forces_batch(self.ctx._h, self._h, n_req, sys_arr, off.ctypes.data, par, _ptr(ids),
                                             _ptr(a_old), _ptr(acc), _ptr(pot), _ptr(n_int),
                                             BATCH_PRESORTED if presorted else 0, _stream(stream, self.ctx.device)))
        return acc, pot, n_int

    def autotune(self, systems, offsets, params, ids, acc, a_old=None, pot=None, n_int=None, presorted=False,
                 reps: int = 3, stream=None):
        """``tpm_plan_autotune``: keeps the fastest group size; returns (G, ms)."""
        n_req, sys_arr, off, par = self._args(systems, offsets, params)
        g, ms = C.c_int(), C.c_float()
        _check(_lib.tpm_plan_autotune(self.ctx._h, self._h, n_req, sys_arr, off.ctypes.data, par, _ptr(ids),
                                      _ptr(a_old), _ptr(acc), _ptr(pot), _ptr(n_int),
                                      BATCH_PRESORTED if presorted else 0, int(reps),
                                      _stream(stream, self.ctx.device), C.byref(g), C.byref(ms)))
        return g.value, ms.value

    def sync_status(self, stream=None):
        _check(_lib.tpm_plan_sync_status(self.ctx._h, self._h, _stream(stream, self.ctx.device)))


class Context:
    """A libtreepm context on one CUDA device (``tpm_create``)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        h = C.c_void_p()
        _check(_lib.tpm_create(C.byref(h), int(device), int(budget_bytes)))
        self._h = h
        self.device = int(device)

    def close(self):
        if getattr(self, "_h", None):
            _lib.tpm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def memory(self):
        used, budget = C.c_size_t(), C.c_size_t()
        _check(_lib.tpm_memory(self._h, C.byref(used), C.byref(budget)))
        return used.value, budget.value

    def create_plan(self, max_ids: int, max_requests: int) -> Plan:
        return Plan(self, max_ids, max_requests)

    def build_tree(self, pos, mass, params: BuildParams, stream=None, hsoft=None) -> "System":
        """``tpm_build_tree``: pos (n, 3) float64, mass (n,) float32, on host or
        device; with ``hsoft`` (n,) float32 per-particle spline supports,
        ``tpm_build_tree_soft``."""
        n = int(pos.shape[0])
        if tuple(pos.shape) != (n, 3) or int(mass.shape[0]) != n:
            raise ValueError("pos must be (n, 3) and mass (n,)")
        _dtype_check(pos, "float64")
        _dtype_check(mass, "float32")
        out = C.c_uint64()
        cp = params._c()
        if hsoft is None:
            _check(_lib.tpm_build_tree(self._h, _ptr(pos), _ptr(mass), n, C.byref(cp), _stream(stream, self.device),
                                       C.byref(out)))
        else:
            if int(hsoft.shape[0]) != n:
                raise ValueError("hsoft must be (n,)")
            _dtype_check(hsoft, "float32")
            _check(_lib.tpm_build_tree_soft(self._h, _ptr(pos), _ptr(mass), _ptr(hsoft), n, C.byref(cp),
                                            _stream(stream, self.device), C.byref(out)))
        return System(self, out.value, n, params)


def _dtype_check(x, name):
    dt = str(x.dtype).replace("torch.", "")
    if dt != name:
        raise TypeError("expected %s, got %s" % (name, dt))


def _numel(x) -> int:
    return int(x.size) if isinstance(x, np.ndarray) else int(x.numel())


def _check_force_arrays(n_act, active_ids, a_old, acc, pot, n_int):
    """Types and sizes of a force call's arrays (the C ABI takes bare pointers,
    so an undersized output would be written past its end)."""
    if active_ids is not None and str(active_ids.dtype).replace("torch.", "") not in ("uint32", "int32"):
        raise TypeError("active_ids must be 32-bit indices, got %s" % active_ids.dtype)
    if a_old is not None:
        _dtype_check(a_old, "float32")
        if _numel(a_old) < n_act:
            raise ValueError("a_old holds %d values for %d active particles" % (_numel(a_old), n_act))
    if acc is None or tuple(acc.shape) != (n_act, 3):
        raise ValueError("acc must have shape (%d, 3)" % n_act)
    _dtype_check(acc, "float32")
    if pot is not None:
        _dtype_check(pot, "float32")
        if _numel(pot) < n_act:
            raise ValueError("pot holds %d values for %d active particles" % (_numel(pot), n_act))
    if n_int is not None:
        if str(n_int.dtype).replace("torch.", "") not in ("uint32", "int32"):
            raise TypeError("n_int must be 32-bit integers, got %s" % n_int.dtype)
        if _numel(n_int) < n_act:
            raise ValueError("n_int holds %d values for %d active particles" % (_numel(n_int), n_act))


class System:
    """A resident particle system (``tpm_sys``)."""

    def __init__(self, ctx: Context, handle: int, n: int, params: BuildParams):
        self.ctx, self.handle, self.n, self.params = ctx, handle, n, params

    def release(self):
        if self.handle:
            _check(_lib.tpm_release(self.ctx._h, self.handle))
            self.handle = 0

    def pm_long_range(self, fp: ForceParams, stream=None):
        cp = fp._c()
        _check(_lib.tpm_pm_long_range(self.ctx._h, self.handle, C.byref(cp), _stream(stream, self.ctx.device)))

    def compute_forces(self, active_ids=None, a_old=None, fp: ForceParams = None, acc=None, pot=None, n_int=None,
                       stream=None, want_pot=True, want_nint=True):
        """``tpm_compute_forces``.  Inputs and outputs may be torch tensors on
        the device or on the host (or numpy arrays).  Missing outputs are
        allocated on the device of the context as torch tensors."""
        import torch

        fp = fp or ForceParams()
        n_act = self.n if active_ids is None else int(active_ids.shape[0])
        dev = torch.device("cuda", self.ctx.device)
        if acc is None:
            acc = torch.empty((n_act, 3), dtype=torch.float32, device=dev)
        if pot is None and want_pot:
            pot = torch.empty(n_act, dtype=torch.float32, device=dev)
        if n_int is None and want_nint:
            n_int = torch.empty(n_act, dtype=torch.int32, device=dev)
        _check_force_arrays(n_act, active_ids, a_old, acc, pot, n_int)
        cp = fp._c()
        _check(_lib.tpm_compute_forces(self.ctx._h, self.handle, _ptr(active_ids), n_act, _ptr(a_old), C.byref(cp),
                                       _ptr(acc), _ptr(pot), _ptr(n_int), _stream(stream, self.ctx.device)))
        return acc, pot, n_int

    def compute_forces_noalloc(self, active_ids, acc, a_old=None, fp: ForceParams = None, pot=None, n_int=None,
                               stream=None):
        """``tpm_compute_forces_noalloc``: the same evaluation without any
        device allocation, for callers that cannot let the library allocate.
        Every array must already live on the device (the caller allocates
        acc, pot and n_int); at most ``NOALLOC_MAX_ACTIVE`` active particles."""
        fp = fp or ForceParams()
        n_act = int(active_ids.shape[0])
        _check_force_arrays(n_act, active_ids, a_old, acc, pot, n_int)
        cp = fp._c()
        _check(_lib.tpm_compute_forces_noalloc(self.ctx._h, self.handle, _ptr(active_ids), n_act, _ptr(a_old),
                                               C.byref(cp), _ptr(acc), _ptr(pot), _ptr(n_int),
                                               _stream(stream, self.ctx.device)))
        return acc, pot, n_int

    def diagnostics(self, acc, pot=None, vel=None, stream=None) -> dict:
        """``tpm_diagnostics``: FP64 total force, its scale sum m |a|, potential
        energy, and with velocities kinetic energy and momentum, over all
        particles (device tensors in the caller's order)."""
        out = np.zeros(9, np.float64)
        _check(_lib.tpm_diagnostics(self.ctx._h, self.handle, _ptr(acc), _ptr(pot), _ptr(vel), out.ctypes.data,
                                    _stream(stream, self.ctx.device)))
        return {"total_force": out[0:3].copy(), "potential_energy": float(out[3]), "kinetic_energy": float(out[4]),
                "momentum": out[5:8].copy(), "force_scale": float(out[8])}

    def sync_status(self, stream=None):
        """``tpm_sync_status``: wait for the stream and raise if device work
        recorded an error for this system."""
        _check(_lib.tpm_sync_status(self.ctx._h, self.handle, _stream(stream, self.ctx.device)))

    def tree_info(self):
        n, nn = C.c_int64(), C.c_int64()
        x0 = np.zeros(3)
        L0 = np.zeros(1)
        _check(_lib.tpm_tree_info(self.ctx._h, self.handle, C.byref(n), C.byref(nn), x0.ctypes.data,
                                  L0.ctypes.data))
        return dict(n=n.value, n_nodes=nn.value, x0=x0, L0=float(L0[0]))

    def tree_export(self) -> dict:
        info = self.tree_info()
        n, m = info["n"], info["n_nodes"]
        out = dict(key=np.zeros(n, np.uint64), perm=np.zeros(n, np.uint32), level=np.zeros(m, np.uint8),
                   prefix=np.zeros(m, np.uint64), first=np.zeros(m, np.uint32), count=np.zeros(m, np.uint32),
                   skip=np.zeros(m, np.uint32), mass=np.zeros(m), com=np.zeros((m, 3)), xtree=np.zeros((n, 3)))
        _check(_lib.tpm_tree_export(self.ctx._h, self.handle, *[out[k].ctypes.data for k in
                                                                ("key", "perm", "level", "prefix", "first", "count",
                                                                 "skip", "mass", "com", "xtree")]))
        out.update(info)
        return out

    def pm_export(self, mesh: int) -> np.ndarray:
        """``tpm_pm_export``: the potential mesh, ``mesh`` points per side (pm_n
        for a periodic system, 2 pm_n for the zero-padded mesh of an open one)."""
        phi = np.zeros(mesh ** 3, np.float32)
        _check(_lib.tpm_pm_export(self.ctx._h, self.handle, phi.ctypes.data, phi.size))
        return phi.reshape(mesh, mesh, mesh)


def launch_counts():
    """(own kernel launches, CUB primitive calls) since the library was loaded."""
    k, c = C.c_uint64(), C.c_uint64()
    _check(_lib.tpm_launch_counts(C.byref(k), C.byref(c)))
    return k.value, c.value


def version() -> int:
    return int(_lib.tpm_version())
