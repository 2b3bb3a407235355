"""CPU oracle for the TreePM gravity force path (FP64).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this
package; the library under ``paper_1909_04667_gb300`` never does, and this
package never imports it.  The two share only the seeded generators in
``workloads``.

Pieces (paper section in brackets):

* ``kforce`` / ``kpot``          spline softening, Newtonian beyond h   [Sec. 3.2]
* ``gshort_force`` / ``gshort_pot`` short-range split factors             [Sec. 3.4]
* ``direct``                     softened O(N^2) sum, open boundaries   [Sec. 3]
* ``Tree``                       key-prefix oct-tree, monopoles, walk    [Sec. 3.1, 3.4]
* ``ewald``                      periodic exact force (Ewald)            [Sec. 2.2, 3.1]
* ``pm_potential`` / ``pm_interpolate``  periodic PM long-range part      [Sec. 3.3, 3.4]
* ``insertion_tree``             the paper's one-by-one insertion build
                                 (brute force, for pinning the node set) [Sec. 3.1]
* ``diagnostics``                total force, energies, momentum (FP64
                                 sums as written)                        [Sec. 7]

The C part (``treepm_oracle.c``) is compiled with gcc by ``build()``; the PM
part is numpy with ``numpy.fft`` as the FFT step.  Every function is pinned by
the CPU tests against closed forms, quadrature, brute force or invariants.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "treepm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXLEVEL = 21


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP on)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class WalkParams(C.Structure):
    _fields_ = [("G", C.c_double), ("h", C.c_double), ("crit", C.c_int), ("theta", C.c_double),
                ("alpha", C.c_double), ("box_guard", C.c_int), ("treepm", C.c_int), ("rs", C.c_double),
                ("rcut", C.c_double), ("ewald", C.c_int), ("etab", C.c_void_p), ("ent", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i64, vp = C.c_double, C.c_int64, C.c_void_p
            lib.orc_kforce.restype = d
            lib.orc_kforce.argtypes = [d, d]
            lib.orc_kpot.restype = d
            lib.orc_kpot.argtypes = [d, d]
            lib.orc_gshort_force.restype = d
            lib.orc_gshort_force.argtypes = [d, d]
            lib.orc_gshort_pot.restype = d
            lib.orc_gshort_pot.argtypes = [d, d]
            lib.orc_direct.restype = None
            lib.orc_direct.argtypes = [i64, vp, vp, i64, vp, d, d, vp, vp, C.c_int]
            lib.orc_tree_build.restype = vp
            lib.orc_tree_build.argtypes = [i64, vp, vp, C.c_int, d, vp, C.c_int]
            lib.orc_tree_free.restype = None
            lib.orc_tree_free.argtypes = [vp]
            lib.orc_tree_nnodes.restype = i64
            lib.orc_tree_nnodes.argtypes = [vp]
            lib.orc_tree_root.restype = None
            lib.orc_tree_root.argtypes = [vp, vp, vp]
            lib.orc_tree_export.restype = None
            lib.orc_tree_export.argtypes = [vp] + [vp] * 10
            lib.orc_tree_walk.restype = None
            lib.orc_tree_walk.argtypes = [vp, i64, vp, vp, C.POINTER(WalkParams), vp, vp, vp, C.c_int]
            lib.orc_ewald.restype = None
            lib.orc_ewald.argtypes = [i64, vp, vp, i64, vp, d, d, d, d, C.c_int, vp, vp, C.c_int]
            lib.orc_direct_soft.restype = None
            lib.orc_direct_soft.argtypes = [i64, vp, vp, vp, i64, vp, d, vp, vp, C.c_int]
            lib.orc_tree_set_soft.restype = None
            lib.orc_tree_set_soft.argtypes = [vp, vp]
            lib.orc_ewald_correction.restype = None
            lib.orc_ewald_correction.argtypes = [d, d, d, d, vp]
            lib.orc_ewald_table.restype = None
            lib.orc_ewald_table.argtypes = [d, C.c_int, vp, C.c_int]
            lib.orc_num_threads.restype = C.c_int
            lib.orc_num_threads.argtypes = []
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(_load().orc_num_threads())


# ---------------------------------------------------------------- kernels
def kforce(r: float, h: float) -> float:
    """Spline-softened force factor: a = -G m (x_i - x_j) kforce(r)."""
    return _load().orc_kforce(float(r), float(h))


def kpot(r: float, h: float) -> float:
    """Spline-softened potential factor: phi = G m kpot(r)."""
    return _load().orc_kpot(float(r), float(h))


def gshort_force(r: float, rs: float) -> float:
    return _load().orc_gshort_force(float(r), float(rs))


def gshort_pot(r: float, rs: float) -> float:
    return _load().orc_gshort_pot(float(r), float(rs))


# ---------------------------------------------------------------- direct sum
def direct_soft(pos, mass, hsoft, targets, G: float, nthreads: int = 0):
    """FP64 direct sum with per-particle spline supports ``hsoft``; a pair
    interacts with the larger of its two supports (Sec. 3.2)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float32)
    hsoft = np.ascontiguousarray(hsoft, dtype=np.float32)
    targets = np.ascontiguousarray(targets, dtype=np.uint32)
    acc = np.zeros((len(targets), 3))
    pot = np.zeros(len(targets))
    _load().orc_direct_soft(len(pos), _p(pos), _p(mass), _p(hsoft), len(targets), _p(targets), G, _p(acc), _p(pot),
                            nthreads)
    return acc, pot


def direct(pos, mass, targets, G: float, h: float, nthreads: int = 0):
    """Softened FP64 direct sum on ``targets`` (open boundaries)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float32)
    targets = np.ascontiguousarray(targets, dtype=np.uint32)
    acc = np.zeros((len(targets), 3))
    pot = np.zeros(len(targets))
    _load().orc_direct(len(pos), _p(pos), _p(mass), len(targets), _p(targets), G, h, _p(acc), _p(pot), nthreads)
    return acc, pot


# ---------------------------------------------------------------- tree
class Tree:
    """Key-prefix oct-tree of the oracle (FP64 monopoles), pre-order nodes."""

    def __init__(self, pos, mass, bucket: int = 1, periodic: bool = False, box: float = 1.0, shift=(0.0, 0.0, 0.0),
                 hsoft=None):
        """``hsoft``: per-particle spline supports (Sec. 3.2), else the walk's
        uniform ``h``."""
        self._lib = _load()
        self.pos = np.ascontiguousarray(pos, dtype=np.float64)
        self.mass = np.ascontiguousarray(mass, dtype=np.float32)
        self.hsoft = None if hsoft is None else np.ascontiguousarray(hsoft, dtype=np.float32)
        self.n = len(self.pos)
        self.bucket = int(bucket)
        self.periodic = bool(periodic)
        self.box = float(box)
        sh = np.ascontiguousarray(shift, dtype=np.float64)
        self._h = self._lib.orc_tree_build(self.n, _p(self.pos), _p(self.mass), int(periodic), float(box), _p(sh),
                                           self.bucket)
        if not self._h:
            raise ValueError("oracle tree build rejected its arguments")
        self.nnodes = int(self._lib.orc_tree_nnodes(self._h))
        x0 = np.zeros(3)
        L0 = np.zeros(1)
        self._lib.orc_tree_root(self._h, _p(x0), _p(L0))
        self.x0, self.L0 = x0, float(L0[0])
        if self.hsoft is not None:
            self._lib.orc_tree_set_soft(self._h, _p(self.hsoft))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_tree_free(h)
            self._h = None

    def export(self) -> dict:
        n, m = self.n, self.nnodes
        out = dict(key=np.zeros(n, np.uint64), perm=np.zeros(n, np.uint32), level=np.zeros(m, np.uint8),
                   prefix=np.zeros(m, np.uint64), first=np.zeros(m, np.uint32), count=np.zeros(m, np.uint32),
                   skip=np.zeros(m, np.uint32), mass=np.zeros(m), com=np.zeros((m, 3)), xtree=np.zeros((n, 3)))
        self._lib.orc_tree_export(self._h, *[_p(out[k]) for k in
                                             ("key", "perm", "level", "prefix", "first", "count", "skip", "mass",
                                              "com", "xtree")])
        return out

    def walk(self, targets, G: float, h: float, crit: str = "bh", theta: float = 0.7, alpha: float = 0.0025,
             a_old=None, box_guard: bool = True, treepm: bool = False, rs: float = 0.0, rcut: float = 0.0,
             ewald: bool = False, ewald_nt: int = 64, nthreads: int = 0):
        """Per-particle walk for ``targets`` (original indices).  Returns
        (acc (k,3), pot (k,), n_int (k,)) in FP64 / uint32.  With ``ewald`` (a
        periodic tree without ``treepm``) every term gets the Ewald correction
        interpolated from ``ewald_table(box, ewald_nt)``."""
        targets = np.ascontiguousarray(targets, dtype=np.uint32)
        k = len(targets)
        tab = ewald_table(self.box, ewald_nt) if ewald else None
        prm = WalkParams(G, h, 0 if crit == "bh" else 1, theta, alpha, int(box_guard), int(treepm), rs, rcut,
                         int(ewald), tab.ctypes.data if ewald else None, int(ewald_nt))
        ao = None
        if a_old is not None:
            ao = np.ascontiguousarray(a_old, dtype=np.float32)
            assert len(ao) == k
        acc = np.zeros((k, 3))
        pot = np.zeros(k)
        nint = np.zeros(k, np.uint32)
        self._lib.orc_tree_walk(self._h, k, _p(targets), _p(ao) if ao is not None else None, C.byref(prm), _p(acc),
                                _p(pot), _p(nint), nthreads)
        return acc, pot, nint


# ---------------------------------------------------------------- Ewald
def ewald_correction(box: float, d) -> np.ndarray:
    """(fx, fy, fz, phi): what the nearest image of a unit mass at separation
    d (source - target) misses of the periodic field (G = 1, Sec. 3.1)."""
    out = np.zeros(4)
    _load().orc_ewald_correction(float(box), float(d[0]), float(d[1]), float(d[2]), _p(out))
    return out


_EWALD_TABLES = {}


def ewald_table(box: float, nt: int = 64) -> np.ndarray:
    """The correction on the grid (i, j, k) box / (2 nt), 0 <= i, j, k <= nt,
    shape (nt+1, nt+1, nt+1, 4); computed once per (box, nt)."""
    key = (float(box), int(nt))
    if key not in _EWALD_TABLES:
        tab = np.zeros((nt + 1, nt + 1, nt + 1, 4))
        _load().orc_ewald_table(float(box), int(nt), _p(tab), 0)
        _EWALD_TABLES[key] = tab
    return _EWALD_TABLES[key]


def ewald_params(box: float, tol_erfc: float = 4.1, rreal_frac: float = 0.3):
    """Splitting with alpha r_E = tol_erfc and the k cutoff set so that
    exp(-k^2 / 4 alpha^2) matches erfc(alpha r_E) (k_max = 2 alpha tol_erfc)."""
    rreal = rreal_frac * box
    alpha = tol_erfc / rreal
    kmax = int(math.ceil(2.0 * alpha * tol_erfc * box / (2.0 * math.pi)))
    return alpha, rreal, kmax


def ewald(pos, mass, targets, G: float, box: float, alpha: float = None, rreal: float = None, kmax: int = None,
          nthreads: int = 0):
    """Periodic Ewald-summed force and potential (FP64) on ``targets``."""
    if alpha is None:
        alpha, rreal, kmax = ewald_params(box)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float32)
    targets = np.ascontiguousarray(targets, dtype=np.uint32)
    acc = np.full((len(targets), 3), np.nan)
    pot = np.full(len(targets), np.nan)
    _load().orc_ewald(len(pos), _p(pos), _p(mass), len(targets), _p(targets), G, box, alpha, rreal, kmax, _p(acc),
                      _p(pot), nthreads)
    return acc, pot


# ---------------------------------------------------------------- PM (numpy)
def _cic_weights(pos, box, ngrid):
    """Cloud-in-cell: mesh points at x = i * box / ngrid; a particle at t = x / dx
    gives weight (1 - f) to cell floor(t) and f to the next (periodic)."""
    t = np.asarray(pos, dtype=np.float64) * (ngrid / box)
    i0 = np.floor(t)
    f = t - i0
    i0 = i0.astype(np.int64) % ngrid
    return i0, f


def pm_potential(pos, mass, box: float, ngrid: int, rs: float, G: float = 1.0) -> np.ndarray:
    """Long-range mesh potential (Sec. 3.3, 3.4), FP64.

    CIC deposit of mass onto ngrid^3 mesh points, density = mass / dx^3;
    Phi_k = -4 pi G rho_k / k^2 * exp(-k^2 r_s^2) / W(k)^2 with
    W = prod_a sinc^2(k_a dx / 2) (CIC assignment and interpolation windows),
    Phi_0 = 0 (the mean density is subtracted); inverse FFT.
    """
    dx = box / ngrid
    i0, f = _cic_weights(pos, box, ngrid)
    m = np.asarray(mass, dtype=np.float64)
    rho = np.zeros(ngrid ** 3)
    for cx in (0, 1):
        wx = f[:, 0] if cx else 1.0 - f[:, 0]
        ix = (i0[:, 0] + cx) % ngrid
        for cy in (0, 1):
            wy = f[:, 1] if cy else 1.0 - f[:, 1]
            iy = (i0[:, 1] + cy) % ngrid
            for cz in (0, 1):
                wz = f[:, 2] if cz else 1.0 - f[:, 2]
                iz = (i0[:, 2] + cz) % ngrid
                np.add.at(rho, (ix * ngrid + iy) * ngrid + iz, m * wx * wy * wz)
    rho = rho.reshape(ngrid, ngrid, ngrid) / dx ** 3
    rhok = np.fft.rfftn(rho)
    kf = 2.0 * math.pi / box
    n = np.fft.fftfreq(ngrid, d=1.0 / ngrid)
    nz = np.fft.rfftfreq(ngrid, d=1.0 / ngrid)
    kx = (kf * n)[:, None, None]
    ky = (kf * n)[None, :, None]
    kz = (kf * nz)[None, None, :]
    k2 = kx * kx + ky * ky + kz * kz
    w = (np.sinc(kx * dx / (2.0 * math.pi)) * np.sinc(ky * dx / (2.0 * math.pi)) *
         np.sinc(kz * dx / (2.0 * math.pi))) ** 2
    k2s = np.where(k2 > 0, k2, 1.0)
    green = -4.0 * math.pi * G / k2s * np.exp(-k2 * rs * rs) / (w * w)
    green[0, 0, 0] = 0.0
    phi = np.fft.irfftn(rhok * green, s=(ngrid, ngrid, ngrid), axes=(0, 1, 2))
    return phi


def mesh_forces(phi: np.ndarray, box: float, grad: str = "fd4"):
    """The three force meshes a = -grad Phi of a periodic potential mesh.

    ``fd4``: the 4-point finite difference (Sec. 3.3 leaves the stencil open)
      dPhi/dx ~ [4/3 (Phi_{+1} - Phi_{-1}) / 2 - 1/3 (Phi_{+2} - Phi_{-2}) / 4] / dx.
    ``ik``: the spectral derivative, a_k = -i k Phi_k per axis, with the
      Nyquist mode of each axis (whose derivative a real mesh cannot carry) set
      to zero.
    """
    ngrid = phi.shape[0]
    dx = box / ngrid
    if grad == "fd4":
        out = []
        for ax in range(3):
            d1 = np.roll(phi, -1, axis=ax) - np.roll(phi, 1, axis=ax)
            d2 = np.roll(phi, -2, axis=ax) - np.roll(phi, 2, axis=ax)
            out.append(-((4.0 / 3.0) * d1 / 2.0 - (1.0 / 3.0) * d2 / 4.0) / dx)
        return out
    if grad != "ik":
        raise ValueError("grad must be 'fd4' or 'ik'")
    phik = np.fft.rfftn(phi)
    kf = 2.0 * math.pi / box
    n = np.fft.fftfreq(ngrid, d=1.0 / ngrid)
    nz = np.fft.rfftfreq(ngrid, d=1.0 / ngrid)
    n = np.where(np.abs(n) == ngrid // 2, 0.0, n)
    nz = np.where(nz == ngrid // 2, 0.0, nz)
    ks = [(kf * n)[:, None, None], (kf * n)[None, :, None], (kf * nz)[None, None, :]]
    return [np.fft.irfftn(-1j * k * phik, s=phi.shape, axes=(0, 1, 2)) for k in ks]


def pm_interpolate(phi: np.ndarray, pos, box: float, grad: str = "fd4"):
    """Mesh force -grad Phi (``mesh_forces``: 4-point difference or spectral),
    then CIC interpolation of the force and of Phi to the particles."""
    ngrid = phi.shape[0]
    grads = mesh_forces(phi, box, grad)
    fields = [g.ravel() for g in grads] + [phi.ravel()]
    i0, f = _cic_weights(pos, box, ngrid)
    out = np.zeros((len(i0), 4))
    for cx in (0, 1):
        wx = f[:, 0] if cx else 1.0 - f[:, 0]
        ix = (i0[:, 0] + cx) % ngrid
        for cy in (0, 1):
            wy = f[:, 1] if cy else 1.0 - f[:, 1]
            iy = (i0[:, 1] + cy) % ngrid
            for cz in (0, 1):
                wz = f[:, 2] if cz else 1.0 - f[:, 2]
                iz = (i0[:, 2] + cz) % ngrid
                idx = (ix * ngrid + iy) * ngrid + iz
                w = wx * wy * wz
                for c in range(4):
                    out[:, c] += w * fields[c][idx]
    return out[:, :3], out[:, 3]


def treepm(pos, mass, targets, box: float, ngrid: int, asmth: float, rcut_cells: float, G: float, h: float,
           crit: str = "bh", theta: float = 0.5, alpha: float = 0.005, a_old=None, bucket: int = 8,
           shift=(0.0, 0.0, 0.0), nthreads: int = 0, grad: str = "fd4"):
    """Periodic TreePM force (Sec. 3.4): short-range tree walk plus PM (mesh
    force by ``grad``: the 4-point difference or the spectral derivative)."""
    rs = asmth * box / ngrid
    rcut = rcut_cells * rs
    tree = Tree(pos, mass, bucket=bucket, periodic=True, box=box, shift=shift)
    a_s, p_s, nint = tree.walk(targets, G, h, crit=crit, theta=theta, alpha=alpha, a_old=a_old, treepm=True, rs=rs,
                               rcut=rcut, nthreads=nthreads)
    phi = pm_potential(pos, mass, box, ngrid, rs, G)
    a_l, p_l = pm_interpolate(phi, np.asarray(pos)[np.asarray(targets, dtype=np.int64)], box, grad)
    return a_s + a_l, p_s + p_l, nint


# ---------------------------------------------------------------- isolated PM
def _erf(x: np.ndarray) -> np.ndarray:
    """Elementwise FP64 erf (scipy's when installed, else the math module's)."""
    try:
        from scipy.special import erf

        return erf(x)
    except ImportError:
        return np.vectorize(math.erf)(x)


def pm_region_isolated(pos):
    """Mesh region of the nonperiodic PM (Sec. 3.3): a cube of side L_pm = the
    tree root's side (smallest power of two >= 1.25 x the largest extent of
    the bounding box; extent 1 for a single point) centred on the bounding
    box, so that at least a tenth of L_pm stays free on every side.  Returns
    (corner (3,), L_pm)."""
    pos = np.asarray(pos, dtype=np.float64)
    lo, hi = pos.min(axis=0), pos.max(axis=0)
    ext = float(np.max(hi - lo))
    if not ext > 0.0:
        ext = 1.0
    f, e = math.frexp(1.25 * ext)
    side = math.ldexp(1.0, e - 1) if f == 0.5 else math.ldexp(1.0, e)
    corner = (lo + hi) * 0.5 - 0.5 * side
    return corner, side


def pm_potential_isolated(pos, mass, corner, side: float, ngrid: int, rs: float, G: float = 1.0) -> np.ndarray:
    """Long-range potential with nonperiodic boundaries (Sec. 3.3: zero padding
    and the Green's function of isolated boundaries), FP64.

    CIC masses on ngrid^3 mesh points x = corner + i dx (dx = side / ngrid)
    inside a zero-padded (2 ngrid)^3 mesh; the potential is the convolution
    Phi(p) = sum_q m_q g(p - q) with the long-range kernel of the Gaussian
    split, g(r) = -G erf(r / 2 r_s) / r (g(0) = -G / (sqrt(pi) r_s)), sampled
    at the mesh separations min(|i|, 2 ngrid - |i|) dx, so the circular
    convolution of the padded mesh is the open one for every mesh point of
    the unpadded region.  The CIC windows are divided out in k-space as in
    the periodic mesh (W(k)^2, W = prod_a sinc^2(k_a dx / 2)).  Returns the
    (2 ngrid)^3 potential; only [0, ngrid]^3 is physical."""
    n2 = 2 * ngrid
    dx = side / ngrid
    t = (np.asarray(pos, dtype=np.float64) - np.asarray(corner)) * (ngrid / side)
    i0 = np.floor(t)
    f = t - i0
    i0 = i0.astype(np.int64)
    if i0.min() < 0 or i0.max() + 1 >= ngrid:
        raise ValueError("particles outside the mesh region")
    m = np.asarray(mass, dtype=np.float64)
    rho = np.zeros(n2 ** 3)
    for cx in (0, 1):
        wx = f[:, 0] if cx else 1.0 - f[:, 0]
        for cy in (0, 1):
            wy = f[:, 1] if cy else 1.0 - f[:, 1]
            for cz in (0, 1):
                wz = f[:, 2] if cz else 1.0 - f[:, 2]
                idx = ((i0[:, 0] + cx) * n2 + i0[:, 1] + cy) * n2 + i0[:, 2] + cz
                np.add.at(rho, idx, m * wx * wy * wz)
    rho = rho.reshape(n2, n2, n2)
    d = np.minimum(np.arange(n2), n2 - np.arange(n2)) * dx
    r = np.sqrt(d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2)
    with np.errstate(invalid="ignore", divide="ignore"):
        g = _erf(r / (2.0 * rs)) / r
    g[0, 0, 0] = 1.0 / (math.sqrt(math.pi) * rs)
    g *= -G
    n = np.fft.fftfreq(n2, d=1.0 / n2)
    nz = np.fft.rfftfreq(n2, d=1.0 / n2)
    sx = np.sinc(n / n2)  # sinc(k dx / 2) with k = 2 pi n / (n2 dx)
    sz = np.sinc(nz / n2)
    w = (sx[:, None, None] * sx[None, :, None] * sz[None, None, :]) ** 2
    phik = np.fft.rfftn(rho) * np.fft.rfftn(g) / (w * w)
    return np.fft.irfftn(phik, s=(n2, n2, n2), axes=(0, 1, 2))


def pm_interpolate_isolated(phi: np.ndarray, pos, corner, side: float, ngrid: int):
    """4-point finite-difference force (a = -grad Phi) and the potential,
    CIC-interpolated to ``pos`` from the physical part of an isolated mesh."""
    dx = side / ngrid
    grads = []
    for ax in range(3):
        d1 = np.roll(phi, -1, axis=ax) - np.roll(phi, 1, axis=ax)
        d2 = np.roll(phi, -2, axis=ax) - np.roll(phi, 2, axis=ax)
        grads.append(-((4.0 / 3.0) * d1 / 2.0 - (1.0 / 3.0) * d2 / 4.0) / dx)
    n2 = phi.shape[0]
    fields = [g.ravel() for g in grads] + [phi.ravel()]
    t = (np.asarray(pos, dtype=np.float64) - np.asarray(corner)) * (ngrid / side)
    i0 = np.floor(t)
    f = t - i0
    i0 = i0.astype(np.int64)
    if i0.min() < 2 or i0.max() + 3 > ngrid:
        raise ValueError("the difference stencil leaves the physical mesh")
    out = np.zeros((len(i0), 4))
    for cx in (0, 1):
        wx = f[:, 0] if cx else 1.0 - f[:, 0]
        for cy in (0, 1):
            wy = f[:, 1] if cy else 1.0 - f[:, 1]
            for cz in (0, 1):
                wz = f[:, 2] if cz else 1.0 - f[:, 2]
                idx = ((i0[:, 0] + cx) * n2 + i0[:, 1] + cy) * n2 + i0[:, 2] + cz
                w = wx * wy * wz
                for c in range(4):
                    out[:, c] += w * fields[c][idx]
    return out[:, :3], out[:, 3]


def treepm_isolated(pos, mass, targets, ngrid: int, asmth: float, rcut_cells: float, G: float, h: float,
                    crit: str = "bh", theta: float = 0.5, alpha: float = 0.0025, a_old=None, bucket: int = 8,
                    shift=(0.0, 0.0, 0.0), nthreads: int = 0, hsoft=None):
    """TreePM with nonperiodic boundaries (Sec. 3.3, 3.4): short-range walk of
    the open tree with the erfc split and cutoff, plus the isolated mesh;
    r_s = asmth x the mesh spacing of ``pm_region_isolated``."""
    corner, side = pm_region_isolated(pos)
    rs = asmth * side / ngrid
    tree = Tree(pos, mass, bucket=bucket, shift=shift, hsoft=hsoft)
    a_s, p_s, nint = tree.walk(targets, G, h, crit=crit, theta=theta, alpha=alpha, a_old=a_old, treepm=True, rs=rs,
                               rcut=rcut_cells * rs, nthreads=nthreads)
    phi = pm_potential_isolated(pos, mass, corner, side, ngrid, rs, G)
    a_l, p_l = pm_interpolate_isolated(phi, np.asarray(pos)[np.asarray(targets, dtype=np.int64)], corner, side, ngrid)
    return a_s + a_l, p_s + p_l, nint


# ---------------------------------------------------------------- insertion tree
def diagnostics(mass, acc, pot=None, vel=None) -> dict:
    """Conservation diagnostics of a force evaluation [Sec. 7], each a plain
    FP64 sum over the particles: total force sum_i m_i a_i, its scale
    sum_i m_i |a_i|, potential energy 1/2 sum_i m_i phi_i, kinetic energy
    1/2 sum_i m_i |v_i|^2 and momentum sum_i m_i v_i (zero without pot / vel)."""
    m = np.asarray(mass, np.float64)
    a = np.asarray(acc, np.float64).reshape(-1, 3)
    out = {"total_force": (m[:, None] * a).sum(axis=0),
           "force_scale": float((m * np.sqrt((a * a).sum(axis=1))).sum()),
           "potential_energy": 0.0, "kinetic_energy": 0.0, "momentum": np.zeros(3)}
    if pot is not None:
        out["potential_energy"] = float(0.5 * (m * np.asarray(pot, np.float64)).sum())
    if vel is not None:
        v = np.asarray(vel, np.float64).reshape(-1, 3)
        out["kinetic_energy"] = float(0.5 * (m * (v * v).sum(axis=1)).sum())
        out["momentum"] = (m[:, None] * v).sum(axis=0)
    return out


def insertion_tree(pos, x0, L0: float, bucket: int = 1, order=None):
    """The paper's construction (Sec. 3.1), brute force: start from the cubic
    root, insert particles one at a time, descending by comparing coordinates
    with each cell's geometric centre; a leaf that would hold more than
    ``bucket`` particles is split and its particles pushed one level down,
    recursively, up to level 21.  Returns {(level, ix, iy, iz): count}.
    """
    pos = np.asarray(pos, dtype=np.float64)
    x0 = [float(v) for v in x0]
    nodes = {}  # (level, ix, iy, iz) -> list of particle ids if leaf, or None if internal

    def centre(level, ix, iy, iz):
        side = L0 / (1 << level)
        return (x0[0] + (ix + 0.5) * side, x0[1] + (iy + 0.5) * side, x0[2] + (iz + 0.5) * side)

    def child_of(cell, p):
        level, ix, iy, iz = cell
        c = centre(level, ix, iy, iz)
        bx = 1 if pos[p, 0] >= c[0] else 0
        by = 1 if pos[p, 1] >= c[1] else 0
        bz = 1 if pos[p, 2] >= c[2] else 0
        return (level + 1, 2 * ix + bx, 2 * iy + by, 2 * iz + bz)

    def put(cell, p):
        while True:
            if cell not in nodes:
                nodes[cell] = [p]
                return
            content = nodes[cell]
            if content is None:
                cell = child_of(cell, p)
                continue
            content.append(p)
            if len(content) > bucket and cell[0] < MAXLEVEL:
                nodes[cell] = None
                for q in content:
                    put(child_of(cell, q), q)
            return

    ids = range(len(pos)) if order is None else order
    root = (0, 0, 0, 0)
    for p in ids:
        put(root, p)

    counts = {}

    def count(cell):
        content = nodes[cell]
        if content is not None:
            counts[cell] = len(content)
            return len(content)
        level, ix, iy, iz = cell
        tot = 0
        for o in range(8):
            ch = (level + 1, 2 * ix + (o & 1), 2 * iy + ((o >> 1) & 1), 2 * iz + ((o >> 2) & 1))
            if ch in nodes:
                tot += count(ch)
        counts[cell] = tot
        return tot

    count(root)
    return counts


def prefix_to_cell(level: int, prefix: int):
    """(level, Morton prefix) -> (level, ix, iy, iz)."""
    ix = iy = iz = 0
    for b in range(level):
        ix |= ((prefix >> (3 * b)) & 1) << b
        iy |= ((prefix >> (3 * b + 1)) & 1) << b
        iz |= ((prefix >> (3 * b + 2)) & 1) << b
    return (level, ix, iy, iz)
