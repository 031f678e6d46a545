"""HSMA oracle: a plain FP64 CPU implementation of the harmonic surface
mapping algorithm (arXiv:1806.04801), used to check the CUDA path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with the CUDA path and must never be used as a fallback for it.

The C primitives live in ``hsma_oracle.c`` (compiled on first use, or by
``build()``); ``oracle.hsma`` composes them in the paper's order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hsma_oracle.c")
_LIB = os.path.join(_HERE, "libhsma_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C primitives with gcc (plain -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    """The oracle's C library (compiled on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_long)
_ip = ctypes.POINTER(ctypes.c_int)


def _declare(L):
    L.hsmo_num_shells.restype = ctypes.c_int
    L.hsmo_num_shells.argtypes = [ctypes.c_double, ctypes.c_double]
    L.hsmo_inset.restype = ctypes.c_long
    L.hsmo_inset.argtypes = [ctypes.c_long, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double,
                             ctypes.c_long, _dp, _dp, _lp, _ip]
    L.hsmo_coulomb.restype = None
    L.hsmo_coulomb.argtypes = [ctypes.c_long, _dp, _dp, ctypes.c_long, _dp, _lp, _dp, _dp, ctypes.c_int]
    L.hsmo_basis.restype = None
    L.hsmo_basis.argtypes = [ctypes.c_long, _dp, ctypes.c_int, ctypes.c_double, _dp]
    L.hsmo_lstsq.restype = ctypes.c_int
    L.hsmo_lstsq.argtypes = [ctypes.c_long, ctypes.c_long, _dp, _dp, _dp, _dp]
    L.hsmo_monitor_sphere.restype = None
    L.hsmo_monitor_sphere.argtypes = [ctypes.c_int, ctypes.c_double, _dp]
    L.hsmo_wrap_into_box.restype = None
    L.hsmo_wrap_into_box.argtypes = [ctypes.c_long, _dp, _dp, _dp]
    L.hsmo_monitor_faces.restype = ctypes.c_int
    L.hsmo_monitor_faces.argtypes = [ctypes.c_int, _dp, _dp]
    L.hsmo_quadrature.restype = None
    L.hsmo_quadrature.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp]
    L.hsmo_ewald.restype = None
    L.hsmo_ewald.argtypes = [ctypes.c_long, _dp, _dp, _dp, ctypes.c_double, ctypes.c_int,
                             ctypes.c_int, _dp, _dp]
    L.hsmo_ewald_cells.restype = ctypes.c_double
    L.hsmo_ewald_cells.argtypes = [ctypes.c_long, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_long, _lp, _dp, _dp]
    L.hsmo_ewald_sf.restype = None
    L.hsmo_ewald_sf.argtypes = [ctypes.c_long, _dp, _dp, _dp, ctypes.c_double, ctypes.c_int,
                                ctypes.c_int, _dp, _dp]


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


# --------------------------------------------------------------------------
# Thin wrappers over the C primitives (argument marshalling only).
# --------------------------------------------------------------------------

def num_shells(Rs: float, La: float) -> int:
    """Image shells needed along an axis: the smallest K with (K + 1/2) L >= Rs (in-set of Sec. II.A)."""
    return int(lib().hsmo_num_shells(float(Rs), float(La)))


def inset(c, q, L, bc: int, Rs: float):
    """In-set of Sec. II.A (sources + images with |r| < Rs); centred coords."""
    c = _d(c).reshape(-1, 3)
    q = _d(q)
    L = _d(L)
    n = c.shape[0]
    K = [num_shells(Rs, La) for La in L]
    cap = n * (2 * K[0] + 1) * (2 * K[1] + 1) * (2 * K[2] + 1)
    xyz = np.empty((cap, 3))
    qq = np.empty(cap)
    src = np.empty(cap, dtype=np.int64)
    sh = np.empty((cap, 3), dtype=np.int32)
    m = lib().hsmo_inset(n, _ptr(c), _ptr(q), _ptr(L), int(bc), float(Rs), cap, _ptr(xyz),
                         _ptr(qq), _ptr(src, _lp), _ptr(sh, _ip))
    if m < 0:
        raise RuntimeError("in-set capacity exceeded")
    return xyz[:m].copy(), qq[:m].copy(), src[:m].copy(), sh[:m].copy()


def coulomb(sxyz, sq, txyz, tskip=None, field: bool = True, nthreads: int = 1):
    """pot[t] = sum_s q_s/|x_t - y_s|, field[t] = sum_s q_s (x_t - y_s)/|.|^3."""
    sxyz = _d(sxyz).reshape(-1, 3)
    sq = _d(sq)
    txyz = _d(txyz).reshape(-1, 3)
    nt = txyz.shape[0]
    pot = np.empty(nt)
    fld = np.empty((nt, 3)) if field else None
    sk = None if tskip is None else np.ascontiguousarray(tskip, dtype=np.int64)
    lib().hsmo_coulomb(sxyz.shape[0], _ptr(sxyz), _ptr(sq), nt, _ptr(txyz), _ptr(sk, _lp),
                       _ptr(pot), _ptr(fld), int(nthreads))
    return (pot, fld) if field else pot


def basis(pts, P: int, Rs: float):
    """Real solid harmonics r^n P_n^m cos/sin(m phi) scaled by Rs^-n at points (Eq. "harmonic"), unnormalised."""
    pts = _d(pts).reshape(-1, 3)
    out = np.empty((pts.shape[0], (P + 1) ** 2))
    lib().hsmo_basis(pts.shape[0], _ptr(pts), int(P), float(Rs), _ptr(out))
    return out


def lstsq(A, b):
    """Least squares min ||A x - b|| by column-equilibrated Householder QR; returns x and R's diagonal."""
    A = _d(A)
    b = _d(b)
    m, n = A.shape
    x = np.empty(n)
    rd = np.empty(n)
    st = lib().hsmo_lstsq(m, n, _ptr(A), _ptr(b), _ptr(x), _ptr(rd))
    if st != 0:
        raise np.linalg.LinAlgError("rank-deficient least-squares matrix")
    return x, rd


def monitor_sphere(nm: int, R0: float):
    """Fibonacci latitude grid of nm points on the sphere of radius R0 (monitoring points, Sec. II.A)."""
    out = np.empty((nm, 3))
    lib().hsmo_monitor_sphere(int(nm), float(R0), _ptr(out))
    return out


def wrap_into_box(pts, L):
    """Nearest periodic image inside the centred box (the partner x~ of a monitoring point, Sec. II.A)."""
    pts = _d(pts).reshape(-1, 3)
    L = _d(L)
    out = np.empty_like(pts)
    lib().hsmo_wrap_into_box(pts.shape[0], _ptr(pts), _ptr(L), _ptr(out))
    return out


def monitor_faces(K: int, L):
    """About K points on the walls of a grounded box, split by area (monitoring points, Sec. II.A)."""
    L = _d(L)
    out = np.empty((K, 3))
    k = lib().hsmo_monitor_faces(int(K), _ptr(L), _ptr(out))
    return out[:k].copy()


def quadrature(F2: int, F1: int, R: float):
    """Fibonacci integration nodes (unit directions) and weights on the sphere of radius R (Sec. II.B)."""
    n = 2 * (F2 + 1)
    dirs = np.empty((n, 3))
    w = np.empty(n)
    lib().hsmo_quadrature(int(F2), int(F1), float(R), _ptr(dirs), _ptr(w))
    return dirs, w


def ewald(xyz, q, L, beta: float, nreal: int, kmax: int):
    """Tinfoil Ewald potentials (self term removed) and fields at each charge."""
    xyz = _d(xyz).reshape(-1, 3)
    q = _d(q)
    L = _d(L)
    n = xyz.shape[0]
    pot = np.empty(n)
    fld = np.empty((n, 3))
    lib().hsmo_ewald(n, _ptr(xyz), _ptr(q), _ptr(L), float(beta), int(nreal), int(kmax),
                     _ptr(pot), _ptr(fld))
    return pot, fld


def ewald_cells(xyz, q, L, pick=None, tol: float = 1e-12, nthreads: int | None = None, energy: bool = True):
    """Ewald sum of a large neutral periodic system (tinfoil) with a cell list
    for the real-space pairs and structure factors for the reciprocal part:
    the energy, and the potentials (self term removed) and fields at the
    particles ``pick``.  The splitting beta and the cutoffs follow from tol:
    erfc(beta rc) and exp(-kcut^2 / 4 beta^2) are both about tol.  With
    energy=False only the picked particles are evaluated (real space for
    them alone; rc = L/3, the largest the cell lists allow, which keeps the
    reciprocal part small) and the energy is None.  Otherwise rc = L/3 up to
    20000 charges and L/4 beyond (four cells per axis: fewer real-space
    pairs, more k vectors).
    Returns (energy, pot[pick], field[pick])."""
    import math
    xyz = _d(xyz).reshape(-1, 3)
    q = _d(q)
    L = _d(L)
    n = xyz.shape[0]
    pick = np.asarray([] if pick is None else pick, dtype=np.int64)
    x = math.sqrt(-math.log(tol))          # beta rc
    kx = 2.0 * math.sqrt(-math.log(tol))   # kcut / beta
    lmin = float(L.min())
    # cells of rc: with three per axis every pair is visited; four halve that
    rc = 0.333 * lmin if (not energy or n <= 20000) else 0.25 * lmin
    beta = x / rc
    kcut = kx * beta
    pot = np.empty(len(pick))
    fld = np.empty((len(pick), 3))
    th = int(nthreads or os.cpu_count() or 1)
    e = lib().hsmo_ewald_cells(n, _ptr(xyz), _ptr(q), _ptr(L), beta, rc, kcut, th, 1 if energy else 0, len(pick),
                               _ptr(pick, _lp), _ptr(pot), _ptr(fld))
    if not np.isfinite(e):
        raise ValueError("box too small for the cell lists")
    return (float(e) if energy else None), pot, fld


def ewald_sf(xyz, q, L, beta: float, nreal: int, kmax: int):
    """Ewald as ``ewald`` with structure factors (O(N K) reciprocal part)."""
    xyz = _d(xyz).reshape(-1, 3)
    q = _d(q)
    L = _d(L)
    n = xyz.shape[0]
    pot = np.empty(n)
    fld = np.empty((n, 3))
    lib().hsmo_ewald_sf(n, _ptr(xyz), _ptr(q), _ptr(L), float(beta), int(nreal), int(kmax),
                        _ptr(pot), _ptr(fld))
    return pot, fld
