"""CPU oracle for the GKE with one homogeneous direction (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the product (CUDA) path never does.

``gke1h_oracle.c`` evaluates the terms for a flow homogeneous in x only (the
variant the paper's conclusions (Sec. 5) point to: the second inhomogeneous
direction z is handled like the wall-normal one) directly from their
definitions, as averages of increment products over x and snapshots, with
5-point stencils in Y1, Y2, Z1, Z2.  It never forms a correlation in Fourier
space.

Index conventions of the output (shared with what it is compared against):
  * cross-section point p = iy nz + iz;
  * ordered pair (p1, p2), separation index m_x in [0, nx), r_x = m_x Lx / nx;
  * terms: A, Phi_x, Phi_y, Phi_z, psi_y, psi_z, xi, residual.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gke1h_oracle.c")
_LIB = os.path.join(_HERE, "_gke1h_oracle.so")

COMPONENTS = ("A", "Bx", "By", "Bz", "Cy", "Cz", "Py", "Pz",
              "Qxy", "Qyy", "Qzy", "Qxz", "Qyz", "Qzz",
              "Rxy", "Ryy", "Rzy", "Rxz", "Ryz", "Rzz",
              "GxA", "dY1A", "dY2A", "dZ1A", "dZ2A")
TERMS = ("A", "Phi_x", "Phi_y", "Phi_z", "psi_y", "psi_z", "xi", "residual")
PROFILES = ("U", "V", "W", "P", "dUdy", "dUdz", "dVdy", "dVdz", "dWdy", "dWdz", "eps")

_lib = None


def _compile(src: str, out: str) -> None:
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-D_DEFAULT_SOURCE", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile gke1h_oracle.c (gcc, OpenMP) into oracle/_gke1h_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        _compile(_SRC, _LIB)
    return _LIB


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def compile_source(src_text: str, out_path: str) -> str:
    """Compile C source text of this oracle into `out_path` (planted-mistake copies)."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    _compile(c_path, out_path)
    return out_path


def load_library(path: str):
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    i = ctypes.c_int
    d = ctypes.c_double
    lib.oracle1h_full.argtypes = [dp, i, i, i, i, dp, dp, d, d, dp, dp, dp, i]
    lib.oracle1h_points.argtypes = [dp, i, i, i, i, dp, dp, d, d, i, ip, dp, dp, i]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def full(phys: np.ndarray, y: np.ndarray, z: np.ndarray, Lx: float, nu: float, nthreads: int = 0, lib=None):
    """All components and terms on the full square of ordered pairs.

    phys: float64 [ns][4][ny][nz][nx] (u, v, w, p including the mean).
    Returns dict(comp=[25][P][P][nx], terms=[8][P][P][nx], prof=[11][P]),
    P = ny nz, names COMPONENTS, TERMS, PROFILES.
    """
    phys = np.ascontiguousarray(phys, dtype=np.float64)
    ns, nf, ny, nz, nx = phys.shape
    assert nf == 4 and len(y) == ny and len(z) == nz
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    P = ny * nz
    comp = np.zeros((len(COMPONENTS), P, P, nx))
    terms = np.zeros((len(TERMS), P, P, nx))
    prof = np.zeros((len(PROFILES), P))
    rc = (lib or _load()).oracle1h_full(_dp(phys), ns, nx, ny, nz, _dp(y), _dp(z), Lx, nu, _dp(comp),
                                        _dp(terms), _dp(prof), nthreads)
    if rc != 0:
        raise ValueError(f"oracle1h_full failed ({rc})")
    return {"comp": comp, "terms": terms, "prof": prof}


def points(phys: np.ndarray, y: np.ndarray, z: np.ndarray, Lx: float, nu: float, pts, nthreads: int = 0):
    """Components and terms (all but the residual) at pts[n] = (p1, p2, m_x).

    Returns dict(comp=[n][25], terms=[n][7], prof=[11][P])."""
    phys = np.ascontiguousarray(phys, dtype=np.float64)
    ns, nf, ny, nz, nx = phys.shape
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.int32).reshape(-1, 3))
    n = len(pts)
    W = len(COMPONENTS) + len(TERMS) - 1
    out = np.zeros((n, W))
    prof = np.zeros((len(PROFILES), ny * nz))
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    rc = _load().oracle1h_points(_dp(phys), ns, nx, ny, nz, _dp(y), _dp(z), Lx, nu, n,
                                 pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(out), _dp(prof), nthreads)
    if rc != 0:
        raise ValueError(f"oracle1h_points failed ({rc})")
    nc = len(COMPONENTS)
    return {"comp": out[:, :nc], "terms": out[:, nc:], "prof": prof}
