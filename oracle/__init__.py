"""CPU oracle for the GKE terms (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (CUDA) path never does, and
this package imports nothing from it.

``gke_oracle.c`` evaluates every term of the Generalised Kolmogorov Equation
for plane channel flow directly from its definition (Sec. 2 of Gatti et al.,
Eq. 1-6) as averages of increment products over x, z and snapshots, with the
Y1/Y2 derivatives of Step 3 (Eq. 10-11) by a 5-point finite-difference
stencil.  It never forms a two-point correlation in Fourier space.

Index conventions shared with the results it is compared against (these are
conventions of the *output*, not code):
  * ordered pair (i1, i2): Y1 = y[i1], Y2 = y[i2];
  * separation index (m_z, m_x) in [0, nz) x [0, nx), r = (m_x Lx/nx, m_z Lz/nz);
  * terms: A = <du^2>, Phi_x, Phi_y, Phi_z, phi, xi, residual.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gke_oracle.c")
_LIB = os.path.join(_HERE, "_gke_oracle.so")

COMPONENTS = ("A", "Bx", "By", "Bz", "C", "P", "Q", "R", "GxA", "GzA", "dY1A", "dY2A")
TERMS = ("A", "Phi_x", "Phi_y", "Phi_z", "phi", "xi", "residual")
PROFILES = ("U", "V", "W", "P", "dUdy", "eps")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into oracle/_gke_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def load_library(path: str):
    """Open a compiled copy of the oracle at `path` with its entry points typed.

    The tests use it to load deliberately broken copies of gke_oracle.c (a
    planted mistake must make a pin fail); everything else goes through the
    default library built by build()."""
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.oracle_full.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, dp,
                                ctypes.c_int]
    lib.oracle_points.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                  ip, dp, dp, ctypes.c_int]
    lib.oracle_fd_weights.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
    lib.oracle_fd_weights.restype = ctypes.c_int
    return lib


def compile_source(src_text: str, out_path: str) -> str:
    """Compile C source text of the oracle (gcc, OpenMP) into `out_path`."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-D_DEFAULT_SOURCE", "-o", out_path, c_path, "-lm"])
    return out_path


def source_text() -> str:
    """The oracle's C source."""
    with open(_SRC) as f:
        return f.read()


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def fd_weights(y: np.ndarray, j: int):
    """(l0, w[5]): first-derivative weights at row j on nodes l0..l0+4."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    w = np.zeros(5)
    l0 = _load().oracle_fd_weights(_dp(y), len(y), j, _dp(w))
    return l0, w


def mirror_augment(phys: np.ndarray) -> np.ndarray:
    """The snapshot set doubled by the mirror images about the centreline.

    Mirror sampling (Sec. 3.2, Step 2): the channel is statistically
    symmetric under the inversion of the wall-normal axis, y -> 2h - y, which
    maps a flow field to another flow field with the same statistics:
    u(x, 2h - y, z), -v(x, 2h - y, z), w(x, 2h - y, z), p(x, 2h - y, z).
    Each snapshot's image is one more sample.  On a grid symmetric about the
    centreline the image of plane j is plane ny - 1 - j.
    """
    phys = np.asarray(phys, dtype=np.float64)
    img = phys[:, :, ::-1].copy()
    img[:, 1] *= -1.0
    return np.concatenate([phys, img], axis=0)


def wedge_pairs(ny: int):
    """Pairs (i1, i2) of the half-channel wedge, row-major: i1 <= i2 and
    i1 + i2 <= ny - 1, i.e. Y1 <= h and Y1 <= Y2 <= 2h - Y1 (Sec. 3.2, Step 2)."""
    return [(a, b) for a in range(ny) for b in range(a, ny - a)]


def full(phys: np.ndarray, y: np.ndarray, Lx: float, Lz: float, nu: float, nthreads: int = 0,
         mirror: bool = False, lib=None):
    """All components and terms on the full square of ordered pairs.

    phys: float64 [ns][4][ny][nz][nx] (u, v, w, p including the mean).
    mirror: average over the snapshots and their mirror images
    (mirror_augment; y must be symmetric about its centre).
    Returns dict(comp=[12][ny][ny][nz][nx], terms=[7][ny][ny][nz][nx],
    prof=[6][ny]) with names COMPONENTS, TERMS, PROFILES.
    lib: a library from load_library() instead of the default build.
    """
    if mirror:
        phys = mirror_augment(phys)
    phys = np.ascontiguousarray(phys, dtype=np.float64)
    ns, nf, ny, nz, nx = phys.shape
    assert nf == 4
    y = np.ascontiguousarray(y, dtype=np.float64)
    comp = np.zeros((len(COMPONENTS), ny, ny, nz, nx))
    terms = np.zeros((len(TERMS), ny, ny, nz, nx))
    prof = np.zeros((len(PROFILES), ny))
    rc = (lib or _load()).oracle_full(_dp(phys), ns, nx, nz, ny, _dp(y), Lx, Lz, nu, _dp(comp), _dp(terms),
                                      _dp(prof), nthreads)
    if rc != 0:
        raise ValueError(f"oracle_full failed ({rc})")
    return {"comp": comp, "terms": terms, "prof": prof}


def points(phys: np.ndarray, y: np.ndarray, Lx: float, Lz: float, nu: float, pts, nthreads: int = 0,
           mirror: bool = False):
    """Components and terms (all but the residual) at points (i1, i2, m_z, m_x).

    mirror: as in full().  Returns dict(comp=[n][12], terms=[n][6],
    prof=[6][ny]); eps in prof is NaN on planes no point touches.
    """
    if mirror:
        phys = mirror_augment(phys)
    phys = np.ascontiguousarray(phys, dtype=np.float64)
    ns, nf, ny, nz, nx = phys.shape
    y = np.ascontiguousarray(y, dtype=np.float64)
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.int32).reshape(-1, 4))
    W = len(COMPONENTS) + len(TERMS) - 1
    out = np.zeros((len(pts), W))
    prof = np.zeros((len(PROFILES), ny))
    rc = _load().oracle_points(_dp(phys), ns, nx, nz, ny, _dp(y), Lx, Lz, nu, len(pts),
                               pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(out), _dp(prof),
                               nthreads)
    if rc != 0:
        raise ValueError(f"oracle_points failed ({rc})")
    return {"comp": out[:, :len(COMPONENTS)], "terms": out[:, len(COMPONENTS):], "prof": prof}
