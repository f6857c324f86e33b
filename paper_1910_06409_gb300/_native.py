"""ctypes binding of the C ABI in include/gke.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own.  Pointers may be torch tensors (device or host),
numpy arrays or raw integer addresses.  The library must have been built
(``paper_1910_06409_gb300.build.build()``); a missing library is an error,
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgke.so")

GKE_OK = 0
STATUS = {0: "GKE_OK", -1: "GKE_ERR_ARG", -2: "GKE_ERR_STATE", -3: "GKE_ERR_OOM", -4: "GKE_ERR_CUDA",
          -5: "GKE_ERR_NONFINITE", -6: "GKE_ERR_IO", -7: "GKE_ERR_UNSUPPORTED"}
GKE_PREC_F64, GKE_PREC_BF16X3, GKE_PREC_F32 = 0, 1, 2
GKE_DOMAIN_TRIANGLE, GKE_DOMAIN_WEDGE = 0, 1
TERMS = ("A", "Phi_x", "Phi_y", "Phi_z", "phi", "xi", "residual")
PROFILES = ("U", "V", "W", "P", "dUdy", "eps")
GKE_NTERM, GKE_NPROF = len(TERMS), len(PROFILES)

# every symbol include/gke.h declares
EXPORTS = ("gke_plan", "gke_accumulate_mean", "gke_set_mean", "gke_accumulate_snapshot", "gke_finalize_terms",
           "gke_compute", "gke_compute_graph", "gke_pair_labels", "gke_npair", "gke_separation_labels",
           "gke_terms_bytes", "gke_term_set", "gke_plan_knobs", "gke_reset", "gke_checkpoint",
           "gke_restore", "gke_merge", "gke_fd_weights", "gke_set_timing", "gke_stage_times",
           "gke_launch_count", "gke_compute_noalloc", "gke_last_error", "gke_destroy",
           "gke_velocity_vorticity",
           "gke1h_plan", "gke1h_compute", "gke1h_npair", "gke1h_pair_labels", "gke1h_set_timing",
           "gke1h_stage_times",
           "gke1h_launch_count", "gke1h_last_error", "gke1h_destroy")
# the variant with one homogeneous direction (include/gke1h.h)
TERMS_1H = ("A", "Phi_x", "Phi_y", "Phi_z", "psi_y", "psi_z", "xi", "residual")
PROFILES_1H = ("U", "V", "W", "P", "dUdy", "dUdz", "dVdy", "dVdz", "dWdy", "dWdz", "eps")
GKE1H_NTERM, GKE1H_NPROF = len(TERMS_1H), len(PROFILES_1H)
STAGES = ("mean", "products", "correlate", "combine", "terms", "stencil")


class gke_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nz", ctypes.c_int), ("ny", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Lz", ctypes.c_double), ("nu", ctypes.c_double),
                ("y", ctypes.POINTER(ctypes.c_double)),
                ("max_snap", ctypes.c_int), ("precision", ctypes.c_int), ("pair_domain", ctypes.c_int),
                ("under_x", ctypes.c_int * 4), ("under_z", ctypes.c_int * 4), ("term_mask", ctypes.c_uint),
                ("tune_cache", ctypes.c_char_p)]


class gke1h_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("Lx", ctypes.c_double), ("nu", ctypes.c_double),
                ("y", ctypes.POINTER(ctypes.c_double)), ("z", ctypes.POINTER(ctypes.c_double)),
                ("max_snap", ctypes.c_int), ("precision", ctypes.c_int)]


class GkeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libgke.so (raises OSError if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} not found: build it with paper_1910_06409_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, cp, i, d = ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_double
        dp = ctypes.POINTER(ctypes.c_double)
        sig = {
            "gke_plan": (i, [ctypes.POINTER(gke_desc), vp, ctypes.POINTER(vp)]),
            "gke_accumulate_mean": (i, [vp, vp, i]),
            "gke_velocity_vorticity": (i, [vp, vp, vp, i, vp]),
            "gke_set_mean": (i, [vp, vp]),
            "gke_accumulate_snapshot": (i, [vp, vp, i]),
            "gke_finalize_terms": (i, [vp, vp, vp]),
            "gke_compute": (i, [vp, vp, i, vp, vp]),
            "gke_compute_graph": (i, [vp, vp, i, vp, vp]),
            "gke_pair_labels": (i, [vp, vp, vp, vp, vp]),
            "gke_npair": (ctypes.c_longlong, [vp]),
            "gke_separation_labels": (i, [vp, vp, vp, vp, vp]),
            "gke_terms_bytes": (ctypes.c_longlong, [vp]),
            "gke_reset": (i, [vp]),
            "gke_checkpoint": (i, [vp, cp]),
            "gke_restore": (i, [vp, cp]),
            "gke_merge": (i, [vp, cp]),
            "gke_fd_weights": (i, [dp, i, i, dp]),
            "gke_term_set": (ctypes.c_uint, [ctypes.c_uint]),
            "gke_plan_knobs": (i, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int)]),
            "gke_set_timing": (i, [vp, i]),
            "gke_stage_times": (i, [vp, vp]),
            "gke_launch_count": (ctypes.c_longlong, [vp]),
            "gke_compute_noalloc": (i, [ctypes.POINTER(gke_desc), vp, i, vp, vp, vp]),
            "gke_last_error": (cp, [vp]),
            "gke_destroy": (None, [vp]),
            "gke1h_plan": (i, [ctypes.POINTER(gke1h_desc), vp, ctypes.POINTER(vp)]),
            "gke1h_compute": (i, [vp, vp, i, vp, vp]),
            "gke1h_npair": (ctypes.c_longlong, [vp]),
            "gke1h_pair_labels": (ctypes.c_longlong, [i, i, dp, dp, vp, vp, vp, vp, vp, vp]),
            "gke1h_set_timing": (i, [vp, i]),
            "gke1h_stage_times": (i, [vp, vp]),
            "gke1h_launch_count": (ctypes.c_longlong, [vp]),
            "gke1h_last_error": (cp, [vp]),
            "gke1h_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def ptr(x) -> int | None:
    """Address of a torch tensor / numpy array / int (None stays None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(status: int, plan) -> None:
    if status != GKE_OK:
        msg = lib().gke_last_error(plan)
        raise GkeError(status, msg.decode() if msg else "")


def gke_plan(nx, nz, ny, Lx, Lz, nu, y, max_snap, precision=GKE_PREC_F64, stream=None,
             pair_domain=GKE_DOMAIN_TRIANGLE, under_x=(0, 0, 0, 0), under_z=(0, 0, 0, 0), term_mask=0,
             tune_cache=None):
    import numpy as np
    yy = np.ascontiguousarray(y, dtype=np.float64)
    desc = gke_desc(nx, nz, ny, Lx, Lz, nu, yy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), max_snap,
                    precision, pair_domain, (ctypes.c_int * 4)(*under_x), (ctypes.c_int * 4)(*under_z), term_mask,
                    None if tune_cache is None else str(tune_cache).encode())
    out = ctypes.c_void_p()
    st = lib().gke_plan(ctypes.byref(desc), stream, ctypes.byref(out))
    _check(st, None)
    return out.value


def gke_accumulate_mean(plan, fields, nsnap):
    _check(lib().gke_accumulate_mean(plan, ptr(fields), nsnap), plan)


def gke_set_mean(plan, mean):
    _check(lib().gke_set_mean(plan, ptr(mean)), plan)


def gke_accumulate_snapshot(plan, fields, nsnap):
    _check(lib().gke_accumulate_snapshot(plan, ptr(fields), nsnap), plan)


def gke_finalize_terms(plan, terms, profiles=None):
    _check(lib().gke_finalize_terms(plan, ptr(terms), ptr(profiles)), plan)


def gke_velocity_vorticity(plan, v_eta, mean_uw, nsnap, fields):
    _check(lib().gke_velocity_vorticity(plan, ptr(v_eta), ptr(mean_uw), nsnap, ptr(fields)), plan)


def gke_compute(plan, fields, nsnap, terms, profiles=None):
    _check(lib().gke_compute(plan, ptr(fields), nsnap, ptr(terms), ptr(profiles)), plan)


def gke_compute_graph(plan, fields, nsnap, terms, profiles=None):
    _check(lib().gke_compute_graph(plan, ptr(fields), nsnap, ptr(terms), ptr(profiles)), plan)


def gke_plan_knobs(plan):
    """(transform scratch per pair chunk in MiB, wavenumbers per combine CTA, source)."""
    w, kc, src = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().gke_plan_knobs(plan, ctypes.byref(w), ctypes.byref(kc), ctypes.byref(src)), plan)
    return w.value, kc.value, src.value


def gke_term_set(term_mask: int) -> int:
    return lib().gke_term_set(term_mask)


def gke_pair_labels(plan):
    import numpy as np
    n = lib().gke_npair(plan)
    Y, ry = np.zeros(n), np.zeros(n)
    i1, i2 = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.int32)
    _check(lib().gke_pair_labels(plan, ptr(Y), ptr(ry), ptr(i1), ptr(i2)), plan)
    return Y, ry, i1, i2


def gke_npair(plan) -> int:
    return lib().gke_npair(plan)


def gke_separation_labels(plan):
    """Kept separation indices (m_z[nrz], m_x[nrx]) as int32 arrays."""
    import numpy as np
    nrz, nrx = ctypes.c_int(), ctypes.c_int()
    _check(lib().gke_separation_labels(plan, ctypes.addressof(nrz), ctypes.addressof(nrx), None, None), plan)
    mz, mx = np.zeros(nrz.value, dtype=np.int32), np.zeros(nrx.value, dtype=np.int32)
    _check(lib().gke_separation_labels(plan, None, None, ptr(mz), ptr(mx)), plan)
    return mz, mx


def gke_terms_bytes(plan) -> int:
    return lib().gke_terms_bytes(plan)


def gke_reset(plan):
    _check(lib().gke_reset(plan), plan)


def gke_checkpoint(plan, path: str):
    _check(lib().gke_checkpoint(plan, path.encode()), plan)


def gke_restore(plan, path: str):
    _check(lib().gke_restore(plan, path.encode()), plan)


def gke_merge(plan, path: str):
    _check(lib().gke_merge(plan, path.encode()), plan)


def gke_fd_weights(y, j):
    import numpy as np
    yy = np.ascontiguousarray(y, dtype=np.float64)
    w = np.zeros(5)
    dp = ctypes.POINTER(ctypes.c_double)
    l0 = lib().gke_fd_weights(yy.ctypes.data_as(dp), len(yy), j, w.ctypes.data_as(dp))
    if l0 < 0:
        raise GkeError(-1, "bad arguments")
    return l0, w


def gke_compute_noalloc(nx, nz, ny, Lx, Lz, nu, y, fields, nsnap, terms, profiles=None, stream=None, term_mask=0):
    """FP64 pass without device allocation (device pointers only); raises GkeError."""
    import numpy as np
    yy = np.ascontiguousarray(y, dtype=np.float64)
    desc = gke_desc(nx, nz, ny, Lx, Lz, nu, yy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nsnap,
                    GKE_PREC_F64, GKE_DOMAIN_TRIANGLE, (ctypes.c_int * 4)(), (ctypes.c_int * 4)(), term_mask, None)
    st = lib().gke_compute_noalloc(ctypes.byref(desc), ptr(fields), nsnap, ptr(terms), ptr(profiles), stream)
    if st != GKE_OK:
        raise GkeError(st, "gke_compute_noalloc")


def gke_set_timing(plan, on: bool):
    _check(lib().gke_set_timing(plan, 1 if on else 0), plan)


def gke_stage_times(plan):
    """dict stage -> device ms since the last read (synchronises the plan's stream)."""
    import numpy as np
    ms = np.zeros(len(STAGES))
    _check(lib().gke_stage_times(plan, ptr(ms)), plan)
    return dict(zip(STAGES, ms.tolist()))


def gke_launch_count(plan) -> int:
    return lib().gke_launch_count(plan)


def gke_last_error(plan) -> str:
    m = lib().gke_last_error(plan)
    return m.decode() if m else ""


def gke_destroy(plan):
    lib().gke_destroy(plan)


# ------------------------------------------------- one homogeneous direction

def _check1h(status: int, plan) -> None:
    if status != GKE_OK:
        msg = lib().gke1h_last_error(plan)
        raise GkeError(status, msg.decode() if msg else "")


def gke1h_plan(nx, ny, nz, Lx, nu, y, z, max_snap, stream=None, precision=GKE_PREC_F64):
    import numpy as np
    yy = np.ascontiguousarray(y, dtype=np.float64)
    zz = np.ascontiguousarray(z, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    desc = gke1h_desc(nx, ny, nz, Lx, nu, yy.ctypes.data_as(dp), zz.ctypes.data_as(dp), max_snap, precision)
    out = ctypes.c_void_p()
    _check1h(lib().gke1h_plan(ctypes.byref(desc), stream, ctypes.byref(out)), None)
    return out.value


def gke1h_compute(plan, fields, nsnap, terms, profiles=None):
    _check1h(lib().gke1h_compute(plan, ptr(fields), nsnap, ptr(terms), ptr(profiles)), plan)


def gke1h_npair(plan) -> int:
    return lib().gke1h_npair(plan)


def gke1h_pair_labels(y, z):
    """(p1, p2, Y1, Z1, Y2, Z2) arrays of the output pairs of grids y, z."""
    import numpy as np
    yy = np.ascontiguousarray(y, dtype=np.float64)
    zz = np.ascontiguousarray(z, dtype=np.float64)
    P = len(yy) * len(zz)
    n = P * (P + 1) // 2
    p1, p2 = np.zeros(n, dtype=np.int32), np.zeros(n, dtype=np.int32)
    Y1, Z1, Y2, Z2 = (np.zeros(n) for _ in range(4))
    dp = ctypes.POINTER(ctypes.c_double)
    got = lib().gke1h_pair_labels(len(yy), len(zz), yy.ctypes.data_as(dp), zz.ctypes.data_as(dp), ptr(p1), ptr(p2),
                                  ptr(Y1), ptr(Z1), ptr(Y2), ptr(Z2))
    if got != n:
        raise GkeError(-1, "bad arguments")
    return p1, p2, Y1, Z1, Y2, Z2


def gke1h_set_timing(plan, on: bool):
    _check1h(lib().gke1h_set_timing(plan, 1 if on else 0), plan)


def gke1h_stage_times(plan):
    import numpy as np
    ms = np.zeros(len(STAGES))
    _check1h(lib().gke1h_stage_times(plan, ptr(ms)), plan)
    return dict(zip(STAGES, ms.tolist()))


def gke1h_launch_count(plan) -> int:
    return lib().gke1h_launch_count(plan)


def gke1h_last_error(plan) -> str:
    m = lib().gke1h_last_error(plan)
    return m.decode() if m else ""


def gke1h_destroy(plan):
    lib().gke1h_destroy(plan)
