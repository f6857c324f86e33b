"""Host-side merge of GKE checkpoint files: the paper's independent jobs over
snapshot subsets, merged before Step 3 (Sec. 3.4).

Each job (a plan on any GPU or machine) writes its partial sums with
gke_checkpoint; this module adds the files on the host into one that
gke_restore loads, with the same result as gke_merge.  File layout (little
endian; the C struct of the library, include/gke.h):

  header   char magic[8] = "GKECKPT\\0"; int32 version (5), nx, nz, ny,
           precision, have_acc, pair_domain, nzt, nxt, term_set, acc_kind,
           reserved; float64 mean_count, snap_count, Lx, Lz, nu
  float64  mean_sum[4][ny]          Step-1 sums of U, V, W, P
  float64  stats[7][ny]             one-point sums
  float64  mean[4][ny]              the mean the spectra were taken about
                                    (only if have_acc)
  complex128 acc[...]               spectra (only if have_acc): per-pair term
                                    spectra (acc_kind 0), the plane spectra
                                    of the split path on one 128-row tile (1)
                                    or the coarse term spectra of the chunked
                                    mode for every triangle pair (2)

The spectra of each job are sums over its snapshots of products of
fluctuations about a Step-1 mean, so jobs add exactly only when they used the
same mean (Step 1 before Step 2, Sec. 3.2); files whose means differ are
refused.

Usage: python -m paper_1910_06409_gb300.merge OUT IN [IN ...]
"""
from __future__ import annotations

import sys

import numpy as np

HEADER = np.dtype([("magic", "S8"), ("version", "<i4"), ("nx", "<i4"), ("nz", "<i4"), ("ny", "<i4"),
                   ("precision", "<i4"), ("have_acc", "<i4"), ("pair_domain", "<i4"), ("nzt", "<i4"),
                   ("nxt", "<i4"), ("term_set", "<i4"), ("acc_kind", "<i4"), ("reserved", "<i4"),
                   ("mean_count", "<f8"), ("snap_count", "<f8"), ("Lx", "<f8"), ("Lz", "<f8"), ("nu", "<f8")])
MAGIC = b"GKECKPT"
VERSION = 5
NSTAT = 7
GRID = ("nx", "nz", "ny", "pair_domain", "nzt", "nxt", "term_set", "acc_kind", "Lx", "Lz", "nu")
MEAN_RTOL = 1e-12             # frozen means closer than this (relative) are the same mean


class CheckpointError(ValueError):
    pass


def read(path: str) -> dict:
    """Header fields and arrays of one checkpoint file."""
    with open(path, "rb") as f:
        raw = f.read()
    if len(raw) < HEADER.itemsize:
        raise CheckpointError(f"{path}: too short for a checkpoint header")
    h = np.frombuffer(raw, dtype=HEADER, count=1)[0]
    if h["magic"] != MAGIC or int(h["version"]) != VERSION:
        raise CheckpointError(f"{path}: not a version-{VERSION} GKE checkpoint")
    ny = int(h["ny"])
    off = HEADER.itemsize
    n_mean, n_stat = 4 * ny, NSTAT * ny
    need = off + 8 * (n_mean + n_stat)
    if len(raw) < need:
        raise CheckpointError(f"{path}: truncated")
    mean_sum = np.frombuffer(raw, dtype="<f8", count=n_mean, offset=off).copy()
    stats = np.frombuffer(raw, dtype="<f8", count=n_stat, offset=off + 8 * n_mean).copy()
    acc = mean = None
    rest = len(raw) - need
    if int(h["have_acc"]):
        if rest <= 8 * n_mean or (rest - 8 * n_mean) % 16:
            raise CheckpointError(f"{path}: truncated accumulator")
        mean = np.frombuffer(raw, dtype="<f8", count=n_mean, offset=need).copy()
        acc = np.frombuffer(raw, dtype="<c16", count=(rest - 8 * n_mean) // 16, offset=need + 8 * n_mean).copy()
    elif rest:
        raise CheckpointError(f"{path}: trailing bytes without accumulator")
    return {"header": {n: h[n].item() for n in HEADER.names}, "mean_sum": mean_sum, "stats": stats,
            "mean": mean, "acc": acc}


def write(path: str, ck: dict) -> None:
    h = np.zeros(1, dtype=HEADER)
    for n, v in ck["header"].items():
        h[n] = v
    h["magic"] = MAGIC
    h["version"] = VERSION
    h["have_acc"] = 1 if ck["acc"] is not None else 0
    if ck["acc"] is not None and ck.get("mean") is None:
        raise CheckpointError("a checkpoint with spectra needs the mean they were taken about")
    with open(path, "wb") as f:
        f.write(h.tobytes())
        f.write(np.ascontiguousarray(ck["mean_sum"], dtype="<f8").tobytes())
        f.write(np.ascontiguousarray(ck["stats"], dtype="<f8").tobytes())
        if ck["acc"] is not None:
            f.write(np.ascontiguousarray(ck["mean"], dtype="<f8").tobytes())
            f.write(np.ascontiguousarray(ck["acc"], dtype="<c16").tobytes())


def same_mean(a: np.ndarray, b: np.ndarray) -> bool:
    """Two frozen Step-1 means equal up to the rounding of their sums."""
    scale = max(float(np.abs(a).max(initial=0.0)), float(np.abs(b).max(initial=0.0)), 1e-300)
    return float(np.abs(a - b).max(initial=0.0)) <= MEAN_RTOL * scale


def merge(paths, out: str) -> dict:
    """Sum the checkpoints `paths` into `out` (sums, sample counts, spectra)."""
    if not paths:
        raise CheckpointError("nothing to merge")
    tot = read(paths[0])
    for p in paths[1:]:
        ck = read(p)
        for n in GRID:
            if ck["header"][n] != tot["header"][n]:
                raise CheckpointError(f"{p}: {n} differs ({ck['header'][n]} vs {tot['header'][n]})")
        tot["mean_sum"] += ck["mean_sum"]
        tot["stats"] += ck["stats"]
        tot["header"]["mean_count"] += ck["header"]["mean_count"]
        tot["header"]["snap_count"] += ck["header"]["snap_count"]
        if ck["acc"] is not None:
            if tot["acc"] is None:
                tot["acc"] = ck["acc"].copy()
                tot["mean"] = ck["mean"].copy()
            elif tot["acc"].shape != ck["acc"].shape:
                raise CheckpointError(f"{p}: accumulator size differs")
            elif not same_mean(tot["mean"], ck["mean"]):
                raise CheckpointError(f"{p}: spectra taken about another Step-1 mean (jobs must share the mean)")
            else:
                tot["acc"] += ck["acc"]
    write(out, tot)
    return tot


def main(argv=None) -> int:
    argv = sys.argv[1:] if argv is None else argv
    if len(argv) < 2:
        print(__doc__.strip().splitlines()[-1], file=sys.stderr)
        return 2
    merge(argv[1:], argv[0])
    return 0


if __name__ == "__main__":
    sys.exit(main())
