"""ctypes front end of oracle/wq_oracle_rows.c (plain C nested WQ sums).

TEST INFRASTRUCTURE ONLY (tests/, smoke(), bench.py cpu_baseline / reference
legs). build_oracle() compiles the C file with gcc; rows_c() evaluates sampled
rows of an Oracle3D, optionally over several host threads (ctypes releases the
GIL during the foreign call, so threads run the C loops in parallel).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wq_oracle_rows.c")
_LIB = os.path.join(_HERE, "libwq_oracle.so")
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the C oracle into oracle/libwq_oracle.so (portable flags only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-o", _LIB, _SRC])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build_oracle()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.wq_oracle_rows.argtypes = [ctypes.c_int, P, P] + [P] * 3 + [P] * 3 + [P] * 6 + \
            [P, ctypes.c_int, ctypes.c_int64, P, P, P]
        lib.wq_oracle_rows.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def row_lengths(orc, rows: np.ndarray) -> np.ndarray:
    out = []
    for r in rows:
        i = orc.row_multi(int(r))
        out.append(int(np.prod([len(d.I[ik]) for d, ik in zip(orc.dirs, i)])))
    return np.array(out, dtype=np.int64)


def rows_c(orc, rows, which: str, threads: int = 1) -> list:
    """Nonzeros of each row (ascending columns) from the C nested sums."""
    lib = _load()
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    lens = row_lengths(orc, rows)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    out = np.zeros(int(offs[-1]))
    keep = []
    def arr(x, dt=np.float64):
        a = np.ascontiguousarray(x, dtype=dt)
        keep.append(a)
        return a
    n = arr(np.array(orc.n), np.int64)
    nqp = arr(np.array(orc.nqp), np.int64)
    W = [arr(d.W) for d in orc.dirs]
    B = [arr(d.B) for d in orc.dirs]
    qlo = [arr([q[0] for q in d.Q], np.int64) for d in orc.dirs]
    qhi = [arr([q[-1] + 1 for q in d.Q], np.int64) for d in orc.dirs]
    coef = arr(orc.coef)
    flag = 1 if which == "mass" else 0

    def run(lo, hi):
        if hi <= lo:
            return
        sub_rows = np.ascontiguousarray(rows[lo:hi])
        sub_off = np.ascontiguousarray(offs[lo:hi] - offs[lo])
        view = out[offs[lo]:offs[hi]]
        buf = np.zeros(len(view))
        lib.wq_oracle_rows(orc.p, _ptr(n), _ptr(nqp), *[_ptr(w) for w in W], *[_ptr(b) for b in B],
                           _ptr(qlo[0]), _ptr(qhi[0]), _ptr(qlo[1]), _ptr(qhi[1]),
                           _ptr(qlo[2]), _ptr(qhi[2]), _ptr(coef), flag,
                           len(sub_rows), _ptr(sub_rows), _ptr(sub_off), _ptr(buf))
        view[:] = buf

    if threads <= 1:
        run(0, len(rows))
    else:
        bounds = np.linspace(0, len(rows), threads * 4 + 1).astype(int)
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(lambda k: run(bounds[k], bounds[k + 1]), range(len(bounds) - 1)))
    res = [out[offs[k]:offs[k + 1]] for k in range(len(rows))]
    if getattr(orc, "nurbs_basis", False):
        res = [v * orc.basis_scale(int(r), which) for r, v in zip(rows, res)]
    return res
