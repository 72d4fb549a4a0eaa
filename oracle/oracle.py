"""FP64 oracle for NDGSBP decoding -- Python entry points.

TEST INFRASTRUCTURE ONLY: the correctness reference for the CUDA decoder.  Only the test suite,
the package smoke check and the CPU-baseline leg of the benchmark import this module.  It shares
no code with the CUDA library (it never imports the package; the package never imports it).

The arithmetic lives in ``ndgsbp_oracle.c`` (plain C, FP64, compiled by ``build()``); this file
marshals numpy arrays into it and adds the small pure-Python references:

* ``brute_force_map``  bitwise-MAP LLRs by enumerating every codeword (tiny codes only).  Belief
  propagation is exact on cycle-free Tanner graphs, so every schedule of the paper must reach
  these values there.
* ``group_sizes`` / ``groups`` / ``budget_iters`` / ``cocsg``  Step 1 and the size relations of
  Sec. II-A and Sec. IV.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ndgsbp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libndgsbp_oracle.so")
_lib = None
_lock = threading.Lock()

ORACLE_EINVAL = -1
ORACLE_EINFEASIBLE = -2


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build (gcc, no fast-math, -O2)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=c99",
                               "-D_POSIX_C_SOURCE=200809L", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            I, D, P, L, U64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_long, ctypes.c_uint64
            lib.oracle_group_sizes.argtypes = [I, I, D, I, P, P, P]
            lib.oracle_groups.argtypes = [I, I, I, D, U64, I, I, P, P, I]
            lib.oracle_budget_iters.argtypes = [I, I, I, D, I]
            lib.oracle_ndgsbp_decode.argtypes = [I, I, P, P, I, P, P, I, P, L, I, D, I, I,
                                                 P, P, P, P, P, I]
            lib.oracle_group_posterior_decode.argtypes = [I, I, P, P, I, P, P, P, L, I, D, I,
                                                          P, P, P, P, P, I]
            lib.oracle_flood_decode.argtypes = [I, I, P, P, P, L, I, D, I, P, P, P, P, P, I]
            lib.oracle_layered_decode.argtypes = [I, I, P, P, P, L, I, D, I, P, P, P, P, P, I]
            lib.oracle_vertical_decode.argtypes = [I, I, P, P, I, P, P, P, L, I, D, I, P, P, P, P, P, I]
            lib.oracle_philox4x32_10.argtypes = [P, P, P]
            lib.oracle_awgn_llr.argtypes = [I, L, D, D, U64, P, P]
            _lib = lib
    return _lib


class swapped_library:
    """Context manager that points this module at another build of the oracle (used by the
    tests that plant a mistake in a copy of the C source and check that a pin catches it)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self._saved = _lib
        lib = ctypes.CDLL(self.path)
        for name in ("oracle_group_sizes", "oracle_groups", "oracle_budget_iters",
                     "oracle_ndgsbp_decode", "oracle_group_posterior_decode",
                     "oracle_flood_decode", "oracle_layered_decode", "oracle_vertical_decode",
                     "oracle_philox4x32_10", "oracle_awgn_llr"):
            getattr(lib, name).argtypes = getattr(self._saved, name).argtypes
        with _lock:
            _lib = lib
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self._saved
        return False


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile a modified copy of the oracle source (tests only)."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-std=c99",
                           "-D_POSIX_C_SOURCE=200809L", "-o", out_path, c_path, "-lm"])
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _check(rc, what):
    if rc < 0:
        raise ValueError(f"oracle {what} failed with code {rc}")
    return rc


# ------------------------------------------------------------------------------------------
# Step 1 and size relations
# ------------------------------------------------------------------------------------------

def group_sizes(M: int, G: int, r: float, cyclic: bool = False):
    """(N_G, o, fresh[G]) from G N_G - (G-1) N_G r = M (Sec. II-A), in the integer reading
    documented in ndgsbp_oracle.c."""
    lib = _load()
    NG = ctypes.c_int()
    o = ctypes.c_int()
    fresh = np.zeros(G, np.int32)
    _check(lib.oracle_group_sizes(M, G, float(r), int(cyclic), ctypes.byref(NG), ctypes.byref(o),
                                  _ptr(fresh)), "group_sizes")
    return NG.value, o.value, fresh


def groups(M: int, G: int, r: float, seed: int, unit: int = 1, cyclic: bool = False,
           natural: bool = False):
    """Step 1 of Sec. II-C.  Returns (grp_ptr[G+1], grp_cn[]) as int32 arrays of CN indices."""
    lib = _load()
    cap = 4 * M + 16
    gp = np.zeros(G + 1, np.int32)
    gc = np.zeros(cap, np.int32)
    n = _check(lib.oracle_groups(M, unit, G, float(r), ctypes.c_uint64(seed & (2**64 - 1)),
                                 int(cyclic), int(natural), _ptr(gp), _ptr(gc), cap), "groups")
    return gp, gc[:n].copy()


def groups_structured(code, G: int, r: float, seed: int):
    """Structure-aware Step 1 (the CoCSG-raising direction the paper names as future work):
    group 1 and every overlap as in Step 1 (linear groups of CNs); the fresh CNs of group g >= 2
    are picked one at a time, each the unused CN adding the most VNs of the previous group's VN
    neighbourhood N(G_{g-1}) that group g does not reach yet; ties go to the earlier CN in the
    Fisher-Yates order of SplitMix64(seed) (the order Step 1 draws from).  Returns (grp_ptr,
    grp_cn) like ``groups``."""
    M = code.M
    NG, o, fresh = group_sizes(M, G, r)
    order = [int(m) for m in groups(M, 1, 0.0, seed, unit=1, cyclic=True)[1]]   # the full draw
    rows = [set(int(v) for v in row) for row in code.rows()]
    out = [order[:NG]]
    used = set(out[0])
    for g in range(1, G):
        prev = out[g - 1]
        nbr = set().union(*(rows[m] for m in prev))
        cur = prev[len(prev) - o:]
        reach = set().union(*(rows[m] for m in cur)) if cur else set()
        for _ in range(int(fresh[g])):
            best, best_gain = None, -1
            for i in range(NG, M):
                m = order[i]
                if m in used:
                    continue
                gain = len((rows[m] & nbr) - reach)
                if gain > best_gain:
                    best, best_gain = m, gain
            used.add(best)
            cur.append(best)
            reach |= rows[best]
        out.append(cur)
    gp = np.zeros(G + 1, np.int32)
    gp[1:] = np.cumsum([len(x) for x in out])
    return gp, np.asarray([m for x in out for m in x], np.int32)


def budget_iters(M: int, G: int, NG: int, r: float, imax: int) -> int:
    """Equal-complexity iteration allowance of Sec. IV: M I_max / (M + (G-1) N_G r)."""
    return int(_load().oracle_budget_iters(M, G, NG, float(r), imax))


def cocsg(code, grp_ptr, grp_cn) -> float:
    """CoCSG l (Sec. I, II-A): the mean, over consecutive group pairs (g-1, g), of the number of
    VNs adjacent to both a CN of G_{g-1} and a CN of G_g."""
    rows = code.rows()
    G = len(grp_ptr) - 1
    if G < 2:
        return 0.0
    vsets = []
    for g in range(G):
        s = set()
        for m in grp_cn[grp_ptr[g]:grp_ptr[g + 1]]:
            s.update(int(v) for v in rows[int(m)])
        vsets.append(s)
    return float(np.mean([len(vsets[g] & vsets[g - 1]) for g in range(1, G)]))


# ------------------------------------------------------------------------------------------
# Decoders
# ------------------------------------------------------------------------------------------

class Result:
    """Per-frame decoder outputs: hard [F, N] uint8, iters [F], synd_ok [F], total [F, N]
    (FP64, Eq. (3)) and c2v [F, E] (CN->VN messages in CSR edge order) when requested."""

    def __init__(self, hard, iters, synd_ok, total, c2v):
        self.hard, self.iters, self.synd_ok, self.total, self.c2v = hard, iters, synd_ok, total, c2v


def _alloc(code, F, want_total, want_c2v):
    hard = np.zeros((F, code.N), np.uint8)
    iters = np.zeros(F, np.int32)
    ok = np.zeros(F, np.uint8)
    tot = np.zeros((F, code.N)) if want_total else None
    c2v = np.zeros((F, code.E)) if want_c2v else None
    return hard, iters, ok, tot, c2v


def _threads(n):
    if n is not None:
        return int(n)
    return max(1, len(os.sched_getaffinity(0)))


def ndgsbp_decode(code, grp_ptr, grp_cn, llr, max_iter: int, llr_max: float = 20.0,
                  early_stop: bool = True, stop_after_subiters: int = -1,
                  want_total: bool = True, want_c2v: bool = False, n_threads=None) -> Result:
    """Steps 2-4 of Sec. II-C over every frame of ``llr`` [F, N].  ``grp_ptr`` is one grouping
    ([G+1]) or several ([K, G+1], cycled by iteration) into ``grp_cn``."""
    lib = _load()
    llr = np.ascontiguousarray(llr, np.float64)
    F = llr.shape[0]
    gp = np.ascontiguousarray(np.atleast_2d(grp_ptr), np.int32)
    K, G1 = gp.shape
    gc = np.ascontiguousarray(grp_cn, np.int32)
    rp = np.ascontiguousarray(code.row_ptr, np.int32)
    ci = np.ascontiguousarray(code.col_idx, np.int32)
    hard, iters, ok, tot, c2v = _alloc(code, F, want_total, want_c2v)
    _check(lib.oracle_ndgsbp_decode(code.M, code.N, _ptr(rp), _ptr(ci), G1 - 1, _ptr(gp), _ptr(gc),
                                    K, _ptr(llr), F, max_iter, float(llr_max), int(early_stop),
                                    int(stop_after_subiters), _ptr(hard), _ptr(iters), _ptr(ok),
                                    _ptr(tot), _ptr(c2v), _threads(n_threads)), "ndgsbp_decode")
    return Result(hard, iters, ok, tot, c2v)


def group_posterior_decode(code, grp_ptr, grp_cn, llr, max_iter: int, llr_max: float = 20.0,
                           early_stop: bool = True, want_total: bool = True,
                           want_c2v: bool = False, n_threads=None) -> Result:
    """Textbook group-shuffled BP in posterior form (independent formulation of Step 2)."""
    lib = _load()
    llr = np.ascontiguousarray(llr, np.float64)
    F = llr.shape[0]
    gp = np.ascontiguousarray(grp_ptr, np.int32)
    gc = np.ascontiguousarray(grp_cn, np.int32)
    rp = np.ascontiguousarray(code.row_ptr, np.int32)
    ci = np.ascontiguousarray(code.col_idx, np.int32)
    hard, iters, ok, tot, c2v = _alloc(code, F, want_total, want_c2v)
    _check(lib.oracle_group_posterior_decode(code.M, code.N, _ptr(rp), _ptr(ci), len(gp) - 1,
                                             _ptr(gp), _ptr(gc), _ptr(llr), F, max_iter,
                                             float(llr_max), int(early_stop), _ptr(hard),
                                             _ptr(iters), _ptr(ok), _ptr(tot), _ptr(c2v),
                                             _threads(n_threads)), "group_posterior")
    return Result(hard, iters, ok, tot, c2v)


def flood_decode(code, llr, max_iter: int, llr_max: float = 20.0, early_stop: bool = True,
                 want_total: bool = True, want_c2v: bool = False, n_threads=None) -> Result:
    """Textbook flooding sum-product (reference for the G = 1 reduction)."""
    lib = _load()
    llr = np.ascontiguousarray(llr, np.float64)
    F = llr.shape[0]
    rp = np.ascontiguousarray(code.row_ptr, np.int32)
    ci = np.ascontiguousarray(code.col_idx, np.int32)
    hard, iters, ok, tot, c2v = _alloc(code, F, want_total, want_c2v)
    _check(lib.oracle_flood_decode(code.M, code.N, _ptr(rp), _ptr(ci), _ptr(llr), F, max_iter,
                                   float(llr_max), int(early_stop), _ptr(hard), _ptr(iters),
                                   _ptr(ok), _ptr(tot), _ptr(c2v), _threads(n_threads)), "flood")
    return Result(hard, iters, ok, tot, c2v)


def layered_decode(code, llr, max_iter: int, llr_max: float = 20.0, early_stop: bool = True,
                   want_total: bool = True, want_c2v: bool = False, n_threads=None) -> Result:
    """Textbook row-serial layered BP (reference for the one-CN-per-group reduction)."""
    lib = _load()
    llr = np.ascontiguousarray(llr, np.float64)
    F = llr.shape[0]
    rp = np.ascontiguousarray(code.row_ptr, np.int32)
    ci = np.ascontiguousarray(code.col_idx, np.int32)
    hard, iters, ok, tot, c2v = _alloc(code, F, want_total, want_c2v)
    _check(lib.oracle_layered_decode(code.M, code.N, _ptr(rp), _ptr(ci), _ptr(llr), F, max_iter,
                                     float(llr_max), int(early_stop), _ptr(hard), _ptr(iters),
                                     _ptr(ok), _ptr(tot), _ptr(c2v), _threads(n_threads)), "layered")
    return Result(hard, iters, ok, tot, c2v)


def vertical_decode(code, grp_ptr, grp_vn, llr, max_iter: int, llr_max: float = 20.0, early_stop: bool = True,
                    want_total: bool = True, want_c2v: bool = False, n_threads=None) -> Result:
    """Vertical group shuffled BP (VN groups, Sec. I): grp_ptr [G+1] into grp_vn, a partition of
    the VNs processed in that order every iteration."""
    lib = _load()
    llr = np.ascontiguousarray(llr, np.float64)
    F = llr.shape[0]
    gp = np.ascontiguousarray(grp_ptr, np.int32)
    gv = np.ascontiguousarray(grp_vn, np.int32)
    rp = np.ascontiguousarray(code.row_ptr, np.int32)
    ci = np.ascontiguousarray(code.col_idx, np.int32)
    hard, iters, ok, tot, c2v = _alloc(code, F, want_total, want_c2v)
    _check(lib.oracle_vertical_decode(code.M, code.N, _ptr(rp), _ptr(ci), len(gp) - 1, _ptr(gp), _ptr(gv),
                                      _ptr(llr), F, max_iter, float(llr_max), int(early_stop), _ptr(hard),
                                      _ptr(iters), _ptr(ok), _ptr(tot), _ptr(c2v), _threads(n_threads)), "vertical")
    return Result(hard, iters, ok, tot, c2v)


# ------------------------------------------------------------------------------------------
# Channel
# ------------------------------------------------------------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: counter (4 x uint32), key (2 x uint32) -> 4 x uint32."""
    lib = _load()
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib.oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def awgn_llr(N: int, n_frames: int, ebn0_db: float, rate: float, seed: int,
             codeword=None) -> np.ndarray:
    """Channel LLRs [n_frames, N] (FP64) from the Philox/Box-Muller definition in
    ndgsbp_oracle.c (the definition the CUDA generator also implements)."""
    lib = _load()
    out = np.zeros((n_frames, N))
    cw = None if codeword is None else np.ascontiguousarray(codeword, np.uint8)
    _check(lib.oracle_awgn_llr(N, n_frames, float(ebn0_db), float(rate),
                               ctypes.c_uint64(seed & (2**64 - 1)), _ptr(cw), _ptr(out)), "awgn")
    return out


# ------------------------------------------------------------------------------------------
# Pure-Python references for tiny codes
# ------------------------------------------------------------------------------------------

def codewords(code) -> np.ndarray:
    """Every codeword of a tiny code (N <= 22), by enumeration of all 2^N words."""
    if code.N > 22:
        raise ValueError("enumeration is for tiny codes only")
    H = code.dense().astype(np.int64)
    words = np.array(list(itertools.product((0, 1), repeat=code.N)), dtype=np.int64)
    synd = (words @ H.T) % 2
    return words[(synd == 0).all(axis=1)].astype(np.uint8)


def brute_force_map(code, llr) -> np.ndarray:
    """Bitwise-MAP LLRs log P(c_n = 0 | y) / P(c_n = 1 | y) for each frame of ``llr`` [F, N],
    by summing the channel likelihood exp(sum_n (1 - 2 c_n) L_n / 2) over all codewords."""
    cws = codewords(code).astype(np.float64)
    llr = np.atleast_2d(np.asarray(llr, np.float64))
    out = np.zeros_like(llr)
    sgn = 1.0 - 2.0 * cws                     # [C, N]
    for f in range(llr.shape[0]):
        a = sgn @ (0.5 * llr[f])              # log-likelihood of each codeword, up to a constant
        a = a - a.max()
        w = np.exp(a)
        p0 = (w[:, None] * (cws == 0)).sum(axis=0)
        p1 = (w[:, None] * (cws == 1)).sum(axis=0)
        out[f] = np.log(p0) - np.log(p1)
    return out
