"""Seeded synthetic inputs: LDPC parity-check matrices, codewords and channel samples.

This module is the only code that the FP64 oracle and the CUDA decoder both consume.  It holds
none of the decoder's arithmetic: it builds the problem that Sec. II-B and II-C of the paper
state (an M x N sparse parity-check matrix H, a BPSK-mapped codeword sent over an AWGN channel
with noise variance sigma^2, channel LLRs L_n = 2 y_n / sigma^2) from fixed seeds, so that both
sides decode the same frames.

Codes are synthetic stand-ins for the paper's MacKay codes, which are not available here:

* ``gallager_code``   regular (dv, dc) Gallager ensemble, 4-cycles removed by column swaps.
* ``qc_code``         quasi-cyclic code from a base matrix: a dual-diagonal parity part and a
                      systematic part with a stated column-degree profile, circulant shifts
                      drawn from a seed while avoiding 4-cycles where the lift size allows.
* ``tree_code``       small cycle-free Tanner graphs (belief propagation is exact on them).
* ``fig1_code``       the eight-VN, four-CN graph of the paper's Fig. 1 discussion (Sec. II-A).

All matrices are returned as ``Code`` objects holding CSR arrays (int32, columns sorted).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Code", "code_from_rows", "gallager_code", "qc_code", "tree_code", "fig1_code",
    "design_rate", "sigma2_from_ebn0", "channel_llr", "random_codeword", "has_4cycle",
    "code_by_name", "CODE_NAMES", "degree_profile", "write_alist", "read_alist",
]


@dataclasses.dataclass
class Code:
    """A binary LDPC code given by its parity-check matrix H (M x N) in CSR form."""
    name: str
    M: int
    N: int
    row_ptr: np.ndarray          # int32 [M+1]
    col_idx: np.ndarray          # int32 [E], sorted within each row
    Z: int = 0                   # lift size for QC codes (rows come in layers of Z), else 0
    base: np.ndarray | None = None   # QC base matrix of circulant shifts, -1 = zero block

    @property
    def E(self) -> int:
        return int(self.row_ptr[-1])

    def rows(self):
        return [self.col_idx[self.row_ptr[m]:self.row_ptr[m + 1]] for m in range(self.M)]

    def dense(self) -> np.ndarray:
        H = np.zeros((self.M, self.N), dtype=np.uint8)
        for m in range(self.M):
            H[m, self.col_idx[self.row_ptr[m]:self.row_ptr[m + 1]]] = 1
        return H

    def row_degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)

    def col_degrees(self) -> np.ndarray:
        return np.bincount(self.col_idx, minlength=self.N).astype(np.int64)


def code_from_rows(rows, N: int, name: str = "custom", Z: int = 0, base=None) -> Code:
    """Build a Code from a list of per-row column lists (duplicates rejected)."""
    row_ptr = [0]
    cols = []
    for r in rows:
        rs = sorted(int(c) for c in r)
        if len(set(rs)) != len(rs):
            raise ValueError("duplicate column in a row")
        if rs and (rs[0] < 0 or rs[-1] >= N):
            raise ValueError("column index out of range")
        cols.extend(rs)
        row_ptr.append(len(cols))
    return Code(name=name, M=len(rows), N=N, row_ptr=np.asarray(row_ptr, np.int32),
                col_idx=np.asarray(cols, np.int32), Z=Z,
                base=None if base is None else np.asarray(base, np.int64))


def has_4cycle(code: Code) -> bool:
    """True if two rows of H share two or more columns (a length-4 cycle in the Tanner graph)."""
    seen = set()
    for r in code.rows():
        r = [int(c) for c in r]
        for a in range(len(r)):
            for b in range(a + 1, len(r)):
                key = (r[a], r[b])
                if key in seen:
                    return True
                seen.add(key)
    return False


def degree_profile(code: Code) -> dict:
    """Edge-perspective degree fractions lambda_i, rho_j (Sec. II-B)."""
    cd = code.col_degrees()
    rd = code.row_degrees()
    E = float(code.E)
    lam = {int(i): float((cd == i).sum() * i / E) for i in np.unique(cd)}
    rho = {int(j): float((rd == j).sum() * j / E) for j in np.unique(rd)}
    return {"lambda": lam, "rho": rho}


# ----------------------------------------------------------------------------------------
# alist files (MacKay's sparse-matrix text format, in which the paper's codes are published)
# ----------------------------------------------------------------------------------------

def write_alist(code: Code, path: str) -> None:
    """Write H as an alist file: "N M", the largest column and row weights, the N column and M
    row weights, then per column its rows and per row its columns (1-based, zero-padded to
    the largest weight)."""
    cols = [[] for _ in range(code.N)]
    for m, r in enumerate(code.rows()):
        for n in r:
            cols[int(n)].append(m)
    rows = [[int(n) for n in r] for r in code.rows()]
    mc = max((len(c) for c in cols), default=0)
    mr = max((len(r) for r in rows), default=0)
    lines = [f"{code.N} {code.M}", f"{mc} {mr}", " ".join(str(len(c)) for c in cols),
             " ".join(str(len(r)) for r in rows)]
    lines += [" ".join(str(m + 1) for m in c + [-1] * (mc - len(c))) for c in cols]
    lines += [" ".join(str(n + 1) for n in r + [-1] * (mr - len(r))) for r in rows]
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def read_alist(path: str, name: str | None = None) -> Code:
    """Read an alist file (the format written by write_alist); the row lists define H and the
    column lists must agree with them."""
    with open(path) as f:
        tok = [int(t) for t in f.read().split()]
    N, M, mc, mr = tok[0], tok[1], tok[2], tok[3]
    pos = 4
    cw = tok[pos:pos + N]
    pos += N
    rw = tok[pos:pos + M]
    pos += M
    cols = []
    for n in range(N):
        ent = tok[pos:pos + mc]
        pos += mc
        cols.append([m - 1 for m in ent if m > 0])
        if len(cols[-1]) != cw[n]:
            raise ValueError(f"column {n + 1}: weight {cw[n]} but {len(cols[-1])} entries")
    rows = []
    for m in range(M):
        ent = tok[pos:pos + mr]
        pos += mr
        rows.append([n - 1 for n in ent if n > 0])
        if len(rows[-1]) != rw[m]:
            raise ValueError(f"row {m + 1}: weight {rw[m]} but {len(rows[-1])} entries")
    from_cols = sorted((m, n) for n, c in enumerate(cols) for m in c)
    from_rows = sorted((m, n) for m, r in enumerate(rows) for n in r)
    if from_cols != from_rows:
        raise ValueError("column and row lists disagree")
    return code_from_rows(rows, N, name=name or path)


# ----------------------------------------------------------------------------------------
# Regular Gallager ensemble
# ----------------------------------------------------------------------------------------

def gallager_code(N: int, dv: int, dc: int, seed: int, remove_4cycles: bool = True,
                  name: str | None = None) -> Code:
    """Regular (dv, dc) code from Gallager's construction: dv stacked sub-matrices, the first a
    band of dc consecutive ones per row, the others column permutations of it.  4-cycles are
    removed by swapping columns between two rows of the same permuted sub-matrix (degrees and
    the sub-matrix structure are kept)."""
    if N % dc:
        raise ValueError("N must be a multiple of dc")
    rng = np.random.default_rng(seed)
    Ms = N // dc
    perms = [np.arange(N)] + [rng.permutation(N) for _ in range(dv - 1)]

    def rows_of():
        out = []
        for p in perms:
            for i in range(Ms):
                out.append(p[i * dc:(i + 1) * dc])
        return out

    if remove_4cycles:
        for _ in range(100000):
            rows = rows_of()
            owner = {}
            bad = None
            for ri, r in enumerate(rows):
                rs = sorted(int(c) for c in r)
                for a in range(dc):
                    for b in range(a + 1, dc):
                        key = (rs[a], rs[b])
                        if key in owner:
                            bad = (owner[key], ri, key)
                            break
                        owner[key] = ri
                    if bad:
                        break
                if bad:
                    break
            if bad is None:
                break
            r1, r2, (ca, cb) = bad
            # move one shared column out of the row that lives in a permuted sub-matrix
            ri = r2 if r2 >= Ms else r1
            sub = ri // Ms
            if sub == 0:
                sub, ri = r1 // Ms, r1
            p = perms[sub]
            local = ri % Ms
            pos = local * dc + int(np.where(p[local * dc:(local + 1) * dc] == ca)[0][0])
            other = int(rng.integers(0, N))
            p[pos], p[other] = p[other], p[pos]
        else:
            raise RuntimeError("4-cycle removal did not converge")
    rows = rows_of()
    return code_from_rows(rows, N, name=name or f"gallager_{dv}_{dc}_n{N}_s{seed}")


# ----------------------------------------------------------------------------------------
# Quasi-cyclic codes
# ----------------------------------------------------------------------------------------

def _qc_4cycle_free_with(base: np.ndarray, i: int, j: int, s: int, Z: int) -> bool:
    """Would placing shift s at (i, j) close a 4-cycle with the shifts already placed?"""
    mb, nb = base.shape
    for i2 in range(mb):
        if i2 == i or base[i2, j] < 0:
            continue
        for j2 in range(nb):
            if j2 == j or base[i, j2] < 0 or base[i2, j2] < 0:
                continue
            if (s - base[i, j2] + base[i2, j2] - base[i2, j]) % Z == 0:
                return False
    return True


def qc_code(mb: int, nb: int, Z: int, syst_degrees, seed: int, name: str | None = None) -> Code:
    """Quasi-cyclic LDPC code with an mb x nb base matrix lifted by Z.

    The last mb base columns are a dual-diagonal parity part (one weight-3 column at rows
    0, mb//2 and mb-1, then weight-2 columns on the staircase with shift 0).  The first nb-mb
    columns take the degrees in ``syst_degrees``; their rows are chosen to even out row
    degrees and their shifts are drawn uniformly, rejecting shifts that close a 4-cycle (up to
    a bounded number of draws).  Base entry (i, j) with shift s connects CN i*Z + c to VN
    j*Z + (c + s) mod Z for c in [0, Z).
    """
    syst_degrees = list(syst_degrees)
    if len(syst_degrees) != nb - mb:
        raise ValueError("need one degree per systematic base column")
    rng = np.random.default_rng(seed)
    base = -np.ones((mb, nb), dtype=np.int64)
    kp = nb - mb
    # parity part: weight-3 column then staircase
    a = int(rng.integers(1, Z))
    base[0, kp] = a
    base[mb // 2, kp] = int(rng.integers(0, Z)) if mb > 2 else a
    base[mb - 1, kp] = a
    for j in range(1, mb):
        base[j - 1, kp + j] = 0
        base[j, kp + j] = 0
    rowdeg = (base >= 0).sum(axis=1).astype(np.int64)
    order = sorted(range(kp), key=lambda j: -syst_degrees[j])
    for j in order:
        d = syst_degrees[j]
        if d > mb:
            raise ValueError("column degree exceeds base rows")
        keys = rowdeg + rng.random(mb) * 0.5
        rows = np.argsort(keys)[:d]
        for i in sorted(int(x) for x in rows):
            for _attempt in range(200):
                s = int(rng.integers(0, Z))
                if _qc_4cycle_free_with(base, i, j, s, Z):
                    break
            base[i, j] = s
            rowdeg[i] += 1
    rows_out = []
    for i in range(mb):
        for c in range(Z):
            cols = [j * Z + (c + int(base[i, j])) % Z for j in range(nb) if base[i, j] >= 0]
            rows_out.append(cols)
    return code_from_rows(rows_out, nb * Z, name=name or f"qc_{mb}x{nb}_Z{Z}_s{seed}",
                          Z=Z, base=base)


# ----------------------------------------------------------------------------------------
# Named codes used by the tests and the benchmark
# ----------------------------------------------------------------------------------------

def _c_gallager_1008():
    return gallager_code(1008, 3, 6, seed=1008, name="gallager36_n1008")


def _c_qc_2304_r12():
    # VN degrees {2,3,6}: 11 x 2 + 1 x 3 (parity), 6 x 3 + 6 x 6 (systematic)
    return qc_code(12, 24, 96, [6] * 6 + [3] * 6, seed=2304, name="qc_n2304_r12")


def _c_qc_16200_r23():
    # VN degrees {2,3,8}: 14 x 2 + 1 x 3 (parity), 6 x 8 + 24 x 3 (systematic)
    return qc_code(15, 45, 360, [8] * 6 + [3] * 24, seed=16200, name="qc_n16200_r23")


def _c_qc_576_r12():
    return qc_code(12, 24, 24, [6] * 6 + [3] * 6, seed=576, name="qc_n576_r12")


def _c_qc_1152_r23():
    return qc_code(8, 24, 48, [6] * 5 + [3] * 11, seed=1152, name="qc_n1152_r23")


def _c_qc_2304_r34():
    return qc_code(6, 24, 96, [6] * 7 + [3] * 11, seed=2305, name="qc_n2304_r34")


def _c_qc_8192_r2732():
    # 5 x 32 base, Z = 256: design rate 27/32 (5/6 is not reachable at n = 8192)
    return qc_code(5, 32, 256, [5] * 9 + [3] * 18, seed=8192, name="qc_n8192_r2732")


_CODES = {
    "gallager36_n1008": _c_gallager_1008,
    "qc_n2304_r12": _c_qc_2304_r12,
    "qc_n16200_r23": _c_qc_16200_r23,
    "qc_n576_r12": _c_qc_576_r12,
    "qc_n1152_r23": _c_qc_1152_r23,
    "qc_n2304_r34": _c_qc_2304_r34,
    "qc_n8192_r2732": _c_qc_8192_r2732,
}
CODE_NAMES = tuple(_CODES)
_CODE_CACHE: dict = {}


def code_by_name(name: str) -> Code:
    """One of the fixed-seed codes above (cached)."""
    if name not in _CODE_CACHE:
        _CODE_CACHE[name] = _CODES[name]()
    return _CODE_CACHE[name]


# ----------------------------------------------------------------------------------------
# Small graphs
# ----------------------------------------------------------------------------------------

def tree_code(n_vn: int, seed: int, max_cn_deg: int = 4) -> Code:
    """A random cycle-free Tanner graph with n_vn variable nodes: CNs of degree 2..max_cn_deg
    are attached one at a time to a single existing VN plus fresh VNs, so the graph stays a
    tree.  Every VN ends up in at least one CN."""
    rng = np.random.default_rng(seed)
    rows = []
    used = 1
    while used < n_vn:
        d = int(rng.integers(2, max_cn_deg + 1))
        d = min(d, n_vn - used + 1)
        anchor = int(rng.integers(0, used))
        rows.append([anchor] + list(range(used, used + d - 1)))
        used += d - 1
    perm = rng.permutation(n_vn)
    rows = [[int(perm[c]) for c in r] for r in rows]
    return code_from_rows(rows, n_vn, name=f"tree_n{n_vn}_s{seed}")


def fig1_code(x: int) -> Code:
    """The Tanner graph of the Fig. 1 discussion (Sec. II-A): CNs c1..c4, VNs v1..v8 with
    c1 = {v1,v2,v3}, c2 = {v2,v4,v5}, c3 = {v4,v6,v7}, c4 = {v_x, v8}.  The figure itself is
    missing; these neighbourhoods are the ones the text's message sets imply, and x (one of
    1, 3, 5, 7) is the one edge the text leaves open.  Indices here are 0-based."""
    if x not in (1, 3, 5, 7):
        raise ValueError("x must be one of 1, 3, 5, 7")
    rows = [[0, 1, 2], [1, 3, 4], [3, 5, 6], [x - 1, 7]]
    return code_from_rows(rows, 8, name=f"fig1_x{x}")


# ----------------------------------------------------------------------------------------
# Channel (Sec. II-C system model) and codewords
# ----------------------------------------------------------------------------------------

def design_rate(code: Code) -> float:
    return 1.0 - code.M / code.N


def sigma2_from_ebn0(ebn0_db: float, rate: float) -> float:
    """Noise variance for BPSK at the given Eb/N0 and code rate: sigma^2 = 1 / (2 R Eb/N0)."""
    return 1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))


def channel_llr(N: int, n_frames: int, ebn0_db: float, rate: float, seed: int,
                codeword: np.ndarray | None = None, dtype=np.float64) -> np.ndarray:
    """Channel LLRs [n_frames, N] for BPSK (bit 0 -> +1) over AWGN.

    y = (1 - 2 c) + sigma * z with z ~ N(0, 1) from numpy's PCG64 stream seeded by ``seed``,
    and L = 2 y / sigma^2 (Sec. II-C).  ``codeword`` is one word [N] or one per frame
    [n_frames, N]; None sends the all-zero word.  dtype float32 draws and computes in single
    precision (a different stream from float64), for batches too large to hold in float64.
    """
    dtype = np.dtype(dtype)
    s2 = sigma2_from_ebn0(ebn0_db, rate)
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal((n_frames, N), dtype=dtype)
    z *= dtype.type(math.sqrt(s2))
    if codeword is None:
        z += dtype.type(1.0)
    else:
        z += (1.0 - 2.0 * np.broadcast_to(np.asarray(codeword, dtype), (n_frames, N))).astype(dtype)
    z *= dtype.type(2.0 / s2)
    return z


def _gf2_nullspace(code: Code) -> np.ndarray:
    """Basis of the GF(2) null space of H, one codeword per row (uint8 [K, N])."""
    H = code.dense().copy()
    M, N = H.shape
    Hp = np.packbits(H, axis=1)
    pivots = []
    r = 0
    for c in range(N):
        if r >= M:
            break
        byte, bit = divmod(c, 8)
        mask = 0x80 >> bit
        col = (Hp[r:, byte] & mask) != 0
        nz = np.nonzero(col)[0]
        if nz.size == 0:
            continue
        p = r + int(nz[0])
        if p != r:
            Hp[[r, p]] = Hp[[p, r]]
        rows = np.nonzero((Hp[:, byte] & mask) != 0)[0]
        rows = rows[rows != r]
        if rows.size:
            Hp[rows] ^= Hp[r]
        pivots.append(c)
        r += 1
    R = np.unpackbits(Hp[:r], axis=1)[:, :N]
    free = [c for c in range(N) if c not in set(pivots)]
    basis = np.zeros((len(free), N), dtype=np.uint8)
    for i, f in enumerate(free):
        basis[i, f] = 1
        basis[i, pivots] = R[:, f]
    return basis


def random_codeword(code: Code, seed: int) -> np.ndarray:
    """A uniformly random codeword (uint8 [N]) of the code: a random GF(2) combination of a
    null-space basis of H."""
    basis = _gf2_nullspace(code)
    rng = np.random.default_rng(seed)
    coef = rng.integers(0, 2, size=basis.shape[0]).astype(np.uint8)
    word = (coef[:, None] * basis).sum(axis=0) % 2
    return word.astype(np.uint8)
