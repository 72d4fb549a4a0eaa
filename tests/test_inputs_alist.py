"""alist I/O of the input generator (MacKay's sparse-matrix text format).

tests/golden/hamming74.alist holds the textbook (7,4) Hamming code, H rows 1101100, 1011010,
0111001: reading it must give that H (whose 7 columns are the 7 distinct nonzero syndromes, so
it has 16 codewords and corrects any single error), and writing then reading every seeded code
must give back the same CSR arrays.
"""
import itertools
import os

import numpy as np
import pytest

from paper_1202_1060_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_read_hamming74():
    c = I.read_alist(os.path.join(GOLD, "hamming74.alist"))
    H = c.dense()
    want = np.array([[1, 1, 0, 1, 1, 0, 0], [1, 0, 1, 1, 0, 1, 0], [0, 1, 1, 1, 0, 0, 1]], np.uint8)
    assert (H == want).all()
    syndromes = {tuple(H[:, n]) for n in range(7)}
    assert len(syndromes) == 7 and (0, 0, 0) not in syndromes
    words = [w for w in itertools.product((0, 1), repeat=7) if not (H @ np.array(w) % 2).any()]
    assert len(words) == 16


@pytest.mark.parametrize("name", ["gallager36_n1008", "qc_n576_r12", "qc_n2304_r12"])
def test_alist_roundtrip(tmp_path, name):
    c = I.code_by_name(name)
    path = str(tmp_path / f"{name}.alist")
    I.write_alist(c, path)
    d = I.read_alist(path)
    assert (d.M, d.N) == (c.M, c.N)
    np.testing.assert_array_equal(d.row_ptr, c.row_ptr)
    np.testing.assert_array_equal(d.col_idx, c.col_idx)


def test_alist_inconsistent_lists_rejected(tmp_path):
    bad = open(os.path.join(GOLD, "hamming74.alist")).read().splitlines()
    bad[4] = "1 3 0"   # column 1 now claims row 3, which its row lists do not have
    p = tmp_path / "bad.alist"
    p.write_text("\n".join(bad) + "\n")
    with pytest.raises(ValueError):
        I.read_alist(str(p))
