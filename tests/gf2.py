"""Textbook dense GF(2) linear algebra on Python integers, for pinning the oracle.

Independent of the oracle and of the CUDA path: rows are Python ints whose bit j
is column (slot) j; right-hand sides are r-bit ints.  Nothing here knows about
ribbons, buckets or bumping.
"""
from __future__ import annotations


class EchelonBasis:
    """Incremental row-echelon basis keyed by lowest set bit (the pivot)."""

    def __init__(self):
        self.rows = {}  # pivot -> (row, rhs)

    def reduce(self, row: int, rhs: int = 0):
        while row:
            p = (row & -row).bit_length() - 1
            hit = self.rows.get(p)
            if hit is None:
                return row, rhs
            row ^= hit[0]
            rhs ^= hit[1]
        return 0, rhs

    def independent(self, row: int) -> bool:
        return self.reduce(row)[0] != 0

    def add(self, row: int, rhs: int = 0) -> bool:
        red, rr = self.reduce(row, rhs)
        if red == 0:
            return False
        self.rows[(red & -red).bit_length() - 1] = (red, rr)
        return True

    def copy(self):
        b = EchelonBasis()
        b.rows = dict(self.rows)
        return b


def rank(rows) -> int:
    b = EchelonBasis()
    return sum(1 for r in rows if b.add(r))


def solve_free_zero(rows, rhs, ncols: int):
    """Solve rows . Z = rhs over GF(2) with every free column set to 0.

    Gauss-Jordan to reduced row-echelon form; then Z[pivot] = rhs of its row.
    Returns a list of ncols r-bit ints, or None if inconsistent.
    """
    piv = {}  # pivot column -> [row, rhs]
    for row, v in zip(rows, rhs):
        for p, (pr, pv) in piv.items():
            if (row >> p) & 1:
                row ^= pr
                v ^= pv
        if row == 0:
            if v != 0:
                return None
            continue
        p = (row & -row).bit_length() - 1
        # clear column p from every existing row (reduced form)
        for q in list(piv):
            pr, pv = piv[q]
            if (pr >> p) & 1:
                piv[q] = [pr ^ row, pv ^ v]
        piv[p] = [row, v]
    z = [0] * ncols
    for p, (pr, pv) in piv.items():
        z[p] = pv
    return z
