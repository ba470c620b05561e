"""Oracle for Radic's determinant of a non-square matrix (arXiv 1508.01326).

TEST INFRASTRUCTURE ONLY.  This module is the slow, exact CPU statement of
what the GPU library computes.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library under
``paper_1508_01326_gb300/`` never does, and this module imports nothing from
the library.  All arithmetic here is exact (Python integers and
``fractions.Fraction``); floating-point inputs are converted exactly.

What each function follows:

* ``radic_sign``, ``radic_det_exact``, ``radic_terms_exact`` -- Definition 3,
  Eq. (1): the sum over all ascending column sequences j1 < ... < jm of
  (-1)^(r+s) det(A[:, J]), r = 1+2+...+m, s = j1+...+jm (1-based), and 0 when
  m > n.  This is the plain definition written out.
* ``lex_combinations`` -- Definitions 1 and 2 (ascending sequences of
  {1..n} in dictionary order), numbered from 0 as in Table 2.
* ``pascal_table`` -- Table 1 / Table 3: entry (j, i) = C(i+j, j), built by
  the Pascal recurrence of Fig. 1.
* ``unrank_combinatorial_addition`` -- Section 4 ("combinatorial addition",
  worked example q = 49, Theorem 2): rank q -> q-th ascending sequence.
* ``lex_successor`` -- the successor figure of Section 5 ("dictionary
  sequence"): next ascending sequence in dictionary order.
* ``processor_ranges`` -- Section 5: K processors take contiguous rank
  chunks of about C(n,m)/K each.
* ``det_bareiss`` -- the m x m minor determinant (the paper defers it to its
  ref. [7]); here exact fraction-free (Bareiss) elimination on integers.
* ``pfaffian`` / ``radic_det_pfaffian`` -- an independent closed form used
  only as a cross-check at sizes where enumeration is too slow: the minor
  summation formula for Pfaffians (Ishikawa and Wakayama, Linear and
  Multilinear Algebra 39 (1995)).  With T = A diag((-1)^j) and B the skew
  matrix with +1 above the diagonal, every Pf(B_J) = 1, so
  sum_J det(T_J) = Pf(T B T^T) for even m; odd m appends one unit row/column.
* ``radic_grad_exact`` -- d det_R / d a_ij = (-1)^(i+j) det_R(A without row i
  and column j) (1-based), the Laplace expansion of Eq. (1) along row i.
* ``det_mod_p`` / ``crt_signed`` -- exact residues and the unique signed
  integer with given residues (Chinese remainder theorem), for the exact
  multi-modular path.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction
from typing import Iterable, List, Sequence, Tuple

# ---------------------------------------------------------------------------
# Combinatorics of column sets (Definitions 1-2, Theorem 1, Section 4, Section 5)
# ---------------------------------------------------------------------------


def first_member(m: int) -> List[int]:
    """First Member [1, 2, ..., m]: the first ascending sequence in dictionary order (Section 3)."""
    return list(range(1, m + 1))


def lex_combinations(n: int, m: int) -> Iterable[Tuple[int, ...]]:
    """All ascending m-sequences of {1..n} in dictionary order (Definitions 1 and 2)."""
    return itertools.combinations(range(1, n + 1), m)


def pascal_table(n: int, m: int) -> List[List[int]]:
    """Table 1 / Table 3 of Section 4: rows j = 0..m-1, columns i = 0..n-m, entry C(i+j, j).

    Built as Fig. 1 builds it: the first row and the first column are ones and
    every other entry is the sum of its left and upper neighbours.
    """
    cols = n - m + 1
    table = [[0] * cols for _ in range(m)]
    for i in range(cols):
        table[0][i] = 1
    for j in range(m):
        table[j][0] = 1
    for j in range(1, m):
        for i in range(1, cols):
            table[j][i] = table[j][i - 1] + table[j - 1][i]
    return table


def unrank_combinatorial_addition(q: int, n: int, m: int, trace: list | None = None) -> List[int]:
    """Section 4, "combinatorial addition": the q-th (0-based) ascending sequence, 1-based values.

    Start from the First Member.  While q > 0: with the current right-hand
    column `col` of the Pascal table, pick the lowest place whose weight (the
    table entry in that place's row at `col`) still fits into q; walk left
    along that row, summing entries while the sum stays <= q; the number of
    steps p is added to that place and to every place after it (which keeps
    the tail consecutive); subtract the sum from q and continue p columns
    further left.  Theorem 2 states that the result is the q-th sequence.

    If `trace` is a list, the sequence after each addition is appended to it
    (the worked example prints [2,3,4,5,6] and then [2,5,6,7,8] for q = 49).
    """
    total_count = math.comb(n, m)
    if not (0 <= q < total_count):
        raise ValueError(f"rank {q} outside [0, C({n},{m}) = {total_count})")
    table = pascal_table(n, m)
    seq = first_member(m)
    col = n - m
    while q > 0:
        if col < 0:
            raise AssertionError("combinatorial addition ran past the table")
        # Row of the place that changes: the largest row whose entry at `col` fits into q.
        row = 0
        while row + 1 < m and table[row + 1][col] <= q:
            row += 1
        # Walk left along that row.
        acc, p = 0, 0
        while col - p >= 0 and acc + table[row][col - p] <= q:
            acc += table[row][col - p]
            p += 1
        place = m - 1 - row  # 0-based place index; row m-1 is the first place
        seq[place] += p
        for h in range(place + 1, m):
            seq[h] = seq[h - 1] + 1
        if trace is not None:
            trace.append(list(seq))
        q -= acc
        col -= p
    return seq


def lex_successor(seq: Sequence[int], n: int) -> List[int] | None:
    """Section 5 successor figure: next ascending sequence in dictionary order (1-based values).

    The rightmost place that is below its largest possible value n-m+place
    (1-based place) is increased by one and every later place is reset to
    follow it consecutively.  Returns None after the last member.
    """
    m = len(seq)
    out = list(seq)
    i = m - 1
    while i >= 0 and out[i] == n - m + 1 + i:
        i -= 1
    if i < 0:
        return None
    out[i] += 1
    for h in range(i + 1, m):
        out[h] = out[h - 1] + 1
    return out


def processor_ranges(total: int, processors: int) -> List[Tuple[int, int]]:
    """Section 5 work split: processor k takes a contiguous run of ranks.

    The paper gives chunks of C(n,m)/K ranks; when K does not divide the
    count the chunks here have ceil(total/K) ranks and the last is shorter
    (empty chunks are dropped).
    """
    if processors < 1:
        raise ValueError("need at least one processor")
    size = -(-total // processors)
    out = []
    for k in range(processors):
        lo, hi = k * size, min((k + 1) * size, total)
        if lo < hi:
            out.append((lo, hi))
    return out


# ---------------------------------------------------------------------------
# Exact values (Definition 3, Eq. (1))
# ---------------------------------------------------------------------------


def exact_matrix(a) -> Tuple[List[List[int]], int]:
    """Exact integer image of a real matrix: returns (M, d) with a = M / d.

    Every binary64/binary32 value and every integer is a dyadic rational, so
    this conversion is exact; exact rationals are accepted as they are.
    """
    rows = [[Fraction(_as_exact(x)) for x in row] for row in _rows(a)]
    den = 1
    for row in rows:
        for x in row:
            den = math.lcm(den, x.denominator)
    return [[int(x * den) for x in row] for row in rows], den


def _rows(a) -> List[list]:
    if hasattr(a, "tolist"):
        a = a.tolist()
    return [list(r) for r in a]


def _as_exact(x):
    if isinstance(x, bool):
        return int(x)
    if isinstance(x, (int, Fraction)):
        return x
    if isinstance(x, float):
        return Fraction(x)
    # numpy scalar
    if hasattr(x, "dtype") and x.dtype.kind in "iu":
        return int(x)
    return Fraction(float(x))


def det_bareiss(mat: Sequence[Sequence[int]]) -> int:
    """Exact determinant of a square integer matrix by Bareiss fraction-free elimination.

    Every division in the recurrence is exact over the integers; a zero pivot
    is replaced by a lower row with a nonzero entry (one row swap, one sign
    flip).  The 0 x 0 determinant is 1.
    """
    size = len(mat)
    if size == 0:
        return 1
    work = [list(r) for r in mat]
    sign = 1
    prev = 1
    for k in range(size - 1):
        if work[k][k] == 0:
            for i in range(k + 1, size):
                if work[i][k] != 0:
                    work[k], work[i] = work[i], work[k]
                    sign = -sign
                    break
            else:
                return 0
        pivot = work[k][k]
        for i in range(k + 1, size):
            for j in range(k + 1, size):
                num = work[i][j] * pivot - work[i][k] * work[k][j]
                quo, rem = divmod(num, prev)
                assert rem == 0, "Bareiss division must be exact"
                work[i][j] = quo
            work[i][k] = 0
        prev = pivot
    return sign * work[size - 1][size - 1]


def radic_sign(cols_1based: Sequence[int]) -> int:
    """(-1)^(r+s) of Eq. (1): r = 1+2+...+m, s = sum of the 1-based column indices."""
    m = len(cols_1based)
    r = m * (m + 1) // 2
    s = sum(cols_1based)
    return -1 if (r + s) % 2 else 1


def _minor_int(mat_int: List[List[int]], cols_1based: Sequence[int]) -> List[List[int]]:
    return [[row[c - 1] for c in cols_1based] for row in mat_int]


def radic_det_exact(a) -> Tuple[Fraction, Fraction]:
    """Eq. (1) written out: returns (det_R(A), sum of |terms|) as exact rationals.

    Enumerates all C(n, m) ascending sequences in dictionary order, takes the
    exact determinant of each minor and adds it with its sign.  m > n gives 0
    (Definition 3).
    """
    rows = _rows(a)
    m = len(rows)
    n = len(rows[0]) if m else 0
    if m > n:
        return Fraction(0), Fraction(0)
    mat_int, den = exact_matrix(rows)
    total = 0
    abs_total = 0
    for cols in lex_combinations(n, m):
        d = det_bareiss(_minor_int(mat_int, cols))
        total += radic_sign(cols) * d
        abs_total += abs(d)
    scale = Fraction(1, den ** m)
    return total * scale, abs_total * scale


def radic_terms_exact(a, ranks: Iterable[int]) -> List[Fraction]:
    """Signed terms (-1)^(r+s) det(A[:, J_q]) of Eq. (1) for the given 0-based dictionary ranks q."""
    rows = _rows(a)
    m = len(rows)
    n = len(rows[0])
    mat_int, den = exact_matrix(rows)
    scale = Fraction(1, den ** m)
    out = []
    for q in ranks:
        cols = unrank_combinatorial_addition(int(q), n, m)
        out.append(radic_sign(cols) * det_bareiss(_minor_int(mat_int, cols)) * scale)
    return out


def to_float(x: Fraction) -> float:
    """Correctly rounded binary64 value of an exact rational."""
    return float(x)


# ---------------------------------------------------------------------------
# Independent closed form (minor summation formula for Pfaffians)
# ---------------------------------------------------------------------------


def pfaffian(skew: Sequence[Sequence]) -> Fraction:
    """Exact Pfaffian of a skew-symmetric matrix by congruence elimination.

    Pf(P M P^T) = det(P) Pf(M).  Each step brings a nonzero entry to (0, 1)
    by a symmetric swap (sign flip), clears rows/columns 0 and 1 beyond the
    leading 2 x 2 block with unit-triangular congruences (Pfaffian
    unchanged), and recurses on the trailing block: Pf(M) = M[0][1] Pf(M').
    """
    size = len(skew)
    if size % 2:
        return Fraction(0)
    work = [[Fraction(x) for x in row] for row in skew]
    result = Fraction(1)
    lo = 0
    while lo < size:
        piv = next((j for j in range(lo + 1, size) if work[lo][j] != 0), None)
        if piv is None:
            return Fraction(0)
        if piv != lo + 1:
            _sym_swap(work, lo + 1, piv)
            result = -result
        a01 = work[lo][lo + 1]
        result *= a01
        for i in range(lo + 2, size):
            beta = -work[lo][i] / a01  # e_i += beta e_{lo+1} clears entry (lo, i)
            if beta:
                _sym_add(work, i, lo + 1, beta)
            alpha = work[lo + 1][i] / a01  # e_i += alpha e_lo clears entry (lo+1, i)
            if alpha:
                _sym_add(work, i, lo, alpha)
        lo += 2
    return result


def _sym_swap(w, i, j):
    w[i], w[j] = w[j], w[i]
    for row in w:
        row[i], row[j] = row[j], row[i]


def _sym_add(w, i, j, c):
    """Row i += c * row j and column i += c * column j (a congruence)."""
    w[i] = [x + c * y for x, y in zip(w[i], w[j])]
    for row in w:
        row[i] += c * row[j]


def radic_det_pfaffian(a) -> Fraction:
    """det_R(A) = (-1)^(m(m+1)/2) Pf(T B T^T) with T = A diag((-1)^j), j 1-based.

    For odd m the (m+1) x (n+1) matrix [[T, 0], [0, 1]] is used, so the
    formula sums det(T_J) over all J of size m.  Exact; m > n gives 0.
    """
    rows = _rows(a)
    m = len(rows)
    n = len(rows[0]) if m else 0
    if m > n:
        return Fraction(0)
    mat_int, den = exact_matrix(rows)
    t = [[(x if (j + 1) % 2 == 0 else -x) for j, x in enumerate(row)] for row in mat_int]
    cols = n
    if m % 2:
        t = [row + [0] for row in t] + [[0] * n + [1]]
        cols = n + 1
    size = len(t)
    # (T B)[i][k] = sum_{j<k} T[i][j] - sum_{j>k} T[i][j]
    tb = []
    for row in t:
        prefix = [0]
        for x in row:
            prefix.append(prefix[-1] + x)
        tot = prefix[-1]
        tb.append([prefix[k] - (tot - prefix[k + 1]) for k in range(cols)])
    g = [[sum(tb[i][k] * t[l][k] for k in range(cols)) for l in range(size)] for i in range(size)]
    r = m * (m + 1) // 2
    val = pfaffian(g)
    if r % 2:
        val = -val
    return val / Fraction(den) ** m


# ---------------------------------------------------------------------------
# Gradient (Laplace expansion of Eq. (1) along a row)
# ---------------------------------------------------------------------------


def radic_grad_exact(a, use_pfaffian: bool = True) -> List[List[Fraction]]:
    """d det_R(A) / d a_ij = (-1)^(i+j) det_R(A with row i and column j removed), 1-based i, j.

    det_R is affine in every single entry, so this is also the exact forward
    difference det_R(A + e_ij) - det_R(A).
    """
    rows = [[_as_exact(x) for x in r] for r in _rows(a)]
    m = len(rows)
    n = len(rows[0])
    det_fn = (lambda x: radic_det_pfaffian(x)) if use_pfaffian else (lambda x: radic_det_exact(x)[0])
    grad = []
    for i in range(m):
        grow = []
        for j in range(n):
            sub = [[x for jj, x in enumerate(r) if jj != j] for ii, r in enumerate(rows) if ii != i]
            val = Fraction(1) if m == 1 else det_fn(sub)
            grow.append(val if (i + j) % 2 == 0 else -val)
        grad.append(grow)
    return grad


# ---------------------------------------------------------------------------
# Residues and reconstruction (exact multi-modular path)
# ---------------------------------------------------------------------------


def det_mod_p(mat_int: Sequence[Sequence[int]], p: int) -> int:
    """det(M) mod p in [0, p), from the exact integer determinant."""
    return det_bareiss(mat_int) % p


def radic_det_mod_p(a_int, p: int) -> int:
    """det_R(A) mod p for an integer matrix, from the exact value of Eq. (1)."""
    val, _ = radic_det_exact(a_int)
    assert val.denominator == 1
    return int(val) % p


def crt_signed(residues: Sequence[int], primes: Sequence[int]) -> int:
    """The unique integer x in (-P/2, P/2], P = prod(primes), with x = r_k mod p_k."""
    big = 1
    for p in primes:
        big *= p
    x = 0
    for r, p in zip(residues, primes):
        other = big // p
        x += r * other * pow(other, -1, p)
    x %= big
    if x > big // 2:
        x -= big
    return x


def is_prime(p: int) -> bool:
    """Deterministic trial division (adequate for 31-bit numbers)."""
    if p < 2:
        return False
    if p % 2 == 0:
        return p == 2
    f = 3
    while f * f <= p:
        if p % f == 0:
            return False
        f += 2
    return True
