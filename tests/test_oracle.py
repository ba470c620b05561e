"""Pins for the exact oracle against what the paper prints and what mathematics fixes.

Every pin here is independent of the oracle's own formulas: printed tables
and the worked example of the paper, the definition of dictionary order
(itertools), the Leibniz permutation expansion, textbook special cases
(m = n is the ordinary determinant, m = 1 is the alternating sum),
invariants (row swap, row linearity), exact finite differences, and the
Chinese remainder theorem.  The last block plants mistakes in the oracle and
checks that a pin catches each one.
"""
import itertools
import math
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle.radic_oracle as orc
from tests.conftest import read_golden_rows


# ---------------------------------------------------------------------------
# Combinatorics: Table 2, worked example, Table 3b, Theorem 1, Theorem 2
# ---------------------------------------------------------------------------


def _table2():
    return {int(r[0]): [int(x) for x in r[1:]] for r in read_golden_rows("table2_lex_n8_m5.txt")}


def test_table2_is_dictionary_order():
    table = _table2()
    assert sorted(table) == list(range(56))
    assert [table[q] for q in range(56)] == [list(c) for c in orc.lex_combinations(8, 5)]


def test_table2_by_combinatorial_addition():
    table = _table2()
    for q in range(56):
        assert orc.unrank_combinatorial_addition(q, 8, 5) == table[q], q


def test_table2_by_successor_walk():
    table = _table2()
    seq = orc.first_member(5)
    for q in range(56):
        assert seq == table[q]
        seq = orc.lex_successor(seq, 8)
    assert seq is None


def test_worked_example_q49():
    rows = read_golden_rows("unrank_example_q49.txt")
    kv = {r[0]: r[1:] for r in rows if r[0] in ("n", "m", "q", "result")}
    steps = [[int(x) for x in r[1:]] for r in rows if r[0] == "step"]
    n, m, q = int(kv["n"][0]), int(kv["m"][0]), int(kv["q"][0])
    trace = []
    out = orc.unrank_combinatorial_addition(q, n, m, trace=trace)
    assert out == [int(x) for x in kv["result"]]
    assert trace == steps


def test_pascal_table3b():
    rows = [[int(x) for x in r] for r in read_golden_rows("table3b_pascal_n8_m5.txt")]
    assert orc.pascal_table(8, 5) == rows


@pytest.mark.parametrize("n", range(1, 13))
def test_theorem1_count(n):
    for m in range(1, n + 1):
        assert sum(1 for _ in orc.lex_combinations(n, m)) == math.comb(n, m)
        # hockey stick of the proof of Theorem 1
        assert sum(math.comb(n - t, m - 1) for t in range(1, n - m + 2)) == math.comb(n, m)


@pytest.mark.parametrize("n", range(1, 11))
def test_theorem2_bijection(n):
    for m in range(1, n + 1):
        listing = [list(c) for c in orc.lex_combinations(n, m)]
        got = [orc.unrank_combinatorial_addition(q, n, m) for q in range(len(listing))]
        assert got == listing, (n, m)


def test_unrank_large_spot_checks():
    # q = 0 and q = C-1 are the first and last members (Section 3).
    for n, m in [(32, 8), (40, 12), (64, 32), (28, 6)]:
        c = math.comb(n, m)
        assert orc.unrank_combinatorial_addition(0, n, m) == list(range(1, m + 1))
        assert orc.unrank_combinatorial_addition(c - 1, n, m) == list(range(n - m + 1, n + 1))
    # a successor step agrees with adding one to the rank
    rng = random.Random(7)
    for _ in range(200):
        n = rng.randint(2, 40)
        m = rng.randint(1, n)
        c = math.comb(n, m)
        if c < 2:
            continue
        q = rng.randrange(c - 1)
        a = orc.unrank_combinatorial_addition(q, n, m)
        assert orc.lex_successor(a, n) == orc.unrank_combinatorial_addition(q + 1, n, m)


def test_processor_ranges():
    for total in [0, 1, 7, 220, 10_518_300]:
        for k in [1, 2, 3, 7, 1024, 1216]:
            rs = orc.processor_ranges(total, k)
            assert sum(hi - lo for lo, hi in rs) == total
            for (a, b), (c, d) in zip(rs, rs[1:]):
                assert b == c
            if rs:
                assert rs[0][0] == 0 and rs[-1][1] == total
                assert max(hi - lo for lo, hi in rs) == -(-total // k)


# ---------------------------------------------------------------------------
# Minor determinant
# ---------------------------------------------------------------------------


def _leibniz(mat):
    size = len(mat)
    tot = 0
    for perm in itertools.permutations(range(size)):
        inv = sum(1 for i in range(size) for j in range(i + 1, size) if perm[i] > perm[j])
        prod = 1
        for i in range(size):
            prod *= mat[i][perm[i]]
        tot += -prod if inv % 2 else prod
    return tot


def test_bareiss_matches_leibniz():
    rng = random.Random(11)
    for _ in range(300):
        size = rng.randint(1, 6)
        lo = rng.choice([-1, -3, -9, -100])
        mat = [[rng.randint(lo, -lo) for _ in range(size)] for _ in range(size)]
        if rng.random() < 0.2:  # force a zero leading pivot
            mat[0][0] = 0
        assert orc.det_bareiss(mat) == _leibniz(mat)


def test_bareiss_special_cases():
    assert orc.det_bareiss([]) == 1
    assert orc.det_bareiss([[5]]) == 5
    assert orc.det_bareiss([[1, 2], [2, 4]]) == 0
    assert orc.det_bareiss([[0, 1], [1, 0]]) == -1
    assert orc.det_bareiss([[2, 7, 1], [0, 3, 5], [0, 0, 4]]) == 24


# ---------------------------------------------------------------------------
# Radic determinant, Definition 3 / Eq. (1)
# ---------------------------------------------------------------------------


def _rand_int_matrix(rng, m, n, lo=-9):
    return [[rng.randint(lo, -lo) for _ in range(n)] for _ in range(m)]


def test_square_is_ordinary_det():
    rng = random.Random(3)
    for size in range(1, 7):
        for _ in range(10):
            a = _rand_int_matrix(rng, size, size)
            val, _ = orc.radic_det_exact(a)
            assert val == _leibniz(a)
    x = np.random.default_rng(0).uniform(-1, 1, (5, 5))
    val, _ = orc.radic_det_exact(x)
    assert abs(float(val) - np.linalg.det(x)) < 1e-14


def test_single_row_is_alternating_sum():
    assert orc.radic_det_exact([[3, 1, 4, 1, 5]])[0] == 3 - 1 + 4 - 1 + 5
    rng = random.Random(5)
    for n in range(1, 12):
        row = [rng.randint(-50, 50) for _ in range(n)]
        assert orc.radic_det_exact([row])[0] == sum(v if j % 2 == 0 else -v for j, v in enumerate(row))


def test_two_by_three_by_hand():
    a, b, c, d, e, f = 2, -3, 5, 7, 11, -13
    # J = {1,2}: r+s = 3+3 even; {1,3}: 3+4 odd; {2,3}: 3+5 even
    want = (a * e - b * d) - (a * f - c * d) + (b * f - c * e)
    assert orc.radic_det_exact([[a, b, c], [d, e, f]])[0] == want


def test_wider_than_tall_is_zero_when_m_gt_n():
    assert orc.radic_det_exact([[1, 2], [3, 4], [5, 6]]) == (0, 0)
    assert orc.radic_det_pfaffian([[1, 2], [3, 4], [5, 6]]) == 0


def test_row_swap_flips_sign_and_row_linearity():
    rng = random.Random(9)
    for _ in range(40):
        m = rng.randint(2, 4)
        n = rng.randint(m, 7)
        a = _rand_int_matrix(rng, m, n)
        base, _ = orc.radic_det_exact(a)
        i, k = rng.sample(range(m), 2)
        sw = [row[:] for row in a]
        sw[i], sw[k] = sw[k], sw[i]
        assert orc.radic_det_exact(sw)[0] == -base
        # linear in row i: det(.., u + c v, ..) = det(.., u, ..) + c det(.., v, ..)
        v = [rng.randint(-9, 9) for _ in range(n)]
        c = rng.randint(-5, 5)
        mixed = [row[:] for row in a]
        mixed[i] = [x + c * y for x, y in zip(a[i], v)]
        only_v = [row[:] for row in a]
        only_v[i] = v
        assert orc.radic_det_exact(mixed)[0] == base + c * orc.radic_det_exact(only_v)[0]


def test_terms_sum_to_det_and_abs_sum():
    rng = random.Random(13)
    a = _rand_int_matrix(rng, 3, 7)
    val, abs_sum = orc.radic_det_exact(a)
    terms = orc.radic_terms_exact(a, range(math.comb(7, 3)))
    assert sum(terms) == val
    assert sum(abs(t) for t in terms) == abs_sum


def test_exact_conversion_of_floats():
    x = np.array([[0.1, -2.5e-7, 3.0], [1e10, 2.0 ** -60, -1.0]])
    mat, den = orc.exact_matrix(x)
    for i in range(2):
        for j in range(3):
            assert Fraction(mat[i][j], den) == Fraction(float(x[i, j]))
    y = x.astype(np.float32)
    mat, den = orc.exact_matrix(y)
    assert Fraction(mat[0][0], den) == Fraction(float(np.float32(0.1)))


def test_row_power_of_two_scaling_of_real_inputs():
    # Every term of Eq. (1) is a determinant, linear in each row, so scaling
    # row i by 2^-e_i multiplies det_R by 2^-e_i.  With e_i the exponent of
    # the lowest set bit of row i's nonzero entries the scaled rows are
    # integers: det_R(A) = 2^(sum e_i) det_R(M), the reading the exact mode
    # uses for binary32 and binary64 inputs.  A dropped or doubled exponent,
    # or a wrongly signed one, fails here.
    rng = np.random.default_rng(11)
    for m, n in [(1, 4), (2, 5), (3, 7), (4, 8)]:
        k = rng.integers(-30, 31, (m, n))
        s = rng.integers(0, 6, (m, n))
        r = rng.integers(-5, 6, (m, 1))
        a = k * np.ldexp(1.0, -s) * np.ldexp(1.0, r)
        e = []
        for i in range(m):
            lows = []
            for x in a[i]:
                f = Fraction(float(x))
                if f != 0:
                    lows.append((f.numerator & -f.numerator).bit_length() - 1 - (f.denominator.bit_length() - 1))
            e.append(min(lows) if lows else 0)
        mat = [[int(Fraction(float(a[i, j])) / Fraction(2) ** e[i]) for j in range(n)] for i in range(m)]
        assert all(Fraction(float(a[i, j])) == mat[i][j] * Fraction(2) ** e[i] for i in range(m) for j in range(n))
        want, _ = orc.radic_det_exact(np.array(mat, dtype=np.int64))
        got, _ = orc.radic_det_exact(a)
        assert got == Fraction(want) * Fraction(2) ** sum(e)


# ---------------------------------------------------------------------------
# Pfaffian closed form
# ---------------------------------------------------------------------------


def test_pfaffian_small_textbook():
    assert orc.pfaffian([[0, 3], [-3, 0]]) == 3
    a, b, c, d, e, f = 2, -1, 4, 3, 5, -7
    m = [[0, a, b, c], [-a, 0, d, e], [-b, -d, 0, f], [-c, -e, -f, 0]]
    # Pf = a f - b e + c d for the 4 x 4 skew matrix [[0,a,b,c],[.,0,d,e],[.,.,0,f]]
    assert orc.pfaffian(m) == a * f - b * e + c * d
    assert orc.pfaffian([[0, 1, 0], [-1, 0, 0], [0, 0, 0]]) == 0


def test_pfaffian_squared_is_det():
    rng = random.Random(17)
    for _ in range(60):
        size = rng.choice([2, 4, 6, 8])
        upper = [[rng.randint(-6, 6) for _ in range(size)] for _ in range(size)]
        sk = [[0] * size for _ in range(size)]
        for i in range(size):
            for j in range(i + 1, size):
                if rng.random() < 0.8:
                    sk[i][j] = upper[i][j]
                    sk[j][i] = -upper[i][j]
        assert orc.pfaffian(sk) ** 2 == orc.det_bareiss(sk)


def test_closed_form_matches_definition():
    rng = random.Random(19)
    for _ in range(150):
        n = rng.randint(1, 8)
        m = rng.randint(1, n)
        a = _rand_int_matrix(rng, m, n, lo=rng.choice([-1, -3, -9]))
        assert orc.radic_det_pfaffian(a) == orc.radic_det_exact(a)[0], (m, n, a)
    for _ in range(20):
        n = rng.randint(2, 8)
        m = rng.randint(1, n)
        x = np.random.default_rng(rng.randint(0, 1 << 30)).uniform(-1, 1, (m, n))
        assert orc.radic_det_pfaffian(x) == orc.radic_det_exact(x)[0]


# ---------------------------------------------------------------------------
# Gradient
# ---------------------------------------------------------------------------


def test_gradient_is_exact_forward_difference():
    rng = random.Random(23)
    for _ in range(12):
        n = rng.randint(2, 6)
        m = rng.randint(1, min(n, 4))
        a = _rand_int_matrix(rng, m, n)
        base, _ = orc.radic_det_exact(a)
        g = orc.radic_grad_exact(a, use_pfaffian=False)
        gp = orc.radic_grad_exact(a, use_pfaffian=True)
        for i in range(m):
            for j in range(n):
                bumped = [row[:] for row in a]
                bumped[i][j] += 1
                assert orc.radic_det_exact(bumped)[0] - base == g[i][j] == gp[i][j]


# ---------------------------------------------------------------------------
# Residues and CRT
# ---------------------------------------------------------------------------


def test_crt_signed_roundtrip():
    primes = [2147483647, 2147483629, 2147483587]
    for p in primes:
        assert orc.is_prime(p)
    big = primes[0] * primes[1] * primes[2]
    rng = random.Random(29)
    for _ in range(200):
        x = rng.randint(-(big // 2) + 1, big // 2)
        assert orc.crt_signed([x % p for p in primes], primes) == x


def test_det_mod_p_matches_exact():
    rng = random.Random(31)
    p = 2147483629
    for _ in range(50):
        size = rng.randint(1, 6)
        mat = [[rng.randint(-3, 3) for _ in range(size)] for _ in range(size)]
        assert orc.det_mod_p(mat, p) == _leibniz(mat) % p


# ---------------------------------------------------------------------------
# Planted mistakes: each must be caught by one of the pins above
# ---------------------------------------------------------------------------


def test_planted_sign_mistake_is_caught(monkeypatch):
    # r taken as 1+...+(m-1): wrong for every m
    def bad_sign(cols):
        m = len(cols)
        return -1 if (m * (m - 1) // 2 + sum(cols)) % 2 else 1

    monkeypatch.setattr(orc, "radic_sign", bad_sign)
    with pytest.raises(AssertionError):
        test_square_is_ordinary_det()


def test_planted_zero_based_s_is_caught(monkeypatch):
    def bad_sign(cols):
        m = len(cols)
        return -1 if (m * (m + 1) // 2 + sum(c - 1 for c in cols)) % 2 else 1

    monkeypatch.setattr(orc, "radic_sign", bad_sign)
    with pytest.raises(AssertionError):
        test_square_is_ordinary_det()


def test_planted_unrank_off_by_one_is_caught(monkeypatch):
    good = orc.pascal_table

    def bad_table(n, m):
        t = good(n, m)
        if m > 1 and len(t[0]) > 1:
            t[1][1] += 1
        return t

    monkeypatch.setattr(orc, "pascal_table", bad_table)
    with pytest.raises(AssertionError):
        test_table2_by_combinatorial_addition()


def test_planted_dropped_term_is_caught(monkeypatch):
    good = orc.lex_combinations

    def dropped(n, m):
        combos = list(good(n, m))
        return iter(combos[:-1])

    monkeypatch.setattr(orc, "lex_combinations", dropped)
    with pytest.raises(AssertionError):
        test_single_row_is_alternating_sum()


def test_planted_missing_pivot_sign_is_caught(monkeypatch):
    def bad_bareiss(mat):
        size = len(mat)
        if size == 0:
            return 1
        w = [list(r) for r in mat]
        prev = 1
        for k in range(size - 1):
            if w[k][k] == 0:
                for i in range(k + 1, size):
                    if w[i][k] != 0:
                        w[k], w[i] = w[i], w[k]  # sign flip forgotten
                        break
                else:
                    return 0
            for i in range(k + 1, size):
                for j in range(k + 1, size):
                    w[i][j] = (w[i][j] * w[k][k] - w[i][k] * w[k][j]) // prev
            prev = w[k][k]
        return w[-1][-1]

    monkeypatch.setattr(orc, "det_bareiss", bad_bareiss)
    with pytest.raises(AssertionError):
        test_bareiss_matches_leibniz()


def test_planted_pfaffian_sign_mistake_is_caught(monkeypatch):
    good = orc.pfaffian
    monkeypatch.setattr(orc, "pfaffian", lambda sk: -good(sk))
    with pytest.raises(AssertionError):
        test_closed_form_matches_definition()


# ---------------------------------------------------------------------------
# Binary64 host enumeration (oracle/radic_cpu.c), the timed CPU baseline
# ---------------------------------------------------------------------------


def test_cpu_enumeration_matches_exact_values():
    from oracle import cpu_enum

    rng = np.random.default_rng(77)
    for m, n in [(1, 7), (2, 5), (3, 9), (5, 5), (4, 11), (6, 12), (7, 9), (3, 2)]:
        a = rng.uniform(-1, 1, (m, n))
        val, abs_sum = orc.radic_det_exact(a)
        s, sa, th = cpu_enum.radic_cpu_sum(a)
        assert th >= 1
        assert abs(s - float(val)) <= 1e-12 * max(float(abs_sum), 1e-300)
        assert abs(sa - float(abs_sum)) <= 1e-12 * max(float(abs_sum), 1e-300)


def test_cpu_enumeration_rank_ranges_and_integers():
    from oracle import cpu_enum

    a = np.random.default_rng(78).integers(-9, 10, (4, 10)).astype(np.float64)
    total = math.comb(10, 4)
    for q0, count in [(0, 1), (17, 50), (total - 3, 10), (5, total)]:
        terms = orc.radic_terms_exact(a, range(q0, min(q0 + count, total)))
        s, sa, _ = cpu_enum.radic_cpu_sum(a, q0, count)
        assert abs(s - float(sum(terms))) <= 1e-13 * float(sum(abs(t) for t in terms))
        assert abs(sa - float(sum(abs(t) for t in terms))) <= 1e-13 * float(sum(abs(t) for t in terms))
