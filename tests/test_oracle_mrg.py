"""Pins the oracle's MRG32k3a (L'Ecuyer 1999) against the mathematics.

No printed known-answer vectors are available, so the pins are properties that
a wrong multiplier, sign, index or matrix layout breaks:

* full period: sympy (independently of the oracle) checks that each
  component's characteristic polynomial z^3 - a12 z + a13 (mod m1) and
  z^3 - a21 z^2 + a23 (mod m2) is primitive, the published design property;
  the oracle's transition matrices must then have order exactly m^3 - 1;
* skip-ahead by matrix powers equals sequential stepping (brute force);
* powers compose: A^(2^a) A^(2^b) = A^(2^a + 2^b), A^(2^76) = (A^(2^75))^2;
* the seeded state follows the stated reading; the first words follow from
  the recursion evaluated with Python integers (a cross-check of the C
  arithmetic, not an independent pin);
* statistics of the combined output.
"""

import numpy as np
import pytest

import oracle

M1 = 2**32 - 209
M2 = 2**32 - 22853
A12, A13 = 1403580, 810728
A21, A23 = 527612, 1370589


def _gf_poly_pow_mod(base, e, mod_poly, p):
    from sympy.polys.domains import ZZ
    from sympy.polys.galoistools import gf_pow_mod

    return gf_pow_mod(base, e, mod_poly, p, ZZ)


def _prime_factors(n):
    from sympy import factorint

    return sorted(factorint(n).keys())


@pytest.mark.parametrize("comp", [1, 2])
def test_characteristic_polynomial_is_primitive(comp):
    """sympy only: the published multipliers give a full-period recursion."""
    from sympy.polys.domains import ZZ
    from sympy.polys.galoistools import gf_irreducible_p

    p = M1 if comp == 1 else M2
    # coefficients, highest degree first, reduced mod p
    if comp == 1:
        poly = [1, 0, (-A12) % p, A13 % p]  # z^3 - a12 z + a13
    else:
        poly = [1, (-A21) % p, 0, A23 % p]  # z^3 - a21 z^2 + a23
    assert gf_irreducible_p(poly, p, ZZ)
    order = p**3 - 1
    z = [1, 0]
    assert _gf_poly_pow_mod(z, order, poly, p) == [1]
    for q in _prime_factors(order):
        assert _gf_poly_pow_mod(z, order // q, poly, p) != [1]


@pytest.mark.parametrize("comp", [1, 2])
def test_transition_matrix_has_full_period(comp):
    p = M1 if comp == 1 else M2
    order = p**3 - 1
    eye = np.eye(3, dtype=np.uint64)
    assert np.array_equal(oracle.mrg_matrix_power(comp, order), eye)
    for q in _prime_factors(order):
        assert not np.array_equal(oracle.mrg_matrix_power(comp, order // q), eye)


def _matmul_mod(a, b, m):
    a = [[int(x) for x in row] for row in a]
    b = [[int(x) for x in row] for row in b]
    return np.array([[sum(a[i][k] * b[k][j] for k in range(3)) % m for j in range(3)]
                     for i in range(3)], dtype=np.uint64)


@pytest.mark.parametrize("comp", [1, 2])
def test_matrix_powers_compose(comp):
    m = M1 if comp == 1 else M2
    for a, b in [(0, 0), (3, 7), (40, 41), (63, 64), (75, 76), (100, 127)]:
        lhs = _matmul_mod(oracle.mrg_matrix_power(comp, 2**a), oracle.mrg_matrix_power(comp, 2**b), m)
        assert np.array_equal(lhs, oracle.mrg_matrix_power(comp, 2**a + 2**b))
    sq = _matmul_mod(oracle.mrg_matrix_power(comp, 2**75), oracle.mrg_matrix_power(comp, 2**75), m)
    assert np.array_equal(sq, oracle.mrg_matrix_power(comp, 2**76))
    assert np.array_equal(oracle.mrg_matrix_power(comp, 0), np.eye(3, dtype=np.uint64))


def test_seeded_state_reading():
    st = oracle.mrg_seed_state(2021)
    assert st.tolist() == [1, 1, 2021, 1, 1, 1]
    st = oracle.mrg_seed_state(M1 + 5)
    assert st.tolist() == [1, 1, 5, 1, 1, 1]


def test_first_words_follow_recursion():
    """Cross-check of the C arithmetic with Python integers."""
    for seed in [0, 1, 2021, 0x12345678, 2**64 - 1]:
        x1 = [1, 1, seed % M1]
        x2 = [1, 1, 1]
        expect = []
        for _ in range(200):
            n1 = (A12 * x1[1] - A13 * x1[0]) % M1
            n2 = (A21 * x2[2] - A23 * x2[0]) % M2
            x1 = [x1[1], x1[2], n1]
            x2 = [x2[1], x2[2], n2]
            expect.append((n1 - n2) % M1)
        got = oracle.words(oracle.ENGINE_MRG, seed, 0, 200)
        assert got.tolist() == expect


def test_skip_equals_stepping_exhaustive_small():
    seed = 2021
    seq = oracle.words(oracle.ENGINE_MRG, seed, 0, 3000)
    for k in range(0, 2048):
        assert int(oracle.words(oracle.ENGINE_MRG, seed, k, 1)[0]) == int(seq[k])


def test_skip_equals_stepping_random_large():
    seed = 0xDEADBEEF
    n = 2_000_000
    seq = oracle.words(oracle.ENGINE_MRG, seed, 0, n)
    rng = np.random.Generator(np.random.PCG64(7))
    for k in rng.integers(0, n - 64, size=64):
        k = int(k)
        assert np.array_equal(oracle.words(oracle.ENGINE_MRG, seed, k, 64), seq[k:k + 64])


def test_state_skip_equals_steps():
    st_a = oracle.mrg_seed_state(99)
    st_b = st_a.copy()
    for _ in range(12345):
        oracle.mrg_step(st_a)
    oracle.mrg_skip(st_b, 12345)
    assert np.array_equal(st_a, st_b)


def test_skips_add():
    """A^a then A^b equals A^(a+b) on states, for offsets beyond 2^64."""
    seed = 5
    for a, b in [(2**76, 2**76), (2**76 * 3, 17), (2**64 - 1, 2), (2**100, 2**90 + 5)]:
        s1 = oracle.mrg_seed_state(seed)
        oracle.mrg_skip(s1, a)
        oracle.mrg_skip(s1, b)
        s2 = oracle.mrg_seed_state(seed)
        oracle.mrg_skip(s2, a + b)
        assert np.array_equal(s1, s2)
        assert np.array_equal(oracle.words(oracle.ENGINE_MRG, seed, a + b, 8),
                              _words_from_state(s2, 8))


def _words_from_state(st, n):
    st = st.copy()
    return np.array([oracle.mrg_step(st) for _ in range(n)], dtype=np.uint32)


def test_mrg_statistics():
    from scipy import stats

    w = oracle.words(oracle.ENGINE_MRG, 2021, 0, 1 << 20)
    assert int(w.max()) < M1
    ks = stats.kstest(w.astype(np.float64) / M1, "uniform")
    assert ks.pvalue > 1e-4
    # lag-1 serial correlation of the scaled words
    u = w.astype(np.float64) / M1 - 0.5
    r = float(np.dot(u[:-1], u[1:]) / np.dot(u, u))
    assert abs(r) < 5.0 / np.sqrt(u.size)
