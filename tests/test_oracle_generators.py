"""Pins of the oracle's point generators (Xu & Okten, Sec. 2 and Sec. 3).

Each test checks the oracle against something other than itself: published
known-answer vectors, an independent library (Triton's Philox, scipy's
Halton and Sobol', sympy's primes), exact rational arithmetic of
Algorithms 1 and 2, or invariants that a dropped term / wrong index breaks.
"""
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1408_5526_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ Philox
def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers():
    for ctr, key, want in _kat():
        assert list(O.philox4x32_10(ctr, key)) == want


_TRITON_SCRIPT = r"""
import os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl
@triton.jit
def k(c_ptr, out_ptr, seed, n: tl.constexpr):
    o = tl.arange(0, n)
    c0 = tl.load(c_ptr + 4 * o + 0).to(tl.uint32)
    c1 = tl.load(c_ptr + 4 * o + 1).to(tl.uint32)
    c2 = tl.load(c_ptr + 4 * o + 2).to(tl.uint32)
    c3 = tl.load(c_ptr + 4 * o + 3).to(tl.uint32)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * o + 0, a.to(tl.int64))
    tl.store(out_ptr + 4 * o + 1, b.to(tl.int64))
    tl.store(out_ptr + 4 * o + 2, c.to(tl.int64))
    tl.store(out_ptr + 4 * o + 3, d.to(tl.int64))
seed = int(sys.argv[1])
ctr = np.array([int(x) for x in sys.argv[2:]], dtype=np.int64)
n = len(ctr) // 4
out = torch.zeros(4 * n, dtype=torch.int64)
k[(1,)](torch.from_numpy(ctr), out, seed, n)
print(" ".join(str(int(x) & 0xffffffff) for x in out))
"""


def test_philox_matches_triton_implementation():
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    seed = int(rng.integers(0, 2**63))
    ctr = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64)
    r = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT, str(seed)] + [str(int(x)) for x in ctr.ravel()],
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + r.stderr[-200:])
    got = np.array([int(x) for x in r.stdout.split()], dtype=np.uint64).reshape(16, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(16):
        assert list(O.philox4x32_10(ctr[i], key)) == list(got[i])


def test_philox_path_stream_layout_and_uniformity():
    # word (j mod 4) of the call with counter (n_lo, n_hi16 | (j/4) << 16, m, inst << 8)
    seed = 0x123456789ABCDEF
    for (m, j, n) in [(0, 0, 0), (3, 5, 77), (63, 39, 65535), (2, 359, (1 << 40) + 5)]:
        w = O.philox4x32_10([n & 0xFFFFFFFF, ((n >> 32) & 0xFFFF) | ((j >> 2) << 16), m, 0],
                            [seed & 0xFFFFFFFF, seed >> 32])
        assert O.lib().orc_philox_path_word(seed, 0, m, j, n) == int(w[j & 3])
    q = O.Sequence(O.PHILOX, 4, 2, seed)
    raw = q.points(20000, transform=O.RAW)
    counts = np.bincount((raw >> 28).astype(np.int64).ravel(), minlength=16)
    exp = raw.size / 16
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 45.0     # 15 dof, p ~ 1e-4


# ------------------------------------------------------------------ primes, digits
def test_first_primes_match_sympy():
    sympy = pytest.importorskip("sympy")
    p = O.first_primes(400)
    assert list(p) == list(sympy.primerange(2, int(p[-1]) + 1))
    assert p[359] == 2423


@pytest.mark.parametrize("p", [2, 3, 5, 19, 173, 2423])
def test_halton_K_is_largest_fitting(p):
    K = O.halton_K(p)
    assert p ** (K + 1) <= 2**64 - 1 < p ** (K + 2)
    assert O.ipow(p, K + 1) == p ** (K + 1)


def test_van_der_corput_textbook_prefix():
    with open(os.path.join(GOLDEN, "van_der_corput_prefix.txt")) as f:
        rows = [tuple(int(x) for x in l.split()) for l in f if l.strip() and not l.startswith("#")]
    for b, n, num, den in rows:
        K = O.halton_K(b)
        got = O.permuted_vdc_numerator(b, K, np.arange(b), n)
        assert Fraction(got, b ** (K + 1)) == Fraction(num, den)


def test_halton_matches_scipy_unscrambled():
    qmc = pytest.importorskip("scipy.stats.qmc")
    s, n = 360, 1500
    P = O.first_primes(s)
    ref = qmc.Halton(d=s, scramble=False).random(n)
    for j in [0, 1, 2, 7, 39, 100, 359]:
        p = int(P[j])
        K = O.halton_K(p)
        ident = np.arange(p)
        got = np.array([O.permuted_vdc_numerator(p, K, ident, i) / float(p ** (K + 1)) for i in range(n)])
        np.testing.assert_allclose(got, ref[:, j], rtol=0, atol=1e-14)


# ------------------------------------------------------------------ Algorithms 1-3
def _alg2_orbit(p, K, sigma, n0, count):
    """Algorithm 2 (recursive odometer, Sec. 3.1) in exact rationals.  The
    start n0 holds K digits, all of them permuted (reading c2)."""
    a = [0] * (K + 2)
    rest = n0
    for k in range(K):
        a[k] = rest % p
        rest //= p
    S = [Fraction(0)] * (K + 3)
    for j in range(K - 1, -1, -1):
        S[j] = S[j + 1] + Fraction(int(sigma[a[j]]), p ** (j + 1))
    out = [S[0]]
    for _ in range(count - 1):
        m = 0
        while a[m] + 1 >= p:
            m += 1
        S[m] = S[m + 1] + Fraction(int(sigma[a[m] + 1]), p ** (m + 1))
        a[m] += 1
        for i in range(m - 1, -1, -1):
            a[i] = 0
            S[i] = S[i + 1] + Fraction(int(sigma[0]), p ** (i + 1))
        out.append(S[0])
    return out


def _struckmeier_orbit(p, x0, count):
    """Algorithm 1 (von Neumann-Kakutani T_p, eqs. bk, tp, k) in exact
    rationals: k is the integer with p^-k < 1 - x <= p^-(k-1)."""
    out = [x0]
    x = x0
    for _ in range(count - 1):
        k = 1
        while not (Fraction(1, p ** k) < 1 - x):
            k += 1
        b = Fraction(p + 1 - p ** k, p ** k)
        x = x + b
        out.append(x)
    return out


@pytest.mark.parametrize("p,K", [(2, 1), (2, 4), (3, 2), (3, 3), (5, 2), (7, 1)])
def test_counter_based_equals_recursive_and_struckmeier(p, K):
    rng = np.random.default_rng(p * 100 + K)
    D = p ** (K + 1)
    for trial in range(4):
        n0 = int(rng.integers(0, p ** K))
        count = D - p ** K - n0          # stay below p^(K+1) after the carry
        sigma = O.halton_perm(1000 + trial, 0, trial, K, p, identity=(trial == 0))
        alg3 = [Fraction(O.permuted_vdc_numerator(p, K, sigma, n0 + i), D) for i in range(count)]
        assert alg3 == _alg2_orbit(p, K, sigma, n0, count)
        if trial == 0:   # identity permutation: T_p orbit of phi_p(n0)
            assert alg3 == _struckmeier_orbit(p, alg3[0], count)


def test_struckmeier_floor_boundary_case():
    # base 2 from x = 0: 0, 1/2, 1/4, 3/4, 1/8 -- the 4th step sits on 1 - x = 2^-2
    assert _struckmeier_orbit(2, Fraction(0), 5) == [0, Fraction(1, 2), Fraction(1, 4), Fraction(3, 4),
                                                     Fraction(1, 8)]


@pytest.mark.parametrize("p", [2, 3, 5, 7])
def test_step_constant_is_odometer_increment(p):
    # b_k^p = (p + 1 - p^k) / p^k equals phi_p(n+1) - phi_p(n) when n ends in k-1 digits p-1
    for k in range(1, 6):
        n = p ** (k - 1) - 1 + 3 * p ** k       # k-1 trailing (p-1) digits, then a digit < p-1
        K = O.halton_K(p)
        ident = np.arange(p)
        D = p ** (K + 1)
        diff = Fraction(O.permuted_vdc_numerator(p, K, ident, n + 1) - O.permuted_vdc_numerator(p, K, ident, n), D)
        assert diff == Fraction(p + 1 - p ** k, p ** k)


@pytest.mark.parametrize("j", [0, 1, 4, 39, 200])
def test_random_start_is_within_eps_of_omega(j):
    # Algorithm 3 step (1): |phi_p(n0) - omega| < p^-K with omega = U / 2^64
    seed, inst, m = 99, 3, 5
    p = int(O.first_primes(j + 1)[j])
    K = O.halton_K(p)
    w = O.philox4x32_10([j, 0, m, 1 | (inst << 8)], [seed & 0xFFFFFFFF, seed >> 32])
    omega = Fraction(int(w[0]) | (int(w[1]) << 32), 2**64)
    n0 = O.halton_start(seed, inst, m, j, p, K)
    assert 0 <= n0 < p ** K
    phi = Fraction(O.permuted_vdc_numerator(p, K, np.arange(p), n0), p ** (K + 1))
    assert abs(phi - omega) < Fraction(1, p ** K)


def test_permutations_are_uniform_bijections():
    p = 5
    first = np.zeros((p, p), dtype=np.int64)
    for m in range(4000):
        s = O.halton_perm(17, 0, m, 2, p)
        assert sorted(s.tolist()) == list(range(p))
        for pos in range(p):
            first[pos, s[pos]] += 1
    exp = 4000 / p
    assert np.all(np.abs(first - exp) < 5 * np.sqrt(exp))


@pytest.mark.parametrize("seq", [O.HALTON_RS, O.RASRAP])
def test_halton_stratification_any_start(seq):
    # p^k consecutive points hit every cell of width p^-k exactly once (eq. perm)
    q = O.Sequence(seq, 8, 3, seed=11)
    N = 2500
    raw = q.points(N, offset=37, transform=O.RAW)
    P = O.first_primes(8)
    for m in range(3):
        for j in range(8):
            p = int(P[j])
            D = p ** (O.halton_K(p) + 1)
            for k in (1, 2, 3):
                if p ** k > N:
                    continue
                for start in (0, 13):
                    blk = raw[m, j, start:start + p ** k].astype(object)
                    cells = sorted(int(x) * p ** k // D for x in blk)
                    assert cells == list(range(p ** k))


# ------------------------------------------------------------------ Sobol'
def test_sobol_matches_scipy_point_sets():
    qmc = pytest.importorskip("scipy.stats.qmc")
    poly, vinit = inputs.joe_kuo_table()
    s = 360
    V = O.sobol_directions(s, poly, vinit)
    k = 11
    ref = qmc.Sobol(d=s, scramble=False, bits=32).random_base2(k)
    ref_u = np.round(ref * 2.0**32).astype(np.uint64)
    for kk in (1, 4, 7, 11):   # every prefix of length 2^kk is the same point set
        n = 1 << kk
        ours = np.array([[O.sobol_binary(V[j], i) for j in range(s)] for i in range(n)], dtype=np.uint64)
        a = sorted(map(tuple, ours.tolist()))
        b = sorted(map(tuple, ref_u[:n].tolist()))
        assert a == b


def test_sobol_first_dimension_is_van_der_corput():
    poly, vinit = inputs.joe_kuo_table()
    V = O.sobol_directions(2, poly, vinit)
    for n in range(64):
        want = int(format(n, "032b")[::-1], 2)
        assert O.sobol_binary(V[0], n) == want


def test_digital_shift_keeps_stratification():
    q = O.Sequence(O.SOBOL_DS, 40, 2, seed=5, joe_kuo=inputs.joe_kuo_table())
    raw = q.points(1024, transform=O.RAW)
    for m in range(2):
        for j in range(40):
            for k in (3, 6, 10):
                blk = raw[m, j, :1 << k] >> (32 - k)
                assert sorted(blk.tolist()) == list(range(1 << k))


def _lms_rows(seed, inst, m, j):
    import ctypes as C
    rows = np.zeros(32, dtype=np.uint32)
    O.lib().orc_sobol_lms_rows(seed, inst, m, j, rows.ctypes.data_as(C.POINTER(C.c_uint32)))
    return rows


def test_lms_matrices_are_random_unit_lower_triangular():
    # Sec. 3.2 (Matousek): nonsingular lower-triangular scrambling matrices
    ones = np.zeros((32, 32))
    for m in range(10):
        for j in range(20):
            rows = _lms_rows(7, 0, m, j)
            for r in range(32):
                row = int(rows[r])
                assert (row >> (31 - r)) & 1 == 1                 # unit diagonal
                assert row & ((1 << (31 - r)) - 1) == 0           # nothing right of it
                for l in range(r):
                    ones[r, l] += (row >> (31 - l)) & 1
    frac = ones[np.tril_indices(32, -1)] / 200.0
    assert 0.35 < frac.mean() < 0.65 and frac.min() > 0.3 and frac.max() < 0.7


def test_lms_equals_explicit_gf2_matrix_product():
    # y = L (C n) + e over GF(2), written as plain 0/1 matrix algebra: C's column k holds
    # the digits of direction number v_k (digit l = 2^-(l+1)), n's digit k is bit k.
    poly, vinit = inputs.joe_kuo_table()
    s, M, seed = 12, 3, 21
    q = O.Sequence(O.SOBOL_LMS, s, M, seed, joe_kuo=(poly, vinit))
    V = O.sobol_directions(s, poly, vinit)
    digits = lambda x: np.array([(int(x) >> (31 - l)) & 1 for l in range(32)], dtype=np.int64)
    rng = np.random.default_rng(3)
    for m in range(M):
        for j in range(s):
            rows = _lms_rows(seed, 0, m, j)
            Lm = np.array([digits(r) for r in rows])                    # row r = output digit r
            Cm = np.array([digits(v) for v in V[j]]).T                  # column k = v_k
            e = digits(O.sobol_shift(seed, 0, m, j))
            for n in [0, 1, 2, 3, 1023, 65535] + rng.integers(0, 1 << 31, 6).tolist():
                nb = np.array([(n >> k) & 1 for k in range(32)], dtype=np.int64)
                y = (Lm @ ((Cm @ nb) % 2) + e) % 2
                want = sum(int(y[l]) << (31 - l) for l in range(32))
                assert q.raw(m, j, n)[0] == want


def test_lms_keeps_stratification_and_the_two_dimensional_net():
    q = O.Sequence(O.SOBOL_LMS, 40, 2, seed=9, joe_kuo=inputs.joe_kuo_table())
    raw = q.points(1024, transform=O.RAW)
    for m in range(2):
        for j in range(40):
            for k in (3, 6, 10):
                assert sorted((raw[m, j, :1 << k] >> (32 - k)).tolist()) == list(range(1 << k))
        # dimensions 0 and 1 of Sobol' form a (0, m, 2)-net in base 2, and a nonsingular
        # lower-triangular scrambling plus a shift keeps it: every elementary box of volume
        # 2^-8 holds exactly one of the first 2^8 points
        x, y = raw[m, 0, :256], raw[m, 1, :256]
        for k1 in range(9):
            cells = (x >> (32 - k1) if k1 else 0 * x) * (1 << (8 - k1)) + (y >> (24 + k1) if k1 < 8 else 0 * y)
            assert len(set(cells.tolist())) == 256


def test_lms_differs_from_the_shift_alone():
    jk = inputs.joe_kuo_table()
    a = O.Sequence(O.SOBOL_LMS, 8, 1, seed=4, joe_kuo=jk).points(64, transform=O.RAW)
    b = O.Sequence(O.SOBOL_DS, 8, 1, seed=4, joe_kuo=jk).points(64, transform=O.RAW)
    assert np.all(a[0, :, 0] == b[0, :, 0])          # point 0: x = 0, so L x = 0, only the shift
    assert np.mean(a != b) > 0.8


# ------------------------------------------------------------------ Table 1 CPU generators
@pytest.mark.parametrize("seq", [O.HALTON_RS, O.RASRAP])
@pytest.mark.parametrize("n_start", [0, 1, 8191, 123456])
def test_algorithm2_stream_equals_counter_based(seq, n_start):
    # Algorithm 2 (recursive odometer with cached suffix sums) and Algorithm 3 (counter-based)
    # give the same numerators; the runs cross carries of many digits in small bases
    q = O.Sequence(seq, 30, 2, seed=17)
    count = 3000
    got = q.stream(n_start, count, threads=2)
    ref = q.points(n_start + count, transform=O.RAW)[:, :, n_start:]
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("seq", [O.SOBOL_DS, O.SOBOL_LMS])
@pytest.mark.parametrize("n_start", [0, 5, 1023, 77777])
def test_gray_code_stream_is_the_gray_permutation(seq, n_start):
    # Antonov-Saleev: element c of the stream is the point of index g(n_start + c)
    q = O.Sequence(seq, 24, 2, seed=3, joe_kuo=inputs.joe_kuo_table())
    count = 2048
    got = q.stream(n_start, count, threads=2)
    for m in range(2):
        for j in (0, 1, 7, 23):
            for c in range(0, count, 97):
                n = n_start + c
                assert int(got[m, j, c]) == q.raw(m, j, n ^ (n >> 1))[0]
    # each aligned block of 2^k Gray-order points is the same set as the binary-order block
    if n_start == 0:
        ref = q.points(count, transform=O.RAW)
        for k in (4, 11):
            assert sorted(got[1, 5, :1 << k].tolist()) == sorted(ref[1, 5, :1 << k].tolist())


# ------------------------------------------------------------------ inverse normal
def test_ndtri_matches_scipy():
    special = pytest.importorskip("scipy.special")
    qs = np.concatenate([np.logspace(-20, np.log10(0.4999), 400), [0.5 - 1e-9, 0.25, 0.1]])
    for q in qs:
        x = O.ndtri_lower(q)
        ref = special.ndtri(q)
        assert abs(x - ref) <= 2e-14 * max(1.0, abs(ref)), (q, x, ref)


def test_ndtri_round_trip_and_symmetry():
    import math
    for q in [1e-18, 3e-12, 1e-6, 0.01, 0.2, 0.49]:
        x = O.ndtri_lower(q)
        # one ulp of x moves q by |x| ulp relative
        assert abs(0.5 * math.erfc(-x / math.sqrt(2)) - q) <= 4e-16 * max(1.0, x * x) * 8 * q
    for u in [0.125, 0.375, 0.0625]:
        assert O.ndtri(u) == -O.ndtri(1.0 - u)
    assert O.ndtri_lower(0.5) == 0.0


def test_normal_uses_exact_complement():
    # raw = D-1 is the largest uniform; its normal is +Phi^-1(1 - 1/(2D)) computed
    # from q = 1/(2D), never from 1 - u.
    q = O.Sequence(O.PHILOX, 4, 1, seed=3)
    z = q.points(4096, transform=O.NORMAL)
    raw = q.points(4096, transform=O.RAW)
    D = 2.0**32
    for (j, i) in zip(*np.unravel_index(np.argsort(raw[0].ravel())[-3:], raw[0].shape)):
        r = int(raw[0, j, i])
        want = -O.ndtri_lower((2**32 - 1 - r + 0.5) / D)
        assert z[0, j, i] == want and want > 3.0
