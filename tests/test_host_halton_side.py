"""The u <= 1/2 side test of the CUDA path's digit split of a Halton coordinate (Sec. 3.1).

The kernels write a coordinate's numerator as num = R P + S with R < p^L the permuted low
digits and S < P the permuted high digits, D = p^L P, and take the exact side num <= D-1-num
(the normal transform needs it, eq. (perm) puts u = (num + 1/2)/D) as one integer compare,
R < floor(p^L / 2) + tie with tie = [p^L odd and 2 S <= P - 1].  This checks that reading by
brute force over every (R, S) of small bases, including the middle R = (p^L - 1)/2 where the
high digits decide; a float comparison cannot see that case, as both sides round to 1/2.
"""
import pytest


@pytest.mark.parametrize("p, L, H", [(2, 3, 2), (3, 2, 2), (3, 3, 1), (5, 2, 2), (7, 1, 3), (11, 2, 1)])
def test_threshold_side_test_is_exact(p, L, H):
    pL, P = p**L, p**H
    D = pL * P
    for S in range(P):
        thr = pL // 2 + (1 if (pL & 1) and S <= P - 1 - S else 0)
        for R in range(pL):
            num = R * P + S
            assert (num <= D - 1 - num) == (R < thr), (p, L, H, R, S)


def test_middle_is_decided_by_the_high_digits():
    # p^L odd: at R = (p^L - 1)/2 both halves occur, as S runs over [0, P)
    p, L, H = 3, 2, 2
    pL, P = p**L, p**H
    R = (pL - 1) // 2
    sides = {(R * P + S) <= pL * P - 1 - (R * P + S) for S in range(P)}
    assert sides == {True, False}
