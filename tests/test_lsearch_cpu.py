"""Host-side pins of the logarithmic searches (Section 3): the constants the
library computes (P, Q, U, F, S, J, L) and the readings of the garbled lines
are checked by simulating each algorithm exactly as the paper states it, on
integer positions, for every possible answer.

For a query z with X_a <= z < X_{a+1} (0 <= a <= N-1) the comparison
z >= X_r is true exactly for r <= a, and false on the padding (X_N > z).  So
every algorithm can be run on the index alone, and must return a, never read
past its layout, and (LeadBit) never read past Q - 1."""
import numpy as np
import pytest

from paper_1506_08620_gb300 import _abi


@pytest.fixture(scope="module")
def L():
    return _abi.lib()


def consts(L, method, n_knots):
    import ctypes
    c = (ctypes.c_int64 * 4)()
    n = ctypes.c_int64()
    assert L.ds_lsearch_constants(method, n_knots, c, ctypes.byref(n)) == _abi.DS_OK
    return list(c), n.value


SIZES = list(range(2, 300)) + [511, 512, 513, 1023, 1024, 1025, 4095, 4096, 65535, 65536, 65537]


def _ge(a):
    return lambda r: r <= a


def test_classicmod_iterations(L):
    for n in SIZES:
        N = n - 1
        c, length = consts(L, _abi.DS_LS_CLASSICMOD, n)
        assert length == n and 2 ** c[0] >= N and (c[0] == 0 or 2 ** (c[0] - 1) < N)
        for a in range(0, N, max(1, N // 97)):
            lo, hi = 0, N
            for _ in range(c[0]):
                mid = (lo + hi) // 2
                if mid > a:
                    hi = mid
                else:
                    lo = mid
            assert lo == a


def test_leadbit_padding_q(L):
    for n in SIZES:
        N = n - 1
        c, length = consts(L, _abi.DS_LS_LEADBIT, n)
        P, Q = c[0], c[1]
        assert P == 1 << (N.bit_length() - 1)           # 2^floor(log2 N)
        # Q by the paper's definition
        s, ubar_s = 0, None
        k = P
        while k:
            s += k
            if ubar_s is None and s >= N:
                ubar_s = s
            k //= 2
        assert Q == 1 + ubar_s and length == max(Q, n)
        worst = 0
        for a in range(N):
            i, k = 0, P
            while k:
                r = i | k
                worst = max(worst, r)
                if r <= a:
                    i = r
                k //= 2
            assert i == a
        assert worst <= Q - 1  # the padded array covers every index formed
        # and Q is not larger than needed by more than the formula's own margin
        assert Q - 1 <= 2 * P - 1


def test_leadbit_nopad_u(L):
    for n in SIZES:
        N = n - 1
        c, length = consts(L, _abi.DS_LS_LEADBIT_NOPAD, n)
        P, U = c[0], c[1]
        assert length == n
        # U = sup{u : sum_{k=1..u} P/2^(k-1) <= N}: the first U indices never pass N
        assert sum(P >> k for k in range(U)) <= N
        assert U == (P.bit_length()) or sum(P >> k for k in range(U + 1)) > N
        for a in range(N):
            i, k = 0, P
            for _ in range(U):
                r = i | k
                assert r <= N
                if r <= a:
                    i = r
                k //= 2
            while k:
                r = i | k
                w = min(r, N)
                if w <= a:
                    i = r
                k //= 2
            assert i == a


def test_offset_constants_and_size_update(L):
    # the size update of Algorithm naiveoffset is read as S <- S - H
    for n in SIZES:
        N = n - 1
        c, length = consts(L, _abi.DS_LS_OFFSET, n)
        F0, S0, J = c[0], c[1], c[2]
        assert F0 == (N + 1) // 2 and S0 == N + 1 - F0 and J == (N + 1).bit_length() - 1
        for a in range(N):
            i = F0 if F0 <= a else 0
            S = S0
            for _ in range(J):
                h = S // 2
                F = i + h
                assert F <= N
                if F <= a:
                    i = F
                S -= h
            assert i == a


def test_eytzinger_layout_and_mask(L):
    # M = not(2L) is read as not(2^L): i = P - 2^L for X_0 <= z < X_N
    for n in SIZES[:200] + SIZES[-6:]:
        N = n - 1
        c, length = consts(L, _abi.DS_LS_EYTZINGER, n)
        Lh = c[0]
        assert Lh == 1 + (N + 2).bit_length() - 1 and length == 2 ** Lh - 1 and length >= n
        # breadth-first layout of the padded sorted array by an in-order walk
        rank = np.empty(length, dtype=np.int64)
        counter = iter(range(length))

        def walk(k):
            if k < length:
                walk(2 * k + 1)
                rank[k] = next(counter)
                walk(2 * k + 2)
        walk(0)
        for a in range(0, N, max(1, N // 61)):
            P = 2 if rank[0] <= a else 1
            for _ in range(1, Lh):
                P = 2 * P + (2 if min(rank[P], N) <= a else 1)
            assert P - 2 ** Lh == a and (P & ~(2 ** Lh)) == a


def test_bad_arguments(L):
    import ctypes
    c = (ctypes.c_int64 * 4)()
    n = ctypes.c_int64()
    assert L.ds_lsearch_constants(9, 10, c, ctypes.byref(n)) == _abi.DS_E_ARG
    assert L.ds_lsearch_constants(_abi.DS_LS_OFFSET, 1, c, ctypes.byref(n)) == _abi.DS_E_ARG
