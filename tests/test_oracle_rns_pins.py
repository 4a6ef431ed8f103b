"""Pins for the RNS oracle (BConv and Rescale): the Chinese remainder
reconstruction from sympy fixes what each output must be -- BConv returns
X + alpha Q for one 0 <= alpha < L in every target prime, BConv into Q
itself returns the input, Rescale returns round(X / q_last) by exact
rational rounding -- and planted mistakes (no Qhat^-1 factor, floor instead
of round, the wrong prime dropped) each fail one of them."""
import math
import types
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from oracle import rns_oracle as R
from paper_2410_05934_gb300 import workloads as W

sympy = pytest.importorskip("sympy")
from sympy.ntheory.modular import crt  # noqa: E402

Q5 = W.POOL50[:5]
P3 = W.POOL50[40:43]


def _rand(Q, n, seed):
    rng = np.random.default_rng(seed)
    return np.array([rng.integers(0, q, n, dtype=np.uint64) for q in Q])


def _crt(x, Q, k):
    return int(crt([int(q) for q in Q], [int(x[i, k]) for i in range(len(Q))])[0])


def _check_bconv(r, x, Q, P):
    y = r.bconv(x, Q, P)
    big = math.prod(int(q) for q in Q)
    for k in range(x.shape[1]):
        X = _crt(x, Q, k)
        alphas = [a for a in range(len(Q)) if all(int(y[j, k]) == (X + a * big) % int(p) for j, p in enumerate(P))]
        assert len(alphas) == 1, (k, alphas)


def _check_rescale(r, x, Q):
    y = r.rescale(x, Q)
    ql = int(Q[-1])
    for k in range(x.shape[1]):
        X = _crt(x, Q, k)
        Y = math.floor(Fraction(X, ql) + Fraction(1, 2))
        assert [int(y[i, k]) for i in range(len(Q) - 1)] == [Y % int(q) for q in Q[:-1]], k


def test_bconv_is_x_plus_alpha_q():
    _check_bconv(R, _rand(Q5, 64, 1), Q5, P3)


def test_bconv_into_q_itself_is_identity():
    x = _rand(Q5, 32, 2)
    assert np.array_equal(R.bconv(x, Q5, Q5), x)


def test_rescale_is_rounded_division():
    x = _rand(Q5, 64, 3)
    _check_rescale(R, x, Q5)
    # values next to the rounding boundary: X = m q_last + floor(q_last / 2) (+1)
    ql = int(Q5[-1])
    big = math.prod(int(q) for q in Q5)
    Xs = [(7 * ql + ql // 2) % big, (7 * ql + ql // 2 + 1) % big, 0, big - 1, ql // 2, ql // 2 + 1]
    x = np.array([[X % int(q) for X in Xs] for q in Q5], dtype=np.uint64)
    _check_rescale(R, x, Q5)


def test_rescale_in_the_ntt_domain_matches_coefficients():
    Q = [W.POOL50[0], W.POOL50[1], W.POOL50[2]]
    n = 64
    x = _rand(Q, n, 4)
    xn = np.array([O.ntt_forward(x[i], q) for i, q in enumerate(Q)])
    want = R.rescale(x, Q)
    got = R.rescale_ntt(xn, Q)
    for i in range(2):
        assert np.array_equal(O.ntt_inverse(got[i], Q[i]), want[i])
    idx = [0, 5, 63]
    assert np.array_equal(R.rescale_ntt(xn, Q, idx=idx), got[:, idx])


# ---- planted mistakes --------------------------------------------------------

def _bconv_no_inverse(x, Q, P):
    big = R.prod(Q)
    out = np.zeros((len(P), x.shape[1]), dtype=np.uint64)
    for k in range(x.shape[1]):
        for j, p in enumerate(P):
            out[j, k] = sum(int(x[i, k]) * (big // int(Q[i]) % int(p)) for i in range(len(Q))) % int(p)
    return out


def _rescale_floor(x, Q):
    ql = int(Q[-1])
    out = np.zeros((len(Q) - 1, x.shape[1]), dtype=np.uint64)
    for i in range(len(Q) - 1):
        qi = int(Q[i])
        inv = pow(ql % qi, -1, qi)
        for k in range(x.shape[1]):
            out[i, k] = (int(x[i, k]) - int(x[-1, k])) % qi * inv % qi
    return out


def _rescale_wrong_prime(x, Q):
    return R.rescale(x[::-1].copy(), list(Q)[::-1])[::-1].copy()


MUTANTS = {"bconv_no_inverse": dict(bconv=_bconv_no_inverse), "rescale_floor": dict(rescale=_rescale_floor),
           "rescale_wrong_prime": dict(rescale=_rescale_wrong_prime)}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistakes(name):
    m = types.SimpleNamespace(bconv=R.bconv, rescale=R.rescale)
    for k, v in MUTANTS[name].items():
        setattr(m, k, v)
    failed = 0
    for check in (lambda: _check_bconv(m, _rand(Q5, 16, 5), Q5, P3),
                  lambda: _check_rescale(m, _rand(Q5, 16, 6), Q5)):
        try:
            check()
        except AssertionError:
            failed += 1
    assert failed >= 1, name
