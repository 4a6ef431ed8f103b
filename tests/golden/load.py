"""Reader of the hand-derived known-answer fixtures in this folder."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def _ints(s):
    return [int(v) for v in s.split()]


def negacyclic_q17():
    """[("ntt", q, log2n, psi, a, A)] and [("mul", q, log2n, a, b, c)] entries."""
    ntt, mul = [], []
    with open(os.path.join(HERE, "negacyclic_q17.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, body = line.split(":", 1)
            kind, *params = head.split()
            if kind == "ntt":
                lhs, rhs = body.split("->")
                ntt.append((int(params[0]), int(params[1]), int(params[2]), _ints(lhs), _ints(rhs)))
            elif kind == "mul":
                lhs, rhs = body.split("->")
                a, b = lhs.split("*")
                mul.append((int(params[0]), int(params[1]), _ints(a), _ints(b), _ints(rhs)))
    return ntt, mul
