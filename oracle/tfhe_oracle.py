"""TFHE external product and CMux step -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU baseline leg may use
this module.  It states, as plainly as possible, the batched CMux gate that
the paper builds its LUT evaluation on (Sec. II-B "TFHE Scheme": RLWE and
RGSW ciphertexts, blind rotation by repeated CMux with an external product;
Sec. IV-A: all ciphertexts of one iteration share one key RGSW(s_i)):

  RLWE ciphertext  d = (d_0, d_1) = (B(x), A(x)), polynomials of R_q
  gadget           B = 2^beta, l levels, g_j = round(q / B^(j+1)), j = 0..l-1
  decomposition    of v in Z_q: t = round(v B^l / q) mod B^l, written with
                   signed digits e_0..e_(l-1) in [-B/2, B/2) (e_0 most
                   significant) such that sum_j e_j B^(l-1-j) = t (mod B^l);
                   then sum_j e_j g_j ~ v (mod q)
  RGSW key         K = rows K_p = (K_p,0, K_p,1), p = i*l + j  (2l rows)
  external product K [x] d = sum_{i, j} Dec_j(d_i) * K_(i*l+j)   (per output c)
  CMux step        acc' = acc + K [x] (x^a * acc - acc)          (a in [0, 2N))

The key is given in the NTT domain (the bit-reversed evaluation order of the
forward transform, Eq. 1); the oracle brings it back with the O(N^2)
definition of the inverse and multiplies with the O(N^2) schoolbook product,
so no fast transform is involved anywhere here.

Readings where the paper is silent (also listed in the design notes): the
gadget is the approximate one over a prime q (top beta*l bits, rounded), the
key rows are ordered input polynomial first then level, and x^a for
a in [N, 2N) is -x^(a-N) (x^N = -1).
"""
import numpy as np

from . import oracle as O


def gadget(q, log2_base, levels):
    """g_j = round(q / B^(j+1)) for j = 0..levels-1 (B = 2^log2_base)."""
    return [(q + (1 << (log2_base * (j + 1) - 1))) >> (log2_base * (j + 1)) for j in range(levels)]


def decompose(v, q, log2_base, levels):
    """Signed digits [e_0, ..., e_(l-1)] of v in [0, q), most significant first."""
    base = 1 << log2_base
    t = ((v << (log2_base * levels)) + q // 2) // q          # round(v B^l / q), no ties for odd q
    t %= 1 << (log2_base * levels)
    digits = [0] * levels
    for j in reversed(range(levels)):                        # least significant digit first
        e = t % base
        t //= base
        if e >= base // 2:
            e -= base
            t += 1
        digits[j] = e
    return digits                                            # a carry out of the top is q ~ 0


def rotate(p, a, q):
    """x^a * p(x) mod (x^N + 1, q) for a in [0, 2N), by moving coefficients."""
    n = len(p)
    out = [0] * n
    for m in range(n):
        k = m + a
        sign = 1
        while k >= n:                                        # x^N = -1
            k -= n
            sign = -sign
        out[k] = (out[k] + sign * int(p[m])) % q
    return out


def digit_polys(d, q, log2_base, levels):
    """[2l][N] residues: row i*l + j is Dec_j(d_i) with negative digits as q + e."""
    rows = []
    for poly in d:
        digs = [decompose(int(v), q, log2_base, levels) for v in poly]
        for j in range(levels):
            rows.append([e % q for e in (dd[j] for dd in digs)])
    return np.array(rows, dtype=np.uint64)


def key_coefficients(key_ntt, q):
    """The key's rows back in the coefficient domain ([2l][2][N]), by the
    inverse-transform definition."""
    key_ntt = np.asarray(key_ntt, dtype=np.uint64)
    return np.array([[O.ntt_inverse(key_ntt[p, c], q) for c in range(2)] for p in range(key_ntt.shape[0])],
                    dtype=np.uint64)


def external_product(d, key_ntt, q, log2_base, levels, key_coef=None, idx=None):
    """K [x] d for one RLWE ciphertext d ([2][N]); all coefficients, or those at idx."""
    d = np.asarray(d, dtype=np.uint64)
    kc = key_coefficients(key_ntt, q) if key_coef is None else key_coef
    dig = digit_polys(d, q, log2_base, levels)
    n = d.shape[1]
    width = n if idx is None else len(idx)
    out = [[0] * width for _ in range(2)]
    for p in range(2 * levels):
        for c in range(2):
            if idx is None:
                prod = O.schoolbook(dig[p], kc[p, c], q)
            else:
                prod = O.schoolbook_at(dig[p], kc[p, c], q, np.asarray(idx, dtype=np.uint32))
            out[c] = [(x + int(y)) % q for x, y in zip(out[c], prod)]
    return np.array(out, dtype=np.uint64)


def cmux_rotate(acc, a, key_ntt, q, log2_base, levels, key_coef=None, idx=None):
    """One blind-rotation step of one ciphertext: acc + K [x] (x^a acc - acc)."""
    acc = np.asarray(acc, dtype=np.uint64)
    diff = np.array([[(r - int(x)) % q for r, x in zip(rotate(acc[i], a, q), acc[i])] for i in range(2)],
                    dtype=np.uint64)
    ep = external_product(diff, key_ntt, q, log2_base, levels, key_coef=key_coef, idx=idx)
    base = acc if idx is None else acc[:, np.asarray(idx)]
    return np.array([[(int(x) + int(y)) % q for x, y in zip(base[c], ep[c])] for c in range(2)],
                    dtype=np.uint64)
