"""A literal exterior algebra for Gaussian Grassmann integrals on tiny spaces (test helper).

Elements are dicts from sorted generator tuples to coefficients; multiplication sorts the
concatenated generators and counts transpositions for the sign.  With the action
S = sum_ij A[i, j] qbar_i q_j, < X > = int X e^{-S} / int e^{-S} takes the coefficient of the
top monomial; e^{-S} is the finite series up to S^N.  It checks the permutation formulas of
the oracle's Wick and baryon contractions independently of them.
"""


def _mono_mul(a, b):
    """Product of two monomials (sorted generator tuples): (sign, monomial) or None."""
    if set(a) & set(b):
        return None
    seq = list(a) + list(b)
    sign = 1
    for i in range(len(seq)):              # bubble sort counting swaps
        for j in range(len(seq) - 1 - i):
            if seq[j] > seq[j + 1]:
                seq[j], seq[j + 1] = seq[j + 1], seq[j]
                sign = -sign
    return sign, tuple(seq)


def _mul(x, y):
    out = {}
    for ma, ca in x.items():
        for mb, cb in y.items():
            r = _mono_mul(ma, mb)
            if r is None:
                continue
            s, m = r
            out[m] = out.get(m, 0) + s * ca * cb
    return out


def _add(x, y, scale=1.0):
    out = dict(x)
    for m, c in y.items():
        out[m] = out.get(m, 0) + scale * c
    return out


class Grassmann:
    """q_j is generator j, qbar_i is generator N + i."""

    def __init__(self, A):
        self.N = A.shape[0]
        S = {}
        for i in range(self.N):
            for j in range(self.N):
                if A[i, j] != 0:
                    S = _add(S, _mul(self.qbar(i), self.q(j)), A[i, j])
        w, term = {(): 1.0}, {(): 1.0}
        for k in range(1, self.N + 1):                       # e^{-S} terminates at S^N
            term = {m: -c / k for m, c in _mul(term, S).items()}
            w = _add(w, term)
        self.weight = w
        self.top = tuple(range(2 * self.N))
        self.Z = w.get(self.top, 0)

    def q(self, j):
        return {(j,): 1.0}

    def qbar(self, i):
        return {(self.N + i,): 1.0}

    def bilinear(self, M, off_bar, off_q):
        out = {}
        n = M.shape[0]
        for i in range(n):
            for j in range(n):
                if M[i, j] != 0:
                    out = _add(out, _mul(self.qbar(off_bar + i), self.q(off_q + j)), M[i, j])
        return out

    def expect(self, x):
        return _mul(x, self.weight).get(self.top, 0) / self.Z


