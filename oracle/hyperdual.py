"""Hyper-dual numbers for exact second derivatives (oracle).

TEST INFRASTRUCTURE ONLY.  A hyper-dual number a + b e1 + c e2 + d e1e2 with
e1^2 = e2^2 = 0 carries f, f' (twice) and f'' exactly through arithmetic
(Fike and Alonso, AIAA 2011-886).  Seeding x_k = x_k + e1 + e2 makes the e1e2
part of u(x) equal to d^2 u / d x_k^2 with no truncation error; the oracle uses
this to build f = -Laplace(u) for the manufactured solutions (Section 3.1).

Pinned in tests/test_oracle_manufactured.py against a hand-derived closed form
of the Laplacian in cylindrical coordinates, against finite differences, and
primitive by primitive (log, sin, cos, products, quotients) against
hand-differentiated first and second derivatives.
"""
import numpy as np


class HD:
    __slots__ = ("a", "b", "c", "d")

    def __init__(self, a, b=0.0, c=0.0, d=0.0):
        self.a = np.asarray(a, dtype=np.float64)
        self.b = np.broadcast_to(np.asarray(b, dtype=np.float64), self.a.shape)
        self.c = np.broadcast_to(np.asarray(c, dtype=np.float64), self.a.shape)
        self.d = np.broadcast_to(np.asarray(d, dtype=np.float64), self.a.shape)

    @staticmethod
    def lift(x):
        return x if isinstance(x, HD) else HD(x)

    def apply(self, f0, f1, f2):
        """f(self) given f, f', f'' evaluated at the real part."""
        return HD(f0, f1 * self.b, f1 * self.c, f1 * self.d + f2 * self.b * self.c)

    def __add__(self, o):
        o = HD.lift(o)
        return HD(self.a + o.a, self.b + o.b, self.c + o.c, self.d + o.d)

    __radd__ = __add__

    def __neg__(self):
        return HD(-self.a, -self.b, -self.c, -self.d)

    def __sub__(self, o):
        return self + (-HD.lift(o))

    def __rsub__(self, o):
        return HD.lift(o) - self

    def __mul__(self, o):
        o = HD.lift(o)
        return HD(self.a * o.a,
                  self.a * o.b + self.b * o.a,
                  self.a * o.c + self.c * o.a,
                  self.a * o.d + self.b * o.c + self.c * o.b + self.d * o.a)

    __rmul__ = __mul__

    def reciprocal(self):
        a = self.a
        return self.apply(1.0 / a, -1.0 / (a * a), 2.0 / (a * a * a))

    def __truediv__(self, o):
        return self * HD.lift(o).reciprocal()

    def __rtruediv__(self, o):
        return HD.lift(o) * self.reciprocal()


def sin(x):
    if isinstance(x, HD):
        return x.apply(np.sin(x.a), np.cos(x.a), -np.sin(x.a))
    return np.sin(x)


def cos(x):
    if isinstance(x, HD):
        return x.apply(np.cos(x.a), -np.sin(x.a), -np.cos(x.a))
    return np.cos(x)


def log(x):
    if isinstance(x, HD):
        return x.apply(np.log(x.a), 1.0 / x.a, -1.0 / (x.a * x.a))
    return np.log(x)


def laplacian(u, X):
    """Sum over k of d^2 u / d x_k^2 at points X[..., 3] for a function u(x, y, z)."""
    total = np.zeros(X.shape[:-1])
    for k in range(3):
        args = [HD(X[..., j], 1.0 if j == k else 0.0, 1.0 if j == k else 0.0) for j in range(3)]
        total = total + u(*args).d
    return total
