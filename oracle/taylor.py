"""Second-order truncated Taylor arithmetic in one variable t (oracle).

A ``Jet`` holds f(0), f'(0), f''(0) of a function of t, elementwise over
numpy arrays. Composing Jets with the operations below gives exact first and
second derivatives along a line, e.g. for E(x + t p): E, g^T p and p^T H p.
Branches (region selection in distance queries, clamping) are decided on the
value part, which is exactly how the underlying piecewise function behaves
away from region boundaries.
"""
from __future__ import annotations

import numpy as np


class Jet:
    __slots__ = ("v", "d", "dd")
    __array_ufunc__ = None          # make numpy defer to the reflected operators

    def __init__(self, v, d=None, dd=None):
        self.v = np.asarray(v, dtype=np.float64)
        self.d = np.zeros_like(self.v) if d is None else np.asarray(d, dtype=np.float64)
        self.dd = np.zeros_like(self.v) if dd is None else np.asarray(dd, dtype=np.float64)

    # --- arithmetic ---------------------------------------------------------
    def __add__(self, o):
        if isinstance(o, Jet):
            return Jet(self.v + o.v, self.d + o.d, self.dd + o.dd)
        return Jet(self.v + o, self.d, self.dd)

    __radd__ = __add__

    def __neg__(self):
        return Jet(-self.v, -self.d, -self.dd)

    def __sub__(self, o):
        return self + (-o)

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        if isinstance(o, Jet):
            return Jet(self.v * o.v, self.v * o.d + self.d * o.v,
                       self.v * o.dd + 2.0 * self.d * o.d + self.dd * o.v)
        return Jet(self.v * o, self.d * o, self.dd * o)

    __rmul__ = __mul__

    def recip(self):
        iv = 1.0 / self.v
        return Jet(iv, -self.d * iv * iv, 2.0 * self.d * self.d * iv ** 3 - self.dd * iv * iv)

    def __truediv__(self, o):
        if isinstance(o, Jet):
            return self * o.recip()
        return Jet(self.v / o, self.d / o, self.dd / o)

    def __rtruediv__(self, o):
        return self.recip() * o

    def __getitem__(self, k):
        return Jet(self.v[k], self.d[k], self.dd[k])

    def sum(self, axis=None):
        return Jet(self.v.sum(axis), self.d.sum(axis), self.dd.sum(axis))

    @property
    def shape(self):
        return self.v.shape


def apply(f0, f1, f2, x):
    """Chain rule for a scalar function with value/derivative arrays f0, f1,
    f2 already evaluated at x.v."""
    return Jet(f0, f1 * x.d, f2 * x.d * x.d + f1 * x.dd)


def val(x):
    return x.v if isinstance(x, Jet) else np.asarray(x)


def sqrt(x):
    if not isinstance(x, Jet):
        return np.sqrt(x)
    s = np.sqrt(x.v)
    with np.errstate(divide="ignore", invalid="ignore"):
        return apply(s, 0.5 / s, -0.25 / (s * x.v), x)


def log(x):
    if not isinstance(x, Jet):
        return np.log(x)
    return apply(np.log(x.v), 1.0 / x.v, -1.0 / (x.v * x.v), x)


def absolute(x):
    if not isinstance(x, Jet):
        return np.abs(x)
    sg = np.where(x.v < 0, -1.0, 1.0)
    return Jet(x.v * sg, x.d * sg, x.dd * sg)


def where(mask, a, b):
    if not isinstance(a, Jet) and not isinstance(b, Jet):
        return np.where(mask, a, b)
    a = a if isinstance(a, Jet) else Jet(np.broadcast_to(np.asarray(a, dtype=np.float64), np.shape(mask)))
    b = b if isinstance(b, Jet) else Jet(np.broadcast_to(np.asarray(b, dtype=np.float64), np.shape(mask)))
    return Jet(np.where(mask, a.v, b.v), np.where(mask, a.d, b.d), np.where(mask, a.dd, b.dd))


def clip01(x):
    """Clamp to [0, 1]; a clamped value is a constant (zero derivatives)."""
    if not isinstance(x, Jet):
        return np.clip(x, 0.0, 1.0)
    lo, hi = x.v < 0.0, x.v > 1.0
    out = Jet(np.clip(x.v, 0.0, 1.0), x.d.copy(), x.dd.copy())
    out.d[lo | hi] = 0.0
    out.dd[lo | hi] = 0.0
    return out


def dot(a, b):
    """Sum over the last axis of a * b."""
    return (a * b).sum(axis=-1)


def cross(a, b):
    def c(i):
        return a[..., i]

    def e(i):
        return b[..., i]
    x = c(1) * e(2) - c(2) * e(1)
    y = c(2) * e(0) - c(0) * e(2)
    z = c(0) * e(1) - c(1) * e(0)
    return stack3(x, y, z)


def stack3(x, y, z):
    if isinstance(x, Jet) or isinstance(y, Jet) or isinstance(z, Jet):
        x, y, z = (q if isinstance(q, Jet) else Jet(q) for q in (x, y, z))
        return Jet(np.stack([x.v, y.v, z.v], -1), np.stack([x.d, y.d, z.d], -1),
                   np.stack([x.dd, y.dd, z.dd], -1))
    return np.stack([x, y, z], -1)


def expand(x, axis=-1):
    """Insert a length-1 axis (for broadcasting a per-row scalar)."""
    if isinstance(x, Jet):
        return Jet(np.expand_dims(x.v, axis), np.expand_dims(x.d, axis), np.expand_dims(x.dd, axis))
    return np.expand_dims(x, axis)


def line(x, p):
    """The Jet of x + t p at t = 0."""
    return Jet(np.asarray(x, dtype=np.float64), np.asarray(p, dtype=np.float64))
