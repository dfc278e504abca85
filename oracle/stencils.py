"""1-D building blocks of the derivative estimates (paper Sec. 3 and the
appendix "Stencil Structure").

The paper fits polynomials through coarse cell centres around each coarse cell
and reads the derivatives off the fit.  The reading used here: every
derivative D^alpha is a tensor product of 1-D stencils, one per axis.  Along
an axis with alpha_d = 0 the stencil is a point evaluation on c's line; along
an axis with alpha_d > 0 it is the exact alpha_d-th derivative, at c, of the
Lagrange polynomial through a window of consecutive cell centres.  The window
is centred on c where possible (the appendix favours central differences) and
shifted inward at the ends of the available data (biased towards the centre of
the pre-image patch, since there is no diagonal data).

Everything here is exact rational arithmetic (``fractions.Fraction``); the
callers round the weights to float64 once.
"""
from fractions import Fraction
from functools import lru_cache


class Unsupported(ValueError):
    """The available data range is too short for the requested stencil."""


def window_length(exactness_degree):
    """Smallest odd number of points that fits a polynomial of the given degree.

    A Lagrange fit through L points reproduces degree L-1, so L >= E+1; odd
    lengths allow a centred window."""
    need = exactness_degree + 1
    return need if need % 2 == 1 else need + 1


def window(centre, lo, hi, exactness_degree):
    """Consecutive integer positions used for one 1-D derivative stencil.

    centre: index of the expansion point; [lo, hi]: available indices
    (inclusive); exactness_degree E: the stencil must be exact on polynomials
    of degree E.  The odd window of ``window_length(E)`` points is centred on
    ``centre`` and shifted inward to fit [lo, hi].  If [lo, hi] is shorter than
    that but still holds E+1 points, the whole range is used.  Shorter ranges
    raise Unsupported."""
    avail = hi - lo + 1
    need = exactness_degree + 1
    if avail < need:
        raise Unsupported(f"range [{lo},{hi}] holds {avail} points, need {need}")
    length = window_length(exactness_degree)
    if avail < length:
        return tuple(range(lo, hi + 1))
    start = centre - length // 2
    start = max(lo, min(start, hi - length + 1))
    return tuple(range(start, start + length))


def _poly_mul_linear(coeffs, root_shift):
    """Multiply a polynomial in t (coefficient list, ascending) by (t - root_shift)."""
    out = [Fraction(0)] * (len(coeffs) + 1)
    for i, c in enumerate(coeffs):
        out[i + 1] += c
        out[i] -= c * root_shift
    return out


@lru_cache(maxsize=None)
def lagrange_derivative_weights(points, x0, order):
    """Weights w_i with sum_i w_i f(points[i]) = f^(order)(x0) exactly for
    every polynomial f of degree < len(points).

    Built from the Lagrange basis: l_i(x) = prod_{j != i} (x - x_j)/(x_i - x_j)
    is expanded in powers of t = x - x0; the order-th derivative at t = 0 is
    order! times the coefficient of t^order."""
    points = tuple(Fraction(p) for p in points)
    x0 = Fraction(x0)
    if order >= len(points):
        return tuple(Fraction(0) for _ in points)
    factorial = 1
    for r in range(2, order + 1):
        factorial *= r
    weights = []
    for i, xi in enumerate(points):
        coeffs = [Fraction(1)]
        denom = Fraction(1)
        for j, xj in enumerate(points):
            if j == i:
                continue
            # (x - x_j) = t - (x_j - x0)
            coeffs = _poly_mul_linear(coeffs, xj - x0)
            denom *= xi - xj
        weights.append(coeffs[order] * factorial / denom)
    return tuple(weights)


def multi_indices(max_degree, dim=3):
    """All alpha in N^dim with |alpha| <= max_degree, ordered by total degree
    then lexicographically (1 + 3 + 6 = 10 for degree 2, 20 for degree 3,
    the coefficient counts the paper gives in Sec. 3)."""
    out = []
    for total in range(max_degree + 1):
        for a in range(total, -1, -1):
            for b in range(total - a, -1, -1):
                c = total - a - b
                if dim == 3:
                    out.append((a, b, c))
    return out


def exactness_degree(alpha, axis, order):
    """E_d = m - |alpha| + alpha_d: the highest power along axis d of a
    monomial of total degree <= m whose D^alpha derivative is non-zero.  The
    axis-d stencil of D^alpha must be exact up to that degree for the tensor
    stencil to reproduce every polynomial of total degree <= m."""
    return order - sum(alpha) + alpha[axis]
