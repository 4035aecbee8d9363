"""Exact centred finite-difference coefficients for the Laplacian, derived, not typed.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The heat-equation kernel of Sec. 4.1 uses second-order centred differences; the SMC
kernel of Sec. 4.2 uses 8th-order stencils that span 9 cells per direction.  Both are
members of one family: the (2R+1)-point centred approximation of d^2/dx^2 of maximal
order 2R,

    (L_R u)_i = c_0 u_i + sum_{m=1..R} c_m (u_{i+m} + u_{i-m}).

The c_m follow from the moment conditions obtained by applying L_R to the monomials
x^{2k} at x = 0 (odd monomials vanish by symmetry):

    k = 0:        c_0 + 2 sum_m c_m         = 0
    k = 1:        2 sum_m c_m m^2           = 2           (the second derivative of x^2)
    k = 2..R:     2 sum_m c_m m^{2k}        = 0

The flux (conservative) form used by the kernel (fluxes on faces, then their divergence,
Sec. 4.1) writes the same operator as F_{i+1/2} - F_{i-1/2} with

    F_{i+1/2} = sum_{m=1..R} b_m (u_{i+m} - u_{i+1-m}),     b_m = sum_{j>=m} c_j,

and ``flux_coefficients`` checks that identity term by term in exact arithmetic.
"""
from fractions import Fraction


def _solve(a, rhs):
    """Gaussian elimination over the rationals (a is square, nonsingular)."""
    n = len(a)
    m = [list(row) + [r] for row, r in zip(a, rhs)]
    for col in range(n):
        piv = next(r for r in range(col, n) if m[r][col] != 0)
        m[col], m[piv] = m[piv], m[col]
        for r in range(n):
            if r != col and m[r][col] != 0:
                f = m[r][col] / m[col][col]
                m[r] = [x - f * y for x, y in zip(m[r], m[col])]
    return [m[i][n] / m[i][i] for i in range(n)]


def laplacian_coefficients(R):
    """[c_0, c_1, ..., c_R] as Fractions for the (2R+1)-point centred Laplacian of order 2R."""
    if R < 1:
        raise ValueError("R >= 1")
    # unknowns c_1..c_R; equations k = 1..R
    a = [[Fraction(2 * m ** (2 * k)) for m in range(1, R + 1)] for k in range(1, R + 1)]
    rhs = [Fraction(2)] + [Fraction(0)] * (R - 1)
    c = _solve(a, rhs)
    c0 = -2 * sum(c)
    return [c0] + c


def flux_coefficients(R):
    """[b_1, ..., b_R] with b_m = sum_{j>=m} c_j; asserts that the flux difference
    F_{i+1/2} - F_{i-1/2} reproduces the direct stencil exactly."""
    c = laplacian_coefficients(R)
    b = [sum(c[m:], Fraction(0)) for m in range(1, R + 1)]
    # expand F_{i+1/2} - F_{i-1/2} into weights on u_{i+s}, s = -R..R
    w = {s: Fraction(0) for s in range(-R, R + 1)}
    for m, bm in enumerate(b, start=1):
        w[m] += bm          # u_{i+m}        in F_{i+1/2}
        w[1 - m] -= bm      # u_{i+1-m}      in F_{i+1/2}
        w[m - 1] -= bm      # u_{i-1+m}      in F_{i-1/2}
        w[-m] += bm         # u_{i-m}        in F_{i-1/2}
    assert w[0] == c[0], (w[0], c[0])
    for m in range(1, R + 1):
        assert w[m] == c[m] and w[-m] == c[m], (m, w[m], w[-m], c[m])
    return b


def symbol(R, theta):
    """Fourier symbol of L_R: sigma_R(theta) = c_0 + 2 sum_m c_m cos(m theta) (float)."""
    import math
    c = laplacian_coefficients(R)
    return float(c[0]) + 2.0 * sum(float(c[m]) * math.cos(m * theta) for m in range(1, R + 1))
