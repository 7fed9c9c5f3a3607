"""Real spherical harmonics (FP64) for "SH-evaluated color" (Eq. 2, c_i).

Test infrastructure only (see the package docstring).

The paper gives no convention. The reading: real SH of degrees 0..3 with the
Condon-Shortley phase, index k = l*l + l + m (m = -l..l), and

    Y_l0  = K_l0 P_l(z)
    Y_lm  = sqrt(2) K_lm P_l^m(z) cos(m phi)      m > 0
    Y_l-m = sqrt(2) K_lm P_l^m(z) sin(m phi)      m > 0
    K_lm  = sqrt((2l+1)/(4 pi) * (l-m)! / (l+m)!)

with P_l^m(z) = (-1)^m (1-z^2)^(m/2) d^m/dz^m P_l(z) and P_l from Rodrigues'
formula. Everything is derived here from those definitions (no tabulated
constants). On the unit sphere (1-z^2)^(m/2) e^{i m phi} = (x + i y)^m, so each
Y_lm is a polynomial in the direction's components and differentiable.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np
from numpy.polynomial import polynomial as npoly
import torch


@lru_cache(maxsize=None)
def legendre_coeffs(l: int) -> tuple:
    """Ascending coefficients of P_l(x) = 1/(2^l l!) d^l/dx^l (x^2-1)^l."""
    p = np.array([1.0])
    for _ in range(l):
        p = npoly.polymul(p, np.array([-1.0, 0.0, 1.0]))
    for _ in range(l):
        p = npoly.polyder(p)
    return tuple(p / (2.0 ** l * math.factorial(l)))


@lru_cache(maxsize=None)
def legendre_deriv_coeffs(l: int, m: int) -> tuple:
    """Ascending coefficients of d^m/dx^m P_l(x)."""
    p = np.array(legendre_coeffs(l))
    for _ in range(m):
        p = npoly.polyder(p)
    return tuple(p) if len(p) else (0.0,)


def norm_const(l: int, m: int) -> float:
    m = abs(m)
    return math.sqrt((2 * l + 1) / (4.0 * math.pi) * math.factorial(l - m) / math.factorial(l + m))


def _polyval(coeffs, z):
    out = torch.zeros_like(z)
    for c in reversed(coeffs):
        out = out * z + c
    return out


def num_coeffs(degree: int) -> int:
    return (degree + 1) ** 2


def sh_basis(dirs: torch.Tensor, degree: int) -> torch.Tensor:
    """Y_k(dir) for k < (degree+1)^2; dirs [..., 3] unit vectors -> [..., K]."""
    x, y, z = dirs.unbind(-1)
    out = []
    # (x + i y)^m as (re, im), built by repeated complex multiplication
    pow_re = [torch.ones_like(x)]
    pow_im = [torch.zeros_like(x)]
    for _ in range(degree):
        re, im = pow_re[-1], pow_im[-1]
        pow_re.append(re * x - im * y)
        pow_im.append(re * y + im * x)
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            q = _polyval(legendre_deriv_coeffs(l, am), z)
            if m == 0:
                out.append(norm_const(l, 0) * q)
            else:
                fac = math.sqrt(2.0) * norm_const(l, am) * (-1.0) ** am
                out.append(fac * q * (pow_re[am] if m > 0 else pow_im[am]))
    return torch.stack(out, dim=-1)
