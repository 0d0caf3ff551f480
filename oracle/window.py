"""Kaiser-Bessel window for the NUFFT steps (oracle; test infrastructure).

Sec. 3 asks for a window Psi with compact support that is positive on the
central interval and whose Fourier transform is concentrated and known in
closed form, and names the Kaiser-Bessel function as the usual choice.  In grid
units (one unit = one oversampled grid cell) the window of width w is

    phi(x)   = I0(beta * sqrt(1 - (2x/w)^2))     for |x| <= w/2, else 0,
    phihat(xi) = int phi(x) exp(-2 pi i xi x) dx
               = w * sinh(sqrt(beta^2 - (pi w xi)^2)) / sqrt(beta^2 - (pi w xi)^2)

(sin instead of sinh once (pi w xi) > beta).  The paper gives no shape
parameter; beta = pi * sqrt((w/sigma)^2 (sigma - 1/2)^2 - 0.8) is the
published choice of Beatty, Nishimura and Pauly (2005) for oversampling sigma.
"""
from __future__ import annotations

import numpy as np


def kb_beta(width, sigma):
    return np.pi * np.sqrt((width / sigma) ** 2 * (sigma - 0.5) ** 2 - 0.8)


def kb_phi(x, width, beta):
    """phi(x) in grid units; zero outside |x| <= width/2."""
    x = np.asarray(x, dtype=np.float64)
    t = 1.0 - (2.0 * x / width) ** 2
    inside = t >= 0.0
    return np.where(inside, np.i0(beta * np.sqrt(np.where(inside, t, 0.0))), 0.0)


def kb_phi_deriv(x, width, beta):
    """d phi / dx by the chain rule with d/dz I0(z) = I1(z), I1 from its
    power series."""
    x = np.asarray(x, dtype=np.float64)
    t = 1.0 - (2.0 * x / width) ** 2
    inside = t > 0.0
    s = np.sqrt(np.where(inside, t, 1.0))
    z = beta * s
    # d/dx [beta * sqrt(t)] = beta * (1/(2 sqrt t)) * (-8x/w^2)
    dz = beta * (-4.0 * x / width ** 2) / s
    return np.where(inside, _i1(z) * dz, 0.0)


def _i1(z):
    """Modified Bessel function I1 by its power series sum (z/2)^(2k+1)/(k!(k+1)!)."""
    z = np.asarray(z, dtype=np.float64)
    h = 0.5 * z
    term = h.copy()
    total = term.copy()
    q = h * h
    for k in range(1, 200):
        term = term * q / (k * (k + 1))
        total = total + term
        if np.all(np.abs(term) <= 1e-18 * np.abs(total)):
            break
    return total


def kb_phihat(xi, width, beta):
    """Continuous Fourier transform of kb_phi at frequency xi (cycles per
    grid unit)."""
    xi = np.asarray(xi, dtype=np.float64)
    a = np.pi * width * xi
    s = beta * beta - a * a
    out = np.empty_like(s)
    pos = s > 0
    neg = s < 0
    zer = ~(pos | neg)
    r = np.sqrt(np.abs(s))
    out[pos] = width * np.sinh(r[pos]) / r[pos]
    out[neg] = width * np.sin(r[neg]) / r[neg]
    out[zer] = width
    return out
