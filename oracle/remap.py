"""Strategy-1 remap to the mean-position grid, and fields at lifted
positions (test infrastructure).

TEST INFRASTRUCTURE ONLY: used by tests/ (and bench.py's cpu_baseline leg),
never by the product path.  Shares no code with the CUDA library.

Sec. 3.1, Eq. (remap-strat1): f~^L(x, tau) = fbar^L(Xi^{-1}(x, tau+T), tau).
Strategy 1 delivers f~^L and the mean positions Xi^{-1}(x, tau+T) at the
grid points x, i.e. fbar^L at the scattered points Xi^{-1}(x).  The paper
leaves the interpolation open (Sec. 5 warns that these points may cluster).
The reading taken here evaluates fbar^L at the grid points y instead, through
the lift map Xi = (Xi^{-1})^{-1} (Eq. (Xi-def)):

    fbar^L(y) = f~^L(Xi(y)),   Xi(y) = y + xi(y),

where the displacement xi solves Xi^{-1}(y + xi) = y.  With the periodic
displacement d = x - Xi^{-1}(x) (= D/T of the Strategy-1 solver) this is
the fixed point xi = d(y + xi), found by the iteration

    xi^0 = 0,   xi^{k+1} = d_I(y + xi^k),   k < iters,

(a contraction while |grad d| < 1, i.e. while Xi^{-1} stays invertible),
and f~^L is then read at y + xi.  Off-grid values d_I and f~^L(y + xi) are
bilinear interpolants, the same rule as the Strategy-2 solver (Sec. 4.2.1):
cell index i + floor(xi/dx) taken periodically, weight xi/dx - floor(xi/dx).
The xi found this way is the Strategy-2 displacement (Xi = x + xi, Sec. 3.2).
"""
from __future__ import annotations

import numpy as np


def grid(N):
    """Grid coordinates X[j, i] = x_i, Y[j, i] = y_j with x_i = 2 pi i / N."""
    x = 2 * np.pi * np.arange(N) / N
    return np.meshgrid(x, x)


def bilinear_at_displacement(f, xi_x, xi_y):
    """Bilinear periodic interpolation of the grid field f at (x_i + xi_x, y_j + xi_y)."""
    N = f.shape[0]
    inv_dx = N / (2.0 * np.pi)
    cx = xi_x * inv_dx
    cy = xi_y * inv_dx
    fx = np.floor(cx)
    fy = np.floor(cy)
    ax = cx - fx
    ay = cy - fy
    i = np.arange(N)[None, :]
    j = np.arange(N)[:, None]
    i0 = (i + fx.astype(np.int64)) % N
    j0 = (j + fy.astype(np.int64)) % N
    i1 = (i0 + 1) % N
    j1 = (j0 + 1) % N
    return ((1 - ax) * (1 - ay) * f[j0, i0] + ax * (1 - ay) * f[j0, i1]
            + (1 - ax) * ay * f[j1, i0] + ax * ay * f[j1, i1])


def remap_strategy1(ftilde, pos_x, pos_y, iters=20):
    """Remap Strategy-1 means onto the mean-position grid (Eq. remap-strat1).

    ftilde: dict name -> N x N field f~^L on the grid x; pos_x, pos_y: the
    mean positions Xi^{-1}(x, tau+T) at the grid points (unwrapped, as the
    solver reports them).  Returns (fbar dict, Xi_x, Xi_y, resid) with
    resid = max |xi^iters - xi^(iters-1)| per point (the last update).
    """
    N = pos_x.shape[0]
    X, Y = grid(N)
    d_x = X - pos_x
    d_y = Y - pos_y
    xi_x = np.zeros_like(d_x)
    xi_y = np.zeros_like(d_y)
    resid = np.zeros_like(d_x)
    for _ in range(iters):
        nx = bilinear_at_displacement(d_x, xi_x, xi_y)
        ny = bilinear_at_displacement(d_y, xi_x, xi_y)
        resid = np.maximum(np.abs(nx - xi_x), np.abs(ny - xi_y))
        xi_x, xi_y = nx, ny
    fbar = {k: bilinear_at_displacement(v, xi_x, xi_y) for k, v in ftilde.items()}
    return fbar, X + xi_x, Y + xi_y, resid


def lift(fields, pos_x, pos_y):
    """Fields evaluated at given positions, f(Xi(x)), by the bilinear rule.

    With Xi the Strategy-2 lift map (Sec. 3.2; Xi = x + xi), this gives the
    instantaneous field at the particles' positions: Sec. 4.2.2 forms the
    Lagrangian perturbation fbar^L(x) - f(x + xi(x, tau+T), tau+T), and
    Sec. 4.2.1 notes that the Lagrangian mean PV is the rearrangement
    qbar^L(x) = q(Xi(x), t).
    """
    N = pos_x.shape[0]
    X, Y = grid(N)
    return {k: bilinear_at_displacement(v, pos_x - X, pos_y - Y) for k, v in fields.items()}


def shells(N):
    """Number of wavenumber shells of the 2/3 box: round(sqrt(2) K) + 1."""
    K = (N - 1) // 3
    return int(np.floor(np.sqrt(2.0) * K + 0.5)) + 1


def spectrum(f):
    """Shell-summed spectrum of a real field on the 2/3 box (Sec. 4.2.2's
    enstrophy spectra when f is the vorticity).

    F = FFT(f)/N^2, kept for |kx|, |ky| <= K; shell n = round(|k|) collects
    |F(k)|^2 / 2 over the whole plane, so the shells sum to half the mean
    square of the box-limited field (Parseval).
    """
    N = f.shape[0]
    K = (N - 1) // 3
    F = np.fft.fft2(f) / (N * N)
    k = np.fft.fftfreq(N, 1.0 / N)
    KX, KY = np.meshgrid(k, k)
    box = (np.abs(KX) <= K) & (np.abs(KY) <= K)
    sh = np.floor(np.sqrt(KX * KX + KY * KY) + 0.5).astype(np.int64)
    out = np.zeros(shells(N))
    np.add.at(out, sh[box], 0.5 * np.abs(F[box]) ** 2)
    return out
