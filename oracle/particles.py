"""Brute-force particle tracking and trajectory averaging (test infrastructure).

TEST INFRASTRUCTURE ONLY; used by tests/ to pin the oracle to the paper's
definitions, never by the product path.

This is the approach the paper replaces (Sec. 1: seed particles, track them,
average along the Lagrangian time series), applied on tiny grids to give the
Lagrangian means directly from their definitions:

* flow map, Eq. (flowmap): d phi/dt = u(phi, t);
* Lagrangian mean position, Eq. (barLbphi): phibar^L(a) = (1/T) int phi ds;
* trajectory mean of f, Eqs. (barLf), (tildeLf): (1/T) int f(phi(a, s), s) ds,
  attached either to phibar^L(a) (overbar) or to phi(a, tau+T) (tilde).

The particle ODEs are integrated with classical RK4 whose stage velocities are
the oracle's own RK4 stage fields, evaluated at the particle positions by
exact Fourier sums (no interpolation).
"""
from __future__ import annotations

import numpy as np


def fourier_eval(F, kx_max, xs, ys):
    """Evaluate the real field whose rfft2-half-plane spectrum is F at points.

    f(x, y) = Re sum_ky F[ky, 0] e^{i ky y}
              + 2 Re sum_{kx >= 1} sum_ky F[ky, kx] e^{i (kx x + ky y)},
    the continuous counterpart of numpy.fft.irfft2 scaled by N^2.
    """
    N = F.shape[0]
    kyv = np.fft.fftfreq(N, d=1.0 / N)
    sel_y = np.nonzero(np.abs(F).sum(axis=1) > 0)[0]
    sel_x = np.arange(min(F.shape[1], kx_max + 1))
    Fs = F[np.ix_(sel_y, sel_x)]
    ey = np.exp(1j * np.outer(ys, kyv[sel_y]))          # (P, ny)
    ex = np.exp(1j * np.outer(xs, sel_x.astype(float)))  # (P, nx)
    w = np.where(sel_x == 0, 1.0, 2.0)
    g = ey @ Fs                                          # (P, nx): sum over ky
    return np.real(np.sum(g * ex * w[None, :], axis=1))


class ParticleTracker:
    """Particles seeded at every grid point at tau; follow the oracle's stages."""

    def __init__(self, oracle, fields=("zeta", "h", "u", "v")):
        self.o = oracle
        N = oracle.N
        x = oracle.x
        X, Y = np.meshgrid(x, x)  # X[j, i] = x_i, Y[j, i] = y_j
        self.px = X.ravel().copy()
        self.py = Y.ravel().copy()
        self.a_x = self.px.copy()
        self.a_y = self.py.copy()
        self.fields = tuple(fields)
        self.int_px = np.zeros_like(self.px)  # int phi_x dt
        self.int_py = np.zeros_like(self.py)
        self.int_f = {f: np.zeros_like(self.px) for f in self.fields}
        self.T = 0.0

    def _vel_and_f(self, sw_stage, px, py):
        o = self.o
        uh, vh, hh = sw_stage
        K = o.K
        u = fourier_eval(uh, K, px, py)
        v = fourier_eval(vh, K, px, py)
        vals = {}
        zh = 1j * o.kx * vh - 1j * o.ky * uh
        for f in self.fields:
            if f == "u":
                vals[f] = u
            elif f == "v":
                vals[f] = v
            elif f == "h":
                # the oracle state carries eta = h - 1, and so do its means
                vals[f] = fourier_eval(hh, K, px, py)
            elif f == "zeta":
                vals[f] = fourier_eval(zh, K, px, py)
            elif f == "q":
                zeta = fourier_eval(zh, K, px, py)
                h = 1.0 + fourier_eval(hh, K, px, py)
                vals[f] = (o.f0 + zeta) / h
        return u, v, vals

    def advance(self, stages, dt):
        """One RK4 step of (phi, int phi, int f) given the 4 SW stage states."""
        x0, y0 = self.px, self.py
        u1, v1, f1 = self._vel_and_f(stages[0], x0, y0)
        x1, y1 = x0 + 0.5 * dt * u1, y0 + 0.5 * dt * v1
        u2, v2, f2 = self._vel_and_f(stages[1], x1, y1)
        x2, y2 = x0 + 0.5 * dt * u2, y0 + 0.5 * dt * v2
        u3, v3, f3 = self._vel_and_f(stages[2], x2, y2)
        x3, y3 = x0 + dt * u3, y0 + dt * v3
        u4, v4, f4 = self._vel_and_f(stages[3], x3, y3)
        # position integral: d/dt int phi = phi, with RK4 stage positions
        self.int_px += dt / 6.0 * (x0 + 2 * x1 + 2 * x2 + x3)
        self.int_py += dt / 6.0 * (y0 + 2 * y1 + 2 * y2 + y3)
        for f in self.fields:
            self.int_f[f] += dt / 6.0 * (f1[f] + 2 * f2[f] + 2 * f3[f] + f4[f])
        self.px = x0 + dt / 6.0 * (u1 + 2 * u2 + 2 * u3 + u4)
        self.py = y0 + dt / 6.0 * (v1 + 2 * v2 + 2 * v3 + v4)
        self.T += dt

    def means(self):
        """Trajectory means: end position, mean position, mean of each f."""
        T = self.T
        return dict(end_x=self.px, end_y=self.py,
                    mean_x=self.int_px / T, mean_y=self.int_py / T,
                    f={f: self.int_f[f] / T for f in self.fields})


def run_interval_with_particles(oracle, strategy, n_steps, fields=("zeta", "h", "u", "v")):
    """Run one averaging interval on the oracle while tracking particles.

    Returns (tracker, spectral LM state at the end of the interval, T).
    """
    tr = ParticleTracker(oracle, fields)
    stages = []
    oracle.lmean_begin(strategy, fields=fields, pos=True, eulerian=False, n_steps=n_steps)
    oracle._stage_hook = lambda st: stages.append(st["sw"])
    try:
        for _ in range(n_steps):
            stages.clear()
            oracle.lmean_step(1)
            tr.advance(stages, oracle.dt)
    finally:
        oracle._stage_hook = None
    lm = oracle.lm
    state = dict(G={f: lm["G"][f].copy() for f in lm["fields"]},
                 P=[p.copy() for p in lm["P"]])
    return tr, state, n_steps * oracle.dt
