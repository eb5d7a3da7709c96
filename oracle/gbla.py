"""Semi-Lagrangian discretisation of Strategy 1 (test infrastructure).

TEST INFRASTRUCTURE ONLY: used by tests/, never by the product path; shares
no code with the CUDA library.

App. B: the grid-based Lagrangian average is a semi-Lagrangian
discretisation of Eqs. (gtilde-evol) and (Xi-1evol).  After each time step
of the dynamics, at every grid point X with departure point
Y = X - dt u(X, t_{n+1}) (a backward difference of Eq. (flowmap)):

* backward Euler, Eq. (sdiscrete_gtilde):
      g(X, t_{n+1}) = g(Y, t_n) + dt f(X, t_{n+1});
* trapezoidal rule, Eq. (sdiscrete_gtilde_trapez) written for g = s f~:
      g(X, t_{n+1}) = g(Y, t_n) + dt [f(Y, t_n) + f(X, t_{n+1})]/2;
* mean positions, Eq. (sdiscrete_Xi-1) (f = x): carried, as in the spectral
  solver, through the periodic displacement D = s (x - Xi^{-1}), for which
  the same steps read D(X) = D(Y) + s_n (X - Y) + dt (X - Y) w, with w = 1/2
  for the trapezoidal rule (Eq. (sdiscrete_Xi-1) exactly) and w = 0 for
  backward Euler (the same substitution in Eq. (sdiscrete_gtilde)), where
  X - Y = dt u(X, t_{n+1}).

Values at Y need interpolation (App. B): "linear" (bilinear, the rule of the
Strategy-2 solver: cell i + floor(d/dx), weight the remainder) or "cubic"
(tensor-product 4-point Lagrange interpolation on the cells i-1 .. i+2), the
paper leaving the cubic scheme unnamed.  At the end, f~^L = g/T and
Xi^{-1} = X - D/T; Eq. (remap-strat1) then gives fbar^L (oracle.remap).
"""
from __future__ import annotations

import numpy as np


def _cells(N, dx_, dy_):
    """Cell indices and fractions of displacements (dx_, dy_) from each node."""
    inv = N / (2.0 * np.pi)
    cx = dx_ * inv
    cy = dy_ * inv
    fx = np.floor(cx)
    fy = np.floor(cy)
    i = np.arange(N)[None, :]
    j = np.arange(N)[:, None]
    return ((i + fx.astype(np.int64)) % N, (j + fy.astype(np.int64)) % N, cx - fx, cy - fy)


def interp_linear(f, dx_, dy_):
    N = f.shape[0]
    i0, j0, ax, ay = _cells(N, dx_, dy_)
    i1, j1 = (i0 + 1) % N, (j0 + 1) % N
    return ((1 - ax) * (1 - ay) * f[j0, i0] + ax * (1 - ay) * f[j0, i1]
            + (1 - ax) * ay * f[j1, i0] + ax * ay * f[j1, i1])


def lagrange4(a):
    """Weights of the cubic Lagrange interpolant through nodes -1, 0, 1, 2 at a."""
    return (-a * (a - 1) * (a - 2) / 6, (a + 1) * (a - 1) * (a - 2) / 2,
            -(a + 1) * a * (a - 2) / 2, (a + 1) * a * (a - 1) / 6)


def interp_cubic(f, dx_, dy_):
    N = f.shape[0]
    i0, j0, ax, ay = _cells(N, dx_, dy_)
    wx = lagrange4(ax)
    wy = lagrange4(ay)
    out = np.zeros_like(f)
    for q, wyq in zip(range(-1, 3), wy):
        row = np.zeros_like(f)
        jq = (j0 + q) % N
        for p, wxp in zip(range(-1, 3), wx):
            row = row + wxp * f[jq, (i0 + p) % N]
        out = out + wyq * row
    return out


class SLInterval:
    """One averaging interval of the semi-Lagrangian Strategy 1 on an oracle run.

    fields: names among zeta, h, u, v, q (f~^L of each); scheme: "euler" or
    "trapezoid"; interp: "linear" or "cubic".  step(n) advances the oracle's
    dynamics by n RK4 steps, applying the semi-Lagrangian update after each.
    """

    def __init__(self, oracle, fields=("zeta", "h", "u", "v"), scheme="trapezoid", interp="linear", n_steps=1):
        self.o = oracle
        self.fields = tuple(fields)
        self.scheme = scheme
        self.interp = interp_linear if interp == "linear" else interp_cubic
        self.n_steps = n_steps
        self.done = 0
        if oracle.model == "euler2d" and ("h" in self.fields or "q" in self.fields):
            raise ValueError("euler2d averages zeta, u and v only")
        N = oracle.N
        self.g = {f: np.zeros((N, N)) for f in self.fields}
        self.D = [np.zeros((N, N)), np.zeros((N, N))]
        self.f_prev = self._fields()

    def _velocity(self, ph):
        if self.o.model == "kinematic":
            N = self.o.N
            return np.full((N, N), self.o.adv[0]), np.full((N, N), self.o.adv[1])
        return ph["u"], ph["v"]

    def _fields(self):
        o = self.o
        u, v, h = o.fields()
        if o.model == "euler2d":
            return {"u": u, "v": v, "zeta": h}  # the third field is the vorticity
        zeta = o.phys(o.dx(o.vh) - o.dy(o.uh))
        return {"u": u, "v": v, "h": h, "zeta": zeta, "q": (o.f0 + zeta) / h}

    def step(self, n=1):
        for _ in range(n):
            if self.done >= self.n_steps:
                raise RuntimeError("interval complete")
            dt = self.o.dt
            s_n = self.done * dt
            self.o.step(1)
            ph = self._fields()
            ux, uy = self._velocity(ph)
            # departure point Y = X - dt u(X, t_{n+1}), as a displacement
            ddx, ddy = -dt * ux, -dt * uy
            for f in self.fields:
                gy = self.interp(self.g[f], ddx, ddy)
                if self.scheme == "euler":
                    self.g[f] = gy + dt * ph[f]
                else:
                    self.g[f] = gy + dt * (self.interp(self.f_prev[f], ddx, ddy) + ph[f]) / 2
            w = 0.0 if self.scheme == "euler" else 0.5
            self.D = [self.interp(self.D[0], ddx, ddy) + (s_n + w * dt) * dt * ux,
                      self.interp(self.D[1], ddx, ddy) + (s_n + w * dt) * dt * uy]
            self.f_prev = ph
            self.done += 1

    def end(self):
        if self.done != self.n_steps:
            raise RuntimeError("interval not complete")
        T = self.n_steps * self.o.dt
        N = self.o.N
        x = 2 * np.pi * np.arange(N) / N
        X, Y = np.meshgrid(x, x)
        out = {f: self.g[f] / T for f in self.fields}
        out["pos_x"] = X - self.D[0] / T
        out["pos_y"] = Y - self.D[1] / T
        return out
