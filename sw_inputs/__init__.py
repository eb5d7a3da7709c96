"""Seeded synthetic initial conditions for the rotating shallow-water runs.

This module only draws inputs: physical fields u, v, h on an N x N grid of the
doubly periodic domain [0, 2*pi)^2, row-major with y the slow index
(``a[j, i]`` is the value at x_i = i*dx, y_j = j*dx, dx = 2*pi/N).  It holds
none of the Lagrangian-mean method and none of the shallow-water time step; the
oracle and the CUDA library both receive the arrays it returns, unchanged.

Workload recipe (the paper's turbulence-plus-Poincare-wave experiment of
Sec. 4.2.1 needs an externally generated Navier-Stokes turbulence field that
is not available; this generator stands in for it):

* balanced part: streamfunction with energy spectrum E(k) ~ k^4 exp(-2 (k/6)^2),
  random phases, restricted to the 2/3-dealiased square box, geostrophically
  balanced height eta = (f0/c2) psi, scaled so that rms(zeta) = Ro * f0;
* wave part: a sum of linear Poincare modes over the lattice annulus
  k_lo <= |k| <= k_hi (one of each +-k pair), random phase and random branch
  of the dispersion relation omega = sqrt(f0^2 + c2 |k|^2), with the
  eigenvector of Sec. 4.2.1, Eq. (initial_wave) generalised to any k; the
  amplitude is set so that the wave energy 1/2 <|u|^2 + c2 eta^2> is a stated
  multiple of that of the balanced part.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "box_cutoff",
    "balanced_turbulence",
    "poincare_waves",
    "turbulence_plus_waves",
    "mode1_wave",
    "uniform_flow",
    "vortex_pair",
    "paper_sw_setup",
    "PAPER_SW",
    "random_smooth_field",
    "smooth_flow",
    "wave_frequency",
    "wave_period",
    "interval_steps",
    "Workload",
    "WORKLOADS",
]


def box_cutoff(N: int) -> int:
    """Largest retained integer wavenumber per axis under the 2/3 rule."""
    return (N - 1) // 3


def _wavenumbers(N: int):
    kx = np.arange(N // 2 + 1, dtype=np.float64)[None, :]
    ky = np.fft.fftfreq(N, d=1.0 / N)[:, None]
    return kx, ky


def _quad_energy(u, v, eta, c2):
    return 0.5 * float(np.mean(u * u + v * v + c2 * eta * eta))


def balanced_turbulence(N: int, ro: float, rng: np.random.Generator,
                        f0: float = 1.0, c2: float = 1.0, kpeak: float = 6.0):
    """Geostrophically balanced random flow; returns (u, v, eta).

    rms(zeta) = ro * f0 (the Rossby number read as rms vorticity over f0).
    """
    K = box_cutoff(N)
    kx, ky = _wavenumbers(N)
    kk = np.sqrt(kx * kx + ky * ky)
    inbox = (np.abs(kx) <= K) & (np.abs(ky) <= K) & (kk > 0)
    kks = np.where(kk > 0, kk, 1.0)
    spec = kks ** 4 * np.exp(-2.0 * (kks / kpeak) ** 2)
    amp = np.where(inbox, np.sqrt(spec / kks ** 3), 0.0)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=amp.shape)
    psi_hat = amp * np.exp(1j * phase)
    psi = np.fft.irfft2(psi_hat, s=(N, N))
    psi_hat = np.fft.rfft2(psi)
    u = np.fft.irfft2(-1j * ky * psi_hat, s=(N, N))
    v = np.fft.irfft2(1j * kx * psi_hat, s=(N, N))
    zeta = np.fft.irfft2(-(kx * kx + ky * ky) * psi_hat, s=(N, N))
    scale = ro * f0 / math.sqrt(float(np.mean(zeta * zeta)))
    psi *= scale
    u *= scale
    v *= scale
    eta = (f0 / c2) * psi
    return u, v, eta


def wave_frequency(k: float, f0: float = 1.0, c2: float = 1.0) -> float:
    """Poincare-wave frequency omega = sqrt(f0^2 + c2 k^2)."""
    return math.sqrt(f0 * f0 + c2 * k * k)


def wave_period(k: float, f0: float = 1.0, c2: float = 1.0) -> float:
    return 2.0 * math.pi / wave_frequency(k, f0, c2)


def interval_steps(periods: float, k_lo: float, dt: float,
                   f0: float = 1.0, c2: float = 1.0) -> int:
    """RK4 steps in an averaging interval of `periods` wave periods at |k| = k_lo."""
    return int(round(periods * wave_period(k_lo, f0, c2) / dt))


def _wave_modes(k_lo: float, k_hi: float):
    kmax = int(math.floor(k_hi))
    out = []
    for kx in range(0, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            if kx == 0 and ky <= 0:
                continue
            kk = math.hypot(kx, ky)
            if k_lo <= kk <= k_hi:
                out.append((kx, ky))
    return out


def poincare_waves(N: int, k_lo: float, k_hi: float, rng: np.random.Generator,
                   f0: float = 1.0, c2: float = 1.0, amplitude: float = 1.0):
    """Sum of linear Poincare modes with height amplitude `amplitude` each."""
    x = 2.0 * np.pi * np.arange(N) / N
    X = x[None, :]
    Y = x[:, None]
    u = np.zeros((N, N))
    v = np.zeros((N, N))
    eta = np.zeros((N, N))
    for kx, ky in _wave_modes(k_lo, k_hi):
        k2 = float(kx * kx + ky * ky)
        om = wave_frequency(math.sqrt(k2), f0, c2)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        sigma = 1.0 if rng.uniform() < 0.5 else -1.0
        th = kx * X + ky * Y + phi
        ct = np.cos(th)
        st = np.sin(th)
        A = amplitude
        eta += A * ct
        u += A * (kx * sigma * om * ct - f0 * ky * st) / k2
        v += A * (ky * sigma * om * ct + f0 * kx * st) / k2
    return u, v, eta


def turbulence_plus_waves(N: int, ro: float = 0.1, ratio: float = 1.0,
                          k_lo: float = 4.0, k_hi: float = 6.0, seed: int = 1001,
                          f0: float = 1.0, c2: float = 1.0):
    """Balanced turbulence plus Poincare waves; returns (u, v, h) with h = 1 + eta."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ub, vb, eb = balanced_turbulence(N, ro, rng, f0, c2)
    if ratio > 0.0:
        uw, vw, ew = poincare_waves(N, k_lo, k_hi, rng, f0, c2)
        ev = _quad_energy(ub, vb, eb, c2)
        ew0 = _quad_energy(uw, vw, ew, c2)
        s = math.sqrt(ratio * ev / ew0)
        ub = ub + s * uw
        vb = vb + s * vw
        eb = eb + s * ew
    return ub, vb, 1.0 + eb


def mode1_wave(N: int, a: float, f0: float, c2: float, t: float = 0.0):
    """Right-travelling mode-1 Poincare wave of Sec. 4.2.1, Eq. (initial_wave).

    With f0 = 1/Ro and c2 = 1/Fr^2 this is u' = a cos(x - w t),
    v' = a/(w Ro) sin(x - w t), h' = a/w cos(x - w t); returns (u, v, h=1+h').
    """
    om = wave_frequency(1.0, f0, c2)
    x = 2.0 * np.pi * np.arange(N) / N
    th = np.broadcast_to(x[None, :] - om * t, (N, N))
    return a * np.cos(th), (a * f0 / om) * np.sin(th), 1.0 + (a / om) * np.cos(th)


# Sec. 4.2.1's first shallow-water set-up: Ro = 0.1, Fr = 0.5, Re = 3840,
# mode-1 wave amplitude a = -1.8, forward Euler with dt = 1.25e-4 over
# T = 2.2 (3.6 wave periods, omega = 10.2), on a 256^2 grid.
PAPER_SW = {"ro": 0.1, "fr": 0.5, "re": 3840.0, "a": -1.8, "dt": 1.25e-4, "T": 2.2, "N": 256}


def paper_sw_setup(N: int = 256, seed: int = 1004, kpeak: float = 6.0, urms: float = 0.3):
    """Initial condition and parameters of Sec. 4.2.1's first example, with
    synthetic balanced turbulence standing in for the paper's Navier-Stokes
    field: geostrophic flow of rms velocity urms (in units of the paper's
    velocity scale U) in balance with its depth, plus the mode-1 Poincare
    wave of Eq. (initial_wave) at t = 0.  At the paper's Ro = 0.1, Fr = 0.5
    the balanced depth is (f0/c2) psi; with urms = 1 this synthetic field
    drives the depth negative during the interval (at any spectral peak from
    6 to 20), so the default is urms = 0.3, which keeps h above 0.4.
    Returns ((u, v, h), params) with params f0 = 1/Ro, c2 = 1/Fr^2, nu = 1/Re
    (Laplacian on momentum), dt, n_steps."""
    P = PAPER_SW
    f0, c2 = 1.0 / P["ro"], 1.0 / P["fr"] ** 2
    rng = np.random.Generator(np.random.PCG64(seed))
    ub, vb, eb = balanced_turbulence(N, 1.0, rng, f0, c2, kpeak=kpeak)
    s = urms / math.sqrt(float(np.mean(ub * ub + vb * vb)))  # balance is linear: rescale
    uw, vw, hw = mode1_wave(N, P["a"], f0, c2)
    params = {"f0": f0, "c2": c2, "nu": 1.0 / P["re"], "dt": P["dt"],
              "n_steps": int(round(P["T"] / P["dt"]))}
    return (s * ub + uw, s * vb + vw, 1.0 + s * eb + (hw - 1.0)), params


def vortex_pair(N: int):
    """Initial vorticity of Sec. 4.1's two-dimensional test flow: two
    like-signed Gaussian vortices that merge, exp(-(x - pi + 0.1)^2 - (y - pi +
    pi/3)^2) + exp(-(x - pi - 0.1)^2 - (y - pi - pi/3)^2) on [0, 2 pi)^2.
    Returns (u, v, zeta) with u = v = 0 placeholders (the two-dimensional
    Euler model derives the velocity from zeta)."""
    x = 2.0 * np.pi * np.arange(N) / N
    X, Y = np.meshgrid(x, x)
    zeta = (np.exp(-(X - np.pi + 0.1) ** 2 - (Y - np.pi + np.pi / 3) ** 2)
            + np.exp(-(X - np.pi - 0.1) ** 2 - (Y - np.pi - np.pi / 3) ** 2))
    return np.zeros((N, N)), np.zeros((N, N)), zeta


def uniform_flow(N: int, U0: float, V0: float, h0: float = 1.0):
    return (np.full((N, N), float(U0)), np.full((N, N), float(V0)),
            np.full((N, N), float(h0)))


def random_smooth_field(N: int, kmax: int, rng: np.random.Generator, amp: float = 1.0):
    """Real band-limited random field with |kx|, |ky| <= kmax, zero mean, rms = amp."""
    kx, ky = _wavenumbers(N)
    sel = (np.abs(kx) <= kmax) & (np.abs(ky) <= kmax) & ((kx != 0) | (ky != 0))
    c = (rng.standard_normal((N, N // 2 + 1))
         + 1j * rng.standard_normal((N, N // 2 + 1)))
    f = np.fft.irfft2(np.where(sel, c, 0.0), s=(N, N))
    return amp * f / math.sqrt(float(np.mean(f * f)))


def smooth_flow(N: int, kmax: int, seed: int, uamp: float = 0.05,
                eamp: float = 0.02):
    """Smooth random (u, v, h) with wavenumbers |kx|, |ky| <= kmax (tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = random_smooth_field(N, kmax, rng, uamp)
    v = random_smooth_field(N, kmax, rng, uamp)
    e = random_smooth_field(N, kmax, rng, eamp)
    return u, v, 1.0 + e


@dataclass(frozen=True)
class Workload:
    """A named synthetic workload (grid, generator and averaging set-up)."""

    name: str
    N: int
    ro: float
    ratio: float
    k_lo: float
    k_hi: float
    periods: float
    intervals: int
    dt: float = 5e-3
    f0: float = 1.0
    c2: float = 1.0
    alpha: float = 10.0  # hyperviscous damping rate at the cutoff wavenumber
    seed: int = 1001
    strategies: tuple = (1,)
    precisions: tuple = ("f64",)

    @property
    def n_steps(self) -> int:
        return interval_steps(self.periods, self.k_lo, self.dt, self.f0, self.c2)

    @property
    def nu8(self) -> float:
        K = box_cutoff(self.N)
        return self.alpha / float(K) ** 8

    def initial_condition(self):
        return turbulence_plus_waves(self.N, self.ro, self.ratio, self.k_lo,
                                     self.k_hi, self.seed, self.f0, self.c2)


WORKLOADS = {
    # 64^2, FP64, Strategy 1, one interval of 4 wave periods at |k| = 4.
    "plain-64": Workload("plain-64", 64, 0.1, 1.0, 4.0, 6.0, 4.0, 1, seed=1001),
    # 256^2, FP32 and FP64, Strategies 1 and 2, 4 intervals of 3.6 periods.
    "plain-256": Workload("plain-256", 256, 0.1, 1.0, 4.0, 6.0, 3.6, 4, seed=1002,
                          strategies=(1, 2), precisions=("f32", "f64")),
    # 1024^2 precision form: Ro 0.05, ratio 2, waves 8..12, one interval.
    "precision-1024": Workload("precision-1024", 1024, 0.05, 2.0, 8.0, 12.0, 3.6, 1,
                               seed=1003, precisions=("f32", "f64")),
}
