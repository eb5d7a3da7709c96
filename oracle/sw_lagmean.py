"""FP64 CPU oracle: pseudospectral rotating shallow water + Lagrangian-mean PDEs.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only tests/, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of bench.py may use it.  It shares no code with the
CUDA library (no kernels, headers, tables or helpers); the two meet only
through the seeded input arrays of ``sw_inputs``.

Plain and slow by design: numpy FP64, full-grid real FFTs (``numpy.fft.rfft2``
and ``irfft2`` as library primitives), no fusion, no blocking.  Each step cites
the passage of Kafiabad & Vanneste, "Computing Lagrangian means" (JFM 2023,
arXiv 2208.02682) it follows.

What is computed (one averaging interval [tau, tau+T], Sec. 2, Eq. (ave)):

* (model "euler2d") two-dimensional incompressible inviscid flow, the test
  flow of Sec. 4.1: the vorticity zeta is carried in the depth slot and
  obeys d_t zeta + div(u zeta) = 0, with the velocity slaved to it through
  the streamfunction (lap psi = zeta, u = -d_y psi, v = d_x psi); the mean of
  zeta, which no periodic velocity carries, is kept and conserved;
* the shallow-water dynamics, Sec. 4.2, Eq. (sw_eqs_dimless), written with
  f0 = 1/Ro and c2 = g H = 1/Fr^2, for the depth perturbation eta = h - 1
  (the mean depth is the scale H, so h = 1 + eta; carrying eta instead of h
  keeps its digits: averages of h are eta averages plus 1), in
  vector-invariant form
  u_t = (f0 + zeta) v - d_x(c2 h + |u|^2/2), v_t = -(f0 + zeta) u - d_y(...),
  h_t = -div(h u), zeta = d_x v - d_y u (Sec. 4.2.1 prints d_x u for the second
  term; read as d_y u); the Laplacian viscosity is replaced by a hyperviscosity
  -nu8 |k|^8 acting on u, v and h;
* Strategy 1, Sec. 4.1, Eq. (gtilde-evol): (d_t + u.grad) g = f for
  g = (t - tau) f~, with f~^L = g(tau+T)/T (Sec. 4.1);
  mean positions from Eq. (Xi-1evol) through the periodic displacement
  D = (t - tau)(x - Xi^{-1}), which obeys (d_t + u.grad) D = (t - tau) u (this
  follows from Eq. (Xi-1evol) by the same substitution as Eq. (gtilde-evol);
  the paper does not write it), so Xi^{-1}(x, tau+T) = x - D/T;
* Strategy 2, Sec. 4.2, Eqs. (xi_evol), (barf_xi): xi = Xi - x and
  g = (t - tau) fbar, advected by w = xi/(t - tau), forced by u and f evaluated
  at x + xi by bilinear interpolation (Sec. 4.2.1); at t = tau, where xi = 0,
  w takes its limit u/2 (the partial mean position is x + u s/2 + O(s^2));
* Eulerian means, Eq. (ave): E = int f dt, mean E/T;
* time stepping: classical RK4 with a diagonal integrating factor
  exp(-nu |k|^8 t); optionally the paper's own steppers, Heun (Sec. 4.1) and
  forward Euler (Sec. 4.2.1), with the same integrating factor, and the
  paper's Laplacian viscosity (-nu |k|^2 on u and v only, as in Eq.
  sw_momentum_dimless) in place of the hyperviscosity;
  the Lagrangian-mean fields share the RK stages with the dynamics (on-the-fly
  computation, Sec. 5).

Spectral convention: F_hat = rfft2(F) / N^2 on the kx >= 0 half-plane, kept only
inside the square 2/3 box |kx|, |ky| <= K = floor((N-1)/3); physical values are
irfft2(F_hat) * N^2 (the imaginary part on the kx = 0 column is discarded by
the real inverse transform).

Parity pins (tests/test_oracle_*.py): closed forms for a uniform inertial
oscillation, uniform advection and the Stokes drift of a small Poincare wave,
linear dispersion, exact mass conservation, fourth-order energy drift, PV
material conservation, agreement of Strategies 1 and 2, brute-force particle
tracking with trajectory averaging (``oracle.particles``), and Strategy 2's
uniform-flow closed form under every stepper (which pins the s = 0 limit
under forward Euler).  Parity unpinned: in the "xi_first" scheme, the time
level of gbar's advecting velocity (xi_{m+1}/s_{m+1}); the scheme itself is
pinned by its uniform-flow closed form and its first-order convergence, but
other consistent levels would pass those too.
"""
from __future__ import annotations

import math

import numpy as np

LM_FIELDS = ("zeta", "h", "u", "v", "q")


class SWOracle:
    """Shallow-water state plus (optionally) one open averaging interval."""

    _stage_hook = None  # test hook: called with each RK stage state

    def __init__(self, N, dt, u, v, h, f0=1.0, c2=1.0, nu8=0.0, lm_nu8=None,
                 model="sw", adv=(0.0, 0.0), stepper="rk4", visc="hyper8"):
        if N % 2 or N < 8:
            raise ValueError("N must be even and >= 8")
        self.N = int(N)
        self.dt = float(dt)
        self.f0 = float(f0)
        self.c2 = float(c2)
        self.nu8 = float(nu8)
        self.lm_nu8 = float(nu8 if lm_nu8 is None else lm_nu8)
        if model not in ("sw", "kinematic", "euler2d"):
            raise ValueError(model)
        self.model = model
        self.adv = (float(adv[0]), float(adv[1]))
        if stepper not in ("rk4", "heun", "euler") or visc not in ("hyper8", "laplace"):
            raise ValueError((stepper, visc))
        self.stepper = stepper
        # nu8 is the coefficient of the viscous term -nu8 |k|^(2p): p = 4
        # (hyperviscosity) or p = 1 (the paper's Laplacian, Eq. sw_momentum_dimless)
        self.visc_p = 4 if visc == "hyper8" else 1
        N = self.N
        self.K = (N - 1) // 3
        self.kx = np.arange(N // 2 + 1, dtype=np.float64)[None, :]
        self.ky = np.fft.fftfreq(N, d=1.0 / N)[:, None]
        self.mask = ((self.kx <= self.K) & (np.abs(self.ky) <= self.K)).astype(np.float64)
        self.k2 = self.kx ** 2 + self.ky ** 2
        self.x = 2.0 * np.pi * np.arange(N) / N
        self.t = 0.0
        self.uh = self.spec(np.asarray(u, dtype=np.float64))
        self.vh = self.spec(np.asarray(v, dtype=np.float64))
        if model == "euler2d":
            # the third field is the vorticity; u and v follow from it
            self.hh = self.spec(np.asarray(h, dtype=np.float64))
            self.uh, self.vh = self.velocity_from_vorticity(self.hh)
        else:
            # depth perturbation eta = h - 1 (spectral)
            self.hh = self.spec(np.asarray(h, dtype=np.float64))
            self.hh[0, 0] -= 1.0
        self.lm = None

    # -- transforms --------------------------------------------------------
    def spec(self, f):
        """Physical -> spectral, truncated to the 2/3 box."""
        return np.fft.rfft2(f) / float(self.N * self.N) * self.mask

    def phys(self, F):
        """Spectral -> physical values on the N x N grid."""
        return np.fft.irfft2(F, s=(self.N, self.N)) * float(self.N * self.N)

    def velocity_from_vorticity(self, zh):
        """Streamfunction psi with lap psi = zeta (zero mean): psi_hat =
        -zeta_hat/|k|^2, u = -d_y psi, v = d_x psi, i.e. u_hat = i ky zeta_hat/|k|^2
        and v_hat = -i kx zeta_hat/|k|^2 (zero at k = 0)."""
        inv = np.zeros_like(self.k2)
        nz = self.k2 > 0
        inv[nz] = 1.0 / self.k2[nz]
        return 1j * self.ky * zh * inv, -1j * self.kx * zh * inv

    def dx(self, F):
        return 1j * self.kx * F

    def dy(self, F):
        return 1j * self.ky * F

    # -- bilinear interpolation at x + xi (Sec. 4.2.1) ---------------------
    def interp(self, f, xi_x, xi_y):
        """Bilinear interpolation of the grid field f at (x_i + xi_x, y_j + xi_y).

        Displacements are converted to cell units d = xi/dx; the cell index is
        i + floor(d) (periodic) and the weight d - floor(d).
        """
        N = self.N
        inv_dx = N / (2.0 * np.pi)
        dxc = xi_x * inv_dx
        dyc = xi_y * inv_dx
        fx = np.floor(dxc)
        fy = np.floor(dyc)
        ax = dxc - fx
        ay = dyc - fy
        I = np.arange(N)[None, :]
        J = np.arange(N)[:, None]
        i0 = (I + fx.astype(np.int64)) % N
        j0 = (J + fy.astype(np.int64)) % N
        i1 = (i0 + 1) % N
        j1 = (j0 + 1) % N
        return ((1 - ax) * (1 - ay) * f[j0, i0] + ax * (1 - ay) * f[j0, i1]
                + (1 - ax) * ay * f[j1, i0] + ax * ay * f[j1, i1])

    # -- interval bookkeeping ---------------------------------------------
    def lmean_begin(self, strategy, fields=("zeta", "h", "u", "v"), pos=True,
                    eulerian=True, n_steps=1, scheme="coupled"):
        """Open an averaging interval at tau = current time (Sec. 2: each
        interval [tau_n, tau_n + T] is computed independently).  Initial
        conditions g = D = 0 (Strategy 1, g = (t - tau) f~ at t = tau) and
        xi = g = 0 (Strategy 2, Xi(x, tau) = x).

        scheme "coupled": the mean fields share the dynamics' stages.
        scheme "xi_first": the paper's discretisation of Eqs. (xi_evol),
        (barf_xi) in Sec. 4.2 / 4.2.1 (Strategy 2, forward Euler): the mean
        equations step by 2 dt every other dynamics step, xi first, then gbar
        with the updated xi (see _euler_step)."""
        if strategy not in (1, 2):
            raise ValueError("strategy must be 1 or 2")
        if scheme not in ("coupled", "xi_first"):
            raise ValueError(scheme)
        if scheme == "xi_first" and (strategy != 2 or self.stepper != "euler" or int(n_steps) % 2):
            raise ValueError("xi_first needs Strategy 2, forward Euler and an even n_steps")
        fields = tuple(f for f in LM_FIELDS if f in fields)
        if self.model == "euler2d" and ("h" in fields or "q" in fields):
            raise ValueError("euler2d averages zeta, u and v only")
        if strategy == 2:
            pos = True  # xi is part of the Strategy-2 dynamics
        z = lambda: np.zeros_like(self.uh)
        self.lm = dict(strategy=strategy, fields=fields, pos=bool(pos),
                       eulerian=bool(eulerian), n_steps=int(n_steps), done=0, scheme=scheme,
                       G={f: z() for f in fields},
                       P=[z(), z()] if pos else None,
                       E={f: z() for f in fields} if eulerian else None)

    # -- right-hand side ---------------------------------------------------
    def _rhs(self, st, s):
        """Right-hand sides of all evolved fields at interval time s = t - tau."""
        if self._stage_hook is not None:
            self._stage_hook(st)
        uh, vh, hh = st["sw"]  # hh: depth perturbation eta (euler2d: vorticity)
        if self.model == "euler2d":
            uh, vh = self.velocity_from_vorticity(hh)
            zh = hh
        else:
            zh = self.dx(vh) - self.dy(uh)
        u = self.phys(uh)
        v = self.phys(vh)
        eta = self.phys(hh)
        zeta = self.phys(zh)
        out = {}
        if self.model == "euler2d":
            # vorticity equation of Sec. 4.1's test flow: d_t zeta = -div(u zeta);
            # u and v take no tendency of their own (they follow zeta)
            Nh = -self.dx(self.spec(u * zeta)) - self.dy(self.spec(v * zeta))
            Nu, Nv = np.zeros_like(uh), np.zeros_like(vh)
            au, av = u, v
            uh_adv, vh_adv = uh, vh
        elif self.model == "sw":
            # Eq. (sw_momentum_dimless), (sw_mass_dimless), vector-invariant form;
            # grad h = grad eta and h u = u + eta u.
            B = self.c2 * hh + self.spec(0.5 * (u * u + v * v))
            Nu = self.f0 * vh + self.spec(zeta * v) - self.dx(B)
            Nv = -self.f0 * uh - self.spec(zeta * u) - self.dy(B)
            Nh = -self.dx(self.spec(u + eta * u)) - self.dy(self.spec(v + eta * v))
            au, av = u, v
            uh_adv, vh_adv = uh, vh
        else:
            # Passive advection of the whole state by a constant velocity.
            cx, cy = self.adv
            ikc = 1j * (self.kx * cx + self.ky * cy)
            Nu, Nv, Nh = -ikc * uh, -ikc * vh, -ikc * hh
            au = np.full((self.N, self.N), cx)
            av = np.full((self.N, self.N), cy)
            uh_adv, vh_adv = self.spec(au), self.spec(av)
        out["sw"] = (Nu, Nv, Nh)
        lm = self.lm
        if lm is None:
            return out
        need_q = "q" in lm["fields"]
        # the average of h is carried as the average of eta (the constant
        # 1 contributes exactly s = t - tau to g and E; added at the end)
        fphys = {"zeta": zeta, "h": eta, "u": u, "v": v}
        fhat = {"zeta": zh, "h": hh, "u": uh, "v": vh}
        if need_q:
            fphys["q"] = (self.f0 + zeta) / (1.0 + eta)  # potential vorticity, Sec. 4.2.1
            fhat["q"] = self.spec(fphys["q"])
        if lm["strategy"] == 1:
            # Eq. (gtilde-evol): d_t g = f - u.grad g.
            out["G"] = {}
            for f in lm["fields"]:
                G = st["G"][f]
                adv = au * self.phys(self.dx(G)) + av * self.phys(self.dy(G))
                out["G"][f] = fhat[f] - self.spec(adv)
            if lm["pos"]:
                # d_t D = s u - u.grad D (from Eq. (Xi-1evol)).
                Dx, Dy = st["P"]
                adx = au * self.phys(self.dx(Dx)) + av * self.phys(self.dy(Dx))
                ady = au * self.phys(self.dx(Dy)) + av * self.phys(self.dy(Dy))
                out["P"] = [s * uh_adv - self.spec(adx), s * vh_adv - self.spec(ady)]
        else:
            # Eqs. (xi_evol), (barf_xi) with w = xi/s (s > 0) or u/2 (s = 0).
            Xx, Xy = st["P"]
            xi_x = self.phys(Xx)
            xi_y = self.phys(Xy)
            if s > 0.0:
                wx = xi_x / s
                wy = xi_y / s
            else:
                wx = 0.5 * au
                wy = 0.5 * av
            uI = self.interp(au, xi_x, xi_y)
            vI = self.interp(av, xi_x, xi_y)
            wgx = wx * self.phys(self.dx(Xx)) + wy * self.phys(self.dy(Xx))
            wgy = wx * self.phys(self.dx(Xy)) + wy * self.phys(self.dy(Xy))
            out["P"] = [self.spec(uI - wx - wgx), self.spec(vI - wy - wgy)]
            if lm["scheme"] == "xi_first":
                # gbar steps with the updated xi, at its own time s + dt
                wx, wy = xi_x / (s + self.dt), xi_y / (s + self.dt)
            out["G"] = {}
            for f in lm["fields"]:
                G = st["G"][f]
                fI = self.interp(fphys[f], xi_x, xi_y)
                wg = wx * self.phys(self.dx(G)) + wy * self.phys(self.dy(G))
                out["G"][f] = self.spec(fI - wg)
        if lm["eulerian"]:
            out["E"] = {f: fhat[f] for f in lm["fields"]}  # Eq. (ave)
        return out

    # -- RK4 with integrating factor ---------------------------------------
    def _state(self):
        st = {"sw": (self.uh, self.vh, self.hh)}
        if self.lm is not None:
            st["G"] = self.lm["G"]
            if self.lm["P"] is not None:
                st["P"] = self.lm["P"]
            if self.lm["E"] is not None:
                st["E"] = self.lm["E"]
        return st

    def _factors(self):
        """Half-step integrating factors exp(L dt/2), L = -nu |k|^(2p), per
        field of (u, v, h): the Laplacian of Eq. (sw_momentum_dimless) acts on
        the momentum only (the mass equation, Eq. sw_mass_dimless, has no
        viscous term); the hyperviscosity acts on u, v and h."""
        k8 = self.k2 ** self.visc_p
        e_sw = np.exp(-self.nu8 * k8 * self.dt * 0.5)
        e_h = np.ones_like(k8) if self.visc_p == 1 else e_sw
        e_lm = np.exp(-self.lm_nu8 * k8 * self.dt * 0.5)
        return {"sw": (e_sw, e_sw, e_h), "G": e_lm, "P": e_lm, "E": np.ones_like(k8)}

    @staticmethod
    def _map(fn, *trees):
        """Apply fn leafwise over matching state trees."""
        t0 = trees[0]
        if isinstance(t0, dict):
            return {k: SWOracle._map(fn, *[t[k] for t in trees]) for k in t0}
        if isinstance(t0, (list, tuple)):
            return type(t0)(SWOracle._map(fn, *[t[i] for t in trees]) for i in range(len(t0)))
        return fn(*trees)

    def _efac_tree(self, st, fac):
        """Factor tree matching the state: a tuple of factors is per field, a
        single factor applies to every field of its group."""
        return {k: (fac[k] if isinstance(fac[k], tuple) else self._map(lambda _x, f=fac[k]: f, v))
                for k, v in st.items()}

    def _step(self, s0):
        {"rk4": self._rk4_step, "heun": self._heun_step, "euler": self._euler_step}[self.stepper](s0)

    def _heun_step(self, s0):
        """Heun's method (the paper's stepper in Sec. 4.1) with the integrating
        factor: a = N(y_n), y1 = E^2 (y_n + dt a), b = N(y1, t + dt),
        y_{n+1} = E^2 y_n + dt/2 (E^2 a + b)."""
        dt = self.dt
        y = self._state()
        E = self._efac_tree(y, self._factors())
        m = self._map
        a = self._rhs(y, s0)
        y1 = m(lambda yy, aa, e: e * e * (yy + dt * aa), y, a, E)
        b = self._rhs(y1, s0 + dt)
        yn = m(lambda yy, aa, bb, e: e * e * yy + (dt / 2.0) * (e * e * aa + bb), y, a, b, E)
        self._commit(yn)

    def _euler_step(self, s0):
        """Forward Euler (the paper's stepper in Sec. 4.2.1) with the
        integrating factor: y_{n+1} = E^2 (y_n + dt N(y_n)).

        With the "xi_first" scheme (Sec. 4.2: xi is updated first and the
        updated xi used for gbar; Sec. 4.2.1: the mean equations' step is
        twice the dynamics' step), step 2m advances xi by 2 dt from the flow
        at t_2m, xi_{m+1} = E^4 (xi_m + 2 dt R_xi(xi_m, t_2m)), and step
        2m + 1 advances gbar with the updated xi at its time s_{m+1} = (2m +
        2) dt and the flow at t_2m+1, gbar_{m+1} = E^4 (gbar_m + 2 dt
        R_g(gbar_m, xi_{m+1})); the Eulerian accumulators step with dt.
        The time level of gbar's advecting velocity xi_{m+1}/s_{m+1} is a
        reading (the paper does not state it) that no pin distinguishes:
        other consistent choices converge at the same first order."""
        dt = self.dt
        y = self._state()
        E = self._efac_tree(y, self._factors())
        a = self._rhs(y, s0)
        yn = self._map(lambda yy, aa, e: e * e * (yy + dt * aa), y, a, E)
        lm = self.lm
        if lm is not None and lm["scheme"] == "xi_first":
            step2 = lambda yy, aa, e: (e * e) * (e * e) * (yy + 2.0 * dt * aa)
            keep = lambda yy, aa, e: yy
            even = lm["done"] % 2 == 0
            yn["P"] = self._map(step2 if even else keep, y["P"], a["P"], E["P"])
            yn["G"] = self._map(keep if even else step2, y["G"], a["G"], E["G"])
        self._commit(yn)

    def _commit(self, yn):
        self.uh, self.vh, self.hh = yn["sw"]
        if self.model == "euler2d":
            self.uh, self.vh = self.velocity_from_vorticity(self.hh)
        if self.lm is not None:
            self.lm["G"] = yn["G"]
            if "P" in yn:
                self.lm["P"] = yn["P"]
            if "E" in yn:
                self.lm["E"] = yn["E"]
        self.t += self.dt

    def _rk4_step(self, s0):
        dt = self.dt
        y = self._state()
        E = self._efac_tree(y, self._factors())
        m = self._map
        a = self._rhs(y, s0)
        y1 = m(lambda yy, aa, e: e * (yy + 0.5 * dt * aa), y, a, E)
        b = self._rhs(y1, s0 + 0.5 * dt)
        y2 = m(lambda yy, bb, e: e * yy + 0.5 * dt * bb, y, b, E)
        c = self._rhs(y2, s0 + 0.5 * dt)
        y3 = m(lambda yy, cc, e: e * e * yy + dt * e * cc, y, c, E)
        d = self._rhs(y3, s0 + dt)
        yn = m(lambda yy, aa, bb, cc, dd, e:
               e * e * yy + (dt / 6.0) * (e * e * aa + 2.0 * e * (bb + cc) + dd),
               y, a, b, c, d, E)
        self.uh, self.vh, self.hh = yn["sw"]
        if self.model == "euler2d":
            self.uh, self.vh = self.velocity_from_vorticity(self.hh)
        if self.lm is not None:
            self.lm["G"] = yn["G"]
            if "P" in yn:
                self.lm["P"] = yn["P"]
            if "E" in yn:
                self.lm["E"] = yn["E"]
        self.t += dt

    def step(self, nsteps):
        """Advance the dynamics only (no interval open)."""
        if self.lm is not None:
            raise RuntimeError("an averaging interval is open")
        for _ in range(int(nsteps)):
            self._step(0.0)

    def lmean_step(self, nsteps):
        lm = self.lm
        if lm is None:
            raise RuntimeError("no averaging interval open")
        if lm["done"] + nsteps > lm["n_steps"]:
            raise ValueError("more steps than remain in the interval")
        for _ in range(int(nsteps)):
            # s = t - tau counted in whole steps (never accumulated).
            self._step(lm["done"] * self.dt)
            lm["done"] += 1

    def lmean_end(self):
        """Close the interval; total means as physical FP64 fields.

        Strategy 1: f~^L = g/T and Xi^{-1}(x, tau+T) = x - D/T (Sec. 4.1).
        Strategy 2: fbar^L = g/T and Xi(x, tau+T) = x + xi (Sec. 3.2, 4.2).
        Eulerian: E/T (Eq. (ave)).
        """
        lm = self.lm
        if lm is None or lm["done"] != lm["n_steps"]:
            raise RuntimeError("interval not complete")
        T = lm["n_steps"] * self.dt
        out = {}
        one = {"h": 1.0}
        for f in lm["fields"]:
            out[f] = self.phys(lm["G"][f]) / T + one.get(f, 0.0)
        X = self.x[None, :] + 0.0 * self.x[:, None]
        Y = self.x[:, None] + 0.0 * self.x[None, :]
        if lm["pos"]:
            if lm["strategy"] == 1:
                dxp = self.phys(lm["P"][0]) / T
                dyp = self.phys(lm["P"][1]) / T
                out["pos_x"] = X - dxp
                out["pos_y"] = Y - dyp
            else:
                out["pos_x"] = X + self.phys(lm["P"][0])
                out["pos_y"] = Y + self.phys(lm["P"][1])
        if lm["eulerian"]:
            for f in lm["fields"]:
                out["E_" + f] = self.phys(lm["E"][f]) / T + one.get(f, 0.0)
        self.lm = None
        return out

    # -- diagnostics -------------------------------------------------------
    def fields(self):
        """Physical u, v, h (euler2d: u, v, zeta)."""
        if self.model == "euler2d":
            return self.phys(self.uh), self.phys(self.vh), self.phys(self.hh)
        return self.phys(self.uh), self.phys(self.vh), 1.0 + self.phys(self.hh)

    def diag(self):
        """Domain means: mass <h>, energy <h|u|^2/2 + c2 h^2/2>, potential
        enstrophy <h q^2/2> with q = (f0 + zeta)/h.  euler2d: mean vorticity,
        kinetic energy <|u|^2/2> and enstrophy <zeta^2/2>."""
        if self.model == "euler2d":
            u, v, zeta = self.fields()
            return (float(np.mean(zeta)), float(np.mean(0.5 * (u * u + v * v))),
                    float(np.mean(0.5 * zeta * zeta)))
        u, v, h = self.fields()
        zeta = self.phys(self.dx(self.vh) - self.dy(self.uh))
        q = (self.f0 + zeta) / h
        return (float(np.mean(h)),
                float(np.mean(0.5 * h * (u * u + v * v) + 0.5 * self.c2 * h * h)),
                float(np.mean(0.5 * h * q * q)))

    def spectral_state(self):
        """Copy of the spectral SW state (u, v, eta; kx >= 0 half-plane arrays)."""
        return self.uh.copy(), self.vh.copy(), self.hh.copy()


def rel_l2(a, b):
    """||a - b||_2 / ||b||_2 over the grid."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = math.sqrt(float(np.sum(b * b)))
    return math.sqrt(float(np.sum((a - b) ** 2))) / (nb if nb > 0 else 1.0)
