"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test fixes one part of the oracle by a closed form, a conservation law,
a symmetry, an independent library routine, a brute-force recount on a tiny
input, a physical law (Shan-Chen coexistence, Laplace), or a value printed in
a cited source (tests/golden/).  A dropped term, a wrong sign or index, or a
transposed operand anywhere in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2504_10539_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- generator

def test_splitmix64_published_vector():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) if l.strip() and l[0] != "#"]
    assert [O.splitmix64(1234567, k) for k in range(5)] == vals


def test_uniform01_range_and_moments():
    u = np.array([O.uniform01(7, k) for k in range(200000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 4e-3
    assert abs(u.var() - 1.0 / 12.0) < 2e-3


# ----------------------------------------------------------------------------- lattice

def test_velocity_set_isotropy():
    cx, cy, w = O.lattice_tables()
    assert sorted(zip(cx.tolist(), cy.tolist())) == sorted((a, b) for a in (-1, 0, 1) for b in (-1, 0, 1))
    # weight depends on |c|^2 only: 4/9, 1/9, 1/36
    for i in range(9):
        assert w[i] == {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}[cx[i] ** 2 + cy[i] ** 2]
    assert abs(w.sum() - 1) < 1e-15
    # second- and fourth-order isotropy of D2Q9 (c_s^2 = 1/3)
    assert abs((w * cx * cx).sum() - 1 / 3) < 1e-15 and abs((w * cx * cy).sum()) < 1e-15
    assert abs((w * cx ** 4).sum() - 1 / 3) < 1e-15 and abs((w * cx ** 2 * cy ** 2).sum() - 1 / 9) < 1e-15


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (2.3, 0.05, -0.02), (0.11, -0.1, 0.07)])
def test_equilibrium_moments(rho, ux, uy):
    cx, cy, _ = O.lattice_tables()
    feq = O.equilibrium(rho, ux, uy)
    assert abs(feq.sum() - rho) < 1e-14 * rho
    assert abs((feq * cx).sum() - rho * ux) < 1e-15 and abs((feq * cy).sum() - rho * uy) < 1e-15
    # second moment: rho c_s^2 delta + rho u u
    assert abs((feq * cx * cx).sum() - (rho / 3 + rho * ux * ux)) < 1e-14
    assert abs((feq * cy * cy).sum() - (rho / 3 + rho * uy * uy)) < 1e-14
    assert abs((feq * cx * cy).sum() - rho * ux * uy) < 1e-15


def test_stream_moves_each_direction_by_its_velocity():
    cx, cy, _ = O.lattice_tables()
    nx, ny = 5, 7
    for x0, y0 in [(2, 3), (0, 0), (4, 6)]:
        f = np.zeros((9, ny, nx))
        for i in range(9):
            f[i, y0, x0] = i + 1.0
        g = O.stream(f)
        for i in range(9):
            assert g[i, (y0 + cy[i]) % ny, (x0 + cx[i]) % nx] == i + 1.0
            assert np.count_nonzero(g[i]) == 1


# ----------------------------------------------------------------------------- pseudopotential and force

def test_psi_limits():
    # psi(0) = 0, psi'(0) = 1, psi(rho0 ln 2) = rho0/2, psi -> rho0
    assert O.psi(0.0, 1.0) == 0.0
    assert abs(O.psi(1e-8, 1.0) / 1e-8 - 1.0) < 1e-7
    for rho0 in (1.0, 2.0):
        assert abs(O.psi(rho0 * math.log(2.0), rho0) - rho0 / 2) < 1e-15
    assert abs(O.psi(60.0, 1.0) - 1.0) < 1e-15


def _force_bruteforce(psi, G):
    """F(x) = -G psi(x) sum over the 8 neighbour displacements d of w(|d|^2) psi(x+d) d,
    enumerating displacements directly (no velocity table)."""
    ny, nx = psi.shape
    wt = {1: 1.0 / 9.0, 2: 1.0 / 36.0}
    Fx = np.zeros_like(psi)
    Fy = np.zeros_like(psi)
    for y in range(ny):
        for x in range(nx):
            sx = sy = 0.0
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dx == 0 and dy == 0:
                        continue
                    p = psi[(y + dy) % ny, (x + dx) % nx]
                    sx += wt[dx * dx + dy * dy] * p * dx
                    sy += wt[dx * dx + dy * dy] * p * dy
            Fx[y, x] = -G * psi[y, x] * sx
            Fy[y, x] = -G * psi[y, x] * sy
    return Fx, Fy


def test_force_bruteforce_5x7():
    rng = np.random.default_rng(3)
    psi = rng.uniform(0.1, 1.0, size=(7, 5))
    Fx, Fy = O.sc_force(psi, -5.5)
    Bx, By = _force_bruteforce(psi, -5.5)
    assert np.abs(Fx - Bx).max() < 1e-15 and np.abs(Fy - By).max() < 1e-15


def test_force_sums_to_zero_on_periodic_lattice():
    rng = np.random.default_rng(4)
    psi = rng.uniform(0.0, 1.0, size=(33, 20))
    Fx, Fy = O.sc_force(psi, -5.0)
    scale = np.abs(Fx).sum() + np.abs(Fy).sum()
    assert abs(Fx.sum()) < 1e-13 * scale and abs(Fy.sum()) < 1e-13 * scale


def test_force_sine_closed_form():
    # psi = A + B sin(k x): sum_i w_i psi(x+c_i) c_ix = B cos(kx) sin(k) / 3, F_y = 0
    nx, ny, A, B, G = 24, 3, 0.6, 0.2, -5.5
    k = 2 * np.pi / nx
    x = np.arange(nx)
    psi = np.broadcast_to(A + B * np.sin(k * x), (ny, nx)).copy()
    Fx, Fy = O.sc_force(psi, G)
    expect = -G * psi[0] * B * np.cos(k * x) * np.sin(k) / 3.0
    assert np.abs(Fx - expect[None, :]).max() < 1e-15
    assert np.abs(Fy).max() < 1e-15


# ----------------------------------------------------------------------------- collision and step

@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0, 1.3])
def test_collision_conserves_mass_and_adds_force_to_momentum(tau):
    # With u_eq = u + tau F / rho, BGK changes each cell's momentum by exactly F.
    cx, cy, _ = O.lattice_tables()
    rng = np.random.default_rng(5)
    f = wl.random_populations(6, 5, seed=6)
    Fx = rng.uniform(-0.02, 0.02, size=(5, 6))
    Fy = rng.uniform(-0.02, 0.02, size=(5, 6))
    fp = O.collide(f, Fx, Fy, tau)
    assert np.abs(fp.sum(0) - f.sum(0)).max() < 1e-15
    djx = np.tensordot(cx, fp - f, axes=1)
    djy = np.tensordot(cy, fp - f, axes=1)
    assert np.abs(djx - Fx).max() < 1e-15 and np.abs(djy - Fy).max() < 1e-15


def test_collision_fixed_point_at_equilibrium():
    nx, ny = 4, 3
    f = np.zeros((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            f[:, y, x] = O.equilibrium(0.5 + 0.1 * x, 0.01 * y, -0.02)
    fp = O.collide(f, np.zeros((ny, nx)), np.zeros((ny, nx)), 0.7)
    assert np.abs(fp - f).max() < 1e-16


def test_collision_relaxation_rate():
    # Without force, the non-equilibrium part is multiplied by (1 - 1/tau).
    f = wl.random_populations(3, 2, seed=8)
    rho = f.sum(0)
    cx, cy, _ = O.lattice_tables()
    ux = np.tensordot(cx, f, axes=1) / rho
    uy = np.tensordot(cy, f, axes=1) / rho
    feq = np.stack([O.equilibrium(rho[y, x], ux[y, x], uy[y, x]) for y in range(2) for x in range(3)], 1).reshape(9, 2, 3)
    for tau in (0.7, 1.0, 1.6):
        fp = O.collide(f, np.zeros((2, 3)), np.zeros((2, 3)), tau)
        assert np.abs((fp - feq) - (1 - 1 / tau) * (f - feq)).max() < 1e-15


def test_step_conserves_mass_and_total_momentum():
    cx, cy, _ = O.lattice_tables()
    f = wl.random_populations(13, 11, seed=9, lo=0.05, hi=0.4)
    M0 = O.mass(f)
    J0 = (np.tensordot(cx, f, axes=1).sum(), np.tensordot(cy, f, axes=1).sum())
    O.step(f, 50, -5.5, 0.9)
    assert abs(O.mass(f) - M0) < 1e-13 * M0
    J1 = (np.tensordot(cx, f, axes=1).sum(), np.tensordot(cy, f, axes=1).sum())
    assert abs(J1[0] - J0[0]) < 1e-12 and abs(J1[1] - J0[1]) < 1e-12


def test_step_uniform_flow_is_stationary():
    # Uniform density (zero force) moving at constant u: f^eq(rho, u) is a fixed point.
    nx, ny = 6, 4
    fe = O.equilibrium(0.8, 0.03, -0.01)
    f = np.repeat(fe[:, None, None], ny * nx, axis=1).reshape(9, ny, nx).copy()
    g = f.copy()
    O.step(g, 5, -5.5, 0.8)
    assert np.abs(g - f).max() < 1e-15


def _coexistence(G, rho0=1.0):
    """Shan-Chen mechanical-stability coexistence for p = rho/3 + G psi^2/6:
    p(rho_g) = p(rho_l) and int_{rho_g}^{rho_l} (p0 - p) psi'/psi^2 drho = 0."""
    from scipy.integrate import quad
    from scipy.optimize import fsolve
    psi = lambda r: rho0 * (1 - np.exp(-r / rho0))
    dpsi = lambda r: np.exp(-r / rho0)
    p = lambda r: r / 3 + G * psi(r) ** 2 / 6

    def eqs(v):
        rg, rl = v
        p0 = p(rg)
        return [p(rl) - p(rg), quad(lambda r: (p0 - p(r)) * dpsi(r) / psi(r) ** 2, rg, rl)[0]]

    return fsolve(eqs, [0.1, 2.3])


@pytest.mark.parametrize("G", [-5.5, -6.0])
def test_flat_interface_reaches_shan_chen_coexistence(G):
    rg, rl = _coexistence(G)
    nx, ny = 4, 64
    y = np.arange(ny)
    prof = 0.15 + 1.85 * 0.5 * (np.tanh((y - 16) / 2.0) - np.tanh((y - 48) / 2.0))
    rho = np.broadcast_to(prof[:, None], (ny, nx)).copy()
    f = O.init_equilibrium(rho)
    O.step(f, 6000, G, 1.0)
    r = O.density(f)
    # x-invariant exactly, plateaus at the coexistence densities
    assert np.array_equal(r, np.broadcast_to(r[:, :1], r.shape))
    assert abs(r[32, 0] - rl) < 0.02 * rl
    assert abs(r[0, 0] - rg) < 0.02 * rg
    # the bulk pressure used by the Laplace estimator is equal in both phases
    pl, pg = O.pressure(r[32, 0], G), O.pressure(r[0, 0], G)
    assert abs(pl - pg) < 0.02 * abs(pg)
    # physical velocity u + F/(2 rho), averaged over two steps, vanishes
    cx, cy, _ = O.lattice_tables()
    us = []
    for _ in range(2):
        rr = O.density(f)
        Fx, Fy = O.sc_force(np.vectorize(O.psi)(rr), G)
        us.append((np.tensordot(cy, f, axes=1) + 0.5 * Fy) / rr)
        O.step(f, 1, G, 1.0)
    assert np.abs(0.5 * (us[0] + us[1])).max() < 1e-3


def test_laplace_pressure_jump_linear_in_inverse_radius():
    n, G = 64, -5.5
    pts = []
    for R in (8, 10, 12, 16):
        f = O.init_equilibrium(O.init_rho(n, n, [(n / 2, n / 2, R)], 2.0, 0.15, 2.0, 0.0, 1))
        O.step(f, 3000, G, 1.0)
        L = O.laplace(O.density(f), n / 2, n / 2, 2.0, G)
        pts.append((1.0 / L["R_eq"], L["dP"]))
    x, y = np.array(pts).T
    A = np.vstack([x, np.ones_like(x)]).T
    (sigma, b), *_ = np.linalg.lstsq(A, y, rcond=None)
    r2 = 1 - ((y - A @ [sigma, b]) ** 2).sum() / ((y - y.mean()) ** 2).sum()
    assert r2 >= 0.99 and sigma > 0
    assert abs(b) < 0.1 * y.min()


def test_laplace_top_hat_closed_form():
    """A top-hat droplet (rho = a on the cells within R0 of the centre, b elsewhere; the centre
    off the grid and near a corner, so the disk wraps across both periodic edges): the
    equimolar radius is sqrt(n_disk / pi) exactly (the excess mass is n_disk (a - b)), and the
    inner and outer regions hold a and b alone, so rho_in = a, rho_out = b, p_in = p(a),
    p_out = p(b) exactly, on both iterations."""
    nx, ny, a, b, R0, G = 53, 47, 2.1, 0.12, 9.3, -5.5
    cx, cy = 50.6, 3.2
    dx = np.abs(np.arange(nx) - cx)
    dx = np.minimum(dx, nx - dx)
    dy = np.abs(np.arange(ny) - cy)
    dy = np.minimum(dy, ny - dy)
    d = np.hypot(dx[None, :], dy[:, None])
    rho = np.where(d < R0, a, b)
    L = O.laplace(rho, cx, cy, 1.0, G)
    assert L["R_eq"] == pytest.approx(np.sqrt((d < R0).sum() / np.pi), rel=1e-14)
    assert L["rho_in"] == pytest.approx(a, rel=1e-15) and L["rho_out"] == pytest.approx(b, rel=1e-15)
    assert L["p_in"] == pytest.approx(O.pressure(a, G), rel=1e-14)
    assert L["p_out"] == pytest.approx(O.pressure(b, G), rel=1e-14)


def test_laplace_regions_by_brute_force():
    """A radially varying droplet on a small non-square lattice, centred across the periodic
    corner: the estimator's two iterations recomputed cell by cell (pure-Python loops over the
    minimum-image distance, inner region d < R_eq / 2, outer region d > R_eq + 4 width, starting
    from rho_in = max rho, rho_out = min rho) give the oracle's six numbers.  A region radius or
    boundary off by a cell, a missed periodic image or one iteration fewer fails this."""
    nx, ny, G, width = 29, 23, -5.3, 1.5
    cx, cy = 27.4, 1.8
    rng = np.random.default_rng(3)
    rho = np.empty((ny, nx))
    for y in range(ny):
        for x in range(nx):
            ddx = min(abs(x - cx), nx - abs(x - cx))
            ddy = min(abs(y - cy), ny - abs(y - cy))
            d = (ddx * ddx + ddy * ddy) ** 0.5
            rho[y, x] = 0.2 + 0.9 * (1.0 - np.tanh((d - 6.0) / width)) + 0.05 * np.cos(d)
    rho += 0.01 * rng.random((ny, nx))
    rin, rout = rho.max(), rho.min()
    for _ in range(2):
        excess = sum(rho[y, x] - rout for y in range(ny) for x in range(nx))
        req = (excess / (np.pi * (rin - rout))) ** 0.5
        inner, outer = [], []
        for y in range(ny):
            for x in range(nx):
                ddx = min(abs(x - cx), nx - abs(x - cx))
                ddy = min(abs(y - cy), ny - abs(y - cy))
                d = (ddx * ddx + ddy * ddy) ** 0.5
                if d < 0.5 * req:
                    inner.append(rho[y, x])
                if d > req + 4.0 * width:
                    outer.append(rho[y, x])
        rin, rout = sum(inner) / len(inner), sum(outer) / len(outer)
        pin = sum(O.pressure(r, G) for r in inner) / len(inner)
        pout = sum(O.pressure(r, G) for r in outer) / len(outer)
    L = O.laplace(rho, cx, cy, width, G)
    for key, val in (("R_eq", req), ("rho_in", rin), ("rho_out", rout), ("p_in", pin), ("p_out", pout),
                     ("dP", pin - pout)):
        assert L[key] == pytest.approx(val, rel=1e-12, abs=1e-14), key


def test_centred_droplet_keeps_d4_symmetry():
    n = 64
    f = O.init_equilibrium(O.init_rho(n, n, [(32.0, 32.0, 12.0)], 2.0, 0.15, 2.0, 0.0, 1))
    O.step(f, 200, -5.5, 1.0)
    r = O.density(f)
    idx = (-np.arange(n)) % n  # x -> 64 - x reflection about the centre column 32
    assert np.abs(r - r[:, idx]).max() < 1e-12
    assert np.abs(r - r[idx, :]).max() < 1e-12
    assert np.abs(r - r.T).max() < 1e-12


def test_step_is_independent_of_thread_count():
    f0 = wl.random_populations(37, 29, seed=10, lo=0.02, hi=0.3)
    nt = O.num_threads()
    outs = []
    for t in (1, max(2, nt)):
        O.set_num_threads(t)
        f = f0.copy()
        O.step(f, 7, -5.5, 1.0)
        outs.append(f)
    O.set_num_threads(nt)
    assert np.array_equal(outs[0], outs[1])


# ----------------------------------------------------------------------------- initial state

def test_init_profile_closed_form():
    n, R, W = 64, 12.0, 2.0
    rho = O.init_rho(n, n, [(32.0, 32.0, R)], 2.0, 0.15, W, 0.0, 1)
    assert abs(rho[32, 32] - (0.15 + 1.85 * 0.5 * (1 - math.tanh(-R / W)))) < 1e-15
    assert abs(rho[32, 44] - (2.0 + 0.15) / 2) < 1e-15       # distance exactly R
    assert abs(rho[32, 20] - (2.0 + 0.15) / 2) < 1e-15
    # minimum image: column 0 is 32 away, same as column 64 would be
    assert abs(rho[32, 0] - (0.15 + 1.85 * 0.5 * (1 - math.tanh((32 - R) / W)))) < 1e-15
    # overlapping droplets take the max, not the sum
    two = O.init_rho(n, n, [(20.0, 32.0, 8.0), (30.0, 32.0, 8.0)], 2.0, 0.15, W, 0.0, 1)
    assert two.max() <= 2.0 + 1e-15


def test_init_noise_is_counter_based():
    nx, ny, amp, seed = 8, 5, 0.01, 42
    base = O.init_rho(nx, ny, [], 2.0, 0.15, 2.0, 0.0, seed)
    noisy = O.init_rho(nx, ny, [], 2.0, 0.15, 2.0, amp, seed)
    assert np.all(base == 0.15)
    for y in range(ny):
        for x in range(nx):
            u = O.uniform01(seed, y * nx + x)
            assert noisy[y, x] == 0.15 + amp * (2 * u - 1)
    f = O.init_equilibrium(noisy)
    _, _, w = O.lattice_tables()
    assert np.array_equal(f, w[:, None, None] * noisy[None])


# ----------------------------------------------------------------------------- metrics (Eqs. 9-16)

@pytest.mark.parametrize("n", [16, 24, 64])
def test_metrics_sine_closed_forms(n):
    a, b, ny = 1.0, 0.7, 8
    rho = wl.sine_rho(n, ny, a, b)
    m = O.metrics_rho(rho)
    s = math.sin(2 * math.pi / n)
    x = np.arange(n)
    N = n * ny
    assert abs(m["G_max"] - b * s) < 1e-14
    assert abs(m["E_int"] - N * b * b * s * s / 2) < 1e-12 * N
    assert abs(m["W_eff"] - np.abs(np.cos(2 * np.pi * x / n)).mean()) < 1e-13
    assert abs(m["delta_rho"] - 2 * b) < 1e-14
    assert abs(m["mass"] - a * N) < 1e-12 * N
    g = np.abs(b * np.cos(2 * np.pi * x / n) * s)
    assert m["count"] == ny * int((g > 0.01).sum()) and abs(m["W"] - m["count"] / N) < 1e-16


def test_metrics_bruteforce_4x4():
    rng = np.random.default_rng(12)
    rho = rng.uniform(0.1, 2.3, size=(4, 4))
    m = O.metrics_rho(rho, threshold=0.3)
    gs = []
    for y in range(4):
        for x in range(4):
            gx = (rho[y][(x + 1) % 4] - rho[y][(x - 1) % 4]) / 2
            gy = (rho[(y + 1) % 4][x] - rho[(y - 1) % 4][x]) / 2
            gs.append(math.hypot(gx, gy))
    assert abs(m["G_max"] - max(gs)) < 1e-15
    assert abs(m["sum_g"] - sum(gs)) < 1e-14
    assert abs(m["E_int"] - sum(g * g for g in gs)) < 1e-14
    assert abs(m["W_eff"] - sum(gs) / (max(gs) * 16)) < 1e-15
    assert m["count"] == sum(g > 0.3 for g in gs)
    assert abs(m["delta_rho"] - (rho.max() - rho.min())) < 1e-15


def test_metrics_threshold_is_strict():
    """Eq. 9 counts the cells whose gradient magnitude is above the threshold: a triangular
    density wave of step 1/4 (exact in binary) has |grad rho| = 1/4 exactly in 6 of every 8
    columns and 0 in the other 2, so a threshold of 1/4 counts none of them and one just below
    counts all six; G_max, W_eff and E_int follow exactly."""
    row = np.array([1.0, 1.25, 1.5, 1.75, 2.0, 1.75, 1.5, 1.25])
    ny = 3
    rho = np.tile(row, (ny, 1))
    at = O.metrics_rho(rho, threshold=0.25)
    below = O.metrics_rho(rho, threshold=0.25 - 2 ** -20)
    assert at["count"] == 0 and at["W"] == 0.0
    assert below["count"] == 6 * ny and below["W"] == 0.75
    assert at["G_max"] == 0.25 and at["W_eff"] == 0.75 and at["E_int"] == 6 * ny * 0.0625
    assert at["delta_rho"] == 1.0 and at["mass"] == ny * row.sum()


def test_metrics_uniform_field_has_no_interface():
    m = O.metrics_rho(np.full((5, 6), 1.3))
    assert m["G_max"] == 0.0 and m["W_eff"] == 0.0 and m["E_int"] == 0.0 and m["W"] == 0.0


def test_paper_tables_fix_lattice_units():
    """Tables I/II are consistent only if |grad rho| is in lattice units (dx = 1):
    E_int = sum g^2 <= N G_max^2 and (sum g)^2 <= N sum g^2 with sum g = W_eff G_max N
    bound N from both sides, and a 100x100 lattice (r = nx/6 ~ 16.7) lies inside
    both rows' ranges; with dx = 1/nx the bound E_int <= N G_max^2 fails."""
    t = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))
    for row in ("pure_lbm", "pinn_lbm"):
        r = t[row]
        n_lo = r["E_int"] / r["G_max"] ** 2                           # from sum g^2 <= N G_max^2
        n_hi = r["E_int"] / (r["W_eff"] ** 2 * r["G_max"] ** 2)       # from (sum g)^2 <= N sum g^2
        assert n_lo <= 100 * 100 <= n_hi
        # with dx = 1/nx the energy carries dx^2 = 1/N while g scales by nx: bound fails
        assert r["E_int"] > r["G_max"] ** 2


# ----------------------------------------------------------------------------- network (Sec. III-B)

def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(13)
    v = np.concatenate([rng.normal(0, 3, 20000), rng.uniform(-1, 1, 20000) * 1e-3,
                        [1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 0.0, 1.0]])
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    got = np.array([O.round_bf16(float(np.float32(x))) for x in v])
    assert np.array_equal(got, ref)
    assert O.round_bf16(1 + 2 ** -8) == 1.0                    # tie to even
    assert O.round_bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6         # tie to even (up)


def test_mlp_zero_weights_give_output_bias():
    blob = np.zeros(wl.mlp_blob_size(), dtype=np.float32)
    blob[-3:] = [0.5, -0.25, 0.125]
    for mode in (O.MLP_F64, O.MLP_BF16):
        assert np.array_equal(O.mlp_forward(blob, 0.3, -0.7, mode), [0.5, -0.25, 0.125])


def test_mlp_is_odd_without_biases():
    blob = wl.mlp_weights(21, zero_bias=True)
    for xy in [(0.3, -0.7), (-0.99, 0.01), (0.5, 0.5)]:
        a = O.mlp_forward(blob, *xy)
        b = O.mlp_forward(blob, -xy[0], -xy[1])
        assert np.array_equal(a, -b)


def _offsets(dims=wl.MLP_DIMS):
    offs, o = [], 0
    for l in range(len(dims) - 1):
        offs.append((o, o + dims[l + 1] * dims[l]))
        o += dims[l + 1] * dims[l] + dims[l + 1]
    return offs


def test_mlp_single_path_composition():
    """Weights with one non-zero path  x -> h1[3] -> h2[70] -> h3[5] -> h4[40] -> out[1]
    give out = w5 tanh(w4 tanh(w3 tanh(w2 tanh(w1 x + b1) + b2) + b3) + b4) + b5;
    a transposed W[out][in], a missing or extra tanh, or a wrong layer order breaks it."""
    dims = wl.MLP_DIMS
    blob = np.zeros(wl.mlp_blob_size(), dtype=np.float32)
    offs = _offsets()
    path = [(3, 1), (70, 3), (5, 70), (40, 5), (1, 40)]   # (out, in) per layer; input 1 = y
    ws = [0.75, -1.25, 0.5, 2.0, -0.625]
    bs = [0.125, 0.25, -0.5, 0.0625, 0.375]
    for l, ((o, i), w, b) in enumerate(zip(path, ws, bs)):
        wo, bo = offs[l]
        blob[wo + o * dims[l] + i] = w
        blob[bo + o] = b
    y = -0.3
    h = y
    for l in range(4):
        h = math.tanh(ws[l] * h + bs[l])
    expect = ws[4] * h + bs[4]
    out = O.mlp_forward(blob, 0.9, y, O.MLP_F64)
    assert abs(out[1] - expect) < 1e-15
    assert out[0] == 0.0 and out[2] == 0.0


def _bf16_bits(v):
    """Nearest BF16 value (ties to even) by integer rounding of the FP64 bit pattern: 45 of the
    52 mantissa bits dropped (BF16 keeps 7), the carry running into the exponent; normal
    numbers only.  An independent route to the rounding the oracle does with frexp/nearbyint."""
    import struct
    b = struct.unpack("<Q", struct.pack("<d", v))[0]
    drop = 45
    lower, half = b & ((1 << drop) - 1), 1 << (drop - 1)
    b >>= drop
    if lower > half or (lower == half and (b & 1)):
        b += 1
    return struct.unpack("<d", struct.pack("<Q", b << drop))[0]


def test_mlp_bf16_emulation_single_path_closed_form():
    """The tensor-core form rounds exactly these values to BF16: the activations h1, h2, h3 that
    feed the MMA layers 2-4 and the weights of those layers; layer 1, the biases, h4 and
    layer 5 stay exact.  One non-zero path gives a closed form.  Its biases in layers 1-3 cancel
    the path's input down to four rounding steps of it, so that one rounding more or less
    anywhere (an activation, a weight, a bias) changes a later BF16 activation and with it the
    output by more than 1e-12, while the oracle must match the closed form to the last bit."""
    dims = wl.MLP_DIMS
    offs = _offsets()
    path = [(3, 1), (70, 3), (5, 70), (40, 5), (1, 40)]
    R = _bf16_bits
    ws = [float(np.float32(w)) for w in (0.7071, -1.2345, 0.55555, 1.9999, -0.6180)]
    y = -0.3
    bs, h = [], y
    for l in range(3):
        w = R(ws[l]) if l >= 1 else ws[l]
        bs.append(float(np.float32(-w * h + 4 * abs(w * h) * 2 ** -9)))
        h = R(math.tanh(w * h + bs[l]))
    bs += [float(np.float32(0.0789)), float(np.float32(0.3691))]
    blob = np.zeros(wl.mlp_blob_size(), dtype=np.float32)
    for l, ((o, i), w, b) in enumerate(zip(path, ws, bs)):
        wo, bo = offs[l]
        blob[wo + o * dims[l] + i] = w
        blob[bo + o] = b

    def closed_form(round_h=(1, 1, 1, 0), round_w=(0, 1, 1, 1, 0), round_b=False):
        h = y
        for l in range(4):
            w = R(ws[l]) if round_w[l] else ws[l]
            b = R(bs[l]) if round_b else bs[l]
            h = math.tanh(w * h + b)
            if round_h[l]:
                h = R(h)
        w5 = R(ws[4]) if round_w[4] else ws[4]
        return w5 * h + bs[4]

    expect = closed_form()
    out = O.mlp_forward(blob, 0.9, y, O.MLP_BF16)
    assert out[1] == expect
    assert out[0] == 0.0 and out[2] == 0.0
    # the pin's power: every other reading of what is rounded gives a visibly different output
    alternatives = [closed_form(round_h=(0, 1, 1, 0)), closed_form(round_h=(1, 0, 1, 0)),
                    closed_form(round_h=(1, 1, 0, 0)), closed_form(round_h=(1, 1, 1, 1)),
                    closed_form(round_w=(1, 1, 1, 1, 0)), closed_form(round_w=(0, 0, 1, 1, 0)),
                    closed_form(round_w=(0, 1, 0, 1, 0)), closed_form(round_w=(0, 1, 1, 0, 0)),
                    closed_form(round_w=(0, 1, 1, 1, 1)), closed_form(round_b=True)]
    assert min(abs(a - expect) for a in alternatives) > 1e-12


# ----------------------------------------------------------------------------- stencil-input network
# A variant that is not in the paper: the network also reads the density of the cell and its
# 8 neighbours (inputs 2..10, velocity order c_0..c_8, periodic).

STENCIL_DIMS = (11, 64, 128, 128, 64, 3)


def test_stencil_network_blob_size_and_zero_weights():
    n = wl.mlp_blob_size(STENCIL_DIMS)
    assert O.mlp_blob_size(11) == n == wl.mlp_blob_size() + 64 * 9
    blob = np.zeros(n, dtype=np.float32)
    blob[-3:] = [0.5, -0.25, 0.125]
    out = O.mlp_forward_n(blob, np.arange(11) * 0.1, O.MLP_F64)
    assert np.array_equal(out, [0.5, -0.25, 0.125])


def test_stencil_network_gathers_each_neighbour_periodically():
    """A single path from input 2 + i to output 0 gives tanh^4 of the density of neighbour
    c_i, which numpy's roll of the density field fixes independently of the oracle's gather."""
    nx, ny = 7, 5
    rho = np.random.default_rng(31).uniform(0.1, 2.0, (ny, nx))
    cx, cy, _ = O.lattice_tables()
    offs = _offsets(STENCIL_DIMS)
    for i in range(9):
        blob = np.zeros(wl.mlp_blob_size(STENCIL_DIMS), dtype=np.float32)
        blob[offs[0][0] + 0 * 11 + 2 + i] = 1.0
        for l in range(1, 5):
            blob[offs[l][0]] = 1.0          # W_l[0][0]
        out = O.mlp_field(blob, nx, ny, O.MLP_F64, n_in=11, rho=rho)
        neighbour = np.roll(rho, shift=(-int(cy[i]), -int(cx[i])), axis=(0, 1))
        assert np.allclose(out[0], np.tanh(np.tanh(np.tanh(np.tanh(neighbour)))), rtol=0, atol=1e-15), i
        assert np.all(out[1] == 0.0) and np.all(out[2] == 0.0)


def test_stencil_network_is_odd_without_biases():
    blob = wl.mlp_weights(24, dims=STENCIL_DIMS, zero_bias=True)
    rng = np.random.default_rng(25)
    for _ in range(20):
        v = rng.uniform(-2, 2, 11)
        assert np.allclose(O.mlp_forward_n(blob, -v), -O.mlp_forward_n(blob, v), rtol=0, atol=1e-14)


def test_stencil_network_coupled_run_keeps_mass_and_momentum():
    n = 32
    f = O.init_equilibrium(O.init_rho(n, n, [(16.0, 16.0, 7.0)], 2.0, 0.15, 2.0, 0.01, 5))
    M0 = O.mass(f)
    P0 = np.array(O.momentum(f)).sum(axis=(1, 2))
    blob = wl.mlp_weights(26, dims=STENCIL_DIMS)
    assert O.run(f, 100, -5.5, 1.0, K=50, blob=blob, M0=M0, n_in=11) == 0
    assert abs(O.mass(f) - M0) < 1e-12 * M0
    assert np.abs(np.array(O.momentum(f)).sum(axis=(1, 2)) - P0).max() < 1e-10


def test_mlp_bf16_emulation_close_to_fp64():
    blob = wl.mlp_weights(22)
    rng = np.random.default_rng(23)
    for _ in range(50):
        x, y = rng.uniform(-1, 1, 2)
        a = O.mlp_forward(blob, x, y, O.MLP_F64)
        b = O.mlp_forward(blob, x, y, O.MLP_BF16)
        # each BF16 rounding is <= 2^-9 relative; three rounded activation layers and
        # three rounded weight layers, damped by the ~1/sqrt(3) gain per layer
        assert np.abs(a - b).max() < 2e-2
        assert np.abs(a - b).max() > 0.0


# ----------------------------------------------------------------------------- correction (Sec. II-C)

def _droplet_state(n=32, steps=100):
    f = O.init_equilibrium(O.init_rho(n, n, [(n / 2, n / 2, n / 5)], 2.0, 0.15, 2.0, 0.01, 3))
    O.step(f, steps, -5.5, 1.0)
    return f


def test_correction_projects_mass_and_keeps_momentum():
    cx, cy, _ = O.lattice_tables()
    f = _droplet_state()
    M0 = O.mass(f) * (1 + 1e-4)          # also pulls the mass to a different target
    J0 = (np.tensordot(cx, f, axes=1).sum(), np.tensordot(cy, f, axes=1).sum())
    g = O.grad_mag(O.density(f))
    f_before = f.copy()
    st = O.correct(f, wl.mlp_weights(31), 0.1, 0.05, M0)
    assert st == 0
    assert abs(O.mass(f) - M0) < 1e-13 * M0
    J1 = (np.tensordot(cx, f, axes=1).sum(), np.tensordot(cy, f, axes=1).sum())
    assert abs(J1[0] - J0[0]) < 1e-13 and abs(J1[1] - J0[1]) < 1e-13
    # cells without gradient are untouched bit for bit; others changed
    flat = g == 0
    assert np.array_equal(f[:, flat], f_before[:, flat])
    assert np.abs(f - f_before).max() > 1e-6


def test_correction_keeps_non_equilibrium_part():
    cx, cy, _ = O.lattice_tables()
    f = _droplet_state()
    f0 = f.copy()
    assert O.correct(f, wl.mlp_weights(32), 0.2, 0.05, O.mass(f)) == 0

    def neq(h):
        rho = h.sum(0)
        ux, uy = np.tensordot(cx, h, axes=1) / rho, np.tensordot(cy, h, axes=1) / rho
        ny, nx = rho.shape
        fe = np.zeros_like(h)
        for yy in range(ny):
            for xx in range(nx):
                fe[:, yy, xx] = O.equilibrium(rho[yy, xx], ux[yy, xx], uy[yy, xx])
        return h - fe

    assert np.abs(neq(f) - neq(f0)).max() < 1e-13


def test_correction_with_zero_gain_is_identity():
    f = _droplet_state()
    f0 = f.copy()
    assert O.correct(f, wl.mlp_weights(33), 0.0, 0.0, O.mass(f)) == 0
    assert np.array_equal(f, f0)


def test_correction_moves_interface_density_toward_network():
    # M = M0 and beta_rho in (0,1]: every interface cell moves toward rho^ up to the
    # (small) projection term; on aggregate the m-weighted misfit shrinks.
    f = _droplet_state()
    blob = wl.mlp_weights(34)
    n = f.shape[1]
    rho = O.density(f)
    g = O.grad_mag(rho)
    m = g / g.max()
    out = O.mlp_field(blob, n, n)
    before = (m * (rho - out[0]) ** 2).sum()
    assert O.correct(f, blob, 0.5, 0.0, O.mass(f)) == 0
    after = (m * (O.density(f) - out[0]) ** 2).sum()
    assert after < before


def test_correction_closed_form_on_a_sine_field_at_rest():
    """A density wave rho = a + b sin(theta), theta = 2 pi x / nx, at rest, with a network whose
    output is its bias (rho^, u^) everywhere.  Eq. 16 gives g = |b cos(theta) sin(2 pi / nx)|,
    so the mask m = g / G_max is |cos(theta)|; the sums of m sin(theta) and m^2 sin(theta) over
    a period vanish, so the m-weighted projections remove exactly (rho^ - a) and a u^:
    rho' = rho - beta_rho m b sin(theta) (whatever rho^ is), j' = beta_u m u^ (rho' - a), and every
    cell ends at the equilibrium of (rho', j' / rho').  A mask not normalised by G_max, a
    projection weighted otherwise, or a dropped gain fails it."""
    nx, ny, a, b = 16, 4, 1.0, 0.3
    f = O.init_equilibrium(wl.sine_rho(nx, ny, a, b))
    f0 = f.copy()
    blob = np.zeros(wl.mlp_blob_size(), dtype=np.float32)
    blob[-3:] = [0.9, 0.05, -0.03]
    rh, ux, uy = (float(v) for v in blob[-3:])
    beta, beta_u = 0.3, 0.2
    assert O.correct(f, blob, beta, beta_u, O.mass(f0), O.MLP_F64) == 0
    th = 2 * np.pi * np.arange(nx) / nx
    m = np.abs(np.cos(th))
    rp = a + b * np.sin(th) - beta * m * b * np.sin(th)
    for x in range(nx):
        fe = O.equilibrium(rp[x], beta_u * m[x] * ux * (rp[x] - a) / rp[x],
                           beta_u * m[x] * uy * (rp[x] - a) / rp[x])
        for y in range(ny):
            assert np.abs(f[:, y, x] - fe).max() < 1e-15, (x, y)
    # the closed form is not the identity, and rho^ does not enter it
    assert np.abs(f - f0).max() > 1e-3
    blob[-3] = 1.7
    f2 = f0.copy()
    assert O.correct(f2, blob, beta, beta_u, O.mass(f0), O.MLP_F64) == 0
    assert np.abs(f2 - f).max() < 1e-15


def test_correction_rejects_nonphysical_result():
    f = _droplet_state()
    f0 = f.copy()
    # rho^ = 200 * tanh(tanh(tanh(tanh(2 x^)))) spans about +-100 across the domain; the
    # projection removes only the m-weighted mean, so interface cells on the left go negative
    dims = wl.MLP_DIMS
    blob = np.zeros(wl.mlp_blob_size(), dtype=np.float32)
    offs = _offsets()
    for l, w in enumerate([2.0, 1.0, 1.0, 1.0, 200.0]):
        blob[offs[l][0]] = w              # W_l[0][0]
    assert O.correct(f, blob, 1.0, 0.0, O.mass(f)) == -4
    assert np.array_equal(f, f0)


def test_run_applies_correction_after_every_kth_step():
    blob = wl.mlp_weights(35)
    f0 = _droplet_state(n=16, steps=20)
    M0 = O.mass(f0)
    a = f0.copy()
    assert O.run(a, 10, -5.5, 1.0, K=5, blob=blob, M0=M0) == 0
    b = f0.copy()
    for _ in range(2):
        O.step(b, 5, -5.5, 1.0)
        assert O.correct(b, blob, 0.1, 0.01, M0) == 0
    assert np.array_equal(a, b)
    c = f0.copy()
    assert O.run(c, 4, -5.5, 1.0, K=5, blob=blob, M0=M0) == 0
    d = f0.copy()
    O.step(d, 4, -5.5, 1.0)
    assert np.array_equal(c, d)
