"""Pins of the training oracle (oracle/train.py, Eqs. 3-8) against facts that do not come
from it: the C oracle's own forward pass, central differences, symbolic derivatives
(sympy), PyTorch autograd and PyTorch's Adam.  Each part of the training step (tangent
forward, the three loss terms, the output-level derivatives, the reverse pass, the
optimizer) fails at least one of them if a term, sign or index is wrong.
"""
import numpy as np
import pytest

import oracle as O
import oracle.train as T
from paper_2504_10539_gb300 import workloads as wl

G, RHO0 = -5.5, 1.0


def small_problem(nx=12, ny=10, seed=0):
    rng = np.random.default_rng(seed)
    N = nx * ny
    t = np.stack([1.0 + 0.5 * rng.random(N), 0.1 * rng.standard_normal(N), 0.1 * rng.standard_normal(N)], axis=1)
    iface = rng.random(N) > 0.5
    return t, iface


def blob64(seed):
    return np.asarray(wl.mlp_weights(seed), dtype=np.float32).astype(np.float64)


# ----------------------------------------------------------------------------- forward

def test_value_channel_equals_c_oracle_network():
    blob = wl.mlp_weights(21)
    nx, ny = 9, 7
    (o, _, _), _ = T.forward(T.unpack(blob), T.cell_inputs(nx, ny))
    ref = O.mlp_field(blob, nx, ny, O.MLP_F64)           # independent C forward pass
    assert np.abs(o - ref.reshape(3, -1).T).max() < 1e-13


def test_tangents_equal_central_differences_of_the_c_network():
    blob = wl.mlp_weights(22)
    X = np.array([[0.3, -0.2], [-0.9, 0.7], [0.0, 0.0]])
    (_, ox, oy), _ = T.forward(T.unpack(blob), X)
    h = 1e-5
    for i, (x, y) in enumerate(X):
        dx = (O.mlp_forward(blob, x + h, y) - O.mlp_forward(blob, x - h, y)) / (2 * h)
        dy = (O.mlp_forward(blob, x, y + h) - O.mlp_forward(blob, x, y - h)) / (2 * h)
        assert np.abs(ox[i] - dx).max() < 1e-8 and np.abs(oy[i] - dy).max() < 1e-8


# ----------------------------------------------------------------------------- loss terms

def test_residuals_match_symbolic_derivatives():
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    rho = 1.0 + 0.3 * sp.sin(0.7 * x) * sp.cos(0.4 * y)
    u = 0.1 * sp.cos(0.5 * x + 0.2 * y)
    v = 0.05 * sp.sin(0.3 * x) * sp.exp(0.1 * y)
    psi = RHO0 * (1 - sp.exp(-rho / RHO0))
    p = rho / 3 + G * psi ** 2 / 6
    rc = sp.diff(rho * u, x) + sp.diff(rho * v, y)
    rmx = sp.diff(rho * u * u, x) + sp.diff(rho * u * v, y) + sp.diff(p, x)
    rmy = sp.diff(rho * u * v, x) + sp.diff(rho * v * v, y) + sp.diff(p, y)
    fields = [rho, u, v, sp.diff(rho, x), sp.diff(rho, y), sp.diff(u, x), sp.diff(u, y), sp.diff(v, x), sp.diff(v, y)]
    for pt in [(0.3, 1.1), (-2.0, 0.4), (5.0, -3.0)]:
        sub = {x: pt[0], y: pt[1]}
        vals = [float(f.subs(sub)) for f in fields]
        got = T.residuals(*vals, G, RHO0)
        want = [float(e.subs(sub)) for e in (rc, rmx, rmy)]
        assert np.allclose(got, want, rtol=1e-12, atol=1e-14)


def test_uniform_fields_have_zero_residual_and_rest_state_balances_pressure():
    # uniform rho and u: every derivative vanishes
    z = np.zeros(4)
    rc, rmx, rmy = T.residuals(np.full(4, 1.3), np.full(4, 0.1), np.full(4, -0.2), z, z, z, z, z, z, G, RHO0)
    assert np.abs(rc).max() == 0 and np.abs(rmx).max() == 0 and np.abs(rmy).max() == 0
    # at rest the momentum residual is grad p = p'(rho) grad rho, with p' the slope of the C oracle's pressure
    r, gx, gy = 0.8, 0.05, -0.02
    h = 1e-6
    slope = (O.pressure(r + h, G) - O.pressure(r - h, G)) / (2 * h)
    rc, rmx, rmy = T.residuals(np.array([r]), z[:1], z[:1], np.array([gx]), np.array([gy]), z[:1], z[:1], z[:1], z[:1],
                               G, RHO0)
    assert rc[0] == 0 and abs(rmx[0] - slope * gx) < 1e-10 and abs(rmy[0] - slope * gy) < 1e-10


def test_pressure_slope_is_the_derivative_of_the_c_oracle_pressure():
    h = 1e-5
    for r in (0.1, 0.7, 2.0):
        P, dP = T.pressure_slope(np.array(r), G, RHO0)
        assert abs(P - (O.pressure(r + h, G) - O.pressure(r - h, G)) / (2 * h)) < 1e-9
        P2 = T.pressure_slope(np.array(r + h), G, RHO0)[0]
        P1 = T.pressure_slope(np.array(r - h), G, RHO0)[0]
        assert abs(dP - (P2 - P1) / (2 * h)) < 1e-8


def test_interface_term_rewards_steep_interfaces_up_to_its_minimum():
    # one interface cell whose network density rises along x: q = |grad rho_N|^2
    nx = ny = 1
    hp = T.TrainParams(lambda_phys=0.0, alpha1=1.0, alpha2=2.0)
    vals = []
    for gq in (0.0, 0.25, 0.5, 0.75):
        o = np.array([[1.0, 0.0, 0.0]])
        ox = np.array([[gq / 2.0, 0.0, 0.0]])           # d/dx = (2/nx) d/dx^ with nx = 1
        L, terms, *_ = T.losses((o, ox, np.zeros((1, 3))), o.copy(), np.array([True]), nx, ny, G, RHO0, hp)
        q = gq * gq
        assert terms[2] == pytest.approx(-1.0 * q + 2.0 * q * q, abs=1e-15)
        vals.append(terms[2])
    # decreasing up to q* = alpha1 / (2 alpha2) = 0.25 (|grad| = 0.5), rising after
    assert vals[0] > vals[1] > vals[2] < vals[3]
    # a cell outside the interface set contributes nothing
    o = np.array([[1.0, 0.0, 0.0]])
    L, terms, *_ = T.losses((o, np.ones((1, 3)), np.zeros((1, 3))), o, np.array([False]), 1, 1, G, RHO0, hp)
    assert terms[2] == 0.0


@pytest.mark.parametrize("which", ["data", "phys", "int"])
def test_output_level_derivatives_equal_central_differences(which):
    rng = np.random.default_rng(3)
    nx, ny = 5, 4
    N = nx * ny
    o = np.stack([1.0 + 0.5 * rng.random(N), 0.2 * rng.standard_normal(N), 0.2 * rng.standard_normal(N)], axis=1)
    ox, oy = 0.3 * rng.standard_normal((N, 3)), 0.3 * rng.standard_normal((N, 3))
    t, iface = small_problem(nx, ny, 4)
    hp = {"data": T.TrainParams(lambda_phys=0.0, lambda_int=0.0),
          "phys": T.TrainParams(lambda_phys=1.0, lambda_int=0.0),
          "int": T.TrainParams(lambda_phys=0.0, lambda_int=1.0, alpha2=3.0)}[which]
    if which != "data":
        t = o.copy()                                       # the data term is flat here
    L, _, g_o, g_ox, g_oy = T.losses((o, ox, oy), t, iface, nx, ny, G, RHO0, hp)
    h = 1e-6
    for arr, g in ((o, g_o), (ox, g_ox), (oy, g_oy)):
        for idx in [(0, 0), (3, 1), (7, 2), (N - 1, 0), (11, 1)]:
            a0 = arr[idx]
            arr[idx] = a0 + h
            Lp = T.losses((o, ox, oy), t, iface, nx, ny, G, RHO0, hp)[0]
            arr[idx] = a0 - h
            Lm = T.losses((o, ox, oy), t, iface, nx, ny, G, RHO0, hp)[0]
            arr[idx] = a0
            assert abs((Lp - Lm) / (2 * h) - g[idx]) < 1e-8 * max(1.0, abs(g).max())


# ----------------------------------------------------------------------------- reverse pass

def torch_gradient(blob, nx, ny, t, iface, hp):
    """The same loss built from torch operations and differentiated by autograd."""
    torch = pytest.importorskip("torch")
    dt = torch.float64
    layers = [(torch.tensor(W, dtype=dt, requires_grad=True), torch.tensor(b, dtype=dt, requires_grad=True))
              for W, b in T.unpack(blob)]
    X = torch.tensor(T.cell_inputs(nx, ny), dtype=dt, requires_grad=True)
    a = X
    for l, (W, b) in enumerate(layers):
        a = a @ W.T + b
        if l < 4:
            a = torch.tanh(a)
    o = a
    d = [torch.autograd.grad(o[:, k].sum(), X, create_graph=True)[0] for k in range(3)]   # [N, 2] each
    sx, sy = 2.0 / nx, 2.0 / ny
    r, u, v = o[:, 0], o[:, 1], o[:, 2]
    rx, ry = sx * d[0][:, 0], sy * d[0][:, 1]
    ux, uy = sx * d[1][:, 0], sy * d[1][:, 1]
    vx, vy = sx * d[2][:, 0], sy * d[2][:, 1]
    N = nx * ny
    tt = torch.tensor(t, dtype=dt)
    L_data = ((o - tt) ** 2).sum() / N
    psi = RHO0 * (1 - torch.exp(-r / RHO0))
    P = 1.0 / 3.0 + G * psi * torch.exp(-r / RHO0) / 3.0
    rc = u * rx + r * ux + v * ry + r * vy
    rmx = u * u * rx + 2 * r * u * ux + u * v * ry + r * v * uy + r * u * vy + P * rx
    rmy = u * v * rx + r * v * ux + r * u * vx + v * v * ry + 2 * r * v * vy + P * ry
    L_phys = (rc ** 2 + rmx ** 2 + rmy ** 2).sum() / N
    m = torch.tensor(iface)
    q = rx * rx + ry * ry
    L_int = torch.where(m, -hp.alpha1 * q + hp.alpha2 * q * q, torch.zeros_like(q)).sum() / max(1, int(iface.sum()))
    L = L_data + hp.lambda_phys * L_phys + hp.lambda_int * L_int
    L.backward()
    return float(L.detach()), np.concatenate([np.concatenate([W.grad.numpy().ravel(), b.grad.numpy()]) for W, b in layers])


@pytest.mark.parametrize("hp", [T.TrainParams(), T.TrainParams(lambda_phys=3e3, lambda_int=0.0),
                                T.TrainParams(lambda_phys=0.0, lambda_int=1e3, alpha2=50.0)])
def test_gradient_equals_torch_autograd(hp):
    nx, ny = 8, 6
    blob = blob64(23)
    t, iface = small_problem(nx, ny, 5)
    L, _, g = T.loss_and_grad(blob, nx, ny, t, iface, G, RHO0, hp)
    Lt, gt = torch_gradient(blob, nx, ny, t, iface, hp)
    assert abs(L - Lt) < 1e-12 * max(1.0, abs(Lt))
    assert np.abs(g - gt).max() < 1e-11 * np.abs(gt).max()


def test_gradient_equals_central_differences_of_the_loss():
    nx, ny = 6, 5
    blob = blob64(24)
    t, iface = small_problem(nx, ny, 6)
    hp = T.TrainParams(lambda_phys=1e3, lambda_int=1e2, alpha2=20.0)
    L, _, g = T.loss_and_grad(blob, nx, ny, t, iface, G, RHO0, hp)
    rng = np.random.default_rng(1)
    idx = np.concatenate([np.arange(0, 192), rng.integers(192, blob.size, 40), np.arange(blob.size - 3, blob.size)])
    h = 1e-6
    for i in idx:
        wp, wm = blob.copy(), blob.copy()
        wp[i] += h
        wm[i] -= h
        fd = (T.loss_and_grad(wp, nx, ny, t, iface, G, RHO0, hp)[0] - T.loss_and_grad(wm, nx, ny, t, iface, G, RHO0, hp)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 * np.abs(g).max(), i


def test_zero_hidden_weights_give_the_closed_form_bias_gradient():
    # all weights zero: N = b5 everywhere, so dL_data/db5 = 2 (b5 - mean target) and every
    # other gradient vanishes except dL/dW5 = 0 (tanh(0) = 0) -- the network has no slope,
    # so the physics and interface terms see constant fields
    nx, ny = 7, 5
    blob = np.zeros(O.mlp_blob_size())
    blob[-3:] = [0.9, 0.1, -0.3]
    t, iface = small_problem(nx, ny, 7)
    L, terms, g = T.loss_and_grad(blob, nx, ny, t, iface, G, RHO0, T.TrainParams())
    assert np.allclose(g[-3:], 2.0 * (blob[-3:] - t.mean(axis=0)), rtol=0, atol=1e-14)
    assert np.abs(g[:-3]).max() == 0.0
    assert terms[1] == 0.0 and terms[2] == 0.0
    assert L == pytest.approx(np.mean(np.sum((blob[-3:] - t) ** 2, axis=1)), rel=1e-14)


# ----------------------------------------------------------------------------- optimizer

def test_adam_matches_torch_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    w0 = rng.standard_normal(50)
    hp = T.TrainParams(lr=3e-4)
    p = torch.tensor(w0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=hp.lr, betas=(hp.beta1, hp.beta2), eps=hp.eps)
    st = T.AdamState.zeros(50)
    w = w0.copy()
    for k in range(12):
        g = rng.standard_normal(50) * (10.0 ** rng.integers(-6, 2, 50))
        w = T.adam_step(w, g, st, hp)
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        assert np.abs(w - p.detach().numpy()).max() < 1e-15


def test_adam_first_step_is_lr_times_sign():
    g = np.array([1e-3, -2.0, 5e2, -1e-5])
    hp = T.TrainParams()
    w = T.adam_step(np.zeros(4), g, T.AdamState.zeros(4), hp)
    assert np.allclose(w, -hp.lr * g / (np.abs(g) + hp.eps), rtol=1e-14, atol=0)


def test_training_reduces_the_loss_on_a_droplet_and_keeps_the_blob_fp32():
    job = wl.single_64()
    f = O.init_equilibrium(O.init_rho(job.nx, job.ny, job.droplets, job.rho_in, job.rho_out, job.width,
                                      job.noise_amp, job.seed))
    O.step(f, 50, job.G, job.tau)
    blob, hist, st = T.train(job.weights(), f, 12, job.G)
    assert blob.dtype == np.float32 and blob.size == O.mlp_blob_size()
    assert st.t == 12 and hist.shape == (12, 4)
    assert np.all(np.diff(hist[:4, 0]) < 0) and hist[-1, 0] < 0.95 * hist[0, 0]   # descends (Adam may overshoot later)
    assert np.allclose(hist[:, 0], hist[:, 1] + hist[:, 2] + hist[:, 3])
    # Adam's step bound (Kingma and Ba, Sec. 2.1): |step| <= lr (1 - beta1) / sqrt(1 - beta2) per weight
    bound = 12 * 3e-4 * 0.1 / np.sqrt(1e-3)
    moved = np.abs(blob.astype(np.float64) - job.weights().astype(np.float64)).max()
    assert 3e-4 <= moved <= bound * (1 + 1e-6) + 1e-7
