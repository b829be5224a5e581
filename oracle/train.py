"""FP64 oracle of the network's training (Eqs. 3-8, Sec. II-C step 2, Sec. III-B) -- TEST
INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this module; the product library never does.  Plain numpy in FP64; a matrix
product is the only library step, and every other step is written out below in the
paper's order.

The paper leaves the following open; each is the reading this oracle (and the CUDA path)
takes:

T1 Samples: every cell of the lattice, input (x^, y^) = the cell centre mapped to [-1, 1]
   as for the correction.  One epoch is one gradient step on the loss over all cells
   (Sec. III-B counts training epochs per coupling step and names no batch size).
T2 Targets: the lattice state when training starts: rho = sum_i f_i and u = j / rho with
   j = sum_i f_i c_i.
T3 L_data (Eq. 4): mean over the cells of |N - (rho, u_x, u_y)|^2 (the three outputs
   summed).
T4 L_phys (Eqs. 5-7): mean over the cells of r_c^2 + r_mx^2 + r_my^2 with
       r_c = d_x(rho u_x) + d_y(rho u_y)
       r_m = div(rho u u) + grad p,
   evaluated on the network's own fields.  The time derivatives are zero because N has
   no time input (Eq. 2); p is the lattice's equation of state p = rho/3 + G psi(rho)^2/6;
   the stress sigma is not defined in the paper and is taken as zero.
T5 L_int (Eq. 8): mean over the interface cells (lattice |grad rho| of Eq. 16 above the
   Eq. 9 threshold) of -alpha1 q + alpha2 q^2, q = |grad rho_N|^2.  These are the signs the
   text describes (a reward for steep interfaces, bounded by the quartic term); Eq. 8 as
   printed has them the other way round and is unbounded below.  With no interface cell
   the term is zero.
T6 Spatial derivatives of N are taken in lattice units: d/dx = (2 / nx) d/dx^.
T7 Optimizer: Adam (beta1 0.9, beta2 0.999, eps 1e-8) at the paper's learning rate 3e-4
   (Sec. III-B names the rate but not the method), no weight decay.  Its moments and step
   count persist across coupling rounds.
T8 lambda1 = lambda2 = alpha1 = alpha2 = 1 unless given (Eq. 3 and Eq. 8 give no values).
T9 Between rounds the network is the FP32 weight blob the correction reads: each round's
   training starts from it in FP64 and ends by rounding the weights back to FP32.

Blob layout (FP32): W1[64 x 2] b1 W2[128 x 64] b2 W3[128 x 128] b3 W4[64 x 128] b4
W5[3 x 64] b5, each W row-major [out][in].
"""
import dataclasses

import numpy as np

import oracle as O

HIDDEN = (64, 128, 128, 64, 3)   # outputs of layers 1..5 (Sec. III-B)


@dataclasses.dataclass
class TrainParams:
    lr: float = 3e-4
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    lambda_phys: float = 1.0
    lambda_int: float = 1.0
    alpha1: float = 1.0
    alpha2: float = 1.0


def unpack(blob, n_in=2):
    """Blob -> [(W [out, in], b [out])] in FP64."""
    w = np.asarray(blob, dtype=np.float64)
    layers, p, nin = [], 0, n_in
    for nout in HIDDEN:
        W = w[p:p + nout * nin].reshape(nout, nin).copy()
        p += nout * nin
        b = w[p:p + nout].copy()
        p += nout
        layers.append((W, b))
        nin = nout
    assert p == w.size, "blob length does not match the architecture"
    return layers


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def cell_inputs(nx, ny):
    """(x^, y^) of every cell, cell index c = y nx + x."""
    xh = 2.0 * (np.arange(nx) + 0.5) / nx - 1.0
    yh = 2.0 * (np.arange(ny) + 0.5) / ny - 1.0
    X, Y = np.meshgrid(xh, yh)
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def forward(layers, X):
    """Network outputs and their derivatives along x^ and y^ (forward tangents).

    Returns ((o, o_x, o_y), acts) where acts[l] = (a, a_x, a_y) is the input of layer l+1
    and its two tangents.  A hidden layer maps z = W a + b to tanh(z); its tangents are
    z_d = W a_d and tanh'(z) z_d (the bias has no tangent)."""
    n = X.shape[0]
    a = X
    ax = np.tile([1.0, 0.0], (n, 1))
    ay = np.tile([0.0, 1.0], (n, 1))
    acts = []
    for l, (W, b) in enumerate(layers):
        acts.append((a, ax, ay))
        z, zx, zy = a @ W.T + b, ax @ W.T, ay @ W.T
        if l == len(layers) - 1:
            return (z, zx, zy), acts
        a = np.tanh(z)
        s = 1.0 - a * a
        ax, ay = s * zx, s * zy


def pressure_slope(rho, G, rho0):
    """dp/drho and d2p/drho2 of p = rho/3 + G psi^2 / 6, psi = rho0 (1 - exp(-rho/rho0))."""
    e = np.exp(-rho / rho0)
    psi = rho0 * (1.0 - e)
    dpsi, d2psi = e, -e / rho0
    return 1.0 / 3.0 + G * psi * dpsi / 3.0, G * (dpsi * dpsi + psi * d2psi) / 3.0


def residuals(r, u, v, rx, ry, ux, uy, vx, vy, G, rho0):
    """Continuity and momentum residuals of T4 (steady, sigma = 0) from the fields and their
    lattice-unit derivatives, expanded by the product rule."""
    P, _ = pressure_slope(r, G, rho0)
    rc = u * rx + r * ux + v * ry + r * vy
    rmx = u * u * rx + 2 * r * u * ux + u * v * ry + r * v * uy + r * u * vy + P * rx
    rmy = u * v * rx + r * v * ux + r * u * vx + v * v * ry + 2 * r * v * vy + P * ry
    return rc, rmx, rmy


def losses(out, targets, iface, nx, ny, G, rho0, hp):
    """Eq. 3 on the network outputs: returns (L, (L_data, L_phys, L_int), dL/do, dL/do_x,
    dL/do_y), the last three per cell and output, derivatives along x^ and y^."""
    o, ox, oy = out
    N = o.shape[0]
    sx, sy = 2.0 / nx, 2.0 / ny
    r, u, v = o[:, 0], o[:, 1], o[:, 2]
    rx, ux, vx = sx * ox[:, 0], sx * ox[:, 1], sx * ox[:, 2]
    ry, uy, vy = sy * oy[:, 0], sy * oy[:, 1], sy * oy[:, 2]

    e = o - targets                                   # Eq. 4
    L_data = np.sum(e * e) / N
    g_o = 2.0 * e / N

    rc, rmx, rmy = residuals(r, u, v, rx, ry, ux, uy, vx, vy, G, rho0)   # Eqs. 5-7
    L_phys = np.sum(rc * rc + rmx * rmx + rmy * rmy) / N
    P, dP = pressure_slope(r, G, rho0)
    A, B, C = (2.0 * hp.lambda_phys / N) * rc, (2.0 * hp.lambda_phys / N) * rmx, (2.0 * hp.lambda_phys / N) * rmy
    dr = A * (ux + vy) + B * (2 * u * ux + v * uy + u * vy + dP * rx) + C * (v * ux + u * vx + 2 * v * vy + dP * ry)
    du = A * rx + B * (2 * u * rx + 2 * r * ux + v * ry + r * vy) + C * (v * rx + r * vx)
    dv = A * ry + B * (u * ry + r * uy) + C * (u * rx + r * ux + 2 * v * ry + 2 * r * vy)
    drx = A * u + B * (u * u + P) + C * (u * v)
    dry = A * v + B * (u * v) + C * (v * v + P)
    dux = A * r + B * (2 * r * u) + C * (r * v)
    duy = B * (r * v)
    dvx = C * (r * u)
    dvy = A * r + B * (r * u) + C * (2 * r * v)

    q = rx * rx + ry * ry                             # Eq. 8 with the T5 signs
    Ni = int(np.count_nonzero(iface))
    if Ni:
        L_int = np.sum(np.where(iface, -hp.alpha1 * q + hp.alpha2 * q * q, 0.0)) / Ni
        dq = np.where(iface, (hp.lambda_int / Ni) * (-hp.alpha1 + 2.0 * hp.alpha2 * q), 0.0)
    else:
        L_int, dq = 0.0, np.zeros(N)
    drx = drx + 2.0 * dq * rx
    dry = dry + 2.0 * dq * ry

    g_o = g_o + np.stack([dr, du, dv], axis=1)
    g_ox = sx * np.stack([drx, dux, dvx], axis=1)
    g_oy = sy * np.stack([dry, duy, dvy], axis=1)
    L = L_data + hp.lambda_phys * L_phys + hp.lambda_int * L_int
    return L, (L_data, L_phys, L_int), g_o, g_ox, g_oy


def backward(layers, acts, g_o, g_ox, g_oy):
    """Reverse pass through the value and tangent channels: [(dW, db)] per layer."""
    grads = [None] * len(layers)
    dz, dzx, dzy = g_o, g_ox, g_oy
    for l in reversed(range(len(layers))):
        W, _ = layers[l]
        a, ax, ay = acts[l]
        grads[l] = (dz.T @ a + dzx.T @ ax + dzy.T @ ay, dz.sum(axis=0))
        if l == 0:
            break
        da, dax, day = dz @ W, dzx @ W, dzy @ W
        # a = tanh(z), a_d = s z_d with s = 1 - a^2 and ds/dz = -2 a s, so
        # dL/dz = s dL/da - 2 a sum_d a_d dL/da_d and dL/dz_d = s dL/da_d
        s = 1.0 - a * a
        dz = s * da - 2.0 * a * (ax * dax + ay * day)
        dzx, dzy = s * dax, s * day
    return grads


def targets_from_state(f, threshold=0.01):
    """T2 targets (N x 3) and the T5 interface mask from a population array f[9, ny, nx]."""
    rho = O.density(f)
    jx, jy = O.momentum(f)
    t = np.stack([rho.ravel(), (jx / rho).ravel(), (jy / rho).ravel()], axis=1)
    iface = (O.grad_mag(rho) > threshold).ravel()
    return t, iface


def loss_and_grad(blob, nx, ny, targets, iface, G, rho0=1.0, hp=None, n_in=2):
    """Loss terms and the gradient (flat, blob order) at the weights `blob`."""
    hp = hp or TrainParams()
    layers = unpack(blob, n_in)
    out, acts = forward(layers, cell_inputs(nx, ny))
    L, terms, g_o, g_ox, g_oy = losses(out, targets, iface, nx, ny, G, rho0, hp)
    return L, terms, pack(backward(layers, acts, g_o, g_ox, g_oy))


@dataclasses.dataclass
class AdamState:
    m: np.ndarray
    v: np.ndarray
    t: int = 0

    @staticmethod
    def zeros(n):
        return AdamState(np.zeros(n), np.zeros(n), 0)


def adam_step(w, g, st, hp):
    """One Adam update of w (returned) with gradient g; st is updated in place (T7)."""
    st.t += 1
    st.m = hp.beta1 * st.m + (1.0 - hp.beta1) * g
    st.v = hp.beta2 * st.v + (1.0 - hp.beta2) * g * g
    mh = st.m / (1.0 - hp.beta1 ** st.t)
    vh = st.v / (1.0 - hp.beta2 ** st.t)
    return w - hp.lr * mh / (np.sqrt(vh) + hp.eps)


def train(blob, f, epochs, G, rho0=1.0, hp=None, state=None, threshold=0.01):
    """Sec. II-C step 2: `epochs` full-batch Adam steps on the state f.

    Returns (new FP32 blob, losses [epochs x 4] = (L, L_data, L_phys, L_int) at the
    weights each step started from, Adam state)."""
    hp = hp or TrainParams()
    _, ny, nx = f.shape
    t, iface = targets_from_state(f, threshold)
    w = np.asarray(blob, dtype=np.float32).astype(np.float64)
    state = state or AdamState.zeros(w.size)
    hist = np.zeros((epochs, 4))
    for e in range(epochs):
        L, terms, g = loss_and_grad(w, nx, ny, t, iface, G, rho0, hp)
        hist[e] = (L,) + tuple(terms)
        w = adam_step(w, g, state, hp)
    return w.astype(np.float32), hist, state


def run_trained(f, nsteps, G, tau, K, blob, epochs, rho0=1.0, hp=None, mode=O.MLP_F64, beta_rho=0.1, beta_u=0.01,
                M0=None, threshold=0.01, state=None, step0=0):
    """The coupled loop of Sec. II-C: after every step whose count (from step0) is a multiple
    of K, train for `epochs` epochs on the current state, then correct with the trained
    network.  f is advanced in place.  Returns (status, blob, Adam state)."""
    if M0 is None:
        M0 = O.mass(f)
    blob = np.asarray(blob, dtype=np.float32)
    s = step0
    while s < step0 + nsteps:
        n = min(K - s % K, step0 + nsteps - s)
        O.step(f, n, G, tau, rho0)
        s += n
        if s % K == 0:
            blob, _, state = train(blob, f, epochs, G, rho0, hp, state, threshold)
            st = O.correct(f, blob, beta_rho, beta_u, M0, mode)
            if st != 0:
                return st, blob, state
    return 0, blob, state
