"""Learned mean-Oseen solve: a small convolutional network Phi on the velocity-node
lattice that approximates K^{-1} r, where K = tau^-1 M + A_0 + N(w_avg) is the
spatial factor of the inner preconditioner of eq. (11_prec).  Used in place of
K^{-1} inside M^{-1} = (I - C)^{-1} (x) I (x) K^{-1}, column by column of the
spatial core, so a train stays a train; the flexible GMRES of Algorithm 4.2
(which stores the preconditioned vectors) absorbs the nonlinearity of Phi, and
the exact K^{-1} stays available as a fallback.  The paper itself has no learned
component: this module is the CPU reference for that extension (forward pass,
backward pass, loss, training pairs from exact solves with K, Adam updates).

Oracle (test infrastructure only; see oracle/__init__.py).

Network: 3x3 convolutions with zero padding ("same" size), channels
5 -> C -> C -> C -> 2 with ReLU after the first three.  Input channels: the two
residual components (scaled to unit norm), the two components of w_avg, and the
domain mask; output: the two components of the correction, read at the free
nodes and scaled back by the residual norm (so Phi(a r) = a Phi(r) for a > 0).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .solver import mean_oseen_matrix, mean_velocity_field
from .tt import TT


# ---------------------------------------------------------------- convolution
def conv3x3(x, W, b):
    """y[o, i, j] = b[o] + sum_{c, p, q} W[o, c, p, q] x[c, i + p - 1, j + q - 1],
    x taken as zero outside the image.  x: (C, H, Wd), W: (O, C, 3, 3), b: (O,)."""
    C, H, Wd = x.shape
    xp = np.zeros((C, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    y = np.empty((W.shape[0], H, Wd))
    for o in range(W.shape[0]):
        acc = np.full((H, Wd), float(b[o]))
        for c in range(C):
            for p in range(3):
                for q in range(3):
                    acc += W[o, c, p, q] * xp[c, p:p + H, q:q + Wd]
        y[o] = acc
    return y


def conv3x3_backward(x, W, gy):
    """Gradients of sum(gy * conv3x3(x, W, b)) with respect to x, W and b."""
    C, H, Wd = x.shape
    xp = np.zeros((C, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    gW = np.empty_like(W)
    gxp = np.zeros_like(xp)
    for o in range(W.shape[0]):
        for c in range(C):
            for p in range(3):
                for q in range(3):
                    gW[o, c, p, q] = np.sum(gy[o] * xp[c, p:p + H, q:q + Wd])
                    gxp[c, p:p + H, q:q + Wd] += W[o, c, p, q] * gy[o]
    gb = gy.sum(axis=(1, 2))
    return gxp[:, 1:-1, 1:-1], gW, gb


# ---------------------------------------------------------------- network
def init_params(channels=64, seed=0, c_in=5, c_out=2, depth=4):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases; the last layer is
    scaled down so an untrained net starts near zero output."""
    rng = np.random.default_rng(seed)
    sizes = [c_in] + [channels] * (depth - 1) + [c_out]
    params = []
    for k in range(depth):
        fan_in = sizes[k] * 9
        W = rng.standard_normal((sizes[k + 1], sizes[k], 3, 3)) * np.sqrt(2.0 / fan_in)
        if k == depth - 1:
            W *= 0.1
        params.append((W, np.zeros(sizes[k + 1])))
    return params


def net_forward(params, x):
    """Output image and the cache of layer inputs and pre-activations."""
    cache = []
    h = x
    for k, (W, b) in enumerate(params):
        z = conv3x3(h, W, b)
        cache.append((h, z))
        h = np.maximum(z, 0.0) if k < len(params) - 1 else z
    return h, cache


def net_backward(params, cache, gy):
    """Gradients [(gW, gb)] of sum(gy * output) and the gradient for the input."""
    grads = [None] * len(params)
    g = gy
    for k in range(len(params) - 1, -1, -1):
        h, z = cache[k]
        if k < len(params) - 1:
            g = g * (z > 0.0)
        gx, gW, gb = conv3x3_backward(h, params[k][0], g)
        grads[k] = (gW, gb)
        g = gx
    return grads, g


# ---------------------------------------------------------------- lattice I/O
def features(lat, r, wavg, n_nodes):
    """Input image (5, ny, nx) for the free-dof residual r = (r_x; r_y) and the
    full-node field wavg = (w_x; w_y), and the scale ||r|| that was divided out."""
    nv = lat.free.size
    s = float(np.linalg.norm(r))
    s = s if s > 0.0 else 1.0
    img = np.zeros((5, lat.ny, lat.nx))
    for comp in range(2):
        v = np.zeros(n_nodes)
        v[lat.free] = r[comp * nv:(comp + 1) * nv] / s
        img[comp, lat.iy, lat.ix] = v
        img[2 + comp, lat.iy, lat.ix] = wavg[comp * n_nodes:(comp + 1) * n_nodes]
    img[4] = lat.mask
    return img, s


def read_free(lat, y, s):
    """(2, ny, nx) output image -> free-dof vector (u_x; u_y), times s."""
    return s * np.concatenate([y[0, lat.iy[lat.free], lat.ix[lat.free]],
                               y[1, lat.iy[lat.free], lat.ix[lat.free]]])


def scatter_free(lat, g):
    """Adjoint of read_free (s = 1): free-dof vector -> (2, ny, nx) image."""
    nv = lat.free.size
    img = np.zeros((2, lat.ny, lat.nx))
    img[0, lat.iy[lat.free], lat.ix[lat.free]] = g[:nv]
    img[1, lat.iy[lat.free], lat.ix[lat.free]] = g[nv:]
    return img


def apply_net(params, lat, r, wavg, n_nodes):
    """Phi(r): the learned approximation of K^{-1} r on both components."""
    x, s = features(lat, r, wavg, n_nodes)
    y, _ = net_forward(params, x)
    return read_free(lat, y, s)


# ---------------------------------------------------------------- training
def training_pairs(disc, w, residuals, smooth_sweeps=0, omega=2.0 / 3.0):
    """(r, K^{-1} r) pairs for K of eq. (11_prec) built from the convection TT w.
    Each residual row (both components) is first smoothed by `smooth_sweeps`
    weighted-Jacobi sweeps of K (r <- r - omega D^-1 K r per component), so the
    set mixes rough and smooth right-hand sides."""
    K = mean_oseen_matrix(disc, w)
    lu = spla.splu(K)
    dinv = 1.0 / K.diagonal()
    nv = disc.n_v
    R, T = [], []
    for r in residuals:
        r = np.array(r, dtype=np.float64)
        for _ in range(smooth_sweeps):
            for comp in range(2):
                rc = r[comp * nv:(comp + 1) * nv]
                r[comp * nv:(comp + 1) * nv] = rc - omega * dinv * (K @ rc)
        t = np.concatenate([lu.solve(r[:nv]), lu.solve(r[nv:])])
        R.append(r)
        T.append(t)
    return np.array(R), np.array(T)


def loss_and_grads(params, lat, wavg, n_nodes, R, T):
    """Mean over the batch of ||Phi(r) - t||^2 / ||t||^2 and its gradients."""
    total = 0.0
    acc = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    for r, t in zip(R, T):
        x, s = features(lat, r, wavg, n_nodes)
        y, cache = net_forward(params, x)
        e = read_free(lat, y, s) - t
        den = float(t @ t)
        total += float(e @ e) / den
        gy = scatter_free(lat, 2.0 * e * s / den)
        grads, _ = net_backward(params, cache, gy)
        acc = [(aW + gW, ab + gb) for (aW, ab), (gW, gb) in zip(acc, grads)]
    n = len(R)
    return total / n, [(gW / n, gb / n) for gW, gb in acc]


class Adam:
    """Adam updates (Kingma and Ba, 2015): bias-corrected first and second moment
    estimates of the gradient, step lr * m_hat / (sqrt(v_hat) + eps)."""

    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        out = []
        for k, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for j, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[k][j] + (1 - self.b1) * g
                v = self.b2 * self.v[k][j] + (1 - self.b2) * g * g
                self.m[k] = tuple(m if i == j else self.m[k][i] for i in range(2))
                self.v[k] = tuple(v if i == j else self.v[k][i] for i in range(2))
                mh = m / (1 - self.b1 ** self.t)
                vh = v / (1 - self.b2 ** self.t)
                new.append(p - self.lr * mh / (np.sqrt(vh) + self.eps))
            out.append((new[0], new[1]))
        return out


# ---------------------------------------------------------------- use in M^{-1}
class LearnedMinv:
    """M^{-1} z with Phi in place of K^{-1}: (I - C)^{-1} on core 1 and Phi on every
    column of core 3 (both components together)."""

    def __init__(self, params, disc, lat, w):
        self.params, self.d, self.lat = params, disc, lat
        self.wavg = mean_velocity_field(w) if w is not None else np.zeros(2 * disc.n_nodes)
        self.cum = np.tril(np.ones((disc.n_t, disc.n_t)))

    def __call__(self, z):
        cols = [apply_net(self.params, self.lat, z.z3[k], self.wavg, self.d.n_nodes)
                for k in range(z.z3.shape[0])]
        return TT(self.cum @ z.z1, z.z2, np.array(cols))
