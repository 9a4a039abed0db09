"""The learned mean-Oseen solve on the GPU against its CPU reference
(oracle/learned.py): forward pass, loss and gradients with the same
(BF16-representable) weights, one Adam step against its closed form, the
training targets against the exact solve, and the network inside the inner
solve with the exact fallback keeping the Picard solve correct.

Two modes.  CUDA-core mode: FP32 activations, BF16 weights; with weights that are
exactly representable in BF16 on both sides, the remaining difference is FP32
rounding of sums of at most 9 x 64 products per layer: 1e-5 relative for the
network output and loss, 1e-4 for gradients (sums over every pixel and image).
Tensor-core mode (the default): convolutions with 16k output channels take BF16
activations as operands; the reference rounds the same operands to BF16 (round
to nearest even), so what remains is FP32 accumulation plus the rare operand
whose FP32 and FP64 values round to neighbouring BF16 numbers: 1e-3 relative."""
import numpy as np
import pytest

import synth
from oracle import learned as L
from oracle.solver import mean_velocity_field
from oracle.system import Discretisation
from oracle.tt import TT
from synth.lattice import gaussian_residuals, node_lattice

pytestmark = pytest.mark.gpu


def _bf16(a):
    """Round float64 values to the nearest BF16 (ties to even) and back."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _flat(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params]).astype(np.float32)


def _unflat(flat, like):
    out, o = [], 0
    for W, b in like:
        nW, nb = W.size, b.size
        out.append((flat[o:o + nW].reshape(W.shape).astype(np.float64),
                    flat[o + nW:o + nW + nb].astype(np.float64)))
        o += nW + nb
    return out


@pytest.fixture(scope="module")
def setup():
    from paper_1906_06785_gb300 import binding
    prob = synth.preset("tiny")
    d = Discretisation(prob)
    lat = node_lattice(prob.mesh)
    ctx = binding.Context()
    P = ctx.problem(prob)
    # a convection field: the lifting plus a random velocity
    u = TT(*synth.random_tt(d.n_t, d.n_xi, d.n_u, 2, 2, seed=3)).scale(0.3)
    w = d.full_velocity(u)
    op = P.op(ctx.tt(w.z1, w.z2, w.z3))
    rng = np.random.default_rng(5)
    params = [(_bf16(W), _bf16(rng.standard_normal(b.shape) * 0.05))
              for W, b in L.init_params(channels=8, seed=1, depth=4)]
    net = binding.NetHandle(P, 8, 4, _flat(params))
    net.set_tensor_cores(False)
    return dict(binding=binding, prob=prob, d=d, lat=lat, ctx=ctx, P=P, w=w, op=op, params=params, net=net)


def _simt(net):
    net.set_tensor_cores(False)
    return net


def test_lattice_matches_the_mesh(setup):
    n, nx, ny = setup["net"].info()
    lat = setup["lat"]
    assert (nx, ny) == (lat.nx, lat.ny)
    assert n == sum(W.size + b.size for W, b in setup["params"])


def test_forward_matches_oracle(setup):
    d, lat, w = setup["d"], setup["lat"], setup["w"]
    R = gaussian_residuals(d.n_v, 3, seed=9)
    wavg = mean_velocity_field(w)
    want = np.array([L.apply_net(setup["params"], lat, r, wavg, d.n_nodes) for r in R])
    got = setup["net"].apply(setup["op"], R)
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)


def test_loss_and_gradients_match_oracle(setup):
    d, lat, w = setup["d"], setup["lat"], setup["w"]
    R0 = gaussian_residuals(d.n_v, 4, seed=10)
    R, T = L.training_pairs(d, w, R0)
    wavg = mean_velocity_field(w)
    lo, go = L.loss_and_grads(setup["params"], lat, wavg, d.n_nodes, R, T)
    lg, gg = setup["net"].loss_grad(setup["op"], R, T)
    assert abs(lg - lo) <= 1e-5 * lo
    for (gW, gb), (hW, hb) in zip(go, _unflat(gg, setup["params"])):
        assert np.linalg.norm(hW - gW) <= 1e-4 * np.linalg.norm(gW)
        assert np.linalg.norm(hb - gb) <= 1e-4 * np.linalg.norm(gb) + 1e-7


def test_one_training_step_is_adam_on_the_exact_targets(setup):
    """tt_net_train computes t = K^-1 r itself (banded FP64 solve); one batch, one
    epoch = one Adam step, whose first update is theta - lr g / (|g| + 1e-8)."""
    from paper_1906_06785_gb300 import binding
    d, w = setup["d"], setup["w"]
    net = _simt(binding.NetHandle(setup["P"], 8, 4, _flat(setup["params"])))
    R0 = gaussian_residuals(d.n_v, 6, seed=12)
    R, T = L.training_pairs(d, w, R0)
    _, g = net.loss_grad(setup["op"], R, T)
    theta0 = net.params().astype(np.float64)
    lr = 1e-3
    losses = net.train(setup["op"], R0, epochs=1, batch=6, lr=lr)
    theta1 = net.params().astype(np.float64)
    g = g.astype(np.float64)
    want = theta0 - lr * g / (np.abs(g) + 1e-8)
    assert np.abs(theta1 - want).max() <= 1e-6
    assert losses.shape == (1,) and losses[0] > 0


def test_smoothed_training_targets_match_oracle(setup):
    """Group g of the residuals gets g weighted-Jacobi sweeps of K before t = K^-1 r.
    The pairs the training builds are checked through the loss: the first batch's
    loss (taken before its Adam step) equals loss_grad on the oracle's smoothed
    pairs."""
    from paper_1906_06785_gb300 import binding
    d, w = setup["d"], setup["w"]
    net = _simt(binding.NetHandle(setup["P"], 8, 4, _flat(setup["params"])))
    R0 = gaussian_residuals(d.n_v, 4, seed=13)
    parts = [L.training_pairs(d, w, R0[g:g + 1], smooth_sweeps=g) for g in range(4)]
    R = np.vstack([p[0] for p in parts])
    T = np.vstack([p[1] for p in parts])
    lo, _ = net.loss_grad(setup["op"], R, T)
    losses = net.train(setup["op"], R0, epochs=1, batch=4, lr=1e-30, smooth_max=3)
    assert abs(losses[0] - lo) <= 1e-5 * lo


def test_training_reduces_the_loss(setup):
    from paper_1906_06785_gb300 import binding
    d = setup["d"]
    net = binding.NetHandle(setup["P"], 8, 4, _flat(setup["params"]))
    R0 = gaussian_residuals(d.n_v, 256, seed=14)
    losses = net.train(setup["op"], R0, epochs=10, batch=32, lr=3e-3, smooth_max=2)
    assert losses[-1] < 0.8 * losses[0] and losses[-1] < losses[1]


def test_learned_inner_solve_keeps_the_picard_solve_correct(setup):
    """With the network in the inner preconditioner (exact K^-1 as fallback) the
    Picard solve reaches the same tolerance and the same solution as without it."""
    from paper_1906_06785_gb300 import binding
    prob = setup["prob"]
    tol = synth.problem.Tolerances(tol_picard=1e-9, tol_gmres=1e-4, eps_gmres=1e-10, eps_soln=1e-12,
                                   eps_conv=1e-10)
    P = setup["P"]
    net = binding.NetHandle(P, 8, 4, _flat(setup["params"]))
    R0 = gaussian_residuals(setup["d"].n_v, 256, seed=15)
    net.train(setup["op"], R0, epochs=4, batch=32, lr=3e-3, smooth_max=2)
    u0, p0, s0, c0 = P.picard(binding.opts_from(tol))
    u1, p1, s1, c1 = P.picard(binding.opts_from(tol, learned=net))
    assert c0 == binding.TT_OK and c1 == binding.TT_OK
    from ttfull import full
    assert s1.res[s1.picard_its] <= tol.tol_picard * s1.fnorm
    du = np.linalg.norm(full(u1) - full(u0)) / np.linalg.norm(full(u0))
    assert du < 1e-6
    print(f"exact: picard {s0.picard_its} gmres {list(s0.gmres_its[:s0.picard_its + 1])} "
          f"inner {list(s0.inner_its[:s0.picard_its + 1])}; learned: picard {s1.picard_its} "
          f"gmres {list(s1.gmres_its[:s1.picard_its + 1])} inner {list(s1.inner_its[:s1.picard_its + 1])} "
          f"fallbacks {list(s1.fallbacks[:s1.picard_its + 1])}")


# ------------------------------------------------------------------ tensor-core mode
def _tc_forward(params, x):
    """Forward pass with the operands the tensor-core convolutions see: the input of
    every layer with 16k output channels rounded to BF16."""
    cache, h = [], x
    for k, (W, b) in enumerate(params):
        xin = _bf16(h) if W.shape[0] % 16 == 0 else h
        z = L.conv3x3(xin, W, b)
        cache.append((h, z))
        h = np.maximum(z, 0.0) if k < len(params) - 1 else z
    return h, cache


def _tc_backward(params, cache, gy):
    """Backward pass as the kernels run it: weight and bias gradients on CUDA cores from
    the FP32 layer inputs, the input gradient of layer k > 0 as a convolution whose
    operand (the output gradient) is rounded to BF16 when it has 16k output channels."""
    grads, g = [None] * len(params), gy
    for k in range(len(params) - 1, -1, -1):
        h, z = cache[k]
        if k < len(params) - 1:
            g = g * (z > 0.0)
        _, gW, gb = L.conv3x3_backward(h, params[k][0], g)
        grads[k] = (gW, gb)
        if k > 0:
            gin = _bf16(g) if params[k][0].shape[1] % 16 == 0 else g
            g, _, _ = L.conv3x3_backward(h, params[k][0], gin)
    return grads


@pytest.fixture(scope="module")
def tc(setup):
    from paper_1906_06785_gb300 import binding
    rng = np.random.default_rng(6)
    params = [(_bf16(W), _bf16(rng.standard_normal(b.shape) * 0.05))
              for W, b in L.init_params(channels=32, seed=2, depth=4)]
    net = binding.NetHandle(setup["P"], 32, 4, _flat(params))
    return params, net


def test_tensor_core_forward_matches_oracle(setup, tc):
    d, lat, w = setup["d"], setup["lat"], setup["w"]
    params, net = tc
    wavg = mean_velocity_field(w)
    R = gaussian_residuals(d.n_v, 5, seed=21)
    want = []
    for r in R:
        x, s = L.features(lat, r, wavg, d.n_nodes)
        y, _ = _tc_forward(params, x)
        want.append(L.read_free(lat, y, s))
    want = np.array(want)
    got = net.apply(setup["op"], R)
    assert np.linalg.norm(got - want) <= 1e-3 * np.linalg.norm(want)
    # and it is a BF16-level perturbation of the FP32-activation network
    net.set_tensor_cores(False)
    simt = net.apply(setup["op"], R)
    net.set_tensor_cores(True)
    assert np.linalg.norm(got - simt) <= 3e-2 * np.linalg.norm(simt)


def test_tensor_core_gradients_match_oracle(setup, tc):
    d, lat, w = setup["d"], setup["lat"], setup["w"]
    params, net = tc
    wavg = mean_velocity_field(w)
    R0 = gaussian_residuals(d.n_v, 4, seed=22)
    R, T = L.training_pairs(d, w, R0)
    total = 0.0
    acc = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    for r, t in zip(R, T):
        x, s = L.features(lat, r, wavg, d.n_nodes)
        y, cache = _tc_forward(params, x)
        e = L.read_free(lat, y, s) - t
        den = float(t @ t)
        total += float(e @ e) / den
        gr = _tc_backward(params, cache, L.scatter_free(lat, 2.0 * e * s / den))
        acc = [(aW + gW, ab + gb) for (aW, ab), (gW, gb) in zip(acc, gr)]
    lo = total / len(R)
    go = [(gW / len(R), gb / len(R)) for gW, gb in acc]
    lg, gg = net.loss_grad(setup["op"], R, T)
    assert abs(lg - lo) <= 1e-3 * lo
    for (gW, gb), (hW, hb) in zip(go, _unflat(gg, params)):
        assert np.linalg.norm(hW - gW) <= 1e-3 * np.linalg.norm(gW)
        assert np.linalg.norm(hb - gb) <= 1e-3 * np.linalg.norm(gb) + 1e-7


def test_tensor_core_network_at_workload_size():
    """64 channels on the small workload's 49 x 17 lattice, 300 columns (3 batches of
    at most 128 images, ragged last one): the tensor-core network equals the CUDA-core
    one to BF16 operand precision, and both stay finite."""
    from paper_1906_06785_gb300 import binding
    from synth.lattice import he_normal_params
    prob = synth.preset("small")
    ctx = binding.Context()
    P = ctx.problem(prob)
    op = P.op(None)
    net = binding.NetHandle(P, 64, 4, he_normal_params(64, 4, seed=3))
    assert net.info()[1:] == (49, 17)
    R = gaussian_residuals(prob.n_v, 300, seed=31)
    a = net.apply(op, R)
    net.set_tensor_cores(False)
    b = net.apply(op, R)
    assert np.isfinite(a).all() and np.isfinite(b).all() and np.linalg.norm(b) > 0
    assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b)
