"""The oracle's element-wise error scales of the BF16/FP32 network
arithmetic (oracle.learned.forward_scales / backward_scales), pinned on the
CPU: a numpy model of that arithmetic (tests/bf16_emulation.py) stays within
16 S + D of the oracle at every element, the scales are small against the
values they bound, and mistakes planted in the oracle's network (a flipped
weight, transposed kernel offsets, a dropped tile, a wrong bias, a wrong
tanh derivative, a shifted weight gradient) are caught at some element."""
import numpy as np
import pytest

from oracle import learned as L
from paper_1812_07977_gb300 import problems

import bf16_emulation as E

PER = (True, True, True)
C = 16.0
NORM = {"in_mean": np.array([1.5, 0.0, 0.0, 0.0, 2.5]),
        "in_scale": np.array([0.5, 0.5, 0.0625, 0.0625, 0.0625]),
        "out_scale": 2.0 ** np.array([-10.0, -9.0, -9.0, -10.0, -8.0]),
        "res_scale": 2.0 ** np.array([-13.0, -13.0, -13.0, -13.0, -12.0])}
SHAPE = (16, 12, 8)     # nx, ny, nz
DT = 2.0 ** -7
GAMMA = 1.4


def _prims(U):
    rho = U[0]
    v = U[1:4] / rho
    p = (GAMMA - 1.0) * (U[4] - 0.5 * rho * (v * v).sum(0))
    return np.stack([rho, v[0], v[1], v[2], p])


def _params(bf16_weights):
    p = L.init_params(4)
    rng = np.random.default_rng(4)
    for k in L.ORDER:
        if k.startswith("w"):
            p[k] = E.bf16(p[k]).astype(np.float64) if bf16_weights else \
                p[k].astype(np.float32).astype(np.float64)
        else:
            p[k] = (0.1 * rng.standard_normal(p[k].shape)).astype(np.float32).astype(np.float64)
    return p


def _case(bf16_weights):
    nx, ny, nz = SHAPE
    U = problems.shear_layer(16, 0.05, modes=8, seed=3)[:, :nz, :ny, :nx].copy()
    W = _prims(U)
    p = _params(bf16_weights)
    inv_d = np.array([nx, ny, nz], dtype=np.float64)
    q = {k: v * (1.0 + 0.3 * np.random.default_rng(1).standard_normal(v.shape))
         for k, v in p.items()}
    phi_q, _ = L.forward(q, W, NORM, PER)
    r = L.laplacian_update(phi_q, DT, inv_d, PER)
    fw = L.forward_scales(p, W, NORM, PER, GAMMA, U, weights_exact=bf16_weights)
    bw = L.backward_scales(p, fw, r, DT, inv_d, NORM, PER, weights_exact=bf16_weights)
    return p, W, U, r, inv_d, fw, bw


@pytest.fixture(scope="module")
def exact_case():
    return _case(True)


def _within(got, ref, S, D):
    return np.all(np.abs(np.asarray(got, np.float64) - ref) <= C * S + D)


def test_scales_agree_with_the_plain_network(exact_case):
    p, W, U, r, inv_d, fw, bw = exact_case
    phi, (x, h1, h2) = L.forward(p, W, NORM, PER)
    assert np.allclose(fw["o"] * NORM["out_scale"][:, None, None, None], phi, rtol=1e-13,
                       atol=0)
    for a, b in ((fw["x"], x), (fw["h1"], h1), (fw["h2"], h2)):
        assert np.array_equal(a, b) or np.allclose(a, b, rtol=1e-14, atol=1e-15)
    _, g = L.loss_and_grads(p, W, r, DT, inv_d, NORM, PER)
    for k in L.ORDER:
        assert np.allclose(bw["grads"][k], g[k], rtol=1e-12, atol=1e-12 * np.abs(g[k]).max())


@pytest.mark.parametrize("bf16_weights", [True, False])
def test_emulated_arithmetic_within_scales(bf16_weights):
    p, W, U, r, inv_d, fw, bw = _case(bf16_weights)
    f = E.forward(p, W, NORM, PER)
    for k in ("x", "h1", "h2", "o"):
        assert _within(f[k], fw[k], fw["S" + k], fw["D" + k]), k
    if not bf16_weights:
        return       # weight rounding adds coherently in the gradients
    b = E.backward(p, f, r, DT, inv_d, NORM, PER)
    for k, s in (("g_o", "go"), ("g_a2", "g2"), ("g_a1", "g1")):
        assert _within(b[k], bw[k], bw["S" + s], bw["D" + s]), k
    for k in L.ORDER:
        assert _within(b["grads"][k], bw["grads"][k], bw["S"][k], bw["D"][k]), k


def test_scales_are_small_against_the_values(exact_case):
    fw, bw = exact_case[5], exact_case[6]
    def med(v, S, D):
        return float(np.median((C * S + D) / np.maximum(np.abs(v), 1e-300)))
    assert med(fw["h1"], fw["Sh1"], fw["Dh1"]) < 0.15
    assert med(fw["h2"], fw["Sh2"], fw["Dh2"]) < 0.25
    assert med(fw["o"], fw["So"], fw["Do"]) < 0.5
    for k in ("w1", "w2", "w3"):
        assert med(bw["grads"][k], bw["S"][k], bw["D"][k]) < 1.0, k


def _caught(got, ref, S, D):
    return bool(np.any(np.abs(got - ref) > C * S + D))


def test_planted_forward_mistakes_are_caught(exact_case):
    p, W, U, r, inv_d, fw, bw = exact_case
    def out(q):
        phi, (x, h1, h2) = L.forward(q, W, NORM, PER)
        return phi / NORM["out_scale"][:, None, None, None], h1, h2
    ref_o = fw["o"]
    # one weight of layer 2 (of 864 per output) with its sign flipped
    q = {k: v.copy() for k, v in p.items()}
    q["w2"][np.unravel_index(np.argmax(np.abs(q["w2"])), q["w2"].shape)] *= -1.0
    o, h1, h2 = out(q)
    assert _caught(h2, fw["h2"], fw["Sh2"], fw["Dh2"])
    # layer 2 with its z and x kernel offsets transposed
    q = {k: v.copy() for k, v in p.items()}
    q["w2"] = np.ascontiguousarray(np.swapaxes(q["w2"], 2, 4))
    o, _, _ = out(q)
    assert _caught(o, ref_o, fw["So"], fw["Do"])
    # a bias of layer 1 off by 0.1 (the size of the biases)
    q = {k: v.copy() for k, v in p.items()}
    q["b1"][5] += 0.1
    _, h1, _ = out(q)
    assert _caught(h1, fw["h1"], fw["Sh1"], fw["Dh1"])
    # a dropped 8 x 8 x 4 tile of the output
    o = ref_o.copy()
    o[:, :4, :8, :8] = 0.0
    assert _caught(o, ref_o, fw["So"], fw["Do"])


def test_planted_backward_mistakes_are_caught(exact_case):
    p, W, U, r, inv_d, fw, bw = exact_case
    # tanh derivative taken as 1 - h instead of 1 - h^2
    g_h2 = L.conv3_input_grad(p["w3"], bw["g_o"], PER)
    wrong = g_h2 * (1.0 - fw["h2"])
    assert _caught(wrong, bw["g_a2"], bw["Sg2"], bw["Dg2"])
    # adjoint convolution without the kernel flip (correlation instead)
    flipped = p["w3"][:, :, ::-1, ::-1, ::-1]
    wrong = L.conv3_input_grad(flipped, bw["g_o"], PER) * (1.0 - fw["h2"] ** 2)
    assert _caught(wrong, bw["g_a2"], bw["Sg2"], bw["Dg2"])
    # weight gradient of layer 2 with the input shifted by one cell in x
    wrong = L.conv3_weight_grad(np.roll(fw["h1"], 1, axis=3), bw["g_a2"], PER)
    assert _caught(wrong, bw["grads"]["w2"], bw["S"]["w2"], bw["D"]["w2"])
    # one offset's weight gradient of layer 1 dropped
    wrong = bw["grads"]["w1"].copy()
    wrong[:, :, 0, 1, 2] = 0.0
    assert _caught(wrong, bw["grads"]["w1"], bw["S"]["w1"], bw["D"]["w1"])
