"""Pins of the learned-correction oracle (oracle/learned.py): the 3x3x3
convolution against a direct 7-loop sum, its backward pass and the whole
loss gradient against central finite differences, the adjoint identities,
and the conservation / uniform-state properties of the correction."""
import numpy as np
import pytest

from oracle import learned as L

PER = (True, True, True)
MIX = (True, False, True)


def _conv_brute(x, w, b, periodic):
    ci, nz, ny, nx = x.shape
    co = w.shape[0]
    out = np.zeros((co, nz, ny, nx))

    def src(g, n, per):
        if per:
            return g % n
        return min(max(g, 0), n - 1)

    for o in range(co):
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    s = b[o]
                    for c in range(ci):
                        for a in range(3):
                            for bb in range(3):
                                for cc in range(3):
                                    s += w[o, c, a, bb, cc] * x[
                                        c, src(k + a - 1, nz, periodic[2]),
                                        src(j + bb - 1, ny, periodic[1]),
                                        src(i + cc - 1, nx, periodic[0])]
                    out[o, k, j, i] = s
    return out


@pytest.mark.parametrize("periodic", [PER, (False, False, False), MIX])
def test_conv3_matches_direct_sum(periodic):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 4, 5))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    np.testing.assert_allclose(L.conv3(x, w, b, periodic), _conv_brute(x, w, b, periodic),
                               rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("periodic", [PER, (False, False, False), MIX])
def test_conv3_backward_adjoint(periodic):
    # <gout, conv3(x, w, 0)> is bilinear: its x- and w-gradients must satisfy
    # <gx, x> = <gout, conv(x)> = <gw, w>
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 4, 3, 5))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    gout = rng.standard_normal((2, 4, 3, 5))
    y = L.conv3(x, w, np.zeros(2), periodic)
    gx, gw, gb = L.conv3_backward(x, w, gout, periodic)
    s = float((gout * y).sum())
    assert abs(float((gx * x).sum()) - s) <= 1e-10 * abs(s)
    assert abs(float((gw * w).sum()) - s) <= 1e-10 * abs(s)
    np.testing.assert_allclose(gb, gout.sum(axis=(1, 2, 3)))


def _problem(seed=3, shape=(4, 3, 5), periodic=PER):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    W = np.stack([1.5 + 0.3 * rng.standard_normal(shape), 0.3 * rng.standard_normal(shape),
                  0.3 * rng.standard_normal(shape), 0.1 * rng.standard_normal(shape),
                  2.5 + 0.3 * rng.standard_normal(shape)])
    r = 1e-3 * rng.standard_normal((5,) + shape)
    norm = {"in_mean": np.array([1.5, 0.0, 0.0, 0.0, 2.5]),
            "in_scale": np.array([0.5, 0.5, 0.5, 0.5, 0.5]),
            "out_scale": np.array([1e-3, 2e-3, 2e-3, 1e-3, 3e-3]),
            "res_scale": np.array([1e-3, 1e-3, 1e-3, 1e-3, 2e-3])}
    p = L.init_params(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.1 * rng.standard_normal(p[k].shape)
    return p, W, r, norm


@pytest.mark.parametrize("periodic", [PER, MIX])
def test_loss_gradient_matches_finite_differences(periodic):
    p, W, r, norm = _problem(periodic=periodic)
    dt, inv_d = 0.01, np.array([4.0, 3.0, 5.0])
    loss, g = L.loss_and_grads(p, W, r, dt, inv_d, norm, periodic)
    flat, gflat = L.flatten(p), L.flatten(g)
    rng = np.random.default_rng(7)
    # a random direction through all parameters ...
    v = rng.standard_normal(flat.size)
    eps = 1e-6
    lp = L.loss_and_grads(L.unflatten(flat + eps * v), W, r, dt, inv_d, norm, periodic)[0]
    lm = L.loss_and_grads(L.unflatten(flat - eps * v), W, r, dt, inv_d, norm, periodic)[0]
    fd = (lp - lm) / (2 * eps)
    assert abs(fd - gflat @ v) <= 1e-6 * abs(fd), (fd, gflat @ v)
    # ... and single parameters of every tensor
    o = 0
    for k in L.ORDER:
        n = int(np.prod(L.SHAPES[k]))
        for idx in rng.choice(n, 3, replace=False):
            e = np.zeros(flat.size)
            e[o + idx] = 1.0
            lp = L.loss_and_grads(L.unflatten(flat + eps * e), W, r, dt, inv_d, norm, periodic)[0]
            lm = L.loss_and_grads(L.unflatten(flat - eps * e), W, r, dt, inv_d, norm, periodic)[0]
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - gflat[o + idx]) <= 1e-5 * abs(fd) + 1e-12, (k, idx, fd, gflat[o + idx])
        o += n


def test_correction_is_conservative_and_vanishes_for_constant_phi():
    rng = np.random.default_rng(4)
    phi = rng.standard_normal((5, 4, 6, 5))
    dU = L.laplacian_update(phi, 0.1, np.array([1.0, 2.0, 3.0]), PER)
    assert np.all(np.abs(dU.reshape(5, -1).sum(1)) < 1e-12)
    const = np.ones((5, 4, 6, 5)) * rng.standard_normal((5, 1, 1, 1))
    for periodic in (PER, (False, False, False)):
        assert np.all(L.laplacian_update(const, 0.1, np.array([1.0, 2.0, 3.0]), periodic) == 0)


@pytest.mark.parametrize("periodic", [PER, MIX])
def test_correction_adjoint(periodic):
    rng = np.random.default_rng(5)
    phi = rng.standard_normal((5, 3, 4, 5))
    g = rng.standard_normal((5, 3, 4, 5))
    inv_d = np.array([2.0, 3.0, 4.0])
    a = float((g * L.laplacian_update(phi, 0.3, inv_d, periodic)).sum())
    b = float((phi * L.laplacian_update_adjoint(g, 0.3, inv_d, periodic)).sum())
    assert abs(a - b) <= 1e-12 * abs(a)


def test_uniform_state_gets_no_correction():
    p, _, _, norm = _problem()
    W = np.broadcast_to(np.array([1.2, 0.1, -0.2, 0.0, 2.0])[:, None, None, None],
                        (5, 4, 3, 5)).copy()
    phi, _ = L.forward(p, W, norm, PER)
    dU = L.laplacian_update(phi, 0.05, np.array([4.0, 3.0, 5.0]), PER)
    assert np.abs(dU).max() < 1e-15
