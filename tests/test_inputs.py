"""The seeded input generators shared by the oracle and the CUDA path
(paper_1812_07977_gb300/problems.py): the random-number generator against
its published test vector, and each workload recipe against its stated
structure and ranges (CPU only)."""
import math

import numpy as np
import pytest

from paper_1812_07977_gb300 import problems

# First outputs of SplitMix64 seeded with 1234567, as published with the
# generator's reference implementation.
SPLITMIX64_1234567 = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                      4593380528125082431, 16408922859458223821]


def _prims(U, gamma=problems.GAMMA):
    rho = U[0]
    v = U[1:4] / rho
    p = (gamma - 1.0) * (U[4] - 0.5 * rho * (v * v).sum(0))
    return rho, v, p


def test_splitmix64_published_vector():
    g = problems.SplitMix64(1234567)
    assert [int(x) for x in g.next_u64(5)] == SPLITMIX64_1234567
    # drawing in pieces continues the same stream
    g1, g2 = problems.SplitMix64(99), problems.SplitMix64(99)
    a = g1.next_u64(7)
    b = np.concatenate([g2.next_u64(3), g2.next_u64(4)])
    assert np.array_equal(a, b)


def test_uniform_in_unit_interval():
    u = problems.SplitMix64(5).uniform(200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1.0 / 12.0) < 0.002
    # the top 53 bits: multiples of 2^-53
    assert np.all(u * 2.0**53 == np.floor(u * 2.0**53))


def test_oblique_riemann_states_and_plane():
    n = (12, 10, 8)
    U = problems.riemann_oblique(*n)
    rho, v, p = _prims(U)
    x = (np.arange(n[0]) + 0.5) / n[0]
    y = (np.arange(n[1]) + 0.5) / n[1]
    z = (np.arange(n[2]) + 0.5) / n[2]
    s = (x[None, None, :] - 0.5) + (y[None, :, None] - 0.5) + (z[:, None, None] - 0.5)
    left = s < 0
    assert np.array_equal(rho, np.where(left, 1.0, 0.125))
    assert np.allclose(p, np.where(left, 1.0, 0.1), rtol=1e-15, atol=0)
    assert np.all(v == 0.0)


def test_batched_workload_recipe():
    spec = problems.batched_riemann(seed=12345, count=16)
    again = problems.batched_riemann(seed=12345, count=16)
    lengths = set(range(16, 129, 8))
    for s, t in zip(spec, again):
        assert s["shape"] == t["shape"] and np.array_equal(s["U0"], t["U0"])
        assert set(s["shape"]) <= lengths
        for side in (s["left"], s["right"]):
            rho, vx, vy, vz, p = side
            assert 0.1 <= rho <= 10.0 and 0.1 <= p <= 10.0
            assert vx * vx + vy * vy + vz * vz <= 1.0
        assert abs(float(np.linalg.norm(s["normal"])) - 1.0) < 1e-14
        nx, ny, nz = s["shape"]
        assert s["U0"].shape == (5, nz, ny, nx)
        rho, v, p = _prims(s["U0"])
        # every cell holds one of the two states
        on_left = np.isclose(rho, s["left"][0], rtol=1e-15, atol=0)
        on_right = np.isclose(rho, s["right"][0], rtol=1e-15, atol=0)
        assert np.all(on_left | on_right)
    # the draws differ from mesh to mesh and with the seed
    assert len({s["shape"] for s in spec}) > 8
    other = problems.batched_riemann(seed=7, count=4)
    assert [s["shape"] for s in other] != [s["shape"] for s in spec[:4]]


@pytest.mark.parametrize("modes", [0, 8])
def test_shear_layer_structure(modes):
    n, amp, p0, gamma = 16, 0.05, 2.5, 5.0 / 3.0
    U = problems.shear_layer(n, amp, gamma=gamma, p0=p0, modes=modes, seed=3)
    rho, v, p = _prims(U, gamma)
    y = (np.arange(n) + 0.5) / n
    inside = (np.abs(y - 0.5) < 0.25)[None, :, None]
    assert np.array_equal(rho, np.broadcast_to(np.where(inside, 2.0, 1.0), rho.shape))
    assert np.allclose(v[0], np.broadcast_to(np.where(inside, 0.5, -0.5), rho.shape),
                       rtol=0, atol=1e-15)
    assert np.allclose(p, p0, rtol=1e-13, atol=0)
    assert np.abs(v[1]).max() <= amp * (1 + 1e-12) and np.abs(v[2]).max() <= amp * (1 + 1e-12)
    if modes == 0:
        # the 2D perturbation: vy = amp sin(4 pi x), the same in every y and z
        x = (np.arange(n) + 0.5) / n
        assert np.allclose(v[1], np.broadcast_to(amp * np.sin(4 * math.pi * x), rho.shape),
                           rtol=0, atol=1e-15)
        assert np.all(v[2] == 0.0)
    else:
        assert np.abs(v[2]).max() > 0.0


def test_shear_layer_device_matches_host():
    torch = pytest.importorskip("torch")
    n, amp, gamma = 12, 0.01, 5.0 / 3.0
    a = problems.shear_layer(n, amp, gamma=gamma, modes=8, seed=0)
    b = problems.shear_layer_device(n, amp, gamma=gamma, modes=8, seed=0, device="cpu")
    assert isinstance(b, torch.Tensor) and tuple(b.shape) == a.shape
    assert np.allclose(b.numpy(), a, rtol=1e-14, atol=1e-15)


def test_oblique_slab_equals_the_slice_of_the_whole_state():
    whole = problems.riemann_oblique(24, 20, 16)
    for k0, k1 in ((0, 4), (6, 10), (13, 16)):
        slab = problems.riemann_oblique(24, 20, 16, planes=(k0, k1))
        assert np.array_equal(slab, whole[:, k0:k1])
