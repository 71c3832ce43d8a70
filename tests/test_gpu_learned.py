"""Learned flux correction on the GPU (fv_net_*, fv_step_learned) against the
FP64 numpy oracle (oracle/learned.py) on the same parameters and states.

The GPU network runs in BF16 (weights and activations; 8-bit significand)
with FP32 accumulation.  On this small, ragged mesh (every tensor-core tile
partly outside it) the network output is checked element by element against
the oracle's error scales (16 S + D, oracle.learned.forward_scales), and the
loss and each parameter tensor's gradient against gates about three times
the measured BF16-level error (relative L2 below 1%, cosine above 0.9999);
the element-wise gradient checks at the full-tile 64^3 mesh are in
test_gpu_learned_elementwise.py."""
import numpy as np
import pytest

import oracle
from oracle import learned as L
from paper_1812_07977_gb300 import problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PER = (True, True, True)
NORM = {"in_mean": np.array([1.0, 0.0, 0.0, 0.0, 1.0]),
        "in_scale": np.array([0.2, 0.3, 0.3, 0.3, 0.2]),
        "out_scale": np.array([1e-3, 2e-3, 2e-3, 1e-3, 3e-3]),
        "res_scale": np.array([1e-4, 1e-4, 1e-4, 1e-4, 2e-4])}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def _prims(U):
    rho = U[0]
    v = U[1:4] / rho
    p = 0.4 * (U[4] - 0.5 * rho * (v * v).sum(0))
    return np.stack([rho, v[0], v[1], v[2], p])


def _setup(shape=(12, 10, 9), seed=4):
    U0 = problems.random_smooth_periodic(*shape, seed=seed)
    p = L.init_params(seed)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.1 * rng.standard_normal(p[k].shape)
    from paper_1812_07977_gb300.fv import Mesh, Net
    mesh = Mesh(*shape, bc=("periodic",) * 3)
    mesh.set_state(U0)
    net = Net()
    net.set_params(L.flatten(p))
    net.set_scales(NORM["in_mean"], NORM["in_scale"], NORM["out_scale"], NORM["res_scale"])
    return U0, p, mesh, net


def _inv_d(shape):
    return np.array([shape[0], shape[1], shape[2]], dtype=np.float64)  # unit cube


def test_forward_matches_oracle():
    U0, p, mesh, net = _setup()
    o = net.forward(mesh).cpu().numpy().astype(np.float64)
    p32 = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in p.items()}
    fw = L.forward_scales(p32, _prims(U0), NORM, PER, 1.4, U0)
    ref = fw["o"]
    err = np.abs(o - ref)
    ratio = (err / (16.0 * fw["So"] + fw["Do"])).max()
    rel2 = np.linalg.norm(o - ref) / np.linalg.norm(ref)
    print("forward: max err / (16 S + D)", ratio, "rel L2", rel2)
    assert ratio <= 1.0 and rel2 < 1e-2
    mesh.close()
    net.close()


def test_loss_and_gradients_match_oracle():
    shape = (12, 10, 9)
    U0, p, mesh, net = _setup(shape)
    rng = np.random.default_rng(8)
    r = 1e-4 * rng.standard_normal((5,) + shape[::-1])
    dt = 0.01
    loss = net.train_step(mesh, torch.from_numpy(r).cuda(), dt, 0.0)
    g = net.grads().astype(np.float64)
    Lref, gref = L.loss_and_grads(p, _prims(U0), r, dt, _inv_d(shape), NORM, PER)
    print("loss", loss, Lref)
    assert abs(loss - Lref) <= 2e-2 * Lref
    gr = L.unflatten(g)
    # a constant shift of the last layer's output gives a constant phi and no
    # correction, so the exact gradient of b3 is zero: both sides must be at
    # round-off compared with the other gradients
    gscale = np.abs(gref["w3"]).max()
    assert np.abs(gr["b3"]).max() < 1e-4 * gscale and np.abs(gref["b3"]).max() < 1e-9 * gscale
    for k in L.ORDER[:-1]:
        a, b = gr[k].ravel(), gref[k].ravel()
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        print(k, "rel L2", rel, "cos", cos)
        assert rel < 1e-2 and cos > 0.9999, k
    mesh.close()
    net.close()


def test_training_reduces_the_loss():
    shape = (16, 16, 8)
    U0, p, mesh, net = _setup(shape, seed=6)
    # a reachable target: the correction of a perturbed copy of the network
    q = {k: v * (1.0 + 0.3 * np.random.default_rng(1).standard_normal(v.shape))
         for k, v in p.items()}
    phi, _ = L.forward(q, _prims(U0), NORM, PER)
    r = L.laplacian_update(phi, 0.01, _inv_d(shape), PER)
    rt = torch.from_numpy(r).cuda()
    losses = [net.train_step(mesh, rt, 0.01, 2e-3) for _ in range(60)]
    print("loss", losses[0], "->", losses[-1])
    assert losses[-1] < 0.5 * losses[0]
    mesh.close()
    net.close()


def test_asynchronous_steps_match_synchronous_steps():
    """Train steps without a loss read (no host wait) compute the same
    parameters bit for bit, and fv_net_take_loss returns the sum of the
    losses the synchronous steps report (the same operations, the same
    order), then zero."""
    shape = (16, 16, 8)
    r = None
    out = []
    for sync in (True, False):
        U0, p, mesh, net = _setup(shape, seed=6)
        phi, _ = L.forward(p, _prims(U0), NORM, PER)
        r = L.laplacian_update(1.2 * phi, 0.01, _inv_d(shape), PER)
        rt = torch.from_numpy(r).cuda()
        total = 0.0
        for _ in range(5):
            v = net.train_step(mesh, rt, 0.01, 2e-3, sync=sync)
            if sync:
                total += v
        if not sync:
            total, n = net.take_loss()
            assert n == 5
            assert net.take_loss() == (0.0, 0)
        params, grads = net.params(), net.grads()
        out.append((total, params, grads))
        mesh.close()
        net.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


def test_zero_network_gives_the_plain_step_bitwise():
    shape = (12, 10, 9)
    U0 = problems.random_smooth_periodic(*shape, seed=2)
    from paper_1812_07977_gb300.fv import Mesh, Net
    a = Mesh(*shape, bc=("periodic",) * 3)
    b = Mesh(*shape, bc=("periodic",) * 3)
    a.set_state(U0)
    b.set_state(U0)
    with Net() as net:
        net.set_params(np.zeros(net.nparam, dtype=np.float32))
        for _ in range(3):
            dt = a.reduce_dt(0.4)
            net.step(a, dt)
            b.step(dt)
    assert np.array_equal(a.get_state().cpu().numpy(), b.get_state().cpu().numpy())
    a.close()
    b.close()


def test_corrected_step_is_conservative():
    shape = (12, 10, 9)
    U0, p, mesh, net = _setup(shape)
    from paper_1812_07977_gb300.fv import Mesh
    plain = Mesh(*shape, bc=("periodic",) * 3)
    plain.set_state(U0)
    for _ in range(3):
        dt = mesh.reduce_dt(0.4)
        net.step(mesh, dt)
        plain.step(dt)
    a, b = mesh.conserved_sums(), plain.conserved_sums()
    got = mesh.get_state().cpu().numpy()
    assert np.abs(got - plain.get_state().cpu().numpy()).max() > 0   # it did correct
    scale = np.abs(U0).reshape(5, -1).sum(1) / U0[0].size
    assert np.all(np.abs(a - b) <= 1e-9 * scale), (a - b) / scale
    mesh.close()
    plain.close()
    net.close()


def test_rejects_non_periodic_mesh():
    from paper_1812_07977_gb300.fv import FvError, Mesh, Net
    with Mesh(8, 8, 8) as m, Net() as net:
        m.set_state(problems.uniform(8, 8, 8, 1.0, (0, 0, 0), 1.0))
        with pytest.raises(FvError):
            net.forward(m)


def test_bounded_mbarrier_wait(tmp_path):
    """The tensor-core kernels' wait for their MMAs is bounded: on an
    mbarrier that nothing arrives at it gives up after its poll limit (the
    kernel then records FV_ERR_TIMEOUT instead of hanging), and on a completed
    phase it returns at once (tests/cuda/mbar_wait_check.cu)."""
    import os
    import subprocess
    from paper_1812_07977_gb300.build import ARCH, CSRC, INCLUDE, nvcc
    here = os.path.dirname(os.path.abspath(__file__))
    exe = str(tmp_path / "mbar_wait_check")
    subprocess.run([nvcc(), *ARCH, "-O3", "-std=c++17", "-I", CSRC, "-I", INCLUDE,
                    os.path.join(here, "cuda", "mbar_wait_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0 and "expired 1 completed 1" in r.stdout, r.stdout + r.stderr
