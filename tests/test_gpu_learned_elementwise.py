"""Element-by-element parity of the learned correction's tensor-core kernels
with the FP64 oracle (oracle/learned.py) at the configured coarse mesh, 64^3
periodic (full 8 x 16 x 4 tiles of the tcgen05 convolutions, 512 of them).

Every intermediate value the library exposes (fv_net_get_buffer) and every
gradient is compared with the oracle's exact value, each element against its
own error scale from the oracle (forward_scales / backward_scales): the
propagated effect of the BF16 roundings (S, a standard-deviation scale) plus
a worst-case bound of the FP32 accumulation, element-wise FP32 arithmetic
and tanhf (D).  The gate is |gpu - oracle| <= 16 S + D for every element.
The weights are BF16 values (so their rounding, which is the same in every
cell and would add coherently in the weight gradients, is zero) and the
normalisation constants, dt and the residual scales are binary fractions
(exact in FP32)."""
import numpy as np
import pytest

from oracle import learned as L
from paper_1812_07977_gb300 import problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PER = (True, True, True)
C_SIGMA = 16.0
NORM = {"in_mean": np.array([1.5, 0.0, 0.0, 0.0, 2.5]),
        "in_scale": np.array([0.5, 0.5, 0.0625, 0.0625, 0.0625]),
        "out_scale": 2.0 ** np.array([-10.0, -9.0, -9.0, -10.0, -8.0]),
        "res_scale": 2.0 ** np.array([-13.0, -13.0, -13.0, -13.0, -12.0])}
N = 64
DT = 2.0 ** -7
GAMMA = 1.4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def _bf16(a):
    """Round to BF16 values (round to nearest even), returned as float64."""
    t = torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.to(torch.float64).numpy()


def _prims(U):
    rho = U[0]
    v = U[1:4] / rho
    p = (GAMMA - 1.0) * (U[4] - 0.5 * rho * (v * v).sum(0))
    return np.stack([rho, v[0], v[1], v[2], p])


def _check(name, got, ref, S, D, c=C_SIGMA):
    got = np.asarray(got, dtype=np.float64)
    assert got.shape == ref.shape, (name, got.shape, ref.shape)
    err = np.abs(got - ref)
    bound = c * S + D
    ratio = float((err / np.where(bound > 0, bound, np.inf)).max())
    rel = float(np.linalg.norm(err) / max(np.linalg.norm(ref), 1e-300))
    print(f"{name}: {ref.size} elements, max |err|/({c:g} S + D) = {ratio:.3f}, "
          f"relative L2 error {rel:.2e}, median bound / |value| "
          f"{np.median(bound / np.maximum(np.abs(ref), 1e-300)):.2e}")
    bad = err > bound
    assert not bad.any(), (f"{name}: {int(bad.sum())} elements outside their bound; worst at "
                           f"{np.unravel_index(np.argmax(err - bound), err.shape)}")
    return ratio


@pytest.fixture(scope="module")
def case():
    from paper_1812_07977_gb300.fv import Mesh, Net
    U0 = problems.shear_layer(N, 0.05, modes=8, seed=3)
    p = L.init_params(4)
    rng = np.random.default_rng(4)
    for k in L.ORDER:
        if k.startswith("w"):
            p[k] = _bf16(p[k])
        else:
            p[k] = np.asarray(0.1 * rng.standard_normal(p[k].shape), np.float32).astype(np.float64)
    W = _prims(U0)
    inv_d = np.array([N, N, N], dtype=np.float64)
    # a residual the network could produce: the correction of a perturbed copy
    q = {k: v * (1.0 + 0.3 * np.random.default_rng(1).standard_normal(v.shape))
         for k, v in p.items()}
    phi_q, _ = L.forward(q, W, NORM, PER)
    r = L.laplacian_update(phi_q, DT, inv_d, PER)
    mesh = Mesh(N, N, N, bc=("periodic",) * 3)
    mesh.set_state(U0)
    net = Net()
    net.set_params(L.flatten(p))
    net.set_scales(NORM["in_mean"], NORM["in_scale"], NORM["out_scale"], NORM["res_scale"])
    o = net.forward(mesh).cpu().numpy()
    fwd = {k: net.buffer(k, mesh).float().cpu().numpy() for k in ("features", "h1", "h2")}
    fwd["out"] = o
    loss = net.train_step(mesh, torch.from_numpy(r).cuda(), DT, 0.0)
    bwd = {k: net.buffer(k, mesh).cpu().numpy() for k in ("grad_out", "grad_a2", "grad_a1")}
    grads = L.unflatten(net.grads().astype(np.float64))
    mesh.close()
    net.close()
    fw = L.forward_scales(p, W, NORM, PER, GAMMA, U0, weights_exact=True)
    bw = L.backward_scales(p, fw, r, DT, inv_d, NORM, PER, weights_exact=True)
    Lref, _ = L.loss_and_grads(p, W, r, DT, inv_d, NORM, PER)
    return dict(fwd=fwd, bwd=bwd, grads=grads, loss=loss, fw=fw, bw=bw, Lref=Lref)


def test_forward_elementwise_64(case):
    """Features, both hidden activations and the network output."""
    f, fw = case["fwd"], case["fw"]
    x = f["features"]
    assert np.all(x[5:] == 0.0)       # the three pad channels
    _check("features x", x[:5], fw["x"], fw["Sx"], fw["Dx"])
    _check("h1", f["h1"], fw["h1"], fw["Sh1"], fw["Dh1"])
    _check("h2", f["h2"], fw["h2"], fw["Sh2"], fw["Dh2"])
    _check("o", f["out"], fw["o"], fw["So"], fw["Do"])


def test_input_gradients_elementwise_64(case):
    """dL/do from the loss kernels, and the two input-gradient (adjoint)
    convolutions followed by the tanh backward."""
    b, bw = case["bwd"], case["bw"]
    _check("dL/do", b["grad_out"], bw["g_o"], bw["Sgo"], bw["Dgo"])
    _check("dL/da2", b["grad_a2"], bw["g_a2"], bw["Sg2"], bw["Dg2"])
    _check("dL/da1", b["grad_a1"], bw["g_a1"], bw["Sg1"], bw["Dg1"])


def test_weight_and_bias_gradients_elementwise_64(case):
    """All three weight gradients (tcgen05 weight-gradient kernels with the
    fixed-order tile sums) and the FP32 bias gradients."""
    g, bw = case["grads"], case["bw"]
    for k in L.ORDER:
        _check("grad " + k, g[k], bw["grads"][k], bw["S"][k], bw["D"][k])


def test_loss_64(case):
    bw = case["bw"]
    e, de = bw["e"], C_SIGMA * bw["Se"] + bw["De"]
    bound = float(np.mean(2.0 * np.abs(e) * de + de * de))
    print("loss", case["loss"], "oracle", case["Lref"], "bound", bound)
    assert abs(case["loss"] - case["Lref"]) <= bound
