"""A numpy model of the learned correction's device arithmetic, for the CPU
tests of the oracle's error scales: BF16 operands (round to nearest even),
products exact and sums accumulated in FP32 (numpy's float32 matrix
products: another order than the tensor cores', the same precision), FP32
element-wise operations.  Test infrastructure: it only exercises the
scales; the library is compared with the oracle itself."""
import numpy as np

from oracle import learned as L


def bf16(a):
    """Round to the nearest BF16 value (ties to even), as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _conv(x, w, b, periodic):
    _, nz, ny, nx = x.shape
    xp = L.pad(x, periodic)
    out = np.zeros((w.shape[0], nz * ny * nx), np.float32)
    for a in range(3):
        for bb in range(3):
            for c in range(3):
                sl = np.ascontiguousarray(xp[:, a:a + nz, bb:bb + ny, c:c + nx])
                out += w[:, :, a, bb, c] @ sl.reshape(x.shape[0], -1)
    out = out.reshape(w.shape[0], nz, ny, nx)
    if b is not None:
        out = out + b.astype(np.float32)[:, None, None, None]
    return out


def _adjoint(g, w, periodic):
    _, nz, ny, nx = g.shape
    gg = bf16(g).reshape(g.shape[0], -1)
    wb = bf16(w)
    gxp = np.zeros((w.shape[1], nz + 2, ny + 2, nx + 2), np.float32)
    for a in range(3):
        for bb in range(3):
            for c in range(3):
                gxp[:, a:a + nz, bb:bb + ny, c:c + nx] += (
                    wb[:, :, a, bb, c].T @ gg).reshape(w.shape[1], nz, ny, nx)
    return L.unpad_adjoint(gxp, periodic).astype(np.float32)


def _wgrad(g, x, periodic):
    _, nz, ny, nx = x.shape
    xp = L.pad(x, periodic)
    gg = bf16(g).reshape(g.shape[0], -1)
    gw = np.zeros((g.shape[0], x.shape[0], 3, 3, 3), np.float32)
    for a in range(3):
        for bb in range(3):
            for c in range(3):
                sl = np.ascontiguousarray(xp[:, a:a + nz, bb:bb + ny, c:c + nx])
                gw[:, :, a, bb, c] = gg @ sl.reshape(x.shape[0], -1).T
    return gw


def _stencil(f, dt, inv_d, scale):
    out = np.zeros_like(f)
    for a in range(3):
        ax = 3 - a
        st = np.roll(f, -1, axis=ax) - np.float32(2) * f + np.roll(f, 1, axis=ax)
        out = out + np.float32(inv_d[a]) * st
    return -np.float32(dt) * scale.astype(np.float32)[:, None, None, None] * out


def forward(p, W, norm, periodic):
    mean = norm["in_mean"].astype(np.float32)[:, None, None, None]
    scale = norm["in_scale"].astype(np.float32)[:, None, None, None]
    x = bf16((W.astype(np.float32) - mean) / scale)
    h1 = bf16(np.tanh(_conv(x, bf16(p["w1"]), p["b1"], periodic)))
    h2 = bf16(np.tanh(_conv(h1, bf16(p["w2"]), p["b2"], periodic)))
    o = _conv(h2, bf16(p["w3"]), p["b3"], periodic)
    return {"x": x, "h1": h1, "h2": h2, "o": o}


def backward(p, f, r, dt, inv_d, norm, periodic):
    osc, sig = norm["out_scale"], norm["res_scale"].astype(np.float32)[:, None, None, None]
    du = _stencil(f["o"], dt, inv_d, osc)
    e = (du - r.astype(np.float32)) / sig
    g = np.float32(2) * e / (sig * np.float32(e.size))
    go = _stencil(g, dt, inv_d, osc)
    g2 = _adjoint(go, p["w3"], periodic) * (np.float32(1) - f["h2"] * f["h2"])
    g1 = _adjoint(g2, p["w2"], periodic) * (np.float32(1) - f["h1"] * f["h1"])
    grads = {"w3": _wgrad(go, f["h2"], periodic), "b3": go.sum((1, 2, 3)),
             "w2": _wgrad(g2, f["h1"], periodic), "b2": g2.sum((1, 2, 3)),
             "w1": _wgrad(g1, f["x"], periodic), "b1": g1.sum((1, 2, 3))}
    return {"g_o": go, "g_a2": g2, "g_a1": g1, "grads": grads}
