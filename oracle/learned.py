"""FP64 numpy oracle of the learned flux correction (test infrastructure only;
the product library never imports it).

The network and the correction follow this project's reading of the
learned-correction extension (the paper itself has no learned part):
  x   = (W - in_mean) / in_scale           5 channels of cell primitives
  h1  = tanh(conv3(x;  w1, b1))            5 -> 32 channels
  h2  = tanh(conv3(h1; w2, b2))            32 -> 32
  phi = out_scale * conv3(h2; w3, b3)      32 -> 5, linear
conv3 is a 3x3x3 cross-correlation with "same" padding (periodic or
clamped per axis, like the mesh's ghost cells):
  out[co, k, j, i] = b[co] + sum_{ci, a, b, c} w[co, ci, a, b, c]
                     * in[ci, k+a-1, j+b-1, i+c-1]
The face-flux correction along axis d at the face between cells L and R is
phi[R] - phi[L]; the update of a cell is minus the divergence of it:
  dU = -sum_d (dt / dx_d) (phi[i+e_d] - 2 phi[i] + phi[i-e_d])
which is conservative (it telescopes) and zero for a constant phi.
Training minimises  L = mean_{q, cells} ((dU - r) / sigma_q)^2  for a
residual r = (fine solution averaged to the coarse mesh) - (coarse step).
"""
from __future__ import annotations

import numpy as np

C_IN, C_HID, C_OUT = 5, 32, 5
SHAPES = {"w1": (C_HID, C_IN, 3, 3, 3), "b1": (C_HID,),
          "w2": (C_HID, C_HID, 3, 3, 3), "b2": (C_HID,),
          "w3": (C_OUT, C_HID, 3, 3, 3), "b3": (C_OUT,)}
ORDER = ("w1", "b1", "w2", "b2", "w3", "b3")


def param_count() -> int:
    return int(sum(np.prod(SHAPES[k]) for k in ORDER))


def unflatten(flat):
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(SHAPES[k])
        o += n
    return out


def flatten(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in ORDER])


def pad(x, periodic):
    """Pad the three spatial axes of a (C, nz, ny, nx) array by one cell:
    wrap where periodic[a] (a = 0 x, 1 y, 2 z), else repeat the edge."""
    for a in range(3):
        axis = 3 - a
        w = [(0, 0)] * 4
        w[axis] = (1, 1)
        x = np.pad(x, w, mode="wrap" if periodic[a] else "edge")
    return x


def conv3(x, w, b, periodic):
    """3x3x3 "same" cross-correlation, written as 27 shifted matrix products."""
    _, nz, ny, nx = x.shape
    xp = pad(x, periodic)
    out = np.broadcast_to(b[:, None, None, None], (w.shape[0], nz, ny, nx)).copy()
    for a in range(3):
        for bb in range(3):
            for c in range(3):
                sl = xp[:, a:a + nz, bb:bb + ny, c:c + nx]
                out += np.einsum("oi,izyx->ozyx", w[:, :, a, bb, c], sl)
    return out


def conv3_backward(x, w, gout, periodic):
    """Gradients of sum(gout * conv3(x, w, b)) with respect to x, w and b."""
    _, nz, ny, nx = x.shape
    xp = pad(x, periodic)
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for a in range(3):
        for bb in range(3):
            for c in range(3):
                sl = xp[:, a:a + nz, bb:bb + ny, c:c + nx]
                gw[:, :, a, bb, c] = np.einsum("ozyx,izyx->oi", gout, sl)
                gxp[:, a:a + nz, bb:bb + ny, c:c + nx] += np.einsum(
                    "oi,ozyx->izyx", w[:, :, a, bb, c], gout)
    # fold the padding back onto the cells it copies
    gx = unpad_adjoint(gxp, periodic)
    return gx, gw, gout.sum(axis=(1, 2, 3))


def unpad_adjoint(gp, periodic):
    """Adjoint of pad(): add each padded cell's gradient to its source cell."""
    for a in (2, 1, 0):
        axis = 3 - a
        n = gp.shape[axis] - 2
        lo = np.take(gp, [0], axis=axis)
        hi = np.take(gp, [n + 1], axis=axis)
        core = np.take(gp, range(1, n + 1), axis=axis).copy()
        first = [slice(None)] * 4
        last = [slice(None)] * 4
        first[axis] = slice(0, 1)
        last[axis] = slice(n - 1, n)
        if periodic[a]:
            core[tuple(last)] += lo
            core[tuple(first)] += hi
        else:
            core[tuple(first)] += lo
            core[tuple(last)] += hi
        gp = core
    return gp


def forward(p, W, norm, periodic):
    """phi and the activations for primitives W (5, nz, ny, nx)."""
    x = (W - norm["in_mean"][:, None, None, None]) / norm["in_scale"][:, None, None, None]
    h1 = np.tanh(conv3(x, p["w1"], p["b1"], periodic))
    h2 = np.tanh(conv3(h1, p["w2"], p["b2"], periodic))
    o = conv3(h2, p["w3"], p["b3"], periodic)
    phi = norm["out_scale"][:, None, None, None] * o
    return phi, (x, h1, h2)


def laplacian_update(phi, dt, inv_d, periodic):
    """dU = -sum_d dt inv_d[d] (phi[i+e_d] - 2 phi[i] + phi[i-e_d])."""
    dU = np.zeros_like(phi)
    php = pad(phi, periodic)
    _, nz, ny, nx = phi.shape
    c = php[:, 1:-1, 1:-1, 1:-1]
    for a in range(3):
        axis = 3 - a
        lo = [slice(None), slice(1, -1), slice(1, -1), slice(1, -1)]
        hi = list(lo)
        lo[axis] = slice(0, -2)
        hi[axis] = slice(2, None)
        dU -= dt * inv_d[a] * (php[tuple(hi)] - 2.0 * c + php[tuple(lo)])
    return dU


def laplacian_update_adjoint(g, dt, inv_d, periodic):
    """Adjoint of laplacian_update (its transpose) applied to g."""
    gp = np.zeros((g.shape[0], g.shape[1] + 2, g.shape[2] + 2, g.shape[3] + 2))
    for a in range(3):
        axis = 3 - a
        lo = [slice(None), slice(1, -1), slice(1, -1), slice(1, -1)]
        hi = list(lo)
        lo[axis] = slice(0, -2)
        hi[axis] = slice(2, None)
        gp[tuple(hi)] -= dt * inv_d[a] * g
        gp[tuple(lo)] -= dt * inv_d[a] * g
        gp[:, 1:-1, 1:-1, 1:-1] += 2.0 * dt * inv_d[a] * g
    return unpad_adjoint(gp, periodic)


def loss_and_grads(p, W, r, dt, inv_d, norm, periodic):
    """L = mean(((dU - r) / sigma)^2) and dL/dparams (dict)."""
    phi, (x, h1, h2) = forward(p, W, norm, periodic)
    dU = laplacian_update(phi, dt, inv_d, periodic)
    sig = norm["res_scale"][:, None, None, None]
    e = (dU - r) / sig
    n = e.size
    L = float(np.mean(e * e))
    g_dU = 2.0 * e / sig / n
    g_phi = laplacian_update_adjoint(g_dU, dt, inv_d, periodic)
    g_o = g_phi * norm["out_scale"][:, None, None, None]
    g_h2, gw3, gb3 = conv3_backward(h2, p["w3"], g_o, periodic)
    g_a2 = g_h2 * (1.0 - h2 * h2)
    g_h1, gw2, gb2 = conv3_backward(h1, p["w2"], g_a2, periodic)
    g_a1 = g_h1 * (1.0 - h1 * h1)
    _, gw1, gb1 = conv3_backward(x, p["w1"], g_a1, periodic)
    return L, {"w1": gw1, "b1": gb1, "w2": gw2, "b2": gb2, "w3": gw3, "b3": gb3}


def init_params(seed: int, scale: float = 1.0):
    """Seeded initial parameters (uniform, fan-in scaled), from SplitMix64."""
    from paper_1812_07977_gb300.problems import SplitMix64
    g = SplitMix64(seed)
    p = {}
    for k in ORDER:
        shape = SHAPES[k]
        n = int(np.prod(shape))
        if k.startswith("w"):
            fan_in = shape[1] * 27
            bound = scale * np.sqrt(3.0 / fan_in)
            p[k] = ((2.0 * g.uniform(n) - 1.0) * bound).reshape(shape)
        else:
            p[k] = np.zeros(shape)
    return p
