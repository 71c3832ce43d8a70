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


def _shifted(xp, a, bb, c, shape):
    """The (C, nz*ny*nx) matrix of input cells at offset (a, bb, c) - 1."""
    nz, ny, nx = shape
    return xp[:, a:a + nz, bb:bb + ny, c:c + nx].reshape(xp.shape[0], -1)


def conv3(x, w, b, periodic):
    """3x3x3 "same" cross-correlation, written as 27 shifted matrix products
    (channels x cells, one per offset)."""
    _, nz, ny, nx = x.shape
    xp = pad(x, periodic)
    out = np.broadcast_to(b[:, None], (w.shape[0], nz * ny * nx)).copy()
    for a in range(3):
        for bb in range(3):
            for c in range(3):
                out += w[:, :, a, bb, c] @ _shifted(xp, a, bb, c, (nz, ny, nx))
    return out.reshape(w.shape[0], nz, ny, nx)


def conv3_weight_grad(x, gout, periodic):
    """dW of sum(gout * conv3(x, w, b)): per offset, gout times the shifted
    input, summed over the cells."""
    _, nz, ny, nx = x.shape
    xp = pad(x, periodic)
    g = gout.reshape(gout.shape[0], -1)
    gw = np.zeros((gout.shape[0], x.shape[0], 3, 3, 3))
    for a in range(3):
        for bb in range(3):
            for c in range(3):
                gw[:, :, a, bb, c] = g @ _shifted(xp, a, bb, c, (nz, ny, nx)).T
    return gw


def conv3_input_grad(w, gout, periodic):
    """dX of sum(gout * conv3(x, w, b)): each offset's transposed weights
    times gout, added at the shifted cells, the padding folded back."""
    _, nz, ny, nx = gout.shape
    g = gout.reshape(gout.shape[0], -1)
    gxp = np.zeros((w.shape[1], nz + 2, ny + 2, nx + 2))
    for a in range(3):
        for bb in range(3):
            for c in range(3):
                gxp[:, a:a + nz, bb:bb + ny, c:c + nx] += (
                    w[:, :, a, bb, c].T @ g).reshape(w.shape[1], nz, ny, nx)
    return unpad_adjoint(gxp, periodic)


def conv3_backward(x, w, gout, periodic):
    """Gradients of sum(gout * conv3(x, w, b)) with respect to x, w and b."""
    return (conv3_input_grad(w, gout, periodic), conv3_weight_grad(x, gout, periodic),
            gout.sum(axis=(1, 2, 3)))


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


# ---------------------------------------------------------------------------
# Element-wise error scales of the BF16 / FP32 network arithmetic.
#
# The library's network rounds its operands to BF16 (weights; the features
# and the two hidden activations, which it stores as BF16; the 5- and
# 32-channel gradients fed to the adjoint and weight-gradient convolutions)
# and accumulates in FP32.  For each quantity of forward() and
# loss_and_grads() the functions below compute, in FP64 from the oracle's own
# values (no value of the library enters), two per-element numbers:
#   S  the scale of the BF16 rounding errors that reach it: every rounding
#      to BF16 is a relative error of at most U_BF16, taken as an independent
#      zero-mean variable of variance U_BF16^2 (a conservative variance: a
#      uniform error on [-u, u] has u^2/3), and S^2 is the variance of their
#      first-order effect, propagated through each contraction with squared
#      weights -- the probabilistic rounding-error analysis of Higham & Mary
#      (SIAM J. Sci. Comput. 41, 2019), in which a length-n inner product's
#      error grows like sqrt(n) u rather than n u;
#   D  a deterministic bound of the errors made where the value itself is
#      formed: FP32 accumulation, taken in the worst case (products of BF16
#      operands are exact in FP32; the tensor cores round, possibly by
#      truncation, once per MMA of 16 products, so K terms cost at most
#      K/16 * 2^-22 of the sum of their magnitudes), the FP32 element-wise
#      operations (a few 2^-24 each) and tanhf (2 ulp).  Downstream, an
#      input's D counts like its S: an error of unknown sign, independent
#      from one input element to the next (S^2 + D^2 enters the variance).
# A library value v_dev of exact value v is expected within
#   |v_dev - v| <= c S + D,
# c a number of standard deviations (the tests use 10).  The parameters the
# library holds are taken to be exactly `p` (FP32 values), each weight
# reaching the tensor cores rounded once to BF16 -- unless `weights_exact`
# says that every weight already is a BF16 value.  A weight's rounding error
# is the same in every cell, so its effect on a sum over cells (a weight
# gradient) is coherent, not random: tests that check weight gradients use
# BF16-valued weights, for which it is zero.

U_BF16 = 2.0 ** -8           # unit roundoff of BF16 (8-bit significand)
ACC_MMA = 2.0 ** -22         # one tensor-core accumulation step (16 products)
TANH_ABS = 2.0 ** -21        # |tanhf(a) - tanh(a)| on the device (2 ulp of |t| <= 1)
K_SECOND = 12.0              # error size, in units of S, taken in second-order terms


def _mma_steps(ci):
    """MMA steps of 16 products per output value of a 3x3x3 convolution with
    ci input channels (the channels padded to a multiple of 16)."""
    return 27 * ((ci + 15) // 16)


def _sq_conv(x, w, periodic):
    """conv3 of x >= 0 with w^2 (or |w| for absolute sums) and no bias."""
    return conv3(x, w, np.zeros(w.shape[0]), periodic)


def _var(S, D):
    """Variance an input error of scale S and bound D contributes downstream."""
    return S * S + D * D


def _layer(v, Sv, Dv, w, b, ci, periodic, uw):
    """A convolution with BF16 weights and inputs, FP32 accumulation, bias
    added in FP32; uw: the weights' relative rounding error (U_BF16, or 0
    for BF16-valued weights).  Returns the exact output and its (S, D)."""
    a = conv3(v, w, b, periodic)
    w2 = w * w
    # input errors and the weights' BF16 rounding (uw |w| per weight)
    S2 = _sq_conv(_var(Sv, Dv), w2, periodic) + uw ** 2 * _sq_conv(v * v, w2, periodic)
    S = np.sqrt(S2)
    A = _sq_conv(np.abs(v), np.abs(w), periodic) + K_SECOND * S
    D = _mma_steps(ci) * ACC_MMA * A + 2.0 ** -23 * (np.abs(a) + A + np.abs(b)[:, None, None, None])
    return a, S, D


def forward_scales(p, W, norm, periodic, gamma, U, weights_exact=False):
    """forward() with error scales.  W: primitives, U: the conserved state
    they come from (the library converts U to primitives in FP32, then
    normalises and rounds to BF16).  Returns {x, h1, h2, o} (o = phi /
    out_scale, the raw network output), the pre-activations a1, a2 and
    S*, D* of x, h1, h2 and o."""
    mean = norm["in_mean"][:, None, None, None]
    scale = norm["in_scale"][:, None, None, None]
    x = (W - mean) / scale
    # FP32 primitives are a few ulp off (the pressure cancels against the
    # kinetic energy, so its error scales with E), then the FP32 normalisation
    ke = 0.5 * W[0] * (W[1] ** 2 + W[2] ** 2 + W[3] ** 2)
    mag = np.abs(W) + np.abs(mean)
    mag[4] += (gamma - 1.0) * (np.abs(U[4]) + ke)
    out = {"x": x, "Sx": U_BF16 * np.abs(x), "Dx": (1 + U_BF16) * 2.0 ** -20 * mag / scale}
    v, Sv, Dv = x, out["Sx"], out["Dx"]
    for layer, (wk, bk, ci) in enumerate((("w1", "b1", C_IN), ("w2", "b2", C_HID),
                                          ("w3", "b3", C_HID))):
        a, Sa, Da = _layer(v, Sv, Dv, p[wk], p[bk], ci, periodic,
                           0.0 if weights_exact else U_BF16)
        if layer < 2:
            h = np.tanh(a)
            d = 1.0 - h * h
            # the slope of tanh over |a| +- Da is at most sech^2(max(0, |a| - Da))
            dmax = 1.0 - np.tanh(np.maximum(0.0, np.abs(a) - Da)) ** 2
            Sh = np.sqrt((d * Sa) ** 2 + (U_BF16 * h) ** 2)
            # (second order in Sa: the slope changes by at most 2 |a| Sa-ish;
            # bounded by taking the slope's maximum over |a| +- (Da + K Sa))
            dmx = 1.0 - np.tanh(np.maximum(0.0, np.abs(a) - Da - K_SECOND * Sa)) ** 2
            Dh = (1 + U_BF16) * (dmax * Da + (dmx - d) * K_SECOND * Sa + TANH_ABS)
            n = str(layer + 1)
            out["a" + n], out["h" + n], out["Sh" + n], out["Dh" + n] = a, h, Sh, Dh
            v, Sv, Dv = h, Sh, Dh
        else:
            out["o"], out["So"], out["Do"] = a, Sa, Da
    return out


def _stencil(f, dt, inv_d, scale, periodic, weights):
    """dt scale sum_d inv_d^k (w0 f(i+e) + w1 f(i) + w0 f(i-e)) for f >= 0."""
    fp = pad(f, periodic)
    c = fp[:, 1:-1, 1:-1, 1:-1]
    out = np.zeros_like(f)
    k, w0, w1 = weights
    for a in range(3):
        axis = 3 - a
        lo = [slice(None), slice(1, -1), slice(1, -1), slice(1, -1)]
        hi = list(lo)
        lo[axis] = slice(0, -2)
        hi[axis] = slice(2, None)
        out += inv_d[a] ** k * (w0 * fp[tuple(hi)] + w1 * c + w0 * fp[tuple(lo)])
    return (dt * scale[:, None, None, None]) ** k * out


def _through_stencil(f, Sf, Df, dt, inv_d, scale, periodic):
    """(S, D) of the FP32 stencil dt scale sum_d inv_d (f(i+e) - 2 f(i) + f(i-e))
    (the correction and its adjoint) from f's (S, D)."""
    S = np.sqrt(_stencil(_var(Sf, Df), dt, inv_d, scale, periodic, (2, 1.0, 4.0)))
    Sabs = _stencil(np.abs(f) + Df + K_SECOND * Sf, dt, inv_d, scale, periodic, (1, 1.0, 2.0))
    return S, 2.0 ** -20 * Sabs


def backward_scales(p, fw, r, dt, inv_d, norm, periodic, weights_exact=False):
    """loss_and_grads() with error scales, from forward_scales()'s output fw
    and the FP64 residual r.  Returns the exact g_o (dL/do), g_a2 and g_a1
    (gradients of the tanh layers' pre-activations), grads (dict) and
    S*, D* of g_o, g_a2, g_a1 and of every gradient tensor (dicts S, D)."""
    osc, sig = norm["out_scale"], norm["res_scale"]
    sig4 = sig[:, None, None, None]
    o = fw["o"]
    phi = osc[:, None, None, None] * o
    dU = laplacian_update(phi, dt, inv_d, periodic)
    n = dU.size
    e = (dU - r) / sig4
    g_dU = 2.0 * e / sig4 / n
    g_o = laplacian_update_adjoint(g_dU, dt, inv_d, periodic) * osc[:, None, None, None]
    # the loss kernel: dU by the FP32 stencil, e = (dU - r) / sigma, 2 e / (sigma N)
    Sdu, Ddu = _through_stencil(o, fw["So"], fw["Do"], dt, inv_d, osc, periodic)
    Se = Sdu / sig4
    De = (1 + 2.0 ** -21) * (Ddu + 2.0 ** -23 * (np.abs(dU) + np.abs(r) + Ddu
                                                  + K_SECOND * Sdu)) / sig4 \
        + 2.0 ** -22 * (np.abs(e) + K_SECOND * Se)
    Sg = 2.0 * Se / (sig4 * n)
    Dg = (1 + 2.0 ** -22) * 2.0 * De / (sig4 * n) + 2.0 ** -22 * (np.abs(g_dU) + K_SECOND * Sg)
    # its adjoint: the same stencil
    Sgo, Dgo = _through_stencil(g_dU, Sg, Dg, dt, inv_d, osc, periodic)
    out = {"g_o": g_o, "Sgo": Sgo, "Dgo": Dgo, "e": e, "Se": Se, "De": De}
    u2 = U_BF16 ** 2
    grads, S, D = {}, {}, {}
    gout, Sgout, Dgout = g_o, Sgo, Dgo
    ncell = g_o[0].size
    # tensor-memory accumulation of a tile (4 planes x 8 MMAs of 16 cells),
    # then the per-tile partials added in FP32 in tile order
    wg_acc = 32 * ACC_MMA + (-(-ncell // 512)) * 2.0 ** -24
    for wk, bk, ik, ci in (("w3", "b3", "2", C_HID), ("w2", "b2", "1", C_HID),
                           ("w1", "b1", "", C_IN)):
        xin = fw["h" + ik] if ik else fw["x"]
        Sin = fw["Sh" + ik] if ik else fw["Sx"]
        Din = fw["Dh" + ik] if ik else fw["Dx"]
        grads[wk] = conv3_weight_grad(xin, gout, periodic)
        grads[bk] = gout.sum(axis=(1, 2, 3))
        # sum over cells of bf(g_dev) in_dev: the gradient's BF16 rounding and
        # the errors of both factors, then the accumulation
        vg, vi = _var(Sgout, Dgout), _var(Sin, Din)
        S2 = conv3_weight_grad(xin * xin, vg + u2 * gout * gout, periodic) \
            + conv3_weight_grad(vi, gout * gout, periodic)
        S[wk] = np.sqrt(S2)
        ag = np.abs(gout) + K_SECOND * np.sqrt(vg)
        ai = np.abs(xin) + K_SECOND * np.sqrt(vi)
        D[wk] = wg_acc * (1 + U_BF16) * conv3_weight_grad(ai, ag, periodic) \
            + K_SECOND ** 2 * conv3_weight_grad(np.sqrt(vi), np.sqrt(vg), periodic) / ncell ** 0.5
        S[bk] = np.sqrt(vg.sum(axis=(1, 2, 3)))
        D[bk] = (5 + -(-ncell // 512)) * 2.0 ** -24 * ag.sum(axis=(1, 2, 3))
        if wk == "w1":
            break
        # the input gradient: the adjoint convolution of bf(g_dev) with the
        # BF16 weights (FP32 output), then g_a = g_h (1 - y^2), y the layer's
        # BF16 activation
        w = p[wk]
        g_h = conv3_input_grad(w, gout, periodic)
        uw2 = 0.0 if weights_exact else u2
        Sgh = np.sqrt(conv3_input_grad(w * w, vg + (u2 + uw2) * gout * gout, periodic))
        Dgh = _mma_steps(C_OUT if wk == "w3" else C_HID) * ACC_MMA * (1 + U_BF16) ** 2 \
            * (conv3_input_grad(np.abs(w), np.abs(gout), periodic) + K_SECOND * Sgh)
        h, Sh, Dh = fw["h" + ik], fw["Sh" + ik], fw["Dh" + ik]
        d = 1.0 - h * h
        g_a = g_h * d
        # |y^2 - h^2| beyond its random linear part 2 h dy, with |dy| up to
        # Dh + K_SECOND Sh, and the products of two errors likewise
        Sga = np.sqrt((d * Sgh) ** 2 + (d * Dgh) ** 2 + (2.0 * h * g_h) ** 2 * _var(Sh, Dh))
        # second-order terms: |y^2 - h^2 - 2 h dy| = dy^2 and dg dy, with
        # |dy| <= Dh + K Sh and |dg| <= Dgh + K Sgh; the FP32 multiply
        ey, eg = Dh + K_SECOND * Sh, Dgh + K_SECOND * Sgh
        Dga = (np.abs(g_h) + eg) * ey * ey + eg * 2.0 * (np.abs(h) + ey) * ey \
            + 2.0 ** -22 * (np.abs(g_h) + eg) * (np.abs(d) + 2.0 * np.abs(h) * ey + ey * ey)
        out["g_a" + ik], out["Sg" + ik], out["Dg" + ik] = g_a, Sga, Dga
        gout, Sgout, Dgout = g_a, Sga, Dga
    out["grads"], out["S"], out["D"] = grads, S, D
    return out
