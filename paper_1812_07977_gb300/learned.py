"""Training and evaluation of the learned flux correction (fv_net_* in
include/fv.h) on the solver's own fine-mesh runs.

Data: fine runs of a periodic shear layer (FP64 solver) are block-averaged
onto the coarse mesh.  Each sample is a coarse state Uc(t) = avg(Uf(t)), the
coarse CFL step dt, and the residual r = avg(Uf(t + dt)) - RK2coarse(Uc(t), dt):
what the coarse solver misses over one of its steps.  The network is trained
(by the library's own forward/backward kernels and Adam) so that its
correction dU matches r.  Evaluation runs the coarse solver with and without
the correction on a held-out perturbation amplitude, on the same time steps
as a fine reference run, and reports the L1 density error of each: the plain
solver is both the fallback (a corrected step that produces a non-physical
cell is redone without the correction) and the arbiter of the gain.

Tensor reshaping and averaging here are data preparation on the GPU (torch);
the solver steps and every network pass run in the library's kernels.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import problems
from .fv import FvError, Mesh, Net

PERIODIC = ("periodic",) * 3


def block_average(U, f: int):
    """(5, nz, ny, nx) conserved fields averaged over f^3 blocks (the exact
    cell averages of the coarse mesh)."""
    q, nz, ny, nx = U.shape
    return U.reshape(q, nz // f, f, ny // f, f, nx // f, f).mean(dim=(2, 4, 6)).contiguous()


def primitives(U, gamma):
    rho = U[0]
    v = U[1:4] / rho
    p = (gamma - 1.0) * (U[4] - 0.5 * rho * (v * v).sum(0))
    return rho, v, p


def advance(mesh: Mesh, dt_total: float, cfl: float) -> int:
    """Advance a mesh by exactly dt_total with CFL-limited steps."""
    t, n = 0.0, 0
    while t < dt_total:
        dt = min(mesh.reduce_dt(cfl), dt_total - t)
        mesh.step(dt)
        t += dt
        n += 1
    return n


def generate(fine_n: int, factor: int, amplitudes, samples: int, cfl: float = 0.4,
             gamma: float = 1.4, precision: str = "fp64_fma", every: int = 1,
             rollout: bool = False):
    """Training samples from fine runs (one per amplitude); a sample every
    `every` coarse steps.  Each sample's input is the averaged fine state and
    its target the coarse step's residual against the averaged fine state
    one step later.  With `rollout`, a plain coarse run advances on the same
    steps and adds samples whose input is its own (drifted) state and whose
    target brings it back to the averaged fine state, so the network also
    learns from the states a coarse run actually visits.  Returns a list of
    (Uc, dt, residual) CUDA tensors and the number of fine steps taken."""
    import torch
    cn = fine_n // factor
    data = []
    fine_steps = 0
    for amp in amplitudes:
        fine = Mesh(fine_n, fine_n, fine_n, gamma=gamma, bc=PERIODIC, precision=precision)
        coarse = Mesh(cn, cn, cn, gamma=gamma, bc=PERIODIC, precision=precision)
        drift = Mesh(cn, cn, cn, gamma=gamma, bc=PERIODIC, precision=precision)
        fine.set_state(torch.from_numpy(problems.shear_layer(fine_n, amp, gamma=gamma)).cuda())
        drift.set_state(block_average(fine.get_state(), factor))
        for s in range(samples * every):
            Uc = block_average(fine.get_state(), factor)
            coarse.set_state(Uc)
            dt = coarse.reduce_dt(cfl)
            coarse.step(dt)
            stepped = coarse.get_state()
            Ud = drift.get_state().clone()
            drift.step(dt)
            fine_steps += advance(fine, dt, cfl)
            target = block_average(fine.get_state(), factor)
            if s % every == 0:
                data.append((Uc, dt, (target - stepped).contiguous()))
                if rollout:
                    data.append((Ud, dt, (target - drift.get_state()).contiguous()))
        for m in (fine, coarse, drift):
            m.close()
    return data, fine_steps


def fit_scales(data, gamma: float = 1.4):
    """Input normalisation, residual scale and output scale from the data."""
    import torch
    def prims(U):
        rho, v, p = primitives(U, gamma)
        return torch.stack([rho, v[0], v[1], v[2], p])

    W = torch.stack([prims(U) for U, _, _ in data])
    in_mean = W.mean(dim=(0, 2, 3, 4)).cpu().numpy()
    in_scale = np.maximum(W.std(dim=(0, 2, 3, 4)).cpu().numpy(), 1e-6)
    R = torch.stack([r for _, _, r in data])
    res_scale = np.maximum(R.std(dim=(0, 2, 3, 4)).cpu().numpy(), 1e-12)
    n = data[0][0].shape[-1]
    dt = float(np.mean([d for _, d, _ in data]))
    # the correction is ~ 12 (dt / dx) * |phi| for an O(1) network output
    out_scale = res_scale / (12.0 * dt * n)
    return in_mean, in_scale, out_scale, res_scale


def reference_run(fine_n: int, factor: int, amp: float, nsteps: int, cfl: float = 0.4,
                  gamma: float = 1.4, precision: str = "fp64_fma"):
    """A fine run averaged to the coarse mesh on the plain coarse run's time
    steps: (initial coarse state, [(dt, averaged fine state after the step)],
    the plain coarse run's L1 density errors)."""
    import torch
    cn = fine_n // factor
    U0 = torch.from_numpy(problems.shear_layer(fine_n, amp, gamma=gamma)).cuda()
    fine = Mesh(fine_n, fine_n, fine_n, gamma=gamma, bc=PERIODIC, precision=precision)
    plain = Mesh(cn, cn, cn, gamma=gamma, bc=PERIODIC, precision=precision)
    fine.set_state(U0)
    Uc0 = block_average(U0, factor)
    plain.set_state(Uc0)
    steps, err = [], []
    for _ in range(nsteps):
        dt = plain.reduce_dt(cfl)
        plain.step(dt)
        advance(fine, dt, cfl)
        ref = block_average(fine.get_state(), factor)
        steps.append((dt, ref))
        err.append(float((plain.get_state()[0] - ref[0]).abs().mean()))
    fine.close()
    plain.close()
    return Uc0, steps, err


def rollout_error(net: Net, ref, gamma: float = 1.4, precision: str = "fp64_fma",
                  timing: bool = False):
    """L1 density errors of the corrected coarse run against a reference
    run.  A corrected step that produces a non-physical cell is redone
    without the correction (the plain solver is the fallback)."""
    import torch
    Uc0, steps, _ = ref
    cn = Uc0.shape[-1]
    m = Mesh(cn, cn, cn, gamma=gamma, bc=PERIODIC, precision=precision)
    m.set_state(Uc0)
    err, fallbacks, t_net = [], 0, 0.0
    cur = Uc0.clone()
    for dt, target in steps:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.step(m, dt)
        bad = m.counters()[0]          # synchronises
        t_net += time.perf_counter() - t0
        if bad:
            fallbacks += 1
            m.set_state(cur)
            m.step(dt)
        try:
            cur = m.get_state()
        except FvError:                # non-physical even without the correction
            err.append(float("inf"))
            break
        err.append(float((cur[0] - target[0]).abs().mean()))
    m.close()
    out = {"l1_rho": err, "fallbacks": fallbacks}
    if timing:
        out["corrected_step_ms"] = 1e3 * t_net / max(len(steps), 1)
    return out


def train(net: Net, data, epochs: int, lr: float, gamma: float = 1.4, seed: int = 0,
          precision: str = "fp64_fma", val=None, log=None, noise: float = 0.0,
          denoise: bool = False):
    """Adam over the samples for `epochs` epochs.  With a validation
    reference run `val`, the parameters of the epoch with the lowest mean
    validation rollout error are kept (model selection against the plain solver).

    With `noise` > 0 each sample's input is perturbed by Gaussian noise of
    `noise` times each conserved field's standard deviation while the target
    stays the sample's residual: training-noise injection against the drift
    of long rollouts (as in Sanchez-Gonzalez et al. 2020, "Learning to
    Simulate Complex Physics with Graph Networks").  With `denoise`, the
    target instead becomes what brings the coarse step of the perturbed state
    to the averaged fine state; a flux-form correction cannot remove white
    noise, so that variant does not train."""
    import torch
    cn = data[0][0].shape[-1]
    mesh = Mesh(cn, cn, cn, gamma=gamma, bc=PERIODIC, precision=precision)
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device="cuda").manual_seed(seed)
    sd = torch.stack([U for U, _, _ in data]).std(dim=(0, 2, 3, 4))[:, None, None, None]
    losses, val_err = [], []
    best = (float("inf"), None, -1)
    t_train = 0.0   # the training steps only (each epoch's steps, to the host's read of their loss)
    steps = 0
    for ep in range(epochs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in rng.permutation(len(data)):
            Uc, dt, r = data[i]
            if noise > 0.0:
                Un = Uc + noise * sd * torch.randn(Uc.shape, generator=gen, device="cuda",
                                                   dtype=Uc.dtype)
                if denoise:
                    # target state = coarse step of Uc + r; the residual of
                    # the perturbed input against it
                    mesh.set_state(Uc)
                    mesh.step(dt)
                    target = mesh.get_state() + r
                    mesh.set_state(Un)
                    mesh.step(dt)
                    r = (target - mesh.get_state()).contiguous()
                Uc = Un
            mesh.set_state(Uc)
            net.train_step(mesh, r, dt, lr, sync=False)   # the loss stays on the device
            steps += 1
        tot, n = net.take_loss()
        t_train += time.perf_counter() - t0
        losses.append(tot / max(n, 1))
        if val is not None:
            e = float(np.mean(rollout_error(net, val, gamma, precision)["l1_rho"]))
            val_err.append(e)
            if e < best[0]:
                best = (e, net.params(), ep)
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4g}" + (f" val {val_err[-1]:.4g}" if val_err else ""))
    mesh.close()
    if best[1] is not None:
        net.set_params(best[1])
    return losses, t_train, steps, val_err, best[2]


def evaluate(net: Net, fine_n: int, factor: int, amp: float, nsteps: int, cfl: float = 0.4,
             gamma: float = 1.4, precision: str = "fp64_fma"):
    """L1 density error against the averaged fine run, plain vs corrected,
    on the plain coarse run's time steps."""
    ref = reference_run(fine_n, factor, amp, nsteps, cfl, gamma, precision)
    ro = rollout_error(net, ref, gamma, precision, timing=True)
    return {"l1_rho_plain": ref[2], "l1_rho_learned": ro["l1_rho"], "fallbacks": ro["fallbacks"],
            "corrected_step_ms": ro["corrected_step_ms"]}


def run(fine_n=256, factor=4, train_amps=(0.01, 0.04, 0.07, 0.1), val_amp=0.085,
        test_amp=0.055, samples=24, every=2, epochs=20, lr=1e-3, eval_steps=48, val_steps=16,
        seed=0, rollout=False, log=None, noise=0.0, denoise=False):
    """The whole workflow: data from fine runs, training with model selection
    on a validation amplitude, evaluation on a held-out test amplitude.  If no
    epoch's correction beats the plain solver on the validation run, the
    plain solver is kept (use_learned False).  Returns a summary."""
    t0 = time.perf_counter()
    data, fine_steps = generate(fine_n, factor, train_amps, samples, every=every, rollout=rollout)
    val = reference_run(fine_n, factor, val_amp, val_steps)
    t_data = time.perf_counter() - t0
    val_plain = float(np.mean(val[2]))
    with Net() as net:
        net.set_params(initial_params(seed, net.nparam, scale=0.5))
        net.set_scales(*fit_scales(data))
        losses, t_train, train_steps, val_err, best_ep = train(net, data, epochs, lr, seed=seed,
                                                               val=val, log=log, noise=noise,
                                                               denoise=denoise)
        ev = evaluate(net, fine_n, factor, test_amp, eval_steps)
    use = min(val_err) < val_plain
    return {"fine": fine_n, "coarse": fine_n // factor, "samples": len(data),
            "fine_steps_for_data": fine_steps, "data_s": t_data, "train_s": t_train,
            "train_steps": train_steps, "train_step_ms": 1e3 * t_train / max(train_steps, 1),
            "loss_first": losses[0], "loss_last": losses[-1], "best_epoch": best_ep,
            "val_l1_rho_plain": val_plain, "val_l1_rho_learned_best": min(val_err),
            "use_learned": bool(use), "noise": noise, **ev}


def initial_params(seed: int, nparam: int, scale: float = 1.0):
    """Seeded fan-in-scaled uniform weights, zero biases (SplitMix64), in the
    parameter order of include/fv.h."""
    g = problems.SplitMix64(seed)
    shapes = [((32, 5, 27), True), ((32,), False), ((32, 32, 27), True), ((32,), False),
              ((5, 32, 27), True), ((5,), False)]
    out = []
    for shape, is_w in shapes:
        n = int(np.prod(shape))
        if is_w:
            bound = scale * math.sqrt(3.0 / (shape[1] * 27))
            out.append((2.0 * g.uniform(n) - 1.0) * bound)
        else:
            out.append(np.zeros(n))
    flat = np.concatenate(out).astype(np.float32)
    assert flat.size == nparam
    return flat
