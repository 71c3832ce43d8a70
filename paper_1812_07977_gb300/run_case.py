"""Run a fixed number of RK2 steps of one workload at one precision and
print the face counts, the time per step and a digest of the final state:
the small, deterministic command that profilers (ncu) and timing runs wrap.

    python -m paper_1812_07977_gb300.run_case PRECISION N STATE STEPS [FUSED]
        [--warmup W] [--tune KEY=VALUE ...]

PRECISION  fp64 | fp64_fma | fp64_ff | fp32_bulk
N          cells per axis of the N^3 mesh
STATE      oblique  -- the oblique Sod problem (plane normal (1,1,1)/sqrt 3,
                       outflow boundaries): long runs of equal cells, so most
                       faces reuse their neighbour's flux
           smooth   -- a seeded random smooth periodic state: no two
                       neighbours equal, every face evaluated
           uniform  -- the Sod left state everywhere (outflow): every face
                       reuses its neighbour's flux, the per-cell floor
STEPS      RK2 steps, each with its CFL time step (Courant number 0.4), timed
           with CUDA events on the mesh's stream
FUSED      for fp64 / fp64_fma: 1 = the fused per-tile substep kernel,
           0 = the per-axis sweeps (default 1)
--warmup W untimed steps first (the timed steps continue from their state)
--tune     Mesh.set_tuning keys (kchunk, occupancy, tile_y, ...), applied
           after the mesh is created
"""
from __future__ import annotations

import argparse
import hashlib
import sys

import torch

from . import problems
from .fv import Mesh


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(usage=__doc__)
    ap.add_argument("precision")
    ap.add_argument("n", type=int)
    ap.add_argument("state", choices=["oblique", "smooth", "uniform"])
    ap.add_argument("steps", type=int)
    ap.add_argument("fused", type=int, nargs="?", default=1)
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--tune", action="append", default=[])
    a = ap.parse_args(sys.argv[1:] if argv is None else argv)
    n = a.n
    torch.cuda.set_device(0)
    if a.state == "smooth":
        U0 = problems.random_smooth_periodic(n, n, n, seed=12345)
        bc = ("periodic",) * 3
    elif a.state == "uniform":
        U0 = problems.uniform(n, n, n, 1.0, (0.0, 0.0, 0.0), 1.0)
        bc = ("outflow",) * 3
    else:
        U0 = problems.riemann_oblique(n, n, n)
        bc = ("outflow",) * 3
    m = Mesh(n, n, n, precision=a.precision, bc=bc)
    if a.precision in ("fp64", "fp64_fma"):
        m.set_tuning("fp64_fused", a.fused)
    for kv in a.tune:
        key, value = kv.split("=", 1)
        m.set_tuning(key, int(value))
    m.set_state(torch.from_numpy(U0).cuda())
    for _ in range(a.warmup):
        m.step(m.reduce_dt(0.4))
    stream = m.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(a.steps):
        m.step(m.reduce_dt(0.4))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(a.steps, 1)
    digest = hashlib.sha256(m.get_state().cpu().numpy().tobytes()).hexdigest()[:16]
    print("ok", a.precision, n, a.state, a.steps, "tune", a.tune, "faces", m.face_counts(),
          f"ms_per_step {ms:.4f}", f"Gzu_s {n ** 3 / ms / 1e6:.4f}", "bits", digest)
    return 0


if __name__ == "__main__":
    sys.exit(main())
