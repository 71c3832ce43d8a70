"""FP32-bulk path (FV_PREC_FP32_BULK): FP32 reconstruction and fluxes on an
FP64 state.  It is not bitwise, so it is checked by its error against the FP64
oracle on the same seeded inputs, per field, and by the invariants that stay
exact in any precision: uniform states, zero transverse momentum of a planar
problem, identical lines of a planar problem, round-off conservation.

Error measures per field q after the run:
  linf_rel[q] = max|gpu - oracle| / max|oracle|
  l1_rel[q]   = sum|gpu - oracle| / sum|oracle|
"""
import math

import numpy as np
import pytest

import oracle
from paper_1812_07977_gb300 import problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUT, PER = 0, 1


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def _mesh32(n, bc=(OUT, OUT, OUT), theta=2.0):
    from paper_1812_07977_gb300.fv import Mesh
    return Mesh(*n, theta=theta, bc=tuple("periodic" if b == PER else "outflow" for b in bc),
                precision="fp32_bulk")


def _errors(got, ref):
    d = np.abs(got - ref).reshape(5, -1)
    r = np.abs(ref).reshape(5, -1)
    linf = d.max(1) / np.maximum(r.max(1), 1e-300)
    l1 = d.sum(1) / np.maximum(r.sum(1), 1e-300)
    return linf, l1


def _run_pair(n, U0, nsteps=None, t_end=None, bc=(OUT, OUT, OUT), theta=2.0):
    om = oracle.mesh(*n, theta=theta, bc=bc)
    Uo = oracle.ghosted_from_interior(om, U0)
    m = _mesh32(n, bc, theta)
    m.set_state(torch.from_numpy(np.ascontiguousarray(U0)).cuda())
    t, steps, dt_rel = 0.0, 0, 0.0
    while True:
        if nsteps is not None and steps >= nsteps:
            break
        if t_end is not None and not t < t_end:
            break
        dt = m.reduce_dt(0.4)
        dto, _, _ = oracle.reduce_dt(om, Uo, 0.4)
        dt_rel = max(dt_rel, abs(dt - dto) / dto)
        if t_end is not None:
            dto = min(dto, t_end - t)
        m.step(dto)                       # both advance with the oracle's dt
        oracle.step(om, Uo, dto)
        t += dto
        steps += 1
    got = m.get_state().cpu().numpy()
    m.close()
    return got, oracle.interior(Uo), dt_rel, steps


def test_sod_32_to_t02_error_against_fp64():
    n = (32, 32, 32)
    got, ref, dt_rel, steps = _run_pair(n, problems.riemann_planar(*n), t_end=0.2)
    linf, l1 = _errors(got, ref)
    print("sod32 fp32_bulk linf", linf, "l1", l1, "dt", dt_rel, "steps", steps)
    assert dt_rel < 1e-6
    for q in (0, 1, 4):
        assert l1[q] < 2e-6 and linf[q] < 1e-4, (q, l1, linf)
    # planar problem: transverse momenta exactly zero, every (j, k) line equal
    assert not np.any(got[2]) and not np.any(got[3])
    assert np.all(got == got[:, :1, :1, :])


def test_oblique_ragged_error_against_fp64():
    n = (45, 38, 33)
    got, ref, _, _ = _run_pair(n, problems.riemann_oblique(*n), nsteps=20)
    linf, l1 = _errors(got, ref)
    print("oblique fp32_bulk linf", linf, "l1", l1)
    assert np.all(l1 < 2e-6) and np.all(linf < 1e-4), (l1, linf)


@pytest.mark.parametrize("theta", [1.0, 0.0])
def test_other_limiters(theta):
    n = (24, 20, 18)
    got, ref, _, _ = _run_pair(n, problems.random_smooth_periodic(*n, seed=8), nsteps=10,
                               bc=(PER, PER, PER), theta=theta)
    linf, l1 = _errors(got, ref)
    assert np.all(l1 < 2e-6) and np.all(linf < 2e-5), (l1, linf)


def test_uniform_state_preserved_exactly():
    n = (33, 10, 9)
    U0 = problems.uniform(*n, 0.7, (0.3, -1.1, 0.25), 1.9)
    m = _mesh32(n)
    m.set_state(U0)
    for _ in range(4):
        m.step(m.reduce_dt(0.4))
    assert np.array_equal(m.get_state().cpu().numpy(), U0)
    m.close()


def test_flux_reuse_is_exact_and_counts_fallbacks():
    """Uniform regions with a block of equal non-physical cells (every face
    there falls back): the fused kernel reuses fluxes along z (runs of equal
    cells) and across planes (faces whose four cells equal the previous
    plane's).  One plane per z chunk turns the plane-to-plane reuse off; the
    state must not change by a bit, and the counts must match the oracle's."""
    n = (40, 36, 33)
    nx, ny, nz = n
    U0 = problems.uniform(nx, ny, nz, 1.0, (0.2, -0.1, 0.05), 1.0)
    U0[4, 10:22, 5:30, 8:20] = -1.0
    U0[0, :, 20:, :] = 0.5
    om = oracle.mesh(*n)
    Uo = oracle.ghosted_from_interior(om, U0)
    _, bad, fb = oracle.compute_update(om, Uo, 1e-3)
    from paper_1812_07977_gb300.fv import FvError, ERR_NONPHYSICAL
    out = []
    for kchunk in (32, 1):
        m = _mesh32(n)
        m.set_tuning("kchunk", kchunk)
        m.set_state(U0)
        m.substep(1, 1e-3)
        st = torch.empty(U0.shape, dtype=torch.float64, device="cuda")
        with pytest.raises(FvError) as e:  # the state is copied, then the latch reported
            m.get_state(st)
        assert e.value.status == ERR_NONPHYSICAL
        out.append((st.cpu().numpy(), m.counters(), m.face_counts()))
        m.close()
    (a, ca, fa), (b, cb, fbc) = out
    assert np.array_equal(a, b, equal_nan=True)
    assert ca == cb == (bad, fb)
    assert fa[0] < fbc[0]          # the plane-to-plane reuse did skip faces


@pytest.mark.parametrize("theta", [2.0, 1.5])
def test_stage2_cfl_maximum_same_dt(theta):
    """The second substep takes the CFL maximum of the state it writes;
    fv_reduce_dt then uses it instead of its own pass.  A run that does and
    one whose dt pass runs every step (fv_fill_ghosts in between drops the
    maximum) agree bit for bit on every dt and on the state; so does the
    first dt of a fresh mesh on the same state."""
    n = (37, 22, 19)
    runs = []
    for refresh in (False, True):
        m = _mesh32(n, theta=theta)
        m.set_state(problems.riemann_oblique(*n))
        dts = []
        for _ in range(6):
            dts.append(m.reduce_dt(0.4))
            if refresh:
                m.fill_ghosts()
            m.step(dts[-1])
        dts.append(m.reduce_dt(0.4))
        runs.append((dts, m.get_state().cpu().numpy(), m.counters()))
        m.close()
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1].view(np.uint64), runs[1][1].view(np.uint64))
    assert runs[0][2] == runs[1][2]
    m = _mesh32(n, theta=theta)
    m.set_state(runs[0][1])
    assert m.reduce_dt(0.4) == runs[0][0][-1]
    m.close()


@pytest.mark.parametrize("shape", [(32, 8), (32, 4), (32, 16), (64, 4), (64, 8), (128, 4)])
def test_tile_shapes_same_bits(shape):
    """The fused kernel built for tiles of 32 to 128 columns by 4 to 16 rows
    (128 to 512 threads; the short tiles have more halo cells than threads)
    gives the default 16 x 8 tile's bits, dt and counts, on a ragged mesh
    with z chunks."""
    n = (45, 38, 33)
    out = []
    for tx, ty in ((16, 8), shape):
        m = _mesh32(n)
        # through built shapes only: width 32 first, then the height
        m.set_tuning("tile_x", 32)
        m.set_tuning("tile_y", ty)
        m.set_tuning("tile_x", tx)
        m.set_tuning("kchunk", 7)
        m.set_state(problems.riemann_oblique(*n))
        dts = []
        for _ in range(4):
            dts.append(m.reduce_dt(0.4))
            m.step(dts[-1])
        out.append((dts, m.get_state().cpu().numpy(), m.counters()))
        m.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1].view(np.uint64), out[1][1].view(np.uint64))
    assert out[0][2] == out[1][2]


@pytest.mark.parametrize("n,bc", [((45, 38, 33), (OUT, OUT, OUT)), ((45, 38, 33), (PER, PER, PER)),
                                  ((3, 1, 2), (OUT, PER, OUT)), ((2, 5, 1), (PER, OUT, PER)),
                                  ((1, 1, 1), (OUT, OUT, OUT)), ((1, 2, 3), (PER, PER, PER))])
def test_ghosts_filled_after_each_substep(n, bc):
    """After each substep the ghost cells of its output hold their source
    cells: the ghosted state is unchanged by another ghost fill (outflow,
    periodic and axes of 1-3 cells)."""
    m = _mesh32(n, bc=bc)
    U0 = (problems.random_smooth_periodic(*n, seed=4) if PER in bc
          else problems.riemann_oblique(*n))
    m.set_state(U0)
    for _ in range(2):
        m.step(m.reduce_dt(0.4))
    a = m.get_ghosted_state().cpu().numpy()
    m.fill_ghosts()
    b = m.get_ghosted_state().cpu().numpy()
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    m.substep(1, 1e-4)                 # the stage-1 output (U1) as well
    a = m.get_ghosted_state().cpu().numpy()
    m.fill_ghosts()
    b = m.get_ghosted_state().cpu().numpy()
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    m.close()


def test_conservation_periodic():
    n = (20, 16, 24)
    U0 = problems.random_smooth_periodic(*n, seed=99)
    m = _mesh32(n, bc=(PER, PER, PER))
    m.set_state(U0)
    s0 = m.conserved_sums()
    for _ in range(40):
        m.step(m.reduce_dt(0.4))
    s1 = m.conserved_sums()
    scale = np.abs(U0).reshape(5, -1).mean(1)
    drift = np.abs(s1 - s0) / scale
    print("fp32_bulk conservation drift", drift)
    assert np.all(drift < 1e-9), drift
    m.close()


def test_near_vacuum_pressure_recovered_in_fp64():
    """A fast, cold flow (kinetic energy 99.95% of E): (gamma-1)(E - ke) in
    FP32 loses ~3 digits of p.  The FP64 recovery of the cell pressures makes
    the pressure error after 5 steps smaller than with the recovery turned off
    (measured 1.6e-4 against 2.7e-4); what remains comes from the FP32 energy
    fluxes, which carry the kinetic energy's rounding into E."""
    n = (32, 8, 8)
    x = problems.cell_centres(32)
    rho = np.broadcast_to(1.0 + 0.1 * np.sin(2 * math.pi * x), (8, 8, 32))
    p = np.broadcast_to(0.01 * (1.0 + 0.2 * np.cos(2 * math.pi * x)), (8, 8, 32))
    U0 = problems.conserved_from_primitive(rho, 10.0, 0.0, 0.0, p)

    def pressure(U):
        ke = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
        return 0.4 * (U[4] - ke)

    errs = {}
    for ratio in (0.99, 2.0):
        om = oracle.mesh(*n, bc=(PER, PER, PER))
        Uo = oracle.ghosted_from_interior(om, U0)
        m = _mesh32(n, bc=(PER, PER, PER))
        m.set_tuning("vacuum_ratio", ratio)
        m.set_state(U0)
        for _ in range(5):
            dt = oracle.reduce_dt(om, Uo, 0.4)[0]
            m.step(dt)
            oracle.step(om, Uo, dt)
        got = m.get_state().cpu().numpy()
        m.close()
        ref = oracle.interior(Uo)
        errs[ratio] = np.abs(pressure(got) - pressure(ref)).max() / np.abs(pressure(ref)).max()
    print("near-vacuum pressure error: recovery on", errs[0.99], "off", errs[2.0])
    assert errs[0.99] < 5e-4
    assert errs[0.99] < 0.8 * errs[2.0], errs


def test_fp32_full_size_sampled_windows():
    """The timed workload at 256^3 in the benchmark's launch configuration:
    after two steps, 8^3 windows against the FP64 oracle on the sub-box
    around each (dependence radius 4 cells per step)."""
    n = 256
    U0 = problems.riemann_oblique(n, n, n)
    from paper_1812_07977_gb300.fv import Mesh
    m = Mesh(n, n, n, precision="fp32_bulk")
    m.set_state(torch.from_numpy(U0).cuda())
    dts = []
    for _ in range(2):
        dt = m.reduce_dt(0.4)
        dts.append(dt)
        m.step(dt)
    got = m.get_state().cpu().numpy()
    m.close()
    halo, w = 8, 8
    for (i0, j0, k0) in [(0, 0, 0), (124, 124, 124), (128, 120, 131), (n - w,) * 3, (60, 200, 128)]:
        lo = [max(0, c - halo) for c in (i0, j0, k0)]
        hi = [min(n, c + w + halo) for c in (i0, j0, k0)]
        sub = np.ascontiguousarray(U0[:, lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]])
        ns = [hi[a] - lo[a] for a in range(3)]
        om = oracle.mesh(*ns, lx=ns[0] / n, ly=ns[1] / n, lz=ns[2] / n)
        Uo = oracle.ghosted_from_interior(om, sub)
        for dt in dts:
            oracle.step(om, Uo, dt)
        ref = oracle.interior(Uo)[:, k0 - lo[2]:k0 - lo[2] + w, j0 - lo[1]:j0 - lo[1] + w,
                                  i0 - lo[0]:i0 - lo[0] + w]
        win = got[:, k0:k0 + w, j0:j0 + w, i0:i0 + w]
        err = np.abs(win - ref).reshape(5, -1).max(1) / np.abs(U0).max()
        assert np.all(err < 1e-5), ((i0, j0, k0), err)


def test_integer_conversions_match_hardware(tmp_path):
    """d2f / f2d (the FP32-bulk path's integer-pipe conversions) equal the
    hardware conversions bit for bit on edge cases and 2^26 random inputs."""
    import os
    import subprocess
    from paper_1812_07977_gb300.build import ARCH, CSRC, INCLUDE, nvcc
    here = os.path.dirname(os.path.abspath(__file__))
    exe = str(tmp_path / "conversions_check")
    subprocess.run([nvcc(), *ARCH, "-O3", "-std=c++17", "-I", CSRC, "-I", INCLUDE,
                    os.path.join(here, "cuda", "conversions_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0 and "mismatches 0" in r.stdout, r.stdout + r.stderr


def test_fp32_bulk_dt_is_the_oracles_bitwise():
    """FP64 is kept for the CFL time step: the FP32-bulk path takes every
    cell's speed in FP64 (the FP64 method's operations; FP32 interval bounds
    only skip cells that cannot raise the maximum), so its dt is the
    oracle's, bit for bit -- from the separate pass after set_state, on
    states whose speeds span many orders of magnitude, near ties and operands
    outside the bound's range, and from stage 2's maximum of the state it
    writes."""
    from test_gpu_parity import _wide_range_states
    from paper_1812_07977_gb300.fv import Mesh
    n = (128, 120, 96)
    for seed, U0 in enumerate(_wide_range_states(*n, seed=3)):
        om = oracle.mesh(*n, ly=2.0)
        dto, _, bad = oracle.reduce_dt(om, oracle.ghosted_from_interior(om, U0), 0.4)
        with Mesh(*n, ly=2.0, precision="fp32_bulk") as m:
            m.set_state(U0)
            assert m.reduce_dt(0.4) == dto, seed
            assert m.counters()[0] == bad
    for U0, bc in ((problems.riemann_oblique(33, 17, 9), (OUT, OUT, OUT)),
                   (problems.random_smooth_periodic(20, 24, 16, seed=11), (PER, PER, PER))):
        nn = U0.shape[1:][::-1]
        om = oracle.mesh(*nn, bc=bc)
        m = _mesh32(nn, bc)
        m.set_state(U0)
        for _ in range(4):
            dt = m.reduce_dt(0.4)        # after the first step: stage 2's maximum
            U = m.get_state().cpu().numpy()
            dto, _, _ = oracle.reduce_dt(om, oracle.ghosted_from_interior(om, U), 0.4)
            assert dt == dto
            m.step(dt)
        m.close()


def test_tile_shape_changes_must_stay_built():
    """Width, height and occupancy changes that would leave the built shapes
    are rejected, and the mesh keeps its shape."""
    from paper_1812_07977_gb300.fv import FvError
    m = _mesh32((16, 16, 16))
    with pytest.raises(FvError):
        m.set_tuning("tile_x", 128)     # (128, 8) is not built
    with pytest.raises(FvError):
        m.set_tuning("tile_y", 4)       # (16, 4) is not built
    m.set_tuning("tile_x", 32)
    m.set_tuning("tile_y", 4)
    m.set_tuning("tile_x", 128)
    with pytest.raises(FvError):
        m.set_tuning("occupancy", 3)
    with pytest.raises(FvError):
        m.set_tuning("tile_x", 48)
    m.close()

