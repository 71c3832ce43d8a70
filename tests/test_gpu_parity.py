"""GPU parity: every stage of the CUDA path against the oracle on the same
seeded inputs, through the C ABI.

The FP64 path (FV_PREC_FP64) performs the method's operations in the
oracle's order without contraction, so the comparison is bitwise (equality,
which also satisfies the 1e-12 relative target).  The FMA-contracted
variant is held to the 1e-12 target: |gpu - oracle| <= 1e-12 * max|oracle|
per field (field-scale relative error; the momenta vanish in places, so an
elementwise relative error has no meaningful denominator there).
"""
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


def _pair(nx, ny, nz, U0, bc=(OUT, OUT, OUT), theta=2.0, precision="fp64", l=(1.0, 1.0, 1.0),
          gamma=1.4):
    from paper_1812_07977_gb300.fv import Mesh
    om = oracle.mesh(nx, ny, nz, lx=l[0], ly=l[1], lz=l[2], gamma=gamma, theta=theta, bc=bc)
    Uo = oracle.ghosted_from_interior(om, U0)
    m = Mesh(nx, ny, nz, lx=l[0], ly=l[1], lz=l[2], gamma=gamma, theta=theta,
             bc=tuple("periodic" if b == PER else "outflow" for b in bc), precision=precision)
    m.set_state(torch.from_numpy(np.ascontiguousarray(U0)).cuda())
    return om, Uo, m


def _field_rel_err(got, ref):
    scale = np.abs(ref).reshape(5, -1).max(1)
    return (np.abs(got - ref).reshape(5, -1).max(1) / np.maximum(scale, 1e-300))


def _run_both(om, Uo, m, nsteps, cfl=0.4):
    for _ in range(nsteps):
        dt = m.reduce_dt(cfl)
        dto, _, bad = oracle.reduce_dt(om, Uo, cfl)
        assert bad == 0
        assert dt == dto, (dt, dto)
        m.step(dt)
        oracle.step(om, Uo, dt)


SIZES = [(4, 4, 4), (5, 7, 3), (1, 9, 1), (33, 17, 9), (48, 40, 36)]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("bc", [(OUT, OUT, OUT), (PER, PER, PER), (PER, OUT, PER)])
def test_ghost_fill_bitwise(n, bc):
    nx, ny, nz = n
    rng = np.random.default_rng(nx * 100 + ny)
    U0 = rng.standard_normal((5, nz, ny, nx))
    om, Uo, m = _pair(nx, ny, nz, U0, bc=bc)
    got = m.get_ghosted_state().cpu().numpy()
    assert np.array_equal(got, Uo)
    m.close()


@pytest.mark.parametrize("n", SIZES)
def test_reduce_dt_bitwise(n):
    nx, ny, nz = n
    U0 = problems.random_smooth_periodic(nx, ny, nz, seed=5)
    om, Uo, m = _pair(nx, ny, nz, U0, l=(1.0, 2.0, 0.5))
    dt = m.reduce_dt(0.4)
    dto, _, _ = oracle.reduce_dt(om, Uo, 0.4)
    assert dt == dto
    m.close()


@pytest.mark.parametrize("n", [(5, 7, 3), (33, 17, 9), (48, 40, 36)])
@pytest.mark.parametrize("theta", [2.0, 1.0, 0.0, 1.3])
def test_substep1_bitwise(n, theta):
    nx, ny, nz = n
    U0 = problems.random_smooth_periodic(nx, ny, nz, seed=17)
    om, Uo, m = _pair(nx, ny, nz, U0, theta=theta, bc=(PER, OUT, PER))
    dt = 0.3 * oracle.reduce_dt(om, Uo, 0.4)[0]
    dU, bad, fb = oracle.compute_update(om, Uo, dt)
    m.substep(1, dt)
    got = m.get_state().cpu().numpy()
    ref = oracle.interior(Uo) + oracle.interior(dU)
    assert np.array_equal(got, ref)
    m.substep(2, dt)
    m.close()


def test_sod_32_to_t02_bitwise():
    """Plain FP64 3D Sod shock tube, 32^3, outflow, CFL 0.4, to t = 0.2."""
    n = 32
    U0 = problems.riemann_planar(n, n, n)
    om, Uo, m = _pair(n, n, n, U0)
    t = 0.0
    steps = 0
    while t < 0.2:
        dt = m.reduce_dt(0.4)
        dto, _, _ = oracle.reduce_dt(om, Uo, 0.4)
        assert dt == dto
        dt = min(dt, 0.2 - t)
        m.step(dt)
        oracle.step(om, Uo, dt)
        t += dt
        steps += 1
    got = m.get_state().cpu().numpy()
    assert steps > 40
    assert np.array_equal(got, oracle.interior(Uo))
    assert np.array_equal(m.get_ghosted_state().cpu().numpy(), Uo)
    m.close()


@pytest.mark.parametrize("theta", [2.0, 1.0])
def test_oblique_ragged_bitwise(theta):
    nx, ny, nz = 48, 40, 36
    om, Uo, m = _pair(nx, ny, nz, problems.riemann_oblique(nx, ny, nz), theta=theta)
    _run_both(om, Uo, m, 25)
    assert np.array_equal(m.get_state().cpu().numpy(), oracle.interior(Uo))
    m.close()


def test_periodic_random_bitwise_and_conserved_sums():
    n = (20, 24, 16)
    U0 = problems.random_smooth_periodic(*n, seed=3)
    om, Uo, m = _pair(*n, U0, bc=(PER, PER, PER))
    _run_both(om, Uo, m, 20)
    assert np.array_equal(m.get_state().cpu().numpy(), oracle.interior(Uo))
    assert np.array_equal(m.conserved_sums(), oracle.conserved_sums(om, Uo))
    m.close()


def _wide_range_states(nx, ny, nz, seed):
    """Physical states whose speeds span many orders of magnitude: rho and p
    log-uniform over 1e-30 .. 1e30 in a slab of four columns (partly
    outside the FP32 bound's operand range; at rest there, with a 1e-45 y
    velocity in two of them, and p / rho within 1e-2 .. 1e2), 1e-3 .. 1e3
    with velocities up to 10 elsewhere; a fast cell where it is visited
    last, or first; and a uniform state perturbed by 1e-13 (near ties)."""
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    rho = 10.0 ** rng.uniform(-3, 3, shape)
    p = 10.0 ** rng.uniform(-3, 3, shape)
    v = rng.uniform(-10, 10, (3,) + shape)
    rho[:, :, :4] = 10.0 ** rng.uniform(-30, 30, (nz, ny, 4))
    p[:, :, :4] = rho[:, :, :4] * 10.0 ** rng.uniform(-2, 2, (nz, ny, 4))
    v[..., :4] = 0.0            # at rest where rho, p span 1e-30 .. 1e30
    v[1, ..., 2:4] = 1e-45
    out = []
    for where in (-1, 0):
        r2, p2, v2 = rho.copy(), p.copy(), v.copy()
        r2.reshape(-1)[where] = 1e-3
        p2.reshape(-1)[where] = 1e3
        v2[0].reshape(-1)[where] = 50.0
        out.append(problems.conserved_from_primitive(r2, v2[0], v2[1], v2[2], p2))
    # nearly tied speeds: a uniform state perturbed by 1e-13 relative
    e = 1.0 + 1e-13 * rng.uniform(-1, 1, (5,) + shape)
    out.append(problems.conserved_from_primitive(e[0], 0.3 * e[1], -0.2 * e[2], 0.1 * e[3], e[4]))
    return out


def test_reduce_dt_wide_range_bitwise():
    """The time-step pass skips the FP64 speed of cells whose FP32 bound
    cannot raise the running maximum: on states where many cells are skipped
    and the bound's edge cases occur, dt stays the oracle's bits (exact
    build) and within a few ulps (FMA build).  Each thread visits several
    cells at this size."""
    from paper_1812_07977_gb300.fv import Mesh
    n = (128, 120, 96)
    for seed, U0 in enumerate(_wide_range_states(*n, seed=3)):
        om = oracle.mesh(*n, ly=2.0)
        dto, _, bad = oracle.reduce_dt(om, oracle.ghosted_from_interior(om, U0), 0.4)
        assert bad == 0
        for prec in ("fp64", "fp64_fma"):
            with Mesh(*n, ly=2.0, precision=prec) as m:
                m.set_state(U0)
                dt = m.reduce_dt(0.4)
            if prec == "fp64":
                assert dt == dto, (seed, dt, dto)
            else:
                assert abs(dt - dto) <= 1e-14 * dto, (seed, dt, dto)


def test_fma_dt_within_a_few_ulps():
    """The FMA build's CFL time step (Newton-Raphson sound speed, contracted
    sums) against the oracle's, on random and Riemann states."""
    from paper_1812_07977_gb300.fv import Mesh
    for U0 in (problems.random_smooth_periodic(20, 24, 16, seed=11),
               problems.riemann_oblique(33, 17, 9)):
        n = U0.shape[1:][::-1]
        om = oracle.mesh(*n)
        dto, _, _ = oracle.reduce_dt(om, oracle.ghosted_from_interior(om, U0), 0.4)
        with Mesh(*n, precision="fp64_fma") as m:
            m.set_state(U0)
            assert abs(m.reduce_dt(0.4) - dto) <= 1e-14 * dto


def test_fma_variant_within_1e12():
    n = 32
    U0 = problems.riemann_oblique(n, n, n)
    om, Uo, m = _pair(n, n, n, U0, precision="fp64_fma")
    for _ in range(60):
        dt = oracle.reduce_dt(om, Uo, 0.4)[0]
        m.step(dt)
        oracle.step(om, Uo, dt)
    err = _field_rel_err(m.get_state().cpu().numpy(), oracle.interior(Uo))
    assert np.all(err <= 1e-12), err
    m.close()


def test_fma_variant_periodic_and_near_vacuum_within_1e12():
    """The FMA build (contraction, Newton-Raphson reciprocal and sound speed)
    on a smooth periodic state and on a near-vacuum tube where faces fall
    back to first order and the sound speed takes its tiny-operand path."""
    n = (20, 24, 16)
    om, Uo, m = _pair(*n, problems.random_smooth_periodic(*n, seed=5), bc=(PER, PER, PER),
                      precision="fp64_fma")
    for _ in range(30):
        dt = oracle.reduce_dt(om, Uo, 0.4)[0]
        m.step(dt)
        oracle.step(om, Uo, dt)
    err = _field_rel_err(m.get_state().cpu().numpy(), oracle.interior(Uo))
    assert np.all(err <= 1e-12), err
    m.close()
    nx = 8
    p = np.array([6.0, 6.0, 6.0, 1.0, 1e-20, 1e-20, 1e-20, 1e-20])
    z = np.zeros(nx)
    U0 = problems.conserved_from_primitive(np.ones(nx), z, z, z, p).reshape(5, 1, 1, nx)
    om, Uo, m = _pair(nx, 1, 1, np.ascontiguousarray(U0), precision="fp64_fma")
    dU, bad, fb = oracle.compute_update(om, Uo, 1e-3)
    m.substep(1, 1e-3)
    ref = oracle.interior(Uo) + oracle.interior(dU)
    assert np.all(_field_rel_err(m.get_state().cpu().numpy(), ref) <= 1e-12)
    assert m.counters() == (0, fb) and fb == 1
    m.close()


def test_newton_forms_against_ieee(tmp_path):
    """recip_nr and sound_speed_nr (the FMA build's divide and square root)
    against IEEE division and square root: within a few ulps inside the
    seed range, bitwise outside it and on special values."""
    import os
    import subprocess
    from paper_1812_07977_gb300.build import ARCH, CSRC, INCLUDE, nvcc
    here = os.path.dirname(os.path.abspath(__file__))
    exe = str(tmp_path / "newton_check")
    subprocess.run([nvcc(), *ARCH, "-O3", "-std=c++17", "-I", CSRC, "-I", INCLUDE,
                    os.path.join(here, "cuda", "newton_check.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    f = r.stdout.split()
    recip, speed, outside = int(f[1]), int(f[3]), int(f[5])
    assert recip <= 2 and speed <= 4 and outside == 0, r.stdout


def test_face_fallback_count_matches():
    nx = 8
    p = np.array([6.0, 6.0, 6.0, 1.0, 1e-20, 1e-20, 1e-20, 1e-20])
    z = np.zeros(nx)
    U0 = problems.conserved_from_primitive(np.ones(nx), z, z, z, p).reshape(5, 1, 1, nx)
    om, Uo, m = _pair(nx, 1, 1, np.ascontiguousarray(U0))
    dU, bad, fb = oracle.compute_update(om, Uo, 1e-3)
    m.substep(1, 1e-3)
    assert np.array_equal(m.get_state().cpu().numpy(), oracle.interior(Uo) + oracle.interior(dU))
    assert m.counters() == (0, fb) and fb == 1
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp64_fma"])
def test_uniform_runs_with_nonphysical_block(precision):
    """Long runs of equal cells (where the sweeps reuse the previous face's
    flux) that contain a block of equal non-physical cells (every face there
    falls back to first order): the fallback count, the non-physical count
    and the state after one substep match the oracle; bitwise for the exact
    build.  Lines along all three axes, several warps of lines."""
    nx, ny, nz = 40, 36, 33
    U0 = problems.uniform(nx, ny, nz, 1.0, (0.2, -0.1, 0.05), 1.0)
    U0[4, 10:22, 5:30, 8:20] = -1.0            # negative energy: p < 0 there
    U0[0, :, 20:, :] = 0.5                     # a density jump across y
    from paper_1812_07977_gb300.fv import FvError, ERR_NONPHYSICAL
    om, Uo, m = _pair(nx, ny, nz, U0, precision=precision)
    dU, bad, fb = oracle.compute_update(om, Uo, 1e-3)
    m.substep(1, 1e-3)
    out = torch.empty(U0.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(FvError) as e:      # the state is copied, then the latch reported
        m.get_state(out)
    assert e.value.status == ERR_NONPHYSICAL
    got = out.cpu().numpy()
    ref = oracle.interior(Uo) + oracle.interior(dU)
    assert m.counters() == (bad, fb) and bad > 0 and fb > 0
    ok = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), ok)
    if precision == "fp64":
        assert np.array_equal(got[ok], ref[ok])
    else:
        scale = np.abs(np.where(ok, ref, 0)).reshape(5, -1).max(1)[:, None, None, None]
        assert np.all(np.abs(np.where(ok, got - ref, 0)) <= 1e-12 * scale)
    m.close()


def test_signed_zeros_bit_for_bit():
    """The reuse shortcuts (reused fluxes, zero flux differences, the RK
    combine of cells with no flux difference) must give the bits the full
    arithmetic gives, signed zeros included: a state whose momenta are -0 in
    one half-space and +0 in the other, with a pressure jump, compared with
    the oracle as bit patterns after 3 steps (exact build)."""
    n = (40, 36, 33)
    nx, ny, nz = n
    U0 = problems.uniform(nx, ny, nz, 1.0, (0.0, 0.0, 0.0), 1.0)
    U0[1:4, :, :, : nx // 2] = -0.0
    U0[4, :, :, nx // 2 + 3:] = 0.25
    U0[0, :, ny // 2:, :] = 0.5
    assert np.signbit(U0[1]).any() and not np.signbit(U0[1]).all()
    om, Uo, m = _pair(*n, U0)
    _run_both(om, Uo, m, 3)
    got = m.get_state().cpu().numpy()
    ref = np.ascontiguousarray(oracle.interior(Uo))
    assert np.array_equal(np.ascontiguousarray(got).view(np.uint64), ref.view(np.uint64))
    m.close()


def test_face_counts():
    """fv_get_face_counts: the FP64 sweeps evaluate every face of a state
    without equal neighbours and reuse almost every flux of a uniform state
    (one evaluated face per grid line and sweep); the fused kernels (FP64 and
    FP32-bulk) evaluate every face of the first (tile and chunk edges twice)
    and reuse most of the second."""
    from paper_1812_07977_gb300.fv import Mesh
    n = (40, 36, 33)
    nx, ny, nz = n
    defined = 2 * ((nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1))
    lines = 2 * (ny * nz + nx * nz + nx * ny)
    for prec, fused in (("fp64", 0), ("fp64_fma", 0), ("fp64", 1), ("fp64_fma", 1),
                        ("fp32_bulk", 1)):
        with Mesh(*n, bc=("periodic",) * 3, precision=prec) as m:
            m.set_tuning("sweep_segments", 1)
            if prec != "fp32_bulk":
                m.set_tuning("fp64_fused", fused)
            m.set_state(problems.random_smooth_periodic(*n, seed=9))
            m.step(m.reduce_dt(0.4))
            ev, de = m.face_counts()
            assert de == defined
            assert (ev == de) if not fused else (ev >= de)
        with Mesh(*n, precision=prec) as m:
            m.set_tuning("sweep_segments", 1)
            if prec != "fp32_bulk":
                m.set_tuning("fp64_fused", fused)
            m.set_state(problems.uniform(*n, 1.0, (0.3, 0.2, 0.1), 1.0))
            m.step(m.reduce_dt(0.4))
            ev, de = m.face_counts()
            assert de == defined
            assert (ev == lines) if not fused else (ev < de // 4)
            m.set_state(problems.uniform(*n, 1.0, (0.3, 0.2, 0.1), 1.0))
            assert m.face_counts() == (0, 0)


def _segments_of(n, segments):
    seg = -(-n // min(segments, n))
    return -(-n // seg)


@pytest.mark.parametrize("segments", [2, 3, 7, 64])
def test_sweep_segments_bitwise_and_counted(segments):
    """Grid lines cut into segments give the unsegmented sweeps' bits
    (exact build against the oracle, FMA build against itself unsegmented);
    each extra segment evaluates one face twice, which the face count shows,
    and a fallback face on a segment boundary is counted once."""
    from paper_1812_07977_gb300.fv import Mesh
    n = (33, 17, 29)
    U0 = problems.riemann_oblique(*n)
    om, Uo, m = _pair(*n, U0)
    m.set_tuning("fp64_fused", 0)
    m.set_tuning("sweep_segments", segments)
    _run_both(om, Uo, m, 4)
    got = m.get_state().cpu().numpy()
    assert np.array_equal(got.view(np.uint64), oracle.interior(Uo).view(np.uint64))
    m.close()
    states = []
    for sg in (1, segments):
        with Mesh(*n, precision="fp64_fma") as mf:
            mf.set_tuning("fp64_fused", 0)
            mf.set_tuning("sweep_segments", sg)
            mf.set_state(torch.from_numpy(U0).cuda())
            for _ in range(4):
                mf.step(mf.reduce_dt(0.4))
            states.append(mf.get_state().cpu().numpy())
    assert np.array_equal(states[0].view(np.uint64), states[1].view(np.uint64))
    # a state without equal neighbours: every face evaluated, boundaries twice
    nx, ny, nz = n
    with Mesh(*n, bc=("periodic",) * 3, precision="fp64_fma") as mp:
        mp.set_tuning("fp64_fused", 0)
        mp.set_tuning("sweep_segments", segments)
        mp.set_state(problems.random_smooth_periodic(*n, seed=9))
        mp.step(mp.reduce_dt(0.4))
        ev, de = mp.face_counts()
    extra = 2 * sum((_segments_of(a, segments) - 1) * lines for a, lines in
                    ((nx, ny * nz), (ny, nx * nz), (nz, nx * ny)))
    assert ev == de + extra, (ev, de, extra)
    # near-vacuum tube: the one fallback face (between cells 3 and 4) is a
    # segment boundary for 2 segments of 4 cells
    tx = 8
    p = np.array([6.0, 6.0, 6.0, 1.0, 1e-20, 1e-20, 1e-20, 1e-20])
    z = np.zeros(tx)
    Ut = problems.conserved_from_primitive(np.ones(tx), z, z, z, p).reshape(5, 1, 1, tx)
    om, Uo, m = _pair(tx, 1, 1, np.ascontiguousarray(Ut))
    m.set_tuning("fp64_fused", 0)
    m.set_tuning("sweep_segments", 2 if segments == 64 else segments)
    dU, bad, fb = oracle.compute_update(om, Uo, 1e-3)
    m.substep(1, 1e-3)
    assert np.array_equal(m.get_state().cpu().numpy(), oracle.interior(Uo) + oracle.interior(dU))
    assert m.counters() == (0, fb) and fb == 1
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "fp64_fma"])
def test_primitives_from_the_dt_pass_same_bits(precision):
    """fv_reduce_dt's pass leaves the state's primitives for the next
    substep 1; a run that uses them and one that converts again (fv_fill_ghosts
    in between drops them) give the same dt and state bits, and the same
    counts."""
    from paper_1812_07977_gb300.fv import Mesh
    n = (37, 22, 19)
    runs = []
    for refresh in (False, True):
        with Mesh(*n, precision=precision) as m:
            m.set_state(torch.from_numpy(problems.riemann_oblique(*n)).cuda())
            dts = []
            for _ in range(5):
                dts.append(m.reduce_dt(0.4))
                if refresh:
                    m.fill_ghosts()
                m.step(dts[-1])
            runs.append((dts, m.get_state().cpu().numpy(), m.counters()))
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1].view(np.uint64), runs[1][1].view(np.uint64))
    assert runs[0][2] == runs[1][2]


def test_driver_loop_with_short_names():
    """Algorithm 1's loop through the wrapper's short names (set, dt, step,
    get) with dt clamped to the end time, against the oracle's loop: the same
    dts and state bits."""
    from paper_1812_07977_gb300.fv import Mesh
    n = (20, 6, 5)
    U0 = problems.riemann_planar(*n)
    om = oracle.mesh(*n)
    Uo = oracle.ghosted_from_interior(om, U0)
    T = 0.05
    with Mesh(*n) as m:
        m.set(U0)
        t = 0.0
        while t < T:
            dt = min(m.dt(0.4), T - t)
            dto = min(oracle.reduce_dt(om, Uo, 0.4)[0], T - t)
            assert dt == dto
            m.step(dt)
            oracle.step(om, Uo, dto)
            t += dt
        got = m.get().cpu().numpy()
    assert np.array_equal(got, oracle.interior(Uo))


def test_host_buffers_match_device_buffers():
    n = (16, 12, 10)
    U0 = problems.riemann_oblique(*n)
    from paper_1812_07977_gb300.fv import Mesh
    a = Mesh(*n)
    b = Mesh(*n)
    a.set_state(torch.from_numpy(U0).cuda())
    b.set_state(U0.copy())                      # numpy host buffer
    for _ in range(3):
        dt = a.reduce_dt(0.4)
        a.step(dt)
        b.step(b.reduce_dt(0.4))
    host = np.empty_like(U0)
    b.get_state(host)
    pinned = torch.empty(U0.shape, dtype=torch.float64).pin_memory()
    a.get_state(pinned)
    assert np.array_equal(host, pinned.numpy())
    a.close()
    b.close()


def test_nonphysical_state_is_reported():
    from paper_1812_07977_gb300.fv import FvError, Mesh, ERR_NONPHYSICAL
    n = (6, 5, 4)
    U0 = problems.uniform(*n, 1.0, (0.0, 0.0, 0.0), 1.0)
    U0[4, 1, 2, 3] = -1.0
    with Mesh(*n) as m:
        m.set_state(U0)
        with pytest.raises(FvError) as e:
            m.reduce_dt(0.4)
        assert e.value.status == ERR_NONPHYSICAL
        assert m.counters()[0] == 1
        m.set_state(problems.uniform(*n, 1.0, (0.0, 0.0, 0.0), 1.0))   # clears the latch
        assert m.reduce_dt(0.4) > 0


def test_call_order_and_handle_errors():
    from paper_1812_07977_gb300.fv import FvError, Mesh, ERR_INVALID_ARG, ERR_BAD_HANDLE
    n = (6, 5, 4)
    m = Mesh(*n)
    m.set_state(problems.uniform(*n, 1.0, (0.1, 0.0, 0.0), 1.0))
    m.substep(1, 1e-3)
    for bad in (lambda: m.step(1e-3), lambda: m.reduce_dt(0.4), lambda: m.substep(1, 1e-3)):
        with pytest.raises(FvError) as e:
            bad()
        assert e.value.status == ERR_INVALID_ARG
    with pytest.raises(FvError):
        m.step(float("nan"))
    m.substep(2, 1e-3)
    h = m.handle
    m.close()
    lib = m._lib
    assert lib.fv_step(h, 1e-3) == ERR_BAD_HANDLE


@pytest.mark.parametrize("precision", ["fp64", "fp64_fma"])
def test_full_size_256_sampled_windows(precision):
    """The timed workload (oblique Riemann problem, 256^3, outflow) in the
    benchmark's launch configuration: after two steps, windows of the GPU
    state match the oracle run on the sub-box around each window (the
    result in a window depends only on inputs within 4 cells per step):
    bitwise for the exact build, within 1e-12 of each field's scale for the
    FMA build that the benchmark times."""
    n = 256
    U0 = problems.riemann_oblique(n, n, n)
    om_full = oracle.mesh(n, n, n)
    from paper_1812_07977_gb300.fv import Mesh
    m = Mesh(n, n, n, precision=precision)
    m.set_state(torch.from_numpy(U0).cuda())
    dts = []
    for _ in range(2):
        dt = m.reduce_dt(0.4)
        dts.append(dt)
        m.step(dt)
    got = m.get_state().cpu().numpy()
    m.close()
    # the first dt against the oracle over the whole mesh (the FMA build's
    # Newton-Raphson sound speed is within a few ulps)
    dto, _, _ = oracle.reduce_dt(om_full, oracle.ghosted_from_interior(om_full, U0), 0.4)
    if precision == "fp64":
        assert dts[0] == dto
    else:
        assert abs(dts[0] - dto) <= 1e-14 * dto
    halo = 4 * len(dts)
    w = 8
    starts = [0, 60, 124, 128, 200, n - w]
    rng = np.random.default_rng(0)
    windows = [(a, a, a) for a in starts] + [tuple(rng.choice(starts, 3)) for _ in range(4)]
    pairs = []
    for (i0, j0, k0) in windows:
        lo = [max(0, c - halo) for c in (i0, j0, k0)]
        hi = [min(n, c + w + halo) for c in (i0, j0, k0)]
        sub = U0[:, lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        ns = [hi[a] - lo[a] for a in range(3)]
        om = oracle.mesh(*ns, lx=ns[0] / n, ly=ns[1] / n, lz=ns[2] / n)
        Uo = oracle.ghosted_from_interior(om, np.ascontiguousarray(sub))
        for dt in dts:
            oracle.step(om, Uo, dt)
        ref = oracle.interior(Uo)[:, k0 - lo[2]:k0 - lo[2] + w, j0 - lo[1]:j0 - lo[1] + w,
                                  i0 - lo[0]:i0 - lo[0] + w]
        pairs.append(((i0, j0, k0), got[:, k0:k0 + w, j0:j0 + w, i0:i0 + w], ref))
    # field scale: the largest |value| of each field over all windows (the
    # momenta start at zero, so the initial state gives them no scale)
    scale = np.max([np.abs(r).reshape(5, -1).max(1) for _, _, r in pairs], axis=0)
    for where, win, ref in pairs:
        if precision == "fp64":
            assert np.array_equal(win, ref), where
        else:
            err = np.abs(win - ref).reshape(5, -1).max(1)
            assert np.all(err <= 1e-12 * scale), (where, err / np.maximum(scale, 1e-300))


def _window_refs(U0_dev, n, dts, windows, w, gamma):
    """Oracle runs on the sub-boxes around each window (outflow at their cut:
    the window depends only on inputs within 4 cells per step)."""
    halo = 4 * len(dts)
    refs = []
    for (i0, j0, k0) in windows:
        lo = [c - halo for c in (i0, j0, k0)]
        hi = [c + w + halo for c in (i0, j0, k0)]
        sub = U0_dev[:, lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].cpu().numpy()
        ns = [hi[a] - lo[a] for a in range(3)]
        om = oracle.mesh(*ns, lx=ns[0] / n, ly=ns[1] / n, lz=ns[2] / n, gamma=gamma)
        Uo = oracle.ghosted_from_interior(om, np.ascontiguousarray(sub))
        for dt in dts:
            oracle.step(om, Uo, dt)
        refs.append(oracle.interior(Uo)[:, halo:halo + w, halo:halo + w, halo:halo + w])
    return refs


def test_shear_layer_512_sampled_windows():
    """The 512^3 periodic shear-layer workload (gamma 5/3, 8-mode seeded
    perturbation): two FP64 steps (exact build) match the oracle bit for bit
    on interior windows, and two FP32-bulk steps of the graph-replayed batch
    of one mesh (its own CFL steps) stay within FP32 rounding of the oracle
    run on the same steps."""
    from paper_1812_07977_gb300.fv import Batch, Mesh
    n, g53, w = 512, 5.0 / 3.0, 8
    U0 = problems.shear_layer_device(n, 0.01, gamma=g53, modes=8, seed=2024, device="cuda")
    rng = np.random.default_rng(1)
    windows = [(100, 100, 100), (250, 120, 380), (400, 255, 60)] + \
        [tuple(int(v) for v in rng.integers(16, n - 16 - w, 3)) for _ in range(3)]
    m = Mesh(n, n, n, gamma=g53, bc=("periodic",) * 3)
    m.set_state(U0)
    dts = []
    for _ in range(2):
        dts.append(m.reduce_dt(0.4))
        m.step(dts[-1])
    got = m.get_state()
    m.close()
    for (i0, j0, k0), ref in zip(windows, _window_refs(U0, n, dts, windows, w, g53)):
        win = got[:, k0:k0 + w, j0:j0 + w, i0:i0 + w].cpu().numpy()
        assert np.array_equal(win, ref), (i0, j0, k0)
    del got
    stream = torch.cuda.Stream()
    b = Batch([(n, n, n)], gamma=g53, bc=("periodic",) * 3, stream=stream)
    b.set_state(0, U0)
    dts32 = []
    for _ in range(2):
        b.step(0.4, use_graph=True)
        dts32.append(float(b.dts()[0]))
    got = b.get_state(0)
    b.close()
    # field scales; the three momenta share the momentum magnitude's (vy and
    # vz are 1% perturbations, FP32 rounds the O(1) fluxes that move them)
    scale = U0.abs().reshape(5, -1).amax(1).cpu().numpy()
    scale[1:4] = scale[1:4].max()
    for (i0, j0, k0), ref in zip(windows, _window_refs(U0, n, dts32, windows, w, g53)):
        win = got[:, k0:k0 + w, j0:j0 + w, i0:i0 + w].cpu().numpy()
        err = np.abs(win - ref).reshape(5, -1).max(1) / scale
        assert np.all(err < 1e-6), ((i0, j0, k0), err)


@pytest.mark.parametrize("kchunk", [1, 5, 32])
def test_fused_and_sweeps_same_bits(kchunk):
    """The fused FP64 kernel (one launch per substep over 32 x 8 tiles and z
    chunks) and the per-axis sweeps compute the same operations in the same
    order: the exact build gives the oracle's bits both ways -- on ragged
    meshes (tiles cut at every edge), z chunks of several sizes, outflow and
    periodic faces, a non-default limiter -- with the same dt, fallback and
    non-physical counts."""
    from paper_1812_07977_gb300.fv import Mesh
    cases = [((45, 19, 23), problems.riemann_oblique(45, 19, 23), (OUT, OUT, OUT), 2.0),
             ((33, 10, 12), problems.random_smooth_periodic(33, 10, 12, seed=3),
              (PER, OUT, PER), 1.3)]
    for n, U0, bc, theta in cases:
        runs = []
        for fused in (1, 0):
            om, Uo, m = _pair(*n, U0, bc=bc, theta=theta)
            m.set_tuning("fp64_fused", fused)
            m.set_tuning("kchunk", kchunk)
            _run_both(om, Uo, m, 4)
            got = m.get_state().cpu().numpy()
            assert np.array_equal(got.view(np.uint64),
                                  np.ascontiguousarray(oracle.interior(Uo)).view(np.uint64))
            runs.append(m.counters())
            m.close()
        assert runs[0] == runs[1]


def test_fused_fma_matches_sweeps_fma_within_1e12():
    """The FMA build in its two forms (fused kernel and sweeps) stays within
    1e-12 of each field's scale of the other after 20 steps of the oblique
    problem (the contractions can differ between the two kernels)."""
    from paper_1812_07977_gb300.fv import Mesh
    n = (40, 36, 33)
    U0 = problems.riemann_oblique(*n)
    out = []
    for fused in (1, 0):
        with Mesh(*n, precision="fp64_fma") as m:
            m.set_tuning("fp64_fused", fused)
            m.set_state(U0)
            for _ in range(20):
                m.step(m.reduce_dt(0.4))
            out.append(m.get_state().cpu().numpy())
    assert np.all(_field_rel_err(out[0], out[1]) <= 1e-12)
