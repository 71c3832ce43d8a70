"""The float-float build (FV_PREC_FP64_FF): FP64 state, primitives, RK
combine and CFL time step; differences, limited slopes, face states, HLL
fluxes and the flux divergence in float-float arithmetic on the FP32 pipe.
It is held to the FP64 target against the oracle: |gpu - oracle| <= 1e-12 of
each field's scale, after as many steps as the FMA build's tests take, and
in the benchmark's 256^3 launch configuration; plus the exact invariants
(uniform states, round-off conservation) and its operand-range guard."""
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


def _mesh(n, bc=(OUT, OUT, OUT), theta=2.0, **kw):
    from paper_1812_07977_gb300.fv import Mesh
    return Mesh(*n, theta=theta, bc=tuple("periodic" if b == PER else "outflow" for b in bc),
                precision="fp64_ff", **kw)


def _field_rel_err(got, ref):
    scale = np.abs(ref).reshape(5, -1).max(1)
    return np.abs(got - ref).reshape(5, -1).max(1) / np.maximum(scale, 1e-300)


def _run(n, U0, steps=None, t_end=None, bc=(OUT, OUT, OUT), theta=2.0):
    """Both sides advance with the oracle's dt; returns the GPU and oracle
    states, the largest relative dt difference and the step count."""
    om = oracle.mesh(*n, bc=bc, theta=theta)
    Uo = oracle.ghosted_from_interior(om, U0)
    m = _mesh(n, bc, theta)
    m.set_state(torch.from_numpy(np.ascontiguousarray(U0)).cuda())
    t, k, dtrel = 0.0, 0, 0.0
    while (steps is None or k < steps) and (t_end is None or t < t_end):
        dto, _, _ = oracle.reduce_dt(om, Uo, 0.4)
        dt = m.reduce_dt(0.4)
        dtrel = max(dtrel, abs(dt - dto) / dto)
        if t_end is not None:
            dto = min(dto, t_end - t)
        m.step(dto)
        oracle.step(om, Uo, dto)
        t += dto
        k += 1
    got = m.get_state().cpu().numpy()
    m.close()
    return got, oracle.interior(Uo), dtrel, k


def test_ff_oblique_60_steps_within_1e12():
    n = (32, 32, 32)
    got, ref, dtrel, k = _run(n, problems.riemann_oblique(*n), steps=60)
    err = _field_rel_err(got, ref)
    print("oblique 32^3, 60 steps: field errors", err, "dt", dtrel)
    assert np.all(err <= 1e-12), err
    assert dtrel <= 1e-14


def test_ff_sod_32_to_t02_within_1e12():
    n = (32, 32, 32)
    got, ref, dtrel, k = _run(n, problems.riemann_planar(*n), t_end=0.2)
    err = _field_rel_err(got, ref)
    print("Sod 32^3 to t = 0.2:", k, "steps, field errors", err)
    assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("theta", [2.0, 1.3])
def test_ff_periodic_random_within_1e12_and_conservative(theta):
    n = (20, 24, 16)
    U0 = problems.random_smooth_periodic(*n, seed=5)
    got, ref, dtrel, k = _run(n, U0, steps=30, bc=(PER, PER, PER), theta=theta)
    err = _field_rel_err(got, ref)
    print("periodic random, theta", theta, "30 steps: field errors", err)
    assert np.all(err <= 1e-12), err
    # the face fluxes telescope: the sums move by round-off of the FP64 state only
    s0, s1 = U0.reshape(5, -1).sum(1), got.reshape(5, -1).sum(1)
    scale = np.abs(U0).reshape(5, -1).sum(1)
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale), (s1 - s0) / scale


def test_ff_uniform_state_exact():
    n = (40, 12, 9)
    U0 = problems.uniform(*n, 1.3, (0.2, -0.1, 0.05), 0.9)
    m = _mesh(n)
    m.set_state(U0)
    for _ in range(3):
        m.step(m.reduce_dt(0.4))
    assert np.array_equal(m.get_state().cpu().numpy(), U0)
    m.close()


def test_ff_full_size_256_sampled_windows():
    """The timed workload (oblique Riemann problem, 256^3) in the benchmark's
    launch configuration: after two steps, windows of the state against the
    oracle on the sub-box around each (the result in a window depends only
    on inputs within 4 cells per step), within 1e-12 of each field's scale;
    the first dt within 1e-14 of the oracle's."""
    n = 256
    U0 = problems.riemann_oblique(n, n, n)
    m = _mesh((n, n, n))
    m.set_state(torch.from_numpy(U0).cuda())
    dts = []
    for _ in range(2):
        dts.append(m.reduce_dt(0.4))
        m.step(dts[-1])
    got = m.get_state().cpu().numpy()
    m.close()
    om_full = oracle.mesh(n, n, n)
    dto, _, _ = oracle.reduce_dt(om_full, oracle.ghosted_from_interior(om_full, U0), 0.4)
    assert abs(dts[0] - dto) <= 1e-14 * dto
    halo, w = 8, 8
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
    scale = np.max([np.abs(r).reshape(5, -1).max(1) for _, _, r in pairs], axis=0)
    worst = 0.0
    for where, win, ref in pairs:
        err = np.abs(win - ref).reshape(5, -1).max(1) / np.maximum(scale, 1e-300)
        worst = max(worst, float(err.max()))
        assert np.all(err <= 1e-12), (where, err)
    print("256^3 windows after two steps: worst field error", worst)


def test_ff_face_counts_and_fallbacks():
    """Every face of a state without equal neighbours is evaluated (tile and
    chunk edges twice); the near-vacuum-free oblique problem has no
    fallback faces, like the oracle."""
    n = (40, 36, 33)
    nx, ny, nz = n
    defined = 2 * ((nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1))
    m = _mesh(n, bc=(PER, PER, PER))
    m.set_state(problems.random_smooth_periodic(*n, seed=9))
    m.step(m.reduce_dt(0.4))
    ev, de = m.face_counts()
    assert de == defined and ev >= de
    assert m.counters() == (0, 0)
    m.close()


def test_ff_operand_range_is_guarded():
    """A state with a primitive outside the float-float range (a pressure
    of 1e-20) is reported at the next synchronising call, not stepped
    silently."""
    from paper_1812_07977_gb300.fv import FvError, ERR_INVALID_ARG
    nx = 8
    p = np.array([6.0, 6.0, 6.0, 1.0, 1e-20, 1e-20, 1e-20, 1e-20])
    z = np.zeros(nx)
    U0 = problems.conserved_from_primitive(np.ones(nx), z, z, z, p).reshape(5, 1, 1, nx)
    m = _mesh((nx, 1, 1))
    m.set_state(np.ascontiguousarray(U0))
    m.step(1e-3)
    with pytest.raises(FvError) as e:
        m.get_state()
    assert e.value.status == ERR_INVALID_ARG
    m.close()


def test_ff_launch_settings_same_bits():
    """The float-float kernel built for one or two CTAs per SM, with tiles of
    32 x 8, 12 or 16 and 16 x 16 columns and z chunks of several sizes,
    computes the same operations: the same bits (45 x 29 x 30: ragged tiles
    of every shape)."""
    n = (45, 29, 30)
    U0 = problems.riemann_oblique(*n)
    out = []
    for occ, ty, tx, kc in ((2, 16, 16, 64), (1, 16, 16, 64), (2, 16, 16, 7), (2, 8, 32, 64),
                            (1, 8, 32, 1), (2, 8, 32, 9), (1, 16, 32, 5)):
        m = _mesh(n)
        # through built shapes only: occupancy 1, the width, the height
        m.set_tuning("occupancy", 1)
        m.set_tuning("tile_x", tx)
        m.set_tuning("tile_y", ty)
        m.set_tuning("occupancy", occ)
        m.set_tuning("kchunk", kc)
        m.set_state(U0)
        for _ in range(3):
            m.step(m.reduce_dt(0.4))
        out.append((m.get_state().cpu().numpy(), m.counters()))
        m.close()
    for st, ct in out[1:]:
        assert np.array_equal(st.view(np.uint64), out[0][0].view(np.uint64))
        assert ct == out[0][1]


def test_ff_tile_changes_must_stay_built():
    """Shape changes that would leave the built (tile x, tile y, CTAs per SM)
    are rejected and leave the mesh as it was: from the default 16 x 16 at 2
    CTAs per SM, 32 x 16 exists only at one CTA per SM."""
    from paper_1812_07977_gb300.fv import FvError
    m = _mesh((16, 16, 16))
    with pytest.raises(FvError):
        m.set_tuning("tile_x", 32)      # (32, 16, 2) is not built
    with pytest.raises(FvError):
        m.set_tuning("tile_y", 8)       # (16, 8, 2) is not built
    m.set_tuning("occupancy", 1)
    m.set_tuning("tile_x", 32)
    with pytest.raises(FvError):
        m.set_tuning("occupancy", 2)    # (32, 16, 2)
    with pytest.raises(FvError):
        m.set_tuning("tile_y", 12)
    m.set_tuning("tile_y", 8)
    m.set_tuning("occupancy", 2)
    m.close()


def _z_invariant(n, seed):
    """A smooth periodic state that varies in x and y only: every z plane of
    every tile equals the one below, so after a chunk's first plane each
    plane skips its slope and face passes while its x and y flux
    differences are not zero."""
    nx, ny, nz = n
    U2 = problems.random_smooth_periodic(nx, ny, 1, seed=seed)
    return np.ascontiguousarray(np.repeat(U2, nz, axis=1))


def _short_chunks(make_mesh):
    def make(n, bc):
        m = make_mesh(n, bc)
        m.set_tuning("kchunk", 11)
        return m
    return make


def _runs_with_plane_skip(make_mesh, n, U0, bc, steps):
    out = []
    for skip in (1, 0):
        m = make_mesh(n, bc)
        m.set_tuning("plane_skip", skip)
        m.set_state(U0)
        dts = []
        for _ in range(steps):
            dts.append(m.reduce_dt(0.4))
            m.step(dts[-1])
        out.append((dts, m.get_state().cpu().numpy(), m.counters(), m.face_counts()))
        m.close()
    return out


@pytest.mark.parametrize("state", ["oblique", "z_invariant", "planar_x", "smooth"])
def test_ff_plane_skip_same_bits(state):
    """Skipping the slope and face passes of tile planes equal to the plane
    below changes nothing: the same state bits, dt, counters and face counts
    as running every pass, on a ragged mesh with short z chunks (transitions
    between skipped and evaluated planes: the oblique problem; every plane
    after a chunk's first skipped with non-zero x / y divergence: a
    z-invariant state; a planar tube along x; a smooth state, where every
    face is evaluated and the steps after the first switch to the kernel
    built without the skip)."""
    n = (45, 29, 30)
    if state == "oblique":
        U0, bc = problems.riemann_oblique(*n), (OUT, OUT, OUT)
    elif state == "z_invariant":
        U0, bc = _z_invariant(n, 5), (PER, PER, PER)
    elif state == "smooth":
        U0, bc = problems.random_smooth_periodic(*n, seed=8), (PER, PER, PER)
    else:
        U0, bc = problems.riemann_planar(*n), (OUT, OUT, OUT)
    out = _runs_with_plane_skip(_short_chunks(_mesh), n, U0, bc, 4)
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1].view(np.uint64), out[1][1].view(np.uint64))
    assert out[0][2] == out[1][2]
    assert out[0][3] == out[1][3]


def test_ff_z_invariant_against_oracle():
    """The z-invariant state (every plane after a chunk's first takes the
    plane skip) against the oracle: within 1e-12 of each field's scale, and
    still z-invariant bit for bit."""
    n = (40, 24, 20)
    U0 = _z_invariant(n, 6)
    got, ref, dtrel, _ = _run(n, U0, steps=12, bc=(PER, PER, PER))
    assert _field_rel_err(got, ref).max() <= 1e-12
    assert dtrel <= 1e-12
    assert np.array_equal(got.view(np.uint64), np.repeat(got[:, :1], n[2], axis=1).view(np.uint64))
