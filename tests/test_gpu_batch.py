"""Batches (fv_batch_*): many uneven meshes advanced by one persistent
launch per substep, optionally replayed from a CUDA graph.

Each mesh of a batch performs exactly the single-mesh FP32-bulk arithmetic
(same per-cell operations, whatever the work decomposition), so after the
same steps it must equal a single FP32-bulk Mesh bit for bit; that Mesh is
itself checked against the FP64 oracle in test_gpu_fp32.py, and one batch
mesh is checked against the oracle here as well.
"""
import numpy as np
import pytest

import oracle
from paper_1812_07977_gb300 import problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)


def _small_batch(count=7, seed=3):
    lengths = (8, 16, 24, 33, 40)
    return problems.batched_riemann(seed=seed, count=count, lengths=lengths)


def _single_runs(spec, nsteps):
    from paper_1812_07977_gb300.fv import Mesh
    out = []
    for s in spec:
        m = Mesh(*s["shape"], precision="fp32_bulk")
        m.set_state(s["U0"])
        for _ in range(nsteps):
            m.step(m.reduce_dt(0.4))
        out.append(m.get_state().cpu().numpy())
        m.close()
    return out


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_single_meshes_bitwise(use_graph):
    from paper_1812_07977_gb300.fv import Batch
    spec = _small_batch()
    ref = _single_runs(spec, 6)
    with Batch([s["shape"] for s in spec]) as b:
        for m, s in enumerate(spec):
            b.set_state(m, s["U0"])
        for _ in range(6):
            b.step(0.4, use_graph=use_graph)
        for m in range(len(spec)):
            got = b.get_state(m).cpu().numpy()
            assert np.array_equal(got, ref[m]), m


@pytest.mark.parametrize("kchunk,occ,tile_y", [(8, 2, 8), (5, 3, 8), (64, 2, 8), (7, 2, 4),
                                                (16, 2, 16), (3, 2, 16)])
def test_batch_result_independent_of_tuning(kchunk, occ, tile_y):
    from paper_1812_07977_gb300.fv import Batch
    spec = _small_batch(count=5, seed=11)
    ref = _single_runs(spec, 3)
    with Batch([s["shape"] for s in spec]) as b:
        b.set_tuning(kchunk, occ, tile_y)
        for m, s in enumerate(spec):
            b.set_state(m, s["U0"])
        for _ in range(3):
            b.step(0.4)
        for m in range(len(spec)):
            assert np.array_equal(b.get_state(m).cpu().numpy(), ref[m]), m


def test_batch_dt_per_mesh_matches_oracle():
    from paper_1812_07977_gb300.fv import Batch
    spec = _small_batch(count=6, seed=5)
    with Batch([s["shape"] for s in spec]) as b:
        for m, s in enumerate(spec):
            b.set_state(m, s["U0"])
        b.step(0.4)
        dts = b.dts()
    for m, s in enumerate(spec):
        om = oracle.mesh(*s["shape"])
        dto, _, _ = oracle.reduce_dt(om, oracle.ghosted_from_interior(om, s["U0"]), 0.4)
        assert dts[m] == dto, (m, dts[m], dto)


def test_batch_stage2_maxima_give_the_oracles_dt():
    """The second substep takes each mesh's FP64 CFL maximum of the state it
    writes; the next step's dt is the oracle's dt of that state, bit for bit."""
    from paper_1812_07977_gb300.fv import Batch
    spec = _small_batch(count=6, seed=9)
    with Batch([s["shape"] for s in spec]) as b:
        for m, s in enumerate(spec):
            b.set_state(m, s["U0"])
        for _ in range(3):
            b.step(0.4)
            states = [b.get_state(m).cpu().numpy() for m in range(len(spec))]
            b.step(0.4)
            dts = b.dts()
            for m, s in enumerate(spec):
                om = oracle.mesh(*s["shape"])
                dto, _, _ = oracle.reduce_dt(om, oracle.ghosted_from_interior(om, states[m]), 0.4)
                assert dts[m] == dto, (m, dts[m], dto)


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_dt_follows_set_state(use_graph):
    """The second substep leaves each mesh's CFL maximum for the next step;
    a state set in between replaces it: the step after set_state uses the dt
    of the new state (here the initial one, so the first step's dt)."""
    from paper_1812_07977_gb300.fv import Batch
    spec = _small_batch(count=5, seed=7)
    with Batch([s["shape"] for s in spec]) as b:
        for m, s in enumerate(spec):
            b.set_state(m, s["U0"])
        b.step(0.4, use_graph=use_graph)
        first = b.dts()
        for _ in range(3):
            b.step(0.4, use_graph=use_graph)
        assert not np.array_equal(b.dts(), first)
        b.set_state(2, spec[2]["U0"])
        b.step(0.4, use_graph=use_graph)
        assert b.dts()[2] == first[2]


def test_batch_mesh_against_fp64_oracle():
    from paper_1812_07977_gb300.fv import Batch
    spec = _small_batch(count=4, seed=9)
    with Batch([s["shape"] for s in spec]) as b:
        for m, s in enumerate(spec):
            b.set_state(m, s["U0"])
        dts = []
        for _ in range(5):
            b.step(0.4)
            dts.append(b.dts())
        for m, s in enumerate(spec):
            om = oracle.mesh(*s["shape"])
            Uo = oracle.ghosted_from_interior(om, s["U0"])
            for d in dts:
                oracle.step(om, Uo, d[m])
            ref = oracle.interior(Uo)
            got = b.get_state(m).cpu().numpy()
            err = np.abs(got - ref).reshape(5, -1).max(1) / np.abs(ref).max()
            assert np.all(err < 1e-5), (m, err)


def test_autotune_restores_state_and_picks_a_candidate():
    from paper_1812_07977_gb300.fv import Batch
    spec = _small_batch(count=5, seed=21)
    with Batch([s["shape"] for s in spec]) as b:
        for m, s in enumerate(spec):
            b.set_state(m, s["U0"])
        kc, occ, ty, ms = b.autotune(0.4)
        assert kc in (8, 16, 32, 64) and (ty, occ) in ((4, 2), (8, 2), (8, 3), (16, 2))
        assert ms > 0
        for m, s in enumerate(spec):
            assert np.array_equal(b.get_state(m).cpu().numpy(), s["U0"])
        assert b.counters() == (0, 0)


def test_batch_full_workload_graph_runs():
    """The 96-mesh workload (axis lengths 16..128): a few graph steps stay
    physical and agree with the non-graph steps bit for bit."""
    from paper_1812_07977_gb300.fv import Batch
    spec = problems.batched_riemann()
    shapes = [s["shape"] for s in spec]
    outs = []
    for use_graph in (True, False):
        with Batch(shapes) as b:
            for m, s in enumerate(spec):
                b.set_state(m, torch.from_numpy(s["U0"]).cuda())
            for _ in range(3):
                b.step(0.4, use_graph=use_graph)
            assert b.counters()[0] == 0
            outs.append([b.get_state(m).cpu().numpy() for m in (0, 17, 95)])
    for a, c in zip(*outs):
        assert np.array_equal(a, c)


def test_batch_rejects_bad_arguments():
    from paper_1812_07977_gb300.fv import Batch, FvError
    with Batch([(8, 8, 8), (16, 8, 4)]) as b:
        with pytest.raises(FvError):
            b.set_state(2, np.zeros((5, 8, 8, 8)))
        with pytest.raises(FvError):
            b.set_tuning(0, 2)
        with pytest.raises(FvError):
            b.set_tuning(8, 4)
        with pytest.raises(FvError):
            b.set_tuning(8, 2, 12)
        with pytest.raises(FvError):
            b.set_tuning(8, 3, 16)
        with pytest.raises(FvError):
            b.step(-1.0)


@pytest.mark.parametrize("shapes", [((16, 8, 2), (64, 4, 2), (128, 4, 2)),
                                    ((32, 4, 2), (64, 8, 2), (64, 4, 2)),
                                    ((16, 8, 2), (16, 8, 2), (32, 16, 2))])
def test_batch_class_tunings_same_bits(shapes):
    """Each size class with its own tile shape (16, 32, 64 or 128 columns
    wide) and z chunk gives every mesh the bits of its single-mesh run: the
    tiles change only which thread computes a face, not how."""
    from paper_1812_07977_gb300.fv import Batch
    spec = problems.batched_riemann(seed=21, count=7, lengths=(8, 16, 24, 40, 56, 72, 100))
    ref = _single_runs(spec, 3)
    with Batch([s["shape"] for s in spec]) as b:
        for cls, (tx, ty, occ) in enumerate(shapes):
            b.set_class_tuning(cls, tx, ty, occ, (5, 16, 64)[cls])
            assert b.class_tuning(cls)["tile_x"] == tx
        assert sum(b.class_tuning(c)["meshes"] for c in range(3)) == len(spec)
        for m, s in enumerate(spec):
            b.set_state(m, s["U0"])
        for _ in range(3):
            b.step(0.4)
        for m in range(len(spec)):
            assert np.array_equal(b.get_state(m).cpu().numpy(), ref[m]), m


def test_batch_autotune_per_class_restores_state():
    """The autotuner leaves a valid configuration per class and the state it
    found; stepping afterwards matches single-mesh runs."""
    from paper_1812_07977_gb300.fv import Batch
    spec = problems.batched_riemann(seed=22, count=6, lengths=(16, 40, 72))
    ref = _single_runs(spec, 2)
    with Batch([s["shape"] for s in spec]) as b:
        for m, s in enumerate(spec):
            b.set_state(m, s["U0"])
        kc, occ, ty, ms = b.autotune(0.4)
        assert ms > 0
        for cls in range(3):
            t = b.class_tuning(cls)
            assert t["tile_x"] in (16, 32, 64, 128) and t["kchunk"] in (8, 16, 32, 64)
        for _ in range(2):
            b.step(0.4)
        for m in range(len(spec)):
            assert np.array_equal(b.get_state(m).cpu().numpy(), ref[m]), m
