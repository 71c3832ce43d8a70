"""bench.py's CPU legs without a GPU: the oracle timed on several host
cores (one spawned process per core, each on its own slab of the workload)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_oracle_on_two_cores_runs_distinct_slabs():
    rate, seconds, steps, S = bench.oracle_on_cores(2, 2, warmup=0, steps=1)
    assert steps == 1 and S == 2 and seconds > 0
    assert rate > 0
    # the slabs of one call are distinct and inside the mesh
    first = max(0, bench.N // 2 - 2 * S // 2)
    starts = [min(first + i * S, bench.N - S) for i in range(2)]
    assert len(set(starts)) == 2 and all(0 <= k and k + S <= bench.N for k in starts)


def test_slab_worker_is_the_oracle_on_that_slab():
    """The worker steps the oracle on the slab of the whole problem's initial
    state, so its sample is the workload's own cells."""
    cells, n, el = bench._oracle_slab((bench.N // 2 - 1, 2, 0, 1, 0.0))
    assert cells == bench.N * bench.N * 2 and n == 1 and el > 0
