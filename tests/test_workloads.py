"""The seeded input generators (no arithmetic of the method): shapes and
distributions of the ragged batch, and that instance k does not depend on how
many instances are drawn."""
import numpy as np

from paper_2605_31425_gb300 import workloads


def test_ragged_shapes_follow_the_stated_distribution():
    sh = [workloads.ragged_shape(k, 1004) for k in range(4096)]
    m = np.array([a for a, _ in sh])
    d = np.array([b for _, b in sh])
    assert m.min() >= 100 and m.max() <= 100_000
    assert set(d.tolist()) == set(workloads.RAGGED_DIMS)
    # log-uniform m: log10 m roughly uniform on [2, 5] (quartiles near 2.75, 3.5, 4.25)
    q = np.quantile(np.log10(m), [0.25, 0.5, 0.75])
    assert np.all(np.abs(q - [2.75, 3.5, 4.25]) < 0.1)
    counts = np.array([np.sum(d == v) for v in workloads.RAGGED_DIMS])
    assert counts.min() > 700


def test_ragged_instances_are_prefix_stable():
    a = workloads.ragged(5, 9)
    b = workloads.ragged(3, 9)
    for (C1, R1), (C2, R2) in zip(a, b):
        assert np.array_equal(C1, C2) and np.array_equal(R1, R2)
    C, R = workloads.ragged_instance(4, 9)
    m, d = workloads.ragged_shape(4, 9)
    assert C.shape == (m, d) and R.shape == (m,)
    assert R.min() >= 0.0 and R.max() < 0.1
