"""Host-side measurement logic of bench.py (no GPU): the time-to-gap stopping rule, the
field-of-view scaling of the batched jobs' TV weight and the all-cores oracle figure."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


ORIG_ENV = {k for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS") if os.environ.get(k) == "1"}


def test_first_within_takes_the_first_evaluation_inside_the_target():
    hist = [[10, 2.0, 0, 0], [20, 1.001, 0, 0], [30, 1.00005, 0, 0], [40, 1.0, 0, 0]]
    assert bench.first_within(hist, 1.0, 1e-4) == 30
    assert bench.first_within(hist, 1.0, 1e-2) == 20
    assert bench.first_within(hist, 0.5, 1e-4) is None
    # negative objectives: the gap is relative to |F*|
    assert bench.first_within([[5, -0.99995, 0, 0]], -1.0, 1e-4) == 5


def test_stop_after_last_prox():
    theta = np.array([0, 1, 0, 0, 1, 0, 0, 0, 1, 0])
    assert bench.stop_after_last_prox(8, theta) == 5     # last prox below 8 is iteration 4
    assert bench.stop_after_last_prox(9, theta) == 9     # iteration 8 is a prox step
    assert bench.stop_after_last_prox(1, theta) == 1     # no prox yet: run to the evaluation
    assert bench.stop_after_last_prox(10, theta) == 9


def test_job_alpha_field_of_view():
    w2 = dict(alpha=0.02, alpha_fov=True)
    assert bench.job_alpha(w2, dict(side=512)) == pytest.approx(0.02 * 256 ** 2)
    w3 = dict(alpha=0.01, alpha_fov=True, dims=3)
    assert bench.job_alpha(w3, dict(side=96)) == pytest.approx(0.01 * 64 ** 2)
    assert bench.job_alpha(dict(alpha=0.3), dict(side=128)) == 0.3


def test_oracle_all_cores_runs_spawned_single_threaded_samples():
    """The all-cores oracle figure: one spawned process per requested core, each timing the
    single-core sample on its own copy of the problem; per-reconstruction seconds scale the
    samples by the counts, and the throughput is processes / that time."""
    import bench
    counts = {"iterations": 10, "prox_calls": 2, "snapshots": 1}
    out = bench.oracle_all_cores("par2d_64", counts, 10, procs=2)
    assert out["processes"] == 2 and out["s_per_reconstruction"] > 0
    # both figures are rounded (seconds to 0.01): they agree to that rounding
    per = out["s_per_reconstruction"]
    assert abs(out["reconstructions_per_hour"] - 2 * 3600.0 / per) <= 2 * 3600.0 * 0.006 / per ** 2 + 1e-3
    for k in bench._SINGLE_THREAD_ENV:   # the parent's environment is restored
        assert os.environ.get(k) != "1" or k in ORIG_ENV
