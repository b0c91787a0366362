"""Host-side logic of the request loop (no GPU): percentiles and request bookkeeping."""
import pytest

from paper_2602_09527_gb300 import serve


def test_percentile_interpolates_order_statistics():
    v = [5.0, 1.0, 3.0, 2.0, 4.0]
    assert serve.percentile(v, 0) == 1.0
    assert serve.percentile(v, 100) == 5.0
    assert serve.percentile(v, 50) == 3.0
    assert serve.percentile(v, 25) == 2.0
    assert serve.percentile([1.0, 2.0], 50) == pytest.approx(1.5)
    assert serve.percentile([], 50) != serve.percentile([], 50)   # NaN


def test_request_defaults():
    r = serve.Request(key=1, b=None, arrival=0.5, alpha=0.01, gamma=1.0, seed=3)
    assert r.admitted is None and r.finished is None and r.n_subsets == 0 and r.storage == "FP32"
