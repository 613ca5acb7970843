"""The checkerboard experiment driver on a small case: the consistent matrix, which generated
the data, reconstructs the 16 x 16 checkerboard almost exactly; the line-based comparators,
which did not, leave a larger error."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim", [2, 3])
def test_checkerboard_small(dim):
    from paper_2511_12235_gb300 import experiments
    res = experiments.run_case(16, dim, max_iters=300)
    main = res["area" if dim == 2 else "volume"]
    for k, v in res.items():
        assert math.isfinite(v["mse"]) and v["spectral_norm"] > 0, k
    assert main["mse"] < 1e-3
    assert main["mse"] < min(res["line_siddon"]["mse"], res["line_joseph"]["mse"])
