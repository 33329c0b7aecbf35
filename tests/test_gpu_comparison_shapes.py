"""The comparison workloads of section 4 on the GPU path: the unit Gaussian on
[-7, 7]^d (d = 2, 8, 16), the 2-D Rosenbrock on [-10, 10]^2 and the array of 49
Gaussians, against their closed forms (erf products, the Rosenbrock 1-D erf
quadrature, Table 1's value for the array).  Batched (m = N/100) to keep the
test short; bench.py --comparison-shapes runs the sequential case."""
import math

import numpy as np
import pytest

from tests import analytic as A
from paper_2608_28514_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2608_28514_gb300 import _native
    _native.lib()
    return _native


@pytest.mark.parametrize("maker,N", [(lambda: W.gauss_unit_box7(2), 1000), (lambda: W.gauss_unit_box7(8), 1000),
                                     (lambda: W.gauss_unit_box7(16), 1000), (W.rosenbrock2d_box10, 500),
                                     (W.array49, 500)])
def test_comparison_shapes_recover_closed_forms(nat, maker, N):
    p = maker()
    truth = A.logz(p)
    n = 16
    h = nat.ns_create_batch([(p, N, N // 100, 5 * p.d, 1e-3, 40 + s) for s in range(n)])
    nat.ns_run(h)
    res = [nat.ns_summary(h, r) for r in range(n)]
    nat.ns_destroy(h)
    z = np.array([r["log_z"] for r in res])
    assert all(r["status"] == 0 for r in res)
    se = max(z.std(ddof=1), np.mean([r["log_z_err"] for r in res])) / math.sqrt(n)
    assert abs(z.mean() - truth) < 4 * se + 0.01, (p.name, z.mean(), truth, se)
