"""The HRG-versus-GIRG experiment (Sec. 5, threshold variants): the subgraph and
supergraph scales found by bisection agree with the exact ones the oracle derives
pair by pair, and the missing / additional edge counts agree with set differences
of the oracle's all-pairs graphs."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle as O  # noqa: E402
from paper_1905_06706_gb300.coupling import Coupling  # noqa: E402

pytestmark = pytest.mark.gpu


def test_coupling_matches_oracle():
    n, alpha, seed = 3000, 0.75, 5
    R = 2.0 * math.log(n) + 0.5
    r, X = O.hrg_points(n, alpha, R, seed)
    w = np.array([O.hrg_weight(x, R) for x in r])
    W = O.exact_sum(w)
    hrg = O.edge_set(O.hrg_allpairs(X, r, R, 0.0, seed))
    # the scale at which each pair joins the GIRG: r_uv = K w_u w_v / W
    u, v = np.triu_indices(n, 1)
    D = (X[u].astype(np.int64) - X[v].astype(np.int64)) % (1 << 32)
    D = np.minimum(D, (1 << 32) - D)
    k_uv = (D * 2.0 ** -32) / ((w[u] * w[v]) / W)
    is_h = np.isin(u.astype(np.int64) * (1 << 32) + v, np.fromiter(hrg, dtype=np.int64))
    k_sub, k_sup = k_uv[~is_h].min(), k_uv[is_h].max()

    cp = Coupling(n, alpha, R, seed)
    assert cp.hrg_edges == len(hrg)
    res = cp.run(grid=(0.5 * k_sub, k_sub * 3.0, k_sup), rel_tol=1e-7)
    assert res["K_sub"] == pytest.approx(k_sub, rel=2e-6)
    assert res["K_super"] == pytest.approx(k_sup, rel=2e-6)
    assert res["d_girg"] <= res["d_hrg"] <= res["D_girg"]
    for pt in res["curve"]:
        g = O.edge_set(O.girg_allpairs(X.reshape(n, 1), w, W, 0.0, None, 0, K=pt["K"]))
        assert pt["missing"] == len(hrg - g)
        assert pt["additional"] == len(g - hrg)
        assert pt["girg_degree"] == pytest.approx(2.0 * len(g) / n)
