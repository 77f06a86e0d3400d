"""The autotuner's host logic: its default level cap is the library's and the oracle's rule
(so a tuned offset means the same on every side), request classes, and how a table is
applied to requests (a cap the caller fixed is kept)."""
import oracle as O
from paper_1905_06706_gb300 import autotune as at


def test_default_level_cap_is_the_oracle_rule():
    for n in (2, 10, 1000, 12_345, 10**6, 1 << 24, (1 << 31) - 1):
        for d in (1, 2, 3, 4, 5, 8):
            for T in (0.0, 0.3, 0.7):
                assert at.default_level_cap(n, d, T) == O.level_cap(n, d, T), (n, d, T)


def test_request_classes_and_apply():
    assert at.request_class(5_000, 2, 0.5) == "d2_T>0_n0"
    assert at.request_class(50_000, 3, 0.0) == "d3_T0_n1"
    assert at.request_class(900_000, 1, 0.2) == "d1_T>0_n2"
    table = {"level_cap": {"d2_T>0_n2": {"level_cap": 8, "default": 9, "ms": {"8": 1.0, "9": 1.2}}}}
    q = dict(n=1_000_000, d=2, beta=2.5, T=0.5, avg_deg=10.0, seed=1)
    assert at.apply(table, q)["level_cap"] == 8
    assert at.apply(table, dict(q, level_cap=5))["level_cap"] == 5      # fixed by the caller
    assert "level_cap" not in at.apply(table, dict(q, d=1))             # class not tuned
    assert abs(at.expected_gain(table) - 1.2) < 1e-12
    reqs = [dict(q, n=n) for n in (200_000, 300_000, 400_000)] + [dict(q, n=2_000, d=1)]
    s = at.class_samples(reqs)
    assert s["d2_T>0_n2"]["n"] == 300_000 and s["d1_T>0_n0"]["n"] == 2_000
