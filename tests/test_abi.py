"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/girg_gb300.h declares; parameter validation happens on the host before
any CUDA call (so these run without a GPU)."""
import ctypes
import os
import re

import pytest

import paper_1905_06706_gb300 as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "girg_gb300.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:girg|hrg)_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return gg.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(gg.SIGNATURES), set(names) ^ set(gg.SIGNATURES)


def test_status_strings(lib):
    assert gg.status_string(0) == "ok"
    assert "too small" in gg.status_string(gg.GIRG_E_CAPACITY)
    assert gg.status_string(99) == "unknown status"


def _params(**kw):
    base = dict(n=1000, d=2, beta=2.5, T=0.5, avg_deg=10.0, c=0.0, w_min=1.0, seed=1,
                edge_bytes=4, precision=0, level_cap=0)
    base.update(kw)
    return gg.GirgParams(**base)


@pytest.mark.parametrize("bad", [dict(n=1), dict(n=2 ** 31), dict(d=0), dict(d=9),
                                 dict(beta=2.0), dict(T=1.0), dict(T=-0.1), dict(w_min=0.0),
                                 dict(edge_bytes=2), dict(precision=2), dict(avg_deg=0.0),
                                 dict(avg_deg=999.0), dict(level_cap=-1)])
def test_invalid_parameters_rejected_on_host(lib, bad):
    p = _params(**bad)
    m = ctypes.c_int64(-1)
    st = lib.girg_generate(ctypes.byref(p), None, 0, ctypes.byref(m), None, None)
    assert st == gg.GIRG_E_PARAM
    assert m.value == -1  # nothing was written


def test_noalloc_refuses_pointers_the_gpu_cannot_use(lib):
    """Pageable host buffers (and, on a machine without a GPU, every pointer) are
    refused by the no-allocation entry point before any device work."""
    import numpy as np
    X = np.zeros(1000, dtype=np.uint32)
    w = np.ones(1000, dtype=np.float64)
    out = np.zeros((4000, 2), dtype=np.int32)
    m = ctypes.c_int64(-1)
    st = lib.girg_allpairs_noalloc(1000, 1, X.ctypes.data, w.ctypes.data, 1000.0, 0.5, 1.0, 1,
                                   0, 4, out.ctypes.data, len(out), ctypes.byref(m), None)
    assert st == gg.GIRG_E_PARAM and m.value == -1 and not out.any()


def test_issue_probe_rejects_bad_arguments(lib):
    """The issue-rate probe checks its kind, trip count and result pointers on the host."""
    ms, wi = ctypes.c_float(-1.0), ctypes.c_int64(-1)
    for kind, iters in ((3, 10), (-1, 10), (0, 0), (2, (1 << 24) + 1)):
        st = lib.girg_issue_probe(kind, iters, None, ctypes.byref(ms), ctypes.byref(wi))
        assert st == gg.GIRG_E_PARAM
    assert lib.girg_issue_probe(0, 10, None, None, ctypes.byref(wi)) == gg.GIRG_E_PARAM
    assert ms.value == -1.0 and wi.value == -1


def test_weight_layer_from_bit_fields_matches_oracle(lib):
    """The kernels take the weight layer of Sec. 3.1 from the bit fields of w and w_min
    (no division); it equals the oracle's floor(log2) of the rounded quotient at every
    layer boundary w_min 2^k, one and two ulps on either side, for minimum weights with
    small and large mantissas, and on random weights, subnormals and extremes (positive
    finite weights, the generator's domain)."""
    import math
    import random
    import oracle as O
    rng = random.Random(5)
    mins = [1.0, 1.37, 1.9999999999999998, 1.0000000000000002, 0.75, 3e-300, 5e-324,
            2.5e-308, 1e300, 7.0]
    cases = []
    for wm in mins:
        for k in range(-2, 66):
            if math.frexp(wm)[1] + k > 1024:  # beyond the doubles
                break
            b = math.ldexp(wm, k)
            x = b
            for _ in range(2):
                x = math.nextafter(x, 0.0)
            for _ in range(5):
                cases.append((x, wm))
                x = math.nextafter(x, math.inf)
        for _ in range(200):
            x = wm * math.exp(rng.uniform(0.0, 45.0))
            if math.isfinite(x):
                cases.append((x, wm))
    cases += [(5e-324, 5e-324), (1e-308, 5e-324), (2e-320, 1e-320), (1e300, 1e290)]
    for x, wm in cases:
        got = lib.girg_det_eval(7, x, wm)
        assert got == O.layer_of(x, wm), (x, wm, got)


def test_invalid_hrg_and_points_rejected(lib):
    m = ctypes.c_int64(0)
    for hp in (gg.HrgParams(1000, 0.5, 0.5, 0.0, 10.0, 1, 4, 0, 0),    # alpha must exceed 1/2
               gg.HrgParams(1000, 0.75, 0.5, 0.0, 0.0, 1, 4, 0, 0),    # R or avg_deg needed
               gg.HrgParams(1000, 0.75, 0.5, 999.0, 0.0, 1, 4, 0, 0),  # avg_deg < n - 1
               gg.HrgParams(1000, 0.75, 1.0, 0.0, 10.0, 1, 4, 0, 0),   # T < 1
               gg.HrgParams(1000, 0.75, 0.5, 0.0, 10.0, 1, 2, 0, 0)):  # edge_bytes 4 or 8
        assert lib.hrg_generate(ctypes.byref(hp), None, 0, ctypes.byref(m), None,
                                None) == gg.GIRG_E_PARAM
    assert lib.girg_points(0, 2, 2.5, 1.0, 1, None, None, None) == gg.GIRG_E_PARAM
    assert lib.girg_allpairs(10, 1, None, None, 0.0, 0.5, 1.0, 1, 0, 4, None, 0,
                             ctypes.byref(m), None) == gg.GIRG_E_PARAM
    assert lib.girg_generate_from_points(10, 1, None, None, 0.5, -1.0, 1, 0, 0, 4, None, 0,
                                         ctypes.byref(m), None) == gg.GIRG_E_PARAM


def test_struct_layout_matches_header(tmp_path):
    """ctypes field offsets equal the C compiler's for both parameter structs."""
    import subprocess
    fields = {"girg_params": [f for f, _ in gg.GirgParams._fields_],
              "hrg_params": [f for f, _ in gg.HrgParams._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "girg_gb300.h"',
             "int main(void) {"]
    for st, names in fields.items():
        lines.append(f'printf("%zu\\n", sizeof({st}));')
        for f in names:
            lines.append(f'printf("%zu\\n", offsetof({st}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    expect = []
    for cls in (gg.GirgParams, gg.HrgParams):
        expect.append(ctypes.sizeof(cls))
        expect.extend(getattr(cls, f).offset for f, _ in cls._fields_)
    assert out == expect


def test_host_deterministic_math_matches_oracle_bitwise(lib):
    """The library's FP64 elementary functions (used for the type-II tables) and the
    oracle's independent implementation give identical bits."""
    import numpy as np

    import oracle as O
    rng = np.random.default_rng(21)
    xs = np.concatenate([np.exp(rng.uniform(-700, 700, 2000)), rng.uniform(0, 3, 2000)])
    for x in xs:
        assert lib.girg_det_eval(0, x, 0.0) == O.det_log(x)
        assert lib.girg_det_eval(5, 1.0 + x, 0.0) == O.det_acosh(1.0 + x)
    for x in rng.uniform(-0.999, 3, 3000):
        assert lib.girg_det_eval(1, x, 0.0) == O.det_log1p(x)
    for x in rng.uniform(-745, 709, 3000):
        assert lib.girg_det_eval(2, x, 0.0) == O.det_exp(x)
    for x, y in zip(np.exp(rng.uniform(-50, 50, 3000)), rng.uniform(-8, 8, 3000)):
        assert lib.girg_det_eval(3, x, y) == O.det_pow(x, y)
    for x in rng.uniform(0, 0.5, 3000):
        assert lib.girg_det_eval(4, x, 0.0) == O.det_sinpi(x)
    for wu, wv in rng.uniform(1, 50, (2000, 2)):
        assert lib.girg_det_eval(6, wu, wv) == O.girg_p(2, 0.75, 0.5, 1000.0, wu, wv, 2 ** 30)


# ------------------------------------------------------------------ HRG radius (host code)

@pytest.mark.parametrize("alpha,T,R", [(0.75, 0.0, 12.0), (0.75, 0.5, 20.0), (0.9, 0.3, 31.0),
                                       (0.6, 0.8, 25.0)])
def test_hrg_expected_degree_matches_oracle(lib, alpha, T, R):
    import oracle as O
    n = 10 ** 6
    got = gg.hrg_expected_avg_degree(n, alpha, T, R)
    ref = O.hrg_avg_degree(n, alpha, T, R)
    assert abs(got - ref) <= 1e-9 * ref


@pytest.mark.parametrize("n,alpha,T,deg", [(10 ** 7, 0.75, 0.5, 10.0), (10 ** 4, 0.75, 0.0, 8.0),
                                           (10 ** 5, 1.1, 0.7, 20.0)])
def test_hrg_radius_matches_oracle(lib, n, alpha, T, deg):
    import oracle as O
    R = gg.hrg_solve_radius(n, alpha, T, deg)
    assert abs(R - O.hrg_solve_R(n, alpha, T, deg)) <= 1e-9 * R
    assert abs(gg.hrg_expected_avg_degree(n, alpha, T, R) - deg) <= 1e-11 * deg


def test_hrg_radius_rejects_bad_targets(lib):
    out = ctypes.c_double(0.0)
    assert lib.hrg_solve_radius(1000, 0.75, 0.5, 0.0, ctypes.byref(out)) == gg.GIRG_E_PARAM
    assert lib.hrg_solve_radius(1000, 0.75, 0.5, 999.0, ctypes.byref(out)) == gg.GIRG_E_PARAM
    assert lib.hrg_expected_avg_degree(1000, 0.75, 0.5, -1.0, ctypes.byref(out)) == gg.GIRG_E_PARAM
