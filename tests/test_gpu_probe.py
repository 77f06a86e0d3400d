"""The issue-rate probe that gives the pair kernels' issue roofline its measured
denominator: every instruction kind runs, reports its launch time and the warp
instructions it issues by construction, and the rates land between a quarter of and a
little above the nominal issue rate (4 schedulers per SM, one warp instruction each per
cycle, at the GPU's maximum clock)."""
import pytest

torch = pytest.importorskip("torch")

import paper_1905_06706_gb300 as gg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_issue_probe_rates(kind):
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    iters = 200
    gg.issue_probe(kind, iters)  # warm-up
    ms, wi = gg.issue_probe(kind, iters)
    assert wi == sms * 2 * 32 * iters * 128  # two 1024-thread blocks per SM, 128 per trip
    assert ms > 0.0
    rate = wi / (ms / 1e3)
    nominal = 4 * sms * 2.2e9  # above the 2.07 GHz maximum clock, as an upper bound
    assert 0.25 * 4 * sms * 1.0e9 < rate < 1.1 * nominal


def test_issue_probe_rejects_bad_kind():
    with pytest.raises(gg.GirgError):
        gg.issue_probe(3, 10)
