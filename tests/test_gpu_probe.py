"""The random-access ceiling probe (maiter_probe_random_rate): it measures
something (positive rates for every kind), and the rate falls once the array
outgrows L2 (126 MB): 2^20 words stay resident, 2^27 words (512 MB) do not."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_05785_b300 as m
    m.lib()
    return m


def test_every_kind_reports_a_rate(mt):
    for kind in (mt.PROBE_RED_F32, mt.PROBE_RED_F64, mt.PROBE_MIN_U32, mt.PROBE_LOAD_32):
        assert mt.probe_random_rate(kind, 16) > 1.0


def test_rate_falls_when_the_array_leaves_l2(mt):
    resident = mt.probe_random_rate(mt.PROBE_RED_F32, 20)
    spilled = mt.probe_random_rate(mt.PROBE_RED_F32, 27)
    assert spilled < 0.7 * resident
