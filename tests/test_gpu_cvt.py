"""The integer-pipe binary32 <-> binary64 conversions of the mixed-precision
kernels against the hardware conversions, bit for bit: every binary32 value
widened; every binary32 value's binary64 image, its neighbours, the midpoints
to the next binary32 value (the ties) and their neighbours narrowed, plus
pseudo-random binary64 patterns (IEEE 754 roundTiesToEven)."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10192_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)


def test_conversions_equal_the_hardware_ones():
    from paper_1912_10192_gb300 import hamr
    wbad, wfirst, nbad, nfirst = hamr.check_conversions(nrandom=1 << 26, seed=10192)
    assert wbad == 0, "widening differs first at binary32 pattern %#x" % (wfirst & 0xffffffff)
    assert nbad == 0, "narrowing differs first at binary64 pattern %#x" % (nfirst & 0xffffffffffffffff)
