"""The FP64 pipe probe measures plausible rates on the GPU: the FMA rate near the nominal
FP64 peak, the FP64 tensor-core (DMMA) rate no higher than a plain FMA can reach."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    from paper_1606_03135_gb300 import probe as P
    r = P.measure(iters=4000, repeats=2)
    assert 0.5 < r["dfma"]["tflops"] < 3.0, r
    assert 0.1 < r["dmma"]["tflops"] < 3.0, r
    assert 0.1 < r["mixed"]["tflops"] < 3.0, r
