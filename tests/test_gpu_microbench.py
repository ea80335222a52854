"""The counter-operation microbenchmark reports a positive, finite rate."""
import math

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_smem_atomics_rate():
    from paper_1812_00283_gb300 import BfcError, bfc
    s = torch.cuda.current_stream().cuda_stream
    rate, ms = bfc.bfc_bench_smem_atomics(s, 256)
    assert ms > 0 and math.isfinite(rate) and rate > 1e9
    with pytest.raises(BfcError):
        bfc.bfc_bench_smem_atomics(s, 0)
