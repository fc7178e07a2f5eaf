"""The measurement probes run and give plausible figures on the GPU: the integer
issue-rate probe (the roofline's denominator) and the shared-memory pattern
probe (whose launches the bank-counter profile reads)."""
import pytest

import probes
from paper_2511_12009_gb300 import nq

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nq.lib()


def test_alu_probe_rates():
    lop3 = nq.probe_alu(0, 256)
    assert 20 < lop3["per_clk_per_sm"] < 140  # lanes per clock per SM
    assert 500 < lop3["sm_mhz"] < 3000


@pytest.mark.parametrize("kind,mask,density", [(k, m, d) for k, m, d, _ in probes.CASES])
def test_smem_probe_runs(kind, mask, density):
    ms = nq.probe_smem(kind, mask, density, iters=16, slots=8)
    assert 0 < ms < 1000


def test_smem_probe_rejects_bad_arguments():
    with pytest.raises(nq.NQError):
        nq.probe_smem(7)
    with pytest.raises(nq.NQError):
        nq.probe_smem(0, slots=17)
