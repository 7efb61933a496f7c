"""Failure detection on the GPU without a fault: bounded device-side waits.

Every mbarrier wait of the tensor-core GEMM pipeline has a time limit; when
one runs out, the kernel sets an error flag, waits for the transfers and
MMAs it has already issued, releases its tensor memory and returns, and the
host reports TN_E_TIMEOUT.  The library's test hook TN_TEST_TC_WAIT_NS sets
the limit of the producer's and the MMA issuer's waits to zero nanoseconds,
so the first wait that is not satisfied at once gives up; the next call,
with the normal limit, must succeed on the same context.
"""
import numpy as np
import pytest

from paper_2405_14060_gb300 import tn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_gemm_wait_gives_up_then_recovers(monkeypatch):
    # a GEMM-form contraction: m = 512, n = 768, k = 384 over three tiles
    sizes, la, lb, lc = [8, 64, 3, 256, 128, 3], [0, 1, 4, 5], [4, 5, 2, 3], [0, 1, 2, 3]
    rng = np.random.default_rng(5)
    A = rng.random([sizes[v] for v in la])
    B = rng.random([sizes[v] for v in lb])
    ref = np.einsum(A, la, B, lb, lc)
    tA = torch.tensor(A, dtype=torch.float32, device="cuda")
    tB = torch.tensor(B, dtype=torch.float32, device="cuda")
    tC = torch.zeros([sizes[v] for v in lc], dtype=torch.float32, device="cuda")
    monkeypatch.setenv("TN_TEST_TC_WAIT_NS", "0")
    with pytest.raises(tn.TNError) as e:
        tn.contract_dev(sizes, la, tA, lb, tB, lc, tC, prec="tf32")
    assert e.value.status == 6, e.value            # TN_E_TIMEOUT
    monkeypatch.delenv("TN_TEST_TC_WAIT_NS")
    for _ in range(2):
        tC.zero_()
        tn.contract_dev(sizes, la, tA, lb, tB, lc, tC, prec="tf32")
        err = np.max(np.abs(tC.cpu().numpy() - ref)) / np.max(np.abs(ref))
        assert err <= 2e-3
    torch.cuda.synchronize()
