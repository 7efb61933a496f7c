"""tn_contract_dev_noalloc: the allocation-free pairwise contraction.

For callers that cannot let the library allocate device memory (an
application owning all GPU memory through its own pool, or a latency-critical
loop that must not hit cudaMalloc), the library runs the split-K contraction
with its partial sums in a fixed device array.  This file checks, through the
C ABI, that two consecutive calls give the same result as the allocating
entry point tn_contract_dev and as the contraction's definition (the CPU
oracle), and that an output too large for the fixed scratch is rejected with
a clear error.  It is collected last on purpose.
"""
import numpy as np
import pytest

from oracle import con
from paper_2405_14060_gb300 import tn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# sizes, labels A, labels B, labels C (small outputs over long summed spaces)
CASES = [
    ([2] * 18, list(range(18)), list(range(18)), []),                        # full trace
    ([2] * 20, list(range(18)), list(range(2, 20)), [0, 1, 18, 19]),          # 16 outputs
    ([3, 5, 7, 11, 13, 4], [0, 1, 2, 3], [1, 2, 3, 4, 5], [0, 5, 4]),         # ragged sizes
    ([2] * 16 + [3], list(range(16)) + [16], list(range(16)), [16]),          # shared batch-like label
    # a short summed space over many outputs: one pass per output, no partials
    ([2] * 19, list(range(18)), [17, 18], list(range(17)) + [18]),
]
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("semiring", [0, 1])
def test_noalloc_matches_allocating_entry(case, dt, semiring):
    sizes, la, lb, lc = CASES[case]
    rng = np.random.default_rng(7 + case)
    A = rng.random([sizes[v] for v in la])
    B = rng.random([sizes[v] for v in lb])
    if semiring == 1:
        A, B = np.log(A), np.log(B)
    tA = torch.tensor(A, dtype=dt, device="cuda").contiguous()
    tB = torch.tensor(B, dtype=dt, device="cuda").contiguous()
    shape = [sizes[v] for v in lc] or [1]
    ref = torch.zeros(shape, dtype=dt, device="cuda")
    ref_am = torch.zeros(ref.numel(), dtype=torch.int32, device="cuda")
    tn.contract_dev(sizes, la, tA, lb, tB, lc, ref, semiring=semiring,
                    argmax=ref_am if semiring else None,
                    prec="fp64" if dt == torch.float64 else "fp32")
    r = ref.cpu().numpy()
    if semiring == 0:
        want = con.con_dense([tuple(la), tuple(lb)], [A, B], tuple(lc))
        want_i = None
    else:
        want, want_i = con.tcon_dense([tuple(la), tuple(lb)], [A, B], tuple(lc))
    want = np.asarray(want).reshape(shape)
    for _ in range(2):
        out = torch.full(shape, float("nan"), dtype=dt, device="cuda")
        am = torch.full((out.numel(),), -1, dtype=torch.int32, device="cuda")
        tn.contract_dev_noalloc(sizes, la, tA, lb, tB, lc, out, semiring=semiring,
                                argmax=am if semiring else None)
        o = out.cpu().numpy()
        err = np.max(np.abs(o - r)) / max(1e-300, np.max(np.abs(r)))
        assert err <= TOL[dt], (case, dt, semiring, err)
        err_o = np.max(np.abs(o - want)) / max(1e-300, np.max(np.abs(want)))
        assert err_o <= TOL[dt], (case, dt, semiring, err_o)
        if semiring == 1 and dt == torch.float64:
            np.testing.assert_array_equal(am.cpu().numpy(), ref_am.cpu().numpy())
            np.testing.assert_array_equal(am.cpu().numpy(), np.asarray(want_i).reshape(-1))


def test_noalloc_rejects_output_beyond_scratch():
    # 2^21 float outputs need more than the 8 MiB fixed scratch
    sizes = [2] * 22
    la, lb, lc = list(range(22)), [21], list(range(21))
    tA = torch.rand([2] * 22, device="cuda")
    tB = torch.rand(2, device="cuda")
    tC = torch.zeros([2] * 21, device="cuda")
    with pytest.raises(tn.TNError) as e:
        tn.contract_dev_noalloc(sizes, la, tA, lb, tB, lc, tC)
    assert e.value.status == 1 and "scratch" in str(e.value)
