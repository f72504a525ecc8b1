"""Failure detection without a GPU fault: a device-side wait that runs out.

The tuning key test_wait_timeout makes the split-precision product issue no
copies and give every mbarrier wait a 1 ms budget, so the MMA issuer's wait
for its first operand tile runs out: the CTA records QML_ETIMEOUT in the
status word, the other roles see it and leave their waits, TMEM is freed
and the kernel returns.  The call reports status 5 and the context stays
usable: the same product then runs normally and is correct."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_21149_gb300 import api as A
    from paper_2605_21149_gb300 import build
    build.build()
    return A


def td(x):
    return torch.as_tensor(np.asarray(x), device="cuda").t().contiguous().t()


@pytest.mark.parametrize("m,nn,kk", [(128, 128, 64), (300, 200, 1100)])
def test_split_wait_timeout_is_reported(api, m, nn, kk):
    rng = np.random.default_rng(m + kk)
    A, B = rng.normal(size=(m, kk)), rng.normal(size=(kk, nn))
    C = td(np.zeros((m, nn)))
    api.tune_set("test_wait_timeout", 1)
    try:
        with pytest.raises(api.QMLError) as ei:
            api.gemm(td(A), td(B), C, precision=1)
    finally:
        api.tune_set("test_wait_timeout", 0)
    assert ei.value.status == 5, str(ei.value)
    # the context is intact: the same split product now runs and is right
    api.gemm(td(A), td(B), C, precision=1)
    ref = A @ B
    assert np.abs(C.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max() * kk
    x = torch.ones(1000, device="cuda").sum().item()
    assert x == 1000.0
