"""Split-precision GEMM (bf16 digits on tcgen05, exact FP32 chunks, float64
recombination) through qml_gemm with precision QML_SPLIT_BF16.

Pins (P14): products of small integer matrices are exact (which holds only if
the tensor-core FP32 accumulation of every digit chunk is exact); on random
float64 operands the error stays inside the bound the digit count predicts,
|dC_ij| <= 4 (S/4 + 1) K 2^(e_i + f_j - beta S), with beta = 6, S = 8."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPLIT = 1
BETA, S = 6, 8


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_21149_gb300 import api as A
    from paper_2605_21149_gb300 import build
    build.build()
    return A


def td(x):
    return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda").t().contiguous().t()


def _exp(v):
    m = np.abs(v).max()
    return 0 if m == 0 else np.frexp(m)[1]


def bound(opA, opB):
    K = opA.shape[1]
    ea = np.array([_exp(r) for r in opA])
    eb = np.array([_exp(c) for c in opB.T])
    return 4 * (S / 4 + 1) * K * np.ldexp(1.0, ea[:, None] + eb[None, :] - BETA * S)


@pytest.mark.parametrize("ta,tb,m,n,k", [(0, 0, 128, 128, 64), (0, 1, 130, 67, 65),
                                         (1, 0, 300, 257, 1000), (1, 1, 1, 1, 1)])
def test_split_exact_on_integers(api, ta, tb, m, n, k):
    rng = np.random.default_rng(m * 7 + n + k)
    A = rng.integers(-1000, 1001, size=(k, m) if ta else (m, k)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(n, k) if tb else (k, n)).astype(np.float64)
    ref = ((A.T if ta else A).astype(np.int64) @ (B.T if tb else B).astype(np.int64)).astype(np.float64)
    C = api.gemm(td(A), td(B), transA=bool(ta), transB=bool(tb), precision=SPLIT)
    assert np.array_equal(C.cpu().numpy(), ref)


@pytest.mark.parametrize("ta,tb,m,n,k", [(0, 0, 200, 130, 300), (0, 1, 257, 129, 4100),
                                         (1, 0, 64, 500, 9000), (1, 1, 333, 77, 128)])
def test_split_error_bound_random(api, ta, tb, m, n, k):
    rng = np.random.default_rng(k)
    A = rng.normal(size=(k, m) if ta else (m, k)) * np.exp(rng.normal(size=(1, m) if ta else (m, 1)))
    B = rng.normal(size=(n, k) if tb else (k, n))
    opA, opB = (A.T if ta else A), (B.T if tb else B)
    ref = opA @ opB
    C0 = rng.normal(size=(m, n))
    Cd = td(C0)
    api.gemm(td(A), td(B), Cd, transA=bool(ta), transB=bool(tb), alpha=0.5, beta=2.0,
             precision=SPLIT)
    err = np.abs(Cd.cpu().numpy() - (0.5 * ref + 2.0 * C0))
    # float64 rounding of the final fma adds one ulp of |2 C0|
    assert np.all(err <= 0.5 * bound(opA, opB) + 4e-16 * np.abs(2.0 * C0) + 1e-300)
    # and it is at float64 quality in practice
    assert np.abs(Cd.cpu().numpy() - (0.5 * ref + 2.0 * C0)).max() <= 1e-12 * np.abs(ref).max()


def test_split_syrk_shared_digits_lower(api):
    """X^T X with A == B (digits shared) into the lower triangle only."""
    rng = np.random.default_rng(11)
    n, k = 700, 300
    X = rng.normal(size=(n, k))
    W0 = rng.normal(size=(k, k))
    Wd = td(W0)
    Xd = td(X)
    api.gemm(Xd, Xd, Wd, transA=True, lower=True, precision=SPLIT)
    out = Wd.cpu().numpy()
    ref = X.T @ X
    il, iu = np.tril_indices(k), np.triu_indices(k, 1)
    assert np.abs(out[il] - ref[il]).max() <= 1e-12 * np.abs(ref).max()
    assert np.array_equal(out[iu], W0[iu])


@pytest.mark.parametrize("ta,tb,m,n,k,lower,beta", [
    (1, 0, 700, 700, 300, True, 0.0),    # X^T X, 6 tile rows, shared digits
    (0, 1, 640, 640, 512, True, 1.0),    # trailing-update shape, 5 tile rows
    (0, 0, 300, 257, 1000, False, 1.0),  # 3 tile rows, ragged N
    (1, 1, 129, 77, 33, False, 0.0),     # 2 tile rows, the second holds one row
    (0, 0, 100, 300, 64, False, 0.0),    # one tile row: one CTA per tile
])
def test_split_pairs_match_single(api, ta, tb, m, n, k, lower, beta):
    """Tile-row pairs in clusters of two (B digit tiles shared by multicast,
    tuning key ozaki_pairs = 1, the default) give the same bits as one CTA
    per tile (ozaki_pairs = 0), including tiles past the last row and, for a
    lower C, tiles above the diagonal (computed, not stored)."""
    rng = np.random.default_rng(m + 3 * n + 7 * k)
    if lower and ta == 1:
        A = rng.normal(size=(k, m))
        B = A
    elif lower:
        A = rng.normal(size=(m, k))
        B = A
    else:
        A = rng.normal(size=(k, m) if ta else (m, k))
        B = rng.normal(size=(n, k) if tb else (k, n))
    tbv = (not ta) if lower else bool(tb)
    C0 = rng.normal(size=(m, n))
    Ad = td(A)
    Bd = Ad if B is A else td(B)
    outs = []
    try:
        for pairs in (1, 0):
            api.tune_set("ozaki_pairs", pairs)
            Cd = td(C0)
            api.gemm(Ad, Bd, Cd, transA=bool(ta), transB=tbv, alpha=-1.0 if beta else 1.0,
                     beta=beta, lower=lower, precision=SPLIT)
            outs.append(Cd.cpu().numpy())
    finally:
        api.tune_set("ozaki_pairs", 1)
    assert np.array_equal(outs[0], outs[1])
    opA = A.T if ta else A
    opB = B.T if tbv else B
    ref = (-1.0 if beta else 1.0) * (opA @ opB) + beta * C0
    if lower:
        il, iu = np.tril_indices(m), np.triu_indices(m, 1)
        assert np.abs(outs[0][il] - ref[il]).max() <= 1e-12 * np.abs(ref).max()
        assert np.array_equal(outs[0][iu], C0[iu])
    else:
        assert np.abs(outs[0] - ref).max() <= 1e-12 * np.abs(ref).max()

