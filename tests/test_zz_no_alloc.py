"""qml_potrf_noalloc against qml_potrf, through the C ABI.

qml_potrf_noalloc serves callers that cannot allocate device memory (a host
runtime that owns all GPU memory and only hands out pre-allocated buffers, or
hot loops that cannot pay for cudaMalloc's device synchronisation); it keeps
its scratch in a static device array shared by every call.  The first test
calls it on shapes no other test uses, before anything else has run them, and
checks that it left no trace of the float64 tile autotuner (which allocates):
no new "dgemm:" entry in the tuning table, and no less free device memory
across a repeated call once CUDA has loaded the kernels' modules.  Calls in a
row (different sizes, so later ones run on leftover scratch) must reproduce
qml_potrf on the same matrices.  This file is
collected last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_21149_gb300 import _native, build
    build.build()
    return _native.load()


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.normal(size=(n, n))
    return G @ G.T / n + np.eye(n)


def _colmajor_dev(A):
    return torch.as_tensor(A, dtype=torch.float64, device="cuda").t().contiguous().t()


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dgemm_entries(lib):
    need = lib.qml_tune_table(None, 0)
    buf = ctypes.create_string_buffer(int(need) + 1)
    lib.qml_tune_table(buf, len(buf))
    return {ln.split()[0] for ln in buf.value.decode().splitlines() if ln.startswith("dgemm:")}


def _dev_pair(A):
    return _colmajor_dev(A), torch.zeros(1, dtype=torch.float64, device="cuda")


def _noalloc(lib, out, ld):
    n = out.shape[0]
    st = lib.qml_potrf_noalloc(n, out.data_ptr(), n, ld.data_ptr(), _stream())
    assert st == 0, lib.qml_last_error()


def _potrf(lib, A):
    ref = _colmajor_dev(A)
    ld = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.qml_potrf(A.shape[0], ref.data_ptr(), A.shape[0], ld.data_ptr(), 0, _stream())
    assert st == 0, lib.qml_last_error()
    return ref, ld


def _check_pair(lib, n, seed):
    """Two calls of qml_potrf_noalloc on n x n matrices.  The first may meet a
    shape nothing has tuned: the tuning table must gain no "dgemm:" entry.
    The second (same shape, another matrix) runs with every kernel module
    already loaded -- CUDA loads modules lazily on first use, which takes
    device memory for code and for the static scratch array itself -- and
    must leave free device memory unchanged.  Both match qml_potrf."""
    mats = [_spd(n, seed), _spd(n, seed + 1)]
    out0, ld0 = _dev_pair(mats[0])
    out1, ld1 = _dev_pair(mats[1])  # every buffer exists before memory is read
    torch.cuda.synchronize()
    tuned0 = _dgemm_entries(lib)
    _noalloc(lib, out0, ld0)
    assert _dgemm_entries(lib) == tuned0, "qml_potrf_noalloc ran the allocating tile autotuner"
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    _noalloc(lib, out1, ld1)
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0, (free0, free1)
    for A, out, ld in ((mats[0], out0, ld0), (mats[1], out1, ld1)):
        ref, ld_ref = _potrf(lib, A)
        L, Lr = torch.tril(out).cpu().numpy(), torch.tril(ref).cpu().numpy()
        assert np.abs(L - Lr).max() <= 1e-12 * np.abs(Lr).max(), n
        assert abs(ld.item() - ld_ref.item()) <= 1e-12 * abs(ld_ref.item())


def test_noalloc_first_on_unseen_shapes(lib):
    """Shapes no other test factors (ragged tails of 59 and 55 columns), run
    through qml_potrf_noalloc before qml_potrf has tuned them."""
    for n in (1531, 2999):
        _check_pair(lib, n, 7000 + n)


@pytest.mark.parametrize("sizes", [(1000, 257), (4096, 65)])
def test_noalloc_matches_potrf_two_calls(lib, sizes):
    for n in sizes:
        _check_pair(lib, n, 100 + n)


def test_noalloc_rejects_oversize_and_host(lib):
    n = 4097
    A = torch.eye(8, dtype=torch.float64, device="cuda")
    st = lib.qml_potrf_noalloc(n, A.data_ptr(), n, None, _stream())
    assert st == 1 and b"4096" in lib.qml_last_error()
    h = np.eye(4)
    st = lib.qml_potrf_noalloc(4, h.ctypes.data, 4, None, _stream())
    assert st == 1 and b"device pointers" in lib.qml_last_error()
