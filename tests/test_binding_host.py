"""The Python binding's marshalling (paper_2605_21149_gb300/api.py), on the
host: every matrix handed to the C ABI is float64 and column-major (rows x
cols at the pointer, element (i, j) at i + j rows), whether it came as a
numpy array in either order, a row-major torch tensor, a column-major torch
view (passed through without a copy) or a vector."""
import ctypes

import numpy as np
import pytest

from paper_2605_21149_gb300 import api

torch = pytest.importorskip("torch")


def _read_colmajor(ptr, rows, cols):
    buf = (ctypes.c_double * (rows * cols)).from_address(ptr)
    return np.ctypeslib.as_array(buf).reshape(cols, rows).T.copy()


@pytest.mark.parametrize("order", ["C", "F"])
def test_numpy_matrix_is_column_major(order):
    x = np.arange(5 * 3, dtype=np.float32).reshape(5, 3).copy(order=order)
    keep = []
    p = api._mat(x, 5, 3, keep)
    np.testing.assert_array_equal(_read_colmajor(p, 5, 3), x.astype(np.float64))


def test_torch_row_major_is_copied_column_major():
    x = torch.arange(4 * 6, dtype=torch.float32).reshape(4, 6)
    keep = []
    p = api._mat(x, 4, 6, keep)
    np.testing.assert_array_equal(_read_colmajor(p, 4, 6), x.double().numpy())


def test_torch_column_major_view_passes_through():
    base = torch.randn(7, 5, dtype=torch.float64)  # contiguous (cols, rows)
    x = base.t()  # (5, 7) with strides (1, 5): column-major
    keep = []
    p = api._mat(x, 5, 7, keep)
    assert p == base.data_ptr()
    np.testing.assert_array_equal(_read_colmajor(p, 5, 7), x.numpy())


def test_vectors_and_flat_inputs():
    keep = []
    v = torch.arange(6, dtype=torch.int64)
    p = api._vec(v, keep)
    np.testing.assert_array_equal(_read_colmajor(p, 6, 1)[:, 0], np.arange(6, dtype=np.float64))
    # a flat array taken as a matrix is read column by column
    flat = np.arange(12, dtype=np.float64)
    p = api._mat(flat, 4, 3, keep)
    np.testing.assert_array_equal(_read_colmajor(p, 4, 3), flat.reshape(4, 3))
    # a one-column torch matrix given as a vector
    t = torch.arange(5, dtype=torch.float64)
    p = api._mat(t, 5, 1, keep)
    np.testing.assert_array_equal(_read_colmajor(p, 5, 1)[:, 0], t.numpy())
    assert api._vec(None, keep) is None


def test_host_outputs_are_column_major():
    out = api._empty(3, 4, False)
    assert out.shape == (3, 4) and out.flags["F_CONTIGUOUS"] and out.dtype == np.float64


def test_problem_struct_from_workload():
    """qml_problem filled from a workload in host mode: sizes, spectra ids,
    pointers to the geometry, transfer, spectra and the column-major noise."""
    from paper_2605_21149_gb300 import synth
    wl = synth.make_workload("QU nside4 lmax7", 4, 7, False, True, 30.0, ("EE", "BB", "EB"), 4, 3)
    edges = [3, 5, 7]  # bins l = 3..4 and 5..6 of the window
    prob = api.Problem.from_workload(wl, device=False, precision=1, bin_edges=edges,
                                     window=(3, 6), basis=api.BASIS_AUTO)
    p = prob._p
    assert (p.has_T, p.has_P) == (0, 1)
    assert p.npix_T == 0 and p.npix_P == len(wl.theta_P)
    assert prob.n == 2 * len(wl.theta_P) == wl.n
    assert (p.lmin, p.lmax) == (3, 6) and (p.lmin_sig, p.lmax_sig) == (wl.lmin, wl.lmax)
    assert p.nspec == 3 and [p.spec[i] for i in range(3)] == [1, 2, 5]
    assert p.precision == 1 and p.basis == api.BASIS_AUTO
    assert p.nbins == 2 and prob.na == 3 * 2
    got_edges = np.ctypeslib.as_array((ctypes.c_int32 * 3).from_address(p.bin_edges))
    np.testing.assert_array_equal(got_edges, edges)
    th = np.ctypeslib.as_array((ctypes.c_double * p.npix_P).from_address(p.theta_P))
    np.testing.assert_array_equal(th, wl.theta_P)
    cl = np.ctypeslib.as_array((ctypes.c_double * wl.cl_fid.size).from_address(p.cl_fid))
    np.testing.assert_array_equal(cl, wl.cl_fid.reshape(-1))
    np.testing.assert_array_equal(_read_colmajor(p.N, wl.n, wl.n), wl.N())
    assert not p.theta_T and not p.transfer_T
