"""Argument marshalling of the Python binding (host side, no GPU).

Inputs that already are float64 in the layout the C-ABI reads (contiguous
vectors; column-major matrices, any leading dimension >= rows) are passed in
place; everything else is converted once.  Either way the pointer handed to
the library must address the same values in the stated layout.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1907_01995_gb300 import api  # noqa: E402


def read(ptr, count):
    return np.ctypeslib.as_array((ctypes.c_double * count).from_address(ptr)).copy()


def read_colmajor(ptr, m, n, ld):
    flat = read(ptr, ld * (n - 1) + m)
    return np.stack([flat[j * ld: j * ld + m] for j in range(n)], axis=1)


def test_vec_in_place_and_converted():
    keep = api._Keep()
    a = torch.arange(7, dtype=torch.float64)
    assert keep.vec(a, 7) == a.data_ptr()                       # read in place
    f = torch.arange(7, dtype=torch.float32) / 3
    p = keep.vec(f, 7)
    assert p != f.data_ptr() and np.array_equal(read(p, 7), f.double().numpy())
    s = torch.arange(14, dtype=torch.float64)[::2]              # strided view
    p = keep.vec(s, 7)
    assert np.array_equal(read(p, 7), s.numpy())
    m = torch.arange(6, dtype=torch.float64).reshape(2, 3)       # contiguous 2-D: row-major flat
    assert np.array_equal(read(keep.vec(m, 6), 6), np.arange(6.0))
    n = np.linspace(0.0, 1.0, 5)
    assert np.array_equal(read(keep.vec(n, 5), 5), n)
    with pytest.raises(ValueError):
        keep.vec(a, 8)
    with pytest.raises(ValueError):
        keep.vec(n, 4)
    assert keep.vec(None) is None


@pytest.mark.parametrize("kind", ["colmajor", "padded", "rowmajor", "float32", "numpy_c",
                                  "numpy_f"])
def test_colmajor_layouts(kind):
    rng = np.random.default_rng(3)
    m, n = 7, 5
    ref = rng.normal(size=(m, n))
    keep = api._Keep()
    if kind == "colmajor":
        a = torch.tensor(ref).t().contiguous().t()
    elif kind == "padded":
        big = torch.zeros((n, m + 3), dtype=torch.float64)
        big[:, :m] = torch.tensor(ref.T)
        a = big.t()[:m]
    elif kind == "rowmajor":
        a = torch.tensor(ref)
    elif kind == "float32":
        a = torch.tensor(ref, dtype=torch.float32).t().contiguous().t()
        ref = a.double().numpy()
    elif kind == "numpy_c":
        a = np.ascontiguousarray(ref)
    else:
        a = np.asfortranarray(ref)
    ptr, rows, cols, ld = keep.colmajor(a)
    assert (rows, cols) == (m, n) and ld >= m
    if kind in ("colmajor", "padded"):
        assert ptr == a.data_ptr()                                 # read in place
        assert ld == a.stride(1)
    assert np.array_equal(read_colmajor(ptr, m, n, ld), ref)


def test_make_problem_points_at_the_data():
    rng = np.random.default_rng(5)
    A = rng.normal(size=(9, 4))
    b = rng.normal(size=9)
    keep = api._Keep()
    At = torch.tensor(A).t().contiguous().t()
    bt = torch.tensor(b)
    pr = api.make_problem(keep, At, bt, phi="l1l2", lambda1=0.25)
    assert (pr.m, pr.n, pr.lda) == (9, 4, 9)
    assert pr.A == At.data_ptr() and pr.b == bt.data_ptr()
    assert np.array_equal(read_colmajor(pr.A, 9, 4, pr.lda), A)
    assert pr.lambda1 == 0.25
    pr2 = api.make_problem(api._Keep(), A, b, phi="l1l2", lambda1=0.25)
    assert (pr2.m, pr2.n, pr2.lda) == (9, 4, 9)


def test_stream_handle_without_a_device_is_the_default_stream():
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    assert api._stream_handle(None) == 0
    assert api._stream_handle(1234) == 1234
