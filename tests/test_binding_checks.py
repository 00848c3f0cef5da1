"""Length checks of the Python binding (no GPU): every vector handed to the C ABI must have
exactly the entries of its grid level, since the library receives bare pointers.  A stand-in
for the loaded library answers the size queries; CPU tensors of the right length get past the
length check and stop at the CUDA-tensor check, wrong lengths stop at the length check."""
import ctypes

import pytest
import torch

from paper_1604_07994_gb300 import sdx

N = 4  # finest grid 4^3 cells, level 1 has 2^3 cells


class _FakeLib:
    """Answers sdx_level_size / sdx_batch_size; any compute entry point would be a test bug."""

    def sdx_level_size(self, h, level, pn, pnodes, pfree):
        n = N >> level
        pn._obj.value, pnodes._obj.value, pfree._obj.value = n, (n + 1) ** 3, 0
        return sdx.OK

    def sdx_batch_size(self, h, i, pn, pnodes, pfree):
        n = (4, 2)[i]
        pn._obj.value, pnodes._obj.value, pfree._obj.value = n, (n + 1) ** 3, 0
        return sdx.OK

    def __getattr__(self, name):
        def entry(*args):
            raise AssertionError(f"{name} reached the library")
        return entry


@pytest.fixture
def hier(monkeypatch):
    monkeypatch.setattr(sdx, "_lib", _FakeLib())
    H = sdx.Hierarchy.__new__(sdx.Hierarchy)
    H._h, H._borrowed, H.n, H.nn = ctypes.c_void_p(1), True, N, (N + 1) ** 3
    return H


def _v(m, dtype=torch.float64):
    return torch.zeros(m, dtype=dtype)


NN0, NN1 = (N + 1) ** 3, (N // 2 + 1) ** 3


def _calls(H, good0, good1, good0_f32, f3):
    return [
        lambda: H.sdx_apply(0, good0, good0),
        lambda: H.sdx_residual(0, good0, good0, good0),
        lambda: H.sdx_rhs(f3, good0),
        lambda: H.sdx_uzawa(0, good0, good0),
        lambda: H.sdx_smooth_pass(0, 0, 0, good0, good0),
        lambda: H.sdx_smooth_pass_noalloc(0, 0, good0, good0),
        lambda: H.sdx_apply_f32(0, good0_f32, good0_f32),
        lambda: H.sdx_smooth_pass_f32(0, 1, 0, good0_f32, good0_f32),
        lambda: H.sdx_restrict(0, good0, good1),
        lambda: H.sdx_prolong_add(0, good1, good0),
        lambda: H.sdx_apply(1, good1, good1),
        lambda: H.sdx_vcycle(good0, good0),
        lambda: H.sdx_solve(good0, good0),
    ]


def test_right_lengths_pass_the_length_check(hier):
    for call in _calls(hier, _v(4 * NN0), _v(4 * NN1), _v(4 * NN0, torch.float32), _v(3 * NN0)):
        with pytest.raises(ValueError, match="CUDA"):
            call()


@pytest.mark.parametrize("k", range(13))
def test_wrong_lengths_are_rejected(hier, k):
    """One argument of each entry point one element short (or the fine/coarse vectors of the
    transfers swapped)."""
    good0, good1 = _v(4 * NN0), _v(4 * NN1)
    short0 = _v(4 * NN0 - 1)
    f32 = _v(4 * NN0, torch.float32)
    bad = [
        lambda: hier.sdx_apply(0, good0, short0),
        lambda: hier.sdx_residual(0, good0, short0, good0),
        lambda: hier.sdx_rhs(_v(3 * NN0 + 1), good0),
        lambda: hier.sdx_uzawa(0, short0, good0),
        lambda: hier.sdx_smooth_pass(0, 0, 0, good0, short0),
        lambda: hier.sdx_smooth_pass_noalloc(0, 0, short0, good0),
        lambda: hier.sdx_apply_f32(0, f32, _v(4 * NN0 - 1, torch.float32)),
        lambda: hier.sdx_smooth_pass_f32(0, 1, 0, _v(4 * NN0 + 4, torch.float32), f32),
        lambda: hier.sdx_restrict(0, good1, good0),
        lambda: hier.sdx_prolong_add(0, good0, good1),
        lambda: hier.sdx_apply(1, good0, good0),
        lambda: hier.sdx_vcycle(good0, short0),
        lambda: hier.sdx_solve(short0, good0),
    ]
    with pytest.raises(ValueError, match="elements where"):
        bad[k]()


def test_raw_pointers_are_passed_through(hier):
    assert sdx._vecs((1234, 10), (None, 10)) == [1234, None]


def test_batch_vectors_are_checked_per_instance(monkeypatch):
    monkeypatch.setattr(sdx, "_lib", _FakeLib())
    B = sdx.Batch.__new__(sdx.Batch)
    B._h, B.count = ctypes.c_void_p(1), 2
    B._lens = [4 * B.sdx_batch_size(i)[1] for i in range(2)]
    assert B._lens == [4 * 125, 4 * 27]
    good = [_v(500), _v(108)]
    with pytest.raises(ValueError, match="2 instances"):
        B.sdx_batch_solve(good[:1], good[:1])
    with pytest.raises(ValueError, match="elements where"):
        B.sdx_batch_vcycle([good[0], _v(107)], good)
    with pytest.raises(ValueError, match="CUDA"):
        B.sdx_batch_solve(good, good)
    B._h = None  # nothing to free
