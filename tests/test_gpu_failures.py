"""Failure detection on the GPU, injected from the host: every error becomes a
status code, later kernels of the call do nothing, and the context stays usable.
No test faults, traps or hangs a GPU."""
import numpy as np
import pytest
import torch

from paper_2105_00039_gb300 import populations as P

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def U():
    from paper_2105_00039_gb300 import ugmech
    ugmech.load()
    return ugmech


def _healthy(U):
    st = P.small_uniform(1)
    x = torch.from_numpy(st).to(DEV)
    srt, perm, start, info, status = U.grid_build(x)
    F = U.compute_forces(srt, start, info)
    assert int(status.item()) == 0 and torch.isfinite(F).all()


def test_error_stops_the_rest_of_the_call(U):
    st = P.small_uniform(2)
    st[5, 0] = np.nan
    x = torch.from_numpy(st).to(DEV)
    n = len(st)
    sp = U.Stepper(n, 100000, x.device)
    perm = U.iota(n, x.device)
    before = x.clone()
    sp.step(x, perm, U.Params(), 5)
    with pytest.raises(U.UgError) as e:
        sp.check()
    assert e.value.code == U.UG_EBADSTATE
    assert torch.equal(x[~torch.isnan(x)], before[~torch.isnan(before)])   # rows untouched
    _healthy(U)


def test_preset_status_makes_calls_no_ops(U):
    st = P.small_uniform(3)
    x = torch.from_numpy(st).to(DEV)
    status = U.new_status(DEV)
    status.fill_(U.UG_ECAPACITY)                          # an earlier error in the same call chain
    srt, perm, start, info, status = U.grid_build(x, status=status, check=False)
    assert int(status.item()) == U.UG_ECAPACITY
    assert int(start.abs().sum().item()) == 0             # nothing was written
    _healthy(U)


def test_workspace_too_small_is_rejected_on_the_host(U):
    lib = U.load()
    st = P.small_uniform(4)
    x = torch.from_numpy(st).to(DEV)
    ws = torch.empty(1024, dtype=torch.uint8, device=DEV)
    perm = U.iota(len(st), x.device)
    status = U.new_status(DEV)
    rc = lib.ug_step(U._ptr(x), U._ptr(perm), len(st), U.Params().c(), 1, 10000, U._ptr(ws),
                     ws.numel(), U._ptr(status), U._stream())
    assert rc == U.UG_EWORKSPACE and int(status.item()) == 0


def test_pairs_once_error_stops_the_rest_of_the_call(U):
    st = P.small_uniform(2)
    st[7, 1] = np.inf
    x = torch.from_numpy(st).to(DEV)
    sp = U.Stepper(len(st), 100000, x.device)
    perm = U.iota(len(st), x.device)
    before = x.clone()
    sp.step(x, perm, U.Params(), 5, pairs_once=True)
    with pytest.raises(U.UgError) as e:
        sp.check()
    assert e.value.code == U.UG_EBADSTATE
    assert torch.equal(x, before)                         # rows untouched
    _healthy(U)


def test_fixed_point_overflow_is_reported(U):
    """A force component beyond the fixed-point range (2^30) is recorded as
    UG_EBADSTATE instead of wrapping around silently."""
    st = P.small_uniform(5)
    x = torch.from_numpy(st).to(DEV)
    srt, perm, start, info, _ = U.grid_build(x)
    with pytest.raises(U.UgError) as e:
        U.forces_symmetric(srt, start, info, U.Params(k=1e12))
    assert e.value.code == U.UG_EBADSTATE
    _healthy(U)
