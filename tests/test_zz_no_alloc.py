"""The allocation-free grid build (ug_grid_build_noalloc) against ug_grid_build.

ug_grid_build_noalloc serves callers that may not allocate device memory when
they call the library (they get only their inputs and outputs), so it keeps its
scratch in a fixed array inside the library.  Its results must be the same as
ug_grid_build's -- exactly, since the grid is integer and index work -- on two
calls in a row, the second one reusing the scratch the first left behind.  This
file is collected last so that a run stopping at its first failure has already
run everything else.
"""
import ctypes

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


def _noalloc(U, x, margin, max_boxes, perm_in=None):
    n = x.shape[0]
    lib = U.load()
    srt = torch.empty_like(x)
    perm = torch.empty(n, dtype=torch.int32, device=DEV)
    start = torch.zeros(max_boxes + 1, dtype=torch.int32, device=DEV)
    info = torch.zeros(48, dtype=torch.uint8, device=DEV)
    status = U.new_status(DEV)
    rc = lib.ug_grid_build_noalloc(U._ptr(x), U._ptr(perm_in), n, float(margin), U._ptr(srt), U._ptr(perm),
                                   U._ptr(start), max_boxes, U._ptr(info), U._ptr(status),
                                   U._stream())
    assert rc == 0, U.strerror(rc)
    U.check_status(status, "ug_grid_build_noalloc")
    return srt, perm, start, info


def test_noalloc_grid_build_matches_workspace_version(U):
    cases = [(P.small_uniform(0), 0.0),
             (P.jittered_lattice(30000, 32, 9.0, 1.5, 9.0, 11.0, 3), 1.5)]
    for st, margin in cases:                       # two calls in a row, different inputs
        x = torch.from_numpy(st).to(DEV)
        mb = U.estimate_max_boxes(x, margin, slack=1.2)
        a_srt, a_perm, a_start, a_info, _ = U.grid_build(x, contact_margin=margin, max_boxes=mb)
        b_srt, b_perm, b_start, b_info = _noalloc(U, x, margin, mb)
        nb = U.grid_info_from_bytes(a_info)["nboxes"]
        assert torch.equal(a_info, b_info)
        assert torch.equal(a_start[: nb + 1], b_start[: nb + 1])
        assert torch.equal(a_perm, b_perm)
        assert torch.equal(a_srt, b_srt)


def test_noalloc_with_input_ids_and_after_a_failed_call(U):
    """Ids carried through the sort, and a call that fails (a NaN row: the
    bounds kernel records UG_EBADSTATE and the later kernels stop) followed by
    a clean call, which must still equal ug_grid_build: every call clears the
    parts of the shared scratch that must start at zero."""
    st = P.uniform_cube(5000, 90.0, 8.0, 12.0, 11)
    x = torch.from_numpy(st).to(DEV)
    ids = torch.from_numpy(np.random.default_rng(3).permutation(len(st)).astype(np.int32)).to(DEV)
    mb = U.estimate_max_boxes(x, 0.0, slack=1.2)
    a_srt, a_perm, a_start, a_info, _ = U.grid_build(x, perm_in=ids, max_boxes=mb)
    b_srt, b_perm, b_start, b_info = _noalloc(U, x, 0.0, mb, perm_in=ids)
    nb = U.grid_info_from_bytes(a_info)["nboxes"]
    assert torch.equal(a_info, b_info) and torch.equal(a_perm, b_perm)
    assert torch.equal(a_start[: nb + 1], b_start[: nb + 1]) and torch.equal(a_srt, b_srt)
    bad = st.copy()
    bad[1234, 1] = np.nan
    with pytest.raises(U.UgError) as e:
        _noalloc(U, torch.from_numpy(bad).to(DEV), 0.0, mb)
    assert e.value.code == U.UG_EBADSTATE
    c_srt, c_perm, c_start, c_info = _noalloc(U, x, 0.0, mb)
    a_srt, a_perm, a_start, a_info, _ = U.grid_build(x, max_boxes=mb)
    assert torch.equal(a_info, c_info) and torch.equal(a_perm, c_perm)
    assert torch.equal(a_start[: nb + 1], c_start[: nb + 1]) and torch.equal(a_srt, c_srt)


def test_noalloc_rejects_sizes_beyond_its_scratch(U):
    lib = U.load()
    big = 1 << 18
    x = torch.zeros((big + 1, 4), dtype=torch.float32, device=DEV)
    dummy = torch.zeros(16, dtype=torch.int32, device=DEV)
    rc = lib.ug_grid_build_noalloc(U._ptr(x), None, big + 1, 0.0, U._ptr(x), U._ptr(dummy),
                                   U._ptr(dummy), 1000, U._ptr(dummy), U._ptr(dummy), U._stream())
    assert rc == U.UG_EWORKSPACE
    rc = lib.ug_grid_build_noalloc(U._ptr(x), None, 10, 0.0, U._ptr(x), U._ptr(dummy),
                                   U._ptr(dummy), (1 << 20) + 1, U._ptr(dummy), U._ptr(dummy),
                                   U._stream())
    assert rc == U.UG_EWORKSPACE
    # argument checks come before the size limits, as in ug_grid_build
    rc = lib.ug_grid_build_noalloc(None, None, big + 1, 0.0, U._ptr(x), U._ptr(dummy),
                                   U._ptr(dummy), 1000, U._ptr(dummy), U._ptr(dummy), U._stream())
    assert rc == U.UG_EINVAL
