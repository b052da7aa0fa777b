"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/ugmech.h declares, and its
argument validation answers before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2105_00039_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ugmech.h")


@pytest.fixture(scope="module")
def lib():
    path = _build.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ug_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ug_grid_build", "ug_compute_forces", "ug_apply_displacement", "ug_step",
                     "ug_step_batched", "ug_step_backward"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2105_00039_gb300 import ugmech
    assert sorted(ugmech.EXPORTED) == sorted(ugmech._SIG)
    assert set(declared_functions()) == set(ugmech.EXPORTED)


def test_built_for_sm103a_only():
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_strerror_and_version(lib):
    lib.ug_strerror.restype = ctypes.c_char_p
    assert lib.ug_strerror(0) == b"ok"
    assert b"max_boxes" in lib.ug_strerror(-3)
    assert lib.ug_version() >= 10000


def test_workspace_sizes_monotone(lib):
    lib.ug_workspace_bytes.restype = ctypes.c_size_t
    lib.ug_backward_workspace_bytes.restype = ctypes.c_size_t
    a = lib.ug_workspace_bytes(1000, 1, 1000)
    b = lib.ug_workspace_bytes(2000, 1, 1000)
    c = lib.ug_workspace_bytes(1000, 1, 5000)
    d = lib.ug_workspace_bytes(1000, 64, 1000)   # one grid record per simulation
    assert a % 256 == 0 and a < b and a < c and a < d
    assert b - a >= 1000 * (16 + 4 * 4)
    e = lib.ug_backward_workspace_bytes(1000, 1000, 10)
    f = lib.ug_backward_workspace_bytes(1000, 1000, 20)
    assert e > a and f - e >= 10 * 1000 * 36


class _Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in
                ("k", "gamma", "adherence", "dt", "density", "max_disp", "contact_margin")]


def test_argument_validation_without_device(lib):
    P = ctypes.c_void_p
    lib.ug_step.argtypes = [P, P, ctypes.c_uint32, _Params, ctypes.c_int32, ctypes.c_uint32, P,
                            ctypes.c_size_t, P, P]
    p = _Params(2, 1, 0.1, 1, 0.02, 3, 0)
    assert lib.ug_step(None, None, 0, p, 1, 100, None, 0, None, None) == 0      # n = 0: no-op
    assert lib.ug_step(None, None, 10, p, 0, 100, None, 0, None, None) == 0     # nsteps = 0
    assert lib.ug_step(None, None, 10, p, -1, 100, None, 0, None, None) == -1   # nsteps < 0
    assert lib.ug_step(None, None, 10, p, 1, 100, None, 0, None, None) == -1    # null pointers
    fake = ctypes.c_void_p(0x10000)
    bad_align = ctypes.c_void_p(0x10008)
    assert lib.ug_step(bad_align, fake, 10, p, 1, 100, fake, 1 << 30, fake, None) == -1
    assert lib.ug_step(fake, fake, 10, p, 1, 10, fake, 1 << 30, fake, None) == -1   # max_boxes < 27
    assert lib.ug_step(fake, fake, 10, p, 1, 100, fake, 16, fake, None) == -5       # workspace
    neg = _Params(2, 1, 0.1, 1, 0.02, 3, -1)
    assert lib.ug_step(fake, fake, 10, neg, 1, 100, fake, 1 << 30, fake, None) == -1
    lib.ug_grid_build.argtypes = [P, P, ctypes.c_uint32, ctypes.c_float, P, P, P, ctypes.c_uint32,
                                  P, P, ctypes.c_size_t, P, P]
    assert lib.ug_grid_build(fake, None, 10, 0.0, fake, fake, fake, 100, fake, fake, 16, fake,
                             None) == -5
    lib.ug_step_batched.argtypes = [P, P, P, ctypes.c_uint32, ctypes.c_uint32, P, ctypes.c_int32,
                                    ctypes.c_uint32, P, P, ctypes.c_size_t, P, P]
    assert lib.ug_step_batched(fake, fake, fake, 0, 10, fake, 1, 100, None, fake, 1 << 30, fake,
                               None) == -1                                          # nsims = 0


def test_ladder_validation_without_device(lib):
    P = ctypes.c_void_p
    lib.ug_ladder_workspace_bytes.restype = ctypes.c_size_t
    lib.ug_forces_ladder.argtypes = [ctypes.c_int32, P, ctypes.c_uint32, _Params, ctypes.c_uint32,
                                     P, P, ctypes.c_size_t, P, P]
    p = _Params(2, 1, 0.1, 1, 0.02, 3, 0)
    fake = ctypes.c_void_p(0x10000)
    need = lib.ug_ladder_workspace_bytes(1000, 5000)
    assert need >= lib.ug_workspace_bytes(1000, 1, 5000) + 4 * (1000 + 5000)
    for bad_version in (-1, 4):
        assert lib.ug_forces_ladder(bad_version, fake, 10, p, 100, fake, fake, 1 << 30, fake,
                                    None) == -1
    assert lib.ug_forces_ladder(0, fake, 0, p, 100, None, None, 0, None, None) == 0   # n = 0
    assert lib.ug_forces_ladder(1, None, 10, p, 100, fake, fake, 1 << 30, fake, None) == -1
    assert lib.ug_forces_ladder(2, fake, 10, p, 10, fake, fake, 1 << 30, fake, None) == -1
    assert lib.ug_forces_ladder(3, fake, 1000, p, 5000, fake, fake, need - 1, fake, None) == -5


def test_agent_count_limit_without_device(lib):
    P = ctypes.c_void_p
    lib.ug_step.argtypes = [P, P, ctypes.c_uint32, _Params, ctypes.c_int32, ctypes.c_uint32, P,
                            ctypes.c_size_t, P, P]
    p = _Params(2, 1, 0.1, 1, 0.02, 3, 0)
    fake = ctypes.c_void_p(0x10000)
    too_many = (1 << 30) + 1
    assert lib.ug_step(fake, fake, too_many, p, 1, 100, fake, 1 << 62, fake, None) == -1
    lib.ug_iota.argtypes = [P, ctypes.c_uint32, P]
    assert lib.ug_iota(fake, too_many, None) == -1


def test_every_entry_point_validates_without_device():
    """Each call below fails its host-side checks (or is a documented no-op)
    before any device work: fake but aligned pointers, one bad argument each."""
    from paper_2105_00039_gb300 import ugmech as U
    lib = U.load()
    P = ctypes.c_void_p
    p = U.Params().c()
    neg = U.Params(contact_margin=-1.0).c()
    fake = P(0x10000)
    odd = P(0x10008)                  # 8-byte aligned only
    big = 1 << 62                     # workspace size that passes every size check
    over = 0x7fffff01                 # max_boxes above 2^31 - 256
    too_many = (1 << 30) + 1
    EINVAL, EWORKSPACE = U.UG_EINVAL, U.UG_EWORKSPACE

    # forces, pairs, displacement
    assert lib.ug_compute_forces(None, None, None, 0, p, None, None, None) == 0
    assert lib.ug_compute_forces(fake, fake, fake, too_many, p, fake, fake, None) == EINVAL
    assert lib.ug_compute_forces(odd, fake, fake, 10, p, fake, fake, None) == EINVAL
    assert lib.ug_compute_forces(fake, None, fake, 10, p, fake, fake, None) == EINVAL
    assert lib.ug_compute_forces(fake, fake, fake, 10, p, odd, fake, None) == EINVAL
    assert lib.ug_compute_forces(fake, fake, fake, 10, p, fake, None, None) == EINVAL
    assert lib.ug_list_pairs(fake, fake, fake, 10, 0.0, 8, fake, None, fake, None) == EINVAL
    assert lib.ug_list_pairs(fake, fake, fake, 10, 0.0, 0, None, None, fake, None) == EINVAL
    assert lib.ug_apply_displacement(fake, fake, 10, p, fake, odd, fake, None) == EINVAL
    assert lib.ug_apply_displacement(fake, fake, 10, p, None, None, fake, None) == EINVAL

    # grid build
    gb = lambda mb, m, bs: lib.ug_grid_build(fake, None, 10, m, fake, fake, bs, mb, fake, fake,
                                             big, fake, None)
    assert gb(over, 0.0, fake) == EINVAL
    assert gb(100, -1.0, fake) == EINVAL
    assert gb(100, 0.0, P(0x10004)) == EINVAL          # box table not 16-byte aligned

    # fused steps
    for step in (lib.ug_step, lib.ug_step_pairs_once):
        assert step(fake, fake, 10, p, -1, 100, fake, big, fake, None) == EINVAL
        assert step(fake, fake, 10, p, 1, 26, fake, big, fake, None) == EINVAL
        assert step(fake, fake, 10, p, 1, over, fake, big, fake, None) == EINVAL
        assert step(fake, fake, 10, neg, 1, 100, fake, big, fake, None) == EINVAL
        assert step(fake, fake, 10, p, 1, 100, odd, big, fake, None) == EINVAL   # ws alignment
        assert step(fake, fake, 10, p, 1, 100, fake, 16, fake, None) == EWORKSPACE
    events = (ctypes.c_void_p * 6)()
    assert lib.ug_step_traced(fake, fake, 10, p, 1, 100, fake, big, fake, None, None, 7) == EINVAL
    assert lib.ug_step_traced(fake, fake, 10, p, 1, 100, fake, big, fake, None, events, 6) == EINVAL

    # batched and its tuner
    def tuning(block, apl, mode):
        t = U.ug_tuning()
        t.sweep_block, t.agents_per_lane, t.pair_mode = block, apl, mode
        return ctypes.byref(t)
    sb = lambda mb, t: lib.ug_step_batched(fake, fake, fake, 2, 10, fake, 1, mb, t, fake, big,
                                           fake, None)
    assert sb(over, None) == EINVAL
    assert sb(100, tuning(96, 2, 0)) == EINVAL
    assert sb(100, tuning(128, 3, 0)) == EINVAL
    assert sb(100, tuning(128, 2, 2)) == EINVAL
    assert lib.ug_step_batched(fake, fake, fake, 2, 10, fake, 1, 100, None, fake, 16, fake,
                               None) == EWORKSPACE
    best = U.ug_tuning()
    assert lib.ug_tune_batched(fake, fake, 2, 10, fake, 100, None, fake, big, None) == EINVAL
    assert lib.ug_tune_batched(None, None, 0, 0, None, 0, ctypes.byref(best), None, 0, None) == 0
    assert (best.sweep_block, best.agents_per_lane, best.pair_mode) == (128, 2, 0)
    assert lib.ug_tune_batched(fake, fake, 0, 10, fake, 100, ctypes.byref(best), fake, big,
                               None) == EINVAL
    assert lib.ug_tune_batched(fake, fake, 2, 10, fake, over, ctypes.byref(best), fake, big,
                               None) == EINVAL
    assert lib.ug_tune_batched(fake, fake, 2, 10, fake, 100, ctypes.byref(best), fake, 16,
                               None) == EWORKSPACE

    # adjoint (n > 0 and nsteps > 0 throughout: the zero cases touch the device)
    bw = lambda ck, mb, prm, ws_bytes, gp=fake, st=fake: lib.ug_step_backward(
        ck, 10, prm, 2, mb, fake, fake, gp, fake, ws_bytes, st, None)
    assert lib.ug_step_backward(fake, 10, p, -1, 100, fake, fake, fake, fake, big, fake,
                                None) == EINVAL
    assert bw(fake, 100, p, big, gp=None) == EINVAL
    assert bw(fake, 100, p, big, st=None) == EINVAL
    assert bw(odd, 100, p, big) == EINVAL
    assert bw(fake, 26, p, big) == EINVAL
    assert bw(fake, over, p, big) == EINVAL
    assert bw(fake, 100, neg, big) == EINVAL
    assert bw(fake, 100, p, 16) == EWORKSPACE

    # every pair once, forces only
    fs = lambda ws, ws_bytes: lib.ug_forces_symmetric(1, fake, fake, fake, 10, p, fake, ws,
                                                      ws_bytes, fake, None)
    assert fs(odd, big) == EINVAL
    assert fs(fake, 32 * 10 - 1) == EWORKSPACE

    # row reordering helpers
    for fn in (lib.ug_scatter_rows, lib.ug_gather_rows):
        assert fn(odd, fake, 10, fake, None) == EINVAL
        assert fn(fake, None, 10, fake, None) == EINVAL
        assert fn(fake, fake, 10, odd, None) == EINVAL
        assert fn(fake, fake, too_many, fake, None) == EINVAL
