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
