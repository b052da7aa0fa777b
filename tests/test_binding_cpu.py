"""The Python binding's argument checks, on the host: every tensor is checked
against the others (dtype, layout, row counts, device) before the library is
called, so that no kernel can read or write past a buffer.  The library is
replaced by a recorder and the device test by "yes", so the checks run on CPU
tensors; a 'meta' tensor stands in for an argument on another device."""
import pytest
import torch

from paper_2105_00039_gb300 import ugmech as U


class _Recorder:
    """Stands in for the loaded library: records each call, returns success."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if not name.startswith("ug_"):
            raise AttributeError(name)

        def fn(*args):
            self.calls.append((name, args))
            return 1024 if name.endswith("_bytes") else 0
        return fn


@pytest.fixture
def rec(monkeypatch):
    r = _Recorder()
    monkeypatch.setattr(U, "load", lambda *a, **k: r)
    monkeypatch.setattr(U, "_on_gpu", lambda t: True)
    monkeypatch.setattr(U, "_stream", lambda: None)
    monkeypatch.setattr(U, "workspace",
                        lambda nbytes, device: torch.empty(max(int(nbytes), 256), dtype=torch.uint8))
    return r


def _rows(n):
    return torch.rand(n, 4) + 1.0


def _ids(n):
    return torch.arange(n, dtype=torch.int32)


def _grid():
    return torch.zeros(101, dtype=torch.int32), torch.zeros(48, dtype=torch.uint8)


def test_valid_calls_reach_the_library_with_their_sizes(rec):
    st = _rows(10)
    U.grid_build(st, _ids(10), max_boxes=100)
    start, info = _grid()
    U.compute_forces(st, start, info)
    U.list_pairs(st, start, info, max_per_agent=8)
    U.forces_symmetric(st, start, info)
    U.forces_ladder(st, 2, max_boxes=100)
    U.apply_displacement(st, _rows(10), out=_rows(10))
    U.scatter_rows(st, _ids(10))
    U.gather_rows(st, _ids(10))
    U.step_backward(st, U.Params(), 2, 100, _rows(10))
    sp = U.Stepper(10, 100, torch.device("cpu"), nsims=2)
    sp.step(_rows(7), _ids(7), U.Params(), 1)
    sp.step(_rows(10), _ids(10), U.Params(), 1, pairs_once=True)

    class _Event:
        cuda_event = 0
    sp.step_traced(_rows(9), _ids(9), U.Params(), 1, [_Event()] * 7)
    sp.step_batched(_rows(10), _ids(10), torch.tensor([0, 4, 10], dtype=torch.int32),
                    torch.zeros(2, 7), 1)
    U.tune_batched(st, torch.tensor([0, 4, 10], dtype=torch.int32), torch.zeros(2, 7), 2, 100)
    names = [c[0] for c in rec.calls]
    for fn in ("ug_grid_build", "ug_compute_forces", "ug_list_pairs", "ug_forces_symmetric",
               "ug_forces_ladder", "ug_apply_displacement", "ug_scatter_rows", "ug_gather_rows",
               "ug_step_backward", "ug_step", "ug_step_pairs_once", "ug_step_traced",
               "ug_step_batched", "ug_tune_batched"):
        assert fn in names, fn
    steps = [c[1] for c in rec.calls if c[0] in ("ug_step", "ug_step_pairs_once")]
    assert [a[2] for a in steps] == [7, 10]           # the rows given, not the room held
    traced = [c[1] for c in rec.calls if c[0] == "ug_step_traced"]
    assert traced[0][2] == 9 and traced[0][-1] == 7


@pytest.mark.parametrize("case", [
    "force_rows", "out_rows", "perm_in_len", "scatter_perm_len", "gather_perm_dtype",
    "grad_out_rows", "box_start_dtype", "info_short", "status_dtype", "stepper_too_many",
    "stepper_perm_len", "sim_offset_len", "sim_offset_dtype", "params_dev_shape",
    "tune_params_shape", "other_device", "rows_shape", "rows_layout", "ws_dtype"])
def test_mismatched_arguments_are_refused_before_the_library(rec, case):
    st = _rows(10)
    start, info = _grid()
    off = torch.tensor([0, 4, 10], dtype=torch.int32)
    sp = U.Stepper(10, 100, torch.device("cpu"), nsims=2)
    calls = {
        "force_rows": lambda: U.apply_displacement(st, _rows(9)),
        "out_rows": lambda: U.apply_displacement(st, _rows(10), out=_rows(11)),
        "perm_in_len": lambda: U.grid_build(st, _ids(9), max_boxes=100),
        "scatter_perm_len": lambda: U.scatter_rows(st, _ids(9)),
        "gather_perm_dtype": lambda: U.gather_rows(st, torch.arange(10)),
        "grad_out_rows": lambda: U.step_backward(st, U.Params(), 2, 100, _rows(9)),
        "box_start_dtype": lambda: U.compute_forces(st, start.float(), info),
        "info_short": lambda: U.list_pairs(st, start, info[:40]),
        "status_dtype": lambda: U.forces_symmetric(st, start, info,
                                                   status=torch.zeros(1, dtype=torch.int64)),
        "stepper_too_many": lambda: sp.step(_rows(11), _ids(11), U.Params(), 1),
        "stepper_perm_len": lambda: sp.step(_rows(8), _ids(9), U.Params(), 1),
        "sim_offset_len": lambda: sp.step_batched(st, _ids(10), off[:2], torch.zeros(2, 7), 1),
        "sim_offset_dtype": lambda: sp.step_batched(st, _ids(10), off.long(), torch.zeros(2, 7), 1),
        "params_dev_shape": lambda: sp.step_batched(st, _ids(10), off, torch.zeros(3, 7), 1),
        "tune_params_shape": lambda: U.tune_batched(st, off, torch.zeros(2, 6), 2, 100),
        "other_device": lambda: U.apply_displacement(st, torch.empty(10, 4, device="meta")),
        "rows_shape": lambda: U.compute_forces(torch.rand(10, 3), start, info),
        "rows_layout": lambda: U.compute_forces(torch.rand(4, 10).t(), start, info),
        "ws_dtype": lambda: U.step_backward(st, U.Params(), 2, 100, _rows(10),
                                            ws=torch.empty(1024, dtype=torch.float32)),
    }
    before = len(rec.calls)
    with pytest.raises(ValueError):
        calls[case]()
    assert not [c for c in rec.calls[before:] if not c[0].endswith("_bytes")]
