"""Python binding of libugmech (include/ugmech.h) through ctypes.

Argument marshalling only: every step of the mechanical-interaction path runs in
the library's CUDA kernels.  PyTorch provides device memory and the stream.
There is no CPU fallback: if the library cannot be loaded, every call raises.

Row layout: float32 tensors of shape (n, 4) = (x, y, z, diameter), contiguous on
the GPU.  Ids, permutations and box tables are int32 tensors (read as uint32 by
the library; values stay below 2^31).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, fields

import torch

from . import _build

_LIB = None

UG_OK, UG_EINVAL, UG_EBADSTATE, UG_EGRID_TOO_LARGE = 0, -1, -2, -3
UG_ECAPACITY, UG_EWORKSPACE, UG_ETIMEOUT, UG_ECUDA = -4, -5, -6, -7

EXPORTED = ("ug_strerror", "ug_version", "ug_workspace_bytes", "ug_grid_build",
            "ug_compute_forces", "ug_list_pairs", "ug_apply_displacement", "ug_step",
            "ug_step_traced",
            "ug_step_batched", "ug_tune_batched", "ug_backward_workspace_bytes",
            "ug_step_backward", "ug_iota", "ug_scatter_rows", "ug_gather_rows",
            "ug_grid_build_noalloc", "ug_ladder_workspace_bytes", "ug_forces_ladder",
            "ug_forces_symmetric", "ug_step_pairs_once")


class UgError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class ug_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in
                ("k", "gamma", "adherence", "dt", "density", "max_disp", "contact_margin")]


class ug_grid_info(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_float * 3), ("edge", ctypes.c_float),
                ("dims", ctypes.c_int32 * 3), ("box_base", ctypes.c_uint32),
                ("nboxes", ctypes.c_uint32), ("agent_base", ctypes.c_uint32),
                ("nagents", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class ug_tuning(ctypes.Structure):
    _fields_ = [("sweep_block", ctypes.c_int32), ("agents_per_lane", ctypes.c_int32),
                ("pair_mode", ctypes.c_int32), ("neighbour_walk", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 4)]


assert ctypes.sizeof(ug_grid_info) == 48


@dataclass
class Params:
    """Eq. 1's kappa (k) and gamma, and the displacement rules of Sec. III."""
    k: float = 2.0
    gamma: float = 1.0
    adherence: float = 0.1
    dt: float = 1.0
    density: float = 0.02
    max_disp: float = 3.0
    contact_margin: float = 0.0

    def c(self) -> ug_params:
        return ug_params(*[float(getattr(self, f.name)) for f in fields(self)])

    def as_tensor(self, device) -> torch.Tensor:
        return torch.tensor([float(getattr(self, f.name)) for f in fields(self)],
                            dtype=torch.float32, device=device)


_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
_SIG = {
    "ug_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "ug_version": (ctypes.c_int, []),
    "ug_workspace_bytes": (ctypes.c_size_t, [_U32, _U32, _U32]),
    "ug_grid_build": (ctypes.c_int, [_P, _P, _U32, ctypes.c_float, _P, _P, _P, _U32, _P, _P,
                                     ctypes.c_size_t, _P, _P]),
    "ug_grid_build_noalloc": (ctypes.c_int, [_P, _P, _U32, ctypes.c_float, _P, _P, _P, _U32, _P,
                                             _P, _P]),
    "ug_compute_forces": (ctypes.c_int, [_P, _P, _P, _U32, ug_params, _P, _P, _P]),
    "ug_list_pairs": (ctypes.c_int, [_P, _P, _P, _U32, ctypes.c_float, _U32, _P, _P, _P, _P]),
    "ug_apply_displacement": (ctypes.c_int, [_P, _P, _U32, ug_params, _P, _P, _P, _P]),
    "ug_step": (ctypes.c_int, [_P, _P, _U32, ug_params, ctypes.c_int32, _U32, _P,
                               ctypes.c_size_t, _P, _P]),
    "ug_step_pairs_once": (ctypes.c_int, [_P, _P, _U32, ug_params, ctypes.c_int32, _U32, _P,
                               ctypes.c_size_t, _P, _P]),
    "ug_step_traced": (ctypes.c_int, [_P, _P, _U32, ug_params, ctypes.c_int32, _U32, _P,
                                      ctypes.c_size_t, _P, _P, ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.c_int32]),
    "ug_step_batched": (ctypes.c_int, [_P, _P, _P, _U32, _U32, _P, ctypes.c_int32, _U32,
                                       ctypes.POINTER(ug_tuning), _P, ctypes.c_size_t, _P, _P]),
    "ug_tune_batched": (ctypes.c_int, [_P, _P, _U32, _U32, _P, _U32, ctypes.POINTER(ug_tuning),
                                       _P, ctypes.c_size_t, _P]),
    "ug_backward_workspace_bytes": (ctypes.c_size_t, [_U32, _U32, ctypes.c_int32]),
    "ug_step_backward": (ctypes.c_int, [_P, _U32, ug_params, ctypes.c_int32, _U32, _P, _P, _P,
                                        _P, ctypes.c_size_t, _P, _P]),
    "ug_iota": (ctypes.c_int, [_P, _U32, _P]),
    "ug_ladder_workspace_bytes": (ctypes.c_size_t, [_U32, _U32]),
    "ug_forces_symmetric": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _U32, ug_params, _P, _P,
                                           ctypes.c_size_t, _P, _P]),
    "ug_forces_ladder": (ctypes.c_int, [ctypes.c_int32, _P, _U32, ug_params, _U32, _P, _P,
                                        ctypes.c_size_t, _P, _P]),
    "ug_scatter_rows": (ctypes.c_int, [_P, _P, _U32, _P, _P]),
    "ug_gather_rows": (ctypes.c_int, [_P, _P, _U32, _P, _P]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libugmech.so (building it first if asked).  Raises if unavailable."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libugmech not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIG.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load(False).ug_strerror(code).decode()
    except Exception:
        return f"status {code}"


# ------------------------------------------------------------------ marshalling
def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# Argument checks.  Every tensor handed to the library is checked for dtype,
# layout and size against the others before any call, so that no kernel reads
# or writes past a buffer; the device is checked last (one helper, _on_gpu).
def _on_gpu(t: torch.Tensor) -> bool:
    return t.is_cuda


def _device(t: torch.Tensor, name: str, device=None):
    if not _on_gpu(t):
        raise ValueError(f"{name} must be a CUDA tensor")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, the other arguments on {device}")


def _rows(t: torch.Tensor, name: str, n: int | None = None, device=None) -> torch.Tensor:
    if not (t.dtype == torch.float32 and t.dim() == 2 and t.shape[1] == 4 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 tensor of shape (n, 4)")
    if n is not None and t.shape[0] != n:
        raise ValueError(f"{name} must have {n} rows, not {t.shape[0]}")
    _device(t, name, device)
    return t


def _ids(t: torch.Tensor, n: int, name: str, device=None) -> torch.Tensor:
    if not (t.dtype == torch.int32 and t.numel() == n and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous int32 tensor with {n} entries")
    _device(t, name, device)
    return t


def _buf(t: torch.Tensor, dtype, numel: int, name: str, device, exact: bool = False):
    """A contiguous buffer of `dtype` with at least (or, exact, exactly) `numel` entries."""
    ok = t.dtype == dtype and t.is_contiguous() and (t.numel() == numel if exact else
                                                     t.numel() >= numel)
    if not ok:
        raise ValueError(f"{name} must be a contiguous {dtype} tensor with "
                         f"{'' if exact else 'at least '}{numel} entries")
    _device(t, name, device)
    return t


def _grid(box_start: torch.Tensor, info: torch.Tensor, device):
    """The box table and grid record of grid_build: int32 [max_boxes + 1], 48 bytes."""
    _buf(box_start, torch.int32, 28, "box_start", device)
    _buf(info, torch.uint8, 48, "info", device)


def _batch(sim_offset: torch.Tensor, params_dev: torch.Tensor, nsims: int, device):
    """Per-simulation arguments of the batched calls: int32 [nsims + 1] offsets
    and float32 [nsims, 7] parameter rows, on the rows' device."""
    _buf(sim_offset, torch.int32, nsims + 1, "sim_offset", device, exact=True)
    if not (params_dev.dtype == torch.float32 and params_dev.dim() == 2 and
            tuple(params_dev.shape) == (nsims, 7) and params_dev.is_contiguous()):
        raise ValueError(f"params_dev must be a contiguous float32 tensor of shape ({nsims}, 7)")
    _device(params_dev, "params_dev", device)


def _status(status: torch.Tensor | None, device) -> torch.Tensor:
    if status is None:
        return new_status(device)
    return _buf(status, torch.int32, 1, "status", device)


def _check(rc: int, where: str):
    if rc != UG_OK:
        raise UgError(rc, where)


def new_status(device) -> torch.Tensor:
    return torch.zeros(1, dtype=torch.int32, device=device)


def check_status(status: torch.Tensor, where: str = "device"):
    """Synchronise with the status word and raise if a kernel reported an error."""
    code = int(status.item())
    if code != UG_OK:
        raise UgError(code, where)


def workspace(nbytes: int, device) -> torch.Tensor:
    """A 256-byte aligned byte buffer (torch's allocator aligns to 512)."""
    t = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    if t.data_ptr() % 256:
        raise RuntimeError("workspace allocation is not 256-byte aligned")
    return t


def estimate_max_boxes(state: torch.Tensor, contact_margin: float = 0.0, slack: float = 1.5,
                       extra_extent: float = 0.0) -> int:
    """Box-table capacity for a population (host-side sizing of the workspace).

    dims per axis = extent / edge + 3; `slack` multiplies the product and
    `extra_extent` pads each axis for agents that will move."""
    lo = state[:, :3].amin(0).double().cpu()
    hi = state[:, :3].amax(0).double().cpu()
    e = float(state[:, 3].amax().item()) + 2.0 * contact_margin
    dims = [math.floor((float(hi[a] - lo[a]) + 2 * extra_extent) / e) + 4 for a in range(3)]
    return int(max(27, math.ceil(dims[0] * dims[1] * dims[2] * slack)))


def grid_info_from_bytes(raw: torch.Tensor) -> dict:
    b = bytes(raw.cpu().numpy().tobytes())
    g = ug_grid_info.from_buffer_copy(b[:48])
    return dict(origin=list(g.origin), edge=g.edge, dims=list(g.dims), box_base=g.box_base,
                nboxes=g.nboxes, agent_base=g.agent_base, nagents=g.nagents, reserved=g.reserved)


# ------------------------------------------------------------------ entry points
def version() -> int:
    return load().ug_version()


def workspace_bytes(n: int, nsims: int, max_boxes: int) -> int:
    return int(load().ug_workspace_bytes(n, nsims, max_boxes))


def grid_build(state: torch.Tensor, perm_in: torch.Tensor | None = None,
               contact_margin: float = 0.0, max_boxes: int | None = None,
               status: torch.Tensor | None = None, check: bool = True):
    """Uniform grid (Sec. IV-A): returns (state_sorted, perm_sorted, box_start,
    info_bytes, status)."""
    lib = load()
    _rows(state, "state")
    n = state.shape[0]
    dev = state.device
    if perm_in is not None:
        _ids(perm_in, n, "perm_in", dev)
    status = _status(status, dev)
    if max_boxes is None:
        max_boxes = estimate_max_boxes(state, contact_margin, slack=1.0)
    st_sorted = torch.empty_like(state)
    perm_sorted = torch.empty(n, dtype=torch.int32, device=dev)
    box_start = torch.zeros(max_boxes + 1, dtype=torch.int32, device=dev)
    info = torch.zeros(48, dtype=torch.uint8, device=dev)
    ws = workspace(lib.ug_workspace_bytes(n, 1, max_boxes), dev)
    rc = lib.ug_grid_build(_ptr(state), _ptr(perm_in), n, float(contact_margin), _ptr(st_sorted),
                           _ptr(perm_sorted), _ptr(box_start), max_boxes, _ptr(info), _ptr(ws),
                           ws.numel(), _ptr(status), _stream())
    _check(rc, "ug_grid_build")
    if check:
        check_status(status, "ug_grid_build")
    return st_sorted, perm_sorted, box_start, info, status


def compute_forces(state_sorted, box_start, info, params: Params = Params(), status=None,
                   check: bool = True) -> torch.Tensor:
    """(Fx, Fy, Fz, contacts) per sorted row (Eq. 1 over the 27-box neighbourhood)."""
    lib = load()
    _rows(state_sorted, "state_sorted")
    n = state_sorted.shape[0]
    _grid(box_start, info, state_sorted.device)
    status = _status(status, state_sorted.device)
    force = torch.empty_like(state_sorted)
    rc = lib.ug_compute_forces(_ptr(state_sorted), _ptr(box_start), _ptr(info), n, params.c(),
                               _ptr(force), _ptr(status), _stream())
    _check(rc, "ug_compute_forces")
    if check:
        check_status(status, "ug_compute_forces")
    return force


def list_pairs(state_sorted, box_start, info, contact_margin: float = 0.0,
               max_per_agent: int = 64, status=None, check: bool = True):
    """Contact lists: (count[n], nbr[n, max_per_agent]) in sorted-row indices."""
    lib = load()
    _rows(state_sorted, "state_sorted")
    n = state_sorted.shape[0]
    _grid(box_start, info, state_sorted.device)
    status = _status(status, state_sorted.device)
    count = torch.empty(n, dtype=torch.int32, device=state_sorted.device)
    nbr = torch.full((n, max_per_agent), -1, dtype=torch.int32, device=state_sorted.device)
    rc = lib.ug_list_pairs(_ptr(state_sorted), _ptr(box_start), _ptr(info), n,
                           float(contact_margin), max_per_agent, _ptr(count), _ptr(nbr),
                           _ptr(status), _stream())
    _check(rc, "ug_list_pairs")
    if check:
        check_status(status, "ug_list_pairs")
    return count, nbr


def forces_symmetric(state_sorted, box_start, info, params: Params = Params(),
                     each_pair_once: bool = True, status=None, check: bool = True) -> torch.Tensor:
    """(Fx, Fy, Fz, contacts) per sorted row with Newton's third law: each pair
    evaluated once and added to both agents (fixed-point sums), or from both
    sides when each_pair_once is False (same bits)."""
    lib = load()
    _rows(state_sorted, "state_sorted")
    n = state_sorted.shape[0]
    _grid(box_start, info, state_sorted.device)
    status = _status(status, state_sorted.device)
    force = torch.empty_like(state_sorted)
    ws = workspace(32 * n + 256, state_sorted.device)
    rc = lib.ug_forces_symmetric(int(bool(each_pair_once)), _ptr(state_sorted), _ptr(box_start),
                                 _ptr(info), n, params.c(), _ptr(force), _ptr(ws), ws.numel(),
                                 _ptr(status), _stream())
    _check(rc, "ug_forces_symmetric")
    if check:
        check_status(status, "ug_forces_symmetric")
    return force


def forces_ladder(state, version: int, params: Params = Params(), max_boxes: int | None = None,
                  status=None, check: bool = True) -> torch.Tensor:
    """The paper's GPU version `version` (0..3) of the force computation:
    (Fx, Fy, Fz, contacts) per row in the caller's order, float64."""
    lib = load()
    _rows(state, "state")
    n = state.shape[0]
    if max_boxes is None:
        max_boxes = estimate_max_boxes(state, params.contact_margin)
    ws = workspace(lib.ug_ladder_workspace_bytes(n, max_boxes), state.device)
    force = torch.empty((n, 4), dtype=torch.float64, device=state.device)
    status = _status(status, state.device)
    rc = lib.ug_forces_ladder(int(version), _ptr(state), n, params.c(), max_boxes, _ptr(force),
                              _ptr(ws), ws.numel(), _ptr(status), _stream())
    _check(rc, "ug_forces_ladder")
    if check:
        check_status(status, "ug_forces_ladder")
    return force


def apply_displacement(state, force, params: Params = Params(), out=None, want_disp=True,
                       status=None, check: bool = True):
    """Adherence, integration and cap (Sec. III): returns (new_state, disp)."""
    lib = load()
    _rows(state, "state")
    n = state.shape[0]
    dev = state.device
    _rows(force, "force", n, dev)
    out = torch.empty_like(state) if out is None else _rows(out, "out", n, dev)
    disp = torch.empty_like(state) if want_disp else None
    status = _status(status, dev)
    rc = lib.ug_apply_displacement(_ptr(state), _ptr(force), n, params.c(), _ptr(out), _ptr(disp),
                                   _ptr(status), _stream())
    _check(rc, "ug_apply_displacement")
    if check:
        check_status(status, "ug_apply_displacement")
    return out, disp


class Stepper:
    """Holds the workspace for repeated fused steps on populations of up to n
    agents (and up to nsims simulations, max_boxes boxes in total).

    step() advances `state` (m, 4) and `perm` (m,) in place, m <= n; both stay
    on the device in box order.  Calls are asynchronous; status is checked on
    demand."""

    def __init__(self, n: int, max_boxes: int, device, nsims: int = 1):
        self.lib = load()
        self.n, self.max_boxes, self.nsims = int(n), int(max_boxes), int(nsims)
        self.ws = workspace(self.lib.ug_workspace_bytes(self.n, self.nsims, self.max_boxes), device)
        self.status = new_status(device)

    def _agents(self, state, perm) -> int:
        _rows(state, "state")
        m = state.shape[0]
        if m > self.n:
            raise ValueError(f"state has {m} rows; this Stepper has room for {self.n}")
        _ids(perm, m, "perm")
        _device(state, "state", self.ws.device)
        _device(perm, "perm", self.ws.device)
        return m

    def step(self, state, perm, params: Params, nsteps: int = 1, pairs_once: bool = False):
        """nsteps fused steps; pairs_once selects ug_step_pairs_once (each pair
        evaluated once, faster on dense grids)."""
        m = self._agents(state, perm)
        fn = self.lib.ug_step_pairs_once if pairs_once else self.lib.ug_step
        rc = fn(_ptr(state), _ptr(perm), m, params.c(), int(nsteps), self.max_boxes,
                _ptr(self.ws), self.ws.numel(), _ptr(self.status), _stream())
        _check(rc, "ug_step_pairs_once" if pairs_once else "ug_step")

    def step_traced(self, state, perm, params: Params, nsteps: int, events):
        """step() with caller-created torch.cuda.Event objects recorded between
        kernels (len(events) >= 2 + 5 * nsteps; each must have been recorded once
        so that its CUDA handle exists)."""
        m = self._agents(state, perm)
        arr = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
        rc = self.lib.ug_step_traced(_ptr(state), _ptr(perm), m, params.c(), int(nsteps),
                                     self.max_boxes, _ptr(self.ws), self.ws.numel(),
                                     _ptr(self.status), _stream(), arr, len(events))
        _check(rc, "ug_step_traced")

    def step_batched(self, state, perm, sim_offset, params_dev, nsteps: int = 1,
                     tuning: ug_tuning | None = None):
        """nsteps fused steps of every simulation: sim_offset (nsims + 1,) int32
        on the device, sim_offset[nsims] = number of rows; params_dev (nsims, 7)."""
        m = self._agents(state, perm)
        _batch(sim_offset, params_dev, self.nsims, self.ws.device)
        rc = self.lib.ug_step_batched(_ptr(state), _ptr(perm), _ptr(sim_offset), self.nsims,
                                      m, _ptr(params_dev), int(nsteps), self.max_boxes,
                                      ctypes.byref(tuning) if tuning is not None else None,
                                      _ptr(self.ws), self.ws.numel(), _ptr(self.status),
                                      _stream())
        _check(rc, "ug_step_batched")

    def check(self, where="ug_step"):
        check_status(self.status, where)


class BatchedGraph:
    """Many simulations advanced by one CUDA-graph launch: ug_step_batched for
    nsteps steps, captured once and replayed.

    state, perm, sim_offset and params_dev are the caller's device tensors; the
    graph reads and writes them in place at every replay (their addresses are
    fixed at capture, their contents are not), so a caller refills state and
    perm between replays as it likes.  Construction runs the step once
    uncaptured on scratch copies (so that every kernel is loaded before the
    capture) and leaves the caller's tensors untouched.  A replay runs on the
    current stream; stepper.check() reads the status after it."""

    def __init__(self, stepper: "Stepper", state, perm, sim_offset, params_dev, nsteps: int,
                 tuning: ug_tuning | None = None):
        self.stepper = stepper
        dev = state.device
        stepper.step_batched(state.clone(), perm.clone(), sim_offset, params_dev, nsteps, tuning)
        torch.cuda.current_stream(dev).synchronize()
        stepper.check("BatchedGraph warm-up")
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side):
                stepper.step_batched(state, perm, sim_offset, params_dev, nsteps, tuning)
        torch.cuda.current_stream(dev).wait_stream(side)

    def replay(self):
        self.graph.replay()


def iota(n: int, device) -> torch.Tensor:
    p = torch.empty(n, dtype=torch.int32, device=device)
    _check(load().ug_iota(_ptr(p), n, _stream()), "ug_iota")
    return p


def scatter_rows(rows, perm):
    """rows_by_id[perm[s]] = rows[s]."""
    _rows(rows, "rows")
    _ids(perm, rows.shape[0], "perm", rows.device)
    out = torch.empty_like(rows)
    _check(load().ug_scatter_rows(_ptr(rows), _ptr(perm), rows.shape[0], _ptr(out), _stream()),
           "ug_scatter_rows")
    return out


def gather_rows(rows_by_id, perm):
    """rows[s] = rows_by_id[perm[s]]."""
    _rows(rows_by_id, "rows_by_id")
    _ids(perm, rows_by_id.shape[0], "perm", rows_by_id.device)
    out = torch.empty_like(rows_by_id)
    _check(load().ug_gather_rows(_ptr(rows_by_id), _ptr(perm), rows_by_id.shape[0], _ptr(out),
                                 _stream()), "ug_gather_rows")
    return out


def simulate(state_by_id: torch.Tensor, params: Params = Params(), nsteps: int = 1,
             max_boxes: int | None = None) -> torch.Tensor:
    """Public one-call API: nsteps fused steps of a population given in id order
    (host or device tensor); returns the final rows in id order on the same
    device as the input."""
    host = not state_by_id.is_cuda
    dev = torch.device("cuda") if host else state_by_id.device
    st = state_by_id.to(dev, non_blocking=True).contiguous()
    if st is state_by_id:
        st = st.clone()
    n = st.shape[0]
    if max_boxes is None:
        max_boxes = estimate_max_boxes(st, params.contact_margin,
                                       extra_extent=params.max_disp * nsteps if nsteps < 8 else 0.0)
    sp = Stepper(n, max_boxes, dev)
    perm = iota(n, dev)
    sp.step(st, perm, params, nsteps)
    out = scatter_rows(st, perm)
    sp.check("simulate")
    return out.to("cpu") if host else out


class Simulation:
    """User-facing runner for one population size: takes rows in id order from
    host (pinned) memory, runs nsteps fused steps on the GPU and returns the rows
    in id order to host memory.  Device buffers and the workspace are reused
    between calls."""

    def __init__(self, n: int, max_boxes: int, device="cuda"):
        self.n = int(n)
        self.device = torch.device(device)
        self.stepper = Stepper(n, max_boxes, self.device)
        self.x = torch.empty((n, 4), dtype=torch.float32, device=self.device)
        self.perm = torch.empty(n, dtype=torch.int32, device=self.device)
        self.by_id = torch.empty_like(self.x)

    def run(self, state_host: torch.Tensor, params: Params, nsteps: int,
            out_host: torch.Tensor | None = None, pairs_once: bool = False,
            sync: bool = True) -> torch.Tensor:
        """Rows in id order in, nsteps steps, rows in id order out.  With sync
        (the default) the call waits for the copy back and raises on a device
        error; with sync=False the caller synchronises the current stream and
        calls stepper.check() before reading out_host."""
        if out_host is None:
            out_host = torch.empty((self.n, 4), dtype=torch.float32, pin_memory=True)
        self.x.copy_(state_host, non_blocking=True)
        lib = self.stepper.lib
        _check(lib.ug_iota(_ptr(self.perm), self.n, _stream()), "ug_iota")
        self.stepper.step(self.x, self.perm, params, nsteps, pairs_once=pairs_once)
        _check(lib.ug_scatter_rows(_ptr(self.x), _ptr(self.perm), self.n, _ptr(self.by_id),
                                   _stream()), "ug_scatter_rows")
        out_host.copy_(self.by_id, non_blocking=True)
        if sync:
            torch.cuda.current_stream(self.device).synchronize()
            self.stepper.check("Simulation.run")
        return out_host


def backward_workspace_bytes(n: int, max_boxes: int, nsteps: int) -> int:
    return int(load().ug_backward_workspace_bytes(n, max_boxes, nsteps))


def step_backward(ckpt_state, params: Params, nsteps: int, max_boxes: int, grad_out,
                  ws=None, status=None):
    """dL/d(ckpt rows) and (dL/dk, dL/dgamma) for nsteps steps from ckpt_state."""
    lib = load()
    _rows(ckpt_state, "ckpt_state")
    n = ckpt_state.shape[0]
    dev = ckpt_state.device
    _rows(grad_out, "grad_out", n, dev)
    status = _status(status, dev)
    if ws is None:
        ws = workspace(lib.ug_backward_workspace_bytes(n, max_boxes, nsteps), dev)
    else:
        _buf(ws, torch.uint8, 256, "ws", dev)
    grad_in = torch.empty_like(ckpt_state)
    gp = torch.zeros(2, dtype=torch.float32, device=dev)
    rc = lib.ug_step_backward(_ptr(ckpt_state), n, params.c(), int(nsteps), max_boxes,
                              _ptr(grad_out), _ptr(grad_in), _ptr(gp), _ptr(ws), ws.numel(),
                              _ptr(status), _stream())
    _check(rc, "ug_step_backward")
    return grad_in, gp, status


def tune_batched(state, sim_offset, params_dev, nsims: int, max_boxes: int) -> ug_tuning:
    """The fastest (sweep_block, agents_per_lane, pair_mode, neighbour_walk) for
    these simulations, timed on scratch copies of the rows (state is only read)."""
    lib = load()
    _rows(state, "state")
    _batch(sim_offset, params_dev, nsims, state.device)
    n = state.shape[0]
    ws = workspace(lib.ug_workspace_bytes(n, nsims, max_boxes) + 20 * n + 1024, state.device)
    best = ug_tuning()
    rc = lib.ug_tune_batched(_ptr(state), _ptr(sim_offset), nsims, n, _ptr(params_dev), max_boxes,
                             ctypes.byref(best), _ptr(ws), ws.numel(), _stream())
    _check(rc, "ug_tune_batched")
    return best
