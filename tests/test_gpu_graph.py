"""The batched step as one CUDA graph (ugmech.BatchedGraph) through the C ABI.

A replay must give the same bits as the uncaptured ug_step_batched call on the
same inputs, and a second replay after the caller refills its rows must give
them again (the graph reads the caller's buffers in place).  Construction must
leave the caller's rows untouched.
"""
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


@pytest.mark.parametrize("pair_mode", [0, 1])
def test_graph_replay_equals_uncaptured_call(U, pair_mode):
    st, offs = P.batched_population(nsims=12, nmin=300, nmax=6000, seed=4)
    n = len(st)
    x0 = torch.from_numpy(st).to(DEV)
    off_t = torch.from_numpy(offs.astype(np.int32)).to(DEV)
    pdev = torch.stack([U.Params(k=2.0 + 0.05 * s).as_tensor(DEV) for s in range(12)])
    parts = [x0[int(offs[k]):int(offs[k + 1])] for k in range(12)]
    mb = sum(4 * U.estimate_max_boxes(p, 0.0, slack=1.0, extra_extent=24.0) + 1000 for p in parts)
    t = U.ug_tuning()
    t.pair_mode = pair_mode
    # uncaptured reference
    sp = U.Stepper(n, mb, x0.device, nsims=12)
    xa, pa = x0.clone(), U.iota(n, x0.device)
    sp.step_batched(xa, pa, off_t, pdev, 10, t)
    sp.check("uncaptured")
    # the graph, on its own buffers
    sp2 = U.Stepper(n, mb, x0.device, nsims=12)
    xb, pb = x0.clone(), U.iota(n, x0.device)
    g = U.BatchedGraph(sp2, xb, pb, off_t, pdev, 10, t)
    torch.cuda.synchronize()
    assert torch.equal(xb, x0) and torch.equal(pb, U.iota(n, x0.device))
    for _ in range(2):
        xb.copy_(x0)
        pb.copy_(U.iota(n, x0.device))
        g.replay()
        torch.cuda.synchronize()
        sp2.check("replay")
        assert torch.equal(xb, xa) and torch.equal(pb, pa)
