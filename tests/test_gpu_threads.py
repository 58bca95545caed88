"""Host threads: the library keeps its per-call caches per host thread and
initialises each plan's page-locked tables once, so plans may be used from
several threads, each on its own stream (and one plan from two threads with
separate workspaces)."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle as O
import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sc():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    import paper_2007_08056_gb300 as mod
    mod.load()
    return mod


def spec(t):
    return (t.signs, t.charge, t.dims)


def test_two_threads_two_streams(sc):
    c = WL.cc_ladder(8, 128, 64)
    u, v = WL.draw_pair(c)
    o = O.plan(c.einsum, O.Group(c.moduli), O.Sym(*spec(c.u)), O.Sym(*spec(c.v)))
    want = O.contract_blockloop(o, u, v)
    shared = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "split_bf16")
    ud, vd = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
    torch.cuda.synchronize()

    def work(k):
        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()
        own = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), ("split_bf16", "tf32")[k % 2])
        ws = torch.empty(int(shared.info.workspace_bytes), dtype=torch.uint8, device="cuda")
        outs = []
        with torch.cuda.stream(stream):
            for i in range(4):
                p = shared if i % 2 == 0 else own
                outs.append((p.info.precision, p.contract(ud, vd, workspace=ws if p is shared else None)))
            stream.synchronize()
        return [(prec, w.cpu().numpy()) for prec, w in outs]

    with ThreadPoolExecutor(max_workers=3) as ex:
        results = list(ex.map(work, range(3)))
    tol = {1: 1e-10, 2: 1e-2}
    for res in results:
        for prec, got in res:
            assert np.linalg.norm(got - want) <= tol[prec] * np.linalg.norm(want)
