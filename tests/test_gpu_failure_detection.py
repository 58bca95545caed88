"""Failure detection without a GPU fault: a kernel whose bounded wait runs out
(on a barrier that nothing completes) records the timeout in the workspace's
error word and returns; the host reads the status, and the context goes on
to run a correct contraction."""
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


def test_bounded_wait_expires_and_is_reported(sc):
    c = WL.Z3_ORDER4
    p = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "split_bf16")
    ws = torch.zeros(int(p.info.workspace_bytes), dtype=torch.uint8, device="cuda")
    sc.selftest_bounded_wait(ws, wait_cycles=2_000_000)   # ~1 ms
    with pytest.raises(sc.SymctrError) as ei:
        p.check_device_error(ws)
    assert ei.value.status == 9           # SYMCTR_ERR_DEVICE_TIMEOUT
    p.check_device_error(ws)              # the word was cleared
    # the context is intact: a contraction on the same stream is still correct
    u, v = WL.draw_pair(c)
    w = p.contract(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), workspace=ws)
    torch.cuda.synchronize()
    p.check_device_error(ws)
    o = O.plan(c.einsum, O.Group(c.moduli), O.Sym(*spec(c.u)), O.Sym(*spec(c.v)))
    want = O.contract_blockloop(o, u, v)
    assert np.linalg.norm(w.cpu().numpy() - want) <= 1e-10 * np.linalg.norm(want)


def test_selftest_argument_errors(sc):
    small = torch.zeros(128, dtype=torch.uint8, device="cuda")
    with pytest.raises(sc.SymctrError) as ei:
        sc.selftest_bounded_wait(small)
    assert ei.value.status == 7           # SYMCTR_ERR_WORKSPACE
