"""symctr_contract_static_scratch: the contraction for callers that cannot
allocate device memory (they receive only their input and output buffers), so
the library uses its own static device array as scratch.

Its results are compared, through the C ABI, with symctr_contract on a
caller-provided workspace, on two calls in a row with different inputs (the
static array keeps the previous call's contents, so the second call checks
that nothing stale leaks through).  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import workloads as WL

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the split-BF16 tolerance used by the parity tests


def spec(t):
    return (t.signs, t.charge, t.dims)


def rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    n = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (n if n > 0 else 1.0))


@pytest.fixture(scope="module")
def sc():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    import paper_2007_08056_gb300 as mod
    mod.load()
    return mod


def test_static_scratch_matches_workspace_path(sc):
    c = WL.Z3_ORDER4
    plan = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "split_bf16")
    assert plan.info.workspace_bytes <= 64 << 20
    for seed in (0, 1):
        u = torch.from_numpy(WL.draw(c.u, c.moduli, seed=c.u.seed + 100 * seed)).cuda()
        v = torch.from_numpy(WL.draw(c.v, c.moduli, seed=c.v.seed + 100 * seed)).cuda()
        ref = plan.contract(u, v)
        out = torch.full_like(ref, float("nan"))
        plan.contract_static_scratch(u, v, out=out)
        torch.cuda.synchronize()
        assert rel(out, ref) <= TOL


def test_static_scratch_split_k_path(sc):
    """The MPS contraction X.A uses split-K: its int64 partial sums live in the
    shared array and must be cleared on every call."""
    E = torch.from_numpy(WL.draw(WL.MPS_E, (8,))).cuda()
    A = torch.from_numpy(WL.draw(WL.MPS_A, (8,))).cuda()
    p1 = sc.Plan(WL.MPS_STEP1, (8,), spec(WL.MPS_E), spec(WL.MPS_A), "split_bf16")
    X = p1.contract(E, A)
    p2 = sc.Plan(WL.MPS_STEP2, (8,), p1.sym_w, spec(WL.MPS_A), "split_bf16")
    assert p2.info.workspace_bytes <= 64 << 20
    for scale in (1.0, -3.0):
        ref = p2.contract(X * scale, A)
        out = torch.full_like(ref, float("nan"))
        p2.contract_static_scratch(X * scale, A, out=out)
        torch.cuda.synchronize()
        assert rel(out, ref) <= TOL


def test_static_scratch_rejects_oversized_plans(sc):
    c = WL.cc_ladder(8, 128, 64)
    plan = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "split_bf16")
    assert plan.info.workspace_bytes > 64 << 20
    u = torch.zeros(plan.shape_u, dtype=torch.float64, device="cuda")
    v = torch.zeros(plan.shape_v, dtype=torch.float64, device="cuda")
    with pytest.raises(sc.SymctrError) as ei:
        plan.contract_static_scratch(u, v)
    assert ei.value.status == 7
    assert "static scratch" in str(ei.value)
