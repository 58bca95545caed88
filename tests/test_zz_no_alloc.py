"""symctr_contract_static_scratch: the contraction for callers that cannot
allocate device memory (they receive only their input and output buffers), so
the library uses its own static device array as scratch.

Its results are compared, through the C ABI, with the CPU float64 oracle and,
bit for bit, with symctr_contract on a caller-provided workspace (the same
kernels on the same inputs are deterministic), on two calls in a row with
different inputs: the static array keeps the previous call's contents, so the
second call checks that nothing stale leaks through.  This file is collected
last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import workloads as WL

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the split-BF16 tolerance used by the parity tests


def spec(t):
    return (t.signs, t.charge, t.dims)


def rel_np(a, b):
    n = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (n if n > 0 else 1.0))


@pytest.fixture(scope="module")
def sc():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    import paper_2007_08056_gb300 as mod
    mod.load()
    return mod


def test_static_scratch_matches_oracle_and_workspace_path(sc):
    c = WL.Z3_ORDER4
    plan = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "split_bf16")
    o = O.plan(c.einsum, O.Group(c.moduli), O.Sym(*spec(c.u)), O.Sym(*spec(c.v)))
    assert plan.info.workspace_bytes <= 64 << 20
    for seed in (0, 1):
        uh = WL.draw(c.u, c.moduli, seed=c.u.seed + 100 * seed)
        vh = WL.draw(c.v, c.moduli, seed=c.v.seed + 100 * seed)
        u, v = torch.from_numpy(uh).cuda(), torch.from_numpy(vh).cuda()
        ref = plan.contract(u, v)
        out = torch.full_like(ref, float("nan"))
        plan.contract_static_scratch(u, v, out=out)
        torch.cuda.synchronize()
        plan.check_static_scratch_error()
        assert torch.equal(out, ref)
        assert rel_np(out.cpu().numpy(), O.contract_blockloop(o, uh, vh)) <= TOL


def test_static_scratch_split_k_path(sc):
    """The MPS contraction X.A uses split-K: its int64 partial sums live in the
    shared array and must be cleared on every call."""
    g = (WL.MPS_G,)
    Eh, Ah = WL.draw(WL.MPS_E, g), WL.draw(WL.MPS_A, g)
    E, A = torch.from_numpy(Eh).cuda(), torch.from_numpy(Ah).cuda()
    p1 = sc.Plan(WL.MPS_STEP1, g, spec(WL.MPS_E), spec(WL.MPS_A), "split_bf16")
    X = p1.contract(E, A)
    p2 = sc.Plan(WL.MPS_STEP2, g, p1.sym_w, spec(WL.MPS_A), "split_bf16")
    assert p2.info.workspace_bytes <= 64 << 20
    sw = p1.sym_w
    o2 = O.plan(WL.MPS_STEP2, O.Group(g), O.Sym(sw.signs, sw.charge, sw.dims), O.Sym(*spec(WL.MPS_A)))
    Xh = X.cpu().numpy()
    for scale in (1.0, -3.0):
        ref = p2.contract(X * scale, A)
        out = torch.full_like(ref, float("nan"))
        p2.contract_static_scratch(X * scale, A, out=out)
        torch.cuda.synchronize()
        p2.check_static_scratch_error()
        assert torch.equal(out, ref)
        assert rel_np(out.cpu().numpy(), O.contract_blockloop(o2, Xh * scale, Ah)) <= TOL


def test_static_scratch_allocates_nothing(sc):
    """Once warm, a call changes neither torch's allocation count nor the
    device's free memory."""
    c = WL.Z3_ORDER4
    plan = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "split_bf16")
    u, v = (torch.from_numpy(x).cuda() for x in WL.draw_pair(c))
    out = torch.empty(plan.shape_w, dtype=torch.float64, device="cuda")
    plan.contract_static_scratch(u, v, out=out)   # warm: module load, symbol lookup
    torch.cuda.synchronize()
    lib = ctypes.CDLL(sc.library_path())
    before_alloc = torch.cuda.memory_allocated()
    free_before, _ = torch.cuda.mem_get_info()
    st = lib.symctr_contract_static_scratch(ctypes.c_void_p(plan._h.value), ctypes.c_void_p(u.data_ptr()),
                                            ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == 0
    assert torch.cuda.memory_allocated() == before_alloc
    assert torch.cuda.mem_get_info()[0] == free_before


def test_static_scratch_streams_over_irreps(sc):
    """A plan whose one-pass workspace exceeds the 64 MiB array but whose
    smallest pass fits runs in several passes over Q."""
    c = WL.cc_ladder(8, 96, 32)
    plan = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "split_bf16")
    assert plan.info.workspace_bytes_min <= 64 << 20 < plan.info.workspace_bytes
    uh, vh = WL.draw_pair(c)
    u, v = torch.from_numpy(uh).cuda(), torch.from_numpy(vh).cuda()
    out = torch.full(plan.shape_w, float("nan"), dtype=torch.float64, device="cuda")
    plan.contract_static_scratch(u, v, out=out)
    torch.cuda.synchronize()
    plan.check_static_scratch_error()
    o = O.plan(c.einsum, O.Group(c.moduli), O.Sym(*spec(c.u)), O.Sym(*spec(c.v)))
    assert rel_np(out.cpu().numpy(), O.contract_blockloop(o, uh, vh)) <= TOL


def test_static_scratch_rejects_oversized_plans(sc):
    c = WL.cc_ladder(8, 160, 64)
    plan = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "split_bf16")
    assert plan.info.workspace_bytes_min > 64 << 20
    u = torch.zeros(plan.shape_u, dtype=torch.float64, device="cuda")
    v = torch.zeros(plan.shape_v, dtype=torch.float64, device="cuda")
    with pytest.raises(sc.SymctrError) as ei:
        plan.contract_static_scratch(u, v)
    assert ei.value.status == 7
    assert "static scratch" in str(ei.value)


def test_static_scratch_reports_nonfinite_input(sc):
    """A non-finite input is recorded in the static array's error word and
    read back (and cleared) through symctr_check_device_error(NULL)."""
    c = WL.Z3_ORDER4
    plan = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "split_bf16")
    uh, vh = WL.draw_pair(c)
    uh = uh.copy()
    uh.flat[17] = np.nan
    u, v = torch.from_numpy(uh).cuda(), torch.from_numpy(vh).cuda()
    out = torch.empty(plan.shape_w, dtype=torch.float64, device="cuda")
    plan.contract_static_scratch(u, v, out=out)
    with pytest.raises(sc.SymctrError) as ei:
        plan.check_static_scratch_error()
    assert ei.value.status == 11
    plan.check_static_scratch_error()   # the word was cleared
