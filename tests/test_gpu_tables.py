"""The offset tables of the aligned forms (the same integers whichever way the
kernels reach them) read from page-locked host memory, copied into the
workspace, or from a device copy attached with symctr_plan_attach_tables give
bit-identical results, in one pass and with Q-streaming."""
import pytest
import torch

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


def raw_contract(sc, p, u, v, w, ws):
    """symctr_contract without the binding's automatic table attachment."""
    st = sc.load().symctr_contract(p._h, u.data_ptr(), v.data_ptr(), w.data_ptr(), ws.data_ptr(),
                                   ws.numel(), torch.cuda.current_stream().cuda_stream)
    assert st == 0, sc.load().symctr_last_error_detail()


CASES = {
    # tables below 1 MiB: read in place from host memory when not attached
    "mps_step1": lambda: (WL.MPS_STEP1, (8,), WL.MPS_E, WL.MPS_A),
    # tables above 1 MiB: copied into the workspace when not attached
    "cc_ladder_G8_V256_O64": lambda: (WL.CC_LADDER.einsum, WL.CC_LADDER.moduli, WL.CC_LADDER.u,
                                      WL.CC_LADDER.v),
}


@pytest.mark.parametrize("precision", ["split_bf16", "tf32"])
@pytest.mark.parametrize("case", list(CASES))
def test_attached_tables_bit_identical(sc, case, precision):
    es, moduli, tu, tv = CASES[case]()
    u = torch.from_numpy(WL.draw(tu, moduli)).cuda()
    v = torch.from_numpy(WL.draw(tv, moduli)).cuda()
    p = sc.Plan(es, moduli, spec(tu), spec(tv), precision)
    ws = p.workspace()
    host = torch.empty(p.shape_w, dtype=torch.float64, device="cuda")
    raw_contract(sc, p, u, v, host, ws)
    ws_min = torch.empty(int(p.info.workspace_bytes_min), dtype=torch.uint8, device="cuda")
    host_q = torch.empty_like(host)
    raw_contract(sc, p, u, v, host_q, ws_min)
    p.attach_tables()
    assert p._tables is not None and p._tables.numel() == p.info.table_bytes
    dev = p.contract(u, v)
    dev_q = p.contract(u, v, workspace=ws_min)
    torch.cuda.synchronize()
    p.check_device_error()
    p.check_device_error(ws_min)
    assert torch.equal(dev, host)
    assert torch.equal(dev_q, host_q)
    # detached: the host tables again
    assert sc.load().symctr_plan_attach_tables(p._h, None, 0, None) == 0
    again = torch.empty_like(host)
    raw_contract(sc, p, u, v, again, ws)
    torch.cuda.synchronize()
    assert torch.equal(again, host)
    del u, v, ws, ws_min, p
    torch.cuda.empty_cache()


def test_attach_rejects_small_buffer_on_device(sc):
    p = sc.Plan(WL.MPS_STEP1, (8,), spec(WL.MPS_E), spec(WL.MPS_A), "split_bf16")
    small = torch.empty(int(p.info.table_bytes) - 256, dtype=torch.uint8, device="cuda")
    st = sc.load().symctr_plan_attach_tables(p._h, small.data_ptr(), small.numel(),
                                            torch.cuda.current_stream().cuda_stream)
    assert st == 7
