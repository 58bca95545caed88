"""Backward (adjoint) contractions on shapes that take the tcgen05 path.

gU = einsum(w, v -> u)(gW, V) and gV = einsum(u, w -> v)(U, gW) are themselves
irrep-aligned contractions (the adjoint of Alg. 2's contraction step); here
their aligned GEMMs are at least 128 x 128 x 128 per irrep, so the split-BF16
and TF32 forms run on the tensor cores (asserted through plan.info.tensor_core
of the equivalent forward plans).  Results are compared with the oracle's
gradients (oracle.grad_u / grad_v, the block loop of the adjoint contractions)
in full at the reduced CC-ladder size, and on per-tile samples at a sweep
point, at each form's tolerance.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as WL
from test_gpu_configs import TOL, oplan, spec, tile_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sc():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    import paper_2007_08056_gb300 as mod
    mod.load()
    return mod


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def adjoint_plans(sc, p, precision):
    """The forward plans equivalent to the library's two backward contractions."""
    lhs, lw = p.einsum.replace(" ", "").split("->")
    lu, lv = lhs.split(",")
    bu = sc.Plan(f"{lw},{lv}->{lu}", p.moduli, p.sym_w, p.sym_v, precision, sym_w=p.sym_u)
    bv = sc.Plan(f"{lu},{lw}->{lv}", p.moduli, p.sym_u, p.sym_w, precision, sym_w=p.sym_v)
    return bu, bv


@pytest.mark.parametrize("precision", ["split_bf16", "tf32"])
def test_backward_cc_ladder_reduced(sc, precision):
    """CC ladder at virtual 8 x 8, occupied 8 x 4: forward M = K = 512, N = 128;
    the adjoints are 512 x 512 x 128 (gU) and 512 x 128 x 512 (gV) per irrep."""
    c = WL.cc_ladder(8, 64, 32)
    p = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), precision)
    assert (p.info.M, p.info.K, p.info.N) == (512, 512, 128)
    for q in adjoint_plans(sc, p, precision):
        assert q.info.tensor_core == 1
    u, v = WL.draw_pair(c)
    gw = np.random.default_rng(3901).standard_normal(p.shape_w)
    ud, vd, gwd = (torch.from_numpy(x).cuda() for x in (u, v, gw))
    gu, gv = p.backward(gwd, ud, vd)
    torch.cuda.synchronize()
    p.check_device_error()
    o = oplan(c)
    assert rel(gu.cpu().numpy(), O.grad_u(o, gw, v)) <= TOL[precision]
    assert rel(gv.cpu().numpy(), O.grad_v(o, u, gw)) <= TOL[precision]


@pytest.mark.parametrize("precision", ["split_bf16", "tf32"])
def test_autograd_function_cc_ladder_reduced(sc, precision):
    """SymContract (the torch.autograd.Function) on the same shapes: loss =
    <W, R>, so dL/dW = R and the gradients are the adjoint contractions of R."""
    c = WL.cc_ladder(8, 64, 32)
    p = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), precision)
    u, v = WL.draw_pair(c)
    r = np.random.default_rng(3902).standard_normal(p.shape_w)
    ud = torch.from_numpy(u).cuda().requires_grad_(True)
    vd = torch.from_numpy(v).cuda().requires_grad_(True)
    loss = (sc.contract(p, ud, vd) * torch.from_numpy(r).cuda()).sum()
    loss.backward()
    torch.cuda.synchronize()
    o = oplan(c)
    assert rel(ud.grad.cpu().numpy(), O.grad_u(o, r, v)) <= TOL[precision]
    assert rel(vd.grad.cpu().numpy(), O.grad_v(o, u, r)) <= TOL[precision]


@pytest.mark.parametrize("precision", ["split_bf16", "tf32"])
def test_backward_sweep_point_per_tile(sc, precision):
    """The CC-ladder sweep at G = 16, virtual 256, occupied 64 (forward M = K =
    4096, N = 256 per irrep), operands drawn on the device.  gU and gV are
    checked on one sample in every 128 x 128 tile of every irrep of their own
    aligned GEMMs."""
    torch.cuda.empty_cache()
    c = WL.cc_ladder(16, 256, 64)
    gen = torch.Generator(device="cuda").manual_seed(5216)
    u = torch.randn(WL.reduced_shape(c.moduli, c.u.dims), generator=gen, device="cuda",
                    dtype=torch.float64).mul_(c.u.scale)
    v = torch.randn(WL.reduced_shape(c.moduli, c.v.dims), generator=gen, device="cuda",
                    dtype=torch.float64).mul_(c.v.scale)
    p = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), precision)
    assert (p.info.M, p.info.K, p.info.N) == (4096, 4096, 256)
    bu, bv = adjoint_plans(sc, p, precision)
    assert bu.info.tensor_core == 1 and bv.info.tensor_core == 1
    gw = torch.randn(p.shape_w, generator=gen, device="cuda", dtype=torch.float64)
    gu, gv = p.backward(gw, u, v)
    torch.cuda.synchronize()
    p.check_device_error()
    lhs, lw = c.einsum.split("->")
    lu, lv = lhs.split(",")
    o = oplan(c)
    g = O.Group(c.moduli)
    ou = O.plan(f"{lw},{lv}->{lu}", g, o.sym_w, o.sym_v)
    ov = O.plan(f"{lu},{lw}->{lv}", g, o.sym_u, o.sym_w)
    err_u, n_u = tile_check(ou, gw, v, gu, per=1, seed=61)
    err_v, n_v = tile_check(ov, u, gw, gv, per=1, seed=62)
    assert n_u == 16 * 32 * 32 and n_v == 16 * 32 * 2
    assert err_u <= TOL[precision]
    assert err_v <= TOL[precision]
    del u, v, gw, gu, gv
    torch.cuda.empty_cache()
