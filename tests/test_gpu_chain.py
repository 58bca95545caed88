"""Contraction chains that stay aligned (Sec. 2.1: the aligned result W_hat is
itself a reduced form of W, with the extra symmetry mode Q): a plan chained
with w_aligned writes W_hat[b][m][n] without the map back of Alg. 2's output
step, and a plan chained with u_from / v_from reads that W_hat as its operand.

Checked against the oracle: the aligned result against the oracle's W_hat of
the standard result (align_w, the dense-delta route, at the irreps of the
plan's batches), the chained step's result against the oracle's block loop on
the standard forms, in every precision form.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as WL
from test_oracle_pins import random_general_case

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "split_bf16": 1e-10, "tf32": 1e-2}


@pytest.fixture(scope="module")
def sc():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    import paper_2007_08056_gb300 as mod
    mod.load()
    return mod


def spec(t):
    return (t.signs, t.charge, t.dims)


def osym(s):
    return O.Sym(s.signs, s.charge, s.dims, s.sectors, s.sector_dims)


def rel(a, b):
    n = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (n if n > 0 else 1.0))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("precision", ["fp64", "split_bf16", "tf32"])
def test_mps_transfer_chain(sc, precision):
    """X = E.A kept as X_hat, E' = X.A reading X_hat (config 2's two steps)."""
    g = (WL.MPS_G,)
    E, A = WL.draw(WL.MPS_E, g), WL.draw(WL.MPS_A, g)
    p1 = sc.Plan(WL.MPS_STEP1, g, spec(WL.MPS_E), spec(WL.MPS_A), precision).chain(w_aligned=True)
    p2 = sc.Plan(WL.MPS_STEP2, g, p1.sym_w, spec(WL.MPS_A), precision).chain(u_from=p1)
    Xh = p1.contract(dev(E), dev(A))
    E2 = p2.contract(Xh, dev(A))
    torch.cuda.synchronize()
    p1.check_device_error()
    p2.check_device_error()
    G = O.Group(g)
    o1 = O.plan(WL.MPS_STEP1, G, O.Sym(*spec(WL.MPS_E)), O.Sym(*spec(WL.MPS_A)))
    o2 = O.plan(WL.MPS_STEP2, G, o1.sym_w, O.Sym(*spec(WL.MPS_A)))
    X = O.contract_blockloop(o1, E, A)
    want_xh = O.align_w(o1, X)[p1.q_values()]
    assert tuple(Xh.shape) == want_xh.shape
    assert rel(Xh.cpu().numpy(), want_xh) <= TOL[precision]
    assert rel(E2.cpu().numpy(), O.contract_blockloop(o2, X, A)) <= 2 * TOL[precision]
    # a chained plan has no backward
    with pytest.raises(sc.SymctrError) as ei:
        p2.backward(torch.zeros(p2.shape_w, dtype=torch.float64, device="cuda"), Xh, dev(A))
    assert ei.value.status == 5


@pytest.mark.parametrize("precision", ["fp64", "split_bf16", "tf32"])
def test_chain_through_v(sc, precision):
    """W = U.V kept aligned and read as the second operand of Y = L.W, whose
    contracted mode is W's free-U mode (Z_4, tensor-core-sized blocks)."""
    rng = np.random.default_rng(8100)
    G = (4,)
    su, sv = ((1, -1), (1,), (40, 48)), ((1, -1), (2,), (48, 36))
    q1 = sc.Plan("ij,jk->ik", G, su, sv, precision).chain(w_aligned=True)
    sl = ((1, -1), (3,), (44, 40))
    q2 = sc.Plan("li,ik->lk", G, sl, q1.sym_w, precision).chain(v_from=q1)
    u = rng.standard_normal(q1.shape_u)
    v = rng.standard_normal(q1.shape_v)
    l = rng.standard_normal(q2.shape_u)
    Wh = q1.contract(dev(u), dev(v))
    Y = q2.contract(dev(l), Wh)
    torch.cuda.synchronize()
    q2.check_device_error()
    Gr = O.Group(G)
    o1 = O.plan("ij,jk->ik", Gr, O.Sym(*su), O.Sym(*sv))
    o2 = O.plan("li,ik->lk", Gr, O.Sym(*sl), o1.sym_w)
    W = O.contract_blockloop(o1, u, v)
    assert rel(Y.cpu().numpy(), O.contract_blockloop(o2, l, W)) <= 2 * TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_chain_general_symmetry(sc, precision):
    """A chain under sub-group coefficients and padded sectors: the aligned
    intermediate holds exact zeros where its entries are absent."""
    rng = np.random.default_rng(8200)
    G = O.Group((8,))
    H = {"a": 8, "b": 4, "c": 8, "d": 2}
    D = {"a": 12, "b": 16, "c": 12, "d": 10}
    SD = {c: tuple(int(rng.integers(D[c] // 2, D[c] + 1)) for _ in range(H[c])) for c in H}
    mk = lambda lab, signs, z: O.Sym(signs, z, tuple(D[c] for c in lab), tuple(H[c] for c in lab),
                                     tuple(SD[c] for c in lab))
    s_ab, s_bc, s_cd = mk("ab", (1, -1), (0,)), mk("bc", (1, -1), (4,)), mk("cd", (1, 1), (2,))
    o1 = O.plan("ab,bc->ac", G, s_ab, s_bc)
    o2 = O.plan("ac,cd->ad", G, o1.sym_w, s_cd)
    as_spec = lambda s: (s.signs, s.charge, s.dims, s.sectors, s.sector_dims)
    p1 = sc.Plan("ab,bc->ac", (8,), as_spec(s_ab), as_spec(s_bc), precision).chain(w_aligned=True)
    p2 = sc.Plan("ac,cd->ad", (8,), p1.sym_w, as_spec(s_cd), precision).chain(u_from=p1)
    a = O.sanitize(G, s_ab, rng.standard_normal(O.reduced_shape(G, s_ab)))
    b = O.sanitize(G, s_bc, rng.standard_normal(O.reduced_shape(G, s_bc)))
    c = O.sanitize(G, s_cd, rng.standard_normal(O.reduced_shape(G, s_cd)))
    Wh = p1.contract(dev(a), dev(b))
    Y = p2.contract(Wh, dev(c))
    torch.cuda.synchronize()
    p2.check_device_error()
    W = O.contract_blockloop(o1, a, b)
    want_wh = O.align_w(o1, W)[p1.q_values()]
    assert rel(Wh.cpu().numpy(), want_wh) <= TOL[precision]
    assert not Wh.cpu().numpy()[want_wh == 0].any() or precision != "fp64"
    assert rel(Y.cpu().numpy(), O.contract_blockloop(o2, W, c)) <= 2 * TOL[precision]
