"""Complex tensors (Sec. 1: entries may be complex) through
symctr_contract_complex, in the three precision forms, against the oracle's
block loop on complex reduced forms; conjugated operands carry the negated law
(the MPS transfer contraction uses conj(A))."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as WL

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


def negated(sp):
    signs, charge, dims = sp
    return (tuple(-c for c in signs), tuple(-z for z in charge), dims)


def cdraw(moduli, sp, seed):
    rng = np.random.default_rng(seed)
    shape = O.reduced_shape(O.Group(moduli), O.Sym(*sp))
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [WL.Z3_ORDER4] + [c for c in WL.small_cases() if c.name in ("mm_G4", "sigma_plus_G5", "z2xz3_order4")]


@pytest.mark.parametrize("precision", ["fp64", "split_bf16", "tf32"])
@pytest.mark.parametrize("conj", [(False, False), (True, False), (False, True), (True, True)],
                         ids=["UV", "cU-V", "U-cV", "cU-cV"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_complex_contraction(sc, case, conj, precision):
    cu, cv = conj
    su, sv = spec(case.u), spec(case.v)
    u = cdraw(case.moduli, su, 11)
    v = cdraw(case.moduli, sv, 12)
    # the plan sees the operands as contracted: a conjugated operand has the negated law
    pu, pv = (negated(su) if cu else su), (negated(sv) if cv else sv)
    p = sc.Plan(case.einsum, case.moduli, pu, pv, precision)
    w = p.contract_complex(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), conj_u=cu, conj_v=cv)
    torch.cuda.synchronize()
    p.check_device_error()
    o = O.plan(case.einsum, O.Group(case.moduli), O.Sym(*pu), O.Sym(*pv))
    want = O.contract_blockloop(o, np.conj(u) if cu else u, np.conj(v) if cv else v)
    assert rel(w.cpu().numpy(), want) <= TOL[precision]


@pytest.mark.parametrize("precision", ["split_bf16", "fp64"])
def test_mps_transfer_with_conjugate(sc, precision):
    """E' = sum E A conj(A) with complex A: X = E.A, then E' = X.conj(A) (conj(A)
    carries A's negated law)."""
    g = WL.MPS_G
    sE, sA = spec(WL.MPS_E), spec(WL.MPS_A)
    E = cdraw((g,), sE, 21)
    A = cdraw((g,), sA, 22)
    p1 = sc.Plan(WL.MPS_STEP1, (g,), sE, sA, precision)
    p2 = sc.Plan(WL.MPS_STEP2, (g,), p1.sym_w, negated(sA), precision)
    Ad = torch.from_numpy(A).cuda()
    X = p1.contract_complex(torch.from_numpy(E).cuda(), Ad)
    Ep = p2.contract_complex(X, Ad, conj_v=True)
    torch.cuda.synchronize()
    p2.check_device_error()
    G = O.Group((g,))
    o1 = O.plan(WL.MPS_STEP1, G, O.Sym(*sE), O.Sym(*sA))
    Xr = O.contract_blockloop(o1, E, A)
    o2 = O.plan(WL.MPS_STEP2, G, o1.sym_w, O.Sym(*negated(sA)))
    want = O.contract_blockloop(o2, Xr, np.conj(A))
    assert rel(Ep.cpu().numpy(), want) <= TOL[precision]
