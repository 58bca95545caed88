"""GPU parity on the contraction families of Table 1 (MM, CC_1, CC_2, CC_3,
MPS, PEPS) with the shapes of Table 2 (type a: few large sectors; type b:
many small ones), scaled so that the oracle's block loop finishes in seconds.

Table 1 gives index patterns but no charge signs; each case below states the
signs it uses (contracted modes carry opposite or equal signs in U and V, the
two cases the remark after Eq. ctr allows).  Every case runs in the three
precision forms against the oracle's block loop (Algorithm 1 generalised)."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as WL

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "split_bf16": 1e-10, "tf32": 1e-2}

# (label, einsum, moduli, (signs_u, charge_u, dims_u), (signs_v, charge_v, dims_v))
CASES = [
    # MM_a: G = 2, N = 10000 -> 2 sectors of 96; MM_b: G = 100, N = 2000 -> 20 of 40
    ("MM_a", "ij,jk->ik", (2,), ((1, -1), (0,), (96, 96)), ((1, -1), (0,), (96, 96))),
    ("MM_b", "ij,jk->ik", (20,), ((1, -1), (3,), (40, 40)), ((1, -1), (5,), (40, 40))),
    # CC_1: w[i,j,m,n] = sum_{k,l} u[i,j,k,l] v[m,n,k,l]  (CC_1a: N_i..l = 32, N_m,n = 16 -> /4)
    ("CC1_a", "ijkl,mnkl->ijmn", (8,), ((1, 1, -1, -1), (0,), (8, 8, 8, 8)),
     ((1, 1, -1, -1), (0,), (4, 4, 8, 8))),
    ("CC1_b", "ijkl,mnkl->ijmn", (4,), ((1, 1, -1, -1), (1,), (8, 8, 8, 8)),
     ((1, 1, -1, -1), (2,), (4, 4, 8, 8))),
    # CC_2: w[i,j,m,k] = sum_{o,p} u[o,p,i,j] v[o,p,k,m]
    ("CC2_a", "opij,opkm->ijmk", (8,), ((1, 1, -1, -1), (0,), (4, 4, 8, 8)),
     ((-1, -1, 1, 1), (0,), (4, 4, 8, 4))),
    ("CC2_b", "opij,opkm->ijmk", (4,), ((1, 1, -1, -1), (3,), (8, 8, 16, 16)),
     ((-1, -1, 1, 1), (1,), (8, 8, 16, 8))),
    # CC_3: w[i,j,m,n] = sum_{o,p} u[o,p,m,n] v[o,p,i,j]
    ("CC3_a", "opmn,opij->ijmn", (8,), ((1, 1, -1, -1), (0,), (4, 4, 4, 4)),
     ((1, 1, -1, -1), (0,), (4, 4, 8, 8))),
    ("CC3_b", "opmn,opij->ijmn", (4,), ((1, -1, 1, -1), (2,), (8, 8, 8, 8)),
     ((-1, 1, 1, -1), (1,), (8, 8, 16, 16))),
    # MPS: W[i,j,l,m] = sum_k U[i,j,k] V[k,l,m] with N_l = 1 (MPS_a: G = 2,
    # N_i = N_k = N_m = 3000, N_j = 10 -> 96 and 10; MPS_b: G = 5, 700 -> 40)
    ("MPS_a", "ijk,klm->ijlm", (2,), ((1, 1, -1), (0,), (96, 10, 96)),
     ((1, 1, -1), (0,), (96, 1, 96))),
    ("MPS_b", "ijk,klm->ijlm", (5,), ((1, 1, -1), (2,), (40, 10, 40)),
     ((1, 1, -1), (4,), (40, 1, 40))),
    # PEPS: W[i,j,m,n] = sum_{k,l} U[i,j,k,l] V[k,l,m,n] (PEPS_a: G = 2, N_i,j = 400,
    # N_k..n = 20 -> 40 and 8; PEPS_b: G = 10, 64 and 8 -> 16 and 4)
    ("PEPS_a", "ijkl,klmn->ijmn", (2,), ((1, 1, -1, -1), (0,), (40, 40, 8, 8)),
     ((1, 1, -1, -1), (0,), (8, 8, 8, 8))),
    ("PEPS_b", "ijkl,klmn->ijmn", (10,), ((1, 1, -1, -1), (0,), (16, 16, 4, 4)),
     ((1, 1, -1, -1), (7,), (4, 4, 4, 4))),
]


@pytest.fixture(scope="module")
def sc():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    import paper_2007_08056_gb300 as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def references():
    """Inputs and oracle results, computed once per case."""
    out = {}
    for k, (label, es, moduli, su, sv) in enumerate(CASES):
        g = O.Group(moduli)
        o = O.plan(es, g, O.Sym(*su), O.Sym(*sv))
        rng = np.random.default_rng(7000 + k)
        u = rng.standard_normal(O.reduced_shape(g, O.Sym(*su)))
        v = rng.standard_normal(O.reduced_shape(g, O.Sym(*sv)))
        out[label] = (u, v, O.contract_blockloop(o, u, v))
    return out


@pytest.mark.parametrize("precision", ["fp64", "split_bf16", "tf32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_table_contraction(sc, references, case, precision):
    label, es, moduli, su, sv = case
    u, v, want = references[label]
    p = sc.Plan(es, moduli, su, sv, precision)
    w = p.contract(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda())
    torch.cuda.synchronize()
    p.check_device_error()
    got = w.cpu().numpy()
    assert got.shape == want.shape
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel <= TOL[precision], f"{label} {precision}: {rel:.3e}"
