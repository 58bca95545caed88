"""GPU parity for the generalized symmetry of Eq. symtsr: modes with H | G
sectors and coefficient +-G/H, and non-uniform sector sizes held in blocks
padded with zeros to a fixed size (Sec. 1).

Every precision form runs its usual kernels; the index maps come from the
plan's offset tables, where absent aligned rows and columns (an implicit sector
equation without a solution, or a padding position) are marked and read as
zero.  Results are compared with the oracle's block loop at each form's
tolerance; the inputs carry large garbage in every entry that is not part of
the tensor, which must change nothing, and the output must hold exact zeros
there.
"""
import numpy as np
import pytest
import torch

import oracle as O
from test_oracle_pins import GEN_STV, random_general_case

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "split_bf16": 1e-10, "tf32": 1e-2}


@pytest.fixture(scope="module")
def sc():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    import paper_2007_08056_gb300 as mod
    mod.load()
    return mod


def as_spec(sym):
    return (sym.signs, sym.charge, sym.dims, sym.sectors, sym.sector_dims)


def garbage(group, sym, red, rng):
    """red with large noise in every entry that is not part of the tensor."""
    part = O.sanitize(group, sym, np.ones_like(red)) != 0
    return np.where(part, red, rng.standard_normal(red.shape) * 1e6), part


def rel(a, b):
    n = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (n if n > 0 else 1.0))


def check(sc, p, u, v, precision, rng, want_tc=None):
    plan = sc.Plan(f"{p.lu},{p.lv}->{p.lw}", p.group.moduli, as_spec(p.sym_u), as_spec(p.sym_v),
                   precision)
    assert plan.info.general == 1
    if want_tc is not None:
        assert plan.info.tensor_core == want_tc
    want = O.contract_blockloop(p, u, v)
    ug, _ = garbage(p.group, p.sym_u, u, rng)
    vg, _ = garbage(p.group, p.sym_v, v, rng)
    w = plan.contract(torch.from_numpy(ug).cuda(), torch.from_numpy(vg).cuda(),
                      out=torch.full(plan.shape_w, np.nan, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    plan.check_device_error()
    got = w.cpu().numpy()
    part = O.sanitize(p.group, p.sym_w, np.ones(got.shape)) != 0
    assert not got[~part].any()                 # padding and absent entries: exact zeros
    assert rel(got, want) <= TOL[precision]
    return plan


@pytest.mark.parametrize("precision", ["fp64", "split_bf16", "tf32"])
def test_general_small_cases(sc, precision):
    """Random small contractions over all (s, t, v) shapes of the oracle pins,
    G = 4, 6, 8, 12, random sector counts, signs, charges and sector sizes."""
    rng = np.random.default_rng(6100)
    for (s, t, v) in GEN_STV:
        for G, sigma in [(4, -1), (6, 1), (8, -1), (12, 1)]:
            if G ** (s + t + v) > 30000:
                continue
            p, u, vv = random_general_case(s, t, v, G, rng, sigma)
            check(sc, p, u, vv, precision, rng)


def cc_like(rng, G=8, dv=12, do=6, seed_sd=True):
    """A CC-ladder-shaped contraction, w[a,b,i,j] = sum v[a,b,c,d] t[c,d,i,j],
    with sub-group modes (b: G/2 sectors, d: 2 sectors, j: G/2) and padded
    non-uniform sectors (virtual blocks of 6..12, occupied of 3..6): aligned
    M = K = 1152, N = 288 per irrep, on the tensor cores."""
    H = {"a": G, "b": G // 2, "c": G, "d": 2, "i": G, "j": G // 2}
    D = {"a": dv, "b": dv, "c": dv, "d": dv, "i": do, "j": do}
    SD = {c: tuple(int(rng.integers(D[c] // 2, D[c] + 1)) for _ in range(H[c])) for c in H}
    sym = lambda lab, signs, z: O.Sym(signs, z, tuple(D[c] for c in lab), tuple(H[c] for c in lab),
                                      tuple(SD[c] for c in lab))
    su = sym("abcd", (1, 1, -1, -1), (0,))
    sv = sym("cdij", (1, 1, -1, -1), (2,))
    p = O.plan("abcd,cdij->abij", O.Group((G,)), su, sv)
    u = rng.standard_normal(O.reduced_shape(p.group, su)) / np.sqrt(dv * dv * G)
    v = rng.standard_normal(O.reduced_shape(p.group, sv))
    return p, u, v


@pytest.mark.parametrize("precision", ["fp64", "split_bf16", "tf32"])
def test_general_cc_ladder_shape(sc, precision):
    rng = np.random.default_rng(6200)
    p, u, v = cc_like(rng)
    G, M, N, K = O.aligned_dims(p)
    assert (M, N, K) == (1152, 288, 1152)
    plan = check(sc, p, u, v, precision, rng, want_tc=0 if precision == "fp64" else 1)
    assert plan.info.n_q > 1


def test_general_align_bit_exact(sc):
    """symctr_align on a general plan: the gather (+1) reproduces the oracle's
    aligned entries bit for bit with absent ones zero, for U, V and W; the
    scatter (-1) of W writes every valid entry and zeros elsewhere."""
    rng = np.random.default_rng(6300)
    for trial in range(3):
        p, u, v = cc_like(rng, G=4, dv=6, do=4) if trial == 0 else \
            random_general_case(2, 2, 2, 6, rng, -1)
        plan = sc.Plan(f"{p.lu},{p.lv}->{p.lw}", p.group.moduli, as_spec(p.sym_u),
                       as_spec(p.sym_v), "split_bf16")
        G, M, N, K = O.aligned_dims(p)
        w = O.contract_blockloop(p, u, v)
        qs = plan.q_values()
        extents = {0: (M, K, u), 1: (N, K, v), 2: (M, N, w)}
        for op, (R, Cn, red) in extents.items():
            ext = plan.align(op, +1, torch.from_numpy(red).cuda()).cpu().numpy()
            assert ext.shape == (len(qs), R, Cn)
            for b, Q in enumerate(qs):
                r, c = np.arange(R)[:, None], np.arange(Cn)[None, :]
                ok = O.aligned_valid(p, op, Q, r, c)
                assert np.array_equal(ext[b], np.where(ok, red[O.aligned_index(p, op, Q, r, c)], 0.0))
        wh = rng.standard_normal((len(qs), M, N))
        back = plan.align(2, -1, torch.from_numpy(wh).cuda()).cpu().numpy()
        want = np.zeros_like(w)
        for b, Q in enumerate(qs):
            r, c = np.arange(M)[:, None], np.arange(N)[None, :]
            ok = O.aligned_valid(p, 2, Q, r, c)
            idx = O.aligned_index(p, 2, Q, r, c)
            want[tuple(i[ok] for i in idx)] = wh[b][ok]
        assert np.array_equal(back, want)


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_general_backward(sc, precision):
    """The adjoint contractions of a general plan (their own general plans,
    built by the library) against the oracle's gradients."""
    rng = np.random.default_rng(6400)
    p, u, v = cc_like(rng)
    plan = sc.Plan(f"{p.lu},{p.lv}->{p.lw}", p.group.moduli, as_spec(p.sym_u), as_spec(p.sym_v),
                   precision)
    gw = O.sanitize(p.group, p.sym_w, rng.standard_normal(plan.shape_w))
    gu, gv = plan.backward(torch.from_numpy(gw).cuda(), torch.from_numpy(u).cuda(),
                           torch.from_numpy(v).cuda())
    torch.cuda.synchronize()
    plan.check_device_error()
    assert rel(gu.cpu().numpy(), O.grad_u(p, gw, v)) <= TOL[precision]
    assert rel(gv.cpu().numpy(), O.grad_v(p, u, gw)) <= TOL[precision]
