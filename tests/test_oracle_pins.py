"""Pins of the CPU oracle to things other than itself (CPU only).

Each test ties an oracle route to a fixed point the paper or plain
mathematics provides: hand-worked examples (tests/golden), brute force on
tiny inputs, closed-form counts, special cases that reduce to a textbook
routine, and invariants of the paper's proof.  The mutation tests at the
end plant plausible mistakes in a copy of the oracle and check that these
pins catch them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import oracle.symoracle as OS
import workloads as WL

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_fixture(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=", 1)
            out[k.strip()] = json.loads(v.strip())
    return out


def mk(c):
    g = O.Group(c.moduli)
    su = O.Sym(c.u.signs, c.u.charge, c.u.dims)
    sv = O.Sym(c.v.signs, c.v.charge, c.v.dims)
    return O.plan(c.einsum, g, su, sv)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    n = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (n if n > 0 else 1.0))


# --------------------------------------------------------------------------
# hand-worked examples
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["mm_z2_d1.txt", "mm_z2_d2_charged.txt", "order4_z2_d1.txt"])
def test_golden_hand_worked(name):
    fx = load_fixture(name)
    g = O.Group(fx["moduli"])
    su = O.Sym(tuple(fx["signs_u"]), tuple(fx["charge_u"]), tuple(fx["dims_u"]))
    sv = O.Sym(tuple(fx["signs_v"]), tuple(fx["charge_v"]), tuple(fx["dims_v"]))
    p = O.plan(fx["einsum"], g, su, sv)
    assert list(p.sym_w.signs) == fx["signs_w"]
    assert list(p.sym_w.charge) == fx["charge_w"]
    u = np.array(fx["u"], dtype=float).reshape(O.reduced_shape(g, su))
    v = np.array(fx["v"], dtype=float).reshape(O.reduced_shape(g, sv))
    want = np.array(fx["w"], dtype=float).reshape(O.reduced_shape(g, p.sym_w))
    # every route must reproduce the hand-worked integers exactly
    assert np.array_equal(O.contract_blockloop(p, u, v), want)
    assert np.array_equal(O.contract_aligned(p, u, v), want)
    w3, forb = O.contract_dense_einsum(p, u, v)
    assert np.array_equal(w3, want) and forb == 0.0
    assert np.array_equal(O.restrict(g, p.sym_w, O.contract_dense_loops(p, u, v))[0], want)


def test_api_listing_shape():
    fx = load_fixture("api_listing.txt")
    g = O.Group(fx["moduli"])
    s = O.Sym(tuple(fx["signs"]), tuple(fx["charge"]), tuple(fx["dims"]))
    assert list(O.reduced_shape(g, s)) == fx["reduced_shape"]
    assert list(WL.reduced_shape(fx["moduli"], fx["dims"])) == fx["reduced_shape"]


def test_table1_block_product_counts():
    """Alg. 1 loop performs G^(s+t+v-2) block products; dense would be G^(s+t+v)."""
    with open(os.path.join(GOLDEN, "table1_costs.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for label, spec, sym_exp, naive_exp in rows:
        lu, lv, lw = O.parse_einsum(spec)
        for G in (2, 3, 4):
            g = O.Group([G])
            # signs chosen so that the contracted coefficients differ by a sign
            su = O.Sym(tuple([1] * (len(lu) // 2) + [-1] * (len(lu) - len(lu) // 2)), (0,),
                       tuple([1] * len(lu)))
            cu = dict(zip(lu, su.signs))
            sv_signs = tuple(-cu[c] if c in lu else 1 for c in lv)
            sv = O.Sym(sv_signs, (0,), tuple([1] * len(lv)))
            p = O.plan(spec, g, su, sv)
            assert p.s + p.t + p.v - 2 == int(sym_exp)
            assert p.s + p.t + p.v == int(naive_exp)
            cnt = [0]
            rng = np.random.default_rng(0)
            O.contract_blockloop(p, rng.standard_normal(O.reduced_shape(g, su)),
                                 rng.standard_normal(O.reduced_shape(g, sv)), cnt)
            assert cnt[0] == G ** int(sym_exp)


# --------------------------------------------------------------------------
# reduced form <-> dense
# --------------------------------------------------------------------------

SYMS = [
    ((3,), O.Sym((1, 1, -1, -1), (0,), (2, 1, 2, 3))),
    ((4,), O.Sym((1, -1, 1), (3,), (2, 3, 1))),
    ((2, 3), O.Sym((1, 1, -1), (1, 2), (1, 2, 2))),
    ((5,), O.Sym((-1,), (2,), (3,))),
    ((2,), O.Sym((), (0,), ())),
]


@pytest.mark.parametrize("moduli,sym", SYMS)
def test_expand_restrict_roundtrip(moduli, sym):
    g = O.Group(moduli)
    rng = np.random.default_rng(1)
    red = rng.standard_normal(O.reduced_shape(g, sym))
    dense = O.expand(g, sym, red)
    back, forb = O.restrict(g, sym, dense)
    assert np.array_equal(back, red)
    assert forb == 0.0
    # closed form: the reduced form stores G^(N-1) of the G^N blocks (Sec. 2.1)
    n = sym.order
    allowed, total = O.count_stored_blocks(g, sym)
    assert total == g.order ** n
    assert allowed == (g.order ** (n - 1) if n else 1)
    assert np.count_nonzero(dense) == red.size


def test_expand_places_blocks_by_hand():
    """x = q*D + b placement and the implicit last sector, checked by hand:
    Z_3, signs (+,-), Z = 1, D = (1, 2).  Allowed: q0 - q1 = 1 -> q1 = q0 - 1."""
    g = O.Group([3])
    s = O.Sym((1, -1), (1,), (1, 2))
    red = np.arange(1.0, 7.0).reshape(3, 1, 2)
    dense = O.expand(g, s, red)
    want = np.zeros((3, 6))
    want[0, 4:6] = [1, 2]     # q0=0 -> q1=2
    want[1, 0:2] = [3, 4]     # q0=1 -> q1=0
    want[2, 2:4] = [5, 6]     # q0=2 -> q1=1
    assert np.array_equal(dense, want)


# --------------------------------------------------------------------------
# contraction routes against brute force
# --------------------------------------------------------------------------

def random_case(s, t, v, G, rng, sigma, moduli=None):
    labels = iter("abcdefghijklmnop")
    FU = [next(labels) for _ in range(s)]
    C = [next(labels) for _ in range(v)]
    FV = [next(labels) for _ in range(t)]
    lu = "".join(FU + C)
    lv = "".join(C + FV)
    # shuffle operand mode orders and the output order
    lu = "".join(rng.permutation(list(lu))) if lu else ""
    lv = "".join(rng.permutation(list(lv))) if lv else ""
    lw = "".join(rng.permutation(FU + FV)) if (FU or FV) else ""
    moduli = moduli or (G,)
    g = O.Group(moduli)
    dims = {c: int(rng.integers(1, 3)) for c in lu + lv}
    su_signs = {c: int(rng.choice([-1, 1])) for c in lu}
    sv_signs = {c: (sigma * su_signs[c] if c in C else int(rng.choice([-1, 1]))) for c in lv}
    zu = tuple(int(rng.integers(0, m)) for m in moduli)
    zv = tuple(int(rng.integers(0, m)) for m in moduli)
    su = O.Sym(tuple(su_signs[c] for c in lu), zu, tuple(dims[c] for c in lu))
    sv = O.Sym(tuple(sv_signs[c] for c in lv), zv, tuple(dims[c] for c in lv))
    p = O.plan(f"{lu},{lv}->{lw}", g, su, sv)
    u = rng.standard_normal(O.reduced_shape(g, su))
    vv = rng.standard_normal(O.reduced_shape(g, sv))
    return p, u, vv


STV = [(s, t, v) for s in range(4) for t in range(4) for v in range(4) if 1 <= s + t + v <= 5]


@pytest.mark.parametrize("s,t,v", STV)
def test_routes_agree_with_dense_bruteforce(s, t, v):
    rng = np.random.default_rng(100 * s + 10 * t + v)
    for G, sigma, moduli in [(2, -1, None), (3, 1, None), (4, -1, None), (6, 1, (2, 3))]:
        if G ** (s + t + v) > 5000:
            continue
        p, u, vv = random_case(s, t, v, G, rng, sigma, moduli)
        w3, forb = O.contract_dense_einsum(p, u, vv)
        assert forb == 0.0                       # off-sector blocks of W are exactly zero
        w4 = O.contract_blockloop(p, u, vv)
        w5 = O.contract_aligned(p, u, vv)
        assert rel(w4, w3) <= 1e-13
        assert rel(w5, w3) <= 1e-13


def test_dense_loops_match_einsum_tiny():
    rng = np.random.default_rng(7)
    for (s, t, v) in [(1, 1, 1), (2, 1, 1), (1, 2, 2), (0, 1, 1), (1, 1, 0), (0, 0, 2)]:
        p, u, vv = random_case(s, t, v, 2, rng, -1)
        dense_loop = O.contract_dense_loops(p, u, vv)
        U = O.expand(p.group, p.sym_u, u)
        V = O.expand(p.group, p.sym_v, vv)
        assert np.allclose(dense_loop, np.einsum(f"{p.lu},{p.lv}->{p.lw}", U, V),
                           rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("case", WL.small_cases(), ids=lambda c: c.name)
def test_small_workloads_all_routes(case):
    p = mk(case)
    u, v = WL.draw_pair(case)
    w3, forb = O.contract_dense_einsum(p, u, v)
    assert forb == 0.0
    assert rel(O.contract_blockloop(p, u, v), w3) <= 1e-13
    assert rel(O.contract_aligned(p, u, v), w3) <= 1e-13
    # one entry at a time, straight from Eq. ctr
    w4 = O.contract_blockloop(p, u, v)
    rng = np.random.default_rng(3)
    for _ in range(5):
        idx = tuple(int(rng.integers(0, n)) for n in w4.shape)
        assert abs(O.contract_element(p, u, v, idx) - w4[idx]) <= 1e-12 * (1 + abs(w4[idx]))


@pytest.mark.parametrize("case", WL.small_cases(), ids=lambda c: c.name)
def test_lazy_element_matches_block_loop(case):
    """The callback form used for operands that only live on a device sums the
    same terms as the block loop."""
    p = mk(case)
    u, v = WL.draw_pair(case)
    w4 = O.contract_blockloop(p, u, v)
    rng = np.random.default_rng(4)
    for _ in range(5):
        idx = tuple(int(rng.integers(0, n)) for n in w4.shape)
        got = O.contract_element_lazy(p, lambda i: u[i], lambda i: v[i], idx)
        assert abs(got - w4[idx]) <= 1e-12 * (1 + abs(w4[idx]))


def test_g1_is_plain_dense():
    """G = 1: the reduced form is the dense tensor; the contraction is np.einsum."""
    rng = np.random.default_rng(5)
    g = O.Group([1])
    su = O.Sym((1, -1, 1), (0,), (3, 4, 2))
    sv = O.Sym((-1, 1), (0,), (2, 5))
    p = O.plan("abk,kc->bca", g, su, sv)
    u = rng.standard_normal(O.reduced_shape(g, su))
    v = rng.standard_normal(O.reduced_shape(g, sv))
    ud = u.reshape(3, 4, 2)
    vd = v.reshape(2, 5)
    want = np.einsum("abk,kc->bca", ud, vd)
    assert np.allclose(O.contract_blockloop(p, u, v).reshape(want.shape), want, rtol=1e-14)
    assert np.allclose(O.contract_aligned(p, u, v).reshape(want.shape), want, rtol=1e-14)


def test_mm_block_diagonal_matmul():
    """Table 1 'MM': with Z = 0 and signs (+,-) both matrices are block diagonal
    and W_Q = U_Q V_Q for each irrep Q (cost G N^3)."""
    rng = np.random.default_rng(6)
    G = 5
    g = O.Group([G])
    su = O.Sym((1, -1), (0,), (4, 3))
    sv = O.Sym((1, -1), (0,), (3, 6))
    p = O.plan("ij,jk->ik", g, su, sv)
    u = rng.standard_normal((G, 4, 3))
    v = rng.standard_normal((G, 3, 6))
    want = np.stack([u[q] @ v[q] for q in range(G)])
    assert np.allclose(O.contract_blockloop(p, u, v), want, rtol=1e-14)
    assert np.allclose(O.contract_aligned(p, u, v), want, rtol=1e-14)


def test_product_group_equals_cyclic_crt():
    """Z_2 x Z_3 is isomorphic to Z_6 (q -> (q mod 2, q mod 3)); results agree
    after relabelling the sectors of every stored axis."""
    rng = np.random.default_rng(8)
    g6, g23 = O.Group([6]), O.Group([2, 3])
    # label in Z_2xZ_3 flattening for each Z_6 label
    lab = [g23.label((q % 2, q % 3)) for q in range(6)]
    z6 = 5
    z23 = (z6 % 2, z6 % 3)
    su6 = O.Sym((1, 1, -1), (z6,), (2, 1, 2))
    sv6 = O.Sym((1, -1), (0,), (2, 3))
    su23 = O.Sym(su6.signs, z23, su6.dims)
    sv23 = O.Sym(sv6.signs, (0, 0), sv6.dims)
    p6 = O.plan("abk,kc->acb", g6, su6, sv6)
    p23 = O.plan("abk,kc->acb", g23, su23, sv23)
    u6 = rng.standard_normal(O.reduced_shape(g6, su6))
    v6 = rng.standard_normal(O.reduced_shape(g6, sv6))

    def relabel(x, nsec):
        y = np.empty_like(x)
        for qs in itertools.product(range(6), repeat=nsec):
            y[tuple(lab[q] for q in qs)] = x[qs]
        return y
    u23 = relabel(u6, 2)
    v23 = relabel(v6, 1)
    w6 = O.contract_blockloop(p6, u6, v6)
    w23 = O.contract_blockloop(p23, u23, v23)
    assert np.allclose(relabel(w6, 2), w23, rtol=1e-14)
    assert np.allclose(O.contract_aligned(p23, u23, v23), w23, rtol=1e-13)


def test_bilinear_and_operand_swap():
    rng = np.random.default_rng(9)
    p, u, v = random_case(2, 2, 2, 3, rng, -1)
    u2 = rng.standard_normal(u.shape)
    a, b = 1.7, -0.3
    lhs = O.contract_blockloop(p, a * u + b * u2, v)
    rhs = a * O.contract_blockloop(p, u, v) + b * O.contract_blockloop(p, u2, v)
    assert rel(lhs, rhs) <= 1e-13
    # swapping the operands (einsum with operands exchanged) gives the same W
    q = O.plan(f"{p.lv},{p.lu}->{p.lw}", p.group, p.sym_v, p.sym_u)
    wq = O.contract_blockloop(q, v, u)
    # same nonzero set; W's law may come out globally negated
    Wp = O.expand(p.group, p.sym_w, O.contract_blockloop(p, u, v))
    Wq = O.expand(q.group, q.sym_w, wq)
    assert rel(Wq, Wp) <= 1e-13


# --------------------------------------------------------------------------
# closed-form counts of the order-4 example
# --------------------------------------------------------------------------

def test_order4_counts_config1():
    p = mk(WL.Z3_ORDER4)
    G, M, N, K = O.aligned_dims(p)
    D = 4
    assert (G, M, N, K) == (3, D * D * 3, D * D * 3, D * D * 3)
    useful = 2 * len(O.q_set(p)) * M * N * K
    assert useful == 2 * D ** 6 * G ** 4 == 663_552          # G^4 block products of D^6 work
    assert 2 * (D * G) ** 6 == 5_971_968                      # dense: G^6 of them
    cnt = [0]
    u, v = WL.draw_pair(WL.Z3_ORDER4)
    O.contract_blockloop(p, u, v, cnt)
    assert cnt[0] == G ** 4


def test_q_sets_of_degenerate_shapes():
    """s = 0 leaves Q = Z_U; t = 0 leaves sigma*Q = Z_V; v = 0 leaves Q = 0."""
    by = {c.name: mk(c) for c in WL.small_cases()}
    assert O.q_set(by["s0_G4"]) == [3]
    assert O.q_set(by["t0_G2"]) == [1]          # sigma = -1, Z_V = 1 -> Q = 1 (mod 2)
    assert O.q_set(by["outer_v0_G3"]) == [0]
    assert O.q_set(by["z3_order4_G3_D4"]) == [0, 1, 2]


# --------------------------------------------------------------------------
# aligned transforms are bijections (uniqueness of Q in the proof, Sec. 2.3)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", WL.small_cases(), ids=lambda c: c.name)
def test_alignment_is_a_permutation(case):
    """Each aligned form holds every stored entry exactly once, the remaining
    positions being zero (Q is unique for each sector tuple)."""
    p = mk(case)
    u, v = WL.draw_pair(case)
    uh, vh = O.align_u(p, u), O.align_v(p, v)
    for red, al in ((u, uh), (v, vh)):
        pad = np.zeros(al.size - red.size)
        assert np.array_equal(np.sort(al.ravel()), np.sort(np.concatenate([red.ravel(), pad])))
    # the product of the aligned forms vanishes outside the Q set
    qs = O.q_set(p)
    wh = np.matmul(uh, np.transpose(vh, (0, 2, 1)))
    absent = [q for q in range(p.group.order) if q not in qs]
    assert not wh[absent].any()
    # W: align_w is the exact inverse of mapback_w on W's reduced form
    w = O.contract_blockloop(p, u, v)
    assert np.array_equal(O.mapback_w(p, O.align_w(p, w)), w)


@pytest.mark.parametrize("s,t,v", [(1, 1, 1), (2, 1, 2), (2, 2, 2), (0, 2, 1), (1, 0, 2),
                                   (2, 1, 0), (3, 1, 1), (1, 3, 1)])
def test_aligned_index_matches_dense_delta_route(s, t, v):
    """Entry-by-entry positions of the aligned forms (aligned_index) against
    the dense generalized-Kronecker-delta route of Alg. 2 (align_u, align_v,
    mapback_w): every entry of U_hat, V_hat and W_hat, over every Q of the
    Q set, with shuffled mode orders, random charges, sigma = +-1 and a
    product group."""
    rng = np.random.default_rng(500 + 100 * s + 10 * t + v)
    for G, sigma, moduli in [(3, -1, None), (4, 1, None), (6, -1, (2, 3))]:
        if G ** (s + t + v) > 3000:
            continue
        p, u, vv = random_case(s, t, v, G, rng, sigma, moduli)
        Gn, M, N, K = O.aligned_dims(p)
        uh, vh = O.align_u(p, u), O.align_v(p, vv)
        wh = rng.standard_normal((Gn, M, N))
        w = O.mapback_w(p, wh)
        for Q in O.q_set(p):
            m, n, k = np.arange(M)[:, None], np.arange(N)[:, None], np.arange(K)[None, :]
            if p.lu:
                assert np.array_equal(u[O.aligned_index(p, 0, Q, m, k)], uh[Q])
            if p.lv:
                assert np.array_equal(vv[O.aligned_index(p, 1, Q, n, k)], vh[Q])
            if p.lw:
                assert np.array_equal(w[O.aligned_index(p, 2, Q, m, np.arange(N)[None, :])], wh[Q])


# --------------------------------------------------------------------------
# gradients
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", WL.small_cases(), ids=lambda c: c.name)
def test_adjoint_identity(case):
    p = mk(case)
    u, v = WL.draw_pair(case)
    rng = np.random.default_rng(11)
    y = rng.standard_normal(O.reduced_shape(p.group, p.sym_w))
    w = O.contract_blockloop(p, u, v)
    lhs = float(np.sum(w * y))
    gu = O.grad_u(p, y, v)
    gv = O.grad_v(p, u, y)
    assert gu.shape == u.shape and gv.shape == v.shape
    scale = float(np.sum(np.abs(w * y))) + 1e-300
    assert abs(lhs - float(np.sum(u * gu))) <= 1e-13 * scale
    assert abs(lhs - float(np.sum(v * gv))) <= 1e-13 * scale


def test_finite_differences_quadratic_loss():
    """L = sum W^2 is quadratic, so central differences are exact up to roundoff."""
    rng = np.random.default_rng(12)
    p, u, v = random_case(2, 1, 2, 3, rng, -1)

    def loss_u(x):
        return float(np.sum(O.contract_blockloop(p, x, v) ** 2))

    def loss_v(x):
        return float(np.sum(O.contract_blockloop(p, u, x) ** 2))
    w = O.contract_blockloop(p, u, v)
    gu = O.grad_u(p, 2 * w, v)
    gv = O.grad_v(p, u, 2 * w)
    for seed in range(3):
        du = np.random.default_rng(50 + seed).standard_normal(u.shape)
        dv = np.random.default_rng(60 + seed).standard_normal(v.shape)
        fd_u = O.central_difference(loss_u, u, du, 1e-6)
        fd_v = O.central_difference(loss_v, v, dv, 1e-6)
        assert abs(fd_u - np.sum(gu * du)) <= 1e-7 * abs(fd_u)
        assert abs(fd_v - np.sum(gv * dv)) <= 1e-7 * abs(fd_v)


# --------------------------------------------------------------------------
# planted mistakes are caught by the pins above
# --------------------------------------------------------------------------

def test_planted_wrong_output_law_is_caught(monkeypatch):
    """A sign slip in the derived output law (Z_W = Z_U + sigma Z_V) must break
    agreement with the dense brute force on a charged case."""
    fx = load_fixture("mm_z2_d2_charged.txt")
    rng = np.random.default_rng(13)
    p, u, v = random_case(1, 1, 1, 3, rng, -1)
    p_bad = O.Plan(p.lu, p.lv, p.lw, p.FU, p.C, p.FV, p.sigma, p.sym_u, p.sym_v,
                   O.Sym(p.sym_w.signs, p.group.norm([a + p.sigma * b for a, b in
                                                      zip(p.sym_u.charge, p.sym_v.charge)]),
                         p.sym_w.dims), p.group)
    if p_bad.sym_w.charge == p.sym_w.charge:
        pytest.skip("charges coincide for this draw")
    w3, forb = O.contract_dense_einsum(p_bad, u, v)
    assert forb > 0.0          # the dense result has entries the wrong law forbids
    assert fx["charge_w"] == [1]


def test_planted_wrong_delta_sign_is_caught(monkeypatch):
    """Writing delta2 with +Q instead of -Q (the sign confusion of Alg. 2 / Sec. 2.3)
    breaks route O5 against the brute force whenever G > 2."""
    rng = np.random.default_rng(14)
    p, u, v = random_case(2, 2, 2, 3, rng, -1)
    good = O.contract_aligned(p, u, v)
    orig = OS._deltas

    def bad(pp):
        d1, d2, d3 = orig(pp)
        G = pp.group
        cu = dict(zip(pp.lu, pp.sym_u.signs))
        d2b = O.delta(G, [cu[c] for c in pp.C] + [1], tuple(0 for _ in G.moduli))
        return d1, d2b, d3
    monkeypatch.setattr(OS, "_deltas", bad)
    w3, _ = O.contract_dense_einsum(p, u, v)
    assert rel(good, w3) <= 1e-13
    assert rel(O.contract_aligned(p, u, v), w3) > 1e-3


def test_planted_transposed_operand_is_caught():
    """Contracting against the wrong axis order of V must fail the brute force."""
    rng = np.random.default_rng(15)
    g = O.Group([3])
    su = O.Sym((1, -1, -1), (0,), (2, 2, 2))
    sv = O.Sym((1, 1, -1), (0,), (2, 2, 3))
    p = O.plan("akl,klb->ab", g, su, sv)
    u = rng.standard_normal(O.reduced_shape(g, su))
    v = rng.standard_normal(O.reduced_shape(g, sv))
    good, _ = O.contract_dense_einsum(p, u, v)
    q = O.plan("alk,klb->ab", g, su, sv)
    assert rel(O.contract_blockloop(q, u, v), good) > 1e-3


# --------------------------------------------------------------------------
# complex tensors (Sec. 1: entries may be complex; conj(T) carries the
# negated law, i.e. negated coefficients and target charge)
# --------------------------------------------------------------------------

def _negated(sym):
    return O.Sym(tuple(-c for c in sym.signs), tuple(-z for z in sym.charge), sym.dims)


def _complexify(rng, a):
    return a + 1j * rng.standard_normal(a.shape)


@pytest.mark.parametrize("s,t,v", [(1, 1, 1), (2, 1, 2), (2, 2, 2), (0, 2, 1), (1, 0, 2), (2, 1, 0)])
def test_complex_block_loop_matches_dense_bruteforce(s, t, v):
    """The block loop on complex reduced forms equals the dense complex einsum
    of the expanded tensors (Eq. ctr), with exact zeros off-sector."""
    rng = np.random.default_rng(900 + 100 * s + 10 * t + v)
    for G, sigma, moduli in [(3, -1, None), (4, 1, None), (6, -1, (2, 3))]:
        p, u, vv = random_case(s, t, v, G, rng, sigma, moduli)
        uc, vc = _complexify(rng, u), _complexify(rng, vv)
        w3, forb = O.contract_dense_einsum(p, uc, vc)
        assert forb == 0.0 and np.iscomplexobj(w3)
        w4 = O.contract_blockloop(p, uc, vc)
        assert np.iscomplexobj(w4)
        assert rel(w4, w3) <= 1e-13


@pytest.mark.parametrize("case", WL.small_cases()[:5], ids=lambda c: c.name)
def test_complex_product_is_four_real_contractions(case):
    """(Ur + i Ui)(Vr + i Vi) = (UrVr - UiVi) + i(UrVi + UiVr), contraction
    by contraction, against the complex route."""
    p = mk(case)
    rng = np.random.default_rng(31)
    ur, ui, vr, vi = (rng.standard_normal(O.reduced_shape(p.group, sy))
                      for sy in (p.sym_u, p.sym_u, p.sym_v, p.sym_v))
    want = O.contract_blockloop(p, ur + 1j * ui, vr + 1j * vi)
    real = O.contract_blockloop(p, ur, vr) - O.contract_blockloop(p, ui, vi)
    imag = O.contract_blockloop(p, ur, vi) + O.contract_blockloop(p, ui, vr)
    assert rel(real + 1j * imag, want) <= 1e-13


def test_conjugate_operand_carries_the_negated_law():
    """conj(V) stored under the negated law has the same reduced array as V
    (same allowed blocks, same implicit sector) with conjugated entries, and
    contracting U with it matches the dense einsum of U and conj(dense V)."""
    rng = np.random.default_rng(77)
    for (s, t, v) in [(1, 1, 1), (2, 1, 2), (1, 2, 1)]:
        for G, sigma, moduli in [(3, 1, None), (6, -1, (2, 3))]:
            p, u, vv = random_case(s, t, v, G, rng, sigma, moduli)
            uc, vc = _complexify(rng, u), _complexify(rng, vv)
            sv_neg = _negated(p.sym_v)
            assert O.reduced_shape(p.group, sv_neg) == O.reduced_shape(p.group, p.sym_v)
            dense_conj = np.conj(O.expand(p.group, p.sym_v, vc))
            assert np.array_equal(O.expand(p.group, sv_neg, np.conj(vc)), dense_conj)
            pc = O.plan(f"{p.lu},{p.lv}->{p.lw}", p.group, p.sym_u, sv_neg)
            got = O.contract_blockloop(pc, uc, np.conj(vc))
            W = np.einsum(f"{p.lu},{p.lv}->{p.lw}", O.expand(p.group, p.sym_u, uc), dense_conj)
            want, forb = O.restrict(p.group, pc.sym_w, W)
            assert forb == 0.0
            assert rel(got, want) <= 1e-13


# --------------------------------------------------------------------------
# generalized symmetry (Eq. symtsr): sub-group coefficients c = +-G/H and
# non-uniform sector sizes held in zero-padded blocks (Sec. 1)
# --------------------------------------------------------------------------

def _divisors(n):
    return [d for d in range(1, n + 1) if n % d == 0]


def random_general_case(s, t, v, G, rng, sigma, pad=True, sub=True):
    """A random contraction whose modes have random sector counts H | G and,
    with pad, random true block sizes d(q) in [0, D] (some modes uniform)."""
    labels = iter("abcdefghijklmnop")
    FU = [next(labels) for _ in range(s)]
    C = [next(labels) for _ in range(v)]
    FV = [next(labels) for _ in range(t)]
    lu = "".join(rng.permutation(FU + C)) if FU or C else ""
    lv = "".join(rng.permutation(C + FV)) if C or FV else ""
    lw = "".join(rng.permutation(FU + FV)) if (FU or FV) else ""
    g = O.Group((G,))
    H = {c: (int(rng.choice(_divisors(G))) if sub else G) for c in lu + lv}
    D = {c: int(rng.integers(1, 4)) for c in lu + lv}
    SD = {}
    for c in lu + lv:
        if pad and rng.random() < 0.7:
            SD[c] = tuple(int(rng.integers(0, D[c] + 1)) for _ in range(H[c]))
        else:
            SD[c] = tuple([D[c]] * H[c])
    su_signs = {c: int(rng.choice([-1, 1])) for c in lu}
    sv_signs = {c: (sigma * su_signs[c] if c in C else int(rng.choice([-1, 1]))) for c in lv}
    zu, zv = (int(rng.integers(0, G)),), (int(rng.integers(0, G)),)

    def sym(lab, signs, z):
        return O.Sym(tuple(signs[c] for c in lab), z, tuple(D[c] for c in lab),
                     tuple(H[c] for c in lab), tuple(SD[c] for c in lab))
    su, sv = sym(lu, su_signs, zu), sym(lv, sv_signs, zv)
    p = O.plan(f"{lu},{lv}->{lw}", g, su, sv)
    u = rng.standard_normal(O.reduced_shape(g, su))
    vv = rng.standard_normal(O.reduced_shape(g, sv))
    return p, u, vv


GEN_STV = [(1, 1, 1), (2, 1, 1), (1, 2, 2), (2, 2, 1), (0, 2, 1), (1, 0, 2), (2, 1, 0), (3, 1, 1),
           (0, 0, 2)]


@pytest.mark.parametrize("s,t,v", GEN_STV)
def test_general_routes_agree_with_compact_dense_bruteforce(s, t, v):
    """Sub-group coefficients and padded non-uniform blocks: the block loop
    (O4), the dense-delta aligned route (O5) and entry-by-entry Eq. ctr agree
    with the dense einsum over the compact unfolded tensors (O3), whose
    forbidden blocks are exactly zero."""
    rng = np.random.default_rng(900 + 100 * s + 10 * t + v)
    for G, sigma in [(4, -1), (6, 1), (8, -1), (12, 1)]:
        if G ** (s + t + v) > 30000:
            continue
        for _ in range(2):
            p, u, vv = random_general_case(s, t, v, G, rng, sigma)
            w3, forb = O.contract_dense_einsum(p, u, vv)
            assert forb == 0.0
            w4 = O.contract_blockloop(p, u, vv)
            w5 = O.contract_aligned(p, u, vv)
            assert rel(w4, w3) <= 1e-13
            assert rel(w5, w3) <= 1e-13
            if w3.ndim:
                for _ in range(4):
                    ix = tuple(int(rng.integers(0, d)) for d in w3.shape)
                    e = O.contract_element(p, u, vv, ix)
                    el = O.contract_element_lazy(p, lambda i: u[i], lambda i: vv[i], ix)
                    assert abs(e - w3[ix]) <= 1e-12 * (1 + abs(w3[ix]))
                    assert abs(el - w3[ix]) <= 1e-12 * (1 + abs(w3[ix]))


def test_dense_loops_match_einsum_general():
    rng = np.random.default_rng(77)
    for (s, t, v) in [(1, 1, 1), (2, 1, 1), (1, 1, 2)]:
        p, u, vv = random_general_case(s, t, v, 6, rng, -1)
        W = O.contract_dense_loops(p, u, vv)
        Wr, _ = O.restrict(p.group, p.sym_w, W)
        assert rel(Wr, O.contract_blockloop(p, u, vv)) <= 1e-13


def test_subgroup_modes_relabel_to_the_smaller_cyclic_group():
    """Every mode with H sectors and coefficient +-G/H, remainders multiples
    of G/H: the law sum (G/H) c q == (G/H) z (mod G) is the Z_H law sum c q == z
    (mod H), so the reduced forms and the result equal those of the Z_H
    contraction with +-1 coefficients."""
    rng = np.random.default_rng(31)
    for G, h in [(8, 4), (12, 3), (6, 2), (8, 2)]:
        k = G // h
        for spec_, su_s, sv_s in [("abkl,klij->abij", (1, 1, -1, -1), (1, 1, -1, -1)),
                                  ("iak,kjb->ijab", (1, -1, 1), (1, 1, -1))]:
            lu, rest = spec_.split(",")
            lv = rest.split("->")[0]
            du = tuple(int(rng.integers(1, 4)) for _ in lu)
            dv = tuple(du[lu.index(c)] if c in lu else int(rng.integers(1, 4)) for c in lv)
            zu, zv = int(rng.integers(0, h)), int(rng.integers(0, h))
            gen = O.plan(spec_, O.Group((G,)),
                         O.Sym(su_s, (k * zu,), du, tuple([h] * len(lu))),
                         O.Sym(sv_s, (k * zv,), dv, tuple([h] * len(lv))))
            small = O.plan(spec_, O.Group((h,)), O.Sym(su_s, (zu,), du), O.Sym(sv_s, (zv,), dv))
            assert O.reduced_shape(gen.group, gen.sym_u) == O.reduced_shape(small.group, small.sym_u)
            u = rng.standard_normal(O.reduced_shape(small.group, small.sym_u))
            v = rng.standard_normal(O.reduced_shape(small.group, small.sym_v))
            assert np.array_equal(O.contract_blockloop(gen, u, v), O.contract_blockloop(small, u, v))


def test_uniform_sector_sizes_are_the_plain_form():
    """sector_dims all equal to D (and H = G) describe the plain tensor: the
    same result, bit for bit."""
    rng = np.random.default_rng(32)
    for c in WL.small_cases()[:6]:
        p = mk(c)
        G = p.group.order
        full = lambda sym: O.Sym(sym.signs, sym.charge, sym.dims, tuple([G] * sym.order),
                                 tuple(tuple([d] * G) for d in sym.dims))
        if len(p.group.moduli) != 1:
            continue
        pg = O.plan(c.einsum, p.group, full(p.sym_u), full(p.sym_v))
        u, v = WL.draw_pair(c)
        assert np.array_equal(O.contract_blockloop(pg, u, v), O.contract_blockloop(p, u, v))


def test_padding_is_read_as_zero_and_written_as_zero():
    """Garbage in the padding of the inputs changes nothing; the padding of
    the output and its entries without a solution are zero (Sec. 1: blocks are
    padded with zeros)."""
    rng = np.random.default_rng(33)
    for (s, t, v) in [(2, 1, 1), (1, 2, 2), (2, 2, 1)]:
        p, u, vv = random_general_case(s, t, v, 8, rng, 1)
        w = O.contract_blockloop(p, u, vv)
        cu, cv = O.sanitize(p.group, p.sym_u, u), O.sanitize(p.group, p.sym_v, vv)
        assert np.array_equal(O.contract_blockloop(p, cu, cv), w)
        noise_u = np.where(cu == 0, rng.standard_normal(u.shape) * 1e3, cu)
        noise_v = np.where(cv == 0, rng.standard_normal(vv.shape) * 1e3, cv)
        assert np.array_equal(O.contract_blockloop(p, noise_u, noise_v), w)
        assert np.array_equal(O.sanitize(p.group, p.sym_w, w), w)


@pytest.mark.parametrize("s,t,v", [(1, 1, 1), (2, 1, 2), (2, 2, 1), (0, 2, 1), (1, 0, 2), (2, 1, 0)])
def test_general_aligned_index_matches_dense_delta_route(s, t, v):
    """aligned_index / aligned_valid against align_u, align_v, mapback_w for
    sub-group coefficients and padding: valid entries sit where the dense
    route puts them, absent ones are zero in the dense route's aligned forms."""
    rng = np.random.default_rng(1500 + 100 * s + 10 * t + v)
    for G, sigma in [(4, 1), (6, -1), (8, 1)]:
        if G ** (s + t + v) > 5000:
            continue
        p, u, vv = random_general_case(s, t, v, G, rng, sigma)
        Gn, M, N, K = O.aligned_dims(p)
        uh, vh = O.align_u(p, u), O.align_v(p, vv)
        wh = rng.standard_normal((Gn, M, N))
        w = O.mapback_w(p, wh)
        for Q in range(G):
            m, n, k = np.arange(M)[:, None], np.arange(N)[:, None], np.arange(K)[None, :]
            for op, red, al, r in ((0, u, uh, m), (1, vv, vh, n)):
                if not (p.lu if op == 0 else p.lv):
                    continue
                ok = O.aligned_valid(p, op, Q, r, k)
                assert np.array_equal(np.where(ok, red[O.aligned_index(p, op, Q, r, k)], 0.0), al[Q])
            if p.lw:
                nn = np.arange(N)[None, :]
                ok = O.aligned_valid(p, 2, Q, m, nn)
                got = w[O.aligned_index(p, 2, Q, m, nn)]
                assert np.array_equal(got[ok], wh[Q][ok])


def test_general_adjoint_identity():
    """<W(U, V), Y> = <U, gU(Y)> = <V, gV(Y)> with sub-group coefficients and
    padding (the gradients are the adjoint contractions, O6)."""
    rng = np.random.default_rng(34)
    for (s, t, v) in [(1, 1, 1), (2, 1, 2), (2, 2, 1)]:
        p, u, vv = random_general_case(s, t, v, 6, rng, -1)
        u, vv = O.sanitize(p.group, p.sym_u, u), O.sanitize(p.group, p.sym_v, vv)
        y = O.sanitize(p.group, p.sym_w, rng.standard_normal(O.reduced_shape(p.group, p.sym_w)))
        w = O.contract_blockloop(p, u, vv)
        a = float(np.sum(w * y))
        b = float(np.sum(u * O.grad_u(p, y, vv)))
        c = float(np.sum(vv * O.grad_v(p, u, y)))
        assert abs(a - b) <= 1e-12 * (1 + abs(a)) and abs(a - c) <= 1e-12 * (1 + abs(a))


def test_planted_wrong_subgroup_solve_is_caught(monkeypatch):
    """Plant a plausible mistake in the sub-group solve (forgetting that
    c q == r (mod G) with c = G/H needs r divisible by G/H and q = r / (G/H)):
    the brute-force pin against the compact dense einsum catches it."""
    def wrong(self, coef, sectors, coeffs, labels, z):
        rest = self.charge(coeffs, labels)[0]
        return ((1 if coef > 0 else -1) * (self.norm(z)[0] - rest)) % sectors
    rng = np.random.default_rng(35)
    cases = [random_general_case(2, 1, 1, 8, rng, -1) for _ in range(4)]
    monkeypatch.setattr(O.Group, "solve_coef", wrong)
    caught = 0
    for p, u, vv in cases:
        w3, _ = O.contract_dense_einsum(p, u, vv)
        if rel(O.contract_blockloop(p, u, vv), w3) > 1e-6:
            caught += 1
    assert caught > 0
