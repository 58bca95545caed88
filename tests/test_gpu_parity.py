"""GPU parity: the CUDA path (through the C ABI) against the CPU float64 oracle.

Tolerances (relative Frobenius error against the oracle's block loop):
  fp64        <= 1e-12   (float64 FMA; summation order differs)
  split_bf16  <= 1e-10   (5 BF16 slices of 8 bits: truncation ~2^-39 per
                          operand entry relative to its row maximum)
  tf32        <= 1e-2    (operands rounded to 11 significant bits)
Alignment transforms are compared bit for bit.
"""
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


def dev(a):
    return torch.from_numpy(np.array(a, dtype=np.float64, order="C", copy=True)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    n = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (n if n > 0 else 1.0))


def oplan(einsum, moduli, su, sv):
    return O.plan(einsum, O.Group(moduli), O.Sym(*su), O.Sym(*sv))


def spec(t):
    return (t.signs, t.charge, t.dims)


def run_case(sc, einsum, moduli, su, sv, u, v, precision, check_err=True):
    p = sc.Plan(einsum, moduli, su, sv, precision)
    w = p.contract(dev(u), dev(v))
    torch.cuda.synchronize()
    if check_err:
        p.check_device_error()
    o = oplan(einsum, moduli, su, sv)
    want = O.contract_blockloop(o, u, v)
    return rel(host(w), want), p, w, want


# ---------------------------------------------------------------------------
# small contractions spanning (s, t, v), sigma, charges, product groups
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "split_bf16", "tf32"])
@pytest.mark.parametrize("case", WL.small_cases(), ids=lambda c: c.name)
def test_small_cases(sc, case, precision):
    u, v = WL.draw_pair(case)
    e, p, _, _ = run_case(sc, case.einsum, case.moduli, spec(case.u), spec(case.v), u, v, precision)
    assert e <= TOL[precision], (case.name, precision, e)


@pytest.mark.parametrize("case", WL.small_cases(), ids=lambda c: c.name)
def test_alignment_bit_exact(sc, case):
    """symctr_align against the oracle's delta-tensor transforms, both directions."""
    u, v = WL.draw_pair(case)
    p = sc.Plan(case.einsum, case.moduli, spec(case.u), spec(case.v))
    o = oplan(case.einsum, case.moduli, spec(case.u), spec(case.v))
    qs = O.q_set(o)
    w = O.contract_blockloop(o, u, v)
    for operand, red, al in ((0, u, O.align_u(o, u)), (1, v, O.align_v(o, v)),
                             (2, w, O.align_w(o, w))):
        got = host(p.align(operand, +1, dev(red)))
        assert np.array_equal(got, al[qs]), (case.name, operand)
        back = host(p.align(operand, -1, dev(al[qs])))
        # entries whose irrep carries no work come back as zero
        full = O.mapback_w(o, al) if operand == 2 else None
        if operand == 2:
            assert np.array_equal(back, full)
        elif len(qs) == p.info.group_order or al[[q for q in range(p.info.group_order)
                                                  if q not in qs]].size == 0:
            assert np.array_equal(back, red)
        else:
            kept = np.isin(red, al[qs])
            assert np.array_equal(back[kept], red[kept]) and not back[~kept].any()


def test_mapback_zero_fill_outer_product(sc):
    """v = 0: W entries whose irrep carries no work must be written as zeros."""
    case = [c for c in WL.small_cases() if c.name == "outer_v0_G3"][0]
    u, v = WL.draw_pair(case)
    for prec in ("fp64", "split_bf16"):
        p = sc.Plan(case.einsum, case.moduli, spec(case.u), spec(case.v), prec)
        w = torch.full(p.shape_w, 7.0, dtype=torch.float64, device="cuda")
        p.contract(dev(u), dev(v), out=w)
        want = O.contract_blockloop(oplan(case.einsum, case.moduli, spec(case.u), spec(case.v)), u, v)
        assert rel(host(w), want) <= 1e-12


@pytest.mark.parametrize("p_dim", [2, 3])
def test_gemv_and_adjoints_many_chunks(sc, p_dim):
    """A GEMV under Z_2 x Z_3 (M = p_dim, N = 1, K = 6^3 * 12^4 per irrep)
    and its two adjoints in float64: an outer product (K = 1, p_dim short
    rows) and a product with K = p_dim, both over 4.5M long-side rows, so that
    the short-K kernel's persistent blocks walk several row chunks each (the
    block offsets of every chunk after the first are computed without the
    per-irrep staging) and the skinny kernel splits K over every resident
    warp.  p_dim = 3 takes the short-K kernel's loop over a run-time K."""
    moduli = (2, 3)
    st = ((1, 1, -1, -1, 1), (0, 0), (12, 12, 12, 12, p_dim))
    se = ((-1, -1, 1, 1), (0, 0), (12, 12, 12, 12))
    T = WL.draw(WL.TensorSpec(*st, 1.0, 4301), moduli)
    Env = WL.draw(WL.TensorSpec(*se, 1e-3, 4302), moduli)
    py = sc.Plan("uldrp,uldr->p", moduli, st, se, "fp64")
    Td, Ed = dev(T), dev(Env)
    y = py.contract(Td, Ed)
    oy = oplan("uldrp,uldr->p", moduli, st, se)
    y_ref = O.contract_blockloop(oy, T, Env)
    assert rel(host(y), y_ref) <= 1e-12
    gy = np.random.default_rng(4303).standard_normal(y_ref.shape)
    gT, gE = py.backward(dev(gy), Td, Ed)
    torch.cuda.synchronize()
    assert rel(host(gT), O.grad_u(oy, gy, Env)) <= 1e-12
    assert rel(host(gE), O.grad_v(oy, T, gy)) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_outer_product_fills_only_unwritten_sectors(sc, precision):
    """An outer product under Z_2 x Z_3 (W's sector combinations: 6^4, one in
    six written by the single irrep that carries work) into an output filled
    with 7.0 first: the zero fill skips the written sector blocks, so every
    other entry must still come out exactly zero and every written one must
    match the oracle."""
    moduli = (2, 3)
    su = ((-1, -1, 1, 1), (0, 0), (6, 6, 6, 6))
    sv = ((1,), (0, 0), (2,))
    u = WL.draw(WL.TensorSpec(*su, 1.0, 4311), moduli)
    v = WL.draw(WL.TensorSpec(*sv, 1.0, 4312), moduli)
    p = sc.Plan("uldr,p->uldrp", moduli, su, sv, precision)
    w = torch.full(p.shape_w, 7.0, dtype=torch.float64, device="cuda")
    p.contract(dev(u), dev(v), out=w)
    want = O.contract_blockloop(oplan("uldr,p->uldrp", moduli, su, sv), u, v)
    got = host(w)
    assert not got[want == 0].any()
    assert rel(got, want) <= 1e-12


# ---------------------------------------------------------------------------
# the paper-shaped workloads
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "split_bf16", "tf32"])
def test_config1_order4_z3(sc, precision):
    c = WL.Z3_ORDER4
    u, v = WL.draw_pair(c)
    e, p, _, _ = run_case(sc, c.einsum, c.moduli, spec(c.u), spec(c.v), u, v, precision)
    assert (p.info.M, p.info.N, p.info.K) == (48, 48, 48)
    assert e <= TOL[precision], e


@pytest.mark.parametrize("precision", ["fp64", "split_bf16", "tf32"])
def test_config2_mps_transfer(sc, precision):
    E = WL.draw(WL.MPS_E, (8,))
    A = WL.draw(WL.MPS_A, (8,))
    e1, p1, X, want_x = run_case(sc, WL.MPS_STEP1, (8,), spec(WL.MPS_E), spec(WL.MPS_A), E, A,
                                 precision)
    assert e1 <= TOL[precision], e1
    p2 = sc.Plan(WL.MPS_STEP2, (8,), p1.sym_w, spec(WL.MPS_A), precision)
    E2 = p2.contract(X, dev(A))
    o2 = oplan(WL.MPS_STEP2, (8,), (p1.sym_w.signs, p1.sym_w.charge, p1.sym_w.dims), spec(WL.MPS_A))
    want = O.contract_blockloop(o2, want_x, A)
    assert rel(host(E2), want) <= 2 * TOL[precision]


def test_tf32_long_k_few_tiles_is_deterministic(sc):
    """E' = X.A in the TF32 form (M = N = 128, K = 2048, 8 irreps: 8 tiles,
    each accumulating all of K in TMEM): repeated calls give the same bits, and
    the result matches the oracle at the TF32 tolerance."""
    A = WL.draw(WL.MPS_A, (8,))
    p1 = sc.Plan(WL.MPS_STEP1, (8,), spec(WL.MPS_E), spec(WL.MPS_A), "fp64")
    X = torch.randn(p1.shape_w, dtype=torch.float64, generator=torch.Generator().manual_seed(77))
    p2 = sc.Plan(WL.MPS_STEP2, (8,), p1.sym_w, spec(WL.MPS_A), "tf32")
    assert (p2.info.M, p2.info.N, p2.info.K, p2.info.n_q) == (128, 128, 2048, 8)
    Xd, Ad = X.cuda(), dev(A)
    first = p2.contract(Xd, Ad)
    again = [p2.contract(Xd, Ad) for _ in range(3)]
    torch.cuda.synchronize()
    p2.check_device_error()
    assert all(torch.equal(first, a) for a in again)
    o2 = oplan(WL.MPS_STEP2, (8,), (p1.sym_w.signs, p1.sym_w.charge, p1.sym_w.dims), spec(WL.MPS_A))
    assert rel(host(first), O.contract_blockloop(o2, X.numpy(), A)) <= TOL["tf32"]


@pytest.mark.parametrize("precision", ["fp64", "split_bf16", "tf32"])
def test_cc_ladder_reduced_size(sc, precision):
    """Config 3's contraction at block size 8/4 (G = 8): M = K = 512, N = 128,
    several tiles in M, eight exact-flush chunks in K."""
    c = WL.cc_ladder(8, 64, 32)
    u, v = WL.draw_pair(c)
    e, p, _, _ = run_case(sc, c.einsum, c.moduli, spec(c.u), spec(c.v), u, v, precision)
    assert (p.info.M, p.info.K, p.info.N) == (512, 512, 128)
    assert e <= TOL[precision], e


@pytest.mark.parametrize("precision", ["split_bf16", "tf32", "fp64"])
def test_ragged_tiles(sc, precision):
    """M, N not multiples of 128 and K not a multiple of 32 (ragged tails)."""
    su = ((1, -1, 1), (0,), (5, 9, 7))          # a b k
    sv = ((-1, 1), (0,), (7, 11))               # k c
    G = 3
    u = np.random.default_rng(31).standard_normal((G, G, 5, 9, 7))
    v = np.random.default_rng(32).standard_normal((G, 7, 11))
    e, p, _, _ = run_case(sc, "abk,kc->abc", (G,), su, sv, u, v, precision)
    assert (p.info.M, p.info.N, p.info.K) == (135, 11, 7)
    assert e <= TOL[precision], e
    # a tensor-core-sized ragged case
    su2 = ((1, 1, -1), (1,), (13, 11, 37))
    sv2 = ((1, -1, 1), (2,), (37, 29, 5))
    u2 = np.random.default_rng(33).standard_normal((G, G, 13, 11, 37))
    v2 = np.random.default_rng(34).standard_normal((G, G, 37, 29, 5))
    e2, p2, _, _ = run_case(sc, "abk,kcd->abcd", (G,), su2, sv2, u2, v2, precision)
    assert p2.info.M == G * 13 * 11 and p2.info.K == 37
    assert e2 <= TOL[precision], e2


@pytest.mark.parametrize("k_blocks", [1, 3, 64, 257])
def test_split_exactness_all_positive(sc, k_blocks):
    """All-positive data makes every slice-pair partial sum grow linearly with K:
    without exact flushes of the top diagonals the FP32 accumulators would
    round.  K up to 8224 (257 stages of 32)."""
    G, Dm, Dn = 2, 130, 70
    Dk = 32 * k_blocks
    su = ((1, -1), (0,), (Dm, Dk))
    sv = ((1, -1), (0,), (Dk, Dn))
    rng = np.random.default_rng(40 + k_blocks)
    u = rng.random((G, Dm, Dk))
    v = rng.random((G, Dk, Dn))
    e, p, _, _ = run_case(sc, "ij,jk->ik", (G,), su, sv, u, v, "split_bf16")
    assert e <= 1e-10, e


@pytest.mark.parametrize("D_j,prep", [(96, 12), (4100, 0)])
def test_split_extreme_exponents(sc, D_j, prep):
    """Rows scaled by very different powers of two, a zero row, a row of
    subnormals and a row of V of subnormals below 2^-1042 (high words all
    zero), through the short-row kernel (K = 96) and the two-phase kernel
    (K = 4100)."""
    G = 2
    su = ((1, -1), (0,), (64, D_j))
    sv = ((1, -1), (0,), (D_j, 48))
    rng = np.random.default_rng(50)
    u = rng.standard_normal((G, 64, D_j)) * np.exp2(rng.integers(-300, 300, size=(G, 64, 1)))
    v = rng.standard_normal((G, D_j, 48)) * np.exp2(rng.integers(-300, 300, size=(G, 1, 48)))
    u[0, 5, :] = 0.0
    u[1, 7, :] = 1e-310 * rng.standard_normal(D_j)
    # k 2^-1050, |k| <= 127: every high word zero (the scale comes from the
    # low words); at the clamped scale 2^(8S-1076) these sit one digit below
    # the top, so their products with U's last digit fall into the dropped
    # diagonals: that column is accurate to ~2^-32 of its scale only
    v[0, :, 9] = np.ldexp(rng.integers(-127, 128, size=D_j).astype(np.float64), -1050)
    p = sc.Plan("ij,jk->ik", (G,), su, sv, "split_bf16")
    assert p.info.single_read_prep == prep
    got = host(p.contract(dev(u), dev(v)))
    p.check_device_error()
    want = O.contract_blockloop(oplan("ij,jk->ik", (G,), su, sv), u, v)
    # the natural error scale of a dot product: sum_j |u_ij| |v_jk| (the same
    # form as the float64 GEMM bound), evaluated in float64 without overflow
    scale = np.einsum("qij,qjk->qik", np.abs(u), np.abs(v))
    assert np.all(got[0, 5] == 0.0)
    ok = scale > 1e-290
    tiny = np.zeros_like(ok)
    tiny[0, :, 9] = True
    assert np.all(np.abs(got - want)[ok & ~tiny] <= 1e-11 * scale[ok & ~tiny])
    assert np.all(np.abs(got - want)[ok & tiny] <= 1e-8 * scale[ok & tiny])


def test_nonfinite_input_is_reported(sc):
    c = WL.Z3_ORDER4
    u, v = WL.draw_pair(c)
    u = u.copy()
    u[0, 0, 0, 0, 0, 0, 0] = np.inf
    p = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "split_bf16")
    p.contract(dev(u), dev(v))
    with pytest.raises(sc.SymctrError) as ei:
        p.check_device_error()
    assert ei.value.status == 11
    p.check_device_error()  # the word was cleared


# ---------------------------------------------------------------------------
# gradients
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
@pytest.mark.parametrize("case", [WL.Z3_ORDER4] + [c for c in WL.small_cases()
                                                   if c.name in ("sigma_plus_G5", "z2xz3_order4",
                                                                 "outer_v0_G3", "s0_G4", "t0_G2")],
                         ids=lambda c: c.name)
def test_backward_matches_oracle_gradient(sc, case, precision):
    u, v = WL.draw_pair(case)
    p = sc.Plan(case.einsum, case.moduli, spec(case.u), spec(case.v), precision)
    o = oplan(case.einsum, case.moduli, spec(case.u), spec(case.v))
    y = np.random.default_rng(77).standard_normal(p.shape_w)
    gu, gv = p.backward(dev(y), dev(u), dev(v))
    torch.cuda.synchronize()
    tol = max(TOL[precision], 1e-12)
    assert rel(host(gu), O.grad_u(o, y, v)) <= tol
    assert rel(host(gv), O.grad_v(o, u, y)) <= tol


def test_autograd_function(sc):
    c = WL.Z3_ORDER4
    u, v = WL.draw_pair(c)
    p = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "fp64")
    ut = dev(u).requires_grad_(True)
    vt = dev(v).requires_grad_(True)
    w = sc.contract(p, ut, vt)
    loss = (w * w).sum()
    loss.backward()
    o = oplan(c.einsum, c.moduli, spec(c.u), spec(c.v))
    wref = O.contract_blockloop(o, u, v)
    assert rel(host(ut.grad), O.grad_u(o, 2 * wref, v)) <= 1e-12
    assert rel(host(vt.grad), O.grad_v(o, u, 2 * wref)) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "split_bf16", "tf32"])
def test_no_irrep_carries_work(sc, precision):
    """A full contraction whose laws admit no irrep Q (s = t = 0 and
    Z_U != sigma Z_V): every block product is forbidden, W is exactly zero."""
    su, sv = ((1, -1), (1,), (3, 3)), ((1, -1), (2,), (3, 3))
    p = sc.Plan("ij,ij->", (4,), su, sv, precision)
    assert p.info.n_q == 0
    o = oplan("ij,ij->", (4,), su, sv)
    rng = np.random.default_rng(5)
    u = rng.standard_normal(O.reduced_shape(o.group, o.sym_u))
    v = rng.standard_normal(O.reduced_shape(o.group, o.sym_v))
    w = p.contract(dev(u), dev(v))
    p.check_device_error()
    assert O.contract_blockloop(o, u, v) == 0.0
    assert host(w) == 0.0


@pytest.mark.parametrize("k_sectors,D", [(2, 64), (2, 4096), (4, 8192)])
def test_split_bit_exact_on_integer_inputs(sc, k_sectors, D):
    """Integer entries with |x| <= 2^12 are exactly two balanced BF16 digits
    at their row scale, so every slice-pair product lands in the exact
    diagonals 0..2: the split form must return the exact integer matrix
    product rounded once to float64, bit for bit.  Rows at the maximum
    magnitude (all digits at the bound) drive every drain to its limit."""
    G = k_sectors
    su = ((1, -1), (0,), (128, D))
    sv = ((1, -1), (0,), (D, 96))
    rng = np.random.default_rng(600 + D)
    u = rng.integers(-4096, 4097, size=(G, 128, D)).astype(np.float64)
    v = rng.integers(-4096, 4097, size=(G, D, 96)).astype(np.float64)
    u[:, :4, :] = 4096.0          # all-maximum rows and columns
    v[:, :, :3] = 4096.0
    u[:, 4:6, :] = -4096.0
    p = sc.Plan("ij,jk->ik", (G,), su, sv, "split_bf16")
    got = host(p.contract(dev(u), dev(v)))
    p.check_device_error()
    # exact integer products (|sum| <= D * 2^24 < 2^63), rounded once to float64
    want = np.stack([np.matmul(u[q].astype(np.int64), v[q].astype(np.int64)) for q in range(G)])
    assert np.array_equal(got, want.astype(np.float64))


@pytest.mark.parametrize("einsum,D_i,D_j,prep", [("ij,jk->ik", 1024, 4096, 1), ("ij,kj->ik", 1024, 4096, 1 | 8),
                                                  ("ij,kj->ik", 1024, 1000, 4 | 8),
                                                  ("ij,jk->ik", 1024, 2000, 4 | 8),
                                                  ("ij,jk->ik", 1024, 3000, 1), ("ij,jk->ik", 500, 3000, 4),
                                                  ("ij,jk->ik", 512, 10000, 1), ("ij,jk->ik", 256, 16384, 1),
                                                  ("ij,jk->ik", 128, 24578, 1), ("ij,jk->ik", 64, 65536, 1)])
def test_single_read_prep_bit_exact_on_integer_inputs(sc, einsum, D_i, D_j, prep):
    """The single-read preparations on shapes that take them (plan bits 0/1:
    rows streamed by bulk copies of contiguous runs, by one CTA up to K = 8192
    and by clusters of 2 to 8 CTAs holding one segment each beyond; 2/3: whole
    short rows per CTA, gathered along the rows or across them; neither: the
    two-phase kernel), alone and side by side: integer inputs of two BF16 digits must give
    the exact integer product rounded once, bit for bit."""
    G, D_k = 2, 72
    su = ((1, -1), (0,), (D_i, D_j))
    sv = ((1, -1), (0,), (D_j, D_k) if einsum == "ij,jk->ik" else (D_k, D_j))
    rng = np.random.default_rng(611 + D_j)
    u = rng.integers(-4096, 4097, size=(G, D_i, D_j)).astype(np.float64)
    v = rng.integers(-4096, 4097, size=(G,) + sv[2]).astype(np.float64)
    u[:, :4, :] = 4096.0
    u[:, 4:6, :] = -4096.0
    u[:, 6, :] = 0.0              # an all-zero row
    # a row of subnormals k * 2^-1050, |k| <= 127: every high word is zero (the
    # row scale comes from the exact pass over the whole bit patterns) and the
    # row scale is the clamped one, 2^(8S - 1076) = 2^-1036 at S = 5, at which
    # each entry is the single BF16 digit k * 2^-8 below the top: its products
    # with V's two digits stay in the exact diagonals
    ks = rng.integers(-127, 128, size=(G, D_j))
    u[:, 7, :] = np.ldexp(ks.astype(np.float64), -1050)
    p = sc.Plan(einsum, (G,), su, sv, "split_bf16")
    assert p.info.single_read_prep == prep
    got = host(p.contract(dev(u), dev(v)))
    p.check_device_error()
    vm = v if einsum == "ij,jk->ik" else np.swapaxes(v, 1, 2)
    ui = u.copy()
    ui[:, 7, :] = 0.0
    # integer sums below 2^53: exact in float64 in any order
    want = np.stack([np.matmul(ui[q], vm[q]) for q in range(G)])
    for q in range(G):
        want[q, 7, :] = np.ldexp(ks[q].astype(np.float64) @ vm[q], -1050)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("D_j", [4096, 16384])
def test_single_read_prep_nonfinite_is_reported(sc, D_j):
    """A NaN in an operand prepared by the single-read kernel sets the device
    error word (and nothing traps)."""
    G, D_i, D_k = 2, 16777216 // (2 * D_j), 64
    p = sc.Plan("ij,jk->ik", (G,), ((1, -1), (0,), (D_i, D_j)), ((1, -1), (0,), (D_j, D_k)),
                "split_bf16")
    assert p.info.single_read_prep & 1
    rng = np.random.default_rng(612)
    u = rng.standard_normal((G, D_i, D_j))
    u[1, 77, D_j - 1234] = np.nan   # in the last CTA's segment of a cluster
    v = rng.standard_normal((G, D_j, D_k))
    p.contract(dev(u), dev(v))
    with pytest.raises(sc.SymctrError) as ei:
        p.check_device_error()
    assert ei.value.status == 11


@pytest.mark.parametrize("precision", ["split_bf16", "tf32"])
def test_mps_step_repeatable(sc, precision):
    """The MPS transfer step (both contractions, the second reading the first's
    output): against the oracle, and bit-identical over repeated calls."""
    E = WL.draw(WL.MPS_E, (8,))
    A = WL.draw(WL.MPS_A, (8,))
    p1 = sc.Plan(WL.MPS_STEP1, (8,), spec(WL.MPS_E), spec(WL.MPS_A), precision)
    p2 = sc.Plan(WL.MPS_STEP2, (8,), p1.sym_w, spec(WL.MPS_A), precision)
    Ed, Ad = dev(E), dev(A)
    X = p1.contract(Ed, Ad)
    E2 = p2.contract(X, Ad)
    again = p2.contract(p1.contract(Ed, Ad), Ad)
    torch.cuda.synchronize()
    p1.check_device_error()
    p2.check_device_error()
    assert torch.equal(E2, again)
    o1 = oplan(WL.MPS_STEP1, (8,), spec(WL.MPS_E), spec(WL.MPS_A))
    o2 = oplan(WL.MPS_STEP2, (8,), (p1.sym_w.signs, p1.sym_w.charge, p1.sym_w.dims), spec(WL.MPS_A))
    Xr = O.contract_blockloop(o1, E, A)
    assert rel(host(X), Xr) <= TOL[precision]
    assert rel(host(E2), O.contract_blockloop(o2, Xr, A)) <= 2 * TOL[precision]


def test_mps_nonfinite_is_reported(sc):
    """An infinity in E (read by the preparation of X = E.A) sets the device
    error word."""
    E = WL.draw(WL.MPS_E, (8,)).copy()
    A = WL.draw(WL.MPS_A, (8,))
    E[3, 5, 7] = np.inf
    p1 = sc.Plan(WL.MPS_STEP1, (8,), spec(WL.MPS_E), spec(WL.MPS_A), "split_bf16")
    p1.contract(dev(E), dev(A))
    with pytest.raises(sc.SymctrError) as ei:
        p1.check_device_error()
    assert ei.value.status == 11
