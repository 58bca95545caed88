"""C ABI checks that need no GPU: the library loads, exports every entry point
that include/symctr.h declares, and its host-side planner agrees with the
oracle's charge algebra (derived output law, aligned GEMM extents, irrep
set) and reports the documented error statuses."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2007_08056_gb300 as sc
import workloads as WL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "symctr.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"SYMCTR_API\s+[\w\s\*]+?\b(symctr_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = sc.load()
    names = declared_symbols()
    assert "symctr_contract" in names and "symctr_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings():
    lib = sc.load()
    for code, name in sc.STATUS.items():
        assert lib.symctr_status_string(code).decode() == name


def oracle_plan(c):
    g = O.Group(c.moduli)
    return O.plan(c.einsum, g, O.Sym(c.u.signs, c.u.charge, c.u.dims),
                  O.Sym(c.v.signs, c.v.charge, c.v.dims))


CASES = WL.small_cases() + [WL.CC_LADDER, WL.cc_ladder(16, 512, 128)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
@pytest.mark.parametrize("precision", ["fp64", "split_bf16", "tf32"])
def test_planner_matches_oracle(case, precision):
    p = sc.Plan(case.einsum, case.moduli, (case.u.signs, case.u.charge, case.u.dims),
                (case.v.signs, case.v.charge, case.v.dims), precision)
    o = oracle_plan(case)
    G, M, N, K = O.aligned_dims(o)
    i = p.info
    assert (i.group_order, i.M, i.N, i.K) == (G, M, N, K)
    assert (i.s, i.t, i.v, i.sigma) == (o.s, o.t, o.v, o.sigma)
    assert p.sym_w.signs == o.sym_w.signs
    assert p.sym_w.charge == o.sym_w.charge
    assert p.sym_w.dims == o.sym_w.dims
    qs = O.q_set(o)
    assert p.q_values() == qs
    assert i.useful_flops == 2.0 * len(qs) * M * N * K
    assert p.shape_u == O.reduced_shape(o.group, o.sym_u)
    assert p.shape_w == O.reduced_shape(o.group, o.sym_w)
    assert i.workspace_bytes >= 256
    if precision == "split_bf16":
        assert i.n_slices == 5


def test_config_extents():
    """Aligned GEMM extents of the paper-shaped workloads."""
    p = sc.Plan(WL.CC_LADDER.einsum, (8,), (WL.PP, (0,), (32,) * 4), (WL.PP, (0,), (32, 32, 8, 8)))
    assert (p.info.M, p.info.K, p.info.N, p.info.n_q) == (8192, 8192, 512, 8)
    assert p.useful_flops == 549_755_813_888
    s1 = sc.Plan(WL.MPS_STEP1, (8,), (WL.MPS_E.signs, (0,), WL.MPS_E.dims),
                 (WL.MPS_A.signs, (0,), WL.MPS_A.dims))
    assert (s1.info.M, s1.info.K, s1.info.N) == (128, 128, 2048)
    s2 = sc.Plan(WL.MPS_STEP2, (8,), s1.sym_w, (WL.MPS_A.signs, (0,), WL.MPS_A.dims))
    assert (s2.info.M, s2.info.K, s2.info.N) == (128, 2048, 128)
    assert s2.sym_w.signs == WL.MPS_E.signs
    y = sc.Plan(WL.PEPS_Y, WL.PEPS_MODULI, (WL.PEPS_T.signs, (0, 0), WL.PEPS_T.dims),
                (WL.PEPS_ENV.signs, (0, 0), WL.PEPS_ENV.dims))
    assert (y.info.M, y.info.N, y.info.K, y.info.n_q) == (2, 1, 6 ** 3 * 16 ** 4, 1)


def plan_status(einsum, moduli, su, sv, sw=None):
    try:
        sc.Plan(einsum, moduli, su, sv, sym_w=sw)
        return 0
    except sc.SymctrError as e:
        return e.status


def test_error_statuses():
    pp = ((1, 1, -1, -1), (0,), (2, 2, 2, 2))
    assert plan_status("abkl,klij->abij", (3,), pp, pp) == 0
    assert plan_status("abkl,klij", (3,), pp, pp) == 1                     # no arrow
    assert plan_status("aakl,klij->ij", (3,), pp, pp) == 1                  # trace label
    assert plan_status("abkl,klij->abijk", (3,), pp, pp) == 1               # batch label
    assert plan_status("abkl,klij->abi", (3,), pp, pp) == 1                 # free label dropped
    mixed = ((1, -1, 1, -1), (0,), (2, 2, 2, 2))                             # k: sigma=-1, l: +1
    assert plan_status("abkl,klij->abij", (3,), pp, mixed) == 2
    assert plan_status("abkl,klij->abij", (3,), pp, ((1, 1, -1, -1), (0,), (3, 2, 2, 2))) == 3
    assert plan_status("abkl,klij->abij", (300,), pp, pp) == 5               # group too large
    # an output law that contradicts the derived one; its global negation is accepted
    assert plan_status("abkl,klij->abij", (3,), pp, pp, ((1, 1, -1, -1), (1,), (2,) * 4)) == 4
    assert plan_status("abkl,klij->abij", (3,), pp, pp, ((-1, -1, 1, 1), (0,), (2,) * 4)) == 0
    big = ((1,) * 9, (0,), (1,) * 9)
    assert plan_status("abcdefghi,a->bcdefghi", (2,), big, ((-1,), (0,), (1,))) == 5
    # an empty sector (D = 0) is rejected
    assert plan_status("abkl,klij->abij", (3,), pp, ((1, 1, -1, -1), (0,), (2, 2, 2, 0))) == 3


def test_null_arguments():
    lib = sc.load()
    out = ctypes.c_void_p()
    st = lib.symctr_plan_create(None, 1, None, None, None, None, None, None, None, None, None, 0,
                                0, ctypes.byref(out))
    assert st == 6
    assert lib.symctr_plan_query(None, None) == 6
    assert lib.symctr_contract(None, None, None, None, None, 0, None) == 6
    assert lib.symctr_contract_complex(None, 0, 0, None, None, None, None, 0, None) == 6
    assert lib.symctr_selftest_bounded_wait(None, 0, 0, None) == 6


def test_workspace_too_small_is_rejected_before_any_launch():
    """The size check happens on the host, so it needs no GPU."""
    p = sc.Plan(WL.Z3_ORDER4.einsum, (3,), (WL.PP, (0,), (4,) * 4), (WL.PP, (0,), (4,) * 4),
                "split_bf16")
    lib = sc.load()
    fake = ctypes.c_void_p(4096)
    st = lib.symctr_contract(p._h, fake, fake, fake, fake, 16, None)
    assert st == 7


def test_attach_tables_argument_checks():
    """symctr_plan_attach_tables checks its arguments on the host before any
    CUDA call; detaching (NULL buffer) touches no device either."""
    lib = sc.load()
    assert lib.symctr_plan_attach_tables(None, None, 0, None) == 6
    spec = lambda t: (t.signs, t.charge, t.dims)
    p = sc.Plan(WL.MPS_STEP1, (8,), spec(WL.MPS_E), spec(WL.MPS_A), "split_bf16")
    # forward tables (U, V and W rows and columns per irrep) plus the backward plans'
    own = 8 * 8 * (2 * p.info.M + 2 * p.info.N + 2 * p.info.K)
    assert p.info.table_bytes >= own and p.info.table_bytes % 256 == 0
    n = int(p.info.table_bytes)
    assert lib.symctr_plan_attach_tables(p._h, ctypes.c_void_p(4096), n - 1, None) == 7
    assert lib.symctr_plan_attach_tables(p._h, ctypes.c_void_p(4096 + 16), n, None) == 12
    assert lib.symctr_plan_attach_tables(p._h, None, 0, None) == 0
    # the float64 form keeps no tables
    p64 = sc.Plan(WL.MPS_STEP1, (8,), spec(WL.MPS_E), spec(WL.MPS_A), "fp64")
    assert p64.info.table_bytes == 0
    assert lib.symctr_plan_attach_tables(p64._h, ctypes.c_void_p(4096), 0, None) == 0


def test_engine_of_each_form_is_reported():
    """plan.info.tensor_core: the tensor-core forms run on tcgen05 for
    GEMM-shaped problems; GEMV shapes and the float64 form use the float64
    CUDA-core kernels."""
    c = WL.CC_LADDER
    spec = lambda t: (t.signs, t.charge, t.dims)
    for prec, want in (("split_bf16", 1), ("tf32", 1), ("fp64", 0)):
        assert sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), prec).info.tensor_core == want
    peps = sc.Plan(WL.PEPS_Y, WL.PEPS_MODULI, spec(WL.PEPS_T), spec(WL.PEPS_ENV), "split_bf16")
    assert peps.info.M == 2 and peps.info.tensor_core == 0


def test_preparation_kernel_of_each_operand_is_reported():
    """plan.info.single_read_prep: bits 0/1 (U/V) for rows of long contiguous
    runs (streamed by bulk copies), bits 2/3 for short rows (padded K <= 4096,
    whole rows per CTA); neither: the two-phase kernel (scan, grid barrier,
    slicing).  TF32 and float64 plans prepare no slices."""
    spec = lambda t: (t.signs, t.charge, t.dims)
    c = WL.CC_LADDER
    cc = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "split_bf16").info
    assert cc.K > 4096 and cc.single_read_prep == 1
    for prec, want in (("split_bf16", 12), ("tf32", 0), ("fp64", 0)):
        p1 = sc.Plan(WL.MPS_STEP1, (WL.MPS_G,), spec(WL.MPS_E), spec(WL.MPS_A), prec)
        p2 = sc.Plan(WL.MPS_STEP2, (WL.MPS_G,), p1.sym_w, spec(WL.MPS_A), prec)
        assert p1.info.single_read_prep == want and p2.info.single_read_prep == want
    # ij,jk: U's rows run along K, V's rows are the unit-stride side (at most
    # K = 2048 on the short-row kernel)
    for K, want in ((2048, 12), (2049, 4), (4096, 4), (4097, 0), (8192, 0)):
        p = sc.Plan("ij,jk->ik", (2,), ((1, -1), (0,), (64, K)), ((1, -1), (0,), (K, 64)),
                    "split_bf16")
        assert p.info.K == K and p.info.single_read_prep == want
    # U's rows are runs of 4096 contiguous entries (bulk copies); V's rows run
    # along K too and take the short-row kernel, or are the unit-stride side
    # and take the two-phase kernel
    p = sc.Plan("ij,kj->ik", (2,), ((1, -1), (0,), (1024, 4096)), ((1, -1), (0,), (64, 4096)),
                "split_bf16")
    assert p.info.single_read_prep == 1 | 8
    p = sc.Plan("ij,jk->ik", (2,), ((1, -1), (0,), (1024, 4096)), ((1, -1), (0,), (4096, 64)),
                "split_bf16")
    assert p.info.single_read_prep == 1
    # rows of runs longer than one CTA's buffers (K > 8192): the cluster form of the
    # bulk-copy kernel, up to K = 65536
    for K, want in ((16384, 1), (65536, 1), (65538, 0)):  # 2 x 256 x K >= 4M entries
        p = sc.Plan("ij,jk->ik", (2,), ((1, -1), (0,), (256, K)), ((1, -1), (0,), (K, 72)), "split_bf16")
        assert p.info.single_read_prep == want
    # short rows with runs: the short-row kernel
    p = sc.Plan("ij,kj->ik", (2,), ((1, -1), (0,), (4096, 1024)), ((1, -1), (0,), (64, 1024)),
                "split_bf16")
    assert p.info.single_read_prep == 4 | 8


def test_zero_fill_of_unwritten_sector_blocks():
    """plan.info.zero_fill_numel: the entries of W a contraction zeroes before
    the GEMM writes the rest (Alg. 2: entries of irreps that carry no work are
    zero).  In a uniform plan only the sector blocks no irrep writes are
    zeroed; the count is compared with the oracle's own sector bookkeeping
    (the share of W's sector combinations whose implicit sector puts them in
    an irrep that carries work)."""
    spec = lambda t: (t.signs, t.charge, t.dims)
    # an outer product under Z_2 x Z_3: one irrep carries work, and it writes
    # one sixth of W's 6^4 sector combinations
    su, sv = ((-1, -1, 1, 1), (0, 0), (6, 6, 6, 6)), ((1,), (0, 0), (2,))
    for prec in ("fp64", "split_bf16"):
        p = sc.Plan("uldr,p->uldrp", (2, 3), su, sv, prec)
        assert p.info.n_q == 1 and p.info.aligned_numel_w * 6 == p.info.numel_w
        assert p.info.zero_fill_numel == p.info.numel_w - p.info.aligned_numel_w
    # the same count from the oracle's plan: W entries outside the live irrep
    o = O.plan("uldr,p->uldrp", O.Group((2, 3)), O.Sym(*su), O.Sym(*sv))
    G, M, N, K = O.aligned_dims(o)
    assert int(np.prod(O.reduced_shape(o.group, o.sym_w))) - M * N == p.info.zero_fill_numel
    # irreps covering W: nothing zeroed (the CC ladder, config 4's GEMV)
    c = WL.CC_LADDER
    assert sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), "split_bf16").info.zero_fill_numel == 0
    y = sc.Plan(WL.PEPS_Y, WL.PEPS_MODULI, spec(WL.PEPS_T), spec(WL.PEPS_ENV), "fp64")
    assert y.info.numel_w == y.info.aligned_numel_w and y.info.zero_fill_numel == 0
    # no irrep carries work: all of W
    p0 = sc.Plan("ij,ij->", (4,), ((1, -1), (1,), (3, 3)), ((1, -1), (2,), (3, 3)), "fp64")
    assert p0.info.n_q == 0 and p0.info.zero_fill_numel == p0.info.numel_w
    # general plans zero all of W
    gp, _, _ = _general_cases()[0]
    q = sc.Plan(f"{gp.lu},{gp.lv}->{gp.lw}", gp.group.moduli, _as_spec(gp.sym_u), _as_spec(gp.sym_v),
                "fp64")
    assert q.info.zero_fill_numel == q.info.numel_w


class _FakeTensor:
    def __init__(self, dev):
        self.dev = dev

    def get_device(self):
        return self.dev


def test_tensors_on_another_device_are_rejected(monkeypatch):
    """The library launches on the current device; a tensor elsewhere is
    refused before anything is launched (checked without a GPU)."""
    monkeypatch.setattr(sc.torch.cuda, "current_device", lambda: 0)
    sc.Plan._same_device(_FakeTensor(0), None, _FakeTensor(0))
    with pytest.raises(ValueError):
        sc.Plan._same_device(_FakeTensor(0), _FakeTensor(1))


# --------------------------------------------------------------------------
# generalized symmetry (Eq. symtsr: H | G sectors, coefficient +-G/H; padded
# non-uniform sectors): the planner against the oracle's plan
# --------------------------------------------------------------------------

def _general_cases():
    import sys
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from test_oracle_pins import random_general_case
    rng = np.random.default_rng(2024)
    out = []
    for (s, t, v) in [(1, 1, 1), (2, 1, 1), (1, 2, 2), (2, 2, 1), (0, 2, 1), (1, 0, 2), (2, 1, 0),
                      (3, 1, 1)]:
        for G in (4, 6, 8, 12):
            out.append(random_general_case(s, t, v, G, rng, int(rng.choice([-1, 1]))))
    return out


def _as_spec(sym):
    return (sym.signs, sym.charge, sym.dims, sym.sectors, sym.sector_dims)


@pytest.mark.parametrize("precision", ["fp64", "split_bf16"])
def test_general_planner_matches_oracle(precision):
    for p, _, _ in _general_cases():
        q = sc.Plan(f"{p.lu},{p.lv}->{p.lw}", p.group.moduli, _as_spec(p.sym_u), _as_spec(p.sym_v),
                    precision)
        G, M, N, K = O.aligned_dims(p)
        assert (q.info.M, q.info.N, q.info.K) == (M, N, K)
        assert q.info.general == 1 and q.info.sigma == p.sigma
        assert q.shape_u == O.reduced_shape(p.group, p.sym_u)
        assert q.shape_w == O.reduced_shape(p.group, p.sym_w)
        assert q.sym_w.signs == p.sym_w.signs and q.sym_w.charge == p.sym_w.charge
        assert q.sym_w.sectors == p.sym_w.sectors and q.sym_w.sector_dims == p.sym_w.sector_dims
        # every form reads the general index maps from tables (none when no irrep carries work)
        assert q.info.table_bytes > 0 or q.info.n_q == 0


def test_general_plan_errors():
    spec = "ab,bc->ac"
    ok_u = ((1, -1), (0,), (2, 2), (4, 4))
    ok_v = ((1, -1), (0,), (2, 2), (4, 2))
    sc.Plan(spec, (8,), ok_u, ok_v)   # valid
    cases = [
        (((1, -1), (0,), (2, 2), (3, 4)), ok_v, (8,), 3),        # 3 does not divide 8
        (ok_u, ((1, -1), (0,), (2, 2), (2, 2)), (8,), 3),        # contracted b: 4 vs 2 sectors
        (((1, -1), (0,), (2, 2), (4, 4), ((1, 2, 2, 3), (2, 2, 2, 2))), ok_v, (8,), 3),  # 3 > D
        (((1, -1), (0, 0), (2, 2), (2, 6)), ((1, -1), (0, 0), (2, 2), (6, 6)), (2, 3), 5),   # product group
    ]
    for su, sv, mod, want in cases:
        with pytest.raises(sc.SymctrError) as ei:
            sc.Plan(spec, mod, su, sv)
        assert ei.value.status == want, (su, sv)


def test_chain_layouts_and_errors():
    """symctr_plan_chain: shapes of the aligned layouts, one chain per plan,
    sources that are not the operand, split free-U modes."""
    spec = lambda t: (t.signs, t.charge, t.dims)
    g = (WL.MPS_G,)
    p1 = sc.Plan(WL.MPS_STEP1, g, spec(WL.MPS_E), spec(WL.MPS_A), "split_bf16").chain(w_aligned=True)
    assert p1.shape_w == (8, 128, 2048) and p1.info.numel_w == 8 * 128 * 2048 and p1.info.chained
    p2 = sc.Plan(WL.MPS_STEP2, g, p1.sym_w, spec(WL.MPS_A), "split_bf16").chain(u_from=p1)
    assert p2.shape_u == (8, 128, 2048) and p2.info.numel_u == 8 * 128 * 2048
    with pytest.raises(sc.SymctrError) as ei:
        p2.chain(w_aligned=True)
    assert ei.value.status == 12
    other = sc.Plan(WL.MPS_STEP2, g, spec(WL.MPS_A), spec(WL.MPS_A), "split_bf16")
    with pytest.raises(sc.SymctrError) as ei:
        other.chain(u_from=sc.Plan("ab,bc->ac", g, ((1, -1), (0,), (128, 64)), ((1, -1), (0,), (64, 3))))
    assert ei.value.status == 3
    r1 = sc.Plan("ab,cd->abcd", (4,), ((1, -1), (0,), (2, 3)), ((1, -1), (0,), (2, 3)))
    r2 = sc.Plan("abcd,be->acde", (4,), r1.sym_w, ((-1, 1), (0,), (3, 2)))
    with pytest.raises(sc.SymctrError) as ei:
        r2.chain(u_from=r1)
    assert ei.value.status == 5


def test_spec_lengths_are_checked():
    """The binding refuses a symmetry spec whose length differs from its
    operand's order (the C ABI reads one entry per mode)."""
    with pytest.raises(ValueError):
        sc.Plan("ab,abc->c", (4,), ((1, -1), (0,), (2, 3)), ((1, -1), (0,), (2, 3)))
