"""Plain, slow CPU float64 oracle for cyclic-group-symmetric tensor contraction.

TEST INFRASTRUCTURE (see the package docstring): only tests/, the smoke
check and the benchmark's CPU-baseline legs use this module.  It imports
nothing from the CUDA path and the CUDA path imports nothing from it.

What the paper fixes, and how each route below follows it
----------------------------------------------------------
* A tensor with cyclic group symmetry is an order-2N "unfolded" tensor
  t[i1 I1, ..., iN IN] that vanishes unless sum_mu c_mu I_mu == Z (mod G)
  (Eq. ex1 and the unfolded rule of Sec. 1; general form Eq. symtsr, with
  coefficients c_mu = +-1 here).  The full index of a mode is x = q*D + b
  (q = sector / irrep label, b = index inside the block).
* Its standard reduced form drops one sector index (Sec. 2.1 and its
  footnote; Eq. redform).  Reading used here: the LAST mode's sector is the
  implicit one, so the stored array has shape [G]*(N-1) + [D_0..D_{N-1}],
  and q_{N-1} = c_{N-1} * (Z - sum_{mu<N-1} c_mu q_mu).
* Product groups Z_m1 x ... x Z_mr (Sec. 3): a label is a tuple, flattened
  mixed-radix with the first modulus most significant; all charge
  arithmetic is componentwise.
* Contraction (Eq. ctr): W = sum over the shared modes of U * V.

Routes
------
O1 expand / O2 restrict  : reduced form <-> dense tensor with zero blocks.
O3 dense brute force     : Eq. ctr on the dense tensors (pure-Python loops
                           for tiny cases, numpy.einsum otherwise).
O4 block loop            : Algorithm 1 generalised to any (s, t, v): loop
                           over the sectors of W's explicit modes and all
                           but one contracted mode, derive the other two
                           sectors by mod-G arithmetic, multiply blocks.
O5 aligned, dense deltas : Algorithm 2 with the transformations done, as
                           the paper's library does them, as einsum
                           contractions with dense generalized Kronecker
                           delta tensors (Sec. 3), the aligned contraction
                           as a batched matmul.
O6 gradients             : adjoint contractions, again by the block loop.
O7 finite differences    : central differences of a scalar loss (FP64).

Readings of points the paper leaves open:
* Q == sum_{k in C} c^U_k q_k (Alg. 2 coefficient vector c^(B) = [c^U_2; -1]
  with remainder 0); the three aligned deltas are
    delta1[F_U..., Q] : sum c^U_{F_U} q + Q         == Z_U
    delta2[C...,   Q] : sum c^U_C     q - Q         == 0
    delta3[F_V..., Q] : sum c^V_{F_V} q + sigma*Q   == Z_V
  where sigma = +-1 is the common ratio c^V_k / c^U_k over the contracted
  modes (Sec. 2.2 remark that the contracted coefficients may differ by a
  sign; sigma = -1 when nothing is contracted).
* Output law: c^W = (c^U_{F_U}, -sigma c^V_{F_V}), Z_W = Z_U - sigma Z_V.
* Canonical aligned layouts: U_hat[Q, m, kappa], V_hat[Q, n, kappa],
  W_hat[Q, m, n] with m = (q_{F_U[0..s-2]}, b_{F_U[0..s-1]}),
  kappa = (q_{C[0..v-2]}, b_{C[0..v-1]}), n = (q_{F_V[0..t-2]}, b_{F_V}),
  sector digits before block digits, C order, modes in operand order,
  all G values of Q present (zero where no entry exists).

Parity: every routine is pinned by tests/test_oracle_*.py.  The split and
TF32 precision forms of the CUDA path have no error bound in the paper;
they are compared with this oracle at stated tolerances ("parity unpinned
by the paper" for those tolerances).
"""
from __future__ import annotations

import itertools
import string
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "Group", "Sym", "Plan", "parse_einsum", "plan", "reduced_shape",
    "expand", "restrict", "contract_dense_einsum", "contract_dense_loops",
    "contract_blockloop", "contract_element", "contract_element_lazy", "align_u", "align_v",
    "mapback_w", "align_w", "q_set", "contract_aligned", "delta", "grad_u", "grad_v",
    "central_difference", "count_stored_blocks", "aligned_dims", "aligned_index",
]


# ---------------------------------------------------------------------------
# Group arithmetic
# ---------------------------------------------------------------------------

class Group:
    """Z_m1 x ... x Z_mr with labels flattened mixed-radix (first modulus
    most significant), e.g. Z_2 x Z_3: q = 3*q1 + q2."""

    def __init__(self, moduli: Sequence[int]):
        self.moduli = tuple(int(m) for m in moduli)
        if not self.moduli or any(m < 1 for m in self.moduli):
            raise ValueError("moduli must be positive")
        self.order = int(np.prod(self.moduli))

    def comps(self, q: int) -> Tuple[int, ...]:
        out = []
        for m in reversed(self.moduli):
            out.append(q % m)
            q //= m
        return tuple(reversed(out))

    def label(self, comps: Sequence[int]) -> int:
        q = 0
        for c, m in zip(comps, self.moduli):
            q = q * m + (int(c) % m)
        return q

    def norm(self, z: Sequence[int]) -> Tuple[int, ...]:
        return tuple(int(a) % m for a, m in zip(z, self.moduli))

    def charge(self, signs: Sequence[int], labels: Sequence[int]) -> Tuple[int, ...]:
        """sum_mu c_mu q_mu, componentwise mod m."""
        acc = [0] * len(self.moduli)
        for c, q in zip(signs, labels):
            for i, x in enumerate(self.comps(q)):
                acc[i] += c * x
        return self.norm(acc)

    def conserves(self, signs, labels, z) -> bool:
        return self.charge(signs, labels) == self.norm(z)

    def solve(self, sign: int, signs, labels, z) -> int:
        """Label q with sign*q + sum signs*labels == z (sign = +-1)."""
        rest = self.charge(signs, labels)
        comps = [sign * (a - b) for a, b in zip(self.norm(z), rest)]
        return self.label(comps)


@dataclass(frozen=True)
class Sym:
    """Conservation law and block sizes of one tensor."""
    signs: Tuple[int, ...]
    charge: Tuple[int, ...]
    dims: Tuple[int, ...]

    @property
    def order(self) -> int:
        return len(self.dims)


def reduced_shape(group: Group, sym: Sym) -> Tuple[int, ...]:
    n = sym.order
    if n == 0:
        return ()
    return tuple([group.order] * (n - 1) + list(sym.dims))


def count_stored_blocks(group: Group, sym: Sym) -> Tuple[int, int]:
    """(#allowed blocks, #blocks of the dense tensor), by enumeration."""
    n = sym.order
    allowed = sum(1 for qs in itertools.product(range(group.order), repeat=n)
                  if group.conserves(sym.signs, qs, sym.charge))
    return allowed, group.order ** n


# ---------------------------------------------------------------------------
# O1 / O2: reduced form <-> dense tensor (Eq. symtsr / Eq. redform)
# ---------------------------------------------------------------------------

def _block(qs, dims):
    return tuple(slice(q * d, (q + 1) * d) for q, d in zip(qs, dims))


def _as_real_or_complex(a) -> np.ndarray:
    """float64, or complex128 for complex input (tensors may be complex, Sec. 1)."""
    a = np.asarray(a)
    return a.astype(np.complex128 if np.iscomplexobj(a) else np.float64, copy=False)


def expand(group: Group, sym: Sym, red: np.ndarray) -> np.ndarray:
    """Dense tensor T[x] = red[q_0..q_{N-2}, b_0..b_{N-1}] if the sectors
    conserve charge, else 0, with q = x div D and b = x mod D."""
    red = _as_real_or_complex(red)
    if red.shape != reduced_shape(group, sym):
        raise ValueError(f"reduced shape {red.shape} != {reduced_shape(group, sym)}")
    n = sym.order
    if n == 0:
        ok = group.conserves((), (), sym.charge)
        return red.copy() if ok else np.zeros((), dtype=red.dtype)
    dense = np.zeros([group.order * d for d in sym.dims], dtype=red.dtype)
    for qs in itertools.product(range(group.order), repeat=n):
        if group.conserves(sym.signs, qs, sym.charge):
            dense[_block(qs, sym.dims)] = red[qs[:-1]]
    return dense


def restrict(group: Group, sym: Sym, dense: np.ndarray) -> Tuple[np.ndarray, float]:
    """Inverse of expand.  Also returns max |entry| over forbidden blocks."""
    dense = _as_real_or_complex(dense)
    n = sym.order
    if n == 0:
        ok = group.conserves((), (), sym.charge)
        return (dense.copy() if ok else np.zeros((), dtype=dense.dtype)), (0.0 if ok else float(abs(dense)))
    red = np.zeros(reduced_shape(group, sym), dtype=dense.dtype)
    worst = 0.0
    for qs in itertools.product(range(group.order), repeat=n):
        blk = dense[_block(qs, sym.dims)]
        if group.conserves(sym.signs, qs, sym.charge):
            red[qs[:-1]] = blk
        elif blk.size:
            worst = max(worst, float(np.max(np.abs(blk))))
    return red, worst


# ---------------------------------------------------------------------------
# Einsum parsing and the output law
# ---------------------------------------------------------------------------

def parse_einsum(spec: str) -> Tuple[str, str, str]:
    s = spec.replace(" ", "")
    if "->" not in s or s.count(",") != 1:
        raise ValueError("expected 'u,v->w'")
    lhs, lw = s.split("->")
    lu, lv = lhs.split(",")
    for lab in (lu, lv, lw):
        if len(set(lab)) != len(lab):
            raise ValueError("repeated label inside one operand")
        if any(ch not in string.ascii_letters for ch in lab):
            raise ValueError("labels must be letters")
    free = [c for c in lu if c not in lv] + [c for c in lv if c not in lu]
    if sorted(free) != sorted(lw):
        raise ValueError("output must list exactly the free labels")
    return lu, lv, lw


@dataclass
class Plan:
    lu: str
    lv: str
    lw: str
    FU: List[str]
    C: List[str]
    FV: List[str]
    sigma: int
    sym_u: Sym
    sym_v: Sym
    sym_w: Sym
    group: Group

    @property
    def s(self): return len(self.FU)

    @property
    def t(self): return len(self.FV)

    @property
    def v(self): return len(self.C)

    def dim(self, lab: str) -> int:
        if lab in self.lu:
            return self.sym_u.dims[self.lu.index(lab)]
        return self.sym_v.dims[self.lv.index(lab)]


def plan(spec: str, group: Group, sym_u: Sym, sym_v: Sym) -> Plan:
    lu, lv, lw = parse_einsum(spec)
    if len(lu) != sym_u.order or len(lv) != sym_v.order:
        raise ValueError("operand order mismatch")
    C = [c for c in lu if c in lv]
    FU = [c for c in lu if c not in lv]
    FV = [c for c in lv if c not in lu]
    sig = None
    for c in C:
        cu, cv = sym_u.signs[lu.index(c)], sym_v.signs[lv.index(c)]
        if sym_u.dims[lu.index(c)] != sym_v.dims[lv.index(c)]:
            raise ValueError(f"dimension mismatch on contracted mode {c}")
        r = cu * cv
        if sig is None:
            sig = r
        elif sig != r:
            raise ValueError("contracted signs must agree up to one global sign")
    if sig is None:
        sig = -1
    signs_w, dims_w = [], []
    for c in lw:
        if c in FU:
            signs_w.append(sym_u.signs[lu.index(c)])
            dims_w.append(sym_u.dims[lu.index(c)])
        else:
            signs_w.append(-sig * sym_v.signs[lv.index(c)])
            dims_w.append(sym_v.dims[lv.index(c)])
    zw = group.norm([a - sig * b for a, b in zip(group.norm(sym_u.charge),
                                                  group.norm(sym_v.charge))])
    sym_w = Sym(tuple(signs_w), zw, tuple(dims_w))
    return Plan(lu, lv, lw, FU, C, FV, sig, sym_u, sym_v, sym_w, group)


# ---------------------------------------------------------------------------
# O3: dense brute force (Eq. ctr)
# ---------------------------------------------------------------------------

def contract_dense_einsum(p: Plan, u_red, v_red) -> Tuple[np.ndarray, float]:
    """Expand, contract densely with numpy.einsum, restrict.  Returns the
    output reduced form and the max |entry| in W's forbidden blocks."""
    U = expand(p.group, p.sym_u, u_red)
    V = expand(p.group, p.sym_v, v_red)
    W = np.einsum(f"{p.lu},{p.lv}->{p.lw}", U, V)
    return restrict(p.group, p.sym_w, W)


def contract_dense_loops(p: Plan, u_red, v_red) -> np.ndarray:
    """Eq. ctr as explicit Python loops over every full index (tiny only).
    Returns the dense output tensor."""
    U = expand(p.group, p.sym_u, u_red)
    V = expand(p.group, p.sym_v, v_red)
    G = p.group.order
    full = {c: G * p.dim(c) for c in set(p.lu + p.lv)}
    W = np.zeros([full[c] for c in p.lw], dtype=np.float64)
    for widx in itertools.product(*[range(full[c]) for c in p.lw]):
        env = dict(zip(p.lw, widx))
        acc = 0.0
        for cidx in itertools.product(*[range(full[c]) for c in p.C]):
            env.update(zip(p.C, cidx))
            acc += U[tuple(env[c] for c in p.lu)] * V[tuple(env[c] for c in p.lv)]
        W[widx] = acc
    return W


# ---------------------------------------------------------------------------
# O4: loop over symmetry blocks (Algorithm 1, generalised)
# ---------------------------------------------------------------------------

def _red_index(sectors: Dict[str, int], labels: str):
    """Sector part of a reduced-form index: all modes but the last."""
    return tuple(sectors[c] for c in labels[:-1])


def contract_blockloop(p: Plan, u_red, v_red, counter: Optional[list] = None) -> np.ndarray:
    """Loop over the sectors of W's explicit modes and of all contracted
    modes but the last; derive the last contracted sector from U's law and
    W's implicit sector from W's law (Algorithm 1 for s=t=v=2); multiply the
    two blocks (numpy.tensordot) and accumulate into W's reduced form."""
    G = p.group
    u_red = _as_real_or_complex(u_red)
    v_red = _as_real_or_complex(v_red)
    w_red = np.zeros(reduced_shape(G, p.sym_w), dtype=np.result_type(u_red, v_red))
    lw = p.lw
    wsig = dict(zip(lw, p.sym_w.signs))
    usig = dict(zip(p.lu, p.sym_u.signs))
    vsig = dict(zip(p.lv, p.sym_v.signs))
    explicit_w = list(lw[:-1])
    c_free = p.C[:-1]
    # contracted axes of the U and V blocks, in the order of p.C
    ax_u = [p.lu.index(c) for c in p.C]
    ax_v = [p.lv.index(c) for c in p.C]
    out_labels = [c for c in p.lu if c not in p.C] + [c for c in p.lv if c not in p.C]
    perm = [out_labels.index(c) for c in lw]
    for qw in itertools.product(range(G.order), repeat=len(explicit_w)):
        sec = dict(zip(explicit_w, qw))
        if lw:
            last = lw[-1]
            sec[last] = G.solve(wsig[last], [wsig[c] for c in explicit_w], qw,
                                p.sym_w.charge)
        for qc in itertools.product(range(G.order), repeat=len(c_free)):
            sec.update(zip(c_free, qc))
            if p.C:
                cl = p.C[-1]
                known = [c for c in p.lu if c != cl]
                sec[cl] = G.solve(usig[cl], [usig[c] for c in known],
                                  [sec[c] for c in known], p.sym_u.charge)
            else:
                # nothing contracted: both operand laws must hold separately
                if not G.conserves([usig[c] for c in p.lu], [sec[c] for c in p.lu],
                                   p.sym_u.charge):
                    continue
            if not G.conserves([vsig[c] for c in p.lv], [sec[c] for c in p.lv],
                               p.sym_v.charge):
                continue
            ub = u_red[_red_index(sec, p.lu)] if p.lu else u_red
            vb = v_red[_red_index(sec, p.lv)] if p.lv else v_red
            blk = np.tensordot(ub, vb, axes=(ax_u, ax_v))
            if perm:
                blk = np.transpose(blk, perm)
            if lw:
                w_red[_red_index(sec, lw)] += blk
            else:
                w_red += blk
            if counter is not None:
                counter[0] += 1
    if not lw and not G.conserves((), (), p.sym_w.charge):
        w_red[...] = 0.0
    return w_red


def contract_element(p: Plan, u_red, v_red, w_index: Tuple[int, ...]) -> float:
    """One entry of W's reduced form, straight from Eq. ctr: fix W's sectors
    and block indices, sum over every allowed contracted sector tuple and
    every contracted block index."""
    G = p.group
    lw = p.lw
    nw = len(lw)
    wsig = dict(zip(lw, p.sym_w.signs))
    usig = dict(zip(p.lu, p.sym_u.signs))
    vsig = dict(zip(p.lv, p.sym_v.signs))
    if nw == 0:
        if not G.conserves((), (), p.sym_w.charge):
            return 0.0
        sec, blk = {}, {}
    else:
        sec = dict(zip(lw[:-1], w_index[:nw - 1]))
        blk = dict(zip(lw, w_index[nw - 1:]))
        sec[lw[-1]] = G.solve(wsig[lw[-1]], [wsig[c] for c in lw[:-1]],
                              [sec[c] for c in lw[:-1]], p.sym_w.charge)
    total = 0.0
    for qc in itertools.product(range(G.order), repeat=len(p.C)):
        sec.update(zip(p.C, qc))
        if not G.conserves([usig[c] for c in p.lu], [sec[c] for c in p.lu], p.sym_u.charge):
            continue
        if not G.conserves([vsig[c] for c in p.lv], [sec[c] for c in p.lv], p.sym_v.charge):
            continue
        ub = np.asarray(u_red)[_red_index(sec, p.lu)] if p.lu else np.asarray(u_red)
        vb = np.asarray(v_red)[_red_index(sec, p.lv)] if p.lv else np.asarray(v_red)
        # fix the free block indices, keep the contracted ones (ordered as p.C)
        ui = tuple(blk[c] if c in blk else slice(None) for c in p.lu)
        vi = tuple(blk[c] if c in blk else slice(None) for c in p.lv)
        us, vs = ub[ui], vb[vi]
        cu = [c for c in p.lu if c in p.C]
        cv = [c for c in p.lv if c in p.C]
        vs = np.transpose(vs, [cv.index(c) for c in cu]) if cv else vs
        total += float(np.sum(us * vs))
    return total


def contract_element_lazy(p: Plan, u_get, v_get, w_index: Tuple[int, ...]) -> float:
    """contract_element for operands too large to hold on the host: the same
    sum (Eq. ctr, over every allowed contracted sector tuple and contracted
    block index), with the operands read through callbacks.
    u_get(index) / v_get(index) return the reduced-form sub-array at `index`,
    a tuple of ints and full slices in the reduced form's axis order."""
    G = p.group
    lw = p.lw
    nw = len(lw)
    wsig = dict(zip(lw, p.sym_w.signs))
    usig = dict(zip(p.lu, p.sym_u.signs))
    vsig = dict(zip(p.lv, p.sym_v.signs))
    if nw == 0:
        if not G.conserves((), (), p.sym_w.charge):
            return 0.0
        sec, blk = {}, {}
    else:
        sec = dict(zip(lw[:-1], w_index[:nw - 1]))
        blk = dict(zip(lw, w_index[nw - 1:]))
        sec[lw[-1]] = G.solve(wsig[lw[-1]], [wsig[c] for c in lw[:-1]],
                              [sec[c] for c in lw[:-1]], p.sym_w.charge)
    cu = [c for c in p.lu if c in p.C]
    cv = [c for c in p.lv if c in p.C]
    total = 0.0
    for qc in itertools.product(range(G.order), repeat=len(p.C)):
        sec.update(zip(p.C, qc))
        if not G.conserves([usig[c] for c in p.lu], [sec[c] for c in p.lu], p.sym_u.charge):
            continue
        if not G.conserves([vsig[c] for c in p.lv], [sec[c] for c in p.lv], p.sym_v.charge):
            continue
        ui = _red_index(sec, p.lu) + tuple(blk[c] if c in blk else slice(None) for c in p.lu)
        vi = _red_index(sec, p.lv) + tuple(blk[c] if c in blk else slice(None) for c in p.lv)
        us = np.asarray(u_get(ui), dtype=np.float64)
        vs = np.asarray(v_get(vi), dtype=np.float64)
        vs = np.transpose(vs, [cv.index(c) for c in cu]) if cv else vs
        total += float(np.sum(us * vs))
    return total


# ---------------------------------------------------------------------------
# O5: Algorithm 2 with dense generalized Kronecker deltas
# ---------------------------------------------------------------------------

def delta(group: Group, coeffs: Sequence[int], z: Sequence[int]) -> np.ndarray:
    """Dense generalized Kronecker delta: 1 where sum coeffs*q == z."""
    n = len(coeffs)
    d = np.zeros([group.order] * n, dtype=np.float64)
    for qs in itertools.product(range(group.order), repeat=n):
        if group.conserves(coeffs, qs, z):
            d[qs] = 1.0
    return d


class _Letters:
    def __init__(self):
        self.pool = iter(string.ascii_letters)
        self.map: Dict[str, str] = {}

    def __call__(self, key: str) -> str:
        if key not in self.map:
            self.map[key] = next(self.pool)
        return self.map[key]


def aligned_dims(p: Plan) -> Tuple[int, int, int, int]:
    """(G, M, N, K) of the canonical aligned forms."""
    G = p.group.order

    def size(mods):
        if not mods:
            return 1
        n = G ** (len(mods) - 1)
        for c in mods:
            n *= p.dim(c)
        return n
    return G, size(p.FU), size(p.FV), size(p.C)


def _deltas(p: Plan):
    G = p.group
    zero = tuple(0 for _ in G.moduli)
    cu = dict(zip(p.lu, p.sym_u.signs))
    cv = dict(zip(p.lv, p.sym_v.signs))
    d1 = delta(G, [cu[c] for c in p.FU] + [1], p.sym_u.charge)
    d2 = delta(G, [cu[c] for c in p.C] + [-1], zero)
    d3 = delta(G, [cv[c] for c in p.FV] + [p.sigma], p.sym_v.charge)
    return d1, d2, d3


def _align(p: Plan, red, labels: str, sym: Sym, free: List[str], d_free, d2):
    """Aligned form [G, size(free), size(C)] of one operand via einsum with
    the operand's own delta and the two alignment deltas."""
    G = p.group
    L = _Letters()
    Q = L("Q")
    n = len(labels)
    own = delta(G, list(sym.signs), sym.charge) if n else None
    red_sub = "".join(L("q" + c) for c in labels[:-1]) + "".join(L("b" + c) for c in labels)
    ops, subs = [np.asarray(red, dtype=np.float64)], [red_sub]
    if n:
        ops.append(own)
        subs.append("".join(L("q" + c) for c in labels))
    ops.append(d_free)
    subs.append("".join(L("q" + c) for c in free) + Q)
    ops.append(d2)
    subs.append("".join(L("q" + c) for c in p.C) + Q)
    out = (Q + "".join(L("q" + c) for c in free[:-1]) + "".join(L("b" + c) for c in free)
           + "".join(L("q" + c) for c in p.C[:-1]) + "".join(L("b" + c) for c in p.C))
    res = np.einsum(",".join(subs) + "->" + out, *ops, optimize=True)
    Gn, M, N, K = aligned_dims(p)
    rows = M if free is p.FU else N
    return np.ascontiguousarray(res.reshape(Gn, rows, K))


def align_u(p: Plan, u_red) -> np.ndarray:
    """U_hat[Q, m, kappa] (Alg. 2, input transformation of U)."""
    d1, d2, _ = _deltas(p)
    return _align(p, u_red, p.lu, p.sym_u, p.FU, d1, d2)


def align_v(p: Plan, v_red) -> np.ndarray:
    """V_hat[Q, n, kappa] (Alg. 2, input transformation of V), kappa-major rows."""
    _, d2, d3 = _deltas(p)
    # delta2 is written with U's contracted signs; V's law uses sigma * those,
    # so the same delta selects the same Q for V's contracted sectors.
    return _align(p, v_red, p.lv, p.sym_v, p.FV, d3, d2)


def mapback_w(p: Plan, w_hat) -> np.ndarray:
    """W's standard reduced form from W_hat[Q, m, n] (Alg. 2, output step)."""
    G = p.group
    d1, _, d3 = _deltas(p)
    L = _Letters()
    Q = L("Q")
    Gn, M, N, K = aligned_dims(p)
    shp = [Gn] + [Gn] * max(p.s - 1, 0) + [p.dim(c) for c in p.FU] \
        + [Gn] * max(p.t - 1, 0) + [p.dim(c) for c in p.FV]
    what = np.asarray(w_hat, dtype=np.float64).reshape(shp)
    w_sub = (Q + "".join(L("q" + c) for c in p.FU[:-1]) + "".join(L("b" + c) for c in p.FU)
             + "".join(L("q" + c) for c in p.FV[:-1]) + "".join(L("b" + c) for c in p.FV))
    ops = [what, d1, d3]
    subs = [w_sub, "".join(L("q" + c) for c in p.FU) + Q, "".join(L("q" + c) for c in p.FV) + Q]
    if p.lw:
        ops.append(delta(G, list(p.sym_w.signs), p.sym_w.charge))
        subs.append("".join(L("q" + c) for c in p.lw))
    out = "".join(L("q" + c) for c in p.lw[:-1]) + "".join(L("b" + c) for c in p.lw)
    res = np.einsum(",".join(subs) + "->" + out, *ops, optimize=True)
    if not p.lw and not G.conserves((), (), p.sym_w.charge):
        res = np.zeros(())
    return np.array(res, dtype=np.float64, order="C")


def align_w(p: Plan, w_red) -> np.ndarray:
    """W_hat[Q, m, n] from W's standard reduced form (inverse of mapback_w;
    the input transformation a gradient dL/dW goes through)."""
    G = p.group
    d1, _, d3 = _deltas(p)
    L = _Letters()
    Q = L("Q")
    ops = [np.asarray(w_red, dtype=np.float64)]
    subs = ["".join(L("q" + c) for c in p.lw[:-1]) + "".join(L("b" + c) for c in p.lw)]
    if p.lw:
        ops.append(delta(G, list(p.sym_w.signs), p.sym_w.charge))
        subs.append("".join(L("q" + c) for c in p.lw))
    ops += [d1, d3]
    subs += ["".join(L("q" + c) for c in p.FU) + Q, "".join(L("q" + c) for c in p.FV) + Q]
    out = (Q + "".join(L("q" + c) for c in p.FU[:-1]) + "".join(L("b" + c) for c in p.FU)
           + "".join(L("q" + c) for c in p.FV[:-1]) + "".join(L("b" + c) for c in p.FV))
    res = np.einsum(",".join(subs) + "->" + out, *ops, optimize=True)
    Gn, M, N, K = aligned_dims(p)
    return np.ascontiguousarray(res.reshape(Gn, M, N))


def q_set(p: Plan) -> List[int]:
    """Labels Q for which the aligned forms can hold nonzero entries: those
    where delta1, delta2 and delta3 can all be satisfied."""
    d1, d2, d3 = _deltas(p)
    out = []
    for q in range(p.group.order):
        if d1[..., q].any() and d2[..., q].any() and d3[..., q].any():
            out.append(q)
    return out


def contract_aligned(p: Plan, u_red, v_red) -> np.ndarray:
    """Algorithm 2: align both operands, batched matmul over Q, map back."""
    uh = align_u(p, u_red)
    vh = align_v(p, v_red)
    wh = np.matmul(uh, np.transpose(vh, (0, 2, 1)))
    return mapback_w(p, wh)


# ---------------------------------------------------------------------------
# O5b: the reduced-form position of single aligned entries (the App. A.4
# layouts of Alg. 2's aligned forms, evaluated entry by entry), for checks
# that sample a few rows and columns of an aligned problem too large to form
# ---------------------------------------------------------------------------

def _comps_arr(group: Group, q):
    """Components of (arrays of) flattened labels, first modulus first."""
    q = np.asarray(q, dtype=np.int64)
    out = []
    for m in reversed(group.moduli):
        out.append(q % m)
        q = q // m
    return list(reversed(out))


def _label_arr(group: Group, comps):
    q = np.zeros(np.broadcast(*comps).shape if len(comps) > 1 else np.shape(comps[0]), dtype=np.int64)
    for c, m in zip(comps, group.moduli):
        q = q * m + np.mod(c, m)
    return q


def _group_digits(p: Plan, labels: List[str], coeffs: List[int], target, r):
    """Sector and block digits of aligned index r over the modes `labels`
    (sector digits of all but the last mode, then every block digit, C
    order); the last mode's sector solves sum coeffs * q == target, where
    target is a list of component arrays.  Returns ({label: sector},
    {label: block})."""
    G = p.group
    n = len(labels)
    if n == 0:
        return {}, {}
    shape = [G.order] * (n - 1) + [p.dim(c) for c in labels]
    digits = np.unravel_index(np.asarray(r, dtype=np.int64), shape)
    sec = {c: digits[i] for i, c in enumerate(labels[:-1])}
    blk = {c: digits[n - 1 + i] for i, c in enumerate(labels)}
    rest = [0] * len(G.moduli)
    for c, k in zip(labels[:-1], coeffs[:-1]):
        for j, x in enumerate(_comps_arr(G, sec[c])):
            rest[j] = rest[j] + k * x
    last = coeffs[-1]   # +-1: its own inverse
    sec[labels[-1]] = _label_arr(G, [last * (t - x) for t, x in zip(target, rest)])
    return sec, blk


def aligned_index(p: Plan, operand: int, Q: int, r, c) -> Tuple[np.ndarray, ...]:
    """Reduced-form index of U_hat[Q, r, c] (operand 0: r = m over the free
    modes of U, c = kappa over the contracted ones), V_hat[Q, r, c] (1: r = n
    over the free modes of V, c = kappa) or W_hat[Q, r, c] (2: r = m, c = n),
    as a tuple of integer arrays broadcast over r and c.  The implicit
    sectors follow Alg. 2's three deltas: sum c^U_{F_U} q + Q == Z_U,
    sum c^U_C q == Q, sum c^V_{F_V} q + sigma Q == Z_V."""
    G = p.group
    cu = dict(zip(p.lu, p.sym_u.signs))
    cv = dict(zip(p.lv, p.sym_v.signs))
    qc = _comps_arr(G, Q)
    zu = [np.int64(z) for z in G.norm(p.sym_u.charge)]
    zv = [np.int64(z) for z in G.norm(p.sym_v.charge)]
    t_fu = [a - b for a, b in zip(zu, qc)]
    t_c = qc
    t_fv = [a - p.sigma * b for a, b in zip(zv, qc)]
    groups = {0: ((p.FU, [cu[x] for x in p.FU], t_fu), (p.C, [cu[x] for x in p.C], t_c), p.lu),
              1: ((p.FV, [cv[x] for x in p.FV], t_fv), (p.C, [cu[x] for x in p.C], t_c), p.lv),
              2: ((p.FU, [cu[x] for x in p.FU], t_fu), (p.FV, [cv[x] for x in p.FV], t_fv), p.lw)}
    (rl, rk, rt), (cl, ck, ct), labels = groups[operand]
    r, c = np.broadcast_arrays(np.asarray(r, dtype=np.int64), np.asarray(c, dtype=np.int64))
    sec, blk = _group_digits(p, rl, rk, rt, r)
    s2, b2 = _group_digits(p, cl, ck, ct, c)
    sec.update(s2)
    blk.update(b2)
    full = np.zeros(r.shape, dtype=np.int64)
    return tuple(full + sec[x] for x in labels[:-1]) + tuple(full + blk[x] for x in labels)


# ---------------------------------------------------------------------------
# O6 / O7: gradients and finite differences
# ---------------------------------------------------------------------------

def _sub_plan(spec: str, group: Group, sym_a: Sym, sym_b: Sym) -> Plan:
    return plan(spec, group, sym_a, sym_b)


def grad_u(p: Plan, gw_red, v_red) -> np.ndarray:
    """dL/dU for L = <W, gW>: gU = einsum(lw,lv->lu)(gW, V), block loop."""
    q = _sub_plan(f"{p.lw},{p.lv}->{p.lu}", p.group, p.sym_w, p.sym_v)
    return contract_blockloop(q, gw_red, v_red)


def grad_v(p: Plan, u_red, gw_red) -> np.ndarray:
    """dL/dV for L = <W, gW>: gV = einsum(lu,lw->lv)(U, gW), block loop."""
    q = _sub_plan(f"{p.lu},{p.lw}->{p.lv}", p.group, p.sym_u, p.sym_w)
    return contract_blockloop(q, u_red, gw_red)


def central_difference(f, x: np.ndarray, direction: np.ndarray, h: float = 1e-6) -> float:
    """(f(x + h d) - f(x - h d)) / (2h), all in float64."""
    return (f(x + h * direction) - f(x - h * direction)) / (2.0 * h)
