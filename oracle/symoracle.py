"""Plain, slow CPU float64 oracle for cyclic-group-symmetric tensor contraction.

TEST INFRASTRUCTURE (see the package docstring): only tests/, the smoke
check and the benchmark's CPU-baseline legs use this module.  It imports
nothing from the CUDA path and the CUDA path imports nothing from it.

What the paper fixes, and how each route below follows it
----------------------------------------------------------
* A tensor with cyclic group symmetry is an order-2N "unfolded" tensor
  t[i1 I1, ..., iN IN] that vanishes unless sum_mu c_mu I_mu == Z (mod G)
  (Eq. ex1 and the unfolded rule of Sec. 1; general form Eq. symtsr).  In
  the general form mode mu has H_mu sectors (H_mu divides G) and coefficient
  c_mu = +-G/H_mu; Sym.sectors gives H_mu (default G, i.e. c_mu = +-1).
  Product groups keep H_mu = G on every mode.
* Block sizes: uniform per mode (D_mu), or non-uniform d_mu(q) <= D_mu per
  sector (Sym.sector_dims), held in blocks padded with zeros to D_mu (Sec. 1:
  non-uniform blocks are padded to a fixed size).  The dense tensor of a mode
  is compact: sector q occupies full indices off(q) .. off(q) + d(q) - 1,
  off(q) = sum_{q' < q} d(q'); with uniform blocks x = q*D + b.
  Padding entries of a reduced form are not part of the tensor: every route
  reads them as zero, and results hold zeros there.
* Its standard reduced form drops one sector index (Sec. 2.1 and its
  footnote; Eq. redform).  Reading used here: the LAST mode's sector is the
  implicit one, so the stored array has shape [H_0..H_{N-2}] + [D_0..D_{N-1}]
  ([G]*(N-1) + dims with c = +-1), and q_{N-1} solves
  c_{N-1} q_{N-1} == Z - sum_{mu<N-1} c_mu q_mu (mod G).  With a sub-group
  coefficient on the last mode some explicit sector tuples leave no
  solution: those entries of the reduced form are not part of the tensor
  either (read as zero, written as zero).
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
O5b aligned entries      : the reduced-form position of single entries of the
                           aligned forms (for sampled checks of large cases).
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
    "aligned_valid", "full_dims", "sanitize",
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

    def solve_coef(self, coef: int, sectors: int, coeffs, labels, z) -> Optional[int]:
        """Sector q in [0, sectors) with coef*q + sum coeffs*labels == z, where
        coef = +-G/sectors (Eq. symtsr), or None when no such q exists."""
        if abs(coef) == 1:
            return self.solve(coef, coeffs, labels, z)
        if len(self.moduli) != 1:
            raise ValueError("sub-group coefficients need a single cyclic factor")
        G = self.order
        step = G // sectors
        rest = self.charge(coeffs, labels)[0]
        r = ((1 if coef > 0 else -1) * (self.norm(z)[0] - rest)) % G
        return r // step if r % step == 0 else None


@dataclass(frozen=True)
class Sym:
    """Conservation law and block sizes of one tensor.
    signs       : +-1 per mode (the sign of c_mu).
    charge      : remainder Z, one entry per modulus.
    dims        : block size D_mu per mode (the padded size when sectors differ).
    sectors     : H_mu per mode (divides G; c_mu = sign * G / H_mu), or None
                  for H_mu = G on every mode.
    sector_dims : per mode, the true block size d_mu(q) <= D_mu of each of its
                  H_mu sectors, or None for uniform blocks."""
    signs: Tuple[int, ...]
    charge: Tuple[int, ...]
    dims: Tuple[int, ...]
    sectors: Optional[Tuple[int, ...]] = None
    sector_dims: Optional[Tuple[Tuple[int, ...], ...]] = None

    @property
    def order(self) -> int:
        return len(self.dims)

    @property
    def general(self) -> bool:
        return self.sectors is not None or self.sector_dims is not None

    def nsec(self, group: Group, mu: int) -> int:
        return group.order if self.sectors is None else int(self.sectors[mu])

    def coef(self, group: Group, mu: int) -> int:
        return int(self.signs[mu]) * (group.order // self.nsec(group, mu))

    def coefs(self, group: Group) -> Tuple[int, ...]:
        return tuple(self.coef(group, mu) for mu in range(self.order))

    def bdim(self, mu: int, q: int) -> int:
        """True block size of sector q of mode mu."""
        return int(self.dims[mu]) if self.sector_dims is None else int(self.sector_dims[mu][q])


def _sym_check(group: Group, sym: Sym):
    for mu in range(sym.order):
        h = sym.nsec(group, mu)
        if h < 1 or group.order % h:
            raise ValueError("sector counts must divide the group order")
        if h != group.order and len(group.moduli) != 1:
            raise ValueError("sub-group coefficients need a single cyclic factor")
        if sym.sector_dims is not None:
            if len(sym.sector_dims[mu]) != h or not all(0 <= d <= sym.dims[mu] for d in sym.sector_dims[mu]):
                raise ValueError("sector_dims: one size in [0, D] per sector")


def reduced_shape(group: Group, sym: Sym) -> Tuple[int, ...]:
    n = sym.order
    if n == 0:
        return ()
    return tuple([sym.nsec(group, mu) for mu in range(n - 1)] + list(sym.dims))


def full_dims(group: Group, sym: Sym) -> Tuple[int, ...]:
    """Dims of the dense (unfolded, compact) tensor: sum over sectors of d(q)."""
    return tuple(sum(sym.bdim(mu, q) for q in range(sym.nsec(group, mu))) for mu in range(sym.order))


def _offsets(group: Group, sym: Sym, mu: int) -> List[int]:
    off, acc = [], 0
    for q in range(sym.nsec(group, mu)):
        off.append(acc)
        acc += sym.bdim(mu, q)
    return off


def count_stored_blocks(group: Group, sym: Sym) -> Tuple[int, int]:
    """(#allowed blocks, #blocks of the dense tensor), by enumeration."""
    n = sym.order
    hs = [sym.nsec(group, mu) for mu in range(n)]
    allowed = sum(1 for qs in itertools.product(*[range(h) for h in hs])
                  if group.conserves(sym.coefs(group), qs, sym.charge))
    return allowed, int(np.prod(hs)) if hs else 1


# ---------------------------------------------------------------------------
# O1 / O2: reduced form <-> dense tensor (Eq. symtsr / Eq. redform)
# ---------------------------------------------------------------------------

def _block(group: Group, sym: Sym, qs, offs=None):
    """Slices of the dense tensor holding the block of sector tuple qs."""
    offs = offs or [_offsets(group, sym, mu) for mu in range(sym.order)]
    return tuple(slice(offs[mu][q], offs[mu][q] + sym.bdim(mu, q)) for mu, q in enumerate(qs))


def _valid(sym: Sym, qs):
    """Slices of a padded block that hold its true entries."""
    return tuple(slice(0, sym.bdim(mu, q)) for mu, q in enumerate(qs))


def _as_real_or_complex(a) -> np.ndarray:
    """float64, or complex128 for complex input (tensors may be complex, Sec. 1)."""
    a = np.asarray(a)
    return a.astype(np.complex128 if np.iscomplexobj(a) else np.float64, copy=False)


def _sectors(group: Group, sym: Sym):
    return itertools.product(*[range(sym.nsec(group, mu)) for mu in range(sym.order)])


def expand(group: Group, sym: Sym, red: np.ndarray) -> np.ndarray:
    """Dense tensor T: the block of every sector tuple (q_0..q_{N-1}) whose
    charge sum_mu c_mu q_mu == Z is red[q_0..q_{N-2}] cut to its true sizes,
    placed at the sectors' compact offsets; every other entry is 0."""
    red = _as_real_or_complex(red)
    _sym_check(group, sym)
    if red.shape != reduced_shape(group, sym):
        raise ValueError(f"reduced shape {red.shape} != {reduced_shape(group, sym)}")
    n = sym.order
    if n == 0:
        ok = group.conserves((), (), sym.charge)
        return red.copy() if ok else np.zeros((), dtype=red.dtype)
    dense = np.zeros(full_dims(group, sym), dtype=red.dtype)
    offs = [_offsets(group, sym, mu) for mu in range(n)]
    coefs = sym.coefs(group)
    for qs in _sectors(group, sym):
        if group.conserves(coefs, qs, sym.charge):
            dense[_block(group, sym, qs, offs)] = red[qs[:-1]][_valid(sym, qs)]
    return dense


def restrict(group: Group, sym: Sym, dense: np.ndarray) -> Tuple[np.ndarray, float]:
    """Inverse of expand (padding and the entries of sector tuples with no
    solution are 0).  Also returns max |entry| over forbidden blocks."""
    dense = _as_real_or_complex(dense)
    _sym_check(group, sym)
    n = sym.order
    if n == 0:
        ok = group.conserves((), (), sym.charge)
        return (dense.copy() if ok else np.zeros((), dtype=dense.dtype)), (0.0 if ok else float(abs(dense)))
    red = np.zeros(reduced_shape(group, sym), dtype=dense.dtype)
    worst = 0.0
    offs = [_offsets(group, sym, mu) for mu in range(n)]
    coefs = sym.coefs(group)
    for qs in _sectors(group, sym):
        blk = dense[_block(group, sym, qs, offs)]
        if group.conserves(coefs, qs, sym.charge):
            red[qs[:-1]][_valid(sym, qs)] = blk
        elif blk.size:
            worst = max(worst, float(np.max(np.abs(blk))))
    return red, worst


def sanitize(group: Group, sym: Sym, red) -> np.ndarray:
    """The reduced form with every entry that is not part of the tensor
    (padding, sector tuples without a solution) set to 0; the array itself
    when the tensor has neither."""
    red = _as_real_or_complex(red)
    if not sym.general:
        return red
    return restrict(group, sym, expand(group, sym, red))[0]


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

    def nsec(self, lab: str) -> int:
        """Sector count H of the mode labelled lab."""
        if lab in self.lu:
            return self.sym_u.nsec(self.group, self.lu.index(lab))
        return self.sym_v.nsec(self.group, self.lv.index(lab))


def plan(spec: str, group: Group, sym_u: Sym, sym_v: Sym) -> Plan:
    lu, lv, lw = parse_einsum(spec)
    if len(lu) != sym_u.order or len(lv) != sym_v.order:
        raise ValueError("operand order mismatch")
    _sym_check(group, sym_u)
    _sym_check(group, sym_v)
    C = [c for c in lu if c in lv]
    FU = [c for c in lu if c not in lv]
    FV = [c for c in lv if c not in lu]
    sig = None
    for c in C:
        i, j = lu.index(c), lv.index(c)
        if sym_u.dims[i] != sym_v.dims[j]:
            raise ValueError(f"dimension mismatch on contracted mode {c}")
        if sym_u.nsec(group, i) != sym_v.nsec(group, j):
            raise ValueError(f"sector count mismatch on contracted mode {c}")
        if [sym_u.bdim(i, q) for q in range(sym_u.nsec(group, i))] != \
                [sym_v.bdim(j, q) for q in range(sym_v.nsec(group, j))]:
            raise ValueError(f"sector size mismatch on contracted mode {c}")
        r = sym_u.signs[i] * sym_v.signs[j]
        if sig is None:
            sig = r
        elif sig != r:
            raise ValueError("contracted signs must agree up to one global sign")
    if sig is None:
        sig = -1
    signs_w, dims_w, sec_w, sd_w = [], [], [], []
    for c in lw:
        if c in FU:
            i = lu.index(c)
            signs_w.append(sym_u.signs[i])
            src, mu = sym_u, i
        else:
            j = lv.index(c)
            signs_w.append(-sig * sym_v.signs[j])
            src, mu = sym_v, j
        dims_w.append(src.dims[mu])
        sec_w.append(src.nsec(group, mu))
        sd_w.append(tuple(src.bdim(mu, q) for q in range(src.nsec(group, mu))))
    zw = group.norm([a - sig * b for a, b in zip(group.norm(sym_u.charge),
                                                  group.norm(sym_v.charge))])
    general = sym_u.general or sym_v.general
    sym_w = Sym(tuple(signs_w), zw, tuple(dims_w),
                tuple(sec_w) if general else None, tuple(sd_w) if general else None)
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
    full = dict(zip(p.lu, U.shape))
    full.update(zip(p.lv, V.shape))
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
    two blocks (numpy.tensordot) and accumulate into W's reduced form.  A
    sector equation without a solution (sub-group coefficients) skips the
    tuple; padded blocks take part with their padding read as zero."""
    G = p.group
    u_red = sanitize(G, p.sym_u, u_red)
    v_red = sanitize(G, p.sym_v, v_red)
    w_red = np.zeros(reduced_shape(G, p.sym_w), dtype=np.result_type(u_red, v_red))
    lw = p.lw
    wco = dict(zip(lw, p.sym_w.coefs(G)))
    uco = dict(zip(p.lu, p.sym_u.coefs(G)))
    vco = dict(zip(p.lv, p.sym_v.coefs(G)))
    explicit_w = list(lw[:-1])
    c_free = p.C[:-1]
    # contracted axes of the U and V blocks, in the order of p.C
    ax_u = [p.lu.index(c) for c in p.C]
    ax_v = [p.lv.index(c) for c in p.C]
    out_labels = [c for c in p.lu if c not in p.C] + [c for c in p.lv if c not in p.C]
    perm = [out_labels.index(c) for c in lw]
    for qw in itertools.product(*[range(p.nsec(c)) for c in explicit_w]):
        sec = dict(zip(explicit_w, qw))
        if lw:
            last = lw[-1]
            q = G.solve_coef(wco[last], p.nsec(last), [wco[c] for c in explicit_w], qw,
                             p.sym_w.charge)
            if q is None:
                continue
            sec[last] = q
        for qc in itertools.product(*[range(p.nsec(c)) for c in c_free]):
            sec.update(zip(c_free, qc))
            if p.C:
                cl = p.C[-1]
                known = [c for c in p.lu if c != cl]
                q = G.solve_coef(uco[cl], p.nsec(cl), [uco[c] for c in known],
                                 [sec[c] for c in known], p.sym_u.charge)
                if q is None:
                    continue
                sec[cl] = q
            else:
                # nothing contracted: both operand laws must hold separately
                if not G.conserves([uco[c] for c in p.lu], [sec[c] for c in p.lu],
                                   p.sym_u.charge):
                    continue
            if not G.conserves([vco[c] for c in p.lv], [sec[c] for c in p.lv],
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


def _w_sectors(p: Plan, w_index):
    """Sectors and block indices of W's entry w_index, or None when the entry
    is not part of W (no solution for the implicit sector, or padding)."""
    G = p.group
    lw = p.lw
    nw = len(lw)
    if nw == 0:
        return ({}, {}) if G.conserves((), (), p.sym_w.charge) else None
    wco = p.sym_w.coefs(G)
    sec = dict(zip(lw[:-1], w_index[:nw - 1]))
    blk = dict(zip(lw, w_index[nw - 1:]))
    q = G.solve_coef(wco[-1], p.nsec(lw[-1]), wco[:-1], [sec[c] for c in lw[:-1]],
                     p.sym_w.charge)
    if q is None:
        return None
    sec[lw[-1]] = q
    if any(blk[c] >= p.sym_w.bdim(i, sec[c]) for i, c in enumerate(lw)):
        return None
    return sec, blk


def _sym_of(p: Plan, lab: str) -> Tuple[Sym, int]:
    return (p.sym_u, p.lu.index(lab)) if lab in p.lu else (p.sym_v, p.lv.index(lab))


def contract_element(p: Plan, u_red, v_red, w_index: Tuple[int, ...]) -> float:
    """One entry of W's reduced form, straight from Eq. ctr: fix W's sectors
    and block indices, sum over every allowed contracted sector tuple and
    every contracted block index."""
    G = p.group
    found = _w_sectors(p, w_index)
    if found is None:
        return 0.0
    sec, blk = found
    u_red = sanitize(G, p.sym_u, u_red)
    v_red = sanitize(G, p.sym_v, v_red)
    uco, vco = p.sym_u.coefs(G), p.sym_v.coefs(G)
    total = 0.0
    for qc in itertools.product(*[range(p.nsec(c)) for c in p.C]):
        sec.update(zip(p.C, qc))
        if not G.conserves(uco, [sec[c] for c in p.lu], p.sym_u.charge):
            continue
        if not G.conserves(vco, [sec[c] for c in p.lv], p.sym_v.charge):
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
    found = _w_sectors(p, w_index)
    if found is None:
        return 0.0
    sec, blk = found
    uco, vco = p.sym_u.coefs(G), p.sym_v.coefs(G)
    cu = [c for c in p.lu if c in p.C]
    cv = [c for c in p.lv if c in p.C]
    total = 0.0
    for qc in itertools.product(*[range(p.nsec(c)) for c in p.C]):
        sec.update(zip(p.C, qc))
        if not G.conserves(uco, [sec[c] for c in p.lu], p.sym_u.charge):
            continue
        if not G.conserves(vco, [sec[c] for c in p.lv], p.sym_v.charge):
            continue
        # the contracted block indices run over the true sizes of their sectors
        cut = {c: slice(0, _sym_of(p, c)[0].bdim(_sym_of(p, c)[1], sec[c])) for c in p.C}
        ui = _red_index(sec, p.lu) + tuple(blk[c] if c in blk else cut[c] for c in p.lu)
        vi = _red_index(sec, p.lv) + tuple(blk[c] if c in blk else cut[c] for c in p.lv)
        us = np.asarray(u_get(ui), dtype=np.float64)
        vs = np.asarray(v_get(vi), dtype=np.float64)
        vs = np.transpose(vs, [cv.index(c) for c in cu]) if cv else vs
        total += float(np.sum(us * vs))
    return total


# ---------------------------------------------------------------------------
# O5: Algorithm 2 with dense generalized Kronecker deltas
# ---------------------------------------------------------------------------

def delta(group: Group, coeffs: Sequence[int], z: Sequence[int],
          extents: Optional[Sequence[int]] = None) -> np.ndarray:
    """Dense generalized Kronecker delta: 1 where sum coeffs*q == z, each q
    running over its extent (default G)."""
    n = len(coeffs)
    ext = [group.order] * n if extents is None else [int(e) for e in extents]
    d = np.zeros(ext, dtype=np.float64)
    for qs in itertools.product(*[range(e) for e in ext]):
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
    """(G, M, N, K) of the canonical aligned forms: per group of modes, the
    sector counts of all but its last mode times every block size."""
    G = p.group.order

    def size(mods):
        if not mods:
            return 1
        n = 1
        for c in mods[:-1]:
            n *= p.nsec(c)
        for c in mods:
            n *= p.dim(c)
        return n
    return G, size(p.FU), size(p.FV), size(p.C)


def _deltas(p: Plan):
    G = p.group
    zero = tuple(0 for _ in G.moduli)
    cu = dict(zip(p.lu, p.sym_u.coefs(G)))
    cv = dict(zip(p.lv, p.sym_v.coefs(G)))

    def ext(mods):
        return [p.nsec(c) for c in mods] + [G.order]
    d1 = delta(G, [cu[c] for c in p.FU] + [1], p.sym_u.charge, ext(p.FU))
    d2 = delta(G, [cu[c] for c in p.C] + [-1], zero, ext(p.C))
    d3 = delta(G, [cv[c] for c in p.FV] + [p.sigma], p.sym_v.charge, ext(p.FV))
    return d1, d2, d3


def _own_delta(p: Plan, sym: Sym, labels: str):
    G = p.group
    return delta(G, list(sym.coefs(G)), sym.charge, [p.nsec(c) for c in labels])


def _align(p: Plan, red, labels: str, sym: Sym, free: List[str], d_free, d2):
    """Aligned form [G, size(free), size(C)] of one operand via einsum with
    the operand's own delta and the two alignment deltas."""
    G = p.group
    L = _Letters()
    Q = L("Q")
    n = len(labels)
    own = _own_delta(p, sym, labels) if n else None
    red_sub = "".join(L("q" + c) for c in labels[:-1]) + "".join(L("b" + c) for c in labels)
    ops, subs = [sanitize(G, sym, np.asarray(red, dtype=np.float64))], [red_sub]
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
    # delta2 is written with U's contracted coefficients; V's law uses sigma
    # times those, so the same delta selects the same Q for V's contracted sectors.
    return _align(p, v_red, p.lv, p.sym_v, p.FV, d3, d2)


def mapback_w(p: Plan, w_hat) -> np.ndarray:
    """W's standard reduced form from W_hat[Q, m, n] (Alg. 2, output step)."""
    G = p.group
    d1, _, d3 = _deltas(p)
    L = _Letters()
    Q = L("Q")
    Gn, M, N, K = aligned_dims(p)
    shp = [Gn] + [p.nsec(c) for c in p.FU[:-1]] + [p.dim(c) for c in p.FU] \
        + [p.nsec(c) for c in p.FV[:-1]] + [p.dim(c) for c in p.FV]
    what = np.asarray(w_hat, dtype=np.float64).reshape(shp)
    w_sub = (Q + "".join(L("q" + c) for c in p.FU[:-1]) + "".join(L("b" + c) for c in p.FU)
             + "".join(L("q" + c) for c in p.FV[:-1]) + "".join(L("b" + c) for c in p.FV))
    ops = [what, d1, d3]
    subs = [w_sub, "".join(L("q" + c) for c in p.FU) + Q, "".join(L("q" + c) for c in p.FV) + Q]
    if p.lw:
        ops.append(_own_delta(p, p.sym_w, p.lw))
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
    ops = [sanitize(G, p.sym_w, np.asarray(w_red, dtype=np.float64))]
    subs = ["".join(L("q" + c) for c in p.lw[:-1]) + "".join(L("b" + c) for c in p.lw)]
    if p.lw:
        ops.append(_own_delta(p, p.sym_w, p.lw))
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
    {label: block}, valid), valid marking the indices whose equation has a
    solution and whose block digits lie inside their sectors' true sizes."""
    G = p.group
    n = len(labels)
    r = np.asarray(r, dtype=np.int64)
    if n == 0:
        # no modes: the equation reads 0 == target
        ok = all(int(np.mod(t, m)) == 0 for t, m in zip(target, G.moduli))
        return {}, {}, np.full(r.shape, ok, dtype=bool)
    shape = [p.nsec(c) for c in labels[:-1]] + [p.dim(c) for c in labels]
    digits = np.unravel_index(r, shape)
    sec = {c: digits[i] for i, c in enumerate(labels[:-1])}
    blk = {c: digits[n - 1 + i] for i, c in enumerate(labels)}
    rest = [0] * len(G.moduli)
    for c, k in zip(labels[:-1], coeffs[:-1]):
        for j, x in enumerate(_comps_arr(G, sec[c])):
            rest[j] = rest[j] + k * x
    last, h = coeffs[-1], p.nsec(labels[-1])
    valid = np.ones(r.shape, dtype=bool)
    if abs(last) == 1:   # its own inverse
        sec[labels[-1]] = _label_arr(G, [last * (t - x) for t, x in zip(target, rest)])
    else:                # last * q == t - rest with last = +-G/h: needs a multiple of G/h
        step = G.order // h
        rhs = np.mod((1 if last > 0 else -1) * (target[0] - rest[0]), G.order)
        valid = valid & (rhs % step == 0)
        sec[labels[-1]] = np.where(valid, rhs // step, 0)
    for c in labels:
        sym, mu = _sym_of(p, c)
        if sym.sector_dims is not None:
            sizes = np.asarray(sym.sector_dims[mu], dtype=np.int64)
            valid = valid & (blk[c] < sizes[sec[c]])
    return sec, blk, valid


def _aligned_entries(p: Plan, operand: int, Q: int, r, c):
    G = p.group
    cu = dict(zip(p.lu, p.sym_u.coefs(G)))
    cv = dict(zip(p.lv, p.sym_v.coefs(G)))
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
    sec, blk, ok_r = _group_digits(p, rl, rk, rt, r)
    s2, b2, ok_c = _group_digits(p, cl, ck, ct, c)
    sec.update(s2)
    blk.update(b2)
    full = np.zeros(r.shape, dtype=np.int64)
    idx = tuple(full + sec[x] for x in labels[:-1]) + tuple(full + blk[x] for x in labels)
    return idx, ok_r & ok_c


def aligned_index(p: Plan, operand: int, Q: int, r, c) -> Tuple[np.ndarray, ...]:
    """Reduced-form index of U_hat[Q, r, c] (operand 0: r = m over the free
    modes of U, c = kappa over the contracted ones), V_hat[Q, r, c] (1: r = n
    over the free modes of V, c = kappa) or W_hat[Q, r, c] (2: r = m, c = n),
    as a tuple of integer arrays broadcast over r and c.  The implicit
    sectors follow Alg. 2's three deltas: sum c^U_{F_U} q + Q == Z_U,
    sum c^U_C q == Q, sum c^V_{F_V} q + sigma Q == Z_V.  Entries that are not
    part of the tensor (aligned_valid is false) get an index inside the array."""
    return _aligned_entries(p, operand, Q, r, c)[0]


def aligned_valid(p: Plan, operand: int, Q: int, r, c) -> np.ndarray:
    """False where the aligned entry is absent: an implicit sector equation
    without a solution (sub-group coefficients) or a padding position."""
    return _aligned_entries(p, operand, Q, r, c)[1]


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
