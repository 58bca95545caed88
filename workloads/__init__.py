"""Seeded synthetic inputs for the irrep-aligned contraction workloads.

This module is shared by the CPU oracle's tests, the GPU tests and the
benchmark.  It holds workload *definitions* (einsum strings, charge signs,
group moduli, sector dimensions, value distributions, seeds) and draws
random reduced-form arrays from them.  It performs none of the method's
arithmetic: no charge conservation, no alignment, no contraction.

A standard reduced form of an order-N tensor over a group of order G with
sector dimensions D_0..D_{N-1} is stored as a C-contiguous float64 array of
shape [G]*(N-1) + [D_0, ..., D_{N-1}] (the sector of the last mode is the
implicit one; Sec. 2.1 footnote on reduced forms, and the API listing of
Sec. 3 whose data has shape [G,G,G,N,N,N,N]).  Every stored entry is an
allowed entry, so an i.i.d. draw over the whole array is a random symmetric
tensor.

Seeds follow "workload k, tensor j -> seed 1000*k + j".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np


def group_order(moduli: Sequence[int]) -> int:
    g = 1
    for m in moduli:
        g *= int(m)
    return g


def reduced_shape(moduli: Sequence[int], dims: Sequence[int]) -> Tuple[int, ...]:
    """Shape of the standard reduced form: [G]*(N-1) + dims (N = len(dims))."""
    n = len(dims)
    g = group_order(moduli)
    if n == 0:
        return ()
    return tuple([g] * (n - 1) + [int(d) for d in dims])


@dataclass(frozen=True)
class TensorSpec:
    """Symmetry and value recipe of one operand."""
    signs: Tuple[int, ...]          # +1 / -1 per mode
    charge: Tuple[int, ...]         # target charge, one entry per modulus
    dims: Tuple[int, ...]           # sector (block) dimension per mode
    scale: float = 1.0              # entries ~ N(0,1) * scale
    seed: int = 0
    positive: bool = False          # entries ~ U[0,1) * scale instead


@dataclass(frozen=True)
class Contraction:
    """One contraction W = einsum(spec, U, V) of cyclic-group tensors."""
    name: str
    einsum: str
    moduli: Tuple[int, ...]
    u: TensorSpec
    v: TensorSpec


def draw(spec: TensorSpec, moduli: Sequence[int], seed: Optional[int] = None) -> np.ndarray:
    """Draw the reduced-form array of one operand (float64, C order)."""
    rng = np.random.default_rng(spec.seed if seed is None else seed)
    shape = reduced_shape(moduli, spec.dims)
    if spec.positive:
        a = rng.random(size=shape)
    else:
        a = rng.standard_normal(size=shape)
    if spec.scale != 1.0:
        a = a * spec.scale
    return np.ascontiguousarray(a, dtype=np.float64)


def draw_pair(c: Contraction) -> Tuple[np.ndarray, np.ndarray]:
    return draw(c.u, c.moduli), draw(c.v, c.moduli)


def direction(moduli: Sequence[int], dims: Sequence[int], seed: int) -> np.ndarray:
    """A random full direction (N(0,1) on every stored entry) for finite differences."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=reduced_shape(moduli, dims))


# ---------------------------------------------------------------------------
# Workload definitions (shapes and distributions of the paper's examples).
# ---------------------------------------------------------------------------

PP = (1, 1, -1, -1)

# Order-4 Z_3 example of Sec. 2.1 / the API listing: w_abij = sum_kl u_abkl v_klij.
Z3_ORDER4 = Contraction(
    name="z3_order4_G3_D4",
    einsum="abkl,klij->abij",
    moduli=(3,),
    u=TensorSpec(PP, (0,), (4, 4, 4, 4), 1.0, 1001),
    v=TensorSpec(PP, (0,), (4, 4, 4, 4), 1.0, 1002),
)

# MPS transfer step, Z_8: E'[g,d] = sum_{a,b,s} E[a,b] A[a,s,g] A[b,s,d],
# evaluated as two contractions X = E.A and E' = X.A.
MPS_G = 8
MPS_E = TensorSpec((1, -1), (0,), (128, 128), 1.0, 2001)
MPS_A = TensorSpec((1, 1, -1), (0,), (128, 2, 128), 1.0, 2002)
MPS_STEP1 = "ab,asg->bsg"
MPS_STEP2 = "bsg,bsd->gd"

# Coupled-cluster particle-particle ladder, Z_8 (Sec. 4.1, Table 1 CC-type).
def cc_ladder(G: int = 8, virt: int = 256, occ: int = 64) -> Contraction:
    dv, do = virt // G, occ // G
    return Contraction(
        name=f"cc_ladder_G{G}_V{virt}_O{occ}",
        einsum="abcd,cdij->abij",
        moduli=(G,),
        u=TensorSpec(PP, (0,), (dv, dv, dv, dv), 1.0 / math.sqrt(virt), 3001),
        v=TensorSpec(PP, (0,), (dv, dv, do, do), 1e-2, 3002),
    )

CC_LADDER = cc_ladder()

# PEPS-style differentiation workload under Z_2 x Z_3 (6 irreps per mode):
# y[p] = sum_{uldr} T[u,l,d,r,p] Env[u,l,d,r]; loss = sum_p y_p^2.
PEPS_MODULI = (2, 3)
PEPS_KLIVE = 6 ** 3 * 16 ** 4
PEPS_T = TensorSpec((1, 1, -1, -1, 1), (0, 0), (16, 16, 16, 16, 2), 1.0, 4001)
PEPS_ENV = TensorSpec((-1, -1, 1, 1), (0, 0), (16, 16, 16, 16),
                      1.0 / math.sqrt(PEPS_KLIVE), 4002)
PEPS_Y = "uldrp,uldr->p"
PEPS_LOSS = "p,p->"

# Scaling sweep of the CC ladder at virtual 512 / occupied 128.
SWEEP_GS = (2, 4, 8, 16)


def sweep_point(G: int) -> Contraction:
    return cc_ladder(G, 512, 128)


# The contraction families of Table 1 at the tensor dimensions of Table 2
# (per-mode sector dims; Table 1 gives no charge signs, these are the ones the
# parity suite uses).  Entries N(0,1) scaled by 1/sqrt(contracted length).
def _t2(label, einsum, G, su, du, sv, dv, k):
    import math as _m
    contracted = [ch for ch in einsum.split("->")[0].split(",")[0] if ch in einsum.split(",")[1].split("->")[0]]
    klen = 1
    lab_u = einsum.split(",")[0]
    for ch in contracted:
        klen *= G * du[lab_u.index(ch)]
    sc = 1.0 / _m.sqrt(klen)
    return Contraction(label, einsum, (G,), TensorSpec(su, (0,), du, sc, 8000 + 2 * k),
                       TensorSpec(sv, (0,), dv, sc, 8001 + 2 * k))


TABLE2 = {c.name: c for c in [
    _t2("CC1_a", "ijkl,mnkl->ijmn", 8, PP, (32, 32, 32, 32), PP, (16, 16, 32, 32), 0),
    _t2("CC2_a", "opij,opkm->ijmk", 8, PP, (16, 16, 32, 32), (-1, -1, 1, 1), (16, 16, 32, 16), 1),
    _t2("CC3_a", "opmn,opij->ijmn", 8, PP, (16, 16, 16, 16), PP, (16, 16, 32, 32), 2),
    _t2("CC1_b", "ijkl,mnkl->ijmn", 16, PP, (16, 16, 16, 16), PP, (8, 8, 16, 16), 3),
    _t2("CC2_b", "opij,opkm->ijmk", 16, PP, (8, 8, 16, 16), (-1, -1, 1, 1), (8, 8, 16, 8), 4),
    _t2("CC3_b", "opmn,opij->ijmn", 16, PP, (8, 8, 8, 8), PP, (8, 8, 16, 16), 5),
    _t2("MM_a", "ij,jk->ik", 2, (1, -1), (10000, 10000), (1, -1), (10000, 10000), 6),
    _t2("MM_b", "ij,jk->ik", 100, (1, -1), (2000, 2000), (1, -1), (2000, 2000), 7),
    _t2("MPS_a", "ijk,klm->ijlm", 2, (1, 1, -1), (3000, 10, 3000), (1, 1, -1), (3000, 1, 3000), 8),
    _t2("MPS_b", "ijk,klm->ijlm", 5, (1, 1, -1), (700, 10, 700), (1, 1, -1), (700, 1, 700), 9),
    _t2("PEPS_a", "ijkl,klmn->ijmn", 2, PP, (400, 400, 20, 20), PP, (20, 20, 20, 20), 10),
    _t2("PEPS_b", "ijkl,klmn->ijmn", 10, PP, (64, 64, 8, 8), PP, (8, 8, 8, 8), 11),
]}


def small_cases() -> List[Contraction]:
    """Small contractions (seconds on the oracle) spanning the (s,t,v) shapes,
    sigma = +-1, nonzero target charges and a product group."""
    out = [Z3_ORDER4]
    out.append(Contraction("mm_G4", "ij,jk->ik", (4,),
                           TensorSpec((1, -1), (0,), (5, 7), 1.0, 11),
                           TensorSpec((1, -1), (0,), (7, 3), 1.0, 12)))
    out.append(Contraction("mps_like_G3_Z1", "ijk,klm->ijlm", (3,),
                           TensorSpec((1, 1, -1), (1,), (3, 2, 4), 1.0, 13),
                           TensorSpec((1, -1, -1), (2,), (4, 3, 2), 1.0, 14)))
    out.append(Contraction("sigma_plus_G5", "iak,kjb->ijab", (5,),
                           TensorSpec((1, -1, 1), (2,), (2, 3, 3), 1.0, 15),
                           TensorSpec((1, 1, -1), (4,), (3, 2, 2), 1.0, 16)))
    out.append(Contraction("z2xz3_order4", "abkl,klij->aibj", (2, 3),
                           TensorSpec(PP, (1, 2), (2, 3, 2, 2), 1.0, 17),
                           TensorSpec(PP, (0, 1), (2, 2, 3, 2), 1.0, 18)))
    out.append(Contraction("outer_v0_G3", "ab,c->acb", (3,),
                           TensorSpec((1, -1), (1,), (3, 2), 1.0, 19),
                           TensorSpec((1,), (2,), (4,), 1.0, 20)))
    out.append(Contraction("full_ctr_s0t0_G4", "ab,ab->", (4,),
                           TensorSpec((1, -1), (0,), (3, 5), 1.0, 21),
                           TensorSpec((-1, 1), (0,), (3, 5), 1.0, 22)))
    out.append(Contraction("s0_G4", "kl,klj->j", (4,),
                           TensorSpec((1, 1), (3,), (3, 2), 1.0, 23),
                           TensorSpec((-1, -1, 1), (1,), (3, 2, 4), 1.0, 24)))
    out.append(Contraction("t0_G2", "ikl,lk->i", (2,),
                           TensorSpec((1, -1, 1), (1,), (3, 2, 4), 1.0, 25),
                           TensorSpec((-1, 1), (1,), (4, 2), 1.0, 26)))
    return out


# Generic contractions of Eq. ctr (Sec. 5.1.1, sensitivity to contraction
# type): s free modes of U, t free modes of V, v contracted modes, every mode
# with G = 4 sectors of the same size D, D chosen so that the contraction's
# symmetry-reduced work 2 G^(s+t+v-2) D^(s+t+v) is as close as an integer D
# gets to 80e9 flops.  Signs: U's free modes +1, contracted -1; V's contracted
# +1 (sigma = -1), free -1; zero remainders.  Entries N(0,1) scaled by
# 1/sqrt(contracted length).
GENERIC_G = 4
GENERIC_FLOPS = 80e9
GENERIC_STV = [(s, t, v) for s in (1, 2, 3) for t in (1, 2, 3) for v in (1, 2, 3)]


def generic_dim(s: int, t: int, v: int, G: int = GENERIC_G, flops: float = GENERIC_FLOPS) -> int:
    n = s + t + v
    return max(1, int(round((flops / (2.0 * G ** (n - 2))) ** (1.0 / n))))


def generic_contraction(s: int, t: int, v: int, G: int = GENERIC_G,
                        flops: float = GENERIC_FLOPS) -> Contraction:
    D = generic_dim(s, t, v, G, flops)
    letters = iter("abcdefghijklmnop")
    FU = "".join(next(letters) for _ in range(s))
    C = "".join(next(letters) for _ in range(v))
    FV = "".join(next(letters) for _ in range(t))
    scale = 1.0 / math.sqrt((G * D) ** v)
    seed = 9000 + 100 * s + 10 * t + v
    return Contraction(
        name=f"generic_s{s}t{t}v{v}_G{G}_D{D}",
        einsum=f"{FU}{C},{C}{FV}->{FU}{FV}",
        moduli=(G,),
        u=TensorSpec(tuple([1] * s + [-1] * v), (0,), tuple([D] * (s + v)), scale, seed),
        v=TensorSpec(tuple([1] * v + [-1] * t), (0,), tuple([D] * (v + t)), 1.0, seed + 1),
    )
