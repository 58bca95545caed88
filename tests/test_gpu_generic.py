"""GPU parity on the generic contractions of Eq. ctr (Sec. 5.1.1): every
(s, t, v) with s, t, v in 1..3 (free modes of U, free modes of V, contracted
modes), G = 4 and one sector size D per contraction chosen for about 80e9
useful flops, operands drawn on the device.

The split-BF16 form runs every point at full size and is checked on one
sample in every 128 x 128 tile of every irrep of the aligned GEMM (the
oracle's aligned rows gathered entry by entry, oracle.aligned_index, and
multiplied in float64) plus entries straight from Eq. ctr.  TF32 runs a few
points at full size; the float64 form (about 1 TFLOP/s on GB300) runs every
point at 2e9 flops.  Also here: the small aligned shapes (M or N from 8 to 31,
K from 1 to 17) that the tensor-core forms took over from the float64 kernels.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as WL
from test_gpu_configs import TOL, oplan, sample_indices, sampled_rel, spec, tile_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sc():
    if not torch.cuda.is_available():
        pytest.fail("a GPU test ran without a visible GPU")
    import paper_2007_08056_gb300 as mod
    mod.load()
    return mod


def device_operands(c):
    gen = torch.Generator(device="cuda").manual_seed(c.u.seed)
    u = torch.randn(WL.reduced_shape(c.moduli, c.u.dims), generator=gen, device="cuda",
                    dtype=torch.float64).mul_(c.u.scale)
    v = torch.randn(WL.reduced_shape(c.moduli, c.v.dims), generator=gen, device="cuda",
                    dtype=torch.float64).mul_(c.v.scale)
    return u, v


def run_point(sc, c, precision, elements=4):
    torch.cuda.empty_cache()
    u, v = device_operands(c)
    p = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), precision)
    if precision != "fp64":
        assert p.info.tensor_core == 1
    w = p.contract(u, v)
    torch.cuda.synchronize()
    p.check_device_error()
    o = oplan(c)
    err, count = tile_check(o, u, v, w, per=1, seed=c.u.seed)
    idx = sample_indices(p.shape_w, elements, c.u.seed + 1)
    want = [O.contract_element_lazy(o, lambda i: u[i].cpu().numpy(), lambda i: v[i].cpu().numpy(), ix)
            for ix in idx]
    got = [w[ix].item() for ix in idx]
    del u, v, w, p
    torch.cuda.empty_cache()
    return max(err, sampled_rel(got, want)), count


@pytest.mark.parametrize("stv", WL.GENERIC_STV, ids=lambda x: "s%dt%dv%d" % x)
def test_generic_split_full_size(sc, stv):
    c = WL.generic_contraction(*stv)
    err, count = run_point(sc, c, "split_bf16")
    assert count > 0
    assert err <= TOL["split_bf16"]


@pytest.mark.parametrize("stv", [(1, 1, 1), (2, 2, 2), (3, 1, 1), (1, 3, 3), (3, 3, 1)],
                         ids=lambda x: "s%dt%dv%d" % x)
def test_generic_tf32_full_size(sc, stv):
    err, _ = run_point(sc, WL.generic_contraction(*stv), "tf32")
    assert err <= TOL["tf32"]


@pytest.mark.parametrize("stv", WL.GENERIC_STV, ids=lambda x: "s%dt%dv%d" % x)
def test_generic_fp64_reduced(sc, stv):
    err, _ = run_point(sc, WL.generic_contraction(*stv, flops=2e9), "fp64")
    assert err <= TOL["fp64"]


@pytest.mark.parametrize("precision", ["split_bf16", "tf32"])
def test_small_aligned_shapes_on_tensor_cores(sc, precision):
    """Matrix products W = U V under Z_2 with aligned M, N in 8..40 and K in
    1..17 (the K padding to 32 and the row padding of the 128-row tiles carry
    zeros): full comparison with the oracle's block loop."""
    rng = np.random.default_rng(7700)
    for (dm, dn, dk) in [(8, 20, 6), (20, 8, 1), (9, 12, 3), (16, 16, 8), (11, 17, 2), (15, 31, 9),
                         (33, 8, 17)]:
        c = WL.Contraction("mm_small", "ij,jk->ik", (2,),
                           WL.TensorSpec((1, -1), (0,), (dm, dk), 1.0, 1),
                           WL.TensorSpec((1, -1), (0,), (dk, dn), 1.0, 2))
        p = sc.Plan(c.einsum, c.moduli, spec(c.u), spec(c.v), precision)
        assert (p.info.M, p.info.N, p.info.K) == (dm, dn, dk) and p.info.tensor_core == 1
        u = rng.standard_normal(p.shape_u)
        v = rng.standard_normal(p.shape_v)
        w = p.contract(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda())
        torch.cuda.synchronize()
        p.check_device_error()
        want = O.contract_blockloop(oplan(c), u, v)
        got = w.cpu().numpy()
        assert np.linalg.norm(got - want) <= TOL[precision] * np.linalg.norm(want)
