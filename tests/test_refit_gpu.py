"""srp_bvh_refit: a BVH built at one set of hinge angles and refitted on the
device to the vertices of another traces the same forces as a fresh host
build at the new angles (closest hits do not depend on the boxes), with the
same grid centre and radius.  Only the grouping of sums may differ: the
span pre-pass projects the trees' boxes four levels down, so the two trees
split the live batches into tiles differently and the FP32 tile sums round
differently (about 1e-9 of |F|); the bound is 1e-7 of |F|, far below one
ray's deposit at 256^2 rays (about 5e-5)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def srp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_10712_gb300 as srp
    return srp


def _forces(srp, ctx, b, rho, sun, K):
    return srp.srp_force(ctx, [b], rho[None], sun, np.zeros((1, 3)), rays_x=256, max_bounces=K)[0]


@pytest.mark.parametrize("case,width", [("box_wing", 4), ("satellite", 4), ("satellite", 8)])
def test_refit_matches_fresh_build(srp, case, width):
    ctx = srp.Context(0)
    m = W.box_wing() if case == "box_wing" else W.config5_designs(1, t_lo=8000, t_hi=12000)[0]
    rho = W.random_reflectances(m.n_groups, seed=3).astype(np.float32)
    sun = W.fibonacci_directions(16)
    a0, a1 = np.array([0.3, -0.5]), np.array([0.45, -0.2])
    v0 = srp.srp_design_instantiate(m.verts, m.vhinge, m.hinges, a0)
    v1 = srp.srp_design_instantiate(m.verts, m.vhinge, m.hinges, a1)
    b = srp.srp_build_bvh(ctx, v0, m.tris, m.group, width)
    srp.srp_bvh_refit(ctx, b, v1, m.tris)
    fresh = srp.srp_build_bvh(ctx, v1, m.tris, m.group, width)
    ib, ifr = b.info(), fresh.info()
    assert ib["center"] == ifr["center"] and ib["radius"] == ifr["radius"]
    for K in (1, 3):
        fr = _forces(srp, ctx, b, rho, sun, K)
        ff = _forces(srp, ctx, fresh, rho, sun, K)
        scale = np.abs(ff[:, :3]).max()
        assert np.max(np.abs(fr - ff)) <= 1e-7 * scale + 1e-300, (K, np.max(np.abs(fr - ff)), scale)
    # refitting back to the build's vertices restores its forces
    srp.srp_bvh_refit(ctx, b, v0, m.tris)
    b0 = srp.srp_build_bvh(ctx, v0, m.tris, m.group, width)
    f0, g0 = _forces(srp, ctx, b, rho, sun, 3), _forces(srp, ctx, b0, rho, sun, 3)
    assert np.max(np.abs(f0 - g0)) <= 1e-7 * np.abs(g0[:, :3]).max()
    b.close(); fresh.close(); b0.close()


def test_refit_rejects_other_meshes(srp):
    ctx = srp.Context(0)
    m = W.box_wing()
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, 4)
    with pytest.raises(srp.SRPError) as e:
        srp.srp_bvh_refit(ctx, b, m.verts, m.tris[:-1])
    assert e.value.code == srp.SRP_EINVAL
    bad = m.tris.copy()
    bad[0, 0] = m.verts.shape[0]
    with pytest.raises(srp.SRPError) as e:
        srp.srp_bvh_refit(ctx, b, m.verts, bad)
    assert e.value.code == srp.SRP_EINVAL
    b.close()
