"""GPU parity of the thermal-emitter estimator (srp_force_thermal through the
C ABI) against the FP64 oracle on the same Philox packets.

Bar: sample counts exact; (F, tau) within 1e-5 of the free-recoil scale
Fs = 2/3 P sum(emit A) (|F_gpu - F_or| <= 1e-5 Fs, |tau_gpu - tau_or| <=
1e-5 Fs R) -- the net force of a symmetric emitter can cancel to far below
its parts, so the parts set the scale; a packet grazing an edge within FP32
rounding may pick the neighbouring triangle."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

C_LIGHT = 299792458.0


@pytest.fixture(scope="module")
def srp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_10712_gb300 as srp
    return srp


@pytest.fixture(scope="module")
def ctx(srp):
    return srp.Context(0)


def _scale(verts, tris, group, emit, P):
    v = verts.astype(np.float64)
    A = 0.5 * np.linalg.norm(np.cross(v[tris[:, 1]] - v[tris[:, 0]], v[tris[:, 2]] - v[tris[:, 0]]), axis=1)
    return (2.0 / 3.0) * P * float(np.sum(np.asarray(emit, np.float64)[group] * A))


def _parity(ft, fo, Fs, R, tol=1e-5, what=""):
    ef = np.linalg.norm(np.asarray(ft)[:3] - fo[:3]) / Fs
    et = np.linalg.norm(np.asarray(ft)[3:] - fo[3:]) / (Fs * R)
    assert ef <= tol and et <= tol, (what, ef, et, ft, fo)


def test_worked_number_on_gpu(srp, ctx):
    """Sec. 5.9 worked example (tests/golden/paper_worked_examples.txt):
    70 kW from a Lambertian emitter -> 70e3 * 2/3 / c N, ~1.55e-4 N."""
    from conftest import golden
    g = golden("paper_worked_examples.txt")
    m = W.flat_plate((2.0, 1.0), 2)
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, 4)
    ft, n = srp.srp_force_thermal(ctx, [b], np.zeros((1, 1, 2), np.float32),
                                  np.array([[g["thermal_power_w"] / 2.0]], np.float32),
                                  np.zeros((1, 3)), 100.0, pressure=1.0 / C_LIGHT, out_samples=True)
    assert n[0] == 200
    f = g["thermal_recoil_fraction"] * g["thermal_power_w"] / C_LIGHT
    assert np.allclose(ft[0, :3], [0.0, 0.0, -f], rtol=1e-6, atol=1e-16)
    assert abs(np.linalg.norm(ft[0, :3]) - g["thermal_recoil_n"]) < g["printed_rel_tol"] * g["thermal_recoil_n"]


@pytest.mark.parametrize("width", [4, 8])
def test_boxwing_parity(srp, ctx, width):
    """Box-wing: the bus faces emit (different powers per face group), the
    panels and the other faces absorb and reflect (random rho)."""
    m = W.box_wing()
    rho = W.random_reflectances(64, seed=6)
    emit = np.zeros(64, np.float32)
    emit[:12] = np.linspace(100.0, 700.0, 12)
    com = np.array([0.05, -0.1, 0.2])
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, width)
    dens = 5.0e4
    ft, sg, n = srp.srp_force_thermal(ctx, [b], rho[None], emit[None], com[None], dens, out_sigma=True,
                                      out_samples=True, seed=3, pressure=1.0 / C_LIGHT)
    fo, so, no = oracle.force_thermal(m.verts, m.tris, m.group, rho, emit, com, density=dens, seed=3,
                                      P=1.0 / C_LIGHT)
    assert int(n[0]) == no
    Fs = _scale(m.verts, m.tris, m.group, emit, 1.0 / C_LIGHT)
    _parity(ft[0], fo, Fs, b.info()["radius"], what=f"W{width}")
    assert np.all(np.abs(sg[0] - so) <= 1e-3 * so.max())


def test_satellite_parity(srp, ctx):
    """Small procedural satellite: dish and boxes, a third of the groups
    emitting; packets hit the dish, the boxes and the panels."""
    m = W.procedural_satellite(dish_segments=64, dish_rings=20, n_boxes=60)
    rng = np.random.default_rng(7)
    emit = np.where(rng.uniform(size=m.n_groups) < 0.33, rng.uniform(50.0, 500.0, m.n_groups), 0.0).astype(np.float32)
    rho = W.random_reflectances(m.n_groups, seed=9)
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, 4)
    dens = 3000.0
    ft, n = srp.srp_force_thermal(ctx, [b], rho[None], emit[None], np.zeros((1, 3)), dens, seed=8,
                                  out_samples=True)
    fo, _, no = oracle.force_thermal(m.verts, m.tris, m.group, rho, emit, np.zeros(3), density=dens, seed=8)
    assert int(n[0]) == no == oracle.thermal_counts(m.verts, m.tris, m.group, emit, dens).sum()
    _parity(ft[0], fo, _scale(m.verts, m.tris, m.group, emit, 1.0), b.info()["radius"], what="satellite")


def test_multi_design_device_memory(srp, ctx):
    """Three hinge designs with their own emission tables, design_base in
    the counters, device-memory call."""
    m = W.box_wing_7group()
    angles = np.array([[0.0, 0.0], [0.7, -0.2], [-1.2, 1.0]])
    D = 3
    rho = np.stack([W.random_reflectances(7, seed=30 + d) for d in range(D)])
    emit = np.zeros((D, 7), np.float32)
    emit[0, 0] = 300.0; emit[1, :3] = [100.0, 0.0, 250.0]; emit[2, 5] = 80.0
    com = np.zeros((D, 3))
    verts = [srp.srp_design_instantiate(m.verts, m.vhinge, m.hinges, a) for a in angles]
    bvhs = [srp.srp_build_bvh(ctx, v, m.tris, m.group, 4) for v in verts]
    dev = torch.device("cuda", 0)
    ft, n = srp.srp_force_thermal(ctx, bvhs, torch.from_numpy(rho).to(dev), torch.from_numpy(emit).to(dev),
                                  torch.from_numpy(com).to(dev), 2.0e4, design_base=11, seed=2, out_samples=True)
    torch.cuda.synchronize()
    ft = ft.cpu().numpy(); n = n.cpu().numpy()
    for d in range(D):
        fo, _, no = oracle.force_thermal(verts[d], m.tris, m.group, rho[d], emit[d], com[d], density=2.0e4, seed=2,
                                         design_index=11 + d)
        assert n[d] == no
        _parity(ft[d], fo, _scale(verts[d], m.tris, m.group, emit[d], 1.0), bvhs[d].info()["radius"],
                what=f"design {d}")


def test_edge_cases_and_errors(srp, ctx):
    m = W.box_wing()
    b = srp.srp_build_bvh(ctx, m.verts, m.tris, m.group, 4)
    rho = W.random_reflectances(64, seed=1)
    # nothing emits: zero force, zero samples
    ft, n = srp.srp_force_thermal(ctx, [b], rho[None], np.zeros((1, 64), np.float32), np.zeros((1, 3)), 100.0,
                                  out_samples=True)
    assert n[0] == 0 and np.all(ft == 0.0)
    ft = srp.srp_force_thermal(ctx, [], np.zeros((0, 64, 2), np.float32), np.zeros((0, 64), np.float32),
                               np.zeros((0, 3)), 100.0)
    assert ft.shape == (0, 6)
    bad = np.zeros((1, 64), np.float32); bad[0, 3] = -1.0
    with pytest.raises(srp.SRPError, match="SRP_EINVAL"):
        srp.srp_force_thermal(ctx, [b], rho[None], bad, np.zeros((1, 3)), 100.0)
    with pytest.raises(srp.SRPError, match="SRP_EUNSUPPORTED"):
        srp.srp_force_thermal(ctx, [b], rho[None], np.ones((1, 64), np.float32), np.zeros((1, 3)), 100.0,
                              max_bounces=3)
    ft = srp.srp_force_thermal(ctx, [b], rho[None], np.ones((1, 64), np.float32), np.zeros((1, 3)), 100.0)
    assert np.all(np.isfinite(ft))
