"""GPU parity of per-sample-design tracing (srp_trace_samples through the C
ABI) against the FP64 brute-force oracle on the same Philox samples.

Each sample instantiates its own hinge angles (FP32 rotation on the GPU,
FP64 then rounded in the oracle) and traces one ray, so a ray that grazes a
triangle edge within FP32 rounding may hit the neighbour: samples whose hit
lists agree must agree to 1e-5 of the sample weight P (2R)^2 (torque: times
R); the share of samples whose lists differ is bounded (0.2 %)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def srp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_10712_gb300 as srp
    return srp


@pytest.fixture(scope="module")
def ctx(srp):
    return srp.Context(0)


def _inputs(m, N, G, seed):
    rng = np.random.default_rng(seed)
    ang = rng.uniform(-np.pi / 2, np.pi / 2, size=(N, m.hinges.shape[0]))
    rho = rng.uniform(0.0, 0.5, size=(N, G, 2)).astype(np.float32)
    sun = rng.normal(size=(N, 3)); sun /= np.linalg.norm(sun, axis=1, keepdims=True)
    com = rng.uniform(-0.2, 0.2, size=(N, 3))
    return ang, rho, sun, com


def _compare(y, h, yo, ho, w0, R, max_frac=2e-3):
    same = np.all(h == ho, axis=1)
    assert (~same).mean() <= max_frac, (~same).sum()
    ef = np.abs(y[same, :3] - yo[same, :3]).max(initial=0.0)
    et = np.abs(y[same, 3:] - yo[same, 3:]).max(initial=0.0)
    assert ef <= 1e-5 * w0 and et <= 1e-5 * w0 * R, (ef / w0, et / (w0 * R))
    return same


@pytest.mark.parametrize("K", [1, 3])
def test_boxwing_per_sample_parity(srp, ctx, K):
    m = W.box_wing()
    N = 8192
    ang, rho, sun, com = _inputs(m, N, 64, seed=K)
    center, R = np.zeros(3), 6.0
    y, h = srp.srp_trace_samples(ctx, m.verts, m.vhinge, m.hinges, m.tris, m.group, ang, rho, sun, com, center, R,
                                 want_hits=True, max_bounces=K, seed=7, pressure=2.0, sun_base=100)
    yo, ho = oracle.trace_samples(m.verts, m.vhinge, m.hinges, m.tris, m.group, ang, rho, sun, com, center, R, K=K,
                                  seed=7, P=2.0, sample_base=100)
    same = _compare(y, h, yo, ho, 2.0 * (2 * R) ** 2, R)
    assert np.count_nonzero(h[:, 0] >= 0) > N // 20     # the rays do hit (~8 % of the square)


def test_satellite_per_sample_parity_and_device_mode(srp, ctx):
    """~3k-triangle hinged satellite (one warp per block, 145 KB of shared
    memory), K = 3; device-memory call equals the host call bit for bit."""
    m = W.procedural_satellite(dish_segments=64, dish_rings=20, n_boxes=60)
    N = 2048
    ang, rho, sun, com = _inputs(m, N, 64, seed=11)
    center, R = np.zeros(3), 7.0
    y, h = srp.srp_trace_samples(ctx, m.verts, m.vhinge, m.hinges, m.tris, m.group, ang, rho, sun, com, center, R,
                                 want_hits=True, max_bounces=3, seed=3)
    yo, ho = oracle.trace_samples(m.verts, m.vhinge, m.hinges, m.tris, m.group, ang, rho, sun, com, center, R, K=3,
                                  seed=3)
    _compare(y, h, yo, ho, (2 * R) ** 2, R, max_frac=5e-3)
    dev = torch.device("cuda", 0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    yd, hd = srp.srp_trace_samples(ctx, m.verts, m.vhinge, m.hinges, m.tris, m.group, t(ang), t(rho), t(sun), t(com),
                                   center, R, want_hits=True, max_bounces=3, seed=3)
    torch.cuda.synchronize()
    assert np.array_equal(yd.cpu().numpy(), y) and np.array_equal(hd.cpu().numpy(), h)


def test_full_satellite_streaming_parity(srp, ctx):
    """The 49,776-triangle satellite (streaming instantiation: each test
    rotates its triangle from the base mesh), K = 2."""
    m = W.procedural_satellite()
    N = 512
    ang, rho, sun, com = _inputs(m, N, 64, seed=21)
    center, R = np.zeros(3), 7.0
    y, h = srp.srp_trace_samples(ctx, m.verts, m.vhinge, m.hinges, m.tris, m.group, ang, rho, sun, com, center, R,
                                 want_hits=True, max_bounces=2, seed=5)
    yo, ho = oracle.trace_samples(m.verts, m.vhinge, m.hinges, m.tris, m.group, ang, rho, sun, com, center, R, K=2,
                                  seed=5)
    _compare(y, h, yo, ho, (2 * R) ** 2, R, max_frac=1e-2)


def test_projected_area_pin_on_gpu(srp, ctx):
    """Absorbing box-wing lit along -z, random hinge angles: the sample mean
    converges to -P (1 + 40/pi) z (see the oracle pin)."""
    m = W.box_wing()
    N = 1 << 20
    rng = np.random.default_rng(2)
    ang = rng.uniform(-np.pi / 2, np.pi / 2, size=(N, 2))
    y = srp.srp_trace_samples(ctx, m.verts, m.vhinge, m.hinges, m.tris, m.group, ang, np.zeros((N, 64, 2), np.float32),
                              np.tile([0.0, 0.0, 1.0], (N, 1)), np.zeros((N, 3)), np.zeros(3), 6.0, seed=9)
    A = 144.0
    p = (1.0 + 40.0 / np.pi) / A
    assert abs(y[:, 2].mean() + (1.0 + 40.0 / np.pi)) <= 3 * 1.2 * A * np.sqrt(p * (1 - p) / N)


def test_errors(srp, ctx):
    m = W.box_wing()
    N = 4
    ang, rho, sun, com = _inputs(m, N, 64, seed=1)
    with pytest.raises(srp.SRPError, match="SRP_EINVAL"):
        srp.srp_trace_samples(ctx, m.verts, np.full(m.V, 5, np.int32), m.hinges, m.tris, m.group, ang, rho, sun, com,
                              np.zeros(3), 6.0)
    with pytest.raises(srp.SRPError, match="SRP_EINVAL"):
        srp.srp_trace_samples(ctx, m.verts, m.vhinge, m.hinges, m.tris, m.group, ang, rho, sun, com, np.zeros(3), 0.0)
    y = srp.srp_trace_samples(ctx, m.verts, m.vhinge, m.hinges, m.tris, m.group, ang[:0], rho[:0], sun[:0], com[:0],
                              np.zeros(3), 6.0)
    assert y.shape == (0, 6)
