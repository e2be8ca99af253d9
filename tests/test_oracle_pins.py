"""Pins of the FP64 oracle against facts fixed outside it: published test
vectors, closed forms of the radiation-pressure integrals (Sec. 2.1 box-wing
and cannonball models; Sec. 3.2 force and torque integrals), exact counts and
symmetry/linearity invariants.  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _stat_ok(a, b, sa, sb, k=3.0, floor=1e-12):
    """|a-b| <= k*sqrt(sa^2+sb^2) per component (plus a round-off floor)."""
    tol = k * np.sqrt(np.asarray(sa) ** 2 + np.asarray(sb) ** 2) + floor
    return np.all(np.abs(np.asarray(a) - np.asarray(b)) <= tol), np.abs(np.asarray(a) - np.asarray(b)) / (tol)


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


# ---------------------------------------------------------------- ONB
def test_onb_orthonormal_right_handed():
    rng = np.random.default_rng(3)
    ns = list(rng.normal(size=(200, 3))) + [[0, 0, 1.0], [0, 0, -1.0], [1e-9, 0, -1.0], [1, 0, 0]]
    for n in ns:
        n = np.asarray(n, float) / np.linalg.norm(n)
        b1, b2 = oracle.onb(n)
        M = np.stack([b1, b2, n])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-12)
        assert np.allclose(np.cross(b1, b2), n, atol=1e-12)


# ---------------------------------------------------------------- plate
def _centre_count(R, nx, half):
    """Number of pixel-centre rays of the 2R grid inside |coord| < half."""
    dx = 2 * R / nx
    c = -R + (np.arange(nx) + 0.5) * dx
    return int(np.sum(np.abs(c) < half))


@pytest.mark.parametrize("rs,rd", [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (0.3, 0.2)])
def test_plate_facing_sun_exact(rs, rd):
    """Plate normal to the sun, pixel centres (no jitter): every deposit is
    the per-plate law, so F = P a count [(1-rs) d - (2 rs + 2/3 rd) n]
    with count the pixel centres inside the plate (exact, FP64)."""
    p = W.flat_plate((2.0, 1.0), 2)
    rho = np.array([[rs, rd]])
    e = np.array([0, 0, 1.0])
    nx = 200
    ft, _ = oracle.force(p.verts, p.tris, p.group, rho, e, np.zeros(3), nx=nx, jitter=0, K=1)
    c, R = oracle.grid(p.verts)
    cnt = _centre_count(R, nx, 1.0) * _centre_count(R, nx, 0.5)
    a = (2 * R / nx) ** 2
    d = -e
    n = e  # facing normal
    F = a * cnt * ((1 - rs) * d - (2 * rs + 2 / 3 * rd) * n)
    assert np.allclose(ft[0, :3], F, rtol=1e-12, atol=1e-15)
    # centred plate, symmetric pixel centres: torque zero to round-off
    assert np.all(np.abs(ft[0, 3:]) < 1e-12)
    # COM 0.5 m below the plate's centre along -y: every hit point sits at
    # r = x - com, whose mean is (0, 0.5, 0), so tau = r x F = (0.5 F_z, 0, 0)
    # (the right-hand cross product, torque about the COM)
    ft2, _ = oracle.force(p.verts, p.tris, p.group, rho, e, np.array([0.0, -0.5, 0.0]), nx=nx, jitter=0, K=1)
    assert np.allclose(ft2[0, :3], F, rtol=1e-12, atol=1e-15)
    assert np.allclose(ft2[0, 3:], [0.5 * F[2], 0.0, 0.0], rtol=1e-12, atol=1e-13)


def test_plate_absorber_forms():
    """The flat-plate forms of an absorber, a mirror and a Lambertian plate at cos = 1."""
    p = W.flat_plate((2.0, 1.0), 2)
    A = 2.0
    e = np.array([0, 0, 1.0]); d = -e; n = e
    for (rs, rd), F in [((0, 0), A * d), ((1, 0), -2 * A * n + 0 * d), ((0, 1), A * (d - 2 / 3 * n))]:
        got = oracle.facet_law(p.verts, p.tris, p.group, np.array([[rs, rd]]), e, np.zeros(3))
        assert np.allclose(got[:3], F, atol=1e-12)


@pytest.mark.parametrize("theta_deg", [20.0, 55.0])
def test_tilted_plate_statistical(theta_deg):
    """Tilted plate with stratified jitter: estimator agrees with
    P A cos [(1-rs) d - (2 rs cos + 2/3 rd) n] within 3 sigma."""
    p = W.flat_plate((2.0, 1.0), 2)
    rho = np.array([[0.25, 0.35]])
    th = math.radians(theta_deg)
    e = np.array([math.sin(th), 0.3 * math.sin(th), math.cos(th)])
    e /= np.linalg.norm(e)
    ft, sg = oracle.force(p.verts, p.tris, p.group, rho, e, np.zeros(3), nx=256, K=1, seed=11)
    ref = oracle.facet_law(p.verts, p.tris, p.group, rho, e, np.zeros(3))
    ok, r = _stat_ok(ft[0, :3], ref[:3], sg[0, :3], 0)
    assert ok, r


# ---------------------------------------------------------------- convex bodies
def test_box_per_facet_law_and_bounce_invariance():
    """Convex box: K=1 matches the per-facet law (3 sigma); K=3 agrees with
    K=1 in expectation (reflected rays never re-hit a convex body)."""
    bv, bt = W.axis_box((0.1, -0.2, 0.3), (0.5, 0.7, 1.1), 0)
    verts = bv.astype(np.float32); tris = bt.astype(np.int32)
    group = np.arange(12, dtype=np.int32) // 2
    rho = W.random_reflectances(6, seed=4)
    e = np.array([0.3, -0.5, 0.8]); e /= np.linalg.norm(e)
    com = np.array([0.0, 0.1, 0.0])
    f1, s1 = oracle.force(verts, tris, group, rho, e, com, nx=256, K=1, seed=1)
    f3, s3 = oracle.force(verts, tris, group, rho, e, com, nx=256, K=3, seed=2)
    ref = oracle.facet_law(verts, tris, group, rho, e, com)
    ok, r = _stat_ok(f1[0], ref, s1[0], 0)
    assert ok, r
    ok, r = _stat_ok(f3[0], f1[0], s3[0], s1[0])
    assert ok, r


def test_icosphere_cannonball():
    """Icosphere -> sphere: per-facet law converges to the cannonball force
    P pi R^2 (1 + 4 rd/9) d (specular adds nothing on a sphere), torque 0;
    the MC estimate agrees with the facet law."""
    e = np.array([0.2, 0.4, -0.9]); e /= np.linalg.norm(e)
    rs, rd = 0.3, 0.4
    rho = np.array([[rs, rd]])
    errs, terrs = [], []
    for s in (1, 2, 3):
        m = W.icosphere(s)
        F = oracle.facet_law(m.verts, m.tris, m.group, rho, e, np.zeros(3))
        ball = math.pi * (1 + 4 * rd / 9) * (-e)
        errs.append(np.linalg.norm(F[:3] - ball) / np.linalg.norm(ball))
        terrs.append(np.linalg.norm(F[3:]) / np.linalg.norm(ball))
    assert errs[2] < 0.02 and errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1], errs
    assert terrs[2] < 1e-3 and terrs[2] < terrs[0], terrs
    m = W.icosphere(2)
    ft, sg = oracle.force(m.verts, m.tris, m.group, rho, e, np.zeros(3), nx=192, K=1, seed=5)
    ref = oracle.facet_law(m.verts, m.tris, m.group, rho, e, np.zeros(3))
    ok, r = _stat_ok(ft[0], ref, sg[0], 0)
    assert ok, r


def test_all_absorber_counts_hits():
    """All-absorber body: F = P a (number of rays hitting) d, so F/(P a) is an
    integer vector multiple of d."""
    m = W.box_wing()
    rho = np.zeros((64, 2))
    e = W.SUN_C1
    nx = 128
    ft, _ = oracle.force(m.verts, m.tris, m.group, rho, e, np.zeros(3), nx=nx, K=1, seed=3)
    c, R = oracle.grid(m.verts)
    a = (2 * R / nx) ** 2
    cnt = -ft[0, :3] / e / a
    assert np.allclose(cnt, cnt[0], rtol=1e-9)
    assert abs(cnt[0] - round(cnt[0])) < 1e-6 and cnt[0] > 100


def test_v_groove_retroreflector_multibounce():
    """90-degree mirror V-groove lit along its bisector: every entering ray is
    reflected twice and leaves reversed, so the expected force is
    2 P A_aperture d.  Exercises the sampled-branch bounce path (K=3)."""
    L, a = 1.0, 1.0
    s = a / math.sqrt(2)
    # walls through the x axis (groove axis), opening toward +z
    v = np.array([[-L / 2, 0, 0], [L / 2, 0, 0], [L / 2, s, s], [-L / 2, s, s],
                  [-L / 2, -s, s], [L / 2, -s, s]], dtype=np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3], [0, 4, 5], [0, 5, 1]], dtype=np.int32)
    g = np.zeros(4, np.int32)
    rho = np.array([[1.0, 0.0]])
    e = np.array([0, 0, 1.0])
    ft, sg = oracle.force(v, t, g, rho, e, np.zeros(3), nx=256, K=3, seed=9)
    ap = L * 2 * s
    ref = 2 * ap * (-e)
    ok, r = _stat_ok(ft[0, :3], ref, sg[0, :3], 0, k=4.0, floor=3e-3 * np.linalg.norm(ref))
    assert ok, (ft[0, :3], ref, sg[0, :3])
    # K=2 closes the second hit with the expected reflection: same mean
    f2, s2 = oracle.force(v, t, g, rho, e, np.zeros(3), nx=256, K=2, seed=10)
    ok, r = _stat_ok(f2[0, :3], ref, s2[0, :3], 0, k=4.0, floor=3e-3 * np.linalg.norm(ref))
    assert ok, (f2[0, :3], ref)


def test_boxwing_mirror_symmetry():
    """Box-wing with one material and the sun in the x-z plane is mirror
    symmetric in y: F_y, tau_x, tau_z vanish (3 sigma)."""
    m = W.box_wing()
    rho = np.tile(np.array([[0.2, 0.3]], np.float32), (64, 1))
    e = np.array([0.4, 0.0, 0.9]); e /= np.linalg.norm(e)
    ft, sg = oracle.force(m.verts, m.tris, m.group, rho, e, np.zeros(3), nx=256, K=3, seed=21)
    for j in (1, 3, 5):
        assert abs(ft[0, j]) <= 3 * sg[0, j] + 1e-9 * np.linalg.norm(ft[0, :3]), (j, ft[0], sg[0])


def test_rotation_equivariance():
    """Rotating the mesh and the sun together rotates F and tau (3 sigma)."""
    m = W.box_wing()
    rho = W.random_reflectances(64, seed=0)
    e = W.SUN_C1
    Rm = oracle.rotation(np.array([1.0, 1.0, 0.0]) / math.sqrt(2), 0.7)
    v2 = (m.verts.astype(np.float64) @ Rm.T).astype(np.float32)
    f1, s1 = oracle.force(m.verts, m.tris, m.group, rho, e, np.zeros(3), nx=256, K=2, seed=1)
    f2, s2 = oracle.force(v2, m.tris, m.group, rho, Rm @ e, np.zeros(3), nx=256, K=2, seed=2)
    rot = np.concatenate([Rm @ f1[0, :3], Rm @ f1[0, 3:]])
    srot = np.concatenate([np.abs(Rm) @ s1[0, :3], np.abs(Rm) @ s1[0, 3:]])
    ok, r = _stat_ok(f2[0], rot, s2[0], srot)
    assert ok, r


def test_mc_convergence_rate():
    """Error of the sampled-bounce estimate falls like N^-1/2: log-log slope
    of the RMS error over seeds vs the ray count in [-0.6, -0.4]."""
    L, a = 1.0, 1.0
    s = a / math.sqrt(2)
    v = np.array([[-L / 2, 0, 0], [L / 2, 0, 0], [L / 2, s, s], [-L / 2, s, s],
                  [-L / 2, -s, s], [L / 2, -s, s]], dtype=np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3], [0, 4, 5], [0, 5, 1]], dtype=np.int32)
    g = np.zeros(4, np.int32)
    rho = np.array([[0.4, 0.5]])
    e = np.array([0.1, 0.2, 1.0]); e /= np.linalg.norm(e)
    ref, _ = oracle.force(v, t, g, rho, e, np.zeros(3), nx=1024, K=3, seed=1000)
    ns, errs = [], []
    for nx in (32, 64, 128, 256):
        err = []
        for sd in range(12):
            f, _ = oracle.force(v, t, g, rho, e, np.zeros(3), nx=nx, K=3, seed=sd)
            err.append(np.sum((f[0, :3] - ref[0, :3]) ** 2))
        ns.append(nx * nx); errs.append(math.sqrt(np.mean(err)))
    slope = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert -0.6 <= slope <= -0.4, (slope, errs)


def test_sigma_matches_seed_spread():
    """The collapsed-strata sigma is consistent with the spread of the
    estimate over independent seeds (it may only over-estimate mildly)."""
    m = W.box_wing()
    rho = W.random_reflectances(64, seed=0)
    fs, ss = [], []
    for sd in range(16):
        f, s = oracle.force(m.verts, m.tris, m.group, rho, W.SUN_C1, np.zeros(3), nx=96, K=3, seed=100 + sd)
        fs.append(f[0]); ss.append(s[0])
    spread = np.std(np.asarray(fs), axis=0, ddof=1)
    sig = np.mean(np.asarray(ss), axis=0)
    ratio = sig[:3] / spread[:3]
    assert np.all((ratio > 0.6) & (ratio < 2.5)), ratio


# ---------------------------------------------------------------- reductions
def test_ray_subset_consistent():
    """A ray subset (offset, stride) traced in four parts sums to the full
    grid; thread count does not change the result."""
    m = W.box_wing()
    rho = W.random_reflectances(64, seed=0)
    nx = 64
    f, s = oracle.force(m.verts, m.tris, m.group, rho, W.SUN_C1, np.zeros(3), nx=nx, K=3)
    f1, s1 = oracle.force(m.verts, m.tris, m.group, rho, W.SUN_C1, np.zeros(3), nx=nx, K=3, threads=1)
    assert np.array_equal(f, f1) and np.array_equal(s, s1)
    parts = [oracle.force(m.verts, m.tris, m.group, rho, W.SUN_C1, np.zeros(3), nx=nx, K=3,
                          ray_offset=o, ray_stride=4, ray_count=nx * nx // 4)[0] for o in range(4)]
    assert np.allclose(sum(parts), f, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- area estimator (Sec. 3.2 "Estimation")
def test_area_estimator_convex_force_exact():
    """Convex box: sunlit facets are fully visible and the back facets are
    shadowed, and the force deposit of a sample does not depend on its
    point, so the area estimate of F equals the per-facet law exactly;
    the torque (point-dependent) agrees within 3 sigma."""
    bv, bt = W.axis_box((0.1, -0.2, 0.3), (0.5, 0.7, 1.1), 0)
    verts = bv.astype(np.float32); tris = bt.astype(np.int32)
    group = np.arange(12, dtype=np.int32) // 2
    rho = W.random_reflectances(6, seed=4)
    e = np.array([0.3, -0.5, 0.8]); e /= np.linalg.norm(e)
    com = np.array([0.0, 0.1, 0.0])
    ft, sg = oracle.force_area(verts, tris, group, rho, e, com, density=2000.0, seed=3)
    ref = oracle.facet_law(verts, tris, group, rho, e, com)
    assert np.allclose(ft[0, :3], ref[:3], rtol=1e-12, atol=1e-14)
    ok, r = _stat_ok(ft[0, 3:], ref[3:], sg[0, 3:], 0)
    assert ok, r


def test_area_estimator_shadowed_plate_and_counts():
    """A plate entirely in the shadow of a larger plate above it receives no
    force; sample counts are max(1, ceil(density * area))."""
    top = W.flat_plate((4.0, 4.0), 2)
    low = W.flat_plate((1.0, 1.0), 2)
    v = np.concatenate([top.verts + np.array([0, 0, 1.0], np.float32), low.verts])
    t = np.concatenate([top.tris, low.tris + 4]).astype(np.int32)
    g = np.array([0, 0, 1, 1], np.int32)
    rho = np.array([[0.0, 0.0], [0.3, 0.2]])
    e = np.array([0.0, 0.1, 1.0]); e /= np.linalg.norm(e)
    ft, _ = oracle.force_area(v, t, g, rho, e, np.zeros(3), density=500.0, seed=1)
    ft_top, _ = oracle.force_area(v[:4], t[:2], g[:2], rho, e, np.zeros(3), density=500.0, seed=1)
    assert np.allclose(ft[0, :3], ft_top[0, :3], rtol=1e-12)   # the low plate adds nothing
    c = oracle.area_counts(v, t, 500.0)
    assert list(c) == [4000, 4000, 250, 250]


def test_area_estimator_matches_ray_grid():
    """Both estimators target the same integral (single bounce): box-wing
    with self-shadowing, 3 sigma."""
    m, rho, sun, com = W.config1()
    fa, sa = oracle.force_area(m.verts, m.tris, m.group, rho, sun, com, density=3000.0, seed=2)
    fg, sgg = oracle.force(m.verts, m.tris, m.group, rho, sun, com, nx=512, K=1, seed=2)
    ok, r = _stat_ok(fa[0], fg[0], sa[0], sgg[0])
    assert ok, r


def _gauss_square(half, n):
    """Gauss-Legendre nodes and weights over [-half, half]^2."""
    x, w = np.polynomial.legendre.leggauss(n)
    return np.meshgrid(half * x, half * x, indexing="ij"), np.outer(half * w, half * w)


def test_area_interreflection_closed_form():
    """One Lambertian interreflection (K = 2): a sunlit diffuse square A
    (side 2, z = 0, rho_d = 0.5) and a square B (side 0.5, rho_s = 0.3,
    rho_d = 0.4) one metre above its centre, sun 70 degrees off the normal
    so that B's shadow falls beside A.  A reflects radiance
    L = rho_d P cos(70)/pi toward B's underside (normal -z); a beam arriving
    there along d at cos_B = d.z pushes it by the per-plate law
    (1 - rs) d - (2 rs cos_B + 2/3 rd)(-z), whose z part is
    (1 + rs) cos_B + 2/3 rd.  With cos_A = cos_B = h/r and
    dOmega = cos_A dA_A / r^2 the force is L [(1 + rs) I3 + 2/3 rd I2] along
    +z, I_k = int_B int_A h^k / r^(k+2) dA_A dA_B (Gauss-Legendre), and the
    x, y parts cancel by symmetry.  B's underside is not sunlit and A's lit
    side sees only B's dark underside, so nothing else is gathered:
    F(K=2) - F(K=1) on the same samples (the direct part is identical) is
    that term, within 3 sigma of the sampled directions."""
    va, ta = _plate((2.0, 2.0))
    vb, tb = _plate((0.5, 0.5), z=1.0)
    v = np.concatenate([va, vb]).astype(np.float32)
    t = np.concatenate([ta, tb + 4]).astype(np.int32)
    g = np.array([0, 0, 1, 1], np.int32)
    rho = np.array([[0.0, 0.5], [0.3, 0.4]])
    th = np.deg2rad(70.0)
    e = np.array([np.sin(th), 0.0, np.cos(th)])
    f1, _ = oracle.force_area(v, t, g, rho, e, np.zeros(3), density=1.0e5, seed=4)
    f2, s2 = oracle.force_area(v, t, g, rho, e, np.zeros(3), density=1.0e5, seed=4, K=2)
    (ax, ay), wa = _gauss_square(1.0, 24)
    (bx, by), wb = _gauss_square(0.25, 12)
    r2 = (ax.ravel()[:, None] - bx.ravel()[None, :]) ** 2 + (ay.ravel()[:, None] - by.ravel()[None, :]) ** 2 + 1.0
    I3 = float(wa.ravel() @ (r2 ** -2.5) @ wb.ravel())
    I2 = float(wa.ravel() @ (r2 ** -2.0) @ wb.ravel())
    L = 0.5 * np.cos(th) / np.pi
    want = np.array([0.0, 0.0, L * ((1.0 + 0.3) * I3 + (2.0 / 3.0) * 0.4 * I2)])
    got = f2[0, :3] - f1[0, :3]
    assert np.all(np.abs(got - want) <= 3.0 * s2[0, :3] + 1e-12), (got, want, s2[0, :3])
    assert s2[0, 2] < 0.02 * want[2]   # the pin resolves the term to about 2 %


def test_area_interreflection_convex_body_adds_nothing():
    """A closed convex box sees no other lit surface from outside, and from
    inside every gathered point is shadowed by the box itself: K = 2 gives
    the K = 1 estimate bit for bit."""
    bv, bt = W.axis_box((0.1, -0.2, 0.3), (0.5, 0.7, 1.1), 0)
    verts = bv.astype(np.float32); tris = bt.astype(np.int32)
    group = np.arange(12, dtype=np.int32) // 2
    rho = W.random_reflectances(6, seed=4)
    e = np.array([0.3, -0.5, 0.8]); e /= np.linalg.norm(e)
    f1, s1 = oracle.force_area(verts, tris, group, rho, e, np.zeros(3), density=800.0, seed=3)
    f2, s2 = oracle.force_area(verts, tris, group, rho, e, np.zeros(3), density=800.0, seed=3, K=2)
    assert np.array_equal(f1, f2) and np.array_equal(s1, s2)


def test_area_interreflection_matches_two_bounce_grid():
    """With no specular reflection (rho_s = 0) the grid estimator at K = 2
    (primary hit, one sampled Lambertian bounce, closed form at the second
    hit) and the area estimator with one gathered interreflection estimate
    the same truncated integral (light reflected once, by reciprocity of the
    transport between the two surfaces): box-wing with both panels hinged
    toward the bus, 3 sigma.  Their difference from K = 1 is resolved."""
    m = W.box_wing()
    v = oracle.instantiate(m.verts, m.vhinge, m.hinges, np.array([0.9, -0.8]))
    rho = W.random_reflectances(64, seed=6)
    rho[:, 0] = 0.0
    rho[:, 1] = 0.3 + rho[:, 1]
    e = np.array([0.2, 0.4, 0.9]); e /= np.linalg.norm(e)
    com = np.zeros(3)
    fa, sa = oracle.force_area(v, m.tris, m.group, rho, e, com, density=6000.0, seed=5, K=2)
    fg, sgg = oracle.force(v, m.tris, m.group, rho, e, com, nx=512, K=2, seed=5)
    ok, r = _stat_ok(fa[0], fg[0], sa[0], sgg[0])
    assert ok, r
    f1, _ = oracle.force_area(v, m.tris, m.group, rho, e, com, density=6000.0, seed=5)
    assert np.linalg.norm(fa[0, :3] - f1[0, :3]) > 6.0 * np.linalg.norm(sa[0, :3])


# ---------------------------------------------------------------- thermal emitters (Sec. 5.9)
C_LIGHT = 299792458.0


def _plate(size, z=0.0, flip=False):
    m = W.flat_plate(size, 2)
    v = m.verts.copy(); v[:, 2] += z
    t = m.tris.copy()
    if flip:
        t = t[:, ::-1].copy()
    return v.astype(np.float32), t.astype(np.int32)


def test_thermal_worked_number():
    """Sec. 5.9 worked example (tests/golden/paper_worked_examples.txt):
    70 kW from a Lambertian emitter recoil with 2/3 of the collimated
    momentum flux, about 1.55e-4 N, 1.55e-7 m/s^2 on 1000 kg.  An isolated
    plate (nothing to hit) emitting 70 kW from one side."""
    from conftest import golden
    g = golden("paper_worked_examples.txt")
    v, t = _plate((2.0, 1.0))
    emit = np.array([g["thermal_power_w"] / 2.0], np.float32)    # W/m^2 over the 2 m^2 plate
    ft, sg, n = oracle.force_thermal(v, t, np.zeros(2, np.int32), np.zeros((1, 2)), emit, np.zeros(3),
                                     density=100.0, P=1.0 / C_LIGHT)
    f = g["thermal_recoil_fraction"] * g["thermal_power_w"] / C_LIGHT
    assert np.allclose(ft[:3], [0.0, 0.0, -f], rtol=1e-6, atol=1e-15)
    tol = g["printed_rel_tol"]
    assert abs(np.linalg.norm(ft[:3]) - g["thermal_recoil_n"]) < tol * g["thermal_recoil_n"]
    assert abs(np.linalg.norm(ft[:3]) / 1000.0 - g["thermal_accel_m_s2"]) < tol * g["thermal_accel_m_s2"]
    assert n == 200


def test_thermal_cube_cancels():
    """All six faces of a closed cube emitting equally: the recoils cancel
    and outward emission never hits the convex cube."""
    bv, bt = W.axis_box((0.0, 0.0, 0.0), (0.5, 0.5, 0.5), 0)
    ft, sg, n = oracle.force_thermal(bv.astype(np.float32), bt.astype(np.int32), np.zeros(12, np.int32),
                                     np.array([[0.3, 0.2]]), np.array([1000.0], np.float32), np.zeros(3),
                                     density=400.0, P=1.0 / C_LIGHT)
    assert np.all(np.abs(ft[:3]) <= 1e-12 * 1000.0 / C_LIGHT * 6)
    assert np.all(np.abs(ft[3:]) <= 4.0 * sg[3:] + 1e-18)
    assert n == 12 * 200


def test_thermal_enclosure_conserves_momentum():
    """An emitter inside a closed absorbing box: every packet is absorbed
    inside the body, so recoil and deposits cancel in expectation (3 sigma)
    while each alone is large; an absorbing plate above an upward emitter is
    pushed up and the net force stays between 0 and the free recoil."""
    bv, bt = W.axis_box((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 0)
    box_t = bt[:, ::-1].astype(np.int32)                 # inward-facing walls (they do not emit)
    pv, pt = _plate((0.5, 0.5), z=-0.5)
    v = np.concatenate([bv, pv]).astype(np.float32)
    t = np.concatenate([box_t, pt + 8]).astype(np.int32)
    g = np.array([0] * 12 + [1] * 2, np.int32)
    rho = np.zeros((2, 2))
    emit = np.array([0.0, 500.0], np.float32)
    ft, sg, n = oracle.force_thermal(v, t, g, rho, emit, np.zeros(3), density=40000.0, P=1.0 / C_LIGHT, seed=3)
    free = (2.0 / 3.0) * 500.0 * 0.25 / C_LIGHT
    assert n == 2 * 5000
    assert np.all(np.abs(ft[:3]) <= 4.0 * sg[:3] + 1e-20)
    assert np.linalg.norm(ft[:3]) < 0.02 * free
    # plate over the emitter: partial absorption
    tv, tt = _plate((2.0, 2.0), z=0.5)
    v2 = np.concatenate([pv, tv]).astype(np.float32)
    t2 = np.concatenate([pt, tt + 4]).astype(np.int32)
    ft2, sg2, _ = oracle.force_thermal(v2, t2, np.array([1, 1, 0, 0], np.int32), rho, emit, np.zeros(3),
                                       density=40000.0, P=1.0 / C_LIGHT, seed=4)
    assert -free < ft2[2] < 0.0 and ft2[2] > -free + 10 * sg2[2]


@pytest.mark.parametrize("rho_hit", [(1.0, 0.0), (0.0, 1.0), (0.0, 0.0)])
def test_thermal_reflector_push(rho_hit):
    """A large plate close above a small upward emitter catches almost every
    packet.  A perfect mirror (rho_s = 1) takes 2 cos w along its normal,
    a perfect Lambertian reflector (rho_d = 1) takes w omega + 2/3 w n; with
    E[cos] = 2/3 and E[omega] = 2/3 n both give 4/3 w and the net is
    -2/3 + 4/3 = +2/3 of the free recoil; an absorber takes 2/3 w: net 0."""
    pv, pt = _plate((0.2, 0.2))
    mv, mt = _plate((40.0, 40.0), z=0.05)
    v = np.concatenate([pv, mv]).astype(np.float32)
    t = np.concatenate([pt, mt + 4]).astype(np.int32)
    g = np.array([0, 0, 1, 1], np.int32)
    rho = np.array([[0.0, 0.0], list(rho_hit)])
    ft, sg, _ = oracle.force_thermal(v, t, g, rho, np.array([1.0, 0.0], np.float32), np.zeros(3),
                                     density=2.0e5, P=1.0, seed=5)
    free = (2.0 / 3.0) * 0.04
    want = 0.0 if rho_hit == (0.0, 0.0) else free
    assert abs(ft[2] - want) < 0.01 * free + 3 * sg[2]


# ---------------------------------------------------------------- per-sample designs (Sec. 3.2, Alg. 1 NNLoss)
def _boxwing_absorber_samples(angles, N, seed):
    m = W.box_wing()
    e = np.array([0.0, 0.0, 1.0])
    R = 6.0
    y, hits = oracle.trace_samples(m.verts, m.vhinge, m.hinges, m.tris, m.group, angles,
                                   np.zeros((N, 64, 2)), np.tile(e, (N, 1)), np.zeros((N, 3)), np.zeros(3), R,
                                   K=1, seed=seed, P=1.0)
    return y, hits, R


def test_samples_absorbing_boxwing_projected_area():
    """Absorbing box-wing lit along -z: the panels (5 x 2 m, hinged about y
    beside the bus) project 10 cos(theta) each and the bus top 1 m^2, with no
    mutual shadowing, so one ray over the 12 x 12 m square deposits
    P (2R)^2 d with probability A_proj / (2R)^2: per design the mean is
    -P (1 + 10 cos t1 + 10 cos t2) z, and over theta ~ U[-pi/2, pi/2]^2 it is
    -P (1 + 40/pi) z.  3 sigma of the binomial spread."""
    N = 1 << 17
    rng = np.random.default_rng(1)
    ang = rng.uniform(-np.pi / 2, np.pi / 2, size=(N, 2))
    y, hits, R = _boxwing_absorber_samples(ang, N, seed=5)
    A = 4 * R * R
    p = (1.0 + 40.0 / np.pi) / A
    mean = y[:, 2].mean()
    sd = A * np.sqrt(p * (1 - p) / N) * 1.2          # (the per-design p varies; 20 % margin on the spread)
    assert abs(mean + (1.0 + 40.0 / np.pi)) <= 3 * sd, (mean, sd)
    assert np.all(np.abs(y[:, :2]) <= 1e-9 * A)
    # conditional: fixed angles
    fixed = np.tile([0.7, -0.2], (N, 1))
    y2, _, _ = _boxwing_absorber_samples(fixed, N, seed=6)
    want = 1.0 + 10 * np.cos(0.7) + 10 * np.cos(0.2)
    p2 = want / A
    assert abs(y2[:, 2].mean() + want) <= 3 * A * np.sqrt(p2 * (1 - p2) / N)


def test_samples_design_changes_hits():
    """A panel rotated by 90 degrees is edge-on to a sun along z: no sample
    hits it; at 0 degrees it is hit."""
    N = 4096
    m = W.box_wing()
    e = np.tile([0.0, 0.0, 1.0], (N, 1))
    y, hits = oracle.trace_samples(m.verts, m.vhinge, m.hinges, m.tris, m.group, np.tile([np.pi / 2, 0.0], (N, 1)),
                                   np.zeros((N, 64, 2)), e, np.zeros((N, 3)), np.zeros(3), 6.0, K=1, seed=2)
    assert not np.any(np.isin(hits[:, 0], [12, 13]))          # panel 1 (triangles 12, 13) edge-on
    assert np.any(np.isin(hits[:, 0], [14, 15]))


def test_samples_mean_matches_grid_estimate():
    """With one fixed design, the mean of the per-sample estimates (one ray
    each, K = 3, reflective materials) converges to the ray-grid estimate of
    the same design: 3 sigma of the sample mean."""
    m, rho, _, com = W.config1()
    N = 1 << 16
    ang = np.tile([0.4, -0.6], (N, 1))
    v = oracle.instantiate(m.verts, m.vhinge, m.hinges, ang[0])
    e = np.array([0.3, -0.2, 0.9]); e /= np.linalg.norm(e)
    c, R = oracle.grid(v)
    y, _ = oracle.trace_samples(m.verts, m.vhinge, m.hinges, m.tris, m.group, ang, np.tile(rho, (N, 1, 1)),
                                np.tile(e, (N, 1)), np.tile(com, (N, 1)), c, R, K=3, seed=4)
    fg, sg = oracle.force(v, m.tris, m.group, rho, e[None], com, nx=512, K=3, seed=1)
    se = y.std(axis=0) / np.sqrt(N)
    assert np.all(np.abs(y.mean(axis=0) - fg[0]) <= 3 * np.sqrt(se ** 2 + sg[0] ** 2) + 1e-12)


# ---------------------------------------------------------------- watertight intersection
def _tiled_square():
    """[-1,1]^2 at z = 0 in 8 x 8 cells of 0.25 m, each split along a
    diagonal (alternating direction), plus two unreferenced vertices at
    z = +-2 so that the grid radius is R = 2 about the origin: pixel centres
    then fall exactly on lattice vertices, edges and diagonals."""
    k = np.arange(9) * 0.25 - 1.0
    X, Y = np.meshgrid(k, k, indexing="ij")
    v = np.stack([X.ravel(), Y.ravel(), np.zeros(81)], axis=1)
    v = np.concatenate([v, [[0.0, 0.0, 2.0], [0.0, 0.0, -2.0]]])
    tris = []
    for i in range(8):
        for j in range(8):
            a, b, c, d = 9 * i + j, 9 * (i + 1) + j, 9 * (i + 1) + j + 1, 9 * i + j + 1
            tris += [[a, b, c], [a, c, d]] if (i + j) % 2 == 0 else [[a, b, d], [b, c, d]]
    return v.astype(np.float32), np.array(tris, np.int32)


def _contains(v, t, p):
    """Closed point-in-triangle test in the z = 0 plane (exact for these
    dyadic coordinates)."""
    a, b, c = v[t[0], :2].astype(np.float64), v[t[1], :2].astype(np.float64), v[t[2], :2].astype(np.float64)
    cr = lambda o, q, r: (q[0] - o[0]) * (r[1] - o[1]) - (q[1] - o[1]) * (r[0] - o[0])
    s = [cr(a, b, p), cr(b, c, p), cr(c, a, p)]
    return all(x >= 0 for x in s) or all(x <= 0 for x in s)


@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 16), (8, 16), (16, 8), (32, 32)])
def test_watertight_edges_vertices_and_ties(nx, ny):
    """Woop-Benthin-Wald watertight intersection in the oracle: rays through
    shared vertices (8 x 8), cell diagonals (16 x 16), vertical and
    horizontal shared edges (8 x 16, 16 x 8) of the tiled square all hit it,
    once each: the all-absorber force is exactly -P a z times the number of
    pixel centres inside; each ray's triangle is the smallest index among
    the triangles that contain its point (the tie rule on equal t)."""
    v, t = _tiled_square()
    g = np.zeros(len(t), np.int32)
    e = np.array([0.0, 0.0, 1.0])
    c, R = oracle.grid(v)
    assert np.array_equal(c, np.zeros(3)) and R == 2.0
    ft, _ = oracle.force(v, t, g, np.zeros((1, 2)), e, np.zeros(3), nx=nx, ny=ny, K=1, jitter=0)
    dx, dy = 4.0 / nx, 4.0 / ny
    xs = -2.0 + (np.arange(nx) + 0.5) * dx
    ys = -2.0 + (np.arange(ny) + 0.5) * dy
    inside = int(np.sum(np.abs(xs) < 1.0)) * int(np.sum(np.abs(ys) < 1.0))
    assert ft[0, 2] == -inside * dx * dy and ft[0, 0] == 0.0 and ft[0, 1] == 0.0
    # the grid's u axis is +x and its v axis -y for a sun along +z (the ONB of
    # the travel direction -z)
    for i in range(nx * ny):
        p = np.array([xs[i % nx], -ys[i // nx]])
        f, _ = oracle.primary_hit(v, t, e, i, nx=nx, ny=ny, jitter=0)
        owners = [k for k in range(len(t)) if _contains(v, t[k], p)]
        assert f == (min(owners) if owners else -1), (i, p, f, owners)


def test_parallel_triangle_is_never_hit():
    """A triangle whose plane contains the travel direction is never hit,
    including by rays that lie in its plane."""
    v = np.array([[-1.0, 0.25, -1.0], [1.0, 0.25, -1.0], [0.0, 0.25, 1.0], [0.0, 0.0, 2.0], [0.0, 0.0, -2.0],
                  [0.0, -0.25, 0.0]], np.float32)
    t = np.array([[0, 1, 2]], np.int32)
    assert oracle.grid(v)[1] == 2.0
    for nx in (8, 16):      # with 8 x 8 a row of pixel centres lies in the plane y = 0.25
        ft, _ = oracle.force(v, t, np.zeros(1, np.int32), np.zeros((1, 2)), np.array([0.0, 0.0, 1.0]),
                             np.zeros(3), nx=nx, K=1, jitter=0)
        assert np.all(ft == 0.0)
        assert all(oracle.primary_hit(v, t, np.array([0.0, 0.0, 1.0]), i, nx=nx, jitter=0)[0] == -1
                   for i in range(nx * nx))
