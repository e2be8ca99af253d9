"""The synthetic inputs are the recipe the design notes state: triangle
counts, material groups, hinges, the log-uniform design sizes, the
Fibonacci and orbit-state generators, and determinism in their seeds (the
parity tests and the benchmark depend on every side drawing the same
inputs)."""
import math

import numpy as np

import workloads as W


def test_box_wing_and_satellite_recipe():
    b = W.box_wing()
    assert b.tris.shape == (16, 3) and b.hinges.shape == (2, 6)
    assert np.array_equal(b.group, np.arange(16))                 # facet f -> group f
    assert np.allclose(np.linalg.norm(b.hinges[:, 3:], axis=1), 1.0)
    b7 = W.box_wing_7group()
    assert b7.n_groups == 7 and b7.group.max() == 6
    m = W.procedural_satellite()
    assert m.tris.shape[0] == 49776 and m.n_groups == 64
    assert m.group.min() >= 0 and m.group.max() <= 63
    assert np.array_equal(m.tris, W.procedural_satellite().tris)
    assert np.array_equal(m.group, W.procedural_satellite().group)
    assert np.isfinite(m.verts).all() and m.tris.min() >= 0 and m.tris.max() < m.verts.shape[0]


def test_config5_sizes_log_uniform_and_deterministic():
    d = W.config5_designs(16)
    T = np.array([x.tris.shape[0] for x in d])
    assert T.min() >= 0.8 * 5000 and T.max() <= 1.2 * 200000
    assert np.array_equal(T, [x.tris.shape[0] for x in W.config5_designs(16)])
    # log-uniform draws: the logs spread over most of [log 5k, log 200k]
    lt = np.log(T)
    assert lt.max() - lt.min() > 0.5 * (math.log(200000) - math.log(5000))


def test_direction_and_orbit_generators():
    f = W.fibonacci_directions(4096)
    assert np.allclose(np.linalg.norm(f, axis=1), 1.0)
    i = np.arange(4096)
    assert np.allclose(f[:, 2], 1.0 - (2.0 * i + 1.0) / 4096)
    assert abs(f.mean(axis=0)).max() < 1e-3                      # evenly spread
    z = W.orbit_states(64, seed=7)
    r, v, q = z[:, :3], z[:, 3:6], z[:, 6:10]
    assert np.allclose(np.linalg.norm(r, axis=1), 26560e3)
    assert np.allclose(np.linalg.norm(v, axis=1), math.sqrt(3.986004418e14 / 26560e3))
    assert np.allclose(np.einsum("ij,ij->i", r, v), 0.0, atol=1e-6 * 26560e3 * 4e3)
    h = np.cross(r, v)
    assert np.allclose(h[:, 2] / np.linalg.norm(h, axis=1), math.cos(math.radians(55.0)))   # inclination
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0)
    assert np.array_equal(z, W.orbit_states(64, seed=7)) and not np.array_equal(z, W.orbit_states(64, seed=8))
