"""Pins of the oracle's clusters -> hits transform (local pixel coordinates
to global positions through per-module placement)."""
import numpy as np

from oracle import oracle
from paper_2004_04334_gb300 import synth

PR, PC = synth.PITCH_ROW, synth.PITCH_COL


def test_identity_placement_is_the_local_frame():
    origin = np.zeros((1, 3), np.float32)
    rot = np.eye(3, dtype=np.float32)[None]
    # module centre, first pixel, last pixel
    x = np.array([79.5, 0.0, 159.0])
    y = np.array([207.5, 0.0, 415.0])
    gx, gy, gz = oracle.hits(np.zeros(3), x, y, origin, rot, PR, PC)
    np.testing.assert_allclose(gx, [0.0, -0.795, 0.795], atol=1e-12)
    np.testing.assert_allclose(gy, [0.0, -3.1125, 3.1125], atol=1e-12)
    np.testing.assert_allclose(gz, 0.0, atol=0)


def test_quarter_turn_and_translation():
    origin = np.array([[1.0, 2.0, 3.0]], np.float32)
    rot = np.array([[[0, -1, 0], [1, 0, 0], [0, 0, 1]]], np.float32)  # 90 degrees about z
    gx, gy, gz = oracle.hits([0], [89.5], [217.5], origin, rot, PR, PC)  # u = 0.1, v = 0.15
    np.testing.assert_allclose([gx[0], gy[0], gz[0]], [1.0 - 0.15, 2.0 + 0.1, 3.0], atol=1e-7)


def test_barrel_hits_lie_on_their_layer_and_keep_distances():
    M = 64
    origin, rot = synth.barrel_geometry(M)
    rng = np.random.default_rng(0)
    n = 500
    mod = rng.integers(0, M, n)
    x = rng.uniform(0, 159, n)
    y = rng.uniform(0, 415, n)
    gx, gy, gz = oracle.hits(mod, x, y, origin, rot, PR, PC)
    u = (x - 79.5) * PR
    v = (y - 207.5) * PC
    r2 = origin[mod, 0].astype(np.float64) ** 2 + origin[mod, 1].astype(np.float64) ** 2
    # a point on a module tangent to the cylinder: |g_xy|^2 = r^2 + v^2, and z moves with u
    np.testing.assert_allclose(gx ** 2 + gy ** 2, r2 + v ** 2, rtol=1e-6)
    np.testing.assert_allclose(gz, origin[mod, 2] + u, atol=1e-6)
    # rigid placement: distances between hits of one module equal local distances
    same = np.flatnonzero(mod == mod[0])
    i, j = same[0], same[-1]
    d_glob = np.sqrt((gx[i] - gx[j]) ** 2 + (gy[i] - gy[j]) ** 2 + (gz[i] - gz[j]) ** 2)
    d_loc = np.hypot(u[i] - u[j], v[i] - v[j])
    assert abs(d_glob - d_loc) < 1e-6
