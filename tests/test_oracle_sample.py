"""Pins of oracle/sample.py (CPU only): samplers against closed forms (order 1 and 3 reproduce
affine fields, order 3 interpolates, order 0 rounds to the nearest voxel), isosurface points
of a planar level set at the plane, and mCD 0 for identical grids and about the offset for
two parallel planes."""
import numpy as np

from oracle import sample, vdb


def _plane(offset, n=24):
    a = np.arange(n)
    g = np.stack(np.meshgrid(a, a, a, indexing="ij"), -1).reshape(-1, 3)
    d = g[:, 0] + 0.5 * g[:, 1] - 0.25 * g[:, 2] - offset
    sel = np.abs(d) < 3.0
    return vdb.build(g[sel], d[sel].astype(np.float32))


def _dense_affine(n=16):
    a = np.arange(n)
    g = np.stack(np.meshgrid(a, a, a, indexing="ij"), -1).reshape(-1, 3)
    f = (0.5 * g[:, 0] - 0.25 * g[:, 1] + 0.125 * g[:, 2] + 1.0).astype(np.float32)
    return vdb.build(g, f)


def test_samplers_closed_forms():
    g = _dense_affine()
    r = np.random.default_rng(0)
    p = r.uniform(2.0, 12.0, (500, 3))
    f = 0.5 * p[:, 0] - 0.25 * p[:, 1] + 0.125 * p[:, 2] + 1.0
    assert np.allclose(sample.sample(g, 0.0, p, 1), f, atol=1e-12)
    assert np.allclose(sample.sample(g, 0.0, p, 3), f, atol=1e-12)      # Catmull-Rom reproduces lines
    nearest = np.floor(p + 0.5)
    assert np.allclose(sample.sample(g, 0.0, p, 0), 0.5 * nearest[:, 0] - 0.25 * nearest[:, 1] + 0.125 * nearest[:, 2] + 1.0)
    q = g["ijk"][::37].astype(np.float64)
    for order in (0, 1, 3):                                              # integer points: the voxel value
        assert np.allclose(sample.sample(g, 0.0, q, order), g["val"][::37], atol=1e-12)
    far = np.array([[100.0, 100.0, 100.0]])
    assert np.all(sample.sample(g, 7.0, far, 1) == 7.0)                  # background outside


def test_isosurface_of_a_plane_and_mcd():
    g = _plane(10.3)
    pts = sample.isosurface(g, 3.0)
    assert len(pts) > 100
    d = pts[:, 0] + 0.5 * pts[:, 1] - 0.25 * pts[:, 2] - 10.3
    assert np.abs(d).max() < 1e-5                                        # on the plane (float32 values)
    assert sample.mcd(g, g, 3.0) < 1e-6
    h = _plane(10.8)
    want = 0.5                                                           # |SDF| shift of the plane's value
    assert abs(sample.mcd(g, h, 3.0) - want) < 0.02
