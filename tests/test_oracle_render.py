"""Pins of oracle/render.py (CPU only): the camera and slab clipping by closed forms, and the
compositing by constant-density media, where transmittance is exp(-sigma rho length) and
radiance 1 - T (emission equal to the density absorbed)."""
import numpy as np

from oracle import render


def test_camera_and_clipping():
    cam = dict(eye=[64.0, 64.0, -100.0], target=[64.0, 64.0, 0.0], up=[0.0, 1.0, 0.0], fov_deg=90.0,
               width=4, height=2, step=1.0, max_steps=10, sigma=1.0)
    eye, d, t_in, t_out = render.rays(cam, np.zeros(3), np.full(3, 128.0))
    # looking down +z; pixel (x, y) film point (u, v) = ((2(x+1/2)/4 - 1) * 2, 1 - 2(y+1/2)/2) for tan 45 = 1, aspect 2
    u = np.array([-1.5, -0.5, 0.5, 1.5]); v = np.array([0.5, -0.5])
    want = np.stack([np.tile(-u, 2), np.repeat(v, 4), np.ones(8)], -1)   # r = f x up = -x
    want /= np.linalg.norm(want, axis=1, keepdims=True)
    assert np.allclose(d, want, atol=1e-15)
    # the central rays (film (+-0.5, +-0.5)) enter the box at z = 0 and leave through a
    # side face, 64 voxels off the axis
    c = [1, 2, 5, 6]
    assert np.allclose(t_in[c] * d[c, 2], 100.0)
    assert np.allclose(t_out[c] * np.abs(d[c, 0]), 64.0) and np.allclose(t_out[c] * np.abs(d[c, 1]), 64.0)
    # a camera beside the box looking away misses it
    _, _, ti, to = render.rays(dict(cam, target=[64.0, 64.0, -200.0]), np.zeros(3), np.full(3, 128.0))
    assert np.all(ti > to)


class _Const:
    def __init__(self, rho):
        self.rho = rho


def test_constant_medium_closed_form(monkeypatch):
    rho, sigma, step = 0.3, 0.05, 0.5
    monkeypatch.setattr(render.codec, "query", lambda model, p, keys: (np.full(len(p), rho), None))
    model = dict(log2_extent=7, origin=np.zeros(3, np.int64))
    cam = dict(eye=[64.0, 64.0, -10.0], target=[64.0, 64.0, 10.0], up=[0.0, 1.0, 0.0], fov_deg=1.0,
               width=1, height=1, step=step, max_steps=1000, sigma=sigma)
    img = render.render(model, cam, None)
    n = int(128 / step)                                  # samples inside the 128-voxel box
    T = np.exp(-sigma * rho * step * n)
    assert np.isclose(img[0, 0, 1], T, rtol=1e-12) and np.isclose(img[0, 0, 0], rho * (1 - T), rtol=1e-12)
