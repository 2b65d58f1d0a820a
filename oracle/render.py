"""Ray marching of a density model on [Hash,5,4,NN(3)] in FP64 (test infrastructure).

Section 4 renders the Bunny Cloud by ray marching directly on the in-memory model.  The
renderer here follows the library's statement: a pinhole camera (view axis f from the eye
to the target, r = f x up normalised, u = r x f; pixel (x, y) has film coordinates
(2(x + 1/2)/W - 1) tan(fov/2) W/H along r and (1 - 2(y + 1/2)/H) tan(fov/2) along u); each
ray is clipped to the model's domain box by slab intersection (from t = 0); samples at
t_in + (k + 1/2) step for k < max_steps while t <= t_out; density = the point query of the
codec (trilinear over regressed active corners, background elsewhere) clamped at 0;
emission-absorption front to back: alpha = 1 - exp(-sigma rho step), L += T alpha rho,
T *= 1 - alpha.  Output [H, W, 2] = (L, T).
"""
from __future__ import annotations

import numpy as np

from . import codec


def rays(cam: dict, lo: np.ndarray, hi: np.ndarray):
    """Unit directions [H*W, 3] (row-major pixels) and box entry / exit distances."""
    eye = np.asarray(cam["eye"], np.float64)
    f = np.asarray(cam["target"], np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(cam["up"], np.float64))
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    W, H = cam["width"], cam["height"]
    th = np.tan(np.radians(cam["fov_deg"]) / 2.0)
    x, y = np.meshgrid(np.arange(W), np.arange(H))
    fu = ((2.0 * (x + 0.5) / W - 1.0) * th * W / H).reshape(-1)
    fv = ((1.0 - 2.0 * (y + 0.5) / H) * th).reshape(-1)
    d = f[None] + fu[:, None] * r[None] + fv[:, None] * u[None]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t_in = np.zeros(len(d))
    t_out = np.full(len(d), np.inf)
    for a in range(3):
        par = d[:, a] == 0
        miss = par & ((eye[a] < lo[a]) | (eye[a] > hi[a]))
        with np.errstate(divide="ignore", invalid="ignore"):
            t0 = (lo[a] - eye[a]) / d[:, a]
            t1 = (hi[a] - eye[a]) / d[:, a]
        a0, a1 = np.minimum(t0, t1), np.maximum(t0, t1)
        t_in = np.where(par, t_in, np.maximum(t_in, a0))
        t_out = np.where(par, t_out, np.minimum(t_out, a1))
        t_in = np.where(miss, 1.0, t_in)
        t_out = np.where(miss, 0.0, t_out)
    return eye, d, t_in, t_out


def render(model: dict, cam: dict, active_keys: np.ndarray) -> np.ndarray:
    E = 1 << model["log2_extent"]
    lo = np.asarray(model["origin"], np.float64)
    eye, d, t_in, t_out = rays(cam, lo, lo + E)
    n = len(d)
    L = np.zeros(n)
    T = np.ones(n)
    step, sigma = cam["step"], cam["sigma"]
    for k in range(cam["max_steps"]):
        t = t_in + (k + 0.5) * step
        inside = (t_in <= t_out) & (t <= t_out)
        rho = np.zeros(n)
        if inside.any():
            p = eye[None] + t[inside, None] * d[inside]
            rho[inside] = np.maximum(codec.query(model, p, active_keys)[0], 0.0)
        alpha = 1.0 - np.exp(-sigma * rho * step)
        L += T * alpha * rho
        T *= 1.0 - alpha
    return np.stack([L, T], -1).reshape(cam["height"], cam["width"], 2)
