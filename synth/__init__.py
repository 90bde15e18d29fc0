"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds none of the rendering arithmetic: it only draws primitive
parameters, ray origins/directions and request streams with numpy's PCG64
generator, so both sides receive bit-identical float32 inputs.  The shapes follow
the workloads stated for this library (unit-cube fields of 256 to 2M Gabor
primitives, 4- or 6-octave pyramids, ~1:16 base:residual ratios as in the
paper's assets, Sec. 6 and the procedural cloud of Sec. 7.3).

Parameter layout (dict of float32 numpy arrays, SoA):
  mu (N,3) | quat (N,4) as (w,x,y,z) | log_scale (N,3) | omega (N,3) |
  phase (N,) | weight (N,) | band (N,) uint8 (octave index, 0 = Gaussians)
plus the metadata keys ``omega_frame`` ("world" or "local") and
``weight_mode`` ("peak").
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi


def _uniform_quaternions(rng, n):
    """Uniform random rotations (Shoemake's subgroup algorithm), (w,x,y,z)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(TWO_PI * u2), a * np.cos(TWO_PI * u2),
                  b * np.sin(TWO_PI * u3), b * np.cos(TWO_PI * u3)], axis=1)
    return q


def _unit_vectors(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size))


def absorption_field(n=256, seed=0):
    """Absorption-only test field: n Gabor primitives in the unit cube.

    Means uniform; per-axis scales log-uniform in [0.02, 0.1]; uniform random
    rotations; carrier frequency f (cycles/unit) with log(1+f) uniform on
    [0, ln 9] (so f spans [0, 8]) and |omega| = 2 pi f in a uniformly random
    direction (world frame); phase uniform in [0, 2 pi); peak weights uniform
    in [0.5, 2].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = rng.random((n, 3))
    s = _log_uniform(rng, 0.02, 0.1, (n, 3))
    q = _uniform_quaternions(rng, n)
    f = np.power(9.0, rng.random(n)) - 1.0
    om = _unit_vectors(rng, n) * (TWO_PI * f)[:, None]
    phase = rng.uniform(0.0, TWO_PI, n)
    w = rng.uniform(0.5, 2.0, n)
    return {
        "mu": mu.astype(np.float32), "quat": q.astype(np.float32),
        "log_scale": np.log(s).astype(np.float32), "omega": om.astype(np.float32),
        "phase": phase.astype(np.float32), "weight": w.astype(np.float32),
        "band": None, "omega_frame": "world", "weight_mode": "peak",
    }


def octave_counts(n, octaves):
    """N_o = N0 4^o with N0 = floor(N / sum 4^o); the remainder goes to the top octave."""
    total = sum(4 ** o for o in range(octaves))
    n0 = n // total
    counts = [n0 * 4 ** o for o in range(octaves)]
    counts[-1] += n - sum(counts)
    return counts


def octave_field(n, octaves, seed=0, s_range=(0.02, 0.1), tau_target=4.0,
                 omega_range=(0.7, 1.5)):
    """Pyramid field: octave o has N0 4^o primitives with scales s_range 2^-o.

    Octave 0 holds Gaussians (zero carrier, zero phase), octaves >= 1 hold Gabor
    kernels in the tied form of Sec. 4.2 (whitened-frame carrier (w,w,w), w
    uniform in omega_range, so the world frequency doubles as the scale halves).
    Peak weights c_rho U[0.5, 2] with c_rho chosen so the Gaussian band has a
    mean optical depth of tau_target per unit path:
    c_rho = tau_target / (N0 * 1.25 * (2 pi)^1.5 * E[s]^3), E[s] the mean of the
    log-uniform scale distribution.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = octave_counts(n, octaves)
    lo, hi = s_range
    mean_s = (hi - lo) / math.log(hi / lo)
    c_rho = tau_target / (counts[0] * 1.25 * (TWO_PI ** 1.5) * mean_s ** 3)
    parts = {k: [] for k in ("mu", "quat", "log_scale", "omega", "phase", "weight", "band")}
    for o, no in enumerate(counts):
        parts["mu"].append(rng.random((no, 3)))
        s = _log_uniform(rng, lo, hi, (no, 3)) * 2.0 ** (-o)
        parts["log_scale"].append(np.log(s))
        parts["quat"].append(_uniform_quaternions(rng, no))
        if o == 0:
            parts["omega"].append(np.zeros((no, 3)))
            parts["phase"].append(np.zeros(no))
        else:
            w = rng.uniform(omega_range[0], omega_range[1], no)
            parts["omega"].append(np.repeat(w[:, None], 3, axis=1))
            parts["phase"].append(rng.uniform(0.0, TWO_PI, no))
        parts["weight"].append(c_rho * rng.uniform(0.5, 2.0, no))
        parts["band"].append(np.full(no, o, np.uint8))
    out = {k: np.concatenate(v).astype(np.float32) for k, v in parts.items() if k != "band"}
    out["band"] = np.concatenate(parts["band"]).astype(np.uint8)
    out["omega_frame"] = "local"
    out["weight_mode"] = "peak"
    out["c_rho"] = c_rho
    out["octave_counts"] = counts
    return out


def orthographic_rays(res=64, z0=-0.5, t_far=2.0):
    """res x res rays along +z through pixel centres of the unit square.

    Ray r = j*res + i starts at ((i+0.5)/res, (j+0.5)/res, z0) with t in [0, t_far].
    """
    i = (np.arange(res) + 0.5) / res
    x, y = np.meshgrid(i, i)  # y varies along rows
    o = np.stack([x.ravel(), y.ravel(), np.full(res * res, z0)], axis=1).astype(np.float32)
    d = np.tile(np.array([0.0, 0.0, 1.0], np.float32), (res * res, 1))
    tr = np.tile(np.array([0.0, t_far], np.float32), (res * res, 1))
    return o, d, tr


def random_rays(n, seed=0, t_far=3.0):
    """Rays from random points on a sphere of radius 1.5 around the cube centre,
    aimed at random points inside the unit cube."""
    rng = np.random.Generator(np.random.PCG64(seed))
    o = 0.5 + 1.5 * _unit_vectors(rng, n)
    tgt = rng.random((n, 3))
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    tr = np.tile(np.array([0.0, t_far]), (n, 1))
    return o.astype(np.float32), d.astype(np.float32), tr.astype(np.float32)


DEFAULT_CAMERA = {"eye": (0.5, 0.5, -1.0), "look_at": (0.5, 0.5, 0.5), "up": (0.0, 1.0, 0.0),
                  "vfov_deg": 45.0}
LIGHT_DIR = (1.0, 1.0, -1.0)  # direction towards the light (normalised by the consumers)


def perturb(params, rel=0.01, seed=1):
    """Multiply every float parameter by (1 + rel N(0,1)), element-wise."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = dict(params)
    for k in ("mu", "quat", "log_scale", "omega", "phase", "weight"):
        a = np.asarray(params[k], np.float64)
        out[k] = (a * (1.0 + rel * rng.standard_normal(a.shape))).astype(np.float32)
    return out


def request_stream(n_requests, rate_hz, seed=0, n_assets=4,
                   resolutions=(128, 256, 512, 1024), lods=(3, 2, 1, 0), spps=(1, 4, 16, 64)):
    """Poisson arrivals of render requests with random cameras on a sphere.

    Each request: arrival time (s), asset index, square resolution, LoD band
    cutoff, spp and a camera eye on a sphere of radius 1.5 about the cube centre.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    eyes = 0.5 + 1.5 * _unit_vectors(rng, n_requests)
    reqs = []
    for k in range(n_requests):
        reqs.append({
            "t_arrive": float(t[k]), "asset": int(rng.integers(n_assets)),
            "res": int(resolutions[rng.integers(len(resolutions))]),
            "lod": int(lods[rng.integers(len(lods))]),
            "spp": int(spps[rng.integers(len(spps))]),
            "eye": tuple(float(x) for x in eyes[k]), "seed": int(k),
        })
    return reqs
