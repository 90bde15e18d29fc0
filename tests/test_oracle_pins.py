"""Pins for the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(App. A.3, A.4, Sec. 4.4), library routines (scipy erf / Rotation / quad),
brute force, invariants, Philox known-answer vectors, estimator expectations
and finite differences.  CPU only.
"""
import math
import os

import numpy as np
import pytest
from scipy import special, stats
from scipy.spatial.transform import Rotation

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _single(mu, quat, s, omega, phase, weight, frame="world", mode="peak", k=3.0):
    p = {"mu": np.array([mu], np.float32), "quat": np.array([quat], np.float32),
         "log_scale": np.log(np.array([s], np.float64)).astype(np.float32),
         "omega": np.array([omega], np.float32), "phase": np.array([phase], np.float32),
         "weight": np.array([weight], np.float32)}
    return oracle.Field(p, weight_mode=mode, omega_frame=frame, k_sigma=k), p


def _geom(p, i=0):
    """Sigma^-1, R, s from the float32 inputs, via scipy's Rotation (independent)."""
    q = p["quat"][i].astype(np.float64)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    s = np.exp(p["log_scale"][i].astype(np.float64))
    return R @ np.diag(1.0 / s ** 2) @ R.T, R, s


def _rand_prim(rng, omega_scale=20.0):
    mu = rng.random(3)
    q = rng.standard_normal(4)
    s = np.exp(rng.uniform(np.log(0.02), np.log(0.1), 3))
    om = rng.standard_normal(3) * omega_scale
    return mu, q, s, om, rng.uniform(0, 2 * np.pi), rng.uniform(0.5, 2.0)


def _ray_near(rng, mu, spread):
    v = rng.standard_normal(3)
    v /= np.linalg.norm(v)
    o = np.asarray(mu, np.float64) + spread * rng.standard_normal(3) - 1.0 * v
    return o, v


# --------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(vals[0:4], vals[4:6])
        assert [int(x) for x in out] == vals[6:10]


# --------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("mode", ["peak", "normalized"])
def test_full_line_closed_form_appendix_a4(mode):
    """Oracle quadrature over the whole line equals the boxed infinite-domain
    integral of App. A.4 (a, beta, gamma, B, delta of App. A.1), phase added."""
    rng = np.random.default_rng(1)
    for trial in range(16):
        mu, q, s, om, ph, w = _rand_prim(rng)
        f, p = _single(mu, q, s, om, ph, w, mode=mode, k=40.0)
        Sinv, R, s64 = _geom(p)
        o, v = _ray_near(rng, p["mu"][0], 0.05)
        d = o - p["mu"][0].astype(np.float64)
        omw = p["omega"][0].astype(np.float64)
        a = v @ Sinv @ v; beta = v @ Sinv @ d; gamma = d @ Sinv @ d
        B = omw @ v; delta = omw @ d + float(p["phase"][0])
        amp = float(p["weight"][0])
        if mode == "normalized":
            amp /= math.sqrt(8 * math.pi ** 3 * np.linalg.det(np.linalg.inv(Sinv)))
        exact = amp * math.sqrt(2 * math.pi / a) * math.exp(-0.5 * (gamma - beta ** 2 / a)) \
            * math.exp(-B ** 2 / (2 * a)) * math.cos(delta - beta * B / a)
        got = f.chord_integral(0, o, v, -np.inf, np.inf)
        scale = amp * math.sqrt(2 * math.pi / a) * math.exp(-0.5 * (gamma - beta ** 2 / a))
        assert abs(got - exact) <= 1e-10 * scale + 1e-300, (trial, got, exact)


def test_whitened_form_sec44_matches_unwhitened():
    """Sec. 4.4 whitened form with W = S^-1 R^T and k_W = S R^T omega equals the
    oracle; the literal W = R^T S^-1, k_W = W omega does not (reading of Eq. 11)."""
    rng = np.random.default_rng(2)
    literal_bad = 0
    for trial in range(12):
        mu, q, s, om, ph, w = _rand_prim(rng, omega_scale=10.0)
        f, p = _single(mu, q, s, om, ph, w, mode="normalized", k=40.0)
        Sinv, R, s64 = _geom(p)
        o, v = _ray_near(rng, p["mu"][0], 0.03)
        m = p["mu"][0].astype(np.float64)
        omw = p["omega"][0].astype(np.float64)
        phase = float(p["phase"][0])
        alpha = float(p["weight"][0])
        det_sigma = np.prod(s64) ** 2

        def whitened(W, kW):
            pW = W @ (o - m); Wv = W @ v; nWv = np.linalg.norm(Wv); vW = Wv / nWv
            b = pW @ vW; c = pW @ pW; Om = kW @ vW; dd = kW @ pW + phase
            K = 1.0 / (2 * math.pi * math.sqrt(det_sigma) * nWv)
            return alpha * K * math.exp(-0.5 * (c - b * b + Om * Om)) * math.cos(dd - Om * b)

        W = np.diag(1 / s64) @ R.T
        got = f.chord_integral(0, o, v, -np.inf, np.inf)
        ref = whitened(W, np.diag(s64) @ R.T @ omw)
        env = alpha / math.sqrt(8 * math.pi ** 3 * det_sigma) * math.sqrt(2 * math.pi / (v @ Sinv @ v))
        assert abs(got - ref) <= 1e-10 * env
        Wl = R.T @ np.diag(1 / s64)
        lit = whitened(Wl, Wl @ omw)
        if abs(lit - got) > 1e-6 * env:
            literal_bad += 1
    assert literal_bad >= 10


def _clip_chord(Sinv, m, o, v, k, tmin, tmax):
    d = o - m
    a = v @ Sinv @ v; beta = v @ Sinv @ d
    ts = -beta / a
    pp = d + ts * v
    r2 = pp @ Sinv @ pp
    if r2 >= k * k:
        return None
    hw = math.sqrt((k * k - r2) / a)
    lo, hi = max(ts - hw, tmin), min(ts + hw, tmax)
    return (lo, hi, a, beta, d @ Sinv @ d) if lo < hi else None


def test_zero_frequency_erf_form():
    """omega = 0, k = 3: the truncated chord integral equals the real-erf closed form."""
    rng = np.random.default_rng(3)
    for trial in range(24):
        mu, q, s, _, _, w = _rand_prim(rng)
        f, p = _single(mu, q, s, (0, 0, 0), 0.0, w, k=3.0)
        Sinv, _, _ = _geom(p)
        m = p["mu"][0].astype(np.float64)
        o, v = _ray_near(rng, m, 0.04)
        tmin, tmax = (0.0, np.inf) if trial % 2 == 0 else (0.9, 1.02)
        cc = _clip_chord(Sinv, m, o, v, 3.0, tmin, tmax)
        has, lo, hi = f.chord(0, o, v, tmin, tmax)
        assert has == (cc is not None)
        if cc is None:
            continue
        lo_r, hi_r, a, beta, gamma = cc
        assert abs(lo - lo_r) < 1e-12 and abs(hi - hi_r) < 1e-12
        amp = float(p["weight"][0])
        sa = math.sqrt(a / 2)
        exact = amp * math.sqrt(math.pi / (2 * a)) * math.exp(-0.5 * (gamma - beta ** 2 / a)) * (
            math.erf(sa * (hi_r + beta / a)) - math.erf(sa * (lo_r + beta / a)))
        got = f.chord_integral(0, o, v, tmin, tmax)
        assert abs(got - exact) <= 1e-12 * amp * math.sqrt(2 * math.pi / a)


def test_finite_segment_complex_erf_appendix_a3():
    """omega != 0, k = 3: the truncated chord integral equals the finite-domain
    complex-erf closed form of App. A.3 (scipy's complex erf)."""
    rng = np.random.default_rng(4)
    checked = 0
    for trial in range(40):
        mu, q, s, om, ph, w = _rand_prim(rng, omega_scale=15.0)
        f, p = _single(mu, q, s, om, ph, w, k=3.0)
        Sinv, _, _ = _geom(p)
        m = p["mu"][0].astype(np.float64)
        o, v = _ray_near(rng, m, 0.04)
        cc = _clip_chord(Sinv, m, o, v, 3.0, 0.0, np.inf)
        if cc is None:
            continue
        lo, hi, a, beta, gamma = cc
        omw = p["omega"][0].astype(np.float64)
        B = omw @ v
        delta = omw @ (o - m) + float(p["phase"][0])
        if abs(B) / math.sqrt(a) > 4.0:
            continue
        amp = float(p["weight"][0])
        al = math.sqrt(a / 2)
        zeta = (-beta + 1j * B) / math.sqrt(2 * a)
        r2 = gamma - beta ** 2 / a
        pref = amp * math.sqrt(math.pi / (2 * a)) * math.exp(-0.5 * r2 - B * B / (2 * a))
        val = pref * (np.exp(1j * (delta - beta * B / a)) *
                      (special.erf(al * hi - zeta) - special.erf(al * lo - zeta))).real
        got = f.chord_integral(0, o, v, 0.0, np.inf)
        assert abs(got - val) <= 1e-11 * amp * math.sqrt(2 * math.pi / a), (trial, got, val)
        checked += 1
    assert checked >= 10


def test_chord_matches_brute_force_sampling():
    """Chord endpoints equal the extent of {t : q(t) <= k^2} sampled on a fine grid."""
    rng = np.random.default_rng(5)
    for trial in range(20):
        mu, q, s, om, ph, w = _rand_prim(rng)
        f, p = _single(mu, q, s, om, ph, w, k=3.0)
        Sinv, _, _ = _geom(p)
        m = p["mu"][0].astype(np.float64)
        o, v = _ray_near(rng, m, 0.05)
        ts = np.linspace(0.0, 2.0, 400001)
        y = o[None, :] + ts[:, None] * v[None, :] - m[None, :]
        qq = np.einsum("ni,ij,nj->n", y, Sinv, y)
        inside = np.nonzero(qq <= 9.0)[0]
        has, lo, hi = f.chord(0, o, v, 0.0, 2.0)
        assert has == (inside.size > 0)
        if has:
            dt = ts[1] - ts[0]
            assert abs(ts[inside[0]] - lo) <= dt and abs(ts[inside[-1]] - hi) <= dt


# --------------------------------------------------------------------------- invariants
def _small_octave(n=340, octaves=4, seed=7):
    p = synth.octave_field(n, octaves, seed=seed)
    return oracle.Field(p, weight_mode="peak", omega_frame="local"), p


def test_band_densities_sum_to_full_density():
    f, p = _small_octave()
    occ, _ = f.cells()
    _, _, cell = f.labels()
    rng = np.random.default_rng(8)
    for _ in range(30):
        x = rng.random(3)
        full = f.density(x)
        acc = 0.0
        for b in range(8):
            bits = 0
            for c in range(64):
                if (occ >> c) & 1 and ((c == 0 and b == 0) or (c > 0 and (c - 1) // 8 + 1 == b)):
                    bits |= 1 << c
            if bits:
                acc += f.density(x, mask=bits)
        assert abs(acc - full) <= 1e-12 * (1 + abs(full))


def test_tau_is_sum_of_per_primitive_integrals_and_cutoffs_nest():
    """Eq. 3: tau = sum_i tau_i; band cutoffs add whole bands."""
    f, p = _small_octave()
    o, d, tr = synth.random_rays(16, seed=3)
    T_all, tau_all = f.transmittance(o, d, tr, mode="det")
    band = p["band"]
    per = np.zeros((16, f.n))
    for r in range(16):
        # the transmittance traces the FP32-rounded unit direction v32 as given:
        # int k(o + t v32) dt over [t0, t1] is the integral along the unit vector
        # v32/|v32| over [|v32| t0, |v32| t1], divided by |v32|
        dd = d[r].astype(np.float64)
        v32 = (dd / np.sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2])).astype(np.float32)
        v32 = v32.astype(np.float64)
        nv = np.sqrt(np.sum(v32 * v32))
        for i in range(f.n):
            per[r, i] = f.chord_integral(i, o[r], v32, nv * tr[r, 0], nv * tr[r, 1]) / nv
    assert np.allclose(tau_all, per.sum(1), rtol=0, atol=1e-11)
    assert np.allclose(T_all, np.exp(-tau_all), rtol=1e-14, atol=0)
    prev = np.zeros(16)
    for b in range(4):
        _, tau_b = f.transmittance(o, d, tr, mode="det", lod=oracle.Lod(1, b, 0))
        assert np.allclose(tau_b - prev, per[:, band == b].sum(1), atol=1e-11)
        prev = tau_b
    _, tau_cv = f.transmittance(o, d, tr, mode="det", lod=oracle.Lod(1, 7, 0))
    assert np.allclose(tau_cv, tau_all, atol=1e-12)


def test_phase_shift_by_pi_inverts_transmittance():
    rng = np.random.default_rng(9)
    for _ in range(8):
        mu, q, s, om, ph, w = _rand_prim(rng)
        f1, p1 = _single(mu, q, s, om, ph, w)
        f2, p2 = _single(mu, q, s, om, ph + math.pi, w)
        o, v = _ray_near(rng, p1["mu"][0], 0.03)
        T1, _ = f1.transmittance(o[None], v[None], None, mode="det")
        T2, _ = f2.transmittance(o[None], v[None], None, mode="det")
        # phases are float32 inputs: allow the rounding of ph + pi
        assert abs(T1[0] * T2[0] - 1.0) < 1e-5


def test_rotation_invariance():
    """Rotating the field (means, orientations, world carriers) and the rays
    together leaves every transmittance unchanged."""
    p = synth.absorption_field(64, seed=11)
    f = oracle.Field(p)
    o, d, tr = synth.random_rays(24, seed=5)
    T0, tau0 = f.transmittance(o, d, tr, mode="det")
    Q = Rotation.from_rotvec([0.3, -1.1, 0.7])
    c = np.array([0.5, 0.5, 0.5])
    p2 = dict(p)
    p2["mu"] = (Q.apply(p["mu"].astype(np.float64) - c) + c).astype(np.float32)
    qi = p["quat"].astype(np.float64)
    rq = Q * Rotation.from_quat(np.stack([qi[:, 1], qi[:, 2], qi[:, 3], qi[:, 0]], 1))
    xyzw = rq.as_quat()
    p2["quat"] = np.stack([xyzw[:, 3], xyzw[:, 0], xyzw[:, 1], xyzw[:, 2]], 1).astype(np.float32)
    p2["omega"] = Q.apply(p["omega"].astype(np.float64)).astype(np.float32)
    f2 = oracle.Field(p2)
    o2 = (Q.apply(o.astype(np.float64) - c) + c).astype(np.float32)
    d2 = Q.apply(d.astype(np.float64)).astype(np.float32)
    T1, tau1 = f2.transmittance(o2, d2, tr, mode="det")
    # float32 rounding of the rotated inputs perturbs positions by ~1e-7
    assert np.max(np.abs(tau1 - tau0)) < 2e-4
    assert np.max(np.abs(tau0)) > 0.05


# --------------------------------------------------------------------------- mask sampler
def test_mask_weights_are_reciprocal_probabilities():
    """Sum over outcomes of p * w * 1[cell selected] = 1 (App. B tables), checked
    by Monte Carlo frequencies against the stated probabilities."""
    f, p = _small_octave(n=5460, octaves=6)
    occ, kbar = f.cells()
    lod = oracle.Lod(2, 7, 1)  # uniform + control variate, importance-sampled cones
    v = np.array([0.3, -0.5, 0.81]); v /= np.linalg.norm(v)
    n = 40000
    acc = np.zeros(64)
    picks = np.zeros(64)
    for r in range(n):
        m, w = f.sample_mask(lod, v, seed=3, ray=r, sample=0, bounce=0, tag=oracle.TAG_MASK)
        bits = np.array([(m >> c) & 1 for c in range(64)], bool)
        acc += np.where(bits, w, 0.0)
        picks += bits
    cells = [c for c in range(64) if (occ >> c) & 1]
    assert acc[0] / n == pytest.approx(1.0, abs=1e-12)  # Gaussian band always, weight 1
    # expected frequency of each Gabor cell: 1/G * w_c / W_band
    axes = []
    for k in range(8):
        z = 1 - (k + 0.5) / 8; r_ = math.sqrt(1 - z * z); ph = k * math.pi * (3 - math.sqrt(5))
        axes.append((r_ * math.cos(ph), r_ * math.sin(ph), z))
    G = 5
    for c in cells:
        if c == 0:
            continue
        b = (c - 1) // 8 + 1
        band_cells = [cc for cc in cells if cc > 0 and (cc - 1) // 8 + 1 == b]
        wts = {cc: math.exp(-0.5 * kbar[cc] ** 2 * abs(np.dot(v, axes[(cc - 1) % 8])) ** 2)
               for cc in band_cells}
        pexp = wts[c] / sum(wts.values()) / G
        sd = math.sqrt(pexp * (1 - pexp) / n)
        assert abs(picks[c] / n - pexp) < 5 * sd + 1e-9
        est = acc[c] / n
        sd_w = (1.0 / pexp) * sd
        assert abs(est - 1.0) < 5 * sd_w


# --------------------------------------------------------------------------- estimators
def _three_gabors():
    p = {"mu": np.array([[0.45, 0.5, 0.5], [0.55, 0.52, 0.45], [0.5, 0.47, 0.6]], np.float32),
         "quat": np.array([[1, 0.2, 0.1, 0], [0.9, 0, 0.3, 0.2], [0.7, 0.1, 0, 0.6]], np.float32),
         "log_scale": np.log(np.array([[0.08, 0.06, 0.1], [0.05, 0.09, 0.07], [0.1, 0.1, 0.06]])).astype(np.float32),
         "omega": np.array([[0, 0, 0], [20, -10, 5], [-8, 12, 30]], np.float32),
         "phase": np.array([0.0, 1.0, 4.0], np.float32),
         "weight": np.array([6.0, 3.0, 2.5], np.float32)}
    return p


def test_ratio_tracking_is_unbiased_for_transmittance():
    p = _three_gabors()
    f = oracle.Field(p)
    o = np.array([[0.5, 0.5, -0.5], [0.47, 0.52, -0.5], [0.55, 0.45, -0.5]], np.float32)
    d = np.tile(np.array([0, 0, 1], np.float32), (3, 1))
    T_det, _ = f.transmittance(o, d, None, mode="det")
    blocks = np.array([f.transmittance(o, d, None, mode="rt", spp=4000, seed=s)[0]
                       for s in range(20)])
    mean = blocks.mean(0)
    se = blocks.std(0, ddof=1) / math.sqrt(blocks.shape[0])
    assert np.all(np.abs(mean - T_det) < 4.5 * se + 1e-4), (mean, T_det, se)
    assert np.all(T_det < 0.95)


def test_majorant_bounds_density_and_drives_points():
    """kappa_bar >= |kappa| on the ray, and the tentative points of one chord form a
    Poisson process with intensity equal to that chord's majorant."""
    p = _three_gabors()
    f = oracle.Field(p)
    o = np.array([0.5, 0.5, -0.5]); v = np.array([0.0, 0.0, 1.0])
    ts = np.linspace(0.7, 1.3, 3001)
    for t in ts:
        x = o + t * v
        assert f.majorant(o, v, t) >= abs(f.density(x)) - 1e-12
    # one chord: counts in bins vs integral of its own majorant
    fi = oracle.Field({k: p[k][1:2] for k in ("mu", "quat", "log_scale", "omega", "phase", "weight")})
    has, lo, hi = fi.chord(0, o, v)
    assert has
    edges = np.linspace(lo, hi, 9)
    grid = np.linspace(lo, hi, 40001)
    maj = np.array([fi.majorant(o, v, t) for t in grid])
    expect = np.array([np.trapezoid(maj[(grid >= a) & (grid <= b)], grid[(grid >= a) & (grid <= b)])
                       for a, b in zip(edges[:-1], edges[1:])])
    counts = np.zeros(8)
    nrep = 6000
    for w in range(nrep):
        t, _ = fi.chord_points(0, o, v, seed=1, ray=0, word=w)
        counts += np.histogram(t, edges)[0]
    exp_counts = expect * nrep
    chi2 = np.sum((counts - exp_counts) ** 2 / exp_counts)
    assert chi2 < stats.chi2.ppf(0.9999, 8)


def _gauss_only():
    p = _three_gabors()
    p = dict(p)
    p["omega"] = np.zeros((3, 3), np.float32)
    p["phase"] = np.zeros(3, np.float32)
    return p


@pytest.mark.parametrize("kind", ["gauss", "gabor"])
def test_delta_tracking_collision_distribution(kind):
    """Collision CDF is 1 - exp(-int_0^t max(kappa,0)) (Woodcock tracking of the
    clamped extinction)."""
    p = _gauss_only() if kind == "gauss" else _three_gabors()
    f = oracle.Field(p)
    o = np.array([0.5, 0.5, -0.5]); v = np.array([0.0, 0.0, 1.0])
    grid = np.linspace(0.0, 2.0, 40001)
    kap = np.array([f.density(o + t * v) for t in grid])
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (np.maximum(kap[1:], 0) + np.maximum(kap[:-1], 0)) * np.diff(grid))])
    if kind == "gauss":
        T_det, tau = f.transmittance(o[None].astype(np.float32), v[None].astype(np.float32), None)
        # the trapezoid rule is first order at the k-sigma cut-offs
        assert abs(cum[-1] - tau[0]) < 2e-5
    edges = np.linspace(0.6, 1.4, 17)
    Fe = 1 - np.exp(-np.interp(edges, grid, cum))
    probs = np.concatenate([[Fe[0]], np.diff(Fe), [1 - Fe[-1]]])
    n = 6000
    hits = []
    for r in range(n):
        h, t = f.delta_track(o, v, seed=2, ray=r, word=oracle.stream_word(0, 0, oracle.TAG_TRACK))
        hits.append(t if h else np.inf)
    hits = np.array(hits)
    counts = np.concatenate([[np.sum(hits < edges[0])], np.histogram(hits, edges)[0],
                             [np.sum(hits >= edges[-1])]])
    keep = probs * n > 5
    chi2 = np.sum((counts[keep] - n * probs[keep]) ** 2 / (n * probs[keep]))
    assert chi2 < stats.chi2.ppf(0.9999, keep.sum() - 1)


def test_masked_optical_depth_is_unbiased_and_jensen_bias():
    """E[tau_hat] = tau under uniform + control variate masking with importance-
    sampled cones (Sec. 4.5, per segment unbiased); E[exp(-tau_hat)] equals the
    enumeration over masks and exceeds exp(-tau) (Sec. 4.5.3)."""
    f, p = _small_octave(n=1365, octaves=5, seed=12)
    o, d, tr = synth.random_rays(6, seed=21)
    _, tau = f.transmittance(o, d, tr, mode="det")
    lod = oracle.Lod(2, 7, 1)
    blocks = np.array([f.transmittance(o, d, tr, mode="det", spp=200, seed=s, lod=lod)[1]
                       for s in range(16)])
    mean = blocks.mean(0)
    se = blocks.std(0, ddof=1) / 4.0
    assert np.all(np.abs(mean - tau) < 4.5 * se + 1e-9), (mean, tau, se)
    # Jensen with whole-band masking (cones all): enumerate the G equally likely masks
    lod_b = oracle.Lod(2, 7, 0)
    band_tau = []
    prev = np.zeros(6)
    for b in range(5):
        _, tb = f.transmittance(o, d, tr, mode="det", lod=oracle.Lod(1, b, 0))
        band_tau.append(tb - prev)
        prev = tb
    G = 4
    enum = np.mean([np.exp(-(band_tau[0] + G * band_tau[b])) for b in range(1, 5)], axis=0)
    samples = np.array([np.exp(-f.transmittance(o, d, tr, mode="det", spp=1, seed=s, lod=lod_b)[1])
                        for s in range(3000)])
    se2 = samples.std(0, ddof=1) / math.sqrt(3000)
    assert np.all(np.abs(samples.mean(0) - enum) < 4.5 * se2 + 1e-12)
    assert np.all(enum >= np.exp(-tau) - 1e-15)
    var = np.mean([(band_tau[0] + G * band_tau[b] - tau) ** 2 for b in range(1, 5)], axis=0)
    small = var < 0.05
    if small.any():
        approx = 0.5 * var * np.exp(-tau)
        assert np.all(np.abs((enum - np.exp(-tau))[small] - approx[small]) <= 0.5 * approx[small] + 1e-6)


@pytest.mark.parametrize("flight,spp", [("delta", 20000), ("cdf", 20000)])
def test_single_scatter_mean_matches_nested_quadrature(flight, spp):
    """Mean single-scattering radiance of one pixel equals
    albedo E/(4 pi) int kappa(t) exp(-tau(0,t)) T_light(x(t)) dt (Gaussian field),
    with delta tracking + ratio-tracked NEE and with CDF-inversion free flight +
    closed-form NEE (Sec. 3 Eq. 5, Sec. 4.4): the same expectation."""
    p = _gauss_only()
    f = oracle.Field(p)
    cam = oracle.camera((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), (0, 1, 0), 45.0, 64, 64)
    ro = oracle.render_opts("scatter", spp=spp, max_bounces=1, albedo=0.8, free_flight=flight)
    px, py = 32, 31
    smp = f.render(cam, ro, seed=5, crop=(px, py, 1, 1), samples=True).ravel()
    # reference: nested quadrature with per-sample jittered rays averaged
    ref = []
    rng_idx = range(0, spp, spp // 40)
    light = np.array([1.0, 1.0, -1.0]) / math.sqrt(3.0)
    for s in rng_idx:
        o, v = oracle.camera_ray(cam, 5, px, py, s)
        grid = np.linspace(0.9, 2.1, 1201)
        kap = np.array([f.density(o + t * v) for t in grid])
        cum = np.concatenate([[0.0], np.cumsum(0.5 * (kap[1:] + kap[:-1]) * np.diff(grid))])
        xs = o[None] + grid[:, None] * v[None]
        Tl, _ = f.transmittance(xs.astype(np.float32), np.tile(light, (len(grid), 1)).astype(np.float32),
                                None, mode="det")
        ref.append(0.8 / (4 * math.pi) * np.trapezoid(kap * np.exp(-cum) * Tl, grid))
    ref_mean = float(np.mean(ref))
    # the jitter varies the reference slightly: compare the sample mean with the
    # mean of the per-jitter references, within MC error plus the jitter spread
    se = smp.std(ddof=1) / math.sqrt(smp.size) + np.std(ref) / math.sqrt(len(ref))
    assert abs(smp.mean() - ref_mean) < 4.5 * se
    assert ref_mean > 1e-3


# --------------------------------------------------------------------------- gradient
def test_tomography_gradient_matches_central_differences():
    p = _three_gabors()
    p["phase"] = np.array([0.3, 1.0, 4.0], np.float32)
    cam = oracle.camera((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), (0, 1, 0), 12.0, 6, 6)
    spp = 2
    f = oracle.Field(p)
    target = f.tomo_image(cam, spp, 3) * 0.9 + 0.02
    L, g = f.tomo_loss_grad(cam, spp, 3, target)
    N = 3
    offs = {"mu": 0, "quat": 3 * N, "log_scale": 7 * N, "omega": 10 * N, "phase": 13 * N,
            "weight": 14 * N}
    rng = np.random.default_rng(0)
    checked = 0
    for key, off in offs.items():
        arr = p[key].reshape(-1)
        for j in range(arr.size):
            base = float(arr[j])
            # small steps: finite differences across a tangent chord are biased
            h = 1e-5 * max(abs(base), 0.5)
            pp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
            pm = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
            pp[key].reshape(-1)[j] = np.float32(base + h)
            pm[key].reshape(-1)[j] = np.float32(base - h)
            step = float(pp[key].reshape(-1)[j]) - float(pm[key].reshape(-1)[j])
            Lp, _ = oracle.Field(pp).tomo_loss_grad(cam, spp, 3, target)
            Lm, _ = oracle.Field(pm).tomo_loss_grad(cam, spp, 3, target)
            fd = (Lp - Lm) / step
            an = g[off + j]
            assert abs(fd - an) <= 2e-3 * abs(an) + 1e-5 * np.max(np.abs(g)), (key, j, fd, an)
            checked += 1
    assert checked == 45


# --------------------------------------------------------------------------- radiance gradient
def _positive_field():
    """A wide Gaussian under three small Gabor kernels, k = 6 (the cut lies where
    the kernels are ~1e-8 of their peak), with kappa > 0 wherever a kernel is."""
    p = {"mu": np.array([[0.5, 0.5, 0.5], [0.45, 0.52, 0.5], [0.55, 0.46, 0.55],
                         [0.5, 0.5, 0.42]], np.float32),
         "quat": np.array([[1, 0, 0, 0], [0.9, 0.1, 0.3, 0.2], [0.7, 0.1, 0, 0.6],
                           [1, 0.3, 0, 0.1]], np.float32),
         "log_scale": np.log(np.array([[0.3, 0.3, 0.3], [0.06, 0.05, 0.08], [0.07, 0.07, 0.05],
                                       [0.05, 0.08, 0.06]])).astype(np.float32),
         "omega": np.array([[0, 0, 0], [1.1, 1.1, 1.1], [0.8, 0.8, 0.8], [1.3, 1.3, 1.3]],
                           np.float32),
         "phase": np.array([0.0, 0.7, 2.0, 4.1], np.float32),
         "weight": np.array([2.0, 0.3, 0.25, 0.3], np.float32)}
    return p


def _nested_radiance(p, o, v, albedo=0.8):
    """albedo E/(4 pi) int kappa(t) exp(-tau(0,t)) T_light(x(t)) dt by the
    trapezoid rule on a fine grid, T_light from the deterministic quadrature."""
    f = oracle.Field(p, omega_frame="local", k_sigma=6.0)
    grid = np.linspace(0.0, 3.6, 3601)
    kap = np.array([f.density(o + t * v) for t in grid])
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (kap[1:] + kap[:-1]) * np.diff(grid))])
    light = np.array([1.0, 1.0, -1.0]) / math.sqrt(3.0)
    xs = o[None] + grid[:, None] * v[None]
    Tl, _ = f.transmittance(xs.astype(np.float32), np.tile(light, (len(grid), 1)).astype(np.float32),
                            None, mode="det")
    return albedo / (4 * math.pi) * np.trapezoid(kap * np.exp(-cum) * Tl, grid), kap


def test_radiance_estimator_mean_and_gradient_match_nested_quadrature():
    """The single-scattering radiance adjoint's expected-value estimator has the
    mean of the nested-quadrature radiance, and its gradient (points, majorant
    and draw probabilities held fixed) the central finite differences of it."""
    p = _positive_field()
    o = np.array([0.5, 0.5, -1.0])
    v = np.array([0.0, 0.03, 1.0])
    v /= np.linalg.norm(v)
    I_ref, kap = _nested_radiance(p, o, v)
    assert kap.min() >= 0.0 and I_ref > 1e-3
    f = oracle.Field(p, omega_frame="local", k_sigma=6.0)
    ro = oracle.render_opts("scatter", 1, 1, 0.8)
    vals, grads = [], []
    for seed in range(12):
        val, g = f.radiance_grad_rays(o[None], v[None], ro, 2000, seed, dLdI=np.ones(1))
        vals.append(val[0])
        grads.append(g)
    vals = np.array(vals)
    grads = np.array(grads)
    se = vals.std(ddof=1) / math.sqrt(len(vals))
    assert abs(vals.mean() - I_ref) < 4.5 * se + 1e-6, (vals.mean(), I_ref, se)
    gm = grads.mean(0)
    gse = grads.std(0, ddof=1) / math.sqrt(len(grads))
    N = 4
    offs = {"mu": 0, "quat": 3 * N, "log_scale": 7 * N, "omega": 10 * N, "phase": 13 * N,
            "weight": 14 * N}
    checks = [("mu", 0), ("log_scale", 1), ("weight", 0), ("mu", 4), ("quat", 4),
              ("log_scale", 5), ("omega", 3), ("phase", 1), ("weight", 1), ("mu", 8),
              ("phase", 2)]
    for key, j in checks:
        base = float(p[key].reshape(-1)[j])
        h = 1e-3 * max(abs(base), 0.5)
        pp = {k: v_.copy() for k, v_ in p.items()}
        pm = {k: v_.copy() for k, v_ in p.items()}
        pp[key].reshape(-1)[j] = np.float32(base + h)
        pm[key].reshape(-1)[j] = np.float32(base - h)
        step = float(pp[key].reshape(-1)[j]) - float(pm[key].reshape(-1)[j])
        fd = (_nested_radiance(pp, o, v)[0] - _nested_radiance(pm, o, v)[0]) / step
        an, s_ = gm[offs[key] + j], gse[offs[key] + j]
        assert abs(an - fd) < 4.5 * s_ + 2e-3 * abs(fd) + 1e-6, (key, j, an, fd, s_)


@pytest.mark.parametrize("freq,cone,beta,delta", [(4, 0, 0.3, 0.0), (5, 2, 0.5, 0.0),
                                                  (6, 1, 0.2, 0.0), (2, 4, 0.0, 0.5),
                                                  (3, 4, 0.0, 0.3), (6, 4, 0.6, 0.4)])
def test_strategy_weights_are_reciprocal_probabilities(freq, cone, beta, delta):
    """Power-law (with and without control variate, accumulating) and threshold +
    uniform strategies of the App. B tables: every occupied cell's mean of
    w * 1[selected] is 1, and power-law levels occur with probability
    ((j+1)/n)^(1-beta) - (j/n)^(1-beta)."""
    f, p = _small_octave(n=5460, octaves=6)
    occ, _ = f.cells()
    lod = oracle.Lod(freq, 7, cone, beta, delta)
    v = np.array([0.3, -0.5, 0.81]); v /= np.linalg.norm(v)
    n = 30000
    acc = np.zeros(64)
    sq = np.zeros(64)
    levels = np.zeros(8)
    for r in range(n):
        m, w = f.sample_mask(lod, v, seed=5, ray=r, sample=0, bounce=0, tag=oracle.TAG_MASK)
        bits = np.array([(m >> c) & 1 for c in range(64)], bool)
        x = np.where(bits, w, 0.0)
        acc += x
        sq += x * x
        gab = [b for b in range(1, 8) if any((m >> c) & 1 for c in range(1 + 8 * (b - 1), 9 + 8 * (b - 1)))]
        if freq in (4, 5):
            if freq == 4 and m & 1 and not gab:
                levels[0] += 1
            for b in gab:
                levels[b] += 1
        # the stated weights, exactly: 1/P(level) for a single level, 1/P(level kept)
        # when accumulating (the weight of a band, before the cone factor)
        nb = 6 if freq in (3, 4) else 5
        b32 = float(np.float32(beta))  # the descriptor holds beta as a float
        for b in gab:
            c = next(c for c in range(1 + 8 * (b - 1), 9 + 8 * (b - 1)) if (m >> c) & 1)
            j = b if freq in (3, 4) else b - 1
            if freq in (4, 5):
                wb = 1.0 / (((j + 1) / nb) ** (1 - b32) - (j / nb) ** (1 - b32))
            elif freq == 6:
                wb = 1.0 / (1.0 - (j / nb) ** (1 - b32))
            else:
                wb = float(nb)
            ratio = w[c] / wb
            if cone == 0:
                assert ratio == pytest.approx(1.0, rel=1e-12)
            elif cone in (2, 4):
                assert ratio == pytest.approx(round(ratio), rel=1e-12) or ratio == pytest.approx(1.0)
    cells = [c for c in range(64) if (occ >> c) & 1]
    for c in cells:
        mean = acc[c] / n
        se = math.sqrt(max(sq[c] / n - mean * mean, 0.0) / n)
        assert abs(mean - 1.0) < 5 * se + 1e-9, (c, mean, se)
    if freq in (4, 5):
        nb = 6 if freq == 4 else 5
        first = 0 if freq == 4 else 1
        for j in range(nb):
            pj = ((j + 1) / nb) ** (1 - beta) - (j / nb) ** (1 - beta)
            sd = math.sqrt(pj * (1 - pj) / n)
            assert abs(levels[first + j] / n - pj) < 5 * sd, (j, levels[first + j] / n, pj)


def test_threshold_culling_keeps_perpendicular_bins():
    """Threshold culling (App. B orientation table): a Gabor band keeps exactly the
    bins with |v . o| <= delta, weight 1; with none below the threshold, the
    least aligned bin (largest contribution weight)."""
    f, p = _small_octave(n=5460, octaves=6)
    occ, _ = f.cells()
    axes = []
    for k in range(8):
        z = 1 - (k + 0.5) / 8; r_ = math.sqrt(1 - z * z); ph = k * math.pi * (3 - math.sqrt(5))
        axes.append((r_ * math.cos(ph), r_ * math.sin(ph), z))
    rng = np.random.default_rng(4)
    for t in range(20):
        v = rng.standard_normal(3); v /= np.linalg.norm(v)
        delta = float(rng.uniform(0.0, 0.8))
        m, w = f.sample_mask(oracle.Lod(0, 7, 3, 0.0, delta), v, seed=1, ray=t, sample=0,
                             bounce=0, tag=oracle.TAG_MASK)
        a = [abs(np.float32(v[0]) * np.float32(ax[0]) + np.float32(v[1]) * np.float32(ax[1])
                 + np.float32(v[2]) * np.float32(ax[2])) for ax in axes]
        for b in range(1, 6):
            cells = [1 + 8 * (b - 1) + k for k in range(8) if (occ >> (1 + 8 * (b - 1) + k)) & 1]
            keep = {c for c in cells if a[(c - 1) % 8] <= np.float32(delta)}
            if not keep:
                keep = {min(cells, key=lambda c: a[(c - 1) % 8])}
            got = {c for c in cells if (m >> c) & 1}
            assert got == keep, (t, b, got, keep)
            assert all(w[c] == 1.0 for c in got)
        assert m & 1 and w[0] == 1.0


# --------------------------------------------------------------------------- adaptive clamping
def _field_of(params, **kw):
    return oracle.Field(params, omega_frame=params.get("omega_frame", "world"), **kw)


def test_adaptive_clamping_gaussian_tail_bound():
    """Sec. 4.4 adaptive clamping: a Gaussian's line integral through any point
    at whitened radius r carries at most rho exp(-r^2/2), rho = |A| sqrt(2 pi)
    s_max, so clamping the support at the radius E where rho exp(-E^2/2) = eps
    removes at most eps from any ray's optical depth and never adds to it.  On
    the central ray along the longest axis, E ~ 2 removes rho erfc(E/sqrt 2),
    about a third of eps: both bounds are checked on random and axial rays."""
    rng = np.random.default_rng(31)
    for trial in range(6):
        s = np.exp(rng.uniform(np.log(0.02), np.log(0.1), 3))
        A = rng.uniform(0.5, 2.0)
        rho = A * math.sqrt(2 * math.pi) * s.max()
        eps = rho * math.exp(-0.5 * 2.0 ** 2)  # E = 2 (< k = 3: the clamp is active)
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        p = {"mu": np.array([[0.5, 0.5, 0.5]], np.float32), "quat": q[None].astype(np.float32),
             "log_scale": np.log(s)[None].astype(np.float32),
             "omega": np.zeros((1, 3), np.float32), "phase": np.zeros(1, np.float32),
             "weight": np.array([A], np.float32)}
        full = oracle.Field(p, k_sigma=6.0)
        cl = oracle.Field(p, k_sigma=6.0, clamp_eps=eps)
        assert abs(cl.extents()[0] - 2.0) < 1e-5  # float32 inputs
        _, R, sg = _geom(p)
        ax = R[:, int(np.argmax(sg))]
        rays = [(np.array([0.5, 0.5, 0.5]) - ax, ax)]
        for _ in range(40):
            rays.append(_ray_near(rng, [0.5, 0.5, 0.5], 1.5 * s.max()))
        for j, (o, v) in enumerate(rays):
            d = full.chord_integral(0, o, v) - cl.chord_integral(0, o, v)
            assert -1e-15 <= d <= eps * (1 + 1e-6), (trial, j, d, eps)
            if j == 0:
                assert d >= 0.25 * eps, (d, eps)


def test_adaptive_clamping_limits_and_frequency():
    """eps -> 0 leaves every support at k and every optical depth unchanged;
    supports never exceed k and shrink as the whitened frequency |k_W| grows
    (the frequency-induced decay term of Sec. 4.4); a kernel whose attenuated
    peak integral is below eps is dropped and contributes nothing."""
    rng = np.random.default_rng(32)
    p = synth.octave_field(400, 4, seed=3)
    o, d, tr = synth.random_rays(64, seed=4)
    f0 = _field_of(p)
    ft = _field_of(p, clamp_eps=1e-300)
    assert np.all(ft.extents() == 3.0)
    assert np.array_equal(ft.transmittance(o, d, tr)[1], f0.transmittance(o, d, tr)[1])
    f2 = _field_of(p, clamp_eps=1e-2)
    e = f2.extents()
    assert np.all((e >= 0) & (e <= 3.0)) and e.min() < 2.5
    # one Gabor at increasing carrier frequency along its longest axis
    base = {"mu": np.array([[0.5, 0.5, 0.5]], np.float32), "quat": np.array([[1, 0, 0, 0]], np.float32),
            "log_scale": np.log(np.array([[0.05, 0.03, 0.02]])).astype(np.float32),
            "phase": np.zeros(1, np.float32), "weight": np.array([1.0], np.float32)}
    ext = []
    for w in (0.0, 0.5, 1.0, 1.5, 2.0, 2.5, 3.0):
        q = dict(base, omega=np.array([[w / 0.05, 0, 0]], np.float32))  # |k_W| = w
        ext.append(oracle.Field(q, k_sigma=3.0, clamp_eps=2e-3).extents()[0])
    assert all(a > b for a, b in zip(ext, ext[1:]) if b > 0) and ext[0] < 3.0
    assert ext[-1] == 0.0
    q = dict(base, omega=np.array([[3.0 / 0.05, 0, 0]], np.float32))
    gone = oracle.Field(q, k_sigma=3.0, clamp_eps=2e-3)
    assert gone.chord_integral(0, np.array([0.5, 0.5, -1.0]), np.array([0, 0, 1.0])) == 0.0
    assert not gone.chord(0, np.array([0.5, 0.5, -1.0]), np.array([0, 0, 1.0]))[0]


# --------------------------------------------------------------------------- multiple scattering
def _one_gaussian():
    """One Gaussian (tau ~ 2 through its centre), k = 6 so the cut is negligible."""
    mu = np.array([0.5, 0.5, 0.5])
    s = np.array([0.2, 0.15, 0.12])
    q = np.array([0.9, 0.2, 0.3, 0.1])
    q /= np.linalg.norm(q)
    return {"mu": mu[None].astype(np.float32), "quat": q[None].astype(np.float32),
            "log_scale": np.log(s)[None].astype(np.float32), "omega": np.zeros((1, 3), np.float32),
            "phase": np.zeros(1, np.float32), "weight": np.array([6.0], np.float32)}


def _two_bounce_quadrature(p, o, v, albedo=0.8):
    """First- and second-bounce radiance along the ray o + t v through one
    Gaussian (Sec. 3 path integral, isotropic phase, NEE to the light at every
    collision), every transmittance in closed form (erf):
      L1 = a E/(4 pi) int dt1 kappa(x1) T(o,x1) T_l(x1)
      L2 = a^2 E/(4 pi) int dt1 kappa(x1) T(o,x1) int dw/(4 pi) int dt2 kappa(x2) T(x1,x2) T_l(x2)
    by Gauss-Legendre in t1 and t2 and a 32 x 64 product rule over directions."""
    f = oracle.Field(p, k_sigma=6.0)
    Si, _, _ = _geom(p)
    muf, A = p["mu"][0].astype(np.float64), float(p["weight"][0])

    def depth(x, w, t0, t1):  # int_t0^t1 A exp(-q(x + s w)/2) ds, broadcast over leading axes
        d = x - muf
        a = np.einsum("...i,ij,...j->...", w, Si, w)
        b = np.einsum("...i,ij,...j->...", w, Si, d)
        g = np.einsum("...i,ij,...j->...", d, Si, d)
        c = np.sqrt(a / 2)
        return A * np.exp(-(g - b * b / a) / 2) * np.sqrt(np.pi / (2 * a)) * (
            special.erf(c * (t1 + b / a)) - special.erf(c * (t0 + b / a)))

    def kappa(x):
        d = x - muf
        return A * np.exp(-0.5 * np.einsum("...i,ij,...j->...", d, Si, d))

    light = np.array([1.0, 1.0, -1.0]) / math.sqrt(3.0)
    _, lo, hi = f.chord(0, o, v)
    xn, wn = np.polynomial.legendre.leggauss(40)
    t1 = 0.5 * (hi - lo) * xn + 0.5 * (hi + lo)
    w1 = 0.5 * (hi - lo) * wn
    X1 = o[None] + t1[:, None] * v[None]
    first = w1 * kappa(X1) * np.exp(-depth(np.broadcast_to(o, X1.shape), np.broadcast_to(v, X1.shape), 0.0, t1))
    L1 = albedo / (4 * np.pi) * np.sum(first * np.exp(-depth(X1, np.broadcast_to(light, X1.shape), 0.0, np.inf)))
    mn, mw = np.polynomial.legendre.leggauss(32)
    ph = (np.arange(64) + 0.5) * 2 * np.pi / 64
    M, P = np.meshgrid(mn, ph, indexing="ij")
    W = np.stack([np.sqrt(1 - M ** 2) * np.cos(P), np.sqrt(1 - M ** 2) * np.sin(P), M], -1).reshape(-1, 3)
    Ww = (mw[:, None] * np.full(64, 2 * np.pi / 64)[None]).reshape(-1)  # sums to 4 pi
    un, uw = np.polynomial.legendre.leggauss(48)
    L2 = 0.0
    for i in range(len(t1)):
        d = X1[i] - muf
        a = np.einsum("ki,ij,kj->k", W, Si, W)
        b = np.einsum("ki,ij,j->k", W, Si, d)
        texit = (-b + np.sqrt(b * b - a * (d @ Si @ d - 36.0))) / a  # leave the 6-sigma support
        T2 = 0.5 * texit[:, None] * (un[None] + 1)
        X2 = X1[i][None, None] + T2[..., None] * W[:, None, :]
        inner = np.sum(0.5 * texit[:, None] * uw[None] * kappa(X2)
                       * np.exp(-depth(np.broadcast_to(X1[i], X2.shape), np.broadcast_to(W[:, None, :], X2.shape), 0.0, T2))
                       * np.exp(-depth(X2, np.broadcast_to(light, X2.shape), 0.0, np.inf)), axis=1)
        L2 += first[i] * np.sum(Ww * inner) / (4 * np.pi)
    L2 *= albedo * albedo / (4 * np.pi)
    return L1, L2


def test_multiple_scatter_adjoint_matches_nested_quadrature():
    """The multiple-scattering radiance adjoint (max_bounces = 2: the renderer's
    delta-tracking path differentiated through each segment's accepted point and
    each NEE product, points and majorants held fixed) on one Gaussian: its
    samples are the renderer's samples (same streams, same decisions), their
    mean is the nested-quadrature radiance L1 + L2, and its gradient the central
    finite differences of that quadrature, within 4.5 standard errors, on the
    mean, rotation, scales and weight."""
    p = _one_gaussian()
    f = oracle.Field(p, k_sigma=6.0)
    # the adjoint follows the render's paths: pixel values equal on a small image
    cam = oracle.camera((1.4, 0.3, -0.5), (0.58, 0.44, 0.5), (0, 1, 0), 12.0, 6, 5)
    ro3 = oracle.render_opts("scatter", 3, 3, 0.8)
    img, _ = f.radiance_grad(cam, ro3, 9)
    assert np.abs(img - f.render(cam, ro3, 9)).max() <= 1e-12 * max(1.0, np.abs(img).max())
    o = np.array([1.4, 0.3, -0.5])
    v = np.array([0.58, 0.44, 0.5]) - o
    v /= np.linalg.norm(v)
    L1, L2 = _two_bounce_quadrature(p, o, v)
    ro = oracle.render_opts("scatter", 1, 2, 0.8)
    vals, grads = [], []
    for seed in range(16):
        val, g = f.radiance_grad_rays(o[None], v[None], ro, 16000, seed, dLdI=np.ones(1))
        vals.append(val[0])
        grads.append(g)
    vals, grads = np.array(vals), np.array(grads)
    se = vals.std(ddof=1) / math.sqrt(len(vals))
    assert abs(vals.mean() - (L1 + L2)) < 4.5 * se, (vals.mean(), L1 + L2, se)
    assert L2 > 20 * se  # the second bounce is resolved
    gm = grads.mean(0)
    gse = grads.std(0, ddof=1) / math.sqrt(len(grads))
    offs = {"mu": 0, "quat": 3, "log_scale": 7, "weight": 14}
    for key, j in (("mu", 0), ("mu", 1), ("mu", 2), ("log_scale", 0), ("log_scale", 2),
                   ("quat", 1), ("quat", 2), ("weight", 0)):
        base = float(p[key].reshape(-1)[j])
        h = 1e-3 * max(abs(base), 0.5)
        pp = {k: v_.copy() for k, v_ in p.items()}
        pm = {k: v_.copy() for k, v_ in p.items()}
        pp[key].reshape(-1)[j] = np.float32(base + h)
        pm[key].reshape(-1)[j] = np.float32(base - h)
        step = float(pp[key].reshape(-1)[j]) - float(pm[key].reshape(-1)[j])
        fd = (sum(_two_bounce_quadrature(pp, o, v)) - sum(_two_bounce_quadrature(pm, o, v))) / step
        an, s_ = gm[offs[key] + j], gse[offs[key] + j]
        assert abs(an - fd) < 4.5 * s_ + 2e-3 * abs(fd) + 1e-6, (key, j, an, fd, s_)


@pytest.mark.parametrize("flight", ["delta", "cdf"])
def test_second_bounce_matches_nested_quadrature(flight):
    """Multiple scattering (Sec. 3 path integral with delta tracking, isotropic
    phase, NEE at every collision): on one Gaussian (tau ~ 2 through its
    centre, k = 6 so the cut is negligible) the second-bounce radiance of a
    pixel, the oracle's 2-bounce minus 1-bounce render under shared streams,
    equals the nested quadrature
      a^2 E/(4 pi) int dt1 kappa(x1) T(o,x1) int dw/(4 pi) int dt2 kappa(x2) T(x1,x2) T_l(x2)
    with every transmittance in closed form (scipy erf), within 4.5 standard errors."""
    mu = np.array([0.5, 0.5, 0.5])
    s = np.array([0.2, 0.15, 0.12])
    q = np.array([0.9, 0.2, 0.3, 0.1])
    q /= np.linalg.norm(q)
    p = {"mu": mu[None].astype(np.float32), "quat": q[None].astype(np.float32),
         "log_scale": np.log(s)[None].astype(np.float32), "omega": np.zeros((1, 3), np.float32),
         "phase": np.zeros(1, np.float32), "weight": np.array([6.0], np.float32)}
    f = oracle.Field(p, k_sigma=6.0)
    Si, _, _ = _geom(p)
    muf, A = p["mu"][0].astype(np.float64), float(p["weight"][0])

    def depth(x, w, t0, t1):  # int_t0^t1 A exp(-q(x + s w)/2) ds, broadcast over leading axes
        d = x - muf
        a = np.einsum("...i,ij,...j->...", w, Si, w)
        b = np.einsum("...i,ij,...j->...", w, Si, d)
        g = np.einsum("...i,ij,...j->...", d, Si, d)
        c = np.sqrt(a / 2)
        return A * np.exp(-(g - b * b / a) / 2) * np.sqrt(np.pi / (2 * a)) * (
            special.erf(c * (t1 + b / a)) - special.erf(c * (t0 + b / a)))

    def kappa(x):
        d = x - muf
        return A * np.exp(-0.5 * np.einsum("...i,ij,...j->...", d, Si, d))

    light = np.array([1.0, 1.0, -1.0]) / math.sqrt(3.0)
    # an oblique camera ray that misses the centre: no symmetry hides a wrong direction law
    cam = oracle.camera((1.4, 0.3, -0.5), (0.58, 0.44, 0.5), (0, 1, 0), 1.0, 64, 64)
    px, py, albedo = 32, 31, 0.8
    o, v = oracle.camera_ray(cam, 5, px, py, 0)  # the pixel spans 3e-4 rad: jitter is negligible
    _, lo, hi = f.chord(0, o, v)
    xn, wn = np.polynomial.legendre.leggauss(40)
    t1 = 0.5 * (hi - lo) * xn + 0.5 * (hi + lo)
    w1 = 0.5 * (hi - lo) * wn
    X1 = o[None] + t1[:, None] * v[None]
    first = w1 * kappa(X1) * np.exp(-depth(np.broadcast_to(o, X1.shape), np.broadcast_to(v, X1.shape), 0.0, t1))
    mn, mw = np.polynomial.legendre.leggauss(32)
    ph = (np.arange(64) + 0.5) * 2 * np.pi / 64
    M, P = np.meshgrid(mn, ph, indexing="ij")
    W = np.stack([np.sqrt(1 - M ** 2) * np.cos(P), np.sqrt(1 - M ** 2) * np.sin(P), M], -1).reshape(-1, 3)
    Ww = (mw[:, None] * np.full(64, 2 * np.pi / 64)[None]).reshape(-1)  # sums to 4 pi
    un, uw = np.polynomial.legendre.leggauss(48)
    L2 = 0.0
    for i in range(len(t1)):
        d = X1[i] - muf
        a = np.einsum("ki,ij,kj->k", W, Si, W)
        b = np.einsum("ki,ij,j->k", W, Si, d)
        texit = (-b + np.sqrt(b * b - a * (d @ Si @ d - 36.0))) / a  # leave the 6-sigma support
        T2 = 0.5 * texit[:, None] * (un[None] + 1)
        X2 = X1[i][None, None] + T2[..., None] * W[:, None, :]
        inner = np.sum(0.5 * texit[:, None] * uw[None] * kappa(X2)
                       * np.exp(-depth(np.broadcast_to(X1[i], X2.shape), np.broadcast_to(W[:, None, :], X2.shape), 0.0, T2))
                       * np.exp(-depth(X2, np.broadcast_to(light, X2.shape), 0.0, np.inf)), axis=1)
        L2 += first[i] * np.sum(Ww * inner) / (4 * np.pi)
    L2 *= albedo * albedo / (4 * np.pi)
    spp = 40000
    r1 = f.render(cam, oracle.render_opts("scatter", spp, 1, albedo, free_flight=flight), seed=5,
                  crop=(px, py, 1, 1), samples=True).ravel()
    r2 = f.render(cam, oracle.render_opts("scatter", spp, 2, albedo, free_flight=flight), seed=5,
                  crop=(px, py, 1, 1), samples=True).ravel()
    d2 = r2 - r1
    se = d2.std(ddof=1) / math.sqrt(spp)
    assert abs(d2.mean() - L2) < 4.5 * se, (d2.mean(), L2, se)
    assert L2 > 50 * se  # a resolved second bounce


# --------------------------------------------------------------------------- camera-Nyquist LoD
def test_camera_lod_selection_against_measured_pixel_pitch():
    """Supp. A (LOD Selection): a kernel stays iff its carrier is resolved at
    its depth, |omega| <= pi / (pitch d), with the pixel pitch measured here on
    the camera's own jittered rays (horizontally and vertically, non-square
    image); kernels within 2% of the threshold are not judged."""
    p = synth.absorption_field(400, seed=6)
    p = dict(p, omega=(p["omega"] * 6.0).astype(np.float32))
    f = oracle.Field(p)
    eye, look = np.array([0.3, 0.6, -1.2]), np.array([0.5, 0.5, 0.5])
    W, H, fov = 96, 64, 40.0
    cam = oracle.camera(tuple(eye), tuple(look), (0, 1, 0), fov, W, H)
    fw = (look - eye) / np.linalg.norm(look - eye)
    rt = np.cross([0, 1, 0], fw); rt /= np.linalg.norm(rt)
    up = np.cross(fw, rt)
    pitches = []
    for axis, n, pix in (("x", W, lambda k, s: (k, H // 2)), ("y", H, lambda k, s: (W // 2, k))):
        lo, hi = [], []
        for s in range(400):
            for k, acc in ((0, lo), (n - 1, hi)):
                _, v = oracle.camera_ray(cam, 3, *pix(k, s), s)
                e = rt if axis == "x" else up
                acc.append((v @ e) / (v @ fw))  # image-plane coordinate at unit depth
        span = (max(max(lo), max(hi)) - min(min(lo), min(hi)))  # ~ n pitches
        pitches.append(span / n)
    assert abs(pitches[0] / pitches[1] - 1) < 0.01  # square pixels
    pitch = np.mean(pitches)
    for H2 in (64, 24, 8):
        cam2 = oracle.camera(tuple(eye), tuple(look), (0, 1, 0), fov, W * H2 // H, H2)
        f.set_camera_lod(cam2)
        kept = f.extents() > 0
        pit = pitch * H / H2
        d = np.linalg.norm(p["mu"].astype(np.float64) - eye, axis=1)
        lim = np.pi / (pit * d)
        wn = np.linalg.norm(p["omega"].astype(np.float64), axis=1)
        sure = np.abs(wn / lim - 1) > 0.02
        assert np.array_equal(kept[sure], (wn <= lim)[sure]), H2
        assert 0 < kept.sum() < len(kept) or H2 == 64
    f.set_camera_lod(None)
    assert np.all(f.extents() == 3.0)


def test_camera_lod_selection_limits():
    """A camera that resolves everything leaves every optical depth bit-equal;
    one that resolves no carrier keeps exactly the Gaussian band (the band-0
    cutoff of Sec. 4.5.1), again bit-equal."""
    p = synth.octave_field(500, 4, seed=7)
    o, d, tr = synth.random_rays(48, seed=8)
    f = oracle.Field(p, omega_frame="local")
    base = f.transmittance(o, d, tr)[1]
    g0 = f.transmittance(o, d, tr, lod=oracle.Lod(1, 0, 0))[1]
    c = synth.DEFAULT_CAMERA
    f.set_camera_lod(oracle.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], 1 << 20, 1 << 20))
    assert np.array_equal(f.transmittance(o, d, tr)[1], base)
    f.set_camera_lod(oracle.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], 1, 1))
    assert np.array_equal(f.extents() > 0, f.labels()[0] == 0)
    assert np.array_equal(f.transmittance(o, d, tr)[1], g0)


# --------------------------------------------------------------------------- foveation
def test_foveation_keeps_the_bands_below_the_eccentricity_threshold():
    """Foveation (Supp., Foveated Rendering; reading G23): every sample's path
    keeps the Gaussian band and the Gabor bands whose largest carrier |omega| is
    at most f = max(0, f0 - slope e) (1 + smooth (2 xi - 1)), e the camera ray's
    angle to the gaze ray and xi the camera stream's third uniform.  The
    threshold law is rebuilt here from the camera's own rays and Philox blocks;
    each sample of a foveated render then equals, bit for bit, the same sample
    rendered with the matching band cutoff.  f0 = 0 leaves the Gaussian band
    alone, and an unbounded threshold changes nothing."""
    p = synth.octave_field(2000, 4, seed=6)
    f = oracle.Field(p, omega_frame="local")
    band = f.labels()[0]
    wn = np.array([np.linalg.norm(f.prim(i)[1]) for i in range(f.n)])
    bmax = np.array([wn[band == b].max() if np.any(band == b) else 0.0 for b in range(8)])
    assert np.all(np.diff(bmax[:4]) > 0)  # octaves: carriers grow band by band
    c = synth.DEFAULT_CAMERA
    W = H = 12
    cam = oracle.camera(c["eye"], c["look_at"], c["up"], 30.0, W, H)
    gaze = (3.5, 8.0)
    f0, slope, smooth = 1.1 * bmax[3], 1.1 * bmax[3] / 0.25, 0.3
    fov = {"gaze": gaze, "f0": f0, "slope": slope, "smooth": smooth}
    spp, seed = 4, 5
    ro = oracle.render_opts("scatter", spp, 2, foveation=fov)
    got = f.render(cam, ro, seed, samples=True)
    cuts = [f.render(cam, oracle.render_opts("scatter", spp, 2), seed, lod=oracle.Lod(1, k, 0),
                     samples=True) for k in range(4)]
    # the gaze ray and each sample's threshold, from the camera's float fields
    eye = np.array(cam.eye[:], np.float64)
    fw = np.array(cam.look_at[:], np.float64) - eye
    fw /= np.linalg.norm(fw)
    rt = np.cross(np.array(cam.up[:], np.float64), fw)
    rt /= np.linalg.norm(rt)
    uv = np.cross(fw, rt)
    th = math.tan(0.5 * float(cam.vfov_deg) * math.pi / 180.0)
    g = fw + (2 * float(np.float32(gaze[0])) / W - 1) * th * (W / H) * rt + \
        (1 - 2 * float(np.float32(gaze[1])) / H) * th * uv
    g /= np.linalg.norm(g)
    seen = set()
    for py in range(H):
        for px in range(W):
            for s in range(spp):
                _, v = oracle.camera_ray(cam, seed, px, py, s)
                e = math.acos(min(1.0, max(-1.0, float(v @ g))))
                word = oracle.stream_word(s, 0, oracle.TAG_CAMERA)
                xi = (oracle.philox4x32_10([0, 0xFFFFFFFF, py * W + px, word], [seed, 0])[2] >> 8) / 2.0 ** 24
                thr = max(0.0, f0 - slope * e) * (1 + smooth * (2 * xi - 1))
                k = max(b for b in range(4) if bmax[b] <= thr or b == 0)
                if min(abs(thr - bmax[b]) for b in range(1, 4)) < 1e-9 * bmax[3]:
                    continue  # a threshold on a band's carrier: FP rounding decides
                seen.add(k)
                assert got[py, px, s] == cuts[k][py, px, s], (px, py, s, k)
    assert seen == {0, 1, 2, 3}  # every regime occurs in the frame
    zero = f.render(cam, oracle.render_opts("scatter", spp, 2, foveation=dict(fov, f0=0.0)), seed)
    assert np.array_equal(zero, cuts[0].mean(-1))
    wide = f.render(cam, oracle.render_opts("scatter", spp, 2, foveation=dict(fov, f0=1e30, slope=0.0)), seed)
    assert np.array_equal(wide, f.render(cam, oracle.render_opts("scatter", spp, 2), seed))


# --------------------------------------------------------------------------- uniform-in-segment free flight
def test_segment_free_flight_samples_the_crossing_segment_uniformly():
    """Free flight by uniform sampling within the crossing segment (Sec. 3: the
    cheap approximation of the CDF inversion).  The segments are rebuilt here
    from the chords (entries and exits, and the ray start) and their optical
    depths from a trapezoid integral of the density: every sample lies in the
    segment where tau first reaches its own -ln(1 - xi), at exactly
    e_a + u (e_b - e_a) with u its stream's second uniform; rays whose whole
    tau stays below the target escape; and the segments' frequencies follow
    the CDF increments exp(-tau(e_a)) - exp(-tau(e_b)) (chi^2)."""
    p = _gauss_only()
    f = oracle.Field(p)
    o = np.array([0.5, 0.5, -0.5]); v = np.array([0.0, 0.0, 1.0])
    ev = [0.0]
    for i in range(f.n):
        has, lo, hi = f.chord(i, o, v)
        if has:
            ev += [lo, hi]
    ev = np.unique(np.array(ev))
    assert len(ev) >= 5  # several overlapping chords: several segments
    grid = np.linspace(0.0, 2.0, 40001)
    kap = np.array([f.density(o + t * v) for t in grid])
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (kap[1:] + kap[:-1]) * np.diff(grid))])
    tau_e = np.interp(ev, grid, cum)
    word = oracle.stream_word(0, 0, oracle.TAG_TRACK)
    n = 4000
    seg = np.full(n, -1)
    for r in range(n):
        h, t = f.segment_flight(o, v, seed=3, ray=r, word=word)
        x = oracle.philox4x32_10([0, 0xFFFFFFFF, r, word], [3, 0])
        xi, u = (x[0] >> 8) / 2.0 ** 24, (x[1] >> 8) / 2.0 ** 24
        target = -math.log1p(-xi)
        k = int(np.searchsorted(tau_e, target))  # first event with tau >= target
        if k >= len(ev):
            assert not h, r
            continue
        if abs(tau_e[k] - target) < 1e-6 or abs(tau_e[k - 1] - target) < 1e-6:
            continue  # within the trapezoid rule's error of a segment end
        assert h, r
        assert abs(t - (ev[k - 1] + u * (ev[k] - ev[k - 1]))) < 1e-12, (r, t, ev[k - 1], ev[k], u)
        seg[r] = k
    probs = np.exp(-tau_e[:-1]) - np.exp(-tau_e[1:])
    counts = np.array([np.sum(seg == k) for k in range(1, len(ev))])
    keep = probs * n > 5
    chi2 = np.sum((counts[keep] - n * probs[keep]) ** 2 / (n * probs[keep]))
    assert chi2 < stats.chi2.ppf(0.9999, max(1, keep.sum() - 1))


# --------------------------------------------------------------------------- CDF-inversion free flight
def test_cdf_inversion_free_flight_distribution():
    """Free flight by inversion of the optical-depth CDF (Sec. 3, Sec. 4.4): on a
    non-negative field the sampled distance has CDF 1 - exp(-tau(0, t)) (chi^2
    against a trapezoid integral of the density), each sample solves
    tau(0, t) = -ln(1 - xi) with xi its own stream's first uniform, and a ray
    whose whole optical depth is below the target escapes."""
    p = _gauss_only()
    f = oracle.Field(p)
    o = np.array([0.5, 0.5, -0.5]); v = np.array([0.0, 0.0, 1.0])
    grid = np.linspace(0.0, 2.0, 40001)
    kap = np.array([f.density(o + t * v) for t in grid])
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (kap[1:] + kap[:-1]) * np.diff(grid))])
    edges = np.linspace(0.6, 1.4, 17)
    Fe = 1 - np.exp(-np.interp(edges, grid, cum))
    probs = np.concatenate([[Fe[0]], np.diff(Fe), [1 - Fe[-1]]])
    n = 4000
    word = oracle.stream_word(0, 0, oracle.TAG_TRACK)
    hits = []
    for r in range(n):
        h, t = f.cdf_flight(o, v, seed=2, ray=r, word=word)
        hits.append(t if h else np.inf)
        if r < 40:
            xi = (oracle.philox4x32_10([0, 0xFFFFFFFF, r, word], [2, 0])[0] >> 8) / 2.0 ** 24
            if h:
                tau_t = np.interp(t, grid, cum)
                assert abs(tau_t + math.log1p(-xi)) < 1e-4, (r, tau_t, xi)
            else:
                assert cum[-1] < -math.log1p(-xi) + 1e-4
    hits = np.array(hits)
    counts = np.concatenate([[np.sum(hits < edges[0])], np.histogram(hits, edges)[0],
                             [np.sum(hits >= edges[-1])]])
    keep = probs * n > 5
    chi2 = np.sum((counts[keep] - n * probs[keep]) ** 2 / (n * probs[keep]))
    assert chi2 < stats.chi2.ppf(0.9999, keep.sum() - 1)
