"""Render server (gf_server_*): continuous batching over resident fields (GPU).

Each request's image must be the same alone (gf_render on its field) and in
the mix (batched with requests on other fields, other LoD settings, other
sample counts, admitted while others run).  A pixel's samples run in one
lane and the majorant sums are exact in fixed point, so the two are compared
bit for bit; the oracle pins one request of the mix directly.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_05081_gb300 import api as _api
    return _api


@pytest.fixture(scope="module")
def ctx(api):
    c = api.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def assets(api, ctx):
    p0 = synth.octave_field(3000, 4, seed=8)
    p1 = synth.octave_field(5460, 6, seed=9)
    fields = [api.Field(ctx, p0), api.Field(ctx, p1), api.Field(ctx, p0, precision="fp16")]
    yield (p0, p1), fields
    for f in fields:
        f.free()


def _cam(api, w, h, eye=None):
    c = synth.DEFAULT_CAMERA
    return api.camera(eye or c["eye"], c["look_at"], c["up"], c["vfov_deg"], w, h)


# (asset, width, height, spp, bounces, primary lod, nee lod, seed)
MIX = [
    (0, 40, 32, 4, 1, ("cutoff", 3, "all"), ("cutoff", 3, "all"), 11),
    (1, 24, 24, 2, 3, ("unif_cv", 7, "is"), ("unif_cv", 7, "is"), 12),
    (2, 32, 32, 1, 1, ("cutoff", 1, "all"), ("cutoff", 1, "all"), 13),
    (0, 16, 48, 8, 1, ("all", 7, "all"), ("cutoff", 0, "all"), 14),
    (1, 32, 16, 4, 2, ("uniform", 5, "uniform"), ("cutoff", 2, "all"), 15),
    (0, 33, 17, 3, 1, ("cutoff", 2, "is"), ("cutoff", 2, "is"), 16),
    (2, 24, 40, 2, 1, ("all", 7, "all"), ("all", 7, "all"), 17),
    (1, 48, 24, 1, 1, ("cutoff", 4, "all"), ("cutoff", 4, "all"), 18),
]


def _lod(api, d):
    return api.lod(d[0], d[1], d[2])


def test_server_images_equal_alone_and_in_the_mix(api, ctx, assets):
    _, fields = assets
    # room for three of the largest framebuffers (64-bit sums and floats, 12 bytes
    # per pixel, each part 256-byte aligned): admission is limited by memory
    def fb(w, h):
        return ((w * h * 8 + 255) // 256 + (w * h * 4 + 255) // 256) * 256
    budget = 3 * fb(48, 24)
    srv = api.Server(ctx, fields, mem_budget=budget, max_inflight=8, batch_samples=1024)
    try:
        tickets = []
        for (a, w, h, spp, nb, lp, ln, seed) in MIX:
            ro = api.render_opts("scatter", spp, nb)
            t, out = srv.submit(a, _cam(api, w, h), ro, _lod(api, lp), _lod(api, ln), seed)
            tickets.append((t, out))
        res = [srv.wait(t) for t, _ in tickets]
        st = srv.stats()
    finally:
        srv.close()
    assert all(r["state"] == 2 and r["status"] == 0 for r in res), res
    assert st["completed"] == len(MIX) and st["failed"] == 0
    # the first three requests fill the pool (15360 + 6912 + 12288 bytes of the
    # 41472; the fourth's 9216 would not fit), later ones join as memory frees up
    assert 3 <= st["max_inflight_seen"] <= 8, st
    assert st["max_bytes_seen"] <= budget
    # requests were split over several launches and shared them
    assert sum(r["launches"] for r in res) > st["launches"] >= max(r["launches"] for r in res) > 1
    for (a, w, h, spp, nb, lp, ln, seed), (t, out) in zip(MIX, tickets):
        f = fields[a]
        f.set_lod(_lod(api, lp), _lod(api, ln))
        alone = f.render(_cam(api, w, h), api.render_opts("scatter", spp, nb), seed=seed)
        f.sync()
        mixed = out.numpy()
        assert mixed.shape == (h, w)
        np.testing.assert_array_equal(mixed, alone.cpu().numpy())
        assert np.isfinite(mixed).all() and mixed.max() > 0.0


def test_server_request_matches_oracle(api, ctx, assets):
    (p0, _), fields = assets
    srv = api.Server(ctx, fields, mem_budget=1 << 20, max_inflight=4, batch_samples=512)
    try:
        ro = api.render_opts("scatter", 8, 1)
        lp = api.lod("cutoff", 2)
        t0, _ = srv.submit(1, _cam(api, 32, 32), api.render_opts("scatter", 2, 2), seed=3)
        t, out = srv.submit(0, _cam(api, 20, 20), ro, lp, lp, seed=5)
        r = srv.wait(t)
        srv.wait(t0)
    finally:
        srv.close()
    assert r["state"] == 2
    c = synth.DEFAULT_CAMERA
    co = oracle.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], 20, 20)
    orc = oracle.Field(p0, omega_frame="local")
    lo = oracle.Lod(1, 2, 0)
    smp = orc.render(co, oracle.render_opts("scatter", 8, 1), seed=5, lod=lo, lod_nee=lo,
                     samples=True)
    ref = smp.mean(-1)
    sig = smp.std(-1, ddof=1) / math.sqrt(smp.shape[-1])
    diff = np.sqrt(np.mean((out.numpy() - ref) ** 2))
    noise = np.sqrt(np.mean(sig ** 2))
    assert ref.max() > 1e-3
    assert diff <= 0.01 * noise, (diff, noise)


def test_server_admission_queue_and_errors(api, ctx, assets):
    from paper_2602_05081_gb300 import _abi
    _, fields = assets
    full = 64 * 64 * 12  # one 64x64 framebuffer: 64-bit sums and floats
    srv = api.Server(ctx, fields[:1], mem_budget=full, max_inflight=2, max_queue=3,
                     batch_samples=256)
    try:
        ro = api.render_opts("scatter", 1, 1)
        # a framebuffer larger than the whole pool can never be admitted
        with pytest.raises(_abi.GfError) as e:
            srv.submit(0, _cam(api, 65, 64), ro)
        assert e.value.status == _abi.GF_EINVAL
        with pytest.raises(_abi.GfError) as e:
            srv.submit(1, _cam(api, 8, 8), ro)  # no such asset
        assert e.value.status == _abi.GF_EINVAL
        with pytest.raises(_abi.GfError) as e:
            srv.submit(0, _cam(api, 8, 8), api.render_opts("tomo", 1))
        assert e.value.status == _abi.GF_EINVAL
        with pytest.raises(_abi.GfError) as e:
            srv.submit(0, _cam(api, 8, 8), api.render_opts("scatter", 1, 1, free_flight="cdf"))
        assert e.value.status == _abi.GF_EINVAL
        # a camera LoD selection belongs to one camera: not on a served field
        with pytest.raises(_abi.GfError) as e:
            fields[0].set_lod_camera(_cam(api, 8, 8))
        assert e.value.status == _abi.GF_ESTATE
        # one full-pool request at a time; the queue bound is enforced at submit
        tk = []
        refused = 0
        for k in range(8):
            try:
                tk.append(srv.submit(0, _cam(api, 64, 64), ro, seed=k)[0])
            except _abi.GfError as err:
                assert err.status == _abi.GF_EOVERFLOW
                refused += 1
        res = [srv.wait(t) for t in tk]
        st = srv.stats()
    finally:
        srv.close()
    assert all(r["state"] == 2 for r in res)
    assert st["max_inflight_seen"] == 1
    # a field with a selection cannot be served; without it, again it can
    fields[0].set_lod_camera(_cam(api, 8, 8))
    with pytest.raises(_abi.GfError) as e:
        api.Server(ctx, fields[:1], mem_budget=full)
    assert e.value.status == _abi.GF_ESTATE
    fields[0].set_lod_camera(None)
    api.Server(ctx, fields[:1], mem_budget=full).close()
    # admissions are in arrival order: each admitted after the previous finished
    for a, b in zip(res, res[1:]):
        assert b["t_admit_ms"] >= a["t_done_ms"] - 1e-3
        assert a["t_submit_ms"] <= a["t_admit_ms"] <= a["t_done_ms"]
    assert len(tk) + refused == 8 and len(tk) >= 3
