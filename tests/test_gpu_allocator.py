"""Device memory through the caller's allocator (GPU).

The library allocates every device buffer it owns through the gf_allocator of
its context (include/gf.h); the Python binding passes one backed by PyTorch's
caching allocator.  After gf_reserve, compute calls within the reserved sizes
allocate nothing at all.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_05081_gb300 import api as _api
    return _api


def _cam(api, w, h):
    c = synth.DEFAULT_CAMERA
    return api.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], w, h)


def test_device_memory_comes_from_the_caller_and_reserved_calls_allocate_nothing(api):
    """With PyTorch's caching allocator behind the context: (1) the device memory
    a field takes (load, build, reserve) is exactly what torch's allocator
    reserved in that time, so nothing bypasses it; (2) after gf_reserve, the
    compute calls (transmittance in all modes with device and host buffers,
    chord lists, scattering and tomography renders into device and host
    images, both adjoints) make no allocator call and leave the device's free
    memory unchanged; (3) freeing the field returns every byte."""
    from paper_2602_05081_gb300 import _abi
    ctx = api.Context(0)
    al = ctx.allocator
    assert isinstance(al, api.TorchAllocator)
    p = synth.octave_field(3000, 4, seed=8)
    o, d, tr = synth.random_rays(512, seed=3)
    od, dd, trd = (torch.from_numpy(a).to(DEV) for a in (o, d, tr))
    n = o.shape[0]
    cam = _cam(api, 32, 32)
    T = torch.empty(n, device=DEV)
    tau = torch.empty(n, device=DEV)
    Th, tauh = np.zeros(n, np.float32), np.zeros(n, np.float32)
    img = torch.empty(32, 32, device=DEV)
    img_h = torch.empty(32, 32).pin_memory()
    dL = torch.ones(32, 32, device=DEV)
    grad = None
    ro_s = api.render_opts("scatter", 4, 2)
    ro_1 = api.render_opts("scatter", 2, 1)
    ro_t = api.render_opts("tomo", 2)
    lo = api.lod("unif_cv", 7, "is")

    def compute(f, grad):
        for mode in ("det", "closed", "rt"):
            f.transmittance(od, dd, trd, mode=mode, spp=2, out_T=T,
                            out_tau=None if mode == "rt" else tau)
            f.transmittance(o, d, tr, mode=mode, spp=2, out_T=Th,
                            out_tau=None if mode == "rt" else tauh)
        f.set_lod(api.lod("cutoff", 3))
        f.chords(o[:64], d[:64], tr[:64], cap=256)
        f.set_lod(lo, lo)
        f.render(cam, ro_s, seed=1, out=img)
        f.render(cam, ro_s, seed=1, out=img_h)
        f.render(cam, ro_t, seed=1, out=img)
        f.render_backward(cam, ro_t, 2, dL, grad=grad)
        f.render_backward(cam, ro_1, 2, dL, grad=grad)
        f.sync()

    def field():
        f = api.Field(ctx, p)
        f.reserve(max_rays=n, max_chords=256, max_pixels=32 * 32, render=True, adjoint=True)
        return f

    # a first cycle loads the library's kernels (their code takes device memory once)
    grad = torch.empty(15 * p["phase"].shape[0], device=DEV)
    f = field()
    compute(f, grad)
    f.free()
    torch.cuda.synchronize()
    free0, res0, live0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved(), al.live_bytes
    f = field()
    torch.cuda.synchronize()
    free1, res1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    assert al.live_bytes > live0
    assert free0 - free1 == res1 - res0, (free0 - free1, res1 - res0)
    calls = al.calls_alloc
    compute(f, grad)
    torch.cuda.synchronize()
    assert al.calls_alloc == calls
    assert torch.cuda.mem_get_info()[0] == free1 and torch.cuda.memory_reserved() == res1
    f.free()
    assert al.live_bytes == live0
    with pytest.raises(_abi.GfError):
        _abi.gf_reserve(f.h if f.h else None, max_rays=-1)
    ctx.close()


def test_failed_allocation_is_reported(api):
    """An allocator that refuses makes the call fail with GF_ENOMEM, cleanly."""
    from paper_2602_05081_gb300 import _abi
    state = {"left": 5}

    def on_alloc(user, nbytes, stream):
        if state["left"] <= 0:
            return None
        state["left"] -= 1
        return torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))

    def on_free(user, ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(int(ptr))

    fa, ff = _abi.ALLOC_FN(on_alloc), _abi.FREE_FN(on_free)
    h = _abi.gf_create_ex(0, _abi.gf_allocator(fa, ff, None))
    p = synth.absorption_field(64, seed=0)
    keep = {k: torch.from_numpy(np.ascontiguousarray(p[k])).to(DEV) for k in
            ("mu", "quat", "log_scale", "omega", "phase", "weight")}
    params = _abi.gf_params(64, *(keep[k].data_ptr() for k in
                                  ("mu", "quat", "log_scale", "omega", "phase", "weight")), None)
    with pytest.raises(_abi.GfError) as e:
        _abi.gf_load_field(h, params, _abi.gf_field_opts(0, 0, 0, 3.0, 0.0))
    assert e.value.status == _abi.GF_ENOMEM
    _abi.gf_destroy(h)
