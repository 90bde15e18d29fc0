"""gf_transmittance_static: the transmittance call for callers that cannot allocate.

Callers that are not allowed to call cudaMalloc at call time (an external
memory manager owns the device, the allocation budget is used up, or only host
arrays are available) use gf_transmittance_static, whose scratch is a fixed
8 MiB device array inside the library.  This file runs last so that, if it
fails, a run stopping at the first failure has already run every other test;
it also passes on its own in a fresh process (it builds and loads the library
itself).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_05081_gb300 import _abi, api
    return _abi, api


def test_static_scratch_transmittance_matches_the_allocating_call(lib):
    """Every mode (Gauss-Legendre, closed form, ratio tracking) through the
    static scratch equals gf_transmittance within 1e-5, on two calls in a row,
    with device buffers, host buffers, and host inputs with device outputs;
    the field's device error word stays clear after each call; and, once the
    library's kernels are loaded, the calls leave the device's free memory
    unchanged (nothing is allocated)."""
    _abi, api = lib
    ctx = api.Context(0)
    p = synth.absorption_field(256, seed=0)
    field = api.Field(ctx, p)
    o, d, tr = synth.orthographic_rays(64)
    n = o.shape[0]
    dev = torch.device("cuda", 0)
    od, dd, trd = (torch.from_numpy(a).to(dev) for a in (o, d, tr))
    modes = ((_abi.GF_TR_DETERMINISTIC, 1), (_abi.GF_TR_CLOSED_FORM, 1),
             (_abi.GF_TR_RATIO_TRACKING, 2))
    refs = {}
    for mode, spp in modes:
        ref_T = torch.empty(n, device=dev)
        ref_tau = torch.empty(n, device=dev)
        _abi.gf_transmittance(field.h, od, dd, trd, n, mode, spp, 5, ref_T, ref_tau)
        field.sync()
        refs[mode] = (ref_T.cpu().numpy(), ref_tau.cpu().numpy())
    # load every kernel the static calls use, then hold the device's free memory
    Tw = torch.empty(n, device=dev)
    for mode, spp in modes:
        _abi.gf_transmittance_static(field.h, od, dd, trd, n, mode, spp, 5, Tw, None)
    field.sync()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    outs = {k: (torch.full((n,), -1.0, device=dev), torch.full((n,), -1.0, device=dev))
            for k in range(2)}
    for mode, spp in modes:
        ref, ref_tau = refs[mode]
        det = mode != _abi.GF_TR_RATIO_TRACKING
        # two calls in a row through the static scratch: device buffers, host buffers,
        # then host inputs with device outputs
        for call in range(2):
            T, tau = outs[call]
            T.fill_(-1.0)
            tau.fill_(-1.0)
            _abi.gf_transmittance_static(field.h, od, dd, trd, n, mode, spp, 5, T, tau)
            field.sync()
            assert np.abs(T.cpu().numpy() - ref).max() <= 1e-5, (mode, call)
            if det:
                assert np.abs(tau.cpu().numpy() - ref_tau).max() <= 1e-5, (mode, call)
            Th = np.full(n, -1.0, np.float32)
            tauh = np.full(n, -1.0, np.float32)
            _abi.gf_transmittance_static(field.h, o, d, tr, n, mode, spp, 5, Th, tauh)
            field.sync()
            assert np.abs(Th - ref).max() <= 1e-5, (mode, call)
            if det:
                assert np.abs(tauh - ref_tau).max() <= 1e-5, (mode, call)
            T.fill_(-1.0)
            _abi.gf_transmittance_static(field.h, o, d, tr, n, mode, spp, 5, T, None)
            field.sync()
            assert np.abs(T.cpu().numpy() - ref).max() <= 1e-5, (mode, call)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    # sizes beyond the static capacity are refused before any GPU work
    big = 200001
    with pytest.raises(_abi.GfError) as e:
        _abi.gf_transmittance_static(field.h, np.zeros(3 * big, np.float32),
                                     np.ones(3 * big, np.float32), None, big,
                                     _abi.GF_TR_DETERMINISTIC, 1, 0, np.zeros(big, np.float32))
    assert e.value.status == _abi.GF_EINVAL
    field.free()
    ctx.close()
