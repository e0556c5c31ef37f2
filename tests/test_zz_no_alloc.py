"""The allocation-free likelihood entry point gives the results of gb_loglik.

Some callers must not allocate device memory while they run: a plugin whose
host application hands out all device memory through its own pool, or a
latency-critical loop that cannot take the device-wide synchronisation of
cudaMalloc and cudaFree.  gb_loglik_mixed_noalloc serves them: it keeps all
its scratch in a static device array.  This file calls it through the C ABI
twice in a row, on two different batches (one window of N = 128; many windows
of N = 32 to 1024 at another observation time), and compares each result
with gb_loglik in mixed precision on the same inputs; checks that a call
leaves the device's free memory unchanged, that the status word reports a
non-finite parameter for that call only, and that a capturing stream is
refused.  It is collected last so that a run that stops at the first failure
has run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _cuda(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device=DEV, dtype=dtype)


def _inputs(api, wl):
    """Noise plus the batch's sources (library waveform), all on the device."""
    ctx = api.Context(wl.T)
    dA, dE = wl.noise_A.copy(), wl.noise_E.copy()
    for w, (k0, W, N, doff, coff, nc) in enumerate(wl.windows):
        for s in wl.sources[w]:
            hA, hE, q = ctx.waveform(_cuda(np.asarray(s)[None], torch.float64), N, "fp64")
            j = int(q[0]) - N // 2 + np.arange(N) - k0
            ok = (j >= 0) & (j < W)
            dA[doff + j[ok]] += hA[0].cpu().numpy()[ok]
            dE[doff + j[ok]] += hE[0].cpu().numpy()[ok]
    args = (_cuda(dA, torch.complex128), _cuda(dE, torch.complex128), _cuda(wl.w_A, torch.float64),
            _cuda(wl.w_E, torch.float64), _cuda(wl.theta, torch.float64))
    return ctx, args


def _call(api, wl, args, out, status, stream=None):
    err = ctypes.create_string_buffer(256)
    obs = api.Obs(wl.T, 2.5e9, 0, 0)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = api.lib().gb_loglik_mixed_noalloc(
        ctypes.byref(obs), api.windows_array(wl.windows), len(wl.windows), ptr(args[0]), ptr(args[1]),
        ptr(args[2]), ptr(args[3]), args[0].shape[0], ptr(args[4]), wl.theta.shape[0], ptr(out[0]), ptr(out[1]),
        ptr(out[2]), ptr(status), ctypes.c_void_p(st.cuda_stream), err, 256)
    return rc, err.value.decode()


def _noalloc(api, wl, args):
    n = wl.theta.shape[0]
    out = [torch.zeros(n, dtype=torch.float64, device=DEV) for _ in range(3)]
    status = torch.full((1,), -7, dtype=torch.int32, device=DEV)
    rc, msg = _call(api, wl, args, out, status)
    torch.cuda.synchronize()
    return rc, msg, out, int(status.item())


def test_noalloc_matches_loglik_on_two_calls_in_a_row():
    from paper_2307_03763_gb300 import api, build
    from paper_2307_03763_gb300 import workloads as wk
    build.build()
    batches = [wk.tiny_window(n_cand=700), wk.band_windows(n_win=24, cand_range=(40, 90))]
    for wl in batches:
        ctx, args = _inputs(api, wl)
        ref = [x.clone() for x in ctx.loglik(wl.windows, *args, prec="mixed")]
        rc, msg, out, status = _noalloc(api, wl, args)
        assert rc == 0, msg
        assert status == 0
        scale = max(1.0, float(ref[2].abs().max()))
        assert torch.allclose(out[0], ref[0], rtol=1e-12, atol=1e-12 * scale)
        assert torch.allclose(out[1], ref[1], rtol=1e-12, atol=1e-12 * scale)
        assert torch.allclose(out[2], ref[2], rtol=1e-12, atol=1e-12 * scale)
        ctx.close()


def test_noalloc_rejects_sizes_beyond_its_limits():
    from paper_2307_03763_gb300 import api, build
    build.build()
    obs = api.Obs(1e7, 2.5e9, 0, 0)
    err = ctypes.create_string_buffer(256)
    many = [(1000 + 64 * i, 64, 64, 64 * i, i, 1) for i in range(4097)]
    z = ctypes.c_void_p(0)
    rc = api.lib().gb_loglik_mixed_noalloc(ctypes.byref(obs), api.windows_array(many), len(many), z, z, z, z,
                                           64 * 4097, z, 4097, z, z, z, z, z, err, 256)
    assert rc == api.GB_EINVAL and "4096 windows" in err.value.decode()
    big = [(1000, 200000, 1024, 0, 0, 1), (300000, 70000, 1024, 200000, 1, 1)]
    rc = api.lib().gb_loglik_mixed_noalloc(ctypes.byref(obs), api.windows_array(big), 2, z, z, z, z, 270000, z, 2,
                                           z, z, z, z, z, err, 256)
    assert rc == api.GB_EINVAL and "262144" in err.value.decode()


def test_noalloc_allocates_nothing_and_reports_status_per_call():
    from paper_2307_03763_gb300 import api, build
    from paper_2307_03763_gb300 import workloads as wk
    build.build()
    wl = wk.tiny_window(n_cand=300)
    ctx, args = _inputs(api, wl)
    n = wl.theta.shape[0]
    out = [torch.zeros(n, dtype=torch.float64, device=DEV) for _ in range(3)]
    status = torch.full((1,), -7, dtype=torch.int32, device=DEV)
    rc, msg = _call(api, wl, args, out, status)                  # set-up call
    assert rc == 0, msg
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    rc, msg = _call(api, wl, args, out, status)
    torch.cuda.synchronize()
    assert rc == 0, msg
    assert torch.cuda.mem_get_info()[0] == free0                 # no device memory taken
    assert int(status.item()) == 0
    # a non-finite parameter: NaN rows and status 1 for that call only
    bad = wl.theta.copy()
    bad[7, 3] = np.nan
    args_bad = args[:4] + (_cuda(bad, torch.float64),)
    rc, msg = _call(api, wl, args_bad, out, status)
    torch.cuda.synchronize()
    assert rc == 0, msg
    assert int(status.item()) == 1
    assert np.isnan(float(out[0][7])) and bool(torch.isfinite(out[0][:7]).all())
    rc, msg = _call(api, wl, args, out, status)
    torch.cuda.synchronize()
    assert rc == 0 and int(status.item()) == 0
    # a stream that is capturing a graph is refused before anything is enqueued
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        rc, msg = _call(api, wl, args, out, status, stream=side)
    assert rc == api.GB_EINVAL and "capturing" in msg
    ctx.close()
