"""The allocation-free Sigma_c entry point (gw_sigma_c_static) against the
regular pipeline.

Callers that cannot allocate device memory (their memory belongs to another
allocator, or they run a loop that must not wait on an allocator) pass their
own input and output buffers; the library's fixed scratch table does the
rest.  The output must equal the Sigma_c grid of gw_sigma_diag, on two calls
in a row with different sizes (the shared table is rewritten each time).
This file is collected last so that a failure here comes after every other
test has run.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _static_sigma_c(gwlib, sig_host, j0, n_omega, d_omega, eta):
    import torch
    lib = gwlib.load()
    dev_sig = torch.from_numpy(np.ascontiguousarray(sig_host)).to("cuda")
    ns = sig_host.shape[0]
    out = torch.empty((ns, 2 * n_omega - 1, 2), dtype=torch.float64, device="cuda")
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream()
    code = lib.gw_sigma_c_static(dev_sig.data_ptr(), ns, sig_host.shape[1], j0, n_omega, d_omega, eta,
                                 out.data_ptr(), stream.cuda_stream, err, 256)
    torch.cuda.synchronize()
    assert code == 0, err.value
    o = out.cpu().numpy()
    return o[..., 0] + 1j * o[..., 1]


def test_static_sigma_c_matches_pipeline_twice(gwlib, ctx):
    runs = []
    for cfg, states in ((1, None), (2, None)):
        mol, grid = synth.make_config(cfg)
        h, *_ = gwlib.solve(ctx, mol, grid, prec=gwlib.GW_MIXED)
        try:
            s = h["sigma"].copy()
        finally:
            for k in ("sigma", "W", "chi0", "mol"):
                h[k].free()
        runs.append((s, grid))
    for s, grid in runs:                       # two calls in a row, different sizes
        got = _static_sigma_c(gwlib, s["sigma"], s["j0"], grid.n_omega, grid.d_omega, grid.eta)
        ref = s["sigma_c"]
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_static_sigma_c_allocates_nothing(gwlib, ctx):
    """Once warmed up, a call leaves the device's free memory unchanged: the
    scratch is the library's fixed table, the buffers are the caller's."""
    import torch
    mol, grid = synth.make_config(1)
    h, *_ = gwlib.solve(ctx, mol, grid, prec=gwlib.GW_MIXED)
    try:
        s = h["sigma"].copy()
    finally:
        for k in ("sigma", "W", "chi0", "mol"):
            h[k].free()
    lib = gwlib.load()
    sig = torch.from_numpy(np.ascontiguousarray(s["sigma"])).to("cuda")
    ns, n_sig = s["sigma"].shape
    out = torch.empty((ns, 2 * grid.n_omega - 1, 2), dtype=torch.float64, device="cuda")
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream()

    def call():
        code = lib.gw_sigma_c_static(sig.data_ptr(), ns, n_sig, s["j0"], grid.n_omega, grid.d_omega, grid.eta,
                                     out.data_ptr(), stream.cuda_stream, err, 256)
        torch.cuda.synchronize()
        assert code == 0, err.value

    call()                                          # warm: table address resolved, kernels loaded
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_sigma_c_rejects_oversize(gwlib):
    lib = gwlib.load()
    err = ctypes.create_string_buffer(256)
    code = lib.gw_sigma_c_static(ctypes.c_void_p(16), 1, 70000, 0, 64, 0.01, 0.015, ctypes.c_void_p(16), None,
                                 err, 256)
    assert code == -1
    assert b"exceeds the static table" in err.value
