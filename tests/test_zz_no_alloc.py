"""kn_integrate_noalloc: the integrator for callers that cannot allocate GPU
memory when they integrate -- e.g. a simulation code that hands out all
device memory from its own pool allocated at start-up, or whose per-step
path must avoid cudaMalloc/cudaFree because those can synchronise the
device.  The entry point reads and writes only the caller's buffers and keeps
its work-queue scratch in a fixed device array.

Checked through the C ABI against kn_integrate_batch on the same zones, on
two calls in a row (the second call sees the scratch the first one left).
This file is collected last, so a run that stops at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from kn_inputs import net150, profile_zones

pytestmark = pytest.mark.gpu

NAMES = ("Y0", "T0", "rho0", "tau", "t_start", "t_end", "dt_trial")
OUTS = ("Y", "t", "dt_next", "steps", "rejects", "status")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_5826_gb300 import build, kn
    build.build()
    return torch, kn


def _outputs(torch, Z, N):
    dev = torch.device("cuda")
    f64 = dict(dtype=torch.float64, device=dev)
    return {"Y": torch.empty((Z, N), **f64), "t": torch.empty(Z, **f64), "dt_next": torch.empty(Z, **f64),
            "steps": torch.empty(Z, dtype=torch.int64, device=dev),
            "rejects": torch.empty(Z, dtype=torch.int64, device=dev),
            "status": torch.empty(Z, dtype=torch.int32, device=dev)}


@pytest.mark.parametrize("prec,method", [(1, 0), (0, 0), (1, 1), (0, 1)])
def test_noalloc_matches_batch_on_two_calls(env, prec, method):
    torch, kn = env
    net = net150()
    Z = 300
    z = profile_zones(net, Z, t_end=3e-11)
    opts = kn.Opts(precision=prec, method=method, threads_per_zone=160, threads_per_cta=160 if prec == 0 else 800)
    g = kn.Network(net)
    # set-up: the existing entry point builds the network's tables for these opts
    g.set_zones(z)
    kn.integrate_batch([g], opts)
    ref = g.get()
    dev = torch.device("cuda")
    dz = {k: torch.from_numpy(np.ascontiguousarray(getattr(z, k))).to(dev) for k in NAMES}
    zc = kn._Zones(*[dz[k].data_ptr() for k in NAMES])
    out = _outputs(torch, Z, net.n_species)
    L = kn.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        for v in out.values():
            v.fill_(-1)
        rc = L.kn_integrate_noalloc(g.h, Z, C.byref(zc), C.byref(opts.c()),
                                    *[out[k].data_ptr() for k in OUTS], stream)
        assert rc == kn.KN_OK, L.kn_last_error()
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        assert (got["status"] == 0).all(), call
        assert np.array_equal(got["steps"], ref["steps"]), call
        assert np.array_equal(got["t"], ref["t"]), call
        m = ref["Y"] > 1e-30
        assert np.max(np.abs(got["Y"][m] - ref["Y"][m]) / ref["Y"][m]) <= 1e-12, call
        assert np.all(got["Y"][~m] <= 1e-30), call
    g.close()


def _zone_buffers(torch, Z, N):
    """Device inputs and outputs sized for Z zones of N species, so that a
    call that wrongly got past the host checks would still stay in bounds."""
    dev = torch.device("cuda")
    zin = {k: torch.zeros((Z, N) if k == "Y0" else (Z,), dtype=torch.float64, device=dev) for k in NAMES}
    return zin, _outputs(torch, Z, N)


def test_noalloc_refuses_oversize_unbuilt_tables_and_host_memory(env):
    torch, kn = env
    net = net150()
    N = net.n_species
    g = kn.Network(net)
    L = kn.lib()
    opts = kn.Opts(precision=1, threads_per_zone=160, threads_per_cta=160)
    # one zone over the limit, with buffers of that size
    Z = 65537
    zin, out = _zone_buffers(torch, Z, N)
    zc = kn._Zones(*[zin[k].data_ptr() for k in NAMES])
    rc = L.kn_integrate_noalloc(g.h, Z, C.byref(zc), C.byref(opts.c()), *[out[k].data_ptr() for k in OUTS], None)
    assert rc == kn.KN_ERR_INVALID_ARG
    assert b"KN_NOALLOC_MAX_ZONES" in L.kn_last_error()
    del zin, out
    # a network whose tables were never built for these opts
    Z = 4
    zin, out = _zone_buffers(torch, Z, N)
    zc = kn._Zones(*[zin[k].data_ptr() for k in NAMES])
    rc = L.kn_integrate_noalloc(g.h, Z, C.byref(zc), C.byref(opts.c()), *[out[k].data_ptr() for k in OUTS], None)
    assert rc == kn.KN_ERR_STATE
    assert b"not built" in L.kn_last_error()
    # build the tables, then hand it host memory: refused on the host, no launch
    z = profile_zones(net, Z, t_end=3e-11)
    g.set_zones(z)
    kn.integrate_batch([g], opts)
    torch.cuda.synchronize()
    host_Y = np.zeros((Z, N))
    ptrs = [out[k].data_ptr() for k in OUTS]
    ptrs[0] = host_Y.ctypes.data
    rc = L.kn_integrate_noalloc(g.h, Z, C.byref(zc), C.byref(opts.c()), *ptrs, None)
    assert rc == kn.KN_ERR_INVALID_ARG
    assert b"Y is not device memory" in L.kn_last_error()
    host_T0 = np.ones(Z)
    zc_host = kn._Zones(*[host_T0.ctypes.data if k == "T0" else zin[k].data_ptr() for k in NAMES])
    rc = L.kn_integrate_noalloc(g.h, Z, C.byref(zc_host), C.byref(opts.c()),
                                *[out[k].data_ptr() for k in OUTS], None)
    assert rc == kn.KN_ERR_INVALID_ARG
    assert b"T0 is not device memory" in L.kn_last_error()
    # Y overlapping Y0 without being Y0 (shifted by one species)
    big = torch.zeros((Z + 1) * N, dtype=torch.float64, device="cuda")
    zc_ov = kn._Zones(*[big.data_ptr() if k == "Y0" else zin[k].data_ptr() for k in NAMES])
    ptrs = [out[k].data_ptr() for k in OUTS]
    ptrs[0] = big.data_ptr() + 8
    rc = L.kn_integrate_noalloc(g.h, Z, C.byref(zc_ov), C.byref(opts.c()), *ptrs, None)
    assert rc == kn.KN_ERR_INVALID_ARG
    assert b"overlaps" in L.kn_last_error()
    torch.cuda.synchronize()
    g.close()


def test_noalloc_in_place(env):
    """Y may be Y0 itself: the zones integrate in place and match the batch."""
    torch, kn = env
    net = net150()
    Z = 64
    z = profile_zones(net, Z, t_end=3e-11)
    opts = kn.Opts(precision=1, threads_per_zone=160, threads_per_cta=800)
    g = kn.Network(net)
    g.set_zones(z)
    kn.integrate_batch([g], opts)
    ref = g.get()
    dev = torch.device("cuda")
    dz = {k: torch.from_numpy(np.ascontiguousarray(getattr(z, k))).to(dev) for k in NAMES}
    zc = kn._Zones(*[dz[k].data_ptr() for k in NAMES])
    out = _outputs(torch, Z, net.n_species)
    ptrs = [out[k].data_ptr() for k in OUTS]
    ptrs[0] = dz["Y0"].data_ptr()
    L = kn.lib()
    rc = L.kn_integrate_noalloc(g.h, Z, C.byref(zc), C.byref(opts.c()), *ptrs,
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == kn.KN_OK, L.kn_last_error()
    torch.cuda.synchronize()
    Y = dz["Y0"].cpu().numpy()
    assert np.array_equal(out["steps"].cpu().numpy(), ref["steps"])
    m = ref["Y"] > 1e-30
    assert np.max(np.abs(Y[m] - ref["Y"][m]) / ref["Y"][m]) <= 1e-12
    g.close()
