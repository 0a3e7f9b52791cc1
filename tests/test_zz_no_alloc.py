"""gp_get_csr_noalloc: the copy-out for callers that must not allocate device
memory at the time of the call (another allocator owns the device's memory,
or the process is at its device-memory limit).  It must give exactly what
gp_get_csr gives, call after call, although every call reuses the same static
staging area on the device, and it must leave the device's free memory
untouched.  This file is collected last."""

import ctypes

import numpy as np
import pytest

from paper_2205_09070_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import __graft_entry__ as g
    g.build()
    from paper_2205_09070_gb300 import gpsparse
    assert torch.cuda.is_available()
    return gpsparse


def copy_out(G, gp, fn_name, device_val=False):
    lib = G.load()
    fn = getattr(lib, fn_name)
    sizes = (ctypes.c_int64 * 2)()
    assert fn(gp._h, None, None, None, None, sizes) == G.GP_OK
    na, nnz = int(sizes[0]), int(sizes[1])
    rp = np.zeros(na + 1, np.int64)
    col = np.zeros(nnz, np.int32)
    perm = np.zeros(na, np.int32)
    if device_val:
        val_t = torch.zeros(nnz, dtype=torch.float64, device="cuda")
        vptr = val_t.data_ptr()
    else:
        val = np.zeros(nnz, np.float64)
        vptr = val.ctypes.data
    st = fn(gp._h, rp.ctypes.data, col.ctypes.data, vptr, perm.ctypes.data, sizes)
    assert st == G.GP_OK, G.status_string(st)
    if device_val:
        val = val_t.cpu().numpy()
    return rp, col, val, perm


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_copy_matches_gp_get_csr_on_consecutive_calls(G, prec):
    # two different matrices, two calls each: every no-alloc copy equals the
    # allocating copy of the same assembly, whatever the previous call left
    # in the shared staging area
    probs = [W.grad_3d(seed=3, n=3000), W.small_2d(seed=1)]
    for p in probs:
        gp = G.GP(p.dim, p.n1, p.n2)
        gp.assemble(torch.as_tensor(p.x, device="cuda"), p.h, precision=prec)
        ref = copy_out(G, gp, "gp_get_csr")
        for device_val in (False, True):
            got = copy_out(G, gp, "gp_get_csr_noalloc", device_val=device_val)
            for a, b in zip(ref, got):
                assert np.array_equal(a, b)
        gp.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_leaves_device_memory_untouched(G, prec):
    # on a fresh context, before any allocating copy-out: once the library's
    # kernels and the staging area's address are set up (first call), a
    # further call changes the device's free memory by nothing, while the
    # allocating gp_get_csr grows a context buffer for the same values (a few
    # MiB here, so that the driver cannot serve it from pages it already holds)
    n = 30_000
    p = W.mixture_3d(seed=9, n=n, r_s=0.005 * (5e6 / n) ** (1 / 3))
    gp = G.GP(p.dim, p.n1, p.n2)
    info = gp.assemble(torch.as_tensor(p.x, device="cuda"), p.h, precision=prec)
    assert 300_000 < info["nnz"] <= (1 << 20)
    torch.cuda.synchronize()
    first = copy_out(G, gp, "gp_get_csr_noalloc")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    again = copy_out(G, gp, "gp_get_csr_noalloc")
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    for a, b in zip(first, again):
        assert np.array_equal(a, b)
    ref = copy_out(G, gp, "gp_get_csr")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free1      # the allocating copy-out took memory
    for a, b in zip(ref, again):
        assert np.array_equal(a, b)
    gp.close()


def test_noalloc_rejects_matrices_above_the_staging_size(G):
    p = W.mixture_3d(seed=9, n=120_000, r_s=0.005 * (5e6 / 120_000) ** (1 / 3))
    gp = G.GP(p.dim, p.n1, p.n2)
    info = gp.assemble(torch.as_tensor(p.x, device="cuda"), p.h)
    lib = G.load()
    sizes = (ctypes.c_int64 * 2)()
    assert info["nnz"] > (1 << 20)
    val = np.zeros(info["nnz"], np.float64)
    st = lib.gp_get_csr_noalloc(gp._h, None, None, val.ctypes.data, None, sizes)
    assert st == G.GP_ERR_UNSUPPORTED
    assert int(sizes[1]) == info["nnz"]
    # the pattern alone needs no staging and still comes out
    rp = np.zeros(info["n_active"] + 1, np.int64)
    assert lib.gp_get_csr_noalloc(gp._h, rp.ctypes.data, None, None, None, sizes) == G.GP_OK
    assert rp[-1] == info["nnz"]
    gp.close()


def test_noalloc_while_another_stream_captures(G):
    """The call is made while a CUDA graph is being captured on a stream of the
    caller's (relaxed capture mode), with its outputs allocated beforehand: the
    copy-out runs on the context's own stream, the capture is left intact, and
    the outputs equal gp_get_csr's."""
    p = W.small_2d(seed=1, n=600)
    gp = G.GP(p.dim, p.n1, p.n2, p.beta)
    gp.assemble(torch.as_tensor(p.x, device="cuda"), p.h, precision="fp32")
    copy_out(G, gp, "gp_get_csr_noalloc")  # first call on the device: outside any capture
    rp0, col0, val0, perm0 = copy_out(G, gp, "gp_get_csr")
    lib = G.load()
    sizes = (ctypes.c_int64 * 2)()
    assert lib.gp_get_csr_noalloc(gp._h, None, None, None, None, sizes) == G.GP_OK
    rp = np.zeros(int(sizes[0]) + 1, np.int64)
    col = np.zeros(int(sizes[1]), np.int32)
    perm = np.zeros(int(sizes[0]), np.int32)
    val_t = torch.zeros(int(sizes[1]), dtype=torch.float64, device="cuda")
    a = torch.arange(16, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side, capture_error_mode="relaxed"):
            b = a * 2.0
            st = lib.gp_get_csr_noalloc(gp._h, rp.ctypes.data, col.ctypes.data, val_t.data_ptr(),
                                        perm.ctypes.data, sizes)
    assert st == G.GP_OK, G.status_string(st)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(b, a * 2.0)
    assert np.array_equal(rp, rp0) and np.array_equal(col, col0) and np.array_equal(perm, perm0)
    assert np.array_equal(val_t.cpu().numpy(), val0)
    gp.close()
