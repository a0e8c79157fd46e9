"""Plans (tcp_plan_*): the calls that take a plan own no per-call state, so
the first use can be captured into a CUDA graph, and their results equal the
calls without a plan and the FP64 oracle.

The capture uses torch's default (global) capture mode, in which a
synchronising or allocating CUDA call made during the capture fails it; the
stream-ordered pool's high-water mark shows that the plan calls take nothing
from it either.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2209_08450_gb300 as tcp

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def u16(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint16).view(np.int16)).to(DEV)


@pytest.fixture(scope="module")
def ds():
    d = synth.shepp_logan_dataset(ntheta=120, ndet=96, nz=11, center=47.3, seed=2)
    ref = oracle.fbp(d.raw, d.dark, d.flat, d.theta, d.center, "shepp")
    return d, ref


@pytest.mark.parametrize("dtype,kw,tol", [
    (torch.float32, {}, 1e-5),                                   # FP16 hi/lo pairs on the tensor cores
    (torch.float32, {"sino_dtype": torch.float32, "chunk_nz": 4}, 1e-5),  # CUDA cores, ragged chunks
    (torch.float16, {"chunk_nz": 5}, 5e-3),
    (torch.float32, {"algorithm": "fourierrec", "chunk_nz": 4}, None),
])
def test_plan_fbp_captured_on_first_use_replays_equal_to_oracle(ds, dtype, kw, tol):
    d, ref = ds
    raw, dark, flat = u16(d.raw), u16(d.dark), u16(d.flat)
    plan = tcp.Plan(d.theta, 96, 11, d.center, dtype=dtype, **kw)
    vol = torch.full((11, 96, 96), float("nan"), dtype=dtype, device=DEV)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=s):  # the plan's first call is the captured one
        plan.fbp(raw, dark, flat, out=vol, stream=s)
    assert torch.isnan(vol).all()  # nothing ran during the capture
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
    got = vol.double().cpu().numpy()
    direct = tcp.fbp(raw, dark, flat, d.theta, d.center, dtype=dtype, **kw)
    torch.cuda.synchronize()
    if tol is None:  # FourierRec: against the oracle's band-limited backprojection of the same rows
        from oracle import fourierrec as frc
        p = oracle.normalize(d.raw, oracle.frame_mean(d.dark), oracle.frame_mean(d.flat))
        q = oracle.filter_sino(p, d.center, "shepp", "edge")
        ref = frc.backproject_gridding(q, d.theta, 48.0, 96, width=10)
        tol = 1e-5
    assert rel(got, ref) <= tol
    assert torch.equal(vol, direct)  # the same kernels on the same tables as the call without a plan
    plan.close()


def test_plan_fbp_host_buffers_captured(ds):
    d, ref = ds
    raw = torch.from_numpy(d.raw.view(np.int16)).pin_memory()
    dark = torch.from_numpy(d.dark.view(np.int16)).pin_memory()
    flat = torch.from_numpy(d.flat.view(np.int16)).pin_memory()
    vol = torch.full((11, 96, 96), float("nan"), pin_memory=True)
    plan = tcp.Plan(d.theta, 96, 11, d.center, chunk_nz=4, host_raw=True, host_vol=True, host_frames=10,
                    n_buffers=3)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=s):
        plan.fbp(raw, dark, flat, out=vol, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert rel(vol.double().numpy(), ref) <= 1e-5
    plan.close()


def test_plan_calls_take_nothing_from_the_stream_ordered_pool(ds):
    d, ref = ds
    rt = None
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            continue
    if rt is None:
        pytest.skip("CUDA runtime library not found by name")
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    USED_CURRENT, USED_HIGH = 7, 8

    def attr(a):
        v = ctypes.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, a, ctypes.byref(v)) == 0
        return v.value

    raw, dark, flat = u16(d.raw), u16(d.dark), u16(d.flat)
    plan = tcp.Plan(d.theta, 96, 11, d.center, algorithm="fourierrec", chunk_nz=4)
    plan_lr = tcp.Plan(d.theta, 96, 11, d.center)
    vol = torch.empty((11, 96, 96), device=DEV)
    sino = torch.empty((11, 120, 96), device=DEV)
    torch.cuda.synchronize()
    for fn in (lambda: plan.fbp(raw, dark, flat, out=vol), lambda: plan_lr.fbp(raw, dark, flat, out=vol),
               lambda: plan_lr.project(vol, 48.0, out=sino), lambda: plan_lr.backproject(sino, 48.0, out=vol)):
        zero = ctypes.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, USED_HIGH, ctypes.byref(zero)) == 0
        base = attr(USED_CURRENT)
        fn()
        torch.cuda.synchronize()
        assert attr(USED_HIGH) <= base
    # the calls without a plan do take their scratch from the pool (the check sees it)
    zero = ctypes.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, USED_HIGH, ctypes.byref(zero)) == 0
    base = attr(USED_CURRENT)
    tcp.fbp(raw, dark, flat, d.theta, d.center, out=vol)
    torch.cuda.synchronize()
    assert attr(USED_HIGH) > base
    plan.close()
    plan_lr.close()


def test_plan_filter_backproject_project_equal_the_calls_without_plan():
    rng = np.random.default_rng(5)
    nz, nt, nd, n, c = 7, 90, 104, 100, 51.6
    theta = rng.uniform(0, np.pi, nt)
    q = torch.from_numpy(rng.normal(size=(nz, nt, nd))).float().to(DEV)
    plan = tcp.Plan(theta, nd, nz, c, n=n, filter="parzen", pad="zero")
    a = plan.filter_(q.clone())
    b = tcp.filter_(q.clone(), c, "parzen", "zero")
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    va = plan.backproject(a, nd / 2.0, scale=0.5)
    vb = tcp.backproject(b, theta, nd / 2.0, n=n, scale=0.5)
    torch.cuda.synchronize()
    assert torch.equal(va, vb)
    ref = 0.5 * oracle.backproject(b.double().cpu().numpy(), theta, nd / 2.0, n)
    assert rel(va.double().cpu().numpy(), ref) <= 1e-5
    pa = plan.project(va, c)
    pb = tcp.project(va, theta, c, ndet=nd)
    torch.cuda.synchronize()
    assert torch.equal(pa, pb)


def test_plan_rejects_calls_outside_its_geometry(ds):
    d, ref = ds
    plan = tcp.Plan(d.theta, 96, 6, d.center)
    raw, dark, flat = u16(d.raw), u16(d.dark), u16(d.flat)
    with pytest.raises(tcp.TcpError) as e:  # 11 slices > the plan's 6
        plan.fbp(raw, dark, flat)
    assert e.value.status == 2
    with pytest.raises(tcp.TcpError) as e:  # host raw without an upload ring
        plan.fbp(torch.from_numpy(d.raw[:, :6].copy().view(np.int16)), dark[:, :6], flat[:, :6],
                 out=torch.empty((6, 96, 96), device=DEV))
    assert e.value.status == 1
    out = plan.fbp(raw[:, :6], dark[:, :6], flat[:, :6])  # fewer slices than planned are fine
    torch.cuda.synchronize()
    assert rel(out.double().cpu().numpy(), ref[:6]) <= 1e-5
    assert plan.info()["device_bytes"] > 0
    plan.close()


def test_plan_trace_records_the_pipeline_timeline(ds):
    # the per-chunk timeline of a host-buffer run: every upload precedes its
    # chunk's compute, every download follows it, computes run in order, and
    # the upload of chunk k+1 is issued before chunk k's compute ends
    d, ref = ds
    raw = torch.from_numpy(d.raw.view(np.int16)).pin_memory()
    vol = torch.empty((11, 96, 96), pin_memory=True)
    plan = tcp.Plan(d.theta, 96, 11, d.center, chunk_nz=4, host_raw=True, host_vol=True, trace=True)
    plan.fbp(raw, u16(d.dark), u16(d.flat), out=vol)
    t = plan.trace()
    torch.cuda.synchronize()
    assert rel(vol.double().numpy(), ref) <= 1e-5
    assert t.shape[0] == 4  # 2 + 4 + 4 + 1 slices: half-depth first chunk, short last chunk
    for k in range(t.shape[0]):
        h0, h1, c0, c1, d0, d1 = t[k]
        assert 0 <= h0 <= h1 <= c0 + 1e-3 <= c1 + 1e-3 and c1 <= d0 + 1e-3 <= d1 + 1e-3
        if k:
            assert c0 >= t[k - 1][3] - 1e-3
        if k + 1 < t.shape[0]:
            assert t[k + 1][0] < c1
    plan.close()
