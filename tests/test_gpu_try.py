"""Multi-centre "try" reconstruction (Sec. 2.4) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2209_08450_gb300 as tcp

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def u16(a, pin=False):
    t = torch.from_numpy(np.ascontiguousarray(a).view(np.int16))
    return t.pin_memory() if pin else t.to(DEV)


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-5), (torch.float16, 5e-3), (torch.bfloat16, 5e-3)])
@pytest.mark.parametrize("ndet", [96, 90])  # 90: rows not 16-byte aligned in FP16, FP32 sinograms
def test_try_centers_match_oracle_per_centre(dtype, tol, ndet):
    c0 = ndet / 2 - 0.7
    ds = synth.shepp_logan_dataset(ntheta=121, ndet=ndet, nz=5, center=c0, seed=11)
    centers = c0 + np.array([-3.0, -1.5, 0.0, 0.7, 2.2, 5.1])
    out = tcp.try_centers(u16(ds.raw), u16(ds.dark), u16(ds.flat), ds.theta, centers, slice=3, dtype=dtype)
    torch.cuda.synchronize()
    assert out.shape == (6, ndet, ndet) and out.dtype == dtype
    got = out.double().cpu().numpy()
    for k, c in enumerate(centers):
        ref = oracle.fbp(ds.raw[:, 3:4], ds.dark[:, 3:4], ds.flat[:, 3:4], ds.theta, float(c), "shepp")[0]
        assert rel(got[k], ref) <= tol


def test_try_centers_host_raw_and_consistency_with_fbp():
    ds = synth.shepp_logan_dataset(ntheta=100, ndet=80, nz=4, center=39.2, seed=12)
    centers = np.array([38.0, 39.2, 40.5])
    dm = tcp.frame_mean(u16(ds.dark))
    fm = tcp.frame_mean(u16(ds.flat))
    a = tcp.try_centers(u16(ds.raw, pin=True), dm, fm, ds.theta, centers, slice=1)
    full = tcp.fbp(u16(ds.raw), dm, fm, ds.theta, 39.2)
    torch.cuda.synchronize()
    assert rel(a[1].double().cpu().numpy(), full[1].double().cpu().numpy()) <= 1e-5
    # a wrong axis gives a visibly different image
    assert rel(a[0].double().cpu().numpy(), full[1].double().cpu().numpy()) > 1e-2


def test_try_centers_rejects_bad_arguments():
    ds = synth.shepp_logan_dataset(ntheta=20, ndet=32, nz=2, center=16.0, seed=1)
    raw, dark, flat = u16(ds.raw), u16(ds.dark), u16(ds.flat)
    with pytest.raises(tcp.TcpError):
        tcp.try_centers(raw, dark, flat, ds.theta, [16.0], slice=2)
    with pytest.raises(tcp.TcpError):
        tcp.try_centers(raw, dark, flat, ds.theta, [16.0, float("nan")], slice=0)
    empty = tcp.try_centers(raw, dark, flat, ds.theta, np.zeros(0), slice=0)
    assert empty.shape == (0, 32, 32)


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-5), (torch.float16, 5e-3)])
def test_try_centers_fourierrec(dtype, tol):
    from oracle import fourierrec as frc
    c0 = 24 - 0.4
    ds = synth.shepp_logan_dataset(ntheta=60, ndet=48, nz=3, center=c0, seed=13)
    centers = c0 + np.array([-2.0, 0.0, 1.3, 3.7])
    out = tcp.try_centers(u16(ds.raw), u16(ds.dark), u16(ds.flat), ds.theta, centers, slice=1, dtype=dtype,
                          algorithm="fourierrec")
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    p = oracle.normalize(ds.raw[:, 1:2], oracle.frame_mean(ds.dark[:, 1:2]), oracle.frame_mean(ds.flat[:, 1:2]))
    for k, c in enumerate(centers):
        q = oracle.filter_sino(p, float(c), "shepp", "edge")
        ref = frc.backproject_exact(q, ds.theta, 24.0, 48)[0]
        assert rel(got[k], ref) <= tol
