"""LpRec (tcp_lprec, tcp_fbp algorithm "lprec") against the FP64 oracle.

Parity: the GPU runs the oracle's steps (three spans, log-polar grid with steps
of 1/os pixel at the far radius, cubic B-splines both ways) at the same
oversampling, so the two agree to FP32 rounding (rel-L2 <= 1e-5).  Accuracy:
both converge to the direct cubic-spline backprojection as os grows, and the
GPU's distance to it equals the oracle's to within rounding.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import lprec as olp
import paper_2209_08450_gb300 as tcp

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _theta(nt, theta0=0.0):
    return theta0 + np.arange(nt) * (np.pi / nt)


@pytest.mark.parametrize("nz,nt,nd,n,center,theta0", [
    (3, 60, 48, 48, 24.3, 0.0),      # spans of 20 angles, off-centre axis
    (2, 61, 52, 40, 26.0, 0.3),      # ragged spans (20/21/20), n != ndet, rotated start
    (18, 45, 32, 32, 15.7, -0.2),    # two passes of slices
    (1, 3, 20, 16, 10.0, 0.0),       # one angle per span
])
def test_lprec_matches_oracle_same_oversampling(nz, nt, nd, n, center, theta0):
    rng = np.random.default_rng(nt + nd)
    q = rng.normal(size=(nz, nt, nd))
    th = _theta(nt, theta0)
    got = tcp.lprec(torch.from_numpy(q).float().to(DEV), th, center, n=n).double().cpu().numpy()
    zs = range(nz) if nz <= 3 else (0, 9, 17)
    ref = olp.backproject_lprec(q[list(zs)], th, center, n, os=2.0)
    err = rel(got[list(zs)], ref)
    print("\nLpRec nz=%d nt=%d nd=%d n=%d: rel-L2 vs oracle %.2e" % (nz, nt, nd, n, err))
    assert err <= 1e-5


def test_lprec_converges_to_the_cubic_spline_sums_like_the_oracle():
    rng = np.random.default_rng(3)
    nt, nd, n, c = 90, 48, 48, 24.0
    q = rng.normal(size=(1, nt, nd))
    th = _theta(nt)
    exact = olp.backproject_spline_exact(q, th, c, n)
    qd = torch.from_numpy(q).float().to(DEV)
    errs = []
    for os in (2.0, 4.0):
        got = tcp.lprec(qd, th, c, n=n, oversampling=os).double().cpu().numpy()
        mine = rel(got, exact)
        ref = rel(olp.backproject_lprec(q, th, c, n, os=os), exact)
        print("\nos %.0f: GPU %.3e, oracle %.3e from the spline sums" % (os, mine, ref))
        assert abs(mine - ref) <= 0.02 * ref + 2e-6
        errs.append(mine)
    assert errs[1] < errs[0] / 5  # about tenfold per doubling


@pytest.mark.parametrize("sdt,vdt", [(torch.float16, torch.float32), (torch.bfloat16, torch.bfloat16),
                                     (torch.float32, torch.float16)])
def test_lprec_16bit_storage(sdt, vdt):
    rng = np.random.default_rng(11)
    q = rng.normal(size=(4, 48, 40))
    th = _theta(48)
    qd = torch.from_numpy(q).to(DEV, sdt)
    got = tcp.lprec(qd, th, 20.2, n=40, dtype=vdt, scale=0.25).double().cpu().numpy()
    ref = 0.25 * olp.backproject_lprec(qd.double().cpu().numpy(), th, 20.2, 40)
    assert rel(got, ref) <= 5e-3


def test_lprec_rejections():
    q = torch.zeros((1, 10, 16), device=DEV)
    with pytest.raises(tcp.TcpError) as e:  # not equally spaced
        th = _theta(10)
        th[3] += 1e-3
        tcp.lprec(q, th, 8.0)
    assert e.value.status == 1
    with pytest.raises(tcp.TcpError) as e:  # a full turn instead of a half
        tcp.lprec(q, np.arange(10) * (2 * np.pi / 10), 8.0)
    assert e.value.status == 1
    with pytest.raises(tcp.TcpError) as e:  # fewer than 3 angles
        tcp.lprec(torch.zeros((1, 2, 16), device=DEV), _theta(2), 8.0)
    assert e.value.status == 2
    out = tcp.lprec(torch.zeros((0, 10, 16), device=DEV), _theta(10), 8.0)
    assert out.shape == (0, 16, 16)


def test_fbp_lprec_pipeline_matches_oracle():
    d = synth.shepp_logan_dataset(ntheta=72, ndet=64, nz=5, center=32.4, seed=7)
    p = oracle.normalize(d.raw, oracle.frame_mean(d.dark), oracle.frame_mean(d.flat))
    q = oracle.filter_sino(p, d.center, "shepp", "edge")
    ref = olp.backproject_lprec(q, d.theta, 32.0, 64)
    raw = torch.from_numpy(d.raw.view(np.int16)).to(DEV)
    dark = torch.from_numpy(d.dark.view(np.int16)).to(DEV)
    flat = torch.from_numpy(d.flat.view(np.int16)).to(DEV)
    for chunk in (0, 2):
        out = tcp.fbp(raw, dark, flat, d.theta, d.center, algorithm="lprec", chunk_nz=chunk)
        torch.cuda.synchronize()
        assert rel(out.double().cpu().numpy(), ref) <= 1e-5
    # the same through a plan, captured on first use
    plan = tcp.Plan(d.theta, 64, 5, d.center, algorithm="lprec")
    vol = torch.full((5, 64, 64), float("nan"), device=DEV)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        plan.fbp(raw, dark, flat, out=vol, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert rel(vol.double().cpu().numpy(), ref) <= 1e-5
    # and it approximates the cubic-spline FBP as closely as the oracle's LpRec does
    exact = olp.backproject_spline_exact(q, d.theta, 32.0, 64)
    assert rel(vol.double().cpu().numpy(), exact) <= 1.02 * rel(ref, exact) + 1e-6
    plan.close()


def test_lprec_2048_sampled_voxels_converge_to_the_spline_sums():
    # a 2048^2 slice of the porous workload, 2048 angles, filtered rows: LpRec
    # at oversampling 2 and 4 on sampled voxels against the direct cubic-spline
    # sums (the quantity LpRec approximates); the error falls about tenfold
    # per doubling, as in the oracle's own convergence pin
    import synth.gpu as sgpu
    raw, dark, flat, th, c, mu = sgpu.porous_frames(2048, 2048, 2048, seed=0, device=DEV, slices=np.array([1024]))
    r = raw.cpu().numpy().view(np.uint16)
    p = oracle.normalize(r, oracle.frame_mean(dark.cpu().numpy().view(np.uint16)),
                         oracle.frame_mean(flat.cpu().numpy().view(np.uint16)))
    q = oracle.filter_sino(p, c, "shepp")[0]
    rng = np.random.default_rng(5)
    ix, iy = rng.integers(200, 1848, 300), rng.integers(200, 1848, 300)
    ref = olp.backproject_spline_points(q, th, 1024.0, 2048, ix, iy)
    qd = torch.from_numpy(q[None]).float().to(DEV)
    errs = []
    for os in (2.0, 4.0):
        got = tcp.lprec(qd, th, 1024.0, oversampling=os)[0].double().cpu().numpy()[iy, ix]
        errs.append(rel(got, ref))
    print("\n2048^2 LpRec vs spline sums: os 2 %.2e, os 4 %.2e" % tuple(errs))
    assert errs[1] < errs[0] / 5
    assert errs[1] < 1e-3
