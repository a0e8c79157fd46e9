"""GPU parity of FourierRec (tcp_fourierrec) against the FP64 oracle.

Small cases compare element by element with the exact definition (direct
sums of trigonometric interpolants); larger ones with the FP64 gridding
evaluation at width 10, whose distance to the exact sums is ~1e-9 (pinned in
test_oracle_fourierrec.py).  Tolerances: relative L2 <= 1e-5 for FP32
storage at the default width 7, <= 5e-3 for FP16/BF16 storage.  Sizes give
several grid strips, odd slice counts (an unpaired last slice), ndet that is
not a power of two and n != ndet (oversampling above 2).
"""
import numpy as np
import pytest
import torch

from oracle import fourierrec as fr
import paper_2209_08450_gb300 as tcp

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def host(t):
    return t.double().cpu().numpy()


@pytest.fixture(autouse=True)
def _checked():
    tcp.set_checked(True)
    yield
    tcp.device_check()
    tcp.set_checked(False)


def _case(nz, nt, nd, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(nz, nt, nd)), np.sort(rng.uniform(0, np.pi, nt))


@pytest.mark.parametrize("nz,nt,nd,n,center", [
    (2, 24, 32, 32, 16.3), (3, 19, 25, 22, 12.9), (1, 9, 16, 16, 8.0), (5, 31, 40, 36, 21.45)])
def test_fourierrec_fp32_vs_exact(nz, nt, nd, n, center):
    q, theta = _case(nz, nt, nd, nz * 100 + nt)
    got = tcp.fourierrec(to_dev(q), theta, center, n=n)
    torch.cuda.synchronize()
    want = fr.backproject_exact(q, theta, center, n)
    assert rel(host(got), want) <= 1e-5


@pytest.mark.parametrize("nz,nt,nd,n,center", [(4, 100, 128, 128, 63.7), (3, 64, 96, 100, 47.2)])
def test_fourierrec_fp32_many_strips(nz, nt, nd, n, center):
    q, theta = _case(nz, nt, nd, 7 * nz + nt)
    got = host(tcp.fourierrec(to_dev(q), theta, center, n=n))
    want = fr.backproject_gridding(q, theta, center, n, width=10)
    assert rel(got, want) <= 1e-5
    # same window as the oracle's gridding steps: only FP32 rounding apart
    assert rel(got, fr.backproject_gridding(q, theta, center, n, width=7)) <= 5e-6



def test_fourierrec_ten_pairs_in_one_batch_with_a_partial_near_region():
    # 19 slices = 10 slice pairs in one batch (the near-node table's pairs are
    # applied 8 at a time: two passes, an unpaired last slice), and a 1024-point
    # grid whose nodes within 128 of the zero frequency come from the table
    # while the rest are gathered
    nz, nt, nd, n, c = 19, 90, 300, 300, 151.3
    q, theta = _case(nz, nt, nd, 77)
    got = host(tcp.fourierrec(to_dev(q), theta, c, n=n))
    for z in (0, 9, 18):
        want = fr.backproject_gridding(q[z:z + 1], theta, c, n, width=10)
        assert rel(got[z:z + 1], want) <= 1e-5

def test_fourierrec_width_controls_error():
    q, theta = _case(2, 24, 32, 11)
    exact = fr.backproject_exact(q, theta, 16.3, 32)
    errs = []
    for w in (4, 6, 8):
        got = host(tcp.fourierrec(to_dev(q), theta, 16.3, n=32, width=w))
        ref = rel(fr.backproject_gridding(q, theta, 16.3, 32, width=w), exact)
        e = rel(got, exact)
        assert e <= 2 * ref + 2e-6, (w, e, ref)
        errs.append(e)
    assert errs[0] > errs[1] > errs[2]


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_fourierrec_16bit(dtype):
    q, theta = _case(3, 48, 64, 5)
    got = host(tcp.fourierrec(to_dev(q, dtype), theta, 32.3, n=64))
    assert rel(got, fr.backproject_exact(q, theta, 32.3, 64)) <= 5e-3


def test_fourierrec_scale_strides_and_special_angles():
    rng = np.random.default_rng(9)
    nz, nt, nd, n = 2, 6, 24, 24
    q = rng.normal(size=(nz, nt, nd))
    theta = np.array([0.0, np.pi / 2, np.pi / 2, 1.0, np.pi, 2.5])  # axis-aligned and repeated angles
    big = torch.zeros((nz, nt, nd + 9), dtype=torch.float32, device=DEV)
    big[:, :, 4:4 + nd] = to_dev(q)
    view = big[:, :, 4:4 + nd]  # row stride nd + 9, offset start
    got = host(tcp.fourierrec(view, theta, 12.0, n=n, scale=np.pi / nt))
    want = fr.backproject_exact(q, theta, 12.0, n) * (np.pi / nt)
    assert rel(got, want) <= 1e-5


def test_fourierrec_no_angles_gives_zeros():
    out = torch.full((2, 8, 8), 7.0, device=DEV)
    tcp.fourierrec(torch.zeros((2, 0, 8), device=DEV), np.zeros(0), 4.0, out=out)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0


def test_fourierrec_full_size_sampled():
    # 2048 angles x 2048 detector pixels -> 2048^2 slices, 18 slices = 9 pairs
    # (two workspace batches, the second ragged); sampled voxels against the
    # exact sums
    nz, nt, nd, n = 18, 2048, 2048, 2048
    rng = np.random.default_rng(2048)
    theta = np.arange(nt) * (np.pi / nt)
    g = torch.Generator(device=DEV).manual_seed(7)
    sino = torch.randn((nz, nt, nd), generator=g, device=DEV)
    center = nd / 2 + 0.37
    vol = tcp.fourierrec(sino, theta, center, n=n)
    torch.cuda.synchronize()
    for z in (0, 9, 17):
        ix = rng.integers(0, n, 10)
        iy = rng.integers(0, n, 10)
        want = fr.backproject_exact_points(host(sino[z]), theta, center, n, ix, iy)
        got = host(vol[z])[iy, ix]
        assert rel(got, want) <= 1e-5, z


@pytest.mark.parametrize("where", ["device", "host"])
@pytest.mark.parametrize("dt", [torch.float32, torch.float16])
def test_fbp_fourierrec_ellipsoids(where, dt):
    import oracle
    import synth
    ds = synth.ellipsoid_dataset(ntheta=60, ndet=48, nz=5, count=10, seed=4)
    raw = torch.from_numpy(np.ascontiguousarray(ds.raw, np.uint16).view(np.int16))
    dark = torch.from_numpy(np.ascontiguousarray(ds.dark, np.uint16).view(np.int16))
    flat = torch.from_numpy(np.ascontiguousarray(ds.flat, np.uint16).view(np.int16))
    if where == "device":
        raw, dark, flat = raw.to(DEV), dark.to(DEV), flat.to(DEV)
    else:
        raw = raw.pin_memory()
    got = tcp.fbp(raw, dark, flat, ds.theta, ds.center, dtype=dt, chunk_nz=3, algorithm="fourierrec")
    torch.cuda.synchronize()
    nd = ds.raw.shape[2]
    p = oracle.normalize(ds.raw, oracle.frame_mean(ds.dark), oracle.frame_mean(ds.flat))
    q = oracle.filter_sino(p, ds.center, "shepp", "edge")
    ref = fr.backproject_exact(q, ds.theta, nd / 2.0, nd)
    assert rel(host(got), ref) <= (1e-5 if dt == torch.float32 else 5e-3)


def test_fourierrec_after_cache_clear():
    # the cached twiddle, deconvolution and sorted-angle tables are rebuilt
    q, theta = _case(2, 24, 32, 21)
    a = host(tcp.fourierrec(to_dev(q), theta, 16.3, n=32))
    tcp.cache_clear()
    b = host(tcp.fourierrec(to_dev(q), theta, 16.3, n=32))
    np.testing.assert_array_equal(a, b)


def test_fourierrec_angles_outside_half_turn():
    # angles in [-pi, 2 pi): folded to [0, pi) with the sign of k flipped
    rng = np.random.default_rng(12)
    nz, nt, nd, n = 3, 40, 48, 48
    q = rng.normal(size=(nz, nt, nd))
    theta = rng.uniform(-np.pi, 2 * np.pi, nt)
    got = host(tcp.fourierrec(to_dev(q), theta, 23.6, n=n))
    assert rel(got, fr.backproject_exact(q, theta, 23.6, n)) <= 1e-5


def test_fourierrec_4096_wide_sampled():
    # n = ndet = 4096: grid L = 8192 and period M = 8192 (odd powers of two:
    # the FFTs end with a radix-2 stage), one-column strips in the column pass
    nz, nt, nd, n = 2, 24, 4096, 4096
    rng = np.random.default_rng(4096)
    theta = np.sort(rng.uniform(0, np.pi, nt))
    q = rng.normal(size=(nz, nt, nd))
    vol = tcp.fourierrec(to_dev(q), theta, nd / 2 - 0.3, n=n)
    torch.cuda.synchronize()
    for z in range(nz):
        ix = rng.integers(0, n, 12)
        iy = rng.integers(0, n, 12)
        want = fr.backproject_exact_points(q[z], theta, nd / 2 - 0.3, n, ix, iy)
        assert rel(host(vol[z])[iy, ix], want) <= 1e-5, z


@pytest.mark.parametrize("nd,n", [(2, 2), (3, 4), (5, 6), (1, 2)])
def test_fourierrec_tiny(nd, n):
    # grids of 4 and 8 points (window clamped to the grid), single-stage FFTs
    rng = np.random.default_rng(nd * 10 + n)
    q = rng.normal(size=(3, 7, nd))
    theta = np.sort(rng.uniform(0, np.pi, 7))
    got = host(tcp.fourierrec(to_dev(q), theta, nd / 2 + 0.2, n=n))
    assert rel(got, fr.backproject_exact(q, theta, nd / 2 + 0.2, n)) <= 1e-5
