"""GPU parity: every CUDA kernel against the FP64 oracle on the same seeded inputs.

Tolerances: relative L2 <= 1e-5 for FP32 storage, <= 5e-3 for FP16/BF16
storage (FP32 accumulation), per result.  Sizes span several 32x32 tiles and
leave ragged tails (n, ndet, nz, ntheta not multiples of the tile, the slice
block or the angle stage).
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2209_08450_gb300 as tcp

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
TOL = {torch.float32: 1e-5, torch.float16: 5e-3, torch.bfloat16: 5e-3}


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def u16(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint16).view(np.int16)).to(DEV)


def host(t):
    return t.double().cpu().numpy()


@pytest.fixture(autouse=True)
def _checked():
    tcp.set_checked(True)
    yield
    tcp.device_check()
    tcp.set_checked(False)


# ------------------------------------------------------------- backproject --

def _bp_case(nz, nt, nd, n, center, seed, uniform=False):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(nz, nt, nd))
    theta = synth.uniform_theta(nt) if uniform else rng.uniform(-0.3, 2 * np.pi, nt)
    return q, theta, center


@pytest.mark.parametrize("nz,nt,nd,n,center", [
    (11, 181, 203, 200, 101.37), (3, 64, 96, 96, 48.0), (1, 7, 33, 70, 20.5), (17, 37, 64, 33, 31.9)])
def test_backproject_fp32(nz, nt, nd, n, center):
    q, theta, c = _bp_case(nz, nt, nd, n, center, nz * 1000 + nt)
    got = host(tcp.backproject(to_dev(q), theta, c, n=n))
    ref = oracle.backproject(q, theta, c, n)
    assert rel(got, ref) <= 1e-5
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))



def _angle_major(x):
    """The same values stored [theta][z][j] (planes first for F16X2), viewed [z][theta][j]."""
    if x.dim() == 4:
        return x.permute(0, 2, 1, 3).contiguous().permute(0, 2, 1, 3)
    return x.permute(1, 0, 2).contiguous().permute(1, 0, 2)


@pytest.mark.parametrize("kind,kernel,nz", [("f32", 0, 13), ("f32", 2, 13), ("f16", 1, 40), ("bf16", 1, 33),
                                            ("f16x2", 1, 131), ("f16x2", 1, 20), ("f16", 0, 5)])
def test_backproject_angle_major_sinograms_give_identical_volumes(kind, kernel, nz):
    # tcp_backproject reads any strides; the angle-major layout (what tcp_fbp's
    # chunks and normalize_filter use) changes the tensor-core kernel's copy
    # shape, not its arithmetic: the volumes are bit-identical, and equal to
    # the oracle within the path's tolerance
    nt, nd, n, c = 67, 96, 90, 47.6
    q, theta, _ = _bp_case(nz, nt, nd, n, c, 100 + nz)
    if kind == "f16x2":
        v = to_dev(q) * 1024.0
        hi = v.half()
        sino = torch.stack([hi, (v - hi.float()).half()])
        scale, vdt, tol = 1.0 / 1024.0, torch.float32, 1e-5
    else:
        dt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[kind]
        sino, scale, vdt = to_dev(q, dt), 1.0, torch.float32
        tol = 1e-5 if kind == "f32" else 5e-3
    try:
        tcp.set_backproject_config(8 if kind == "f32" else 4, 16, 4, kernel=kernel)
        a = tcp.backproject(sino, theta, c, n=n, dtype=vdt, scale=scale)
        b = tcp.backproject(_angle_major(sino), theta, c, n=n, dtype=vdt, scale=scale)
        torch.cuda.synchronize()
    finally:
        tcp.set_backproject_config(None)
    assert torch.equal(a, b)
    assert rel(host(b), oracle.backproject(q, theta, c, n)) <= tol


def test_normalize_filter_output_is_angle_major_and_equals_a_contiguous_output():
    ds = synth.shepp_logan_dataset(ntheta=48, ndet=80, nz=6, center=40.3, seed=9)
    raw, dark, flat = u16(ds.raw), u16(ds.dark), u16(ds.flat)
    for dt in (torch.float32, torch.float16, "f16x2"):
        got = tcp.normalize_filter(raw, dark, flat, ds.center, dtype=dt)
        split = dt == "f16x2"
        if split:
            assert got.stride() == (48 * 6 * 80, 80, 6 * 80, 1)
            ref = torch.empty((2, 6, 48, 80), dtype=torch.float16, device=DEV)
        else:
            assert got.stride() == (80, 6 * 80, 1)
            ref = torch.empty((6, 48, 80), dtype=dt, device=DEV)
        tcp.normalize_filter(raw, dark, flat, ds.center, out=ref)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


@pytest.mark.parametrize("cfg", [(8, 16, 4), (4, 32, 4), (4, 16, 4), (16, 8, 2), (8, 16, 2), (2, 16, 4),
                                 (1, 32, 4), (4, 16, 16), (2, 16, 16), (4, 32, 16), (8, 16, 16)])
def test_backproject_every_config(cfg):
    q, theta, c = _bp_case(13, 50, 70, 65, 35.2, 7)
    ref = oracle.backproject(q, theta, c, 65)
    try:
        tcp.set_backproject_config(*cfg)
        got = host(tcp.backproject(to_dev(q), theta, c, n=65))
    finally:
        tcp.set_backproject_config(None)
    assert rel(got, ref) <= 1e-5


@pytest.mark.parametrize("sdt", [torch.float16, torch.bfloat16, torch.float32])
@pytest.mark.parametrize("vdt", [torch.float16, torch.bfloat16, torch.float32])
def test_backproject_16bit_storage(sdt, vdt):
    q, theta, c = _bp_case(9, 120, 100, 96, 50.5, 3, uniform=True)
    qd = to_dev(q, sdt)
    got = host(tcp.backproject(qd, theta, c, n=96, dtype=vdt))
    # against the oracle on the stored (rounded) samples and on the exact ones
    ref_stored = oracle.backproject(host(qd), theta, c, 96)
    ref_exact = oracle.backproject(q, theta, c, 96)
    tol = max(TOL[sdt], TOL[vdt])
    assert rel(got, ref_stored) <= tol
    assert rel(got, ref_exact) <= tol


@pytest.mark.parametrize("nz,nt,nd,n,center", [
    (11, 181, 203, 200, 101.37), (3, 64, 96, 96, 48.0), (1, 7, 33, 70, 20.5), (17, 37, 64, 33, 31.9)])
def test_backproject_register_reuse_blocks(nz, nt, nd, n, center):
    # 4 x 4 voxel blocks per thread walking the less-varying axis (checked
    # mode is on: a floor step other than 0 or +1 would set the error word);
    # angles over two turns cover all four walk directions
    q, theta, c = _bp_case(nz, nt, nd, n, center, nz * 1000 + nt)
    ref = oracle.backproject(q, theta, c, n)
    for cfg in ((4, 16, 16), (8, 16, 16)):
        try:
            tcp.set_backproject_config(*cfg)
            got = host(tcp.backproject(to_dev(q), theta, c, n=n))
        finally:
            tcp.set_backproject_config(None)
        assert rel(got, ref) <= 1e-5
        assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))
    assert tcp.device_check() == 0


@pytest.mark.parametrize("cfg", [(8, 16, 4), (16, 8, 4), (4, 16, 4), (8, 16, 8)])
@pytest.mark.parametrize("nz,nt,nd,n,center", [
    (11, 181, 203, 200, 101.37), (3, 64, 96, 96, 48.0), (1, 7, 33, 70, 20.5), (17, 37, 64, 33, 31.9)])
def test_backproject_slice_pairs(cfg, nz, nt, nd, n, center):
    # kernel 2: FP32 slice pairs with packed FMAs and sample reuse down each
    # column (checked mode is on: a floor step other than 0 or +1 along the
    # walk sets the error word); odd slice counts leave half a pair
    q, theta, c = _bp_case(nz, nt, nd, n, center, nz * 1000 + nt)
    ref = oracle.backproject(q, theta, c, n)
    try:
        tcp.set_backproject_config(*cfg, kernel=2)
        got = host(tcp.backproject(to_dev(q), theta, c, n=n))
        got16 = host(tcp.backproject(to_dev(q), theta, c, n=n, dtype=torch.float16))
    finally:
        tcp.set_backproject_config(None)
    assert rel(got, ref) <= 1e-5
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))
    assert rel(got16, ref) <= 5e-3
    assert tcp.device_check() == 0


def test_backproject_slice_pairs_special_angles():
    # sin exactly 0, +-1, +-1/sqrt(2) and just inside / outside the 0.99 reuse bound
    q, _, c = _bp_case(6, 18, 80, 72, 40.25, 9)
    th = np.array([0.0, np.pi / 4, np.pi / 2, 3 * np.pi / 4, np.pi, 5 * np.pi / 4, 3 * np.pi / 2, 7 * np.pi / 4,
                   np.arcsin(0.99) - 1e-6, np.arcsin(0.99) + 1e-6, np.pi - np.arcsin(0.99), -np.arcsin(0.99) + 1e-7,
                   1e-7, np.pi / 2 + 1e-7, -np.pi / 4, 3.9269, 1.4, -1.4])
    ref = oracle.backproject(q, th, c, 72)
    try:
        tcp.set_backproject_config(8, 16, 4, kernel=2)
        got = host(tcp.backproject(to_dev(q), th, c, n=72))
    finally:
        tcp.set_backproject_config(None)
    assert rel(got, ref) <= 1e-5
    assert tcp.device_check() == 0


def test_backproject_register_reuse_axis_aligned_and_diagonal_angles():
    # slopes of exactly 0, +-1/sqrt(2) and +-1 sit on the walk-axis switch
    q, _, c = _bp_case(5, 16, 80, 72, 40.25, 9)
    theta = np.array([0.0, np.pi / 4, np.pi / 2, 3 * np.pi / 4, np.pi, 5 * np.pi / 4, 3 * np.pi / 2, 7 * np.pi / 4,
                      0.7853, 0.7855, 2.3561, 2.3563, 1e-7, np.pi / 2 + 1e-7, -np.pi / 4, 3.9269])
    ref = oracle.backproject(q, theta, c, 72)
    try:
        tcp.set_backproject_config(4, 16, 16)
        got = host(tcp.backproject(to_dev(q), theta, c, n=72))
    finally:
        tcp.set_backproject_config(None)
    assert rel(got, ref) <= 1e-5
    assert tcp.device_check() == 0


def test_backproject_special_angles_and_constant():
    n, nd, nt = 64, 64, 17
    theta = synth.uniform_theta(nt)
    got = host(tcp.backproject(torch.full((2, nt, nd), 1.5, device=DEV), theta, nd / 2, n=n))
    c = np.arange(n) - n / 2
    X, Y = np.meshgrid(c, c)
    inside = X ** 2 + Y ** 2 < (nd / 2 - 1.5) ** 2
    assert np.max(np.abs(got[:, inside] - 1.5 * nt)) < 1e-4
    q = np.random.default_rng(0).normal(size=(1, 1, nd))
    b = host(tcp.backproject(to_dev(q), np.array([0.0]), nd / 2, n=n))[0]
    assert np.max(np.abs(b - np.broadcast_to(q[0], (n, n)))) < 1e-6


def test_backproject_edge_cases():
    th = np.array([0.3, 1.1])
    # empty slice count
    out = tcp.backproject(torch.zeros((0, 2, 8), device=DEV), th, 4.0, n=8)
    assert out.shape == (0, 8, 8)
    # no angles: zero volume
    out = tcp.backproject(torch.zeros((2, 0, 8), device=DEV), np.zeros(0), 4.0, n=8)
    assert torch.count_nonzero(out) == 0
    # one voxel, one detector pixel
    q = np.array([[[2.0]]])
    got = host(tcp.backproject(to_dev(q), np.array([0.0]), 0.0, n=1))
    assert abs(got[0, 0, 0] - oracle.backproject(q, np.array([0.0]), 0.0, 1)[0, 0, 0]) < 1e-6
    # non-contiguous (strided) volume output
    big = torch.zeros((3, 40, 48), device=DEV)
    view = big[:, 2:34, 5:37]
    q, theta, c = _bp_case(3, 20, 40, 32, 19.0, 11)
    tcp.backproject(to_dev(q), theta, c, out=view)
    assert rel(host(view), oracle.backproject(q, theta, c, 32)) <= 1e-5
    assert torch.count_nonzero(big[:, :2]) == 0 and torch.count_nonzero(big[:, :, :5]) == 0


def test_backproject_large_detector_offsets():
    # a centre far from ndet/2 and a volume wider than the detector
    q, theta, c = _bp_case(2, 45, 50, 90, -7.25, 5)
    got = host(tcp.backproject(to_dev(q), theta, c, n=90))
    assert rel(got, oracle.backproject(q, theta, c, 90)) <= 1e-5


# ----------------------------------------------------------------- project --

@pytest.mark.parametrize("nz,nt,nd,n,center", [(5, 67, 91, 80, 44.6), (9, 30, 40, 64, 33.0), (1, 5, 17, 9, 8.2),
                                               (21, 50, 70, 64, 33.3), (32, 19, 48, 40, 20.0), (16, 9, 24, 33, 12.5),
                                               (16, 11, 31, 40, 15.2), (16, 13, 62, 50, 30.9), (16, 7, 63, 48, -3.0)])
def test_project_fp32(nz, nt, nd, n, center):
    # 16-slice groups read the slice-interleaved copies, the remainder the plain
    # and transposed volume (21 = 16 + 4 + 1); widths 31, 62 and 63 end in a
    # partial 32-bin warp, and a centre of -3 puts bin 0 inside the object
    rng = np.random.default_rng(nz + nt)
    vol = rng.normal(size=(nz, n, n))
    theta = rng.uniform(0, np.pi, nt)
    got = host(tcp.project(to_dev(vol), theta, center, ndet=nd))
    ref = oracle.project(vol, theta, center, nd)
    assert rel(got, ref) <= 1e-5


@pytest.mark.parametrize("nz", [4, 18])
def test_project_is_exact_transpose_on_gpu(nz):
    rng = np.random.default_rng(1)
    n, nt, nd = 100, 73, 111
    theta = rng.uniform(0, np.pi, nt)
    x = to_dev(rng.normal(size=(nz, n, n)))
    y = to_dev(rng.normal(size=(nz, nt, nd)))
    px = tcp.project(x, theta, 52.3, ndet=nd)
    bty = tcp.backproject(y, theta, 52.3, n=n)
    lhs = torch.sum(px.double() * y.double()).item()
    rhs = torch.sum(x.double() * bty.double()).item()
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
def test_project_16bit(dt):
    rng = np.random.default_rng(2)
    vol = rng.uniform(0, 1, size=(3, 64, 64))
    theta = synth.uniform_theta(48)
    vd = to_dev(vol, dt)
    got = host(tcp.project(vd, theta, 32.0, ndet=64, dtype=dt))
    assert rel(got, oracle.project(host(vd), theta, 32.0, 64)) <= 5e-3


# --------------------------------------------------------------- normalize --

@pytest.mark.parametrize("nd", [64, 203])
@pytest.mark.parametrize("means", [False, True])
@pytest.mark.parametrize("dt", [torch.float32, torch.float16, torch.bfloat16])
def test_normalize(nd, means, dt):
    ds = synth.shepp_logan_dataset(ntheta=33, ndet=nd, nz=5, center=nd / 2, seed=nd)
    raw, dark, flat = u16(ds.raw), u16(ds.dark), u16(ds.flat)
    if means:
        dark, flat = tcp.frame_mean(dark), tcp.frame_mean(flat)
        assert rel(host(dark), oracle.frame_mean(ds.dark)) < 1e-7
    got = host(tcp.normalize(raw, dark, flat, dtype=dt))
    ref = oracle.normalize(ds.raw, oracle.frame_mean(ds.dark), oracle.frame_mean(ds.flat))
    assert rel(got, ref) <= TOL[dt]


def test_normalize_special_values_and_strided_chunk():
    raw = np.array([10100, 5100, 100, 50, 65535, 2600, 0, 100], np.uint16).reshape(1, 1, 8)
    raw = np.repeat(raw, 3, axis=1)  # [1][3][8]
    d = np.full((3, 8), 100.0, np.float32)
    f = np.full((3, 8), 10100.0, np.float32)
    f[2] = 100.0  # flat == dark -> clamp
    got = host(tcp.normalize(u16(raw), to_dev(d), to_dev(f)))
    ref = oracle.normalize(raw, d.astype(np.float64), f.astype(np.float64))
    assert np.max(np.abs(got - ref)) < 1e-5
    # a z-chunk of a larger stack is a strided view
    ds = synth.shepp_logan_dataset(ntheta=10, ndet=64, nz=8, center=32.0, seed=1)
    full = u16(ds.raw)
    dm, fm = tcp.frame_mean(u16(ds.dark)), tcp.frame_mean(u16(ds.flat))
    got = host(tcp.normalize(full[:, 3:6], dm[3:6], fm[3:6]))
    ref = oracle.normalize(ds.raw[:, 3:6], oracle.frame_mean(ds.dark)[3:6], oracle.frame_mean(ds.flat)[3:6])
    assert rel(got, ref) <= 1e-6


# ------------------------------------------------------------------ filter --

@pytest.mark.parametrize("nd", [1, 2, 7, 64, 100, 256, 333, 1024, 2048, 2560, 4096])
def test_filter_shepp_edge(nd):
    rng = np.random.default_rng(nd)
    nt = 5
    q = rng.normal(size=(3, nt, nd))
    c = nd / 2 + 1.37
    got = host(tcp.filter_(to_dev(q), c, "shepp"))
    ref = oracle.filter_sino(q, c, "shepp", "edge")
    assert rel(got, ref) <= 1e-5


@pytest.mark.parametrize("kind", ["shepp", "parzen", "ramp", "none"])
@pytest.mark.parametrize("pad", ["edge", "zero"])
def test_filter_kinds_and_pads(kind, pad):
    rng = np.random.default_rng(3)
    q = rng.normal(size=(2, 9, 150)) + 3.0
    got = host(tcp.filter_(to_dev(q), 71.6, kind, pad))
    ref = oracle.filter_sino(q, 71.6, kind, pad)
    assert rel(got, ref) <= 1e-5


@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
def test_filter_16bit(dt):
    rng = np.random.default_rng(4)
    q = rng.uniform(0, 2, size=(4, 31, 256))
    qd = to_dev(q, dt)
    got = host(tcp.filter_(qd, 128.0, "shepp"))
    assert rel(got, oracle.filter_sino(host(to_dev(q, dt)), 128.0, "shepp")) <= 5e-3


def test_filter_explicit_ntheta_and_2d_rows():
    rng = np.random.default_rng(5)
    q = rng.normal(size=(7, 80))
    got = host(tcp.filter_(to_dev(q), 40.0, "ramp", ntheta=100))
    assert rel(got, oracle.filter_sino(q[None], 40.0, "ramp", ntheta=100)[0]) <= 1e-5


# -------------------------------------------------------------- end to end --

def _fbp_gpu(ds, dt=torch.float32, vdt=None, kind="shepp", fused=False):
    if fused:
        sino = tcp.normalize_filter(u16(ds.raw), u16(ds.dark), u16(ds.flat), ds.center, kind, dtype=dt)
    else:
        sino = tcp.normalize(u16(ds.raw), u16(ds.dark), u16(ds.flat), dtype=dt)
        tcp.filter_(sino, ds.center, kind)
    nd = ds.raw.shape[-1]
    return tcp.backproject(sino, ds.theta, nd / 2.0, dtype=vdt or dt)


def test_fbp_shepp_logan_256_fp32():
    ds = synth.shepp_logan_dataset()  # 256 angles, 256 x 16, centre 128, I0 4e4
    got = host(_fbp_gpu(ds))
    ref = oracle.fbp(ds.raw, ds.dark, ds.flat, ds.theta, ds.center, "shepp")
    assert rel(got, ref) <= 1e-5


@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
def test_fbp_shepp_logan_256_16bit(dt):
    # 16-bit storage of the filtered sinogram and the volume (fused
    # normalise+filter rounds once, after filtering)
    ds = synth.shepp_logan_dataset(nz=6)
    got = host(_fbp_gpu(ds, dt, fused=True))
    ref = oracle.fbp(ds.raw, ds.dark, ds.flat, ds.theta, ds.center, "shepp")
    assert rel(got, ref) <= 5e-3


def test_fbp_shepp_logan_fp16_separate_steps():
    # FP16 (11-bit significand) also holds the unfiltered sinogram well enough
    ds = synth.shepp_logan_dataset(nz=4)
    got = host(_fbp_gpu(ds, torch.float16, fused=False))
    ref = oracle.fbp(ds.raw, ds.dark, ds.flat, ds.theta, ds.center, "shepp")
    assert rel(got, ref) <= 5e-3


@pytest.mark.parametrize("nd", [64, 203])
@pytest.mark.parametrize("dt", [torch.float32, torch.float16, torch.bfloat16])
@pytest.mark.parametrize("means", [False, True])
def test_normalize_filter_fused(nd, dt, means):
    ds = synth.shepp_logan_dataset(ntheta=41, ndet=nd, nz=3, center=nd / 2 - 0.7, seed=nd + 1)
    dark, flat = u16(ds.dark), u16(ds.flat)
    if means:
        dark, flat = tcp.frame_mean(dark), tcp.frame_mean(flat)
    got = host(tcp.normalize_filter(u16(ds.raw), dark, flat, ds.center, "shepp", dtype=dt))
    p = oracle.normalize(ds.raw, oracle.frame_mean(ds.dark), oracle.frame_mean(ds.flat))
    ref = oracle.filter_sino(p, ds.center, "shepp", "edge")
    assert rel(got, ref) <= TOL[dt]


def test_fbp_ellipsoids_ragged():
    ds = synth.ellipsoid_dataset(ntheta=150, ndet=173, nz=7, count=20, seed=3)
    got = host(_fbp_gpu(ds, kind="parzen"))
    ref = oracle.fbp(ds.raw, ds.dark, ds.flat, ds.theta, ds.center, "parzen")
    assert rel(got, ref) <= 1e-5


# ---------------------------------------------------------------- pipeline --

@pytest.mark.parametrize("where", ["device", "host"])
@pytest.mark.parametrize("chunk,nbuf", [(5, 2), (16, 2), (3, 3)])
def test_fbp_pipeline(where, chunk, nbuf):
    ds = synth.shepp_logan_dataset(ntheta=120, ndet=96, nz=13, center=47.3, seed=2)
    ref = oracle.fbp(ds.raw, ds.dark, ds.flat, ds.theta, ds.center, "shepp")
    if where == "device":
        raw, dark, flat = u16(ds.raw), u16(ds.dark), u16(ds.flat)
    else:
        raw = torch.from_numpy(ds.raw.view(np.int16)).pin_memory()
        dark = torch.from_numpy(ds.dark.view(np.int16))  # pageable host frames
        flat = torch.from_numpy(ds.flat.view(np.int16)).pin_memory()
    out = tcp.fbp(raw, dark, flat, ds.theta, ds.center, chunk_nz=chunk, n_buffers=nbuf)
    torch.cuda.synchronize()
    assert out.device.type == ("cuda" if where == "device" else "cpu")
    assert rel(host(out), ref) <= 1e-5


def test_fbp_pipeline_16bit_and_means():
    ds = synth.shepp_logan_dataset(ntheta=100, ndet=80, nz=9, center=40.0, seed=4)
    ref = oracle.fbp(ds.raw, ds.dark, ds.flat, ds.theta, ds.center, "shepp")
    dm, fm = tcp.frame_mean(u16(ds.dark)), tcp.frame_mean(u16(ds.flat))
    for dt in (torch.float16, torch.bfloat16):
        out = tcp.fbp(u16(ds.raw), dm, fm, ds.theta, ds.center, dtype=dt, chunk_nz=4)
        torch.cuda.synchronize()
        assert rel(host(out), ref) <= 5e-3


def test_fbp_fp16_many_angles_keeps_filtered_values_in_range():
    # 3000 angles: with pi/N_theta folded into an FP16 sinogram the filtered
    # values would sit in the FP16 subnormal range; the pipeline stores them
    # with a 2^10 headroom and applies pi/N_theta/2^10 in the backprojector.
    import synth.gpu as sgpu
    raw, dark, flat, theta, c, mu = sgpu.ellipsoid_frames(320, 3000, 4, seed=5, device=DEV, count=12)
    nr = raw.cpu().numpy().view(np.uint16)
    ref = oracle.fbp(nr, dark.cpu().numpy().view(np.uint16), flat.cpu().numpy().view(np.uint16), theta, c, "shepp")
    for dt in (torch.float16, torch.bfloat16):
        out = tcp.fbp(raw, dark, flat, theta, c, dtype=dt, chunk_nz=3)
        torch.cuda.synchronize()
        assert rel(host(out), ref) <= 5e-3
    # the same through the public calls
    s = tcp.normalize_filter(raw, dark, flat, c, dtype=torch.float16, weight=1024.0)
    v = tcp.backproject(s, theta, 320 / 2.0, dtype=torch.float32, scale=np.pi / 3000 / 1024.0)
    assert rel(host(v), ref) <= 5e-3


# ------------------------------------------------- tensor-core backprojector --

@pytest.mark.parametrize("stage", [1, 2])
@pytest.mark.parametrize("sdt", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("nz,nt,nd,n,center", [
    (20, 37, 96, 96, 48.0), (3, 50, 72, 70, 35.3), (16, 13, 64, 100, 31.7), (40, 129, 200, 160, 99.2),
    (1, 70, 40, 48, 19.5), (3, 10, 16, 9, 4.2)])
def test_backproject_tensor_cores(sdt, nz, nt, nd, n, center, stage):
    # stage = angles per pipeline stage (the B ring then holds as many stages
    # as shared memory allows); 129 angles leave a ragged last stage
    q, theta, c = _bp_case(nz, nt, nd, n, center, nz + nt + nd)
    qd = to_dev(q, sdt)
    ref = oracle.backproject(host(qd), theta, c, n)
    try:
        tcp.set_backproject_config(8, stage, 4, kernel=1)
        got = host(tcp.backproject(qd, theta, c, n=n, dtype=torch.float32))
        tcp.set_backproject_config(8, 16, 4, kernel=0)
        cuda_core = host(tcp.backproject(qd, theta, c, n=n, dtype=torch.float32))
    finally:
        tcp.set_backproject_config(None)
    assert rel(got, ref) <= 5e-3
    assert rel(got, cuda_core) <= 5e-3


@pytest.mark.parametrize("stage", [1, 2])
def test_backproject_tensor_cores_256_slices_and_scale(stage):
    # one full 256-slice block plus a ragged second block, 16-bit volume
    q, theta, c = _bp_case(300, 24, 64, 64, 32.4, 1)
    qd = to_dev(q, torch.float16)
    try:
        tcp.set_backproject_config(8, stage, 4, kernel=1)
        got = host(tcp.backproject(qd, theta, c, n=64, dtype=torch.float16, scale=0.5))
    finally:
        tcp.set_backproject_config(None)
    ref = 0.5 * oracle.backproject(host(qd), theta, c, 64)
    assert rel(got, ref) <= 5e-3


@pytest.mark.parametrize("stage", [1, 2])
@pytest.mark.parametrize("sdt", [torch.float16, torch.bfloat16])
@pytest.mark.parametrize("nz,nt,nd,n,center", [
    (32, 129, 200, 160, 99.2), (20, 13, 64, 100, 31.7), (48, 37, 96, 96, 48.0), (128, 50, 72, 70, 35.3),
    (130, 24, 64, 64, 32.4)])
def test_backproject_tensor_cores_two_blocks_per_sm(sdt, nz, nt, nd, n, center, stage):
    # kernel 3 sizes the rings for two blocks per SM where the TMEM
    # accumulators (2 x slices per block columns) and the rings fit (130
    # slices take one 144-slice block: one block per SM): the same MMAs in
    # the same order, so the volume is identical to kernel 1's
    q, theta, c = _bp_case(nz, nt, nd, n, center, 7 * nz + nt)
    qd = to_dev(q, sdt)
    try:
        tcp.set_backproject_config(8, stage, 4, kernel=3)
        two = host(tcp.backproject(qd, theta, c, n=n, dtype=torch.float32))
        tcp.set_backproject_config(8, stage, 4, kernel=1)
        one = host(tcp.backproject(qd, theta, c, n=n, dtype=torch.float32))
    finally:
        tcp.set_backproject_config(None)
    assert np.array_equal(two, one)
    assert rel(two, oracle.backproject(host(qd), theta, c, n)) <= 5e-3


def test_backproject_default_for_16bit_sinograms_is_the_two_block_tensor_core_kernel():
    assert tcp.get_backproject_config(64, 720, 512, 512, torch.float16, torch.float32)[3] == 3
    assert tcp.get_backproject_config(256, 2048, 2048, 2048, torch.bfloat16, torch.float16)[3] == 3
    assert tcp.get_backproject_config(16, 720, 512, 512, torch.float16, torch.float32)[3] == 0


# ------------------------------- FP32-accurate split FP16 (F16X2) sinograms --

def _split(q, scale):
    """hi = fp16(q * scale), lo = fp16(q * scale - hi) as a [2][...] tensor."""
    v = to_dev(q) * scale
    hi = v.half()
    lo = (v - hi.float()).half()
    return torch.stack([hi, lo])


@pytest.mark.parametrize("nz,nt,nd,n,center", [
    (20, 37, 96, 96, 48.0), (3, 50, 72, 70, 35.3), (300, 24, 64, 64, 32.4), (1, 70, 40, 48, 19.5),
    (40, 129, 200, 160, 99.2), (2, 33, 16, 9, 4.2)])
def test_backproject_split_fp16_pairs_reach_fp32_tolerance(nz, nt, nd, n, center):
    # three FP16 products per weight/sample pair, accumulated in FP32 on the
    # tensor cores: held to the FP32 tolerance, not the 16-bit one
    q, theta, c = _bp_case(nz, nt, nd, n, center, 7 * nz + nt)
    ref = oracle.backproject(q, theta, c, n)
    got = host(tcp.backproject(_split(q, 1024.0), theta, c, n=n, scale=1.0 / 1024.0))
    assert rel(got, ref) <= 1e-5
    fp32 = host(tcp.backproject(to_dev(q), theta, c, n=n))
    assert rel(got, fp32) <= 1e-5


def test_normalize_filter_split_planes_carry_the_fp32_result():
    ds = synth.shepp_logan_dataset(ntheta=64, ndet=128, nz=5, center=63.2, seed=6)
    raw, dark, flat = u16(ds.raw), u16(ds.dark), u16(ds.flat)
    f32 = tcp.normalize_filter(raw, dark, flat, ds.center, dtype=torch.float32, weight=1024.0)
    sp = tcp.normalize_filter(raw, dark, flat, ds.center, dtype="f16x2", weight=1024.0)
    torch.cuda.synchronize()
    assert sp.shape == (2, 5, 64, 128) and sp.dtype == torch.float16
    v = f32.double()
    pair = sp[0].double() + sp[1].double()
    # |v - hi - lo| <= 2^-22 |v| while lo is normal (|v| >= 2^-3), else <= 2^-25
    bound = torch.clamp(v.abs() * 2.0 ** -22, min=2.0 ** -25) * 1.01
    assert bool(((pair - v).abs() <= bound).all())
    assert bool((sp[0].double() == v.half().double()).all())  # hi is fp16(v)


def test_fbp_default_fp32_volume_uses_split_pairs_and_matches_fp32_sinograms():
    ds = synth.shepp_logan_dataset(ntheta=90, ndet=104, nz=7, center=51.6, seed=8)
    ref = oracle.fbp(ds.raw, ds.dark, ds.flat, ds.theta, ds.center, "shepp")
    raw, dark, flat = u16(ds.raw), u16(ds.dark), u16(ds.flat)
    assert tcp.get_backproject_config(7, 90, 104, 104, "f16x2")[3] == 1
    a = tcp.fbp(raw, dark, flat, ds.theta, ds.center)  # default: F16X2 chunks
    b = tcp.fbp(raw, dark, flat, ds.theta, ds.center, sino_dtype="f16x2", chunk_nz=3)
    c = tcp.fbp(raw, dark, flat, ds.theta, ds.center, sino_dtype=torch.float32)
    torch.cuda.synchronize()
    for v in (a, b, c):
        assert rel(host(v), ref) <= 1e-5
    # two FP32-accurate paths with different rounding orders: the FP32 tolerance
    assert rel(host(a), host(c)) <= 1e-5
    assert torch.equal(a, b)  # slices are independent of the chunking


def test_split_sinogram_rejections():
    q = torch.zeros((2, 4, 10, 36), dtype=torch.float16, device=DEV)  # rows of 72 bytes: not 16-byte aligned
    with pytest.raises(tcp.TcpError):
        tcp.backproject(q, np.linspace(0, np.pi, 10), 18.0, n=36)
    with pytest.raises(tcp.TcpError):  # the in-place filter does not take pairs
        tcp.filter_(torch.zeros((2, 4, 10, 32), dtype=torch.float16, device=DEV), 16.0)


# ------------------------------------------ smooth (3 x 2^k) filter padding --

@pytest.mark.parametrize("nd,pad", [(40, "edge"), (300, "zero"), (24, "edge"), (1536, "edge"), (45, "zero"),
                                    (2560, "edge"), (76, "edge")])
@pytest.mark.parametrize("dt", [torch.float32, torch.float16])
def test_filter_on_smooth_padding(nd, pad, dt):
    # padded lengths 80, 640, 5120, 160 (radix-5 FFT pass) and 48, 3072, 96
    # (radix 3), in place and fused
    rng = np.random.default_rng(nd)
    nz, nt = 3, 5 if nd > 1000 else 17
    q = rng.normal(size=(nz, nt, nd))
    c = nd / 2.0 + 1.37
    ref = oracle.filter_sino(q, c, "shepp", pad, rule="smooth")
    assert tcp.padded_length(nd, smooth=True) == oracle.padded_length(nd, "smooth")
    got = tcp.filter_(to_dev(q, dt), c, "shepp", pad + "_smooth")
    tol = 1e-5 if dt == torch.float32 else 2e-3
    assert rel(host(got), ref) <= tol
    # against the power-of-two padding the result differs (other period) but only slightly
    pow2 = oracle.filter_sino(q, c, "shepp", pad)
    assert rel(ref, pow2) < 0.05


def test_fbp_with_smooth_padding_matches_oracle():
    ds = synth.shepp_logan_dataset(ntheta=80, ndet=96, nz=3, center=47.1, seed=21)
    ref = oracle.fbp(ds.raw, ds.dark, ds.flat, ds.theta, ds.center, "shepp", rule="smooth")
    out = tcp.fbp(u16(ds.raw), u16(ds.dark), u16(ds.flat), ds.theta, ds.center, pad="edge_smooth")
    torch.cuda.synchronize()
    assert tcp.padded_length(96, smooth=True) == 192
    assert rel(host(out), ref) <= 1e-5


@pytest.mark.parametrize("split", [False, True])
def test_tensor_core_window_check_stays_clean(split):
    # checked mode: every weight index is checked against the 32-sample window
    # and any violation is recorded in the device error word; angles over two
    # turns, an axis off the middle, ragged tiles
    rng = np.random.default_rng(31)
    nz, nt, nd, n, c = 40, 96, 200, 184, 123.7
    q = rng.normal(size=(nz, nt, nd))
    theta = rng.uniform(-7.0, 7.0, nt)
    ref = oracle.backproject(q, theta, c, n)
    tcp.set_checked(True)
    try:
        if split:
            got = tcp.backproject(_split(q, 1024.0), theta, c, n=n, scale=1.0 / 1024.0)
            tol = 1e-5
        else:
            qd = to_dev(q, torch.float16)
            got = tcp.backproject(qd, theta, c, n=n, dtype=torch.float32)
            ref = oracle.backproject(host(qd), theta, c, n)
            tol = 5e-3
        torch.cuda.synchronize()
        assert tcp.device_check() == 0
    finally:
        tcp.set_checked(False)
    assert rel(host(got), ref) <= tol
