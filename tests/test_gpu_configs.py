"""Oracle parity of the library's DEFAULT reconstruction paths at the sizes of
the benchmark workloads.

`tcp.fbp` with no options reconstructs an FP32 volume from FP16 hi/lo sinogram
pairs on the tensor cores (split mode: 32-angle TMEM segments added into FP32
running sums), and FP16/BF16 volumes from 16-bit sinograms on the tensor
cores once a chunk holds 32 slices or more.  These tests run exactly those
paths on:
  * the plain Shepp-Logan FBP workload in full (256 angles, 256 pixels x 16
    slices, centre 128);
  * the 1024-pixel, 1500-angle random-ellipsoid workload on 32 seeded slices
    (FP32, FP16, BF16);
  * the 2048-pixel, 2048-angle porous-medium workload on a 256-slice chunk
    (64 TMEM segments per voxel, full 128/256-slice CTAs), compared on sampled
    voxels of several slices.
Every compared voxel enters the relative L2 error; the bar is 1e-5 for FP32
volumes and 5e-3 for 16-bit storage.  The measured errors are printed.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import synth.gpu as sgpu
import paper_2209_08450_gb300 as tcp

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
TOL = {torch.float32: 1e-5, torch.float16: 5e-3, torch.bfloat16: 5e-3}


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def u16(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint16).view(np.int16)).to(DEV)


def np_u16(t):
    return t.cpu().numpy().view(np.uint16)


def _report(name, err, tol, n_vox):
    print("\n%s: rel-L2 %.3e over %d voxels (bar %.0e)" % (name, err, n_vox, tol))


def _default_kernel(nz, nt, nd, n, vdt):
    sd = "f16x2" if vdt == torch.float32 else vdt
    return tcp.get_backproject_config(nz, nt, nd, n, sd, vdt)[3]


# ---------------------------------------------- Shepp-Logan 256^2 x 16, full --

@pytest.fixture(scope="module")
def shepp():
    ds = synth.shepp_logan_dataset()  # 256 angles, 256 x 16 slices, centre 128, I0 4e4
    ref = oracle.fbp(ds.raw, ds.dark, ds.flat, ds.theta, ds.center, "shepp")
    return ds, ref


def test_shepp_logan_256_default_fp32_path(shepp):
    ds, ref = shepp
    assert _default_kernel(16, 256, 256, 256, torch.float32) == 1  # FP16 hi/lo pairs on the tensor cores
    out = tcp.fbp(u16(ds.raw), u16(ds.dark), u16(ds.flat), ds.theta, ds.center)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    err = rel(got, ref)
    _report("Shepp-Logan 256^2 x 16 FP32 (default)", err, 1e-5, got.size)
    assert err <= 1e-5
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16])
def test_shepp_logan_256_16bit_tensor_cores(shepp, dt):
    # 16 slices pick the CUDA-core kernel by default; force the tensor-core
    # kernel so that its 16-bit path is held to the oracle at this size too
    ds, ref = shepp
    for kernel in (None, 1, 3):
        try:
            if kernel:
                tcp.set_backproject_config(8, 2, 4, kernel=kernel)
            out = tcp.fbp(u16(ds.raw), u16(ds.dark), u16(ds.flat), ds.theta, ds.center, dtype=dt)
            torch.cuda.synchronize()
        finally:
            tcp.set_backproject_config(None)
        got = out.double().cpu().numpy()
        err = rel(got, ref)
        _report("Shepp-Logan 256^2 x 16 %s (kernel %s)" % (dt, kernel or "default"), err, 5e-3, got.size)
        assert err <= 5e-3


# ---------------------------- random ellipsoids 1024^2, 1500 angles, 32 slices --

@pytest.fixture(scope="module")
def ellipsoids_1024():
    raw, dark, flat, theta, center, mu = sgpu.ellipsoid_frames(1024, 1500, 32, seed=2, device=DEV, count=64)
    assert 509.5 <= center <= 513.5
    ref = oracle.fbp(np_u16(raw), np_u16(dark), np_u16(flat), theta, center, "shepp")
    return raw, dark, flat, theta, center, ref


@pytest.mark.parametrize("dt", [torch.float32, torch.float16, torch.bfloat16])
def test_ellipsoids_1024_1500_angles_default_paths(ellipsoids_1024, dt):
    raw, dark, flat, theta, center, ref = ellipsoids_1024
    assert _default_kernel(32, 1500, 1024, 1024, dt) == (1 if dt == torch.float32 else 3)
    out = tcp.fbp(raw, dark, flat, theta, center, dtype=dt)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    err = rel(got, ref)
    _report("ellipsoids 1024^2 x 32, 1500 angles, %s (default)" % dt, err, TOL[dt], got.size)
    assert err <= TOL[dt]
    if dt == torch.float32:
        assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_ellipsoids_1024_host_buffers_match_device(ellipsoids_1024):
    # the end-to-end form (pinned host raw, host volume) of the same call
    raw, dark, flat, theta, center, ref = ellipsoids_1024
    raw_h = raw.cpu().pin_memory()
    out = tcp.fbp(raw_h, dark.cpu(), flat.cpu(), theta, center)
    torch.cuda.synchronize()
    assert out.device.type == "cpu"
    err = rel(out.double().numpy(), ref)
    _report("ellipsoids 1024^2 x 32 FP32 from host buffers", err, 1e-5, out.numel())
    assert err <= 1e-5


# ------------------------- porous medium 2048^2, 2048 angles, 256-slice chunk --

@pytest.fixture(scope="module")
def porous_2048():
    nz = 256
    z = np.arange(1024 - nz // 2, 1024 + nz // 2)
    raw, dark, flat, theta, center, mu = sgpu.porous_frames(2048, 2048, 2048, seed=0, device=DEV, slices=z)
    return raw, dark, flat, theta, center


def _sampled_ref(raw, dark, flat, theta, center, zs, npts, seed):
    """FP64 oracle at npts seeded voxels of each slice in zs."""
    rng = np.random.default_rng(seed)
    n = raw.shape[-1]
    out = []
    for z in zs:
        p = oracle.normalize(np_u16(raw[:, z:z + 1]), oracle.frame_mean(np_u16(dark[:, z:z + 1])),
                             oracle.frame_mean(np_u16(flat[:, z:z + 1])))
        q = oracle.filter_sino(p, center, "shepp")[0]
        ix, iy = rng.integers(0, n, npts), rng.integers(0, n, npts)
        out.append((z, ix, iy, oracle.backproject_points(q, theta, n / 2.0, n, ix, iy)))
    return out


@pytest.mark.parametrize("dt", [torch.float32, torch.float16, torch.bfloat16])
def test_porous_2048_2048_angles_256_slices_default_paths(porous_2048, dt):
    raw, dark, flat, theta, center = porous_2048
    nz, n = raw.shape[1], raw.shape[2]
    # 16-bit: kernel 3, which runs a 256-slice block at one block per SM (kernel 1)
    assert _default_kernel(nz, 2048, n, n, dt) == (1 if dt == torch.float32 else 3)
    out = tcp.fbp(raw, dark, flat, theta, center, dtype=dt)  # one 256-slice chunk
    torch.cuda.synchronize()
    # slices at both ends of the chunk, in the middle, and at the 128-slice
    # boundary of the split kernel's CTAs
    zs = [0, 1, 63, 127, 128, 200, 254, 255]
    got_all, ref_all = [], []
    for z, ix, iy, ref in _sampled_ref(raw, dark, flat, theta, center, zs, 3000, 7):
        got = out[z].double().cpu().numpy()[iy, ix]
        got_all.append(got)
        ref_all.append(ref)
        assert rel(got, ref) <= TOL[dt], "slice %d" % z
    err = rel(np.concatenate(got_all), np.concatenate(ref_all))
    _report("porous 2048^2 x 256, 2048 angles, %s (default)" % dt, err, TOL[dt], sum(len(g) for g in got_all))
    assert err <= TOL[dt]
