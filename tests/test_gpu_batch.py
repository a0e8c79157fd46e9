"""Batched uneven datasets in one persistent, graph-captured launch.

Six stacks of widths {512, 768, 1024, 1536, 2048, 2560} and angle counts
{400, 900, 1200, 1800, 2048, 3000}, 32 slices each, distinct centres, uint16
frames with dark/flat, FP16 sinogram storage and FP32 accumulation, the
backprojector configuration autotuned on the batch.  Parity against the FP64
oracle on sampled voxels of one slice per dataset (5e-3, reduced precision).
"""
import numpy as np
import pytest
import torch

import oracle
import synth.gpu as sgpu
import paper_2209_08450_gb300 as tcp
from paper_2209_08450_gb300.batch import Batch, autotune_backproject

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

WIDTHS = (512, 768, 1024, 1536, 2048, 2560)
ANGLES = (400, 900, 1200, 1800, 2048, 3000)


@pytest.fixture(autouse=True)
def _checked():
    tcp.set_checked(True)
    yield
    tcp.device_check()
    tcp.set_checked(False)


def _host_u16(t):
    return t.cpu().numpy().view(np.uint16)


def _datasets(widths, angles, nz, seed0=10, vdt=torch.float32):
    out = []
    for i, (n, nt) in enumerate(zip(widths, angles)):
        raw, dark, flat, theta, c, mu = sgpu.ellipsoid_frames(n, nt, nz, seed=seed0 + i, device=DEV, count=24)
        out.append(dict(raw=raw, dark=dark, flat=flat, theta=theta, center=c,
                        vol=torch.empty((nz, n, n), dtype=vdt, device=DEV)))
    return out


def _means(t, z):
    if t.dim() == 2:  # already FP32 means [nz][ndet]
        return t[z:z + 1].double().cpu().numpy()
    return oracle.frame_mean(_host_u16(t[:, z:z + 1]))


def _check_sampled(d, z, tol, seed=0):
    raw = _host_u16(d["raw"][:, z:z + 1])
    dm, fm = _means(d["dark"], z), _means(d["flat"], z)
    q = oracle.filter_sino(oracle.normalize(raw, dm, fm), d["center"], d.get("filter", "shepp"))[0]
    n = d["vol"].shape[-1]
    rng = np.random.default_rng(seed)
    ix, iy = rng.integers(0, n, 1500), rng.integers(0, n, 1500)
    ref = oracle.backproject_points(q, d["theta"], raw.shape[-1] / 2.0, n, ix, iy)
    got = d["vol"][z].double().cpu().numpy()[iy, ix]
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= tol, err
    return err


def test_uneven_batch_graph_replay_matches_oracle():
    ds = _datasets(WIDTHS, ANGLES, 32)
    b = Batch(ds, sino_dtype=torch.float16, autotune=True)
    info = b.info()
    # the autotuner picks among the CUDA-core configurations (one persistent
    # launch) and the tensor-core kernel (one launch per dataset, one or two
    # blocks per SM)
    if info["kernel"] == 0:
        assert info["config"] in {(8, 16, 4), (4, 32, 4), (4, 16, 4), (16, 8, 2), (8, 16, 2), (2, 16, 4), (1, 32, 4)}
        assert info["grid_blocks"] >= 152
    else:
        assert info["kernel"] in (1, 3) and info["config"][1] in (1, 2)
    assert info["tuned_ms"] > 0
    print("\nbatch autotune: kernel %d config %s, %.1f ms" % (info["kernel"], info["config"], info["tuned_ms"]))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(s)
    s.synchronize()
    first = [d["vol"].clone() for d in ds]
    for d in ds:
        d["vol"].zero_()
    b.capture(s)
    torch.cuda.synchronize()
    assert all(torch.count_nonzero(d["vol"]) == 0 for d in ds)  # capture executes nothing
    b.replay(s)
    s.synchronize()
    for d, f in zip(ds, first):
        assert torch.equal(d["vol"], f)  # deterministic: each unit is computed by one block
    for i, d in enumerate(ds):
        _check_sampled(d, z=(7 * i + 3) % 32, tol=5e-3, seed=i)
    b.close()


def test_batch_of_one_equals_fbp_and_fp32_sinogram():
    ds = _datasets((96, 130), (150, 77), 9, seed0=3)
    for d in ds:
        d["dark"] = tcp.frame_mean(d["dark"])  # F32 means form
    b = Batch(ds, sino_dtype=torch.float32, autotune=False)
    b.run()
    torch.cuda.synchronize()
    for d in ds:
        ref = tcp.fbp(d["raw"], d["dark"], d["flat"], d["theta"], d["center"], sino_dtype=torch.float32)
        torch.cuda.synchronize()
        assert torch.allclose(d["vol"], ref, rtol=0, atol=1e-6 * float(ref.abs().max()))
        _check_sampled(d, z=4, tol=1e-5)
    b.close()


def test_uneven_batch_on_each_kernel_matches_oracle():
    # both backprojectors of a batch, forced: the persistent CUDA-core launch
    # and the tensor-core launches (one and two blocks per SM), on three of
    # the uneven shapes
    ds = _datasets((512, 1536, 2560), (400, 1800, 3000), 32, seed0=20)
    for cfg in ((8, 16, 4, 0), (8, 2, 4, 1), (8, 1, 4, 3)):
        b = Batch(ds, sino_dtype=torch.float16, autotune=False, config=cfg)
        assert b.info()["kernel"] == cfg[3]
        b.run()
        torch.cuda.synchronize()
        for i, d in enumerate(ds):
            _check_sampled(d, z=(11 * i + 5) % 32, tol=5e-3, seed=40 + i)
        b.close()


def test_batch_rejects_bad_items():
    ds = _datasets((64,), (20,), 2)
    ds[0]["vol"] = ds[0]["vol"][:, :, :63]  # not square
    with pytest.raises(tcp.TcpError):
        Batch(ds, autotune=False)


def test_autotune_single_call_picks_a_config_and_is_used():
    g = torch.Generator(device=DEV)
    g.manual_seed(0)
    q = torch.randn((16, 300, 512), generator=g, device=DEV)
    vol = torch.empty((16, 512, 512), device=DEV)
    th = np.linspace(0, np.pi, 300, endpoint=False)
    cfg, ms = autotune_backproject(q, th, 256.0, vol)
    assert ms > 0
    assert tcp.get_backproject_config(16, 300, 512, 512) == cfg
    ref = oracle.backproject(q[:1].double().cpu().numpy(), th, 256.0, 512)
    got = tcp.backproject(q, th, 256.0, out=vol)[:1].double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
