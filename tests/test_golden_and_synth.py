"""Paper-printed FP16 facts and sanity pins of the synthetic-input generators."""
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_fp16_examples():
    # Sec. 2.1 prints three FP16 facts; numpy's IEEE binary16 reproduces them.
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fp16_examples.txt"))
            if l.strip() and not l.startswith("#")]
    for op, a, b, expect in rows:
        if op == "sub":
            got = np.float16(a) - np.float16(b)
        elif op == "mul":
            with np.errstate(over="ignore"):
                got = np.float16(a) * np.float16(b)
        else:
            got = np.finfo(np.float16).max
        assert float(got) == float(expect)
    # A 16-bit detector count does not fit in FP16 (65535 > 65504).
    with np.errstate(over="ignore"):
        assert np.isinf(np.float16(65535.0))


def test_disk_line_integral_is_chord_length():
    th = np.array([0.0, 0.7, 2.0])
    p = synth.ellipse_sinogram([(0.0, 0.0, 5.0, 5.0, 0.3, 2.0)], th, 21, 10.0)
    t = np.arange(21) - 10.0
    ref = np.where(np.abs(t) < 5, 2 * 2.0 * np.sqrt(np.maximum(25 - t ** 2, 0)), 0)
    assert np.max(np.abs(p - ref[None])) < 1e-12


def test_ellipse_integral_conserves_area():
    th = synth.uniform_theta(7)
    ell = [(15.0, -20.0, 900.0, 400.0, 0.4, 1.0)]
    p = synth.ellipse_sinogram(ell, th, 4001, 2000.0)  # unit-spaced samples
    # the integral over s of every projection is the area pi A B (midpoint rule)
    area = np.pi * 900.0 * 400.0
    assert np.max(np.abs(p.sum(axis=1) - area)) < 1e-4 * area


def test_rasterized_area():
    img = synth.rasterize_ellipses([(0.0, 0.0, 20.0, 10.0, 0.5, 1.0)], 64, supersample=8)
    assert abs(img.sum() - np.pi * 200.0) / (np.pi * 200.0) < 0.01


def test_porous_solid_fraction_and_bounds():
    rng = np.random.default_rng(0)
    s = synth.porous_spheres(rng, 1024, 128)
    x0, y0, z0, r, rho = s.T
    assert np.all((r >= 3) & (r <= 40)) and np.all((rho >= 0.2) & (rho <= 1.0))
    assert np.all(np.hypot(x0, y0) + r <= 0.45 * 1024 + 1e-9)
    frac = (4 / 3 * np.pi * r ** 3).sum() / (np.pi * (0.45 * 1024) ** 2 * 128)
    assert 0.4 <= frac < 0.41


def test_frames_statistics_and_seed():
    p = np.zeros((50, 2, 40))
    p[:, :, 10:30] = 1.0
    raw, dark, flat, mu = synth.frames_from_line_integrals(p, np.random.default_rng(1), 4e4, 10, 10)
    assert raw.dtype == np.uint16 and raw.shape == p.shape
    assert abs(mu - 2.0) < 1e-15
    assert abs(dark.mean() - 100) < 1.0
    assert abs(flat.mean() - 40100) < 20
    assert abs(raw[:, :, 15].mean() - (4e4 * np.exp(-2) + 100)) < 10
    raw2, *_ = synth.frames_from_line_integrals(p, np.random.default_rng(1), 4e4, 10, 10)
    assert np.array_equal(raw, raw2)


def test_torch_sphere_generator_matches_host_closed_form():
    import synth.gpu as sgpu
    rng = np.random.default_rng(0)
    sp = synth.porous_spheres(rng, 256, 64)
    zs = np.arange(3) + 0.5
    th = synth.uniform_theta(90)
    a = sgpu.sphere_line_integrals(sp, zs, th, 256, 128.0, "cpu").numpy()
    b = np.stack([synth.sphere_sinogram(sp, z, th, 256, 128.0) for z in zs], 1)
    assert np.max(np.abs(a - b)) < 1e-5 * np.max(np.abs(b)) * 256


def test_torch_ellipsoid_generator_statistics():
    import synth.gpu as sgpu
    raw, dark, flat, theta, c, mu = sgpu.ellipsoid_frames(64, 30, 3, seed=1, device="cpu", count=8)
    assert raw.shape == (30, 3, 64) and dark.shape == (20, 3, 64) and flat.shape == (20, 3, 64)
    u = raw.numpy().view(np.uint16)
    assert u.max() <= 2e4 + 1000 and u.min() >= 0
    assert abs(dark.numpy().view(np.uint16).mean() - 100) < 2
    assert 31.5 - 2 <= c <= 31.5 + 2


def test_oracle_and_library_share_no_code():
    # the FP64 oracle and the CUDA library are independent: no source of the
    # package imports, loads or includes anything of the oracle, and the
    # oracle neither imports the package nor includes its headers; the input
    # generators (synth) hold none of the method's arithmetic and import neither
    import glob
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

    def sources(d, exts):
        return [p for e in exts for p in glob.glob(os.path.join(root, d, "**", "*" + e), recursive=True)]

    pkg = sources("paper_2209_08450_gb300", (".py", ".cu", ".cuh", ".h")) + sources("include", (".h",))
    for p in pkg:
        text = open(p).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), p
        assert "liboracle" not in text and "tcp_oracle" not in text, p
    for p in sources("oracle", (".py", ".c", ".h")):
        text = open(p).read()
        assert not re.search(r"^\s*(import|from)\s+paper_2209_08450_gb300\b", text, re.M), p
        assert not re.search(r'#include\s+"(tcp|tcp_internal)', text), p
        assert "libtcp" not in text, p
    for p in sources("synth", (".py",)):
        text = open(p).read()
        assert not re.search(r"^\s*(import|from)\s+(oracle|paper_2209_08450_gb300)\b", text, re.M), p
