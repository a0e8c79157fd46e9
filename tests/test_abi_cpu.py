"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
function include/tcp.h declares, and rejects bad arguments on the host (no
compute call is made without a GPU)."""
import ctypes

import pytest

from paper_2209_08450_gb300 import _lib
from paper_2209_08450_gb300 import build as tcp_build


@pytest.fixture(scope="module")
def lib():
    tcp_build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _lib.header_functions()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(lib):
    assert lib.tcp_version() == 1
    assert lib.tcp_status_string(0) == b"ok"
    assert lib.tcp_status_string(2) == b"invalid shape"


def _t(dtype, shape, ptr=4096):
    d = _lib.TcpTensor()
    d.data = ptr
    d.dtype = dtype
    d.ndim = len(shape)
    st = 1
    for i in reversed(range(len(shape))):
        d.shape[i] = shape[i]
        d.stride[i] = st
        st *= shape[i]
    return d


def _status(lib, name, *args):
    return getattr(lib, name)(*args)


def test_host_side_argument_checks(lib):
    th = (ctypes.c_double * 4)(0, 0.5, 1.0, 1.5)
    sino = _t(_lib.F32, (2, 4, 16))
    vol = _t(_lib.F32, (2, 16, 16), ptr=1 << 20)
    # null tensor
    assert _status(lib, "tcp_backproject", None, th, 8.0, ctypes.byref(vol), None) == 1
    # wrong slice count
    bad = _t(_lib.F32, (3, 16, 16), ptr=1 << 20)
    assert _status(lib, "tcp_backproject", ctypes.byref(sino), th, 8.0, ctypes.byref(bad), None) == 2
    assert b"slice" in lib.tcp_last_error()
    # non-square volume
    bad = _t(_lib.F32, (2, 16, 15), ptr=1 << 20)
    assert _status(lib, "tcp_backproject", ctypes.byref(sino), th, 8.0, ctypes.byref(bad), None) == 2
    # u16 volume is not a float dtype
    bad = _t(_lib.U16, (2, 16, 16), ptr=1 << 20)
    assert _status(lib, "tcp_backproject", ctypes.byref(sino), th, 8.0, ctypes.byref(bad), None) == 3
    # non-unit innermost stride
    bad = _t(_lib.F32, (2, 16, 16), ptr=1 << 20)
    bad.stride[2] = 2
    assert _status(lib, "tcp_backproject", ctypes.byref(sino), th, 8.0, ctypes.byref(bad), None) == 4
    # non-finite centre and angle
    assert _status(lib, "tcp_backproject", ctypes.byref(sino), th, float("nan"), ctypes.byref(vol), None) == 1
    th_bad = (ctypes.c_double * 4)(0, float("inf"), 1.0, 1.5)
    assert _status(lib, "tcp_project", ctypes.byref(vol), th_bad, 8.0, ctypes.byref(sino), None) == 1
    # overlapping input and output
    alias = _t(_lib.F32, (2, 16, 16), ptr=4096 + 64)
    assert _status(lib, "tcp_backproject", ctypes.byref(sino), th, 8.0, ctypes.byref(alias), None) == 10
    # filter: unknown kind, unknown pad, too wide
    assert _status(lib, "tcp_filter_ex", ctypes.byref(sino), 7, 8.0, 0, 0, None) == 1
    assert _status(lib, "tcp_filter_ex", ctypes.byref(sino), 0, 8.0, 5, 0, None) == 1
    wide = _t(_lib.F32, (1, 2, 5000))
    assert _status(lib, "tcp_filter_ex", ctypes.byref(wide), 0, 8.0, 0, 0, None) == 9
    # normalize: shapes and dtypes
    raw = _t(_lib.U16, (4, 2, 16))
    dark = _t(_lib.F32, (2, 16), ptr=1 << 24)
    out = _t(_lib.F32, (2, 4, 16), ptr=1 << 26)
    badout = _t(_lib.F32, (4, 2, 16), ptr=1 << 26)
    assert _status(lib, "tcp_normalize", ctypes.byref(raw), ctypes.byref(dark), ctypes.byref(dark),
                   ctypes.byref(badout), None) == 2
    rawf = _t(_lib.F32, (4, 2, 16))
    assert _status(lib, "tcp_normalize", ctypes.byref(rawf), ctypes.byref(dark), ctypes.byref(dark),
                   ctypes.byref(out), None) == 3
    darku = _t(_lib.U16, (2, 16), ptr=1 << 24)
    assert _status(lib, "tcp_normalize", ctypes.byref(raw), ctypes.byref(darku), ctypes.byref(dark),
                   ctypes.byref(out), None) == 3
    # config that is not instantiated
    c = _lib.BpConfig(3, 16, 4, 0)
    assert _status(lib, "tcp_set_backproject_config", ctypes.byref(c)) == 9
    # kernel ids: 3 (tensor cores, two blocks per SM) exists, 4 does not
    for ks, kern, want in ((2, 4, 9), (8, 4, 9), (8, 3, 0), (2, 3, 0)):
        c = _lib.BpConfig(ks, 2, 4, kern)
        assert _status(lib, "tcp_set_backproject_config", ctypes.byref(c)) == want
    assert _status(lib, "tcp_set_backproject_config", None) == 0


def test_split_sinogram_descriptor_checks(lib):
    # F16X2 must be 4-d [2][nz][ntheta][ndet] with non-overlapping planes;
    # rejected before any device work
    raw = _t(_lib.U16, (10, 4, 32), ptr=1 << 20)
    dark = _t(_lib.F32, (4, 32), ptr=1 << 21)
    flat = _t(_lib.F32, (4, 32), ptr=1 << 22)
    bad3 = _t(_lib.F16X2, (4, 10, 32), ptr=1 << 23)
    assert _status(lib, "tcp_normalize_filter", ctypes.byref(raw), ctypes.byref(dark), ctypes.byref(flat),
                   ctypes.byref(bad3), 0, 16.0, 0, None) == 2
    three = _t(_lib.F16X2, (3, 4, 10, 32), ptr=1 << 23)
    assert _status(lib, "tcp_normalize_filter", ctypes.byref(raw), ctypes.byref(dark), ctypes.byref(flat),
                   ctypes.byref(three), 0, 16.0, 0, None) == 2
    ovl = _t(_lib.F16X2, (2, 4, 10, 32), ptr=1 << 23)
    ovl.stride[0] = 16  # planes overlap
    assert _status(lib, "tcp_normalize_filter", ctypes.byref(raw), ctypes.byref(dark), ctypes.byref(flat),
                   ctypes.byref(ovl), 0, 16.0, 0, None) == 4
    pair = _t(_lib.F16X2, (2, 4, 10, 32), ptr=1 << 23)
    assert _status(lib, "tcp_normalize", ctypes.byref(raw), ctypes.byref(dark), ctypes.byref(flat),
                   ctypes.byref(pair), None) == 3  # only the fused normalise + filter writes pairs


def test_try_centers_argument_checks(lib):
    raw = _t(_lib.U16, (10, 4, 32), ptr=1 << 20)
    dark = _t(_lib.F32, (4, 32), ptr=1 << 21)
    flat = _t(_lib.F32, (4, 32), ptr=1 << 22)
    vol = _t(_lib.F32, (2, 32, 32), ptr=1 << 23)
    th = (ctypes.c_double * 10)(*[0.1 * i for i in range(10)])
    cs = (ctypes.c_double * 2)(16.0, 17.0)
    bad = (ctypes.c_double * 2)(16.0, float("inf"))
    assert _status(lib, "tcp_try_centers", ctypes.byref(raw), 4, ctypes.byref(dark), ctypes.byref(flat), th, cs, 2,
                   ctypes.byref(vol), 0, None) == 1  # slice outside [0, nz)
    assert _status(lib, "tcp_try_centers", ctypes.byref(raw), 1, ctypes.byref(dark), ctypes.byref(flat), th, bad, 2,
                   ctypes.byref(vol), 0, None) == 1  # non-finite centre
    assert _status(lib, "tcp_try_centers", ctypes.byref(raw), 1, ctypes.byref(dark), ctypes.byref(flat), th, cs, 3,
                   ctypes.byref(vol), 0, None) == 2  # vol is not [ncenters][n][n]


def test_detector_width_limit(lib):
    # padded rows must fit shared memory: ndet <= 4096, checked before any device work
    wide = _t(_lib.F32, (1, 2, 4097), ptr=1 << 20)
    assert _status(lib, "tcp_filter", ctypes.byref(wide), 0, 2048.0, None) == 9


def test_default_config_query(lib):
    c = _lib.BpConfig()
    assert lib.tcp_get_backproject_config(64, 2048, 2048, 2048, 3, 3, ctypes.byref(c)) == 0
    assert c.k_slices in (1, 2, 4, 8, 16) and c.theta_stage in (8, 16, 32)


def test_fourierrec_argument_checks(lib):
    th = (ctypes.c_double * 4)(0, 0.5, 1.0, 1.5)
    sino = _t(_lib.F32, (2, 4, 16))
    vol = _t(_lib.F32, (2, 16, 16), ptr=1 << 20)
    odd = _t(_lib.F32, (2, 15, 15), ptr=1 << 20)
    assert _status(lib, "tcp_fourierrec", ctypes.byref(sino), th, 8.0, ctypes.byref(odd), 1.0, 0, None) == 2
    assert b"even" in lib.tcp_last_error()
    for w in (1, 17):
        assert _status(lib, "tcp_fourierrec", ctypes.byref(sino), th, 8.0, ctypes.byref(vol), 1.0, w, None) == 1
    pair = _t(_lib.F16X2, (2, 2, 4, 16))
    assert _status(lib, "tcp_fourierrec", ctypes.byref(pair), th, 8.0, ctypes.byref(vol), 1.0, 0, None) == 3
    wide = _t(_lib.F32, (2, 4, 8193))
    assert _status(lib, "tcp_fourierrec", ctypes.byref(wide), th, 8.0, ctypes.byref(vol), 1.0, 0, None) == 2
    assert _status(lib, "tcp_fourierrec", ctypes.byref(sino), th, float("nan"), ctypes.byref(vol), 1.0, 0,
                   None) == 1


def test_fbp_algorithm_checks(lib):
    raw = _t(_lib.U16, (4, 2, 16), ptr=1 << 20)
    dark = _t(_lib.F32, (2, 16), ptr=1 << 21)
    flat = _t(_lib.F32, (2, 16), ptr=1 << 22)
    vol = _t(_lib.F32, (2, 16, 16), ptr=1 << 23)
    th = (ctypes.c_double * 4)(0, 0.5, 1.0, 1.5)
    o = _lib.FbpOpts()
    o.algorithm = 7
    assert _status(lib, "tcp_fbp", ctypes.byref(raw), ctypes.byref(dark), ctypes.byref(flat), th, 8.0,
                   ctypes.byref(vol), ctypes.byref(o), None) == 1
    o.algorithm = _lib.ALGORITHMS["fourierrec"]
    o.sino_dtype = _lib.F16X2
    assert _status(lib, "tcp_fbp", ctypes.byref(raw), ctypes.byref(dark), ctypes.byref(flat), th, 8.0,
                   ctypes.byref(vol), ctypes.byref(o), None) == 3
    o.sino_dtype = -1
    odd = _t(_lib.F32, (2, 15, 15), ptr=1 << 23)
    assert _status(lib, "tcp_fbp", ctypes.byref(raw), ctypes.byref(dark), ctypes.byref(flat), th, 8.0,
                   ctypes.byref(odd), ctypes.byref(o), None) == 2


def test_try_centers_ex_algorithm_checks(lib):
    raw = _t(_lib.U16, (10, 4, 32), ptr=1 << 20)
    dark = _t(_lib.F32, (4, 32), ptr=1 << 21)
    flat = _t(_lib.F32, (4, 32), ptr=1 << 22)
    th = (ctypes.c_double * 10)(*[0.1 * i for i in range(10)])
    cs = (ctypes.c_double * 2)(16.0, 17.0)
    vol = _t(_lib.F32, (2, 32, 32), ptr=1 << 23)
    assert _status(lib, "tcp_try_centers_ex", ctypes.byref(raw), 1, ctypes.byref(dark), ctypes.byref(flat), th, cs,
                   2, ctypes.byref(vol), 0, 9, 0, None) == 1  # unknown algorithm
    odd = _t(_lib.F32, (2, 31, 31), ptr=1 << 23)
    assert _status(lib, "tcp_try_centers_ex", ctypes.byref(raw), 1, ctypes.byref(dark), ctypes.byref(flat), th, cs,
                   2, ctypes.byref(odd), 0, 1, 0, None) == 2  # FourierRec needs an even n


@pytest.mark.parametrize("name", ["tcp_normalize", "tcp_normalize_noalloc"])
def test_normalize_rejects_misaligned_and_aliased_buffers(lib, name):
    # both normalisation calls check every descriptor on the host before any
    # launch: a U16 pointer at an odd address or an F32 pointer off its 4-byte
    # alignment is TCP_ERR_ALIGN, a sinogram overlapping raw is TCP_ERR_ALIAS
    fn = getattr(lib, name)
    fn.argtypes = [ctypes.POINTER(_lib.TcpTensor)] * 4 + [ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    raw = _t(_lib.U16, (4, 2, 16), ptr=1 << 20)
    dark = _t(_lib.U16, (3, 2, 16), ptr=1 << 21)
    flat = _t(_lib.U16, (3, 2, 16), ptr=1 << 22)
    out = _t(_lib.F32, (2, 4, 16), ptr=1 << 23)
    args = lambda r, d, f, o: (ctypes.byref(r), ctypes.byref(d), ctypes.byref(f), ctypes.byref(o), None)
    odd_raw = _t(_lib.U16, (4, 2, 16), ptr=(1 << 20) + 1)
    assert fn(*args(odd_raw, dark, flat, out)) == 4
    odd_dark = _t(_lib.U16, (3, 2, 16), ptr=(1 << 21) + 1)
    assert fn(*args(raw, odd_dark, flat, out)) == 4
    off_out = _t(_lib.F32, (2, 4, 16), ptr=(1 << 23) + 2)
    assert fn(*args(raw, dark, flat, off_out)) == 4
    strided = _t(_lib.U16, (4, 2, 16), ptr=1 << 20)
    strided.stride[2] = 2
    assert fn(*args(strided, dark, flat, out)) == 4
    alias = _t(_lib.F32, (2, 4, 16), ptr=(1 << 20) + 64)  # inside raw's 256 bytes
    assert fn(*args(raw, dark, flat, alias)) == 10
    assert b"overlap" in lib.tcp_last_error()


def test_plan_create_validates_its_arguments(lib):
    # every check of tcp_plan_create runs on the host before any CUDA call
    th = (ctypes.c_double * 4)(0, 0.5, 1.0, 1.5)
    h = ctypes.c_void_p(1234)

    def desc(**kw):
        d = _lib.PlanDesc()
        d.ntheta, d.nz, d.ndet, d.n, d.center, d.vol_dtype = 4, 8, 32, 0, 16.0, _lib.F32
        d.opts.sino_dtype = -1
        for k, v in kw.items():
            setattr(d, k, v)
        return d

    create = lambda d, t=th: lib.tcp_plan_create(ctypes.byref(d), t, ctypes.byref(h))
    assert lib.tcp_plan_create(None, th, ctypes.byref(h)) == 1 and h.value is None
    assert lib.tcp_plan_create(ctypes.byref(desc()), th, None) == 1
    assert create(desc(ntheta=0)) == 2
    assert create(desc(nz=-1)) == 2
    assert create(desc(ndet=0)) == 2
    assert create(desc(vol_dtype=_lib.U16)) == 3
    assert create(desc(io=4)) == 1
    assert create(desc(host_frames=-1)) == 1
    assert create(desc(center=float("nan"))) == 1
    assert create(desc(), None) == 1
    bad = (ctypes.c_double * 4)(0, float("inf"), 1.0, 1.5)
    assert create(desc(), bad) == 1
    assert b"theta" in lib.tcp_last_error()
    # calls on a null plan are rejected, destroying NULL is accepted
    t = _t(_lib.F32, (2, 4, 32))
    assert lib.tcp_fbp_plan(None, ctypes.byref(t), ctypes.byref(t), ctypes.byref(t), ctypes.byref(t), None) == 1
    assert lib.tcp_filter_plan(None, ctypes.byref(t), None) == 1
    assert lib.tcp_backproject_plan(None, ctypes.byref(t), 16.0, ctypes.byref(t), 1.0, None) == 1
    assert lib.tcp_project_plan(None, ctypes.byref(t), 16.0, ctypes.byref(t), None) == 1
    assert lib.tcp_plan_info(None, None, None) == 1
    assert lib.tcp_plan_destroy(None) == 0


def test_lprec_argument_checks(lib):
    # host-side checks of tcp_lprec, made before any device work
    sino = _t(_lib.F32, (2, 6, 16))
    vol = _t(_lib.F32, (2, 16, 16), ptr=1 << 20)
    eq = (ctypes.c_double * 6)(*[i * 3.141592653589793 / 6 for i in range(6)])
    uneq = (ctypes.c_double * 6)(*[i * 3.141592653589793 / 6 + (0.01 if i == 2 else 0) for i in range(6)])
    full = (ctypes.c_double * 6)(*[i * 2 * 3.141592653589793 / 6 for i in range(6)])
    assert lib.tcp_lprec(ctypes.byref(sino), uneq, 8.0, ctypes.byref(vol), 1.0, 2.0, None) == 1
    assert b"equally spaced" in lib.tcp_last_error()
    assert lib.tcp_lprec(ctypes.byref(sino), full, 8.0, ctypes.byref(vol), 1.0, 2.0, None) == 1
    assert b"half turn" in lib.tcp_last_error()
    assert lib.tcp_lprec(ctypes.byref(sino), eq, 8.0, ctypes.byref(vol), 1.0, 40.0, None) == 1  # oversampling
    two = _t(_lib.F32, (2, 2, 16))
    assert lib.tcp_lprec(ctypes.byref(two), eq, 8.0, ctypes.byref(vol), 1.0, 2.0, None) == 2
    pair = _t(_lib.F16X2, (2, 2, 6, 16))
    assert lib.tcp_lprec(ctypes.byref(pair), eq, 8.0, ctypes.byref(vol), 1.0, 2.0, None) == 3
    assert lib.tcp_lprec(ctypes.byref(sino), eq, float("nan"), ctypes.byref(vol), 1.0, 2.0, None) == 1
    # tcp_fbp: LpRec oversampling outside 1..8
    raw = _t(_lib.U16, (6, 2, 16), ptr=1 << 22)
    dark = _t(_lib.F32, (2, 16), ptr=1 << 23)
    o = _lib.FbpOpts()
    o.algorithm = _lib.ALGORITHMS["lprec"]
    o.width = 9
    assert lib.tcp_fbp(ctypes.byref(raw), ctypes.byref(dark), ctypes.byref(dark), eq, 8.0, ctypes.byref(vol),
                       ctypes.byref(o), None) == 1


def test_padded_length_matches_the_oracle_rule(lib):
    import oracle
    for nd in (1, 12, 20, 24, 38, 40, 45, 76, 100, 200, 300, 1024, 1536, 2048, 2560, 4096):
        assert lib.tcp_padded_length(nd, 0) == oracle.padded_length(nd)
        assert lib.tcp_padded_length(nd, 2) == oracle.padded_length(nd, "smooth"), nd
    assert lib.tcp_padded_length(0, 0) == -1


def _tc_shape(lib, nz, sdt, stage, blocks):
    sh = _lib.TcShape()
    st = lib.tcp_tc_launch_shape(nz, sdt, stage, blocks, ctypes.byref(sh))
    return st, (sh.slices_per_block, sh.angles_per_stage, sh.blocks_per_sm, sh.weight_stages,
                sh.sinogram_stages, sh.smem_bytes)


@pytest.mark.parametrize("nz,sdt,stage,blocks,want", [
    # FP16, 32 slices, two angles per stage: two blocks per SM fit (2 x 64
    # TMEM columns; rings in half of the 228 KB: 2 weight + 11 sinogram
    # stages, 113440 bytes), one block takes 16 sinogram stages
    (32, _lib.F16, 2, 2, (32, 2, 2, 2, 11, 113440)),
    (32, _lib.F16, 2, 1, (32, 2, 1, 2, 16, 133920)),
    (20, _lib.BF16, 2, 2, (32, 2, 2, 2, 11, 113440)),
    (1, _lib.F16, 1, 2, (16, 1, 2, 3, 32, 84768)),
    # 128 slices: 256 TMEM columns each, two blocks with two sinogram stages
    (128, _lib.F16, 2, 2, (128, 2, 2, 2, 2, 101152)),
    # 144- and 256-slice blocks need more than half the TMEM: one block
    (130, _lib.F16, 1, 2, (144, 1, 1, 3, 19, 227104)),
    (256, _lib.F16, 2, 2, (256, 2, 1, 2, 5, 232224)),
    # FP16 hi/lo pairs: 128 slices, one angle per stage, 4 weight + 6 sinogram
    # stages of both planes, always one block (accumulators and sums fill TMEM)
    (256, _lib.F16X2, 2, 2, (128, 1, 1, 4, 6, 232224)),
])
def test_tensor_core_launch_shape(lib, nz, sdt, stage, blocks, want):
    st, got = _tc_shape(lib, nz, sdt, stage, blocks)
    assert st == 0 and got == want
    assert got[5] <= 232448  # opt-in shared memory per block
    if got[2] == 2:
        assert 2 * (got[5] + 1024) <= 233472  # two blocks per SM, 1 KB reserved each
        assert 2 * (2 * got[0]) <= 512        # both blocks' TMEM accumulators


def test_tensor_core_launch_shape_errors(lib):
    assert _tc_shape(lib, 0, _lib.F16, 2, 2)[0] == 1
    assert _tc_shape(lib, 32, _lib.F32, 2, 2)[0] == 3
    assert lib.tcp_tc_launch_shape(32, _lib.F16, 2, 2, None) == 1


def test_tensor_core_launch_shape_from_python():
    import torch

    import paper_2209_08450_gb300 as tcp
    sh = tcp.tc_launch_shape(32, torch.float16)
    assert (sh["slices_per_block"], sh["blocks_per_sm"], sh["smem_bytes"]) == (32, 2, 113440)
    assert tcp.tc_launch_shape(256, "f16x2")["sinogram_stages"] == 6


def test_tensor_core_launch_shape_limits_hold_for_every_slice_count(lib):
    # every shape the launcher can pick fits the SM: shared memory per block
    # within the opt-in limit (and two blocks with their reserved 1 KB within
    # the SM's 228 KB), both blocks' TMEM accumulators within 512 columns,
    # at least two sinogram stages and no more weight stages than sinogram
    # stages, slices per block a multiple of 16 covering nz or capped
    for sdt in (_lib.F16, _lib.BF16, _lib.F16X2):
        for stage in (1, 2):
            for blocks in (1, 2):
                for nz in range(1, 601):
                    st, (N, S, b, na, nbb, smem) = _tc_shape(lib, nz, sdt, stage, blocks)
                    assert st == 0
                    split = sdt == _lib.F16X2
                    assert N % 16 == 0 and N >= min(nz, 16) and N <= (128 if split else 256)
                    assert N >= nz or N == (128 if split else 256)
                    assert S == (1 if split or stage == 1 else 2)
                    assert 1 <= b <= (1 if split else blocks)
                    assert 2 <= nbb and na <= nbb and na >= 2
                    assert smem <= 232448
                    if b == 2:
                        assert 2 * (smem + 1024) <= 233472
                        cols = 2 * N
                        alloc = 32 if cols <= 32 else 1 << (cols - 1).bit_length()
                        assert 2 * alloc <= 512


def test_tensor_core_blocks_that_share_an_sm_fit_its_tensor_memory(lib):
    # Blocks of any tensor-core launches (side streams can run several at
    # once) that fit one SM's shared memory together (each + 1 KB reserved)
    # also fit its 512 TMEM columns, so no block's allocation waits on another.
    import itertools
    shapes = set()
    for sdt in (_lib.F16, _lib.BF16, _lib.F16X2):
        for stage in (1, 2):
            for blocks in (1, 2):
                for nz in range(1, 300):
                    st, (N, S, b, na, nbb, smem) = _tc_shape(lib, nz, sdt, stage, blocks)
                    assert st == 0
                    cols = 512 if sdt == _lib.F16X2 else 2 * N
                    shapes.add((smem, 32 if cols <= 32 else 1 << (cols - 1).bit_length()))
    for k in (2, 3, 4):
        for combo in itertools.combinations_with_replacement(sorted(shapes), k):
            if sum(s + 1024 for s, _ in combo) <= 233472:
                assert sum(a for _, a in combo) <= 512, combo


def test_batch_argument_checks(lib):
    # rejected on the host before any device work; *out stays NULL
    out = ctypes.c_void_p(1)
    item = _lib.BatchItem()
    item.raw = _t(_lib.U16, (10, 2, 16), ptr=1 << 20)
    item.vol = _t(_lib.F32, (2, 16, 16), ptr=1 << 21)
    item.dark = item.flat = _t(_lib.F32, (2, 16), ptr=1 << 22)
    th = (ctypes.c_double * 10)(*[0.1 * k for k in range(10)])
    item.theta = ctypes.cast(th, ctypes.c_void_p)
    item.center = 8.0
    items = (_lib.BatchItem * 1)(item)
    assert lib.tcp_batch_create(items, 1, None, None, None) == 1  # null output handle
    assert lib.tcp_batch_create(None, 1, None, None, ctypes.byref(out)) == 1 and not out.value
    out = ctypes.c_void_p(1)
    assert lib.tcp_batch_create(items, 0, None, None, ctypes.byref(out)) == 1 and not out.value
    opts = _lib.BatchOpts()
    opts.sino_dtype = _lib.U16
    out = ctypes.c_void_p(1)
    assert lib.tcp_batch_create(items, 1, ctypes.byref(opts), None, ctypes.byref(out)) == 3 and not out.value
    # host pointers (or no GPU at all): refused, nothing created
    out = ctypes.c_void_p(1)
    assert lib.tcp_batch_create(items, 1, None, None, ctypes.byref(out)) != 0 and not out.value
    for fn in ("tcp_batch_run", "tcp_batch_capture", "tcp_batch_replay"):
        assert getattr(lib, fn)(None, None) == 1
    assert lib.tcp_batch_info(None, None, None, None, None) == 1
    assert lib.tcp_batch_destroy(None) == 0


def test_plan_argument_checks(lib):
    # the description and angles are checked on the host before any device
    # work; *out stays NULL on every refusal
    th = (ctypes.c_double * 8)(*[0.1 * k for k in range(8)])

    def desc(**kw):
        d = _lib.PlanDesc()
        d.ntheta, d.nz, d.ndet, d.n, d.center, d.vol_dtype = 8, 4, 32, 32, 16.0, _lib.F32
        for k, v in kw.items():
            setattr(d, k, v)
        return d

    def create(d, theta=th):
        out = ctypes.c_void_p(1)
        st = lib.tcp_plan_create(ctypes.byref(d) if d is not None else None, theta, ctypes.byref(out))
        assert not out.value
        return st

    assert lib.tcp_plan_create(ctypes.byref(desc()), th, None) == 1  # null output handle
    assert create(None) == 1
    assert create(desc(ntheta=0)) == 2
    assert create(desc(nz=-1)) == 2
    assert create(desc(vol_dtype=_lib.U16)) == 3
    assert create(desc(io=4)) == 1
    assert create(desc(host_frames=-1)) == 1
    assert create(desc(center=float("nan"))) == 1
    assert create(desc(), None) == 1
    bad = (ctypes.c_double * 8)(*([0.0] * 7 + [float("inf")]))
    assert create(desc(), bad) == 1
    assert lib.tcp_plan_destroy(None) == 0
    assert lib.tcp_plan_info(None, None, None) == 1
    cnt = ctypes.c_int64()
    assert lib.tcp_plan_trace(None, None, 0, ctypes.byref(cnt)) == 1


def test_lprec_shape_dtype_and_alias_checks(lib):
    # more host-side refusals of tcp_lprec (the angle checks are above), all
    # before any device work
    import math
    nt, nd, n = 12, 32, 32
    sino = _t(_lib.F32, (2, nt, nd), ptr=1 << 20)
    vol = _t(_lib.F32, (2, n, n), ptr=1 << 24)
    eq = (ctypes.c_double * nt)(*[k * math.pi / nt for k in range(nt)])

    def call(s=sino, th=eq, c=16.0, v=vol, scale=1.0, os=2.0):
        return _status(lib, "tcp_lprec", ctypes.byref(s), th, c, ctypes.byref(v), scale, os, None)

    assert call(scale=float("nan")) == 1
    assert call(s=_t(_lib.U16, (2, nt, nd), ptr=1 << 20)) == 3
    assert call(v=_t(_lib.F32, (3, n, n), ptr=1 << 24)) == 2          # slice counts differ
    assert call(v=_t(_lib.F32, (2, n, n + 1), ptr=1 << 24)) == 2      # not square
    assert call(c=float("inf")) == 1
    assert call(th=None) == 1
    assert call(v=_t(_lib.F32, (2, n, n), ptr=(1 << 20) + 64)) == 10   # vol overlaps sino


def test_missing_library_fails_loudly(tmp_path):
    # no CPU or PyTorch fallback: without the built library the binding raises
    import os
    import subprocess
    import sys
    code = ("import paper_2209_08450_gb300._lib as L\n"
            "try:\n    L.load(%r)\nexcept RuntimeError as e:\n    print('raised', 'not built' in str(e))\n"
            % str(tmp_path / "libtcp.so"))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "raised True" in r.stdout
