"""Host-side checks of the C ABI: the library loads, exports every declared symbol, and rejects
bad arguments before any CUDA call (so these run without a GPU)."""
import ctypes
import json
import os
import re

import pytest

import paper_1510_04686_gb300 as negf
from paper_1510_04686_gb300 import negf as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    negf._build.build()
    return negf.library()


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"^\s*[\w\s\*]*?\b(negf_\w+)\s*\(", txt, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"negf_rgf_solve", "negf_lead_selfenergy", "negf_scba_step", "negf_rgf_adjoint"} <= names
    for n in names:
        assert hasattr(lib, n), n


def test_version_defaults_and_strings(lib):
    assert lib.negf_abi_version() == 4
    o = negf.options()
    assert o.eta_lead == 1e-6 and o.eta_device == 1e-6 and o.sr_max_iter == 100
    assert o.precision == negf.PREC_FP64 and o.refine_steps == 2
    assert o.lead_precision == negf.PREC_AUTO and o.refine_max == 6
    assert o.sigma_structure == negf.SIGMA_ORBITAL_DIAG and o.atom_orbitals == 10
    for code in range(9):
        assert lib.negf_status_string(code)
    assert lib.negf_status_string(99) == b"unknown status"


def _dev(n_sys=1, N=4, b=8, hd=1, hu=1):
    return B._Dev(n_sys, N, b, 0, hd, hu)


def test_workspace_size_validation(lib):
    o = negf.options()
    d = _dev()
    for which in (B.WS_LEAD, B.WS_RGF):
        assert lib.negf_workspace_size(ctypes.byref(d), 10, ctypes.byref(o), which) > 0
    assert lib.negf_workspace_size(ctypes.byref(_dev(N=0)), 10, ctypes.byref(o), B.WS_RGF) == 0
    assert lib.negf_workspace_size(ctypes.byref(d), 0, ctypes.byref(o), B.WS_RGF) == 0
    bad = negf.options(precision=7)
    assert lib.negf_workspace_size(ctypes.byref(d), 10, ctypes.byref(bad), B.WS_RGF) == 0
    # the size saturates with the chunk
    o2 = negf.options(chunk=4)
    s4 = lib.negf_workspace_size(ctypes.byref(d), 4, ctypes.byref(o2), B.WS_RGF)
    s100 = lib.negf_workspace_size(ctypes.byref(d), 100, ctypes.byref(o2), B.WS_RGF)
    assert s4 == s100


def test_bad_arguments_rejected_on_host(lib):
    o = negf.options()
    P = ctypes.c_void_p
    fake = P(16)
    d = _dev()
    # missing H_up with N > 1
    r = lib.negf_rgf_solve(ctypes.byref(_dev(hu=0)), 3, fake, fake, None, fake, fake, None, None,
                           None, 0, ctypes.byref(o), None, None, None, None, None, None, fake, fake,
                           1 << 30, None)
    assert r == 1
    # scat_R without scat_L
    r = lib.negf_rgf_solve(ctypes.byref(d), 3, fake, fake, None, fake, fake, fake, None, None,
                           1, ctypes.byref(o), None, None, None, None, None, None, fake, fake, 1 << 30,
                           None)
    assert r == 1
    # workspace too small
    r = lib.negf_rgf_solve(ctypes.byref(d), 3, fake, fake, None, fake, fake, None, None, None,
                           0, ctypes.byref(o), None, None, None, None, None, None, fake, fake, 16,
                           None)
    assert r == 3
    # bad options
    bad = negf.options(kT=0.0)
    r = lib.negf_lead_selfenergy(ctypes.byref(d), 3, fake, fake, ctypes.byref(bad), fake, fake,
                                 None, fake, fake, 1 << 30, None)
    assert r == 1
    r = lib.negf_scba_step(0, 4, 4, fake, 0.01, 0.01, 1, 0.1, 1.0, fake, fake, fake, fake, fake,
                           None)
    assert r == 1
    r = lib.negf_scba_step(1, 4, 4, fake, 0.01, 0.01, 1, 0.1, 0.0, fake, fake, fake, fake, fake,
                           None)
    assert r == 1
    # zero points is a no-op
    r = lib.negf_rgf_solve(ctypes.byref(d), 0, None, None, None, None, None, None, None, None,
                           0, ctypes.byref(o), None, None, None, None, None, None, None, None, 0,
                           None)
    assert r == 0


def test_binding_refuses_cpu_tensors():
    import torch
    with pytest.raises(TypeError):
        negf.Device(torch.zeros((1, 2, 3, 3), dtype=torch.complex128), None)


def test_options_struct_layout():
    # six doubles and eight 32-bit integers, as in include/negf.h
    assert ctypes.sizeof(B._Opt) == 6 * 8 + 10 * 4
    assert ctypes.sizeof(B._Dev) == 4 * 4 + 2 * 8 + 2 * 4
    o = negf.options()
    assert o.sr_host_check == 4


def test_autotune_cache_rejects_stale_records(tmp_path):
    """A cached tensor-core choice is reused only if it was written for this library's set of
    configurations."""
    from paper_1510_04686_gb300 import autotune
    n = autotune._n.tc_config_count()
    good = tmp_path / "good.json"
    good.write_text(json.dumps({"b": 400, "batch": 8, "config": n - 1, "n_configs": n}))
    assert autotune.load_cached(str(good))["config"] == n - 1
    for bad in ({"b": 400, "batch": 8, "config": 1},                        # no count
                {"b": 400, "batch": 8, "config": 1, "n_configs": n + 3},    # other library
                {"b": 400, "batch": 8, "config": n, "n_configs": n},        # out of range
                {"b": 400, "batch": 8, "config": "1", "n_configs": n}):
        p = tmp_path / "bad.json"
        p.write_text(json.dumps(bad))
        assert autotune.load_cached(str(p)) is None
    (tmp_path / "list.json").write_text("[1, 2]")
    assert autotune.load_cached(str(tmp_path / "list.json")) is None
    (tmp_path / "junk.json").write_text("{not json")
    assert autotune.load_cached(str(tmp_path / "junk.json")) is None
    assert autotune.load_cached(str(tmp_path / "missing.json")) is None


def test_mixed_form_rejects_contractions_beyond_its_exact_range(lib):
    """The split-BF16 GEMM keeps 48-bit slices exact for contraction lengths up to 393216; longer
    ones (GEMM K) are refused on the host instead of losing accuracy, and blocks beyond the
    mixed inverse's range (n > 9266) are refused by every sweep entry point."""
    P = ctypes.c_void_p
    fake = P(16)
    mixed, fp64 = B.PREC_MIXED, B.PREC_FP64
    assert lib.negf_zgemm_workspace_size(mixed, 1, 8, 8, 393216) > 0
    assert lib.negf_zgemm_workspace_size(mixed, 1, 8, 8, 393217) == 0
    assert lib.negf_zgemm_workspace_size(fp64, 1, 8, 8, 393217) > 0
    r = lib.negf_zgemm_batched(mixed, 1, 8, 8, 400000, 1.0, 0.0, fake, 0, 400000, 0, fake, 0, 8,
                               0, 0.0, 0.0, fake, 64, 8, fake, 1 << 40, None)
    assert r == 8
    assert lib.negf_zinv_workspace_size(mixed, 1, 28033) == 0
    r = lib.negf_zinv_batched(mixed, 1, 28033, fake, fake, 2, fake, fake, 1 << 40, None)
    assert r == 8
    big = _dev(b=28033)
    o_mixed = negf.options(precision=mixed)
    assert lib.negf_workspace_size(ctypes.byref(big), 1, ctypes.byref(o_mixed), B.WS_RGF) == 0
    r = lib.negf_rgf_solve(ctypes.byref(big), 1, fake, fake, None, fake, fake, None, None, None,
                           0, ctypes.byref(o_mixed), None, None, None, None, None, None, fake,
                           fake, 1 << 40, None)
    assert r == 8
    r = lib.negf_lead_selfenergy(ctypes.byref(big), 1, fake, fake, ctypes.byref(o_mixed), fake,
                                 fake, None, fake, fake, 1 << 40, None)
    assert r == 8
    # the benchmark's and the adjoint workload's block sizes are inside the range
    for b in (40, 400, 800, 3430):
        assert lib.negf_workspace_size(ctypes.byref(_dev(b=b)), 1, ctypes.byref(o_mixed),
                                       B.WS_RGF) > 0


def test_block_inverse_size_limits_are_checked_on_the_host(lib):
    """The Gauss-Jordan panel keeps an n-row column panel in shared memory: n <= 5147 for FP64
    elements and n <= 9266 for the mixed form's FP32 elimination; larger blocks are refused on
    the host (NEGF_ERR_UNSUPPORTED / workspace size 0) instead of failing at launch."""
    P = ctypes.c_void_p
    fake = P(16)
    mixed, fp64 = B.PREC_MIXED, B.PREC_FP64
    assert lib.negf_zinv_workspace_size(fp64, 1, 5147) > 0
    assert lib.negf_zinv_workspace_size(fp64, 1, 5148) == 0
    assert lib.negf_zinv_workspace_size(mixed, 1, 9266) > 0
    assert lib.negf_zinv_workspace_size(mixed, 1, 9267) == 0
    assert lib.negf_zinv_batched(fp64, 1, 5148, fake, fake, 0, fake, fake, 1 << 40, None) == 8
    assert lib.negf_zinv_batched_noalloc(1, 5148, fake, fake, fake, None) == 8
    o_fp64 = negf.options(precision=fp64)
    assert lib.negf_workspace_size(ctypes.byref(_dev(b=5148)), 1, ctypes.byref(o_fp64),
                                   B.WS_RGF) == 0
    assert lib.negf_workspace_size(ctypes.byref(_dev(b=5147)), 1, ctypes.byref(o_fp64),
                                   B.WS_RGF) > 0


def test_precision_tiers_and_their_exact_ranges(lib):
    """Each mixed tier keeps its fixed-point slices exact up to its own contraction length
    (40 bits: K <= 524288, 48 bits: 393216, 56 bits: 98304) and refuses longer ones on the host;
    the decimation's automatic precision is the 56-bit tier where it is exact, else the 48-bit
    one."""
    for prec, kmax in ((B.PREC_MIXED_40, 524288), (B.PREC_MIXED, 393216),
                       (B.PREC_MIXED_56, 98304)):
        assert lib.negf_zgemm_workspace_size(prec, 1, 8, 8, kmax) > 0
        assert lib.negf_zgemm_workspace_size(prec, 1, 8, 8, kmax + 1) == 0
    # 56-bit values need more slices: a larger workspace for the same product
    w48 = lib.negf_zgemm_workspace_size(B.PREC_MIXED, 4, 400, 400, 400)
    w56 = lib.negf_zgemm_workspace_size(B.PREC_MIXED_56, 4, 400, 400, 400)
    w40 = lib.negf_zgemm_workspace_size(B.PREC_MIXED_40, 4, 400, 400, 400)
    assert w40 < w48 < w56
    assert lib.negf_zgemm_workspace_size(4, 1, 8, 8, 8) == 0
    d = _dev(b=400)
    auto = negf.options(precision=B.PREC_MIXED)
    l48 = negf.options(precision=B.PREC_MIXED, lead_precision=B.PREC_MIXED)
    l56 = negf.options(precision=B.PREC_MIXED, lead_precision=B.PREC_MIXED_56)
    size = lambda o, dv=d: lib.negf_workspace_size(ctypes.byref(dv), 8, ctypes.byref(o), B.WS_LEAD)
    assert size(auto) == size(l56) > size(l48) > 0
    # every block the mixed inverse takes (n <= 9266) is inside the 56-bit range
    big = _dev(b=9266)
    assert size(auto, big) == size(l56, big) > size(l48, big) > 0
    for bad in (dict(lead_precision=5), dict(lead_precision=-2), dict(refine_max=17),
                dict(refine_max=-1)):
        o = negf.options(precision=B.PREC_MIXED, **bad)
        assert lib.negf_workspace_size(ctypes.byref(d), 8, ctypes.byref(o), B.WS_LEAD) == 0


def test_interface_support_is_validated(lib):
    """The interface-coupling support (last r rows, first c columns of every hopping block) must
    lie in [0, b]."""
    o = negf.options()
    for r, c, ok in ((0, 0, True), (2, 3, True), (8, 8, True), (9, 0, False), (0, -1, False)):
        d = B._Dev(1, 4, 8, r, 1, 1, c, 0)
        size = lib.negf_workspace_size(ctypes.byref(d), 4, ctypes.byref(o), B.WS_RGF)
        assert (size > 0) == ok, (r, c)


def test_sigma_structure_is_validated(lib):
    """Atom-block scattering self-energies need a known structure and a block width that
    divides b; the check runs on the host before any device work."""
    d = _dev(b=40)
    bad_kind = negf.options(sigma_structure=2)
    assert lib.negf_workspace_size(ctypes.byref(d), 4, ctypes.byref(bad_kind), B.WS_RGF) == 0
    fake = ctypes.c_void_p(1 << 40)
    for A, ok in ((10, True), (8, True), (1, True), (7, False), (0, False), (65, False)):
        o = negf.options(sigma_structure=negf.SIGMA_ATOM_BLOCK, atom_orbitals=A)
        assert negf.sigma_width(o) == A
        if ok:
            continue
        r = lib.negf_rgf_solve(ctypes.byref(d), 1, fake, fake, None, fake, fake, None, None,
                               None, 0, ctypes.byref(o), None, None, None, None, None, None,
                               fake, fake, 1 << 40, None)
        assert r == 1, A
        r = lib.negf_rgf_adjoint(ctypes.byref(d), 1, fake, fake, None, fake, fake, None, None,
                                 None, 0, ctypes.byref(o), None, None, None, fake, fake, fake,
                                 1 << 40, None)
        assert r == 1, A


def test_checkpoint_sizes(lib):
    """negf_rgf_solve's checkpoints hold 5 N b^2 complex numbers per point, and the adjoint that
    reads them needs a smaller workspace than the one that recomputes the sweeps."""
    d = _dev(N=6, b=40)
    o = negf.options()
    assert lib.negf_checkpoint_bytes(ctypes.byref(d), 3) == 5 * 6 * 3 * 40 * 40 * 16
    assert lib.negf_checkpoint_bytes(ctypes.byref(d), 0) == 0
    assert lib.negf_checkpoint_bytes(ctypes.byref(_dev(N=0)), 3) == 0
    full = lib.negf_workspace_size(ctypes.byref(d), 3, ctypes.byref(o), B.WS_ADJOINT)
    ck = lib.negf_workspace_size(ctypes.byref(d), 3, ctypes.byref(o), B.WS_ADJOINT_CKPT)
    assert 0 < ck < full
