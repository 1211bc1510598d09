"""The C-ABI library without a GPU: it loads, exports every function that
include/lbm.h declares, and rejects bad problems before any CUDA call."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_2311_10827_gb300 import build, capi
    build.build()
    return capi


def header_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree(capi):
    assert header_functions() == sorted(capi.EXPORTS)


def test_every_declared_symbol_is_exported(capi):
    L = capi.lib()
    for name in header_functions():
        assert hasattr(L, name), name


def test_defaults(capi):
    p = capi.lbm_params_default()
    assert (p.W, p.M, p.alpha, p.sigma, p.phi_l, p.phi_v) == (4.0, 0.1, 1.0, 1e-3, 1.0, 0.0)
    assert p.precision == capi.LBM_FP32 and p.diag_every == 0 and p.tau_f == 0.0


@pytest.mark.parametrize("field,value", [("W", 0.0), ("W", float("nan")), ("M", -0.1),
                                         ("alpha", 0.0), ("tau_f", 0.5), ("tau_f", 0.2),
                                         ("rho_v", 0.0), ("nu_l", -1.0), ("sigma", -1e-3),
                                         ("precision", 7), ("diag_every", -1)])
def test_invalid_parameters_rejected(capi, field, value):
    p = capi.lbm_params_default()
    setattr(p, field, value)
    rc, h = capi.lbm_create((16, 16), capi.LBM_D2Q9, p)
    assert rc == capi.LBM_ERR_INVALID_ARG and not h.value


def test_equal_phases_and_bad_grids_rejected(capi):
    p = capi.lbm_params_default()
    p.phi_v = p.phi_l
    assert capi.lbm_create((16, 16), 0, p)[0] == capi.LBM_ERR_INVALID_ARG
    p = capi.lbm_params_default()
    for grid in ((0, 16), (16, -1), (16, 16, 2)):
        assert capi.lbm_create(grid, capi.LBM_D2Q9, p)[0] == capi.LBM_ERR_INVALID_ARG
    assert capi.lbm_create((16, 16), 5, p)[0] == capi.LBM_ERR_INVALID_ARG


def test_offset_storage_needs_d3q19(capi):
    """16-bit offset storage exists for the D3Q19 path only."""
    for prec in (capi.LBM_FP32_F16OFF, capi.LBM_FP32_BF16OFF):
        p = capi.lbm_params_default()
        p.precision = prec
        assert capi.lbm_create((16, 16), capi.LBM_D2Q9, p)[0] == capi.LBM_ERR_INVALID_ARG


def test_state_bytes_and_caller_buffers(capi):
    """lbm_state_bytes reports the double-buffered state's sizes without a GPU;
    lbm_create_with_buffers refuses missing or misaligned buffers first."""
    p = capi.lbm_params_default()                      # FP32: rest population pair
    rc, (fb, gb, sb) = capi.lbm_state_bytes((30, 20), capi.LBM_D2Q9, p)
    assert rc == 0 and (fb, gb, sb) == (10 * 600 * 4, 9 * 600 * 4, 600 * 4)
    p.precision = capi.LBM_FP64
    rc, sizes = capi.lbm_state_bytes((30, 20, 7), capi.LBM_D3Q19, p)
    assert rc == 0 and sizes == (19 * 4200 * 8, 19 * 4200 * 8, 4200 * 8)
    p.precision = capi.LBM_FP32_F16OFF                 # 16-bit offsets, 7 FP32 fields, scales
    rc, (fb, gb, sb) = capi.lbm_state_bytes((30, 20, 7), capi.LBM_D3Q19, p)
    pad = lambda b: (b + 255) // 256 * 256
    assert rc == 0 and fb == pad(19 * 4200 * 2) + pad(7 * 4200 * 4) + 256
    assert gb == 19 * 4200 * 2 and sb == 4200 * 4
    p.W = 0.0
    assert capi.lbm_state_bytes((30, 20), capi.LBM_D2Q9, p)[0] == capi.LBM_ERR_INVALID_ARG
    p = capi.lbm_params_default()
    rc, h = capi.lbm_create_with_buffers((16, 16), capi.LBM_D2Q9, p, [0] * 5)
    assert rc == capi.LBM_ERR_INVALID_ARG and not h.value
    rc, h = capi.lbm_create_with_buffers((16, 16), capi.LBM_D2Q9, p, [4096 + 8] * 5)
    assert rc == capi.LBM_ERR_INVALID_ARG and not h.value


def test_null_safety_and_strerror(capi):
    L = capi.lib()
    L.lbm_destroy(None)
    assert L.lbm_time(None) == -1
    assert L.lbm_step(None, 1) == capi.LBM_ERR_INVALID_ARG
    assert L.lbm_sync(None) == capi.LBM_ERR_INVALID_ARG
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert capi.strerror(code) and capi.strerror(code) != "unknown error"
    assert capi.strerror(-99) == "unknown error"


def test_no_cpu_fallback(capi, monkeypatch, tmp_path):
    """The binding refuses to run without the CUDA library."""
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(RuntimeError):
        capi.lib(str(tmp_path / "missing.so"))
