"""Host-side checks of the C ABI: the library builds for sm_103a, loads
without a GPU, and exports every function include/*.h declares."""
import ctypes
import glob
import os
import re

import pytest

from paper_2404_10087_gb300 import _build, ft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(ft_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_binding_surface():
    assert declared_functions() == set(ft.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls_without_gpu():
    lib = ft.load()
    cfg = ft.ft_config()
    lib.ft_config_default(ctypes.byref(cfg))
    assert cfg.precision == ft.FT_FP32 and cfg.scatter == ft.FT_HOGWILD and cfg.det_batch == 4096
    assert ft.ft_status_str(0) == "ok"
    assert ft.ft_status_str(-2) == "coordinate out of range"
    lib.ft_destroy(None)
    assert lib.ft_launch_count(None) == 0


def test_shape_rejection_before_any_device_call():
    """Unsupported shapes are refused on the host (no device query needed)."""
    cfg = ft.make_config()
    for I, J, R in [((10,) * 11, (4,) * 11, 4),     # N > 10
                    ((10,) * 6, (17,) * 6, 4),       # N > 5 at K = 32
                    ((10, 10), (4, 33), 4),          # J > 32
                    ((10, 10), (4, 4), 33),          # R > 32
                    ((10,) * 6, (32,) * 6, 8),       # N * K > 160
                    ((10, 10), (0, 4), 4)]:          # J < 1
        with pytest.raises(ft.FtError) as e:
            ft.ft_workspace_size(I, J, R, 100, cfg)
        assert e.value.status == -3


def test_engine_configuration_rejected_on_host():
    """The tcgen05 engine is BF16 Hogwild only; unknown engines are refused."""
    I, J, R = (10, 10, 10), (16, 16, 16), 16
    for kw in (dict(precision="fp32", engine="tcgen05"), dict(precision="tf32", engine="tcgen05"),
               dict(precision="bf16", scatter="deterministic", engine="tcgen05"),
               dict(precision="bf16", engine=7)):
        cfg = ft.make_config(**kw)
        with pytest.raises(ft.FtError) as e:
            ft.ft_workspace_size(I, J, R, 100, cfg)
        assert e.value.status == -1, kw


def test_core_scheme_configuration():
    """The core phase's storage scheme is a config field (default:
    calculation); unknown schemes are refused on the host."""
    lib = ft.load()
    cfg = ft.ft_config()
    lib.ft_config_default(ctypes.byref(cfg))
    assert cfg.core_scheme == ft.FT_CORE_CALC and cfg.l2_persist == 0 and list(cfg.reserved) == [0]
    with pytest.raises(ft.FtError) as e:
        ft.ft_workspace_size((10, 10, 10), (16, 16, 16), 16, 100, ft.make_config(core_scheme=5))
    assert e.value.status == -1


def test_l2_persist_configuration():
    """l2_persist is 0 or 1; other values are refused on the host."""
    with pytest.raises(ft.FtError) as e:
        ft.ft_workspace_size((10, 10, 10), (16, 16, 16), 16, 100, ft.make_config(l2_persist=2))
    assert e.value.status == -1


def test_context_calls_refuse_a_null_context():
    """The per-context calls return FT_ERR_ARG for a null context before any
    device work."""
    lib = ft.load()
    assert lib.ft_epoch_factors(None, 0.1, 0.1, None, None) == -1
    assert lib.ft_epoch_core(None, 0.1, 0.1, None) == -1
    assert lib.ft_epoch_core_sgd(None, 0.1, 0.1, 100, None) == -1
    assert lib.ft_permute(None, None, None, None, None) == -1
    assert lib.ft_rebind(None, None, None, None) == -1
    assert lib.ft_core_grad(None, None, None) == -1
    assert lib.ft_check(None, None) == -1
