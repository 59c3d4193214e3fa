"""The C-ABI library builds, loads without a GPU and exports every function include/lbm.h
declares; the binding's structure matches the header (no GPU, no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b(lbm_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2101_11856_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_api():
    names = declared_functions()
    for core in ("lbm_create", "lbm_destroy", "lbm_set_state", "lbm_set_solids", "lbm_step", "lbm_macroscopic",
                 "lbm_reductions", "lbm_save", "lbm_load", "lbm_last_error"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_config_layout_matches_header(lib):
    from paper_2101_11856_gb300 import lbm
    cfg = lbm.lbm_config()
    lib.lbm_config_default(ctypes.byref(cfg))
    assert cfg.storage == 0 and list(cfg.face_type) == [0] * 6
    assert cfg.rho0 == 1.0 and cfg.seed == 2101 and cfg.omega_bulk == 1.0 and list(cfg.omega_hi) == [1.0] * 4
    assert cfg.cuda_stream is None and cfg.collision == lbm.COLLISION["acm"] == 0


def test_velocity_table_is_d3q27(lib):
    from paper_2101_11856_gb300 import lbm
    vel = {lbm.lbm_velocity(i) for i in range(27)}
    assert vel == {(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)}
    with pytest.raises(lbm.LBMError):
        lbm.lbm_velocity(27)


def test_create_rejects_bad_arguments_without_touching_the_gpu(lib):
    """Argument validation happens before any CUDA call."""
    from paper_2101_11856_gb300 import lbm
    cfg = lbm.lbm_config_default()
    for args in ((0, 4, 4, 0.1), (4, 4, 4, 0.0), (4, 4, 4, -1.0), (4, 4, 4, float("nan"))):
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_create(*args, cfg=cfg)
        assert e.value.code == lbm.LBM_EINVAL
    bad = lbm.lbm_config_default()
    bad.face_type[0] = lbm.FACE["noslip"]            # -x no-slip with +x periodic
    with pytest.raises(lbm.LBMError):
        lbm.lbm_create(4, 4, 4, 0.1, cfg=bad)
    bad = lbm.lbm_config_default()
    bad.face_type[2], bad.face_type[3] = lbm.FACE["inlet"], lbm.FACE["noslip"]   # inlet on -y
    with pytest.raises(lbm.LBMError):
        lbm.lbm_create(4, 4, 4, 0.1, cfg=bad)
    for coll in (-1, 3):
        bad = lbm.lbm_config_default()
        bad.collision = coll
        with pytest.raises(lbm.LBMError) as e:
            lbm.lbm_create(4, 4, 4, 0.1, cfg=bad)
        assert e.value.code == lbm.LBM_EINVAL


def test_async_binding_refuses_converted_temporaries():
    """The asynchronous transfers read or write the caller's buffer after the call returns, so
    the binding passes float32 C-contiguous buffers as they are and refuses anything that would
    need a temporary copy (which could be freed before the transfer runs)."""
    import numpy as np
    import torch
    from paper_2101_11856_gb300.lbm import _ptr_nocopy
    a = np.zeros((4, 5), np.float32)
    assert _ptr_nocopy(a).value == a.ctypes.data
    t = torch.zeros(6)
    assert _ptr_nocopy(t).value == t.data_ptr()
    assert _ptr_nocopy(None) is None
    for bad in (np.zeros(4), np.zeros((4, 6), np.float32)[:, ::2], torch.zeros(4, dtype=torch.float64),
                torch.zeros(4, 6)[:, ::2], [1.0, 2.0]):
        with pytest.raises(ValueError):
            _ptr_nocopy(bad)


def test_output_binding_refuses_temporaries_and_short_buffers():
    """Outputs are filled in place: a buffer that would need a converted temporary (the caller's
    array would keep stale data) or that is shorter than what the library writes is refused."""
    import numpy as np
    import torch
    from paper_2101_11856_gb300.lbm import _ptr_out
    a = np.zeros((3, 4), np.float32)
    assert _ptr_out(a, 12, "x").value == a.ctypes.data
    t = torch.zeros(5)
    assert _ptr_out(t, 5, "x").value == t.data_ptr()
    for bad in (np.zeros(12), np.zeros((3, 8), np.float32)[:, ::2], torch.zeros(12, dtype=torch.float64),
                torch.zeros(3, 8)[:, ::2], [0.0] * 12, np.zeros(11, np.float32), torch.zeros(11)):
        with pytest.raises(ValueError):
            _ptr_out(bad, 12, "x")
    ro = np.zeros(12, np.float32)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        _ptr_out(ro, 12, "x")


def test_static_force_sum_binding_validates_before_the_call():
    """The allocation-free force sum's binding checks types, shapes and devices itself (the C
    function takes bare pointers and cannot)."""
    import torch
    from paper_2101_11856_gb300.lbm import lbm_sum_forces_static
    g, out = torch.zeros(10, 3), torch.zeros(3, dtype=torch.float64)
    for args in ((torch.zeros(10, 3, dtype=torch.float64), out), (torch.zeros(30), out), (torch.zeros(10, 4), out),
                 (g, torch.zeros(3)), (g, torch.zeros(2, dtype=torch.float64)), (g.numpy(), out),
                 (torch.zeros(3, 10).t(), out)):
        with pytest.raises(ValueError):
            lbm_sum_forces_static(*args)
    with pytest.raises(ValueError):                 # host tensors of the right shapes
        lbm_sum_forces_static(g, out)


def test_context_setters_reject_a_null_context_without_the_gpu(lib):
    """The per-context switches validate their context before anything else."""
    assert lib.lbm_set_pair_kernel(None, 1) == -1     # LBM_EINVAL
    assert lib.lbm_set_pair_kernel(None, 0) == -1
    assert lib.lbm_set_inflow(None, None) == -1
