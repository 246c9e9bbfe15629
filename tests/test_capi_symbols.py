"""The C interface library loads on a machine without a GPU and exports every
entry point declared in include/*.h (no compute calls are made here)."""
import glob
import os
import re

import paper_2509_19777_gb300 as hp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(hplmm_[a-z_0-9]+)\s*\(", txt))
    return names


def test_library_exports_declared_symbols():
    lib = hp.load_library()
    names = declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(hp.EXPORTED) == names


def test_default_options_and_struct_sizes():
    o = hp.hplmm_default_options()
    assert (o.n_mortar, o.beta, o.contact_halfwidth, o.n_st, o.restart, o.max_iters) == (4, 4.0, 2, 1, 30, 300)
    assert o.local_prec == hp.HPLMM_FP64 and o.apply_prec == hp.HPLMM_FP64


def test_missing_library_fails_loudly(tmp_path):
    import importlib
    import pytest
    # the patches are undone before the module is reloaded, so later tests see the library with its
    # argument types bound to the reloaded module's classes
    try:
        with pytest.MonkeyPatch.context() as mp:
            mp.setattr(hp, "LIB_PATH", str(tmp_path / "absent.so"))
            mp.setattr(hp, "_lib", None)
            with pytest.raises(RuntimeError, match="no CPU fallback"):
                hp.load_library()
    finally:
        importlib.reload(hp)


def test_invalid_options_rejected_before_any_device_call():
    # hplmm_create validates the options first and returns HPLMM_ERR_INVALID without touching a device, so
    # this runs on a machine without a GPU
    import ctypes
    lib = hp.load_library()
    bad = [dict(smoother_bulk_warps=3), dict(smoother_bulk_warps=4, smoother_ctas=2),
           dict(smoother_bulk_warps=1, smoother_ctas=2), dict(smoother_ctas=3), dict(restart=0),
           dict(matrix_free_updates=2)]
    for over in bad:
        o = hp.hplmm_default_options()
        for k, v in over.items():
            setattr(o, k, v)
        ctx = ctypes.c_void_p()
        assert lib.hplmm_create(ctypes.byref(ctx), ctypes.byref(o), None) == hp.HPLMM_ERR_INVALID, over
        assert not ctx.value
    assert hp.hplmm_default_options().smoother_bulk_warps == 0
