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


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import importlib
    monkeypatch.setattr(hp, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(hp, "_lib", None)
    try:
        hp.load_library()
    except RuntimeError as e:
        assert "no CPU fallback" in str(e)
    else:
        raise AssertionError("load_library must raise when the library is missing")
    finally:
        importlib.reload(hp)
