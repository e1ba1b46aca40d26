"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/*.h; host-side argument checks answer without one."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header="cmaes.h"):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return set(re.findall(r"\b(cmaes_[a-z_]+)\s*\(", text))


def test_every_header_has_a_library():
    headers = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    assert headers == ["cmaes.h", "cmaes_ozaki.h", "cmaes_probe.h"]


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2409_11765_gb300 import _build
    return _build.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("cmaes_create", "cmaes_create_batch", "cmaes_ask", "cmaes_tell",
                     "cmaes_step_batch", "cmaes_restart", "cmaes_best", "cmaes_get_state",
                     "cmaes_set_state", "cmaes_query", "cmaes_strerror", "cmaes_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    from paper_2409_11765_gb300 import _build
    for header, path in (("cmaes.h", libpath), ("cmaes_ozaki.h", libpath), ("cmaes_probe.h", _build.PROBE_LIB)):
        L = ctypes.CDLL(path)
        names = _declared(header)
        assert names
        missing = [n for n in sorted(names) if not hasattr(L, n)]
        assert not missing, (header, missing)


def test_host_only_calls_without_gpu(libpath):
    import paper_2409_11765_gb300 as eng
    o = eng.cmaes_default_options()
    assert o.precision == 0 and o.ipop_double == 1 and o.stop_mask == 255
    assert o.f_target == float("-inf") and o.cond_max == 1e14
    assert eng.cmaes_strerror(0) == "ok"
    assert eng.cmaes_strerror(4) == "call out of order"
    # argument checks fail before any device work
    with pytest.raises(eng.CmaesError) as e:
        eng.cmaes_create(0, 10, [], 1.0, 1)
    assert e.value.status == 1
    with pytest.raises(eng.CmaesError) as e:
        eng.cmaes_create(3, 1, [0.0, 0.0, 0.0], 1.0, 1)
    assert e.value.status == 1
    with pytest.raises(eng.CmaesError) as e:
        eng.cmaes_create(3, 6, [0.0, 0.0, 0.0], -1.0, 1)
    assert e.value.status == 1
    # a NULL handle is rejected, destroy(NULL) is a no-op
    assert eng.lib().cmaes_sync(None) == 1
    eng.lib().cmaes_destroy(None)
    assert eng.cmaes_count(None) == 0
