"""CPU checks of the C ABI: the shared library builds for sm_103a, loads, and
exports every function that include/*.h declares; without a GPU the context
call fails with a status instead of crashing."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mglma_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    import paper_2412_06347_gb300 as m
    names = declared_functions()
    assert len(names) >= 8
    missing = [n for n in names if not hasattr(m.lib, n)]
    assert not missing, missing
    assert "sm_103a" in m.mglma_version()


def test_python_binding_uses_the_same_names():
    import paper_2412_06347_gb300 as m
    for n in declared_functions():
        assert hasattr(m, n), n


def test_create_fails_cleanly_without_gpu():
    import torch
    import paper_2412_06347_gb300 as m
    if torch.cuda.is_available():
        return
    try:
        m.mglma_create(0)
    except m.MglmaError as e:
        assert e.status in (1, 3)
    else:
        raise AssertionError("mglma_create succeeded without a GPU")
