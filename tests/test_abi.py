"""The C ABI library loads and exports every function include/*.h declares
(no GPU needed: nothing here calls into CUDA)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ess_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1912_09596_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ess_create", "ess_destroy", "ess_volume_upload", "ess_tf_set",
                     "ess_tf_update", "ess_build", "ess_rebuild", "ess_render",
                     "ess_structure_read", "ess_release", "ess_sync"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_without_gpu(libpath):
    from paper_1912_09596_gb300 import ess
    assert os.path.samefile(ess.LIB_PATH, libpath)
    for n in declared_functions():
        assert hasattr(ess, n) or n in ("ess_kind_name",), n


def test_null_context_is_rejected(libpath):
    from paper_1912_09596_gb300 import ess
    assert ess.lib.ess_sync(None) == ess.ERR_ARG
    assert ess.lib.ess_destroy(None) == ess.ERR_ARG
    assert ess.ess_launch_count(None) == 0


def test_binding_constants_match_header(libpath):
    """Every `ESS_NAME = value` enumerator in include/*.h has the same value
    as the binding's NAME constant (structure kinds, dtypes, arrays, status
    codes, request kinds)."""
    from paper_1912_09596_gb300 import ess
    found = 0
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for name, value in re.findall(r"\bESS_(\w+)\s*=\s*(-?\d+)", src):
            assert hasattr(ess, name), "binding lacks %s" % name
            assert getattr(ess, name) == int(value), name
            found += 1
    assert found >= 20
