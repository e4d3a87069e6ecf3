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


STRUCTS = {  # C typedef in include/ess.h -> ctypes mirror in the binding
    "ess_build_params": "BuildParams", "ess_camera": "Camera",
    "ess_render_params": "RenderParams", "ess_render_item": "RenderItem",
    "ess_server_config": "ServerConfig", "ess_request": "Request",
    "ess_request_status": "RequestStatus", "ess_tune_result": "TuneResult",
    "ess_structure_info": "StructureInfo",
}


def test_binding_structs_match_header_layout(libpath, tmp_path):
    """Size and every field offset of each public struct, as the C compiler
    lays it out from include/ess.h, equal the binding's ctypes mirror."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    from paper_1912_09596_gb300 import ess
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "ess.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in getattr(ess, pyname)._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, field, cname, field))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, pyname in STRUCTS.items():
        cls = getattr(ess, pyname)
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert got[(cname, field)] == getattr(cls, field).offset, (cname, field)
