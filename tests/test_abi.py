"""CPU checks of the C ABI: the library builds, loads and exports every
function declared in include/lodge.h, and the ctypes structures used by the
binding have the sizes and field offsets of the C declarations.  No compute
calls (no GPU here)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lodge.h")


@pytest.fixture(scope="module")
def built():
    from paper_2505_23158_gb300 import build
    return build.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lodge_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function(built):
    lib = C.CDLL(built)
    names = declared_functions()
    assert "lodge_render" in names and "lodge_render_backward" in names
    for n in names:
        assert hasattr(lib, n), n
    from paper_2505_23158_gb300 import _capi
    assert sorted(_capi.exported_symbols()) == names


def test_struct_layouts_match_header(tmp_path):
    from paper_2505_23158_gb300 import _capi as A
    prog = tmp_path / "probe.c"
    structs = {"lodge_level_desc": A.lodge_level_desc, "lodge_scene_desc": A.lodge_scene_desc,
               "lodge_camera": A.lodge_camera, "lodge_selection": A.lodge_selection,
               "lodge_frame_stats": A.lodge_frame_stats, "lodge_profile": A.lodge_profile,
               "lodge_request": A.lodge_request, "lodge_request_result": A.lodge_request_result,
               "lodge_serve_opts": A.lodge_serve_opts, "lodge_residency": A.lodge_residency}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-o", str(exe), str(prog)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.split() for l in out if l.strip())
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def test_header_entry_points_document_errors():
    """Each declaration in the header sits under a comment (its contract)."""
    src = open(HEADER).read()
    for n in declared_functions():
        m = re.search(r"(lodge_status|const char\*)\s+" + n + r"\(", src)
        assert m, n
        before = src[:m.start()].rstrip()
        assert before.endswith("*/"), n


def test_no_gpu_fails_loudly(built):
    """Without a usable GPU the library refuses to create a context: the
    product path has no CPU fallback (the oracle is test infrastructure)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2505_23158_gb300.api import Lodge, LodgeError
    with pytest.raises(LodgeError):
        Lodge(0)
