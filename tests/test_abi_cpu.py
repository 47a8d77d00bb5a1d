"""The C ABI library loads and exports every symbol include/pvg.h declares;
the ctypes structures match the C layouts; the product package never
reaches the oracle.  No compute call, no GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2311_18561_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pvg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pvg_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return C.CDLL(build.LIB)


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(abi._SIGS)


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pvg.h"\nint main(void){\n'
                   'printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(pvg_scene_t), sizeof(pvg_camera_t),'
                   ' sizeof(pvg_image_t), sizeof(pvg_image_grad_t), sizeof(pvg_scene_grad_t),'
                   ' sizeof(pvg_config_t), offsetof(pvg_camera_t, t), offsetof(pvg_config_t, dilation));\n'
                   'return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(abi.Scene), C.sizeof(abi.Camera), C.sizeof(abi.Image), C.sizeof(abi.ImageGrad),
            C.sizeof(abi.SceneGrad), C.sizeof(abi.Config), abi.Camera.t.offset, abi.Config.dilation.offset]
    assert got == want


def test_status_strings(lib):
    lib.pvg_status_str.restype = C.c_char_p
    assert lib.pvg_status_str(0) == b"PVG_OK"
    assert lib.pvg_status_str(6) == b"PVG_ERR_OVERFLOW"


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2311_18561_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, flags=re.M), f
                assert "pvg_oracle" not in text, f


def test_serving_struct_layouts_match_c(tmp_path):
    src = tmp_path / "serve_sizes.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pvg.h"\nint main(void){\n'
                   'printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(pvg_serve_config_t), sizeof(pvg_req_stats_t),'
                   ' offsetof(pvg_serve_config_t, gate_timeout_us), offsetof(pvg_serve_config_t, pair_capacity),'
                   ' offsetof(pvg_req_stats_t, gpu_ms), offsetof(pvg_req_stats_t, attempts));\n'
                   'return 0;}\n')
    exe = tmp_path / "serve_sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(abi.ServeConfig), C.sizeof(abi.ReqStats), abi.ServeConfig.gate_timeout_us.offset,
            abi.ServeConfig.pair_capacity.offset, abi.ReqStats.gpu_ms.offset, abi.ReqStats.attempts.offset]
    assert got == want
