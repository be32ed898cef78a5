"""The C ABI library loads and exports every entry point include/nr.h declares,
and its argument checks answer without a GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nr():
    from paper_2306_16541_gb300 import build
    build.build()
    from paper_2306_16541_gb300 import nr as mod
    return mod


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:nr_status|const char \*|void)\s*\**\s*(nr_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["nr_create_subject", "nr_set_pose", "nr_render", "nr_train_step", "nr_destroy"]:
        assert must in names


def test_every_declared_symbol_is_exported(nr):
    lib = C.CDLL(nr.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_argument_errors_without_gpu(nr):
    h = C.c_void_p()
    assert nr.lib.nr_create_subject(None, None, C.byref(h)) == nr.NR_EINVAL
    assert b"NULL" in nr.lib.nr_last_error()
    d = nr.nr_subject_desc()
    d.abi_version = 999
    assert nr.lib.nr_create_subject(C.byref(d), None, C.byref(h)) == nr.NR_EINVAL
    assert b"abi_version" in nr.lib.nr_last_error()
    d.abi_version, d.n_bones = nr.NR_ABI_VERSION, 23
    assert nr.lib.nr_create_subject(C.byref(d), None, C.byref(h)) == nr.NR_EINVAL
    assert nr.lib.nr_destroy(None) == nr.NR_OK
    assert nr.lib.nr_render(None, None, None, None, None) == nr.NR_EINVAL
    assert nr.lib.nr_set_pose(None, None, None, 0, None) == nr.NR_EINVAL


def test_struct_sizes_match_header(nr):
    # nr_camera: 2 u32 + 4 f + 9 f + 3 f + 2 f + u32 + 3 f = 24 * 4 bytes
    assert C.sizeof(nr.nr_camera) == 96
    assert C.sizeof(nr.nr_render_opts) == 24


def _header_constants():
    """#define NR_X <n> and the enumerators of nr_status / nr_dtype, from include/nr.h."""
    text = open(os.path.join(ROOT, "include", "nr.h")).read()
    consts = {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define (NR_\w+) (\d+)u?\b", text, flags=re.M)}
    for body in re.findall(r"typedef enum \{(.*?)\}", text, flags=re.S):
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        for name, val in re.findall(r"(NR_\w+)\s*=\s*(\d+)", body):
            consts[name] = int(val)
    return consts


def test_binding_constants_match_header(nr):
    """Every constant the header defines has the same value in the Python binding."""
    consts = _header_constants()
    assert {"NR_OK", "NR_EUNSUPPORTED", "NR_BF16", "NR_RENDER_F32_TC", "NR_TRAIN_ALL", "NR_PARAM_CNN"} <= set(consts)
    missing = [k for k in consts if not hasattr(nr, k)]
    assert not missing, missing
    wrong = {k: (v, getattr(nr, k)) for k, v in consts.items() if getattr(nr, k) != v}
    assert not wrong, wrong


STRUCTS = ["nr_subject_desc", "nr_camera", "nr_render_opts", "nr_train_batch", "nr_request", "nr_server_stats",
           "nr_server_policy"]


def test_struct_layouts_match_header(nr, tmp_path):
    """sizeof and every field offset of the header's structs, as a C compiler lays them out,
    equal the ctypes structures of the binding."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nr.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("{s} sizeof %zu\\n", sizeof({s}));')
        for name, _ in getattr(nr, s)._fields_:
            lines.append(f'  printf("{s} {name} %zu\\n", offsetof({s}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            s, f, v = ln.split()
            got[(s, f)] = int(v)
    for s in STRUCTS:
        cls = getattr(nr, s)
        assert got[(s, "sizeof")] == C.sizeof(cls), (s, got[(s, "sizeof")], C.sizeof(cls))
        for name, _ in cls._fields_:
            assert got[(s, name)] == getattr(cls, name).offset, (s, name)


@pytest.mark.parametrize("field,value,message", [
    ("level_res", "huge", b"level_res must be 1..65536"),
    ("wvol_res", 300, b"wvol_res must be 2..256"),
    ("log2_T", 9, b"log2_T must be 10..24"),
    ("mlp_hidden_layers", 5, b"mlp_hidden_layers must be 1..4"),
    ("occ_grid", 100, b"occ_grid"),
])
def test_descriptor_checks_without_gpu(nr, field, value, message):
    """A descriptor outside the documented ranges is refused (NR_EINVAL, with the message)
    before any device call."""
    from paper_2306_16541_gb300 import synth
    s = dict(synth.subject(5))
    if value == "huge":
        lv = np.array(s["level_res"], np.uint32)
        lv[-1] = 70000
        s["level_res"] = lv
    else:
        s[field] = value
    with pytest.raises(nr.NRError) as e:
        nr.nr_create_subject(s, stream=0)   # the legacy default stream: no torch CUDA call
    assert e.value.code == nr.NR_EINVAL
    assert message in nr.lib.nr_last_error()


def test_option_and_camera_marshalling(nr):
    """make_opts and make_camera fill the C structs field by field (no device needed)."""
    from paper_2306_16541_gb300 import synth
    o = nr.make_opts("bf16", "f16", True, 1e-4, profile=True, mma2=True, all_bones=True)
    assert (o.mlp_dtype, o.feat_dtype, o.use_occupancy) == (nr.NR_BF16, nr.NR_F16, 1)
    assert abs(o.t_min - 1e-4) < 1e-9
    assert o.flags == nr.NR_RENDER_PROFILE | nr.NR_RENDER_MMA2 | nr.NR_RENDER_ALL_BONES
    o = nr.make_opts("f32", f32_tc=True, tcgen05=True)
    assert o.mlp_dtype == nr.NR_F32 and o.flags == nr.NR_RENDER_F32_TC | nr.NR_RENDER_TCGEN05
    cam = synth.camera(64, 48, 80.0, (0.0, 0.0, 2.5), 32, 1.5, 3.5)
    c = nr.make_camera(cam)
    assert (c.width, c.height, c.n_samples) == (64, 48, 32)
    assert (c.fx, c.fy) == (80.0, 80.0) and (c.t_near, c.t_far) == (1.5, 3.5)
    assert np.allclose(np.array(c.R[:]), np.asarray(cam.R, np.float32).ravel())
    assert np.allclose(np.array(c.t[:]), np.asarray(cam.t, np.float32).ravel())


def test_server_policy_refused_without_a_server(nr):
    """nr_server_set_policy validates its handle before touching a server (no device needed)."""
    pol = nr.nr_server_policy(nr.NR_SERVE_EDF, 40.0, 20.0, 20.0, 0)
    assert nr.lib.nr_server_set_policy(None, C.byref(pol)) == nr.NR_EINVAL
    assert b"nr_server_set_policy" in nr.lib.nr_last_error()


def test_gather_rate_arguments_checked_without_gpu(nr):
    """nr_l2_gather_rate refuses a NULL output, load sizes other than 4 or 16 bytes and tables
    that are not a power of two in [1 MiB, 1 GiB] before it touches a device."""
    v = C.c_double()
    assert nr.lib.nr_l2_gather_rate(0, 32 << 20, 4, None) == nr.NR_EINVAL
    assert nr.lib.nr_l2_gather_rate(0, 32 << 20, 8, C.byref(v)) == nr.NR_EINVAL
    assert b"load_bytes" in nr.lib.nr_last_error()
    assert nr.lib.nr_l2_gather_rate(0, (32 << 20) + 4096, 4, C.byref(v)) == nr.NR_EINVAL
    assert nr.lib.nr_l2_gather_rate(0, 1 << 19, 16, C.byref(v)) == nr.NR_EINVAL
    assert b"table_bytes" in nr.lib.nr_last_error()
