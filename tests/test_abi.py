"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, exports every function include/skyline.h declares, and
every struct of the header has the layout the binding assumes."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = "".join(open(os.path.join(ROOT, "include", h)).read() for h in ("skyline.h", "skyline_diag.h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sky_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2411_14968_gb300 import native
    return native.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "sky_skyline" in names and "sky_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2411_14968_gb300 import native
    assert sorted(native.EXPORTS) == sorted(n for n in _declared())


def test_params_layout_and_defaults(lib):
    from paper_2411_14968_gb300 import native
    p = native.SkyParams()
    lib.sky_params_init(ctypes.byref(p))
    assert p.struct_size == ctypes.sizeof(native.SkyParams)
    assert p.scheme == native.SCHEMES["none"] and p.num_partitions == 1
    assert list(p.slices) == [1] * 8 and p.grid_filter == 1 and p.reps_per_partition == 1
    assert p.merge == 0 and p.exec == 0 and p.rep == 0
    # engine knobs 0 = built-in defaults; images of the values by default
    assert p.chunk_min == p.chunk_max == p.chunk_alpha_x4 == p.dom_block == 0
    assert p.engine_warps == p.engine_cands == 0 and p.images == native.IMAGES["values"]


def test_status_strings(lib):
    for s in range(7):
        assert lib.sky_status_str(s).decode().startswith("SKY_")


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.sky_create(ctypes.byref(h), 0, 0)
    assert st != 0 and not h.value


def test_library_is_built_for_sm_103a():
    from paper_2411_14968_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.LIB_PATH)


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct of the C ABI has, field by field, the offset and size the
    ctypes binding assumes: a small C program compiled against
    include/skyline.h prints sizeof and offsetof of each."""
    import shutil
    import subprocess
    from paper_2411_14968_gb300 import native
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"sky_params": native.SkyParams, "sky_stats": native.SkyStats, "sky_query": native.SkyQuery,
               "sky_serve_config": native.SkyServeConfig, "sky_ticket_info": native.SkyTicketInfo}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "skyline.h"', "int main(void) {"]
    want = []
    for cname, cls in structs.items():
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(cls))
        for f, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f}));')
            want.append(getattr(cls, f).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == want
