"""The C-ABI library builds, loads without a GPU and exports every entry
point declared in include/mmncg.h."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mmncg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mm_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1801_03690_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        pytest.skip("library not built (run __graft_entry__.build())")
    lib = _lib.load()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.EXPORTS), set(names) ^ set(_lib.EXPORTS)


def test_create_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1801_03690_gb300 import _lib, Magnet, MMError
    if not os.path.exists(_lib.LIB_PATH):
        pytest.skip("library not built")
    with pytest.raises(MMError):
        Magnet(device=0)


def test_header_is_plain_c(tmp_path):
    """include/mmncg.h is a C header: it compiles as C99 with -pedantic, so
    callers outside C++ and PyTorch can use the library."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "mmncg.h"\nint main(void) { mm_params p; mm_default_params(&p); return p.jmax; }\n')
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.join(ROOT, "include"), "-c", str(src), "-o", str(tmp_path / "use_header.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_and_calls_host_entry_points(tmp_path):
    """A C program links libmmncg.so and calls two entry points that need no
    GPU: the default parameters of Algorithm 4 and the batch team split
    (blocks in proportion to work, largest remainders, summing to the grid)."""
    import shutil
    import subprocess
    from paper_1801_03690_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None or not os.path.exists(_lib.LIB_PATH):
        pytest.skip("no C compiler or library not built")
    src = tmp_path / "use_lib.c"
    src.write_text(
        '#include <stdio.h>\n#include "mmncg.h"\n'
        "int main(void) {\n"
        "    mm_params p; int64_t work[3] = {100, 400, 900}; int32_t b[3];\n"
        "    mm_default_params(&p);\n"
        "    if (mm_batch_plan(3, work, 60, 1.0, b) != 0) return 1;\n"
        '    printf("%d %g %d %d %d\\n", p.jmax, p.tau_F, b[0], b[1], b[2]);\n'
        "    return 0;\n}\n")
    libdir = os.path.dirname(_lib.LIB_PATH)
    exe = tmp_path / "use_lib"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir,
                        "-lmmncg", f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    jmax, tau, *blocks = r.stdout.split()
    assert int(jmax) == 4 and float(tau) == 1e-10
    assert [int(x) for x in blocks] == [4, 17, 39]          # 60 x (1, 4, 9) / 14, largest remainders
