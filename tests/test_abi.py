"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU and exports every
function include/gcmc.h declares; the binding's structs match the header's field order."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "gcmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gcmc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_2110_15640_gb300 import build
    return build.build()


def test_library_exports_every_declared_function(built):
    names = header_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gcmc_[a-z_0-9]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(built):
    from paper_2110_15640_gb300 import gcmc
    L = gcmc.lib()
    assert L.gcmc_version().startswith(b"gcmc")
    assert set(gcmc.EXPORTED) == set(header_functions())


def test_struct_layouts_match_header():
    from paper_2110_15640_gb300 import gcmc
    import ctypes as C
    # sizes computed from the header's field lists (LP64)
    assert C.sizeof(gcmc.gcmc_grid_desc) == 16 + 7 * 8
    assert C.sizeof(gcmc.gcmc_job) == 8 * 4 + 16
    assert C.sizeof(gcmc.gcmc_launch_cfg) == 24
    assert C.sizeof(gcmc.gcmc_stats) == 16 + 64 + 16 + 8 + 8
    assert C.sizeof(gcmc.gcmc_source_desc) == 24 + 8 + 8 * 3 * 8 + 6 * 8 + 8 + 8 + 8 + 8 + 8 + 4 * 8 + 2 * 8 + 2 * 8 + 8 + 8 + 8 + 8
    assert C.sizeof(gcmc.gcmc_transit_obs) == 8 * 8
    assert C.sizeof(gcmc.gcmc_server_cfg) == 6 * 4 + 8 + 2 * 4
    assert C.sizeof(gcmc.gcmc_server_stats) == 5 * 8 + 2 * 4


def test_missing_library_fails_loudly(monkeypatch):
    """Without the built library the product raises; there is no CPU fallback."""
    from paper_2110_15640_gb300 import gcmc
    monkeypatch.setattr(gcmc, "_lib", None)
    monkeypatch.setattr(gcmc, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "libgcmc.so"))
    with pytest.raises(RuntimeError, match="not built"):
        gcmc.lib()


def test_product_never_uses_the_oracle():
    """The package (CUDA sources, binding, inputs, autotuner) neither imports nor loads the oracle."""
    pkg = os.path.join(ROOT, "paper_2110_15640_gb300")
    hits = []
    for dirpath, dirnames, files in os.walk(pkg):
        dirnames[:] = [d for d in dirnames if d not in ("_build", "__pycache__")]
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp", ".c")):
                src = open(os.path.join(dirpath, f)).read()
                if re.search(r"(import\s+oracle|from\s+oracle|liboracle|oracle\.c|orc_[a-z_]+\s*\()", src):
                    hits.append(f)
    assert not hits, hits


def test_header_is_plain_c_and_links_from_c(built, tmp_path):
    """include/gcmc.h compiles as C11 and as C++ without warnings, and a C program links against the
    library and calls it (gcmc_version needs no GPU)."""
    prog = tmp_path / "use_gcmc.c"
    prog.write_text('#include "gcmc.h"\n#include <stdio.h>\n'
                    'int main(void) {\n'
                    '    gcmc_ctx *ctx = NULL;\n'
                    '    gcmc_status (*create)(int, gcmc_ctx **) = gcmc_create;\n'
                    '    (void)ctx; (void)create;\n'
                    '    printf("%s\\n", gcmc_version());\n'
                    '    return 0;\n'
                    '}\n')
    inc = os.path.join(ROOT, "include")
    libdir = os.path.dirname(built)
    exe = tmp_path / "use_gcmc"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, str(prog), "-o", str(exe),
                    "-L", libdir, "-lgcmc", f"-Wl,-rpath,{libdir}"], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    assert out.startswith("gcmc")
    cpp = tmp_path / "use_gcmc.cpp"
    cpp.write_text('#include "gcmc.h"\nint main() { return gcmc_version() ? 0 : 1; }\n')
    subprocess.run(["g++", "-std=c++17", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, "-fsyntax-only", str(cpp)],
                   check=True, capture_output=True, text=True)
