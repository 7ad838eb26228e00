"""The C-ABI library builds, loads and exports every entry point that
include/mor_spai.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

import paper_2003_12759_gb300 as mor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mor_spai.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?(?:int|void|char\s*\*|const char\s*\*)\s*\**\s*(mor_\w+)\s*\(",
                                 text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_12759_gb300 import build
    build.build()
    return mor.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mor_create", "mor_destroy", "mor_set_system", "mor_build_precond", "mor_update_precond",
                     "mor_solve_shifts", "mor_irka_step", "mor_eval_tf", "mor_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    raw = ctypes.CDLL(mor.LIB_PATH)
    for name in names:
        assert hasattr(raw, name), name
        assert name in mor.SIGNATURES, "binding lacks " + name


def test_binding_structs_match_header_sizes():
    # mor_solve_opts: 11 fields, mor_reduced capacity fixed by MOR_MAX_R / MOR_MAX_IO
    assert ctypes.sizeof(mor.mor_c64) == 16
    assert ctypes.sizeof(mor.mor_csr) == 40
    assert ctypes.sizeof(mor.mor_reduced) == 12 + 4 + 8 * (2 * 64 * 64 + 2 * 64 * 8)
    text = open(HEADER).read()
    assert "#define MOR_MAX_R 64" in text and "#define MOR_MAX_IO 8" in text


def test_product_path_does_not_import_oracle():
    """The CUDA path never routes through the oracle."""
    pkg = os.path.join(ROOT, "paper_2003_12759_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """sizeof / offsetof of the option and statistics structs as gcc lays them
    out from include/mor_spai.h equal the ctypes binding's."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mor_spai.h"\n'
                   'int main(void) { printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mor_solve_opts), '
                   'offsetof(mor_solve_opts, restart), offsetof(mor_solve_opts, max_chain), '
                   'sizeof(mor_solve_stats), sizeof(mor_reduced), sizeof(mor_reduced2), '
                   'offsetof(mor_reduced2, Kr), offsetof(mor_solve_opts, fp64_fallback), '
                   'offsetof(mor_solve_stats, fallback), sizeof(mor_irka_stats), '
                   'offsetof(mor_irka_stats, fallbacks), offsetof(mor_solve_opts, concurrent_sweeps), '
                   'offsetof(mor_solve_opts, reuse), offsetof(mor_solve_opts, moments)); return 0; }\n')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(mor.mor_solve_opts), mor.mor_solve_opts.restart.offset, mor.mor_solve_opts.max_chain.offset,
            ctypes.sizeof(mor.mor_solve_stats), ctypes.sizeof(mor.mor_reduced), ctypes.sizeof(mor.mor_reduced2),
            mor.mor_reduced2.Kr.offset, mor.mor_solve_opts.fp64_fallback.offset, mor.mor_solve_stats.fallback.offset,
            ctypes.sizeof(mor.mor_irka_stats), mor.mor_irka_stats.fallbacks.offset,
            mor.mor_solve_opts.concurrent_sweeps.offset, mor.mor_solve_opts.reuse.offset,
            mor.mor_solve_opts.moments.offset]
    assert got == want


def test_default_options(lib):
    """mor_default_opts fills host memory only (no GPU call)."""
    o = mor.mor_default_opts()
    assert o.solver == mor.MOR_BICGSTAB and o.precision == mor.MOR_MIXED and o.restart == 50
    assert o.tol == 1e-8 and o.precond == 0 and o.max_chain == 0 and o.precond_precision == -1
    assert o.fp64_fallback == 1 and o.concurrent_sweeps == 1
    assert o.reuse == mor.MOR_REUSE_CHAIN and o.moments == 1
