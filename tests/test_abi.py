"""CPU checks of the C-ABI boundary: the library builds, loads, exports every
entry point include/distill_gpu.h declares, and the binding declares the same
set. No compute call is made (there is no GPU here)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(?:dg_status|const char\s*\*)\s*(dg_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def so():
    from paper_2110_15425_gb300 import build
    try:
        return build.build()
    except (RuntimeError, FileNotFoundError) as e:
        pytest.skip(f"nvcc unavailable: {e}")


def test_header_declares_entry_points():
    names = _declared()
    for n in ["dg_create", "dg_compose", "dg_run", "dg_grid_search", "dg_submit", "dg_wait",
              "dg_batch_launch", "dg_philox_words"]:
        assert n in names


def test_library_exports_every_declared_symbol(so):
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dg_\w+)", out))
    missing = _declared() - exported
    assert not missing, missing


def test_binding_matches_header(so):
    from paper_2110_15425_gb300 import binding as B
    assert set(B.EXPORTS) == _declared()
    L = B.lib()
    for n in B.EXPORTS:
        assert hasattr(L, n)


def test_struct_layouts_match_header(so):
    """Compile a tiny C program against the header and compare sizeof/offsetof
    with the ctypes mirrors."""
    from paper_2110_15425_gb300 import binding as B
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "distill_gpu.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(dg_mechanism), sizeof(dg_projection),
         sizeof(dg_stop), sizeof(dg_run_desc), sizeof(dg_grid_desc), sizeof(dg_grid_result),
         sizeof(dg_job), sizeof(dg_job_result));
  printf("%zu %zu %zu %zu\n", offsetof(dg_job, run), offsetof(dg_job, grid),
         offsetof(dg_job, choice), offsetof(dg_grid_desc, positions));
  return 0;
}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    sizes = [int(v) for v in lines[0].split()]
    mine = [C.sizeof(t) for t in (B.dg_mechanism, B.dg_projection, B.dg_stop, B.dg_run_desc,
                                  B.dg_grid_desc, B.dg_grid_result, B.dg_job, B.dg_job_result)]
    assert sizes == mine
    offs = [int(v) for v in lines[1].split()]
    assert offs == [B.dg_job.run.offset, B.dg_job.grid.offset, B.dg_job.choice.offset,
                    B.dg_grid_desc.positions.offset]


def test_error_strings_without_gpu(so):
    from paper_2110_15425_gb300 import binding as B
    assert B.dg_version().startswith("distill-gpu")
    assert isinstance(B.dg_last_error(), str)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2110_15425_gb300 import binding as B
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(RuntimeError):
        B.lib()
