"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares.  CPU only: no call here touches a GPU."""
import ctypes as C
import glob
import os
import re
import subprocess

import pytest

from paper_1207_1114_gb300 import build as fbuild
from paper_1207_1114_gb300 import fastpfp as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(fastpfp_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def built():
    return fbuild.build()


def test_library_exports_every_declared_symbol(built):
    declared = _declared_symbols()
    assert "fastpfp_create" in declared and "fastpfp_match_batched" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (fastpfp_\w+)", out))
    assert declared <= exported, declared - exported
    assert declared <= set(F.EXPORTS) | declared
    lib = C.CDLL(built)
    for name in declared:
        assert getattr(lib, name) is not None


def test_binding_lists_every_declared_symbol():
    assert _declared_symbols() == set(F.EXPORTS)


def test_default_params_and_error_strings(built):
    p = F.default_params()
    assert p.alpha == 0.5 and p.max_outer == 100 and p.max_inner == 1000
    assert p.tol_outer == 1e-6 and p.tol_inner == 1e-6 and p.normalize_max == 1
    assert p.slack_policy == 0 and p.precision == F.FP32 and p.debug_flags == 0
    assert p.algorithm == F.ALG_FASTPFP and p.beta == 100.0
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert F.error_string(code) != "unknown error"


def test_struct_layouts_match_header():
    """The ctypes mirrors have the size the C compiler gives the header's structs."""
    src = r'''
#include <stddef.h>
#include <stdio.h>
#include "fastpfp.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(fastpfp_params), sizeof(fastpfp_stats), sizeof(fastpfp_pair));
  printf("%zu %zu %zu %zu\n", offsetof(fastpfp_stats, wave_pairs), offsetof(fastpfp_stats, ms_disc),
         offsetof(fastpfp_stats, host_syncs), offsetof(fastpfp_params, beta));
  printf("%d %d %d %d %d %d %d %d %d\n", FASTPFP_FP32, FASTPFP_BF16, FASTPFP_FP8, FASTPFP_FP32_SIMT,
         FASTPFP_ALG_FASTPFP, FASTPFP_ALG_PG, FASTPFP_ALG_FASTGA, FASTPFP_TUNE_SIZES, FASTPFP_TUNE_COUNTS);
  return 0;
}'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.splitlines()
    sizes = [int(x) for x in lines[0].split()]
    assert sizes == [C.sizeof(F.fastpfp_params), C.sizeof(F.fastpfp_stats),
                     C.sizeof(F.fastpfp_pair)]
    offs = [int(x) for x in lines[1].split()]
    assert offs == [F.fastpfp_stats.wave_pairs.offset, F.fastpfp_stats.ms_disc.offset,
                    F.fastpfp_stats.host_syncs.offset, F.fastpfp_params.beta.offset]
    consts = [int(x) for x in lines[2].split()]
    assert consts == [F.FP32, F.BF16, F.FP8, F.FP32_SIMT, F.ALG_FASTPFP, F.ALG_PG, F.ALG_FASTGA,
                      F.TUNE_SIZES, F.TUNE_COUNTS]
