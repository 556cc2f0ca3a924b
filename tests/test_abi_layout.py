"""The ctypes structures of the binding match include/kt.h field by field: a C program
compiled against the header prints sizeof and offsetof of every structure and field, and
the binding's ctypes layout must give the same numbers (CPU only; needs gcc)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_0908_0681_gb300 import kt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["kt_model_params", "kt_model_info", "kt_stats", "kt_seq_batch", "kt_move_batch", "kt_sweep_params",
           "kt_sweep_state", "kt_sweep_accum"]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kt.h"', 'int main(void) {']
    for name in STRUCTS:
        cls = getattr(kt, name)
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return dict((k, int(v)) for k, v in (line.split() for line in out.splitlines()))


def test_ctypes_structures_match_the_header(tmp_path):
    c = _c_layout(tmp_path)
    for name in STRUCTS:
        cls = getattr(kt, name)
        assert ctypes.sizeof(cls) == c[name], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == c[f"{name}.{field}"], (name, field)


def test_stats_words_cover_the_structure():
    assert ctypes.sizeof(kt.kt_stats) == 8 * kt.STATS_WORDS


def test_constants_match_the_header(tmp_path):
    """Status codes, precision and flag values, and the sizes the binding hard-codes, are the
    header's (a C program prints them)."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    names = kt.STATUS_NAMES + ["KT_FP64", "KT_FP32_KRYLOV", "KT_DENSITY_ONLY", "KT_SECTOR_BLOCKS", "KT_HOST_ONLY",
                               "KT_FP32_TRIDIAG64",
                               "KT_P_HIST", "KT_SWEEP_NCOUNTERS", "KT_MLP_HIDDEN", "KT_STATIC_SCRATCH_BYTES",
                               "KT_DA_MAX_TRIES"]
    lines = ['#include <stdio.h>', '#include "kt.h"', 'int main(void) {']
    lines += [f'  printf("{n} %lld\\n", (long long)({n}));' for n in names]
    lines += [f'  printf("NOBS{n} %lld\\n", (long long)KT_MEASURE_NOBS({n}));' for n in (3, 5, 7)]
    lines += ['  return 0;', '}']
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "consts"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    c = dict((k, int(v)) for k, v in (line.split() for line in out.splitlines()))
    for code, n in enumerate(kt.STATUS_NAMES):
        assert c[n] == code == getattr(kt, n), n
    for n in names[len(kt.STATUS_NAMES):]:
        assert c[n] == getattr(kt, n), n
    for n in (3, 5, 7):
        assert c[f"NOBS{n}"] == kt.measure_nobs(n)
