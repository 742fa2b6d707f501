"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol include/psdproj.h declares; host-only queries answer without a GPU."""
import os
import re

import pytest

import oracle
from oracle import schedules as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "psdproj.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(psd_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_09165_gb300 import _build, binding
    _build.build()
    return binding.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "psd_project" in names and "psd_project_batched" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_library_schedule_matches_the_paper_tables():
    # The library and the oracle each carry their own transcription of
    # Tables 1 and 2; they must agree digit for digit.
    from paper_2507_09165_gb300 import binding as b
    coef, post = b.psd_schedule("fp16")
    assert coef == [tuple(c) for c in S.HALF_FTILDE]
    assert tuple(post) == S.post_scale("half", 7)
    coef, post = b.psd_schedule("fp32")
    assert coef == [tuple(c) for c in S.SINGLE_FTILDE]
    assert tuple(post) == S.post_scale("single", 10)


def test_gemm_counts():
    from paper_2507_09165_gb300 import binding as b
    assert b.psd_gemm_count("fp16") == 22  # Sec. 3.3 / abstract
    assert b.psd_gemm_count("bf16") == 22
    assert b.psd_gemm_count("fp32") == 31
    assert b.psd_gemm_count("fp8_late") == 22  # the half schedule with e4m3 late stages


def test_host_side_argument_checks():
    from paper_2507_09165_gb300 import binding as b
    L = b.lib()
    assert L.psd_project(-1, 0, 1, 0, 1, None) == 1
    assert L.psd_project(0, 0, 0, 0, 1, None) == 0   # n == 0 is a no-op
    assert L.psd_project(4, 0, 4, 0, 1, None) == 1   # null pointers
    assert L.psd_project(4, 16, 3, 4096, 1, None) == 1   # ld < n
    assert L.psd_project(4, 16, 4, 4096, 9, None) == 1   # bad precision
    # partial overlap of X and out
    assert L.psd_project(4, 4096, 4, 4096 + 8, 1, None) == 1
    assert L.psd_workspace_size(10000, 1) > 4 * 10000 * 10000 * 2
    assert L.psd_workspace_size(-3, 1) == 0
    assert b.psd_status_string(5).startswith("norm bound")


def test_oracle_and_library_share_no_code():
    # The oracle never imports the CUDA package and the package never imports the oracle.
    pkg = os.path.join(ROOT, "paper_2507_09165_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2507_09165_gb300" not in txt, f
    assert oracle.num_threads() >= 1
