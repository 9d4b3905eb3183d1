"""The C-ABI library builds, loads and exports every entry point that include/bingo.h declares (no GPU needed)."""
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "bingo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bingo_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_10233_gb300 import _build

    path = _build.build()
    import paper_2504_10233_gb300 as B

    B.load()
    return path


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("bingo_create", "bingo_apply_updates", "bingo_walk", "bingo_stream_updates", "bingo_export_state",
                 "bingo_server_create", "bingo_server_submit_walk"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib]).decode()
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in _declared() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_declared_symbol(lib):
    import paper_2504_10233_gb300 as B

    assert sorted(B.SIGNATURES) == _declared()
    L = B.load()
    assert L.bingo_version().startswith(b"bingo-gb300")


def test_library_targets_sm103a(lib):
    out = subprocess.run(["cuobjdump", "--list-elf", lib], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2504_10233_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "oracle/" not in txt, f
