"""The product path and the oracle stay apart: nothing in the package imports or
loads the oracle, the CUDA sources include nothing of it, and the oracle includes
nothing of the CUDA library.  Only synth.py (seeded input generators, no NURBS
arithmetic) is shared."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2104_14547_gb300")


def _sources(folder, exts):
    for dirpath, _, files in os.walk(folder):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(dirpath, f)


def test_package_never_imports_the_oracle():
    for path in _sources(PKG, (".py",)):
        text = open(path).read()
        assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), path
        assert "nurbs_oracle" not in text, path


def test_cuda_sources_and_oracle_share_no_headers():
    for path in _sources(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h")):
        for inc in re.findall(r'#include\s+[<"]([^>"]+)[>"]', open(path).read()):
            assert "oracle" not in inc, (path, inc)
    for path in _sources(os.path.join(ROOT, "oracle"), (".c", ".h", ".py")):
        text = open(path).read()
        for inc in re.findall(r'#include\s+[<"]([^>"]+)[>"]', text):
            assert inc in ("math.h", "string.h", "stdlib.h", "stddef.h", "stdint.h"), (path, inc)
        assert "paper_2104_14547_gb300" not in text, path


def test_synth_holds_no_nurbs_arithmetic():
    text = open(os.path.join(PKG, "synth.py")).read()
    for word in ("basis", "find_span", "de Boor", "homog", "_lib", "csrc"):
        assert word not in text, word
