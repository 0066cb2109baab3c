"""Structural rules of the repository, checked on the source text.

* Every entry point declared in include/vla.h is documented by a comment that
  cites the paper passage defining its operation (or states that the paper
  has no counterpart) and states its error behaviour.
* The oracle and the library share no code: the package and its CUDA sources
  never import, include or load anything under oracle/, and the oracle never
  imports the package.
"""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2404_16039_gb300")


def _read(path):
    with open(path, encoding="utf-8") as f:
        return f.read()


def test_every_entry_point_cites_its_passage():
    s = _read(os.path.join(ROOT, "include", "vla.h"))
    comments = [(m.end(), re.sub(r"\s*\n\s*\*\s*", " ", m.group(0))) for m in re.finditer(r"/\*.*?\*/", s, re.S)]
    decls = [(m.start(), m.group(1)) for m in
             re.finditer(r"^(?:vla_status|int32_t|const char \*)\s*(vla_\w+)\(", s, re.M)]
    assert len(decls) > 40
    cite = re.compile(r"Section \d|no counterpart in the paper|paper has no counterpart")
    errors = re.compile(r"VLA_ERR_|errors|cannot fail", re.I)
    uncited, silent = [], []
    for pos, name in decls:
        before = [text for end, text in comments if end <= pos]
        doc = before[-1] if before else ""
        if not cite.search(doc):
            uncited.append(name)
        if name not in ("vla_last_error",) and not errors.search(doc):
            silent.append(name)
    assert not uncited, uncited
    assert not silent, silent          # every entry point states its error behaviour


def test_oracle_and_library_share_no_code():
    lib_sources = glob.glob(os.path.join(PKG, "*.py")) + glob.glob(os.path.join(PKG, "csrc", "*"))
    for path in lib_sources:
        text = _read(path)
        assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), path
        assert "liboracle" not in text and "vla_oracle" not in text, path
        assert not re.search(r'#include\s+["<][^">]*oracle', text), path
    for path in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if path.endswith((".py", ".c", ".h")):
            text = _read(path)
            assert not re.search(r"^\s*(import|from)\s+paper_2404_16039_gb300\b", text, re.M), path
            assert "libvla" not in text and '#include "vla' not in text, path
