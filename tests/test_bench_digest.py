"""The digest that ties committed ncu traffic figures to the kernel sources: it
ignores comments and layout and changes with any code edit."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _digest_of(tmp_path, edit=None):
    pkg = tmp_path / "paper_2004_09350_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_2004_09350_gb300", "csrc"), pkg / "csrc")
    if edit:
        f = pkg / "csrc" / "ms_kernels.cuh"
        f.write_text(edit(f.read_text()))
    old = bench.ROOT
    bench.ROOT = str(tmp_path)
    try:
        return bench.source_digest()
    finally:
        bench.ROOT = old


def test_comments_and_layout_do_not_count(tmp_path):
    base = _digest_of(tmp_path / "a")
    assert base == bench.source_digest()
    assert _digest_of(tmp_path / "b", lambda s: s.replace("namespace ms {", "namespace ms {  // note\n\n/* a\n b */")) == base
    assert _digest_of(tmp_path / "c", lambda s: s.replace("constexpr int kClaim = 128;", "constexpr  int kClaim =  128;")) == base


def test_code_edits_count(tmp_path):
    base = _digest_of(tmp_path / "a")
    assert _digest_of(tmp_path / "b", lambda s: s.replace("constexpr int kClaim = 128;", "constexpr int kClaim = 64;")) != base

