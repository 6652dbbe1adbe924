"""bench.py reports a kernel's DRAM traffic from profiles/ only while the
kernel's sources are those of the capture, keyed by a hash over the csrc files
listed for it.  Every csrc header that those files include (directly or not)
must be in that list, or a change to it would leave a stale figure in force.

CPU only: reads source files.
"""
import os
import re

import bench

CSRC = os.path.join(bench.ROOT, "paper_2504_05148_gb300", "csrc")


def _includes(fname):
    text = open(os.path.join(CSRC, fname)).read()
    return [f for f in re.findall(r'^\s*#include\s+"([^"]+)"', text, flags=re.M)
            if os.path.exists(os.path.join(CSRC, f))]


def test_every_included_header_is_hashed_with_its_kernel():
    files = sorted(os.listdir(CSRC))
    for kernel, prefixes in bench.KERNEL_SOURCES.items():
        pre = prefixes + ("sgmf_internal", "sgmf_api")
        hashed = [f for f in files if f.startswith(pre)]
        assert hashed, kernel
        seen, todo = set(), list(hashed)
        while todo:
            f = todo.pop()
            if f in seen:
                continue
            seen.add(f)
            todo += _includes(f)
        missing = sorted(f for f in seen if not f.startswith(pre))
        assert not missing, f"{kernel}: {missing} not covered by its source hash"


def test_hash_changes_with_a_kernels_header(tmp_path, monkeypatch):
    # the hash follows the file contents, not their names or dates
    import shutil
    root = tmp_path / "repo"
    shutil.copytree(CSRC, root / "paper_2504_05148_gb300" / "csrc")
    monkeypatch.setattr(bench, "ROOT", str(root))
    before = bench.src_hash("cost")
    p = root / "paper_2504_05148_gb300" / "csrc" / "sgmf_cost.cuh"
    p.write_text(p.read_text() + "\n")
    assert bench.src_hash("cost") != before
    assert bench.src_hash("agg_sweep") == bench.src_hash("agg_sweep")
