"""The product path's boundary, checked on the CPU: the package never reaches the oracle, the
binding refuses to load without the compiled library (no fallback), and the committed profile of
the propagate/bin kernel describes the current kernel source (so the bench reports its traffic)."""
import ast
import os
import shutil
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1310_5541_gb300")


def test_package_sources_do_not_import_the_oracle():
    for name in sorted(os.listdir(PKG)):
        if not name.endswith(".py"):
            continue
        tree = ast.parse(open(os.path.join(PKG, name)).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            else:
                continue
            assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), (name, mods)


def test_binding_fails_loudly_without_the_library(tmp_path):
    pkg = tmp_path / "paper_1310_5541_gb300"
    shutil.copytree(PKG, pkg, ignore=shutil.ignore_patterns("*.so", "__pycache__", "csrc"))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "try:\n"
            "    import paper_1310_5541_gb300.pcsir\n"
            "except ImportError as e:\n"
            "    print('refused:', e)\n"
            "    sys.exit(0)\n"
            "sys.exit(1)\n") % str(tmp_path)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "not built" in r.stdout
    assert "oracle" not in r.stdout


def test_committed_propagate_bin_profile_matches_the_kernel_source():
    txt = open(os.path.join(ROOT, "profiles", "k_prop_bin_512x512_h0.5.md")).read()
    assert "kernel source hash: %s" % bench.kernel_source_hash() in txt
    assert bench.profiled_traffic(1 << 24) is not None
