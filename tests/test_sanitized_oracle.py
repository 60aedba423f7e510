"""Opt-in (RST_SANITIZE=1, CPU, about a minute): the oracle and the input
generators rebuilt with AddressSanitizer and UndefinedBehaviorSanitizer, and
the CPU suite run against those builds in a child process.  Any out-of-bounds
access, use after free or undefined arithmetic in the C code fails it."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUNNER = """
import sys
sys.path.insert(0, {tests!r}); sys.path.insert(0, {root!r})
import oracle
oracle._SO = {oso!r}; oracle._lib = None
from paper_2603_11645_gb300 import graphs
graphs._GEN_SO = {gso!r}; graphs._lib = None
import pytest
if __name__ == "__main__":
    sys.exit(pytest.main(["-q", "-x", "-m", "not gpu", "-p", "no:cacheprovider",
                          "--deselect", "tests/test_sanitized_oracle.py::test_c_code_under_sanitizers",
                          "tests/"]))
"""


@pytest.mark.skipif(not os.environ.get("RST_SANITIZE"), reason="opt-in: set RST_SANITIZE=1")
def test_c_code_under_sanitizers(tmp_path):
    flags = ["-O1", "-g", "-std=c11", "-fPIC", "-shared", "-fsanitize=address,undefined",
             "-fno-omit-frame-pointer", "-fno-sanitize-recover=undefined"]
    oso, gso = str(tmp_path / "liboracle.so"), str(tmp_path / "libgraphgen.so")
    subprocess.check_call(["gcc", *flags, os.path.join(ROOT, "oracle", "rst_oracle.c"), "-o", oso])
    subprocess.check_call(["gcc", *flags, os.path.join(ROOT, "paper_2603_11645_gb300", "gen", "graphgen.c"),
                           "-o", gso, "-lm"])
    runner = tmp_path / "run.py"
    runner.write_text(RUNNER.format(tests=os.path.join(ROOT, "tests"), root=ROOT, oso=oso, gso=gso))
    pre = " ".join(subprocess.check_output(["gcc", f"-print-file-name={lib}"], text=True).strip()
                   for lib in ("libasan.so", "libubsan.so"))
    env = dict(os.environ, LD_PRELOAD=pre, ASAN_OPTIONS="detect_leaks=0")
    env.pop("RST_SANITIZE")
    r = subprocess.run([sys.executable, str(runner)], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1800)
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "runtime error" not in out and "AddressSanitizer" not in out, out[-4000:]
