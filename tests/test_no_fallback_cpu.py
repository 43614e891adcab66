"""The product path has no CPU fallback: without the CUDA library every entry point
raises, and nothing in the package reaches the oracle."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1411_5512_gb300")


def test_package_never_reaches_the_oracle():
    pat = re.compile(r"\boracle\b|ea_oracle|libea_oracle")
    hits = []
    for dirpath, _, files in os.walk(PKG):
        if "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp", ".c")):
                path = os.path.join(dirpath, f)
                with open(path, encoding="utf-8") as fh:
                    for n, line in enumerate(fh, 1):
                        if pat.search(line):
                            hits.append("%s:%d: %s" % (os.path.relpath(path, ROOT), n, line.strip()))
    assert not hits, "\n".join(hits)


_MISSING = r"""
import sys
sys.path.insert(0, sys.argv[1])
from paper_1411_5512_gb300 import _lib, job
_lib.load.__defaults__ = ("/nonexistent/libea_gb300.so",)
failures = []
for name, call in [("EAJob", lambda: job.EAJob(16, 0.5, 1, 1)),
                   ("EABatch", lambda: job.EABatch()),
                   ("EAServer", lambda: job.EAServer(1 << 30)),
                   ("restore", lambda: job.EAJob.restore("/nonexistent/job.ckpt")),
                   ("geometry", lambda: job.geometry(16)),
                   ("thresholds", lambda: job.thresholds(0.7)),
                   ("launch_count", lambda: job.launch_count())]:
    try:
        call()
        failures.append(name + " ran without the library")
    except RuntimeError as e:
        if "not built" not in str(e):
            failures.append(name + ": " + str(e))
    except Exception as e:  # a different error: still loud, but say which
        failures.append(name + " raised " + type(e).__name__ + ": " + str(e))
print("\n".join(failures))
sys.exit(1 if failures else 0)
"""


def test_entry_points_raise_without_the_cuda_library():
    p = subprocess.run([sys.executable, "-c", _MISSING, ROOT], capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stdout + p.stderr
