"""The C-ABI library loads without a GPU and exports every entry point include/*.h declares;
the Python binding covers exactly those names."""
import ctypes
import glob
import os
import re
import subprocess

from paper_2605_18515_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(cbspmv_[a-z0-9_]+)\s*\(", text))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cbspmv_analyze", "cbspmv_run", "cbspmv_export_csr", "cbspmv_destroy",
                     "cbspmv_get_stats", "cbspmv_last_error", "cbspmv_default_opts"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib_path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(cbspmv_[a-z0-9_]+)$", out, flags=re.M))
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    lib = ctypes.CDLL(lib_path)          # loads without a GPU
    for name in declared_functions():
        assert hasattr(lib, name)


def test_binding_covers_the_header():
    from paper_2605_18515_gb300 import binding
    assert set(binding.SIGNATURES) == declared_functions()
    assert binding.version().startswith("cbspmv")
    # the Python-level API over those entry points
    for name in ("BlockedMatrix", "Server", "Graph", "analyze_batched", "run_batched", "analyze_tuned"):
        assert callable(getattr(binding, name)), name
    for meth in ("run", "run_multi", "run_host", "time_kernels", "export_csr", "export_blocked", "stats"):
        assert callable(getattr(binding.BlockedMatrix, meth)), meth
    for meth in ("register", "submit_spmv", "submit_cg", "wait", "poll", "stats", "close"):
        assert callable(getattr(binding.Server, meth)), meth
