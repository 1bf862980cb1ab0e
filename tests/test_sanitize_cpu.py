"""The host side of libgfpdot under AddressSanitizer and
UndefinedBehaviorSanitizer: the service's dispatcher, admission, arena and
queue logic (simulation mode), the parameter derivations and reductions, and
argument checking run in a child process against the host-sanitized build of
the library, with libasan preloaded.  Any memory error or undefined
behaviour aborts the child, which fails this test.  No GPU is used."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HOST_TESTS = ["tests/test_server_sim.py", "tests/test_params.py",
              "tests/test_abi.py::test_status_strings",
              "tests/test_abi.py::test_choose_repr_rules_without_context",
              "tests/test_properties_cpu.py"]


def _libasan():
    for cc in ("gcc", "cc"):
        try:
            out = subprocess.run([cc, "-print-file-name=libasan.so"], capture_output=True,
                                 text=True).stdout.strip()
        except FileNotFoundError:
            continue
        if out and os.path.isabs(out) and os.path.exists(out):
            return out
    return None


def test_host_code_clean_under_asan_ubsan(lib):
    asan = _libasan()
    if asan is None:
        pytest.skip("no libasan for the host compiler")
    from paper_cs_0404008_gb300 import build
    build.build(sanitize=True)
    env = dict(os.environ)
    env.update({
        "GFPDOT_SANITIZED": "1",
        "LD_PRELOAD": asan,
        # the interpreter itself is not instrumented and keeps memory until exit;
        # the CUDA driver maps memory inside the shadow gap
        "ASAN_OPTIONS": "detect_leaks=0:protect_shadow_gap=0:abort_on_error=1",
        "UBSAN_OPTIONS": "print_stacktrace=1:halt_on_error=1",
    })
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "not gpu",
                        "-p", "no:cacheprovider", *HOST_TESTS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    tail = (r.stdout + r.stderr)[-4000:]
    assert r.returncode == 0, tail
    assert "AddressSanitizer" not in tail and "runtime error" not in tail, tail
