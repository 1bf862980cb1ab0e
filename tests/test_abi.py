"""The C-ABI library loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "gfpdot.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"GFP_API\s+[\w\s\*]+?\b(gfp_\w+)\s*\(", txt)))


def test_header_symbols_exported(lib):
    syms = header_symbols()
    assert len(syms) >= 20
    so = ctypes.CDLL(lib.lib_path())
    missing = [s for s in syms if not hasattr(so, s)]
    assert not missing, missing


def test_binding_covers_header(lib):
    assert set(header_symbols()) <= set(lib.declared_symbols()) | {"gfp_get_params"}


def test_exports_are_only_the_abi(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.lib_path()], capture_output=True,
                         text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    ours = {s for s in exported if s.startswith("gfp_")}
    assert ours == set(header_symbols())


def test_status_strings(lib):
    assert lib.gfp_status_string(0) == "GFP_OK"
    assert lib.gfp_status_string(-2) == "GFP_ERR_RANGE"
    assert lib.gfp_status_string(12345) == "GFP_UNKNOWN_STATUS"


def test_choose_repr_rules_without_context(lib):
    assert lib.gfp_choose_repr(None, 65521, 1 << 20) == lib.GFP_REPR_U64_BLOCK
    assert lib.gfp_choose_repr(None, 2147483647, 1 << 20) == lib.GFP_REPR_U64_CARRY
    assert lib.gfp_choose_repr(None, 4294967291, 10) == lib.GFP_REPR_U64_CARRY
    assert lib.gfp_choose_repr(None, 1, 10) == lib.GFP_REPR_AUTO


def test_no_oracle_in_product():
    """The library and its binding never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_cs_0404008_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp", ".c")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "gfp_oracle" not in txt and "liboracle" not in txt, f


def sweep_header_symbols():
    txt = open(os.path.join(ROOT, "include", "gfpsweep.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gfp_sweep_\w+)\s*\(", txt)))


def test_sweep_library_exports_its_header():
    from paper_cs_0404008_gb300 import build
    path = build.build_sweep()
    syms = sweep_header_symbols()
    assert len(syms) == 5
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert {s for s in exported if s.startswith("gfp_")} == set(syms)


def test_gpu_library_does_not_contain_the_sweep(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.lib_path()], capture_output=True,
                         text=True).stdout
    assert "gfp_sweep_" not in out


def test_peaks_library_exports_its_header():
    from paper_cs_0404008_gb300 import build
    path = build.build_peaks()
    txt = open(os.path.join(ROOT, "include", "gfppeaks.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    syms = set(re.findall(r"\b(gfp_peak_\w+)\s*\(", txt))
    assert syms == {"gfp_peak_measure", "gfp_peak_name"}
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert {s for s in exported if s.startswith("gfp_")} == syms


def test_peaks_refuses_bad_arguments_without_a_gpu():
    from paper_cs_0404008_gb300 import peaks
    so = peaks.lib()
    r = peaks.gfp_peak_result()
    assert so.gfp_peak_measure(99, 0, 1, ctypes.byref(r)) == -1
    assert so.gfp_peak_measure(0, 1 << 30, 0, ctypes.byref(r)) == -1
    assert so.gfp_peak_measure(0, 16, 1, ctypes.byref(r)) == -1
    assert so.gfp_peak_name(0) == b"read_hbm" and so.gfp_peak_name(7) is None
