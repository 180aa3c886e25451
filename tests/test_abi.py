"""CPU checks of the C-ABI library: it loads and exports every entry point
that include/pbfmm.h declares (no compute call without a GPU)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "pbfmm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", txt, flags=re.M)))


def test_library_exports_declared_symbols():
    import paper_2103_01048_gb300 as pb
    names = declared()
    assert len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", pb.lib_path()], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if " T " in l)
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(pb._lib, n)


def test_binding_names_match_header():
    import paper_2103_01048_gb300 as pb
    assert set(pb.exported_symbols()) <= set(declared())


def test_library_exports_test_hooks():
    """The hooks of include/pbfmm_testing.h and the microbenchmark entry of
    include/pbfmm_peaks.h are exported too."""
    import paper_2103_01048_gb300 as pb
    names = []
    for h in ("pbfmm_testing.h", "pbfmm_peaks.h"):
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:int|int64_t|void)\s+(\w+)\s*\(", txt, flags=re.M)
    assert len(names) >= 6
    out = subprocess.run(["nm", "-D", "--defined-only", pb.lib_path()], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if " T " in l)
    assert not [n for n in names if n not in exported]
