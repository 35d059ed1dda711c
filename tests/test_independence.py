"""The oracle and the CUDA path stay independent: no source of the library
package imports or includes anything of the oracle, no oracle source
refers to the package, its kernels or its header, the shared input module
imports neither side, outside tests/ only the build/smoke entry points
and the benchmark's CPU legs import the oracle, and the package refuses to
import without its CUDA library (no fallback)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def tracked(prefix=""):
    cmd = ["git", "ls-files"] + ([prefix] if prefix else [])
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True).stdout.split()
    if not out:  # not a git checkout: walk the tree instead
        base = os.path.join(ROOT, prefix)
        out = [os.path.relpath(os.path.join(d, f), ROOT) for d, _, fs in os.walk(base) for f in fs
               if "_build" not in d and "__pycache__" not in d]
    return out


def read(rel):
    with open(os.path.join(ROOT, rel), errors="replace") as fh:
        return fh.read()


PY_IMPORT_ORACLE = re.compile(r"^\s*(import oracle\b|from oracle\b)", re.M)


def test_package_does_not_use_the_oracle():
    for rel in tracked("paper_2606_25453_gb300"):
        src = read(rel)
        if rel.endswith(".py"):
            assert not PY_IMPORT_ORACLE.search(src), rel
        if rel.endswith((".cu", ".cuh", ".h", ".c", ".cpp")):
            assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", src), rel
    for rel in tracked("include"):
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", read(rel)), rel


def test_oracle_does_not_use_the_package():
    for rel in tracked("oracle"):
        src = read(rel)
        if rel.endswith(".py"):
            assert not re.search(r"^\s*(import|from)\s+(paper_2606_25453_gb300|synth)\b", src, re.M), rel
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*(emugemm|csrc|emu_internal|emu_device)", src), rel
        assert "libemugemm" not in src, rel


def test_shared_inputs_import_neither_side():
    src = read("synth.py")
    assert not PY_IMPORT_ORACLE.search(src)
    assert "paper_2606_25453_gb300" not in src


def test_only_allowed_modules_import_the_oracle():
    allowed = {"__graft_entry__.py", "bench.py"}
    for rel in tracked():
        if not rel.endswith(".py") or rel.startswith(("tests/", "oracle/")):
            continue
        if PY_IMPORT_ORACLE.search(read(rel)):
            assert rel in allowed, rel


def test_package_import_fails_loudly_without_the_library():
    # the binding has no fallback: with its shared library missing, the
    # import itself raises
    code = (
        "import importlib.util, sys\n"
        "spec = importlib.util.spec_from_file_location('paper_2606_25453_gb300.build', %r)\n"
        "mod = importlib.util.module_from_spec(spec)\n"
        "spec.loader.exec_module(mod)\n"
        "mod.LIB = '/nonexistent/libemugemm.so'\n"
        "sys.modules['paper_2606_25453_gb300.build'] = mod\n"
        "try:\n"
        "    import paper_2606_25453_gb300\n"
        "except ImportError as e:\n"
        "    print('raised:', e)\n"
        "    sys.exit(0)\n"
        "sys.exit(3)\n" % os.path.join(ROOT, "paper_2606_25453_gb300", "build.py"))
    import sys
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "not built" in r.stdout
