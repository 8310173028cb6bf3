"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/sem.h declares (no GPU needed, no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "sem.h")).read()
    return sorted(set(re.findall(r"SEM_API\s+[\w\s\*]*?\b(sem_\w+)\s*\(", txt)))


def test_header_declares_the_hot_path():
    syms = declared_symbols()
    for s in ("sem_setup", "sem_ax", "sem_dssum", "sem_pcg_solve", "sem_pcg_solve_batched",
              "sem_tgv_init", "sem_tgv_step", "sem_destroy", "sem_strerror"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_2608_24348_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_names_are_declared():
    from paper_2608_24348_gb300 import sem
    assert set(sem.EXPORTS) <= set(declared_symbols())


def test_strerror_without_gpu():
    from paper_2608_24348_gb300 import sem
    L = sem.load()
    assert L.sem_strerror(-5).decode() == "solver did not converge"
    assert L.sem_strerror(0).decode() == "ok"


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the CUDA library absent, load() raises."""
    import pytest

    from paper_2608_24348_gb300 import sem
    monkeypatch.setattr(sem, "_lib", None)
    monkeypatch.setattr(sem._build, "LIB", str(tmp_path / "libsem.so"))
    with pytest.raises(RuntimeError, match="CUDA extension is required"):
        sem.load(build_if_missing=False)


def test_package_never_imports_the_oracle():
    """The product package reaches no code under oracle/ (the oracle is test
    infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2608_24348_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                txt = open(os.path.join(dirpath, f), errors="replace").read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), f
                assert "sem_oracle" not in txt and "liboracle" not in txt, f
