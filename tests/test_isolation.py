"""The oracle and the CUDA path share no code, and the product path never
reaches the oracle: only the tests, the smoke check and the bench's CPU
baseline / reference arm (in a child process) import it."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
IMPORT = re.compile(r"^\s*(?:from|import)\s+([A-Za-z_][A-Za-z_0-9.]*)", re.M)


def imports_of(path):
    with open(path) as fh:
        return [m.group(1) for m in IMPORT.finditer(fh.read())]


def test_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2401_09721_gb300")
    for name in sorted(os.listdir(pkg)):
        if name.endswith(".py"):
            mods = imports_of(os.path.join(pkg, name))
            assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), name


def test_cuda_sources_name_no_oracle_file():
    csrc = os.path.join(ROOT, "paper_2401_09721_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name)) as fh:
            text = fh.read()
        assert "fgbd_oracle" not in text and "oracle/" not in text, name


def test_oracle_imports_nothing_of_the_package():
    mods = imports_of(os.path.join(ROOT, "oracle", "fgbd_oracle.py"))
    assert not any(m.startswith("paper_2401_09721_gb300") for m in mods), mods
    assert set(mods) <= {"__future__", "dataclasses", "numpy", "scipy.sparse", "math"}, mods


def test_bench_reaches_the_oracle_only_in_its_child_process():
    with open(os.path.join(ROOT, "bench.py")) as fh:
        text = fh.read()
    # the single import sits in the function the child process runs
    hits = [m.start() for m in re.finditer(r"from oracle import", text)]
    assert len(hits) == 1
    child = text.index("def _oracle_child(")
    nxt = text.index("\ndef ", child + 1)
    assert child < hits[0] < nxt
