"""The C-ABI library loads and exports every entry point declared in include/qsim.h
(no compute call: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "qsim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z][a-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_hot_path_entry_points():
    names = declared_functions()
    for n in ("qsim_create", "qsim_step", "qsim_rollout", "ac_update", "ac_train",
              "qsim_dynamics_step", "qsim_rollout_vjp", "qsim_last_error"):
        assert n in names
    assert len(names) >= 30


def test_library_exports_every_declared_symbol():
    from paper_2311_13081_gb300 import build as b
    lib_path = b.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.qsim_abi_version() == 1
