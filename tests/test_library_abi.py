"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/gint.h declares (CPU only: no compute call is made)."""
import os
import re
import subprocess

import pytest

from paper_2501_08697_gb300 import build as B
from paper_2501_08697_gb300 import gint as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gint.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gint_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    return B.build_library()


def test_header_and_binding_agree():
    assert sorted(G.EXPORTS) == _declared()


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gint_[a-z_]+)\b", out))
    missing = [s for s in _declared() if s not in exported]
    assert not missing, missing


def test_library_targets_sm103a_only(lib_path):
    out = subprocess.run(["cuobjdump", "--list-elf", lib_path], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    archs = set(re.findall(r"sm_(\d+a?)", out.stdout))
    assert archs == {"103a"}, archs


def test_loads_with_ctypes(lib_path):
    lib = G.load()
    for name in G.EXPORTS:
        assert hasattr(lib, name)
    assert lib.gint_last_error() is not None


def _param_counts():
    src = open(os.path.join(ROOT, "include", "gint.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(gint_[a-z_]+)\s*\(([^()]*)\)\s*;", src):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_every_binding_declares_its_argument_types(lib_path):
    """ctypes passes undeclared arguments as C int: a 64-bit device pointer would be cut to 32
    bits.  Every entry point therefore has argtypes, as many as the header declares."""
    lib = G.load()
    counts = _param_counts()
    for name in G.EXPORTS:
        fn = getattr(lib, name)
        if counts.get(name, 0) == 0:
            continue
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == counts[name], (name, len(fn.argtypes), counts[name])


def test_setup_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2501_08697_gb300 import synth as S
    st = S.si_diamond((1, 1, 1), grid=(16, 16, 16))
    with pytest.raises(G.GintError) as e:
        G.setup_structure(st)
    assert e.value.code == G.GINT_ECUDA


@pytest.mark.parametrize("case", ["no_atoms", "grid_zero", "singular_cell", "bad_species", "nan_position",
                                  "bad_batch"])
def test_setup_rejects_invalid_input_on_host(case):
    """gint_setup checks its arguments on the host before it touches a device, so an invalid
    structure is GINT_EINVAL (with a message), GPU or not."""
    import numpy as np
    from paper_2501_08697_gb300 import synth as S
    st = S.si_diamond((1, 1, 1), grid=(16, 16, 16))
    cell, species, tau, grid = st.cell.copy(), st.species.copy(), st.tau.copy(), list(st.grid)
    kw = {}
    if case == "no_atoms":
        species, tau = species[:0], tau[:0]
    elif case == "grid_zero":
        grid[1] = 0
    elif case == "singular_cell":
        cell[2] = cell[0]
    elif case == "bad_species":
        species[3] = 5
    elif case == "nan_position":
        tau[2, 1] = np.nan
    elif case == "bad_batch":
        kw = dict(batch=(4, 4, 3))          # odd along a3
    with pytest.raises(G.GintError) as e:
        G.gint_setup(cell, species, tau, st.tables, grid, **kw)
    assert e.value.code == G.GINT_EINVAL
    assert G.load().gint_last_error()


def test_empty_and_null_calls_on_host():
    """An empty multi-structure call is a no-op; a call without a handle is rejected."""
    lib = G.load()
    assert lib.gint_batched(0, None, None, None, None, None, 0, None) == G.GINT_OK
    assert lib.gint_vlocal(None, None, None, 0, None) == G.GINT_EINVAL
    assert lib.gint_rho(None, None, None, 0, None) == G.GINT_EINVAL
    assert lib.gint_get_status(None) == G.GINT_EINVAL
