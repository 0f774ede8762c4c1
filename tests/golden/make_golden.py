"""Writes the oracle regression fixtures of tests/golden/ (run from the repository root:
python tests/golden/make_golden.py).  Every stored value comes from oracle/ on the seeded
inputs of tests/_cases.py; nothing here runs the CUDA library.

water1_vacuum.txt: one water molecule in a 16-bohr cubic box (64 x 64 x 72 grid), the plane-wave
V(r) and the seeded density matrix of the input generator:
  H      every value of V_mu,nu(R) (Sec. IV.B two-centre template with the local potential),
  rho    rho(r) at 64 seeded grid points (Eq. density_matrix and the sentence after it),
  F      the Pulay force of every atom (Eq. force_lcao, Sec. IV.D, V(r) held fixed),
  charge Sum_r rho(r) dV over the whole grid.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import Oracle                      # noqa: E402
from paper_2501_08697_gb300 import synth as S  # noqa: E402
from tests._cases import inputs                # noqa: E402

NAME = "water1_vacuum"


def golden_values():
    st, V = inputs(NAME)
    o = Oracle.from_structure(st)
    keys, offs = o.pairs()
    DM = S.density_matrix(keys, st.norb_atom, seed=st.seed)
    H = o.vlocal(V)
    rho = o.rho(DM)
    F = o.force(V, DM).reshape(-1)
    npts = int(np.prod(st.grid))
    pts = np.unique((S.uniform(S.stream_key(st.seed, 901), 64) * npts).astype(np.int64))
    dV = abs(np.linalg.det(st.cell)) / npts
    return {"H": H, "rho_pts": pts.astype(np.float64), "rho": rho[pts], "F": F,
            "charge": np.array([rho.sum() * dV])}


def write(path):
    vals = golden_values()
    with open(path, "w") as f:
        f.write(f"# oracle regression fixture: {NAME} (written by tests/golden/make_golden.py)\n")
        for k, v in vals.items():
            f.write(f"{k} {len(v)}\n")
            for x in v:
                f.write(f"{x:.17e}\n")


def read(path):
    out, lines = {}, [l for l in open(path) if not l.startswith("#")]
    i = 0
    while i < len(lines):
        k, n = lines[i].split()
        n = int(n)
        out[k] = np.array([float(x) for x in lines[i + 1:i + 1 + n]])
        i += 1 + n
    return out


if __name__ == "__main__":
    write(os.path.join(HERE, f"{NAME}.txt"))
