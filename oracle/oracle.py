"""ctypes wrapper around gint_oracle.c (plain FP64 reference; test infrastructure only).

Functions follow the definitions cited in gint_oracle.c: V_mu,nu(R) by grid quadrature of
the two-centre template with a local operator (Sec. IV.B), rho(r) from rho_mu,nu(R)
(Eq. density_matrix), and the basis-motion (Pulay) derivative of Eq. force_lcao (Sec. IV.D).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gint_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libgint_oracle.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over grid points)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build_oracle())
            P = C.POINTER
            d, i, i64 = C.c_double, C.c_int, C.c_int64
            lib.oracle_new.restype = C.c_void_p
            lib.oracle_new.argtypes = [P(d), i, P(i), P(d), i, P(i), P(d), P(d), P(i), P(i), P(d), P(d), P(i)]
            lib.oracle_free.argtypes = [C.c_void_p]
            lib.oracle_dV.restype = d
            lib.oracle_dV.argtypes = [C.c_void_p]
            lib.oracle_norb.argtypes = [C.c_void_p, i]
            lib.oracle_radial.restype = d
            lib.oracle_radial.argtypes = [C.c_void_p, i, i, d, P(d)]
            lib.oracle_phi.argtypes = [C.c_void_p, i, P(d), P(d), P(d)]
            lib.oracle_pairs.restype = i64
            lib.oracle_pairs.argtypes = [C.c_void_p, i64, P(i)]
            lib.oracle_vlocal.argtypes = [C.c_void_p, P(d), i64, P(i), P(i64), P(d), i64, P(i64)]
            lib.oracle_rho.argtypes = [C.c_void_p, i64, P(i), P(i64), P(d), P(d), i64, P(i64)]
            lib.oracle_dLdtau.argtypes = [C.c_void_p, P(d), i64, P(i), P(i64), P(d), P(d), i64, P(i64)]
            lib.oracle_dLdeps.argtypes = [C.c_void_p, P(d), i64, P(i), P(i64), P(d), P(d), i64, P(i64)]
            lib.oracle_vlocal_blocks.argtypes = [C.c_void_p, P(d), i64, P(i), P(i64), P(d)]
            lib.oracle_dLdtau_atoms.argtypes = [C.c_void_p, P(d), i64, P(i), P(i64), P(d), i64, P(i), P(d)]
            lib.oracle_points_near_atom.restype = i64
            lib.oracle_points_near_atom.argtypes = [C.c_void_p, i, i64, P(i64)]
            lib.oracle_threads.restype = i
            _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class Oracle:
    """Oracle context for one structure (cell, atoms, species tables, grid)."""

    def __init__(self, cell, species, tau, tables, grid):
        lib = _load()
        self._lib = lib
        self.cell = np.ascontiguousarray(cell, np.float64).reshape(3, 3)
        self.species = np.ascontiguousarray(species, np.int32)
        self.tau = np.ascontiguousarray(tau, np.float64).reshape(-1, 3)
        self.grid = np.ascontiguousarray(grid, np.int32)
        self.tables = tables
        nrad = np.array([len(t.l) for t in tables], np.int32)
        rcut = np.array([t.rcut for t in tables], np.float64)
        dr = np.array([t.dr for t in tables], np.float64)
        ntab = np.array([t.ftab.shape[1] for t in tables], np.int32)
        rad_l = np.ascontiguousarray(np.concatenate([t.l for t in tables]).astype(np.int32))
        d0 = np.ascontiguousarray(np.concatenate([t.dfdr0 for t in tables]).astype(np.float64))
        ftab = np.ascontiguousarray(np.concatenate([t.ftab.reshape(-1) for t in tables]).astype(np.float64))
        self._keep = (nrad, rcut, dr, ntab, rad_l, d0, ftab)
        self.ctx = lib.oracle_new(_p(self.cell, C.c_double), len(self.tau), _p(self.species, C.c_int),
                                  _p(self.tau, C.c_double), len(tables), _p(nrad, C.c_int),
                                  _p(rcut, C.c_double), _p(dr, C.c_double), _p(ntab, C.c_int),
                                  _p(rad_l, C.c_int), _p(d0, C.c_double), _p(ftab, C.c_double),
                                  _p(self.grid, C.c_int))
        self.natoms = len(self.tau)
        self.norb_atom = np.array([lib.oracle_norb(self.ctx, a) for a in range(self.natoms)], np.int64)
        self.dV = lib.oracle_dV(self.ctx)
        self._keys = None

    @classmethod
    def from_structure(cls, st, tau=None):
        return cls(st.cell, st.species, st.tau if tau is None else tau, st.tables, st.grid)

    def __del__(self):
        if getattr(self, "ctx", None):
            self._lib.oracle_free(self.ctx)
            self.ctx = None

    @staticmethod
    def threads() -> int:
        return _load().oracle_threads()

    # ---- pins
    def radial(self, species, irad, r):
        d = C.c_double()
        v = self._lib.oracle_radial(self.ctx, species, irad, float(r), C.byref(d))
        return v, d.value

    def phi(self, species, d, grad=False):
        d = np.ascontiguousarray(d, np.float64)
        phi = np.zeros(64)
        g = np.zeros(64 * 3)
        n = self._lib.oracle_phi(self.ctx, species, _p(d, C.c_double), _p(phi, C.c_double),
                                 _p(g, C.c_double) if grad else None)
        return (phi[:n], g[:3 * n].reshape(n, 3)) if grad else phi[:n]

    # ---- layout
    def pairs(self):
        if self._keys is None:
            n = self._lib.oracle_pairs(self.ctx, 0, None)
            keys = np.zeros((n, 5), np.int32)
            self._lib.oracle_pairs(self.ctx, n, _p(keys, C.c_int))
            nI = self.norb_atom[keys[:, 0]]
            nJ = self.norb_atom[keys[:, 1]]
            offs = np.zeros(n + 1, np.int64)
            offs[1:] = np.cumsum(nI * nJ)
            self._keys, self._offs = keys, offs
        return self._keys, self._offs

    # ---- the method
    def _pts(self, pts):
        if pts is None:
            return 0, None, None
        pts = np.ascontiguousarray(pts, np.int64)
        return len(pts), pts, _p(pts, C.c_int64)

    def vlocal(self, V, pts=None):
        keys, offs = self.pairs()
        V = np.ascontiguousarray(V, np.float64).reshape(-1)
        H = np.zeros(offs[-1], np.float64)
        n, keep, pp = self._pts(pts)
        rc = self._lib.oracle_vlocal(self.ctx, _p(V, C.c_double), len(keys), _p(keys, C.c_int),
                                     _p(offs, C.c_int64), _p(H, C.c_double), n, pp)
        if rc != 0:
            raise RuntimeError(f"oracle_vlocal failed ({rc})")
        return H

    def rho(self, DM, pts=None):
        keys, offs = self.pairs()
        DM = np.ascontiguousarray(DM, np.float64)
        n, keep, pp = self._pts(pts)
        out = np.zeros(n if pts is not None else int(np.prod(self.grid)), np.float64)
        rc = self._lib.oracle_rho(self.ctx, len(keys), _p(keys, C.c_int), _p(offs, C.c_int64),
                                  _p(DM, C.c_double), _p(out, C.c_double), n, pp)
        if rc != 0:
            raise RuntimeError(f"oracle_rho failed ({rc})")
        return out

    def dLdtau(self, V, DM, pts=None):
        keys, offs = self.pairs()
        V = np.ascontiguousarray(V, np.float64).reshape(-1)
        DM = np.ascontiguousarray(DM, np.float64)
        out = np.zeros((self.natoms, 3), np.float64)
        n, keep, pp = self._pts(pts)
        rc = self._lib.oracle_dLdtau(self.ctx, _p(V, C.c_double), len(keys), _p(keys, C.c_int),
                                     _p(offs, C.c_int64), _p(DM, C.c_double), _p(out, C.c_double), n, pp)
        if rc != 0:
            raise RuntimeError(f"oracle_dLdtau failed ({rc})")
        return out

    def force(self, V, DM, pts=None):
        return -self.dLdtau(V, DM, pts)

    def dLdeps(self, V, DM, pts=None):
        """dL/deps_ab (3x3) under a homogeneous strain of cell, atoms and grid with the grid
        values of V held fixed; the stress of Eq. (stress) is -dL/deps / Omega."""
        keys, offs = self.pairs()
        V = np.ascontiguousarray(V, np.float64).reshape(-1)
        DM = np.ascontiguousarray(DM, np.float64)
        out = np.zeros(9, np.float64)
        n, keep, pp = self._pts(pts)
        rc = self._lib.oracle_dLdeps(self.ctx, _p(V, C.c_double), len(keys), _p(keys, C.c_int),
                                     _p(offs, C.c_int64), _p(DM, C.c_double), _p(out, C.c_double), n, pp)
        if rc != 0:
            raise RuntimeError(f"oracle_dLdeps failed ({rc})")
        return out.reshape(3, 3)

    def vlocal_blocks(self, V, sel):
        """The blocks sel (indices into the sorted block list) of V_mu,nu(R), each summed over
        the grid points of all space in the first atom's sphere; returns them concatenated in
        the order of sel (sorted by first atom internally so blocks of one atom share a pass)."""
        keys, offs = self.pairs()
        V = np.ascontiguousarray(V, np.float64).reshape(-1)
        sel = np.asarray(sel, np.int64)
        order = np.argsort(keys[sel, 0], kind="stable")
        s2 = sel[order]
        k2 = np.ascontiguousarray(keys[s2], np.int32)
        sizes = self.norb_atom[k2[:, 0]] * self.norb_atom[k2[:, 1]]
        o2 = np.zeros(len(s2) + 1, np.int64)
        o2[1:] = np.cumsum(sizes)
        out = np.zeros(o2[-1], np.float64)
        self._lib.oracle_vlocal_blocks(self.ctx, _p(V, C.c_double), len(s2), _p(k2, C.c_int), _p(o2, C.c_int64),
                                       _p(out, C.c_double))
        # back to the order of sel
        parts = {int(b): out[o2[i]:o2[i + 1]] for i, b in enumerate(s2)}
        return np.concatenate([parts[int(b)] for b in sel]) if len(sel) else out

    def dLdtau_atoms(self, V, DM, atoms):
        """dL/dtau for the listed atoms (len(atoms) x 3), each summed over its own sphere."""
        keys, offs = self.pairs()
        V = np.ascontiguousarray(V, np.float64).reshape(-1)
        DM = np.ascontiguousarray(DM, np.float64)
        atoms = np.ascontiguousarray(atoms, np.int32)
        out = np.zeros((len(atoms), 3), np.float64)
        rc = self._lib.oracle_dLdtau_atoms(self.ctx, _p(V, C.c_double), len(keys), _p(keys, C.c_int),
                                           _p(offs, C.c_int64), _p(DM, C.c_double), len(atoms),
                                           _p(atoms, C.c_int), _p(out, C.c_double))
        if rc != 0:
            raise RuntimeError(f"oracle_dLdtau_atoms failed ({rc})")
        return out

    def points_near_atom(self, I):
        n = self._lib.oracle_points_near_atom(self.ctx, I, 0, None)
        out = np.zeros(n, np.int64)
        self._lib.oracle_points_near_atom(self.ctx, I, n, _p(out, C.c_int64))
        return out
