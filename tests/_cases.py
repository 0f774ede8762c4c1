"""Shared seeded cases for the parity tests: a structure, its inputs and the oracle's
results (computed once per session)."""
from __future__ import annotations

import functools

import numpy as np

from paper_2501_08697_gb300 import synth as S


def rel_fro(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def block_class_errors(H, ref, keys, offs, norb_atom):
    """Per block shape (rows x cols): the relative Frobenius error over the blocks of that shape
    and the worst relative error of a single block among them (blocks whose reference norm is
    below 1e-12 of the largest block norm are left out of the worst-block figure)."""
    H = np.asarray(H, np.float64)
    ref = np.asarray(ref, np.float64)
    d2, r2, worst = {}, {}, {}
    norms = np.sqrt(np.add.reduceat(ref * ref, offs[:-1])) if len(keys) else np.zeros(0)
    dn = np.sqrt(np.add.reduceat((H - ref) ** 2, offs[:-1])) if len(keys) else np.zeros(0)
    big = norms.max() if len(norms) else 0.0
    for b in range(len(keys)):
        k = f"{norb_atom[keys[b, 0]]}x{norb_atom[keys[b, 1]]}"
        d2[k] = d2.get(k, 0.0) + dn[b] ** 2
        r2[k] = r2.get(k, 0.0) + norms[b] ** 2
        if norms[b] > 1e-12 * big:
            worst[k] = max(worst.get(k, 0.0), dn[b] / norms[b])
    return {k: (float(np.sqrt(d2[k] / r2[k])) if r2[k] > 0 else 0.0, worst.get(k, 0.0)) for k in sorted(d2)}


def structure(name):
    if name == "si8":
        return S.workload("si8")
    if name == "si8_ragged":      # grid not a multiple of the batch, displaced atoms
        return S.si_diamond((1, 1, 1), grid=(30, 34, 38), sigma=0.05, seed=S.BASE_SEED + 61, name="si8_ragged")
    if name == "si16_strained":   # orthorhombic 2x1x1 cell, strained, displaced
        return S.si_diamond((2, 1, 1), sigma=0.05, strain=0.021, seed=S.BASE_SEED + 62, name="si16_strained")
    if name == "water8":          # two species, mixed block shapes 13x13 / 13x5 / 5x5
        return S.water_box(8, (8 * 23.5 ** 3 / 64) ** (1 / 3), seed=S.BASE_SEED + 63, name="water8")
    if name == "water1_vacuum":   # one molecule in a large box: batches with no orbitals
        return S.water_box(1, 16.0, grid=(64, 64, 72), seed=S.BASE_SEED + 64, name="water1_vacuum")
    if name == "si8_2d":          # 18 orbitals per atom (2s2p2d): slots wider than 17 orbitals
        st = S.si_diamond((1, 1, 1), grid=(36, 36, 40), sigma=0.05, seed=S.BASE_SEED + 65, name="si8_2d")
        spec = S.SpeciesSpec("Si", 7.0, [(0, 0.3), (0, 0.8), (1, 0.3), (1, 0.8), (2, 0.5), (2, 1.1)])
        st.tables = [S.species_tables(spec)]
        return st
    if name == "h64_dense":       # 64 one-orbital atoms 3 bohr apart: 40-60 atom images per batch
        spec = S.SpeciesSpec("H", 6.0, [(0, 0.5)])
        L = 12.0
        g = np.arange(4) * 3.0 + 0.7
        tau = np.array([(x, y, z) for x in g for y in g for z in g], np.float64)
        tau = tau + 0.05 * S.normal(S.stream_key(S.BASE_SEED + 66, 11), tau.size).reshape(tau.shape)
        return S.Structure("h64_dense", np.diag([L, L, L]), tau, np.zeros(len(tau), np.int32),
                           [S.species_tables(spec)], (48, 48, 48), S.BASE_SEED + 66)
    if name == "si64":
        return S.workload("si64")
    if name == "water64":
        return S.workload("water64")
    if name == "si512":
        return S.workload("si512")
    raise KeyError(name)


@functools.lru_cache(maxsize=None)
def inputs(name):
    st = structure(name)
    V = S.local_potential(st)
    return st, V


@functools.lru_cache(maxsize=None)
def oracle_full(name):
    """Oracle keys/offsets, H, DM, rho, F for a case small enough to run in full."""
    from oracle import Oracle
    st, V = inputs(name)
    o = Oracle.from_structure(st)
    keys, offs = o.pairs()
    DM = S.density_matrix(keys, st.norb_atom, seed=st.seed)
    H = o.vlocal(V)
    rho = o.rho(DM)
    F = o.force(V, DM)
    return dict(st=st, V=V, keys=keys, offs=offs, DM=DM, H=H, rho=rho, F=F, oracle=o)


@functools.lru_cache(maxsize=None)
def oracle_strain(name):
    """Oracle dL/deps (3x3) for a case small enough to run in full."""
    ref = oracle_full(name)
    return ref["oracle"].dLdeps(ref["V"], ref["DM"])
