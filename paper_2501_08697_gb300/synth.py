"""Seeded synthetic inputs for the LCAO real-space grid integration.

Everything here is *input preparation*: crystal/molecular structures, tabulated radial
functions, the local potential V(r) on the grid and a density matrix rho_mu_nu(R) in the
block layout.  None of the grid-integration arithmetic (orbital evaluation, contraction,
scatter, density, force) lives in this module, so both the CUDA path and the CPU oracle can
draw identical inputs from it without sharing any of the method.

Random numbers come from one counter-based generator, splitmix64 (Steele, Lea, Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): output i of stream k is
mix(k + (i+1)*0x9E3779B97F4A7C15), where mix is the published 64-bit finaliser.

Workloads follow the paper's NAO description (Sec. IV.A-B: strictly localised radial
functions times spherical harmonics, uniform real-space grid), with the concrete sizes of
the five benchmark cases: Si diamond cells of 8/64/512 atoms, a 64-molecule water box and a
mixed set of 32 structures for batched launches.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 250108697


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(*parts: int) -> np.uint64:
    """Derive a 64-bit stream key from integers (seed, stream id, ...)."""
    k = np.uint64(0)
    with np.errstate(over="ignore"):
        for p in parts:
            k = _mix(np.uint64(k + GOLDEN + np.uint64(int(p) & 0xFFFFFFFFFFFFFFFF)))
    return np.uint64(k)


def splitmix_u64(key: np.uint64, n: int, start: int = 0) -> np.ndarray:
    i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(key) + i * GOLDEN)


def uniform(key: np.uint64, n: int, start: int = 0) -> np.ndarray:
    """n doubles in [0, 1) with 53 random bits each."""
    return (splitmix_u64(key, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(key: np.uint64, n: int) -> np.ndarray:
    """n standard normals by Box-Muller on pairs of uniforms."""
    m = (n + 1) // 2
    u = uniform(key, 2 * m)
    u1 = 1.0 - u[0::2]          # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([rad * np.cos(2 * np.pi * u2), rad * np.sin(2 * np.pi * u2)])
    return z[:n]


# --------------------------------------------------------------------------------------
# Species: radial functions f(r) = N r^l exp(-alpha r^2) (1-(r/rc)^2)^3 tabulated on r_i=i*dr
# --------------------------------------------------------------------------------------
@dataclass
class SpeciesSpec:
    name: str
    rcut: float
    radials: list            # [(l, alpha), ...]; orbitals per radial ordered m = 0,+1,-1,+2,-2
    dr: float = 0.01

    @property
    def norb(self) -> int:
        return sum(2 * l + 1 for l, _ in self.radials)

    @property
    def ntab(self) -> int:
        return int(round(self.rcut / self.dr)) + 1


SI = SpeciesSpec("Si", 7.0, [(0, 0.3), (0, 0.8), (1, 0.3), (1, 0.8), (2, 0.5)])
O = SpeciesSpec("O", 7.0, [(0, 0.4), (0, 1.0), (1, 0.4), (1, 1.0), (2, 0.7)])
H = SpeciesSpec("H", 6.0, [(0, 0.5), (0, 1.2), (1, 1.2)])
H_2S = SpeciesSpec("H", 6.0, [(0, 0.5), (0, 1.2)])


def _radial_shape(r, l, alpha, rc):
    x = np.clip(1.0 - (r / rc) ** 2, 0.0, None)
    return r ** l * np.exp(-alpha * r * r) * x ** 3


def radial_norm(l: int, alpha: float, rc: float, panels: int = 200000) -> float:
    """N with int_0^rc f(r)^2 r^2 dr = 1, by composite Simpson on `panels` panels."""
    r = np.linspace(0.0, rc, panels + 1)
    g = (_radial_shape(r, l, alpha, rc) * r) ** 2
    h = rc / panels
    s = g[0] + g[-1] + 4.0 * g[1:-1:2].sum() + 2.0 * g[2:-1:2].sum()
    return 1.0 / math.sqrt(s * h / 3.0)


@dataclass
class SpeciesTables:
    spec: SpeciesSpec
    l: np.ndarray            # [nrad] int32
    ftab: np.ndarray         # [nrad, ntab] float64
    dfdr0: np.ndarray        # [nrad] float64
    norm: np.ndarray         # [nrad]

    @property
    def rcut(self):
        return self.spec.rcut

    @property
    def dr(self):
        return self.spec.dr

    @property
    def ntab(self):
        return self.spec.ntab

    @property
    def norb(self):
        return self.spec.norb


def species_tables(spec: SpeciesSpec) -> SpeciesTables:
    r = np.arange(spec.ntab, dtype=np.float64) * spec.dr
    ls, tabs, d0, norms = [], [], [], []
    for l, a in spec.radials:
        nrm = radial_norm(l, a, spec.rcut)
        f = nrm * _radial_shape(r, l, a, spec.rcut)
        f[r >= spec.rcut] = 0.0
        ls.append(l)
        tabs.append(f)
        d0.append(nrm if l == 1 else 0.0)     # d/dr [N r^l ...] at r = 0
        norms.append(nrm)
    return SpeciesTables(spec, np.array(ls, np.int32), np.array(tabs), np.array(d0), np.array(norms))


def radial_analytic(spec: SpeciesSpec, irad: int, r):
    l, a = spec.radials[irad]
    return radial_norm(l, a, spec.rcut) * _radial_shape(np.asarray(r, float), l, a, spec.rcut)


# --------------------------------------------------------------------------------------
# Structures
# --------------------------------------------------------------------------------------
@dataclass
class Structure:
    name: str
    cell: np.ndarray         # [3,3] rows a1, a2, a3 (bohr)
    tau: np.ndarray          # [natoms, 3] Cartesian (bohr)
    species: np.ndarray      # [natoms] int32 index into `tables`
    tables: list             # [SpeciesTables]
    grid: tuple              # (N1, N2, N3)
    seed: int = BASE_SEED
    meta: dict = field(default_factory=dict)

    @property
    def natoms(self):
        return len(self.tau)

    @property
    def npts(self):
        return int(np.prod(self.grid))

    @property
    def norb_atom(self):
        return np.array([self.tables[s].norb for s in self.species], np.int64)

    @property
    def nbasis(self):
        return int(self.norb_atom.sum())

    @property
    def volume(self):
        return abs(float(np.linalg.det(self.cell)))

    @property
    def dV(self):
        return self.volume / self.npts


_DIAMOND = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                     [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25]])


def grid_for(L: float, h: float = 0.214) -> int:
    """Grid points per axis, a multiple of 4, spacing close to h."""
    return 4 * max(1, int(round(L / (4 * h))))


def si_diamond(rep=(1, 1, 1), a=10.26, grid=None, sigma=0.0, strain=0.0, seed=BASE_SEED,
               name=None) -> Structure:
    a_eff = a * (1.0 + strain)
    frac = []
    for i in range(rep[0]):
        for j in range(rep[1]):
            for k in range(rep[2]):
                frac.append((_DIAMOND + np.array([i, j, k])) / np.array(rep, float))
    frac = np.concatenate(frac)
    cell = np.diag([a_eff * rep[0], a_eff * rep[1], a_eff * rep[2]]).astype(np.float64)
    tau = frac @ cell
    if sigma > 0:
        tau = tau + sigma * normal(stream_key(seed, 11), tau.size).reshape(tau.shape)
    if grid is None:
        grid = tuple(grid_for(cell[i, i]) for i in range(3))
    return Structure(name or f"si{len(tau)}", cell, tau, np.zeros(len(tau), np.int32),
                     [species_tables(SI)], tuple(int(g) for g in grid), seed)


def _rot_from_quat(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def water_box(nmol=64, L=23.5, grid=None, min_oo=5.0, seed=BASE_SEED, h_basis="2s1p",
              name=None) -> Structure:
    """O positions with minimum periodic O-O distance min_oo: a jittered cubic lattice when its
    spacing allows (the 64-molecule box: 4x4x4 in 23.5 bohr), otherwise random sequential
    addition (bounded attempts).  H at 1.809 bohr, HOH angle 104.5 deg, orientation from a
    uniform random quaternion (Shoemake)."""
    n = int(math.ceil(nmol ** (1.0 / 3.0) - 1e-9))
    sp = L / n
    cell = np.diag([L, L, L]).astype(np.float64)

    def min_dist(pos):
        d = pos[:, None, :] - pos[None, :, :]
        d -= L * np.round(d / L)
        return (np.sqrt((d ** 2).sum(-1)) + np.eye(len(pos)) * 1e9).min()

    if sp >= min_oo:
        sites = np.array([[i, j, k] for i in range(n) for j in range(n) for k in range(n)], float)
        pick = np.argsort(uniform(stream_key(seed, 21), len(sites)), kind="stable")[:nmol]
        base = (sites[np.sort(pick)] + 0.5) * sp
        # per-coordinate jitter below (sp - min_oo)/(2 sqrt 3) keeps every distance >= min_oo
        jitter = min(0.4, 0.999 * (sp - min_oo) / (2 * math.sqrt(3)))
        u = uniform(stream_key(seed, 22), 3 * nmol).reshape(nmol, 3)
        opos = base + jitter * (2 * u - 1)
    else:
        opos = np.zeros((0, 3))
        key = stream_key(seed, 24)
        draw = 0
        while len(opos) < nmol:
            for _ in range(100000):
                cand = L * uniform(key, 3, start=draw)
                draw += 3
                if len(opos) == 0:
                    break
                d = opos - cand
                d -= L * np.round(d / L)
                if np.sqrt((d ** 2).sum(-1)).min() >= min_oo:
                    break
            else:
                raise ValueError(f"water_box: cannot place {nmol} molecules {min_oo} bohr apart in {L} bohr")
            opos = np.vstack([opos, cand])
    assert min_dist(opos) >= min_oo - 1e-9
    roh, ang = 1.809, math.radians(104.5)
    h1 = roh * np.array([math.sin(ang / 2), 0.0, math.cos(ang / 2)])
    h2 = roh * np.array([-math.sin(ang / 2), 0.0, math.cos(ang / 2)])
    uq = uniform(stream_key(seed, 23), 3 * nmol).reshape(nmol, 3)
    tau, spc = [], []
    for m in range(nmol):
        u1, u2, u3 = uq[m]
        q = (math.sqrt(1 - u1) * math.sin(2 * math.pi * u2), math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
             math.sqrt(u1) * math.sin(2 * math.pi * u3), math.sqrt(u1) * math.cos(2 * math.pi * u3))
        R = _rot_from_quat(q)
        tau += [opos[m], opos[m] + R @ h1, opos[m] + R @ h2]
        spc += [0, 1, 1]
    hspec = H if h_basis == "2s1p" else H_2S
    if grid is None:
        g = grid_for(L, 0.184)
        grid = (g, g, g)
    return Structure(name or f"water{nmol}", cell, np.array(tau), np.array(spc, np.int32),
                     [species_tables(O), species_tables(hspec)], tuple(int(x) for x in grid), seed)


# --------------------------------------------------------------------------------------
# Local potential V(r) = -1 + sum_k 0.5 cos(G_k . r + theta_k) on the grid
# --------------------------------------------------------------------------------------
def plane_wave_set(cell, nwaves=20, seed=BASE_SEED, gmax_cycles=3.0):
    """Integer vectors n (G = 2 pi B n, B reciprocal rows) with |G| <= gmax_cycles*2pi/L,
    L = volume^(1/3); +n and -n count as one wave.  Drawn without replacement."""
    cell = np.asarray(cell, float)
    L = abs(np.linalg.det(cell)) ** (1.0 / 3.0)
    B = np.linalg.inv(cell).T                  # rows b_i with a_i . b_j = delta_ij
    nmax = int(math.ceil(gmax_cycles * np.linalg.norm(cell, axis=1).max() / L)) + 1
    cand = []
    rng = range(-nmax, nmax + 1)
    for i in rng:
        for j in rng:
            for k in rng:
                n = (i, j, k)
                if n == (0, 0, 0):
                    continue
                if n < (0, 0, 0):                            # keep one of +-n
                    continue
                G = 2 * math.pi * (np.array(n) @ B)
                if np.linalg.norm(G) <= gmax_cycles * 2 * math.pi / L + 1e-12:
                    cand.append(n)
    cand = np.array(sorted(cand))
    order = np.argsort(uniform(stream_key(seed, 31), len(cand)), kind="stable")[:nwaves]
    ns = cand[np.sort(order)]
    theta = 2 * math.pi * uniform(stream_key(seed, 32), len(ns))
    return ns, theta


def local_potential(st: Structure, nwaves=20, amp=0.5, v0=-1.0, seed=None) -> np.ndarray:
    """V on the grid, shape (N1, N2, N3), k fastest.  Each wave is exactly periodic on the
    grid because G . r_ijk = 2 pi (n1 i/N1 + n2 j/N2 + n3 k/N3)."""
    seed = st.seed if seed is None else seed
    ns, theta = plane_wave_set(st.cell, nwaves, seed)
    N1, N2, N3 = st.grid
    V = np.full((N1, N2, N3), v0, dtype=np.float64)
    i = np.arange(N1) / N1
    j = np.arange(N2) / N2
    k = np.arange(N3) / N3
    for n, th in zip(ns, theta):
        ei = np.exp(2j * np.pi * n[0] * i) * np.exp(1j * th)
        ej = np.exp(2j * np.pi * n[1] * j)
        ek = np.exp(2j * np.pi * n[2] * k)
        V += amp * np.real(ei[:, None, None] * ej[None, :, None] * ek[None, None, :])
    return V


# --------------------------------------------------------------------------------------
# Density matrix rho_mu_nu(R): U[-0.1, 0.1], symmetric in the block sense
# --------------------------------------------------------------------------------------
def partner_index(keys: np.ndarray) -> np.ndarray:
    """For block keys (I, J, R1, R2, R3) return the index of (J, I, -R)."""
    keys = np.asarray(keys, np.int64)
    d = {tuple(k): i for i, k in enumerate(keys.tolist())}
    out = np.empty(len(keys), np.int64)
    for i, (I, J, a, b, c) in enumerate(keys.tolist()):
        out[i] = d[(J, I, -a, -b, -c)]
    return out


def density_matrix(keys, norb_atom, seed=BASE_SEED, scale=0.1) -> np.ndarray:
    """Block-store values for the given keys (row-major n_I x n_J per block, blocks in key
    order).  The canonical member of {(I,J,R), (J,I,-R)} (lexicographically smaller key)
    draws its elements; the partner holds the transpose.  A self-partner block (I,I,0) is
    symmetric.  Element (mu, nu) of canonical block (I,J,R) is a function of the key and
    (mu, nu) only, so any key order gives the same values."""
    keys = np.asarray(keys, np.int64)
    norb_atom = np.asarray(norb_atom, np.int64)
    part = partner_index(keys)
    nI = norb_atom[keys[:, 0]]
    nJ = norb_atom[keys[:, 1]]
    offs = np.zeros(len(keys) + 1, np.int64)
    offs[1:] = np.cumsum(nI * nJ)
    out = np.empty(offs[-1], np.float64)
    base = stream_key(seed, 41)
    for b in range(len(keys)):
        p = part[b]
        I, J, r1, r2, r3 = keys[b].tolist()
        canon = tuple(keys[b].tolist()) <= tuple(keys[p].tolist())
        ck = keys[b] if canon else keys[p]
        cI, cJ = int(ck[0]), int(ck[1])
        code = (((int(ck[2]) + 64) * 128 + (int(ck[3]) + 64)) * 128 + (int(ck[4]) + 64))
        k = stream_key(int(base), cI, cJ, code)
        n1, n2 = int(norb_atom[cI]), int(norb_atom[cJ])
        mu = np.arange(n1)[:, None]
        nu = np.arange(n2)[None, :]
        idx = (mu * 64 + nu).astype(np.uint64)
        with np.errstate(over="ignore"):
            u = (_mix(np.uint64(k) + (idx + np.uint64(1)) * GOLDEN) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        blk = scale * (2.0 * u - 1.0)
        if cI == cJ and int(ck[2]) == 0 and int(ck[3]) == 0 and int(ck[4]) == 0:
            blk = np.triu(blk) + np.triu(blk, 1).T
        if not canon:
            blk = blk.T
        out[offs[b]:offs[b + 1]] = blk.reshape(-1)
    return out


# --------------------------------------------------------------------------------------
# The five benchmark workloads
# --------------------------------------------------------------------------------------
def workload(name: str) -> Structure:
    if name == "si8":            # plain FP64 gamma-only case
        return si_diamond((1, 1, 1), grid=(48, 48, 48), seed=BASE_SEED + 1, name="si8")
    if name == "si64":           # differentiation case
        return si_diamond((2, 2, 2), grid=(96, 96, 96), sigma=0.05, seed=BASE_SEED + 2, name="si64")
    if name == "si512":          # precision case
        return si_diamond((4, 4, 4), grid=(192, 192, 192), seed=BASE_SEED + 3, name="si512")
    if name == "water64":        # water-like box
        return water_box(64, 23.5, grid=(128, 128, 128), seed=BASE_SEED + 4, name="water64")
    raise KeyError(name)


def batching_set(seed=BASE_SEED + 5):
    """32 structures of uneven size: Si 8/16/64/216 atoms x 4 isotropic strains in
    [-3%, +3%] (sigma 0.05 bohr displacements), and water boxes of 8..32 molecules."""
    out = []
    eps = 0.03 * (2 * uniform(stream_key(seed, 51), 16) - 1)
    reps = [(1, 1, 1), (2, 1, 1), (2, 2, 2), (3, 3, 3)]
    for a, rep in enumerate(reps):
        for s in range(4):
            e = float(eps[4 * a + s])
            st = si_diamond(rep, sigma=0.05, strain=e, seed=seed + 100 + 4 * a + s,
                            name=f"si{8 * int(np.prod(rep))}_s{s}")
            out.append(st)
    for k in range(16):
        n = 8 + int(round(24 * k / 15))
        L = (n * 23.5 ** 3 / 64) ** (1.0 / 3.0)
        out.append(water_box(n, L, seed=seed + 200 + k, name=f"water{n}"))
    return out
