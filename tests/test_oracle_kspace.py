"""Pins of the k-space oracle (folding of Sec. IV.B and the R-resolved density matrix of Eq.
density_matrix) against closed forms and exact identities."""
import numpy as np
import pytest

from oracle.kspace import fold, monkhorst_pack, orbital_offsets, unfold
from paper_2501_08697_gb300 import synth as S


def _cubic_tight_binding(e0, t):
    """One s orbital per simple-cubic cell: on-site e0, nearest-neighbour hopping t."""
    keys = np.array([[0, 0, 0, 0, 0], [0, 0, -1, 0, 0], [0, 0, 1, 0, 0], [0, 0, 0, -1, 0], [0, 0, 0, 1, 0],
                     [0, 0, 0, 0, -1], [0, 0, 0, 0, 1]], np.int32)
    keys = keys[np.lexsort(keys.T[::-1])]
    X = np.array([e0 if (k[2:] == 0).all() else t for k in keys])
    return keys, np.arange(len(keys) + 1, dtype=np.int64), np.array([1]), X


def test_fold_gives_the_tight_binding_dispersion():
    """E(k) = e0 + 2t (cos 2pi k1 + cos 2pi k2 + cos 2pi k3), the textbook band of the simple
    cubic s band."""
    keys, offs, norb, X = _cubic_tight_binding(-0.3, 0.17)
    rng = np.random.default_rng(7)
    kap = rng.uniform(-0.5, 0.5, (9, 3))
    Hk = fold(keys, offs, norb, X, kap)
    ref = -0.3 + 2 * 0.17 * np.cos(2 * np.pi * kap).sum(axis=1)
    assert np.allclose(Hk[:, 0, 0], ref, rtol=0, atol=1e-14)


@pytest.fixture(scope="module")
def si8_blocks():
    from oracle import Oracle
    st = S.si_diamond((1, 1, 1), grid=(16, 16, 16), sigma=0.05, seed=S.BASE_SEED + 93)
    o = Oracle.from_structure(st)
    keys, offs = o.pairs()
    DM = S.density_matrix(keys, st.norb_atom, seed=st.seed)   # block-symmetric: X(J,I,-R) = X(I,J,R)^T
    return st, keys, offs, DM


def test_folded_block_symmetric_store_is_hermitian_and_periodic(si8_blocks):
    st, keys, offs, X = si8_blocks
    kap = np.array([[0.1, -0.23, 0.37], [0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    Hk = fold(keys, offs, st.norb_atom, X, kap)
    for q in range(len(kap)):
        assert np.abs(Hk[q] - Hk[q].conj().T).max() < 1e-14
    assert np.abs(Hk[1].imag).max() == 0.0                      # Gamma: real, = Sum_R X(R)
    o = orbital_offsets(st.norb_atom)
    I, J = 0, 3
    sel = (keys[:, 0] == I) & (keys[:, 1] == J)
    direct = sum(X[offs[b]:offs[b + 1]].reshape(13, 13) for b in np.nonzero(sel)[0])
    assert np.allclose(Hk[1, o[I]:o[I + 1], o[J]:o[J + 1]].real, direct, rtol=0, atol=1e-15)
    # a reciprocal lattice vector changes nothing
    Hk2 = fold(keys, offs, st.norb_atom, X, kap + np.array([1, -2, 3]))
    assert np.abs(Hk2 - Hk).max() < 1e-12


def test_unfold_inverts_fold_on_a_complete_mesh(si8_blocks):
    """Discrete Fourier orthogonality: with an n^3 mesh wider than the range of R (|n_i| < n/2)
    and weights 1/N_k, unfolding the folded store returns it exactly."""
    st, keys, offs, X = si8_blocks
    nmax = int(np.abs(keys[:, 2:]).max())
    n = 2 * nmax + 1
    kap, w = monkhorst_pack(n, n, n)
    Xk = fold(keys, offs, st.norb_atom, X, kap)
    back = unfold(keys, offs, st.norb_atom, Xk, kap, w)
    assert np.abs(back - X).max() < 1e-13
    # a shifted mesh is complete too
    kap2, w2 = monkhorst_pack(n, n, n, shift=(0.5, 0.25, 0.0))
    back2 = unfold(keys, offs, st.norb_atom, fold(keys, offs, st.norb_atom, X, kap2), kap2, w2)
    assert np.abs(back2 - X).max() < 1e-13


def test_density_matrix_from_eigenvectors_matches_bloch_sum():
    """Eq. density_matrix for the tight-binding band: one orbital, f = 1 below the Fermi level,
    rho(R) = (1/N_k) Sum_k f(k) exp(-i k.R), checked against the explicit Bloch sum."""
    keys, offs, norb, _ = _cubic_tight_binding(0.0, -1.0)
    kap, w = monkhorst_pack(6, 6, 6, shift=(0.5, 0.5, 0.5))
    E = -2 * np.cos(2 * np.pi * kap).sum(axis=1)
    f = (E < 0.3).astype(float)
    Xk = f.reshape(-1, 1, 1).astype(np.complex128)              # c = 1: X(k) = f(k)
    rho = unfold(keys, offs, norb, Xk, kap, w)
    for b, k in enumerate(keys):
        ref = np.sum(w * f * np.cos(2 * np.pi * kap @ k[2:]))
        assert rho[b] == pytest.approx(ref, abs=1e-13)
    assert rho[list(map(tuple, keys[:, 2:])).index((0, 0, 0))] == pytest.approx(f.mean())


def test_density_matrix_of_a_complete_unitary_basis_is_the_identity(si8_blocks):
    """All bands occupied with unitary C(k): rho(k) = 1, so on a complete k mesh rho(R) is the
    identity on the on-site blocks (R = 0) and zero on every other block."""
    from oracle.kspace import density_matrix
    st, keys, offs, _ = si8_blocks
    nmax = int(np.abs(keys[:, 2:]).max())
    n = 2 * nmax + 1
    kap, w = monkhorst_pack(n, n, n)
    N = int(st.norb_atom.sum())
    rng = np.random.default_rng(5)
    C = np.stack([np.linalg.qr(rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N)))[0] for _ in kap])
    rho = density_matrix(keys, offs, st.norb_atom, C, np.ones((len(kap), N)), kap, w)
    for b, k in enumerate(keys):
        blk = rho[offs[b]:offs[b + 1]].reshape(13, 13)
        ref = np.eye(13) if (k[0] == k[1] and (k[2:] == 0).all()) else np.zeros((13, 13))
        assert np.abs(blk - ref).max() < 1e-12


def test_density_matrix_is_block_symmetric_and_counts_electrons(si8_blocks):
    from oracle.kspace import density_matrix
    st, keys, offs, _ = si8_blocks
    kap, w = monkhorst_pack(2, 2, 2, shift=(0.25, 0.25, 0.25))
    kap = np.vstack([kap, -kap])            # closed under k -> -k
    w = np.full(len(kap), 1.0 / len(kap))
    N = int(st.norb_atom.sum())
    rng = np.random.default_rng(6)
    C = rng.normal(size=(len(kap), N, 40)) + 1j * rng.normal(size=(len(kap), N, 40))
    C /= np.linalg.norm(C, axis=1, keepdims=True)                    # unit-norm bands
    f = rng.uniform(0, 2, (len(kap), 40))
    rho = density_matrix(keys, offs, st.norb_atom, C, f, kap, w)
    part = S.partner_index(keys)
    for b in range(len(keys)):
        A = rho[offs[b]:offs[b + 1]].reshape(13, 13)
        B = rho[offs[part[b]]:offs[part[b] + 1]].reshape(13, 13)
        assert np.abs(A - B.T).max() < 1e-14
    # trace of the R = 0 on-site blocks = Sum_k w_k Sum_n f_nk
    tr = sum(np.trace(rho[offs[b]:offs[b + 1]].reshape(13, 13)) for b, k in enumerate(keys)
             if k[0] == k[1] and (k[2:] == 0).all())
    assert tr == pytest.approx((w[:, None] * f).sum(), rel=1e-12)
