"""Density matrix from eigenvectors (Eq. density_matrix) through the C ABI against the k-space
oracle (pinned in test_oracle_kspace).  FP64 on both sides: bound 1e-12 relative (max norm)."""
import numpy as np
import pytest

from oracle.kspace import density_matrix, monkhorst_pack

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_08697_gb300 import gint
    return gint


@pytest.mark.parametrize("name,nbands", [("si8", 20), ("water8", 37), ("si8_gamma", 16)])
def test_density_matrix_matches_oracle(G, name, nbands):
    from paper_2501_08697_gb300 import synth as S
    if name == "water8":
        st = S.water_box(8, (8 * 23.5 ** 3 / 64) ** (1 / 3), grid=(32, 32, 32), seed=S.BASE_SEED + 412)
    else:
        st = S.si_diamond((1, 1, 1), grid=(24, 24, 24), sigma=0.05, seed=S.BASE_SEED + 411)
    h = G.setup_structure(st)
    keys, offs = h.layout()
    N = h.info["nbasis"]
    if name == "si8_gamma":
        kap, w = np.zeros((1, 3)), np.ones(1)
    else:
        kap, w = monkhorst_pack(2, 2, 2, shift=(0.5, 0.5, 0.5))
        kap = np.vstack([kap, [0.1, -0.2, 0.3]])
        w = np.full(len(kap), 1.0 / len(kap))
    rng = np.random.default_rng(21)
    C = rng.normal(size=(len(kap), N, nbands)) + 1j * rng.normal(size=(len(kap), N, nbands))
    if name == "si8_gamma":
        C = C.real + 0j
    f = rng.uniform(0, 2, (len(kap), nbands))
    ref = density_matrix(keys, offs, st.norb_atom, C, f, kap, w)
    dev = torch.device("cuda")
    out = torch.full((len(ref),), float("nan"), dtype=torch.float64, device=dev)
    G.gint_density_matrix(h, kap, w, torch.from_numpy(C).to(dev), torch.from_numpy(f).to(dev), out, "fp64")
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_density_matrix_feeds_rho(G):
    """The produced DM drives gint_rho: the charge Sum rho dV equals <DM, S> computed two ways."""
    from paper_2501_08697_gb300 import synth as S
    st = S.si_diamond((1, 1, 1), grid=(24, 24, 24), sigma=0.05, seed=S.BASE_SEED + 413)
    h = G.setup_structure(st)
    N = h.info["nbasis"]
    dev = torch.device("cuda")
    rng = np.random.default_rng(22)
    C = torch.from_numpy(rng.normal(size=(1, N, 16)) + 0j).to(dev)
    f = torch.full((1, 16), 2.0, dtype=torch.float64, device=dev)
    DM = torch.empty(h.info["nvalues"], dtype=torch.float64, device=dev)
    G.gint_density_matrix(h, np.zeros((1, 3)), [1.0], C, f, DM, "fp64")
    rho = torch.empty(h.info["npts"], dtype=torch.float64, device=dev)
    G.gint_rho(h, DM, rho, "fp64")
    Sg = torch.empty_like(DM)
    G.gint_vlocal(h, torch.ones(h.info["npts"], dtype=torch.float64, device=dev), Sg, "fp64")
    torch.cuda.synchronize()
    assert float(rho.sum()) * h.info["dV"] == pytest.approx(float((DM * Sg).sum()), rel=1e-10)
