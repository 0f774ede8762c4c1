"""Density matrix from eigenvectors (Eq. density_matrix) through the C ABI against the k-space
oracle (pinned in test_oracle_kspace).  FP64: bound 1e-12 relative (max norm); TF32x3 (tensor
cores, 64-term K segments summed in FP32): 1e-6 relative Frobenius."""
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


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
@pytest.mark.parametrize("name,nbands", [("si8", 20), ("water8", 37), ("si8_gamma", 16), ("si8_many", 150)])
def test_density_matrix_matches_oracle(G, name, nbands, prec):
    from paper_2501_08697_gb300 import synth as S
    if name == "water8":
        st = S.water_box(8, (8 * 23.5 ** 3 / 64) ** (1 / 3), grid=(32, 32, 32), seed=S.BASE_SEED + 412)
    else:
        st = S.si_diamond((1, 1, 1), grid=(24, 24, 24), sigma=0.05, seed=S.BASE_SEED + 411)
    h = G.setup_structure(st)
    keys, offs = h.layout()
    N = h.info["nbasis"]
    if name in ("si8_gamma", "si8_many"):
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
    G.gint_density_matrix(h, kap, w, torch.from_numpy(C).to(dev), torch.from_numpy(f).to(dev), out, prec)
    torch.cuda.synchronize()
    assert G.gint_get_status(h) == 0
    got = out.cpu().numpy()
    if prec == "fp64":
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    else:
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        print(f"{name} tf32x3: DM {err:.2e}")
        assert err <= 1e-6


def test_density_matrix_long_band_sum(G):
    """Si64 Gamma with 512 bands: K = 1024 real terms, 16 TMEM segments per output tile, 7 x 7
    tiles of 128 (nbasis 832 is not a multiple of 128)."""
    from paper_2501_08697_gb300 import synth as S
    st = S.workload("si64")
    h = G.setup_structure(st)
    keys, offs = h.layout()
    N = h.info["nbasis"]
    rng = np.random.default_rng(23)
    C = (rng.normal(size=(1, N, 512)) + 1j * rng.normal(size=(1, N, 512))) / np.sqrt(N)
    f = rng.uniform(0, 2, (1, 512))
    kap, w = np.array([[0.25, 0.0, -0.125]]), np.ones(1)
    ref = density_matrix(keys, offs, st.norb_atom, C, f, kap, w)
    dev = torch.device("cuda")
    out = torch.empty(len(ref), dtype=torch.float64, device=dev)
    G.gint_density_matrix(h, kap, w, torch.from_numpy(C).to(dev), torch.from_numpy(f).to(dev), out, "tf32x3")
    torch.cuda.synchronize()
    assert G.gint_get_status(h) == 0
    err = float(np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref))
    print(f"si64 512 bands tf32x3: DM {err:.2e}")
    assert err <= 1e-6


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
