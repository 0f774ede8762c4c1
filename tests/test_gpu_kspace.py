"""k-space transforms through the C ABI (gint_fold / gint_unfold) against the k-space oracle,
whose pins are in test_oracle_kspace.  Pure FP64 on both sides: only the order of additions
differs, so the bound is 1e-13 relative (max norm)."""
import numpy as np
import pytest

from oracle.kspace import fold, monkhorst_pack, unfold

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_08697_gb300 import gint as G
    from paper_2501_08697_gb300 import synth as S
    out = {}
    for name, st in (("si8", S.si_diamond((1, 1, 1), grid=(24, 24, 24), sigma=0.05, seed=S.BASE_SEED + 401)),
                     ("water8", S.water_box(8, (8 * 23.5 ** 3 / 64) ** (1 / 3), grid=(32, 32, 32),
                                            seed=S.BASE_SEED + 402))):
        h = G.setup_structure(st)
        keys, offs = h.layout()
        X = S.density_matrix(keys, st.norb_atom, seed=st.seed)
        rng = np.random.default_rng(11)
        Xg = X * rng.uniform(0.5, 1.5, X.shape)     # also a store that is not block-symmetric
        out[name] = dict(st=st, h=h, keys=keys, offs=offs, X=X, Xg=Xg)
    return G, out


def _fold_gpu(G, c, X, kap):
    dev = torch.device("cuda")
    N = c["h"].info["nbasis"]
    Xk = torch.full((len(kap), N, N), complex("nan"), dtype=torch.complex128, device=dev)
    G.gint_fold(c["h"], torch.from_numpy(X).to(dev), kap, Xk)
    torch.cuda.synchronize()
    return Xk.cpu().numpy()


@pytest.mark.parametrize("name", ["si8", "water8"])
def test_fold_matches_oracle(case, name):
    G, cs = case
    c = cs[name]
    rng = np.random.default_rng(3)
    kap = np.vstack([[0, 0, 0], [0.5, 0, 0.5], rng.uniform(-0.5, 0.5, (5, 3))])
    assert c["h"].info["nbasis"] == int(c["st"].norb_atom.sum())
    for X in (c["X"], c["Xg"]):
        got = _fold_gpu(G, c, X, kap)
        ref = fold(c["keys"], c["offs"], c["st"].norb_atom, X, kap)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["si8", "water8"])
def test_unfold_matches_oracle_and_inverts_fold(case, name):
    G, cs = case
    c = cs[name]
    dev = torch.device("cuda")
    nmax = int(np.abs(c["keys"][:, 2:]).max())
    n = 2 * nmax + 1
    kap, w = monkhorst_pack(n, n, n, shift=(0.5, 0.0, 0.25))
    Xk = _fold_gpu(G, c, c["Xg"], kap)
    out = torch.full((len(c["Xg"]),), float("nan"), dtype=torch.float64, device=dev)
    G.gint_unfold(c["h"], torch.from_numpy(Xk).to(dev), kap, w, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = unfold(c["keys"], c["offs"], c["st"].norb_atom, Xk, kap, w)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(got - c["Xg"]).max() <= 1e-12 * np.abs(c["Xg"]).max()


def test_fold_rejects_bad_input(case):
    G, cs = case
    c = cs["si8"]
    dev = torch.device("cuda")
    N = c["h"].info["nbasis"]
    Xk = torch.empty((1, N, N), dtype=torch.complex128, device=dev)
    with pytest.raises(ValueError):
        G.gint_fold(c["h"], torch.from_numpy(c["X"]).to(dev), np.zeros((1, 2)), Xk)
    with pytest.raises(G.GintError):
        G.gint_fold(c["h"], torch.from_numpy(c["X"]).to(dev), np.zeros((0, 3)), Xk)
