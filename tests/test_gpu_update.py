"""Position updates through the C ABI: a handle moved with gint_update_positions gives the same
batches, description and results (V_mu,nu, rho, force) as a handle built at the new positions,
both when the batch -> atom-image lists are kept (small moves: new slot positions only) and
when they change (seeded N(0, 0.05 bohr) displacements of every atom)."""
import numpy as np
import pytest

from tests._cases import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_08697_gb300 import gint
    return gint


def _run(G, h, V, DM, natoms, prec):
    dev = torch.device("cuda")
    H = torch.empty(h.info["nvalues"], dtype=torch.float64, device=dev)
    rho = torch.empty(h.info["npts"], dtype=torch.float64, device=dev)
    F = torch.empty(3 * natoms, dtype=torch.float64, device=dev)
    G.gint_vlocal(h, V, H, prec)
    G.gint_rho_force(h, V, DM, rho, F, prec)
    return H.cpu().numpy(), rho.cpu().numpy(), F.cpu().numpy()


@pytest.mark.parametrize("name", ["si64", "water8"])
@pytest.mark.parametrize("sigma", [1e-6, 0.05])
def test_update_matches_fresh_handle(G, name, sigma):
    from paper_2501_08697_gb300 import synth as S
    st, Vn = inputs(name)
    dev = torch.device("cuda")
    V = torch.from_numpy(Vn.reshape(-1)).to(dev)
    h = G.setup_structure(st, batch=(4, 4, 8), batch_rho=(4, 4, 8))
    keys, _ = h.layout()
    DM = torch.from_numpy(S.density_matrix(keys, st.norb_atom, seed=st.seed)).to(dev)
    rng = np.random.default_rng(2501 + int(sigma * 1e6))
    tau = st.tau + rng.normal(0.0, sigma, st.tau.shape)
    fresh = G.setup_structure(st, batch=(4, 4, 8), batch_rho=(4, 4, 8), tau=tau)
    k2, _ = fresh.layout()
    if not np.array_equal(k2, keys):
        # a pair crossed the cutoff: the update must refuse and leave the handle as it was
        with pytest.raises(G.GintError) as e:
            G.gint_update_positions(h, tau)
        assert e.value.code == G.GINT_ESTATE
        pytest.skip("the displacement changed the block list")
    G.gint_update_positions(h, tau)
    a, b = G.gint_get_info(h), G.gint_get_info(fresh)
    for k in ("nbatches", "nslots", "max_orbitals", "nbatches_rho", "max_orbitals_rho", "nvalues"):
        assert a[k] == b[k], k
    assert a["flops_useful"] == b["flops_useful"]
    assert abs(a["flops_dense"] - b["flops_dense"]) <= 1e-12 * b["flops_dense"]
    for prec in ("fp64", "fp16x3"):
        H1, r1, F1 = _run(G, h, V, DM, st.natoms, prec)
        H2, r2, F2 = _run(G, fresh, V, DM, st.natoms, prec)
        # same lists and positions: equal up to the last bits of the slot positions.  The force
        # of a split precision is summed in FP32 shared-memory atomics per batch, whose order
        # varies from run to run: it agrees to that rounding (the method's 1e-6 bound) only.
        for x, y, what in ((H1, H2, "H"), (r1, r2, "rho"), (F1, F2, "F")):
            err = np.abs(x - y).max() / np.abs(y).max()
            tol = 1e-6 if (what == "F" and prec != "fp64") else 1e-12
            print(f"{name} sigma {sigma} {prec}: {what} {err:.2e}")
            assert err <= tol, (prec, what, err)
    fresh.close()
    h.close()
