"""Failure detection without faulting the GPU: with a pipeline-wait budget of a few clock
cycles the tensor-core kernels give up on their first unfinished barrier, record GINT_ETIMEOUT
in the handle's status word, drain their in-flight MMAs (with the full budget) and exit.  The
host reads the status; the context stays usable and a normal handle still gives correct results.
Invalid arguments are rejected on the host before any launch."""
import numpy as np
import pytest

from tests._cases import rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_08697_gb300 import gint
    return gint


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x6"])
def test_wait_budget_exhaustion_reports_timeout_and_context_survives(G, prec):
    from paper_2501_08697_gb300 import synth as S
    st = S.si_diamond((2, 1, 1), sigma=0.05, seed=S.BASE_SEED + 401)
    dev = torch.device("cuda")
    V = torch.from_numpy(S.local_potential(st).reshape(-1)).to(dev)
    h_bad = G.setup_structure(st, wait_budget=1)
    keys, _ = h_bad.layout()
    DM = torch.from_numpy(S.density_matrix(keys, st.norb_atom, seed=st.seed)).to(dev)
    H = torch.empty(h_bad.info["nvalues"], dtype=torch.float64, device=dev)
    rho = torch.empty(h_bad.info["npts"], dtype=torch.float64, device=dev)
    G.gint_vlocal(h_bad, V, H, prec)
    torch.cuda.synchronize()
    assert G.gint_get_status(h_bad) == G.GINT_ETIMEOUT
    G.gint_rho(h_bad, DM, rho, prec)
    torch.cuda.synchronize()
    assert G.gint_get_status(h_bad) == G.GINT_ETIMEOUT
    assert G.gint_get_status(h_bad) == G.GINT_OK          # reading the word clears it
    # the context is intact: a default handle computes the right answer
    h = G.setup_structure(st)
    H2 = torch.empty_like(H)
    H64 = torch.empty_like(H)
    G.gint_vlocal(h, V, H2, prec)
    G.gint_vlocal(h, V, H64, "fp64")
    torch.cuda.synchronize()
    assert G.gint_get_status(h) == G.GINT_OK
    assert rel_fro(H2.cpu().numpy(), H64.cpu().numpy()) <= 1e-6


def test_host_validation(G):
    from paper_2501_08697_gb300 import synth as S
    st = S.si_diamond((1, 1, 1), grid=(16, 16, 16))
    bad_species = np.array(st.species).copy()
    bad_species[0] = 5
    with pytest.raises(G.GintError) as e:
        G.gint_setup(st.cell, bad_species, st.tau, st.tables, st.grid)
    assert e.value.code == G.GINT_EINVAL
    with pytest.raises(G.GintError):
        G.gint_setup(st.cell, st.species, st.tau, st.tables, st.grid, batch=(4, 4, 3))   # odd along a3
    with pytest.raises(G.GintError):
        G.gint_setup(np.zeros((3, 3)), st.species, st.tau, st.tables, st.grid)           # singular cell
    tau = st.tau.copy()
    tau[0, 0] = np.nan
    with pytest.raises(G.GintError):
        G.gint_setup(st.cell, st.species, tau, st.tables, st.grid)
    h = G.setup_structure(st)
    keys0, _ = h.layout()
    tau2 = st.tau.copy()
    tau2[0] += [2.0, 1.0, 0.5]                       # a different neighbour topology
    with pytest.raises(G.GintError) as e:
        G.gint_update_positions(h, tau2)
    assert e.value.code == G.GINT_ESTATE
    keys1, _ = h.layout()
    assert np.array_equal(keys0, keys1)             # the handle was left untouched
    tau3 = st.tau.copy()
    tau3[1] += [1e-7, -2e-7, 1e-7]                  # same topology: positions only
    G.gint_update_positions(h, tau3)
