"""Spin channels on one geometry as one multi-structure job (the same handle repeated): collinear
spin (V_up, V_down; DM_up, DM_down) and the four real components of a non-collinear 2x2 spinor
potential.  Each channel must equal the single-structure call (same kernels, only the order of
FP64 atomic additions differs) and the oracle; the total density of collinear spin is the sum of
the channels (Sec. II.A)."""
import numpy as np
import pytest

from tests._cases import rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def geom():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_08697_gb300 import gint as G
    from paper_2501_08697_gb300 import synth as S
    st = S.si_diamond((1, 1, 1), grid=(30, 34, 38), sigma=0.05, seed=S.BASE_SEED + 501)
    h = G.setup_structure(st)
    keys, offs = h.layout()
    V0 = S.local_potential(st).reshape(-1)
    rng = np.random.default_rng(31)
    Vs = [V0 + 0.1 * np.sin(np.arange(V0.size) * (0.01 * (c + 1))) * rng.uniform(0.5, 1.5) for c in range(4)]
    DMs = [S.density_matrix(keys, st.norb_atom, seed=st.seed + c) for c in range(4)]
    return G, S, st, h, Vs, DMs


@pytest.mark.parametrize("nch", [2, 4])
@pytest.mark.parametrize("prec", ["tf32x3", "bf16x6"])
def test_spin_channels_match_single_calls(geom, nch, prec):
    G, S, st, h, Vs, DMs = geom
    dev = torch.device("cuda")
    V = [torch.from_numpy(v).to(dev) for v in Vs[:nch]]
    DM = [torch.from_numpy(d).to(dev) for d in DMs[:nch]]
    H = [torch.empty(h.info["nvalues"], dtype=torch.float64, device=dev) for _ in range(nch)]
    rho = [torch.empty(h.info["npts"], dtype=torch.float64, device=dev) for _ in range(nch)]
    job = G.spin_channels(h, V, H, DM, rho, prec)
    job.launch()
    torch.cuda.synchronize()
    for c in range(nch):
        Hs = torch.empty_like(H[c])
        rs = torch.empty_like(rho[c])
        G.gint_vlocal(h, V[c], Hs, prec)
        G.gint_rho(h, DM[c], rs, prec)
        torch.cuda.synchronize()
        assert rel_fro(H[c].cpu().numpy(), Hs.cpu().numpy()) < 1e-13
        assert rel_fro(rho[c].cpu().numpy(), rs.cpu().numpy()) < 1e-13
    job.close()


def test_collinear_spin_against_oracle(geom):
    from oracle import Oracle
    G, S, st, h, Vs, DMs = geom
    dev = torch.device("cuda")
    V = [torch.from_numpy(v).to(dev) for v in Vs[:2]]
    DM = [torch.from_numpy(d).to(dev) for d in DMs[:2]]
    H = [torch.empty(h.info["nvalues"], dtype=torch.float64, device=dev) for _ in range(2)]
    rho = [torch.empty(h.info["npts"], dtype=torch.float64, device=dev) for _ in range(2)]
    job = G.spin_channels(h, V, H, DM, rho, "tf32x3")
    job.launch()
    torch.cuda.synchronize()
    o = Oracle.from_structure(st)
    for c in range(2):
        assert rel_fro(H[c].cpu().numpy(), o.vlocal(Vs[c])) <= 1e-6
    tot = (rho[0] + rho[1]).cpu().numpy()
    assert rel_fro(tot, o.rho(DMs[0] + DMs[1])) <= 1e-6      # rho = rho_up + rho_down
    job.close()
