"""Differentiation through the C ABI: GintVlocal's hand-written backward (adjoint rho kernel
for dL/dV, grad-phi kernel for dL/dtau) against exact linearity, central finite differences
(h = 1e-4 bohr, FP64) and the oracle's gradient.  Split-precision gradients are compared with
the FP64 analytic gradient (a finite difference of an FP32 objective would be noise)."""
import numpy as np
import pytest

from tests._cases import inputs, rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_08697_gb300 import gint as G
    from paper_2501_08697_gb300 import synth as S
    from paper_2501_08697_gb300.autograd import vlocal
    return G, S, vlocal


def _setup(G, S, name):
    st, V = inputs(name)
    h = G.setup_structure(st)
    keys, offs = h.layout()
    gH = S.density_matrix(keys, st.norb_atom, seed=st.seed + 7)
    return st, V, h, keys, gH


def _loss_at(G, st, V, gH, keys, tau, prec="fp64"):
    """L(tau) = <gH, H(V; tau)> on a handle placed at tau (new handle if the batch lists change)."""
    dev = torch.device("cuda")
    h = G.setup_structure(st, tau=tau)
    k2, _ = h.layout()
    assert np.array_equal(k2, keys), "block list changed under the displacement"
    H = torch.empty(h.info["nvalues"], dtype=torch.float64, device=dev)
    G.gint_vlocal(h, torch.from_numpy(V.reshape(-1)).to(dev), H, prec)
    L = float((H.cpu().numpy() * gH).sum())
    h.close()
    return L


@pytest.mark.parametrize("name", ["si8_ragged", "water8"])
def test_backward_v_is_exact_adjoint(env, name):
    G, S, vlocal = env
    st, V, h, keys, gH = _setup(G, S, name)
    dev = torch.device("cuda")
    Vt = torch.from_numpy(V.reshape(-1)).to(dev).requires_grad_(True)
    tau = torch.from_numpy(st.tau.copy())
    H = vlocal(Vt, tau, h, "fp64")
    gHt = torch.from_numpy(gH).to(dev)
    (H * gHt).sum().backward()
    dV = torch.from_numpy(np.random.default_rng(3).normal(size=V.size)).to(dev)
    with torch.no_grad():
        H2 = vlocal(Vt + dV, tau, h, "fp64")
        lhs = float(((H2 - H) * gHt).sum())
    rhs = float((Vt.grad * dV).sum())
    assert lhs == pytest.approx(rhs, rel=1e-10)


@pytest.mark.parametrize("name", ["si8_ragged", "water8"])
def test_backward_tau_matches_central_differences(env, name):
    G, S, vlocal = env
    st, V, h, keys, gH = _setup(G, S, name)
    dev = torch.device("cuda")
    Vt = torch.from_numpy(V.reshape(-1)).to(dev)
    tau = torch.from_numpy(st.tau.copy()).requires_grad_(True)
    H = vlocal(Vt, tau, h, "fp64")
    (H * torch.from_numpy(gH).to(dev)).sum().backward()
    g = tau.grad.numpy()
    hstep = 1e-4
    for atom in (0, st.natoms - 1):
        for c in range(3):
            tp, tm = st.tau.copy(), st.tau.copy()
            tp[atom, c] += hstep
            tm[atom, c] -= hstep
            fd = (_loss_at(G, st, V, gH, keys, tp) - _loss_at(G, st, V, gH, keys, tm)) / (2 * hstep)
            assert fd == pytest.approx(g[atom, c], rel=1e-6, abs=1e-8 * np.abs(g).max())


def test_backward_tau_matches_oracle(env):
    from oracle import Oracle
    G, S, vlocal = env
    st, V, h, keys, gH = _setup(G, S, "si8_ragged")
    dev = torch.device("cuda")
    tau = torch.from_numpy(st.tau.copy()).requires_grad_(True)
    Vt = torch.from_numpy(V.reshape(-1)).to(dev).requires_grad_(True)
    H = vlocal(Vt, tau, h, "fp64")
    (H * torch.from_numpy(gH).to(dev)).sum().backward()
    o = Oracle.from_structure(st)
    assert rel_fro(tau.grad.numpy(), o.dLdtau(V, gH)) < 1e-10
    assert rel_fro(Vt.grad.cpu().numpy(), st.dV * o.rho(gH)) < 1e-11


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("tf32x3", 1e-6), ("bf16x6", 1e-6), ("bf16x3", 1e-4)])
def test_split_precision_gradients_vs_fp64(env, prec, tol):
    G, S, vlocal = env
    st, V, h, keys, gH = _setup(G, S, "si16_strained")
    dev = torch.device("cuda")
    gHt = torch.from_numpy(gH).to(dev)
    grads = {}
    for p in ("fp64", prec):
        Vt = torch.from_numpy(V.reshape(-1)).to(dev).requires_grad_(True)
        tau = torch.from_numpy(st.tau.copy()).requires_grad_(True)
        (vlocal(Vt, tau, h, p) * gHt).sum().backward()
        grads[p] = (Vt.grad.cpu().numpy(), tau.grad.numpy())
    eV = rel_fro(grads[prec][0], grads["fp64"][0])
    eT = rel_fro(grads[prec][1], grads["fp64"][1])
    print(f"{prec}: dL/dV rel err {eV:.2e}, dL/dtau rel err {eT:.2e}")
    assert eV <= tol and eT <= 2 * tol


def test_differentiation_config_si64(env):
    """The 64-atom differentiation case (96^3 grid, displaced atoms): FP64 autograd gradient
    against central differences on two atoms, and the TF32x3 / FP32 gradients against FP64."""
    G, S, vlocal = env
    st, V, h, keys, gH = _setup(G, S, "si64")
    dev = torch.device("cuda")
    gHt = torch.from_numpy(gH).to(dev)
    grads = {}
    for p in ("fp64", "fp32", "tf32x3"):
        Vt = torch.from_numpy(V.reshape(-1)).to(dev).requires_grad_(True)
        tau = torch.from_numpy(st.tau.copy()).requires_grad_(True)
        (vlocal(Vt, tau, h, p) * gHt).sum().backward()
        grads[p] = (Vt.grad.cpu().numpy(), tau.grad.numpy())
    g = grads["fp64"][1]
    for atom, c in ((3, 0), (41, 2)):
        tp, tm = st.tau.copy(), st.tau.copy()
        tp[atom, c] += 1e-4
        tm[atom, c] -= 1e-4
        fd = (_loss_at(G, st, V, gH, keys, tp) - _loss_at(G, st, V, gH, keys, tm)) / 2e-4
        assert fd == pytest.approx(g[atom, c], rel=1e-6, abs=1e-8 * np.abs(g).max())
    for p in ("fp32", "tf32x3"):
        assert rel_fro(grads[p][0], grads["fp64"][0]) <= 1e-6
        assert rel_fro(grads[p][1], grads["fp64"][1]) <= 2e-6


def test_water_box_split_bf16_with_fd_on_eight_atoms(env):
    """The 64-molecule water box (128^3): forward, adjoint and force in split BF16, FP64
    finite-difference check of the force on 8 atoms."""
    G, S, vlocal = env
    st, V, h, keys, gH = _setup(G, S, "water64")
    dev = torch.device("cuda")
    gHt = torch.from_numpy(gH).to(dev)
    grads = {}
    for p in ("fp64", "bf16x6", "bf16x3"):
        Vt = torch.from_numpy(V.reshape(-1)).to(dev).requires_grad_(True)
        tau = torch.from_numpy(st.tau.copy()).requires_grad_(True)
        (vlocal(Vt, tau, h, p) * gHt).sum().backward()
        grads[p] = (Vt.grad.cpu().numpy(), tau.grad.numpy())
    g = grads["fp64"][1]
    rng = np.random.default_rng(5)
    for atom in rng.choice(st.natoms, 8, replace=False):
        c = int(rng.integers(3))
        tp, tm = st.tau.copy(), st.tau.copy()
        tp[atom, c] += 1e-4
        tm[atom, c] -= 1e-4
        fd = (_loss_at(G, st, V, gH, keys, tp) - _loss_at(G, st, V, gH, keys, tm)) / 2e-4
        assert fd == pytest.approx(g[atom, c], rel=1e-6, abs=1e-8 * np.abs(g).max())
    print("water64 bf16x6 dV %.2e dtau %.2e | bf16x3 dV %.2e dtau %.2e" % (
        rel_fro(grads["bf16x6"][0], grads["fp64"][0]), rel_fro(grads["bf16x6"][1], grads["fp64"][1]),
        rel_fro(grads["bf16x3"][0], grads["fp64"][0]), rel_fro(grads["bf16x3"][1], grads["fp64"][1])))
    assert rel_fro(grads["bf16x6"][0], grads["fp64"][0]) <= 1e-6
    assert rel_fro(grads["bf16x6"][1], grads["fp64"][1]) <= 2e-6
    assert rel_fro(grads["bf16x3"][0], grads["fp64"][0]) <= 1e-4


def test_two_forwards_at_different_tau_before_backward(env):
    """L = <gH, H(V; tau1)> + <gH2, H(V; tau2)> on one handle: the second forward moves the
    handle, and each term's backward must still be taken at its own geometry.  The sum of the
    two gradients is compared with two separate forward/backward passes."""
    G, S, vlocal = env
    st, V, h, keys, gH = _setup(G, S, "si8_ragged")
    dev = torch.device("cuda")
    gH2 = S.density_matrix(keys, st.norb_atom, seed=st.seed + 11)
    gHt, gH2t = torch.from_numpy(gH).to(dev), torch.from_numpy(gH2).to(dev)
    tau1 = st.tau.copy()
    tau2 = st.tau.copy()
    tau2[0] += (0.01, -0.02, 0.015)
    Vt = torch.from_numpy(V.reshape(-1)).to(dev)

    def grad_of(pairs):
        ts = [torch.from_numpy(t.copy()).requires_grad_(True) for t, _ in pairs]
        L = sum((vlocal(Vt, t, h, "fp64") * g).sum() for t, (_, g) in zip(ts, pairs))
        L.backward()
        return [t.grad.numpy().copy() for t in ts]

    g1, g2 = grad_of([(tau1, gHt), (tau2, gH2t)])      # both forwards, then one backward
    (r1,) = grad_of([(tau1, gHt)])
    (r2,) = grad_of([(tau2, gH2t)])
    assert rel_fro(g1, r1) < 1e-12 and rel_fro(g2, r2) < 1e-12
    assert rel_fro(g1, g2) > 1e-3                        # the two geometries do differ
