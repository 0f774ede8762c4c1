"""Strain derivative dL/deps of L = <rho_mu,nu, V_mu,nu> (the grid part of the stress of
Eq. stress, sigma = -dL/deps / Omega) through the C ABI against the FP64 oracle, whose own
strain derivative is pinned to central differences in test_oracle_pins.

Tolerances (relative Frobenius over the 3x3): FP64 1e-11; FP32, TF32x3, BF16x6 1e-6; BF16x3
5e-5 (about 16 significant bits)."""
import numpy as np
import pytest

from tests._cases import oracle_full, oracle_strain, rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 1e-6, "tf32x3": 1e-6, "bf16x6": 1e-6, "bf16x3": 5e-5}


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_08697_gb300 import gint
    return gint


_handles = {}


def _strain(G, name, prec):
    ref = oracle_full(name)
    if name not in _handles:
        _handles[name] = G.setup_structure(ref["st"])
    h = _handles[name]
    dev = torch.device("cuda")
    V = torch.from_numpy(ref["V"].reshape(-1)).to(dev)
    DM = torch.from_numpy(ref["DM"]).to(dev)
    out = torch.full((9,), float("nan"), dtype=torch.float64, device=dev)
    G.gint_strain_derivative(h, V, DM, out, prec)
    torch.cuda.synchronize()
    assert G.gint_get_status(h) == 0
    return out.cpu().numpy().reshape(3, 3)


@pytest.mark.parametrize("name", ["si8", "si8_ragged", "si16_strained", "water8"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32x3", "bf16x3", "bf16x6"])
def test_strain_derivative_parity(G, name, prec):
    ref = oracle_strain(name)
    got = _strain(G, name, prec)
    err = rel_fro(got, ref)
    print(f"{name} {prec}: dL/deps {err:.2e}")
    assert err <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_strain_derivative_si64(G, prec):
    ref = oracle_strain("si64")
    got = _strain(G, "si64", prec)
    err = rel_fro(got, ref)
    print(f"si64 {prec}: dL/deps {err:.2e}")
    assert err <= TOL[prec]


def test_strain_trace_holds_the_volume_term(G):
    """The delta_ab term: dL/deps_aa contains dV Sum V rho = L; removing it leaves the basis
    part, which the force path sums per atom instead of with the displacement."""
    ref = oracle_full("si8")
    got = _strain(G, "si8", "fp64")
    L = float((ref["DM"] * ref["H"]).sum())
    basis = got - L * np.eye(3)
    ref_basis = oracle_strain("si8") - L * np.eye(3)
    assert rel_fro(basis, ref_basis) <= 1e-10
