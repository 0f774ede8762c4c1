"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative Frobenius norm over the whole output): FP64 <= 1e-11; FP32 and the
split tensor-core paths TF32x3 / FP16x3 / BF16x6 <= 1e-6; BF16x3 (about 16 significant bits)
is held to 5e-5 and its error reported.  The block layout is compared bit-exactly.
"""
import numpy as np
import pytest

from tests._cases import inputs, oracle_full, rel_fro

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 1e-6, "tf32x3": 1e-6, "fp16x3": 1e-6, "bf16x6": 1e-6, "bf16x3": 5e-5}
FORCE_TOL = {"fp64": 1e-10, "fp32": 1e-6, "tf32x3": 1e-6, "fp16x3": 1e-6, "bf16x6": 1e-6, "bf16x3": 1e-4}
SIMT = ["fp64", "fp32"]
ALL = ["fp64", "fp32", "tf32x3", "fp16x3", "bf16x3", "bf16x6"]
CASES = ["si8", "si8_ragged", "si16_strained", "water8", "water1_vacuum", "si8_2d"]
TC = ["tf32x3", "fp16x3", "bf16x3", "bf16x6"]


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_08697_gb300 import gint
    gint.load()
    return gint


_handles = {}


def _handle(G, name, batch=None):
    key = (name, batch)
    if key not in _handles:
        st, _ = inputs(name)
        kw = {} if batch is None else dict(batch=batch, batch_rho=batch)
        _handles[key] = G.setup_structure(st, **kw)
    return _handles[key]


def _run(G, name, prec, batch=None):
    ref = oracle_full(name)
    h = _handle(G, name, batch)
    keys, offs = h.layout()
    assert np.array_equal(keys, ref["keys"]) and np.array_equal(offs, ref["offs"])
    dev = torch.device("cuda")
    V = torch.from_numpy(ref["V"].reshape(-1)).to(dev)
    DM = torch.from_numpy(ref["DM"]).to(dev)
    H = torch.empty(h.info["nvalues"], dtype=torch.float64, device=dev)
    rho = torch.empty(h.info["npts"], dtype=torch.float64, device=dev)
    F = torch.empty(3 * h.natoms, dtype=torch.float64, device=dev)
    G.gint_vlocal(h, V, H, prec)
    G.gint_rho_force(h, V, DM, rho, F, prec)
    torch.cuda.synchronize()
    assert G.gint_get_status(h) == 0
    return ref, h, H.cpu().numpy(), rho.cpu().numpy(), F.cpu().numpy().reshape(-1, 3)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("prec", SIMT)
def test_simt_parity(G, name, prec):
    ref, h, H, rho, F = _run(G, name, prec)
    eH, er, eF = rel_fro(H, ref["H"]), rel_fro(rho, ref["rho"]), rel_fro(F, ref["F"])
    print(f"{name} {prec}: H {eH:.2e} rho {er:.2e} F {eF:.2e}")
    assert eH <= TOL[prec]
    assert er <= TOL[prec]
    assert eF <= FORCE_TOL[prec]


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("prec", TC)
def test_tensor_core_parity(G, name, prec):
    ref, h, H, rho, F = _run(G, name, prec)
    eH, er, eF = rel_fro(H, ref["H"]), rel_fro(rho, ref["rho"]), rel_fro(F, ref["F"])
    print(f"{name} {prec}: H {eH:.2e} rho {er:.2e} F {eF:.2e}")
    assert eH <= TOL[prec]
    assert er <= TOL[prec]
    assert eF <= FORCE_TOL[prec]


@pytest.mark.parametrize("batch", [(4, 4, 4), (2, 2, 2), (4, 4, 2), (8, 2, 4)])
@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3", "bf16x6"])
def test_tensor_core_batch_shapes(G, batch, prec):
    """One-tile (<= 128 orbitals), two-tile and split batches; ragged grid.  Batches of at
    most 64 points keep the tensor-core FP32 accumulation within 1e-6 for vlocal."""
    ref, h, H, rho, F = _run(G, "si8_ragged", prec, batch)
    eH, er, eF = rel_fro(H, ref["H"]), rel_fro(rho, ref["rho"]), rel_fro(F, ref["F"])
    print(f"si8_ragged {prec} batch {batch}: H {eH:.2e} rho {er:.2e} F {eF:.2e}")
    assert eH <= 1e-6 and er <= 1e-6 and eF <= 1e-6


@pytest.mark.parametrize("batch", [(4, 4, 4), (8, 4, 4), (2, 2, 2), (8, 8, 2)])
def test_batch_shapes_fp64(G, batch):
    ref, h, H, rho, F = _run(G, "si8_ragged", "fp64", batch)
    assert rel_fro(H, ref["H"]) <= 1e-11
    assert rel_fro(rho, ref["rho"]) <= 1e-11
    assert rel_fro(F, ref["F"]) <= 1e-10


def test_separate_entry_points_match_fused(G):
    ref, h, H, rho, F = _run(G, "water8", "fp64")
    dev = torch.device("cuda")
    V = torch.from_numpy(ref["V"].reshape(-1)).to(dev)
    DM = torch.from_numpy(ref["DM"]).to(dev)
    rho2 = torch.empty_like(V)
    F2 = torch.empty(3 * h.natoms, dtype=torch.float64, device=dev)
    G.gint_rho(h, DM, rho2, "fp64")
    G.gint_force(h, V, DM, F2, "fp64")
    assert rel_fro(rho2.cpu().numpy(), rho) < 1e-14
    assert rel_fro(F2.cpu().numpy(), F.reshape(-1)) < 1e-13


def test_reductions_and_identities_on_gpu(G):
    ref, h, H, rho, F = _run(G, "si8", "fp64")
    dev = torch.device("cuda")
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    rho_t = torch.from_numpy(rho).to(dev)
    G.gint_charge(h, rho_t, out)
    assert out.item() == pytest.approx(rho.sum() * h.info["dV"], rel=1e-13)
    Ht = torch.from_numpy(H).to(dev)
    DMt = torch.from_numpy(ref["DM"]).to(dev)
    G.gint_block_dot(h, DMt, Ht, out)
    tr = out.item()
    assert tr == pytest.approx((ref["DM"] * H).sum(), rel=1e-13)
    # adjoint identity <rho, V> dV = <DM, H> on the GPU outputs
    assert (rho * ref["V"].reshape(-1)).sum() * h.info["dV"] == pytest.approx(tr, rel=1e-11)


def test_block_symmetry_of_gpu_h(G):
    ref, h, H, rho, F = _run(G, "water8", "fp32")
    keys, offs = h.layout()
    from paper_2501_08697_gb300.synth import partner_index
    part = partner_index(keys)
    nI = ref["st"].norb_atom
    for b in range(len(keys)):
        A = H[offs[b]:offs[b + 1]].reshape(nI[keys[b, 0]], -1)
        B = H[offs[part[b]]:offs[part[b] + 1]].reshape(nI[keys[part[b], 0]], -1)
        assert np.array_equal(A, B.T)


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "fp16x3", "bf16x6"])
def test_many_atom_images_per_batch(G, prec):
    """h64_dense: every batch sees 39-53 atom images (one orbital each), more than the
    shared-memory slot-pair tables of the tensor-core kernels hold (28), so vlocal's scatter and
    rho's gather tables read the batch's table from global memory."""
    ref, h, H, rho, F = _run(G, "h64_dense", prec)
    eH, er, eF = rel_fro(H, ref["H"]), rel_fro(rho, ref["rho"]), rel_fro(F, ref["F"])
    print(f"h64_dense {prec}: H {eH:.2e} rho {er:.2e} F {eF:.2e}")
    assert eH <= TOL[prec] and er <= TOL[prec] and eF <= FORCE_TOL[prec]


def test_run_host_matches_device_path(G):
    ref, h, H, rho, F = _run(G, "si8_ragged", "fp64")
    Hh = np.empty(h.info["nvalues"])
    rh = np.empty(h.info["npts"])
    Fh = np.empty(3 * h.natoms)
    G.gint_run_host(h, np.ascontiguousarray(ref["V"].reshape(-1)), ref["DM"], Hh, rh, Fh, "fp64")
    assert rel_fro(Hh, H) < 1e-14 and rel_fro(rh, rho) < 1e-14 and rel_fro(Fh, F.reshape(-1)) < 1e-13


def test_run_host_pinned_repeated_matches_device_path(G):
    """Pinned host buffers (the copies then overlap the kernels on the library's copy stream),
    two calls in a row on the same handle."""
    ref, h, H, rho, F = _run(G, "si8_ragged", "tf32x3")
    pin = lambda n: torch.empty(n, dtype=torch.float64).pin_memory()
    Vh, DMh = pin(h.info["npts"]), pin(h.info["nvalues"])
    Vh.copy_(torch.from_numpy(np.ascontiguousarray(ref["V"].reshape(-1))))
    DMh.copy_(torch.from_numpy(ref["DM"]))
    Hh, rh, Fh = pin(h.info["nvalues"]), pin(h.info["npts"]), pin(3 * h.natoms)
    for _ in range(2):
        for t in (Hh, rh, Fh):
            t.fill_(float("nan"))
        G.gint_run_host(h, Vh, DMh, Hh, rh, Fh, "tf32x3")
        assert rel_fro(Hh.numpy(), H) < 1e-13 and rel_fro(rh.numpy(), rho) < 1e-13
        # the per-batch force sums are FP32 shared-memory additions whose order varies from run
        # to run, so F agrees to FP32 rounding of those sums, well inside the 1e-6 tolerance
        assert rel_fro(Fh.numpy(), F.reshape(-1)) < 1e-6


def test_invalid_arguments_are_rejected_on_host(G):
    h = _handle(G, "si8")
    dev = torch.device("cuda")
    V = torch.zeros(h.info["npts"], dtype=torch.float64, device=dev)
    with pytest.raises(G.GintError) as e:
        G.gint_vlocal(h, V, V, 99)
    assert e.value.code == G.GINT_EINVAL
    with pytest.raises(TypeError):
        G.gint_vlocal(h, V.float(), V, "fp64")
    import ctypes
    lib = G.load()
    assert lib.gint_vlocal(h.ptr, None, None, 0, None) == G.GINT_EINVAL
    assert lib.gint_vlocal(None, None, None, 0, None) == G.GINT_EINVAL
