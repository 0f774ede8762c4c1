"""gint_block_dot_noalloc: the block-store inner product for callers that cannot allocate.

The entry point keeps its partial sums in a static device array instead of handle-owned
scratch, so the call allocates nothing.  It must agree with gint_block_dot, the allocating
entry point, on two calls in a row (the static array keeps the previous call's contents).
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_block_dot_noalloc_matches_block_dot():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_08697_gb300 import gint as G
    from paper_2501_08697_gb300 import synth as S

    lib = G.load()
    dev = torch.device("cuda")
    results = []
    # the larger store first: the second call uses fewer partial sums than the first left behind
    for seed, (name, st) in enumerate([("si16", S.si_diamond((2, 1, 1), grid=(48, 24, 24), sigma=0.05,
                                                             seed=S.BASE_SEED + 82)),
                                       ("si8", S.si_diamond((1, 1, 1), grid=(24, 24, 24), seed=S.BASE_SEED + 81))]):
        h = G.setup_structure(st)
        n = h.info["nvalues"]
        g = torch.Generator().manual_seed(1234 + seed)
        A = torch.rand(n, dtype=torch.float64, generator=g).to(dev) - 0.5
        B = torch.rand(n, dtype=torch.float64, generator=g).to(dev) - 0.5
        ref = torch.zeros(1, dtype=torch.float64, device=dev)
        out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        G.gint_block_dot(h, A, B, ref)
        # through the C ABI directly
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = lib.gint_block_dot_noalloc(h.ptr, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == G.GINT_OK, lib.gint_last_error()
        torch.cuda.synchronize()
        exact = float((A.cpu().numpy() * B.cpu().numpy()).sum())
        assert out.item() == pytest.approx(ref.item(), rel=1e-12, abs=1e-12)
        assert out.item() == pytest.approx(exact, rel=1e-10, abs=1e-10)
        results.append(out.item())
        h.close()
    # two calls in a row on different store sizes gave two different, correct sums
    assert results[0] != results[1]


def test_block_dot_noalloc_rejects_null():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_08697_gb300 import gint as G
    lib = G.load()
    assert lib.gint_block_dot_noalloc(None, None, None, None, None) == G.GINT_EINVAL
