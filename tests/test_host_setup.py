"""Host logic of the set-up and of position updates, on the CPU: gint_setup.cpp is compiled with
host-memory stand-ins for the CUDA runtime calls it makes (tests/host/cuda_stub.cpp), and a
handle moved with gint_update_positions must hold exactly the batches, atom-image slots, slot-pair
tables and padded offsets of a handle set up at the new positions (Sec. IV.B: the batch lists
follow from strict locality, so they are a function of the positions alone).  Covered: unchanged
lists (new positions only), changed lists (per-batch reuse, partial reuse of a batch's old
table), a refused update (block list changed: the handle stays as it was), rho/force lists shared
with the vlocal lists when both use the same batch shape, and the row-layout fallback; and the
cost-balanced CTA ranges of the persistent kernels."""
import ctypes as C
import os
import shutil
import subprocess
from contextlib import contextmanager

import numpy as np
import pytest

from tests._cases import structure

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2501_08697_gb300", "csrc")
HOST = os.path.join(ROOT, "tests", "host")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    out = tmp_path_factory.mktemp("hostsetup")
    so = str(out / "libgint_host.so")
    srcs = [os.path.join(CSRC, "gint_setup.cpp"), os.path.join(HOST, "cuda_stub.cpp"), os.path.join(HOST, "inspect.cpp")]
    # -Bsymbolic: the set-up code calls these stand-ins even where the process has loaded the CUDA
    # runtime already (through torch)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-Wl,-Bsymbolic", "-I", inc, "-I", CSRC,
                           "-I", os.path.join(ROOT, "include"), *srcs, "-o", so, "-lpthread"])
    from paper_2501_08697_gb300 import gint as G
    L = C.CDLL(so)
    P, vp, i32, d = C.POINTER, C.c_void_p, C.c_int, C.c_double
    L.gint_setup.argtypes = [P(vp), P(d), i32, P(i32), P(d), i32, P(G._Species), P(i32), P(G._Options)]
    L.gint_get_info.argtypes = [vp, P(G._Info)]
    L.gint_update_positions.argtypes = [vp, P(d)]
    L.gint_destroy.argtypes = [vp]
    L.gint_block_layout.argtypes = [vp, P(C.c_int64), P(C.c_int64), P(P(C.c_int32)), P(P(C.c_int64))]
    L.gint_last_error.restype = C.c_char_p
    L.inspect_compare.argtypes = [vp, vp]
    L.inspect_summary.argtypes = [vp, i32, P(C.c_longlong)]
    L.inspect_check_tables.argtypes = [vp]
    L.inspect_check_tables.restype = C.c_longlong
    for n in ("gint_setup", "gint_get_info", "gint_update_positions", "gint_destroy", "gint_block_layout",
              "inspect_compare"):
        getattr(L, n).restype = C.c_int
    return L


@contextmanager
def host_lib(L):
    """gint.py's marshalling over the host build (the module's library is put back after)."""
    from paper_2501_08697_gb300 import gint as G
    keep = G._lib
    G._lib = L
    try:
        yield G
    finally:
        G._lib = keep


def _summary(L, h, w):
    out = (C.c_longlong * 6)()
    L.inspect_summary(h._ptr, w, out)
    return dict(zip(("batches", "slots", "entries", "padn", "shared", "max_k"), list(out)))


CASES = [("si8", (4, 4, 8)), ("si64", (4, 4, 8)), ("si64", (4, 4, 4)), ("water8", (4, 4, 8)),
         ("si16_strained", (4, 4, 4)), ("si8_2d", (4, 4, 8)), ("h64_dense", (4, 4, 8))]


@pytest.mark.parametrize("name,batch", CASES)
def test_update_equals_fresh_setup(lib, name, batch):
    st = structure(name)
    rng = np.random.default_rng(2501)
    with host_lib(lib) as G:
        h = G.setup_structure(st, batch=batch, batch_rho=(4, 4, 8))
        assert lib.inspect_check_tables(h._ptr) == 0
        cur, moved = st.tau, 0
        for sigma in (0.0, 1e-6, 0.01, 0.05, 0.05, 0.01):
            tau = st.tau + rng.normal(0.0, sigma, st.tau.shape)
            fresh = G.setup_structure(st, batch=batch, batch_rho=(4, 4, 8), tau=tau)
            if np.array_equal(fresh.layout()[0], h.layout()[0]):
                G.gint_update_positions(h, tau)
                assert lib.inspect_compare(h._ptr, fresh._ptr) == 0, (name, sigma)
                cur, moved = tau, moved + 1
            else:
                # the block list changed: refused, and the handle keeps its lists
                with pytest.raises(G.GintError) as e:
                    G.gint_update_positions(h, tau)
                assert e.value.code == G.GINT_ESTATE
                before = G.setup_structure(st, batch=batch, batch_rho=(4, 4, 8), tau=cur)
                assert lib.inspect_compare(h._ptr, before._ptr) == 0, (name, sigma)
                before.close()
            fresh.close()
        assert moved >= 2
        assert lib.inspect_check_tables(h._ptr) == 0
        h.close()


def test_rho_lists_shared_with_vlocal(lib):
    """Same batch shape: the rho/force set is the vlocal set (and its own slot-pair offsets) when
    every vlocal batch fits the padded layout; another shape or a wider batch builds its own."""
    with host_lib(lib) as G:
        for name in ("si8", "si64"):       # an ideal crystal, and one with displaced atoms
            h = G.setup_structure(structure(name), batch=(4, 4, 8), batch_rho=(4, 4, 8))
            v, r = _summary(lib, h, 0), _summary(lib, h, 1)
            if name == "si8" or v["max_k"] <= 256:
                assert r["shared"] == 1 and r["padn"] == 1
                assert (v["batches"], v["slots"], v["entries"]) == (r["batches"], r["slots"], r["entries"])
            else:
                assert r["shared"] == 0 and r["batches"] >= v["batches"]
            h.close()
        st = structure("si64")
        h = G.setup_structure(st, batch=(4, 4, 4), batch_rho=(4, 4, 8))
        assert _summary(lib, h, 1)["shared"] == 0
        # the comparison sees a change of positions alone
        tau = st.tau + np.random.default_rng(3).normal(0.0, 1e-3, st.tau.shape)
        g = G.setup_structure(st, batch=(4, 4, 4), batch_rho=(4, 4, 8), tau=tau)
        assert lib.inspect_compare(h._ptr, g._ptr) != 0
        g.close()
        h.close()


def test_cta_ranges_cover_and_balance(lib):
    """The persistent kernels' CTA ranges (segment_ranges): within each segment of the batch list
    the non-empty ranges tile it in order, one per CTA, with min(CTAs, batches) of them; each
    range's estimated cost is within one batch's cost of the segment's mean per range; and the
    CTAs that get work rotate from one segment to the next, so short segments land on different
    CTAs."""
    lib.inspect_batches.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_longlong]
    lib.inspect_batches.restype = C.c_longlong
    lib.inspect_segment_ranges.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    npart = 152
    with host_lib(lib) as G:
        h = G.setup_structure(structure("si64"), batch=(4, 4, 8), batch_rho=(4, 4, 8))
        for w in (0, 1):
            n = lib.inspect_batches(h._ptr, w, None, 0)
            buf = np.zeros(4 * n, np.int32)
            lib.inspect_batches(h._ptr, w, buf.ctypes.data, 4 * n)
            pts, nb = buf.reshape(n, 4)[:, 0].astype(float), buf.reshape(n, 4)[:, 1].astype(float)
            # the cost model of the partition (relative cycles per batch, one form per kernel)
            cost = (2000.0 + 2.6 * pts * nb + 0.65 * nb * nb) if w == 0 else (4000.0 + 4.0 * pts * nb + nb * nb)
            for seg in ([0, n], [0, n // 3, n // 3 + 5, n], [0, 7, 20, 30, n]):
                nseg = len(seg) - 1
                out = np.zeros(2 * nseg * npart, np.int32)
                sa = np.array(seg, np.int32)
                lib.inspect_segment_ranges(h._ptr, w, sa.ctypes.data, nseg, npart, out.ctypes.data)
                r = out.reshape(nseg, npart, 2)
                used = []
                for g in range(nseg):
                    lo, hi = seg[g], seg[g + 1]
                    ranges = sorted((int(a), int(b), c) for c, (a, b) in enumerate(r[g]) if b > a)
                    assert len(ranges) == min(npart, hi - lo)
                    assert ranges[0][0] == lo and ranges[-1][1] == hi
                    assert all(ranges[i][1] == ranges[i + 1][0] for i in range(len(ranges) - 1))
                    # ranges are dealt to CTAs in order, starting where the last segment stopped
                    ctas = [c for _, _, c in ranges]
                    assert ctas == [(ctas[0] + i) % npart for i in range(len(ctas))]
                    if used:
                        assert ctas[0] == (used[-1][-1] + 1) % npart
                    used.append(ctas)
                    if hi - lo >= 4 * npart:
                        mean = cost[lo:hi].sum() / len(ranges)
                        cmax = cost[lo:hi].max()
                        for a, b, _ in ranges:
                            assert abs(cost[a:b].sum() - mean) <= cmax * (1 + 1e-9), (w, g, a, b)
        h.close()
