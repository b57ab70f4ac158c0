"""The allocation-free dissipation entry point agrees with the handle-based one.

rve_dissipation_noalloc serves callers that cannot allocate device memory when they need D(phi)
(a framework owning the whole device memory through its own pool, a loop that must not hit the
synchronisation of cudaMalloc, a caller with a fixed memory budget): its scratch is one fixed
array inside the library. This test gives it device buffers it owns itself, calls it twice in a
row with different damage fields (the second call reuses the array left by the first) and
compares D and Gamma with rve_dissipation on an RVE handle, to the 1e-12 relative tolerance of
the other dissipation parity tests. It lives in a file collected last, so that a run stopping at
the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from oracle import material as mat

pytestmark = pytest.mark.gpu


def _tables(m):
    G = m.n_grains
    A = np.zeros((G, 6))
    for g in range(G):
        a = mat.cleavage_tensor(m.R[g], m.cleave_n[g], m.beta[g], m.dim)
        if m.dim == 2:
            A[g, :3] = (a[0, 0], a[1, 1], a[0, 1])
        else:
            A[g] = (a[0, 0], a[1, 1], a[2, 2], a[1, 2], a[0, 2], a[0, 1])
    return np.ascontiguousarray(m.Gc, np.float64), A


@pytest.mark.parametrize("name", ["poly32", "poly3d"])
def test_noalloc_dissipation_matches_handle_path(name):
    torch = pytest.importorskip("torch")
    from paper_2508_07424_gb300 import build, capi
    from paper_2508_07424_gb300.rve import Rve
    build.build()
    w = synth.small_cases()[name]
    m = w.micro
    g = Rve.from_workload(w)
    Gc, A = _tables(m)
    dev = torch.device("cuda", 0)
    gid_d = torch.from_numpy(m.grain_id.reshape(-1).astype(np.int32)).to(dev)
    gc_d = torch.from_numpy(Gc).to(dev)
    a_d = torch.from_numpy(A.reshape(-1)).to(dev)
    out_d = torch.zeros(2, dtype=torch.float64, device=dev)
    n = (C.c_int * 3)(*m.n)
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(21)
    for call in range(2):
        phi = rng.uniform(0.0, 1.0, m.grain_id.shape)
        phi_d = torch.from_numpy(phi.reshape(-1)).to(dev)
        rc = capi.lib().rve_dissipation_noalloc(m.dim, n, w.ell, m.n_grains, gid_d.data_ptr(), gc_d.data_ptr(),
                                                a_d.data_ptr(), phi_d.data_ptr(), out_d.data_ptr(),
                                                stream.cuda_stream)
        assert rc == capi.RVE_OK, rc
        stream.synchronize()
        D_na, G_na = out_d.cpu().numpy()
        D_ref, G_ref = g.dissipation(phi)
        assert abs(D_na - D_ref) < 1e-12 * D_ref, (call, D_na, D_ref)
        assert abs(G_na - G_ref) < 1e-12 * G_ref, (call, G_na, G_ref)
    big = (C.c_int * 3)(1024, 1024, 1)
    rc = capi.lib().rve_dissipation_noalloc(2, big, w.ell, m.n_grains, gid_d.data_ptr(), gc_d.data_ptr(),
                                            a_d.data_ptr(), phi_d.data_ptr(), out_d.data_ptr(), stream.cuda_stream)
    assert rc == capi.RVE_EINVAL
