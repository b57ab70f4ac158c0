"""The allocation-free dissipation entry point agrees with the handle-based one.

rve_dissipation_noalloc serves callers that cannot allocate device memory when they need D(phi)
(a framework owning the whole device memory through its own pool, a loop that must not hit the
synchronisation of cudaMalloc, a caller with a fixed memory budget): its scratch is one fixed
array inside the library. This test gives it device buffers it owns itself, calls it twice in a
row with different damage fields (the second call reuses the array left by the first) and
compares D and Gamma with rve_dissipation on an RVE handle, to the 1e-12 relative tolerance of
the other dissipation parity tests. The grids span the small parity cases, a plate one voxel
thick and the two largest grids that fit the array (512 x 512 and 32^3); the first grids that do
not fit are refused. A grain id outside the tables gives NaN instead of a read past them. It
lives in a file collected last, so that a run stopping at the first failure has already run every
other test.
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


def _workload(name):
    if name == "poly512":
        return synth.Workload(synth.voronoi((512, 512), 40, 31, beta=2.0, sigma_Gc=0.3), ell=3.0)
    if name == "poly32cubed":
        return synth.Workload(synth.voronoi((32, 32, 32), 20, 33, orientation="so3", beta=1.0, sigma_Gc=0.3),
                              ell=2.0)
    return synth.small_cases()[name]


class _Bufs:
    def __init__(self, torch, m):
        dev = torch.device("cuda", 0)
        Gc, A = _tables(m)
        self.torch, self.dev, self.m = torch, dev, m
        self.gid = torch.from_numpy(m.grain_id.reshape(-1).astype(np.int32)).to(dev)
        self.gc = torch.from_numpy(Gc).to(dev)
        self.a = torch.from_numpy(A.reshape(-1)).to(dev)
        self.out = torch.zeros(2, dtype=torch.float64, device=dev)
        self.stream = torch.cuda.current_stream()

    def call(self, capi, dim, n, ell, phi_d, gid=None):
        nn = (C.c_int * 3)(*n)
        g = self.gid if gid is None else gid
        rc = capi.lib().rve_dissipation_noalloc(dim, nn, ell, self.m.n_grains, g.data_ptr(), self.gc.data_ptr(),
                                                self.a.data_ptr(), phi_d.data_ptr(), self.out.data_ptr(),
                                                self.stream.cuda_stream)
        self.stream.synchronize()
        return rc, self.out.cpu().numpy().copy()


@pytest.mark.parametrize("name", ["poly32", "poly3d", "plate3d", "poly512", "poly32cubed"])
def test_noalloc_dissipation_matches_handle_path(name):
    torch = pytest.importorskip("torch")
    from paper_2508_07424_gb300 import build, capi
    from paper_2508_07424_gb300.rve import Rve
    build.build()
    w = _workload(name)
    m = w.micro
    g = Rve.from_workload(w)
    b = _Bufs(torch, m)
    rng = np.random.default_rng(21)
    for call in range(2):
        phi = rng.uniform(0.0, 1.0, m.grain_id.shape)
        phi_d = torch.from_numpy(phi.reshape(-1)).to(b.dev)
        rc, (D_na, G_na) = b.call(capi, m.dim, m.n, w.ell, phi_d)
        assert rc == capi.RVE_OK, rc
        D_ref, G_ref = g.dissipation(phi)
        assert abs(D_na - D_ref) < 1e-12 * D_ref, (call, D_na, D_ref)
        assert abs(G_na - G_ref) < 1e-12 * G_ref, (call, G_na, G_ref)
    g.close()


def test_noalloc_refuses_grids_beyond_the_array_and_flags_bad_ids():
    torch = pytest.importorskip("torch")
    from paper_2508_07424_gb300 import build, capi
    build.build()
    w = synth.small_cases()["poly32"]
    m = w.micro
    b = _Bufs(torch, m)
    phi_d = torch.from_numpy(np.random.default_rng(5).uniform(0, 1, m.grain_id.size)).to(b.dev)
    # the first grids past the 8 MiB scratch: the pointers are never read, the call returns first
    for dim, n in ((3, (64, 64, 64)), (2, (1024, 512, 1)), (2, (512, 1024, 1)), (2, (1024, 1024, 1))):
        rc, _ = b.call(capi, dim, n, w.ell, phi_d)
        assert rc == capi.RVE_EINVAL, (n, rc)
    # a grain id outside [0, n_grains) reads no table entry and makes the result NaN
    bad = b.gid.clone()
    bad[17] = m.n_grains
    bad[300] = -1
    rc, out = b.call(capi, 2, m.n, w.ell, phi_d, gid=bad)
    assert rc == capi.RVE_OK and np.isnan(out).all(), out
    # the next call with valid ids is unaffected
    rc, out = b.call(capi, 2, m.n, w.ell, phi_d)
    assert rc == capi.RVE_OK and np.isfinite(out).all() and out[0] > 0
