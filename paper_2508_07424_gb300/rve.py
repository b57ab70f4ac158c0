"""numpy-facing wrapper of one RVE handle (marshalling only; every step runs in the CUDA library)."""
import ctypes as C

import numpy as np

from . import capi

_FIELD_TENSOR = {capi.RVE_FIELD_EPS, capi.RVE_FIELD_SIGMA, capi.RVE_FIELD_FLUCT1}


def make_config(dim, n, ell, k_res=1e-6, split=0, precision=0, history=1, f=(0, 1, 0, 0, 0, 0), stream=None,
                **kw):
    cfg = capi.rve_config()
    capi.lib().rve_config_default(C.byref(cfg))
    cfg.dim = dim
    cfg.n[0], cfg.n[1], cfg.n[2] = n
    cfg.ell, cfg.k_res, cfg.split, cfg.precision, cfg.history = ell, k_res, split, precision, history
    for i in range(6):
        cfg.f[i] = f[i]
    for k, v in kw.items():
        setattr(cfg, k, v)
    cfg.stream = stream
    return cfg


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_micro(m):
    """rve_micro for a synth.Microstructure-like object; returns (struct, arrays to keep alive)."""
    keep = [np.ascontiguousarray(m.grain_id, np.int32).reshape(-1),
            np.ascontiguousarray(m.C_cubic, np.float64).reshape(-1),
            np.ascontiguousarray(m.R, np.float64).reshape(-1),
            np.ascontiguousarray(m.Gc, np.float64).reshape(-1),
            np.ascontiguousarray(m.cleave_n, np.float64).reshape(-1),
            np.ascontiguousarray(m.beta, np.float64).reshape(-1)]
    gid, Cc, R, Gc, cn, be = keep
    mi = capi.rve_micro()
    mi.grain_id = gid.ctypes.data_as(C.POINTER(C.c_int32))
    mi.n_grains = int(m.C_cubic.shape[0])
    mi.C_cubic, mi.R, mi.Gc, mi.cleave_n, mi.beta = _dptr(Cc), _dptr(R), _dptr(Gc), _dptr(cn), _dptr(be)
    cr = m.crack
    mi.crack_kind, mi.crack_row, mi.crack_x0, mi.crack_len = cr.kind, cr.row, cr.x0, cr.length
    mi.crack_phi_M, mi.crack_stiffness = cr.phi_M, cr.stiffness
    return mi, keep


def workload_config(w, **kw):
    m = w.micro
    return make_config(m.dim, m.n, w.ell, w.k_res, w.split, 0 if w.precision == "fp64" else 1, f=w.f, **kw)


class Rve:
    """One RVE resident on the GPU.

    ``micro`` is a :class:`synth.Microstructure`-like object (grain_id, C_cubic, R, Gc, cleave_n,
    beta, crack). Arrays are copied by the library.
    """

    def __init__(self, cfg):
        self.cfg = cfg
        self.h = capi.rve_handle()
        capi.check(capi.lib().rve_create(C.byref(cfg), C.byref(self.h)), "rve_create")
        nx, ny, nz = cfg.n[0], cfg.n[1], cfg.n[2]
        self.nvox = nx * ny * nz
        self.ns = 3 if cfg.dim == 2 else 6

    @classmethod
    def from_workload(cls, w, **kw):
        r = cls(workload_config(w, **kw))
        r.set_microstructure(w.micro)
        return r

    def set_microstructure(self, m):
        mi, self._keep = make_micro(m)
        capi.check(capi.lib().set_microstructure(self.h, C.byref(mi)), "set_microstructure")

    def step(self, dtau):
        out = capi.rve_step_result()
        capi.check(capi.lib().step_dissipation(self.h, dtau, C.byref(out)), "step_dissipation")
        return {k: getattr(out, k) for k, _ in out._fields_}

    def toughness(self):
        g = C.c_double()
        capi.check(capi.lib().effective_toughness(self.h, C.byref(g)), "effective_toughness")
        return g.value

    def toughness_functional(self):
        g = C.c_double()
        capi.check(capi.lib().effective_toughness_functional(self.h, C.byref(g)), "effective_toughness_functional")
        return g.value

    def get(self, field):
        n = self.nvox * (self.ns if field in _FIELD_TENSOR else 1)
        a = np.empty(n, np.float64)
        capi.check(capi.lib().rve_get_field(self.h, field, _dptr(a), n), "rve_get_field")
        nx, ny, nz = self.cfg.n[0], self.cfg.n[1], self.cfg.n[2]
        if field in _FIELD_TENSOR:
            return a.reshape(self.ns, nz, ny, nx)
        return a.reshape(nz, ny, nx)

    def set(self, field, arr):
        a = np.ascontiguousarray(arr, np.float64).reshape(-1)
        capi.check(capi.lib().rve_set_field(self.h, field, _dptr(a), a.size), "rve_set_field")

    def scalars(self):
        s = capi.rve_scalars()
        capi.check(capi.lib().rve_get_scalars(self.h, C.byref(s)), "rve_get_scalars")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def set_scalars(self, **kw):
        s = capi.rve_scalars()
        capi.check(capi.lib().rve_get_scalars(self.h, C.byref(s)), "rve_get_scalars")
        for k, v in kw.items():
            setattr(s, k, v)
        capi.check(capi.lib().rve_set_scalars(self.h, C.byref(s)), "rve_set_scalars")

    def mech_solve(self):
        it = C.c_int()
        capi.check(capi.lib().rve_mech_solve(self.h, C.byref(it)), "rve_mech_solve")
        return it.value

    def damage_solve(self, E):
        d, it = C.c_double(), C.c_int()
        capi.check(capi.lib().rve_damage_solve(self.h, E, C.byref(d), C.byref(it)), "rve_damage_solve")
        return d.value, it.value

    def dissipation(self, phi):
        a = np.ascontiguousarray(phi, np.float64).reshape(-1)
        d, g = C.c_double(), C.c_double()
        capi.check(capi.lib().rve_dissipation(self.h, _dptr(a), C.byref(d), C.byref(g)), "rve_dissipation")
        return d.value, g.value

    def save(self):
        n = C.c_size_t()
        capi.check(capi.lib().rve_save(self.h, None, C.byref(n)), "rve_save")
        buf = C.create_string_buffer(n.value)
        capi.check(capi.lib().rve_save(self.h, buf, C.byref(n)), "rve_save")
        return buf.raw

    def load(self, blob):
        capi.check(capi.lib().rve_load(self.h, blob, len(blob)), "rve_load")

    def timing(self, on=None, kind=0):
        if on is not None:
            capi.check(capi.lib().rve_timing_enable(self.h, int(on)), "rve_timing_enable")
            return None
        ms, n, b = C.c_double(), C.c_long(), C.c_double()
        capi.check(capi.lib().rve_timing_get(self.h, kind, C.byref(ms), C.byref(n), C.byref(b)), "rve_timing_get")
        return ms.value, n.value, b.value

    def timing_kinds(self):
        """Per kernel class recorded since timing was enabled: {name: (ms, launches, bytes per
        launch, FFT flops per launch)}."""
        out = {}
        for kind, name in ((0, "projection_pass"), (1, "k_axis"), (2, "k_x_fwd"), (3, "k_x_inv"), (4, "k_x_mid"),
                           (5, "k_pointwise"), (6, "all"), (7, "fp64_residual"), (8, "cg_x_fwd"), (9, "cg_x_inv")):
            ms, n, b, f = C.c_double(), C.c_long(), C.c_double(), C.c_double()
            capi.check(capi.lib().rve_timing_get_flops(self.h, kind, C.byref(ms), C.byref(n), C.byref(b), C.byref(f)),
                       "rve_timing_get_flops")
            out[name] = (ms.value, n.value, b.value, f.value)
        return out

    def launches(self):
        return capi.lib().rve_launch_count(self.h)

    def tiles(self):
        y, z = C.c_int(), C.c_int()
        capi.check(capi.lib().rve_tile_config(self.h, C.byref(y), C.byref(z)), "rve_tile_config")
        return y.value, z.value

    def close(self):
        if self.h:
            capi.lib().rve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_batch(rves, dtaus):
    """One increment of each Rve in lockstep (rve_step_batch): the solves of all of them are
    launched together, one kernel launch per pass. Returns the step records; raises on the first
    failing status (the other increments are committed all the same)."""
    n = len(rves)
    hs = (capi.rve_handle * n)(*[r.h for r in rves])
    dt = (C.c_double * n)(*[float(d) for d in dtaus])
    out = (capi.rve_step_result * n)()
    capi.check(capi.lib().rve_step_batch(hs, n, dt, out), "rve_step_batch")
    return [{k: getattr(out[i], k) for k, _ in out[i]._fields_} for i in range(n)]
