"""Shared helpers of the parity tests: oracle <-> library field conversions."""
import numpy as np

import synth
from oracle import solver as S

PAIRS = {2: [(0, 0), (1, 1), (0, 1)], 3: [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]}


def sym_components(T, dim):
    """(d, d, *grid) tensor -> (ns, *grid) components xx, yy, [zz, yz, xz], xy (tensor shear)."""
    S_ = 0.5 * (T + np.swapaxes(T, 0, 1))
    return np.stack([S_[i, j] for (i, j) in PAIRS[dim]])


def tensor_from_components(c, dim):
    d = dim
    out = np.zeros((d, d) + c.shape[1:])
    for k, (i, j) in enumerate(PAIRS[dim]):
        out[i, j] = c[k]
        out[j, i] = c[k]
    return out


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    den = max(np.linalg.norm(b), 1e-300)
    return float(np.linalg.norm(a - b) / den)


def oracle_model(w, **kw):
    return S.Model(w.micro, S.params_from_workload(w, **kw))


def parity_workloads():
    return synth.small_cases()
