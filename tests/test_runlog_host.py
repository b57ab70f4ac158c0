"""Host-side run driver and its per-increment JSON-lines log (no GPU: a scripted stand-in RVE)."""
import io
import json

from paper_2508_07424_gb300 import runlog


class FakeRve:
    """Returns scripted step results like Rve.step; fractures at increment ``f``."""

    def __init__(self, f):
        self.f, self.n = f, 0

    def step(self, dtau):
        self.n += 1
        return {"n": self.n, "E": 0.1 * self.n, "Sigma": 1.0 / self.n, "D": dtau * self.n, "Emec": 0.0,
                "T": 0.5 * self.n, "Gamma": 0.2 * self.n, "tau": dtau * self.n, "mech_iters": 3,
                "dmg_iters": 4, "root_evals": 2, "stag_iters": 1, "fractured": int(self.n >= self.f),
                "stag_err": 1e-9, "flags": 0, "G_inst": float("nan") if self.n == 1 else 2.5}

    def toughness(self):
        return 1.25

    def toughness_functional(self):
        return 1.5


def test_run_logs_every_increment_and_a_summary():
    buf = io.StringIO()
    ticks = iter(range(100))
    s = runlog.run_to_fracture(FakeRve(4), 0.5, 10, log=buf, clock=lambda: float(next(ticks)))
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert [x["n"] for x in lines[:-1]] == [1, 2, 3, 4]
    assert lines[0]["G_inst"] is None                     # NaN becomes null: the log stays JSON
    assert lines[1]["G_inst"] == 2.5 and lines[3]["fractured"] == 1
    assert all(a["wall_s"] < b["wall_s"] for a, b in zip(lines[:-2], lines[1:-1]))
    assert lines[-1] == s and s["summary"] and s["fractured"] and s["increments"] == 4
    assert s["toughness"] == 1.25 and s["toughness_functional"] == 1.5


def test_run_stops_at_the_cap_without_fracture(tmp_path):
    path = tmp_path / "run.jsonl"
    s = runlog.run_to_fracture(FakeRve(100), 0.5, 3, log=str(path))
    lines = path.read_text().splitlines()
    assert len(lines) == 4 and not s["fractured"] and s["toughness"] is None
