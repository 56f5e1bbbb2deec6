"""The paper-experiment driver's bookkeeping on the CPU, with a stand-in simulation
(no GPU): step counts and record spacing, the energy-drift figure, the CSV and the
summary it writes."""
import csv
import json
import os

import pytest

from paper_2502_10640_gb300 import experiments


class FakeSim:
    """Records the calls; diagnostics follow a made-up trajectory."""
    instances = []

    def __init__(self, n, w, dt, eps, tune=None):
        self.n, self.dt, self.done = n, dt, 0
        self.pe_calls = []
        FakeSim.instances.append(self)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def load(self, pos):
        assert pos.shape == (self.n, 3)

    def step(self, k):
        assert k > 0
        self.done += k

    def get_option(self, key):
        return 1

    def diagnostics(self, with_pe=True):
        self.pe_calls.append(with_pe)
        t = self.done * self.dt
        d = {k: float(self.done + 1) for k in experiments.FIELDS}
        d["t"], d["step"] = t, self.done
        d["ke"] = 1.0 + t * 1e8            # kinetic energy grows ...
        d["pe"] = 3.0 - t * 1e8 + (self.done * 1e-9 if with_pe else 0.0)   # ... potential falls
        return d


@pytest.fixture
def fake(monkeypatch):
    FakeSim.instances.clear()
    monkeypatch.setattr(experiments.capi, "Simulation", FakeSim)
    return FakeSim


def test_run_lattice_steps_records_and_energy(fake):
    run = experiments.run_lattice(4, 1e-12, 1e-9, records=7)
    sim = fake.instances[-1]
    assert run["steps"] == 1000 and sim.done == 1000
    # first record, then blocks of 142 steps (the last one shorter) up to the end
    assert len(run["series"]["step"]) == 1 + 8 and run["series"]["step"][-1] == 1000
    assert sim.pe_calls[0] and sim.pe_calls[-1] and not any(sim.pe_calls[1:-1])
    assert run["resident"] is True
    assert run["energy_drift"] == pytest.approx((1000 * 1e-9) / 4.0)


def test_main_writes_csv_and_summary(fake, tmp_path):
    experiments.main(["--t-end", "1e-11", "--records", "3", "--only", "dt", "--out", str(tmp_path)])
    summary = json.load(open(os.path.join(tmp_path, "summary.json")))
    assert [r["dt"] for r in summary] == list(experiments.DT_SWEEP)
    assert all(r["sweep"] == "dt" and r["n"] == 16 ** 3 for r in summary)
    with open(os.path.join(tmp_path, summary[0]["file"])) as f:
        rows = list(csv.reader(f))
    assert rows[0] == list(experiments.FIELDS) and len(rows) >= 3
