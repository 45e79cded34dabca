"""Host logic of the calculation-mode driver (paper_1711_11418_gb300.driver):
the call sequence, the JSON records and the averaging over measurements,
with a stand-in context that records the calls (no GPU, no library)."""
import io
import json
import math

import numpy as np
import pytest

from paper_1711_11418_gb300 import driver


class FakeContext:
    def __init__(self, Ns=3):
        self.calls = []
        self.Ns = Ns
        self.k = 0

    def sample(self, n_warmup, n_samples, sweeps_between):
        self.calls.append(("sample", n_warmup, n_samples, sweeps_between))

    def measure(self, system=0):
        self.calls.append(("measure", system))
        return {"energy": -1.0 - 0.1 * len(self.calls), "variance": 0.5, "stderr_walkers": 0.01,
                "acceptance": 0.3, "max_drift": 1e-7, "n_flagged": 0, "n_recomputes": 2,
                "n_proposals": 10}

    def sr_step(self, dtau, shift_rel, shift_abs, solver=0, cg_eps=1e-10, cg_kmax=1000,
                system=0):
        self.calls.append(("sr_step", dtau, shift_rel, shift_abs, solver, system))
        return {"energy": -1.0, "norm_g": 0.2, "norm_dalpha": 0.01, "cg_iters": 3,
                "n_params": 5, "rel_residual": 1e-13, "fallback": 0}

    def measure_corr(self, system=0):
        self.calls.append(("measure_corr", system))
        self.k += 1
        c = np.zeros((6, self.Ns, self.Ns))
        c[0] = np.eye(self.Ns) * 0.5
        c[1] = np.eye(self.Ns) * 0.5
        c[2] = np.eye(self.Ns) * (1.0 + 0.2 * (self.k % 2))      # n^2 = n + 2D
        c[5] = self.k * np.ones((self.Ns, self.Ns))
        return c


def test_optimize_call_sequence_and_records():
    ctx = FakeContext()
    buf = io.StringIO()
    recs = driver.optimize(ctx, 3, 4, sweeps_between=2, n_warmup=7, dtau=0.02, solver=3,
                           log=buf)
    samples = [c for c in ctx.calls if c[0] == "sample"]
    assert samples == [("sample", 7, 4, 2), ("sample", 0, 4, 2), ("sample", 0, 4, 2)]
    assert [c[0] for c in ctx.calls] == ["sample", "measure", "sr_step"] * 3
    assert all(c[1] == 0.02 and c[4] == 3 for c in ctx.calls if c[0] == "sr_step")
    lines = [json.loads(l) for l in buf.getvalue().splitlines()]
    assert lines == recs and len(lines) == 3
    assert [r["step"] for r in lines] == [0, 1, 2]
    for r in lines:
        for k in ("energy", "stderr_walkers", "acceptance", "max_drift", "sr_norm_g",
                  "sr_cg_iters", "sr_fallback"):
            assert k in r


def test_measure_physics_mean_and_error(tmp_path):
    ctx = FakeContext()
    log = tmp_path / "m.jsonl"
    mean, err, recs = driver.measure_physics(ctx, 4, sweeps_between=3, n_warmup=5, log=str(log))
    assert ctx.calls[0] == ("sample", 5, 0, 0)
    # the chains advance by sweeps only: no sample rows are measured or replaced
    assert [c for c in ctx.calls[1:] if c[0] == "sample"] == [("sample", 3, 0, 0)] * 4
    assert [c[0] for c in ctx.calls[1:]] == ["sample", "measure_corr"] * 4
    # kind 5 takes the values 1, 2, 3, 4: mean 2.5, standard error of the mean
    np.testing.assert_allclose(mean[5], 2.5)
    np.testing.assert_allclose(err[5], np.std([1, 2, 3, 4], ddof=1) / 2.0)
    np.testing.assert_allclose(err[0], 0.0)
    lines = [json.loads(l) for l in log.read_text().splitlines()]
    assert len(lines) == 4 and lines == recs
    # D = (n^2 - n_up - n_dn) / 2 per site: 0.0 or 0.1 on alternate measurements
    assert [round(r["doublons_per_site"], 12) for r in lines] == [0.1, 0.0, 0.1, 0.0]


def test_measure_physics_single_measurement_has_no_error():
    mean, err, _ = driver.measure_physics(FakeContext(), 1)
    assert np.all(np.isnan(err))
    with pytest.raises(ValueError):
        driver.measure_physics(FakeContext(), 0)


def test_stand_in_matches_the_binding():
    """The driver calls Context methods by these names and keywords; the
    stand-in above must accept what the real binding accepts."""
    import inspect
    from paper_1711_11418_gb300 import vmc
    for name in ("sample", "measure", "sr_step", "measure_corr"):
        real = inspect.signature(getattr(vmc.Context, name)).parameters
        fake = inspect.signature(getattr(FakeContext, name)).parameters
        for p in fake:
            assert p in real, (name, p)
        for p, spec in real.items():
            if spec.default is inspect.Parameter.empty:
                assert p in fake, (name, p)
