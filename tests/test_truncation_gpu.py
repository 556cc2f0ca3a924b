"""Truncated and untruncated outer traces give the same physics at low temperature.

Sec. IV.A: keeping only the ground multiplet in the outer trace (N_tr = 4 for the
three-orbital model at half filling) is legitimate when the temperature is below about
1% of the bandwidth; measurements taken at beta/2 are least affected. Here the
three-orbital model with the semicircular bath of bandwidth 4 runs at beta = 50
(T = 0.5% of the bandwidth) once with the ground multiplet only and once with every
eigenstate in the outer trace; double occupancy at beta/2, the densities and the mean
expansion order must agree within 5 standard errors over independent chains.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0908_0681_gb300 import engine, kt, workloads  # noqa: E402


def run(trunc_eps, nw=512, therm=1500, steps=2500, seed=4):
    w = workloads.three_orbital()
    spec = workloads.ModelSpec(w.model.n_orb, w.model.U, w.model.J, mu=w.model.mu, delta=w.model.delta, beta=50.0)
    model = engine.model_from_spec(spec, precision=kt.KT_FP64, trunc_eps=trunc_eps)
    n_kept = kt.kt_model_query(model)["n_kept"]
    table = workloads.semicircular_hybridization(spec.beta, 6, n_tau=2000)
    sw = engine.Sweep(model, table, spec.beta, nw, k_cap=64, n_bins=20, measure_obs=True)
    g = torch.Generator(device="cuda").manual_seed(seed)
    sw.run(torch.rand((therm, nw, 6), dtype=torch.float64, device="cuda", generator=g))
    sw.reset_accumulators()
    sw.run(torch.rand((steps, nw, 6), dtype=torch.float64, device="cuda", generator=g), meas_every=10)
    a = {k: v.cpu().numpy() for k, v in sw.accumulators().items()}
    assert sw.counters()["trace_errors"] == 0
    obs = a["obs_sum"] / a["sign_sum"][:, None]
    return n_kept, {"docc": obs[:, 6:9].mean(1), "n": obs[:, :6].mean(1), "order": a["order_sum"].sum(1) / a["sign_sum"]}


def test_ground_multiplet_truncation_at_low_temperature():
    k_tr, tr = run(1e-10)
    k_all, full = run(0.0)
    assert k_tr == 4 and k_all == 64
    for name in ("docc", "n", "order"):
        a, b = tr[name], full[name]
        se = math.sqrt(a.var(ddof=1) / len(a) + b.var(ddof=1) / len(b))
        assert abs(a.mean() - b.mean()) < 5 * se + 1e-12, (name, a.mean(), b.mean(), se)
