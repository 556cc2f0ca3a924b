"""Parity of kt_measure (observables at tau = beta/2) with the oracle, element by element.

Expected values: oracle.measure in long double (the FP64 oracle decides which
entries are well conditioned: where FP64 and long double differ by more than 1e-8
the exact value is fixed by a symmetry beyond the blocks and only |GPU - ext| <=
ZERO_ATOL is asked). Tolerance on <O> = T_O / T, absolute, for walkers whose trace
is regular: the item weights carry the trace tolerance (1e-10 FP64, 1e-5 FP32) and
the per-row products of the two half vectors add the working precision, so with
values in [0, 1] and items of one sign |error| <= 2 rtol + d 2^-24: 1e-9 for the
FP64 path, 3e-5 for the FP32-Krylov path.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle.oracle import measure as oracle_measure  # noqa: E402
from paper_0908_0681_gb300 import engine, kt, workloads  # noqa: E402
from tests import parity  # noqa: E402

ATOL = {kt.KT_FP64: 1e-9, kt.KT_FP32_KRYLOV: 3e-5}
ZERO_ATOL = {kt.KT_FP64: 1e-6, kt.KT_FP32_KRYLOV: 1e-4}
PRECS = [kt.KT_FP64, kt.KT_FP32_KRYLOV]


def gpu_measure(model, seqs):
    s, l, obs, st = engine.measure(model, engine.DeviceSeqs.from_host(seqs))
    return s.cpu().numpy(), l.cpu().numpy(), obs.cpu().numpy(), st.cpu().numpy()


def check(spec, seqs, prec, label, density_only=False, min_regular=1):
    o64, ox = parity.oracle_pair(spec, density_only=density_only)
    sb = parity.seqbatch(seqs)
    v64, s64, l64 = oracle_measure(o64, sb)
    vx, sx, lx = oracle_measure(ox, sb)
    cls, _, _ = parity.oracle_traces(o64, ox, seqs)
    m = engine.model_from_spec(spec, precision=prec, flags=kt.KT_DENSITY_ONLY if density_only else 0)
    s, l, obs, st = gpu_measure(m, seqs)
    assert (st == kt.KT_OK).all(), (label, np.unique(st))
    # the trace itself as kt_trace
    parity.compare(cls, sx, lx, s, l, prec, ox.nkept, spec.beta * ox.E0, label)
    reg = cls == 2
    assert reg.sum() >= min_regular, label
    assert np.isnan(obs[s == 0]).all(), label
    known = reg[:, None] & np.isfinite(vx)     # the oracle skips S^2 beyond five orbitals
    good = known & (np.abs(v64 - vx) <= 1e-8)
    ill = known & ~good
    err = np.abs(obs - vx)
    assert (err[good] <= ATOL[prec]).all(), (label, float(err[good].max()), np.argwhere(err > ATOL[prec])[:5])
    if ill.any():
        assert (err[ill] <= ZERO_ATOL[prec]).all(), (label, float(err[ill].max()))
    return float(err[good].max()) if good.any() else 0.0


@pytest.mark.parametrize("prec", PRECS)
def test_three_orbital_measure(prec):
    w = workloads.three_orbital()
    seqs = workloads.generate_sequences(w, 2000, seed=1)
    check(w.model, seqs, prec, "three_orbital", min_regular=300)


@pytest.mark.parametrize("prec", PRECS)
def test_five_orbital_measure(prec):
    w = workloads.five_orbital()
    seqs = workloads.generate_sequences(w, 128, seed=3)
    check(w.model, seqs, prec, "five_orbital", min_regular=100)


def test_five_orbital_density_only_measure():
    w = workloads.five_orbital()
    seqs = workloads.generate_sequences(w, 64, seed=4)
    check(w.model, seqs, kt.KT_FP64, "five_orbital density-only", density_only=True)


def test_seven_orbital_measure():
    w = workloads.seven_orbital()
    seqs = workloads.generate_sequences(w, 16, seed=5)
    check(w.model, seqs, kt.KT_FP32_KRYLOV, "seven_orbital", min_regular=8)


@pytest.mark.parametrize("prec", PRECS)
def test_measure_split_edge_cases(prec):
    """Empty sequences, every operator before beta/2, every operator after it, one
    straddling pair, an unbalanced sequence (zero trace: NaN), and the kept multiplet
    alone (n_f = 1/2, no double occupancy, S^2 = 35/4)."""
    w = workloads.five_orbital()
    spec = w.model
    b = spec.beta
    rng = np.random.default_rng(8)
    spins = rng.integers(2, size=spec.n_orb)

    def occupied_pairs(lo, hi, k):
        ops = []
        for f in range(2 * spec.n_orb):
            ts = np.sort(rng.uniform(lo, hi, 2 * k))
            occ = (f % 2) == spins[f // 2]
            for j, t in enumerate(ts):
                ops.append((float(t), f, (0 if occ else 1) if j % 2 == 0 else (1 if occ else 0)))
        return sorted(ops)

    lists = [[], occupied_pairs(0.0, 0.5 * b - 1e-3, 2), occupied_pairs(0.5 * b + 1e-3, b - 1e-3, 2),
             [(0.3 * b, 0, 1 - int(spins[0] == 0)), (0.7 * b, 0, int(spins[0] == 0))], [(0.2 * b, 3, 1)],
             occupied_pairs(0.0, b - 1e-3, 1)]
    offs = np.cumsum([0] + [len(x) for x in lists]).astype(np.int32)
    cat = [op for x in lists for op in x]
    seqs = workloads.Sequences(offs, np.array([o[0] for o in cat]), np.array([o[1] for o in cat], np.uint8),
                               np.array([o[2] for o in cat], np.uint8))
    check(spec, seqs, prec, "edge cases")
    m = engine.model_from_spec(spec, precision=prec)
    s, l, obs, st = gpu_measure(m, seqs)
    lay = engine.measure_layout(spec.n_orb)
    assert np.allclose(obs[0, lay["n"]], 0.5, atol=ATOL[prec]) and np.allclose(obs[0, lay["docc"]], 0, atol=ATOL[prec])
    assert abs(obs[0, lay["S2"]][0] - 8.75) < 10 * ATOL[prec]          # the S = 5/2 sextet
    assert s[4] == 0 and np.isnan(obs[4]).all()


def test_measure_workspace_rules():
    w = workloads.three_orbital()
    seqs = workloads.generate_sequences(w, 8, seed=1)
    m = engine.model_from_spec(w.model, precision=kt.KT_FP64)
    d = engine.DeviceSeqs.from_host(seqs)
    small = engine.workspace(m, seqs.n)   # the trace workspace lacks the measurement regions
    assert kt.kt_measure_workspace_size(m, seqs.n) > kt.kt_workspace_size(m, seqs.n)
    n_orb = w.model.n_orb
    out = [torch.empty(seqs.n, dtype=t, device="cuda") for t in (torch.int8, torch.float64)]
    obs = torch.empty((seqs.n, kt.measure_nobs(n_orb)), dtype=torch.float64, device="cuda")
    st = torch.empty(seqs.n, dtype=torch.int32, device="cuda")
    with pytest.raises(kt.KtError):
        kt.kt_measure(m, d.batch(), out[0], out[1], obs, st, None, small)
    with pytest.raises(kt.KtError):
        kt.kt_measure(m, d.batch(), out[0], out[1], None, st, None, small)
