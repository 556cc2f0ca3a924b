"""Parity of the CUDA path (through the C ABI) with the oracle, element by element.

Sizes: the 3-orbital workload at its full 2,000 sequences; the 5-orbital
workload at 384 walkers (several warps' worth of items per SM, ragged
lengths) for traces and ratios, plus the full 4,096-walker batch with a
sample checked against the oracle; the 7-orbital workload at 48 walkers.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0908_0681_gb300 import engine, kt, workloads  # noqa: E402
from tests import parity  # noqa: E402

PRECS = [kt.KT_FP64, kt.KT_FP32_KRYLOV]


def gpu_trace(model, seqs):
    s, l, st = engine.trace(model, engine.DeviceSeqs.from_host(seqs))
    return s.cpu().numpy(), l.cpu().numpy(), st.cpu().numpy()


def gpu_ratio(model, seqs, cur_s, cur_l, moves):
    s, l, st = engine.trace_ratio(model, engine.DeviceSeqs.from_host(seqs),
                                  torch.as_tensor(np.asarray(cur_s, np.int8), device="cuda"),
                                  torch.as_tensor(np.asarray(cur_l, np.float64), device="cuda"),
                                  engine.DeviceMoves.from_host(moves))
    return s.cpu().numpy(), l.cpu().numpy(), st.cpu().numpy()


@pytest.fixture(scope="module")
def three():
    w = workloads.three_orbital()
    seqs = workloads.generate_sequences(w, 2000, seed=1)
    o64, ox = parity.oracle_pair(w.model)
    cls, sx, lx = parity.oracle_traces(o64, ox, seqs)
    return w, seqs, o64, ox, cls, sx, lx


@pytest.fixture(scope="module")
def five():
    w = workloads.five_orbital()
    seqs = workloads.generate_sequences(w, 384, seed=1)
    o64, ox = parity.oracle_pair(w.model)
    cls, sx, lx = parity.oracle_traces(o64, ox, seqs)
    return w, seqs, o64, ox, cls, sx, lx


@pytest.mark.parametrize("prec", PRECS)
def test_three_orbital_traces(three, prec):
    w, seqs, o64, ox, cls, sx, lx = three
    m = engine.model_from_spec(w.model, precision=prec)
    s, l, st = gpu_trace(m, seqs)
    assert (st == kt.KT_OK).all()
    r = parity.compare(cls, sx, lx, s, l, prec, ox.nkept, w.model.beta * ox.E0, "3-orbital traces")
    assert r["regular"] > 200 and r["structural"] > 500
    # the oracle's per-component exponentials make symmetry zeros exact, and so do the
    # GPU's blocks: every exact zero of one is an exact zero of the other
    assert ((s == 0) == (cls == 0)).all()


@pytest.mark.parametrize("prec", PRECS)
def test_three_orbital_ratios(three, prec):
    w, seqs, o64, ox, cls, sx, lx = three
    moves = workloads.generate_moves(w, seqs, seed=1000)
    cur_s = np.where(cls == 2, sx, 0).astype(np.int8)
    ncls, nsx, nlx = parity.oracle_ratios(o64, ox, seqs, cur_s, lx, moves)
    m = engine.model_from_spec(w.model, precision=prec)
    s, lr, st = gpu_ratio(m, seqs, cur_s, lx, moves)
    reg = cls == 2
    assert (st[~reg] == kt.KT_EZEROWEIGHT).all() and (s[~reg] == 0).all() and np.isnan(lr[~reg]).all()
    assert (st[reg] == kt.KT_OK).all()
    # ratio = T_new / T_cur with T_cur the oracle's: compare the new trace through logratio + cur
    idx = np.nonzero(reg)[0]
    r = parity.compare(ncls[idx], nsx[idx] * cur_s[idx], nlx[idx] - lx[idx], s[idx], lr[idx], prec, ox.nkept,
                       w.model.beta * ox.E0 + lx[idx], "3-orbital ratios")
    assert r["regular"] > 100


@pytest.mark.parametrize("prec", PRECS)
def test_five_orbital_traces(five, prec):
    w, seqs, o64, ox, cls, sx, lx = five
    m = engine.model_from_spec(w.model, precision=prec)
    s, l, st = gpu_trace(m, seqs)
    assert (st == kt.KT_OK).all(), np.unique(st, return_counts=True)
    r = parity.compare(cls, sx, lx, s, l, prec, ox.nkept, w.model.beta * ox.E0, "5-orbital traces")
    assert r["regular"] >= 0.95 * len(cls)


@pytest.mark.parametrize("prec", PRECS)
def test_five_orbital_ratios(five, prec):
    w, seqs, o64, ox, cls, sx, lx = five
    moves = workloads.generate_moves(w, seqs, seed=1001)
    ncls, nsx, nlx = parity.oracle_ratios(o64, ox, seqs, sx, lx, moves)
    m = engine.model_from_spec(w.model, precision=prec)
    s, lr, st = gpu_ratio(m, seqs, sx, lx, moves)
    assert (st == kt.KT_OK).all()
    parity.compare(ncls, nsx * sx, nlx - lx, s, lr, prec, ox.nkept, w.model.beta * ox.E0 + lx, "5-orbital ratios")


def test_five_orbital_ratio_end_to_end_fp32(five):
    """Ratios against the GPU's own current traces (as a sampler uses them), FP32 path:
    within parity.RATIO_RTOL of the oracle ratio (two FP32 traces, each within 1e-5, enter)."""
    w, seqs, o64, ox, cls, sx, lx = five
    moves = workloads.generate_moves(w, seqs, seed=1002)
    m = engine.model_from_spec(w.model, precision=kt.KT_FP32_KRYLOV)
    cs, cl, _ = gpu_trace(m, seqs)
    s, lr, st = gpu_ratio(m, seqs, cs, cl, moves)
    ncls, nsx, nlx = parity.oracle_ratios(o64, ox, seqs, sx, lx, moves)
    assert (st == kt.KT_OK).all()
    reg = ncls == 2
    assert (s[reg] == (nsx * sx)[reg]).all()
    err = np.abs(np.expm1(lr[reg] - (nlx - lx)[reg]))
    assert err.max() <= parity.RATIO_RTOL[kt.KT_FP32_KRYLOV], err.max()


def test_sector_blocks_agree(five):
    """Propagating in whole (n_up, n_dn) sectors (d up to 100) gives the same traces."""
    w, seqs, o64, ox, cls, sx, lx = five
    sub = seqs.subset(range(96))
    m = engine.model_from_spec(w.model, precision=kt.KT_FP64, flags=kt.KT_SECTOR_BLOCKS)
    assert kt.kt_model_query(m)["d_max"] == 100
    s, l, st = gpu_trace(m, sub)
    assert (st == kt.KT_OK).all()
    parity.compare(cls[:96], sx[:96], lx[:96], s, l, kt.KT_FP64, ox.nkept, w.model.beta * ox.E0, "sector blocks")


def test_density_only_model():
    w = workloads.three_orbital()
    seqs = workloads.generate_sequences(w, 400, seed=5)
    o64, ox = parity.oracle_pair(w.model, density_only=True)
    cls, sx, lx = parity.oracle_traces(o64, ox, seqs)
    for prec in PRECS:
        m = engine.model_from_spec(w.model, precision=prec, flags=kt.KT_DENSITY_ONLY)
        s, l, st = gpu_trace(m, seqs)
        assert (st == kt.KT_OK).all()
        parity.compare(cls, sx, lx, s, l, prec, ox.nkept, w.model.beta * ox.E0, "density only")


def test_untruncated_trace_three_orbital():
    """trunc_eps = 0 keeps all 64 states (N_tr = 64, many blocks per walker)."""
    w = workloads.three_orbital()
    seqs = workloads.generate_sequences(w, 200, seed=9)
    o64, ox = parity.oracle_pair(w.model, trunc_eps=0.0)
    cls, sx, lx = parity.oracle_traces(o64, ox, seqs)
    m = engine.model_from_spec(w.model, precision=kt.KT_FP64, trunc_eps=0.0)
    assert kt.kt_model_query(m)["n_kept"] == 64
    s, l, st = gpu_trace(m, seqs)
    assert (st == kt.KT_OK).all()
    parity.compare(cls, sx, lx, s, l, kt.KT_FP64, ox.nkept, w.model.beta * ox.E0, "untruncated")


def test_edge_cases():
    """Empty batch, empty sequences, ragged lengths, a maximal sequence, invalid input."""
    w = workloads.five_orbital()
    spec = w.model
    o64, ox = parity.oracle_pair(spec)
    m = engine.model_from_spec(spec, precision=kt.KT_FP64)
    # empty batch
    empty = workloads.Sequences(np.zeros(1, np.int32), np.zeros(0), np.zeros(0, np.uint8), np.zeros(0, np.uint8))
    s, l, st = gpu_trace(m, empty)
    assert len(s) == 0
    # ragged: K = 0, 2, ..., plus a maximal walker (40 pairs in every flavor)
    rng = np.random.default_rng(3)
    lists = [[]]
    for k in (1, 2, 3, 7, 40):
        spins = rng.integers(2, size=spec.n_orb)
        ops = []
        for f in range(2 * spec.n_orb):
            ts = np.sort(rng.uniform(0, spec.beta, 2 * k))
            occ = (f % 2) == spins[f // 2]
            for j, t in enumerate(ts):
                ops.append((float(t), f, (0 if occ else 1) if j % 2 == 0 else (1 if occ else 0)))
        ops.sort()
        lists.append(ops)
    offs = np.cumsum([0] + [len(x) for x in lists]).astype(np.int32)
    cat = [op for x in lists for op in x]
    seqs = workloads.Sequences(offs, np.array([o[0] for o in cat]), np.array([o[1] for o in cat], np.uint8),
                               np.array([o[2] for o in cat], np.uint8))
    assert offs[-1] - offs[-2] == 800
    cls, sx, lx = parity.oracle_traces(o64, ox, seqs)
    s, l, st = gpu_trace(m, seqs)
    assert (st == kt.KT_OK).all()
    parity.compare(cls, sx, lx, s, l, kt.KT_FP64, ox.nkept, spec.beta * ox.E0, "ragged")
    assert s[0] == 1 and abs(l[0] - (math.log(6) - spec.beta * ox.E0)) < 1e-9  # K = 0: N_tr e^{-beta E0}
    # invalid sequences
    bad = workloads.Sequences(np.array([0, 2, 4, 6], np.int32), np.array([2.0, 1.0, 1.0, spec.beta, 1.0, 2.0]),
                              np.array([0, 0, 0, 0, 99, 0], np.uint8), np.array([1, 0, 1, 0, 1, 0], np.uint8))
    s, l, st = gpu_trace(m, bad)
    assert (st == kt.KT_EINVAL).all() and (s == 0).all()


def test_invalid_moves():
    w = workloads.five_orbital()
    seqs = workloads.generate_sequences(w, 4, seed=2)
    m = engine.model_from_spec(w.model, precision=kt.KT_FP64)
    cs, cl, _ = gpu_trace(m, seqs)
    mv = workloads.generate_moves(w, seqs, seed=3)
    tau, fl, dg = seqs.walker(0)
    c_idx = int(np.nonzero(dg == 0)[0][0])
    mv.kind[:] = [1, 0, 2, 1]
    mv.flavor[:] = [(int(fl[c_idx]) + 1) % (2 * w.model.n_orb), 0, 0, 0]   # removal of an op of another flavor
    mv.rem_idx[:] = [c_idx, 0, 0, 10 ** 6]
    mv.t_dag[1], mv.t_ann[1] = -1.0, 3.0
    s, lr, st = gpu_ratio(m, seqs, cs, cl, mv)
    assert (st == kt.KT_EINVAL).all()
    # zero current weight
    mv2 = workloads.generate_moves(w, seqs, seed=4)
    s, lr, st = gpu_ratio(m, seqs, np.zeros(4, np.int8), cl, mv2)
    assert (st == kt.KT_EZEROWEIGHT).all() and (s == 0).all()


def _full_batch(prec, flags=0):
    """The benchmark's 4,096-walker batch in its launch configuration: GPU current traces,
    then ratios against them; the oracle (FP64 and its long-double twin) evaluates every
    walker's current and edited sequence."""
    w = workloads.five_orbital()
    seqs = workloads.generate_sequences(w, 4096, seed=1)
    moves = workloads.generate_moves(w, seqs, seed=1000)
    m = engine.model_from_spec(w.model, precision=prec, flags=flags)
    cs, cl, cst = gpu_trace(m, seqs)
    s, lr, st = gpu_ratio(m, seqs, cs, cl, moves)
    assert (cst == kt.KT_OK).all() and (st == kt.KT_OK).all()
    assert (cs != 0).all()
    o64, ox = parity.oracle_pair(w.model)
    cls, sx, lx = parity.oracle_traces(o64, ox, seqs)
    ncls, nsx, nlx = parity.oracle_ratios(o64, ox, seqs, sx, lx, moves)
    return w, ox, cs, cl, s, lr, cls, sx, lx, ncls, nsx, nlx


@pytest.mark.parametrize("prec", PRECS)
def test_full_batch_every_walker(prec):
    """Every walker of the benchmark batch: traces within RTOL of the oracle, and the ratios a
    sampler forms from two of the path's own traces within RATIO_RTOL, signs exact."""
    w, ox, cs, cl, s, lr, cls, sx, lx, ncls, nsx, nlx = _full_batch(prec)
    r = parity.compare(cls, sx, lx, cs, cl, prec, ox.nkept, w.model.beta * ox.E0, "full batch traces")
    assert r["regular"] == 4096
    reg = ncls == 2
    assert (s[reg] == (nsx * sx)[reg]).all() and (s[ncls == 0] == 0).all()
    err = np.abs(np.expm1(lr[reg] - (nlx - lx)[reg]))
    assert err.max() <= parity.RATIO_RTOL[prec], err.max()


def test_full_batch_fp64_tridiagonal_ratios_within_1e5():
    """KT_FP32_TRIDIAG64 (FP32 Krylov vectors, tridiagonal exponential to FP64 accuracy):
    every ratio of the benchmark batch, formed end to end from two of the path's own traces,
    is within 1e-5 of the oracle's, and every trace within 5e-6."""
    w, ox, cs, cl, s, lr, cls, sx, lx, ncls, nsx, nlx = _full_batch(kt.KT_FP32_KRYLOV, kt.KT_FP32_TRIDIAG64)
    reg = cls == 2
    assert (cs[reg] == sx[reg]).all()
    assert np.abs(np.expm1(cl[reg] - lx[reg])).max() <= 5e-6
    reg = ncls == 2
    assert (s[reg] == (nsx * sx)[reg]).all()
    err = np.abs(np.expm1(lr[reg] - (nlx - lx)[reg]))
    assert err.max() <= 1e-5, err.max()


@pytest.mark.parametrize("prec", PRECS)
def test_every_tiling_matches_oracle(five, prec):
    """Each compiled lane-group size G gives oracle-parity results (and G = 4 and G = 32
    agree in sign)."""
    w, seqs, o64, ox, cls, sx, lx = five
    sub = seqs.subset(range(160))
    m = engine.model_from_spec(w.model, precision=prec)
    outs = {}
    for g in (4, 8, 16, 32):
        kt.kt_model_set_tiling(m, g)
        assert kt.kt_model_query(m)["group_lanes"] == g
        s, l, st = gpu_trace(m, sub)
        assert (st == kt.KT_OK).all()
        parity.compare(cls[:160], sx[:160], lx[:160], s, l, prec, ox.nkept, w.model.beta * ox.E0, f"G={g}")
        outs[g] = (s, l)
    assert (outs[4][0] == outs[32][0]).all()
    with pytest.raises(kt.KtError):
        kt.kt_model_set_tiling(m, 3)


def test_autotune_picks_a_compiled_tiling(five):
    w, seqs, o64, ox, cls, sx, lx = five
    m = engine.model_from_spec(w.model, precision=kt.KT_FP32_KRYLOV)
    d = engine.DeviceSeqs.from_host(seqs)
    n = seqs.n
    s = torch.empty(n, dtype=torch.int8, device="cuda")
    l = torch.empty(n, dtype=torch.float64, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    g = kt.kt_autotune(m, d.batch(), s, l, st, engine.workspace(m, n))
    assert g in (4, 8, 16, 32) and kt.kt_model_query(m)["group_lanes"] == g
    s2, l2, st2 = gpu_trace(m, seqs)
    parity.compare(cls, sx, lx, s2, l2, kt.KT_FP32_KRYLOV, ox.nkept, w.model.beta * ox.E0, "autotuned")


@pytest.fixture(scope="module")
def seven():
    w = workloads.seven_orbital()
    seqs = workloads.generate_sequences(w, 256, seed=1)   # the full seven-orbital batch
    o64, ox = parity.oracle_pair(w.model)
    cls, sx, lx = parity.oracle_traces(o64, ox, seqs)
    return w, seqs, o64, ox, cls, sx, lx


@pytest.mark.parametrize("prec", PRECS)
def test_seven_orbital_traces_and_ratios(seven, prec):
    """7-orbital f-shell model (16,384 states, blocks up to 35 rows, N_tr = 63), the full batch
    of 256 walkers: traces, ratios against the oracle's current traces (RTOL) and ratios
    against the path's own current traces (RATIO_RTOL)."""
    w, seqs, o64, ox, cls, sx, lx = seven
    m = engine.model_from_spec(w.model, precision=prec)
    info = kt.kt_model_query(m)
    assert info["n_kept"] == ox.nkept == 63 and info["d_max"] == 35
    s, l, st = gpu_trace(m, seqs)
    assert (st == kt.KT_OK).all(), np.unique(st, return_counts=True)
    r = parity.compare(cls, sx, lx, s, l, prec, ox.nkept, w.model.beta * ox.E0, "7-orbital traces")
    assert r["regular"] >= 0.9 * len(cls)
    moves = workloads.generate_moves(w, seqs, seed=1000)
    cur_s = np.where(cls == 2, sx, 0).astype(np.int8)
    ncls, nsx, nlx = parity.oracle_ratios(o64, ox, seqs, cur_s, lx, moves)
    rs, rl, rst = gpu_ratio(m, seqs, cur_s, lx, moves)
    reg = cls == 2
    assert (rst[reg] == kt.KT_OK).all()
    idx = np.nonzero(reg)[0]
    parity.compare(ncls[idx], nsx[idx] * cur_s[idx], nlx[idx] - lx[idx], rs[idx], rl[idx], prec, ox.nkept,
                   w.model.beta * ox.E0 + lx[idx], "7-orbital ratios")
    # as a sampler forms them: against the path's own current traces
    es, el, est = gpu_ratio(m, seqs, s, l, moves)
    both = reg & (ncls == 2)
    assert (est[reg] == kt.KT_OK).all() and (es[both] == (nsx * sx)[both]).all()
    err = np.abs(np.expm1(el[both] - (nlx - lx)[both]))
    assert err.max() <= parity.RATIO_RTOL[prec], err.max()


def test_seven_orbital_energy_window_1e4():
    """The seven-orbital model with the wider truncation threshold trunc_eps = 1e-4 (Sec. IV.C's
    energy window): fewer kept multiplets, the same parity bar for traces and ratios."""
    w = workloads.seven_orbital(trunc_eps=1e-4)
    seqs = workloads.generate_sequences(w, 48, seed=2)
    o64, ox = parity.oracle_pair(w.model)
    cls, sx, lx = parity.oracle_traces(o64, ox, seqs)
    m = engine.model_from_spec(w.model, precision=kt.KT_FP32_KRYLOV)
    info = kt.kt_model_query(m)
    assert info["n_kept"] == ox.nkept < 63
    s, l, st = gpu_trace(m, seqs)
    assert (st == kt.KT_OK).all(), np.unique(st, return_counts=True)
    parity.compare(cls, sx, lx, s, l, kt.KT_FP32_KRYLOV, ox.nkept, w.model.beta * ox.E0, "7-orbital 1e-4 traces")
    moves = workloads.generate_moves(w, seqs, seed=1001)
    cur_s = np.where(cls == 2, sx, 0).astype(np.int8)
    ncls, nsx, nlx = parity.oracle_ratios(o64, ox, seqs, cur_s, lx, moves)
    rs, rl, rst = gpu_ratio(m, seqs, cur_s, lx, moves)
    idx = np.nonzero(cls == 2)[0]
    assert (rst[idx] == kt.KT_OK).all()
    parity.compare(ncls[idx], nsx[idx] * cur_s[idx], nlx[idx] - lx[idx], rs[idx], rl[idx], kt.KT_FP32_KRYLOV,
                   ox.nkept, w.model.beta * ox.E0 + lx[idx], "7-orbital 1e-4 ratios")


@pytest.mark.parametrize("prec", PRECS)
def test_repeated_evaluations_are_bitwise_identical(prec):
    """The full five-orbital batch (4,096 walkers) evaluated four times, with other work
    between the calls: signs, log-ratios and statuses must be bit for bit the same (no
    result may depend on which unit of an item finishes first or on what a warp slot held
    before)."""
    w = workloads.five_orbital()
    seqs = workloads.generate_sequences(w, 4096, seed=1)
    m = engine.model_from_spec(w.model, precision=prec)
    d = engine.DeviceSeqs.from_host(seqs)
    cs, cl, cst = engine.trace(m, d)
    assert int((cst != 0).sum()) == 0
    mv = engine.DeviceMoves.from_host(workloads.generate_moves(w, seqs, seed=1003))
    ref = None
    for k in range(4):
        if k % 2:
            engine.trace(m, engine.DeviceSeqs.from_host(seqs.subset(list(range(0, 4096, 3)))))
        out = [t.cpu().numpy() for t in engine.trace_ratio(m, d, cs, cl, mv)]
        if ref is None:
            ref = out
            assert (out[2] == kt.KT_OK).all(), np.unique(out[2], return_counts=True)
        else:
            for a, b in zip(ref, out):
                assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), k
