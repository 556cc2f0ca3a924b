"""Trace ratios from cached partial states (kt_ratio_cache_*) against the oracle and
against the from-scratch kt_trace_ratio, element by element.

One build of the cache serves several rounds of proposed updates against the same
current configurations. The cached ratio propagates only the edited window between
cached states, so it is the same trace ratio up to rounding: the oracle bars of the
parity tests apply (1e-10 relative FP64, 1e-5 FP32, structural zeros exact), and the
two GPU evaluations differ by at most the sum of their errors. A short cache length
(24 operators) makes most walkers fall back to the full evaluation.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0908_0681_gb300 import engine, kt, workloads  # noqa: E402
from tests import parity  # noqa: E402

PRECS = [kt.KT_FP64, kt.KT_FP32_KRYLOV]
# two evaluations of one ratio, each within RTOL of the exact value, differ by at most about 2 RTOL
PAIR_TOL = parity.RATIO_RTOL


def dev(a, dt):
    return torch.as_tensor(np.asarray(a, dt), device="cuda")


def both_ratios(model, seqs, cur_s, cur_l, moves_list, max_ops):
    d = engine.DeviceSeqs.from_host(seqs)
    cache = engine.RatioCache(model, seqs.n, max_ops)
    cache.build(d)
    cs, cl = dev(cur_s, np.int8), dev(cur_l, np.float64)
    out = []
    for mv in moves_list:
        dm = engine.DeviceMoves.from_host(mv)
        c = [t.cpu().numpy() for t in cache.ratio(d, cs, cl, dm)]
        f = [t.cpu().numpy() for t in engine.trace_ratio(model, d, cs, cl, dm)]
        out.append((c, f))
    return out


def check_round(w, seqs, o64, ox, cls, sx, lx, prec, mv, cached, full, label):
    cur_s = np.where(cls == 2, sx, 0).astype(np.int8)
    reg = cls == 2
    cs, cl, cst = cached
    fs, fl, fst = full
    assert (cst[reg] == kt.KT_OK).all() and (fst[reg] == kt.KT_OK).all(), label
    assert (cst[~reg] == kt.KT_EZEROWEIGHT).all(), label
    ncls, nsx, nlx = parity.oracle_ratios(o64, ox, seqs, cur_s, lx, mv)
    both = reg & (ncls == 2)
    assert (cs[both] == fs[both]).all(), label
    d = np.abs(cl[both] - fl[both])
    assert d.max(initial=0.0) <= PAIR_TOL[prec], (label, float(d.max(initial=0.0)))
    zero = reg & (ncls == 0)
    assert (cs[zero] == 0).all() and (fs[zero] == 0).all(), label
    idx = np.nonzero(reg)[0]
    parity.compare(ncls[idx], nsx[idx] * cur_s[idx], nlx[idx] - lx[idx], cs[idx], cl[idx], prec, ox.nkept,
                   w.model.beta * ox.E0 + lx[idx], label)


@pytest.fixture(scope="module")
def three():
    w = workloads.three_orbital()
    seqs = workloads.generate_sequences(w, 600, seed=5)
    o64, ox = parity.oracle_pair(w.model)
    cls, sx, lx = parity.oracle_traces(o64, ox, seqs)
    return w, seqs, o64, ox, cls, sx, lx


@pytest.fixture(scope="module")
def five():
    w = workloads.five_orbital()
    seqs = workloads.generate_sequences(w, 192, seed=6)
    o64, ox = parity.oracle_pair(w.model)
    cls, sx, lx = parity.oracle_traces(o64, ox, seqs)
    return w, seqs, o64, ox, cls, sx, lx


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("max_ops", [512, 24])
def test_three_orbital_cached_ratios(three, prec, max_ops):
    w, seqs, o64, ox, cls, sx, lx = three
    m = engine.model_from_spec(w.model, precision=prec)
    cur_s = np.where(cls == 2, sx, 0).astype(np.int8)
    moves = [workloads.generate_moves(w, seqs, seed=900 + r) for r in range(3)]
    for r, (c, f) in enumerate(both_ratios(m, seqs, cur_s, lx, moves, max_ops)):
        check_round(w, seqs, o64, ox, cls, sx, lx, prec, moves[r], c, f, f"3-orbital round {r} cache {max_ops}")


@pytest.mark.parametrize("prec", PRECS)
def test_five_orbital_cached_ratios(five, prec):
    w, seqs, o64, ox, cls, sx, lx = five
    m = engine.model_from_spec(w.model, precision=prec)
    cur_s = np.where(cls == 2, sx, 0).astype(np.int8)
    moves = [workloads.generate_moves(w, seqs, seed=950 + r) for r in range(2)]
    for r, (c, f) in enumerate(both_ratios(m, seqs, cur_s, lx, moves, 512)):
        check_round(w, seqs, o64, ox, cls, sx, lx, prec, moves[r], c, f, f"5-orbital round {r}")


def test_cached_window_edge_cases(five):
    """Updates whose window touches the ends of the sequence: an insertion that wraps
    around beta, insertions at the very start and end, the removal of two adjacent
    operators (an empty window), and a removal that wraps (the pair's second operator
    is the first of the sequence)."""
    w, seqs, o64, ox, cls, sx, lx = five
    b = w.model.beta
    m = engine.model_from_spec(w.model, precision=kt.KT_FP64)
    mv = workloads.generate_moves(w, seqs, seed=977)
    n = seqs.n
    for i in range(n):
        tau, fl, dg = seqs.walker(i)
        case = i % 5
        f = int(fl[0]) if len(fl) else 0
        if case == 0:    # wrapping insertion
            mv.kind[i], mv.flavor[i], mv.t_dag[i], mv.t_ann[i] = 0, f, b - 1e-3, 1e-3
        elif case == 1:  # both operators before the first existing one
            t0 = tau[0] if len(tau) else b
            mv.kind[i], mv.flavor[i], mv.t_dag[i], mv.t_ann[i] = 0, f, 0.25 * t0, 0.5 * t0
        elif case == 2:  # both after the last one
            t1 = tau[-1] if len(tau) else 0.0
            mv.kind[i], mv.flavor[i], mv.t_dag[i], mv.t_ann[i] = 0, f, t1 + 0.5 * (b - t1), t1 + 0.25 * (b - t1)
        elif case == 3:  # adjacent pair
            adj = [j for j in range(len(fl) - 1) if fl[j] == fl[j + 1] and dg[j] != dg[j + 1]]
            if adj:
                mv.kind[i], mv.flavor[i], mv.rem_idx[i] = 1, int(fl[adj[0]]), adj[0]
        else:            # the last operator of a flavor with its cyclic successor (wraps)
            g = int(fl[-1])
            last = max(j for j in range(len(fl)) if fl[j] == g)
            firsts = [j for j in range(len(fl)) if fl[j] == g]
            if len(firsts) >= 2 and dg[firsts[0]] != dg[last]:
                mv.kind[i], mv.flavor[i], mv.rem_idx[i] = 1, g, last
    cur_s = np.where(cls == 2, sx, 0).astype(np.int8)
    (c, f), = both_ratios(m, seqs, cur_s, lx, [mv], 512)
    check_round(w, seqs, o64, ox, cls, sx, lx, kt.KT_FP64, mv, c, f, "window edge cases")


def test_rebuild_for_new_configurations(three):
    """One cache object rebuilt for other configurations gives their ratios."""
    w, seqs, o64, ox, cls, sx, lx = three
    m = engine.model_from_spec(w.model, precision=kt.KT_FP64)
    cache = engine.RatioCache(m, 200, 512)
    for part in (range(0, 200), range(200, 400)):
        sub = seqs.subset(list(part))
        c_sub, s_sub, l_sub = cls[list(part)], sx[list(part)], lx[list(part)]
        d = engine.DeviceSeqs.from_host(sub)
        cache.build(d)
        mv = workloads.generate_moves(w, sub, seed=31)
        cur_s = np.where(c_sub == 2, s_sub, 0).astype(np.int8)
        res = [t.cpu().numpy() for t in cache.ratio(d, dev(cur_s, np.int8), dev(l_sub, np.float64),
                                                      engine.DeviceMoves.from_host(mv))]
        full = [t.cpu().numpy() for t in engine.trace_ratio(m, d, dev(cur_s, np.int8), dev(l_sub, np.float64),
                                                             engine.DeviceMoves.from_host(mv))]
        check_round(w, sub, o64, ox, c_sub, s_sub, l_sub, kt.KT_FP64, mv, res, full, "rebuild")


@pytest.mark.parametrize("prec", PRECS)
def test_seven_orbital_cached_ratios(prec):
    """36-row blocks (the 16-lane cached kernel): seven orbitals, N_tr = 63."""
    w = workloads.seven_orbital()
    seqs = workloads.generate_sequences(w, 48, seed=1)
    o64, ox = parity.oracle_pair(w.model)
    cls, sx, lx = parity.oracle_traces(o64, ox, seqs)
    m = engine.model_from_spec(w.model, precision=prec)
    cur_s = np.where(cls == 2, sx, 0).astype(np.int8)
    mv = workloads.generate_moves(w, seqs, seed=1000)
    (c, f), = both_ratios(m, seqs, cur_s, lx, [mv], 512)
    check_round(w, seqs, o64, ox, cls, sx, lx, prec, mv, c, f, "7-orbital cached")


def test_sector_blocks_cached_ratios(five):
    """Whole (n_up, n_dn) sectors (KT_SECTOR_BLOCKS, up to 100 rows: the 32-lane, 128-row
    cached kernel) give the same ratios."""
    w, seqs, o64, ox, cls, sx, lx = five
    m = engine.model_from_spec(w.model, precision=kt.KT_FP64, flags=kt.KT_SECTOR_BLOCKS)
    cur_s = np.where(cls == 2, sx, 0).astype(np.int8)
    sub = list(range(64))
    s2, c2, x2, l2 = seqs.subset(sub), cls[sub], sx[sub], lx[sub]
    mv = workloads.generate_moves(w, s2, seed=1001)
    (c, f), = both_ratios(m, s2, cur_s[sub], l2, [mv], 512)
    check_round(w, s2, o64, ox, c2, x2, l2, kt.KT_FP64, mv, c, f, "sector blocks cached")


def test_stale_lengths_fall_back_to_full_evaluation(three):
    """A cache built for other configurations: walkers whose length differs from the build
    are evaluated in full (correct ratios); the library cannot see other differences."""
    w, seqs, o64, ox, cls, sx, lx = three
    m = engine.model_from_spec(w.model, precision=kt.KT_FP64)
    a = seqs.subset(list(range(0, 200)))
    b = seqs.subset(list(range(200, 400)))
    lens_a, lens_b = np.diff(a.offsets), np.diff(b.offsets)
    cache = engine.RatioCache(m, 200, 512)
    cache.build(engine.DeviceSeqs.from_host(a))
    db = engine.DeviceSeqs.from_host(b)
    c_b, s_b, l_b = cls[200:400], sx[200:400], lx[200:400]
    cur_s = np.where(c_b == 2, s_b, 0).astype(np.int8)
    mv = workloads.generate_moves(w, b, seed=77)
    res = [t.cpu().numpy() for t in cache.ratio(db, dev(cur_s, np.int8), dev(l_b, np.float64),
                                                  engine.DeviceMoves.from_host(mv))]
    full = [t.cpu().numpy() for t in engine.trace_ratio(m, db, dev(cur_s, np.int8), dev(l_b, np.float64),
                                                         engine.DeviceMoves.from_host(mv))]
    diff = lens_a != lens_b
    assert diff.sum() >= 50
    ncls, nsx, nlx = parity.oracle_ratios(o64, ox, b, cur_s, l_b, mv)
    ok = diff & (c_b == 2) & (ncls == 2)
    zero = diff & (c_b == 2) & (ncls == 0)
    assert ok.sum() >= 10
    assert (res[0][ok] == full[0][ok]).all() and (res[0][zero] == 0).all()
    assert np.abs(res[1][ok] - full[1][ok]).max() <= 1e-10


@pytest.mark.parametrize("prec", PRECS)
def test_external_chain_with_propose_and_commit(prec):
    """An external Markov chain on the trace alone (accept when u < |T_new / T_old|) driven
    through kt_ratio_cache_propose / kt_ratio_cache_commit, its sequences edited on the host
    with the library's edit rules: every step's cached ratios equal kt_trace_ratio's on the
    same configurations (FP64 2e-10, FP32 2e-5), over many accepted moves."""
    from oracle.oracle import edit
    w = workloads.five_orbital()
    n = 64
    seqs = workloads.generate_sequences(w, n, seed=12)
    m = engine.model_from_spec(w.model, precision=prec)
    d = engine.DeviceSeqs.from_host(seqs)
    cs, cl, cst = engine.trace(m, d)
    assert (cs.cpu().numpy() != 0).all()
    cache = engine.RatioCache(m, n, 512)
    cache.build(d)
    rng = np.random.default_rng(3)
    ops = [list(zip(*[a.tolist() for a in seqs.walker(i)])) for i in range(n)]
    accepted_total = 0
    for step in range(40):
        cur = workloads.Sequences(np.concatenate([[0], np.cumsum([len(o) for o in ops])]).astype(np.int32),
                                  np.array([t for o in ops for (t, f, g) in o], np.float64),
                                  np.array([f for o in ops for (t, f, g) in o], np.uint8),
                                  np.array([g for o in ops for (t, f, g) in o], np.uint8))
        d = engine.DeviceSeqs.from_host(cur)
        mv = workloads.generate_moves(w, cur, seed=3000 + step)
        dm = engine.DeviceMoves.from_host(mv)
        c = [t.cpu().numpy() for t in cache.propose(d, cs, cl, dm)]
        f = [t.cpu().numpy() for t in engine.trace_ratio(m, d, cs, cl, dm)]
        ok = (c[2] == kt.KT_OK) & (f[2] == kt.KT_OK)
        assert (c[2] == f[2]).all(), step
        nz = ok & (f[0] != 0) & (c[0] != 0)
        assert (c[0][ok & (f[0] != 0)] == f[0][ok & (f[0] != 0)]).all(), step
        assert np.abs(c[1][nz] - f[1][nz]).max(initial=0.0) <= PAIR_TOL[prec], step
        acc = nz & (np.log(rng.uniform(size=n)) < f[1])
        accepted_total += int(acc.sum())
        cache.commit(torch.as_tensor(acc.astype(np.int8), device="cuda"), torch.as_tensor(c[2], device="cuda"))
        for i in np.nonzero(acc)[0]:
            ops[i] = edit(ops[i], int(mv.kind[i]), int(mv.flavor[i]), float(mv.t_dag[i]), float(mv.t_ann[i]),
                          int(mv.rem_idx[i]))
        cs = torch.as_tensor(np.where(acc, c[0] * cs.cpu().numpy(), cs.cpu().numpy()).astype(np.int8), device="cuda")
        cl = torch.as_tensor(np.where(acc, cl.cpu().numpy() + f[1], cl.cpu().numpy()), device="cuda")
    assert accepted_total >= 200


@pytest.mark.parametrize("prec", PRECS)
def test_full_batch_cached_ratios_sampled(prec):
    """The benchmark's 4,096-walker batch and moves, with ratios from the partial-state cache
    (the bench's cached_ratio configuration): every walker against the full GPU evaluation,
    and 48 sampled walkers one by one against the oracle."""
    w = workloads.five_orbital()
    seqs = workloads.generate_sequences(w, 4096, seed=1)
    moves = workloads.generate_moves(w, seqs, seed=1000)
    m = engine.model_from_spec(w.model, precision=prec)
    d = engine.DeviceSeqs.from_host(seqs)
    cs, cl, cst = engine.trace(m, d)
    assert (cst.cpu().numpy() == kt.KT_OK).all() and (cs.cpu().numpy() != 0).all()
    cache = engine.RatioCache(m, seqs.n, max_ops=512)
    cache.build(d)
    dm = engine.DeviceMoves.from_host(moves)
    c = [t.cpu().numpy() for t in cache.ratio(d, cs, cl, dm)]
    f = [t.cpu().numpy() for t in engine.trace_ratio(m, d, cs, cl, dm)]
    assert (c[2] == kt.KT_OK).all() and (f[2] == kt.KT_OK).all()
    assert (c[0] == f[0]).all()
    nz = c[0] != 0
    assert np.abs(c[1][nz] - f[1][nz]).max() <= PAIR_TOL[prec]
    idx = np.random.default_rng(1).choice(4096, 48, replace=False)
    sub = seqs.subset(idx)
    o64, ox = parity.oracle_pair(w.model)
    cls, sx, lx = parity.oracle_traces(o64, ox, sub)
    ncls, nsx, nlx = parity.oracle_ratios(o64, ox, sub, sx, lx, moves.subset(idx))
    reg = ncls == 2
    err = np.abs(np.expm1(c[1][idx][reg] - (nlx - lx)[reg]))
    assert err.max() <= parity.RATIO_RTOL[prec], err.max()
