"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test fixes one part of the oracle to something independent: numbers
printed in the paper (tests/golden/paper_degeneracies.json), closed forms,
invariants, library routines, or a full-space brute force (tests/brute.py).
"""
import json
import math
import os
from itertools import combinations

import numpy as np
import pytest

from oracle.oracle import Model, Params, SeqBatch, classify, edit, ratio
from tests import brute

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_degeneracies.json")))


def mu_half(n, U, J):
    # Sec. IV.B: mu_half = (n - 1/2) U - (n - 1) 5J/2
    return (n - 0.5) * U - (n - 1) * 2.5 * J


def sector_energies(m: Model, N: int):
    out = []
    n = m.p.n_orb
    for nu in range(n + 1):
        nd = N - nu
        if 0 <= nd <= n:
            out.extend(m.block(m.sector_index(nu, nd))[1].tolist())
    return np.sort(out)


# ---------------------------------------------------------------------------
# eigensolver and H_loc construction
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 5])
def test_eigensolver_matches_lapack_and_is_orthonormal(n):
    rng = np.random.default_rng(n)
    m = Model(Params(n, 4.0, 1.0, mu=3.0, delta=tuple(rng.uniform(-0.3, 0.3, n)), beta=5.0))
    for s in range(m.nsec):
        H, w, V = m.block(s)
        if len(w) == 0:
            continue
        assert np.allclose(H, H.T, atol=0)
        np.testing.assert_allclose(w, np.linalg.eigvalsh(H), atol=1e-12 * max(1, np.abs(w).max()))
        assert np.abs(H @ V - V * w).max() < 1e-11 * max(1, np.abs(w).max())
        assert np.abs(V.T @ V - np.eye(len(w))).max() < 1e-13


@pytest.mark.parametrize("n,density_only", [(2, False), (3, False), (3, True)])
def test_hamiltonian_matches_kronecker_brute_force(n, density_only):
    """Sector blocks of the oracle's H equal the full-space Kronecker construction."""
    rng = np.random.default_rng(10 + n)
    U, J, mu = 4.0, 0.8, 2.7
    delta = rng.uniform(-0.4, 0.4, n)
    m = Model(Params(n, U, J, mu=mu, delta=tuple(delta), beta=3.0, density_only=density_only))
    Hf = brute.hamiltonian(n, U, J, U - 2 * J, mu, delta, density_only)
    for s in range(m.nsec):
        xs = m.sector_states(s)
        if len(xs) == 0:
            continue
        H = m.block(s)[0]
        np.testing.assert_allclose(H, Hf[np.ix_(xs, xs)], atol=1e-13)
    # and nothing couples different sectors
    sec = np.zeros(len(Hf), dtype=int)
    for s in range(m.nsec):
        sec[m.sector_states(s)] = s
    assert np.all(Hf[sec[:, None] != sec[None, :]] == 0)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_two_electron_spectrum_closed_form(n):
    """P3: N=2 levels U-3J (x3C(n,2)), U-J (x C(n,2)+n-1), U+(n-1)J (x1) at mu=0, no crystal field.

    Derived from Eq. (H_loc) with U' = U-2J: two electrons in different orbitals form a
    triplet at U'-J and a singlet at U'+J; the n doubly occupied states are coupled by
    pair hopping -J into one state at U+(n-1)J and n-1 states at U-J.
    """
    U, J = 5.0, 0.7
    m = Model(Params(n, U, J, mu=0.0, beta=1.0))
    e = sector_energies(m, 2)
    c2 = n * (n - 1) // 2
    expect = np.sort([U - 3 * J] * (3 * c2) + [U - J] * (c2 + n - 1) + [U + (n - 1) * J])
    np.testing.assert_allclose(e, expect, atol=1e-12)


@pytest.mark.parametrize("n", [2, 3, 5])
def test_particle_hole_symmetry_at_half_filling(n):
    """P8: at mu_half (Sec. IV.B) with no crystal field the N and 2n-N spectra coincide."""
    U, J = 6.0, 1.0
    m = Model(Params(n, U, J, mu=mu_half(n, U, J), beta=1.0))
    for N in range(0, n):
        np.testing.assert_allclose(sector_energies(m, N), sector_energies(m, 2 * n - N), atol=1e-10)


def test_three_orbital_ground_degeneracy_paper():
    """P4: four ground states at half filling, spin 3/2 (Sec. IV.A)."""
    g = GOLD["three_orbital_half_filling"]
    m = Model(Params(3, g["U"], g["J"], mu=mu_half(3, g["U"], g["J"]), beta=50.0, trunc_eps=1.0))
    assert m.nkept == g["ground_degeneracy"]


def test_five_orbital_ground_degeneracies_paper():
    """P4: degeneracies 6, 25, 40, 30, 10, 1 for 5..10 electrons (Sec. IV.C)."""
    g = GOLD["five_orbital_filling_scan"]
    U, J = g["U"], g["J"]
    # middle of each ground-state window in mu - mu_half
    shifts = {5: 0.0, 6: 6.5, 7: 9.5, 8: 12.5, 9: 15.5, 10: 20.0}
    for N, deg in zip(g["electrons"], g["ground_degeneracy"]):
        m = Model(Params(5, U, J, mu=mu_half(5, U, J) + shifts[N], beta=50.0, trunc_eps=1.0))
        assert m.nkept == deg, (N, m.nkept)
        # all kept states hold N electrons
        nsec = [(int(s) // 6, int(s) % 6) for s in m.kept_sec]
        assert all(a + b == N for a, b in nsec)


def test_five_orbital_level_crossing_paper():
    """P4: N_tr = 6, 31, 25 at mu - mu_half = 4.98, 5, 5.02 (Sec. IV.C, Fig. 4)."""
    g = GOLD["five_orbital_level_crossing"]
    U, J = g["U"], g["J"]
    for dmu, ntr in zip(g["mu_minus_mu_half"], g["n_tr"]):
        m = Model(Params(5, U, J, mu=mu_half(5, U, J) + dmu, beta=g["beta"], trunc_eps=1.0))
        assert m.nkept == ntr, (dmu, m.nkept)


def test_spin_rotation_invariance():
    """P6: [H, S^2] = 0 and [H, S^+] = 0 for U' = U - 2J (Sec. IV.A, rotational invariance)."""
    n = 3
    rng = np.random.default_rng(3)
    delta = rng.uniform(-0.2, 0.2, n)
    m = Model(Params(n, 4.0, 1.0, mu=3.3, delta=tuple(delta), beta=1.0))
    dim = 4 ** n
    Hf = np.zeros((dim, dim))
    for s in range(m.nsec):
        xs = m.sector_states(s)
        if len(xs):
            Hf[np.ix_(xs, xs)] = m.block(s)[0]
    c = brute.fermion_ops(n)
    Sp = sum(c[2 * a].T @ c[2 * a + 1] for a in range(n))
    Sz = sum(0.5 * (c[2 * a].T @ c[2 * a] - c[2 * a + 1].T @ c[2 * a + 1]) for a in range(n))
    S2 = Sp @ Sp.T + Sz @ Sz - Sz
    assert np.abs(Hf @ Sp - Sp @ Hf).max() < 1e-12
    assert np.abs(Hf @ S2 - S2 @ Hf).max() < 1e-11


# ---------------------------------------------------------------------------
# traces
# ---------------------------------------------------------------------------

def one(m, ops):
    s, la, lt = m.trace(SeqBatch.from_lists([ops]))
    return int(s[0]), float(la[0]), float(lt[0])


@pytest.mark.parametrize("n", [1, 2, 3])
def test_atomic_limit_partition_function(n):
    """P1: empty sequence, no truncation: T = Z = sum_n exp(-beta E_n) (full-space eigvalsh)."""
    rng = np.random.default_rng(n)
    U, J, mu, beta = 4.0, 0.9, 3.1, 7.0
    delta = rng.uniform(-0.2, 0.2, n)
    m = Model(Params(n, U, J, mu=mu, delta=tuple(delta), beta=beta, trunc_eps=0.0))
    E = np.linalg.eigvalsh(brute.hamiltonian(n, U, J, U - 2 * J, mu, delta))
    logZ = -beta * E.min() + math.log(np.exp(-beta * (E - E.min())).sum())
    s, la, _ = one(m, [])
    assert s == 1
    assert abs(la - logZ) < 1e-12 * max(1.0, abs(logZ))


def test_atomic_limit_truncated():
    """P1: with truncation to the ground multiplet, T = N_tr exp(-beta E0)."""
    U, J = 6.0, 1.0
    m = Model(Params(3, U, J, mu=mu_half(3, U, J), beta=10.0, trunc_eps=1e-10))
    s, la, lt = one(m, [])
    assert s == 1 and m.nkept == 4
    assert abs(lt - math.log(4.0)) < 1e-13
    assert abs(la - (math.log(4.0) - 10.0 * m.E0)) < 1e-12


def test_one_orbital_closed_forms():
    """P2: one orbital, E_0 = 0, E_up = E_dn = -mu, E_updn = U - 2 mu."""
    U, mu, beta = 3.0, 1.1, 4.0
    m = Model(Params(1, U, 0.0, mu=mu, beta=beta, trunc_eps=0.0))
    E0, Es, E2 = 0.0, -mu, U - 2 * mu
    t1, t2 = 0.7, 2.9
    for f in (0, 1):
        # c_f at t1 then c_f^+ at t2
        s, la, _ = one(m, [(t1, f, 0), (t2, f, 1)])
        ex = math.exp(-(beta - t2 + t1) * Es - (t2 - t1) * E0) + math.exp(-(beta - t2 + t1) * E2 - (t2 - t1) * Es)
        assert s == 1 and abs(la - math.log(ex)) < 1e-13
        # reversed order: c_f^+ at t1 then c_f at t2 gives the complementary terms
        s, la, _ = one(m, [(t1, f, 1), (t2, f, 0)])
        ex = math.exp(-(beta - t2 + t1) * E0 - (t2 - t1) * Es) + math.exp(-(beta - t2 + t1) * Es - (t2 - t1) * E2)
        assert s == 1 and abs(la - math.log(ex)) < 1e-13
    # mixed flavors: c_up at t1, c_dn at t2, c_dn^+ at t3, c_up^+ at t4 passes only through |updn>
    t3, t4 = 3.2, 3.6
    s, la, _ = one(m, [(t1, 0, 0), (t2, 1, 0), (t3, 1, 1), (t4, 0, 1)])
    ex = math.exp(-(beta - t4 + t1) * E2 - (t2 - t1) * Es - (t3 - t2) * E0 - (t4 - t3) * Es)
    assert abs(la - math.log(ex)) < 1e-13
    # sign: c_dn c_up |updn> = -c_up c_dn |updn>: swapping the two annihilations flips the sign
    s2, la2, _ = one(m, [(t1, 1, 0), (t2, 0, 0), (t3, 1, 1), (t4, 0, 1)])
    assert s == 1 and s2 == -1 and abs(la2 - la) < 1e-13


def test_unbalanced_sequences_vanish():
    """P6: a sequence that changes the particle number has zero trace."""
    m = Model(Params(2, 4.0, 1.0, mu=2.0, beta=5.0, trunc_eps=0.0))
    assert one(m, [(1.0, 0, 1)])[0] == 0
    assert one(m, [(1.0, 0, 1), (2.0, 1, 0)])[0] == 0  # up in, down out: S_z changes
    assert one(m, [(1.0, 0, 1), (2.0, 0, 1)])[0] == 0   # Pauli


def test_density_expectation_equal_times():
    """P7: (c_f, c_f^+) at equal times gives Tr[e^{-beta H} n_f], independent of tau."""
    n = 2
    rng = np.random.default_rng(7)
    U, J, mu, beta = 4.0, 1.0, 2.5, 3.0
    delta = rng.uniform(-0.3, 0.3, n)
    m = Model(Params(n, U, J, mu=mu, delta=tuple(delta), beta=beta, trunc_eps=0.0))
    Hf = brute.hamiltonian(n, U, J, U - 2 * J, mu, delta)
    E, V = np.linalg.eigh(Hf)
    c = brute.fermion_ops(n)
    w = np.exp(-beta * (E - E.min()))
    Z = w.sum()
    for f in range(2 * n):
        nf = np.einsum("in,ij,jn->n", V, c[f].T @ c[f], V)
        ex_n = math.log((w * nf).sum()) - beta * E.min()
        ex_1mn = math.log((w * (1 - nf)).sum()) - beta * E.min()
        for tau in (0.0, 0.4, 2.9):
            s, la, _ = one(m, [(tau, f, 0), (tau, f, 1)])
            assert s == 1 and abs(la - ex_n) < 1e-12
            s, la, _ = one(m, [(tau, f, 1), (tau, f, 0)])
            assert s == 1 and abs(la - ex_1mn) < 1e-12


def _random_ops(rng, n, beta, kmax, coin=True):
    ops = []
    for f in range(2 * n):
        k = int(rng.integers(0, kmax + 1))
        ts = np.sort(rng.uniform(0, beta, 2 * k))
        first = int(rng.integers(2)) if coin else 1
        for j, t in enumerate(ts):
            ops.append((float(t), f, first if j % 2 == 0 else 1 - first))
    ops.sort()
    return ops


@pytest.mark.parametrize("n", [2, 3])
def test_brute_force_full_space(n):
    """P9: untruncated trace equals the full-space Kronecker/expm brute force."""
    rng = np.random.default_rng(100 + n)
    U, J, mu, beta = 4.0, 1.0, 2.5 * 4.0 - 5.0, 4.0
    delta = rng.uniform(-0.1, 0.1, n)
    m = Model(Params(n, U, J, mu=mu, delta=tuple(delta), beta=beta, trunc_eps=0.0))
    mx = Model(Params(n, U, J, mu=mu, delta=tuple(delta), beta=beta, trunc_eps=0.0), "ext")
    Hf = brute.hamiltonian(n, U, J, U - 2 * J, mu, delta)
    checked = 0
    for _ in range(40):
        ops = _random_ops(rng, n, beta, 3)
        Tb, E0b = brute.trace_all_states(Hf, beta, ops, n)
        s, la, lt = one(m, ops)
        sx, lax, ltx = one(mx, ops)
        if classify([s], [lt], [sx], [ltx])[0] != 2:
            assert abs(Tb) < 1e-10 * 4 ** n
            continue
        checked += 1
        assert s == int(np.sign(Tb))
        assert abs(lt - math.log(abs(Tb))) < 1e-9
    assert checked >= 10


def _gap_threshold(H, beta, n_multiplets, deg_tol=1e-9):
    """A trunc_eps that keeps exactly the lowest n_multiplets multiplets of the full-space H,
    set in the middle (geometrically) of the gap to the next one."""
    E = np.linalg.eigvalsh(H)
    lows = [0]
    for i in range(1, len(E)):
        if E[i] - E[i - 1] > deg_tol * max(1.0, abs(E[i])):
            lows.append(i)
    a, b = E[lows[n_multiplets - 1]] - E[0], E[lows[n_multiplets]] - E[0]
    return math.exp(-beta * 0.5 * (a + b))


@pytest.mark.parametrize("n,n_mult", [(2, 3), (3, 4), (3, 7)])
def test_truncated_trace_full_space_projector(n, n_mult):
    """Truncation type (i) of Sec. II with spin flip and pair hopping on: the truncated trace
    with operators equals Tr[P e^{-(beta-t_K)H} O_K ... O_1 e^{-t_1 H}], P the projector on the
    kept multiplets of the full-space Kronecker H (numpy eigh, whole multiplets) and every
    propagator a full-space scaling-and-squaring exponential. Nothing here uses the oracle's
    sectors, eigensolver or kept-state list."""
    rng = np.random.default_rng(300 + 10 * n + n_mult)
    U, J, beta = 4.0, 1.0, 4.0
    mu = mu_half(n, U, J) + 0.6
    delta = rng.uniform(-0.3, 0.3, n)
    Hf = brute.hamiltonian(n, U, J, U - 2 * J, mu, delta)
    eps = _gap_threshold(Hf, beta, n_mult)
    P, n_keep = brute.kept_projector(Hf, beta, eps)
    assert 1 < n_keep < 4 ** n
    m = Model(Params(n, U, J, mu=mu, delta=tuple(delta), beta=beta, trunc_eps=eps))
    mx = Model(Params(n, U, J, mu=mu, delta=tuple(delta), beta=beta, trunc_eps=eps), "ext")
    assert m.nkept == n_keep
    # the kept set really has multiplets (spin degeneracy survives the crystal field)
    assert n_keep > n_mult
    checked = 0
    for _ in range(40):
        ops = _random_ops(rng, n, beta, 3)
        Tb, E0b = brute.trace_projected(Hf, beta, ops, n, P)
        s, la, lt = one(m, ops)
        sx, lax, ltx = one(mx, ops)
        assert abs(E0b - m.E0) < 1e-12 * max(1.0, abs(E0b))
        if classify([s], [lt], [sx], [ltx])[0] != 2:
            assert abs(Tb) < 1e-10 * n_keep
            continue
        checked += 1
        assert s == int(np.sign(Tb))
        assert abs(lt - math.log(abs(Tb))) < 1e-9
    assert checked >= 10


def test_brute_force_extended_precision_classes():
    """Conditioning classes agree with a 40-digit full-space computation (2 orbitals)."""
    n = 2
    rng = np.random.default_rng(5)
    U, J, mu, beta = 4.0, 1.0, 2.5, 6.0
    m = Model(Params(n, U, J, mu=mu, beta=beta, trunc_eps=0.0))
    mx = Model(Params(n, U, J, mu=mu, beta=beta, trunc_eps=0.0), "ext")
    Hf = brute.hamiltonian(n, U, J, U - 2 * J, mu, np.zeros(n))
    seen = set()
    for _ in range(12):
        ops = _random_ops(rng, n, beta, 2)
        s, la, lt = one(m, ops)
        sx, lax, ltx = one(mx, ops)
        cls = classify([s], [lt], [sx], [ltx])[0]
        Tm, _ = brute.trace_all_states_mp(Hf, beta, ops, n, dps=40)
        seen.add(int(cls))
        if cls == 2:
            assert s * math.exp(lt) / float(Tm) - 1 == pytest.approx(0, abs=1e-11)
        else:
            assert abs(float(Tm)) < 1e-25
    assert 2 in seen


@pytest.mark.parametrize("shift", [0.37, 1.9, 3.3])
def test_cyclic_invariance_untruncated(shift):
    """P10: shifting every time by s modulo beta (wrapped operators move to the front)."""
    n, U, J, mu, beta = 3, 4.0, 1.0, 5.0, 4.0
    m = Model(Params(n, U, J, mu=mu, beta=beta, trunc_eps=0.0))
    mx = Model(Params(n, U, J, mu=mu, beta=beta, trunc_eps=0.0), "ext")
    rng = np.random.default_rng(21)
    done = 0
    for _ in range(30):
        ops = _random_ops(rng, n, beta, 2)
        s, la, lt = one(m, ops)
        sx, _, ltx = one(mx, ops)
        if classify([s], [lt], [sx], [ltx])[0] != 2:
            continue
        wrapped = [((t + shift) - beta, f, d) for (t, f, d) in ops if t + shift >= beta]
        stay = [(t + shift, f, d) for (t, f, d) in ops if t + shift < beta]
        s2, la2, _ = one(m, wrapped + stay)
        assert s2 == s and abs(la2 - la) < 1e-10
        done += 1
    assert done >= 5


def test_orbital_relabelling_invariance():
    """P10: relabelling orbitals (a different Jordan-Wigner order) leaves the trace unchanged."""
    n, U, J, mu, beta = 3, 4.0, 1.0, 5.0, 10.0
    m = Model(Params(n, U, J, mu=mu, beta=beta))
    mx = Model(Params(n, U, J, mu=mu, beta=beta), "ext")
    rng = np.random.default_rng(8)
    perm = [2, 0, 1]
    done = 0
    for _ in range(60):
        ops = _random_ops(rng, n, beta, 3)
        s, la, lt = one(m, ops)
        sx, _, ltx = one(mx, ops)
        if classify([s], [lt], [sx], [ltx])[0] != 2:
            continue
        ops2 = [(t, 2 * perm[f // 2] + f % 2, d) for (t, f, d) in ops]
        s2, la2, _ = one(m, ops2)
        assert s2 == s and abs(la2 - la) < 1e-10
        done += 1
    assert done >= 5


def test_density_only_segment_picture():
    """P5: density-density H_loc (segment formulation, Sec. II): each occupation string
    x(tau) contributes exp(-integral of E_diag(x)) times its Jordan-Wigner signs."""
    n, U, J, mu, beta = 3, 4.0, 1.0, 4.0, 6.0
    rng = np.random.default_rng(4)
    delta = rng.uniform(-0.3, 0.3, n)
    m = Model(Params(n, U, J, mu=mu, delta=tuple(delta), beta=beta, trunc_eps=0.0, density_only=True))
    Hd = np.diag(brute.hamiltonian(n, U, J, U - 2 * J, mu, delta, density_only=True))
    E0 = Hd.min()
    for _ in range(25):
        ops = _random_ops(rng, n, beta, 3)
        total = 0.0
        for x0 in range(4 ** n):
            x, sgn, t_prev, expo, ok = x0, 1, 0.0, 0.0, True
            for (t, f, d) in ops:
                expo += (t - t_prev) * (Hd[x] - E0)
                bit = 1 << f
                if bool(x & bit) == bool(d):
                    ok = False
                    break
                if bin(x & (bit - 1)).count("1") % 2:
                    sgn = -sgn
                x ^= bit
                t_prev = t
            if not ok or x != x0:
                continue
            expo += (beta - t_prev) * (Hd[x] - E0)
            total += sgn * math.exp(-expo)
        s, la, lt = one(m, ops)
        if total == 0.0:
            assert s == 0
        else:
            assert s == int(np.sign(total)) and abs(lt - math.log(abs(total))) < 1e-11


def test_edit_insert_and_remove():
    """Local updates: insertion places each new operator after equal times; removal takes
    an operator and its cyclic successor of the same flavor, which has the other type."""
    ops = [(0.5, 0, 1), (1.0, 1, 0), (2.0, 0, 0), (3.0, 1, 1)]
    new = edit(ops, 0, 2, 1.5, 2.5, 0)
    assert new == [(0.5, 0, 1), (1.0, 1, 0), (1.5, 2, 1), (2.0, 0, 0), (2.5, 2, 0), (3.0, 1, 1)]
    new = edit(ops, 0, 2, 2.5, 1.5, 0)   # anti-segment
    assert new == [(0.5, 0, 1), (1.0, 1, 0), (1.5, 2, 0), (2.0, 0, 0), (2.5, 2, 1), (3.0, 1, 1)]
    assert edit(ops, 1, 0, 0, 0, 0) == [(1.0, 1, 0), (3.0, 1, 1)]
    assert edit(ops, 1, 1, 0, 0, 3) == [(0.5, 0, 1), (2.0, 0, 0)]  # wraps: successor is at index 1
    assert edit(ops, 1, 1, 0, 0, 1) == [(0.5, 0, 1), (2.0, 0, 0)]   # a c and the c^+ after it
    assert edit(ops, 1, 0, 0, 0, 2) == [(1.0, 1, 0), (3.0, 1, 1)]   # wraps: the c at 2, then the c^+ at 0
    assert edit(ops, 1, 0, 0, 0, 1) is None   # index 1 is not of flavor 0
    assert edit([(0.5, 0, 1), (1.0, 0, 1)], 1, 0, 0, 0, 0) is None   # successor of the same type


def _gap_pair(rng, ops, f, beta):
    """Two times in one gap between cyclically consecutive flavor-f operators, in cyclic
    order: an inserted pair there is adjacent in flavor f, so removing its first operator
    (with its cyclic successor) undoes the insertion."""
    ts = sorted(t for t, g, _ in ops if g == f)
    if not ts:
        a, b = np.sort(rng.uniform(0, beta, 2))
        return float(a), float(b)
    k = int(rng.integers(len(ts)))
    lo, hi = ts[k], (ts[k + 1] if k + 1 < len(ts) else ts[0] + beta)
    a, b = np.sort(rng.uniform(lo, hi, 2))
    return float(a % beta), float(b % beta)


def _move(kind, f, t_dag=0.0, t_ann=0.0, rem_idx=0):
    return {"kind": [kind], "flavor": [f], "t_dag": [t_dag], "t_ann": [t_ann], "rem_idx": [rem_idx]}


@pytest.mark.parametrize("n", [2, 3])
def test_ratio_insert_then_remove_is_identity(n):
    """Trace ratio (Sec. II local updates): inserting a pair and removing it again gives
    back the sequence, and the two ratios multiply to one (signs and log-ratios)."""
    rng = np.random.default_rng(40 + n)
    beta = 5.0
    m = Model(Params(n, 4.0, 1.0, mu=mu_half(n, 4.0, 1.0), beta=beta, trunc_eps=1e-8))
    checked = 0
    for _ in range(30):
        ops = _random_ops(rng, n, beta, 2)
        f = int(rng.integers(2 * n))
        a, b = _gap_pair(rng, ops, f, beta)
        d_first = int(rng.integers(2))  # the operator at a: c^+ (segment) or c (anti-segment)
        t_dag, t_ann = (a, b) if d_first else (b, a)
        new = edit(ops, 0, f, t_dag, t_ann, 0)
        idx = new.index((a, f, d_first))
        assert edit(new, 1, f, 0.0, 0.0, idx) == ops
        cur = SeqBatch.from_lists([ops])
        cs, cl, _ = m.trace(cur)
        s1, lr1, ns, nl = ratio(m, cur, cs, cl, _move(0, f, t_dag, t_ann))
        s2, lr2, bs, bl = ratio(m, SeqBatch.from_lists([new]), ns, nl, _move(1, f, rem_idx=idx))
        assert bs[0] == cs[0] and (cs[0] == 0 or bl[0] == cl[0])
        if cs[0] == 0:
            assert s1[0] == 0 and math.isnan(lr1[0])
            continue
        if ns[0] == 0:
            assert s1[0] == 0 and lr1[0] == -math.inf and s2[0] == 0 and math.isnan(lr2[0])
            continue
        checked += 1
        assert s1[0] * s2[0] == 1
        assert s1[0] == cs[0] * ns[0]
        assert lr1[0] + lr2[0] == 0.0
    assert checked >= 8


def test_ratio_matches_full_space_brute_force():
    """Trace ratio T_new / T_cur against the full-space Kronecker/expm traces (2 orbitals,
    untruncated); numerically-zero traces (FP64 and long double disagree) are skipped."""
    n, beta = 2, 4.0
    rng = np.random.default_rng(77)
    U, J, mu = 4.0, 1.0, mu_half(2, 4.0, 1.0)
    m = Model(Params(n, U, J, mu=mu, beta=beta, trunc_eps=0.0))
    mx = Model(Params(n, U, J, mu=mu, beta=beta, trunc_eps=0.0), "ext")
    Hf = brute.hamiltonian(n, U, J, U - 2 * J, mu, np.zeros(n))
    checked = 0
    for _ in range(40):
        ops = _random_ops(rng, n, beta, 2)
        f = int(rng.integers(2 * n))
        t_dag, t_ann = (float(t) for t in rng.uniform(0, beta, 2))
        new = edit(ops, 0, f, t_dag, t_ann, 0)
        cur = SeqBatch.from_lists([ops])
        cs, cl, _ = m.trace(cur)
        s, lr, ns, nl = ratio(m, cur, cs, cl, _move(0, f, t_dag, t_ann))
        ok = [classify([x], [y], [xx], [yy])[0] == 2
              for (x, y), (xx, yy) in (((cs[0], cl[0]), one(mx, ops)[:2]), ((ns[0], nl[0]), one(mx, new)[:2]))]
        if not all(ok):
            continue
        Tc, _ = brute.trace_all_states(Hf, beta, ops, n)
        Tn, _ = brute.trace_all_states(Hf, beta, new, n)
        checked += 1
        assert s[0] == int(np.sign(Tn * Tc))
        assert abs(lr[0] - math.log(abs(Tn / Tc))) < 1e-9
    assert checked >= 10
